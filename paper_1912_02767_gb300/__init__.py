"""GB300-native approximate-ADMM semidefinite programming.

The solver, the PSD projection by warm-started LOBPCG and the batched and
serving drivers live in the CUDA library ``libsdpgpu.so`` built from
``csrc/``; ``sdpgpu`` is its thin ctypes binding (argument marshalling only).
Importing the package does not load the library; ``sdpgpu.load()`` does, and
fails loudly when it has not been built.
"""
__all__ = ["instances", "sdpgpu"]
