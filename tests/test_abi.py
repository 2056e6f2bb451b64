"""The C-ABI library loads and exports every function include/sdpgpu.h
declares (no GPU needed: nothing is called that touches a device)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(?:int|void|const char\s*\*|unsigned long long)\s+(sdp_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1912_02767_gb300 import build_lib, sdpgpu
    build_lib.build()
    return sdpgpu.load()


def test_header_declares_the_api():
    names = declared_functions()
    for must in ["sdp_create", "sdp_setup", "sdp_solve", "sdp_project_psd", "sdp_batch_solve",
                 "sdp_server_submit", "sdp_server_poll", "sdp_destroy"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    from paper_1912_02767_gb300 import sdpgpu
    s = sdpgpu.settings()
    assert s.rho == 1.0 and s.max_iter == 5000 and s.check_every == 40
    assert abs(s.mode_frac - 1 / 3) < 1e-15 and abs(s.expand_frac - 1 / 50) < 1e-15
    assert sdpgpu.status_str(1) == "SOLVED" and sdpgpu.status_str(-4) == "E_NUMERICAL"
    assert sdpgpu.footprint_bytes(64, 64, 64) > 0
