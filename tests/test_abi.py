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


# (size in bytes, floating point?) of the C types the header uses
C_TYPES = {"double": (8, True), "int": (4, False), "unsigned long long": (8, False), "long long": (8, False)}


def header_structs():
    """(name -> [(C type, field)]) of the typedef'd structs of the header."""
    text = open(os.path.join(ROOT, "include", "sdpgpu.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for m in re.finditer(r"typedef struct \{(.*?)\}\s*(\w+);", text, flags=re.S):
        fields = []
        for decl in m.group(1).split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            ctype, names = re.match(r"(unsigned long long|long long|double|int)\s+(.*)", decl).groups()
            fields += [(ctype, nm.strip()) for nm in names.split(",")]
        out[m.group(2)] = fields
    return out


def test_ctypes_mirrors_match_the_header():
    """Field names, order and types of the ctypes structures equal the C
    structs of include/sdpgpu.h (a drift would shift every later field)."""
    import ctypes
    from paper_1912_02767_gb300 import sdpgpu
    hs = header_structs()
    for cname, py in [("sdp_settings", sdpgpu.Settings), ("sdp_info", sdpgpu.Info),
                      ("sdp_proj_info", sdpgpu.ProjInfo), ("sdp_prof_entry", sdpgpu.ProfEntry)]:
        want = [(f,) + C_TYPES[t] for t, f in hs[cname]]
        got = [(f, ctypes.sizeof(t), t in (ctypes.c_double, ctypes.c_float)) for f, t in py._fields_]
        assert got == want, (cname, got, want)


def test_default_rayleigh_ritz_settings(lib):
    from paper_1912_02767_gb300 import sdpgpu
    s = sdpgpu.settings()
    assert s.rr_method == 0 and s.rr_fp32 == 0 and s.precision == sdpgpu.PREC_FP64
    # Algorithm 3's full trial subspace span(X, R, dX) unless soft locking is asked for
    assert s.soft_lock == 0 and s.proj_neg == 0 and s.exact_solver == 0


@pytest.mark.parametrize("field,value", [
    ("rho", 0.0), ("sigma", -1.0), ("alpha", 2.0), ("eps_abs", -1e-4), ("max_iter", 0), ("check_every", 0),
    ("lobpcg_max_iter", 0), ("precision", 3), ("rr_method", 2), ("rr_fp32", 2), ("proj_neg", 2),
    ("exact_solver", 2), ("soft_lock", 2), ("tol_coef", 0.0), ("expand_frac", 0.0), ("mode_frac", 0.6)])
def test_invalid_settings_are_refused_before_any_device_call(lib, field, value):
    """sdp_create checks every setting before it touches the device: an out-of-
    range value returns SDP_E_INVALID and creates nothing (no GPU needed)."""
    import ctypes
    from paper_1912_02767_gb300 import sdpgpu
    s = sdpgpu.settings()
    setattr(s, field, value)
    h = ctypes.c_void_p()
    rc = sdpgpu.load().sdp_create(ctypes.byref(h), ctypes.byref(s), None)
    assert rc == -1 and not h.value, (field, value, rc)
