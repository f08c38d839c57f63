"""C ABI checks that need no GPU: the library loads, exports every entry point
declared in include/nsrgs.h, answers size queries, and rejects bad arguments
before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    import __graft_entry__

    try:
        __graft_entry__.build()
    except Exception as e:  # nvcc missing on this machine
        pytest.skip(f"cannot build libnsrgs.so here: {e}")
    import paper_2604_07372_gb300 as P

    return P


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "nsrgs.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(nsrgs_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert "nsrgs_solve" in names and "nsrgs_step" in names and "nsrgs_spectral_init" in names
    lib = ctypes.CDLL(L.lib_path())
    for name in names:
        assert hasattr(lib, name), f"{name} declared but not exported"


def test_version_and_sizes(L):
    assert "sm_103a" in L.nsrgs_version()
    # symmetric layouts: F32 any d <= 64 (panels up to 8, float32 tiles above), BF16 d <= 8
    # and 8 < d <= 64 (tiles), FP8 d <= 4 and 8 < d <= 64; the dense layout any d <= 64
    assert L.nsrgs_packed_bytes(200, 3, L.F32) > 0
    assert L.nsrgs_packed_bytes(200, 8, L.F32) > 0 and L.nsrgs_packed_bytes(200, 5, L.BF16) > 0
    assert L.nsrgs_packed_bytes(200, 9, L.F32) > 0 and L.nsrgs_packed_bytes(200, 64, L.F32) > 0
    assert L.nsrgs_packed_bytes(200, 65, L.F32) == 0 and L.nsrgs_packed_bytes(200, 65, L.BF16) == 0
    # BF16 / FP8 above d = 8: the tile-upper layout at every d (tile width 16, 32 or 64)
    NT = -(-(200 * 9) // 128)
    assert L.nsrgs_packed_bytes(200, 9, L.BF16) == NT * (NT + 1) // 2 * 32768
    assert L.nsrgs_packed_bytes(200, 25, L.FP8E4M3) > 0 and L.nsrgs_packed_bytes(200, 8, L.FP8E4M3) == 0
    assert L.nsrgs_packed_bytes(200, 5, L.FP8E4M3) == 0 and L.nsrgs_packed_bytes(200, 8, L.FP8E4M3) == 0
    assert L.nsrgs_packed_bytes(200, 16, L.FP8E4M3) * 2 < L.nsrgs_packed_bytes(200, 16, L.BF16) + 4096
    # block-sparse rows: the bound for fully observed data, both triangles, d <= 8
    assert L.nsrgs_packed_bytes(200, 3, L.BCSR_F32) >= 200 * 199 * 9 * 4
    assert L.nsrgs_packed_bytes(200, 3, L.BCSR_BF16) >= 200 * 199 * 9 * 2
    assert L.nsrgs_packed_bytes(200, 9, L.BCSR_F32) == 0
    assert L.nsrgs_packed_bytes(200, 25, L.DENSE_F32) == 200 * 25 * 5000 * 4
    assert L.nsrgs_packed_bytes(1, 3, L.F32) == 0
    # BF16 / FP8 shrink the panels by 2x / 4x (plus small tables)
    f, b, q = (L.nsrgs_packed_bytes(10000, 3, s) for s in (L.F32, L.BF16, L.FP8E4M3))
    assert abs(f / b - 2.0) < 0.01 and abs(f / q - 4.0) < 0.02
    assert L.nsrgs_workspace_bytes(10000, 3) >= 4 * (30064 * 3 * 4)
    assert L.nsrgs_workspace_bytes(1, 3) == 0


def test_bad_arguments_are_rejected_without_a_device(L):
    lib = L.lib()
    A = L._lib._A(0, 1, 3, 0)  # n = 1
    r = lib.nsrgs_solve(ctypes.byref(A), 0.1, 10, 2, 0.0, 1, 50, None, None, None, 0, None)
    assert r == 1 and b"n must be" in lib.nsrgs_last_error()
    A = L._lib._A(0, 100, 65, 0)  # d = 65
    assert lib.nsrgs_solve(ctypes.byref(A), 0.1, 10, 2, 0.0, 1, 50, None, None, None, 0, None) == 1
    A = L._lib._A(16, 100, 3, 0)  # packed must be non-null; given, the next check is the workspace
    assert lib.nsrgs_step(None, 0.1, 2, None, None, None, None, 0, None) == 1
    assert lib.nsrgs_dF(None, None, 10, 3, None, None, 0, None) == 1
    assert lib.nsrgs_pack_upper(None, 10, 3, 0, None, None) == 1
    assert lib.nsrgs_pack_dense(None, 1, 3, 0, None, None) == 1
    # host-buffer solve: size and header checks come before any copy
    buf = (ctypes.c_char * 256)()
    A = L._lib._A(16, 100, 3, 0)
    assert lib.nsrgs_solve_host(ctypes.byref(A), buf, 256, 0.01, 10, 2, 0.0, 1, 50, None, buf, None, None, 0,
                                None) == 1
    assert b"packed_bytes" in lib.nsrgs_last_error()
    assert lib.nsrgs_solve_host(ctypes.byref(A), None, 256, 0.01, 10, 2, 0.0, 1, 50, None, buf, None, None, 0,
                                None) == 1
    hdr = (ctypes.c_longlong * 32)(100, 4, 10)  # block-sparse header for another d
    A = L._lib._A(16, 100, 3, 5)
    assert lib.nsrgs_solve_host(ctypes.byref(A), hdr, 256, 0.01, 10, 2, 0.0, 1, 50, None, buf, None, None, 0,
                                None) == 1
    assert b"header" in lib.nsrgs_last_error()
    # SE(d) form: shapes outside it are rejected before any device work
    assert lib.nsrgs_se_packed_bytes(100, 64, 0) == 0 and lib.nsrgs_se_packed_bytes(100, 3, 2) == 0
    assert lib.nsrgs_se_packed_bytes(100, 8, 0) == lib.nsrgs_packed_bytes(100, 9, 0) > 0  # float32 tiles
    assert lib.nsrgs_se_packed_bytes(100, 3, 0) == lib.nsrgs_packed_bytes(100, 4, 0) > 0
    assert lib.nsrgs_se_workspace_bytes(100, 3) == lib.nsrgs_workspace_bytes(100, 4) > 0
    assert lib.nsrgs_se_pack(buf, buf, 100, 64, 0.1, 0, buf, None) == 1
    assert lib.nsrgs_se_pack(buf, buf, 100, 3, -0.1, 0, buf, None) == 1
    A = L._lib._A(16, 100, 65, 0)  # augmented blocks of 65: outside the form
    assert lib.nsrgs_se_solve(ctypes.byref(A), 0.1, 0.01, 1.0, 5, 2, 0.0, buf, buf, None, buf, 0, None) == 1


def test_static_step_limits_match_the_documented_figures(L):
    """nsrgs_step_static holds its scratch in a fixed 8 MiB array; the largest n per d
    documented in include/nsrgs.h follows from nsrgs_workspace_bytes."""
    cap = 8 << 20
    lib = L.lib()

    def largest_n(d):
        if lib.nsrgs_workspace_bytes(2, d) > cap:
            return None
        lo, hi = 2, 1 << 22
        while lo < hi:
            m = (lo + hi + 1) // 2
            if lib.nsrgs_workspace_bytes(m, d) <= cap:
                lo = m
            else:
                hi = m - 1
        return lo

    header = open(os.path.join(ROOT, "include", "nsrgs.h")).read()
    for d, n in ((3, 46016), (4, 25656), (8, 6025), (16, 931)):
        assert largest_n(d) == n, (d, largest_n(d))
        assert f"n <= {n} at d = {d}" in header
    assert largest_n(32) is None and largest_n(64) is None
    assert "d >= 32\n *    never fits" in header
    # the oversize check comes before any device access
    fn = lib.nsrgs_step_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(L._lib._A), ctypes.c_float, ctypes.c_int] + [ctypes.c_void_p] * 4
    a = L._lib._A(16, 46017, 3, 0)
    assert fn(ctypes.byref(a), 0.1, 2, None, None, None, None) == 1
    assert b"8 MiB" in lib.nsrgs_last_error()
