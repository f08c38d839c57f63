"""Host-side model of the float32 tile-upper layout (NSRGS_F32 at 8 < d <= 64),
without a GPU: the order of the stored 64 x 64 tiles (row after row of the
upper triangle of tiles), the chunk swizzle inside a tile, and the storage rule
(block(row) < block(col), zero elsewhere).  Walking the stored tiles as the
kernel does (Y_I += A_IJ X_J, Y_J += A_IJ^T X_I) must rebuild A_off X, and the
library's packed size must match."""
import math

import numpy as np
import pytest

import synth

T = 64


def nt(n, d):
    return -(-n * d // T)


def row_start(I, NT):
    return I * NT - I * (I - 1) // 2


def tile_ij(t, NT):
    """The kernel's inverse of the order: closed form, then corrected by one step."""
    b = 2.0 * NT + 1.0
    i = int((b - math.sqrt(b * b - 8.0 * t)) * 0.5)
    i = min(max(i, 0), NT - 1)
    while i > 0 and row_start(i, NT) > t:
        i -= 1
    while i + 1 < NT and row_start(i + 1, NT) <= t:
        i += 1
    return i, i + (t - row_start(i, NT))


def swz(r, c):
    return r * 256 + (((c >> 2) ^ ((r >> 2) & 7)) << 4) + (c & 3) * 4


@pytest.mark.parametrize("NT", [1, 2, 3, 7, 64, 250, 501, 2000])
def test_tile_order_inverse(NT):
    ts = range(NT * (NT + 1) // 2) if NT <= 501 else list(range(0, NT * (NT + 1) // 2, 997)) + [NT * (NT + 1) // 2 - 1]
    seq = {}
    t = 0
    if NT <= 501:
        for I in range(NT):
            for J in range(I, NT):
                seq[t] = (I, J)
                t += 1
    for t in ts:
        I, J = tile_ij(t, NT)
        assert 0 <= I <= J < NT
        assert row_start(I, NT) + (J - I) == t
        if seq:
            assert seq[t] == (I, J)


def test_swizzle_is_a_bijection_of_4_byte_words():
    offs = sorted(swz(r, c) for r in range(T) for c in range(T))
    assert offs == list(range(0, T * T * 4, 4))
    # each row's 16 chunks stay inside the row and float4 chunks stay 16-byte aligned
    for r in range(T):
        assert {swz(r, c) // 256 for c in range(T)} == {r}
        assert all(swz(r, c) % 16 == 0 for c in range(0, T, 4))


def conflict_free(addrs):
    """8 lanes of a quarter-warp reading 16 bytes each: distinct 16-byte bank groups
    (address / 16 mod 8), or the same address (a broadcast)."""
    groups = {}
    for a in addrs:
        groups.setdefault((a // 16) % 8, set()).add(a)
    return all(len(v) == 1 for v in groups.values())


def test_kernel_shared_memory_reads_are_conflict_free():
    # row product: 8 consecutive threads share the X column chunk and take rows 4p + i, p = p0 .. p0 + 7
    for p0 in (0, 8):
        for i in range(4):
            for k in range(0, T, 4):
                assert conflict_free([swz(4 * p + i, k) for p in range(p0, p0 + 8)])
    # column product: 8 consecutive threads take columns 4q .. 4q+3, q = q0 .. q0 + 7, of one row
    for q0 in (0, 8):
        for r in range(T):
            assert conflict_free([swz(r, 4 * q) for q in range(q0, q0 + 8)])


def stored_tile(Aoff_upper, I, J, n, d):
    N = n * d
    tile = np.zeros((T, T))
    rows = np.arange(I * T, I * T + T)
    cols = np.arange(J * T, J * T + T)
    for a, r in enumerate(rows):
        if r >= N:
            continue
        for b, c in enumerate(cols):
            if c < N and c // d > r // d:
                tile[a, b] = Aoff_upper[r, c]
    return tile


@pytest.mark.parametrize("n,d", [(2, 9), (5, 16), (9, 25), (7, 13), (12, 40), (3, 64), (30, 11)])
def test_walk_rebuilds_Aoff_X(n, d):
    inst = synth.make_instance(n, d, 0.7, seed=n + d)
    A = inst.dense()
    N = n * d
    Aoff = A.copy()
    for i in range(n):
        Aoff[i * d : (i + 1) * d, i * d : (i + 1) * d] = 0.0
    X = np.random.default_rng(1).standard_normal((N, d))
    NT = nt(n, d)
    Xp = np.zeros((NT * T, d))
    Xp[:N] = X
    Y = np.zeros((NT * T, d))
    hit = np.zeros((NT * T, NT * T), dtype=int)
    for t in range(NT * (NT + 1) // 2):
        I, J = tile_ij(t, NT)
        tl = stored_tile(Aoff, I, J, n, d)
        Y[I * T : I * T + T] += tl @ Xp[J * T : J * T + T]
        Y[J * T : J * T + T] += tl.T @ Xp[I * T : I * T + T]
        hit[I * T : I * T + T, J * T : J * T + T] += tl != 0
    assert np.allclose(Y[:N], Aoff @ X, atol=1e-10)
    assert np.all(Y[N:] == 0.0)
    assert hit.max() <= 1  # every stored element appears in one tile


@pytest.mark.parametrize("n,d", [(2000, 16), (2000, 32), (2000, 64), (500, 25), (3, 9)])
def test_packed_bytes_match_library(n, d):
    L = pytest.importorskip("paper_2604_07372_gb300._lib")
    try:
        lib = L.lib()
    except RuntimeError:
        pytest.skip("libnsrgs.so not built")
    NT = nt(n, d)
    assert lib.nsrgs_packed_bytes(n, d, 0) == NT * (NT + 1) // 2 * T * T * 4
    # about half the dense float32 bytes
    dense = lib.nsrgs_packed_bytes(n, d, 3)
    assert 0.49 < lib.nsrgs_packed_bytes(n, d, 0) / dense < 0.56 or n * d < 1000
