"""Host-side checks of the tile-upper layout of the tensor-core symmetric stream
(BF16 storage at d in {16, 32, 64}), without a GPU.

A NumPy model of the layout: 128 x 128 tiles (I, J) with J >= I, stored in the
kernel's processing order (groups of R row tiles, R = 8 for d in {16, 32} and 4
for d = 64; columns J inside a group; rows inside a column); inside a tile the
128-byte-swizzled order (8-row groups 2048 bytes apart, the two 64-column halves
1024 bytes apart, rows 128 bytes apart, 16-byte chunk k of row r at k ^ (r % 8)).  Checked: (1) the swizzle is a bijection of a
tile onto its 32 KB; (2) every element of the strict block-upper triangle lands
in exactly one stored slot and every other slot holds zero; (3) the two products
each tile feeds (Y_I += A_IJ X_J, Y_J += A_IJ^T X_I) rebuild A_off X; (4) the
MN-major reading of a tile (MN atoms 1024 bytes apart, 8-row K groups 2048
apart) addresses the transposed tile, and the K-major reading (8-row groups 2048
apart) the tile itself; (5) the processing order visits every tile once and the
closed-form position -> (I, J) map (group sizes, then triangular and full
column strips) inverts it; (6) the library's packed-byte count agrees.
"""
import numpy as np
import pytest

import synth

T = 128


def swz(r, c):
    """Byte offset of bfloat16 element (r, c) in a swizzled 128 x 128 tile."""
    s, k, e = c >> 6, (c & 63) >> 3, c & 7
    return (r >> 3) * 2048 + s * 1024 + (r & 7) * 128 + ((k ^ (r & 7)) << 4) + e * 2


def sw128(addr):
    """The 128-byte swizzle as an address map: bits [4:6] ^= bits [7:9]."""
    return addr ^ (((addr >> 7) & 7) << 4)


def test_swizzle_is_a_bijection_of_a_tile():
    r, c = np.meshgrid(np.arange(T), np.arange(T), indexing="ij")
    off = swz(r, c)
    assert off.min() == 0 and off.max() == 32768 - 2
    assert np.unique(off).size == T * T
    assert np.all(off % 2 == 0)


def test_k_major_reading_addresses_the_tile():
    """K-major operand: row m of the 8-row group g of half s, K offset kk*16 elements:
    unswizzled address base + s*1024 + g*2048 + (m%8)*128 + 2*k, then the 128-byte swizzle."""
    for s in (0, 1):
        for m in range(T):
            for k in range(64):
                a = s * 1024 + (m >> 3) * 2048 + (m & 7) * 128 + 2 * k
                assert sw128(a) == swz(m, 64 * s + k)


def test_mn_major_reading_addresses_the_transpose():
    """MN-major operand (A^T, M = tile columns, K = tile rows): MN atom a = m // 64 at
    LBO = 1024, K group g = k // 8 at SBO = 2048, inside an atom k % 8 selects the
    128-byte row and m % 64 the element."""
    for m in range(T):
        for k in range(T):
            a = (m >> 6) * 1024 + (k >> 3) * 2048 + (k & 7) * 128 + 2 * (m & 63)
            assert sw128(a) == swz(k, m)  # element (m, k) of A^T is element (k, m) of the tile


def pack(upper, n, d):
    N = n * d
    NT = -(-N // T)
    A = synth.dense_from_upper(np.asarray(upper, dtype=np.float64), n, d)
    A[np.diag_indices(N)] -= 1.0
    Aoff = np.zeros((NT * T, NT * T))
    Aoff[:N, :N] = A
    bi = np.arange(NT * T) // d
    upper_mask = bi[None, :] > bi[:, None]
    tiles = {}
    for I in range(NT):
        for J in range(I, NT):
            tiles[(I, J)] = np.where(upper_mask[I * T:(I + 1) * T, J * T:(J + 1) * T],
                                     Aoff[I * T:(I + 1) * T, J * T:(J + 1) * T], 0.0)
    return Aoff, tiles, NT


@pytest.mark.parametrize("n,d", [(2, 16), (9, 16), (8, 16), (20, 32), (5, 64), (3, 64)])
def test_tiles_cover_the_upper_triangle_once_and_rebuild_the_product(n, d):
    inst = synth.make_instance(n, d, 0.5, seed=n * d)
    Aoff, tiles, NT = pack(inst.upper, n, d)
    N = n * d
    assert len(tiles) == NT * (NT + 1) // 2
    hit = np.zeros((NT * T, NT * T), dtype=int)
    X = np.zeros((NT * T, d))
    X[:N] = np.random.default_rng(d).standard_normal((N, d))
    Y = np.zeros((NT * T, d))
    for (I, J), t in tiles.items():
        hit[I * T:(I + 1) * T, J * T:(J + 1) * T] += (t != 0)
        Y[I * T:(I + 1) * T] += t @ X[J * T:(J + 1) * T]      # D1 = A_IJ X_J
        Y[J * T:(J + 1) * T] += t.T @ X[I * T:(I + 1) * T]    # D2 = A_IJ^T X_I
    bi = np.arange(NT * T) // d
    strict_upper = (bi[None, :] > bi[:, None]) & (np.arange(NT * T)[:, None] < N) & (np.arange(NT * T)[None, :] < N)
    assert np.all(hit[strict_upper] == 1)
    assert np.all(hit[~strict_upper] == 0)
    assert np.allclose(Y[:N], Aoff[:N, :N] @ X[:N], atol=1e-10)
    assert np.all(Y[N:] == 0.0)


@pytest.mark.parametrize("n,d", [(2, 16), (100, 16), (2000, 16), (50, 32), (1000, 32), (7, 64), (500, 64)])
def test_packed_bytes_match_library(n, d):
    L = pytest.importorskip("paper_2604_07372_gb300._lib")
    try:
        lib = L.lib()
    except RuntimeError:
        pytest.skip("libnsrgs.so not built")
    NT = -(-(n * d) // T)
    assert lib.nsrgs_packed_bytes(n, d, L.BF16) == NT * (NT + 1) // 2 * 32768


def order(NT, R):
    """The processing (and storage) order: (I, J) of every stored tile."""
    out = []
    for g in range(-(-NT // R)):
        I0 = g * R
        Rg = min(R, NT - I0)
        for J in range(I0, NT):
            for r in range(min(Rg, J - I0 + 1)):
                out.append((I0 + r, J))
    return out


def seek(t, NT, R):
    """Position t -> (I, J) as the kernel and the packer compute it."""
    base, g = 0, 0
    while True:
        L = NT - g * R
        Rg = min(R, L)
        cnt = Rg * (Rg + 1) // 2 + (L - Rg) * Rg
        if t < base + cnt:
            break
        base += cnt
        g += 1
    I0, Rg = g * R, min(R, NT - g * R)
    u = t - base
    tri = Rg * (Rg + 1) // 2
    if u < tri:
        c = 0
        while u >= c + 1:
            u -= c + 1
            c += 1
        return I0 + u, I0 + c
    u -= tri
    return I0 + u % Rg, I0 + Rg + u // Rg


@pytest.mark.parametrize("NT,R", [(1, 8), (2, 8), (8, 8), (9, 8), (17, 8), (30, 4), (7, 4), (125, 8)])
def test_processing_order_covers_each_tile_once_and_seek_inverts_it(NT, R):
    seq = order(NT, R)
    assert len(seq) == NT * (NT + 1) // 2
    assert len(set(seq)) == len(seq) and all(I <= J for I, J in seq)
    assert all(seek(t, NT, R) == ij for t, ij in enumerate(seq))
