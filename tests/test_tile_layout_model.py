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
The FP8 form (one byte per element, 16 KB tiles, X as hi and lo E4M3 planes)
gets the same checks of its swizzle and operand readings, plus the accuracy of
the hi / lo split and the folding of the block-row scales.
"""
import numpy as np
import pytest

import synth
import torch

from _tile_model import T, fp8_tile_bytes, order, pow2_scale, seek, sw128, swz, swz8


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


@pytest.mark.parametrize("NT,R", [(1, 8), (2, 8), (8, 8), (9, 8), (17, 8), (30, 4), (7, 4), (125, 8), (20, 6), (5, 6)])
def test_processing_order_covers_each_tile_once_and_seek_inverts_it(NT, R):
    seq = order(NT, R)
    assert len(seq) == NT * (NT + 1) // 2
    assert len(set(seq)) == len(seq) and all(I <= J for I, J in seq)
    assert all(seek(t, NT, R) == ij for t, ij in enumerate(seq))


# ---------------------------------------------------------------- FP8 tiles
# The FP8 (E4M3) form of the layout: the same tiles and order, one byte per
# element, so a tile row is exactly one 128-byte swizzle row (16 KB tiles,
# 8-row groups 1024 bytes apart); X travels as hi and lo E4M3 planes of N rows
# of 128 bytes each.


def test_fp8_swizzle_is_a_bijection_of_a_tile():
    r, c = np.meshgrid(np.arange(T), np.arange(T), indexing="ij")
    off = swz8(r, c)
    assert off.min() == 0 and off.max() == 16384 - 1
    assert np.unique(off).size == T * T
    assert np.array_equal(ts8_row_of(off), r)


def ts8_row_of(o):
    """Row of the byte at offset o of a one-byte tile (the objective pass decodes rows this way)."""
    return (o >> 10) * 8 + ((o >> 7) & 7)


def test_fp8_k_major_reading_addresses_the_tile():
    """K-major operand (SBO = 1024 between 8-row groups; the K = 32 step kk starts 32 kk
    bytes into the row): element (m, 32 kk + k) is at the swizzled unswizzled address."""
    for m in range(T):
        for kk in range(4):
            for k in range(32):
                a = 32 * kk + (m >> 3) * 1024 + (m & 7) * 128 + k
                assert sw128(a) == swz8(m, 32 * kk + k)


def test_fp8_mn_major_reading_addresses_the_transpose():
    """MN-major operand (A^T, M = tile columns = one 128-element MN atom, K = tile rows):
    K = 32 step kk starts at 4096 kk, K groups of 8 rows at SBO = 1024."""
    for kk in range(4):
        for k in range(32):
            kr = 32 * kk + k
            for m in range(T):
                a = 4096 * kk + (k >> 3) * 1024 + (k & 7) * 128 + m
                assert sw128(a) == swz8(kr, m)


@pytest.mark.parametrize("N", [16, 32, 64])
def test_fp8_x_planes_fill_their_tile(N):
    """hi plane (N x 128 bytes) then lo plane: 256 N bytes per 128-row tile, each slot once."""
    nn, k = np.meshgrid(np.arange(N), np.arange(T), indexing="ij")
    off = np.concatenate([swz8(nn, k).ravel(), N * 128 + swz8(nn, k).ravel()])
    assert np.unique(off).size == 2 * N * T and off.max() == 256 * N - 1
    # a K = 32 step of the B operand (N rows, SBO = 1024) reads columns 32 kk .. 32 kk + 31
    for kk in range(4):
        for n in range(N):
            for kc in range(32):
                a = 32 * kk + (n >> 3) * 1024 + (n & 7) * 128 + kc
                assert sw128(a) == swz8(n, 32 * kk + kc)


def e4m3(v):
    """Round float32 values to E4M3 (nearest even, saturating at +-448), back as float32."""
    t = torch.from_numpy(np.asarray(v, dtype=np.float32)).clamp(-448.0, 448.0)
    return t.to(torch.float8_e4m3fn).to(torch.float32).numpy()


def split(v):
    hi = e4m3(v)
    lo = e4m3(np.asarray(v, dtype=np.float32) - hi)
    return hi, lo


def test_fp8_hi_lo_split_carries_x_to_2_pow_minus_8():
    """hi = RN(v), lo = RN(v - hi) in E4M3 (3 mantissa bits each): |v - hi - lo| <= 2^-8 |v|
    for v in the normal range of both planes, and v - hi is exact in float32."""
    rng = np.random.default_rng(5)
    v = (rng.uniform(-1, 1, 200000) * 2.0 ** rng.uniform(-4, 8, 200000)).astype(np.float32)
    hi, lo = split(v)
    r = v.astype(np.float64) - hi
    assert np.array_equal(r, (v - hi).astype(np.float64))  # exact subtraction
    # lo's rounding error is at most 2^-4 |r| <= 2^-8 |v| where r is a normal E4M3 value,
    # else half the subnormal spacing, 2^-10, which is <= 2^-8 |v| for |v| >= 1/4
    big = np.abs(v) >= 0.25
    err = np.abs(v.astype(np.float64) - hi - lo)
    assert np.all(err[big] <= 2.0 ** -8 * np.abs(v[big]))
    assert np.all(err <= 2.0 ** -8 * np.abs(v) + 2.0 ** -10)  # subnormal floor of lo
    # one plane alone is only good to 2^-4
    assert np.max(np.abs(r[big]) / np.abs(v[big])) > 2.0 ** -5


def test_fp8_operand_scale_is_a_power_of_two_in_range():
    for m in [1e-30, 3e-7, 0.0123, 0.5, 1.0, 1.75, 255.9, 3e5, 1e30]:
        g = pow2_scale(m)
        assert np.log2(g) == int(np.log2(g))
        assert 128.0 <= m * g < 256.0, (m, g)
    assert pow2_scale(0.0) == 1.0


@pytest.mark.parametrize("n,d", [(9, 16), (20, 32), (5, 64)])
def test_fp8_scale_folding_rebuilds_the_product(n, d):
    """With A_ij = s_i Q_ij (one scale per block row), the row product is scaled per output
    row after accumulation and the column product takes s_i into its operand (s runs along
    K there): diag(s) Q X + Q^T (diag(s) X) = A_off X."""
    inst = synth.make_instance(n, d, 0.5, seed=n + d)
    Aoff, tiles, NT = pack(inst.upper, n, d)
    N = n * d
    s = np.abs(Aoff[:N, :N]).reshape(n, d, N).max(axis=(1, 2)) / 448.0
    s[s == 0] = 1.0
    srow = np.zeros(NT * T)
    srow[:N] = np.repeat(s, d)
    X = np.zeros((NT * T, d))
    X[:N] = np.random.default_rng(1).standard_normal((N, d))
    Y = np.zeros((NT * T, d))
    for (I, J), t in tiles.items():
        rs = srow[I * T:(I + 1) * T]
        Q = np.divide(t, rs[:, None], out=np.zeros_like(t), where=rs[:, None] > 0)
        Y[I * T:(I + 1) * T] += rs[:, None] * (Q @ X[J * T:(J + 1) * T])
        Y[J * T:(J + 1) * T] += Q.T @ (rs[:, None] * X[I * T:(I + 1) * T])
    assert np.allclose(Y[:N], Aoff[:N, :N] @ X[:N], atol=1e-10)


@pytest.mark.parametrize("n,d", [(2, 16), (100, 16), (50, 32), (1000, 32), (7, 64), (500, 64)])
def test_fp8_packed_bytes_match_library(n, d):
    L = pytest.importorskip("paper_2604_07372_gb300._lib")
    try:
        lib = L.lib()
    except RuntimeError:
        pytest.skip("libnsrgs.so not built")
    assert lib.nsrgs_packed_bytes(n, d, L.FP8E4M3) == fp8_tile_bytes(n, d)
