"""Bit-exact check of the reduced-precision packers (a1): the bytes the GPU
writes into the symmetric panel layout are read back and compared, slot by
slot, with a host quantiser written from the storage rule stated in
include/nsrgs.h:

  * BF16: each float32 element rounded to bfloat16, round to nearest even
    (torch's float32 -> bfloat16 conversion rounds that way);
  * FP8-E4M3: one float32 scale per block row, s_i = max_{j > i} max |A_ij| / 448
    (1 for an all-zero row), computed in float32; the element A_ij / s_i
    (float32 division) rounded to nearest, saturating at +-448 (clamped, then
    torch's float8_e4m3fn conversion, which rounds to nearest even);
  * FP32: the element itself.

Unstored positions of a stored slice (on or below the block diagonal, past
row or column n*d) must hold exact zeros.  The slot order comes from the
NumPy layout model of tests/_panel_model.py, which the CPU tests check
against the library's sizes.  The product test then multiplies with the
host-quantised matrix: the GPU's product must match the float64 product of
those exact stored values to float32 accumulation accuracy, which a different
rounding rule (toward zero, or a per-tensor scale) would not.
"""
import numpy as np
import pytest
import torch

import synth
from _panel_model import Geom, slot_coords, walk

pytestmark = pytest.mark.gpu

F32, BF16, FP8 = 0, 1, 2


@pytest.fixture(scope="module")
def P():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2604_07372_gb300 as P

    return P


def strict_upper(inst):
    """A_off restricted to the strict block-upper triangle (float32), zeros elsewhere."""
    n, d = inst.n, inst.d
    A = inst.dense(dtype=np.float32)
    mask = np.zeros((n * d, n * d), dtype=bool)
    for i in range(n):
        mask[i * d : (i + 1) * d, (i + 1) * d :] = True
    return np.where(mask, A, np.float32(0.0)).astype(np.float32)


def fp8_scales(U, n, d):
    """s_i = max_{j > i} max |A_ij| / 448 in float32 (1 for an all-zero block row)."""
    m = np.abs(U).reshape(n, d, n * d).max(axis=(1, 2)).astype(np.float32)
    return np.where(m > 0, m / np.float32(448.0), np.float32(1.0)).astype(np.float32)


def quantise(vals, storage, scale_rows=None):
    """Host quantiser: float32 values -> the stored bytes (as unsigned integers)."""
    t = torch.from_numpy(np.ascontiguousarray(vals, dtype=np.float32))
    if storage == F32:
        return t.view(torch.int32).numpy().view(np.uint32)
    if storage == BF16:
        return t.to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    q = (t / torch.from_numpy(scale_rows)).clamp(-448.0, 448.0)
    return q.to(torch.float8_e4m3fn).view(torch.uint8).numpy()


def dequantise(U, storage, s, n, d):
    """float64 values of the stored matrix (exact: bf16 and e4m3 values are float32-representable)."""
    if storage == F32:
        return U.astype(np.float64)
    t = torch.from_numpy(U)
    if storage == BF16:
        return t.to(torch.bfloat16).double().numpy()
    rows = np.repeat(s, d)[:, None].astype(np.float32)
    q = (t / torch.from_numpy(rows)).clamp(-448.0, 448.0).to(torch.float8_e4m3fn).double().numpy()
    return q * rows.astype(np.float64)


@pytest.mark.parametrize("storage", [F32, BF16, FP8])
@pytest.mark.parametrize("n,d", [(131, 3), (2000, 3), (131, 4), (2000, 4), (300, 1), (97, 2)])
def test_packed_bytes_match_the_host_quantiser(P, n, d, storage):
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=n * 3 + d, dtype=np.float32)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, storage)
    torch.cuda.synchronize()
    buf = pa.buf.cpu().numpy()
    g = Geom(n, d, storage)
    assert buf.size == g.header_bytes() + g.panel_bytes()
    U = strict_upper(inst)
    N = n * d
    s = None
    if storage == FP8:
        s = fp8_scales(U, n, d)
        off_scale = 16 * (g.nslabs + 1)
        got_s = buf[off_scale : off_scale + 4 * n].view(np.uint32)
        assert np.array_equal(got_s, s.view(np.uint32)), "per-block-row scales differ"
    elem = {F32: np.uint32, BF16: np.uint16, FP8: np.uint8}[storage]
    hb = g.header_bytes()
    checked = 0
    for b, q, W, off in walk(g):
        rows, cols = slot_coords(g, b, q, W)
        inside = (rows < N) & (cols < N)
        vals = np.zeros(rows.shape, dtype=np.float32)
        vals[inside] = U[rows[inside], cols[inside]]
        srow = None
        if storage == FP8:
            srow = np.where(inside, s[np.minimum(rows, N - 1) // d], np.float32(1.0)).astype(np.float32)
        want = quantise(vals, storage, srow)
        got = buf[hb + off : hb + off + W * g.WB].view(elem)
        if not np.array_equal(got, want):
            bad = np.nonzero(got != want)[0][:5]
            raise AssertionError(f"step (b={b}, q={q}): slots {bad} rows {rows[bad]} cols {cols[bad]} "
                                 f"got {got[bad]} want {want[bad]} (value {vals[bad]})")
        checked += int(np.count_nonzero(inside & (cols // d > rows // d)))
    assert checked == n * (n - 1) // 2 * d * d


@pytest.mark.parametrize("storage", [BF16, FP8])
@pytest.mark.parametrize("n,d", [(131, 3), (2000, 3), (1537, 4), (513, 1)])
def test_product_uses_exactly_the_stored_values(P, n, d, storage):
    """Y = A_off X through the reduced-precision panels equals the float64
    product of the host-quantised A to float32 accumulation accuracy."""
    inst = synth.make_instance(n, d, 0.5, seed=n + 11 * d, dtype=np.float32)
    U = strict_upper(inst)
    s = fp8_scales(U, n, d) if storage == FP8 else None
    Uq = dequantise(U, storage, s, n, d)
    Aq = Uq + Uq.T  # the stored upper triangle and its mirror
    X = np.random.default_rng(n).standard_normal((n * d, d)).astype(np.float32)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, storage)
    Y = P.nsrgs_product(pa, torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    ref = Aq @ X.astype(np.float64)
    scale = np.abs(Aq) @ np.abs(X.astype(np.float64))
    err = np.abs(Y.double().cpu().numpy() - ref)
    assert np.all(err <= 2e-6 * scale + 1e-6), float(np.max(err / (scale + 1e-6)))


@pytest.mark.parametrize("n,d", [(131, 3), (200, 4)])
def test_dense_and_upper_sources_pack_the_same_bytes(P, n, d):
    """The tables, the FP8 scales and the panels are the same from either source
    (the header's alignment padding is left unwritten by both)."""
    inst = synth.make_instance(n, d, 0.4, seed=5 * n + d, dtype=np.float32)
    for storage in (BF16, FP8):
        a = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, storage)
        b = P.nsrgs_pack_dense(torch.from_numpy(inst.dense(dtype=np.float32)).cuda(), n, d, storage)
        torch.cuda.synchronize()
        g = Geom(n, d, storage)
        tab = 16 * (g.nslabs + 1)
        parts = [(0, tab), (g.header_bytes(), g.header_bytes() + g.panel_bytes())]
        if storage == FP8:
            parts.append((tab, tab + 4 * n))
        for lo, hi in parts:
            assert torch.equal(a.buf[lo:hi], b.buf[lo:hi]), (storage, lo, hi)
