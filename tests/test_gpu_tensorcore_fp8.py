"""FP8-E4M3 storage on the tile-upper tensor-core stream (NSRGS_FP8E4M3 at d in
{16, 32, 64}; tcgen05 kind::f8f6f4).

  * Packed bytes, bit for bit: every tile against a host quantiser of the
    stated rule (q_ij = RN(A_ij / s_i) saturating at +-448, s_i = max_{j > i}
    max |A_ij| / 448 in float32) placed by the NumPy layout model, and the n
    scales behind the tiles.
  * The product against the exact float64 product of the stored values with the
    operands the kernel multiplies: X as hi + lo E4M3 planes at a power-of-two
    scale (g X for the row product, g' s_i X_i for the column product), to
    float32 accumulation accuracy.  Scaling X by a power of two scales Y by it
    (the same E4M3 codes; only the order of the float32 reductions into Y may
    differ); X = 0 gives Y = 0.
  * Whole solves against the FP64 oracle on the unrounded A, and the objective
    through this layout against the host value of F on the stored matrix.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from _tile_model import T, fp8_tile_bytes, pow2_scale, seek, strip_rows, swz8, tile_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2604_07372_gb300 as P

    return P


def strict_upper(inst):
    """A_off restricted to the strict block-upper triangle (float32), zero elsewhere."""
    n, d = inst.n, inst.d
    A = inst.dense(dtype=np.float32)
    bi = np.arange(n * d) // d
    return np.where(bi[None, :] > bi[:, None], A, np.float32(0.0)).astype(np.float32)


def fp8_scales(U, n, d):
    m = np.abs(U).reshape(n, d, n * d).max(axis=(1, 2)).astype(np.float32)
    return np.where(m > 0, m / np.float32(448.0), np.float32(1.0)).astype(np.float32)


def e4m3_codes(v):
    t = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).clamp(-448.0, 448.0)
    return t.to(torch.float8_e4m3fn)


def e4m3(v):
    return e4m3_codes(v).to(torch.float32).numpy()


def stored(inst):
    """(U, s, Q): the strict upper triangle, the block-row scales and the stored codes' values."""
    n, d = inst.n, inst.d
    U = strict_upper(inst)
    s = fp8_scales(U, n, d)
    rows = np.repeat(s, d)[:, None]
    Q = e4m3(U / rows).astype(np.float64)
    return U, s, Q


def operand(V):
    """hi + lo at the power-of-two scale of max |V|, divided back (float64, exact)."""
    g = pow2_scale(np.max(np.abs(V)))
    v = (V * g).astype(np.float32)
    hi = e4m3(v)
    lo = e4m3(v - hi)
    return (hi.astype(np.float64) + lo) / np.float64(g)


def product_ref(Q, s, X, d):
    srow = np.repeat(s, d).astype(np.float32)
    Xr = operand(X)
    Xc = operand((X * srow[:, None]).astype(np.float32))
    s64 = srow.astype(np.float64)[:, None]
    ref = s64 * (Q @ Xr) + Q.T @ Xc
    scale = s64 * (np.abs(Q) @ np.abs(Xr)) + np.abs(Q).T @ np.abs(Xc)
    return ref, scale


def pack(P, inst):
    return P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), inst.n, inst.d, P.FP8E4M3)


@pytest.mark.parametrize("n,d", [(2, 16), (9, 16), (300, 16), (20, 32), (130, 32), (3, 64), (17, 64), (20, 25),
                                 (9, 12), (5, 48)])
def test_fp8_tiles_match_the_host_quantiser(P, n, d):
    inst = synth.make_instance(n, d, 0.5, seed=4 * n + d, dtype=np.float32)
    pa = pack(P, inst)
    torch.cuda.synchronize()
    buf = pa.buf.cpu().numpy()
    assert buf.size == fp8_tile_bytes(n, d)
    U, s, _ = stored(inst)
    NT = tile_rows(n, d)
    ntiles = NT * (NT + 1) // 2
    off_s = ntiles * 16384
    assert np.array_equal(buf[off_s : off_s + 4 * n].view(np.uint32), s.view(np.uint32)), "block-row scales"
    N = n * d
    Up = np.zeros((NT * T, NT * T), dtype=np.float32)
    Up[:N, :N] = U
    sp = np.ones(NT * T, dtype=np.float32)
    sp[:N] = np.repeat(s, d)
    r, c = np.meshgrid(np.arange(T), np.arange(T), indexing="ij")
    where = swz8(r, c).ravel()
    for t in range(ntiles):
        I, J = seek(t, NT, strip_rows(d, f8=True))
        vals = Up[I * T : (I + 1) * T, J * T : (J + 1) * T] / sp[I * T : (I + 1) * T, None]
        want = np.empty(16384, dtype=np.uint8)
        want[where] = e4m3_codes(vals).view(torch.uint8).numpy().ravel()
        got = buf[t * 16384 : (t + 1) * 16384]
        if not np.array_equal(got, want):
            bad = np.nonzero(got != want)[0][:5]
            raise AssertionError(f"tile {t} = ({I}, {J}): bytes {bad} got {got[bad]} want {want[bad]}")


PRODUCT_CASES = [(2, 16), (20, 16), (8, 16), (300, 16), (1000, 16), (9, 32), (130, 32), (5, 64), (70, 64), (17, 64),
                 (30, 9), (20, 25), (9, 48), (3, 63)]


@pytest.mark.parametrize("n,d", PRODUCT_CASES)
def test_fp8_product_uses_exactly_the_stored_values(P, n, d):
    inst = synth.make_instance(n, d, 0.5, seed=n + 3 * d, dtype=np.float32)
    _, s, Q = stored(inst)
    X = np.random.default_rng(d + n).standard_normal((n * d, d)).astype(np.float32)
    pa = pack(P, inst)
    Y = P.nsrgs_product(pa, torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    ref, scale = product_ref(Q, s, X, d)
    err = np.abs(Y.double().cpu().numpy() - ref)
    assert np.all(err <= 2e-6 * scale + 1e-9 * np.max(scale)), float(np.max(err / (scale + 1e-30)))


@pytest.mark.parametrize("n,d", [(300, 16), (40, 64)])
def test_fp8_product_is_exact_under_power_of_two_scaling(P, n, d):
    """The operand scales are powers of two, so Y(2^k X) = 2^k Y(X) up to the order of the
    float32 reductions into Y (the E4M3 codes are the same); Y(0) = 0."""
    inst = synth.make_instance(n, d, 0.5, seed=n, dtype=np.float32)
    pa = pack(P, inst)
    X = torch.from_numpy(np.random.default_rng(2).standard_normal((n * d, d)).astype(np.float32)).cuda()
    Y0 = P.nsrgs_product(pa, X).clone()
    for k in (-20, 7, 30):
        Yk = P.nsrgs_product(pa, X * (2.0 ** k)).clone()
        torch.cuda.synchronize()
        want = Y0 * (2.0 ** k)
        assert torch.allclose(Yk, want, rtol=1e-5, atol=1e-6 * want.abs().max().item()), k
    Yz = P.nsrgs_product(pa, torch.zeros_like(X))
    torch.cuda.synchronize()
    assert torch.count_nonzero(Yz).item() == 0


@pytest.mark.parametrize("n,d", [(200, 16), (80, 32), (40, 64), (100, 25)])
def test_fp8_solve_within_one_percent_of_the_oracle(P, n, d):
    """Final d_F(X, Z) of an FP8 tile-upper solve within 1% of the FP64 oracle's (unrounded A)."""
    T_, K = 40, 2
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=7 * d, dtype=np.float32)
    Xo, _ = O.nsrgs(inst.dense(), n, d, 1.0 / n, T_, K)
    X, info = P.nsrgs_solve(pack(P, inst), 1.0 / n, T_, K)
    torch.cuda.synchronize()
    Z = inst.Zstack()
    eo = O.dF(Xo, Z, d)
    e8 = O.dF(X.double().cpu().numpy(), Z, d)
    assert info.iters == T_ and not (info.flags & 1), info.as_dict()
    assert abs(e8 - eo) / eo <= 0.01, (eo, e8, info.as_dict())


@pytest.mark.parametrize("n,d", [(300, 16), (40, 64)])
def test_fp8_objective_matches_the_stored_matrix(P, n, d):
    """F(X) of eq. (1) through the FP8 tile layout.  Expanding the square,
    F = ||A_off||^2 / 2 - tr(X^T A_off X) + sum_{i != j} ||X_i X_j^T||^2 / 2: its
    ||A_off||^2 pass (stored triangle once, codes times scales) and its product
    (the kernel's hi / lo operands) against the host value on the stored matrix;
    and within 1e-3 of the oracle's F on the stored matrix with X unrounded."""
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=11 + d, dtype=np.float32)
    _, s, Q = stored(inst)
    X = inst.Zstack().astype(np.float32)
    F = P.nsrgs_objective(pack(P, inst), torch.from_numpy(X).cuda())
    srow = np.repeat(s, d).astype(np.float64)[:, None]
    Aq = srow * Q
    Yref, _ = product_ref(Q, s, X, d)
    X64 = X.astype(np.float64)
    Xb = O.blocks(X64, d)
    Gi = np.swapaxes(Xb, 1, 2) @ Xb
    a2, tr = 2.0 * np.sum(Aq * Aq), np.sum(X64 * Yref)
    xx = np.sum(Gi.sum(axis=0) ** 2) - np.sum(Gi ** 2)
    ref = 0.5 * a2 - tr + 0.5 * xx
    assert abs(F - ref) <= 1e-6 * (0.5 * a2 + abs(tr) + 0.5 * xx), (F, ref)
    Fo = O.objective(Aq + Aq.T, X64, n, d)
    assert abs(F - Fo) <= 1e-3 * abs(Fo), (F, Fo)
