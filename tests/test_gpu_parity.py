"""GPU parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Both sides receive the same float32 inputs from the seeded generator.  Bars:
  * one iteration: max |X_gpu - X_oracle| <= 2e-5 elementwise (float32 A X with
    n terms, then the eta = 1/n step: the error is a few float32 ulps of O(1));
  * whole solves: d_F(X_gpu, X_oracle) / sqrt(nd) <= 1e-5 (the stated bar);
  * reduced-precision storage: final d_F(X, Z) within 1% of the oracle's.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session")
def P():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2604_07372_gb300 as P

    return P


def make(n, d, c=0.3, seed=0, p=1.0):
    return synth.make_instance(n, d, synth.sigma_rule(c, n, d), seed=seed, p=p, dtype=np.float32)


def packed(P, inst, storage):
    up = torch.from_numpy(inst.upper).cuda()
    return P.nsrgs_pack_upper(up, inst.n, inst.d, storage)


def to64(t):
    return t.detach().double().cpu().numpy()


@pytest.mark.parametrize("storage", ["f32", "bf16", "fp8", "dense_f32"])
@pytest.mark.parametrize("n,d", [(2, 3), (5, 2), (131, 3), (257, 4), (513, 1), (2000, 3), (1537, 4)])
def test_product_matches_dense_matmul(P, n, d, storage):
    """a2 alone: Y = A_off X through nsrgs_product vs the float64 product of the same stored values."""
    inst = make(n, d, c=0.5, seed=n + 7 * d)
    A = inst.dense()
    for i in range(n):
        A[i * d : (i + 1) * d, i * d : (i + 1) * d] = 0.0
    X = np.random.default_rng(n).standard_normal((n * d, d)).astype(np.float32)
    pa = packed(P, inst, P.STORAGE[storage])
    Y = P.nsrgs_product(pa, torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    ref = A @ X.astype(np.float64)
    scale = np.abs(A) @ np.abs(X.astype(np.float64))  # sum of |terms| per output
    got = to64(Y)
    if storage in ("f32", "dense_f32"):
        assert np.all(np.abs(got - ref) <= 1e-6 * scale + 1e-6)
    elif storage == "bf16":
        # round to nearest with an 8-bit significand: |err| <= 2^-8 |a| per element
        # (2^-8 is the round-to-nearest worst case; tests/test_gpu_quantiser.py checks
        # the rounding rule itself bit for bit)
        assert np.all(np.abs(got - ref) <= 2.0**-8 * scale + 1e-6 * scale + 1e-6)
    else:
        # e4m3, round to nearest (4-bit significand): |err| <= 2^-4 |a| for normal
        # values, and at most half the subnormal spacing, 2^-10 s_i, below 2^-6 s_i
        s_row = np.abs(A).reshape(n, d, n * d).max(axis=(1, 2)) / 448.0
        S = np.repeat(np.where(s_row > 0, s_row, 1.0), d)
        mask = np.zeros_like(A, dtype=bool)
        for i in range(n):
            mask[i * d : (i + 1) * d, (i + 1) * d :] = True
        Srow = np.where(mask, S[:, None], 0.0)
        Sfull = Srow + Srow.T  # a mirrored element carries its stored block's scale
        sub = 2.0**-10 * (Sfull @ np.abs(X.astype(np.float64)))
        assert np.all(np.abs(got - ref) <= 2.0**-4 * scale + sub + 1e-6 * scale + 1e-6)


STEP_CASES = [(2, 3), (3, 1), (5, 2), (130, 3), (200, 3), (257, 4), (131, 2), (513, 1), (700, 3), (1025, 4)]


@pytest.mark.parametrize("storage", ["f32", "dense_f32"])
@pytest.mark.parametrize("n,d", STEP_CASES)
def test_one_iteration_matches_oracle(P, n, d, storage):
    inst = make(n, d, seed=n * 10 + d)
    A = inst.dense()
    X0, _ = O.spectral_init(A, n, d)
    X0 = X0.astype(np.float32).astype(np.float64)
    ref = O.nsrgs_iteration(A, X0, n, d, 1.0 / n, 2)
    pa = packed(P, inst, P.STORAGE[storage])
    Xin = torch.from_numpy(X0.astype(np.float32)).cuda()
    Xout = torch.empty_like(Xin)
    un = torch.zeros(1, dtype=torch.float64, device="cuda")
    P.nsrgs_step(pa, 1.0 / n, 2, Xin, Xout, upd_norm=un)
    torch.cuda.synchronize()
    got = to64(Xout)
    assert np.max(np.abs(got - ref)) <= 2e-5
    assert abs(un.item() - O.update_norm(ref, X0)) <= 1e-5


def test_step_is_linear_in_A_row_and_column_contributions(P):
    """K = 0 and X = I blocks: X_out - X = -eta P((n-1)I - Y) exercises the row and column paths separately."""
    n, d = 300, 3
    inst = make(n, d, seed=3)
    A = inst.dense()
    Xb = np.tile(np.eye(d), (n, 1))
    ref = O.nsrgs_iteration(A, Xb, n, d, 0.5 / n, 0)
    pa = packed(P, inst, P.F32)
    Xin = torch.from_numpy(Xb.astype(np.float32)).cuda()
    Xout = torch.empty_like(Xin)
    P.nsrgs_step(pa, 0.5 / n, 0, Xin, Xout)
    torch.cuda.synchronize()
    assert np.max(np.abs(to64(Xout) - ref)) <= 2e-5


@pytest.mark.parametrize("n,d", [(200, 3), (1000, 3), (300, 2), (150, 4), (400, 1)])
def test_spectral_init_matches_oracle(P, n, d):
    inst = make(n, d, seed=7 + n)
    X0o, _ = O.spectral_init(inst.dense(), n, d)
    pa = packed(P, inst, P.F32)
    X0, res = P.nsrgs_spectral_init(pa, max_iters=80, tol=1e-6)
    torch.cuda.synchronize()
    assert res <= 1e-6
    assert O.dF(to64(X0), X0o, d) / math.sqrt(n * d) <= 1e-5


FLAG_SPEC_SHIFTED = 1 << 6


@pytest.mark.parametrize("n,d,storage", [(120, 3, "f32"), (100, 4, "f32"), (90, 2, "dense_f32"), (40, 10, "dense_f32"),
                                         (30, 16, "dense_f32")])
def test_spectral_start_takes_the_algebraic_top_d(P, n, d, storage):
    """Algorithm 2's start uses the d largest eigenvalues of A.  Here the d
    eigenvalues of largest magnitude are negative (about -1.5 n, against the
    signal's n), so subspace iteration on A alone would converge to them; the
    start must detect that (its Ritz values fail the positive-definiteness
    test), restart with a larger shift and match the oracle's eigh top d."""
    inst = synth.make_negative_dominated(n, d, seed=40 + n + d)
    A = inst.dense()
    w = np.linalg.eigvalsh(A)
    assert abs(w[0]) > 1.2 * w[-1]  # the construction: magnitude-dominant eigenvalues are negative
    X0o, _ = O.spectral_init(A, n, d)
    pa = packed(P, inst, P.STORAGE[storage])
    X, info = P.nsrgs_solve(pa, 1.0 / n, 0, 2, init=True, spectral_max_iters=400)
    torch.cuda.synchronize()
    assert info.flags & FLAG_SPEC_SHIFTED, info.as_dict()
    assert info.spectral_residual <= 1e-6 and not (info.flags & 4), info.as_dict()
    assert O.dF(to64(X), X0o, d) / math.sqrt(n * d) <= 1e-5
    # nsrgs_spectral_init reports convergence the same way
    X1, res = P.nsrgs_spectral_init(pa, max_iters=400, tol=1e-6)
    torch.cuda.synchronize()
    assert res <= 1e-6 and O.dF(to64(X1), X0o, d) / math.sqrt(n * d) <= 1e-5


@pytest.mark.parametrize("storage", ["f32", "dense_f32"])
def test_solve_config1_parity(P, storage):
    """n = 200, d = 3, sigma by the c = 0.3 rule, spectral start, T = 50, K = 2."""
    n, d, T, K = 200, 3, 50, 2
    inst = make(n, d, seed=2026)
    A = inst.dense()
    Xo, _ = O.nsrgs(A, n, d, 1.0 / n, T, K)
    pa = packed(P, inst, P.STORAGE[storage])
    X, info = P.nsrgs_solve(pa, 1.0 / n, T, K, init=True, spectral_max_iters=80)
    torch.cuda.synchronize()
    assert info.iters == T and info.flags == 0, info.as_dict()
    assert O.dF(to64(X), Xo, d) / math.sqrt(n * d) <= 1e-5
    # a second replay of the cached graph gives the same answer
    X2, info2 = P.nsrgs_solve(pa, 1.0 / n, T, K, init=True, spectral_max_iters=80, X=torch.empty_like(X))
    torch.cuda.synchronize()
    assert O.dF(to64(X2), Xo, d) / math.sqrt(n * d) <= 1e-5


def test_solve_from_given_start(P):
    n, d, T, K = 257, 3, 30, 2
    inst = make(n, d, seed=11)
    A = inst.dense()
    X0, _ = O.spectral_init(A, n, d)
    Xo, _ = O.nsrgs(A, n, d, 1.0 / n, T, K, X0=X0)
    pa = packed(P, inst, P.F32)
    X = torch.from_numpy(X0.astype(np.float32)).cuda()
    X, info = P.nsrgs_solve(pa, 1.0 / n, T, K, init=False, X=X)
    torch.cuda.synchronize()
    assert O.dF(to64(X), Xo, d) / math.sqrt(n * d) <= 1e-5


@pytest.mark.parametrize("storage", ["f32", "bcsr_f32"])
def test_solve_from_host_buffers(P, storage):
    """nsrgs_solve_host: packed A and X in (pinned) host memory, one call, same
    answer as the oracle; from the spectral start and from a given X^0."""
    n, d, T, K = 200, 3, 40, 2
    inst = make(n, d, seed=7, p=0.5 if storage == "bcsr_f32" else 1.0)
    A = inst.dense()
    Xo, _ = O.nsrgs(A, n, d, 1.0 / n, T, K)
    pa = packed(P, inst, P.STORAGE[storage])
    host = torch.empty(pa.nbytes, dtype=torch.uint8, pin_memory=True)
    host.copy_(pa.buf[: pa.nbytes])
    torch.cuda.synchronize()
    pa.buf.zero_()
    Xh = torch.full((n * d, d), float("nan"), dtype=torch.float32, pin_memory=True)
    Xh, info = P.nsrgs_solve_host(pa, host, Xh, 1.0 / n, T, K, init=True, spectral_max_iters=80)
    assert info.iters == T and info.flags == 0, info.as_dict()
    assert O.dF(Xh.double().numpy(), Xo, d) / math.sqrt(n * d) <= 1e-5
    X0, _ = O.spectral_init(A, n, d)
    Xo0, _ = O.nsrgs(A, n, d, 1.0 / n, T, K, X0=X0)
    Xh = torch.from_numpy(X0.astype(np.float32)).contiguous()
    Xh, info = P.nsrgs_solve_host(pa, host, Xh, 1.0 / n, T, K, init=False)
    assert O.dF(Xh.double().numpy(), Xo0, d) / math.sqrt(n * d) <= 1e-5
    # a host buffer of the wrong size is rejected before anything is copied
    with pytest.raises(P.NsrgsError):
        P.nsrgs_solve_host(pa, host[:-16], Xh, 1.0 / n, T, K)


def test_sigma_zero_exact_recovery_gpu(P):
    n, d = 200, 3
    inst = synth.make_instance(n, d, 0.0, seed=5, dtype=np.float32)
    pa = packed(P, inst, P.F32)
    X, info = P.nsrgs_solve(pa, 1.0 / n, 50, 2)
    torch.cuda.synchronize()
    assert O.dF(to64(X), inst.Zstack(), d) / math.sqrt(n * d) <= 1e-5


def test_tol_stops_early_like_the_oracle(P):
    n, d, K, tol = 200, 3, 2, 1e-6
    inst = make(n, d, seed=9)
    A = inst.dense()
    _, hist = O.nsrgs(A, n, d, 1.0 / n, 60, K, history=True)
    t_oracle = next(t + 1 for t, u in enumerate(hist["upd"]) if u < tol)
    pa = packed(P, inst, P.F32)
    X, info = P.nsrgs_solve(pa, 1.0 / n, 60, K, tol=tol)
    torch.cuda.synchronize()
    assert info.last_update_norm < tol
    assert abs(info.iters - t_oracle) <= 1


@pytest.mark.parametrize("n,d", [(50, 1), (64, 2), (200, 3), (333, 4), (100, 8)])
def test_dF_matches_oracle(P, n, d):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n * d, d)).astype(np.float32)
    Y = rng.standard_normal((n * d, d)).astype(np.float32)
    got = P.nsrgs_dF(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), n, d)
    ref = O.dF(X.astype(np.float64), Y.astype(np.float64), d)
    assert abs(got - ref) <= 1e-9 * ref


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
@pytest.mark.parametrize("n", [200, 2000])
def test_reduced_precision_final_error_within_one_percent(P, n, storage):
    d, T, K = 3, 50, 2
    inst = make(n, d, seed=31)
    Z = inst.Zstack()
    # the FP64 oracle on the unrounded A (at n = 2000 the dense A is 6000 x 6000, 288 MB)
    Xo, _ = O.nsrgs(inst.dense(), n, d, 1.0 / n, T, K)
    ref = O.dF(Xo, Z, d)
    X, info = P.nsrgs_solve(packed(P, inst, P.STORAGE[storage]), 1.0 / n, T, K)
    torch.cuda.synchronize()
    got = O.dF(to64(X), Z, d)
    assert abs(got - ref) / ref <= 0.01, (got, ref)


def test_nonfinite_is_reported(P):
    n, d = 64, 3
    inst = make(n, d, seed=1)
    pa = packed(P, inst, P.F32)
    with pytest.raises(P.NsrgsError) as e:
        P.nsrgs_solve(pa, 40.0 / n, 40, 2)
    assert e.value.status in (4,)


@pytest.mark.slow
def test_full_size_sampled_blocks(P):
    """n = 10^4, d = 3 (A is 30000 x 30000): one GPU iteration, 48 sampled blocks checked one by one."""
    n, d = 10000, 3
    inst = make(n, d, seed=77)
    pa = packed(P, inst, P.F32)
    X0, res = P.nsrgs_spectral_init(pa, max_iters=60, tol=1e-6)
    assert res <= 1e-6
    Xout = torch.empty_like(X0)
    P.nsrgs_step(pa, 1.0 / n, 2, X0, Xout)
    torch.cuda.synchronize()
    X0h = to64(X0)
    idx = list(np.random.default_rng(0).choice(n, size=48, replace=False)) + [0, n - 1]
    rows = np.stack([synth.block_row(inst.upper, n, d, int(i)) for i in idx])
    ref = O.nsrgs_rows_update(rows, X0h, idx, n, d, 1.0 / n, 2)
    got = O.blocks(to64(Xout), d)[idx]
    assert np.max(np.abs(got - ref)) <= 2e-5
    # spectral start: Y spans the top-d subspace, X0 blocks orthogonal
    Xb = O.blocks(X0h, d)
    assert np.max(np.abs(np.swapaxes(Xb, 1, 2) @ Xb - np.eye(d))) <= 1e-5


@pytest.mark.parametrize("storage", ["f32", "dense_f32"])
def test_gpm_baseline_matches_oracle(P, storage):
    """The GPM baseline (per-block exact sign) against the oracle's GPM, same start."""
    n, d, T = 200, 3, 30
    inst = make(n, d, seed=44)
    A = inst.dense()
    X0, _ = O.spectral_init(A, n, d)
    ref = O.gpm(A, n, d, T, X0=X0)
    pa = packed(P, inst, P.STORAGE[storage])
    X = torch.from_numpy(X0.astype(np.float32)).cuda()
    X, info = P.nsrgs_gpm_solve(pa, T, init=False, X=X)
    torch.cuda.synchronize()
    assert info.iters == T
    assert O.dF(to64(X), ref, d) / math.sqrt(n * d) <= 1e-5
    # GPM and NS-RGS reach the same fixed point (the oracle pins this too)
    Xn, _ = P.nsrgs_solve(pa, 1.0 / n, 120, 2)
    Xg, _ = P.nsrgs_gpm_solve(pa, 120)
    torch.cuda.synchronize()
    assert O.dF(to64(Xn), to64(Xg), d) / math.sqrt(n * d) <= 1e-5
