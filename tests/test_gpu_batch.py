"""GPU tests of the batched form (nsrgs_batch_solve) through the C ABI.

Each instance is solved alone (nsrgs_solve) and in the batch; the two must
agree to d_F/sqrt(nd) <= 1e-5, and small instances are also checked against
the FP64 oracle with the same bar.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2604_07372_gb300 as P

    return P


def inst(n, d, c, seed, p=1.0):
    return synth.make_instance(n, d, synth.sigma_rule(c, n, d), seed=seed, p=p, dtype=np.float32)


def pack(P, I, storage):
    return P.nsrgs_pack_upper(torch.from_numpy(I.upper).cuda(), I.n, I.d, storage)


def to64(t):
    return t.detach().double().cpu().numpy()


@pytest.mark.parametrize("d", [3, 1, 2, 4])
def test_each_instance_alone_and_in_the_batch(P, d):
    ns = [2, 3, 50, 129, 200, 257, 300, 64, 513, 90]
    insts = [inst(n, d, 0.3, seed=100 * d + k) for k, n in enumerate(ns)]
    packs = [pack(P, I, P.F32) for I in insts]
    etas = [1.0 / I.n for I in insts]
    T, K = 30, 2
    Xs, infos = P.nsrgs_batch_solve(packs, etas, T, K, init=True, spectral_max_iters=60)
    torch.cuda.synchronize()
    for I, pa, X, info in zip(insts, packs, Xs, infos):
        Xa, ia = P.nsrgs_solve(pa, 1.0 / I.n, T, K, init=True, spectral_max_iters=60)
        torch.cuda.synchronize()
        assert info.iters == T, info.as_dict()
        assert O.dF(to64(X), to64(Xa), d) / math.sqrt(I.n * d) <= 1e-5, (I.n, info.as_dict(), ia.as_dict())


def test_batch_matches_oracle(P):
    d, T, K = 3, 40, 2
    insts = [inst(n, d, c, seed=s) for n, c, s in [(120, 0.3, 1), (200, 0.2, 2), (77, 0.4, 3), (160, 0.1, 4)]]
    packs = [pack(P, I, P.F32) for I in insts]
    Xs, infos = P.nsrgs_batch_solve(packs, [1.0 / I.n for I in insts], T, K)
    torch.cuda.synchronize()
    for I, X in zip(insts, Xs):
        Xo, _ = O.nsrgs(I.dense(), I.n, d, 1.0 / I.n, T, K)
        assert O.dF(to64(X), Xo, d) / math.sqrt(I.n * d) <= 1e-5


def test_batch_per_instance_stop_matches_alone(P):
    d, K, tol = 3, 2, 1e-6
    insts = [inst(n, d, c, seed=s) for n, c, s in [(150, 0.3, 5), (400, 0.2, 6), (90, 0.45, 7)]]
    packs = [pack(P, I, P.F32) for I in insts]
    Xs, infos = P.nsrgs_batch_solve(packs, [1.0 / I.n for I in insts], 200, K, tol=tol)
    torch.cuda.synchronize()
    for I, pa, X, info in zip(insts, packs, Xs, infos):
        Xa, ia = P.nsrgs_solve(pa, 1.0 / I.n, 200, K, tol=tol)
        torch.cuda.synchronize()
        assert info.last_update_norm < tol
        assert abs(info.iters - ia.iters) <= 1
        assert O.dF(to64(X), to64(Xa), d) / math.sqrt(I.n * d) <= 1e-5


def test_batch_given_start(P):
    d, T, K = 3, 20, 2
    insts = [inst(n, d, 0.3, seed=s) for n, s in [(100, 8), (233, 9)]]
    packs = [pack(P, I, P.F32) for I in insts]
    X0s = []
    for I in insts:
        X0, _ = O.spectral_init(I.dense(), I.n, d)
        X0s.append(torch.from_numpy(X0.astype(np.float32)).cuda())
    refs = [O.nsrgs(I.dense(), I.n, d, 1.0 / I.n, T, K, X0=to64(x0))[0] for I, x0 in zip(insts, X0s)]
    Xs, infos = P.nsrgs_batch_solve(packs, [1.0 / I.n for I in insts], T, K, init=False, Xs=[x.clone() for x in X0s])
    torch.cuda.synchronize()
    for I, X, ref in zip(insts, Xs, refs):
        assert O.dF(to64(X), ref, d) / math.sqrt(I.n * d) <= 1e-5


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_batch_reduced_precision_within_one_percent(P, storage):
    """Config-4 shape in miniature: n in [50, 2000], c in [0.1, 0.5], own seeds, T = 60, K = 2."""
    rng = np.random.default_rng(42)
    d, T, K = 3, 60, 2
    insts = [inst(int(n), d, float(c), seed=1000 + k) for k, (n, c) in enumerate(zip(rng.integers(50, 2001, 8), rng.uniform(0.1, 0.5, 8)))]
    f32 = [pack(P, I, P.F32) for I in insts]
    red = [pack(P, I, P.STORAGE[storage]) for I in insts]
    etas = [1.0 / I.n for I in insts]
    Xf, _ = P.nsrgs_batch_solve(f32, etas, T, K)
    Xr, _ = P.nsrgs_batch_solve(red, etas, T, K)
    torch.cuda.synchronize()
    for I, a, b in zip(insts, Xf, Xr):
        Z = I.Zstack()
        ea, eb = O.dF(to64(a), Z, d), O.dF(to64(b), Z, d)
        assert abs(eb - ea) / ea <= 0.01, (I.n, ea, eb)


@pytest.mark.parametrize("storage", ["bcsr_f32", "bcsr_bf16"])
def test_block_sparse_batch_alone_and_against_oracle(P, storage):
    """Block-sparse rows in the batched form (warp-per-row kernel over every
    instance's rows): each instance equals its single-instance solve, and the
    F32 batch matches the oracle."""
    d, T, K = 3, 30, 2
    specs = [(2, 0.3, 1.0), (150, 0.3, 0.2), (300, 0.2, 0.05), (77, 0.4, 0.5), (64, 0.3, 1.0)]
    insts = [inst(n, d, c, seed=900 + k, p=p) for k, (n, c, p) in enumerate(specs)]
    st = P.STORAGE[storage]
    packs = [pack(P, I, st) for I in insts]
    Xs, infos = P.nsrgs_batch_solve(packs, [1.0 / I.n for I in insts], T, K, spectral_max_iters=80)
    torch.cuda.synchronize()
    for I, pa, X, info in zip(insts, packs, Xs, infos):
        assert info.iters == T
        Xa, _ = P.nsrgs_solve(pa, 1.0 / I.n, T, K, spectral_max_iters=80)
        torch.cuda.synchronize()
        assert O.dF(to64(X), to64(Xa), d) / math.sqrt(I.n * d) <= 1e-5
        if storage == "bcsr_f32" and I.n > 2:
            Xo, _ = O.nsrgs(I.dense(), I.n, d, 1.0 / I.n, T, K)
            assert O.dF(to64(X), Xo, d) / math.sqrt(I.n * d) <= 1e-5


def test_batched_spectral_start_takes_the_algebraic_top_d(P):
    """An instance whose magnitude-dominant eigenvalues are negative, batched with
    ordinary ones: its spectral phase restarts under a larger shift (flag bit 6)
    and every instance's start and final iterate match the oracle's."""
    d, T, K = 3, 20, 2
    insts = [synth.make_negative_dominated(120, d, seed=3), inst(150, d, 0.3, seed=8),
             synth.make_negative_dominated(90, d, seed=5, beta=2.0), inst(60, d, 0.3, seed=9)]
    packs = [pack(P, I, P.F32) for I in insts]
    Xs, infos = P.nsrgs_batch_solve(packs, [1.0 / I.n for I in insts], T, K, init=True, spectral_max_iters=400)
    torch.cuda.synchronize()
    for k, (I, X, info) in enumerate(zip(insts, Xs, infos)):
        A = I.dense()
        Xo, _ = O.nsrgs(A, I.n, d, 1.0 / I.n, T, K)
        shifted = bool(info.flags & (1 << 6))
        assert shifted == (k in (0, 2)), (k, info.as_dict())
        assert info.iters == T and info.spectral_residual <= 1e-6, info.as_dict()
        assert O.dF(to64(X), Xo, d) / math.sqrt(I.n * d) <= 1e-5, (k, info.as_dict())
