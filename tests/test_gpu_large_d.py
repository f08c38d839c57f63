"""GPU parity for block sizes above 8 (the dimension sweep d in {16, 32, 64} and
the paper's own d = 25): dense storage for A, shared-memory per-block kernels."""
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


def to64(t):
    return t.detach().double().cpu().numpy()


CASES = [(60, 16), (40, 25), (30, 32), (20, 64), (50, 9)]


@pytest.mark.parametrize("n,d", CASES)
def test_one_iteration_large_d(P, n, d):
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=d, dtype=np.float32)
    A = inst.dense()
    X0, _ = O.spectral_init(A, n, d)
    X0 = X0.astype(np.float32).astype(np.float64)
    ref = O.nsrgs_iteration(A, X0, n, d, 1.0 / n, 2)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.DENSE_F32)
    Xout = torch.empty(n * d, d, device="cuda")
    P.nsrgs_step(pa, 1.0 / n, 2, torch.from_numpy(X0.astype(np.float32)).cuda(), Xout)
    torch.cuda.synchronize()
    assert np.max(np.abs(to64(Xout) - ref)) <= 3e-5


@pytest.mark.parametrize("n,d", CASES)
def test_solve_large_d(P, n, d):
    T, K = 30, 2
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=100 + d, dtype=np.float32)
    A = inst.dense()
    X0o, _ = O.spectral_init(A, n, d)
    Xo, _ = O.nsrgs(A, n, d, 1.0 / n, T, K, X0=X0o)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.DENSE_F32)
    X0, res = P.nsrgs_spectral_init(pa, max_iters=80, tol=1e-6)
    torch.cuda.synchronize()
    assert O.dF(to64(X0), X0o, d) / math.sqrt(n * d) <= 1e-5
    X, info = P.nsrgs_solve(pa, 1.0 / n, T, K, spectral_max_iters=80)
    torch.cuda.synchronize()
    assert info.iters == T
    assert O.dF(to64(X), Xo, d) / math.sqrt(n * d) <= 1e-5


@pytest.mark.parametrize("n,d", [(30, 16), (20, 25), (12, 64)])
def test_dF_large_d(P, n, d):
    rng = np.random.default_rng(d)
    X = rng.standard_normal((n * d, d)).astype(np.float32)
    Y = rng.standard_normal((n * d, d)).astype(np.float32)
    got = P.nsrgs_dF(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), n, d)
    ref = O.dF(X.astype(np.float64), Y.astype(np.float64), d)
    assert abs(got - ref) <= 1e-9 * ref


@pytest.mark.parametrize("n,d", [(60, 16), (40, 25), (30, 32), (20, 64), (50, 9)])
def test_gpm_large_d_matches_oracle(P, n, d):
    """The GPM baseline above d = 8 (per-block one-sided Jacobi SVD in a CTA)
    against the oracle's GPM from the same start."""
    T = 10
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=300 + d, dtype=np.float32)
    A = inst.dense()
    X0, _ = O.spectral_init(A, n, d)
    X0 = X0.astype(np.float32).astype(np.float64)
    ref = O.gpm(A, n, d, T, X0=X0)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.DENSE_F32)
    X = torch.from_numpy(X0.astype(np.float32)).cuda()
    X, info = P.nsrgs_gpm_solve(pa, T, init=False, X=X)
    torch.cuda.synchronize()
    assert info.iters == T
    Xb = O.blocks(to64(X), d)
    assert np.max(np.abs(np.swapaxes(Xb, 1, 2) @ Xb - np.eye(d))) <= 1e-4  # exact signs: orthogonal blocks
    assert O.dF(to64(X), ref, d) / math.sqrt(n * d) <= 1e-5


@pytest.mark.parametrize("storage", ["bf16", "dense_bf16"])
def test_gpm_tensor_core_storage_within_one_percent(P, storage):
    """GPM on the tensor-core streams (BF16 A, X rounded to BF16 for the product)
    reaches the float32 GPM's final d_F to the truth within 1%."""
    n, d, T = 300, 16, 20
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=316, dtype=np.float32)
    up = torch.from_numpy(inst.upper).cuda()
    Xf, _ = P.nsrgs_gpm_solve(P.nsrgs_pack_upper(up, n, d, P.DENSE_F32), T)
    Xb, info = P.nsrgs_gpm_solve(P.nsrgs_pack_upper(up, n, d, P.STORAGE[storage]), T)
    torch.cuda.synchronize()
    Z = inst.Zstack()
    ef, eb = O.dF(to64(Xf), Z, d), O.dF(to64(Xb), Z, d)
    assert info.iters == T
    assert abs(eb - ef) / ef <= 0.01, (ef, eb)
