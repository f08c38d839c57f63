"""GPU tests of the float32 symmetric tile stream (NSRGS_F32 at 8 < d <= 64):
the product against the float64 product of the same float32 values, one
iteration and whole solves against the FP64 oracle, the objective and the GPM
baseline on this layout."""
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


PRODUCT_CASES = [(2, 9), (5, 16), (20, 16), (9, 25), (33, 13), (100, 32), (70, 64), (300, 16), (17, 40), (60, 24),
                 (130, 48), (50, 56), (3, 64), (257, 12), (1000, 16)]


@pytest.mark.parametrize("n,d", PRODUCT_CASES)
def test_product_matches_float64(P, n, d):
    inst = synth.make_instance(n, d, 0.5, seed=n + 3 * d, dtype=np.float32)
    A = inst.dense()
    for i in range(n):
        A[i * d : (i + 1) * d, i * d : (i + 1) * d] = 0.0
    X = np.random.default_rng(d + n).standard_normal((n * d, d)).astype(np.float32)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.F32)
    Y = P.nsrgs_product(pa, torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    ref = A @ X.astype(np.float64)
    scale = np.abs(A) @ np.abs(X.astype(np.float64))
    err = np.abs(to64(Y) - ref)
    assert np.all(err <= 1e-6 * scale + 1e-6), float(np.max(err / (scale + 1e-6)))
    # the dense and the upper-block sources pack the same tiles
    pb = P.nsrgs_pack_dense(torch.from_numpy(inst.dense(dtype=np.float32)).cuda(), n, d, P.F32)
    torch.cuda.synchronize()
    assert torch.equal(pa.buf, pb.buf)


@pytest.mark.parametrize("n,d", [(200, 16), (64, 25), (90, 32), (40, 64), (75, 11)])
def test_one_iteration_matches_oracle(P, n, d):
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=5 * n + d, dtype=np.float32)
    A = inst.dense()
    X0, _ = O.spectral_init(A, n, d)
    X0 = X0.astype(np.float32).astype(np.float64)
    ref = O.nsrgs_iteration(A, X0, n, d, 1.0 / n, 2)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.F32)
    Xin = torch.from_numpy(X0.astype(np.float32)).cuda()
    Xout = torch.empty_like(Xin)
    un = torch.zeros(1, dtype=torch.float64, device="cuda")
    P.nsrgs_step(pa, 1.0 / n, 2, Xin, Xout, upd_norm=un)
    torch.cuda.synchronize()
    assert np.max(np.abs(to64(Xout) - ref)) <= 2e-5
    assert abs(un.item() - O.update_norm(ref, X0)) <= 1e-5


@pytest.mark.parametrize("n,d,T", [(200, 16, 30), (120, 25, 20), (60, 64, 15)])
def test_solve_matches_oracle(P, n, d, T):
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=11 * d + n, dtype=np.float32)
    A = inst.dense()
    Xo, _ = O.nsrgs(A, n, d, 1.0 / n, T, 2)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.F32)
    X, info = P.nsrgs_solve(pa, 1.0 / n, T, 2, spectral_max_iters=200)
    torch.cuda.synchronize()
    assert info.iters == T and info.flags == 0, info.as_dict()
    assert O.dF(to64(X), Xo, d) / math.sqrt(n * d) <= 1e-5


def test_table1_setting_on_the_float32_tiles(P):
    """n = 500, d = 25, sigma = 0.1, p = 1, mu = 1/(np), K = 1 (the paper's §4.1 setting):
    the solve with the paper's stopping rule matches the oracle's Rel.Err."""
    n, d, sigma = 500, 25, 0.1
    inst = synth.make_instance(n, d, sigma, seed=2024, dtype=np.float32)
    A = inst.dense()
    Xo, io = O.nsrgs(A, n, d, 1.0 / n, 100, 1, rel_tol=1e-8)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.F32)
    X, info = P.nsrgs_solve_objective(pa, 1.0 / n, 100, 1, rel_tol=1e-8, spectral_max_iters=200)
    torch.cuda.synchronize()
    Z = inst.Zstack()
    ro, rg = O.rel_err(Xo, Z, d), O.rel_err(to64(X), Z, d)
    assert abs(rg - ro) / ro <= 1e-3, (ro, rg)
    assert abs(rg - 2.19e-2) / 2.19e-2 <= 0.05


@pytest.mark.parametrize("n,d", [(150, 16), (40, 33)])
def test_objective_and_gpm_on_the_float32_tiles(P, n, d):
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=d + 7, dtype=np.float32)
    A = inst.dense()
    up = torch.from_numpy(inst.upper).cuda()
    X = torch.from_numpy(inst.Zstack().astype(np.float32)).cuda()
    Ft = P.nsrgs_objective(P.nsrgs_pack_upper(up, n, d, P.F32), X)
    Fo = O.objective(A, inst.Zstack().astype(np.float32).astype(np.float64), n, d)
    assert abs(Ft - Fo) <= 1e-5 * abs(Fo), (Ft, Fo)
    X0, _ = O.spectral_init(A, n, d)
    ref = O.gpm(A, n, d, 10, X0=X0)
    Xg = torch.from_numpy(X0.astype(np.float32)).cuda()
    Xg, info = P.nsrgs_gpm_solve(P.nsrgs_pack_upper(up, n, d, P.F32), 10, init=False, X=Xg)
    torch.cuda.synchronize()
    assert O.dF(to64(Xg), ref, d) / math.sqrt(n * d) <= 1e-5
