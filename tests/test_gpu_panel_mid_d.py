"""GPU parity of the symmetric panel stream for block sizes 5 <= d <= 8.

Above d = 4 each thread loads two columns per row (8 bytes FP32, 4 bytes
BF16) and holds one whole block row; FP8 storage is not offered there.  The
bars are those of the small-d parity tests: the product against the float64
product of the same stored values, one iteration against the oracle
elementwise, a whole solve within d_F / sqrt(nd) <= 1e-5.
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


def to64(t):
    return t.detach().double().cpu().numpy()


def make(n, d, c=0.3, seed=0):
    return synth.make_instance(n, d, synth.sigma_rule(c, n, d), seed=seed, dtype=np.float32)


# ragged slabs (64 block rows per slab), a single block pair, several slabs
PRODUCT_CASES = [(2, 5), (3, 8), (70, 5), (67, 6), (66, 7), (130, 8), (900, 6), (1100, 8), (1601, 7)]


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("n,d", PRODUCT_CASES)
def test_product_mid_d(P, n, d, storage):
    inst = make(n, d, c=0.5, seed=n + 7 * d)
    A = inst.dense()
    for i in range(n):
        A[i * d : (i + 1) * d, i * d : (i + 1) * d] = 0.0
    X = np.random.default_rng(n).standard_normal((n * d, d)).astype(np.float32)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.STORAGE[storage])
    Y = P.nsrgs_product(pa, torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    ref = A @ X.astype(np.float64)
    scale = np.abs(A) @ np.abs(X.astype(np.float64))
    got = to64(Y)
    rel = 1e-6 if storage == "f32" else 2.0**-8
    assert np.all(np.abs(got - ref) <= rel * scale + 1e-5)


def test_fp8_is_refused_above_d4(P):
    inst = make(20, 5)
    with pytest.raises(P.NsrgsError):
        P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), 20, 5, P.FP8E4M3)


@pytest.mark.parametrize("n,d", [(2, 6), (130, 5), (300, 8), (257, 7)])
def test_one_iteration_mid_d(P, n, d):
    inst = make(n, d, seed=n * 10 + d)
    A = inst.dense()
    X0, _ = O.spectral_init(A, n, d)
    X0 = X0.astype(np.float32).astype(np.float64)
    ref = O.nsrgs_iteration(A, X0, n, d, 1.0 / n, 2)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.F32)
    Xout = torch.empty(n * d, d, device="cuda")
    P.nsrgs_step(pa, 1.0 / n, 2, torch.from_numpy(X0.astype(np.float32)).cuda(), Xout)
    torch.cuda.synchronize()
    assert np.max(np.abs(to64(Xout) - ref)) <= 2e-5


@pytest.mark.parametrize("n,d", [(400, 5), (300, 8)])
def test_solve_mid_d(P, n, d):
    T, K = 30, 2
    inst = make(n, d, seed=200 + d)
    A = inst.dense()
    X0o, _ = O.spectral_init(A, n, d)
    Xo, _ = O.nsrgs(A, n, d, 1.0 / n, T, K, X0=X0o)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.F32)
    X, info = P.nsrgs_solve(pa, 1.0 / n, T, K, spectral_max_iters=80)
    torch.cuda.synchronize()
    assert info.iters == T
    assert O.dF(to64(X), Xo, d) / math.sqrt(n * d) <= 1e-5


def test_bf16_solve_mid_d_final_error(P):
    """BF16 storage at d = 8: final d_F(X, Z) within 1% of the oracle's."""
    n, d, T, K = 600, 8, 40, 2
    inst = make(n, d, seed=321)
    A = inst.dense()
    X0o, _ = O.spectral_init(A, n, d)
    Xo, _ = O.nsrgs(A, n, d, 1.0 / n, T, K, X0=X0o)
    Z = inst.Zstack()
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.BF16)
    X, _ = P.nsrgs_solve(pa, 1.0 / n, T, K, spectral_max_iters=80)
    torch.cuda.synchronize()
    e_gpu = O.dF(to64(X), Z, d)
    e_ref = O.dF(Xo, Z, d)
    assert abs(e_gpu - e_ref) <= 0.01 * e_ref
