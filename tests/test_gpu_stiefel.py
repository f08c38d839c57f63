"""GPU parity of the Stiefel form (d x p row-orthonormal blocks; an extension the
paper names, not its method) with the oracle's stiefel_iteration, and its
reduction to Algorithm 2 when p = d.
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


def start(inst, A, n, d, p):
    """[X_i^0, 0] from the oracle's spectral start, rotated by a fixed Q in O(p)."""
    X0, _ = O.spectral_init(A, n, d)
    Q = np.linalg.qr(np.random.default_rng(p).standard_normal((p, p)))[0]
    Xb = np.concatenate([O.blocks(X0, d), np.zeros((n, d, p - d))], axis=2) @ Q
    return Xb.reshape(n * d, p).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("n,d,p", [(200, 3, 5), (120, 3, 3), (90, 4, 8), (40, 16, 24)])
def test_stiefel_iterations_match_oracle(P, n, d, p):
    T, K = 5, 2
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=n + p, dtype=np.float32)
    A = inst.dense()
    X0 = start(inst, A, n, d, p)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.DENSE_F32)
    x0 = torch.from_numpy(X0.astype(np.float32)).cuda()
    X1, info1 = P.nsrgs_stiefel_solve(pa, p, 1.0 / n, 1, K, x0)
    torch.cuda.synchronize()
    ref1 = O.stiefel_iteration(A, X0, n, d, 1.0 / n, K)
    assert info1.iters == 1
    assert np.max(np.abs(to64(X1) - ref1)) <= 2e-5
    XT, info = P.nsrgs_stiefel_solve(pa, p, 1.0 / n, T, K, x0)
    torch.cuda.synchronize()
    ref = X0
    for _ in range(T):
        ref = O.stiefel_iteration(A, ref, n, d, 1.0 / n, K)
    assert info.iters == T
    assert np.linalg.norm(to64(XT) - ref) / math.sqrt(n * d * p) <= 1e-5


def test_stiefel_with_p_equal_d_is_algorithm_2(P):
    n, d, T, K = 300, 3, 10, 2
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=4, dtype=np.float32)
    A = inst.dense()
    X0, _ = O.spectral_init(A, n, d)
    x0 = torch.from_numpy(X0.astype(np.float32)).cuda()
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.DENSE_F32)
    Xs, _ = P.nsrgs_stiefel_solve(pa, d, 1.0 / n, T, K, x0)
    Xa, _ = P.nsrgs_solve(pa, 1.0 / n, T, K, init=False, X=x0.clone())
    torch.cuda.synchronize()
    assert O.dF(to64(Xs), to64(Xa), d) / math.sqrt(n * d) <= 1e-5


def test_stiefel_update_norm_stop(P):
    n, d, p = 150, 3, 4
    inst = synth.make_instance(n, d, synth.sigma_rule(0.2, n, d), seed=6, dtype=np.float32)
    A = inst.dense()
    X0 = start(inst, A, n, d, p)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.DENSE_F32)
    X, info = P.nsrgs_stiefel_solve(pa, p, 1.0 / n, 500, 2, torch.from_numpy(X0.astype(np.float32)).cuda(), tol=1e-6)
    torch.cuda.synchronize()
    assert info.iters < 500 and info.last_update_norm < 1e-6
    Xb = to64(X).reshape(n, d, p)
    assert np.max(np.abs(Xb @ np.swapaxes(Xb, 1, 2) - np.eye(d))) < 1e-4  # rows stay orthonormal


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("n,d,p", [(40, 16, 24), (30, 10, 13), (12, 40, 48)])
def test_stiefel_on_symmetric_tiles(P, n, d, p, storage):
    """d > 8: the product reads the symmetric tiles once (float32 tiles on the CUDA
    cores, bfloat16 tiles on the tensor cores) with X of p columns.  Float32 tiles
    match the oracle as the dense form does; bfloat16 tiles (A and X rounded for the
    product) stay within 1e-3 RMS of it over 5 iterations."""
    T, K = 5, 2
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=n + d + p, dtype=np.float32)
    A = inst.dense()
    X0 = start(inst, A, n, d, p)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.STORAGE[storage])
    x0 = torch.from_numpy(X0.astype(np.float32)).cuda()
    XT, info = P.nsrgs_stiefel_solve(pa, p, 1.0 / n, T, K, x0)
    torch.cuda.synchronize()
    ref = X0
    for _ in range(T):
        ref = O.stiefel_iteration(A, ref, n, d, 1.0 / n, K)
    assert info.iters == T and info.flags == 0, info.as_dict()
    err = np.linalg.norm(to64(XT) - ref) / math.sqrt(n * d * p)
    assert err <= (1e-5 if storage == "f32" else 1e-3), err


def test_stiefel_bf16_tiles_refuse_a_width_class_change(P):
    """The bfloat16 tiles' visiting order depends on the tile width; p must keep d's class."""
    n, d, p = 10, 16, 40
    inst = synth.make_instance(n, d, 0.3, seed=2, dtype=np.float32)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.BF16)
    x0 = torch.zeros(n * d, p, device="cuda")
    with pytest.raises(P.NsrgsError):
        P.nsrgs_stiefel_solve(pa, p, 0.1, 1, 2, x0)
