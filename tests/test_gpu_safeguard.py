"""GPU parity of the safeguarded Newton-Schulz start (beyond the paper; the
oracle's ``ns_safeguard``): a block whose F_i fails Lemma 2.1's precondition
(||I - F_i^T F_i||_F >= 1) starts Algorithm 1 from F_i / ||F_i||_F.

A large step from a random orthogonal start makes many blocks fail the
precondition in the first iteration; one iteration is compared with the
oracle elementwise (2e-5, the one-iteration bar), through the register
epilogue (d <= 8), the shared-memory epilogue (d > 8) and the batched form.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu
SAFEGUARD_FLAG = 1 << 4
PRECOND_FLAG = 1 << 1


@pytest.fixture(scope="module")
def P():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2604_07372_gb300 as P

    return P


def to64(t):
    return t.detach().double().cpu().numpy()


def random_orthogonal_blocks(n, d, seed):
    g = np.random.default_rng(seed).standard_normal((n, d, d))
    u, _, vt = np.linalg.svd(g)
    return (u @ vt).reshape(n * d, d).astype(np.float32)


@pytest.mark.parametrize("n,d,storage,scale", [(300, 3, "f32", 6.0), (200, 4, "dense_f32", 6.0),
                                                (60, 12, "dense_f32", 3.0), (150, 6, "f32", 6.0)])
def test_one_safeguarded_iteration_matches_oracle(P, n, d, storage, scale):
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=n + d, dtype=np.float32)
    A = inst.dense()
    X0 = random_orthogonal_blocks(n, d, 5)
    eta, K = scale / n, 2
    F = O.blocks(X0.astype(np.float64), d) - eta * O.tangent_projection(
        O.blocks(X0.astype(np.float64), d), O.euclidean_gradient(A, X0.astype(np.float64), n, d))
    viol = np.linalg.norm(np.eye(d) - np.swapaxes(F, 1, 2) @ F, axis=(1, 2)) >= 1.0
    assert viol.any() and not viol.all()  # both kinds of block are exercised
    ref = O.nsrgs_iteration(A, X0.astype(np.float64), n, d, eta, K, safeguard=True)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.STORAGE[storage])
    X = torch.from_numpy(X0).cuda()
    X, info = P.nsrgs_solve_ex(pa, eta, 1, K, ns_safeguard=True, init=False, X=X)
    torch.cuda.synchronize()
    assert info.iters == 1
    assert info.flags & SAFEGUARD_FLAG and not info.flags & PRECOND_FLAG
    assert np.max(np.abs(to64(X) - ref)) <= 2e-5
    # without the safeguard the violation is reported and the iterate differs
    X2 = torch.from_numpy(X0).cuda()
    X2, info2 = P.nsrgs_solve_ex(pa, eta, 1, K, ns_safeguard=False, init=False, X=X2)
    torch.cuda.synchronize()
    assert info2.flags & PRECOND_FLAG and not info2.flags & SAFEGUARD_FLAG
    assert np.max(np.abs(to64(X2) - O.nsrgs_iteration(A, X0.astype(np.float64), n, d, eta, K))) <= 2e-5


def test_safeguard_is_a_no_op_where_the_precondition_holds(P):
    n, d, T = 400, 3, 30
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=9, dtype=np.float32)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.F32)
    Xa, ia = P.nsrgs_solve_ex(pa, 1.0 / n, T, 2, ns_safeguard=True)
    Xb, ib = P.nsrgs_solve_ex(pa, 1.0 / n, T, 2, ns_safeguard=False)
    torch.cuda.synchronize()
    assert not ia.flags & SAFEGUARD_FLAG
    # the same arithmetic; only the order of the float32 atomic adds in the A stream varies
    assert O.dF(to64(Xa), to64(Xb), d) / math.sqrt(n * d) <= 1e-6


def test_safeguard_keeps_the_low_p_step_finite(P):
    """p = 0.05 with the paper's mu = 1/(np): the plain GPU iteration becomes non-finite,
    the safeguarded one stays finite with d_F(X, Z) bounded (as the oracle's pin)."""
    n, d, p, T = 400, 3, 0.05, 40
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=7, p=p, dtype=np.float32)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.F32)
    with pytest.raises(P.NsrgsError):
        P.nsrgs_solve_ex(pa, 1.0 / (n * p), T, 2, ns_safeguard=False)
        torch.cuda.synchronize()
    X, info = P.nsrgs_solve_ex(pa, 1.0 / (n * p), T, 2, ns_safeguard=True)
    torch.cuda.synchronize()
    assert info.iters == T and info.flags & SAFEGUARD_FLAG
    Xn = to64(X)
    assert np.all(np.isfinite(Xn))
    assert O.dF(Xn, inst.Zstack(), d) / math.sqrt(n * d) < 1.0


def test_batched_safeguarded_iteration_matches_oracle(P):
    d, K, eta_scale = 3, 2, 6.0
    ns = [120, 301, 57]
    packs, Xs, refs = [], [], []
    for k, n in enumerate(ns):
        inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=40 + k, dtype=np.float32)
        X0 = random_orthogonal_blocks(n, d, 60 + k)
        refs.append(O.nsrgs_iteration(inst.dense(), X0.astype(np.float64), n, d, eta_scale / n, K, safeguard=True))
        packs.append(P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.F32))
        Xs.append(torch.from_numpy(X0).cuda())
    out, infos = P.nsrgs_batch_solve(packs, [eta_scale / n for n in ns], 1, K, init=False, Xs=Xs, ns_safeguard=True)
    torch.cuda.synchronize()
    for X, ref, inf in zip(out, refs, infos):
        assert inf.iters == 1 and inf.flags & SAFEGUARD_FLAG
        assert np.max(np.abs(to64(X) - ref)) <= 2e-5
