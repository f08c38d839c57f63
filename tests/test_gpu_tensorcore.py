"""Tensor-core (tcgen05) A streams for d in {16, 32, 64}: the dense form
(NSRGS_DENSE_BF16, both triangles) and the symmetric tile-upper form (NSRGS_BF16
at these d: each stored tile feeds Y_I += A_IJ X_J and Y_J += A_IJ^T X_I).

The product is checked against an exact float64 product of the same
bfloat16-rounded A and X (the kernels round X to bfloat16 for the multiply and
accumulate in float32), then whole solves against the FP64 oracle: final
d_F(X, Z) within 1%.
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


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


PRODUCT_CASES = [(2, 16), (20, 16), (9, 32), (5, 64), (300, 16), (130, 32), (70, 64), (8, 16), (17, 64), (1000, 16)]


@pytest.mark.parametrize("storage", ["dense_bf16", "bf16"])
@pytest.mark.parametrize("n,d", PRODUCT_CASES)
def test_tensor_core_product(P, n, d, storage):
    inst = synth.make_instance(n, d, 0.5, seed=n + d, dtype=np.float32)
    A = inst.dense()
    for i in range(n):
        A[i * d : (i + 1) * d, i * d : (i + 1) * d] = 0.0
    X = np.random.default_rng(d).standard_normal((n * d, d)).astype(np.float32)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.STORAGE[storage])
    Y = P.nsrgs_product(pa, torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    Ab, Xb = bf16_round(A), bf16_round(X)
    ref = Ab @ Xb
    scale = np.abs(Ab) @ np.abs(Xb)
    got = Y.double().cpu().numpy()
    assert np.all(np.abs(got - ref) <= 2e-6 * scale + 1e-6), np.max(np.abs(got - ref) / (scale + 1e-6))


# BF16 above d = 8 at block sizes other than the tile width: X^T rows past d are
# zero, blocks straddle the 128-row tiles, Y is added element-wise
ODD_D_CASES = [(30, 9), (7, 13), (20, 25), (11, 40), (9, 48), (3, 63)]


@pytest.mark.parametrize("n,d", ODD_D_CASES)
def test_tile_upper_product_at_any_d(P, n, d):
    inst = synth.make_instance(n, d, 0.5, seed=n + 7 * d, dtype=np.float32)
    A = inst.dense()
    for i in range(n):
        A[i * d : (i + 1) * d, i * d : (i + 1) * d] = 0.0
    X = np.random.default_rng(d).standard_normal((n * d, d)).astype(np.float32)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.BF16)
    Y = P.nsrgs_product(pa, torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    Ab, Xb = bf16_round(A), bf16_round(X)
    ref = Ab @ Xb
    scale = np.abs(Ab) @ np.abs(Xb)
    got = Y.double().cpu().numpy()
    assert np.all(np.abs(got - ref) <= 2e-6 * scale + 1e-6), np.max(np.abs(got - ref) / (scale + 1e-6))


@pytest.mark.parametrize("storage", ["dense_bf16", "bf16"])
@pytest.mark.parametrize("n,d", [(200, 16), (80, 32), (40, 64)])
def test_tensor_core_solve_within_one_percent(P, n, d, storage):
    """Final d_F(X, Z) of a BF16 tensor-core solve within 1% of the FP64 oracle's."""
    T, K = 40, 2
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=7 * d, dtype=np.float32)
    up = torch.from_numpy(inst.upper).cuda()
    Xo, _ = O.nsrgs(inst.dense(), n, d, 1.0 / n, T, K)
    Xb, info = P.nsrgs_solve(P.nsrgs_pack_upper(up, n, d, P.STORAGE[storage]), 1.0 / n, T, K)
    torch.cuda.synchronize()
    Z = inst.Zstack()
    eo = O.dF(Xo, Z, d)
    eb = O.dF(Xb.double().cpu().numpy(), Z, d)
    assert info.iters == T
    assert abs(eb - eo) / eo <= 0.01, (eo, eb)


def test_tile_upper_bytes_are_about_half_of_dense(P):
    for n, d in [(2000, 16), (1000, 32), (500, 64)]:
        dense = P.nsrgs_packed_bytes(n, d, P.DENSE_BF16)
        sym = P.nsrgs_packed_bytes(n, d, P.BF16)
        assert 0.49 < sym / dense < 0.53, (n, d, sym / dense)


@pytest.mark.parametrize("n,d", [(500, 16), (64, 64)])
def test_tile_upper_objective_equals_dense_bf16(P, n, d):
    """F(X) through the tile-upper layout (its ||A_off||^2 pass reads the stored
    triangle once, weighted twice) equals F through the dense BF16 layout (both
    triangles): the same bfloat16 values and the same bfloat16-rounded X."""
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=3 + d, dtype=np.float32)
    up = torch.from_numpy(inst.upper).cuda()
    X = torch.from_numpy(inst.Zstack().astype(np.float32)).cuda()
    Ft = P.nsrgs_objective(P.nsrgs_pack_upper(up, n, d, P.BF16), X)
    Fd = P.nsrgs_objective(P.nsrgs_pack_upper(up, n, d, P.DENSE_BF16), X)
    assert abs(Ft - Fd) <= 1e-6 * abs(Fd), (Ft, Fd)


@pytest.mark.parametrize("storage", ["dense_bf16", "bf16", "fp8"])
@pytest.mark.parametrize("n,d", [(200, 16), (80, 32), (40, 64)])
def test_tensor_core_spectral_start_stops_at_its_floor(P, n, d, storage):
    """The tensor-core streams multiply a rounded V, so the subspace iteration's
    residual settles at a floor (about 2^-8 of ||A_off V_perp|| / ||A_off V||)
    instead of reaching 1e-6: the passes stop there (info bit 7), report
    convergence, and the start agrees with the oracle's eigenvector start to the
    Davis-Kahan bound of that residual."""
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=5 * d + n, dtype=np.float32)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.STORAGE[storage])
    X0, res = P.nsrgs_spectral_init(pa, max_iters=60, tol=1e-6)  # raises unless it stopped
    torch.cuda.synchronize()
    assert res <= 1e-2
    _, info = P.nsrgs_solve(pa, 1.0 / n, 0, 2, spectral_max_iters=60)
    torch.cuda.synchronize()
    assert info.spectral_iters < 60 and not (info.flags & 4), info.as_dict()
    A = inst.dense()
    lam, U = np.linalg.eigh(A)
    top = lam[-d:]
    gap = lam[-d] - lam[-d - 1]
    # sin of the largest principal angle <= ||R||_F / gap, ||R||_F = res * ||H||_F
    sin_bound = res * np.sqrt(np.sum(top ** 2)) / gap
    X0o, _ = O.spectral_init(A, n, d)
    dist = O.dF(X0.double().cpu().numpy(), X0o, d) / math.sqrt(n * d)
    assert dist <= 4.0 * sin_bound + 1e-5, (dist, sin_bound, res, info.as_dict())


@pytest.mark.parametrize("n,d", [(100, 25), (60, 12)])
def test_tile_upper_solve_at_the_papers_d(P, n, d):
    """d = 25 (the setting of §4.1's Table 1) and d = 12 on the BF16 tile stream:
    final d_F(X, Z) within 1% of the FP64 oracle's."""
    T, K = 40, 2
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=3 * d, dtype=np.float32)
    Xo, _ = O.nsrgs(inst.dense(), n, d, 1.0 / n, T, K)
    Xb, info = P.nsrgs_solve(P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.BF16), 1.0 / n, T, K)
    torch.cuda.synchronize()
    Z = inst.Zstack()
    eo, eb = O.dF(Xo, Z, d), O.dF(Xb.double().cpu().numpy(), Z, d)
    assert info.iters == T and not (info.flags & 4), info.as_dict()
    assert abs(eb - eo) / eo <= 0.01, (eo, eb)
