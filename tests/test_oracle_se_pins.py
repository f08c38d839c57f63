"""Pins of the oracle's SE(d) form (poses: rotation X_i in O(d) and translation t_i).

The paper names the special Euclidean group as a target of the Newton-Schulz
retraction (§6) without writing the method; the oracle's reading is
    f(X, t) = F(X) + kappa sum_{i<j} w_ij ||t_j - t_i - X_i^T c_ij||^2
with G^X, G^t half its gradient (the term whose tangent projection vanishes on
O(d) dropped, as Algorithm 2 drops X_j^T X_j).  These checks tie it to things
other than itself: finite differences of f, the fixed point of noise-free data,
the reduction to Algorithm 2 at kappa = 0, the gauge symmetry, a closed form of
the translation step, a planted-mistake check, and the gauge-aligned error metric.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth


def inst(n=9, d=3, sigma=0.3, sigma_t=0.2, seed=5, p=1.0):
    s = synth.make_se_instance(n, d, sigma, sigma_t, seed=seed, p=p)
    return s, s.rot.dense(), s.c_square(), s.mask_square()


def rand_orth(rng, n, d):
    return synth.haar_orthogonal(rng, n, d).reshape(n * d, d)


@pytest.mark.parametrize("p", [1.0, 0.6])
def test_translation_gradient_is_half_the_finite_difference(p):
    s, A, C, W = inst(p=p)
    n, d, kappa = 9, 3, 0.7
    rng = np.random.default_rng(1)
    X = rand_orth(rng, n, d)
    t = rng.standard_normal((n, d))
    _, Gt = O.se_gradient(A, C, W, X, t, n, d, kappa)
    h = 1e-5
    fd = np.zeros((n, d))
    for k in range(n):
        for a in range(d):
            tp = t.copy(); tp[k, a] += h
            tm = t.copy(); tm[k, a] -= h
            fd[k, a] = (O.se_objective(A, C, W, X, tp, n, d, kappa) - O.se_objective(A, C, W, X, tm, n, d, kappa)) / (2 * h)
    assert np.max(np.abs(Gt - 0.5 * fd)) < 1e-6 * max(1.0, np.max(np.abs(fd)))


@pytest.mark.parametrize("p", [1.0, 0.6])
def test_rotation_gradient_projects_like_half_the_finite_difference(p):
    """At orthogonal X the tangent projection of G^X equals that of half the full
    Euclidean gradient of f in X (the dropped kappa c c^T X term projects to zero)."""
    s, A, C, W = inst(p=p)
    n, d, kappa = 9, 3, 0.7
    rng = np.random.default_rng(2)
    X = rand_orth(rng, n, d)
    t = rng.standard_normal((n, d))
    GX, _ = O.se_gradient(A, C, W, X, t, n, d, kappa)
    h = 1e-5
    fd = np.zeros((n * d, d))
    for e in range(n * d):
        for a in range(d):
            Xp = X.copy(); Xp[e, a] += h
            Xm = X.copy(); Xm[e, a] -= h
            fd[e, a] = (O.se_objective(A, C, W, Xp, t, n, d, kappa) - O.se_objective(A, C, W, Xm, t, n, d, kappa)) / (2 * h)
    Xb = O.blocks(X, d)
    P1 = O.tangent_projection(Xb, GX)
    P2 = O.tangent_projection(Xb, 0.5 * O.blocks(fd, d))
    assert np.max(np.abs(P1 - P2)) < 1e-5 * max(1.0, np.max(np.abs(P2)))


def test_noise_free_poses_are_a_fixed_point():
    s, A, C, W = inst(sigma=0.0, sigma_t=0.0, p=0.7)
    n, d = 9, 3
    Z = s.rot.Zstack()
    GX, Gt = O.se_gradient(A, C, W, Z, s.tau, n, d, 0.5)
    assert np.max(np.abs(O.tangent_projection(O.blocks(Z, d), GX))) < 1e-12
    assert np.max(np.abs(Gt)) < 1e-12
    Xn, tn = O.se_iteration(A, C, W, Z, s.tau, n, d, 1.0 / n, 0.1, 0.5, 3)
    assert np.max(np.abs(Xn - Z)) < 1e-12 and np.max(np.abs(tn - s.tau)) < 1e-12


def test_kappa_zero_is_algorithm_2_and_keeps_t():
    s, A, C, W = inst()
    n, d = 9, 3
    rng = np.random.default_rng(3)
    X = rand_orth(rng, n, d) + 0.01 * rng.standard_normal((n * d, d))
    t = rng.standard_normal((n, d))
    Xn, tn = O.se_iteration(A, C, W, X, t, n, d, 1.0 / n, 0.3, 0.0, 2)
    assert np.array_equal(Xn, O.nsrgs_iteration(A, X, n, d, 1.0 / n, 2))
    assert np.array_equal(tn, t)


def test_gauge_equivariance():
    """(X Q, Q^T t + v) maps to (X' Q, Q^T t' + v): the objective is invariant under the gauge."""
    s, A, C, W = inst(p=0.8)
    n, d, kappa = 9, 3, 0.4
    rng = np.random.default_rng(4)
    X = rand_orth(rng, n, d)
    t = rng.standard_normal((n, d))
    Q = synth.haar_orthogonal(rng, 1, d)[0]
    v = rng.standard_normal(d)
    Xn, tn = O.se_iteration(A, C, W, X, t, n, d, 1.0 / n, 0.05, kappa, 2)
    Xq, tq = O.se_iteration(A, C, W, X @ Q, t @ Q + v[None, :], n, d, 1.0 / n, 0.05, kappa, 2)
    assert np.max(np.abs(Xq - Xn @ Q)) < 1e-12
    assert np.max(np.abs(tq - (tn @ Q + v[None, :]))) < 1e-12


def test_translation_step_is_exact_in_one_step_on_noise_free_complete_data():
    """At X = Z, t = 0 and mu_t = 1/(kappa n), the step gives t = tau - mean(tau):
    G^t_k = kappa (sum_{i != k} (t_k - t_i) - n tau_k + sum_i tau_i) by hand."""
    s, A, C, W = inst(sigma=0.0, sigma_t=0.0)
    n, d, kappa = 9, 3, 0.8
    Z = s.rot.Zstack()
    _, tn = O.se_iteration(A, C, W, Z, np.zeros((n, d)), n, d, 1.0 / n, 1.0 / (kappa * n), kappa, 2)
    assert np.max(np.abs(tn - (s.tau - s.tau.mean(axis=0)))) < 1e-12


def test_iterations_reduce_the_objective_and_recover_the_poses():
    s, A, C, W = inst(n=40, sigma=0.3, sigma_t=0.1, seed=9)
    n, d, kappa = 40, 3, 1.0 / (4 * 3)
    X0, _ = O.spectral_init(A, n, d)
    t0 = np.zeros((n, d))
    f0 = O.se_objective(A, C, W, X0, t0, n, d, kappa)
    X, t, it = O.se_nsrgs(A, C, W, n, d, 1.0 / n, 1.0 / (kappa * n), kappa, 60, 2, X0, t0)
    f1 = O.se_objective(A, C, W, X, t, n, d, kappa)
    eR, eT = O.se_errors(X, t, s.rot.Z, s.tau, n, d)
    assert it == 60 and f1 < f0
    assert eR / math.sqrt(n * d) < 0.1 and eT < 0.1


def test_planted_mistakes_are_caught():
    """Mutants of the gradient (sign of the cross term, wrong residual index) fail the pins."""
    s, A, C, W = inst()
    n, d, kappa = 9, 3, 0.7
    rng = np.random.default_rng(6)
    X = rand_orth(rng, n, d)
    t = rng.standard_normal((n, d))
    GX, Gt = O.se_gradient(A, C, W, X, t, n, d, kappa)

    def f_t(tt):
        return O.se_objective(A, C, W, X, tt, n, d, kappa)

    h = 1e-5
    fd = np.zeros((n, d))
    for k in range(n):
        for a in range(d):
            tp = t.copy(); tp[k, a] += h
            tm = t.copy(); tm[k, a] -= h
            fd[k, a] = (f_t(tp) - f_t(tm)) / (2 * h)
    bad_sign = -Gt
    bad_index = np.roll(Gt, 1, axis=0)
    assert np.max(np.abs(Gt - 0.5 * fd)) < 1e-6
    assert np.max(np.abs(bad_sign - 0.5 * fd)) > 1e-3
    assert np.max(np.abs(bad_index - 0.5 * fd)) > 1e-3
    # a cross term with the wrong sign breaks the rotation pin
    Xb = O.blocks(X, d)
    GXbad = O.euclidean_gradient(A, X, n, d)
    for i in range(n - 1):
        for j in range(i + 1, n):
            GXbad[i] += kappa * np.outer(C[i, j], t[j] - t[i])
    assert np.max(np.abs(O.tangent_projection(Xb, GXbad) - O.tangent_projection(Xb, GX))) > 1e-3


def test_errors_are_gauge_invariant_and_exact():
    """se_errors: the truth moved by any gauge (X Q, Q^T t + v) scores (0, 0); adding a
    zero-mean perturbation e to the translations scores sqrt(sum ||e_i||^2 / n)."""
    s, _, _, _ = inst(n=12)
    n, d = 12, 3
    rng = np.random.default_rng(8)
    Q = synth.haar_orthogonal(rng, 1, d)[0]
    v = rng.standard_normal(d)
    Z = s.rot.Zstack()
    eR, eT = O.se_errors(Z @ Q, s.tau @ Q + v[None, :], s.rot.Z, s.tau, n, d)
    assert eR < 1e-12 and eT < 1e-12
    e = rng.standard_normal((n, d))
    e -= e.mean(axis=0, keepdims=True)
    _, eT = O.se_errors(Z @ Q, (s.tau + e) @ Q + v[None, :], s.rot.Z, s.tau, n, d)
    assert abs(eT - math.sqrt(float(np.sum(e * e)) / n)) < 1e-12
