"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks an oracle function against something other than the oracle
itself: a closed form derived by hand, a textbook identity, a brute-force
search, a different library routine, or a value printed in the paper.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rot(a):
    return np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])


J = np.array([[0.0, -1.0], [1.0, 0.0]])


def rand_orth(rng, d):
    q, r = np.linalg.qr(rng.standard_normal((d, d)))
    return q * np.sign(np.diag(r))


# ------------------------------------------------------------ Algorithm 1
@pytest.mark.parametrize("d", [1, 3, 5, 25])
def test_ns_singular_value_map(d):
    """One NS step keeps the singular vectors and maps each s to s(3 - s^2)/2."""
    rng = np.random.default_rng(d)
    M = rng.standard_normal((d, d))
    M *= 1.6 / np.linalg.norm(M, 2)  # singular values in (0, 1.6]
    U, s, Vt = np.linalg.svd(M)
    for steps in (1, 2, 3):
        f = s.copy()
        for _ in range(steps):
            f = f * (3.0 - f * f) / 2.0
        expect = U @ np.diag(f) @ Vt
        assert np.allclose(O.newton_schulz(M, steps), expect, atol=1e-12, rtol=0)


def test_ns_lemma_2_1_bound_and_limit():
    """Lemma 2.1: ||S_t - sgn A|| <= ||I - S_t^T S_t|| <= ||I - A^T A||^(2^t)."""
    rng = np.random.default_rng(0)
    for d in (2, 3, 8, 25):
        for _ in range(5):
            U = rand_orth(rng, d)
            V = rand_orth(rng, d)
            s = rng.uniform(0.05, 1.4, size=d)  # |1 - s^2| < 1
            A = U @ np.diag(s) @ V.T
            polar = U @ V.T
            e0 = np.linalg.norm(np.eye(d) - A.T @ A, 2)
            assert e0 < 1
            for t in range(6):
                S = O.newton_schulz(A, t)
                et = np.linalg.norm(np.eye(d) - S.T @ S, 2)
                assert np.linalg.norm(S - polar, 2) <= et + 1e-13
                assert et <= e0 ** (2**t) + 1e-13
            assert np.linalg.norm(O.newton_schulz(A, 12) - polar) < 1e-12


def test_ns_diverges_outside_precondition():
    """Singular value 3 maps to 3(3-9)/2 = -9: far outside ||I - A^T A|| < 1 it blows up."""
    A = np.diag([3.0, 0.5, 1.0])
    assert np.max(np.abs(O.newton_schulz(A, 3))) > 1e3


def test_sgn_is_polar_factor():
    rng = np.random.default_rng(1)
    for d in (1, 2, 3, 7):
        M = rng.standard_normal((d, d))
        Q = O.sgn(M)
        assert np.allclose(Q.T @ Q, np.eye(d), atol=1e-13)
        H = Q.T @ M  # the symmetric positive factor of M = Q H
        assert np.allclose(H, H.T, atol=1e-12)
        assert np.min(np.linalg.eigvalsh(0.5 * (H + H.T))) > 0


# ------------------------------------------------- §2.2 tangent projection
@pytest.mark.parametrize("d", [2, 3, 6])
def test_tangent_projection_identities(d):
    rng = np.random.default_rng(10 + d)
    X = rand_orth(rng, d)
    G = rng.standard_normal((d, d))
    P = O.tangent_projection(X, G)
    # P lies in the tangent space {X H : H skew}
    assert np.allclose(X.T @ P + P.T @ X, 0, atol=1e-13)
    # symmetric directions X S are annihilated, skew directions X H are kept
    S = rng.standard_normal((d, d))
    S = S + S.T
    H = rng.standard_normal((d, d))
    H = H - H.T
    assert np.allclose(O.tangent_projection(X, X @ S), 0, atol=1e-12)
    assert np.allclose(O.tangent_projection(X, X @ H), X @ H, atol=1e-12)
    # idempotent
    assert np.allclose(O.tangent_projection(X, P), P, atol=1e-12)


# ---------------------------------------------------- §2.2 gradient
def test_gradient_is_derivative_of_fi():
    """G_i equals d f_i / d X_i, f_i = 1/2 sum_{j != i} ||X_i X_j^T - A_ij||^2, when X_j in O(d)."""
    rng = np.random.default_rng(3)
    n, d = 5, 3
    inst = synth.make_instance(n, d, 0.7, seed=11)
    A = inst.dense()
    Xb = np.stack([rand_orth(rng, d) for _ in range(n)])
    G = O.euclidean_gradient(A, Xb.reshape(n * d, d), n, d)

    def f_i(i, Xi):
        tot = 0.0
        for j in range(n):
            if j == i:
                continue
            Aij = A[i * d : (i + 1) * d, j * d : (j + 1) * d]
            R = Xi @ Xb[j].T - Aij
            tot += 0.5 * np.sum(R * R)
        return tot

    h = 1e-6
    for i in range(n):
        num = np.zeros((d, d))
        for a in range(d):
            for b in range(d):
                E = np.zeros((d, d))
                E[a, b] = h
                num[a, b] = (f_i(i, Xb[i] + E) - f_i(i, Xb[i] - E)) / (2 * h)
        assert np.allclose(G[i], num, atol=1e-6)


# -------------------------------------- Algorithm 2, closed forms in O(2)
@pytest.mark.parametrize("mu,th,ph", [(0.5, 0.3, -0.7), (0.1, 1.2, 0.4), (0.9, -2.0, 0.25)])
def test_one_iteration_two_nodes_closed_form(mu, th, ph):
    """n = 2, d = 2, X_1 = I, X_2 = R(th), A_12 = R(ph), one NS step.

    By hand: G_1 = I - R(ph + th), P(G_1) = -sin(a) J with a = ph + th, so
    F_1 = I + mu s J (s = sin a), F_1^T F_1 = (1 + mu^2 s^2) I and one NS step
    gives X_1' = (1 - mu^2 s^2 / 2)(I + mu s J).  Likewise
    P(G_2) = s J R(th), F_2 = (I - mu s J) R(th), X_2' = (1 - mu^2 s^2/2)(I - mu s J) R(th).
    """
    n, d = 2, 2
    A = np.block([[np.eye(2), rot(ph)], [rot(ph).T, np.eye(2)]])
    X = np.vstack([np.eye(2), rot(th)])
    Xn = O.nsrgs_iteration(A, X, n, d, mu, 1)
    s = math.sin(th + ph)
    c = 1 - mu * mu * s * s / 2
    assert np.allclose(Xn[:2], c * (np.eye(2) + mu * s * J), atol=1e-14)
    assert np.allclose(Xn[2:], c * (np.eye(2) - mu * s * J) @ rot(th), atol=1e-14)


def test_one_iteration_three_nodes_sums_over_j():
    """n = 3: node 1 sees both neighbours: X_1' = (1 - mu^2 S^2/2)(I + mu S J), S = sum_j sin(ph_j + th_j)."""
    n, d, mu = 3, 2, 0.3
    th2, th3, ph2, ph3, ph23 = 0.4, -1.1, 0.9, 0.2, 2.5
    A = np.eye(6)
    A[0:2, 2:4] = rot(ph2)
    A[0:2, 4:6] = rot(ph3)
    A[2:4, 4:6] = rot(ph23)
    A[2:4, 0:2] = rot(ph2).T
    A[4:6, 0:2] = rot(ph3).T
    A[4:6, 2:4] = rot(ph23).T
    X = np.vstack([np.eye(2), rot(th2), rot(th3)])
    Xn = O.nsrgs_iteration(A, X, n, d, mu, 1)
    S = math.sin(ph2 + th2) + math.sin(ph3 + th3)
    assert np.allclose(Xn[:2], (1 - mu * mu * S * S / 2) * (np.eye(2) + mu * S * J), atol=1e-14)


# ------------------------------------------------ whole-loop properties
def _config1(seed=5, c=0.3, n=200, d=3):
    inst = synth.make_instance(n, d, synth.sigma_rule(c, n, d), seed=seed)
    return inst, inst.dense()


def test_sigma_zero_exact_recovery():
    """sigma = 0: A = Z Z^T, the spectral start is Z up to one rotation and a fixed point."""
    n, d = 200, 3
    inst = synth.make_instance(n, d, 0.0, seed=2)
    A = inst.dense()
    X0, _ = O.spectral_init(A, n, d)
    assert O.dF(X0, inst.Zstack(), d) <= 1e-10
    X, _ = O.nsrgs(A, n, d, 1.0 / n, 50, 2, X0=X0)
    assert O.dF(X, inst.Zstack(), d) <= 1e-10


def test_iterates_stay_orthogonal():
    n, d = 200, 3
    inst, A = _config1()
    X, _ = O.nsrgs(A, n, d, 1.0 / n, 50, 2)
    err = max(np.linalg.norm(b.T @ b - np.eye(d)) for b in O.blocks(X, d))
    assert err <= 1e-8


def test_fixed_point_first_order_condition():
    """At convergence P(G_i) = 0, i.e. X_i^T sum_{j != i} A_ij X_j is symmetric."""
    n, d = 200, 3
    inst, A = _config1()
    X, _ = O.nsrgs(A, n, d, 1.0 / n, 120, 2)
    Xb = O.blocks(X, d)
    AX = O.blocks(A @ X, d) - Xb  # A_ii = I
    M = np.swapaxes(Xb, 1, 2) @ AX
    skew = 0.5 * (M - np.swapaxes(M, 1, 2))
    assert np.max(np.linalg.norm(skew, axis=(1, 2))) / n <= 1e-10


def test_global_rotation_equivariance():
    n, d = 60, 3
    inst, A = _config1(n=n)
    rng = np.random.default_rng(4)
    Q = rand_orth(rng, d)
    X0, _ = O.spectral_init(A, n, d)
    Xa, _ = O.nsrgs(A, n, d, 1.0 / n, 10, 2, X0=X0)
    Xb, _ = O.nsrgs(A, n, d, 1.0 / n, 10, 2, X0=X0 @ Q)
    assert np.allclose(Xb, Xa @ Q, atol=1e-12)


def test_gauge_equivariance():
    """A -> D^T A D, X -> D^T X with D = diag(Z_i) maps iterates to iterates (§5)."""
    n, d = 40, 3
    inst, A = _config1(n=n)
    D = np.zeros((n * d, n * d))
    for i in range(n):
        D[i * d : (i + 1) * d, i * d : (i + 1) * d] = inst.Z[i]
    A2 = D.T @ A @ D
    X0, _ = O.spectral_init(A, n, d)
    Xa, _ = O.nsrgs(A, n, d, 1.0 / n, 6, 2, X0=X0)
    Xb, _ = O.nsrgs(A2, n, d, 1.0 / n, 6, 2, X0=D.T @ X0)
    assert np.allclose(Xb, D.T @ Xa, atol=1e-12)


def test_node_permutation_equivariance():
    n, d = 30, 3
    inst, A = _config1(n=n)
    perm = np.random.default_rng(6).permutation(n)
    idx = (perm[:, None] * d + np.arange(d)[None, :]).ravel()
    A2 = A[np.ix_(idx, idx)]
    X0, _ = O.spectral_init(A, n, d)
    Xa, _ = O.nsrgs(A, n, d, 1.0 / n, 6, 2, X0=X0)
    Xb, _ = O.nsrgs(A2, n, d, 1.0 / n, 6, 2, X0=X0[idx])
    assert np.allclose(Xb, Xa[idx], atol=1e-12)


def test_gpm_and_nsrgs_share_the_fixed_point():
    n, d = 200, 3
    inst, A = _config1()
    Xn, _ = O.nsrgs(A, n, d, 1.0 / n, 150, 3)
    Xg = O.gpm(A, n, d, 150)
    assert O.dF(Xn, Xg, d) / math.sqrt(n * d) <= 1e-9
    # sigma = 0: the ground truth is a GPM fixed point
    inst0 = synth.make_instance(n, d, 0.0, seed=2)
    Z = inst0.Zstack()
    assert O.dF(O.gpm_iteration(inst0.dense(), Z, n, d), Z, d) <= 1e-10


# ------------------------------------------------------------ metrics
def test_dF_closed_form_d1():
    rng = np.random.default_rng(8)
    x = rng.standard_normal(20)
    y = rng.standard_normal(20)
    expect = min(np.linalg.norm(x - y), np.linalg.norm(x + y))
    assert abs(O.dF(x[:, None], y[:, None], 1) - expect) < 1e-12


def test_dF_brute_force_d2_and_nuclear_identity():
    """d = 2: search all rotations and reflections on a fine grid; and
    d_F^2 = ||X||^2 + ||Y||^2 - 2 ||Y^T X||_* (proof of Lemma 7.4)."""
    rng = np.random.default_rng(9)
    X = rng.standard_normal((14, 2))
    Y = rng.standard_normal((14, 2))
    best = np.inf
    refl = np.diag([1.0, -1.0])
    for a in np.linspace(0, 2 * math.pi, 20001):
        for Q in (rot(a), rot(a) @ refl):
            best = min(best, np.linalg.norm(X - Y @ Q))
    val = O.dF(X, Y, 2)
    assert val <= best + 1e-12
    assert val >= best - 1e-6
    nuc = np.sum(np.linalg.svd(Y.T @ X, compute_uv=False))
    assert abs(val**2 - (np.sum(X * X) + np.sum(Y * Y) - 2 * nuc)) < 1e-10


def test_rel_err_gram_identity_and_mse():
    rng = np.random.default_rng(12)
    n, d = 50, 3
    Z = np.vstack([rand_orth(rng, d) for _ in range(n)])
    X = np.vstack([rand_orth(rng, d) for _ in range(n)])
    # ||ZZ^T - XX^T||^2 = ||Z^T Z||^2 + ||X^T X||^2 - 2 ||Z^T X||^2
    num = np.sum((Z.T @ Z) ** 2) + np.sum((X.T @ X) ** 2) - 2 * np.sum((Z.T @ X) ** 2)
    assert abs(O.rel_err(X, Z, d, chunk=17) - math.sqrt(num / np.sum((Z.T @ Z) ** 2))) < 1e-12
    Q = rand_orth(rng, d)
    assert O.mse(Z @ Q, Z, n, d) < 1e-24


# ------------------------------------------------- spectral start
def test_spectral_subspace_courant_fischer():
    """tr(Y^T A Y) equals the sum of the d largest eigenvalues (scipy's eigvalsh)."""
    import scipy.linalg

    for n, d, c in [(30, 3, 0.3), (25, 4, 0.5), (40, 2, 2.0)]:
        inst = synth.make_instance(n, d, synth.sigma_rule(c, n, d), seed=n)
        A = inst.dense()
        X0, Y = O.spectral_init(A, n, d, method="eigh")
        assert np.allclose(Y.T @ Y, np.eye(d), atol=1e-12)
        top = np.sort(scipy.linalg.eigvalsh(A))[-d:]
        assert abs(np.trace(Y.T @ A @ Y) - top.sum()) < 1e-9 * abs(top.sum())
        # the Lanczos route spans the same subspace
        X0b, _ = O.spectral_init(A, n, d, method="eigsh")
        assert O.dF(X0b, X0, d) < 1e-8


# ------------------------------------------------------ generator sanity
def test_noise_operator_norm_bound():
    """Lemma 7.2: a symmetric Gaussian W (W_ii = 0) has ||W|| <= 3 sqrt(nd)."""
    n, d = 120, 3
    inst = synth.make_instance(n, d, 1.0, seed=21)
    Z = inst.Zstack()
    W = inst.dense() - Z @ Z.T  # diagonal blocks: I - Z_i Z_i^T = 0
    assert np.allclose(W, W.T)
    assert np.linalg.norm(W, 2) <= 3 * math.sqrt(n * d)


# ---------------------------------------------------------- Table 1
@pytest.mark.slow
@pytest.mark.parametrize("sigma,p", [(0.1, 1.0), (0.02, 0.5)])
def test_table1_relative_error(sigma, p):
    """Reproduce Table 1's NS-RGS Rel.Err (means of 10 trials) with one seed, within 2%."""
    with open(os.path.join(GOLDEN, "table1_relerr.json")) as f:
        g = json.load(f)
    pt = [q for q in g["points"] if q["sigma"] == sigma and q["p"] == p][0]
    n, d = g["n"], g["d"]
    inst = synth.make_instance(n, d, sigma, seed=1, p=p)
    A = inst.dense()
    X, info = O.nsrgs(A, n, d, 1.0 / (n * p), g["max_iter"], g["Ts"], rel_tol=g["rel_tol"])
    err = O.rel_err(X, inst.Zstack(), d)
    assert abs(err - pt["rel_err"]) / pt["rel_err"] < 0.02


def test_rows_update_matches_full_iteration():
    n, d = 40, 3
    inst, A = _config1(n=n)
    X0, _ = O.spectral_init(A, n, d)
    full = O.blocks(O.nsrgs_iteration(A, X0, n, d, 1.0 / n, 2), d)
    idx = [0, 7, 39]
    rows = np.stack([synth.block_row(inst.upper, n, d, i) for i in idx])
    assert np.allclose(rows[1], A[7 * d : 8 * d]), "block_row must read A's block row"
    part = O.nsrgs_rows_update(rows, X0, idx, n, d, 1.0 / n, 2)
    assert np.allclose(part, full[idx], atol=1e-14)


# ------------------------------- beyond the paper: safeguarded NS start
def test_safeguard_leaves_blocks_that_meet_the_precondition():
    """Where ||I - F_i^T F_i||_F < 1 for every block the safeguarded iteration is
    Algorithm 2 itself, bit for bit."""
    n, d = 120, 3
    inst, A = _config1(n=n)
    X0, _ = O.spectral_init(A, n, d)
    X = X0
    for _ in range(5):
        a = O.nsrgs_iteration(A, X, n, d, 1.0 / n, 2)
        b = O.nsrgs_iteration(A, X, n, d, 1.0 / n, 2, safeguard=True)
        assert np.array_equal(a, b)
        X = a


def test_safeguard_restores_convergence_to_the_polar_factor():
    """A block far outside Lemma 2.1's region: Algorithm 1 from F diverges, from the
    safeguarded start it converges to sgn(F) (the SVD polar factor), unchanged by the scaling."""
    rng = np.random.default_rng(3)
    for d in (2, 3, 5):
        F = 3.0 * rng.standard_normal((d, d))
        assert np.linalg.norm(np.eye(d) - F.T @ F) >= 1.0
        with np.errstate(over="ignore", invalid="ignore"):
            bad = O.newton_schulz(F, 30)
        assert not np.all(np.isfinite(bad)) or np.linalg.norm(bad - O.sgn(F)) > 1e-3
        G = O.ns_safeguard(F)
        assert np.isclose(np.linalg.norm(G), 1.0)
        assert np.allclose(O.sgn(G), O.sgn(F), atol=1e-12)
        assert np.allclose(O.newton_schulz(G, 60), O.sgn(F), atol=1e-10)
        # a block inside the region is returned as it is
        H = O.sgn(F) * 1.05
        assert np.array_equal(O.ns_safeguard(H), H)


def test_safeguard_keeps_the_low_p_step_finite():
    """Sparse data with the paper's step mu = 1/(np) at p = 0.05 (n = 400, d = 3): the
    plain iteration leaves Lemma 2.1's region and blows up within 30 iterations; with the
    safeguarded start the iterates stay finite and d_F(X, Z) stays bounded."""
    n, d, p = 400, 3, 0.05
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=7, p=p)
    A = inst.dense()
    X0, _ = O.spectral_init(A, n, d)
    X = X0
    blew_up = False
    with np.errstate(over="ignore", invalid="ignore"):
        for _ in range(30):
            X = O.nsrgs_iteration(A, X, n, d, 1.0 / (n * p), 2)
            if not np.all(np.isfinite(X)):
                blew_up = True
                break
    assert blew_up
    X = X0
    for _ in range(40):
        X = O.nsrgs_iteration(A, X, n, d, 1.0 / (n * p), 2, safeguard=True)
        assert np.all(np.isfinite(X))
    assert O.dF(X, inst.Zstack(), d) / math.sqrt(n * d) < 1.0


# ---------------------- beyond the paper: Stiefel form (d x p blocks)
def _row_orthonormal(rng, n, d, p):
    g = rng.standard_normal((n, d, p))
    return np.stack([O.polar_rows(b) for b in g])


def test_stiefel_reduces_to_algorithm_2_when_p_equals_d():
    n, d = 60, 3
    inst, A = _config1(n=n)
    X0, _ = O.spectral_init(A, n, d)
    X = X0
    for _ in range(3):
        a = O.nsrgs_iteration(A, X, n, d, 1.0 / n, 2)
        b = O.stiefel_iteration(A, X, n, d, 1.0 / n, 2)
        assert np.allclose(a, b, atol=1e-12)
        X = a


def test_stiefel_gradient_is_the_derivative_of_the_objective():
    """Central differences of F (eq. (1) with d x p blocks) along random directions:
    each X_i enters F through the pairs (i, j) and (j, i), so dF = sum_i <2 G_i, dX_i>
    (G_i is the gradient of f_i = 1/2 sum_{j != i} ||X_i X_j^T - A_ij||^2, as in Algorithm 2)."""
    rng = np.random.default_rng(4)
    n, d, p = 7, 2, 4
    inst = synth.make_instance(n, d, 0.7, seed=3)
    A = inst.dense()
    X = _row_orthonormal(rng, n, d, p).reshape(n * d, p)
    G = O.stiefel_gradient(A, X, n, d).reshape(n * d, p)
    for _ in range(3):
        V = rng.standard_normal(X.shape)
        h = 1e-6
        fd = (O.objective(A, X + h * V, n, d) - O.objective(A, X - h * V, n, d)) / (2 * h)
        assert abs(fd - 2.0 * np.sum(G * V)) <= 1e-6 * max(1.0, abs(fd))


def test_stiefel_projection_lands_in_the_tangent_space():
    rng = np.random.default_rng(5)
    for d, p in [(2, 3), (3, 5), (4, 4)]:
        Xi = _row_orthonormal(rng, 1, d, p)[0]
        G = rng.standard_normal((d, p))
        P = O.stiefel_projection(Xi, G)
        assert np.allclose(P @ Xi.T + Xi @ P.T, 0.0, atol=1e-12)     # tangent
        assert np.allclose(O.stiefel_projection(Xi, P), P, atol=1e-12)  # idempotent
        H = rng.standard_normal((d, d))
        N = (H + H.T) @ Xi  # a normal direction
        assert np.allclose(O.stiefel_projection(Xi, N), 0.0, atol=1e-12)


def test_row_newton_schulz_converges_to_the_polar_factor():
    rng = np.random.default_rng(6)
    for d, p in [(2, 3), (3, 7), (5, 5)]:
        U, _, Vt = np.linalg.svd(rng.standard_normal((d, p)), full_matrices=False)
        s = rng.uniform(0.3, 1.6, size=d)
        M = U @ np.diag(s) @ Vt
        assert np.allclose(O.newton_schulz_rows(M, 40), U @ Vt, atol=1e-12)
        assert np.allclose(O.polar_rows(M), U @ Vt, atol=1e-12)


def test_stiefel_fixed_point_at_sigma_zero():
    """sigma = 0: X_i = [Z_i, 0] Q for any Q in O(p) is left unchanged."""
    rng = np.random.default_rng(7)
    n, d, p = 40, 3, 5
    inst = synth.make_instance(n, d, 0.0, seed=8)
    A = inst.dense()
    Q = np.linalg.qr(rng.standard_normal((p, p)))[0]
    Xb = np.concatenate([inst.Z, np.zeros((n, d, p - d))], axis=2) @ Q
    X = Xb.reshape(n * d, p)
    X1 = O.stiefel_iteration(A, X, n, d, 1.0 / n, 2)
    assert np.allclose(X1, X, atol=1e-12)


# ------------------------------------------------- update norm (retire rule)
@pytest.mark.parametrize("th", [math.pi / 3, 0.25, 2.0])
def test_update_norm_closed_form_two_blocks(th):
    """||X' - X||_F / sqrt(nd) on n = 2 blocks in O(2): X = (I; I), X' = (R(th); I).
    By hand ||R(th) - I||_F^2 = 2((cos th - 1)^2 + sin^2 th) = 4 - 4 cos th, and
    nd = 4 rows, so the norm is sqrt(1 - cos th): a sqrt(n) or sqrt(n d^2)
    normaliser, or a norm over one block only, gives another number."""
    X = np.vstack([np.eye(2), np.eye(2)])
    Xn = np.vstack([rot(th), np.eye(2)])
    assert O.update_norm(Xn, X) == pytest.approx(math.sqrt(1.0 - math.cos(th)), rel=1e-14)
    # symmetric in its arguments and zero at no change
    assert O.update_norm(X, Xn) == pytest.approx(O.update_norm(Xn, X), rel=1e-15)
    assert O.update_norm(X, X) == 0.0
    # three nodes, d = 1: X' - X = (3, 0, 4) gives 5 / sqrt(3)
    assert O.update_norm(np.array([[3.0], [0.0], [4.0]]), np.zeros((3, 1))) == pytest.approx(5.0 / math.sqrt(3.0))


def test_se_update_norm_closed_form():
    """sqrt((||X' - X||_F^2 + ||t' - t||^2) / (nd)) with n = 2, d = 2: the rotation
    part as above (4 - 4 cos th) and a translation change (3, 4) at node 0
    (25), so the norm is sqrt((29 - 4 cos th) / 4)."""
    th = 0.7
    X = np.vstack([np.eye(2), np.eye(2)])
    Xn = np.vstack([rot(th), np.eye(2)])
    t = np.zeros((2, 2))
    tn = np.array([[3.0, 4.0], [0.0, 0.0]])
    want = math.sqrt((29.0 - 4.0 * math.cos(th)) / 4.0)
    assert O.se_update_norm(Xn, X, tn, t, 2, 2) == pytest.approx(want, rel=1e-14)
    # with no translation change it is the rotation-only norm
    assert O.se_update_norm(Xn, X, t, t, 2, 2) == pytest.approx(O.update_norm(Xn, X), rel=1e-14)
