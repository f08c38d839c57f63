"""Plain FP64 NumPy oracle of NS-RGS (Peng, Han, Chen, Huang, arXiv 2604.07372).

TEST INFRASTRUCTURE ONLY: used by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``; never by the CUDA product path.

Everything here is written straight from the paper's definitions, in float64,
with library primitives (matmul, SVD, symmetric eigensolver) as steps and no
blocking, fusion or reordering beyond what the definitions state.

Notation (paper §1.4): X = (X_1; ...; X_n) is nd x d with d x d blocks X_i;
A = [A_ij] is the symmetric nd x nd matrix of pairwise measurements with
A_ii = I_d (self-loops excluded, §2.2 eq. (4)).

Readings of points the paper leaves open (each one also listed in the design
notes of the repository):
  * gradient: Algorithm 2's form G_i = sum_{j != i} (X_i - A_ij X_j), taken
    literally (also for sparse data, where unobserved A_ij = 0);
  * projection: the paper's (G - X_i G^T X_i)/2, applied also when X_i is only
    approximately orthogonal ("pseudo projection", §2.2);
  * all blocks are updated simultaneously from X^t (Algorithm 2 uses X_j^t on
    the right-hand side);
  * Newton-Schulz starts unscaled, S_0 = F_i (Algorithm 1);
  * spectral initialisation takes the eigenvectors of the d largest
    *algebraic* eigenvalues of A;
  * GPM (the paper's comparison method, not written out there) is read as
    X_i <- sgn(sum_j A_ij X_j) including the j = i term A_ii X_i = X_i.

Pins (tests marked "not gpu" in tests/test_oracle_pins.py) tie each function
to something other than itself: the Newton-Schulz singular-value map and
Lemma 2.1's bound, tangent-space identities, a finite-difference check of the
gradient, hand-derived closed forms of one iteration for rotations in O(2),
exact recovery at sigma = 0, equivariance, brute-force minimality of d_F,
Courant-Fischer for the spectral subspace, and Table 1's relative errors.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "sgn",
    "sgn_blocks",
    "newton_schulz",
    "tangent_projection",
    "euclidean_gradient",
    "nsrgs_iteration",
    "ns_safeguard",
    "nsrgs_rows_update",
    "spectral_init",
    "nsrgs",
    "objective",
    "dF",
    "rel_err",
    "mse",
    "update_norm",
    "gpm_iteration",
    "gpm",
    "stiefel_gradient",
    "stiefel_projection",
    "newton_schulz_rows",
    "polar_rows",
    "stiefel_iteration",
    "se_residuals",
    "se_objective",
    "se_gradient",
    "se_iteration",
    "se_update_norm",
    "se_nsrgs",
    "se_errors",
    "blocks",
    "stack",
]


# ---------------------------------------------------------------- helpers
def blocks(X: np.ndarray, d: int) -> np.ndarray:
    """View the nd x d stack X as an (n, d, d) array of blocks X_i."""
    return np.asarray(X, dtype=np.float64).reshape(-1, d, d)


def stack(Xb: np.ndarray) -> np.ndarray:
    """Inverse of ``blocks``: (n, d, d) -> nd x d."""
    n, d, _ = Xb.shape
    return Xb.reshape(n * d, d)


# ------------------------------------------------------ §2.1: matrix sign
def sgn(M: np.ndarray) -> np.ndarray:
    """Matrix sign of a square matrix (§2.1): M = U Sigma V^T (full SVD) -> U V^T."""
    U, _, Vt = np.linalg.svd(np.asarray(M, dtype=np.float64))
    return U @ Vt


def sgn_blocks(Phi: np.ndarray, d: int) -> np.ndarray:
    """Blockwise matrix sign of an nd x d stack (§2.1): (sgn(A_1); ...; sgn(A_n))."""
    Pb = blocks(Phi, d)
    U, _, Vt = np.linalg.svd(Pb)
    return stack(U @ Vt)


# ------------------------------------ §2.1, Algorithm 1: Newton-Schulz
def newton_schulz(M: np.ndarray, Ts: int) -> np.ndarray:
    """Algorithm 1: S_0 = M, S_{t+1} = (1/2) S_t (3 I - S_t^T S_t), t < Ts.

    Accepts one d x d matrix or a stack (n, d, d) of them (applied blockwise).
    """
    S = np.array(M, dtype=np.float64, copy=True)
    d = S.shape[-1]
    I = np.eye(d)
    for _ in range(Ts):
        S = 0.5 * (S @ (3.0 * I - np.swapaxes(S, -1, -2) @ S))
    return S


# ---------------------------------------------- §2.2: tangent projection
def tangent_projection(Xi: np.ndarray, G: np.ndarray) -> np.ndarray:
    """P_{X_i}(G) = (G - X_i G^T X_i) / 2 (§2.2); blockwise on (n, d, d) stacks."""
    Xi = np.asarray(Xi, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    return 0.5 * (G - Xi @ np.swapaxes(G, -1, -2) @ Xi)


# ------------------------------------------ §2.2 / Algorithm 2: gradient
def euclidean_gradient(A: np.ndarray, X: np.ndarray, n: int, d: int) -> np.ndarray:
    """G_i = sum_{j != i} (X_i - A_ij X_j) for every i (Algorithm 2), as (n, d, d).

    sum_{j != i} A_ij X_j is the i-th block of A X minus the diagonal term
    A_ii X_i; the library matmul A @ X serves as the step that forms A X.
    """
    A = np.asarray(A, dtype=np.float64)
    Xb = blocks(X, d)
    AX = blocks(A @ stack(Xb), d)
    Aii = np.stack([A[i * d : (i + 1) * d, i * d : (i + 1) * d] for i in range(n)])
    offdiag = AX - Aii @ Xb
    return (n - 1) * Xb - offdiag


# ------------------- beyond the paper: safeguarded Newton-Schulz start
def ns_safeguard(F: np.ndarray) -> np.ndarray:
    """Safeguarded start of Algorithm 1 (not part of the paper's method).

    Lemma 2.1 needs ||I - F_i^T F_i|| < 1 for the Newton-Schulz iteration to
    converge; the test here uses the Frobenius norm (an upper bound of the
    spectral norm).  A block F_i that fails it is replaced by F_i / ||F_i||_F:
    its singular values move into (0, 1], where the Newton-Schulz map converges
    to the polar factor, and the polar factor itself is unchanged
    (sgn(c F) = sgn(F) for c > 0).  Blocks that pass are left as they are, so
    on data where the precondition always holds this is Algorithm 2 exactly.
    Accepts one d x d matrix or a stack (n, d, d).
    """
    F = np.array(F, dtype=np.float64, copy=True)
    one = F.ndim == 2
    if one:
        F = F[None]
    d = F.shape[-1]
    E = np.eye(d) - np.swapaxes(F, -1, -2) @ F
    bad = np.sqrt(np.sum(E * E, axis=(-2, -1))) >= 1.0
    norms = np.sqrt(np.sum(F * F, axis=(-2, -1)))
    F[bad] = F[bad] / norms[bad][:, None, None]
    return F[0] if one else F


# ------------------------------------------ Algorithm 2: one iteration
def nsrgs_iteration(
    A: np.ndarray, X: np.ndarray, n: int, d: int, mu: float, Ts: int, safeguard: bool = False
) -> np.ndarray:
    """One sweep of Algorithm 2's loop body for all i, every block from X^t.

    G_i = sum_{j != i}(X_i - A_ij X_j);  F_i = X_i - mu P_{X_i}(G_i);
    X_i^{t+1} = S(F_i) with S = Algorithm 1 run for Ts steps.  With
    ``safeguard`` the Newton-Schulz start is ``ns_safeguard(F)`` (beyond the paper).
    """
    Xb = blocks(X, d)
    G = euclidean_gradient(A, X, n, d)
    F = Xb - mu * tangent_projection(Xb, G)
    if safeguard:
        F = ns_safeguard(F)
    return stack(newton_schulz(F, Ts))


def nsrgs_rows_update(Arows: np.ndarray, X: np.ndarray, idx, n: int, d: int, mu: float, Ts: int) -> np.ndarray:
    """Algorithm 2's loop body for the listed blocks i only, as (len(idx), d, d).

    ``Arows[k]`` is the whole k-th listed block row of A (d x nd), so one block
    update costs O(n d^2): this lets a sample of blocks of a very large instance
    be checked one by one.  Same steps as ``nsrgs_iteration``.
    """
    Xs = np.asarray(X, dtype=np.float64)
    Xb = blocks(Xs, d)
    out = []
    for k, i in enumerate(idx):
        Ar = np.asarray(Arows[k], dtype=np.float64)
        off = Ar @ Xs - Ar[:, i * d : (i + 1) * d] @ Xb[i]  # sum_{j != i} A_ij X_j
        G = (n - 1) * Xb[i] - off
        F = Xb[i] - mu * tangent_projection(Xb[i], G)
        out.append(newton_schulz(F, Ts))
    return np.stack(out)


# ---------------------------------------- Algorithm 2: spectral start
def spectral_init(A: np.ndarray, n: int, d: int, method: str = "auto") -> tuple[np.ndarray, np.ndarray]:
    """Spectral initialisation of Algorithm 2.

    Y = eigenvectors of the d largest (algebraic) eigenvalues of A, Y^T Y = I;
    X^0 = sgn_n(Y) (blockwise matrix sign).  Returns (X0, Y).

    ``method='eigh'`` is the full symmetric eigensolver (LAPACK); ``'eigsh'`` the
    ARPACK Lanczos solver for the same top-d eigenpairs, used for large nd
    where the full solve takes minutes.  ``'auto'`` picks eigh for nd <= 4000.
    """
    A = np.asarray(A, dtype=np.float64)
    N = n * d
    if method == "auto":
        method = "eigh" if N <= 4000 else "eigsh"
    if method == "eigh":
        w, V = np.linalg.eigh(A)
        order = np.argsort(w)[::-1][:d]
        Y = V[:, order]
    elif method == "eigsh":
        from scipy.sparse.linalg import eigsh

        v0 = np.ones(N) / math.sqrt(N)
        w, V = eigsh(A, k=d, which="LA", v0=v0, tol=1e-13, maxiter=20 * N)
        Y = V[:, np.argsort(w)[::-1]]
    else:
        raise ValueError(method)
    return sgn_blocks(Y, d), Y


# ----------------------------------------------- eq. (1): objective F
def objective(A: np.ndarray, X: np.ndarray, n: int, d: int) -> float:
    """F(X) = (1/2) sum_{i != j} ||X_i X_j^T - A_ij||_F^2 (eq. (1))."""
    X = np.asarray(X, dtype=np.float64)
    total = 0.0
    for i in range(n):
        rows = slice(i * d, (i + 1) * d)
        R = X[rows] @ X.T - np.asarray(A[rows], dtype=np.float64)  # d x nd: blocks j = 0..n-1
        R[:, i * d : (i + 1) * d] = 0.0  # j = i excluded
        total += float(np.sum(R * R))
    return 0.5 * total


# -------------------------------------------------- Algorithm 2: loop
def nsrgs(
    A: np.ndarray,
    n: int,
    d: int,
    mu: float,
    T: int,
    Ts: int,
    X0: np.ndarray | None = None,
    rel_tol: float | None = None,
    history: bool = False,
    safeguard: bool = False,
):
    """Algorithm 2: spectral start (unless X0 is given), then up to T iterations.

    With ``rel_tol`` set, stops after the first iteration t whose relative
    decrease R^t = (F(X^t) - F(X^{t+1})) / F(X^{t+1}) is below it (§4.1's rule:
    R^t < 1e-8 or 100 iterations).  Returns (X, info) where info holds the
    number of iterations run and, with ``history``, every iterate's update
    norm ||X^{t+1} - X^t||_F / sqrt(nd).  ``safeguard`` as in ``nsrgs_iteration``.
    """
    if X0 is None:
        X0, _ = spectral_init(A, n, d)
    X = np.array(X0, dtype=np.float64, copy=True)
    info = {"iters": 0, "upd": []}
    Fcur = objective(A, X, n, d) if rel_tol is not None else None
    for t in range(T):
        Xn = nsrgs_iteration(A, X, n, d, mu, Ts, safeguard)
        if history:
            info["upd"].append(update_norm(Xn, X))
        info["iters"] = t + 1
        if rel_tol is not None:
            Fn = objective(A, Xn, n, d)
            R = (Fcur - Fn) / Fn if Fn != 0.0 else 0.0
            X, Fcur = Xn, Fn
            if R < rel_tol:
                break
        else:
            X = Xn
    return X, info


# ------------------------------------- §1.4 notations: distance d_F
def dF(X: np.ndarray, Y: np.ndarray, d: int) -> float:
    """d_F(X, Y) = min_{Q in O(d)} ||X - Y Q||_F (§1.4).

    The minimiser is Q* = sgn(Y^T X) (proof of Lemma 7.4); the distance is then
    evaluated directly as ||X - Y Q*||_F rather than through the nuclear-norm
    identity, which keeps resolution near zero.
    """
    X = np.asarray(X, dtype=np.float64).reshape(-1, d)
    Y = np.asarray(Y, dtype=np.float64).reshape(-1, d)
    Q = sgn(Y.T @ X)
    return float(np.linalg.norm(X - Y @ Q))


def rel_err(X: np.ndarray, Z: np.ndarray, d: int, chunk: int = 2048) -> float:
    """Rel.Err = ||Z Z^T - X X^T||_F / ||Z Z^T||_F (§4.1), evaluated by row chunks."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, d)
    Z = np.asarray(Z, dtype=np.float64).reshape(-1, d)
    num = 0.0
    den = 0.0
    for s in range(0, X.shape[0], chunk):
        ZZ = Z[s : s + chunk] @ Z.T
        XX = X[s : s + chunk] @ X.T
        num += float(np.sum((ZZ - XX) ** 2))
        den += float(np.sum(ZZ**2))
    return math.sqrt(num / den)


def mse(Xhat: np.ndarray, X: np.ndarray, n: int, d: int) -> float:
    """MSE = d_F(Xhat, X)^2 / n (§4.2)."""
    return dF(Xhat, X, d) ** 2 / n


def update_norm(Xnew: np.ndarray, Xold: np.ndarray) -> float:
    """||X^{t+1} - X^t||_F / sqrt(nd): the per-iteration change used as a retire rule."""
    Xnew = np.asarray(Xnew, dtype=np.float64)
    Xold = np.asarray(Xold, dtype=np.float64)
    rows = Xnew.size // Xnew.shape[-1]  # nd
    return float(np.linalg.norm(Xnew - Xold) / math.sqrt(rows))


# --------------------------------------------- GPM (comparison method)
def gpm_iteration(A: np.ndarray, X: np.ndarray, n: int, d: int) -> np.ndarray:
    """Generalised power method step X_i <- sgn((A X)_i), with A_ii = I included.

    The paper compares against GPM (§1.1, §4.1) without writing it out; this is
    the reading used here: one full matrix product followed by an exact
    blockwise matrix sign.
    """
    return sgn_blocks(np.asarray(A, dtype=np.float64) @ np.asarray(X, dtype=np.float64), d)


def gpm(A: np.ndarray, n: int, d: int, T: int, X0: np.ndarray | None = None):
    if X0 is None:
        X0, _ = spectral_init(A, n, d)
    X = np.array(X0, dtype=np.float64, copy=True)
    for _ in range(T):
        X = gpm_iteration(A, X, n, d)
    return X


# ---------------------- beyond the paper: Stiefel form (d x p blocks)
# The relaxation of O(d) synchronisation to row-orthonormal blocks X_i in
# R^{d x p} (X_i X_i^T = I_d, p >= d), which §1.2 cites (Stiefel manifold,
# Burer-Monteiro) and §6 names as an extension.  The same objective F (eq. (1))
# and the same three steps as Algorithm 2; with p = d they are Algorithm 2's.
def stiefel_gradient(A: np.ndarray, X: np.ndarray, n: int, d: int) -> np.ndarray:
    """Blockwise Euclidean gradient at X (nd x p) as (n, d, p) blocks, the gradient of
    f_i = 1/2 sum_{j != i} ||X_i X_j^T - A_ij||^2 in X_i (half of dF/dX_i, as in Algorithm 2):
    G_i = sum_{j != i} (X_i X_j^T - A_ij) X_j = X_i (X^T X - X_i^T X_i) - (A_off X)_i.
    (For X_j in O(d), X_j^T X_j = I and this is Algorithm 2's (n-1) X_i - (A_off X)_i.)"""
    A = np.asarray(A, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    Xb = X.reshape(n, d, -1)
    C = X.T @ X
    AX = (A @ X).reshape(n, d, -1)
    Aii = np.stack([A[i * d : (i + 1) * d, i * d : (i + 1) * d] for i in range(n)])
    Y = AX - Aii @ Xb  # (A_off X)_i = sum_{j != i} A_ij X_j
    return Xb @ (C[None, :, :] - np.swapaxes(Xb, -1, -2) @ Xb) - Y


def stiefel_projection(Xi: np.ndarray, G: np.ndarray) -> np.ndarray:
    """Projection onto the tangent space of the row-orthonormal matrices at X_i:
    P(G) = G - sym(G X_i^T) X_i  (tangent vectors H satisfy H X_i^T + X_i H^T = 0).
    With X_i square and orthogonal this is the paper's (G - X_i G^T X_i)/2."""
    Xi = np.asarray(Xi, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    T = G @ np.swapaxes(Xi, -1, -2)
    return G - 0.5 * (T + np.swapaxes(T, -1, -2)) @ Xi


def newton_schulz_rows(M: np.ndarray, Ts: int) -> np.ndarray:
    """Algorithm 1 for a d x p block with full row rank: S <- (3I - S S^T) S / 2,
    Ts times; converges to the polar factor U V^T of M = U Sigma V^T when the
    singular values lie in (0, sqrt(3)).  For square M this is Algorithm 1."""
    S = np.array(M, dtype=np.float64, copy=True)
    d = S.shape[-2]
    I = np.eye(d)
    for _ in range(Ts):
        S = 0.5 * ((3.0 * I - S @ np.swapaxes(S, -1, -2)) @ S)
    return S


def polar_rows(M: np.ndarray) -> np.ndarray:
    """Polar factor U V^T of a full-row-rank d x p matrix (thin SVD)."""
    U, _, Vt = np.linalg.svd(np.asarray(M, dtype=np.float64), full_matrices=False)
    return U @ Vt


def stiefel_iteration(A: np.ndarray, X: np.ndarray, n: int, d: int, mu: float, Ts: int) -> np.ndarray:
    """One sweep of the Stiefel form for all blocks from X (nd x p)."""
    X = np.asarray(X, dtype=np.float64)
    Xb = X.reshape(n, d, -1)
    G = stiefel_gradient(A, X, n, d)
    F = Xb - mu * stiefel_projection(Xb, G)
    return newton_schulz_rows(F, Ts).reshape(n * d, -1)


# ------------------------- beyond the paper: SE(d) form (poses = rotation + translation)
# §6 names the special Euclidean group as a target for the Newton-Schulz retraction
# without writing a method for it; this is the reading the repository builds.
# Unknowns: X_i in O(d) (as in the paper) and t_i in R^d.  Measurements for an
# observed pair i < j (mask w_ij in {0, 1}): A_ij ~ X_i X_j^T (the paper's model) and
# c_ij ~ X_i (t_j - t_i), the translation from i to j in the frame of i.  Objective
#     f(X, t) = F(X) + kappa sum_{i<j} w_ij ||t_j - t_i - X_i^T c_ij||^2
# with F of eq. (1).  One iteration from (X^t, t^t), all blocks at once:
#     G^X_i = sum_{j != i}(X_i - A_ij X_j) - kappa sum_{j>i} w_ij c_ij (t_j - t_i)^T
#     G^t_k = kappa [sum_{i<k} w_ik r_ik - sum_{j>k} w_kj r_kj],  r_ij = t_j - t_i - X_i^T c_ij
#     X_i <- S_K(X_i - mu P_{X_i}(G^X_i))  (Algorithm 1),   t_k <- t_k - mu_t G^t_k.
# G^X and G^t are half the Euclidean gradient of f, like Algorithm 2's G, with the same
# simplification on the manifold: Algorithm 2 uses X_j^T X_j = I, and here the term
# kappa sum_j w_ij c_ij c_ij^T X_i is dropped, whose projection P_{X_i} vanishes when
# X_i is orthogonal (P(M X) = 0 for symmetric M).  G^t is the exact half-gradient.
def se_residuals(Cu: np.ndarray, X: np.ndarray, t: np.ndarray, n: int, d: int) -> np.ndarray:
    """r_ij = t_j - t_i - X_i^T c_ij for every ordered i < j, as an (n, n, d) array (zero elsewhere)."""
    Xb = blocks(X, d)
    t = np.asarray(t, dtype=np.float64).reshape(n, d)
    R = np.zeros((n, n, d))
    for i in range(n - 1):
        c = np.asarray(Cu[i, i + 1 :], dtype=np.float64)  # (m, d)
        R[i, i + 1 :] = t[i + 1 :] - t[i][None, :] - c @ Xb[i]  # (X_i^T c)^T = c^T X_i
    return R


def se_objective(A, Cu, Wm, X, t, n: int, d: int, kappa: float) -> float:
    """f(X, t) = F(X) + kappa sum_{i<j} w_ij ||t_j - t_i - X_i^T c_ij||^2."""
    R = se_residuals(Cu, X, t, n, d)
    W = np.triu(np.asarray(Wm, dtype=np.float64), 1)
    return objective(A, X, n, d) + kappa * float(np.sum(W[:, :, None] * R * R))


def se_gradient(A, Cu, Wm, X, t, n: int, d: int, kappa: float):
    """(G^X as (n, d, d), G^t as (n, d)) of the SE(d) reading, from the pair sums written out."""
    Xb = blocks(X, d)
    t = np.asarray(t, dtype=np.float64).reshape(n, d)
    W = np.triu(np.asarray(Wm, dtype=np.float64), 1)
    GX = euclidean_gradient(A, X, n, d)
    Gt = np.zeros((n, d))
    R = se_residuals(Cu, X, t, n, d)
    for i in range(n - 1):
        for j in range(i + 1, n):
            if W[i, j] == 0.0:
                continue
            c = np.asarray(Cu[i, j], dtype=np.float64)
            GX[i] -= kappa * np.outer(c, t[j] - t[i])
            Gt[j] += kappa * R[i, j]
            Gt[i] -= kappa * R[i, j]
    return GX, Gt


def se_iteration(A, Cu, Wm, X, t, n: int, d: int, mu: float, mu_t: float, kappa: float, Ts: int):
    """One iteration of the SE(d) form for all blocks from (X^t, t^t): (X^{t+1} nd x d, t^{t+1} (n, d))."""
    Xb = blocks(X, d)
    GX, Gt = se_gradient(A, Cu, Wm, X, t, n, d, kappa)
    F = Xb - mu * tangent_projection(Xb, GX)
    tn = np.asarray(t, dtype=np.float64).reshape(n, d) - mu_t * Gt
    return stack(newton_schulz(F, Ts)), tn


def se_update_norm(Xn, X, tn, t, n: int, d: int) -> float:
    """sqrt((||X' - X||_F^2 + ||t' - t||^2) / (n d)), the update norm of the SE(d) form."""
    dx = np.asarray(Xn, dtype=np.float64) - np.asarray(X, dtype=np.float64)
    dt = np.asarray(tn, dtype=np.float64) - np.asarray(t, dtype=np.float64)
    return math.sqrt((float(np.sum(dx * dx)) + float(np.sum(dt * dt))) / (n * d))


def se_nsrgs(A, Cu, Wm, n: int, d: int, mu: float, mu_t: float, kappa: float, T: int, Ts: int, X0, t0,
             tol: float = 0.0):
    """T iterations of the SE(d) form from (X0, t0); with tol > 0, stops after the first
    iteration whose update norm is below tol.  Returns (X, t, iterations run)."""
    X = np.asarray(X0, dtype=np.float64)
    t = np.asarray(t0, dtype=np.float64).reshape(n, d)
    it = 0
    for _ in range(T):
        Xn, tn = se_iteration(A, Cu, Wm, X, t, n, d, mu, mu_t, kappa, Ts)
        un = se_update_norm(Xn, X, tn, t, n, d)
        X, t, it = Xn, tn, it + 1
        if tol > 0.0 and un < tol:
            break
    return X, t, it


def se_errors(X, t, Z, tau, n: int, d: int) -> tuple[float, float]:
    """(d_F(X, Z), translation RMS error) after the global gauge X -> X Q, t -> Q^T t + v:
    Q minimises ||X - Z Q||_F (as in d_F), v is the mean offset."""
    X = np.asarray(X, dtype=np.float64)
    Zs = np.asarray(Z, dtype=np.float64).reshape(n * d, d)
    U, _, Vt = np.linalg.svd(Zs.T @ X)
    Q = U @ Vt
    e = np.asarray(t, dtype=np.float64).reshape(n, d) - np.asarray(tau, dtype=np.float64).reshape(n, d) @ Q
    e -= e.mean(axis=0, keepdims=True)
    return dF(X, Zs, d), math.sqrt(float(np.sum(e * e)) / n)
