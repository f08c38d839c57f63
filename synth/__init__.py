"""Seeded synthetic instances of orthogonal group synchronization.

This module only *generates inputs*.  It holds none of the NS-RGS arithmetic
(no gradient, projection, Newton-Schulz step, spectral initialisation or
distance): both the FP64 CPU oracle and the CUDA library receive the arrays
built here, so the two sides never share method code.

Measurement model (paper §1.1 and eq. (4) of §2.2): for i < j

    A_ij = Z_i Z_j^T + sigma * W_ij,   W_ij with i.i.d. N(0, 1) entries,
    A_ji = A_ij^T,   A_ii = I_d   (W_ii = 0, self-loops excluded).

Ground truth (§4.1): i.i.d. standard Gaussian d x d matrices projected onto
O(d), i.e. the polar factor U V^T of each draw (det = -1 is allowed).

Incomplete observations (§4.1): each unordered pair {i, j} is observed with
probability p; an unobserved pair has A_ij = A_ji = 0.  The mask is symmetric
because A is symmetric; the diagonal is always present.

Noise scale used by the workloads: sigma = c * sqrt(n) / (sqrt(d) + sqrt(ln n))
(natural log), with c stated per workload.

Canonical packed order ("upper-block list"): the n(n-1)/2 blocks (i, j), i < j,
ordered by i, then j; each block d x d row-major.  Block (i, j) sits at index
``upper_index(i, j, n)``.

Random-stream order, fixed so instances are reproducible from (n, d, sigma, p,
seed): one ``numpy.random.Generator(PCG64(seed))``; first the n ground-truth
draws (n*d*d normals), then for each block row i = 0..n-2 the W_ij draws for
j = i+1..n-1 ((n-1-i)*d*d normals) followed, when p < 1, by (n-1-i) uniforms for
the observation mask (pair observed iff uniform < p).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "sigma_rule",
    "haar_orthogonal",
    "upper_index",
    "num_upper_blocks",
    "upper_blocks",
    "dense_from_upper",
    "block_row",
    "Instance",
    "make_instance",
    "SEInstance",
    "make_se_instance",
    "device_se",
]


def sigma_rule(c: float, n: int, d: int) -> float:
    """sigma = c * sqrt(n) / (sqrt(d) + sqrt(ln n))."""
    return float(c) * math.sqrt(n) / (math.sqrt(d) + math.sqrt(math.log(n)))


def haar_orthogonal(rng: np.random.Generator, n: int, d: int) -> np.ndarray:
    """n ground-truth blocks: Gaussian d x d draws projected onto O(d) (§4.1)."""
    g = rng.standard_normal((n, d, d))
    u, _, vt = np.linalg.svd(g)
    return u @ vt


def num_upper_blocks(n: int) -> int:
    return n * (n - 1) // 2


def upper_index(i: int, j: int, n: int) -> int:
    """Index of block (i, j), i < j, in the canonical upper-block list."""
    if not 0 <= i < j < n:
        raise ValueError(f"need 0 <= i < j < n, got i={i} j={j} n={n}")
    return i * n - i * (i + 1) // 2 + (j - i - 1)


def upper_blocks(
    Z: np.ndarray,
    sigma: float,
    rng: np.random.Generator,
    p: float = 1.0,
    dtype=np.float64,
) -> np.ndarray:
    """Canonical upper-block list of A (shape (n(n-1)/2, d, d)).

    Each block row is built in float64 and then stored in ``dtype``.
    """
    n, d, _ = Z.shape
    out = np.empty((num_upper_blocks(n), d, d), dtype=dtype)
    off = 0
    for i in range(n - 1):
        m = n - 1 - i
        w = rng.standard_normal((m, d, d))
        blk = Z[i][None, :, :] @ np.transpose(Z[i + 1 :], (0, 2, 1))
        blk += sigma * w
        if p < 1.0:
            keep = rng.random(m) < p
            blk[~keep] = 0.0
        out[off : off + m] = blk
        off += m
    return out


def dense_from_upper(upper: np.ndarray, n: int, d: int, dtype=np.float64) -> np.ndarray:
    """Symmetric nd x nd matrix with A_ii = I_d and the given upper blocks."""
    U = np.zeros((n * d, n * d), dtype=dtype)
    off = 0
    for i in range(n - 1):
        m = n - 1 - i
        row = upper[off : off + m]  # (m, d, d): blocks (i, i+1..n-1)
        U[i * d : (i + 1) * d, (i + 1) * d :] = np.transpose(row, (1, 0, 2)).reshape(d, m * d)
        off += m
    A = U + U.T
    A[np.diag_indices(n * d)] += 1.0
    return A


def block_row(upper: np.ndarray, n: int, d: int, i: int) -> np.ndarray:
    """Block row i of A (d x nd, float64) read from the canonical upper-block list."""
    R = np.zeros((d, n * d))
    for j in range(n):
        if j == i:
            R[:, j * d : (j + 1) * d] = np.eye(d)
        elif j > i:
            R[:, j * d : (j + 1) * d] = upper[upper_index(i, j, n)]
        else:
            R[:, j * d : (j + 1) * d] = np.asarray(upper[upper_index(j, i, n)]).T
    return R


@dataclass
class Instance:
    """One synthetic instance; ``upper`` is the canonical upper-block list."""

    n: int
    d: int
    sigma: float
    p: float
    seed: int
    Z: np.ndarray
    upper: np.ndarray
    meta: dict = field(default_factory=dict)

    def dense(self, dtype=np.float64) -> np.ndarray:
        return dense_from_upper(self.upper, self.n, self.d, dtype=dtype)

    def Zstack(self) -> np.ndarray:
        """Ground truth stacked as an nd x d matrix (Z_1; ...; Z_n)."""
        return self.Z.reshape(self.n * self.d, self.d)


def device_upper(n: int, d: int, sigma: float, seed: int, p: float = 1.0, device="cuda"):
    """The same measurement model generated on a GPU with torch's seeded RNG.

    Returns (Z (n, d, d) float32, canonical upper-block list (n(n-1)/2, d, d)
    float32) as torch tensors on ``device``.  The random stream differs from
    ``make_instance``'s NumPy stream (so results differ draw by draw, not in
    distribution); it exists for workloads too large to build on the host
    quickly (hundreds of instances, serving streams), where no oracle
    comparison is made.
    """
    import torch

    # ground truth on the host (n small d x d polar factors), noise on the device
    Z = torch.from_numpy(haar_orthogonal(np.random.default_rng(int(seed)), n, d).astype(np.float32)).to(device)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    iu, ju = torch.triu_indices(n, n, offset=1, device=device)
    nb = iu.numel()
    out = torch.empty((nb, d, d), dtype=torch.float32, device=device)
    chunk = max(1, (1 << 24) // (d * d))
    for s in range(0, nb, chunk):
        e = min(nb, s + chunk)
        blk = Z[iu[s:e]] @ Z[ju[s:e]].transpose(1, 2)
        blk += sigma * torch.randn((e - s, d, d), generator=g, device=device, dtype=torch.float32)
        if p < 1.0:
            keep = torch.rand((e - s,), generator=g, device=device) < p
            blk *= keep[:, None, None].to(blk.dtype)
        out[s:e] = blk
    return Z, out


def make_instance(n: int, d: int, sigma: float, seed: int, p: float = 1.0, dtype=np.float64) -> Instance:
    if n < 2 or d < 1:
        raise ValueError("need n >= 2 and d >= 1")
    if not 0.0 < p <= 1.0:
        raise ValueError("need 0 < p <= 1")
    rng = np.random.Generator(np.random.PCG64(seed))
    Z = haar_orthogonal(rng, n, d)
    up = upper_blocks(Z, sigma, rng, p=p, dtype=dtype)
    return Instance(n=n, d=d, sigma=float(sigma), p=float(p), seed=int(seed), Z=Z, upper=up)


def make_negative_dominated(n: int, d: int, seed: int, beta: float = 1.5, sigma: float = 0.2,
                            dtype=np.float32) -> Instance:
    """An instance whose largest-magnitude eigenvalues are negative.

    The measurement model above (small noise sigma) minus beta * n * M_off, where
    M = U U^T for a random orthonormal nd x d basis U and M_off is M with its
    diagonal blocks zeroed (so A_ii = I still holds).  The spectrum then has d
    eigenvalues near n (the ground truth Z, the algebraic top d) and d near
    -beta * n, which dominate in magnitude for beta > 1.  Input for checking
    that a spectral start finds the algebraic top d; a seeded second stream
    [seed, 1] draws U.
    """
    base = make_instance(n, d, sigma, seed, dtype=np.float64)
    U = dense_from_upper(base.upper, n, d) - np.eye(n * d)
    rng = np.random.Generator(np.random.PCG64([seed, 1]))
    Q, _ = np.linalg.qr(rng.standard_normal((n * d, d)))
    U -= beta * n * (Q @ Q.T)
    up = np.empty((num_upper_blocks(n), d, d), dtype=dtype)
    for i in range(n - 1):
        for j in range(i + 1, n):
            up[upper_index(i, j, n)] = U[i * d : (i + 1) * d, j * d : (j + 1) * d]
    return Instance(n=n, d=d, sigma=float(sigma), p=1.0, seed=int(seed), Z=base.Z, upper=up,
                    meta={"beta": float(beta)})


@dataclass
class SEInstance:
    """Poses (Z_i, tau_i) and measurements of the SE(d) form.

    ``rot`` is the rotation instance (exactly ``make_instance`` with the same
    arguments); ``tau`` (n, d) are the true translations; ``c_upper``
    (n(n-1)/2, d) holds c_ij = Z_i (tau_j - tau_i) + sigma_t w_ij for i < j in
    the canonical upper order (zero for an unobserved pair); ``mask_upper``
    (n(n-1)/2,) is 1 for an observed pair.
    """

    rot: Instance
    sigma_t: float
    tau: np.ndarray
    c_upper: np.ndarray
    mask_upper: np.ndarray

    def c_square(self) -> np.ndarray:
        """c as an (n, n, d) float64 array with c[i, j] = c_ij for i < j, zero elsewhere."""
        n, d = self.rot.n, self.rot.d
        out = np.zeros((n, n, d))
        iu, ju = np.triu_indices(n, 1)
        out[iu, ju] = self.c_upper
        return out

    def mask_square(self) -> np.ndarray:
        """Symmetric (n, n) 0/1 observation mask (diagonal 0)."""
        n = self.rot.n
        m = np.zeros((n, n))
        iu, ju = np.triu_indices(n, 1)
        m[iu, ju] = self.mask_upper
        return m + m.T


def make_se_instance(n: int, d: int, sigma: float, sigma_t: float, seed: int, p: float = 1.0,
                     dtype=np.float64) -> SEInstance:
    """Rotation part from ``make_instance(n, d, sigma, seed, p)``; translations from a
    second generator PCG64([seed, 1]): first tau (n*d normals), then the translation
    noise w_ij (n(n-1)/2 * d normals, canonical upper order).  An unobserved pair
    (zero rotation block) has c_ij = 0 and mask 0."""
    rot = make_instance(n, d, sigma, seed, p=p, dtype=dtype)
    rng = np.random.Generator(np.random.PCG64([seed, 1]))
    tau = rng.standard_normal((n, d))
    w = rng.standard_normal((num_upper_blocks(n), d))
    iu, ju = np.triu_indices(n, 1)
    c = np.einsum("kab,kb->ka", rot.Z[iu], tau[ju] - tau[iu]) + sigma_t * w
    mask = np.any(np.asarray(rot.upper) != 0, axis=(1, 2)).astype(np.float64)
    c *= mask[:, None]
    return SEInstance(rot=rot, sigma_t=float(sigma_t), tau=tau, c_upper=c.astype(dtype), mask_upper=mask)


def device_se(n: int, d: int, sigma: float, sigma_t: float, seed: int, device="cuda"):
    """The SE(d) measurement model generated on a GPU (complete graph), for workloads
    too large to build on the host: returns (Z, tau, A upper-block list, c upper list)
    as float32 torch tensors.  Rotation part as ``device_upper``; no oracle comparison."""
    import torch

    Z, up = device_upper(n, d, sigma, seed, device=device)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) + 1)
    tau = torch.randn((n, d), generator=g, device=device, dtype=torch.float32)
    iu, ju = torch.triu_indices(n, n, offset=1, device=device)
    nb = iu.numel()
    c = torch.empty((nb, d), dtype=torch.float32, device=device)
    chunk = 1 << 22
    for s in range(0, nb, chunk):
        e = min(nb, s + chunk)
        c[s:e] = torch.einsum("kab,kb->ka", Z[iu[s:e]], tau[ju[s:e]] - tau[iu[s:e]])
        c[s:e] += sigma_t * torch.randn((e - s, d), generator=g, device=device, dtype=torch.float32)
    return Z, tau, up, c
