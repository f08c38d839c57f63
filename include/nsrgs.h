/*
 * nsrgs.h -- C ABI of the GB300 (sm_103a) NS-RGS library (libnsrgs.so).
 *
 * NS-RGS (Peng, Han, Chen, Huang, arXiv 2604.07372) recovers X = (X_1; ...; X_n),
 * X_i in O(d), from a symmetric nd x nd matrix of pairwise measurements
 * A = [A_ij] with A_ij ~ Z_i Z_j^T (problem statement §1.1; block model eq. (4),
 * §2.2, where self-loops are excluded so A_ii = I_d).  Each iteration of
 * Algorithm 2 forms, for every block i simultaneously from X^t,
 *
 *     G_i = sum_{j != i} (X_i - A_ij X_j)
 *     F_i = X_i - eta * (G_i - X_i G_i^T X_i) / 2          (tangent projection, §2.2)
 *     X_i^{t+1} = S_K(F_i),  S_{k+1} = S_k (3I - S_k^T S_k) / 2   (Algorithm 1, K steps)
 *
 * and starts from the spectral initialisation X^0 = sgn_n(Y), Y the top-d
 * eigenvectors of A (Algorithm 2).
 *
 * Conventions shared by every entry point
 *  - Matrices are row-major.  X is the nd x d stack of d x d blocks, float32.
 *  - "device" pointers are CUDA global-memory pointers on the current device;
 *    "host" pointers are ordinary CPU memory.  The caller owns every buffer:
 *    the library allocates no device memory.  Scratch space ("workspace") is a
 *    caller-provided device buffer of at least nsrgs_workspace_bytes(n, d)
 *    bytes, 256-byte aligned; its contents between calls are unspecified.
 *  - Every call is asynchronous on the caller's stream `st` (a cudaStream_t,
 *    passed as void* so that this header needs no CUDA header), except where a
 *    host output is written: those calls synchronise `st` before returning.
 *  - Errors are returned as nsrgs_status; nothing is thrown across the ABI and
 *    no kernel traps.  nsrgs_last_error() returns a thread-local message for
 *    the last failing call on the calling thread.
 *  - Argument checks: 2 <= n, 1 <= d <= 64, eta > 0 and finite, K >= 0,
 *    T >= 0, non-null pointers, 16-byte aligned device pointers.
 */
#ifndef NSRGS_H
#define NSRGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NSRGS_OK = 0,
  NSRGS_ERR_INVALID_ARG = 1,   /* a size, pointer or parameter is out of contract, or a packed
                                  buffer is inconsistent (an index or address found on the
                                  device to leave its buffer; the access is skipped) */
  NSRGS_ERR_CUDA = 2,          /* a CUDA runtime call failed (message has the CUDA error) */
  NSRGS_ERR_NOMEM = 3,         /* a caller buffer is smaller than the size query returned */
  NSRGS_ERR_NONFINITE = 4,     /* an iterate became NaN or Inf */
  NSRGS_ERR_NS_PRECOND = 5,    /* ||I - F_i^T F_i||_F >= 1 for some i (Lemma 2.1's precondition
                                  checked conservatively); reported through nsrgs_info.flags */
  NSRGS_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
  NSRGS_ERR_NOT_CONVERGED = 7, /* spectral initialisation hit max_iters above tol */
  NSRGS_ERR_UNSUPPORTED = 8    /* valid arguments that this build does not implement */
} nsrgs_status;

/* Storage precision of the packed A.  Arithmetic is float32 in every case.
 *  F32     : A stored as float32.  For d <= 8 the panel layout on the CUDA cores;
 *            for 8 < d <= 64 the float32 tile-upper layout (64 x 64 tiles of the
 *            upper triangle, each feeding Y_I += A_IJ X_J and Y_J += A_IJ^T X_I on
 *            the CUDA cores): half the bytes of DENSE_F32.
 *  BF16    : A rounded to bfloat16 (round to nearest even).  For d <= 8 the panel
 *            layout on the CUDA cores; for 8 < d <= 64 the tile-upper layout
 *            on the tensor cores (128 x 128 tiles of the upper triangle, each feeding
 *            Y_I += A_IJ X_J and Y_J += A_IJ^T X_I through tcgen05 with X rounded to
 *            bfloat16, float32 accumulation in TMEM): half the bytes of DENSE_BF16.
 *  FP8E4M3 : A stored as FP8 E4M3 (round to nearest, saturating at +-448) with one
 *            float32 scale per block row i: s_i = max_{j>i} max|A_ij| / 448 and
 *            A_ij ~ s_i * q_ij.  The per-block-row scale is this library's choice;
 *            the paper does not discuss reduced precision.  For d <= 4 the panel
 *            layout on the CUDA cores (X float32).  For 8 < d <= 64 the
 *            tile-upper layout of BF16 with one byte per element (16 KB tiles, the n
 *            scales behind them) on the tensor cores (tcgen05 kind::f8f6f4): X
 *            enters as two E4M3 planes hi = RN(g X), lo = RN(g X - hi) at a
 *            power-of-two g from max |X| (about 2^-8 relative together), the column
 *            product takes the rows s_i X_i as its operand (the scale runs along K
 *            there) and the row product's result is multiplied by s_i; float32
 *            accumulation in TMEM.  A quarter of DENSE_BF16's bytes.
 *  DENSE_F32: the full nd x nd float32 matrix, both triangles, no symmetric reuse
 *            (twice the bytes of F32).  Works for every d; it is the plain form the
 *            symmetric layouts are measured against.
 *  DENSE_BF16: the full matrix in bfloat16 for d in {16, 32, 64}, multiplied on the
 *            tensor cores (tcgen05, float32 accumulation in TMEM) with X rounded to
 *            bfloat16 for the product; the d x d work stays float32.
 *  BCSR_F32 / BCSR_BF16: block-sparse rows for incomplete observations (§4.1's
 *            sampling model, unobserved A_ij = 0), d <= 8: only blocks with a
 *            nonzero entry are stored, both A_ij and A_ji = A_ij^T, each block row
 *            complete and sorted by j, so one warp owns a row and no atomics are
 *            needed.  Bytes per A pass ~ 2 p (n^2 - n) d^2 E: below the symmetric
 *            panels whenever the observed fraction p < 1/2.  The exact size depends
 *            on the data: nsrgs_bcsr_packed_bytes; nsrgs_packed_bytes returns the
 *            bound for p = 1.  Values are stored in groups of 32 consecutive blocks,
 *            interleaved element by element (element e = r*d + c of block k at
 *            32*d*d*(k/32) + 32*e + k%32, the last group zero-padded), so that a
 *            warp taking 32 blocks reads each element with coalesced loads.  Used
 *            by the single-instance, batched and served forms. */
typedef enum {
  NSRGS_F32 = 0,
  NSRGS_BF16 = 1,
  NSRGS_FP8E4M3 = 2,
  NSRGS_DENSE_F32 = 3,
  NSRGS_DENSE_BF16 = 4,
  NSRGS_BCSR_F32 = 5,
  NSRGS_BCSR_BF16 = 6
} nsrgs_storage;

/* A packed measurement matrix.  `packed` is the device buffer written by
 * nsrgs_pack_upper / nsrgs_pack_dense for the same (n, d, storage).  Only the
 * strict block-upper triangle of A is kept (symmetric layouts): A_ji = A_ij^T
 * and A_ii = I_d are implied, which is the model of eq. (4).  The struct lives
 * in host memory; the library keeps no pointer to it after a call returns. */
typedef struct nsrgs_A {
  const void* packed;
  int n;
  int d;
  int storage; /* nsrgs_storage */
} nsrgs_A;

/* Host-side report filled by nsrgs_solve when `info` is non-null. */
typedef struct nsrgs_info {
  int spectral_iters;      /* subspace iterations run by the spectral initialisation (0 if skipped) */
  int iters;               /* NS-RGS iterations run (< T when tol > 0 stopped the loop early) */
  double last_update_norm; /* ||X^{t+1} - X^t||_F / sqrt(nd) of the last iteration run */
  double spectral_residual;/* ||A V - V H||_F / ||H||_F at the end of the spectral initialisation */
  uint32_t flags;          /* bit 0: non-finite iterate; bit 1: NS precondition violated;
                              bit 2: spectral initialisation not converged;
                              bit 4: the safeguarded Newton-Schulz start acted;
                              bit 6: the spectral initialisation restarted with a larger
                              shift to reach the algebraic top-d (see nsrgs_spectral_init);
                              bit 7: the spectral initialisation stopped at its product's
                              precision floor, above tol (tensor-core storages, and F32 at
                              8 < d <= 64; see nsrgs_spectral_init) */
  double objective;        /* nsrgs_solve_objective: F(X) of eq. (1) at the returned X; NaN otherwise */
  double rel_decrease;     /* nsrgs_solve_objective: the last relative decrease R^t formed; NaN otherwise */
} nsrgs_info;

/* ---------------------------------------------------------------- sizes */

/* Bytes of the packed buffer for (n, d, storage); 0 if the combination is not
 * supported (F32: any d <= 64; BF16: any d <= 64; FP8E4M3: d <= 4 and 8 < d <= 64;
 * DENSE_F32: any d <= 64; DENSE_BF16: d in {16, 32, 64}; BCSR_*: d <= 8, the
 * bound for fully observed data -- see nsrgs_bcsr_packed_bytes for the exact size). */
size_t nsrgs_packed_bytes(int n, int d, int storage);

/* Bytes of scratch workspace that every call below accepts for (n, d). */
size_t nsrgs_workspace_bytes(int n, int d);

/* Exact bytes of a block-sparse packed buffer (storage NSRGS_BCSR_F32 or
 * NSRGS_BCSR_BF16) for the given data: `src` (device, float32) is the canonical
 * upper-block list (src_is_dense = 0) or the dense nd x nd matrix (src_is_dense
 * != 0), as passed to nsrgs_pack_upper / nsrgs_pack_dense.  Counts the blocks
 * with a nonzero entry on the device (using the workspace), then synchronises
 * `st` and writes *bytes (host). */
nsrgs_status nsrgs_bcsr_packed_bytes(const float* src, int src_is_dense, int n, int d, int storage, size_t* bytes,
                                     void* ws, size_t ws_bytes, void* st);

/* ------------------------------------------------------------- packing */

/* Build the packed A from the canonical upper-block list (device, float32):
 * the n(n-1)/2 blocks (i, j), i < j, ordered by i then j, each d x d row-major
 * (block (i, j) at index i*n - i*(i+1)/2 + (j - i - 1)).  `packed` (device,
 * nsrgs_packed_bytes bytes) is fully overwritten.  Model: eq. (4), §2.2. */
nsrgs_status nsrgs_pack_upper(const float* upper, int n, int d, int storage, void* packed, void* st);

/* Same, from the dense symmetric nd x nd float32 matrix A (device, row-major).
 * Only the strict block-upper triangle is read for symmetric layouts; the
 * diagonal blocks are taken to be I_d as in eq. (4). */
nsrgs_status nsrgs_pack_dense(const float* A, int n, int d, int storage, void* packed, void* st);

/* ---------------------------------------------------------- the method */

/* Spectral initialisation (Algorithm 2): X0 (device, nd x d) = sgn_n(Y), Y an
 * orthonormal basis of the eigenvectors of the d largest (algebraic) eigenvalues
 * of A, found by block subspace iteration V <- orth((A_off + cI) V) with float64
 * d x d Gram/Cholesky steps, converged when
 * ||A V - V (V^T A V)||_F / ||V^T A V||_F <= tol.  The shift starts at c = 1
 * (iteration on A itself), which finds the d eigenvalues of largest magnitude.
 * At convergence the basis is accepted when V^T (A_off + cI) V is positive
 * definite: then no eigenvalue left out lies above the captured ones.  Otherwise
 * a negative eigenvalue dominated, and the passes restart from the start vectors
 * with c raised above the negative end of the spectrum (a Gershgorin bound of
 * that d x d matrix), at most 3 times (info flags bit 6).  Restarts count
 * against max_iters; a basis that still fails after the last restart is
 * reported as not converged.  The tensor-core storages (NSRGS_DENSE_BF16, and
 * BF16 / FP8E4M3 at 8 < d <= 64) multiply a rounded V (bfloat16, or E4M3
 * hi + lo planes, about 2^-8 relative), which puts a floor under the residual,
 * typically 1e-4 .. 1e-3: there the passes also count as converged once the
 * residual is at most 1e-2 and no smaller than the previous pass's (info flags
 * bit 7), and the same positive-definiteness test follows.  F32 storage at
 * 8 < d <= 64 (float32 tiles, sums of thousands of float32 products per output)
 * floors near 1e-6 for n d around 10^5 and stops the same way below 1e-4.
 * The per-block matrix sign is exact (float64 one-sided Jacobi SVD).  Returns
 * NSRGS_ERR_NOT_CONVERGED (X0 still written) when max_iters ran out; with
 * `residual` non-null the final residual is written there (host; synchronises). */
nsrgs_status nsrgs_spectral_init(const nsrgs_A* A, float* X0, int max_iters, double tol,
                                 double* residual, void* ws, size_t ws_bytes, void* st);

/* The block product of Algorithm 2's gradient on its own: Y_i = sum_{j != i} A_ij X_j
 * for every i, i.e. Y = A_off X (device, nd x d each, no overlap), streaming the
 * packed A once.  Useful for power/subspace iterations built on this library. */
nsrgs_status nsrgs_product(const nsrgs_A* A, const float* X, float* Y, void* ws, size_t ws_bytes, void* st);

/* One iteration of Algorithm 2 for all blocks: X_out = NS_K(X_in - eta P(G)).
 * X_in and X_out (device, nd x d) must not overlap.  When `upd_norm` (device,
 * one double) is non-null it receives ||X_out - X_in||_F / sqrt(nd). */
nsrgs_status nsrgs_step(const nsrgs_A* A, float eta, int K, const float* X_in, float* X_out,
                        double* upd_norm, void* ws, size_t ws_bytes, void* st);

/* nsrgs_step without a workspace argument, for callers that cannot allocate
 * device memory where they run: e.g. code inside a host program whose memory
 * manager owns the device heap and gives out no scratch buffers, or a
 * latency-critical loop that must not enter an allocator.  The paper has no
 * counterpart; this is a deployment convenience.
 *  - Scratch lives in one fixed 8 MiB (8388608-byte) device array inside the
 *    library; every GPU on which this is called keeps that memory until the
 *    process exits.  (n, d) whose nsrgs_workspace_bytes exceeds 8 MiB is
 *    rejected with NSRGS_ERR_INVALID_ARG: n <= 46016 at d = 3,
 *    n <= 25656 at d = 4, n <= 6025 at d = 8, n <= 931 at d = 16; d >= 32
 *    never fits.
 *  - The first call on a device resolves the array's device address
 *    (cudaGetSymbolAddress) with that device current and caches it; make that
 *    first call before any stream capture, and do not use this entry point
 *    across a cudaDeviceReset of the device (the cached address goes stale).
 *  - No device memory is allocated or freed by any call.
 *  - All calls share the one array: calls that overlap on the GPU (other
 *    streams, other host threads) race and give wrong results; serialise them.
 *    Each call clears the parts that must start at zero.
 *  Arguments, layouts and results are those of nsrgs_step. */
nsrgs_status nsrgs_step_static(const nsrgs_A* A, float eta, int K, const float* X_in, float* X_out,
                               double* upd_norm, void* st);

/* Whole solve (Algorithm 2): when `init` != 0, spectral initialisation into X
 * first (spectral_max_iters passes, tolerance 1e-6); otherwise X holds X^0 on
 * entry.  Then T iterations with step eta and K Newton-Schulz steps; with
 * tol > 0 the loop stops after the first iteration whose update norm
 * ||X^{t+1} - X^t||_F / sqrt(nd) is below tol.  X (device, nd x d) receives the
 * final iterate.  The iteration loop is replayed from a CUDA graph cached per
 * (A, X, workspace, parameters).  `info` (host, nullable) is filled after a
 * synchronisation of `st`.  Returns NSRGS_ERR_NONFINITE if an iterate became
 * non-finite (checked only when info is non-null). */
nsrgs_status nsrgs_solve(const nsrgs_A* A, float eta, int T, int K, double tol, int init,
                         int spectral_max_iters, float* X, nsrgs_info* info, void* ws,
                         size_t ws_bytes, void* st);

/* nsrgs_solve for a packed A and an iterate held in host memory: one call that
 * copies the packed bytes (`packed_host`, `packed_bytes`, laid out as the
 * packers write them: e.g. a host copy of a packed device buffer) into the
 * caller's device buffer A->packed, copies X^0 from X_host into the device
 * buffer X when `init` == 0, runs the solve (Algorithm 2, arguments as
 * nsrgs_solve), copies the final iterate from X to X_host (nd x d float32) and
 * synchronises `st`.  packed_bytes must equal nsrgs_packed_bytes(n, d, storage)
 * for the panel, tile and dense layouts and, for block-sparse rows, the size
 * that the header in packed_host implies (its n and d must match A).  Host
 * buffers in page-locked memory copy asynchronously at the link's rate;
 * pageable ones are staged by the CUDA runtime.  The library keeps no pointer
 * to either host buffer after the call returns.  Errors: NSRGS_ERR_INVALID_ARG
 * for a size or header mismatch or null pointers (nothing is copied), otherwise
 * those of nsrgs_solve; X_host is written only on success. */
nsrgs_status nsrgs_solve_host(const nsrgs_A* A, const void* packed_host, size_t packed_bytes, float eta,
                              int T, int K, double tol, int init, int spectral_max_iters, float* X,
                              float* X_host, nsrgs_info* info, void* ws, size_t ws_bytes, void* st);

/* The least-squares objective of eq. (1) at X (device, nd x d):
 *   F(X) = 1/2 sum_{i != j} ||X_i X_j^T - A_ij||_F^2,
 * with A the stored (packed) matrix.  Evaluated as
 *   1/2 (||X^T X||_F^2 - sum_i ||X_i^T X_i||_F^2) - tr(X^T A_off X) + 1/2 ||A_off||_F^2
 * from one A pass for A_off X, one for ||A_off||_F^2, and float64 sums of the
 * d x d terms.  *F (host) is written after a synchronisation of `st`. */
nsrgs_status nsrgs_objective(const nsrgs_A* A, const float* X, double* F, void* ws, size_t ws_bytes, void* st);

/* Whole solve with the paper's stopping rule (§4.1): as nsrgs_solve, but the
 * loop stops after the first iteration t whose relative decrease
 *   R^t = (F(X^t) - F(X^{t+1})) / F(X^{t+1})
 * is below rel_tol (the paper: 1e-8 with at most 100 iterations), returning
 * X^{t+1}; otherwise after T iterations.  F(X^{t+1}) comes from the product
 * A_off X^{t+1} that the next iteration computes anyway; one extra product
 * follows the last iteration and one pass computes ||A_off||_F^2.  The decrease
 * is evaluated in difference form, tr(X'^T A X') - tr(X^T A X) =
 * tr((X' - X)^T (A X + A X')), so its float32 rounding scales with the update
 * rather than with F.  info->objective = F(X) at the returned X and
 * info->rel_decrease = the last R^t formed.  rel_tol may be any finite value
 * (<= 0: stop only when F does not decrease).  Update-norm fields as nsrgs_solve. */
nsrgs_status nsrgs_solve_objective(const nsrgs_A* A, float eta, int T, int K, double rel_tol, int init,
                                   int spectral_max_iters, float* X, nsrgs_info* info, void* ws,
                                   size_t ws_bytes, void* st);

/* Options of nsrgs_solve_ex.
 *  stop_rule    : NSRGS_STOP_UPDATE_NORM -- stop after the first iteration with
 *                 ||X^{t+1} - X^t||_F / sqrt(nd) < tol (tol = 0: run T iterations),
 *                 as nsrgs_solve; NSRGS_STOP_REL_DECREASE -- the paper's rule
 *                 R^t < tol (§4.1), as nsrgs_solve_objective.
 *  ns_safeguard : nonzero selects a safeguarded Newton-Schulz start, which is not
 *                 part of the paper: a block whose F_i fails Lemma 2.1's
 *                 precondition (checked as ||I - F_i^T F_i||_F >= 1) starts
 *                 Algorithm 1 from F_i / ||F_i||_F, whose singular values lie in
 *                 (0, 1] and whose polar factor is that of F_i.  Blocks that meet
 *                 the precondition are untouched, so where it always holds the
 *                 result is Algorithm 2's.  It keeps large steps on sparse data
 *                 (e.g. the paper's mu = 1/(np) at p = 0.05) finite, where plain
 *                 Newton-Schulz overflows; info->flags bit 4 reports that it acted. */
enum { NSRGS_STOP_UPDATE_NORM = 0, NSRGS_STOP_REL_DECREASE = 1 };
typedef struct nsrgs_solve_opts {
  int stop_rule;
  double tol;
  int ns_safeguard;
} nsrgs_solve_opts;

/* nsrgs_solve / nsrgs_solve_objective with explicit options (opts non-null). */
nsrgs_status nsrgs_solve_ex(const nsrgs_A* A, float eta, int T, int K, const nsrgs_solve_opts* opts, int init,
                            int spectral_max_iters, float* X, nsrgs_info* info, void* ws, size_t ws_bytes,
                            void* st);

/* --------------------------------------------- Stiefel form (extension) */

/* The relaxation of O(d) synchronisation to row-orthonormal blocks X_i in
 * R^{d x p} (X_i X_i^T = I_d, d <= p <= 64): the Stiefel manifold of §1.2 and
 * the extension named in §6; not part of the paper's method.  Same objective
 * (eq. (1)) and the same three steps per iteration, for every block from X^t:
 *   G_i = X_i (X^T X - X_i^T X_i) - sum_{j != i} A_ij X_j
 *   F_i = X_i - eta (G_i - sym(G_i X_i^T) X_i)
 *   X_i^{t+1} = S_K(F_i),  S <- (3I - S S^T) S / 2   (Algorithm 1 by rows).
 * With p = d and X_i orthogonal these are Algorithm 2's steps exactly.  A is
 * NSRGS_DENSE_F32 (any d), or for d > 8 the symmetric tile layouts NSRGS_F32
 * (float32 tiles) and NSRGS_BF16 (tensor-core tiles, X rounded to bfloat16 for
 * the product; p must fall in the same tile-width class as d: both <= 32 or both
 * > 32): the product runs with p columns of X, the tiles read once.  X0 (device,
 * nd x p, row-orthonormal blocks, e.g. [X_i^0, 0] from the O(d) start) is
 * required; X (device, nd x p) receives the last iterate.  tol > 0 stops after
 * the first iteration with ||X^{t+1} - X^t||_F / sqrt(ndp) < tol.  info: iters,
 * last_update_norm, flags (synchronises when non-null). */
size_t nsrgs_stiefel_workspace_bytes(int n, int d, int p);
nsrgs_status nsrgs_stiefel_solve(const nsrgs_A* A, int p, float eta, int T, int K, double tol, const float* X0,
                                 float* X, nsrgs_info* info, void* ws, size_t ws_bytes, void* st);

/* ------------------------------------------------------- SE(d) form
 * Poses (X_i, t_i), X_i in O(d), t_i in R^d: the special Euclidean group that §6
 * names as a target of the Newton-Schulz retraction (the paper writes no method
 * for it; this is the library's reading).  Measurements for pairs i < j: the
 * rotation blocks A_ij ~ X_i X_j^T of the paper's model and translations
 * c_ij ~ X_i (t_j - t_i) (from i to j, in the frame of i); a pair is observed
 * when A_ij has a nonzero entry (unobserved: A_ij = 0, c_ij = 0).  Objective
 *     f(X, t) = F(X) + kappa sum_{i<j observed} ||t_j - t_i - X_i^T c_ij||^2,
 * F of eq. (1).  Each iteration, all nodes at once from (X^t, t^t):
 *     G^X_i = sum_{j != i} (X_i - A_ij X_j) - kappa sum_{j > i} c_ij (t_j - t_i)^T
 *     G^t_i = kappa [deg_i t_i - sum_{j ~ i} t_j - sum_{j < i} X_j^T c_ji + X_i^T sum_{j > i} c_ij]
 *     X_i <- S_K(X_i - eta (G^X_i - X_i G^X_i^T X_i) / 2)   (§2.2, Algorithm 1)
 *     t_i <- t_i - eta_t G^t_i
 * (half the gradient of f, as Algorithm 2's G; the term kappa sum_j c_ij c_ij^T X_i,
 * whose tangent projection vanishes on O(d), is dropped as Algorithm 2 drops
 * X_j^T X_j).  The whole gradient comes from one read of a packed matrix of
 * augmented (d+1) x (d+1) blocks B_ij = [[A_ij, sqrt(kappa) c_ij], [0, w_ij]] in the
 * symmetric layout of that block size (panels up to d + 1 = 8, the float32 or
 * bfloat16 tiles above), multiplied with [[X_j, 0], [sqrt(kappa) t_j^T, 1]].
 * d <= 63 (the node update in registers up to d = 7, a CTA per node above);
 * storage NSRGS_F32 or NSRGS_BF16 (FP8's per-row scale would store the unit
 * weights w_ij inexactly and skew the translations). */

/* Bytes of the packed augmented matrix: nsrgs_packed_bytes(n, d + 1, storage);
 * 0 when (n, d, storage) is outside the form. */
size_t nsrgs_se_packed_bytes(int n, int d, int storage);
/* Workspace bytes of nsrgs_se_solve: nsrgs_workspace_bytes(n, d + 1). */
size_t nsrgs_se_workspace_bytes(int n, int d);
/* Packs the augmented matrix from the canonical upper-block list of A (device,
 * n(n-1)/2 x d x d float32, blocks (i, j) for i < j ordered by i then j) and the
 * matching list of translations c (device, n(n-1)/2 x d float32) into `packed`
 * (device, nsrgs_se_packed_bytes, 16-byte aligned).  kappa >= 0 is folded into
 * the stored blocks (sqrt(kappa) c_ij), so a packed matrix serves one kappa.
 * The result is an nsrgs_A with d + 1 for nsrgs_se_solve. */
nsrgs_status nsrgs_se_pack(const float* upper_a, const float* upper_c, int n, int d, float kappa, int storage,
                           void* packed, void* st);
/* T iterations of the SE(d) form from (X, t) (device: X nd x d, t n x d, both
 * float32, 16-byte aligned), written back in place.  B: an nsrgs_A with
 * B->d = d + 1 describing an nsrgs_se_pack result made with the same kappa.
 * eta > 0 steps the rotations (the paper's 1/n), eta_t >= 0 the translations
 * (1/(kappa n) solves the translation problem of complete noise-free data in
 * one step).  tol > 0 stops after the first iteration with
 * sqrt((||X' - X||_F^2 + ||t' - t||^2) / (nd)) < tol.  X is typically the
 * spectral start of the rotation part (nsrgs_spectral_init on A packed alone)
 * and t zero.  Synchronises `st`; `info` (nullable) receives iters,
 * last_update_norm and flags.  The A stream of each iteration is timed when
 * nsrgs_set_kernel_timing is on.  Errors as nsrgs_solve. */
nsrgs_status nsrgs_se_solve(const nsrgs_A* B, float kappa, float eta, float eta_t, int T, int K, double tol,
                            float* X, float* t, nsrgs_info* info, void* ws, size_t ws_bytes, void* st);

/* ------------------------------------------------------- batched form */

/* One independent instance of a batch. */
typedef struct nsrgs_batch_item {
  const void* packed; /* device, written by nsrgs_pack_* for (n, d, storage) of the batch call */
  int n;
  float eta;          /* step size of this instance */
  float* X;           /* device, nd x d: result; also X^0 on entry when init == 0 */
  int ns_safeguard;   /* nonzero: safeguarded Newton-Schulz start (see nsrgs_solve_opts) */
} nsrgs_batch_item;

/* Workspace bytes for a batch of `count` instances with sizes n[0..count-1] and
 * block size d (1 <= d <= 4); 0 when unsupported. */
size_t nsrgs_batch_workspace_bytes(const int* n, int count, int d);

/* Solves `count` independent instances (Algorithm 2 for each: spectral start
 * when init != 0, then T iterations with K Newton-Schulz steps; tol > 0 stops
 * an instance after its first iteration with update norm below tol) in one
 * CUDA-graph replay or one persistent launch (nsrgs_batch_set_path).  All
 * instances share d (1..4) and the storage (F32, BF16 or FP8E4M3 panels, or
 * BCSR_F32 / BCSR_BF16 block-sparse rows, streamed by a warp-per-row kernel);
 * n and eta differ per instance.  On the tick path each tick is one A-stream
 * launch over every active instance (their steps concatenated and split evenly
 * over the SMs) plus grid-wide launches for the d x d work, so instances in
 * their spectral phase and in their iterations advance in the same tick.  `info` (host array of count, nullable) is filled
 * after a synchronisation.  items, the packed buffers and X must stay valid
 * until the work on `st` completes.  The batched form has no counterpart in
 * the paper beyond running Algorithm 2 on each instance. */
nsrgs_status nsrgs_batch_solve(const nsrgs_batch_item* items, int count, int d, int storage, int T, int K,
                               double tol, int init, int spectral_max_iters, nsrgs_info* info, void* ws,
                               size_t ws_bytes, void* st);

/* How nsrgs_batch_solve runs a batch of panel-stored instances (block-sparse
 * batches always take the tick path):
 *  NSRGS_BATCH_TICKS      : the tick path above -- per tick one A-stream launch over
 *                           every active instance plus grid-wide d x d launches,
 *                           replayed from a CUDA graph;
 *  NSRGS_BATCH_PERSISTENT : one persistent launch (a CTA per SM) in which each CTA
 *                           takes whole instances from a device work counter,
 *                           largest first, and runs each one's spectral start and
 *                           T iterations alone: A passes through the same panel
 *                           pipeline, the d x d work with CTA-local reductions, no
 *                           grid-wide step.  An instance whose panels (stored
 *                           densely with each step's X rows) fit the CTA's stage
 *                           space is loaded into shared memory once and read from
 *                           there on every later pass;
 *  NSRGS_BATCH_AUTO       : (default) the first call for a batch shape (sizes, d,
 *                           storage, T, K, tol, start, pass cap, workspace) runs both
 *                           paths, each a complete solve, times them with CUDA events
 *                           and keeps the faster for later calls of that shape.
 * Both paths compute the same iteration per instance; results agree to the
 * run-to-run spread of the float32 atomic sums.  The setting is process-wide.
 * No counterpart in the paper: these are execution strategies. */
enum { NSRGS_BATCH_AUTO = 0, NSRGS_BATCH_TICKS = 1, NSRGS_BATCH_PERSISTENT = 2 };
nsrgs_status nsrgs_batch_set_path(int path);
/* The path (NSRGS_BATCH_TICKS or NSRGS_BATCH_PERSISTENT) the most recent
 * nsrgs_batch_solve on the calling thread ran with (0 before any call). */
int nsrgs_batch_last_path(void);

/* -------------------------------------------------------- served form */

/* Continuous batching of solves (no counterpart in the paper beyond running
 * Algorithm 2 per request).  A server holds `max_slots` slots and carves every
 * admitted request's packed A and scratch out of a device arena that the
 * caller allocates and keeps alive until nsrgs_server_destroy: admission is by
 * arena (HBM) budget, in arrival order.  Each nsrgs_server_step admits what
 * fits, replays `ticks_per_step` ticks of the batched form over all occupied
 * slots (requests in their spectral phase and in their iterations share each
 * tick), and retires every request that finished (update norm below its
 * tolerance, T_max iterations, or a non-finite iterate); its X is then in the
 * caller's buffer.  A server is used by one host thread at a time. */
typedef struct nsrgs_server nsrgs_server;

typedef struct nsrgs_server_config {
  int d;                   /* block size of every request, 1..4 */
  int storage;             /* NSRGS_F32, NSRGS_BF16 or NSRGS_FP8E4M3 */
  int max_slots;           /* requests in flight at most */
  int K;                   /* Newton-Schulz steps per iteration */
  int spectral_max_iters;  /* subspace-iteration passes cap per request */
  double spectral_tol;     /* subspace residual target (e.g. 1e-6) */
  int ticks_per_step;      /* ticks per nsrgs_server_step call */
  int ns_safeguard;        /* nonzero: safeguarded Newton-Schulz start for every request */
} nsrgs_server_config;

typedef struct nsrgs_server_result {
  uint64_t id;             /* the id nsrgs_server_submit returned */
  int status;              /* NSRGS_OK, NSRGS_ERR_NONFINITE or NSRGS_ERR_TIMEOUT */
  int iters;               /* NS-RGS iterations run */
  int spectral_iters;      /* spectral passes run */
  double last_update_norm; /* ||X^{t+1} - X^t||_F / sqrt(nd) of the last iteration */
  uint32_t flags;          /* as nsrgs_info.flags */
} nsrgs_server_result;

/* Bytes at the start of the arena that the server keeps for its slot table. */
size_t nsrgs_server_table_bytes(int max_slots);

/* Creates a server over `arena` (device, 256-byte aligned, arena_bytes long)
 * working on stream `st`.  *out receives the handle (host object). */
nsrgs_status nsrgs_server_create(const nsrgs_server_config* cfg, void* arena, size_t arena_bytes, void* st,
                                 nsrgs_server** out);

/* Queues a request: `upper` (device, float32 canonical upper-block list of an
 * n-node instance, as for nsrgs_pack_upper) must stay valid until the request
 * is admitted; X (device, nd x d) receives the result.  Iterations stop when
 * the update norm falls below tol (> 0) or after T_max.  NSRGS_ERR_NOMEM when
 * the request could never fit in the arena. */
nsrgs_status nsrgs_server_submit(nsrgs_server* s, const float* upper, int n, float eta, int T_max, double tol,
                                 float* X, uint64_t* id);

/* nsrgs_server_submit for a request stored as block-sparse rows when `sparse` is
 * nonzero (NSRGS_BCSR_F32 for an F32 server, NSRGS_BCSR_BF16 otherwise):
 * packed_bytes is its exact packed size from nsrgs_bcsr_packed_bytes (the
 * admission budget counts it).  With sparse == 0 this is nsrgs_server_submit. */
nsrgs_status nsrgs_server_submit_ex(nsrgs_server* s, const float* upper, int n, float eta, int T_max, double tol,
                                    int sparse, size_t packed_bytes, float* X, uint64_t* id);

/* Admits, runs ticks_per_step ticks, retires; synchronises `st`.  active and
 * queued (nullable) receive the requests in flight and waiting afterwards. */
nsrgs_status nsrgs_server_step(nsrgs_server* s, int* active, int* queued);

/* Moves up to `max` finished results into out (host array); *count receives how many. */
nsrgs_status nsrgs_server_poll(nsrgs_server* s, nsrgs_server_result* out, int max, int* count);

/* Releases the server (not the arena, which the caller owns). */
void nsrgs_server_destroy(nsrgs_server* s);

/* The comparison method of the paper (§1.1, §4.1), the generalised power
 * method, on the same A stream: X_i <- sgn(sum_j A_ij X_j) with A_ii = I, the
 * sign computed exactly per block by a float32 one-sided Jacobi SVD (a thread
 * per block for d <= 8; a CTA per block for 8 < d <= 64, its columns paired
 * round-robin, one warp per pair).  Same start,
 * stop rule, graph replay and info as nsrgs_solve; the paper cites GPM but
 * does not write it out, so this is the reading stated above.  A baseline:
 * NS-RGS replaces exactly this per-block SVD with K Newton-Schulz products. */
nsrgs_status nsrgs_gpm_solve(const nsrgs_A* A, int T, double tol, int init, int spectral_max_iters, float* X,
                             nsrgs_info* info, void* ws, size_t ws_bytes, void* st);

/* d_F(X, Y) = min_{Q in O(d)} ||X - Y Q||_F (§1.4) for two nd x d device stacks,
 * with Q = sgn(Y^T X) from a float64 Jacobi SVD and float64 accumulation.
 * `out` is a host double; the call synchronises `st`. */
nsrgs_status nsrgs_dF(const float* X, const float* Y, int n, int d, double* out, void* ws,
                      size_t ws_bytes, void* st);

/* ------------------------------------------------------ measurement aids */

/* Per-launch timing of the A-stream kernel inside nsrgs_solve.  While enabled
 * (enable != 0), graphs captured by nsrgs_solve carry a CUDA event before and
 * after every A-stream launch of the iteration loop; nsrgs_kernel_timing then
 * reports, for the most recent replay on the calling device, how many such
 * launches ran and their mean duration in milliseconds (it synchronises the
 * device).  The events cost a few microseconds per iteration; the setting is
 * process-wide and part of the graph-cache key.  No counterpart in the paper:
 * this exists to measure the kernel against its memory roofline. */
nsrgs_status nsrgs_set_kernel_timing(int enable);
nsrgs_status nsrgs_kernel_timing(int* launches, double* mean_ms, int* graph_kernel_nodes);

/* Thread-local text of the last error on this thread ("" if none). */
const char* nsrgs_last_error(void);

/* Library version string. */
const char* nsrgs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NSRGS_H */
