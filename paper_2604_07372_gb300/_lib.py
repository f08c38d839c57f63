"""ctypes binding of libnsrgs.so with the ABI's names (include/nsrgs.h).

Arguments are torch tensors on the current CUDA device; the binding passes
their data pointers and ``torch.cuda.current_stream()`` to the C calls and
turns non-zero status codes into ``NsrgsError``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

F32, BF16, FP8E4M3, DENSE_F32, DENSE_BF16, BCSR_F32, BCSR_BF16 = 0, 1, 2, 3, 4, 5, 6
STORAGE = {
    "f32": F32,
    "bf16": BF16,
    "fp8": FP8E4M3,
    "dense_f32": DENSE_F32,
    "dense_bf16": DENSE_BF16,
    "bcsr_f32": BCSR_F32,
    "bcsr_bf16": BCSR_BF16,
}
_STATUS = {
    0: "NSRGS_OK",
    1: "NSRGS_ERR_INVALID_ARG",
    2: "NSRGS_ERR_CUDA",
    3: "NSRGS_ERR_NOMEM",
    4: "NSRGS_ERR_NONFINITE",
    5: "NSRGS_ERR_NS_PRECOND",
    6: "NSRGS_ERR_TIMEOUT",
    7: "NSRGS_ERR_NOT_CONVERGED",
    8: "NSRGS_ERR_UNSUPPORTED",
}

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def lib_path() -> str:
    return os.path.join(_HERE, "libnsrgs.so")


class NsrgsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _A(ctypes.Structure):
    _fields_ = [("packed", ctypes.c_void_p), ("n", ctypes.c_int), ("d", ctypes.c_int), ("storage", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [
        ("spectral_iters", ctypes.c_int),
        ("iters", ctypes.c_int),
        ("last_update_norm", ctypes.c_double),
        ("spectral_residual", ctypes.c_double),
        ("flags", ctypes.c_uint32),
        ("objective", ctypes.c_double),
        ("rel_decrease", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib() -> ctypes.CDLL:
    """Load libnsrgs.so (built by __graft_entry__.build()); raise if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(path)
    vp, i, sz, f, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_float, ctypes.c_double
    Ap = ctypes.POINTER(_A)
    sig = {
        "nsrgs_packed_bytes": (sz, [i, i, i]),
        "nsrgs_workspace_bytes": (sz, [i, i]),
        "nsrgs_bcsr_packed_bytes": (i, [vp, i, i, i, i, ctypes.POINTER(sz), vp, sz, vp]),
        "nsrgs_pack_upper": (i, [vp, i, i, i, vp, vp]),
        "nsrgs_pack_dense": (i, [vp, i, i, i, vp, vp]),
        "nsrgs_spectral_init": (i, [Ap, vp, i, d, ctypes.POINTER(d), vp, sz, vp]),
        "nsrgs_step": (i, [Ap, f, i, vp, vp, vp, vp, sz, vp]),
        "nsrgs_solve": (i, [Ap, f, i, i, d, i, i, vp, ctypes.POINTER(Info), vp, sz, vp]),
        "nsrgs_solve_objective": (i, [Ap, f, i, i, d, i, i, vp, ctypes.POINTER(Info), vp, sz, vp]),
        "nsrgs_solve_host": (i, [Ap, vp, sz, f, i, i, d, i, i, vp, vp, ctypes.POINTER(Info), vp, sz, vp]),
        "nsrgs_se_packed_bytes": (sz, [i, i, i]),
        "nsrgs_se_workspace_bytes": (sz, [i, i]),
        "nsrgs_se_pack": (i, [vp, vp, i, i, f, i, vp, vp]),
        "nsrgs_se_solve": (i, [Ap, f, f, f, i, i, d, vp, vp, ctypes.POINTER(Info), vp, sz, vp]),
        "nsrgs_objective": (i, [Ap, vp, ctypes.POINTER(d), vp, sz, vp]),
        "nsrgs_solve_ex": (i, [Ap, f, i, i, vp, i, i, vp, ctypes.POINTER(Info), vp, sz, vp]),
        "nsrgs_dF": (i, [vp, vp, i, i, ctypes.POINTER(d), vp, sz, vp]),
        "nsrgs_set_kernel_timing": (i, [i]),
        "nsrgs_kernel_timing": (i, [ctypes.POINTER(i), ctypes.POINTER(d), ctypes.POINTER(i)]),
        "nsrgs_last_error": (ctypes.c_char_p, []),
        "nsrgs_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = L
    return L


def _check(status: int) -> None:
    if status != 0:
        raise NsrgsError(status, lib().nsrgs_last_error().decode())


def _stream() -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor | None) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    if not t.is_cuda:
        raise ValueError("tensor must be on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def nsrgs_version() -> str:
    return lib().nsrgs_version().decode()


def nsrgs_packed_bytes(n: int, d: int, storage: int) -> int:
    return int(lib().nsrgs_packed_bytes(n, d, storage))


def nsrgs_workspace_bytes(n: int, d: int) -> int:
    return int(lib().nsrgs_workspace_bytes(n, d))


def workspace(n: int, d: int, device=None) -> torch.Tensor:
    """A device buffer of nsrgs_workspace_bytes(n, d) bytes (torch allocations are 512-byte aligned)."""
    nb = nsrgs_workspace_bytes(n, d)
    if nb == 0:
        raise ValueError("unsupported (n, d)")
    return torch.empty(nb, dtype=torch.uint8, device=device or "cuda")


@dataclass
class PackedA:
    """A packed measurement matrix: the device buffer plus its (n, d, storage)."""

    buf: torch.Tensor
    n: int
    d: int
    storage: int

    def struct(self) -> _A:
        return _A(self.buf.data_ptr(), self.n, self.d, self.storage)

    @property
    def nbytes(self) -> int:
        return self.buf.numel()


def nsrgs_bcsr_packed_bytes(src: torch.Tensor, n: int, d: int, storage: int, dense: bool = False, ws=None) -> int:
    """Exact bytes of a block-sparse packed buffer for this data (counts observed blocks on the device)."""
    w = ws if ws is not None else workspace(n, d, src.device)
    out = ctypes.c_size_t(0)
    _check(lib().nsrgs_bcsr_packed_bytes(_ptr(src), 1 if dense else 0, n, d, storage, ctypes.byref(out), _ptr(w),
                                         w.numel(), _stream()))
    return int(out.value)


def _alloc_packed(n: int, d: int, storage: int, device, src=None, dense=False) -> torch.Tensor:
    if storage in (BCSR_F32, BCSR_BF16) and src is not None and d <= 8:
        nb = nsrgs_bcsr_packed_bytes(src, n, d, storage, dense=dense)
        return torch.empty(nb, dtype=torch.uint8, device=device)
    nb = nsrgs_packed_bytes(n, d, storage)
    if nb == 0:
        raise NsrgsError(8, f"storage {storage} does not support (n={n}, d={d})")
    return torch.empty(nb, dtype=torch.uint8, device=device)


def nsrgs_pack_upper(upper: torch.Tensor, n: int, d: int, storage: int = F32) -> PackedA:
    """Pack the canonical upper-block list (n(n-1)/2, d, d) float32 on the device."""
    assert upper.dtype == torch.float32 and upper.numel() == n * (n - 1) // 2 * d * d
    buf = _alloc_packed(n, d, storage, upper.device, src=upper)
    _check(lib().nsrgs_pack_upper(_ptr(upper), n, d, storage, _ptr(buf), _stream()))
    return PackedA(buf, n, d, storage)


def nsrgs_pack_dense(A: torch.Tensor, n: int, d: int, storage: int = F32) -> PackedA:
    """Pack a dense symmetric (nd, nd) float32 device matrix."""
    assert A.dtype == torch.float32 and A.shape == (n * d, n * d)
    buf = _alloc_packed(n, d, storage, A.device, src=A, dense=True)
    _check(lib().nsrgs_pack_dense(_ptr(A), n, d, storage, _ptr(buf), _stream()))
    return PackedA(buf, n, d, storage)


def _ws(A: PackedA, ws: torch.Tensor | None) -> torch.Tensor:
    return ws if ws is not None else workspace(A.n, A.d, A.buf.device)


def nsrgs_spectral_init(
    A: PackedA, X0: torch.Tensor | None = None, max_iters: int = 50, tol: float = 1e-6, ws=None, strict=True
):
    """Spectral initialisation into X0 (nd, d) float32; returns (X0, residual)."""
    if X0 is None:
        X0 = torch.empty(A.n * A.d, A.d, dtype=torch.float32, device=A.buf.device)
    w = _ws(A, ws)
    res = ctypes.c_double(0.0)
    a = A.struct()
    st = lib().nsrgs_spectral_init(ctypes.byref(a), _ptr(X0), max_iters, tol, ctypes.byref(res), _ptr(w), w.numel(), _stream())
    if st != 7 or strict:
        _check(st)
    return X0, res.value


def nsrgs_step(A: PackedA, eta: float, K: int, X_in: torch.Tensor, X_out: torch.Tensor, upd_norm=None, ws=None):
    """One NS-RGS iteration X_out = NS_K(X_in - eta P(G)); upd_norm: optional device float64 scalar."""
    w = _ws(A, ws)
    a = A.struct()
    _check(
        lib().nsrgs_step(
            ctypes.byref(a), eta, K, _ptr(X_in), _ptr(X_out), _ptr(upd_norm), _ptr(w), w.numel(), _stream()
        )
    )
    return X_out


def nsrgs_solve(
    A: PackedA,
    eta: float,
    T: int,
    K: int,
    tol: float = 0.0,
    init: bool = True,
    spectral_max_iters: int = 50,
    X: torch.Tensor | None = None,
    ws=None,
    info: bool = True,
):
    """Spectral start (init=True) then T iterations; returns (X, Info or None)."""
    if X is None:
        X = torch.empty(A.n * A.d, A.d, dtype=torch.float32, device=A.buf.device)
    w = _ws(A, ws)
    a = A.struct()
    inf = Info() if info else None
    _check(
        lib().nsrgs_solve(
            ctypes.byref(a),
            eta,
            T,
            K,
            tol,
            1 if init else 0,
            spectral_max_iters,
            _ptr(X),
            ctypes.byref(inf) if inf is not None else None,
            _ptr(w),
            w.numel(),
            _stream(),
        )
    )
    return X, inf


def nsrgs_solve_host(
    A: PackedA,
    packed_host: torch.Tensor,
    X_host: torch.Tensor,
    eta: float,
    T: int,
    K: int,
    tol: float = 0.0,
    init: bool = True,
    spectral_max_iters: int = 50,
    X: torch.Tensor | None = None,
    ws=None,
    info: bool = True,
):
    """nsrgs_solve with the packed A and the iterate in host memory: the library
    copies packed_host (uint8, CPU) into A.buf, solves, and writes the final
    iterate into X_host (float32 CPU, nd x d); returns (X_host, Info or None)."""
    for t, name in ((packed_host, "packed_host"), (X_host, "X_host")):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CPU tensor")
    if X_host.dtype != torch.float32 or X_host.numel() != A.n * A.d * A.d:
        raise ValueError("X_host must be float32 with n*d*d elements")
    if X is None:
        X = torch.empty(A.n * A.d, A.d, dtype=torch.float32, device=A.buf.device)
    w = _ws(A, ws)
    a = A.struct()
    inf = Info() if info else None
    _check(
        lib().nsrgs_solve_host(
            ctypes.byref(a),
            ctypes.c_void_p(packed_host.data_ptr()),
            packed_host.numel() * packed_host.element_size(),
            eta,
            T,
            K,
            tol,
            1 if init else 0,
            spectral_max_iters,
            _ptr(X),
            ctypes.c_void_p(X_host.data_ptr()),
            ctypes.byref(inf) if inf is not None else None,
            _ptr(w),
            w.numel(),
            _stream(),
        )
    )
    return X_host, inf


def nsrgs_solve_objective(
    A: PackedA,
    eta: float,
    T: int,
    K: int,
    rel_tol: float = 1e-8,
    init: bool = True,
    spectral_max_iters: int = 50,
    X: torch.Tensor | None = None,
    ws=None,
    info: bool = True,
):
    """Solve with the relative-decrease stopping rule (R^t < rel_tol or T iterations)."""
    if X is None:
        X = torch.empty(A.n * A.d, A.d, dtype=torch.float32, device=A.buf.device)
    w = _ws(A, ws)
    a = A.struct()
    inf = Info() if info else None
    _check(
        lib().nsrgs_solve_objective(
            ctypes.byref(a),
            eta,
            T,
            K,
            rel_tol,
            1 if init else 0,
            spectral_max_iters,
            _ptr(X),
            ctypes.byref(inf) if inf is not None else None,
            _ptr(w),
            w.numel(),
            _stream(),
        )
    )
    return X, inf


STOP_UPDATE_NORM, STOP_REL_DECREASE = 0, 1


class SolveOpts(ctypes.Structure):
    _fields_ = [("stop_rule", ctypes.c_int), ("tol", ctypes.c_double), ("ns_safeguard", ctypes.c_int)]


def nsrgs_solve_ex(
    A: PackedA,
    eta: float,
    T: int,
    K: int,
    stop_rule: int = STOP_UPDATE_NORM,
    tol: float = 0.0,
    ns_safeguard: bool = False,
    init: bool = True,
    spectral_max_iters: int = 50,
    X: torch.Tensor | None = None,
    ws=None,
    info: bool = True,
):
    """nsrgs_solve / nsrgs_solve_objective with explicit options; returns (X, Info or None)."""
    if X is None:
        X = torch.empty(A.n * A.d, A.d, dtype=torch.float32, device=A.buf.device)
    w = _ws(A, ws)
    a = A.struct()
    opts = SolveOpts(stop_rule, tol, 1 if ns_safeguard else 0)
    inf = Info() if info else None
    _check(
        lib().nsrgs_solve_ex(
            ctypes.byref(a),
            eta,
            T,
            K,
            ctypes.byref(opts),
            1 if init else 0,
            spectral_max_iters,
            _ptr(X),
            ctypes.byref(inf) if inf is not None else None,
            _ptr(w),
            w.numel(),
            _stream(),
        )
    )
    return X, inf


def nsrgs_stiefel_solve(A: PackedA, p: int, eta: float, T: int, K: int, X0: torch.Tensor, tol: float = 0.0,
                        X: torch.Tensor | None = None, info: bool = True):
    """Stiefel form (d x p row-orthonormal blocks) from X0 (nd x p); returns (X, Info or None)."""
    L = lib()
    fn = L.nsrgs_stiefel_solve
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(_A), ctypes.c_int, ctypes.c_float, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(Info), ctypes.c_void_p, ctypes.c_size_t,
                   ctypes.c_void_p]
    wb = L.nsrgs_stiefel_workspace_bytes
    wb.restype = ctypes.c_size_t
    wb.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    nbytes = int(wb(A.n, A.d, p))
    if nbytes == 0:
        raise ValueError("unsupported (n, d, p)")
    w = torch.empty(nbytes, dtype=torch.uint8, device=A.buf.device)
    if X is None:
        X = torch.empty(A.n * A.d, p, dtype=torch.float32, device=A.buf.device)
    a = A.struct()
    inf = Info() if info else None
    _check(fn(ctypes.byref(a), p, eta, T, K, tol, _ptr(X0), _ptr(X), ctypes.byref(inf) if inf is not None else None,
              _ptr(w), w.numel(), _stream()))
    return X, inf


def nsrgs_se_pack(upper_a: torch.Tensor, upper_c: torch.Tensor, n: int, d: int, kappa: float,
                  storage: int = F32) -> PackedA:
    """Pack the SE(d) form's augmented matrix from the upper-block lists of A
    ((n(n-1)/2, d, d) float32) and c ((n(n-1)/2, d) float32) on the device; the
    result describes (d + 1)-blocks for nsrgs_se_solve."""
    assert upper_a.dtype == torch.float32 and upper_a.numel() == n * (n - 1) // 2 * d * d
    assert upper_c.dtype == torch.float32 and upper_c.numel() == n * (n - 1) // 2 * d
    nb = int(lib().nsrgs_se_packed_bytes(n, d, storage))
    if nb == 0:
        raise NsrgsError(8, f"the SE(d) form does not support (n={n}, d={d}, storage={storage})")
    buf = torch.empty(nb, dtype=torch.uint8, device=upper_a.device)
    _check(lib().nsrgs_se_pack(_ptr(upper_a.contiguous()), _ptr(upper_c.contiguous()), n, d, kappa, storage,
                               _ptr(buf), _stream()))
    return PackedA(buf, n, d + 1, storage)


def nsrgs_se_solve(B: PackedA, kappa: float, eta: float, eta_t: float, T: int, K: int, X: torch.Tensor,
                   t: torch.Tensor, tol: float = 0.0, ws=None, info: bool = True):
    """T iterations of the SE(d) form from (X (nd x d), t (n x d)), updated in place;
    B from nsrgs_se_pack with the same kappa.  Returns (X, t, Info or None)."""
    n, d = B.n, B.d - 1
    if ws is None:
        ws = torch.empty(int(lib().nsrgs_se_workspace_bytes(n, d)), dtype=torch.uint8, device=B.buf.device)
    a = B.struct()
    inf = Info() if info else None
    _check(lib().nsrgs_se_solve(ctypes.byref(a), kappa, eta, eta_t, T, K, tol, _ptr(X), _ptr(t),
                                ctypes.byref(inf) if inf is not None else None, _ptr(ws), ws.numel(), _stream()))
    return X, t, inf


def nsrgs_objective(A: PackedA, X: torch.Tensor, ws=None) -> float:
    """F(X) of eq. (1) for the stored A."""
    w = _ws(A, ws)
    a = A.struct()
    out = ctypes.c_double(0.0)
    _check(lib().nsrgs_objective(ctypes.byref(a), _ptr(X), ctypes.byref(out), _ptr(w), w.numel(), _stream()))
    return out.value


def nsrgs_dF(X: torch.Tensor, Y: torch.Tensor, n: int, d: int, ws=None) -> float:
    """d_F(X, Y) = min over O(d) of ||X - Y Q||_F, float64 on the device."""
    w = ws if ws is not None else workspace(n, d, X.device)
    out = ctypes.c_double(0.0)
    _check(lib().nsrgs_dF(_ptr(X), _ptr(Y), n, d, ctypes.byref(out), _ptr(w), w.numel(), _stream()))
    return out.value


def nsrgs_set_kernel_timing(enable: bool) -> None:
    _check(lib().nsrgs_set_kernel_timing(1 if enable else 0))


def nsrgs_kernel_timing() -> tuple[int, float, int]:
    """(A-stream launches timed in the last solve replay, their mean ms, kernel nodes of that graph)."""
    n = ctypes.c_int(0)
    ms = ctypes.c_double(0.0)
    k = ctypes.c_int(0)
    _check(lib().nsrgs_kernel_timing(ctypes.byref(n), ctypes.byref(ms), ctypes.byref(k)))
    return n.value, ms.value, k.value


def nsrgs_step_static(A: PackedA, eta: float, K: int, X_in: torch.Tensor, X_out: torch.Tensor, upd_norm=None):
    """nsrgs_step with the library's fixed 8 MiB scratch array instead of a workspace (no allocation)."""
    L = lib()
    fn = L.nsrgs_step_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(_A), ctypes.c_float, ctypes.c_int] + [ctypes.c_void_p] * 4
    a = A.struct()
    _check(fn(ctypes.byref(a), eta, K, _ptr(X_in), _ptr(X_out), _ptr(upd_norm), _stream()))
    return X_out


class _BatchItem(ctypes.Structure):
    _fields_ = [
        ("packed", ctypes.c_void_p),
        ("n", ctypes.c_int),
        ("eta", ctypes.c_float),
        ("X", ctypes.c_void_p),
        ("ns_safeguard", ctypes.c_int),
    ]


def nsrgs_batch_workspace_bytes(ns, d: int) -> int:
    arr = (ctypes.c_int * len(ns))(*ns)
    fn = lib().nsrgs_batch_workspace_bytes
    fn.restype = ctypes.c_size_t
    fn.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int]
    return int(fn(arr, len(ns), d))


def nsrgs_batch_solve(
    packs,
    etas,
    T: int,
    K: int,
    tol: float = 0.0,
    init: bool = True,
    spectral_max_iters: int = 50,
    Xs=None,
    ws=None,
    info: bool = True,
    ns_safeguard: bool = False,
):
    """Solve a batch of PackedA instances (same d and storage); returns (list of X, list of Info or None)."""
    count = len(packs)
    d = packs[0].d
    storage = packs[0].storage
    if Xs is None:
        Xs = [torch.empty(p.n * d, d, dtype=torch.float32, device=p.buf.device) for p in packs]
    items = (_BatchItem * count)()
    for k, (p, e, X) in enumerate(zip(packs, etas, Xs)):
        assert p.d == d and p.storage == storage
        items[k] = _BatchItem(p.buf.data_ptr(), p.n, float(e), X.data_ptr(), 1 if ns_safeguard else 0)
    if ws is None:
        ws = torch.empty(nsrgs_batch_workspace_bytes([p.n for p in packs], d), dtype=torch.uint8, device=packs[0].buf.device)
    infos = (Info * count)() if info else None
    fn = lib().nsrgs_batch_solve
    fn.restype = ctypes.c_int
    fn.argtypes = [
        ctypes.POINTER(_BatchItem), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
        ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Info), ctypes.c_void_p, ctypes.c_size_t,
        ctypes.c_void_p,
    ]
    _check(
        fn(items, count, d, storage, T, K, tol, 1 if init else 0, spectral_max_iters, infos, _ptr(ws), ws.numel(), _stream())
    )
    return Xs, (list(infos) if infos is not None else None)


BATCH_AUTO, BATCH_TICKS, BATCH_PERSISTENT = 0, 1, 2


def nsrgs_batch_set_path(path: int) -> None:
    """Path of nsrgs_batch_solve: BATCH_AUTO (timed once per batch shape), BATCH_TICKS, BATCH_PERSISTENT."""
    fn = lib().nsrgs_batch_set_path
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int]
    _check(fn(path))


def nsrgs_batch_last_path() -> int:
    """The path the most recent nsrgs_batch_solve on this thread ran with."""
    fn = lib().nsrgs_batch_last_path
    fn.restype = ctypes.c_int
    fn.argtypes = []
    return int(fn())


class _ServerConfig(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int),
        ("storage", ctypes.c_int),
        ("max_slots", ctypes.c_int),
        ("K", ctypes.c_int),
        ("spectral_max_iters", ctypes.c_int),
        ("spectral_tol", ctypes.c_double),
        ("ticks_per_step", ctypes.c_int),
        ("ns_safeguard", ctypes.c_int),
    ]


class ServerResult(ctypes.Structure):
    _fields_ = [
        ("id", ctypes.c_uint64),
        ("status", ctypes.c_int),
        ("iters", ctypes.c_int),
        ("spectral_iters", ctypes.c_int),
        ("last_update_norm", ctypes.c_double),
        ("flags", ctypes.c_uint32),
    ]


class Server:
    """nsrgs_server_* over a caller-owned device arena (a torch uint8 tensor)."""

    def __init__(self, d: int, storage: int, max_slots: int, arena_bytes: int, K: int = 2,
                 spectral_max_iters: int = 60, spectral_tol: float = 1e-6, ticks_per_step: int = 4, device=None,
                 ns_safeguard: bool = False):
        L = lib()
        for name, res, args in [
            ("nsrgs_server_table_bytes", ctypes.c_size_t, [ctypes.c_int]),
            ("nsrgs_server_create", ctypes.c_int, [ctypes.POINTER(_ServerConfig), ctypes.c_void_p, ctypes.c_size_t,
                                                   ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
            ("nsrgs_server_submit", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_float,
                                                   ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                                   ctypes.POINTER(ctypes.c_uint64)]),
            ("nsrgs_server_submit_ex", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_float,
                                                      ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_size_t,
                                                      ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
            ("nsrgs_server_step", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
            ("nsrgs_server_poll", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ServerResult), ctypes.c_int,
                                                 ctypes.POINTER(ctypes.c_int)]),
            ("nsrgs_server_destroy", None, [ctypes.c_void_p]),
        ]:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        self._L = L
        self.d = d
        self.arena = torch.empty(arena_bytes, dtype=torch.uint8, device=device or "cuda")
        self._keep = {}
        cfg = _ServerConfig(d, storage, max_slots, K, spectral_max_iters, spectral_tol, ticks_per_step,
                            1 if ns_safeguard else 0)
        self.sparse_storage = BCSR_F32 if storage == F32 else BCSR_BF16
        h = ctypes.c_void_p(0)
        _check(L.nsrgs_server_create(ctypes.byref(cfg), _ptr(self.arena), self.arena.numel(), _stream(), ctypes.byref(h)))
        self._h = h

    def submit(self, upper: torch.Tensor, n: int, eta: float, T_max: int, tol: float, X: torch.Tensor,
               sparse: bool = False, packed_bytes: int = 0) -> int:
        """Queue a request; sparse=True stores it as block-sparse rows (packed_bytes from
        nsrgs_bcsr_packed_bytes with the server's sparse storage, see sparse_storage)."""
        rid = ctypes.c_uint64(0)
        _check(self._L.nsrgs_server_submit_ex(self._h, _ptr(upper), n, eta, T_max, tol, 1 if sparse else 0,
                                              packed_bytes, _ptr(X), ctypes.byref(rid)))
        self._keep[rid.value] = (upper, X)
        return rid.value

    def step(self) -> tuple[int, int]:
        a, q = ctypes.c_int(0), ctypes.c_int(0)
        _check(self._L.nsrgs_server_step(self._h, ctypes.byref(a), ctypes.byref(q)))
        return a.value, q.value

    def poll(self, max_results: int = 4096) -> list[ServerResult]:
        out = (ServerResult * max_results)()
        c = ctypes.c_int(0)
        _check(self._L.nsrgs_server_poll(self._h, out, max_results, ctypes.byref(c)))
        res = [out[i] for i in range(c.value)]
        for r in res:
            self._keep.pop(r.id, None)
        return res

    def close(self):
        if self._h:
            self._L.nsrgs_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nsrgs_product(A: PackedA, X: torch.Tensor, Y: torch.Tensor | None = None, ws=None) -> torch.Tensor:
    """Y = A_off X (Y_i = sum_{j != i} A_ij X_j), streaming the packed A once."""
    if Y is None:
        Y = torch.empty_like(X)
    w = _ws(A, ws)
    fn = lib().nsrgs_product
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(_A), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    a = A.struct()
    _check(fn(ctypes.byref(a), _ptr(X), _ptr(Y), _ptr(w), w.numel(), _stream()))
    return Y


def nsrgs_gpm_solve(A: PackedA, T: int, tol: float = 0.0, init: bool = True, spectral_max_iters: int = 50,
                    X: torch.Tensor | None = None, ws=None, info: bool = True):
    """Generalised power method baseline on the same A stream; returns (X, Info or None)."""
    if X is None:
        X = torch.empty(A.n * A.d, A.d, dtype=torch.float32, device=A.buf.device)
    w = _ws(A, ws)
    a = A.struct()
    inf = Info() if info else None
    fn = lib().nsrgs_gpm_solve
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(_A), ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                   ctypes.POINTER(Info), ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    _check(fn(ctypes.byref(a), T, tol, 1 if init else 0, spectral_max_iters, _ptr(X),
              ctypes.byref(inf) if inf is not None else None, _ptr(w), w.numel(), _stream()))
    return X, inf
