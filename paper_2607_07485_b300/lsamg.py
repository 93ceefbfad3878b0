"""Thin ctypes binding over the C ABI of liblsamg (include/lsamg.h).

Argument marshalling only: every step of set-up and solve runs in the library's CUDA
kernels.  PyTorch supplies device memory and the stream.  Importing this module fails
loudly if the compiled library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblsamg.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"liblsamg.so not built ({LIB_PATH}); run python -m paper_2607_07485_b300.build")
_lib = C.CDLL(LIB_PATH)

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "NOT_SPSD", 3: "SINGULAR", 4: "NO_CONVERGENCE", 5: "CUDA",
          6: "OOM", 7: "DEVICE_TIMEOUT", 8: "NAN", 9: "LIMIT"}

Q = dict(AGG=0, MULT=1, OMEGA_PTR=2, OMEGA_IDX=3, K=4, ZOFF=5, Z=6, CELEM_PTR=7, CELEM_IDX=8,
         GOFF=9, GROWS=10, G=11, COLOUR=12, EPTR=13, EIDX=14, MU=15, CGROUP=16)
_QTYPE = {0: np.int32, 1: np.int32, 2: np.int64, 3: np.int32, 4: np.int32, 5: np.int64, 6: np.float64,
          7: np.int64, 8: np.int32, 9: np.int64, 10: np.int32, 11: np.float64, 12: np.int32,
          13: np.int64, 14: np.int32, 15: np.float64, 16: np.int32}


class LsamgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lsamg error {code} ({STATUS.get(code, '?')}): {msg}")
        self.code = code


class Problem(C.Structure):
    _fields_ = [("n_dofs", C.c_int64), ("n_elems", C.c_int64), ("n_T", C.c_int32),
                ("on_host", C.c_int32), ("elem_dofs", C.c_void_p), ("elem_mats", C.c_void_p),
                ("elem_coef", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("tau_c", C.c_double), ("agg_passes", C.c_int32), ("agg_passes_coarse", C.c_int32),
                ("max_levels", C.c_int32), ("min_coarse", C.c_int32), ("max_density", C.c_double),
                ("vcycle_fp32", C.c_int32), ("maxit", C.c_int32), ("rtol", C.c_double),
                ("chunk_bytes", C.c_int64), ("use_graph", C.c_int32), ("verbose", C.c_int32),
                ("profile", C.c_int32), ("large_dense", C.c_int32), ("split_sweep", C.c_int32),
                ("sweep_block", C.c_int32), ("smoother", C.c_int32), ("closure", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("n", C.c_int64 * 8), ("nnz", C.c_int64 * 8),
                ("n_elems", C.c_int64 * 8), ("n_agg", C.c_int32 * 8), ("n_colours", C.c_int32 * 8),
                ("tau", C.c_double * 8), ("min_gap", C.c_double * 8), ("op_complexity", C.c_double),
                ("grid_complexity", C.c_double), ("setup_seconds", C.c_double),
                ("stage_seconds", C.c_double * 16), ("setup_flops", C.c_double)]


_H = C.c_void_p
_lib.lsamg_options_default.restype = Options
_lib.lsamg_setup.argtypes = [C.POINTER(Problem), C.POINTER(Options), C.c_void_p, C.POINTER(_H)]
_lib.lsamg_apply.argtypes = [_H, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]
_lib.lsamg_solve.argtypes = [_H, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                             C.c_void_p, C.c_void_p]
_lib.lsamg_solve_host.argtypes = [_H, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                  C.c_void_p, C.c_void_p]
_lib.lsamg_gram_spmv.argtypes = [_H, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]
_lib.lsamg_elem_grad.argtypes = [_H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
_lib.lsamg_get_stats.argtypes = [_H, C.POINTER(Stats)]
_lib.lsamg_stage_name.restype = C.c_char_p
_lib.lsamg_stage_name.argtypes = [C.c_int32]
_lib.lsamg_query.argtypes = [_H, C.c_int32, C.c_int32, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]
_lib.lsamg_destroy.argtypes = [_H]
_lib.lsamg_gram_spmv_static.argtypes = [C.c_int64, C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_void_p]
_lib.lsamg_dgemm_nt.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_double, C.c_void_p, C.c_int64, C.c_void_p,
                                C.c_int64, C.c_double, C.c_void_p, C.c_int64, C.c_void_p]
_lib.lsamg_last_error.restype = C.c_char_p
_lib.lsamg_kernel_classes.restype = C.c_int32
_lib.lsamg_kernel_name.restype = C.c_char_p
_lib.lsamg_kernel_name.argtypes = [C.c_int32]
_lib.lsamg_kernel_stats_all.argtypes = [C.c_void_p]
_lib.lsamg_launch_count.restype = C.c_int64

EXPORTS = ["lsamg_options_default", "lsamg_setup", "lsamg_apply", "lsamg_solve", "lsamg_solve_host",
           "lsamg_gram_spmv", "lsamg_elem_grad", "lsamg_get_stats", "lsamg_stage_name", "lsamg_query",
           "lsamg_destroy", "lsamg_last_error", "lsamg_kernel_classes", "lsamg_kernel_name",
           "lsamg_kernel_stats_all", "lsamg_launch_count", "lsamg_gram_spmv_static", "lsamg_dgemm_nt"]


def kernel_stats():
    """Per-kernel-class device time since the previous call (needs the profile option)."""
    k = _lib.lsamg_kernel_classes()
    buf = np.zeros(4 * k, np.float64)
    _check(_lib.lsamg_kernel_stats_all(buf.ctypes.data))
    out = {}
    for c in range(k):
        ms, calls, fl, by = buf[4 * c:4 * c + 4]
        if calls:
            out[_lib.lsamg_kernel_name(c).decode()] = dict(ms=ms, calls=int(calls), flops=fl, bytes=by)
    return out


def _check_static_args(elem_dofs, G, x, y):
    """Reject every input the allocation-free Gram SpMV cannot take safely.  The C entry point
    only sees raw pointers, so a wrong dtype, a strided view, a short output or a tensor on
    another device would make its kernels read or write past the buffers; it must not copy or
    convert either (that would allocate), so it refuses instead.  Raises ValueError."""
    import torch
    for name, t, dt in (("elem_dofs", elem_dofs, torch.int32), ("G", G, torch.float64),
                        ("x", x, torch.float64), ("y", y, torch.float64)):
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if elem_dofs.dim() != 2:
        raise ValueError("elem_dofs must be 2-D [n_elems, n_T]")
    ne, nT = elem_dofs.shape
    if nT < 1:
        raise ValueError("elem_dofs must have n_T >= 1 columns")
    if G.dim() != 3 or G.shape[0] != ne or G.shape[2] != nT:
        raise ValueError(f"G must be [n_elems={ne}, m, n_T={nT}], got {tuple(G.shape)}")
    if x.dim() != 1 or y.dim() != 1 or y.numel() != x.numel():
        raise ValueError("x and y must be 1-D with the same length")
    if not torch.cuda.is_available():
        raise ValueError("the tensors must be CUDA tensors (no CUDA device is available)")
    cur = torch.cuda.current_device()
    for name, t in (("elem_dofs", elem_dofs), ("G", G), ("x", x), ("y", y)):
        if not t.is_cuda or t.device.index != cur:
            raise ValueError(f"{name} must be on the current CUDA device cuda:{cur}, got {t.device}")


def gram_spmv_static(elem_dofs, G, x, y, stream=None):
    """y = sum_T R_T^T G_T^T (G_T x_T) through the allocation-free entry point (no handle), for
    callers that cannot allocate device memory (GPU memory owned by another allocator, or a
    latency-critical loop where cudaMalloc would synchronise the device).
    elem_dofs: int32 [ne, nT], G: float64 [ne, m, nT], x, y: float64 [n], all contiguous on the
    current CUDA device (y is overwritten; nothing is allocated here or in the library; any
    other input raises ValueError before the library is called).  The call synchronises its
    stream, so it cannot be recorded into a CUDA graph; on a capturing stream it is refused."""
    _check_static_args(elem_dofs, G, x, y)
    ne, nT = elem_dofs.shape
    m = G.shape[1]
    _check(_lib.lsamg_gram_spmv_static(int(x.numel()), int(ne), int(nT), int(m), _ptr(elem_dofs), _ptr(G),
                                       _ptr(x), _ptr(y), _stream(stream)))
    return y


def dgemm_nt(A, B, C=None, alpha=1.0, beta=0.0, stream=None):
    """C = alpha A B^T + beta C in FP64 on the tensor cores (lsamg_dgemm_nt).  A: [M, K], B: [N, K],
    C: [M, N] float64 CUDA tensors (row-major torch layout; transposed copies give the library its
    column-major operands)."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    At = A.t().contiguous()
    Bt = B.t().contiguous()
    Ct = (torch.zeros(N, M, dtype=torch.float64, device=A.device) if C is None else C.t().contiguous())
    _check(_lib.lsamg_dgemm_nt(M, N, K, float(alpha), _ptr(At), max(M, 1), _ptr(Bt), max(N, 1), float(beta), _ptr(Ct),
                               max(M, 1), _stream(stream)))
    return Ct.t()


def launch_count():
    return int(_lib.lsamg_launch_count())


def _check(rc, allow=()):
    if rc != 0 and rc not in allow:
        raise LsamgError(rc, _lib.lsamg_last_error().decode())
    return rc


def options(**kw) -> Options:
    o = _lib.lsamg_options_default()
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        if k == "closure" and isinstance(v, str):
            if v not in ("G", "A"):
                raise ValueError(f"closure must be 'G' or 'A', not {v!r}")
            v = 0 if v == "G" else 1
        setattr(o, k, v)
    return o


def _stream(stream):
    if stream is not None:
        return C.c_void_p(stream)
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


class Lsamg:
    """An LS-AMG-DD hierarchy built on the GPU from element DOF maps and element matrices.

    elem_dofs: [ne, nT] int32, elem_mats: [ne, nT, nT] float64, coef: [ne] float64 or None
    (A_T = coef_e * elem_mats_e).  Either all CUDA torch tensors (device path) or all numpy
    arrays (host path, copied in by the library)."""

    def __init__(self, n_dofs, elem_dofs, elem_mats, coef=None, stream=None, **opts):
        self._h = _H()
        self.n = int(n_dofs)
        self.ne = int(elem_dofs.shape[0])
        self.nT = int(elem_dofs.shape[1])
        on_host = isinstance(elem_dofs, np.ndarray)
        self._keep = []
        if on_host:
            d = np.ascontiguousarray(elem_dofs, dtype=np.int32)
            m = np.ascontiguousarray(elem_mats, dtype=np.float64)
            c = None if coef is None else np.ascontiguousarray(coef, dtype=np.float64)
            self._keep = [d, m, c]
            p = Problem(self.n, self.ne, self.nT, 1, d.ctypes.data, m.ctypes.data,
                        None if c is None else c.ctypes.data)
            st = C.c_void_p(stream) if stream is not None else C.c_void_p(0)
        else:
            import torch
            d = elem_dofs.to(torch.int32).contiguous()
            m = elem_mats.to(torch.float64).contiguous()
            c = None if coef is None else coef.to(torch.float64).contiguous()
            self._keep = [d, m, c]
            p = Problem(self.n, self.ne, self.nT, 0, d.data_ptr(), m.data_ptr(),
                        None if c is None else c.data_ptr())
            st = _stream(stream)
        self.opts = options(**opts)
        _check(_lib.lsamg_setup(C.byref(p), C.byref(self.opts), st, C.byref(self._h)))
        self._keep = []

    # ------------------------------------------------------------------ solve-phase calls
    def apply(self, r, fp32=-1, stream=None):
        """z = B^{-1} r (one V-cycle); r: CUDA float64 [n] or [nrhs, n]."""
        import torch
        z = torch.empty_like(r)
        nrhs = 1 if r.dim() == 1 else r.shape[0]
        _check(_lib.lsamg_apply(self._h, _ptr(r.contiguous()), _ptr(z), nrhs, fp32, _stream(stream)))
        return z

    def solve(self, b, x0=None, mode=-1, stream=None, raise_on_noconv=False):
        """Solve A x = b; returns (x, iters[nrhs], relres[nrhs], status)."""
        import torch
        b = b.contiguous()
        nrhs = 1 if b.dim() == 1 else b.shape[0]
        x = torch.zeros_like(b) if x0 is None else x0.clone().contiguous()
        its = np.zeros(nrhs, np.int32)
        rel = np.zeros(nrhs, np.float64)
        rc = _lib.lsamg_solve(self._h, _ptr(b), _ptr(x), nrhs, mode, 0 if x0 is None else 1, _stream(stream),
                              its.ctypes.data, rel.ctypes.data)
        _check(rc, allow=() if raise_on_noconv else (4,))
        return x, its, rel, rc

    def solve_host(self, b, mode=-1, stream=None):
        """Solve with host numpy arrays (copies inside the call)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        nrhs = 1 if b.ndim == 1 else b.shape[0]
        x = np.empty_like(b)
        its = np.zeros(nrhs, np.int32)
        rel = np.zeros(nrhs, np.float64)
        rc = _lib.lsamg_solve_host(self._h, b.ctypes.data, x.ctypes.data, nrhs, mode,
                                   C.c_void_p(stream) if stream is not None else C.c_void_p(0),
                                   its.ctypes.data, rel.ctypes.data)
        _check(rc, allow=(4,))
        return x, its, rel, rc

    def gram_spmv(self, x, level=0, fp32=False, stream=None):
        import torch
        y = torch.empty_like(x)
        _check(_lib.lsamg_gram_spmv(self._h, level, _ptr(x.contiguous()), _ptr(y), 1 if fp32 else 0,
                                    _stream(stream)))
        return y

    def elem_grad(self, lam, x, stream=None):
        import torch
        g = torch.empty(self.ne, dtype=torch.float64, device=x.device)
        _check(_lib.lsamg_elem_grad(self._h, _ptr(lam.contiguous()), _ptr(x.contiguous()), _ptr(g),
                                    _stream(stream)))
        return g

    # ------------------------------------------------------------------ introspection
    def stats(self):
        s = Stats()
        _check(_lib.lsamg_get_stats(self._h, C.byref(s)))
        L = s.n_levels
        return dict(n_levels=L, n=list(s.n[:L]), nnz=list(s.nnz[:L]), n_elems=list(s.n_elems[:L]),
                    n_agg=list(s.n_agg[:L]), n_colours=list(s.n_colours[:L]), tau=list(s.tau[:L]),
                    min_gap=list(s.min_gap[:L]), OC=s.op_complexity, GC=s.grid_complexity,
                    setup_seconds=s.setup_seconds, setup_flops=s.setup_flops,
                    stages={_lib.lsamg_stage_name(i).decode(): s.stage_seconds[i] for i in range(9)})

    def query(self, level, what):
        w = Q[what] if isinstance(what, str) else what
        need = C.c_int64(0)
        _check(_lib.lsamg_query(self._h, level, w, None, 0, C.byref(need)))
        dt = _QTYPE[w]
        out = np.empty(need.value // np.dtype(dt).itemsize, dt)
        if need.value:
            _check(_lib.lsamg_query(self._h, level, w, out.ctypes.data, need.value, C.byref(need)))
        return out

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.lsamg_destroy(self._h)
            self._h = _H()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
