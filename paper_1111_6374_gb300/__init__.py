"""Python binding of ``libgsyeig.so`` (C ABI in ``include/gsyeig.h``).

Argument marshalling only: every step of the eigen-solve runs in the
library's CUDA kernels.  PyTorch supplies device memory and streams.  If
the compiled library is missing (and cannot be built) every entry point
raises; there is no CPU path.

Layout: the library is column-major.  A torch tensor ``M`` is passed as a
column-major matrix when ``M.stride(0) == 1`` (leading dimension
``M.stride(1)``); a row-major contiguous square tensor is accepted for the
symmetric inputs A, B, C (whose two layouts coincide).  Outputs are
returned as column-major views (``colmajor_empty``).
"""
from __future__ import annotations

import ctypes
import os

import torch

from .build import LIB, build as _build_lib

__all__ = ["Solver", "load", "colmajor", "colmajor_empty", "Info", "GsyeigError", "kernel_launches",
           "tridiag_eig_noalloc"]

SMALLEST, LARGEST = 0, 1
_STATUS = {1: "NOT_SPD", 2: "NO_CONVERGENCE", 3: "TIMEOUT", 4: "CUDA_ERROR", 5: "OOM", 6: "NOT_SUPPORTED",
           7: "SCRATCH_TOO_SMALL"}


class GsyeigError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"gsyeig status {status} ({_STATUS.get(status, 'invalid argument')}): {msg}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("krylov_dim", ctypes.c_int64), ("keep", ctypes.c_int64),
                ("max_restarts", ctypes.c_int64), ("seed", ctypes.c_uint64), ("v0", ctypes.c_void_p),
                ("timeout_ms", ctypes.c_double), ("block", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("fp64_gemm", ctypes.c_int32), ("fp64_symv", ctypes.c_int32),
                ("qr_restart", ctypes.c_int32), ("inverse", ctypes.c_int32),
                ("preserve_inputs", ctypes.c_int32), ("verify", ctypes.c_int32), ("implicit", ctypes.c_int32),
                ("wait_limit", ctypes.c_int32), ("start_block", ctypes.c_void_p), ("start_weights", ctypes.c_void_p),
                ("start_cols", ctypes.c_int64), ("ld_start", ctypes.c_int64), ("filter_cut", ctypes.c_double),
                ("filter_edge", ctypes.c_double), ("filter_degree", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("mixed", ctypes.c_int32), ("graph", ctypes.c_int32), ("max_ctas", ctypes.c_int32),
                ("block_start", ctypes.c_int32), ("shift", ctypes.c_double)]


class Problem(ctypes.Structure):
    """gsyeig_problem: one problem of a batch (device pointers)."""
    _fields_ = [("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64),
                ("n", ctypes.c_int64), ("s", ctypes.c_int64), ("which", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("w", ctypes.c_void_p), ("X", ctypes.c_void_p), ("ldx", ctypes.c_int64)]


class Info(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("n", "s", "nconv", "restarts", "matvecs", "krylov_dim", "keep",
                                               "potrf_index", "breakdowns", "kernel_launches")] + \
               [(f, ctypes.c_double) for f in ("ms_gs1", "ms_gs2", "ms_ke", "ms_ke3", "ms_bt1", "ms_total",
                                                "max_ritz_estimate")] + \
               [(f, ctypes.c_int64) for f in ("gemm_launches", "symv_launches")] + \
               [(f, ctypes.c_double) for f in ("gemm_ms", "gemm_flops", "gemm_bytes", "symv_ms", "symv_flops",
                                                "symv_bytes", "orth_ms", "restart_ms", "ritz_ms")] + \
               [("inverse", ctypes.c_int64)] + \
               [(f, ctypes.c_double) for f in ("max_eta", "orth_err")] + \
               [("gemm_core_launches", ctypes.c_int64)] + \
               [(f, ctypes.c_double) for f in ("gemm_core_ms", "gemm_core_flops")] + \
               [("diag_launches", ctypes.c_int64), ("diag_ms", ctypes.c_double), ("tnorm", ctypes.c_double),
                ("filter_matvecs", ctypes.c_int64), ("slice_ms", ctypes.c_double)] + \
               [(f, ctypes.c_int64) for f in ("block_steps", "refine_iters")] + \
               [(f, ctypes.c_double) for f in ("ms_block_lanczos", "ms_refine")] + \
               [(f, ctypes.c_int64) for f in ("refine_stop", "refine_fallback", "symm32_launches")] + \
               [(f, ctypes.c_double) for f in ("symm32_ms", "ms_h2d_first", "host_ms_h2d_enqueue")]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def load(build_if_missing: bool = True):
    """Load the compiled library (building it with nvcc if absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = LIB
    if build_if_missing:
        path = _build_lib()
    if not os.path.exists(path):
        raise RuntimeError(f"libgsyeig.so not found at {path}; run paper_1111_6374_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i64, i32, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "gsyeig_create": ([ctypes.POINTER(vp), i32, vp], i32),
        "gsyeig_destroy": ([vp], i32),
        "gsyeig_default_options": ([ctypes.POINTER(Opts)], i32),
        "gsyeig_set_options": ([vp, ctypes.POINTER(Opts)], i32),
        "gsyeig_strerror": ([i32], ctypes.c_char_p),
        "gsyeig_solve": ([vp, vp, i64, vp, i64, i64, i64, i32, vp, vp, i64, ctypes.POINTER(Info)], i32),
        "gsyeig_potrf": ([vp, vp, i64, i64, ctypes.POINTER(i64)], i32),
        "gsyeig_sygst": ([vp, vp, i64, vp, i64, i64], i32),
        "gsyeig_symv": ([vp, vp, i64, i64, vp, vp], i32),
        "gsyeig_trsm_back": ([vp, vp, i64, i64, vp, i64, i64], i32),
        "gsyeig_syev_lanczos": ([vp, vp, i64, i64, i64, i32, vp, vp, i64, ctypes.POINTER(Info)], i32),
        "gsyeig_tridiag_eig": ([vp, vp, vp, i64, i64, i64, vp, vp, i64], i32),
        "gsyeig_kernel_launches": ([], i64),
        "gsyeig_tridiag_eig_noalloc": ([vp, vp, i64, i64, i64, vp, vp, i64, vp], i32),
        "gsyeig_gemm": ([vp, i32, i32, i64, i64, i64, dp, vp, i64, vp, i64, dp, vp, i64], i32),
        "gsyeig_solve_batched": ([vp, i64, vp, i32, vp, vp], i32),
        "gsyeig_autotuned_block": ([vp, i64], i32),
        "gsyeig_mlp_param_count": ([i32, i32, i32], i64),
        "gsyeig_mlp_workspace_floats": ([i32, i32, i32, i64], i64),
        "gsyeig_mlp_init": ([vp, i32, i32, i32, ctypes.c_uint64, vp], i32),
        "gsyeig_mlp_forward": ([vp, i32, i32, i32, vp, i64, vp, vp, vp], i32),
        "gsyeig_mlp_grad": ([vp, i32, i32, i32, vp, vp, vp, i64, vp, vp, vp, vp], i32),
        "gsyeig_mlp_adam": ([vp, vp, vp, vp, i64, i64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                             ctypes.c_float, vp], i32),
        "gsyeig_ws_features": ([i64, vp, vp, dp, vp, vp, vp], i32),
        "gsyeig_ws_align": ([i64, i64, vp, i64, vp, i64, vp, i64, vp, i64, vp, vp], i32),
        "gsyeig_ws_coef_targets": ([i64, i64, vp, i64, vp, i64, vp, i64, dp, dp, vp, vp], i32),
        "gsyeig_ws_extrapolate": ([i64, i64, vp, i64, vp, i64, vp, dp, dp, vp, i64, vp], i32),
        "gsyeig_ws_shift": ([i64, vp, vp, vp, dp, dp, dp, vp, vp], i32),
        "gsyeig_ws_shift_target": ([vp, vp, vp, dp, dp, vp, vp], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def kernel_launches() -> int:
    return int(load().gsyeig_kernel_launches())


def tridiag_eig_noalloc(d: torch.Tensor, e: torch.Tensor, first: int, cnt: int, vectors: bool = True,
                        stream: torch.cuda.Stream | None = None):
    """Allocation-free tridiagonal eigen-solve (gsyeig_tridiag_eig_noalloc):
    the library allocates nothing; the caller provides the outputs, which this
    wrapper allocates with torch.  Returns (lam, Z) or lam."""
    _check_f64(d, e)
    lib = load()
    m = d.shape[0]
    lam = torch.empty(cnt, device=d.device, dtype=torch.float64)
    Z = colmajor_empty(m, cnt, device=d.device) if vectors else None
    s = stream if stream is not None else torch.cuda.current_stream(d.device)
    st = lib.gsyeig_tridiag_eig_noalloc(d.data_ptr(), e.data_ptr() if e.numel() else None, m, first, cnt,
                                        lam.data_ptr(), Z.data_ptr() if vectors else None, m,
                                        ctypes.c_void_p(s.cuda_stream))
    if st != 0:
        raise GsyeigError(st, "tridiag_eig_noalloc: " + lib.gsyeig_strerror(st).decode())
    return (lam, Z) if vectors else lam


def colmajor_empty(rows: int, cols: int, device="cuda", dtype=torch.float64) -> torch.Tensor:
    """An uninitialised rows x cols tensor with column-major storage."""
    return torch.empty((cols, rows), device=device, dtype=dtype).t()


def colmajor(t: torch.Tensor) -> torch.Tensor:
    """A column-major copy (or the tensor itself if it already is one)."""
    if t.dim() == 2 and t.stride(0) == 1 and t.stride(1) >= max(1, t.shape[0]):
        return t
    return t.t().contiguous().t()


def _ld(t: torch.Tensor, symmetric_ok: bool) -> int:
    if t.dim() != 2:
        raise ValueError("expected a 2-D tensor")
    if t.stride(0) == 1 and t.stride(1) >= max(1, t.shape[0]):
        return t.stride(1)
    if symmetric_ok and t.is_contiguous() and t.shape[0] == t.shape[1]:
        return t.shape[1]  # row-major symmetric: same bytes as column-major
    raise ValueError("expected a column-major tensor (stride(0) == 1)")


def _check_f64(*ts):
    for t in ts:
        if t.dtype != torch.float64:
            raise TypeError("float64 tensors required")


class Solver:
    """One library handle on a CUDA device, bound to a torch stream."""

    def __init__(self, device: int | None = None, stream: torch.cuda.Stream | None = None, **opts):
        self.lib = load()
        dev = torch.cuda.current_device() if device is None else int(device)
        self.device = dev
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        self._h = ctypes.c_void_p()
        self._check(self.lib.gsyeig_create(ctypes.byref(self._h), dev, ctypes.c_void_p(s.cuda_stream)), "create")
        self.opts = Opts()
        self.lib.gsyeig_default_options(ctypes.byref(self.opts))
        if opts:
            self.set_options(**opts)

    def _check(self, st: int, what: str, ok=(0,)):
        if st not in ok:
            msg = self.lib.gsyeig_strerror(st).decode()
            raise GsyeigError(st, f"{what}: {msg}")
        return st

    def set_options(self, **kw):
        """Set fields of gsyeig_opts.  Device tensors for v0, start_block and
        start_weights are kept alive by the solver; a column-major start_block
        also sets start_cols and ld_start."""
        for k, v in kw.items():
            if k in ("v0", "start_block", "start_weights"):
                setattr(self, "_" + k, v)
                if k == "start_block":
                    self.opts.start_cols = 0 if v is None else v.shape[1]
                    self.opts.ld_start = 0 if v is None else _ld(v, False)
                v = None if v is None else v.data_ptr()
            setattr(self.opts, k, v)
        self._check(self.lib.gsyeig_set_options(self._h, ctypes.byref(self.opts)), "set_options")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.gsyeig_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- whole route ------------------------------------------------------
    def solve(self, A: torch.Tensor, B: torch.Tensor, s: int, which: str = "smallest", overwrite: bool = False,
              allow_unconverged: bool = False):
        """s eigenpairs of (A, B): returns (w ascending, X column-major n x s, info dict).

        Device tensors: A becomes C and B's upper triangle U unless
        ``overwrite`` is False (then copies are solved).  CPU tensors: the
        host pointers are handed to the library, which stages them on the
        device and returns w and X on the host."""
        _check_f64(A, B)
        n = A.shape[0]
        on_dev = A.is_cuda
        if on_dev and not overwrite:
            A = A.clone(memory_format=torch.contiguous_format)
            B = B.clone(memory_format=torch.contiguous_format)
        lda, ldb = _ld(A, True), _ld(B, True)
        if on_dev:
            X = colmajor_empty(n, s, device=A.device)
            w = torch.empty(s, device=A.device, dtype=torch.float64)
        else:
            X = torch.empty((s, n), dtype=torch.float64, pin_memory=A.is_pinned()).t()
            w = torch.empty(s, dtype=torch.float64)
        info = Info()
        st = self.lib.gsyeig_solve(self._h, A.data_ptr(), lda, B.data_ptr(), ldb, n, s,
                                   LARGEST if which == "largest" else SMALLEST, w.data_ptr(), X.data_ptr(), X.stride(1),
                                   ctypes.byref(info))
        self._check(st, "solve", ok=(0, 2, 3) if allow_unconverged else (0,))
        d = info.as_dict()
        d["status"] = st
        return w, X, d

    def solve_batched(self, pencils, s, which: str = "smallest", streams: int = 8, overwrite: bool = False):
        """Independent problems [(A_i, B_i), ...] (device tensors) through
        gsyeig_solve_batched; returns [(w_i, X_i, info_i)] in input order."""
        probs = (Problem * len(pencils))()
        outs, keep = [], []
        for i, (A, B) in enumerate(pencils):
            _check_f64(A, B)
            if not overwrite:
                A = A.clone(memory_format=torch.contiguous_format)
                B = B.clone(memory_format=torch.contiguous_format)
            n = A.shape[0]
            si = s[i] if isinstance(s, (list, tuple)) else s
            X = colmajor_empty(n, si, device=A.device)
            w = torch.empty(si, device=A.device, dtype=torch.float64)
            probs[i] = Problem(A.data_ptr(), _ld(A, True), B.data_ptr(), _ld(B, True), n, si,
                               LARGEST if which == "largest" else SMALLEST, 0, w.data_ptr(), X.data_ptr(), X.stride(1))
            outs.append((w, X))
            keep.append((A, B))
        st = (ctypes.c_int32 * len(pencils))()
        infos = (Info * len(pencils))()
        rc = self.lib.gsyeig_solve_batched(self._h, len(pencils), probs, streams, st, infos)
        self._check(rc, "solve_batched")
        return [(w, X, dict(infos[i].as_dict(), status=st[i])) for i, (w, X) in enumerate(outs)]

    def autotuned_block(self, n: int) -> int:
        return int(self.lib.gsyeig_autotuned_block(self._h, n))

    # -- single steps -----------------------------------------------------
    def potrf(self, B: torch.Tensor):
        """In place: U (B = U^T U) in the upper triangle of column-major B; returns 0 or failing pivot."""
        _check_f64(B)
        idx = ctypes.c_int64(0)
        st = self.lib.gsyeig_potrf(self._h, B.data_ptr(), _ld(B, True), B.shape[0], ctypes.byref(idx))
        self._check(st, "potrf", ok=(0, 1))
        return int(idx.value)

    def sygst(self, A: torch.Tensor, U: torch.Tensor):
        """In place: A <- U^-T A U^-1 (lower triangle of A read; C written full)."""
        _check_f64(A, U)
        self._check(self.lib.gsyeig_sygst(self._h, A.data_ptr(), _ld(A, True), U.data_ptr(), _ld(U, False), A.shape[0]),
                    "sygst")
        return A

    def symv(self, C: torch.Tensor, w: torch.Tensor, z: torch.Tensor | None = None):
        _check_f64(C, w)
        n = C.shape[0]
        if z is None:
            z = torch.empty(n, device=C.device, dtype=torch.float64)
        self._check(self.lib.gsyeig_symv(self._h, C.data_ptr(), _ld(C, True), n, w.data_ptr(), z.data_ptr()), "symv")
        return z

    def trsm_back(self, U: torch.Tensor, Y: torch.Tensor):
        """In place: Y <- U^-1 Y (Y column-major n x s)."""
        _check_f64(U, Y)
        self._check(self.lib.gsyeig_trsm_back(self._h, U.data_ptr(), _ld(U, False), U.shape[0], Y.data_ptr(),
                                              _ld(Y, False), Y.shape[1]), "trsm_back")
        return Y

    def syev_lanczos(self, C: torch.Tensor, s: int, which: str = "smallest", allow_unconverged: bool = False):
        _check_f64(C)
        n = C.shape[0]
        Y = colmajor_empty(n, s, device=C.device)
        w = torch.empty(s, device=C.device, dtype=torch.float64)
        info = Info()
        st = self.lib.gsyeig_syev_lanczos(self._h, C.data_ptr(), _ld(C, True), n, s,
                                          LARGEST if which == "largest" else SMALLEST, w.data_ptr(), Y.data_ptr(),
                                          Y.stride(1), ctypes.byref(info))
        self._check(st, "syev_lanczos", ok=(0, 2, 3) if allow_unconverged else (0,))
        d = info.as_dict()
        d["status"] = st
        return w, Y, d

    def gemm(self, A: torch.Tensor, B: torch.Tensor, C: torch.Tensor | None = None, transA: bool = False,
             transB: bool = False, alpha: float = 1.0, beta: float = 0.0):
        """C = alpha op(A) op(B) + beta C on the library's GEMM engine (column-major tensors)."""
        _check_f64(A, B)
        M = A.shape[1] if transA else A.shape[0]
        K = A.shape[0] if transA else A.shape[1]
        N = B.shape[0] if transB else B.shape[1]
        if C is None:
            C = colmajor_empty(M, N, device=A.device)
        self._check(self.lib.gsyeig_gemm(self._h, int(transA), int(transB), M, N, K, alpha, A.data_ptr(),
                                         _ld(A, False), B.data_ptr(), _ld(B, False), beta, C.data_ptr(),
                                         _ld(C, False)), "gemm")
        return C

    def tridiag_eig(self, d: torch.Tensor, e: torch.Tensor, first: int, cnt: int, vectors: bool = True):
        _check_f64(d, e)
        m = d.shape[0]
        lam = torch.empty(cnt, device=d.device, dtype=torch.float64)
        Z = colmajor_empty(m, cnt, device=d.device) if vectors else None
        st = self.lib.gsyeig_tridiag_eig(self._h, d.data_ptr(), e.data_ptr() if e.numel() else None, m, first, cnt,
                                         lam.data_ptr(), Z.data_ptr() if vectors else None, m)
        self._check(st, "tridiag_eig")
        return (lam, Z) if vectors else lam
