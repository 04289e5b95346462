"""Thin ctypes binding of libtstar (include/tstar.h): argument marshalling only.

Tensors are passed as torch tensors in the library's layout: a tensor
X in R^{n1 x n2 x p} is a contiguous float64 torch tensor of shape (p, n2, n1)
(column-major X(i, j, k) at i + n1*(j + n2*k)).  CUDA tensors are passed by
device pointer on the current torch stream; CPU tensors by host pointer (the
library stages them).  Every computation runs inside libtstar; there is no
Python or CPU fallback, and a missing library raises immediately.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtstar.so")

TS_OK, TS_BREAKDOWN, TS_NOT_CONVERGED, TS_SINGULAR = 0, 1, 2, 3
TS_ERR_ARG, TS_ERR_CUDA, TS_ERR_NOMEM, TS_ERR_NONFINITE, TS_ERR_TIMEOUT, TS_ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6
TS_ERR_CORRUPTION = -7
PRECISIONS = {"fp64": 0, "mixed_fp32": 1, "mixed_tf32": 2, "mixed_bf16": 3, "mixed_tf32x3": 4}
ENGINES = {"dfma": 0, "ozaki": 1}
STATUS_NAMES = {0: "ok", 1: "breakdown", 2: "not_converged", 3: "singular", -1: "err_arg", -2: "err_cuda",
                -3: "err_nomem", -4: "err_nonfinite", -5: "err_timeout", -6: "err_unsupported", -7: "err_corruption"}


class SolveOpts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("max_restarts", ctypes.c_int), ("tol", ctypes.c_double),
                ("precision", ctypes.c_int), ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("history", ctypes.POINTER(ctypes.c_double)), ("history_cap", ctypes.c_int),
                ("true_history", ctypes.POINTER(ctypes.c_double)), ("true_history_cap", ctypes.c_int),
                ("fp64_engine", ctypes.c_int), ("ozaki_digits", ctypes.c_int), ("spectral_basis", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("cycles", ctypes.c_int), ("outer", ctypes.c_int),
                ("history_len", ctypes.c_int), ("true_history_len", ctypes.c_int),
                ("applies_fp64", ctypes.c_int), ("applies_low", ctypes.c_int),
                ("normC", ctypes.c_double), ("relres_true", ctypes.c_double), ("relres_est", ctypes.c_double),
                ("ms_total", ctypes.c_double)]


class Instance(ctypes.Structure):
    _fields_ = [("op", ctypes.c_void_p), ("C", ctypes.c_void_p), ("X", ctypes.c_void_p), ("tol", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("gemm_launches", ctypes.c_longlong), ("gemm_ms", ctypes.c_double),
                ("gemm_flops", ctypes.c_double), ("lowp_launches", ctypes.c_longlong), ("lowp_ms", ctypes.c_double),
                ("lowp_flops", ctypes.c_double), ("fft_launches", ctypes.c_longlong), ("fft_ms", ctypes.c_double),
                ("fft_bytes", ctypes.c_double), ("oz_launches", ctypes.c_longlong), ("oz_ms", ctypes.c_double),
                ("oz_flops", ctypes.c_double), ("tba_launches", ctypes.c_longlong), ("tba_ms", ctypes.c_double),
                ("tba_flops", ctypes.c_double), ("oz_pair_flops", ctypes.c_double),
                ("spmm_launches", ctypes.c_longlong), ("spmm_ms", ctypes.c_double), ("spmm_flops", ctypes.c_double),
                ("spmm_bytes", ctypes.c_double), ("host_setup_ms", ctypes.c_double),
                ("graph_build_ms", ctypes.c_double), ("host_cycles_ms", ctypes.c_double)]


class TstarError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

_vp, _i, _u, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_double
_SIGNATURES = {
    "ts_create": (_i, [ctypes.POINTER(_vp), _i]),
    "ts_destroy": (None, [_vp]),
    "ts_last_error": (ctypes.c_char_p, [_vp]),
    "ts_status_string": (ctypes.c_char_p, [_i]),
    "ts_tstar": (_i, [_vp, _vp, _i, _i, _vp, _i, _i, _vp, _vp]),
    "ts_op_create_dense": (_i, [_vp, _vp, _i, _vp, _i, _i, _u, ctypes.POINTER(_vp), _vp]),
    "ts_op_create_csr": (_i, [_vp, _i, _i, _vp, _vp, _vp, _vp, _i, _u, ctypes.POINTER(_vp), _vp]),
    "ts_op_destroy": (None, [_vp]),
    "ts_op_shape": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "ts_sylv_apply": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "ts_sylv_apply_lowp": (_i, [_vp, _vp, _i, _vp, _vp, _vp]),
    "ts_sylv_apply_ozaki": (_i, [_vp, _vp, _i, _vp, _vp, _vp]),
    "ts_solve_opts_default": (None, [ctypes.POINTER(SolveOpts)]),
    "ts_tgmres_solve": (_i, [_vp, _vp, _vp, _vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), _vp]),
    "ts_tfom_solve": (_i, [_vp, _vp, _vp, _vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), _vp]),
    "ts_tba_solve": (_i, [_vp, _vp, _vp, _vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), _vp]),
    "ts_t_bartels_stewart": (_i, [_vp, _vp, _i, _vp, _i, _i, _vp, _vp, _vp]),
    "ts_batched_solve": (_i, [_vp, _i, ctypes.POINTER(Instance), ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo),
                              ctypes.POINTER(_i), _vp]),
    "ts_tstar_noalloc": (_i, [_vp, _i, _i, _vp, _i, _i, _vp, _vp]),
    "ts_workspace_check": (_i, [_vp]),
    "ts_tune_entries": (_i, [_vp, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "ts_stats_enable": (_i, [_vp, _i]),
    "ts_stats_get": (_i, [_vp, ctypes.POINTER(Stats)]),
    "ts_stats_reset": (_i, [_vp]),
    "ts_probe_fp64_peak": (_i, [_vp, ctypes.POINTER(_d), _vp]),
}


def lib():
    """Load libtstar.so (built in-tree by paper_2405_09233_gb300.build); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() (nvcc, sm_103a)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(t) -> int:
    import torch
    assert isinstance(t, torch.Tensor), "expected a torch tensor"
    assert t.dtype == torch.float64, "expected float64"
    assert t.is_contiguous(), "expected a contiguous tensor in (p, n2, n1) layout"
    return t.data_ptr()


def _stream(*tensors):
    import torch
    if any(t.is_cuda for t in tensors):
        return ctypes.c_void_p(torch.cuda.current_stream(tensors[0].device).cuda_stream)
    return ctypes.c_void_p(0)


class Context:
    """A libtstar context on one CUDA device."""

    def __init__(self, device: int = 0):
        self._h = _vp()
        st = lib().ts_create(ctypes.byref(self._h), device)
        if st != TS_OK:
            raise TstarError(st, "ts_create failed")
        self.device = device

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def close(self):
        if self._h:
            lib().ts_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, what: str):
        if st < 0:
            raise TstarError(st, f"{what}: {lib().ts_last_error(self._h).decode()}")
        return st

    def workspace_check(self):
        """Raise TstarError if any workspace buffer was written past its end."""
        self._check(lib().ts_workspace_check(self._h), "ts_workspace_check")

    def probe_fp64_peak(self) -> float:
        """Measured FP64 fused multiply-add rate of the device in TFLOP/s (ts_probe_fp64_peak), on the
        current stream."""
        import torch
        out = ctypes.c_double(0.0)
        st = ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        self._check(lib().ts_probe_fp64_peak(self._h, ctypes.byref(out), st), "ts_probe_fp64_peak")
        return out.value

    def tune_entries(self) -> dict:
        """The autotuner's choices in this context, {key: value} (ts_tune_entries)."""
        need = ctypes.c_size_t(0)
        self._check(lib().ts_tune_entries(self._h, None, 0, ctypes.byref(need)), "ts_tune_entries")
        buf = ctypes.create_string_buffer(need.value)
        self._check(lib().ts_tune_entries(self._h, buf, need.value, ctypes.byref(need)), "ts_tune_entries")
        out = {}
        for line in buf.value.decode().splitlines():
            k, v = line.rsplit(" ", 1)
            out[k] = int(v)
        return out

    # --- statistics ---------------------------------------------------------------------------
    def stats_enable(self, enable: bool = True):
        self._check(lib().ts_stats_enable(self._h, int(enable)), "ts_stats_enable")

    def stats_get(self) -> Stats:
        s = Stats()
        self._check(lib().ts_stats_get(self._h, ctypes.byref(s)), "ts_stats_get")
        return s

    def stats_reset(self):
        self._check(lib().ts_stats_reset(self._h), "ts_stats_reset")

    # --- entry points -------------------------------------------------------------------------
    def tstar(self, A, B, C=None):
        """C = A * B (T-product).  A: (p, n2, n1), B: (p, m, n2) float64 torch tensors."""
        import torch
        p, n2, n1 = A.shape
        pB, m, n2b = B.shape
        assert p == pB and n2 == n2b
        if C is None:
            C = torch.empty((p, m, n1), dtype=torch.float64, device=A.device)
        self._check(lib().ts_tstar(self._h, _ptr(A), n1, n2, _ptr(B), m, p, _ptr(C), _stream(A, B, C)), "ts_tstar")
        return C

    def op_create_dense(self, A, B) -> "Operator":
        p, n, n_ = A.shape
        pB, s, s_ = B.shape
        assert n == n_ and s == s_ and p == pB
        h = _vp()
        self._check(lib().ts_op_create_dense(self._h, _ptr(A), n, _ptr(B), s, p, 0, ctypes.byref(h),
                                             _stream(A, B)), "ts_op_create_dense")
        return Operator(self, h, n, s, p)

    def op_create_csr(self, n, p, rowptr, col, val, B) -> "Operator":
        """Sparse A from p CSR slices (numpy int32 rowptr of length p*(n+1) indexing the shared
        int32 col / float64 val arrays); B: (p, s, s) float64 torch tensor."""
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        col = np.ascontiguousarray(col, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float64)
        pB, s, s_ = B.shape
        assert pB == p and s == s_ and rowptr.size == p * (n + 1)
        h = _vp()
        self._check(lib().ts_op_create_csr(self._h, n, p, rowptr.ctypes.data, col.ctypes.data, val.ctypes.data,
                                           _ptr(B), s, 0, ctypes.byref(h), _stream(B)), "ts_op_create_csr")
        return Operator(self, h, n, s, p)

    def t_bartels_stewart(self, A, B, C, X=None):
        """Small dense STE A*X - X*B = C by t-Bartels-Stewart; (p, n, n), (p, s, s), (p, s, n) tensors.
        Raises TstarError when the library reports TS_SINGULAR (no solution was formed)."""
        import torch
        p, n, _ = A.shape
        s = B.shape[1]
        if X is None:
            X = torch.empty_like(C)
        st = self._check(lib().ts_t_bartels_stewart(self._h, _ptr(A), n, _ptr(B), s, p, _ptr(C), _ptr(X),
                                                    _stream(A, B, C, X)), "ts_t_bartels_stewart")
        if st != 0:   # TS_SINGULAR: X holds no solution
            raise TstarError(st, f"ts_t_bartels_stewart: {lib().ts_last_error(self._h).decode()}")
        return X

    def sylv_apply(self, op: "Operator", X, Y=None):
        import torch
        if Y is None:
            Y = torch.empty_like(X)
        self._check(lib().ts_sylv_apply(self._h, op._h, _ptr(X), _ptr(Y), _stream(X, Y)), "ts_sylv_apply")
        return Y

    def sylv_apply_ozaki(self, op: "Operator", X, Y=None, digits=0):
        """Y = M(X) in FP64 with the slice products on the emulated-FP64 tensor-core engine."""
        import torch
        if Y is None:
            Y = torch.empty_like(X)
        self._check(lib().ts_sylv_apply_ozaki(self._h, op._h, int(digits), _ptr(X), _ptr(Y), _stream(X, Y)),
                    "ts_sylv_apply_ozaki")
        return Y

    def sylv_apply_lowp(self, op: "Operator", X, precision="mixed_bf16", Y=None):
        """Y = M(X) in low precision; X, Y float32 CUDA tensors of shape (p, s, n)."""
        import torch
        assert X.dtype == torch.float32 and X.is_cuda and X.is_contiguous()
        if Y is None:
            Y = torch.empty_like(X)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self._check(lib().ts_sylv_apply_lowp(self._h, op._h, prec, X.data_ptr(), Y.data_ptr(), _stream(X, Y)),
                    "ts_sylv_apply_lowp")
        return Y

    def _solve(self, fn, name, op, C, X, restart, tol, max_restarts, precision, inner_tol, max_outer,
               history_cap, engine="dfma", ozaki_digits=0, spectral=False):
        opts = SolveOpts()
        lib().ts_solve_opts_default(ctypes.byref(opts))
        opts.restart, opts.tol, opts.max_restarts = restart, tol, max_restarts
        opts.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        opts.inner_tol, opts.max_outer = inner_tol, max_outer
        opts.fp64_engine = ENGINES[engine] if isinstance(engine, str) else int(engine)
        opts.ozaki_digits = ozaki_digits
        opts.spectral_basis = 1 if spectral else 0
        hist = np.zeros(history_cap)
        thist = np.zeros(history_cap)
        opts.history = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        opts.history_cap = history_cap
        opts.true_history = thist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        opts.true_history_cap = history_cap
        info = SolveInfo()
        st = self._check(fn(self._h, op._h, _ptr(C), _ptr(X), ctypes.byref(opts), ctypes.byref(info),
                            _stream(C, X)), name)
        return SolveResult(st, info, hist[:min(info.history_len, history_cap)].copy(),
                           thist[:min(info.true_history_len, history_cap)].copy())

    def tgmres_solve(self, op, C, X, restart=20, tol=1e-10, max_restarts=200, precision="fp64",
                     inner_tol=0.0, max_outer=0, history_cap=4096, engine="dfma", ozaki_digits=0, spectral=False):
        """Restarted tGMRES(m); X holds X0 on entry and the solution on return.  engine selects how
        FP64 applications are computed ("dfma" or "ozaki"); spectral=True keeps an FP64 Krylov basis in
        the Fourier domain."""
        return self._solve(lib().ts_tgmres_solve, "ts_tgmres_solve", op, C, X, restart, tol, max_restarts,
                           precision, inner_tol, max_outer, history_cap, engine, ozaki_digits, spectral)

    def tba_solve(self, op, C, X, restart=10, tol=1e-10, max_restarts=100, history_cap=4096, precision="fp64"):
        """Restarted TBAS(m); X holds X0 on entry and the solution on return.  precision "fp64", or
        "mixed_fp32" (FP32 block Krylov cycles, FP64 true residuals and solution)."""
        return self._solve(lib().ts_tba_solve, "ts_tba_solve", op, C, X, restart, tol, max_restarts,
                           precision, 0.0, 0, history_cap)

    def batched_solve(self, ops, Cs, Xs, tols=None, restart=20, tol=1e-10, max_restarts=200, precision="fp64",
                      inner_tol=0.0, max_outer=0, engine="dfma", ozaki_digits=0):
        """Solve len(ops) independent STEs together; Cs/Xs are CUDA float64 tensors (p, s, n) per instance.
        Returns (status, [SolveInfo], [per-instance status])."""
        count = len(ops)
        arr = (Instance * count)()
        for i, (op, C, X) in enumerate(zip(ops, Cs, Xs)):
            arr[i].op = op._h.value if isinstance(op._h, ctypes.c_void_p) else op._h
            arr[i].C = _ptr(C)
            arr[i].X = _ptr(X)
            arr[i].tol = -1.0 if tols is None else float(tols[i])
        opts = SolveOpts()
        lib().ts_solve_opts_default(ctypes.byref(opts))
        opts.restart, opts.tol, opts.max_restarts = restart, tol, max_restarts
        opts.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        opts.inner_tol, opts.max_outer = inner_tol, max_outer
        opts.fp64_engine = ENGINES[engine] if isinstance(engine, str) else int(engine)
        opts.ozaki_digits = ozaki_digits
        infos = (SolveInfo * count)()
        sts = (ctypes.c_int * count)()
        st = self._check(lib().ts_batched_solve(self._h, count, arr, ctypes.byref(opts), infos, sts,
                                                _stream(*Cs)), "ts_batched_solve")
        return st, list(infos), list(sts)

    def tfom_solve(self, op, C, X, restart=20, tol=1e-10, max_restarts=200, history_cap=4096, engine="dfma",
                   ozaki_digits=0, spectral=False):
        """Restarted tFOM(m) (FP64); spectral=True keeps the Krylov basis in the Fourier domain."""
        return self._solve(lib().ts_tfom_solve, "ts_tfom_solve", op, C, X, restart, tol, max_restarts,
                           "fp64", 0.0, 0, history_cap, engine, ozaki_digits, spectral)


class Operator:
    """A prepared operator M(X) = A*X - X*B (owns the Fourier slices of A and B on the device)."""

    def __init__(self, ctx: Context, h, n: int, s: int, p: int):
        self.ctx, self._h, self.n, self.s, self.p = ctx, h, n, s, p

    def close(self):
        if self._h:
            lib().ts_op_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SolveResult:
    def __init__(self, status: int, info: SolveInfo, history: np.ndarray, true_history: np.ndarray):
        self.status = status
        self.status_name = STATUS_NAMES.get(status, str(status))
        self.info = info
        self.history = history
        self.true_history = true_history

    @property
    def relres(self) -> float:
        return self.info.relres_true

    def __repr__(self):
        i = self.info
        return (f"SolveResult({self.status_name}, iters={i.iters}, cycles={i.cycles}, outer={i.outer}, "
                f"relres={i.relres_true:.3e}, fp64_applies={i.applies_fp64}, low_applies={i.applies_low}, "
                f"ms={i.ms_total:.2f})")


def declared_symbols(header: Optional[str] = None):
    """Names of the functions include/tstar.h declares (for the ABI completeness test)."""
    import re
    header = header or os.path.join(_PKG, "..", "include", "tstar.h")
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ts_[a-z0-9_]+)\s*\(", text)))
