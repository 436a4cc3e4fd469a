"""Python binding of the GB300 rational-program library (``include/klr.h``).

Argument marshalling only: every step of the fit and of the evaluation runs in
the library's CUDA kernels.  PyTorch provides device memory and the current
stream.  Importing this package loads ``_lib/libklr.so`` and raises if it is
missing (build it with ``python paper_1911_02373_gb300/build.py`` or
``__graft_entry__.build()``); there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libklr.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                      "(python paper_1911_02373_gb300/build.py)")
_lib = ctypes.CDLL(LIB_PATH)

# status codes and enums of klr.h
OK, EINVAL, ECUDA, ENOMEM, ENOTSUP = 0, 1, 2, 3, 4
F32, F64 = 0, 1
EXP8 = 2      # sample coordinates as uint8 base-2 logarithms (klr_fit)
EXP16 = 3     # one packed code per sample: log2 N | log2 b0 << 6 | log2 b1 << 11 (klr_fit)
FIT_FP64, FIT_DF32, FIT_FP32, FIT_TF32, FIT_BF16 = 0, 1, 2, 3, 4
FIT_OK, FIT_EMPTY, FIT_NONFINITE, FIT_RANK_DEFICIENT, FIT_INEXACT, FIT_SOLVE_FAILED = 0, 1, 2, 4, 8, 16
Q_OK, Q_BAD_METRIC, Q_NONE_FEASIBLE, Q_TIE_RESOLVED, Q_HISTORY, Q_REFINED = 0, 1, 2, 4, 8, 16

#: every entry point declared in include/klr.h
ABI_SYMBOLS = ("klr_ctx_create", "klr_ctx_destroy", "klr_ctx_reserve", "klr_last_error",
               "klr_version", "klr_enumerate_configs", "klr_fit", "klr_eval", "klr_argmin",
               "klr_argmin_noalloc", "klr_mlp_param_count", "klr_mlp_train_step",
               "klr_mlp_predict", "klr_propose", "klr_argmin_candidates", "klr_autotune_fit",
               "klr_autotune_argmin", "klr_tune_export", "klr_tune_import", "klr_fit_gram",
               "klr_fit_solve", "klr_mlp_query_targets", "klr_history_create",
               "klr_history_clear", "klr_history_destroy", "klr_argmin_history",
               "klr_argmin_refined", "klr_fit_heldout", "klr_choose_basis", "klr_probe_peaks")
#: largest query count klr_argmin_noalloc accepts
ARGMIN_NOALLOC_MAX_QUERIES = 65536
ARGMIN_NOALLOC_TIE_RECORDS = 16384   # FP32 near-ties it lists; more are decided in place


class KlrError(RuntimeError):
    def __init__(self, fn, status):
        msg = _lib.klr_last_error().decode()
        super().__init__(f"{fn} returned {status}: {msg}")
        self.status = status


class FitBatch(ctypes.Structure):
    _fields_ = [("n_fits", ctypes.c_int32), ("n_vars", ctypes.c_int32),
                ("degree", ctypes.c_int32), ("n_scale_log2", ctypes.c_int32),
                ("b_scale_log2", ctypes.c_int32), ("sample_dtype", ctypes.c_int32),
                ("offsets", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("x_stride", ctypes.c_int64), ("y", ctypes.c_void_p),
                ("precision", ctypes.c_int32), ("refine_iters", ctypes.c_int32),
                ("var_degree", ctypes.c_int32 * 4)]


class Hw(ctypes.Structure):
    _fields_ = [("n_sm", ctypes.c_int32), ("max_warps_per_sm", ctypes.c_int32),
                ("regs_per_sm", ctypes.c_int32), ("smem_per_sm", ctypes.c_int32),
                ("max_blocks_per_sm", ctypes.c_int32), ("max_threads_per_block", ctypes.c_int32),
                ("mem_latency", ctypes.c_double), ("mem_bandwidth", ctypes.c_double),
                ("clock_hz", ctypes.c_double), ("departure_delay_coal", ctypes.c_double),
                ("departure_delay_uncoal", ctypes.c_double)]


class Program(ctypes.Structure):
    _fields_ = [("n_kernels", ctypes.c_int32), ("n_vars", ctypes.c_int32),
                ("degree", ctypes.c_int32), ("n_scale_log2", ctypes.c_int32),
                ("b_scale_log2", ctypes.c_int32), ("coef_dtype", ctypes.c_int32),
                ("coef", ctypes.c_void_p), ("regs", ctypes.c_void_p), ("smem", ctypes.c_void_p),
                ("metric_lo", ctypes.c_double * 8), ("metric_scale", ctypes.c_double * 8),
                ("var_degree", ctypes.c_int32 * 4)]


class Queries(ctypes.Structure):
    _fields_ = [("q_offsets", ctypes.c_void_p), ("q_N", ctypes.c_void_p),
                ("n_queries", ctypes.c_int64)]


class MlpNet(ctypes.Structure):
    _fields_ = [("n_coef", ctypes.c_int32), ("n_out", ctypes.c_int32), ("params", ctypes.c_void_p),
                ("adam_m", ctypes.c_void_p), ("adam_v", ctypes.c_void_p),
                ("step", ctypes.c_int64), ("hw_feat", ctypes.c_float * 7)]


class Peaks(ctypes.Structure):
    _fields_ = [("fp32_fma_tflops", ctypes.c_double), ("fp32x2_fma_tflops", ctypes.c_double),
                ("fp64_fma_tflops", ctypes.c_double), ("mufu_rcp_tops", ctypes.c_double),
                ("tf32_mma_sync_tflops", ctypes.c_double)]


class MlpRows(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("kernel", ctypes.c_void_p), ("N", ctypes.c_void_p),
                ("cfg_idx", ctypes.c_void_p), ("target", ctypes.c_void_p)]


_vp = ctypes.c_void_p
_lib.klr_last_error.restype = ctypes.c_char_p
_lib.klr_mlp_param_count.restype = ctypes.c_int64
_lib.klr_mlp_param_count.argtypes = [ctypes.c_int32, ctypes.c_int32]
_lib.klr_version.restype = ctypes.c_int
for _name, _args in {
    "klr_ctx_create": [ctypes.POINTER(_vp), ctypes.c_int],
    "klr_ctx_destroy": [_vp],
    "klr_ctx_reserve": [_vp, ctypes.c_int64, ctypes.c_int64],
    "klr_enumerate_configs": [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int,
                              ctypes.POINTER(ctypes.c_int)],
    "klr_fit": [_vp, ctypes.POINTER(FitBatch), _vp, ctypes.c_int32, _vp, _vp, _vp],
    "klr_eval": [_vp, ctypes.POINTER(Program), ctypes.POINTER(Hw), _vp, ctypes.c_int,
                 ctypes.POINTER(Queries), _vp, ctypes.c_int32, _vp],
    "klr_argmin": [_vp, ctypes.POINTER(Program), ctypes.POINTER(Hw), _vp, ctypes.c_int,
                   ctypes.POINTER(Queries), _vp, _vp, ctypes.c_int32, _vp, _vp, _vp, _vp],
    "klr_autotune_fit": [_vp, ctypes.POINTER(FitBatch), _vp, ctypes.c_int32, _vp, _vp,
                         ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float), _vp],
    "klr_autotune_argmin": [_vp, ctypes.POINTER(Program), ctypes.POINTER(Hw), _vp, ctypes.c_int,
                            ctypes.POINTER(Queries), _vp, _vp, ctypes.c_int32, _vp, _vp, _vp,
                            ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float), _vp],
    "klr_fit_gram": [_vp, ctypes.POINTER(FitBatch), _vp],
    "klr_fit_heldout": [_vp, ctypes.POINTER(FitBatch), _vp, ctypes.c_int32, _vp, _vp],
    "klr_choose_basis": [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                         ctypes.c_double, _vp, _vp],
    "klr_history_create": [_vp, ctypes.c_int32, ctypes.POINTER(_vp)],
    "klr_probe_peaks": [_vp, ctypes.POINTER(Peaks), _vp],
    "klr_history_clear": [_vp, _vp],
    "klr_argmin_refined": [_vp, ctypes.POINTER(Program), ctypes.POINTER(Hw), _vp, ctypes.c_int,
                           ctypes.POINTER(Queries), _vp, ctypes.c_double, _vp, _vp, _vp, _vp],
    "klr_history_destroy": [_vp],
    "klr_argmin_history": [_vp, _vp, ctypes.POINTER(Program), ctypes.POINTER(Hw), _vp, ctypes.c_int,
                           ctypes.POINTER(Queries), _vp, _vp, _vp, _vp, _vp, _vp],
    "klr_mlp_query_targets": [_vp, ctypes.c_int64, ctypes.c_int32, _vp, _vp],
    "klr_fit_solve": [_vp, ctypes.POINTER(FitBatch), _vp, ctypes.c_int32, _vp, _vp, _vp],
    "klr_tune_export": [_vp, _vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "klr_tune_import": [_vp, _vp, _vp, ctypes.c_int],
    "klr_argmin_noalloc": [ctypes.POINTER(Program), ctypes.POINTER(Hw), _vp, ctypes.c_int,
                           ctypes.POINTER(Queries), _vp, _vp, _vp, _vp, _vp, _vp],
    "klr_mlp_train_step": [_vp, ctypes.POINTER(MlpNet), _vp, _vp, ctypes.c_int,
                           ctypes.POINTER(MlpRows), ctypes.c_float, ctypes.c_float, ctypes.c_int,
                           _vp, _vp, _vp],
    "klr_mlp_predict": [_vp, ctypes.POINTER(MlpNet), _vp, _vp, ctypes.c_int,
                        ctypes.POINTER(MlpRows), _vp, _vp],
    "klr_propose": [_vp, ctypes.POINTER(MlpNet), _vp, _vp, _vp, ctypes.c_int32,
                    ctypes.POINTER(Hw), _vp, ctypes.c_int, ctypes.POINTER(Queries), ctypes.c_int,
                    _vp, _vp],
    "klr_argmin_candidates": [_vp, ctypes.POINTER(Program), ctypes.POINTER(Hw), _vp, ctypes.c_int,
                              ctypes.POINTER(Queries), _vp, ctypes.c_int, _vp, _vp, _vp, _vp],
}.items():
    getattr(_lib, _name).argtypes = _args
    getattr(_lib, _name).restype = ctypes.c_int32


def _check(fn, status):
    if status != OK:
        raise KlrError(fn, status)


def version() -> int:
    return _lib.klr_version()


def enumerate_configs(dims: int, min_threads: int = 32, max_threads: int = 1024) -> np.ndarray:
    """Configuration set F as an (|F|, 3) int32 array (unused dims are 1)."""
    n = ctypes.c_int(0)
    _check("klr_enumerate_configs",
           _lib.klr_enumerate_configs(dims, min_threads, max_threads, None, 0, ctypes.byref(n)))
    out = np.zeros((n.value, 3), dtype=np.int32)
    _check("klr_enumerate_configs",
           _lib.klr_enumerate_configs(dims, min_threads, max_threads,
                                      out.ctypes.data_as(_vp), n.value, ctypes.byref(n)))
    return out


def _dptr(t):
    """Device address of a CUDA tensor.  The library's kernels read and write
    the addresses they are given, so a tensor in host memory is refused here
    (on a GPU that reaches host memory through a coherent link it would
    otherwise be read or written in place instead of failing)."""
    if not t.is_cuda:
        raise ValueError(f"expected a CUDA tensor, got one on {t.device}")
    return t.data_ptr()


def _ptr(t):
    return None if t is None else ctypes.c_void_p(_dptr(t))


def _iptr(t):
    """Address of an input the kernels only read (klr_fit's samples and
    offsets, klr_argmin's queries): a CUDA tensor, or a page-locked host
    tensor (pin_memory), which the device reads in place through unified
    addressing.  Any other host tensor is refused."""
    if t.is_cuda:
        return t.data_ptr()
    if t.is_pinned() and t.is_contiguous():
        return t.data_ptr()
    raise ValueError("expected a CUDA tensor or a contiguous page-locked host tensor, "
                     f"got one on {t.device}")


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def make_hw(hw: dict) -> Hw:
    return Hw(int(hw["n_sm"]), int(hw["max_warps_per_sm"]), int(hw["regs_per_sm"]),
              int(hw["smem_per_sm"]), int(hw["max_blocks_per_sm"]),
              int(hw["max_threads_per_block"]), float(hw["mem_latency"]),
              float(hw["mem_bandwidth"]), float(hw["clock_hz"]),
              float(hw["departure_delay_coal"]), float(hw["departure_delay_uncoal"]))


class Context:
    """A library context on one CUDA device (owns the scratch memory)."""

    def __init__(self, device: int = 0):
        import torch
        torch.cuda.init()
        self.device = device
        h = _vp()
        _check("klr_ctx_create", _lib.klr_ctx_create(ctypes.byref(h), device))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.klr_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, max_fits: int, max_queries: int):
        _check("klr_ctx_reserve", _lib.klr_ctx_reserve(self._h, max_fits, max_queries))

    # -- F1-F4 ---------------------------------------------------------------
    def fit(self, offsets, x, y, *, n_vars, degree, n_scale_log2, b_scale_log2,
            precision=FIT_DF32, refine_iters=0, coef_dtype=None, out=None, stream=None,
            autotune=False, stage=None, var_degree=None):
        """Fit every CSR fit.  offsets: int64 (F+1,); x: (n_vars, S) float32/64
        rows (N, b0, b1[, b2]), or uint8 base-2 logarithms of them (KLR_EXP8,
        y float32), or an int16 (S,) of packed codes log2 N | log2 b0 << 6 |
        log2 b1 << 11 (KLR_EXP16, y float32); y: (S,) same dtype.  Returns (coef, status, diag)
        device tensors; ``out`` may pass preallocated (coef, status, diag).
        autotune=True times the candidate launch shapes first (klr_autotune_fit)
        and records (choice, ms) in ``self.last_tune``.  stage='gram' or
        'solve' runs one stage only (klr_fit_gram / klr_fit_solve).  offsets,
        x and y may be page-locked host tensors (read in place by the
        kernels); the outputs are on the context's device.
        var_degree: per-variable degree bounds of the basis (else the
        total-degree basis of ``degree``)."""
        import torch
        sdt = (F64 if x.dtype == torch.float64 else EXP8 if x.dtype == torch.uint8
               else EXP16 if x.dtype == torch.int16 else F32)
        cdt = (F64 if sdt == F64 else F32) if coef_dtype is None else coef_dtype
        n_fits = offsets.numel() - 1
        m = _n_monomials(n_vars, degree, var_degree)
        if out is None:
            dev = torch.device("cuda", self.device)
            coef = torch.empty((n_fits, 2 * m), device=dev,
                               dtype=torch.float64 if cdt == F64 else torch.float32)
            status = torch.empty(n_fits, device=dev, dtype=torch.int32)
            diag = torch.empty((n_fits, 4), device=dev, dtype=torch.float64)
        else:
            coef, status, diag = out
        b = FitBatch(n_fits, n_vars, degree, n_scale_log2, b_scale_log2, sdt,
                     _iptr(offsets), _iptr(x), x.stride(0), _iptr(y),
                     precision, refine_iters)
        _set_var_degree(b, var_degree)
        if stage == "gram":
            _check("klr_fit_gram", _lib.klr_fit_gram(self._h, ctypes.byref(b), _stream(stream)))
        elif stage == "solve":
            _check("klr_fit_solve", _lib.klr_fit_solve(self._h, ctypes.byref(b), _ptr(coef), cdt,
                                                       _ptr(status), _ptr(diag), _stream(stream)))
        elif stage is not None:
            raise ValueError(f"stage {stage!r} is not 'gram' or 'solve'")
        elif autotune:
            ch, ms = ctypes.c_int32(-1), ctypes.c_float(0.0)
            _check("klr_autotune_fit",
                   _lib.klr_autotune_fit(self._h, ctypes.byref(b), _ptr(coef), cdt, _ptr(status),
                                         _ptr(diag), ctypes.byref(ch), ctypes.byref(ms),
                                         _stream(stream)))
            self.last_tune = (ch.value, ms.value)
        else:
            _check("klr_fit", _lib.klr_fit(self._h, ctypes.byref(b), _ptr(coef), cdt,
                                           _ptr(status), _ptr(diag), _stream(stream)))
        return coef, status, diag

    def fit_heldout(self, offsets, x, y, coef, *, n_vars, degree, n_scale_log2, b_scale_log2,
                    var_degree=None, out=None, stream=None):
        """Per fit, the RMS relative error of coef on the CSR samples
        (klr_fit_heldout); a float64 device tensor."""
        import torch
        sdt = F64 if x.dtype == torch.float64 else F32
        cdt = F64 if coef.dtype == torch.float64 else F32
        n_fits = offsets.numel() - 1
        if out is None:
            out = torch.empty(n_fits, device=x.device, dtype=torch.float64)
        b = FitBatch(n_fits, n_vars, degree, n_scale_log2, b_scale_log2, sdt,
                     _dptr(offsets), _dptr(x), x.stride(0), _dptr(y), FIT_FP64, 0)
        _set_var_degree(b, var_degree)
        _check("klr_fit_heldout", _lib.klr_fit_heldout(self._h, ctypes.byref(b), _ptr(coef), cdt,
                                                       _ptr(out), _stream(stream)))
        return out

    def choose_basis(self, errors, sizes, tol=0.05, floor=1e-6, out=None, stream=None):
        """klr_choose_basis: per fit (row of the float64 device tensor errors,
        one column per candidate basis of sizes[j] monomials) the chosen
        column, -1 when no error is finite; an int32 device tensor."""
        import torch
        n_fits, n_cand = errors.shape
        errors = errors.contiguous()
        sz = np.ascontiguousarray(np.asarray(sizes, dtype=np.int32))
        if out is None:
            out = torch.empty(n_fits, device=errors.device, dtype=torch.int32)
        _check("klr_choose_basis", _lib.klr_choose_basis(self._h, _ptr(errors), sz.ctypes.data_as(_vp),
                                                         n_fits, n_cand, tol, floor, _ptr(out),
                                                         _stream(stream)))
        return out

    def probe_peaks(self, stream=None):
        """klr_probe_peaks: the device's measured arithmetic peaks (a dict of
        10^12 flop/s or operations/s; synchronous)."""
        pk = Peaks()
        _check("klr_probe_peaks", _lib.klr_probe_peaks(self._h, ctypes.byref(pk), _stream(stream)))
        return {name: float(getattr(pk, name)) for name, _ in Peaks._fields_}

    # -- tuned launch shapes -------------------------------------------------
    def tune_export(self):
        """The context's tuned launch shapes: list of (key, choice)."""
        n = ctypes.c_int(0)
        _check("klr_tune_export", _lib.klr_tune_export(self._h, None, None, 0, ctypes.byref(n)))
        keys = np.zeros(n.value, dtype=np.uint64)
        ch = np.zeros(n.value, dtype=np.int32)
        _check("klr_tune_export",
               _lib.klr_tune_export(self._h, keys.ctypes.data_as(_vp), ch.ctypes.data_as(_vp),
                                    n.value, ctypes.byref(n)))
        return [(int(k), int(c)) for k, c in zip(keys, ch)]

    def tune_import(self, pairs):
        """Store (key, choice) pairs, e.g. from an earlier tune_export()."""
        keys = np.ascontiguousarray([k for k, _ in pairs], dtype=np.uint64)
        ch = np.ascontiguousarray([c for _, c in pairs], dtype=np.int32)
        _check("klr_tune_import",
               _lib.klr_tune_import(self._h, keys.ctypes.data_as(_vp), ch.ctypes.data_as(_vp),
                                    len(pairs)))

    # -- E1-E5 ---------------------------------------------------------------
    @staticmethod
    def program(coef, regs, smem, *, n_vars, degree, n_scale_log2, b_scale_log2,
                metric_lo, metric_scale, var_degree=None) -> Program:
        """The rational program of n_kernels x 8 fitted metrics (coef
        n_kernels x 8 x 2m); var_degree: per-variable bounds of the basis."""
        import torch
        p = Program(regs.numel(), n_vars, degree, n_scale_log2, b_scale_log2,
                    F64 if coef.dtype == torch.float64 else F32,
                    _dptr(coef), _dptr(regs), _dptr(smem))
        _set_var_degree(p, var_degree)
        for i in range(8):
            p.metric_lo[i] = float(metric_lo[i])
            p.metric_scale[i] = float(metric_scale[i])
        p._keep = (coef, regs, smem)
        return p

    def eval(self, prog: Program, hw: Hw, cfg, q_offsets, q_N, out_dtype=F32, out=None,
             stream=None):
        """Cycles table (n_queries, n_cfg)."""
        import torch
        n_q = q_N.numel()
        if out is None:
            out = torch.empty((n_q, cfg.shape[0]), device=q_N.device,
                              dtype=torch.float64 if out_dtype == F64 else torch.float32)
        q = Queries(_dptr(q_offsets), _dptr(q_N), n_q)
        _check("klr_eval", _lib.klr_eval(self._h, ctypes.byref(prog), ctypes.byref(hw),
                                         _ptr(cfg), cfg.shape[0], ctypes.byref(q), _ptr(out),
                                         out_dtype, _stream(stream)))
        return out

    def argmin(self, prog: Program, hw: Hw, cfg, q_offsets, q_N, out_dtype=F32, out=None,
               launch=True, stream=None, autotune=False):
        """Per query: (best index, best cycles, margin, status, launch params).
        autotune=True times the candidate launch shapes first
        (klr_autotune_argmin) and records (choice, ms) in ``self.last_tune``.
        q_offsets and q_N may be page-locked host tensors (read in place by the
        kernels); the outputs are on the context's device."""
        import torch
        n_q = q_N.numel()
        dev = torch.device("cuda", self.device)
        if out is None:
            best = torch.empty(n_q, device=dev, dtype=torch.int32)
            cyc = torch.empty(n_q, device=dev,
                              dtype=torch.float64 if out_dtype == F64 else torch.float32)
            margin = torch.empty(n_q, device=dev, dtype=torch.float32)
            status = torch.empty(n_q, device=dev, dtype=torch.int32)
            lp = torch.empty((n_q, 6), device=dev, dtype=torch.int32) if launch else None
        else:
            best, cyc, margin, status, lp = out
        q = Queries(_iptr(q_offsets), _iptr(q_N), n_q)
        if autotune:
            ch, ms = ctypes.c_int32(-1), ctypes.c_float(0.0)
            _check("klr_autotune_argmin",
                   _lib.klr_autotune_argmin(self._h, ctypes.byref(prog), ctypes.byref(hw),
                                            _ptr(cfg), cfg.shape[0], ctypes.byref(q), _ptr(best),
                                            _ptr(cyc), out_dtype, _ptr(margin), _ptr(status),
                                            _ptr(lp), ctypes.byref(ch), ctypes.byref(ms),
                                            _stream(stream)))
            self.last_tune = (ch.value, ms.value)
        else:
            _check("klr_argmin", _lib.klr_argmin(self._h, ctypes.byref(prog), ctypes.byref(hw),
                                                 _ptr(cfg), cfg.shape[0], ctypes.byref(q),
                                                 _ptr(best), _ptr(cyc), out_dtype, _ptr(margin),
                                                 _ptr(status), _ptr(lp), _stream(stream)))
        return best, cyc, margin, status, lp


class History:
    """Runtime history of argmin decisions on the context's device: a hash
    table from (kernel index, N) to the outputs (klr_history_*)."""

    def __init__(self, ctx: "Context", capacity_log2: int = 20):
        self._h = ctypes.c_void_p()
        _check("klr_history_create",
               _lib.klr_history_create(ctx._h, capacity_log2, ctypes.byref(self._h)))

    def clear(self, stream=None):
        _check("klr_history_clear", _lib.klr_history_clear(self._h, _stream(stream)))

    def close(self):
        if self._h:
            _lib.klr_history_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def argmin_history(ctx: "Context", hist: History, prog: Program, hw: Hw, cfg, q_offsets, q_N,
                   out=None, stream=None):
    """FP32 argmin answered from the history where it can be, the rest
    evaluated and recorded (klr_argmin_history).  Returns (best, cycles,
    margin, status, launch)."""
    import torch
    n_q = q_N.numel()
    dev = q_N.device
    if out is None:
        out = (torch.empty(n_q, device=dev, dtype=torch.int32),
               torch.empty(n_q, device=dev, dtype=torch.float32),
               torch.empty(n_q, device=dev, dtype=torch.float32),
               torch.empty(n_q, device=dev, dtype=torch.int32),
               torch.empty((n_q, 6), device=dev, dtype=torch.int32))
    best, cyc, margin, status, lp = out
    q = Queries(_dptr(q_offsets), _dptr(q_N), n_q)
    _check("klr_argmin_history",
           _lib.klr_argmin_history(ctx._h, hist._h, ctypes.byref(prog), ctypes.byref(hw), _ptr(cfg),
                                   cfg.shape[0], ctypes.byref(q), _ptr(best), _ptr(cyc),
                                   _ptr(margin), _ptr(status), _ptr(lp), _stream(stream)))
    return out


def argmin_refined(ctx: "Context", prog: Program, hw: Hw, cfg, q_offsets, q_N, cycles_table,
                   eps: float, out=None, stream=None):
    """Secondary-metric refinement (occupancy) among the configurations
    within (1 + eps) of the least cycles of klr_eval's FP32 table
    (klr_argmin_refined).  Returns (best, cycles, status)."""
    import torch
    n_q = q_N.numel()
    if out is None:
        out = (torch.empty(n_q, dtype=torch.int32, device=q_N.device),
               torch.empty(n_q, dtype=torch.float32, device=q_N.device),
               torch.empty(n_q, dtype=torch.int32, device=q_N.device))
    best, cyc, st = out
    q = Queries(_dptr(q_offsets), _dptr(q_N), n_q)
    _check("klr_argmin_refined",
           _lib.klr_argmin_refined(ctx._h, ctypes.byref(prog), ctypes.byref(hw), _ptr(cfg),
                                   cfg.shape[0], ctypes.byref(q), _ptr(cycles_table), float(eps),
                                   _ptr(best), _ptr(cyc), _ptr(st), _stream(stream)))
    return out


def mlp_param_count(n_coef: int, n_out: int = 0) -> int:
    """Parameters of the surrogate: per-row output (n_out 0) or n_out
    per-query outputs."""
    return int(_lib.klr_mlp_param_count(n_coef, n_out))


class Surrogate:
    """The learned proposer's parameters and optimiser state (device tensors)
    and the calls that train and use it.  ``init`` is the initial FP32
    parameter vector (drawn by the caller's seeded generator).  n_out = 0:
    one output per (kernel, N, shape) row; n_out = |F|: one output per shape
    for a (kernel, N) row (targets n x n_out, non-finite entries masked)."""

    def __init__(self, ctx: "Context", n_coef: int, init, hw_feat, n_out: int = 0):
        import torch
        self.ctx = ctx
        self.n_coef = n_coef
        self.n_out = n_out
        n = mlp_param_count(n_coef, n_out)
        init = torch.as_tensor(init, dtype=torch.float32)
        if init.numel() != n:
            raise ValueError(f"init has {init.numel()} values, the network {n}")
        self.params = init.cuda().contiguous()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.net = MlpNet(n_coef, n_out, _dptr(self.params), _dptr(self.m),
                          _dptr(self.v), 0)
        for i in range(7):
            self.net.hw_feat[i] = float(hw_feat[i])

    @staticmethod
    def _rows(kernel, N, cfg_idx, target=None):
        return MlpRows(kernel.numel(), _dptr(kernel), _dptr(N),
                       None if cfg_idx is None else _dptr(cfg_idx),
                       None if target is None else _dptr(target))

    def train_step(self, coef, cfg, kernel, N, cfg_idx, target, lr, weight_decay=0.0,
                   apply_update=True, loss=None, grads=None, stream=None):
        import torch
        if loss is None:
            loss = torch.zeros(1, dtype=torch.float32, device=coef.device)
        rows = self._rows(kernel, N, cfg_idx, target)
        _check("klr_mlp_train_step",
               _lib.klr_mlp_train_step(self.ctx._h, ctypes.byref(self.net), _ptr(coef), _ptr(cfg),
                                       cfg.shape[0], ctypes.byref(rows), lr, weight_decay,
                                       int(apply_update), _ptr(loss), _ptr(grads),
                                       _stream(stream)))
        return loss

    def predict(self, coef, cfg, kernel, N, cfg_idx, out=None, stream=None):
        import torch
        if out is None:
            shape = (kernel.numel(), self.n_out) if self.n_out else (kernel.numel(),)
            out = torch.empty(shape, dtype=torch.float32, device=coef.device)
        rows = self._rows(kernel, N, cfg_idx)
        _check("klr_mlp_predict",
               _lib.klr_mlp_predict(self.ctx._h, ctypes.byref(self.net), _ptr(coef), _ptr(cfg),
                                    cfg.shape[0], ctypes.byref(rows), _ptr(out), _stream(stream)))
        return out

    def propose(self, coef, regs, smem, hw: Hw, cfg, q_offsets, q_N, k, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((q_N.numel(), k), dtype=torch.int32, device=coef.device)
        q = Queries(_dptr(q_offsets), _dptr(q_N), q_N.numel())
        _check("klr_propose",
               _lib.klr_propose(self.ctx._h, ctypes.byref(self.net), _ptr(coef), _ptr(regs),
                                _ptr(smem), regs.numel(), ctypes.byref(hw), _ptr(cfg),
                                cfg.shape[0], ctypes.byref(q), k, _ptr(out), _stream(stream)))
        return out


def query_targets(cycles, out=None, stream=None):
    """Per-query centred log2 cycles of an FP32 cycles table (n_q, n_cfg);
    NaN where a shape is not meaningful (klr_mlp_query_targets)."""
    import torch
    if out is None:
        out = torch.empty_like(cycles)
    _check("klr_mlp_query_targets",
           _lib.klr_mlp_query_targets(_ptr(cycles), cycles.shape[0], cycles.shape[1], _ptr(out),
                                      _stream(stream)))
    return out


def argmin_candidates(ctx: "Context", prog: Program, hw: Hw, cfg, q_offsets, q_N, cand,
                      out=None, stream=None):
    """Exact re-ranking of candidate shapes (klr_argmin_candidates)."""
    import torch
    n_q = q_N.numel()
    if out is None:
        out = (torch.empty(n_q, dtype=torch.int32, device=q_N.device),
               torch.empty(n_q, dtype=torch.float32, device=q_N.device),
               torch.empty(n_q, dtype=torch.int32, device=q_N.device))
    best, cyc, st = out
    q = Queries(_dptr(q_offsets), _dptr(q_N), n_q)
    _check("klr_argmin_candidates",
           _lib.klr_argmin_candidates(ctx._h, ctypes.byref(prog), ctypes.byref(hw), _ptr(cfg),
                                      cfg.shape[0], ctypes.byref(q), _ptr(cand), cand.shape[1],
                                      _ptr(best), _ptr(cyc), _ptr(st), _stream(stream)))
    return out


def argmin_noalloc(prog: Program, hw: Hw, cfg, q_offsets, q_N, out, stream=None):
    """klr_argmin_noalloc on the current device: FP32 argmin whose scratch is a
    static device array of the library, for callers that cannot allocate device
    memory.  ``out`` = (best int32, cycles float32, margin float32 or None,
    status int32 or None, launch int32 (n, 6) or None), all preallocated."""
    best, cyc, margin, status, lp = out
    q = Queries(_dptr(q_offsets), _dptr(q_N), q_N.numel())
    _check("klr_argmin_noalloc",
           _lib.klr_argmin_noalloc(ctypes.byref(prog), ctypes.byref(hw), _ptr(cfg), cfg.shape[0],
                                   ctypes.byref(q), _ptr(best), _ptr(cyc), _ptr(margin),
                                   _ptr(status), _ptr(lp), _stream(stream)))
    return out


def _n_monomials(n_vars: int, degree: int, var_degree=None) -> int:
    """Basis size: total degree <= degree, or per-variable bounds var_degree."""
    if var_degree is not None and var_degree[0] > 0:
        m = 1
        for v in range(n_vars):
            m *= int(var_degree[v]) + 1
        return m
    from math import comb
    return comb(n_vars + degree, degree)


def _set_var_degree(struct, var_degree):
    for i in range(4):
        struct.var_degree[i] = int(var_degree[i]) if var_degree is not None and i < len(var_degree) else 0
