"""Python binding of libenkf.so, the GB300 CGD-EnKF analysis-step library.

Argument marshalling only: every step of the analysis runs in the library's CUDA kernels.
PyTorch supplies device memory and the stream; tensors are passed to the C ABI
(include/enkf.h) as raw pointers. There is no CPU fallback: if the library cannot be built
or loaded, or no CUDA device is present, calls raise.
"""
import ctypes
import os

from .build import LIB, build, up_to_date

FP64, FP32, BF16_REFINE, FP16_REFINE = 0, 1, 2, 3
CGD, CGD_REDUCED = 0, 1
_PREC = {"fp64": FP64, "fp32": FP32, "bf16": BF16_REFINE, "fp16": FP16_REFINE}
_VARIANT = {"cgd": CGD, "reduced": CGD_REDUCED}

STATUS = {0: "ok", 1: "invalid_arg", 2: "cuda", 3: "oom", 4: "not_converged", 5: "nonfinite",
          6: "breakdown", 7: "timeout", 8: "unsupported"}

# Every symbol include/enkf.h declares (checked by the test suite against the .so).
EXPORTS = (
    "enkf_config_default", "enkf_create", "enkf_analyze", "enkf_analyze_with_E",
    "enkf_analyze_host", "enkf_get_stats", "enkf_get_column_stats", "enkf_copy_intermediates",
    "enkf_draw_perturbations", "enkf_destroy", "enkf_status_str", "enkf_last_error",
    "enkf_set_phase_timing", "enkf_get_phase_times", "enkf_analyze_noalloc",
    "enkf_get_solve_phases",
)


class Config(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("m", ctypes.c_int64), ("N", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("variant", ctypes.c_int32), ("max_iter", ctypes.c_int32),
        ("tol", ctypes.c_double), ("fixed_iters", ctypes.c_int32), ("max_refine", ctypes.c_int32),
        ("inner_tol", ctypes.c_double), ("refresh_every", ctypes.c_int32),
        ("perturb_obs", ctypes.c_int32), ("warm_start", ctypes.c_int32),
        ("true_residual", ctypes.c_int32), ("grid_blocks", ctypes.c_int32),
        ("precondition", ctypes.c_int32), ("lowprec_terms", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 5),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32), ("iters_max", ctypes.c_int32), ("iters_min", ctypes.c_int32),
        ("refinements", ctypes.c_int32), ("relres_max", ctypes.c_double),
        ("true_relres_max", ctypes.c_double), ("columns_converged", ctypes.c_int32),
        ("grid_blocks", ctypes.c_int32), ("reserved", ctypes.c_double * 4),
    ]


class EnKFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str = None):
    """Load libenkf.so (building it first if it is missing or stale) and declare the
    signatures. Returns the ctypes library."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        if not up_to_date():
            build()
        path = LIB
    lib = ctypes.CDLL(path)
    vp, i32, i64, u64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
    sig = {
        "enkf_config_default": (i32, [ctypes.POINTER(Config), i64, i64, i32]),
        "enkf_create": (i32, [ctypes.POINTER(Config), vp, vp, vp, vp, vp, ctypes.POINTER(vp)]),
        "enkf_analyze": (i32, [vp, vp, dp, u64, u64, vp]),
        "enkf_analyze_with_E": (i32, [vp, vp, dp, dp, vp]),
        "enkf_analyze_host": (i32, [vp, vp, dp, u64, u64, vp]),
        "enkf_get_stats": (i32, [vp, ctypes.POINTER(Stats)]),
        "enkf_get_column_stats": (i32, [vp, vp, vp, vp]),
        "enkf_copy_intermediates": (i32, [vp, dp, dp, dp, dp]),
        "enkf_draw_perturbations": (i32, [u64, u64, dp, i64, i32, dp, vp]),
        "enkf_destroy": (i32, [vp]),
        "enkf_status_str": (ctypes.c_char_p, [i32]),
        "enkf_last_error": (ctypes.c_char_p, [vp]),
        "enkf_set_phase_timing": (i32, [vp, i32]),
        "enkf_get_phase_times": (i32, [vp, vp]),
        "enkf_get_solve_phases": (i32, [vp, vp]),
        "enkf_analyze_noalloc": (i32, [ctypes.POINTER(Config), vp, vp, vp, vp, vp, dp, u64, u64,
                                       vp, vp, ctypes.POINTER(Stats)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(status, handle=None):
    if status != 0:
        msg = load().enkf_last_error(handle).decode(errors="replace")
        raise EnKFError(status, msg)


def default_config(n, m, N, **kw) -> Config:
    cfg = Config()
    _check(load().enkf_config_default(ctypes.byref(cfg), n, m, N))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = _PREC[v]
        if k == "variant" and isinstance(v, str):
            v = _VARIANT[v]
        setattr(cfg, k, v)
    return cfg


class Analysis:
    """One problem shape (n, m, N, H, R) bound to a stream. Wraps enkf_create / enkf_destroy;
    analyze* enqueue one analysis step on the stream."""

    def __init__(self, n, m, N, rowptr, col, w, r, stream=None, **config):
        import numpy as np
        import torch
        if not torch.cuda.is_available():
            raise EnKFError(2, "no CUDA device")
        lib = load()
        self.cfg = default_config(n, m, N, **config)
        self._rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        self._col = np.ascontiguousarray(col, dtype=np.int32)
        self._w = np.ascontiguousarray(w, dtype=np.float64)
        self._r = np.ascontiguousarray(r, dtype=np.float64)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = lib.enkf_create(ctypes.byref(self.cfg), self._rowptr.ctypes.data, self._col.ctypes.data,
                             self._w.ctypes.data, self._r.ctypes.data,
                             ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        _check(st, None)
        self.h = h
        self.n, self.m, self.N = n, m, N
        self.dtype = torch.float64 if self.cfg.precision == FP64 else torch.float32

    def _out(self, Xf, out):
        import torch
        return torch.empty_like(Xf) if out is None else out

    def analyze(self, Xf, y, seed=0, counter=0, out=None):
        out = self._out(Xf, out)
        _check(load().enkf_analyze(self.h, _ptr(Xf), _ptr(y), seed, counter, _ptr(out)), self.h)
        return out

    def analyze_with_E(self, Xf, y, E=None, out=None):
        out = self._out(Xf, out)
        _check(load().enkf_analyze_with_E(self.h, _ptr(Xf), _ptr(y), _ptr(E), _ptr(out)), self.h)
        return out

    def analyze_host(self, Xf, y, seed=0, counter=0, out=None):
        """Host tensors in and out (copies inside the library call)."""
        import torch
        if out is None:
            out = torch.empty_like(Xf)
        _check(load().enkf_analyze_host(self.h, _ptr(Xf), _ptr(y), seed, counter, _ptr(out)), self.h)
        return out

    def stats(self, raise_on_error=False):
        s = Stats()
        st = load().enkf_get_stats(self.h, ctypes.byref(s))
        if raise_on_error:
            _check(st, self.h)
        return dict(status=STATUS.get(s.status, s.status), iters_max=s.iters_max,
                    iters_min=s.iters_min, refinements=s.refinements, relres_max=s.relres_max,
                    true_relres_max=s.true_relres_max, columns_converged=s.columns_converged,
                    grid_blocks=s.grid_blocks)

    def column_stats(self):
        import numpy as np
        it = np.zeros(self.N, np.int32)
        rel = np.zeros(self.N)
        tr = np.zeros(self.N)
        _check(load().enkf_get_column_stats(self.h, it.ctypes.data, rel.ctypes.data, tr.ctypes.data), self.h)
        return it, rel, tr

    def intermediates(self):
        """(HA, D, Z, W) of the last analysis as FP64 device tensors."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        HA = torch.empty((self.m, self.N), dtype=torch.float64, device=dev)
        D = torch.empty_like(HA)
        Z = torch.empty_like(HA)
        W = torch.empty((self.N, self.N), dtype=torch.float64, device=dev)
        _check(load().enkf_copy_intermediates(self.h, _ptr(HA), _ptr(D), _ptr(Z), _ptr(W)), self.h)
        self.stream.synchronize()
        return HA, D, Z, W

    def intermediates_reduced(self):
        """(V, G) of the last CGD-EnKF-Reduced analysis as FP64 device tensors (N x N)."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        V = torch.empty((self.N, self.N), dtype=torch.float64, device=dev)
        G = torch.empty_like(V)
        _check(load().enkf_copy_intermediates(self.h, None, None, _ptr(V), _ptr(G)), self.h)
        self.stream.synchronize()
        return V, G

    def set_phase_timing(self, enable=True, phases=False):
        _check(load().enkf_set_phase_timing(self.h, (2 if phases else 1) if enable else 0), self.h)

    def solve_phases(self):
        """In-kernel phase timers (us) of the last timed solve: set-up, fused passes, barrier 1,
        reduction, barrier 2, scalars, FP64 refreshes."""
        us = (ctypes.c_double * 8)()
        _check(load().enkf_get_solve_phases(self.h, us), self.h)
        return dict(zip(("setup", "pass", "barrier1", "reduce", "barrier2", "scalars", "refresh"), us[:7]))

    def phase_times(self):
        """(innovations, solve, update) kernel milliseconds of the last timed analysis."""
        ms = (ctypes.c_float * 3)()
        _check(load().enkf_get_phase_times(self.h, ms), self.h)
        return tuple(ms)

    def close(self):
        if getattr(self, "h", None):
            load().enkf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def draw_perturbations(seed, counter, r, N, stream=None):
    """E [m][N] (FP64, device) exactly as enkf_analyze draws it; r is a device FP64 tensor."""
    import torch
    E = torch.empty((r.shape[0], N), dtype=torch.float64, device=r.device)
    _check(load().enkf_draw_perturbations(seed, counter, _ptr(r), r.shape[0], N, _ptr(E),
                                          _stream_handle(stream)))
    return E


def analyze_noalloc(cfg, rowptr, col, w, r, Xf, y, seed=0, counter=0, out=None, stream=None):
    """One analysis through enkf_analyze_noalloc, which allocates no device memory (for
    callers that must not allocate, e.g. inside stream capture). rowptr, col, w, r are
    DEVICE tensors (int32, int32, float64, float64); returns (X_a, stats dict)."""
    import torch
    if out is None:
        out = torch.empty_like(Xf)
    s = Stats()
    st = load().enkf_analyze_noalloc(ctypes.byref(cfg), _ptr(rowptr), _ptr(col), _ptr(w), _ptr(r),
                                     _ptr(Xf), _ptr(y), seed, counter, _ptr(out),
                                     _stream_handle(stream), ctypes.byref(s))
    return out, dict(status=STATUS.get(st, st), iters_max=s.iters_max, refinements=s.refinements,
                     true_relres_max=s.true_relres_max, grid_blocks=s.grid_blocks)
