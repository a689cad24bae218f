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
CGD, CGD_REDUCED, SENKF = 0, 1, 2
_PREC = {"fp64": FP64, "fp32": FP32, "bf16": BF16_REFINE, "fp16": FP16_REFINE}
_VARIANT = {"cgd": CGD, "reduced": CGD_REDUCED, "senkf": SENKF}

STATUS = {0: "ok", 1: "invalid_arg", 2: "cuda", 3: "oom", 4: "not_converged", 5: "nonfinite",
          6: "breakdown", 7: "timeout", 8: "unsupported"}

# Every symbol include/enkf.h declares (checked by the test suite against the .so).
EXPORTS = (
    "enkf_config_default", "enkf_create", "enkf_analyze", "enkf_analyze_with_E",
    "enkf_analyze_host", "enkf_get_stats", "enkf_get_column_stats", "enkf_copy_intermediates",
    "enkf_draw_perturbations", "enkf_destroy", "enkf_status_str", "enkf_last_error",
    "enkf_set_phase_timing", "enkf_get_phase_times", "enkf_analyze_noalloc", "enkf_create_tridiag",
    "enkf_get_solve_phases", "enkf_batch_create", "enkf_batch_analyze", "enkf_batch_tune",
    "enkf_batch_get_stats", "enkf_batch_get_plan", "enkf_batch_get_row_floors", "enkf_batch_plan",
    "enkf_batch_set_phase_timing",
    "enkf_batch_get_times", "enkf_selftest_wait_timeout",
    "enkf_mlp_param_count", "enkf_mlp_work_bytes", "enkf_mlp_forward", "enkf_mlp_loss_grad",
    "enkf_mlp_adam", "enkf_mlp_train_epoch", "enkf_mlp_standardize", "enkf_warm_features",
    "enkf_set_warm_model",
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
        ("warm_accept", ctypes.c_int32), ("reduce_order", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32), ("iters_max", ctypes.c_int32), ("iters_min", ctypes.c_int32),
        ("refinements", ctypes.c_int32), ("relres_max", ctypes.c_double),
        ("true_relres_max", ctypes.c_double), ("columns_converged", ctypes.c_int32),
        ("grid_blocks", ctypes.c_int32), ("warm_relres_max", ctypes.c_double),
        ("warm_fallbacks", ctypes.c_double), ("reserved", ctypes.c_double * 2),
    ]


class MlpShape(ctypes.Structure):
    _fields_ = [("in_dim", ctypes.c_int32), ("hidden", ctypes.c_int32), ("layers", ctypes.c_int32),
                ("out_dim", ctypes.c_int32)]


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
        "enkf_create_tridiag": (i32, [ctypes.POINTER(Config), vp, vp, vp, vp, vp, vp, ctypes.POINTER(vp)]),
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
        "enkf_batch_create": (i32, [i32, ctypes.POINTER(Config), vp, vp, vp, vp, vp, ctypes.POINTER(vp)]),
        "enkf_batch_analyze": (i32, [vp, vp, vp, vp, vp, vp]),
        "enkf_batch_tune": (i32, [vp, vp, vp, vp, vp, vp, vp]),
        "enkf_batch_get_stats": (i32, [vp, vp, vp, vp, vp]),
        "enkf_batch_get_plan": (i32, [vp, vp, vp, vp, vp]),
        "enkf_batch_get_row_floors": (i32, [vp, vp]),
        "enkf_batch_set_phase_timing": (i32, [vp, i32]),
        "enkf_batch_get_times": (i32, [vp, vp, vp, vp, vp]),
        "enkf_selftest_wait_timeout": (i32, [i32, ctypes.c_double, vp]),
        "enkf_mlp_param_count": (i64, [ctypes.POINTER(MlpShape)]),
        "enkf_mlp_work_bytes": (i64, [ctypes.POINTER(MlpShape), i32]),
        "enkf_mlp_forward": (i32, [ctypes.POINTER(MlpShape), vp, vp, vp, i32, vp, vp, vp]),
        "enkf_mlp_loss_grad": (i32, [ctypes.POINTER(MlpShape), vp, vp, vp, vp, i32, vp, vp, vp, vp]),
        "enkf_mlp_adam": (i32, [i64, vp, vp, vp, vp, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                ctypes.c_float, vp]),
        "enkf_mlp_train_epoch": (i32, [ctypes.POINTER(MlpShape), vp, vp, vp, vp, vp, vp, i64, i32, i32,
                                       ctypes.c_float, vp, vp, vp, vp]),
        "enkf_mlp_standardize": (i32, [ctypes.POINTER(MlpShape), vp, vp, vp, i64, vp]),
        "enkf_warm_features": (i32, [vp, i32, vp, vp]),
        "enkf_set_warm_model": (i32, [vp, ctypes.POINTER(MlpShape), vp]),
        "enkf_batch_plan": (i32, [i32, ctypes.POINTER(Config), i32, ctypes.c_double, vp, vp, vp, vp, vp,
                                  vp, vp, vp]),
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

    def __init__(self, n, m, N, rowptr, col, w, r, stream=None, r_off=None, **config):
        """r: the diagonal of R; r_off (optional, m - 1 entries): the off-diagonal of a
        symmetric tridiagonal R (enkf_create_tridiag)."""
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
        if r_off is None:
            st = lib.enkf_create(ctypes.byref(self.cfg), self._rowptr.ctypes.data, self._col.ctypes.data,
                                 self._w.ctypes.data, self._r.ctypes.data,
                                 ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        else:
            self._r_off = np.ascontiguousarray(r_off, dtype=np.float64)
            st = lib.enkf_create_tridiag(ctypes.byref(self.cfg), self._rowptr.ctypes.data, self._col.ctypes.data,
                                         self._w.ctypes.data, self._r.ctypes.data, self._r_off.ctypes.data,
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
                    grid_blocks=s.grid_blocks, warm_relres_max=s.warm_relres_max,
                    warm_fallbacks=int(s.warm_fallbacks))

    def warm_features(self, K, targets=True):
        """Training pairs of the last analysis: (F [N][K + N], T [N][N] or None), device FP32."""
        import torch
        F = torch.empty((self.N, K + self.N), dtype=torch.float32, device="cuda")
        T = torch.empty((self.N, self.N), dtype=torch.float32, device="cuda") if targets else None
        _check(load().enkf_warm_features(self.h, K, _ptr(F), _ptr(T)), self.h)
        return F, T

    def set_warm_model(self, shape, params):
        """Attach an MLP (shape: MlpShape or (in, hidden, layers, out); params: device FP32,
        kept referenced here) for analyses with warm_start=1; params=None detaches."""
        if not isinstance(shape, MlpShape):
            shape = MlpShape(*shape)
        self._warm_params = params
        _check(load().enkf_set_warm_model(self.h, ctypes.byref(shape), _ptr(params)), self.h)

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

    def intermediates_senkf(self):
        """W = HA^T diag(HA HA^T + R_N)^{-1} D (N x N, FP64 device tensor) of the last sEnKF
        analysis (X_a = X_f + A W)."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        W = torch.empty((self.N, self.N), dtype=torch.float64, device=dev)
        _check(load().enkf_copy_intermediates(self.h, None, None, None, _ptr(W)), self.h)
        self.stream.synchronize()
        return W

    def set_phase_timing(self, enable=True, phases=False):
        _check(load().enkf_set_phase_timing(self.h, (2 if phases else 1) if enable else 0), self.h)

    def solve_phases(self):
        """In-kernel phase timers (us) of the last timed solve: set-up, fused passes, barrier 1,
        reduction, barrier 2, scalars, FP64 refreshes."""
        us = (ctypes.c_double * 8)()
        _check(load().enkf_get_solve_phases(self.h, us), self.h)
        return dict(zip(("setup", "pass", "barrier1", "reduce", "barrier2", "scalars", "refresh"), us[:7]))

    def phase_times(self):
        """(innovations, solve, update) kernel milliseconds of the last timed analysis; for the
        Reduced and sEnKF variants (Gram pass, N x N stage, update)."""
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


def _ptr_array(items, ctype=ctypes.c_void_p):
    arr = (ctype * len(items))()
    for i, x in enumerate(items):
        arr[i] = x
    return arr


def selftest_wait_timeout(which, timeout_ms=50.0, stream=None):
    """Run a bounded device wait that nothing releases (0: grid barrier, 1: mbarrier) with the
    given limit; returns the library status name ("timeout" is the expected outcome)."""
    st = load().enkf_selftest_wait_timeout(int(which), float(timeout_ms), _stream_handle(stream))
    return STATUS.get(st, st)


def batch_plan(shapes, max_grid, alpha=1.0, row_floors=None):
    """The batched launch planner alone (host only): shapes is a list of (n, m, N), alpha the
    team-scaling exponent in (0, 1], row_floors the fewest rows per CTA of a team for N <= 16,
    <= 32, <= 64, <= 128 (None: 64 each). Returns dict(grid, teams, cta_team, cta_rank,
    team_size, team_first, order) as numpy arrays; order[team_first[teams]:] is the queue."""
    import numpy as np
    cfgs = (Config * len(shapes))()
    for i, (n, m, N) in enumerate(shapes):
        cfgs[i].n, cfgs[i].m, cfgs[i].N = n, m, N
    out = {k: np.zeros(max_grid + 1, dtype=np.int32) for k in ("cta_team", "cta_rank", "team_size", "team_first")}
    order = np.zeros(len(shapes), dtype=np.int32)
    grid, teams = ctypes.c_int32(), ctypes.c_int32()
    fl = None if row_floors is None else np.ascontiguousarray(row_floors, dtype=np.int32)
    _check(load().enkf_batch_plan(len(shapes), cfgs, max_grid, alpha, None if fl is None else fl.ctypes.data,
                                  out["cta_team"].ctypes.data,
                                  out["cta_rank"].ctypes.data, out["team_size"].ctypes.data,
                                  out["team_first"].ctypes.data, order.ctypes.data, ctypes.byref(grid),
                                  ctypes.byref(teams)))
    g, t = grid.value, teams.value
    return dict(grid=g, teams=t, cta_team=out["cta_team"][:g], cta_rank=out["cta_rank"][:g],
                team_size=out["team_size"][:t], team_first=out["team_first"][:t + 1], order=order)


class BatchAnalysis:
    """Many problems of uneven (n, m, N) analysed in one persistent launch replayed from a
    CUDA graph (enkf_batch_create / enkf_batch_analyze). problems: list of dicts with n, m, N,
    rowptr, col, w, r (host arrays). FP32 with Jacobi preconditioning."""

    def __init__(self, problems, stream=None, tol=1e-8, perturb_obs=1, grid_blocks=0, **config):
        import numpy as np
        import torch
        if not torch.cuda.is_available():
            raise EnKFError(2, "no CUDA device")
        lib = load()
        self.count = len(problems)
        self.cfgs = (Config * self.count)()
        self._keep = []
        rp, cl, ww, rr = [], [], [], []
        for i, p in enumerate(problems):
            kw = dict(precision=FP32, precondition=1, tol=tol, perturb_obs=perturb_obs, grid_blocks=grid_blocks)
            kw.update(config)
            c = default_config(p["n"], p["m"], p["N"], **kw)
            self.cfgs[i] = c
            arrs = (np.ascontiguousarray(p["rowptr"], dtype=np.int32), np.ascontiguousarray(p["col"], dtype=np.int32),
                    np.ascontiguousarray(p["w"], dtype=np.float64), np.ascontiguousarray(p["r"], dtype=np.float64))
            self._keep.append(arrs)
            rp.append(arrs[0].ctypes.data)
            cl.append(arrs[1].ctypes.data)
            ww.append(arrs[2].ctypes.data)
            rr.append(arrs[3].ctypes.data)
        self.shapes = [(p["n"], p["m"], p["N"]) for p in problems]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = lib.enkf_batch_create(self.count, self.cfgs, _ptr_array(rp), _ptr_array(cl), _ptr_array(ww),
                                   _ptr_array(rr), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        _check(st, None)
        self.h = h

    def _tables(self, Xf, y, seeds, counters, out):
        import torch
        if out is None:
            out = [torch.empty_like(x) for x in Xf]
        tabs = (_ptr_array([x.data_ptr() for x in Xf]), _ptr_array([v.data_ptr() for v in y]),
                _ptr_array([o.data_ptr() for o in out]))
        sd = _ptr_array([int(v) for v in seeds], ctypes.c_uint64) if seeds is not None else None
        ct = _ptr_array([int(v) for v in counters], ctypes.c_uint64) if counters is not None else None
        return out, tabs, sd, ct

    def analyze(self, Xf, y, seeds=None, counters=None, out=None):
        """Xf: list of device FP32 [n_i][N_i]; y: list of device FP64 [m_i]. Returns X_a list."""
        out, (a, b, c), sd, ct = self._tables(Xf, y, seeds, counters, out)
        _check(load().enkf_batch_analyze(self.h, a, b, sd, ct, c), self.h)
        return out

    def tune(self, Xf, y, seeds=None, counters=None, out=None):
        out, (a, b, c), sd, ct = self._tables(Xf, y, seeds, counters, out)
        best = ctypes.c_double()
        _check(load().enkf_batch_tune(self.h, a, b, sd, ct, c, ctypes.byref(best)), self.h)
        return best.value

    def stats(self):
        import numpy as np
        st = np.zeros(self.count, dtype=np.int32)
        it = np.zeros(self.count, dtype=np.int32)
        rel = np.zeros(self.count, dtype=np.float64)
        ref = np.zeros(self.count, dtype=np.int32)
        load().enkf_batch_get_stats(self.h, st.ctypes.data, it.ctypes.data, rel.ctypes.data, ref.ctypes.data)
        return dict(status=st, iters_max=it, relres_max=rel, refinements=ref)

    def plan(self):
        g, t, a, gr = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double(), ctypes.c_int32()
        _check(load().enkf_batch_get_plan(self.h, ctypes.byref(g), ctypes.byref(t), ctypes.byref(a),
                                          ctypes.byref(gr)), self.h)
        fl = (ctypes.c_int32 * 4)()
        _check(load().enkf_batch_get_row_floors(self.h, fl), self.h)
        return dict(grid=g.value, teams=t.value, alpha=a.value, graphed=gr.value, row_floors=list(fl))

    def set_phase_timing(self, enable=True):
        _check(load().enkf_batch_set_phase_timing(self.h, 1 if enable else 0), self.h)

    def times(self, phases=False):
        """When each problem of the last analysis ran: dict(start_us, end_us, team_size[, phase_us
        [count][8] when phases=True, which needs set_phase_timing(True) before the analysis])."""
        import numpy as np
        t0 = np.zeros(self.count)
        t1 = np.zeros(self.count)
        ts = np.zeros(self.count, dtype=np.int32)
        ph = np.zeros((self.count, 8)) if phases else None
        _check(load().enkf_batch_get_times(self.h, t0.ctypes.data, t1.ctypes.data,
                                           ph.ctypes.data if phases else None, ts.ctypes.data), self.h)
        out = dict(start_us=t0, end_us=t1, team_size=ts)
        if phases:
            out["phase_us"] = ph
        return out

    def close(self):
        if getattr(self, "h", None):
            load().enkf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- learned warm start (MLP)
def _shape(shape):
    return shape if isinstance(shape, MlpShape) else MlpShape(*shape)


def mlp_param_count(shape):
    """Total FP32 parameters of the layout; the trained prefix is this minus 2 (in + out)."""
    return int(load().enkf_mlp_param_count(ctypes.byref(_shape(shape))))


def mlp_trained_count(shape):
    s = _shape(shape)
    return mlp_param_count(s) - 2 * (s.in_dim + s.out_dim)


def _work(shape, batch):
    import torch
    nb = int(load().enkf_mlp_work_bytes(ctypes.byref(_shape(shape)), batch))
    if nb < 0:
        raise EnKFError(1, "bad MLP shape or batch")
    return torch.empty(nb, dtype=torch.uint8, device="cuda")


def mlp_forward(shape, params, X, rows=None, stream=None):
    """Raw predictions Y [batch][out] for rows X (or X[rows]), device FP32."""
    import torch
    s = _shape(shape)
    B = rows.numel() if rows is not None else X.shape[0]
    Y = torch.empty((B, s.out_dim), dtype=torch.float32, device="cuda")
    work = _work(s, B)
    _check(load().enkf_mlp_forward(ctypes.byref(s), _ptr(params), _ptr(X), _ptr(rows), B, _ptr(Y), _ptr(work),
                                   _stream_handle(stream)))
    return Y


def mlp_loss_grad(shape, params, X, T, rows=None, stream=None):
    """(loss tensor [1], gradient [param_count]) of the standardised MSE on a minibatch."""
    import torch
    s = _shape(shape)
    B = rows.numel() if rows is not None else X.shape[0]
    grad = torch.zeros(mlp_param_count(s), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    work = _work(s, B)
    _check(load().enkf_mlp_loss_grad(ctypes.byref(s), _ptr(params), _ptr(X), _ptr(T), _ptr(rows), B, _ptr(grad),
                                     _ptr(loss), _ptr(work), _stream_handle(stream)))
    return loss, grad


def mlp_adam(count, params, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(load().enkf_mlp_adam(count, _ptr(params), _ptr(grad), _ptr(m), _ptr(v), step, lr, beta1, beta2, eps,
                                _stream_handle(stream)))


def mlp_standardize(shape, params, X, T, stream=None):
    _check(load().enkf_mlp_standardize(ctypes.byref(_shape(shape)), _ptr(params), _ptr(X), _ptr(T), X.shape[0],
                                       _stream_handle(stream)))


def mlp_train_epoch(shape, params, m, v, X, T, perm, batch, step0, lr, stream=None):
    """One epoch of minibatch Adam over rows perm (device int32); returns per-batch losses."""
    import torch
    s = _shape(shape)
    rows = perm.numel()
    losses = torch.zeros(rows // batch, dtype=torch.float32, device="cuda")
    grad = torch.zeros(mlp_param_count(s), dtype=torch.float32, device="cuda")
    work = _work(s, batch)
    _check(load().enkf_mlp_train_epoch(ctypes.byref(s), _ptr(params), _ptr(m), _ptr(v), _ptr(X), _ptr(T),
                                       _ptr(perm), rows, batch, step0, lr, _ptr(losses), _ptr(grad), _ptr(work),
                                       _stream_handle(stream)))
    return losses
