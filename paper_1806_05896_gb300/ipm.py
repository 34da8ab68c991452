"""Python binding of libipm (include/ipm.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts numpy
arrays / torch CUDA tensors to pointers and C structs. Importing it never
falls back to anything else: if ``libipm.so`` is missing, loading raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Optional, Sequence

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libipm.so")
_lib = None

OK, EINVAL, ENOMEM, ENOTCONV, EBREAKDOWN, ETIMEOUT, ECUDA, ESTATE = range(8)
PREC_FP64, PREC_MIXED = 0, 1
KRYLOV_MINRES_PD, KRYLOV_GMRES_PT = 0, 1
STOP_PAPER, STOP_KKT, STOP_FIXED = 0, 1, 2
POISSON, CONVDIFF_SUPG, HEAT = 0, 1, 2
KINDS = {"poisson": POISSON, "cd": CONVDIFF_SUPG, "heat": HEAT}

HIST_COLS = ("k", "mu", "xi_p", "xi_d", "xi_c", "kkt_rel", "alpha_P", "alpha_D",
             "krylov_iters", "krylov_relres")

EXPORTED = (
    "ipm_default_options", "ipm_create", "ipm_set_stream", "ipm_set_data",
    "ipm_set_data_device", "ipm_solve", "ipm_get_state", "ipm_get_control", "ipm_get_adjoint",
    "ipm_get_state_device", "ipm_get_control_device", "ipm_get_adjoint_device",
    "ipm_get_history", "ipm_destroy", "ipm_launch_count",
    "ipm_profile_smoother", "ipm_profile_read", "ipm_profile_phases", "ipm_profile_kernel",
    "ipm_profile_kernel_read", "ipm_tuning_report", "ipm_tuning_set", "ipm_set_observation",
    "ipm_strerror", "ipm_last_error",
    "ipm_newton_apply_device", "ipm_newton_apply_ff_device", "ipm_precond_apply_device", "ipm_chebyshev_device",
    "ipm_vcycle_device", "ipm_newton_step_device", "ipm_chebyshev_noalloc",
    "ipm_reset", "ipm_device_bytes", "ipm_server_create", "ipm_server_submit",
    "ipm_server_wait", "ipm_server_stats", "ipm_server_destroy",
)


class Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3)]


class Pde(C.Structure):
    _fields_ = [("kind", C.c_int), ("eps", C.c_double), ("wind", C.c_int), ("T", C.c_double)]


class Bounds(C.Structure):
    _fields_ = [("ua", C.c_double), ("ub", C.c_double), ("ya", C.c_double), ("yb", C.c_double),
                ("ua_v", C.POINTER(C.c_double)), ("ub_v", C.POINTER(C.c_double)),
                ("ya_v", C.POINTER(C.c_double)), ("yb_v", C.POINTER(C.c_double))]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("krylov", C.c_int), ("stop", C.c_int),
                ("sigma", C.c_double), ("alpha0", C.c_double), ("eps_p", C.c_double),
                ("eps_d", C.c_double), ("eps_c", C.c_double), ("mu0", C.c_double),
                ("kkt_tol", C.c_double), ("krylov_tol", C.c_double),
                ("cheb_steps", C.c_int), ("vcycles", C.c_int), ("smooth_pre", C.c_int),
                ("smooth_post", C.c_int), ("max_ipm", C.c_int), ("max_krylov", C.c_int),
                ("restart", C.c_int), ("fixed_iters", C.c_int), ("time_limit_s", C.c_double),
                ("common_step", C.c_int), ("mu_rule", C.c_int), ("kernel_flags", C.c_int)]


class Report(C.Structure):
    _fields_ = [("status", C.c_int), ("ipm_iters", C.c_int), ("krylov_iters_total", C.c_int),
                ("kkt_rel", C.c_double), ("xi_p", C.c_double), ("xi_d", C.c_double),
                ("xi_c", C.c_double), ("mu", C.c_double), ("krylov_relres_max", C.c_double),
                ("seconds", C.c_double)]


class Request(C.Structure):
    _fields_ = [("grid", Grid), ("pde", Pde), ("alpha", C.c_double), ("beta", C.c_double),
                ("bounds", Bounds), ("yd", C.POINTER(C.c_double)), ("opt", Options)]


class IpmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libipm error {code}: {msg}")
        self.code = code


def lib_path() -> str:
    return _LIB_PATH


def load() -> C.CDLL:
    """Load libipm.so (built by ``paper_1806_05896_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libipm.so not built ({_LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(_LIB_PATH)
    P = C.c_void_p
    D = C.POINTER(C.c_double)
    lib.ipm_default_options.argtypes = [C.POINTER(Options)]
    lib.ipm_default_options.restype = None
    lib.ipm_create.argtypes = [C.POINTER(Grid), C.POINTER(Pde), C.c_double, C.c_double,
                               C.POINTER(Bounds), C.POINTER(P)]
    lib.ipm_set_stream.argtypes = [P, P]
    lib.ipm_set_data.argtypes = [P, D, D, D]
    lib.ipm_set_data_device.argtypes = [P, P, P, P]
    lib.ipm_solve.argtypes = [P, C.POINTER(Options), C.POINTER(Report)]
    for nm in ("ipm_get_state", "ipm_get_control", "ipm_get_adjoint"):
        getattr(lib, nm).argtypes = [P, D, C.c_size_t]
        getattr(lib, nm + "_device").argtypes = [P, P, C.c_size_t]
    lib.ipm_get_history.argtypes = [P, D, C.c_int, C.POINTER(C.c_int)]
    lib.ipm_destroy.argtypes = [P]
    lib.ipm_destroy.restype = None
    lib.ipm_launch_count.argtypes = []
    lib.ipm_launch_count.restype = C.c_longlong
    lib.ipm_profile_smoother.argtypes = [P, C.c_int, C.c_int]
    lib.ipm_profile_read.argtypes = [P, D, C.POINTER(C.c_longlong), D]
    lib.ipm_profile_phases.argtypes = [P, C.c_int, D, C.POINTER(C.c_longlong), C.c_int]
    lib.ipm_profile_kernel.argtypes = [P, C.c_int, C.c_int, C.c_int]
    lib.ipm_profile_kernel_read.argtypes = [P, D, C.POINTER(C.c_longlong),
                                            C.POINTER(C.c_longlong), D, D]
    lib.ipm_tuning_report.argtypes = [C.c_char_p, C.c_size_t]
    lib.ipm_tuning_report.restype = C.c_int
    lib.ipm_tuning_set.argtypes = [C.c_int, C.c_int, C.c_int]
    lib.ipm_set_observation.argtypes = [P, D, D]
    lib.ipm_strerror.argtypes = [C.c_int]
    lib.ipm_strerror.restype = C.c_char_p
    lib.ipm_last_error.argtypes = [P]
    lib.ipm_last_error.restype = C.c_char_p
    lib.ipm_newton_apply_device.argtypes = [P, P, P, P, P, P]
    lib.ipm_newton_apply_ff_device.argtypes = [P, P, P, P, P, P]
    lib.ipm_precond_apply_device.argtypes = [P, C.POINTER(Options), C.c_int, P, P, P, P, P]
    lib.ipm_chebyshev_device.argtypes = [P, C.c_int, P, P, P]
    lib.ipm_vcycle_device.argtypes = [P, C.POINTER(Options), C.c_int, P, P, P]
    lib.ipm_newton_step_device.argtypes = [P, C.POINTER(Options), C.POINTER(P), C.c_double, P,
                                           C.POINTER(C.c_int), D]
    lib.ipm_chebyshev_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P, P]
    lib.ipm_reset.argtypes = [P, C.c_double, C.c_double, C.POINTER(Bounds)]
    lib.ipm_device_bytes.argtypes = [P]
    lib.ipm_device_bytes.restype = C.c_size_t
    lib.ipm_server_create.argtypes = [C.c_int, C.c_size_t, C.POINTER(P)]
    lib.ipm_server_submit.argtypes = [P, C.POINTER(Request), C.POINTER(C.c_longlong)]
    lib.ipm_server_wait.argtypes = [P, C.c_longlong, C.POINTER(Report), D, C.c_size_t, D, D]
    lib.ipm_server_stats.argtypes = [P, C.POINTER(C.c_size_t), C.POINTER(C.c_int),
                                     C.POINTER(C.c_longlong)]
    lib.ipm_server_destroy.argtypes = [P]
    lib.ipm_server_destroy.restype = None
    _lib = lib
    return lib


def tuning_report() -> str:
    """Tile shapes the autotuner chose so far (one line per kernel and grid size)."""
    lib = load()
    n = lib.ipm_tuning_report(None, 0)
    buf = C.create_string_buffer(n + 1)
    lib.ipm_tuning_report(buf, n + 1)
    return buf.value.decode()


def tuning_set(kernel: int, n: int, shape: int):
    """Pin (shape >= 0) or forget (shape < 0) a tile shape (see ipm_tuning_set)."""
    rc = load().ipm_tuning_set(kernel, n, shape)
    if rc != OK:
        raise IpmError(rc, "unknown kernel or shape")


def launch_count() -> int:
    """Kernel launches enqueued by libipm so far (this process)."""
    return int(load().ipm_launch_count())


def default_options(**kw) -> Options:
    o = Options()
    load().ipm_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _dptr(a) -> int:
    """Device pointer of a contiguous torch CUDA float64 tensor."""
    if a is None:
        return None
    if not (a.is_cuda and a.dtype.is_floating_point and a.element_size() == 8 and a.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return a.data_ptr()


def _hptr(a):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def chebyshev_noalloc(dim: int, n: int, steps: int, th_y, b, x, stream: Optional[int] = None):
    """Allocation-free Chebyshev semi-iteration (fixed device work array, n^dim <= 274625)."""
    rc = load().ipm_chebyshev_noalloc(dim, n, steps, _dptr(th_y), _dptr(b), _dptr(x), stream)
    if rc != OK:
        raise IpmError(rc, load().ipm_strerror(rc).decode())
    return x


class Server:
    """Native serving loop (worker threads, one CUDA stream each, memory-budget admission)."""

    def __init__(self, workers: int = 4, budget_bytes: int = 64 << 30):
        self._lib = load()
        h = C.c_void_p()
        rc = self._lib.ipm_server_create(workers, budget_bytes, C.byref(h))
        if rc != OK:
            raise IpmError(rc, "ipm_server_create failed")
        self._h = h
        self._keep = {}

    def submit(self, dim, n, alpha, beta, ua, ub, yd, ya=-math.inf, yb=math.inf, kind="poisson",
               eps=1.0, options: Optional[Options] = None, **kw) -> int:
        o = options if options is not None else default_options(**kw)
        yd = np.ascontiguousarray(np.asarray(yd, dtype=np.float64).reshape(-1))
        rq = Request(Grid(dim, (C.c_int * 3)(n, n, n if dim == 3 else 0)),
                     Pde(KINDS[kind], eps, 0, 0.0), alpha, beta,
                     Bounds(ua, ub, ya, yb, None, None, None, None),
                     yd.ctypes.data_as(C.POINTER(C.c_double)), o)
        t = C.c_longlong()
        rc = self._lib.ipm_server_submit(self._h, C.byref(rq), C.byref(t))
        if rc != OK:
            raise IpmError(rc, self._lib.ipm_strerror(rc).decode())
        self._keep[t.value] = yd.size
        return t.value

    def wait(self, ticket: int):
        """(report dict, control as a flat array, latency s, queue time s)."""
        nn = self._keep.pop(ticket)
        u = np.empty(nn)
        r = Report()
        lat = C.c_double()
        q = C.c_double()
        rc = self._lib.ipm_server_wait(self._h, ticket, C.byref(r),
                                       u.ctypes.data_as(C.POINTER(C.c_double)), nn, C.byref(lat),
                                       C.byref(q))
        if rc not in (OK, ENOTCONV):
            raise IpmError(rc, self._lib.ipm_strerror(rc).decode())
        return {f: getattr(r, f) for f, _ in Report._fields_}, u, lat.value, q.value

    def stats(self):
        b = C.c_size_t()
        ns = C.c_int()
        done = C.c_longlong()
        self._lib.ipm_server_stats(self._h, C.byref(b), C.byref(ns), C.byref(done))
        return dict(bytes_in_use=b.value, solvers=ns.value, completed=done.value)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ipm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """One problem instance on the current CUDA device (owns its device memory)."""

    def __init__(self, dim: int, n: int, alpha: float, beta: float, ua, ub,
                 ya=-math.inf, yb=math.inf, kind: str = "poisson", eps: float = 1.0,
                 T: float = 1.0):
        lib = load()
        self._lib = lib
        self.dim, self.n = dim, n
        g = Grid(dim, (C.c_int * 3)(n, n, n if dim == 3 else 0))
        pde = Pde(KINDS[kind], eps, 0, T)
        self.nodal_dim = 3 if kind == "heat" else dim
        keep = []

        def bnd(v):
            a = np.asarray(v, dtype=np.float64)
            if a.ndim == 0:
                return float(a), None
            a = np.ascontiguousarray(a.reshape(-1))
            keep.append(a)
            return 0.0, a.ctypes.data_as(C.POINTER(C.c_double))
        (sua, pua), (sub, pub), (sya, pya), (syb, pyb) = bnd(ua), bnd(ub), bnd(ya), bnd(yb)
        b = Bounds(sua, sub, sya, syb, pua, pub, pya, pyb)
        h = C.c_void_p()
        rc = lib.ipm_create(C.byref(g), C.byref(pde), alpha, beta, C.byref(b), C.byref(h))
        if rc != OK:
            raise IpmError(rc, lib.ipm_last_error(None).decode())
        self._h = h

    # ------------------------------------------------------------------
    def _check(self, rc: int, ok=(OK,)):
        if rc not in ok:
            raise IpmError(rc, self._lib.ipm_last_error(self._h).decode())
        return rc

    @property
    def nodes(self) -> int:
        return self.n ** self.nodal_dim

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ipm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def reset(self, alpha: float, beta: float, ua, ub, ya=-math.inf, yb=math.inf):
        b = Bounds(ua, ub, ya, yb, None, None, None, None)
        self._check(self._lib.ipm_reset(self._h, alpha, beta, C.byref(b)))

    def device_bytes(self) -> int:
        return int(self._lib.ipm_device_bytes(self._h))

    def set_stream(self, stream_handle: Optional[int]):
        self._check(self._lib.ipm_set_stream(self._h, stream_handle))

    def set_observation(self, lo=None, hi=None):
        """Observe only the elements whose centre lies in the box lo < x < hi (None: all)."""
        if lo is None:
            self._check(self._lib.ipm_set_observation(self._h, None, None))
            return
        a = (C.c_double * 3)(*[float(v) for v in lo] + [0.0] * (3 - len(lo)))
        b = (C.c_double * 3)(*[float(v) for v in hi] + [0.0] * (3 - len(hi)))
        self._check(self._lib.ipm_set_observation(self._h, a, b))

    def set_data(self, yd=None, f=None, g=None):
        """Host nodal arrays (n^d, C order, x fastest); None = zero."""
        args = [_hptr(a) for a in (yd, f, g)]
        self._check(self._lib.ipm_set_data(self._h, *[a[1] if a else None for a in args]))

    def set_data_device(self, yd=None, f=None, g=None):
        """Torch CUDA float64 tensors of n^d entries; None = zero."""
        self._check(self._lib.ipm_set_data_device(self._h, _dptr(yd), _dptr(f), _dptr(g)))

    def solve(self, options: Optional[Options] = None, **kw) -> dict:
        o = options if options is not None else default_options(**kw)
        r = Report()
        self._check(self._lib.ipm_solve(self._h, C.byref(o), C.byref(r)), ok=(OK, ENOTCONV))
        return {f: getattr(r, f) for f, _ in Report._fields_}

    def _get(self, name: str):
        out = np.empty(self.nodes)
        self._check(getattr(self._lib, name)(self._h, out.ctypes.data_as(C.POINTER(C.c_double)),
                                             out.size))
        return out.reshape((self.n,) * self.nodal_dim)

    def state(self):
        return self._get("ipm_get_state")

    def control(self):
        return self._get("ipm_get_control")

    def adjoint(self):
        return self._get("ipm_get_adjoint")

    def get_device(self, which: str, out):
        nm = {"state": "ipm_get_state_device", "control": "ipm_get_control_device",
              "adjoint": "ipm_get_adjoint_device"}[which]
        self._check(getattr(self._lib, nm)(self._h, _dptr(out), out.numel()))
        return out

    def profile_smoother(self, enable: bool, every: int = 8):
        self._check(self._lib.ipm_profile_smoother(self._h, int(enable), every))

    def profile_read(self):
        ms = C.c_double()
        cnt = C.c_longlong()
        by = C.c_double()
        self._check(self._lib.ipm_profile_read(self._h, C.byref(ms), C.byref(cnt), C.byref(by)))
        return ms.value, cnt.value, by.value

    KERNELS = ("finest_pre_restrict", "finest_prolong_post", "coarse_cycle", "saddle_operator",
               "mid_level_tiles")

    def profile_kernel(self, kind: int, enable: bool, every: int = 4):
        """Sample CUDA-event timings of one kernel (see KERNELS) on the solver's stream."""
        self._check(self._lib.ipm_profile_kernel(self._h, kind, int(enable), every))

    def profile_kernel_read(self) -> dict:
        ms = C.c_double()
        smp = C.c_longlong()
        calls = C.c_longlong()
        bp = C.c_double()
        bo = C.c_double()
        self._check(self._lib.ipm_profile_kernel_read(self._h, C.byref(ms), C.byref(smp),
                                                      C.byref(calls), C.byref(bp), C.byref(bo)))
        return dict(ms=ms.value, sampled=smp.value, calls=calls.value, bytes_pass=bp.value,
                    bytes_once=bo.value)

    PHASES = ("", "chebyshev", "zblock+coupling", "multigrid", "mass_theta+convert",
              "normalise+norm", "newton_operator", "gs_dots", "gs_updates", "mg_fine_pre",
              "mg_fine_post", "mg_mid_levels", "mg_coarse_cta")

    def profile_phases(self, enable: int):
        """Return accumulated per-stage (ms, count) and reset; enable: 1 on, 0 off, -1 keep."""
        ms = (C.c_double * 16)()
        cnt = (C.c_longlong * 16)()
        self._check(self._lib.ipm_profile_phases(self._h, enable, ms, cnt, 16))
        return {nm: (ms[i], cnt[i]) for i, nm in enumerate(self.PHASES) if nm}

    def history(self) -> list:
        nr = C.c_int()
        self._check(self._lib.ipm_get_history(self._h, None, 0, C.byref(nr)))
        buf = np.zeros((max(nr.value, 1), len(HIST_COLS)))
        self._check(self._lib.ipm_get_history(self._h, buf.ctypes.data_as(C.POINTER(C.c_double)),
                                              nr.value, C.byref(nr)))
        return [dict(zip(HIST_COLS, row)) for row in buf[:nr.value]]

    # ------------------------------------------------------------------
    # component entry points (torch CUDA float64 tensors)
    # ------------------------------------------------------------------
    def newton_apply(self, th_y, th_w, th_v, x, out, float_float: bool = False):
        fn = self._lib.ipm_newton_apply_ff_device if float_float else self._lib.ipm_newton_apply_device
        self._check(fn(self._h, _dptr(th_y), _dptr(th_w), _dptr(th_v), _dptr(x), _dptr(out)))
        return out

    def precond_apply(self, triangular: bool, th_y, th_w, th_v, r, z, options=None, **kw):
        o = options if options is not None else default_options(**kw)
        self._check(self._lib.ipm_precond_apply_device(self._h, C.byref(o), int(triangular),
                                                       _dptr(th_y), _dptr(th_w), _dptr(th_v),
                                                       _dptr(r), _dptr(z)))
        return z

    def chebyshev(self, steps: int, th_y, b, x):
        self._check(self._lib.ipm_chebyshev_device(self._h, steps, _dptr(th_y), _dptr(b), _dptr(x)))
        return x

    def vcycle(self, transpose: bool, m, b, x, options=None, **kw):
        o = options if options is not None else default_options(**kw)
        self._check(self._lib.ipm_vcycle_device(self._h, C.byref(o), int(transpose), _dptr(m),
                                                _dptr(b), _dptr(x)))
        return x

    def newton_step(self, iterate: Sequence, mu: float, dx, options=None, **kw):
        o = options if options is not None else default_options(**kw)
        arr = (C.c_void_p * 10)(*[_dptr(a) for a in iterate])
        it = C.c_int()
        rr = C.c_double()
        self._check(self._lib.ipm_newton_step_device(self._h, C.byref(o), arr, mu, _dptr(dx),
                                                     C.byref(it), C.byref(rr)))
        return it.value, rr.value
