"""Thin ctypes binding of libpdg.so (include/pdg.h).  Argument marshalling only.

Every function of the C ABI is exposed under the same name with the same
arguments (pointers given as integers, numpy arrays or torch tensors).  The
class :class:`Solver` is a small convenience wrapper used by the tests and
``bench.py``.  There is no CPU fallback: importing this module raises if the
CUDA library has not been built (``__graft_entry__.build()``).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libpdg.so")

PDG_OK = 0
PDG_ERR_ARG, PDG_ERR_OOM, PDG_ERR_CUDA, PDG_ERR_STATE, PDG_ERR_TIMEOUT, PDG_ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6
PDG_MODEL_ADVECTION, PDG_MODEL_SHALLOW_WATER, PDG_MODEL_EULER = 0, 1, 2
PDG_MODEL_ISOTHERMAL_D2Q9, PDG_MODEL_ISOTHERMAL_D3Q19 = 3, 4
PDG_MODEL_ISOTHERMAL_D3Q15, PDG_MODEL_ISOTHERMAL_D3Q27 = 5, 6
PDG_SCHEME_M2, PDG_SCHEME_M2_COLLAPSED, PDG_SCHEME_M2KIN, PDG_SCHEME_M4KIN = 0, 1, 2, 3
PDG_PREC_FP64 = 0
PDG_PREC_DF32 = 1
PDG_PREC_TF32 = 2
PDG_PREC_TF32_DFRES = 3
PRECISION = {"fp64": PDG_PREC_FP64, "df32": PDG_PREC_DF32, "tf32": PDG_PREC_TF32, "tf32_df": PDG_PREC_TF32_DFRES}
PDG_OPT_COMPOSE_TT = 1
PDG_OPT_GRAPH = 2
PDG_OPT_DEBUG_TC_STALL = 3
PDG_OPT_RESIDENT = 4
PDG_OPT_COLLISION_AXIS = 5
PDG_OPT_TC_LAYERS = 6
PDG_OPT_CORNER_SWEEP = 7

KIND = {"advection": PDG_MODEL_ADVECTION, "shallow_water": PDG_MODEL_SHALLOW_WATER, "euler": PDG_MODEL_EULER,
        "isothermal_d2q9": PDG_MODEL_ISOTHERMAL_D2Q9, "isothermal_d3q19": PDG_MODEL_ISOTHERMAL_D3Q19,
        "isothermal_d3q15": PDG_MODEL_ISOTHERMAL_D3Q15, "isothermal_d3q27": PDG_MODEL_ISOTHERMAL_D3Q27}
SCHEME = {"M2": PDG_SCHEME_M2, "M2_collapsed": PDG_SCHEME_M2_COLLAPSED, "M2_kin": PDG_SCHEME_M2KIN,
          "M4_kin": PDG_SCHEME_M4KIN}


class pdg_model_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("scheme", ctypes.c_int), ("precision", ctypes.c_int),
                ("reserved", ctypes.c_int), ("lambda_", ctypes.c_double), ("a", ctypes.c_double * 3),
                ("gravity", ctypes.c_double), ("gamma", ctypes.c_double), ("omega", ctypes.c_double),
                ("theta", ctypes.c_double)]


PDG_SOURCE_GRAVITY, PDG_SOURCE_PENALIZATION = 1, 2


class pdg_source_desc(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_int), ("reserved", ctypes.c_int), ("gravity", ctypes.c_double * 3),
                ("K_s", ctypes.c_double), ("kappa", ctypes.c_double), ("x_c", ctypes.c_double * 3),
                ("w_s", ctypes.c_double * 5), ("theta", ctypes.c_double)]


class pdg_info(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("order", ctypes.c_int), ("m", ctypes.c_int), ("nv", ctypes.c_int),
                ("ncell", ctypes.c_int * 3), ("npts", ctypes.c_int * 3), ("npoints", ctypes.c_longlong),
                ("nfields", ctypes.c_longlong), ("w_len", ctypes.c_longlong), ("f_len", ctypes.c_longlong),
                ("h", ctypes.c_double * 3)]


class pdg_request(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_macro", ctypes.c_int * 3), ("n_sub", ctypes.c_int * 3),
                ("order", ctypes.c_int), ("model", pdg_model_desc), ("dt", ctypes.c_double),
                ("nsteps", ctypes.c_int), ("reserved", ctypes.c_int), ("w0", ctypes.c_void_p),
                ("w0_len", ctypes.c_size_t), ("t_arrival", ctypes.c_double)]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libpdg.so not built at {LIB_PATH}; run __graft_entry__.build()")
lib = ctypes.CDLL(LIB_PATH)

_P = ctypes.c_void_p
_I = ctypes.c_int
_SZ = ctypes.c_size_t
_D = ctypes.c_double
_SIGS = {
    "pdg_create_mesh": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_I), ctypes.POINTER(_I), _I,
                             ctypes.POINTER(_D), ctypes.c_uint, _P]),
    "pdg_set_model": (_I, [_P, ctypes.POINTER(pdg_model_desc)]),
    "pdg_set_w": (_I, [_P, _P, _SZ, _I]),
    "pdg_step": (_I, [_P, _D, _I]),
    "pdg_set_source": (_I, [_P, _P]),
    "pdg_get_w": (_I, [_P, _P, _SZ, _I]),
    "pdg_get_f": (_I, [_P, _P, _SZ, _I]),
    "pdg_set_f": (_I, [_P, _P, _SZ, _I]),
    "pdg_get_points": (_I, [_P, _I, _P, _SZ]),
    "pdg_set_inflow": (_I, [_P, _I, _P, _SZ, _I]),
    "pdg_get_info": (_I, [_P, ctypes.POINTER(pdg_info)]),
    "pdg_get_line_coefs": (_I, [_P, _I, _D, _P, _P, _P]),
    "pdg_get_schedule": (_I, [_P, _D, _I, _P, _P, _I, _P]),
    "pdg_get_w_noalloc": (_I, [_P, _P, _SZ]),
    "pdg_synchronize": (_I, [_P]),
    "pdg_timing_enable": (_I, [_P, _I]),
    "pdg_timing_read": (_I, [_P, _P, _P, _I]),
    "pdg_set_launch": (_I, [_P, _I, _I, _I, _I]),
    "pdg_get_launch": (_I, [_P, _I, _P, _P, _P]),
    "pdg_set_option": (_I, [_P, _I, _I]),
    "pdg_autotune": (_I, [_P, _D, _I]),
    "pdg_batch_create": (_I, [ctypes.POINTER(_P), _I, _P, _P]),
    "pdg_batch_step": (_I, [_P, _P, _P, _I]),
    "pdg_batch_elapsed": (_I, [_P, _P, _P]),
    "pdg_batch_autotune": (_I, [_P, _P, _I]),
    "pdg_batch_destroy": (_I, [_P]),
    "pdg_batch_last_error": (ctypes.c_char_p, [_P]),
    "pdg_server_create": (_I, [ctypes.POINTER(_P), _SZ, _I, _I, _P]),
    "pdg_server_now": (_D, [_P]),
    "pdg_server_submit": (_I, [_P, ctypes.POINTER(pdg_request), _P]),
    "pdg_server_iterate": (_I, [_P, _P, _P]),
    "pdg_server_pending": (_I, [_P, _P, _P]),
    "pdg_server_poll": (_I, [_P, _P, _P, _P, _P, _I, _P]),
    "pdg_server_result": (_I, [_P, ctypes.c_longlong, _P, _SZ]),
    "pdg_server_cancel": (_I, [_P, ctypes.c_longlong]),
    "pdg_server_stats": (_I, [_P, _P, _P, _P, _P]),
    "pdg_server_destroy": (_I, [_P]),
    "pdg_server_last_error": (ctypes.c_char_p, [_P]),
    "pdg_debug_fail_allocs": (_I, [_I]),
    "pdg_measure_fma_peak": (_I, [_I, _P, _P, _P]),
    "pdg_plan_sweep": (_I, [_I, _I, _P, _D, _P, _P]),
    "pdg_plan_line": (_I, [_I, _D, _D, _P, _P, _P, _P]),
    "pdg_destroy": (_I, [_P]),
    "pdg_last_error": (ctypes.c_char_p, [_P]),
    "pdg_status_string": (ctypes.c_char_p, [_I]),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args
    globals()[_name] = _fn

EXPORTED = tuple(_SIGS)


def measure_fma_peak(fp64=True, stream=None):
    """pdg_measure_fma_peak: (TFLOP/s, kernel ms) of a multiply-add throughput kernel on the
    current device, FP64 (fp64=True) or FP32."""
    t = ctypes.c_double(0.0)
    ms = ctypes.c_double(0.0)
    st = pdg_measure_fma_peak(1 if fp64 else 0, ctypes.addressof(t), ctypes.addressof(ms), stream)
    if st != PDG_OK:
        raise PdgError(st, "pdg_measure_fma_peak")
    return t.value, ms.value


class PdgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{pdg_status_string(status).decode()}: {msg}")
        self.status = status


def plan_line(d, nu, theta=0.5):
    """pdg_plan_line: dict with E, q, beta, za, zb, gamma1, W, W2 of the line plan."""
    n = d + 1
    E = np.zeros((n, n))
    q = np.zeros(n)
    sc = np.zeros(4)
    win = (ctypes.c_int * 2)()
    st = pdg_plan_line(d, nu, theta, E.ctypes.data, q.ctypes.data, sc.ctypes.data, ctypes.addressof(win))
    if st != PDG_OK:
        raise PdgError(st, f"pdg_plan_line(d={d}, nu={nu}, theta={theta})")
    return {"E": E, "q": q, "beta": sc[0], "za": sc[1], "zb": sc[2], "gamma1": sc[3], "W": win[0], "W2": win[1]}


def plan_sweep(d, nu, theta=0.5):
    """pdg_plan_sweep: (widths, binv) of the tile (len(nu) == 2) or box (len(nu) == 3) sweep."""
    nu = np.ascontiguousarray(nu, dtype=np.float64)
    nc = nu.size
    widths = (ctypes.c_int * nc)()
    nn = (d + 1) ** nc
    binv = np.zeros((nn, nn))
    st = pdg_plan_sweep(nc, d, nu.ctypes.data, theta, ctypes.addressof(widths), binv.ctypes.data)
    if st != PDG_OK:
        raise PdgError(st, f"pdg_plan_sweep(ncomp={nc}, d={d}, nu={nu.tolist()}, theta={theta})")
    return list(widths), binv


def _ptr(x, want_device):
    """(pointer, on_device, length) of a numpy array or torch tensor (FP64, contiguous)."""
    if isinstance(x, np.ndarray):
        if want_device is True:
            raise ValueError("numpy array given where a device buffer is required")
        if x.dtype != np.float64 or not x.flags.c_contiguous:
            raise ValueError("numpy buffers must be contiguous float64")
        return x.ctypes.data, 0, x.size
    import torch  # device memory and streams come from torch

    if not isinstance(x, torch.Tensor):
        raise TypeError(type(x))
    if x.dtype != torch.float64 or not x.is_contiguous():
        raise ValueError("tensors must be contiguous float64")
    return x.data_ptr(), 1 if x.is_cuda else 0, x.numel()


class Solver:
    """Owns one pdg_ctx.  Methods map one-to-one onto the C ABI."""

    def __init__(self, dim, n_macro, n_sub, order, lengths=None, stream=None, periodic=None):
        self.ctx = _P()
        nm = (_I * 3)(*(list(n_macro) + [1] * (3 - len(n_macro))))
        ns = (_I * 3)(*(list(n_sub) + [1] * (3 - len(n_sub))))
        ln = None if lengths is None else (_D * 3)(*(list(lengths) + [1.0] * (3 - len(lengths))))
        st = _P(stream) if stream else None
        mask = (1 << dim) - 1 if periodic is None else sum(1 << a for a in range(dim) if periodic[a])
        r = pdg_create_mesh(ctypes.byref(self.ctx), dim, nm, ns, order, ln, mask, st)
        if r != PDG_OK:
            raise PdgError(r, "pdg_create_mesh")
        self.dim = dim

    def _check(self, r, what):
        if r != PDG_OK:
            raise PdgError(r, f"{what}: {pdg_last_error(self.ctx).decode()}")

    def close(self):
        if self.ctx:
            pdg_destroy(self.ctx)
            self.ctx = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        i = pdg_info()
        self._check(pdg_get_info(self.ctx, ctypes.byref(i)), "pdg_get_info")
        return i

    def set_model(self, kind, lam, a=(0.0, 0.0, 0.0), gravity=9.81, gamma=1.4, omega=2.0, theta=0.5,
                  scheme="M2", precision=PDG_PREC_FP64):
        d = pdg_model_desc()
        d.kind = KIND[kind] if isinstance(kind, str) else int(kind)
        d.scheme = SCHEME[scheme] if isinstance(scheme, str) else int(scheme)
        d.precision = precision
        d.lambda_ = lam
        for i in range(3):
            d.a[i] = float(a[i]) if i < len(a) else 0.0
        d.gravity, d.gamma, d.omega, d.theta = gravity, gamma, omega, theta
        self._check(pdg_set_model(self.ctx, ctypes.byref(d)), "pdg_set_model")

    def points(self, axis):
        n = self.info().npts[axis]
        out = np.empty(n, dtype=np.float64)
        self._check(pdg_get_points(self.ctx, axis, out.ctypes.data, n), "pdg_get_points")
        return out

    def set_w(self, w):
        p, dev, n = _ptr(w, None)
        self._check(pdg_set_w(self.ctx, p, n, dev), "pdg_set_w")

    def set_inflow(self, axis, fb):
        p, dev, n = _ptr(fb, None)
        self._check(pdg_set_inflow(self.ctx, axis, p, n, dev), "pdg_set_inflow")

    def set_f(self, f):
        p, dev, n = _ptr(f, None)
        self._check(pdg_set_f(self.ctx, p, n, dev), "pdg_set_f")

    def step(self, dt, nsteps):
        self._check(pdg_step(self.ctx, dt, nsteps), "pdg_step")

    def set_source(self, gravity=None, K_s=None, kappa=0.0, x_c=(0.0, 0.0), w_s=(1.0, 0.0, 0.0), theta=0.5):
        """Gravity vector and/or penalisation (K_s, kappa, x_c, w_s); no argument removes it."""
        d = pdg_source_desc()
        d.flags = (PDG_SOURCE_GRAVITY if gravity is not None else 0) | \
                  (PDG_SOURCE_PENALIZATION if K_s is not None else 0)
        for i in range(3):
            d.gravity[i] = float(gravity[i]) if gravity is not None and i < len(gravity) else 0.0
            d.x_c[i] = float(x_c[i]) if i < len(x_c) else 0.0
        for i in range(5):
            d.w_s[i] = float(w_s[i]) if i < len(w_s) else 0.0
        d.K_s = float(K_s or 0.0)
        d.kappa = float(kappa)
        d.theta = float(theta)
        self._check(pdg_set_source(self.ctx, ctypes.byref(d)), "pdg_set_source")

    def get_w(self, out=None):
        i = self.info()
        if out is None:
            out = np.empty(i.w_len, dtype=np.float64)
        p, dev, n = _ptr(out, None)
        self._check(pdg_get_w(self.ctx, p, n, dev), "pdg_get_w")
        return out

    def get_f(self, out=None):
        i = self.info()
        if out is None:
            out = np.empty(i.f_len, dtype=np.float64)
        p, dev, n = _ptr(out, None)
        self._check(pdg_get_f(self.ctx, p, n, dev), "pdg_get_f")
        return out

    def line_coefs(self, axis, delta):
        n = self.info().order + 1
        E = np.empty(n * n)
        q = np.empty(n)
        b = np.empty(1)
        self._check(pdg_get_line_coefs(self.ctx, axis, delta, E.ctypes.data, q.ctypes.data, b.ctypes.data),
                    "pdg_get_line_coefs")
        return E.reshape(n, n), q, float(b[0])

    def schedule(self, dt, nsteps):
        """pdg_get_schedule: list of passes, each a dict (kind, axis, ops, fingerprints of the
        transports' line plans as (E00, beta), slot, diagonal sub-step, source sub-step)."""
        cnt = ctypes.c_int(0)
        self._check(pdg_get_schedule(self.ctx, dt, nsteps, None, None, 0, ctypes.byref(cnt)), "pdg_get_schedule")
        n = cnt.value
        ints = np.zeros(8 * max(n, 1), dtype=np.int32)
        dbls = np.zeros(10 * max(n, 1))
        self._check(pdg_get_schedule(self.ctx, dt, nsteps, ints.ctypes.data, dbls.ctypes.data, n,
                                     ctypes.byref(cnt)), "pdg_get_schedule")
        out = []
        for i in range(n):
            I, X = ints[8 * i:8 * i + 8], dbls[10 * i:10 * i + 10]
            nops = int(I[2])
            out.append({"kind": int(I[0]), "axis": int(I[1]), "ops": [int(v) for v in I[3:3 + nops]],
                        "plans": [(float(X[2 * o]), float(X[2 * o + 1])) for o in range(nops)],
                        "slot": int(I[7]), "ddelta": float(X[8]), "sdelta": float(X[9])})
        return out

    def synchronize(self):
        self._check(pdg_synchronize(self.ctx), "pdg_synchronize")

    def timing_enable(self, on=True):
        self._check(pdg_timing_enable(self.ctx, 1 if on else 0), "pdg_timing_enable")

    def timing_read(self):
        """Per kernel kind (0 line pass, 1 line pass with collision, 2 state kernels,
        3 diagonal pass, 4 corner pass): launches and summed ms."""
        la = (ctypes.c_longlong * 5)()
        ms = (ctypes.c_double * 5)()
        self._check(pdg_timing_read(self.ctx, ctypes.addressof(la), ctypes.addressof(ms), 5), "pdg_timing_read")
        return list(la), list(ms)

    def set_launch(self, kind, lpb, nseg, ngroup):
        self._check(pdg_set_launch(self.ctx, kind, lpb, nseg, ngroup), "pdg_set_launch")


    def set_option(self, option, value):
        self._check(pdg_set_option(self.ctx, option, int(value)), "pdg_set_option")

    def get_launch(self, kind):
        v = [ctypes.c_int(), ctypes.c_int(), ctypes.c_int()]
        self._check(pdg_get_launch(self.ctx, kind, *[ctypes.addressof(x) for x in v]), "pdg_get_launch")
        return tuple(x.value for x in v)

    def autotune(self, dt, reps=3):
        self._check(pdg_autotune(self.ctx, dt, reps), "pdg_autotune")


class Batch:
    """Owns one pdg_batch over existing Solver objects (which must outlive it)."""

    def __init__(self, solvers, stream=None):
        self.solvers = list(solvers)
        arr = (_P * len(self.solvers))(*[s.ctx.value for s in self.solvers])
        self.b = _P()
        r = pdg_batch_create(ctypes.byref(self.b), len(self.solvers), ctypes.addressof(arr),
                             _P(stream) if stream else None)
        if r != PDG_OK:
            raise PdgError(r, "pdg_batch_create")

    def _check(self, r, what):
        if r != PDG_OK:
            raise PdgError(r, f"{what}: {pdg_batch_last_error(self.b).decode()}")

    def step(self, dt, nsteps, use_graph=False):
        n = len(self.solvers)
        dts = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (n,)))
        ns = np.ascontiguousarray(np.broadcast_to(np.asarray(nsteps, dtype=np.int32), (n,)))
        self._check(pdg_batch_step(self.b, dts.ctypes.data, ns.ctypes.data, 1 if use_graph else 0),
                    "pdg_batch_step")

    def elapsed(self):
        ms = ctypes.c_double()
        la = ctypes.c_longlong()
        self._check(pdg_batch_elapsed(self.b, ctypes.addressof(ms), ctypes.addressof(la)), "pdg_batch_elapsed")
        return ms.value, la.value

    def autotune(self, dt, reps=3):
        n = len(self.solvers)
        dts = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (n,)))
        self._check(pdg_batch_autotune(self.b, dts.ctypes.data, reps), "pdg_batch_autotune")

    def close(self):
        if self.b:
            pdg_batch_destroy(self.b)
            self.b = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solver_for(cfg, scheme="M2", stream=None, precision=PDG_PREC_FP64):
    """Create a Solver with mesh and model of a workloads.Config."""
    s = Solver(cfg.dim, cfg.n_macro, cfg.n_sub, cfg.order, lengths=cfg.lengths[:cfg.dim], stream=stream)
    prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
    s.set_model(cfg.kind, cfg.lam, a=cfg.a, gravity=cfg.gravity, gamma=cfg.gamma, omega=cfg.omega,
                theta=cfg.theta, scheme=scheme, precision=prec)
    return s


def model_desc(kind, lam, a=(0.0, 0.0, 0.0), gravity=9.81, gamma=1.4, omega=2.0, theta=0.5, scheme="M2",
               precision=PDG_PREC_FP64):
    d = pdg_model_desc()
    d.kind = KIND[kind] if isinstance(kind, str) else int(kind)
    d.scheme = SCHEME[scheme] if isinstance(scheme, str) else int(scheme)
    d.precision = precision
    d.lambda_ = lam
    for i in range(3):
        d.a[i] = float(a[i]) if i < len(a) else 0.0
    d.gravity, d.gamma, d.omega, d.theta = gravity, gamma, omega, theta
    return d


class Server:
    """Owns one pdg_server (continuous batching of independent solves)."""

    def __init__(self, budget_bytes, chunk_steps=10, use_graph=False, stream=None):
        self.s = _P()
        r = pdg_server_create(ctypes.byref(self.s), int(budget_bytes), int(chunk_steps), 1 if use_graph else 0,
                              _P(stream) if stream else None)
        if r != PDG_OK:
            raise PdgError(r, "pdg_server_create")

    def _check(self, r, what):
        if r != PDG_OK:
            raise PdgError(r, f"{what}: {pdg_server_last_error(self.s).decode()}")

    def now(self):
        return pdg_server_now(self.s)

    def submit(self, cfg, w0, nsteps, t_arrival=None, dt=None, scheme="M2", precision=PDG_PREC_FP64):
        """Enqueue a solve of workloads.Config `cfg` from w0 (host array)."""
        w0 = np.ascontiguousarray(np.asarray(w0, dtype=np.float64).reshape(-1))
        q = pdg_request()
        q.dim = cfg.dim
        for a in range(3):
            q.n_macro[a] = cfg.n_macro[a] if a < cfg.dim else 1
            q.n_sub[a] = cfg.n_sub[a] if a < cfg.dim else 1
        q.order = cfg.order
        q.model = model_desc(cfg.kind, cfg.lam, a=cfg.a, gravity=cfg.gravity, gamma=cfg.gamma, omega=cfg.omega,
                             theta=cfg.theta, scheme=scheme,
                             precision=PRECISION[precision] if isinstance(precision, str) else int(precision))
        q.dt = cfg.dt if dt is None else dt
        q.nsteps = int(nsteps)
        q.w0 = w0.ctypes.data
        q.w0_len = w0.size
        q.t_arrival = self.now() if t_arrival is None else t_arrival
        rid = ctypes.c_longlong()
        self._check(pdg_server_submit(self.s, ctypes.byref(q), ctypes.addressof(rid)), "pdg_server_submit")
        return rid.value

    def iterate(self):
        nr, nd = ctypes.c_int(), ctypes.c_int()
        self._check(pdg_server_iterate(self.s, ctypes.addressof(nr), ctypes.addressof(nd)), "pdg_server_iterate")
        return nr.value, nd.value

    def pending(self):
        nw, nr = ctypes.c_int(), ctypes.c_int()
        self._check(pdg_server_pending(self.s, ctypes.addressof(nw), ctypes.addressof(nr)), "pdg_server_pending")
        return nw.value, nr.value

    def poll(self, max_n=4096):
        ids = np.zeros(max_n, dtype=np.int64)
        ta, tb, tc = (np.zeros(max_n) for _ in range(3))
        cnt = ctypes.c_int()
        self._check(pdg_server_poll(self.s, ids.ctypes.data, ta.ctypes.data, tb.ctypes.data, tc.ctypes.data, max_n,
                                    ctypes.addressof(cnt)), "pdg_server_poll")
        n = cnt.value
        return [(int(ids[i]), ta[i], tb[i], tc[i]) for i in range(n)]

    def result(self, rid, w_len):
        out = np.empty(w_len)
        self._check(pdg_server_result(self.s, rid, out.ctypes.data, w_len), "pdg_server_result")
        return out

    def cancel(self, rid):
        self._check(pdg_server_cancel(self.s, rid), "pdg_server_cancel")

    def stats(self):
        it, du, co = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        pk = ctypes.c_size_t()
        self._check(pdg_server_stats(self.s, ctypes.addressof(it), ctypes.addressof(du), ctypes.addressof(co),
                                     ctypes.addressof(pk)), "pdg_server_stats")
        return {"iterations": it.value, "dof_updates": du.value, "completed": co.value, "peak_bytes": pk.value}

    def close(self):
        if self.s:
            pdg_server_destroy(self.s)
            self.s = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
