"""ctypes binding of libkin (include/kin.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts torch
tensors / numpy arrays to pointers and C structs.  There is no CPU fallback:
if libkin.so is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkin.so")

KIN_OK, KIN_ERR_INVALID_ARG, KIN_ERR_CUDA, KIN_ERR_NOMEM, KIN_ERR_MECH = 0, 1, 2, 3, 4
KIN_ERR_STATE_FAILED, KIN_ERR_UNSUPPORTED = 5, 6
LAYOUT_PLAIN, LAYOUT_QUEUE, LAYOUT_WARP, LAYOUT_AUTO = 0, 1, 2, 3
LAYOUT_NAMES = {LAYOUT_PLAIN: "plain", LAYOUT_QUEUE: "queue", LAYOUT_WARP: "warp",
                LAYOUT_AUTO: "auto"}
KEY_GIVEN, KEY_STEP_HEURISTIC, KEY_GIVEN_LOG = 0, 1, 2
COUNTER_NAMES = ("nstep", "naccpt", "nrejct", "nfcn", "njac", "ndec", "nsol", "status")
MAX_SPECIES = 64

# every symbol include/kin.h declares
EXPORTS = ("kin_options_default", "kin_mech_create", "kin_destroy", "kin_integrate",
           "kin_integrate_ex", "kin_integrate_host", "kin_get_stats", "kin_rhs",
           "kin_jacobian", "kin_radau_constants", "kin_status_string", "kin_exp",
           "kin_integrate_static", "kin_mlp_create", "kin_mlp_destroy", "kin_mlp_num_params",
           "kin_mlp_get_params", "kin_mlp_set_params", "kin_mlp_forward", "kin_mlp_grad",
           "kin_mlp_train_step", "kin_moments", "kin_mlp_features", "kin_mlp_targets",
           "kin_mlp_predict", "kin_autotune", "kin_order_states", "kin_mlp_train_step_rows",
           "kin_resolve_options", "kin_conc_analyse", "kin_conc_create", "kin_conc_destroy",
           "kin_integrate_conc", "kin_conc_get_stats", "kin_exprb_create", "kin_exprb_destroy",
           "kin_integrate_exprb", "kin_exprb_get_stats", "kin_exprb_phi", "kin_exprb_chem")


class KinError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        msg = _lib.kin_status_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} (status {code})" if what else msg)


class MechDesc(C.Structure):
    _fields_ = [("ns", C.c_int32), ("nr", C.c_int32), ("W", C.c_void_p), ("nasa", C.c_void_p),
                ("reac", C.c_void_p), ("prod", C.c_void_p), ("arrh", C.c_void_p),
                ("rtype", C.c_void_p), ("eff", C.c_void_p), ("fall", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("layout", C.c_int32), ("lu_fp32", C.c_int32), ("jac_fd", C.c_int32),
                ("max_steps", C.c_int32), ("nit", C.c_int32), ("block", C.c_int32),
                ("grid_per_sm", C.c_int32), ("transform_tol", C.c_int32),
                ("queue_refill", C.c_int32), ("stop_after", C.c_int32), ("h0", C.c_void_p),
                ("z0", C.c_void_p), ("h_first", C.c_void_p), ("z_first", C.c_void_p),
                ("order", C.c_void_p), ("lanes", C.c_int32), ("h_fixed", C.c_double),
                ("order_by", C.c_int32)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load libkin.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            from . import build as _build
            if not _build.up_to_date():
                _build.build()
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libkin.so not found at {LIB_PATH}")
            L = C.CDLL(LIB_PATH)
            vp, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
            L.kin_options_default.argtypes = [vp]
            L.kin_mech_create.argtypes = [vp, C.POINTER(vp)]
            L.kin_destroy.argtypes = [vp]
            L.kin_destroy.restype = None
            L.kin_integrate.argtypes = [vp, vp, vp, vp, i64, d, d, d, vp]
            L.kin_integrate_ex.argtypes = [vp, vp, vp, vp, i64, d, d, d, vp, vp, vp, vp]
            L.kin_integrate_host.argtypes = [vp, vp, vp, vp, i64, d, d, d, vp, vp, vp, vp]
            L.kin_get_stats.argtypes = [vp, vp]
            L.kin_rhs.argtypes = [vp, vp, vp, i64, vp, vp]
            L.kin_jacobian.argtypes = [vp, vp, vp, i64, i32, d, vp, vp, vp]
            L.kin_radau_constants.argtypes = [vp, i32]
            L.kin_exp.argtypes = [vp, vp, vp, i64, vp]
            L.kin_integrate_static.argtypes = [vp, vp, vp, vp, i64, d, d, d, vp, vp]
            L.kin_autotune.argtypes = [vp, vp, vp, vp, i64, d, d, d, vp, vp, vp, i32, vp]
            L.kin_order_states.argtypes = [vp, vp, vp, vp, i64, d, d, i32, vp, vp, vp]
            L.kin_resolve_options.argtypes = [vp, i64, d, vp, vp]
            L.kin_mlp_create.argtypes = [i32, i32, i32, i32, C.c_uint64, C.POINTER(vp)]
            L.kin_mlp_destroy.argtypes = [vp]
            L.kin_mlp_destroy.restype = None
            L.kin_mlp_num_params.argtypes = [vp]
            L.kin_mlp_num_params.restype = i64
            L.kin_mlp_get_params.argtypes = [vp, vp, i64]
            L.kin_mlp_set_params.argtypes = [vp, vp, i64]
            L.kin_mlp_forward.argtypes = [vp, vp, vp, i64, vp]
            L.kin_mlp_grad.argtypes = [vp, vp, vp, i64, vp, vp, vp]
            L.kin_mlp_train_step.argtypes = [vp, vp, vp, i64, C.c_float, vp, vp]
            L.kin_mlp_train_step_rows.argtypes = [vp, vp, vp, i64, vp, i64, C.c_float, vp, vp]
            L.kin_moments.argtypes = [vp, i64, i32, vp, vp, vp]
            L.kin_mlp_features.argtypes = [i32, vp, vp, vp, i64, d, vp, vp, vp, vp]
            L.kin_mlp_targets.argtypes = [i32, vp, vp, i64, vp, vp, vp, vp]
            L.kin_mlp_predict.argtypes = [vp, i32, vp, vp, vp, i64, d, vp, vp, vp, vp, vp, vp,
                                          vp]
            L.kin_conc_analyse.argtypes = [vp, vp, vp, vp]
            L.kin_conc_create.argtypes = [vp, C.POINTER(vp)]
            L.kin_conc_destroy.argtypes = [vp]
            L.kin_integrate_conc.argtypes = [vp, vp, vp, vp, i64, d, d, d, vp, vp, vp, vp]
            L.kin_conc_get_stats.argtypes = [vp, vp]
            L.kin_exprb_create.argtypes = [vp, C.POINTER(vp)]
            L.kin_exprb_destroy.argtypes = [vp]
            L.kin_integrate_exprb.argtypes = [vp, vp, vp, vp, i64, d, d, d, d, vp, i32, vp, vp,
                                              vp]
            L.kin_exprb_get_stats.argtypes = [vp, vp]
            L.kin_exprb_phi.argtypes = [vp, vp, i32, i32, d, vp, vp]
            L.kin_exprb_chem.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp]
            L.kin_status_string.argtypes = [C.c_int]
            L.kin_status_string.restype = C.c_char_p
            _lib = L
    return _lib


def _check(rc, what):
    if rc != KIN_OK:
        raise KinError(rc, what)


def _ptr(t):
    """Device/host pointer of a torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def options(layout="auto", lu_fp32=False, jac_fd=False, max_steps=100000, nit=7, block=0,
            grid_per_sm=0, transform_tol=True, queue_refill=0, stop_after=0, h0=None, z0=None,
            h_first=None, z_first=None, order=None, lanes=0, h_fixed=0.0, order_by=None):
    o = Options()
    _check(lib().kin_options_default(C.byref(o)), "kin_options_default")
    o.layout = {v: k for k, v in LAYOUT_NAMES.items()}[layout] if isinstance(layout, str) \
        else int(layout)
    o.lu_fp32 = int(bool(lu_fp32))
    o.jac_fd = int(bool(jac_fd))
    o.max_steps = int(max_steps)
    o.nit = int(nit)
    o.block = int(block)
    o.grid_per_sm = int(grid_per_sm)
    o.transform_tol = int(bool(transform_tol))
    o.queue_refill = int(queue_refill)
    o.stop_after = int(stop_after)
    o.h0, o.z0, o.h_first, o.z_first = _ptr(h0), _ptr(z0), _ptr(h_first), _ptr(z_first)
    o.order = _ptr(order)
    o.lanes = int(lanes)
    o.h_fixed = float(h_fixed)
    o.order_by = {None: 0, "none": 0, "heuristic": 1}[order_by]
    return o


def mech_desc(mech):
    """(kin_mech_desc, arrays it points at) for a ``synth.Mechanism``-like object."""
    arrs = dict(
        W=np.ascontiguousarray(mech.W, np.float64),
        nasa=np.ascontiguousarray(mech.nasa, np.float64),
        reac=np.ascontiguousarray(mech.reac, np.int32),
        prod=np.ascontiguousarray(mech.prod, np.int32),
        arrh=np.ascontiguousarray(mech.arrh, np.float64),
        rtype=np.ascontiguousarray(mech.rtype, np.int32),
        eff=np.ascontiguousarray(mech.eff, np.float64),
        fall=np.ascontiguousarray(mech.fall, np.float64))
    d = MechDesc(int(mech.ns), int(mech.nr), *(arrs[k].ctypes.data for k in
                                                ("W", "nasa", "reac", "prod", "arrh", "rtype",
                                                 "eff", "fall")))
    return d, arrs


def integrate_static(mech, Y, T, P, dt, rtol=1e-6, atol=1e-10, *, status=None, stream=None):
    """kin_integrate_static: default-option integration that allocates no device
    memory (tables and counters in libkin's fixed device array)."""
    d, keep = mech_desc(mech)
    n = int(T.shape[0])
    rc = lib().kin_integrate_static(C.byref(d), _ptr(Y), _ptr(T), _ptr(P), n, float(dt),
                                    float(rtol), float(atol), _ptr(status), _stream(stream))
    del keep
    _check(rc, "kin_integrate_static")


class Mechanism:
    """A mechanism uploaded to the current CUDA device (kin_mech_create)."""

    def __init__(self, mech):
        self.ns, self.nr = int(mech.ns), int(mech.nr)
        arrs = dict(
            W=np.ascontiguousarray(mech.W, np.float64),
            nasa=np.ascontiguousarray(mech.nasa, np.float64),
            reac=np.ascontiguousarray(mech.reac, np.int32),
            prod=np.ascontiguousarray(mech.prod, np.int32),
            arrh=np.ascontiguousarray(mech.arrh, np.float64),
            rtype=np.ascontiguousarray(mech.rtype, np.int32),
            eff=np.ascontiguousarray(mech.eff, np.float64),
            fall=np.ascontiguousarray(mech.fall, np.float64))
        d = MechDesc(self.ns, self.nr, *(arrs[k].ctypes.data for k in
                                          ("W", "nasa", "reac", "prod", "arrh", "rtype", "eff",
                                           "fall")))
        h = C.c_void_p()
        _check(lib().kin_mech_create(C.byref(d), C.byref(h)), "kin_mech_create")
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("mechanism destroyed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.kin_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- integration --------------------------------------------------------
    def integrate(self, Y, T, P, dt, rtol=1e-6, atol=1e-10, *, status=None, counters=None,
                  stream=None, **opt):
        """Advance device tensors Y [ns, n], T [n] in place over dt (kin_integrate_ex)."""
        n = int(T.shape[0])
        o = options(**opt)
        rc = lib().kin_integrate_ex(self.handle, _ptr(Y), _ptr(T), _ptr(P), n, float(dt),
                                    float(rtol), float(atol), C.byref(o), _ptr(status),
                                    _ptr(counters), _stream(stream))
        _check(rc, "kin_integrate_ex")

    def capture(self, Y, T, P, dt, rtol=1e-6, atol=1e-10, *, status=None, counters=None,
                order_by=None, **opt):
        """Capture one integration into a CUDA graph (torch.cuda.CUDAGraph).

        Each replay() integrates the same buffers in place over dt with the
        launch configuration fixed at capture: one memset node (the batch
        totals) and one integration kernel node.  With order_by="heuristic"
        the graph first orders the states by the starting-step heuristic
        (kin_order_states: key, min/max, histogram, scan and scatter kernels)
        and integrates in that order.  Capture itself runs nothing.
        """
        import torch
        if order_by not in (None, "heuristic"):
            raise ValueError(f"order_by: {order_by!r}")
        g = torch.cuda.CUDAGraph()
        bufs = ()
        if order_by == "heuristic":
            n = int(T.shape[0])
            bufs = (torch.empty(n, dtype=torch.float64, device=T.device),
                    torch.empty(n, dtype=torch.int32, device=T.device))
        with torch.cuda.graph(g, capture_error_mode="relaxed"):
            s = torch.cuda.current_stream()
            if bufs:
                self.order_states(Y, T, P, rtol, atol, key=bufs[0], order=bufs[1], stream=s)
                opt["order"] = bufs[1]
            self.integrate(Y, T, P, dt, rtol, atol, status=status, counters=counters,
                           stream=s, **opt)
        g.kin_buffers = bufs  # the key and order live as long as the graph
        return g

    def integrate_default(self, Y, T, P, dt, rtol=1e-6, atol=1e-10, stream=None):
        """kin_integrate: the default options."""
        n = int(T.shape[0])
        _check(lib().kin_integrate(self.handle, _ptr(Y), _ptr(T), _ptr(P), n, float(dt),
                                   float(rtol), float(atol), _stream(stream)), "kin_integrate")

    def integrate_host(self, Y, T, P, dt, rtol=1e-6, atol=1e-10, *, status=None, counters=None,
                       stream=None, **opt):
        """Advance host arrays (numpy or CPU tensors) in place (kin_integrate_host)."""
        n = int(T.shape[0])
        o = options(**opt)
        rc = lib().kin_integrate_host(self.handle, _ptr(Y), _ptr(T), _ptr(P), n, float(dt),
                                      float(rtol), float(atol), C.byref(o), _ptr(status),
                                      _ptr(counters), _stream(stream) if stream is not None else None)
        _check(rc, "kin_integrate_host")

    def autotune(self, Y, T, P, dt, rtol=1e-6, atol=1e-10, stream=None, **base):
        """kin_autotune: returns (best options as a dict, list of candidate seconds)."""
        b = options(**base)
        best = Options()
        secs = np.full(16, np.nan)
        rc = lib().kin_autotune(self.handle, _ptr(Y), _ptr(T), _ptr(P), int(T.shape[0]), float(dt),
                                float(rtol), float(atol), C.byref(b), C.byref(best),
                                secs.ctypes.data, 16, _stream(stream))
        _check(rc, "kin_autotune")
        secs = secs[~np.isnan(secs)]
        return dict(layout=LAYOUT_NAMES[best.layout], block=best.block,
                    queue_refill=best.queue_refill, grid_per_sm=best.grid_per_sm,
                    lanes=best.lanes), secs.tolist()

    def resolve(self, n, dt, **opt):
        """kin_resolve_options: the launch configuration an integration of n
        states over dt with these options would use (layout "auto" resolved)."""
        o = options(**opt)
        out = Options()
        _check(lib().kin_resolve_options(self.handle, int(n), float(dt), C.byref(o),
                                         C.byref(out)), "kin_resolve_options")
        return dict(layout=LAYOUT_NAMES[out.layout], block=out.block,
                    queue_refill=out.queue_refill, lanes=out.lanes)

    def order_states(self, Y, T, P, rtol=1e-6, atol=1e-10, *, key=None, given_key=None,
                     log_key=False, order=None, stream=None):
        """kin_order_states: (order, key) device tensors, order an int32
        permutation that sorts the key ascending (stiffest first).  With
        given_key (float64 [n], e.g. the predictor's ln h0) that key is used
        as is; otherwise the starting-step heuristic's ln h0 is computed into
        key (a new tensor when key is None).  log_key: sort a positive given key
        (e.g. the predictor's h0) by its logarithm.  order: optional output."""
        import torch
        if given_key is not None:
            key, mode = given_key, (KEY_GIVEN_LOG if log_key else KEY_GIVEN)
        else:
            mode = KEY_STEP_HEURISTIC
        n = int(T.shape[0]) if T is not None else int(key.shape[0])
        dev = (T if T is not None else key).device
        if order is None:
            order = torch.empty(n, dtype=torch.int32, device=dev)
        if key is None:
            key = torch.empty(n, dtype=torch.float64, device=dev)
        _check(lib().kin_order_states(self.handle, _ptr(Y), _ptr(T), _ptr(P), n, float(rtol),
                                      float(atol), mode, _ptr(key), _ptr(order),
                                      _stream(stream)), "kin_order_states")
        return order, key

    def stats(self):
        """Totals of the last integration (kin_get_stats)."""
        out = np.zeros(9, dtype=np.int64)
        rc = lib().kin_get_stats(self.handle, out.ctypes.data)
        if rc not in (KIN_OK, KIN_ERR_STATE_FAILED):
            _check(rc, "kin_get_stats")
        keys = list(COUNTER_NAMES[:7]) + ["failed", "max_steps_state"]
        return dict(zip(keys, out.tolist()))

    # -- unit-level entries ---------------------------------------------------
    def rhs(self, y, P, f, stream=None):
        n = int(P.shape[0])
        _check(lib().kin_rhs(self.handle, _ptr(y), _ptr(P), n, _ptr(f), _stream(stream)), "kin_rhs")

    def exp(self, x, y, stream=None):
        _check(lib().kin_exp(self.handle, _ptr(x), _ptr(y), int(x.numel()), _stream(stream)),
               "kin_exp")

    def jacobian(self, y, P, J, fd=False, h=0.0, scal=None, stream=None):
        n = int(P.shape[0])
        _check(lib().kin_jacobian(self.handle, _ptr(y), _ptr(P), n, int(bool(fd)), float(h),
                                  _ptr(scal), _ptr(J), _stream(stream)), "kin_jacobian")


def conc_analyse(mech):
    """kin_conc_analyse (host only): (var [ns+1], filled pattern [(ns+1)^2] in
    elimination order, counts [nnz J, nnz L+U, real LU ops, real solve ops])."""
    d, keep = mech_desc(mech)
    N = int(mech.ns) + 1
    var = np.zeros(N, dtype=np.int32)
    pat = np.zeros((N, N), dtype=np.uint8)
    cnt = np.zeros(4, dtype=np.int64)
    _check(lib().kin_conc_analyse(C.byref(d), var.ctypes.data, pat.ctypes.data, cnt.ctypes.data),
           "kin_conc_analyse")
    del keep
    return var, pat.astype(bool), cnt


class ConcMechanism:
    """The concentration-based form of a mechanism with its sparse LU
    structure, on the current CUDA device (kin_conc_create)."""

    def __init__(self, mech):
        self.ns, self.nr = int(mech.ns), int(mech.nr)
        d, keep = mech_desc(mech)
        h = C.c_void_p()
        _check(lib().kin_conc_create(C.byref(d), C.byref(h)), "kin_conc_create")
        del keep
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("plan destroyed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.kin_conc_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def integrate(self, Y, T, P, dt, rtol=1e-6, atol=1e-10, *, status=None, counters=None,
                  stream=None, **opt):
        """Advance device tensors Y [ns, n], T [n] in place over dt (kin_integrate_conc)."""
        n = int(T.shape[0])
        opt.setdefault("layout", "warp")
        o = options(**opt)
        rc = lib().kin_integrate_conc(self.handle, _ptr(Y), _ptr(T), _ptr(P), n, float(dt),
                                      float(rtol), float(atol), C.byref(o), _ptr(status),
                                      _ptr(counters), _stream(stream))
        _check(rc, "kin_integrate_conc")

    def stats(self):
        """Totals of the last integration (kin_conc_get_stats)."""
        out = np.zeros(9, dtype=np.int64)
        rc = lib().kin_conc_get_stats(self.handle, out.ctypes.data)
        if rc not in (KIN_OK, KIN_ERR_STATE_FAILED):
            _check(rc, "kin_conc_get_stats")
        keys = list(COUNTER_NAMES[:7]) + ["failed", "max_steps_state"]
        return dict(zip(keys, out.tolist()))


class ExpRosenbrock:
    """exprb43 with Krylov phi-function products for a mechanism on the
    current CUDA device (kin_exprb_create)."""

    def __init__(self, mech):
        self.ns, self.nr = int(mech.ns), int(mech.nr)
        d, keep = mech_desc(mech)
        h = C.c_void_p()
        _check(lib().kin_exprb_create(C.byref(d), C.byref(h)), "kin_exprb_create")
        del keep
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("destroyed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.kin_exprb_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def integrate(self, Y, T, P, dt, rtol=1e-6, atol=1e-10, *, kappa=0.1, h0=None,
                  max_steps=100000, status=None, counters=None, stream=None):
        """Advance device tensors Y [ns, n], T [n] in place over dt (kin_integrate_exprb)."""
        n = int(T.shape[0])
        _check(lib().kin_integrate_exprb(self.handle, _ptr(Y), _ptr(T), _ptr(P), n, float(dt),
                                         float(rtol), float(atol), float(kappa), _ptr(h0),
                                         int(max_steps), _ptr(status), _ptr(counters),
                                         _stream(stream)), "kin_integrate_exprb")

    def phi(self, H, p, tau, out, stream=None):
        """phi_1..phi_p (tau H) e1 of a device matrix H [m, m] into out [m, p]
        (kin_exprb_phi)."""
        m = int(H.shape[0])
        _check(lib().kin_exprb_phi(self.handle, _ptr(H), m, int(p), float(tau), _ptr(out),
                                   _stream(stream)), "kin_exprb_phi")

    def chem(self, y, P, f, f_rates, J, stream=None):
        """Right-hand sides and Jacobians of the state-per-warp kernels
        (kin_exprb_chem): y [N, n], f and f_rates [N, n], J [N*N, n]."""
        n = int(P.shape[0])
        _check(lib().kin_exprb_chem(self.handle, _ptr(y), _ptr(P), n, _ptr(f), _ptr(f_rates),
                                    _ptr(J), _stream(stream)), "kin_exprb_chem")

    def stats(self):
        """Totals of the last integration (kin_exprb_get_stats)."""
        out = np.zeros(9, dtype=np.int64)
        rc = lib().kin_exprb_get_stats(self.handle, out.ctypes.data)
        if rc not in (KIN_OK, KIN_ERR_STATE_FAILED):
            _check(rc, "kin_exprb_get_stats")
        keys = ["nstep", "naccpt", "nrejct", "nfcn", "njac", "krylov_spaces", "krylov_dim",
                "failed", "max_steps_state"]
        return dict(zip(keys, out.tolist()))


def radau_constants():
    """The library's Radau IIA constants (kin_radau_constants): dict of arrays."""
    out = np.zeros(27)
    _check(lib().kin_radau_constants(out.ctypes.data, 27), "kin_radau_constants")
    return dict(c=out[0:3], gamma=out[3], alpha=out[4], beta=out[5],
                T=out[6:15].reshape(3, 3), TI=out[15:24].reshape(3, 3), d=out[24:27])


class MLP:
    """The step/guess predictor (kin_mlp_*).  precision: "bf16" or "fp32"."""

    def __init__(self, din, width, dout, precision="bf16", seed=0):
        h = C.c_void_p()
        p = {"bf16": 0, "fp32": 1}[precision]
        _check(lib().kin_mlp_create(int(din), int(width), int(dout), p, int(seed), C.byref(h)),
               "kin_mlp_create")
        self._h = h
        self.din, self.width, self.dout = int(din), int(width), int(dout)

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.kin_mlp_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def num_params(self):
        return int(lib().kin_mlp_num_params(self._h))

    def get_params(self):
        out = np.zeros(self.num_params(), dtype=np.float32)
        _check(lib().kin_mlp_get_params(self._h, out.ctypes.data, out.size), "kin_mlp_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(lib().kin_mlp_set_params(self._h, p.ctypes.data, p.size), "kin_mlp_set_params")

    def forward(self, X, Y, stream=None):
        _check(lib().kin_mlp_forward(self._h, _ptr(X), _ptr(Y), int(X.shape[0]), _stream(stream)),
               "kin_mlp_forward")

    def grad(self, X, T, grad_out=None, loss_out=None, stream=None):
        _check(lib().kin_mlp_grad(self._h, _ptr(X), _ptr(T), int(X.shape[0]), _ptr(grad_out),
                                  _ptr(loss_out), _stream(stream)), "kin_mlp_grad")

    def train_step(self, X, T, lr, loss_out=None, stream=None):
        _check(lib().kin_mlp_train_step(self._h, _ptr(X), _ptr(T), int(X.shape[0]), float(lr),
                                        _ptr(loss_out), _stream(stream)), "kin_mlp_train_step")

    def train_step_rows(self, X, T, rows, lr, loss_out=None, stream=None):
        """Adam step on the rows (device int32 tensor) of the training set X, T."""
        _check(lib().kin_mlp_train_step_rows(self._h, _ptr(X), _ptr(T), int(X.shape[0]),
                                             _ptr(rows), int(rows.shape[0]), float(lr),
                                             _ptr(loss_out), _stream(stream)),
               "kin_mlp_train_step_rows")

    def predict(self, ns, Y, T, P, dt, norm, h0=None, z0=None, stream=None):
        """norm: dict of device float tensors in_mean, in_std, out_mean, out_std."""
        _check(lib().kin_mlp_predict(self._h, int(ns), _ptr(Y), _ptr(T), _ptr(P), int(T.shape[0]),
                                     float(dt), _ptr(norm["in_mean"]), _ptr(norm["in_std"]),
                                     _ptr(norm["out_mean"]), _ptr(norm["out_std"]), _ptr(h0),
                                     _ptr(z0), _stream(stream)), "kin_mlp_predict")


def moments(X, mean, std, stream=None):
    _check(lib().kin_moments(_ptr(X), int(X.shape[0]), int(X.shape[1]), _ptr(mean), _ptr(std),
                             _stream(stream)), "kin_moments")


def features(ns, Y, T, P, dt, X, mean=None, std=None, stream=None):
    _check(lib().kin_mlp_features(int(ns), _ptr(Y), _ptr(T), _ptr(P), int(T.shape[0]), float(dt),
                                  _ptr(mean), _ptr(std), _ptr(X), _stream(stream)),
           "kin_mlp_features")


def targets(nz, h, z, tgt, mean=None, std=None, stream=None):
    _check(lib().kin_mlp_targets(int(nz), _ptr(h), _ptr(z), int(h.shape[0]), _ptr(mean),
                                 _ptr(std), _ptr(tgt), _stream(stream)), "kin_mlp_targets")
