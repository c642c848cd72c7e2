"""ctypes front end of the FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: this module and the C library it builds may be used
by the test-suite, by the smoke check and by the benchmark's CPU-baseline leg,
and by nothing on the product path.  It shares no code with the CUDA path:
it takes a mechanism as plain arrays (see ``synth.Mechanism``) and states as
numpy arrays.

The functions follow the paper (Curtis, Niemeyer & Sung): the reactor ODE
and Jacobian (Sec. 2.1), the CVODE-style finite-difference Jacobian
(Sec. 2.1, Sec. 3.4), Radau IIA with step control (Sec. 2.1), the error
measure E_i and |E| (Sec. 2.3) and the divergence measure D (Sec. 3.3).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["chem.c", "linalg.c", "radau.c", "batch.c"]
# -O3 with IEEE semantics kept (no fast-math, no FMA contraction, no
# host-specific instruction set), so the x86 and Arm hosts evaluate the same
# expressions in the same order: the oracle is a checker first, and its
# timed CPU baseline is this same build.
CFLAGS = ["-O3", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math", "-ffp-contract=off"]
LIB_NAME = "liboracle.so"
RU = 8314.46261815324  # J/(kmol K), as oracle.h
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain C99 + OpenMP) into oracle/liboracle.so."""
    out = os.path.join(HERE, LIB_NAME)
    srcs = [os.path.join(HERE, s) for s in SOURCES] + [os.path.join(HERE, "oracle.h")]
    if not force and os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(s)
                                                 for s in srcs):
        return out
    cmd = ["gcc", "-std=c99", *CFLAGS, "-o", out + ".tmp"] + [os.path.join(HERE, s) for s in SOURCES] + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(out + ".tmp", out)
    return out


class _Mech(C.Structure):
    _fields_ = [("ns", C.c_int), ("nr", C.c_int),
                ("W", C.c_void_p), ("nasa", C.c_void_p), ("reac", C.c_void_p),
                ("prod", C.c_void_p), ("arrh", C.c_void_p), ("rtype", C.c_void_p),
                ("eff", C.c_void_p), ("fall", C.c_void_p)]


class _Opts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("transform_tol", C.c_int),
                ("nit", C.c_int), ("h0", C.c_double), ("hfixed", C.c_double),
                ("max_steps", C.c_int), ("jac_kind", C.c_int), ("z0", C.c_void_p),
                ("z_first_out", C.c_void_p), ("form", C.c_int), ("atol_scale", C.c_void_p)]


class _Stats(C.Structure):
    _fields_ = [("nstep", C.c_int32), ("naccpt", C.c_int32), ("nrejct", C.c_int32),
                ("nfcn", C.c_int32), ("njac", C.c_int32), ("ndec", C.c_int32),
                ("nsol", C.c_int32), ("status", C.c_int32), ("h_first", C.c_double),
                ("h_last", C.c_double), ("err_last", C.c_double)]


class _Tableau(C.Structure):
    _fields_ = [("c", C.c_double * 3), ("A", C.c_double * 9), ("b", C.c_double * 3),
                ("gamma", C.c_double), ("alpha", C.c_double), ("beta", C.c_double),
                ("T", C.c_double * 9), ("TI", C.c_double * 9), ("e", C.c_double * 3),
                ("gamma0", C.c_double)]


RHS_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double))
JAC_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double),
                     C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double))

COUNTER_NAMES = ("nstep", "naccpt", "nrejct", "nfcn", "njac", "ndec", "nsol", "status")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            vp, d, i = C.c_void_p, C.c_double, C.c_int
            L.orc_thermo.argtypes = [vp, d, vp, vp, vp]
            L.orc_rhs.argtypes = [vp, d, vp, vp]
            L.orc_jac.argtypes = [vp, d, vp, vp]
            L.orc_jac_fd.argtypes = [vp, d, vp, vp, d, vp, vp]
            L.orc_rate_constants.argtypes = [vp, d, vp, vp, vp]
            L.orc_wdot.argtypes = [vp, d, d, vp, vp]
            L.orc_rhs_conc.argtypes = [vp, d, vp, vp]
            L.orc_jac_conc.argtypes = [vp, d, vp, vp]
            L.orc_lu_real.argtypes = [i, vp, vp]
            L.orc_lu_solve_real.argtypes = [i, vp, vp, vp]
            L.orc_lu_cplx.argtypes = [i, vp, vp]
            L.orc_lu_solve_cplx.argtypes = [i, vp, vp, vp]
            L.orc_radau_tableau.argtypes = [vp]
            L.orc_radau.argtypes = [i, RHS_FN, JAC_FN, vp, d, d, vp, vp, vp]
            L.orc_initial_step.argtypes = [i, RHS_FN, vp, d, d, vp, vp, d, d, vp]
            L.orc_initial_step.restype = d
            L.orc_fd_jacobian.argtypes = [i, RHS_FN, vp, d, vp, vp, d, vp, vp]
            L.orc_integrate_batch.argtypes = [vp, C.c_int64, vp, vp, vp, d, vp, vp, vp, i]
            L.orc_num_threads.restype = i
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


class OracleMech:
    """Holds the contiguous arrays a ``orc_mech`` points at."""

    def __init__(self, mech):
        self.ns, self.nr = int(mech.ns), int(mech.nr)
        self.W = np.ascontiguousarray(mech.W, dtype=np.float64)
        self.nasa = np.ascontiguousarray(mech.nasa, dtype=np.float64)
        self.reac = np.ascontiguousarray(mech.reac, dtype=np.int32)
        self.prod = np.ascontiguousarray(mech.prod, dtype=np.int32)
        self.arrh = np.ascontiguousarray(mech.arrh, dtype=np.float64)
        self.rtype = np.ascontiguousarray(mech.rtype, dtype=np.int32)
        self.eff = np.ascontiguousarray(mech.eff, dtype=np.float64)
        self.fall = np.ascontiguousarray(mech.fall, dtype=np.float64)
        self.s = _Mech(self.ns, self.nr, _p(self.W).value, _p(self.nasa).value,
                       _p(self.reac).value, _p(self.prod).value, _p(self.arrh).value,
                       _p(self.rtype).value, _p(self.eff).value, _p(self.fall).value)
        self.ptr = C.cast(C.pointer(self.s), C.c_void_p)


def _as_om(mech):
    return mech if isinstance(mech, OracleMech) else OracleMech(mech)


def thermo(mech, T):
    om = _as_om(mech)
    cp, h, s = (np.zeros(om.ns) for _ in range(3))
    lib().orc_thermo(om.ptr, float(T), _p(cp), _p(h), _p(s))
    return cp, h, s


def rhs(mech, P, y):
    om = _as_om(mech)
    y = np.ascontiguousarray(y, dtype=np.float64)
    f = np.zeros(om.ns)
    rc = lib().orc_rhs(om.ptr, float(P), _p(y), _p(f))
    return f, rc


def jac(mech, P, y):
    om = _as_om(mech)
    y = np.ascontiguousarray(y, dtype=np.float64)
    J = np.zeros((om.ns, om.ns))
    rc = lib().orc_jac(om.ptr, float(P), _p(y), _p(J))
    return J, rc


def jac_fd(mech, P, y, f0, h, scal):
    om = _as_om(mech)
    y = np.ascontiguousarray(y, dtype=np.float64)
    f0 = np.ascontiguousarray(f0, dtype=np.float64)
    scal = np.ascontiguousarray(scal, dtype=np.float64)
    J = np.zeros((om.ns, om.ns))
    rc = lib().orc_jac_fd(om.ptr, float(P), _p(y), _p(f0), float(h), _p(scal), _p(J))
    return J, rc


FORMS = {"massfrac": 0, "conc": 1}


def rhs_conc(mech, P, phi):
    """f(phi) of the concentration-based form, phi = [T, V, n_0..n_{ns-2}]
    per unit mass (chem.c orc_rhs_conc; Sec. 3.3, Sec. 4)."""
    om = _as_om(mech)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    f = np.zeros(om.ns + 1)
    rc = lib().orc_rhs_conc(om.ptr, float(P), _p(phi), _p(f))
    return f, rc


def jac_conc(mech, P, phi):
    om = _as_om(mech)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    J = np.zeros((om.ns + 1, om.ns + 1))
    rc = lib().orc_jac_conc(om.ptr, float(P), _p(phi), _p(J))
    return J, rc


def to_conc(mech, Y, T, P):
    """phi = [T, V, n_0..n_{ns-2}] per unit mass of the states (Y [ns, n] or
    [ns], T, P): n_k = Y_k / W_k, V = Ru T sum_k (Y_k / W_k) / P."""
    W = np.asarray(mech.W, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    nk = Y / (W[:, None] if Y.ndim == 2 else W)
    V = RU * np.asarray(T, dtype=np.float64) * nk.sum(axis=0) / np.asarray(P, dtype=np.float64)
    return np.concatenate([np.atleast_1d(T)[None] if Y.ndim == 2 else [T],
                           np.atleast_1d(V)[None] if Y.ndim == 2 else [V], nk[:-1]])


def from_conc(mech, phi, P):
    """(Y [ns, ...], T) of phi: the bath gas's moles close P V = n Ru T and
    Y_k = W_k n_k over the mixture's mass."""
    W = np.asarray(mech.W, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    T, V, n = phi[0], phi[1], phi[2:]
    nin = np.asarray(P, dtype=np.float64) * V / (RU * T) - n.sum(axis=0)
    nall = np.concatenate([n, np.asarray(nin)[None]])
    w = W[:, None] if phi.ndim == 2 else W
    mass = (w * nall).sum(axis=0)
    return w * nall / mass, T


def rate_constants(mech, T, Cc):
    om = _as_om(mech)
    Cc = np.ascontiguousarray(Cc, dtype=np.float64)
    kf, kr = np.zeros(om.nr), np.zeros(om.nr)
    lib().orc_rate_constants(om.ptr, float(T), _p(Cc), _p(kf), _p(kr))
    return kf, kr


def wdot(mech, T, P, Yfull):
    om = _as_om(mech)
    Yfull = np.ascontiguousarray(Yfull, dtype=np.float64)
    w = np.zeros(om.ns)
    lib().orc_wdot(om.ptr, float(T), float(P), _p(Yfull), _p(w))
    return w


def lu_real(a):
    a = np.array(a, dtype=np.float64, order="C")
    n = a.shape[0]
    ip = np.zeros(n, dtype=np.int32)
    rc = lib().orc_lu_real(n, _p(a), _p(ip))
    return a, ip, rc


def lu_solve_real(lu, ip, b):
    b = np.array(b, dtype=np.float64)
    lib().orc_lu_solve_real(lu.shape[0], _p(lu), _p(ip), _p(b))
    return b


def lu_cplx(a):
    a = np.array(a, dtype=np.complex128, order="C")
    n = a.shape[0]
    ip = np.zeros(n, dtype=np.int32)
    rc = lib().orc_lu_cplx(n, _p(a), _p(ip))
    return a, ip, rc


def lu_solve_cplx(lu, ip, b):
    b = np.array(b, dtype=np.complex128)
    lib().orc_lu_solve_cplx(lu.shape[0], _p(lu), _p(ip), _p(b))
    return b


def tableau():
    tb = _Tableau()
    lib().orc_radau_tableau(C.byref(tb))
    return dict(c=np.array(tb.c), A=np.array(tb.A).reshape(3, 3), b=np.array(tb.b),
                gamma=tb.gamma, alpha=tb.alpha, beta=tb.beta,
                T=np.array(tb.T).reshape(3, 3), TI=np.array(tb.TI).reshape(3, 3),
                e=np.array(tb.e), gamma0=tb.gamma0)


def make_opts(rtol=1e-6, atol=1e-10, transform_tol=True, nit=7, h0=0.0, hfixed=0.0,
              max_steps=100000, jac_kind=0, z0=None, z_first_out=None, form=0,
              atol_scale=None):
    o = _Opts(rtol, atol, int(transform_tol), nit, h0, hfixed, max_steps, jac_kind,
              None if z0 is None else _p(z0).value,
              None if z_first_out is None else _p(z_first_out).value, int(form),
              None if atol_scale is None else _p(atol_scale).value)
    return o


def _rhs_callback(f, n, err):
    """A C right-hand-side callback around f(t, y) -> array."""
    def _f(ctx, t, yp, fp):
        try:
            v = np.asarray(f(t, np.ctypeslib.as_array(yp, (n,)).copy()), dtype=np.float64)
            if not np.all(np.isfinite(v)):
                return 4
            np.ctypeslib.as_array(fp, (n,))[:] = v
            return 0
        except Exception as e:  # pragma: no cover - surfaced by the caller
            err.append(e)
            return 4
    return RHS_FN(_f)


def initial_step(f, y0, t0, t1, rtol, atol):
    """The oracle's starting-step heuristic (orc_initial_step) for y' = f(t, y)
    at (t0, y0), with the tolerances given as they enter the weights
    atol + rtol |y| (no transform).  Returns (h, right-hand sides used)."""
    n = len(y0)
    y = np.ascontiguousarray(y0, dtype=np.float64)
    err = []
    cf = _rhs_callback(f, n, err)
    f0 = np.ascontiguousarray(f(t0, y.copy()), dtype=np.float64)
    nf = C.c_int(0)
    h = lib().orc_initial_step(n, cf, None, float(t0), float(t1), _p(y), _p(f0), float(rtol),
                               float(atol), C.byref(nf))
    if err:
        raise err[0]
    return float(h), int(nf.value)


def fd_jacobian(f, y, h, scal, t=0.0):
    """The oracle's one-sided difference-quotient Jacobian (orc_fd_jacobian) of a
    generic f(t, y) at y with the internal step h and error weights scal."""
    n = len(y)
    y = np.ascontiguousarray(y, dtype=np.float64)
    scal = np.ascontiguousarray(scal, dtype=np.float64)
    err = []
    cf = _rhs_callback(f, n, err)
    f0 = np.ascontiguousarray(f(t, y.copy()), dtype=np.float64)
    J = np.zeros((n, n))
    rc = lib().orc_fd_jacobian(n, cf, None, float(t), _p(y), _p(f0), float(h), _p(scal), _p(J))
    if err:
        raise err[0]
    return J, rc


def radau(f, jacobian, y0, t0, t1, **kw):
    """Integrate y' = f(t, y) with the oracle's Radau IIA (Python callbacks).

    f(t, y) -> array;  jacobian(t, y) -> (n, n) array.  Returns (y, stats dict).
    """
    n = len(y0)
    y = np.array(y0, dtype=np.float64)
    err = []

    def _f(ctx, t, yp, fp):
        try:
            v = np.asarray(f(t, np.ctypeslib.as_array(yp, (n,)).copy()), dtype=np.float64)
            if not np.all(np.isfinite(v)):
                return 4
            np.ctypeslib.as_array(fp, (n,))[:] = v
            return 0
        except Exception as e:  # pragma: no cover - surfaced below
            err.append(e)
            return 4

    def _j(ctx, t, yp, f0p, h, scalp, Jp):
        try:
            Jv = np.asarray(jacobian(t, np.ctypeslib.as_array(yp, (n,)).copy()), dtype=np.float64)
            np.ctypeslib.as_array(Jp, (n * n,))[:] = Jv.reshape(-1)
            return 0
        except Exception as e:  # pragma: no cover
            err.append(e)
            return 4

    cf, cj = RHS_FN(_f), JAC_FN(_j)
    z0 = kw.pop("z0", None)
    zf = kw.pop("z_first_out", None)
    z0a = None if z0 is None else np.ascontiguousarray(z0, dtype=np.float64)
    o = make_opts(z0=z0a, z_first_out=zf, **kw)
    st = _Stats()
    lib().orc_radau(n, cf, cj, None, float(t0), float(t1), _p(y), C.byref(o), C.byref(st))
    if err:
        raise err[0]
    stats = {k: getattr(st, k) for k in ("nstep", "naccpt", "nrejct", "nfcn", "njac", "ndec",
                                         "nsol", "status", "h_first", "h_last", "err_last")}
    return y, stats


def integrate(mech, states, dt, *, rtol=1e-6, atol=1e-10, jac_kind=0, nthreads=0,
              max_steps=100000, h0=0.0, hfixed=0.0, transform_tol=True, nit=7,
              form="massfrac"):
    """Integrate a batch of states over dt.  Returns (Y, T, counters[n, 8]).
    form "conc" integrates the concentration-based form: the tolerances weigh
    phi = [T, V, n_0..n_{ns-2}], the moles with absolute tolerance atol / W_k."""
    om = _as_om(mech)
    Y = np.array(states.Y, dtype=np.float64, order="C")
    T = np.array(states.T, dtype=np.float64)
    P = np.ascontiguousarray(states.P, dtype=np.float64)
    n = T.shape[0]
    cnt = np.zeros((n, 8), dtype=np.int32)
    o = make_opts(rtol=rtol, atol=atol, jac_kind=jac_kind, max_steps=max_steps, h0=h0,
                  hfixed=hfixed, transform_tol=transform_tol, nit=nit, form=FORMS[form])
    lib().orc_integrate_batch(om.ptr, n, _p(Y), _p(T), _p(P), float(dt), C.byref(o), None,
                              _p(cnt), int(nthreads))
    return Y, T, cnt


def num_threads() -> int:
    return int(lib().orc_num_threads())


def error_norm(y, y_true, atol=1e-10, rtol=1e-6):
    """E_i of Sec. 2.3: the weighted root-mean-square of (y - yhat)/(atol + |yhat| rtol)
    over the state vector, one value per state.  y, y_true: [N, n]."""
    y = np.asarray(y, dtype=np.float64)
    yt = np.asarray(y_true, dtype=np.float64)
    w = (y - yt) / (atol + np.abs(yt) * rtol)
    return np.sqrt(np.mean(w * w, axis=0))


def divergence(d):
    """Warp divergence D of Sec. 3.3 for step counts d[n] grouped in warps of 32."""
    d = np.asarray(d, dtype=np.float64)
    nw = d.shape[0] // 32
    d = d[: nw * 32].reshape(nw, 32)
    mx = d.max(axis=1)
    return 1.0 - d.sum(axis=1) / (32.0 * np.where(mx > 0, mx, 1.0))


def state_vector(states):
    """[N, n] state vectors y = [T, Y_0..Y_{ns-2}] of a ``States`` batch."""
    return np.concatenate([states.T[None, :], states.Y[:-1, :]], axis=0)
