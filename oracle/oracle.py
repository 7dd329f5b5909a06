"""ctypes front end of the CPU oracle -- TEST INFRASTRUCTURE.

Marshals a flat mechanism description (the synthetic generator's ``MechDesc`` arrays) into the
oracle's own C struct and exposes its entry points with numpy arrays.  State vectors are
``y = (T, Y_1..Y_n)``.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from . import build as _build

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class _OMech(C.Structure):
    _fields_ = [("n", C.c_int), ("R", C.c_int),
                ("W", _dp), ("lo", _dp), ("hi", _dp), ("Tmid", _dp),
                ("rptr", _ip), ("rsp", _ip), ("rnu", _ip),
                ("pptr", _ip), ("psp", _ip), ("pnu", _ip),
                ("A", _dp), ("b", _dp), ("Ea", _dp),
                ("type", _ip), ("rev", _ip),
                ("eptr", _ip), ("esp", _ip), ("eval", _dp),
                ("troe", _dp), ("low", _dp)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.oracle_rhs.argtypes = [C.c_void_p, C.c_double, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.oracle_thermo.argtypes = [C.c_void_p, C.c_double, _dp, _dp, _dp]
        L.oracle_jacobian.argtypes = [C.c_void_p, C.c_double, _dp, _dp, _dp]
        L.oracle_jacobian_cs.argtypes = [C.c_void_p, C.c_double, _dp, C.c_double, _dp]
        L.oracle_rhs_param_cs.argtypes = [C.c_void_p, C.c_double, _dp, C.c_int, C.c_int, C.c_double, _dp]
        L.oracle_tableau.argtypes = [C.c_int, _dp]
        L.oracle_step.argtypes = [C.c_void_p, C.c_double, _dp, C.c_double, _dp, _dp, C.c_int]
        L.oracle_integrate.argtypes = [C.c_void_p, C.c_double, _dp, C.c_double, C.c_double, C.c_double,
                                       C.c_double, C.c_int, _dp, _ip, _ip, _dp, _ip, C.c_int, _ip, C.c_int]
        L.oracle_replay.argtypes = [C.c_void_p, C.c_double, _dp, _dp, C.c_int, C.c_int]
        L.oracle_replay_sens_cs.argtypes = [C.c_void_p, C.c_double, _dp, _dp, C.c_int, C.c_int, C.c_int,
                                            C.c_double, _dp]
        L.oracle_integrate_batch.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp, C.c_double, C.c_double,
                                             C.c_int, _dp, _ip, _ip, _ip, C.c_int, _dp, C.c_int, C.c_int]
        L.oracle_integrate_batch_tab.argtypes = L.oracle_integrate_batch.argtypes + [C.c_void_p]
        L.oracle_replay_tab.argtypes = [C.c_void_p, C.c_double, _dp, _dp, C.c_int, C.c_int, C.c_void_p]
        L.oracle_tab_build.argtypes = [C.c_void_p, C.c_double]
        L.oracle_tab_build.restype = C.c_void_p
        L.oracle_tab_free.argtypes = [C.c_void_p]
        L.oracle_tab_info.argtypes = [C.c_void_p, _ip, _dp]
        L.oracle_tab_eval.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_double]
        L.oracle_tab_eval.restype = C.c_double
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _i(a):
    return a.ctypes.data_as(_ip) if a is not None else None


STATUS = {0: "OK", 1: "MAXSTEPS", 2: "HMIN", 3: "NONFINITE", 4: "BADINPUT"}


class Oracle:
    """The oracle bound to one mechanism (keeps the marshalled arrays alive)."""

    def __init__(self, mech):
        self.mech = mech
        self.n = mech.n_species
        self.R = mech.n_reactions
        self.m = self.n + 1
        f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
        self._keep = dict(
            W=f64(mech.W), lo=f64(mech.nasa_lo).ravel(), hi=f64(mech.nasa_hi).ravel(), Tmid=f64(mech.T_mid),
            rptr=i32(mech.reac_ptr), rsp=i32(mech.reac_sp), rnu=i32(mech.reac_nu),
            pptr=i32(mech.prod_ptr), psp=i32(mech.prod_sp), pnu=i32(mech.prod_nu),
            A=f64(mech.A), b=f64(mech.b), Ea=f64(mech.Ea), type=i32(mech.rtype), rev=i32(mech.reversible),
            eptr=i32(mech.eff_ptr), esp=i32(mech.eff_sp), eval=f64(mech.eff_alpha),
            troe=f64(mech.troe).ravel(), low=f64(mech.low).ravel())
        k = self._keep
        self._s = _OMech(self.n, self.R, _d(k["W"]), _d(k["lo"]), _d(k["hi"]), _d(k["Tmid"]),
                         _i(k["rptr"]), _i(k["rsp"]), _i(k["rnu"]), _i(k["pptr"]), _i(k["psp"]), _i(k["pnu"]),
                         _d(k["A"]), _d(k["b"]), _d(k["Ea"]), _i(k["type"]), _i(k["rev"]),
                         _i(k["eptr"]), _i(k["esp"]), _d(k["eval"]), _d(k["troe"]), _d(k["low"]))
        self._p = C.addressof(self._s)
        self.L = lib()

    # -------------------------------------------------------------- pointwise
    def state(self, T, Y):
        y = np.empty(self.m)
        y[0] = T
        y[1:] = Y
        return y

    def rhs(self, T, p, Y, want_gross=False):
        """Returns dict: f (m), wdot (n), gross (m) [if asked], qf, qr, kf, kr (R)."""
        y = self.state(T, Y)
        f = np.empty(self.m); w = np.empty(self.n)
        g = np.empty(self.m) if want_gross else None
        qf, qr, kf, kr = (np.empty(self.R) for _ in range(4))
        self.L.oracle_rhs(self._p, p, _d(y), _d(f), _d(w), _d(g), _d(qf), _d(qr), _d(kf), _d(kr))
        return dict(f=f, wdot=w, gross=g, qf=qf, qr=qr, kf=kf, kr=kr)

    def thermo(self, T):
        cp, h, s = np.empty(self.n), np.empty(self.n), np.empty(self.n)
        self.L.oracle_thermo(self._p, T, _d(cp), _d(h), _d(s))
        return cp, h, s

    def jacobian(self, T, p, Y, want_gross=False):
        y = self.state(T, Y)
        J = np.empty((self.m, self.m))
        G = np.empty((self.m, self.m)) if want_gross else None
        self.L.oracle_jacobian(self._p, p, _d(y), _d(J), _d(G))
        return (J, G) if want_gross else J

    def jacobian_cs(self, T, p, Y, eps=1e-30):
        y = self.state(T, Y)
        J = np.empty((self.m, self.m))
        self.L.oracle_jacobian_cs(self._p, p, _d(y), eps, _d(J))
        return J

    def rhs_param_cs(self, T, p, Y, kind, j, eps=1e-30):
        y = self.state(T, Y)
        df = np.empty(self.m)
        self.L.oracle_rhs_param_cs(self._p, p, _d(y), kind, j, eps, _d(df))
        return df

    def tableau(self, method=0):
        """Coefficients of method 0 (RODAS3), 1 (ROS2) or 2 (RODAS4) in the k-form of the oracle's step
        (arrays padded to six stages)."""
        S = 6
        out = np.zeros(2 + 2 * S * S + 2 * S + 1)
        self.L.oracle_tableau(method, _d(out))
        o = 2 + 2 * S * S
        return dict(s=int(out[0]), gamma=out[1], alpha=out[2:2 + S * S].reshape(S, S),
                    gam=out[2 + S * S:o].reshape(S, S), b=out[o:o + S].copy(), bhat=out[o + S:o + 2 * S].copy(),
                    err_order=int(out[o + 2 * S]))

    def step(self, y, p, h, method=0):
        y = np.ascontiguousarray(y, dtype=np.float64)
        yn, ye = np.empty(self.m), np.empty(self.m)
        rc = self.L.oracle_step(self._p, p, _d(y), h, _d(yn), _d(ye), method)
        if rc:
            raise RuntimeError("singular iteration matrix")
        return yn, ye

    # -------------------------------------------------------------- integration
    def integrate(self, T, p, Y, dt, rtol=1e-6, atol=1e-12, h0=0.0, max_steps=100000, trace=False, method=0):
        y = self.state(T, Y)
        h_out = C.c_double(0.0); ns = C.c_int(0); na = C.c_int(0); tl = C.c_int(0)
        cap = 200000 if trace else 0
        th = np.empty(cap) if trace else None
        ta = np.empty(cap, dtype=np.int32) if trace else None
        st = self.L.oracle_integrate(self._p, p, _d(y), dt, rtol, atol, h0, max_steps, C.byref(h_out),
                                     C.byref(ns), C.byref(na), _d(th), _i(ta), cap, C.byref(tl), method)
        out = dict(T=y[0], Y=y[1:].copy(), y=y, h=h_out.value, nsub=ns.value, nacc=na.value, status=st)
        if trace:
            L = min(tl.value, cap)
            out["trace_h"] = th[:L].copy()
            out["trace_acc"] = ta[:L].copy()
        return out

    # -------------------------------------------------------------- tabulated temperature functions
    def tab_build(self, tol=1e-10):
        """Build (once per tolerance) the oracle's own tables of exp(+-g_k), k_f and F_cent; returns
        (handle, degrees[4], interval count, range (T_lo, T_hi, u_lo, du))."""
        if not hasattr(self, "_tabs"):
            self._tabs = {}
        if tol not in self._tabs:
            t = self.L.oracle_tab_build(self._p, tol)
            deg = np.zeros(4, dtype=np.int32)
            rng = np.zeros(4)
            ni = self.L.oracle_tab_info(t, _i(deg), _d(rng))
            self._tabs[tol] = (t, deg, ni, rng)
        return self._tabs[tol]

    def tab_eval(self, tol, cls, f, T):
        t = self.tab_build(tol)[0]
        return self.L.oracle_tab_eval(self._p, t, cls, f, float(T))

    def __del__(self):
        try:
            for t in getattr(self, "_tabs", {}).values():
                self.L.oracle_tab_free(t[0])
        except Exception:
            pass

    def replay(self, y0, p, hs, method=0, tab_tol=0.0):
        y = np.array(y0, dtype=np.float64)
        hs = np.ascontiguousarray(hs, dtype=np.float64)
        if tab_tol > 0:
            rc = self.L.oracle_replay_tab(self._p, p, _d(y), _d(hs), len(hs), method, self.tab_build(tab_tol)[0])
            if rc:
                raise RuntimeError("singular iteration matrix in replay")
            return y
        rc = self.L.oracle_replay(self._p, p, _d(y), _d(hs), len(hs), method)
        if rc:
            raise RuntimeError("singular iteration matrix in replay")
        return y

    def replay_sens_cs(self, y0, p, hs, kind, j, eps=1e-30):
        y0 = np.ascontiguousarray(y0, dtype=np.float64)
        hs = np.ascontiguousarray(hs, dtype=np.float64)
        dy = np.empty(self.m)
        rc = self.L.oracle_replay_sens_cs(self._p, p, _d(y0), _d(hs), len(hs), kind, j, eps, _d(dy))
        if rc:
            raise RuntimeError("singular iteration matrix in replay")
        return dy

    def integrate_batch(self, T, p, Y, dt, rtol=1e-6, atol=1e-12, h_io=None, max_steps=100000, nthreads=0,
                        trace_cap=0, method=0, tab_tol=0.0):
        """Structure-of-arrays batch (Y[k, c]); returns a dict of new arrays and the thread count."""
        N = int(T.shape[0])
        T = np.array(T, dtype=np.float64)
        Yc = np.array(Y, dtype=np.float64, order="C")
        p = np.ascontiguousarray(p, dtype=np.float64)
        dt = np.ascontiguousarray(dt, dtype=np.float64)
        h = np.zeros(N) if h_io is None else np.array(h_io, dtype=np.float64)
        ns = np.zeros(N, dtype=np.int32); na = np.zeros(N, dtype=np.int32); st = np.zeros(N, dtype=np.int32)
        tr = np.zeros((trace_cap, N)) if trace_cap > 0 else None
        tab = self.tab_build(tab_tol)[0] if tab_tol > 0 else None
        used = self.L.oracle_integrate_batch_tab(self._p, N, _d(T), _d(p), _d(Yc), _d(dt), rtol, atol, max_steps,
                                                 _d(h), _i(ns), _i(na), _i(st), nthreads, _d(tr), trace_cap, method,
                                                 tab)
        out = dict(T=T, Y=Yc, h=h, nsub=ns, nacc=na, status=st, threads=used)
        if tr is not None:
            out["trace"] = tr
        return out
