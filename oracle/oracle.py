"""ctypes loader for the FP64 CPU oracle (conv_oracle.cpp).

TEST INFRASTRUCTURE: imported only by the tests, the smoke check and the
benchmark's CPU-baseline leg.  The product library never imports this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "conv_oracle.cpp")
LIB = os.path.join(HERE, "libconv_oracle.so")
# Tests that plant mistakes in a copy of the oracle point this at the mutant.
_OVERRIDE = os.environ.get("CONV_ORACLE_LIB")

F_TRIGGERED, F_ACTIVE, F_LIMITED, F_NEWTON, F_BADINPUT = 1, 2, 4, 8, 16
EXIT_SHIFT = 8


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2 -ffp-contract=off, OpenMP)."""
    stale = (not os.path.exists(LIB)) or os.path.getmtime(LIB) < max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "conv_oracle.h")))
    if force or stale:
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c++17",
               "-o", tmp, SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


class DeepParams(C.Structure):
    _fields_ = [("capelmt", C.c_double), ("lambda_default", C.c_double),
                ("tau_default", C.c_double), ("c0", C.c_double), ("alpha_dd", C.c_double),
                ("p_launch_min", C.c_double), ("p_top_lim", C.c_double), ("q_min", C.c_double),
                ("ent_zscale", C.c_double), ("n_newton_lcl", C.c_int32),
                ("n_newton_h", C.c_int32), ("n_plumes", C.c_int32), ("reserved", C.c_int32),
                ("plume_spread", C.c_double)]


class ShallowParams(C.Structure):
    _fields_ = [("eps_s", C.c_double), ("tke", C.c_double), ("c_m", C.c_double),
                ("cin_scale", C.c_double), ("cin_max", C.c_double), ("a_w", C.c_double),
                ("b_w", C.c_double), ("ql_crit", C.c_double), ("p_lcl_min", C.c_double),
                ("p_lfc_min", C.c_double), ("p_top_lim", C.c_double),
                ("n_newton_lcl", C.c_int32), ("n_newton_h", C.c_int32), ("evap_k", C.c_double)]


def deep_params(**kw) -> DeepParams:
    d = dict(capelmt=70.0, lambda_default=1e-3, tau_default=3600.0, c0=2e-3, alpha_dd=0.2,
             p_launch_min=60000.0, p_top_lim=4000.0, q_min=1e-12, ent_zscale=1000.0,
             n_newton_lcl=6, n_newton_h=15, n_plumes=1, reserved=0, plume_spread=4.0)
    d.update(kw)
    return DeepParams(**d)


def shallow_params(**kw) -> ShallowParams:
    d = dict(eps_s=2e-3, tke=1.0, c_m=0.03, cin_scale=10.0, cin_max=50.0, a_w=1.0, b_w=2.0,
             ql_crit=1e-3, p_lcl_min=70000.0, p_lfc_min=50000.0, p_top_lim=4000.0,
             n_newton_lcl=6, n_newton_h=15, evap_k=0.0)
    d.update(kw)
    return ShallowParams(**d)


class Out(C.Structure):
    _fields_ = [("dTdt", C.c_void_p), ("dqdt", C.c_void_p), ("prec", C.c_void_p),
                ("flags", C.c_void_p), ("kb", C.c_void_p), ("klcl", C.c_void_p),
                ("ktop", C.c_void_p), ("kaux", C.c_void_p), ("cape", C.c_void_p),
                ("mb", C.c_void_p), ("cons_err", C.c_void_p)]


class Flux(C.Structure):
    _fields_ = [("mu", C.c_void_p), ("du", C.c_void_p), ("md", C.c_void_p)]


N32 = 32


class DeepDiag(C.Structure):
    _fields_ = ([(n, C.c_int32) for n in
                 ("k_top_lim", "kb", "klcl", "kel", "khmin", "jt", "jd", "triggered", "active",
                  "limited")]
                + [(n, C.c_double) for n in
                   ("TL", "pL", "cape", "F", "mb", "sumR", "sumE", "alpha_eff", "prec")]
                + [(n, C.c_double * N32) for n in
                   ("Tp", "qp", "b", "eta", "hu", "qtu", "rain", "etad", "hd", "qd", "E1",
                    "dh", "dq", "dT", "m", "z_mid")]
                + [("z_int", C.c_double * 33)]
                + [(n, C.c_double * N32) for n in ("h", "hs", "p_mid")]
                + [("p_int", C.c_double * 33)])


class ShallowDiag(C.Structure):
    _fields_ = ([(n, C.c_int32) for n in
                 ("k_top_lim", "klcl", "klfc", "kts", "exit_code", "active")]
                + [(n, C.c_double) for n in ("TL", "pL", "cin", "mb", "prec")]
                + [(n, C.c_double * N32) for n in
                   ("b", "hu", "qtu", "qtpre", "w2", "rf", "Tu", "dh", "dq", "dT", "m", "z_mid")]
                + [("z_int", C.c_double * 33)]
                + [(n, C.c_double * N32) for n in ("h", "p_mid")]
                + [("p_int", C.c_double * 33)])


_lib = None


def lib():
    global _lib
    if _lib is None:
        if _OVERRIDE:
            L = C.CDLL(_OVERRIDE)
        else:
            build()
            L = C.CDLL(LIB)
        d, i, p = C.c_double, C.c_int, C.c_void_p
        L.oracle_es.restype = d
        L.oracle_es.argtypes = [d]
        L.oracle_qs.restype = d
        L.oracle_qs.argtypes = [d, d]
        L.oracle_dqsdT.restype = d
        L.oracle_dqsdT.argtypes = [d, d]
        L.oracle_lcl.restype = d
        L.oracle_lcl.argtypes = [d, d, d, i, C.POINTER(d), C.POINTER(d)]
        L.oracle_hinv.restype = d
        L.oracle_hinv.argtypes = [d, d, d, d, i, C.POINTER(d)]
        L.oracle_heights.argtypes = [i, p, p, p, p, p, p]
        L.oracle_levels.argtypes = [i, p, p, d, d, p, p]
        L.oracle_deep_column_diag.argtypes = [i, p, p, d, p, p, d, d, d, C.POINTER(DeepParams), d,
                                              C.POINTER(DeepDiag)]
        L.oracle_shallow_column_diag.argtypes = [i, p, p, d, p, p, d, C.POINTER(ShallowParams),
                                                 C.POINTER(ShallowDiag)]
        L.oracle_deep.argtypes = [i, i, i, p, p, d, p, p, p, p, p, C.POINTER(DeepParams), d,
                                  C.POINTER(Out), i]
        L.oracle_shallow.argtypes = [i, i, i, p, p, d, p, p, p, C.POINTER(ShallowParams),
                                     C.POINTER(Out), i]
        L.oracle_deep_shallow.argtypes = [i, i, i, p, p, d, p, p, p, p, p, C.POINTER(DeepParams),
                                          C.POINTER(ShallowParams), d, C.POINTER(Out),
                                          C.POINTER(Out), i]
        L.oracle_deep_adjoint.argtypes = [i, i, i, p, p, d, p, p, p, p, p, C.POINTER(DeepParams),
                                          d, p, p, p, p, p, p, p, i]
        L.oracle_deep_shallow_adjoint.argtypes = [i, i, i, p, p, d, p, p, p, p, p,
                                                  C.POINTER(DeepParams), C.POINTER(ShallowParams),
                                                  d, p, p, p, p, p, p, p, p, p, i]
        L.oracle_deep_shallow_tracers.argtypes = [i, i, i, p, p, d, p, p, p, p, p,
                                                  C.POINTER(DeepParams), C.POINTER(ShallowParams),
                                                  d, i, p, p, p, C.POINTER(Flux), C.POINTER(Flux),
                                                  i]
        L.oracle_count_ops.argtypes = [i, i, i, p, p, d, p, p, p, C.POINTER(DeepParams),
                                       C.POINTER(ShallowParams), d, p, p]
        L.oracle_count_ops_by_pass.argtypes = [i, i, i, p, p, d, p, p, p, C.POINTER(DeepParams),
                                               C.POINTER(ShallowParams), d, p, p, p, p]
        L.oracle_deep_shallow_momentum.argtypes = [i, i, i, p, p, d, p, p, p, p, p,
                                                   C.POINTER(DeepParams),
                                                   C.POINTER(ShallowParams), d, d, d, p, p, p,
                                                   i]
        L.oracle_deep_shallow_counted.argtypes = [i, i, i, p, p, d, p, p, p,
                                                  C.POINTER(DeepParams), C.POINTER(ShallowParams),
                                                  d, C.POINTER(Out), C.POINTER(Out)]
        for fn in ("oracle_deep", "oracle_shallow", "oracle_deep_shallow", "oracle_deep_adjoint",
                   "oracle_deep_shallow_tracers", "oracle_deep_shallow_counted",
                   "oracle_deep_shallow_momentum",
                   "oracle_deep_shallow_adjoint", "oracle_count_ops", "oracle_count_ops_by_pass"):
            getattr(L, fn).restype = i
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _c64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def new_out(pver: int, ld: int) -> dict:
    return dict(dTdt=np.zeros((pver, ld)), dqdt=np.zeros((pver, ld)), prec=np.zeros(ld),
                flags=np.zeros(ld, np.int32), kb=np.zeros(ld, np.int32),
                klcl=np.zeros(ld, np.int32), ktop=np.zeros(ld, np.int32),
                kaux=np.zeros(ld, np.int32), cape=np.zeros(ld), mb=np.zeros(ld),
                cons_err=np.zeros(ld))


def _out_struct(o: dict) -> Out:
    return Out(*[o[n].ctypes.data for n in ("dTdt", "dqdt", "prec", "flags", "kb", "klcl", "ktop",
                                            "kaux", "cape", "mb", "cons_err")])


def _trim(o: dict, n: int) -> dict:
    return {k: (v[:, :n] if v.ndim == 2 else v[:n]) for k, v in o.items()}


def deep(g, par: DeepParams | None = None, dt: float | None = None, threads: int = 1,
         lam=None, tau=None) -> dict:
    """Deep scheme over a ``soundings.Columns`` grid; returns [pver][n] / [n] arrays."""
    par = par or deep_params()
    dt = g.dt if dt is None else dt
    T, q, ps = _c64(g.T), _c64(g.q), _c64(g.ps)
    lam = _c64(lam if lam is not None else g.lam)
    tau = _c64(tau if tau is not None else g.tau)
    n, pver = g.n_cols, g.pver
    o = new_out(pver, n)
    hyai, hybi = _c64(g.hyai), _c64(g.hybi)
    rc = lib().oracle_deep(n, pver, n, _ptr(hyai), _ptr(hybi), 1e5, _ptr(T), _ptr(q), _ptr(ps),
                           _ptr(lam), _ptr(tau), C.byref(par), dt, C.byref(_out_struct(o)), threads)
    assert rc == 0
    return o


def shallow(g, par: ShallowParams | None = None, threads: int = 1, T=None, q=None) -> dict:
    par = par or shallow_params()
    T = _c64(g.T if T is None else T)
    q = _c64(g.q if q is None else q)
    ps = _c64(g.ps)
    n, pver = g.n_cols, g.pver
    o = new_out(pver, n)
    hyai, hybi = _c64(g.hyai), _c64(g.hybi)
    rc = lib().oracle_shallow(n, pver, n, _ptr(hyai), _ptr(hybi), 1e5, _ptr(T), _ptr(q),
                              _ptr(ps), C.byref(par), C.byref(_out_struct(o)), threads)
    assert rc == 0
    return o


def deep_shallow(g, dpar=None, spar=None, dt=None, threads: int = 1, lam=None, tau=None):
    """Deep then shallow (on the deep-updated state); returns (deep_out, shallow_out)."""
    dpar = dpar or deep_params()
    spar = spar or shallow_params()
    dt = g.dt if dt is None else dt
    T, q, ps = _c64(g.T), _c64(g.q), _c64(g.ps)
    lam = _c64(lam if lam is not None else g.lam)
    tau = _c64(tau if tau is not None else g.tau)
    n, pver = g.n_cols, g.pver
    od, os_ = new_out(pver, n), new_out(pver, n)
    hyai, hybi = _c64(g.hyai), _c64(g.hybi)
    rc = lib().oracle_deep_shallow(n, pver, n, _ptr(hyai), _ptr(hybi), 1e5, _ptr(T), _ptr(q),
                                   _ptr(ps), _ptr(lam), _ptr(tau), C.byref(dpar), C.byref(spar),
                                   dt, C.byref(_out_struct(od)), C.byref(_out_struct(os_)),
                                   threads)
    assert rc == 0
    return od, os_


def deep_shallow_tracers(g, tracers, dpar=None, spar=None, dt=None, threads: int = 1, lam=None,
                         tau=None, T=None, q=None):
    """Convective transport of passive tracers ([ntr][pver][n]) by the fused step.

    Returns (tend_deep, tend_shallow, flux_deep, flux_shallow): tendencies
    [ntr][pver][n] (the shallow one of the deep-updated tracers) and dicts of the
    mass-flux profiles mu, du, md ([pver][n])."""
    dpar = dpar or deep_params()
    spar = spar or shallow_params()
    dt = g.dt if dt is None else dt
    T = _c64(g.T if T is None else T)
    q = _c64(g.q if q is None else q)
    ps = _c64(g.ps)
    lam = _c64(lam if lam is not None else g.lam)
    tau = _c64(tau if tau is not None else g.tau)
    n, pver = g.n_cols, g.pver
    tr = _c64(tracers)
    assert tr.ndim == 3 and tr.shape[1:] == (pver, n), tr.shape
    ntr = tr.shape[0]
    td, ts = np.zeros_like(tr), np.zeros_like(tr)
    fd = {k: np.zeros((pver, n)) for k in ("mu", "du", "md")}
    fs = {k: np.zeros((pver, n)) for k in ("mu", "du", "md")}
    hyai, hybi = _c64(g.hyai), _c64(g.hybi)
    rc = lib().oracle_deep_shallow_tracers(
        n, pver, n, _ptr(hyai), _ptr(hybi), 1e5, _ptr(T), _ptr(q), _ptr(ps), _ptr(lam), _ptr(tau),
        C.byref(dpar), C.byref(spar), dt, ntr, _ptr(tr), _ptr(td), _ptr(ts),
        C.byref(Flux(*[fd[k].ctypes.data for k in ("mu", "du", "md")])),
        C.byref(Flux(*[fs[k].ctypes.data for k in ("mu", "du", "md")])), threads)
    assert rc == 0
    return td, ts, fd, fs


def deep_shallow_momentum(g, uv, c_up=0.7, c_down=0.7, dpar=None, spar=None, dt=None,
                          threads: int = 1, lam=None, tau=None):
    """Convective momentum transport of the wind components uv ([2][pver][n], u
    then v) by the fused step, with the plumes' pressure-gradient coefficients.
    Returns (tend_deep, tend_shallow), each [2][pver][n]."""
    dpar = dpar or deep_params()
    spar = spar or shallow_params()
    dt = g.dt if dt is None else dt
    T, q, ps = _c64(g.T), _c64(g.q), _c64(g.ps)
    lam = _c64(lam if lam is not None else g.lam)
    tau = _c64(tau if tau is not None else g.tau)
    n, pver = g.n_cols, g.pver
    w = _c64(uv)
    assert w.shape == (2, pver, n), w.shape
    td, ts = np.zeros_like(w), np.zeros_like(w)
    hyai, hybi = _c64(g.hyai), _c64(g.hybi)
    rc = lib().oracle_deep_shallow_momentum(
        n, pver, n, _ptr(hyai), _ptr(hybi), 1e5, _ptr(T), _ptr(q), _ptr(ps), _ptr(lam), _ptr(tau),
        C.byref(dpar), C.byref(spar), dt, float(c_up), float(c_down), _ptr(w), _ptr(td),
        _ptr(ts), threads)
    assert rc == 0
    return td, ts


def deep_adjoint(g, gP, gH, w_heat=None, par=None, dt=None, threads: int = 1, lam=None,
                 tau=None):
    """Tangent-mode gradients of J = gP*P + gH*sum w m cp dTdt (deep scheme)."""
    par = par or deep_params()
    dt = g.dt if dt is None else dt
    n, pver = g.n_cols, g.pver
    T, q, ps = _c64(g.T), _c64(g.q), _c64(g.ps)
    lam = _c64(lam if lam is not None else g.lam)
    tau = _c64(tau if tau is not None else g.tau)
    gP, gH, w = _c64(gP), _c64(gH), _c64(w_heat)
    gT, gq = np.zeros((pver, n)), np.zeros((pver, n))
    gl, gt = np.zeros(n), np.zeros(n)
    hyai, hybi = _c64(g.hyai), _c64(g.hybi)
    rc = lib().oracle_deep_adjoint(n, pver, n, _ptr(hyai), _ptr(hybi), 1e5, _ptr(T), _ptr(q),
                                   _ptr(ps), _ptr(lam), _ptr(tau), C.byref(par), dt, _ptr(gP),
                                   _ptr(gH), _ptr(w), _ptr(gT), _ptr(gq), _ptr(gl), _ptr(gt),
                                   threads)
    assert rc == 0
    return gT, gq, gl, gt


def deep_shallow_adjoint(g, gPd=None, gHd=None, gPs=None, gHs=None, w_heat=None, dpar=None,
                         spar=None, dt=None, threads: int = 1, lam=None, tau=None):
    """Tangent-mode gradients of J = gPd*Pd + gHd*Hd + gPs*Ps + gHs*Hs of the fused
    deep -> shallow step, H = sum w m cp dTdt of each scheme."""
    dpar = dpar or deep_params()
    spar = spar or shallow_params()
    dt = g.dt if dt is None else dt
    n, pver = g.n_cols, g.pver
    T, q, ps = _c64(g.T), _c64(g.q), _c64(g.ps)
    lam = _c64(lam if lam is not None else g.lam)
    tau = _c64(tau if tau is not None else g.tau)
    seeds = [_c64(x) for x in (gPd, gHd, gPs, gHs)]
    w = _c64(w_heat)
    gT, gq = np.zeros((pver, n)), np.zeros((pver, n))
    gl, gt = np.zeros(n), np.zeros(n)
    hyai, hybi = _c64(g.hyai), _c64(g.hybi)
    rc = lib().oracle_deep_shallow_adjoint(
        n, pver, n, _ptr(hyai), _ptr(hybi), 1e5, _ptr(T), _ptr(q), _ptr(ps), _ptr(lam),
        _ptr(tau), C.byref(dpar), C.byref(spar), dt, *[_ptr(x) for x in seeds], _ptr(w),
        _ptr(gT), _ptr(gq), _ptr(gl), _ptr(gt), threads)
    assert rc == 0
    return gT, gq, gl, gt


def advance(T, q, deep, shallow, dt, T_relax=None, q_relax=None, tau_relax=0.0):
    """State advance of the multi-step column driver (numpy, FP64):
    T + dt*((dTdt_deep + dTdt_shallow) + (T_relax - T)/tau_relax), likewise q,
    floored at 0; no relaxation for tau_relax <= 0."""
    rt = 1.0 / tau_relax if tau_relax > 0 else 0.0
    Tr = T if T_relax is None else T_relax
    qr = q if q_relax is None else q_relax
    fT = (deep["dTdt"] + shallow["dTdt"]) + (Tr - T) * rt
    fq = (deep["dqdt"] + shallow["dqdt"]) + (qr - q) * rt
    return T + dt * fT, np.maximum(q + dt * fq, 0.0)


def column_model(g, steps, tau_relax=86400.0, threads: int = 1, record=None):
    """Runs the oracle's fused step `steps` times from g's state, relaxing towards
    the initial profiles; record(step, T, q, deep, shallow) after every step.
    Returns the final (T, q)."""
    import copy
    T, q = g.T.copy(), g.q.copy()
    for s in range(steps):
        sub = copy.copy(g)
        sub.T, sub.q = T, q
        d, sh = deep_shallow(sub, threads=threads)
        T, q = advance(T, q, d, sh, g.dt, g.T, g.q, tau_relax)
        if record:
            record(s, T, q, d, sh)
    return T, q


def count_ops(g, dpar=None, spar=None, dt=None):
    """Operation counts (add, mul, div, exp, log, pow, sqrt, -) summed over columns."""
    dpar = dpar or deep_params()
    spar = spar or shallow_params()
    dt = g.dt if dt is None else dt
    T, q, ps = _c64(g.T), _c64(g.q), _c64(g.ps)
    cd, ct = np.zeros(8), np.zeros(8)
    hyai, hybi = _c64(g.hyai), _c64(g.hybi)
    rc = lib().oracle_count_ops(g.n_cols, g.pver, g.n_cols, _ptr(hyai), _ptr(hybi), 1e5, _ptr(T),
                                _ptr(q), _ptr(ps), C.byref(dpar), C.byref(spar), dt, _ptr(cd),
                                _ptr(ct))
    assert rc == 0
    return cd, ct


def count_ops_by_pass(g, dpar=None, spar=None, dt=None, e2=False):
    """(trigger_pass[13], plume_pass[13], n_triggered) summed over g's columns;
    with e2=True also the E2 LFC-search operations (8 categories)."""
    dpar = dpar or deep_params()
    spar = spar or shallow_params()
    dt = g.dt if dt is None else dt
    T, q, ps = _c64(g.T), _c64(g.q), _c64(g.ps)
    a, b, nt, e = np.zeros(13), np.zeros(13), np.zeros(1), np.zeros(8)
    hyai, hybi = _c64(g.hyai), _c64(g.hybi)
    rc = lib().oracle_count_ops_by_pass(g.n_cols, g.pver, g.n_cols, _ptr(hyai), _ptr(hybi), 1e5,
                                        _ptr(T), _ptr(q), _ptr(ps), C.byref(dpar), C.byref(spar),
                                        dt, _ptr(a), _ptr(b), _ptr(nt), _ptr(e))
    assert rc == 0
    return (a, b, float(nt[0]), e) if e2 else (a, b, float(nt[0]))


def deep_shallow_counted(g, dpar=None, spar=None, dt=None):
    """The fused step through the counting instantiation (default lambda, tau):
    (deep, shallow) output dicts as deep_shallow returns them."""
    dpar = dpar or deep_params()
    spar = spar or shallow_params()
    dt = g.dt if dt is None else dt
    n, pver = g.n_cols, g.pver
    T, q, ps = _c64(g.T), _c64(g.q), _c64(g.ps)
    hyai, hybi = _c64(g.hyai), _c64(g.hybi)
    od, os_ = new_out(pver, n), new_out(pver, n)
    rc = lib().oracle_deep_shallow_counted(n, pver, n, _ptr(hyai), _ptr(hybi), 1e5, _ptr(T),
                                           _ptr(q), _ptr(ps), C.byref(dpar), C.byref(spar), dt,
                                           C.byref(_out_struct(od)), C.byref(_out_struct(os_)))
    assert rc == 0
    return od, os_


def deep_column_diag(pver, hyai, hybi, T, q, ps, lam=1e-3, tau=3600.0, par=None, dt=1800.0):
    par = par or deep_params()
    d = DeepDiag()
    T, q = _c64(T), _c64(q)
    hyai, hybi = _c64(hyai), _c64(hybi)
    lib().oracle_deep_column_diag(pver, _ptr(hyai), _ptr(hybi), 1e5, _ptr(T), _ptr(q), ps, lam,
                                  tau, C.byref(par), dt, C.byref(d))
    return d


def shallow_column_diag(pver, hyai, hybi, T, q, ps, par=None):
    par = par or shallow_params()
    d = ShallowDiag()
    T, q = _c64(T), _c64(q)
    hyai, hybi = _c64(hyai), _c64(hybi)
    lib().oracle_shallow_column_diag(pver, _ptr(hyai), _ptr(hybi), 1e5, _ptr(T), _ptr(q), ps,
                                     C.byref(par), C.byref(d))
    return d


def es(T):
    return lib().oracle_es(float(T))


def qs(T, p):
    return lib().oracle_qs(float(T), float(p))


def dqsdT(T, p):
    return lib().oracle_dqsdT(float(T), float(p))


def lcl(Tb, qb, pb, n_newton=6):
    TL, pL = C.c_double(), C.c_double()
    last = lib().oracle_lcl(float(Tb), float(qb), float(pb), n_newton, C.byref(TL), C.byref(pL))
    return TL.value, pL.value, last


def hinv(h, gz, p, T_start, n_extra=15):
    last = C.c_double()
    T = lib().oracle_hinv(float(h), float(gz), float(p), float(T_start), n_extra, C.byref(last))
    return T, last.value


def levels(pver, hyai, hybi, ps):
    p_int, p_mid = np.zeros(pver + 1), np.zeros(pver)
    hyai, hybi = _c64(hyai), _c64(hybi)
    lib().oracle_levels(pver, _ptr(hyai), _ptr(hybi), 1e5, float(ps), _ptr(p_int), _ptr(p_mid))
    return p_int, p_mid


def heights(T, q, p_int, p_mid):
    pver = len(T)
    z_int, z_mid = np.zeros(pver + 1), np.zeros(pver)
    T, q, p_int, p_mid = _c64(T), _c64(q), _c64(p_int), _c64(p_mid)
    lib().oracle_heights(pver, _ptr(T), _ptr(q), _ptr(p_int), _ptr(p_mid), _ptr(z_int),
                         _ptr(z_mid))
    return z_int, z_mid
