"""Pins of the FP64 CPU oracle against facts it does not compute itself.

Each test checks one step of the column schemes against a closed form, a
published value, an independent root finder, a brute-force scan or a different
formulation of the same budget, so that a dropped term, a wrong sign or a
shifted level index in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S
from tests import physics_ref as P

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- saturation
def test_es_reference_table(oracle):
    """Bolton eq. 10 against tabulated saturation vapour pressure (golden file)."""
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "saturation_vapour_pressure.txt"))
            if l.strip() and not l.startswith("#")]
    for tc, es in rows:
        got = oracle.es(273.15 + float(tc))
        assert abs(got / float(es) - 1.0) < 3e-3, (tc, got, es)


def test_es_at_freezing_is_exact(oracle):
    assert oracle.es(273.15) == 611.2


@pytest.mark.parametrize("T,p", [(300.0, 1e5), (270.0, 5e4), (220.0, 2e4), (250.0, 900.0),
                                 (330.0, 1.2e4), (330.0, 5.0e3)])
def test_dqsdT_matches_central_difference(oracle, T, p):
    h = 1e-4
    fd = (oracle.qs(T + h, p) - oracle.qs(T - h, p)) / (2 * h)
    an = oracle.dqsdT(T, p)
    assert abs(an - fd) <= 1e-7 * abs(an), (an, fd)


def test_qs_definition_and_clamp(oracle):
    # ordinary branch: qs = eps es / (p - (1-eps) es)
    T, p = 295.0, 85000.0
    es = oracle.es(T)
    assert oracle.qs(T, p) == pytest.approx(P.EPS * es / (p - (1 - P.EPS) * es), rel=1e-15)
    # clamped branch (es close to p): denominator floored at 1e-3 p
    T, p = 330.0, 5.0e3
    es = oracle.es(T)
    assert p - (1 - P.EPS) * es < 1e-3 * p
    assert oracle.qs(T, p) == pytest.approx(P.EPS * es / (1e-3 * p), rel=1e-15)


# ---------------------------------------------------------------- levels and heights
@pytest.mark.parametrize("pver", [26, 30, 32])
@pytest.mark.parametrize("ps", [1e5, 9.2e4])
def test_levels_mass_and_monotonicity(oracle, pver, ps):
    a, b = S.hybrid_coefficients(pver)
    p_int, p_mid = oracle.levels(pver, a, b, ps)
    assert p_int[0] == pytest.approx(300.0, rel=1e-14)
    assert p_int[-1] == pytest.approx(ps, rel=1e-15)
    assert np.all(np.diff(p_int) > 0) and np.all(np.diff(p_mid) > 0)
    m = np.diff(p_int) / P.GRAV
    assert m.sum() == pytest.approx((ps - 300.0) / P.GRAV, rel=1e-14)
    assert np.all((p_mid > p_int[:-1]) & (p_mid < p_int[1:]))


def test_isothermal_heights_closed_form(oracle):
    pver = 30
    a, b = S.hybrid_coefficients(pver)
    p_int, p_mid = oracle.levels(pver, a, b, 1e5)
    T0, q0 = 250.0, 2e-3
    z_int, z_mid = oracle.heights(np.full(pver, T0), np.full(pver, q0), p_int, p_mid)
    H = P.RD * T0 * (1 + P.ZVIR * q0) / P.GRAV
    np.testing.assert_allclose(z_int, H * np.log(1e5 / p_int), rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(z_mid, H * np.log(1e5 / p_mid), rtol=1e-12, atol=1e-9)


# ---------------------------------------------------------------- LCL and inversion
@pytest.mark.parametrize("Tb,rh,pb", [(300.0, 0.8, 98000.0), (290.0, 0.5, 95000.0),
                                      (305.0, 0.95, 99000.0), (275.0, 0.3, 70000.0),
                                      (260.0, 0.6, 60000.0)])
def test_lcl_against_bisection_and_bolton(oracle, Tb, rh, pb):
    qb = rh * oracle.qs(Tb, pb)
    TL, pL, last = oracle.lcl(Tb, qb, pb)
    # defining equation: saturated at the LCL on the dry adiabat
    assert pL == pytest.approx(pb * (TL / Tb) ** (1 / P.KAPPA), rel=1e-14)
    assert oracle.qs(TL, pL) == pytest.approx(qb, rel=1e-12)
    assert TL == pytest.approx(P.lcl_by_bisection(oracle, Tb, qb, pb), abs=1e-9)
    # Bolton's empirical fit (stated 0.1 K) with RH from vapour pressures
    e = qb * pb / (P.EPS + (1 - P.EPS) * qb)
    assert abs(TL - P.bolton_tl(Tb, e / oracle.es(Tb))) < 0.3
    assert last < 1e-9


def test_lcl_saturated_launch_is_launch_point(oracle):
    Tb, pb = 295.0, 97000.0
    qb = 1.001 * oracle.qs(Tb, pb)
    TL, pL, _ = oracle.lcl(Tb, qb, pb)
    assert TL == Tb and pL == pb


@pytest.mark.parametrize("h_off,p,Tenv", [(5e3, 60000.0, 265.0), (-3e3, 85000.0, 288.0),
                                          (1.2e4, 25000.0, 235.0), (0.0, 5000.0, 210.0)])
def test_moist_inversion_against_bisection(oracle, h_off, p, Tenv):
    gz = 4.0e4
    h = P.CP * Tenv + gz + P.LV * oracle.qs(Tenv, p) + h_off
    T, last = oracle.hinv(h, gz, p, Tenv)
    assert T == pytest.approx(P.saturated_temperature(oracle, h, gz, p), abs=1e-9)
    assert abs(P.CP * T + gz + P.LV * oracle.qs(T, p) - h) < 1e-8 * h
    assert last < 1e-7  # the loop ended on its convergence test


@pytest.mark.parametrize("dT", [-40.0, -15.0, 20.0, 45.0])
def test_moist_inversion_far_start_converges(oracle, dT):
    """A start 15-45 K from the root (a parcel far warmer or colder than the
    environment): the convergence-tested loop reaches the bisection root, while
    a fixed 1 + 1 steps does not; a cap of 0 extra steps takes exactly one
    Newton step from the start."""
    p, gz = 50000.0, 5.5e4
    Tsol = 262.0
    h = P.CP * Tsol + gz + P.LV * oracle.qs(Tsol, p)
    T, last = oracle.hinv(h, gz, p, Tsol + dT)
    assert T == pytest.approx(P.saturated_temperature(oracle, h, gz, p), abs=1e-9)
    assert last < 1e-7
    T1, last1 = oracle.hinv(h, gz, p, Tsol + dT, n_extra=1)
    assert abs(T1 - Tsol) > 1e-3 and last1 > 1e-4
    T0, _ = oracle.hinv(h, gz, p, Tsol + dT, n_extra=0)
    T00 = Tsol + dT
    qs = oracle.qs(T00, p)
    f = P.CP * T00 + gz + P.LV * qs - h
    assert T0 == pytest.approx(T00 - f / (P.CP + P.LV * oracle.dqsdT(T00, p)), rel=1e-14)


# ---------------------------------------------------------------- deep scheme
@pytest.fixture(scope="module")
def cols():
    return S.column_set(128)


def _col(g, i):
    return g.T[:, i].copy(), g.q[:, i].copy(), float(g.ps[i])


def _deep_diags(oracle, g, idx, **kw):
    return [oracle.deep_column_diag(g.pver, g.hyai, g.hybi, *_col(g, i), **kw) for i in idx]


def test_deep_launch_level_brute_force(oracle, cols):
    for i in range(cols.n_cols):
        T, q, ps = _col(cols, i)
        d = oracle.deep_column_diag(cols.pver, cols.hyai, cols.hybi, T, q, ps)
        h = np.array(d.h[: cols.pver])
        p_mid = np.array(d.p_mid[: cols.pver])
        cand = [k for k in range(cols.pver) if p_mid[k] >= 60000.0]
        best = max(h[k] for k in cand)
        assert d.kb == max(k for k in cand if h[k] == best)


def test_deep_launch_level_tie_keeps_lowest(oracle, cols):
    """An exact tie of h between layers kb-1 and kb keeps the lower layer kb."""
    i = next(i for i in range(cols.n_cols)
             if oracle.deep_column_diag(cols.pver, cols.hyai, cols.hybi, *_col(cols, i)).kb
             == cols.pver - 1)
    T, q, ps = _col(cols, i)
    kb = cols.pver - 1

    def h_at(qv):
        q2 = q.copy()
        q2[kb - 1] = qv
        d = oracle.deep_column_diag(cols.pver, cols.hyai, cols.hybi, T, q2, ps)
        return d.h[kb - 1], d.h[kb], d.kb

    # bisection over the float64 bit patterns of q[kb-1] for h[kb-1] == h[kb]
    lo = np.float64(q[kb - 1]).view(np.int64)
    hi = np.float64(0.09).view(np.int64)
    assert h_at(q[kb - 1])[0] < h_at(q[kb - 1])[1] < h_at(0.09)[0]
    while hi - lo > 1:
        mid = (lo + hi) // 2
        a, b, _ = h_at(np.int64(mid).view(np.float64))
        lo, hi = (mid, hi) if a < b else (lo, mid)
    a, b, k_tie = h_at(np.int64(hi).view(np.float64))
    assert a == b, "no exactly representable tie found"
    assert k_tie == kb
    a, b, k_up = h_at(np.int64(hi + 1).view(np.float64))
    if a > b:
        assert k_up == kb - 1


def test_deep_parcel_cape_brute_force(oracle, cols):
    """Parcel temperatures from independent root finders, EL by scan, CAPE by sum."""
    checked = 0
    for i in range(0, cols.n_cols, 3):
        T, q, ps = _col(cols, i)
        d = oracle.deep_column_diag(cols.pver, cols.hyai, cols.hybi, T, q, ps)
        if d.klcl < d.k_top_lim:
            continue
        p_int, p_mid = P.levels(cols.hyai, cols.hybi, ps)
        z_mid = np.array(d.z_mid[: cols.pver])
        kb, klcl, ktl = d.kb, d.klcl, d.k_top_lim
        # LCL level: largest k <= kb with p_mid <= pL
        assert klcl == max(k for k in range(kb + 1) if p_mid[k] <= d.pL)
        Tv = T * (1 + P.ZVIR * q)
        b = np.full(cols.pver, np.nan)
        hb = d.h[kb]
        for k in range(ktl, klcl + 1):
            Tp = P.saturated_temperature(oracle, hb, P.GRAV * z_mid[k], p_mid[k])
            b[k] = Tp * (1 + P.ZVIR * oracle.qs(Tp, p_mid[k])) - Tv[k]
            assert d.Tp[k] == pytest.approx(Tp, abs=1e-8)
        for k in range(klcl + 1, kb + 1):  # closed-form dry adiabat below the LCL
            assert d.Tp[k] == pytest.approx(T[kb] * (p_mid[k] / p_mid[kb]) ** P.KAPPA, rel=1e-14)
        pos = [k for k in range(ktl, klcl + 1) if b[k] > 0]
        kel = min(pos) if pos else -1
        assert d.kel == kel
        if kel >= 0:
            cape = max(0.0, sum(P.RD * b[k] * math.log(p_int[k + 1] / p_int[k])
                                for k in range(kel, klcl + 1)))
            assert d.cape == pytest.approx(cape, rel=1e-9, abs=1e-9)
        checked += 1
    assert checked > 10


@pytest.fixture(scope="module")
def active_diags(oracle, cols):
    ds = []
    for i in range(cols.n_cols):
        d = oracle.deep_column_diag(cols.pver, cols.hyai, cols.hybi, *_col(cols, i))
        if d.active:
            ds.append((i, d))
    assert len(ds) > 15
    return ds


def test_deep_plume_closed_forms(oracle, cols, active_diags):
    """Telescoped plume budgets and the entrainment profile in closed form."""
    for i, d in active_diags:
        T, q, ps = _col(cols, i)
        kb, jt = d.kb, d.jt
        z = np.array(d.z_mid[: cols.pver])
        h = np.array(d.h[: cols.pver])
        eta = np.array(d.eta[: cols.pver])
        lam, ze = 1e-3, 1000.0
        for k in range(jt, kb + 1):
            assert eta[k] == pytest.approx((1 + (z[k] - z[kb]) / ze) ** (lam * ze), rel=1e-13)
        rain = np.array(d.rain[: cols.pver])
        for k in range(jt + 1, kb):
            # eta_k h_u,k = h_kb + sum_{j=k}^{kb-1} (eta_j - eta_j+1) h_j
            s_h = h[kb] + sum((eta[j] - eta[j + 1]) * h[j] for j in range(k, kb))
            assert eta[k] * d.hu[k] == pytest.approx(s_h, rel=1e-12)
            s_q = q[kb] + sum((eta[j] - eta[j + 1]) * q[j] for j in range(k, kb)) - rain[k:kb].sum()
            assert eta[k] * d.qtu[k] == pytest.approx(s_q, rel=1e-10, abs=1e-15)
            # implicit rain: R/eta = c0 dz (liquid left after rain)
            dz = d.z_int[k] - d.z_int[k + 1]
            qt = d.qtu[k] + rain[k] / eta[k]
            Ts = P.saturated_temperature(oracle, d.hu[k], P.GRAV * z[k], d.p_mid[k])
            l = max(0.0, qt - oracle.qs(Ts, d.p_mid[k]))
            assert rain[k] / eta[k] == pytest.approx(2e-3 * dz * (l - rain[k] / eta[k]),
                                                     rel=1e-7, abs=1e-14)
        # cloud top: first layer at/above the min-h* layer with h_u <= h*, h* the
        # saturated moist static energy cp T + g z + Lv qs(T, p) of the environment
        hs = _saturated_mse(oracle, T, z, d.p_mid)
        np.testing.assert_allclose(np.array(d.hs[: cols.pver]), hs, rtol=1e-14, atol=0)
        khmin = max(range(d.k_top_lim, d.klcl), key=lambda k: (-hs[k], k))
        assert d.khmin == khmin
        cands = [k for k in range(khmin, d.k_top_lim - 1, -1) if d.hu[k] <= hs[k]]
        assert jt == (cands[0] if cands else d.k_top_lim)


def _saturated_mse(oracle, T, z, p_mid):
    return np.array([P.CP * T[k] + P.GRAV * z[k] + P.LV * oracle.qs(T[k], p_mid[k])
                     for k in range(len(T))])


def test_deep_downdraft_closed_forms(oracle, cols, active_diags):
    for i, d in active_diags:
        T, q, ps = _col(cols, i)
        kb, jt, jd = d.kb, d.jt, d.jd
        # the downdraft starts at the minimum of the environment's h* between
        # the cloud top and the LCL (ties: the lower layer)
        hs = _saturated_mse(oracle, T, np.array(d.z_mid[: cols.pver]), d.p_mid)
        rng = list(range(jt + 1, d.klcl))
        if not rng:
            assert jd == -1
            continue
        assert jd == min(rng, key=lambda k: (hs[k], -k))
        etad = np.array(d.etad[: cols.pver])
        E1 = np.array(d.E1[: cols.pver])
        qd = np.array(d.qd[: cols.pver])
        eprev = np.concatenate([[0.0], etad[jd:kb - 1]])
        sumE = etad[kb - 1] * qd[kb - 1] - np.sum((etad[jd:kb] - eprev) * q[jd:kb])
        assert E1[jd:kb].sum() == pytest.approx(sumE, rel=1e-9, abs=1e-15)
        if 0.2 * d.sumE > d.sumR:
            assert d.alpha_eff * d.sumE == pytest.approx(d.sumR, rel=1e-14)
        else:
            assert d.alpha_eff == 0.2
        assert d.prec >= 0.0


def test_deep_tendencies_match_interface_flux_budget(cols, active_diags):
    """C8 per-layer formula against an interface-flux budget of the drafts.

    H_i = U_i h_u,i - U_i h_{i-1} - D_i h_d,{i-1} + D_i h_i through interface i
    (updraft U_i = eta_i for jt < i <= kb, downdraft D_i = alpha eta_d,{i-1} for
    jd < i <= kb, each with its own upwind compensating flux);
    m_k dh_k = H_{k+1} - H_k, m_k dq_k = Q_{k+1} - Q_k - R_k + alpha E_k.
    """
    for i, d in active_diags:
        T, q, ps = _col(cols, i)
        n, kb, jt, jd, a = cols.pver, d.kb, d.jt, d.jd, d.alpha_eff
        h = np.array(d.h[:n])
        H = np.zeros(n + 1)
        Q = np.zeros(n + 1)
        for ii in range(jt + 1, kb + 1):
            H[ii] += d.eta[ii] * (d.hu[ii] - h[ii - 1])
            Q[ii] += d.eta[ii] * (d.qtu[ii] - q[ii - 1])
        if jd >= 0:
            for ii in range(jd + 1, kb + 1):
                D = a * d.etad[ii - 1]
                H[ii] += D * (h[ii] - d.hd[ii - 1])
                Q[ii] += D * (q[ii] - d.qd[ii - 1])
        m = np.array(d.m[:n])
        dh = (H[1:] - H[:-1]) / m
        src = -np.array(d.rain[:n]) + (a * np.array(d.E1[:n]) if jd >= 0 else 0.0)
        dq = (Q[1:] - Q[:-1] + src) / m
        scale_h = np.abs(dh).max()
        scale_q = np.abs(dq).max()
        np.testing.assert_allclose(np.array(d.dh[:n]), dh, rtol=0, atol=1e-10 * scale_h)
        np.testing.assert_allclose(np.array(d.dq[:n]), dq, rtol=0, atol=1e-10 * scale_q)


def test_closure_F_is_cape_derivative(oracle, cols, active_diags):
    """F equals dCAPE/dM_b of the parcel-fixed CAPE (central difference)."""
    for i, d in active_diags[:12]:
        T, q, ps = _col(cols, i)
        kb, kel, klcl = d.kb, d.kel, d.klcl
        p_int, p_mid = P.levels(cols.hyai, cols.hybi, ps)
        z = np.array(d.z_mid[: cols.pver])
        dT = np.array(d.dT[: cols.pver])
        dq = np.array(d.dq[: cols.pver])
        dhb = P.CP * dT[kb] + P.LV * dq[kb]

        def cape(eps):
            hb = d.h[kb] + eps * dhb
            s = 0.0
            for k in range(kel, klcl + 1):
                Tp = P.saturated_temperature(oracle, hb, P.GRAV * z[k], p_mid[k])
                Tvp = Tp * (1 + P.ZVIR * oracle.qs(Tp, p_mid[k]))
                Tk, qk = T[k] + eps * dT[k], q[k] + eps * dq[k]
                s += P.RD * (Tvp - Tk * (1 + P.ZVIR * qk)) * math.log(p_int[k + 1] / p_int[k])
            return s

        e = 1e-3 * abs(d.cape / d.F)
        fd = (cape(e) - cape(-e)) / (2 * e)
        assert d.F == pytest.approx(fd, rel=2e-5)
        if not d.limited:
            assert d.mb == pytest.approx(-d.cape / (3600.0 * d.F), rel=1e-14)


def test_deep_grid_invariants(oracle):
    g = S.latlon_grid(24, 36)
    od = oracle.deep(g, threads=4)
    fl = od["flags"]
    act = (fl & oracle.F_ACTIVE) > 0
    assert act.any() and (~act).any()
    # not active => every output exactly zero
    for k in ("dTdt", "dqdt"):
        assert np.all(od[k][:, ~act] == 0.0)
    assert np.all(od["prec"][~act] == 0.0) and np.all(od["mb"][~act] == 0.0)
    assert np.all(od["ktop"][~act] == -1)
    trig = (fl & oracle.F_TRIGGERED) > 0
    assert np.all(od["cape"][trig] > 70.0) and np.all(od["cape"][~trig] <= 70.0)
    # conservation: sum m cp dTdt = Lv P, sum m dqdt = -P
    for i in np.where(act)[0]:
        p_int, _ = P.levels(g.hyai, g.hybi, g.ps[i])
        m = np.diff(p_int) / P.GRAV
        P_ = od["prec"][i]
        e = np.sum(m * P.CP * od["dTdt"][:, i])
        w = np.sum(m * od["dqdt"][:, i])
        sc = np.sum(m * P.CP * np.abs(od["dTdt"][:, i]))
        assert abs(e - P.LV * P_) <= 1e-12 * sc
        assert abs(w + P_) <= 1e-12 * sc / P.LV
        assert od["cons_err"][i] < 1e-12
    assert np.all(od["prec"] >= 0.0)
    # limiter keeps q + dt dqdt >= q_min
    qn = g.q + g.dt * od["dqdt"]
    assert np.all(qn[:, act] >= 1e-12 - 1e-14 * g.q[:, act])  # q - (q - q_min) rounds at ulp(q)


def test_closure_linear_in_inverse_tau(oracle):
    g = S.latlon_grid(24, 36)
    o1 = oracle.deep(g, threads=4)
    o2 = oracle.deep(g, threads=4, tau=np.full(g.n_cols, 7200.0))
    act = (o1["flags"] & oracle.F_ACTIVE) > 0
    unl = act & ((o1["flags"] & oracle.F_LIMITED) == 0) & ((o2["flags"] & oracle.F_LIMITED) == 0)
    assert unl.sum() > 5
    np.testing.assert_allclose(o2["prec"][unl], 0.5 * o1["prec"][unl], rtol=1e-14)
    np.testing.assert_allclose(o2["dTdt"][:, unl], 0.5 * o1["dTdt"][:, unl], rtol=1e-13,
                               atol=1e-30)


def test_undilute_limit_lambda_zero(oracle, cols, active_diags):
    for i, _ in active_diags[:10]:
        T, q, ps = _col(cols, i)
        d = oracle.deep_column_diag(cols.pver, cols.hyai, cols.hybi, T, q, ps, lam=0.0)
        if not d.triggered or d.jt < 0:
            continue
        for k in range(max(d.jt, 0) + 1, d.kb + 1):
            assert d.eta[k] == 1.0
            assert d.hu[k] == pytest.approx(d.h[d.kb], rel=1e-15)


# ---------------------------------------------------------------- shallow scheme
def _sh(oracle, g, i, T=None, q=None):
    T0, q0, ps = _col(g, i)
    return oracle.shallow_column_diag(g.pver, g.hyai, g.hybi, T0 if T is None else T,
                                      q0 if q is None else q, ps)


def test_shallow_exit_paths_and_zero_outputs(oracle):
    g = S.column_set(256)
    so = oracle.shallow(g, threads=4)
    codes = (so["flags"] >> oracle.EXIT_SHIFT) & 7
    act = (so["flags"] & oracle.F_ACTIVE) > 0
    assert act.any()
    assert np.all(codes[act] == 0)
    for c in (1, 2, 3, 4):
        sel = codes == c
        if sel.any():
            assert np.all(so["dTdt"][:, sel] == 0) and np.all(so["dqdt"][:, sel] == 0)
            assert np.all(so["prec"][sel] == 0) and np.all(so["mb"][sel] == 0)
    # E1 by construction: a very dry surface layer lifts far before saturating
    t, qq, ps = S.profiles(30, np.array([300.0]), np.array([0.10]))
    d = oracle.shallow_column_diag(30, g.hyai, g.hybi, t[:, 0], qq[:, 0], float(ps[0]))
    assert d.exit_code == 1 and d.pL < 70000.0
    # E2 by construction: cold dry column has no LFC below 500 hPa
    t, qq, ps = S.profiles(30, np.array([280.0]), np.array([0.40]))
    d = oracle.shallow_column_diag(30, g.hyai, g.hybi, t[:, 0], qq[:, 0], float(ps[0]))
    assert d.exit_code == 2
    assert np.bincount(codes, minlength=5)[3] > 0  # E3 occurs in this set


@pytest.mark.parametrize("warm", [0.0, 3.0])
def test_shallow_lfc_cin_brute_force(oracle, warm):
    """warm > 0 heats the source layer by that many kelvin: a superadiabatic
    surface layer whose dry-lifted parcel is buoyant below its LCL, where the
    LFC must still not be placed."""
    g = S.column_set(96)
    n = dry_buoyant = 0
    for i in range(g.n_cols):
        T, q, ps = _col(g, i)
        T[-1] += warm
        d = _sh(oracle, g, i, T=T)
        if d.exit_code == 1:
            continue
        p_int, p_mid = P.levels(g.hyai, g.hybi, ps)
        ks = g.pver - 1
        z = np.array(d.z_mid[: g.pver])
        Tv = T * (1 + P.ZVIR * q)
        b = {}
        klfc = -1
        for k in range(ks, d.k_top_lim - 1, -1):
            if p_mid[k] < 50000.0:
                break
            if k > d.klcl:
                Tp, qp = T[ks] * (p_mid[k] / p_mid[ks]) ** P.KAPPA, q[ks]
            else:
                Tp = P.saturated_temperature(oracle, d.h[ks], P.GRAV * z[k], p_mid[k])
                qp = oracle.qs(Tp, p_mid[k])
            b[k] = Tp * (1 + P.ZVIR * qp) - Tv[k]
            if k <= d.klcl and b[k] > 0:
                klfc = k
                break
        dry_buoyant += any(b[k] > 0 for k in b if k > d.klcl)
        assert d.klfc == klfc
        if klfc >= 0:
            cin = sum(P.RD * max(0.0, -b[k]) * math.log(p_int[k + 1] / p_int[k])
                      for k in range(klfc + 1, ks + 1))
            assert d.cin == pytest.approx(cin, rel=1e-9, abs=1e-9)
            n += 1
    assert n > 10
    if warm > 0:
        assert dry_buoyant > 10


def test_shallow_budget_and_closure(oracle):
    g = S.column_set(256)
    n = 0
    for i in range(g.n_cols):
        d = _sh(oracle, g, i)
        if not d.active:
            continue
        T, q, ps = _col(g, i)
        ks, kts = g.pver - 1, d.kts
        rho = d.p_mid[ks] / (P.RD * T[ks] * (1 + P.ZVIR * q[ks]))
        assert d.mb == pytest.approx(rho * 0.03 * math.exp(-d.cin / 10.0), rel=1e-13)
        # interface-flux budget of the constant-mass-flux plume
        h = np.array(d.h[: g.pver])
        H = np.zeros(g.pver + 1)
        Q = np.zeros(g.pver + 1)
        for ii in range(kts + 1, ks + 1):
            H[ii] = d.mb * (d.hu[ii] - h[ii - 1])
            Q[ii] = d.mb * (d.qtu[ii] - q[ii - 1])
        m = np.array(d.m[: g.pver])
        rf = np.array(d.rf[: g.pver])
        rf[: kts + 1] = 0.0
        dh = (H[1:] - H[:-1]) / m
        dq = (Q[1:] - Q[:-1] - d.mb * rf) / m
        np.testing.assert_allclose(np.array(d.dh[: g.pver]), dh, rtol=0,
                                   atol=1e-10 * np.abs(dh).max())
        np.testing.assert_allclose(np.array(d.dq[: g.pver]), dq, rtol=0,
                                   atol=1e-10 * np.abs(dq).max())
        assert d.prec == pytest.approx(d.mb * rf.sum(), rel=1e-12, abs=1e-300)
        # rain comes out of the condensate only: never more than the liquid the
        # plume carries (total water above saturation at its temperature), so a
        # saturated plume stays saturated after the rain-out
        for k in range(kts + 1, ks):
            qs_u = oracle.qs(d.Tu[k], d.p_mid[k])
            assert 0.0 <= rf[k] <= max(d.qtpre[k] - qs_u, 0.0) * (1 + 1e-12), k
            if d.qtpre[k] >= qs_u:
                assert d.qtu[k] >= qs_u * (1 - 1e-12), k
        # w2 above the LFC stays positive up to the top, fails (or hits the limit) above it
        w2 = np.array(d.w2[: g.pver])
        assert np.all(w2[kts:ks + 1] > 0)
        assert kts == d.k_top_lim or w2[kts - 1] <= 0
        assert kts < d.klcl
        n += 1
    assert n > 10


def test_shallow_grid_conservation(oracle):
    g = S.latlon_grid(24, 36)
    od, so = oracle.deep_shallow(g, threads=4)
    act = (so["flags"] & oracle.F_ACTIVE) > 0
    assert act.any()
    assert np.all(so["prec"] >= 0)
    assert np.all(so["cons_err"][act] < 1e-12)


def _deep_shallow_column(oracle, g, par, min_layers):
    """First column whose shallow plume rises min_layers above its LFC under par."""
    for i in range(g.n_cols):
        T, q, ps = _col(g, i)
        d = oracle.shallow_column_diag(g.pver, g.hyai, g.hybi, T, q, ps, par=par)
        if d.klfc >= 0 and d.exit_code in (0, 4) and d.klfc - max(d.kts, d.k_top_lim) >= min_layers:
            return i, d
    raise AssertionError("no suitable shallow column")


def test_shallow_w2_pure_drag_closed_form(oracle):
    """a = 0: w2 decays as w2_0 exp(-2 b eps (z - z_LFC)) and never reaches zero."""
    g = S.column_set(256)
    i, d = _deep_shallow_column(oracle, g, oracle.shallow_params(a_w=0.0), 3)
    zi = np.array(d.z_int[: g.pver + 1])
    for k in range(d.k_top_lim, d.klfc):
        want = (2.0 / 3.0) * np.exp(-2 * 2.0 * 2e-3 * (zi[k] - zi[d.klfc]))
        assert d.w2[k] == pytest.approx(want, rel=1e-12)
    assert d.kts == d.k_top_lim


def test_shallow_w2_buoyancy_work_without_drag(oracle):
    """b = 0: the change of w2 across a layer is 2 a B dz, B from an independent
    saturation adjustment of the plume state."""
    g = S.latlon_grid(48, 72)
    i, d = _deep_shallow_column(oracle, g, oracle.shallow_params(b_w=0.0), 2)
    T, q, ps = _col(g, i)
    Tv = T * (1 + P.ZVIR * q)
    zi = np.array(d.z_int[: g.pver + 1])
    n = 0
    for k in range(d.klfc - 1, max(d.kts, d.k_top_lim + 1) - 1, -1):
        p, gz = d.p_mid[k], P.GRAV * d.z_mid[k]
        qt = d.qtpre[k]
        Ts = P.saturated_temperature(oracle, d.hu[k], gz, p)
        if qt >= oracle.qs(Ts, p):
            Tu, qv = Ts, oracle.qs(Ts, p)
        else:
            Tu, qv = (d.hu[k] - gz - P.LV * qt) / P.CP, qt
        B = P.GRAV * (Tu * (1 + P.ZVIR * qv) - Tv[k]) / Tv[k]
        assert d.w2[k] - d.w2[k + 1] == pytest.approx(2 * B * (zi[k] - zi[k + 1]), rel=1e-8,
                                                      abs=1e-9)
        n += 1
    assert n >= 2


def test_shallow_drag_lowers_w2(oracle):
    """More drag never raises w2 nor the cloud top."""
    g = S.column_set(256)
    for i in range(0, g.n_cols, 5):
        T, q, ps = _col(g, i)
        d1 = oracle.shallow_column_diag(g.pver, g.hyai, g.hybi, T, q, ps,
                                        par=oracle.shallow_params(b_w=1.0))
        d2 = oracle.shallow_column_diag(g.pver, g.hyai, g.hybi, T, q, ps,
                                        par=oracle.shallow_params(b_w=3.0))
        if d1.klfc < 0 or d1.exit_code in (1, 2, 3):
            continue
        assert d2.kts >= d1.kts
        for k in range(max(d1.kts, d2.kts), d1.klfc):
            assert d2.w2[k] <= d1.w2[k] * (1 + 1e-15)
