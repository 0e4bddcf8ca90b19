"""Pins of the oracle's tangent of the fused deep -> shallow step (shallow
convection on the deep-updated state) against central finite differences of
the FP64 oracle's forward step and against exact identities."""
import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S
from tests import physics_ref as P

LV = 2.501e6


@pytest.fixture(scope="module")
def grid():
    g = S.latlon_grid(24, 36, tau_range=(1800.0, 7200.0))
    g.lam = 5e-4 + 1.5e-3 * S.uniform(20171105, 0, np.arange(g.n_cols), 0)
    return g


def _seeds(n, seed):
    c = np.arange(n)
    return [2.0 * S.uniform(seed, 0, c, j) - 1.0 for j in range(4)]


def _step_J(oracle, g, T, q, lam, tau, seeds):
    """J of every column and the decisions of both schemes."""
    sub = S.Columns("c", g.pver, T, q, g.ps, g.hyai, g.hybi, lam, tau, g.dt)
    od, os_ = oracle.deep_shallow(sub, threads=4)
    p_int = g.hyai[:, None] * 1e5 + g.hybi[:, None] * g.ps[None, :]
    p_mid = 0.5 * (p_int[1:] + p_int[:-1])
    m = np.diff(p_int, axis=0) / P.GRAV
    w = p_mid / g.ps[None, :]
    gPd, gHd, gPs, gHs = seeds
    J = (gPd * od["prec"] + gHd * np.sum(w * m * P.CP * od["dTdt"], axis=0)
         + gPs * os_["prec"] + gHs * np.sum(w * m * P.CP * os_["dTdt"], axis=0))
    dec = np.stack([o[k] for o in (od, os_) for k in ("flags", "kb", "klcl", "ktop", "kaux")])
    return J, dec, od, os_


def test_step_tangent_matches_central_differences(oracle, grid):
    g = grid
    n = g.n_cols
    seeds = _seeds(n, 3)
    ad = dict(zip(("gT", "gq", "gl", "gt"), oracle.deep_shallow_adjoint(
        g, *seeds, threads=4)))
    J0, dec0, od, os_ = _step_J(oracle, g, g.T, g.q, g.lam, g.tau, seeds)
    both = ((od["flags"] & oracle.F_ACTIVE) > 0) & ((os_["flags"] & oracle.F_ACTIVE) > 0)
    ok = both & (np.abs(od["cape"] - 70.0) >= 5.0)
    assert ok.sum() >= 30
    kinked = np.zeros(n, bool)
    fd = {"gT": np.zeros((g.pver, n)), "gq": np.zeros((g.pver, n)), "gl": np.zeros(n),
          "gt": np.zeros(n)}
    cmp = {"gT": np.ones((g.pver, n), bool), "gq": g.q > 1e-6, "gl": np.ones(n, bool),
           "gt": np.ones(n, bool)}
    for var, k in ([("gT", k) for k in range(g.pver)] + [("gq", k) for k in range(g.pver)]
                   + [("gl", None), ("gt", None)]):
        h = {"gT": np.full(n, 3e-4), "gl": np.full(n, 1e-9), "gt": np.full(n, 3.6e-3)}.get(var)
        if var == "gq":
            h = np.where(cmp["gq"][k], 2e-8, 0.0)
        Js = []
        for sgn in (1.0, -1.0):
            T, q, lam, tau = g.T.copy(), g.q.copy(), g.lam.copy(), g.tau.copy()
            if var == "gT":
                T[k] += sgn * h
            elif var == "gq":
                q[k] += sgn * h
            elif var == "gl":
                lam = lam + sgn * h
            else:
                tau = tau + sgn * h
            J, dec, _, _ = _step_J(oracle, g, T, q, lam, tau, seeds)
            ok &= np.all(dec == dec0, axis=0)
            Js.append(J)
        hs = np.where(h > 0, h, 1.0)
        fwd, bwd = (Js[0] - J0) / hs, (J0 - Js[1]) / hs
        scale = np.maximum(np.abs(np.atleast_2d(ad[var])).max(axis=0), 1e-300)
        kinked |= (np.abs(fwd - bwd) > 1e-3 * scale) & (h > 0)
        c = (Js[0] - Js[1]) / (2 * hs)
        if k is None:
            fd[var] = c
        else:
            fd[var][k] = c
    use = ok & ~kinked
    assert use.sum() >= 0.7 * ok.sum() and use.sum() >= 20, (use.sum(), ok.sum())
    xs = {"gT": 300.0, "gq": 0.02, "gl": 1e-3, "gt": 3600.0}
    for var in fd:
        a = np.atleast_2d(ad[var])
        den = np.maximum(np.abs(a).max(axis=0), np.abs(J0) / xs[var])
        err = np.where(np.atleast_2d(cmp[var]), np.abs(np.atleast_2d(fd[var]) - a), 0.0)
        rel = err.max(axis=0)[use] / den[use]
        assert rel.max() <= 1e-6, f"{var}: {rel.max():.3e}"


def test_shallow_energy_balance_of_gradients(oracle):
    """The shallow tendencies conserve column enthalpy: with w = 1,
    sum m cp dTdt_shallow = Lv P_shallow identically, so the gradients agree
    (checked where the shallow plume rains; without rain both sides vanish)."""
    g = S.latlon_grid(48, 72)
    n = g.n_cols
    one, w1 = np.ones(n), np.ones(g.pver)
    aP = oracle.deep_shallow_adjoint(g, None, None, one, None, w_heat=w1, threads=4)
    aH = oracle.deep_shallow_adjoint(g, None, None, None, one, w_heat=w1, threads=4)
    _, os_ = oracle.deep_shallow(g, threads=4)
    act = ((os_["flags"] & oracle.F_ACTIVE) > 0) & (os_["prec"] > 0)
    assert act.sum() > 20
    for x, y in zip(aH, aP):
        x, y = np.atleast_2d(x)[:, act], LV * np.atleast_2d(y)[:, act]
        den = np.maximum(np.abs(y).max(axis=0), 1e-300)
        assert (np.abs(x - y).max(axis=0) / den).max() <= 1e-10


def test_deep_seeds_reproduce_deep_tangent_and_zeros_off_schemes(oracle, grid):
    g = grid
    n = g.n_cols
    gPd, gHd, gPs, gHs = _seeds(n, 9)
    a = oracle.deep_shallow_adjoint(g, gPd, gHd, None, None, threads=4)
    b = oracle.deep_adjoint(g, gPd, gHd, threads=4)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    full = oracle.deep_shallow_adjoint(g, gPd, gHd, gPs, gHs, threads=4)
    od, os_ = oracle.deep_shallow(g, threads=4)
    idle = ((od["flags"] & oracle.F_ACTIVE) == 0) & ((os_["flags"] & oracle.F_ACTIVE) == 0)
    assert idle.sum() > 50
    for x in full:
        assert np.all(np.atleast_2d(x)[:, idle] == 0.0)
