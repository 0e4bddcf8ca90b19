"""Invariants of the two schemes that hold for any valid column, checked on
randomly perturbed soundings rather than the generator's smooth profiles:
temperature inversions and superadiabatic layers, moist and dry layers, surface
pressures from mountains to sea level, random entrainment rates and closure
times.  For every column: the column's enthalpy and water budgets close
(cons_err <= 1e-12) wherever a scheme is active; precipitation is non-negative;
a scheme that is not active leaves exactly zero tendencies, precipitation and
mass flux; the flags are consistent (active implies triggered; the exit code of
an inactive shallow column is set); the level indices are ordered
(cloud top above the LCL, the LCL at or above the launch level); and after the
deep step no humidity falls below q_min where the deep scheme acted."""
import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S


def _random_columns(seed, n=1500, pver=30):
    rng = np.random.default_rng(seed)
    ts = rng.uniform(278.0, 306.0, n)
    rh = rng.uniform(0.3, 0.97, n)
    ps = rng.uniform(6.0e4, 1.04e5, n)
    T, q, ps = S.profiles(pver, ts, rh, ps)
    # red-noise perturbations in the vertical: inversions, superadiabatic
    # layers, moist and dry layers
    noise_T = np.cumsum(rng.normal(0.0, 0.8, (pver, n)), axis=0)
    noise_T -= noise_T.mean(axis=0)
    T = T + noise_T
    q = q * np.exp(rng.normal(0.0, 0.25, (pver, n)))
    a, b = S.hybrid_coefficients(pver)
    lam = rng.uniform(2e-4, 3e-3, n)
    tau = rng.uniform(1800.0, 14400.0, n)
    return S.Columns(f"random-{seed}", pver, T, q, ps, a, b, lam, tau, 1800.0)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_invariants_on_random_columns(oracle, seed):
    g = _random_columns(seed)
    d, s = oracle.deep_shallow(g, threads=4, lam=g.lam, tau=g.tau)
    F = oracle
    for o, deep in ((d, True), (s, False)):
        act = (o["flags"] & F.F_ACTIVE) > 0
        trig = (o["flags"] & F.F_TRIGGERED) > 0
        bad = (o["flags"] & F.F_BADINPUT) > 0
        assert act.sum() > 30 and (~act & ~bad).sum() > 30, (deep, act.sum())
        assert np.all(trig[act])
        assert np.all(o["cons_err"][act] <= 1e-12), (deep, o["cons_err"][act].max())
        assert np.all(o["prec"] >= 0.0)
        off = ~act
        assert np.all(o["dTdt"][:, off] == 0.0) and np.all(o["dqdt"][:, off] == 0.0)
        assert np.all(o["prec"][off] == 0.0) and np.all(o["mb"][off] == 0.0)
        assert np.all(o["mb"][act] > 0.0)
        kb, klcl, kt = o["kb"][act], o["klcl"][act], o["ktop"][act]
        assert np.all(kt < klcl) and np.all(klcl <= kb)
        if deep:
            qn = g.q + g.dt * d["dqdt"]
            qmin = F.deep_params().q_min
            assert np.all(qn[:, act] >= qmin * (1 - 1e-9) - 1e-18)
        else:
            codes = (o["flags"] >> F.EXIT_SHIFT) & 7
            assert np.all(codes[act] == 0)
            assert np.all(codes[off & ~bad] > 0)


def test_newton_convergence_test_on_rough_columns(oracle):
    """The moist inversions test convergence for termination (stop after the
    first correction below 1e-7 K, at most 1 + n_newton_h steps).  On these
    columns a parcel can lie 10-50 K from the environment temperature its solve
    starts from: a fixed count of 1 + 4 steps leaves such solves unconverged
    (and flags them), while the default cap converges every solve, and raising
    the cap changes nothing (the test, not the cap, ends every loop)."""
    g = _random_columns(7, n=3000)
    d, s = oracle.deep_shallow(g, threads=4)
    assert not ((d["flags"] | s["flags"]) & oracle.F_NEWTON).any()
    d4, _ = oracle.deep_shallow(g, dpar=oracle.deep_params(n_newton_h=4),
                                spar=oracle.shallow_params(n_newton_h=4), threads=4)
    assert ((d4["flags"] & oracle.F_NEWTON) > 0).sum() > 100
    d40, s40 = oracle.deep_shallow(g, dpar=oracle.deep_params(n_newton_h=40),
                                   spar=oracle.shallow_params(n_newton_h=40), threads=4)
    for a, b in ((d, d40), (s, s40)):
        for k in ("flags", "kb", "klcl", "ktop", "kaux"):
            assert np.array_equal(a[k], b[k]), k
        for k in ("dTdt", "dqdt", "prec", "cape", "mb"):
            assert np.array_equal(a[k], b[k]), k


def test_bad_input_columns(oracle):
    """Columns outside the accepted input ranges (surface pressure 500-1200 hPa,
    temperature 100-400 K, humidity [0, 0.1) kg/kg, NaN anywhere) are flagged as
    bad input with zero outputs in both schemes; columns just inside the ranges
    are not."""
    g = _random_columns(11, n=12)
    T, q, ps = g.T.copy(), g.q.copy(), g.ps.copy()
    ps[0] = 4.99e4
    ps[1] = 1.21e5
    T[5, 2] = float("nan")
    T[10, 3] = 401.0
    q[20, 4] = -1e-9
    q[25, 5] = 0.1
    q[3, 6] = float("nan")
    ps[7] = 5.01e4
    T[0, 8] = 101.0
    g2 = type(g)(g.name, g.pver, T, q, ps, g.hyai, g.hybi, g.lam, g.tau, g.dt)
    d, s = oracle.deep_shallow(g2, threads=2)
    want = np.zeros(g.n_cols, bool)
    want[:7] = True
    for o in (d, s):
        got = (o["flags"] & oracle.F_BADINPUT) > 0
        assert np.array_equal(got, want), got
        assert np.all(o["flags"][want] == oracle.F_BADINPUT)
        assert np.all(o["dTdt"][:, want] == 0.0) and np.all(o["dqdt"][:, want] == 0.0)
        assert np.all(o["prec"][want] == 0.0)
