"""Pins of the oracle's shallow rain evaporation (a scheme variant, off by
default): rain made in a plume layer falls through the environment layers
below it and each layer evaporates the fraction 1 - exp(-k max(qs - q, 0) dz)
of the flux arriving from above.

Pinned against what the mathematics fixes: the decisions and the deep scheme
are untouched; evaporation only moves water and heat between the rain and the
layers (column enthalpy and water still close, per level cp dT = -Lv dq, the
evaporated total equals the precipitation lost); precipitation falls
monotonically with k and vanishes as k -> infinity where every layer below the
rain is unsaturated, and no rain evaporates where every such layer is
saturated or supersaturated; and for small k the loss matches the first-order
expansion sum_j G_j (qs_j - q_j) dz_j, G_j the rain made above layer j (so rain
does not evaporate in the layer that makes it)."""
import copy

import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S
from tests import physics_ref as P


@pytest.fixture(scope="module")
def grid():
    return S.latlon_grid(24, 36)


# a lower autoconversion threshold than the default makes most shallow plumes of
# this grid rain, so every pin sees many raining columns
QL = 1e-4


@pytest.fixture(scope="module")
def base(oracle, grid):
    return oracle.deep_shallow(grid, spar=oracle.shallow_params(ql_crit=QL), threads=4)


def _run(oracle, g, k, **kw):
    return oracle.deep_shallow(g, spar=oracle.shallow_params(ql_crit=QL, evap_k=k), threads=4,
                               **kw)


def _act(o, oracle):
    return (o["flags"] & oracle.F_ACTIVE) > 0


def _layer_mass(g):
    p_int = g.hyai[:, None] * 1e5 + g.hybi[:, None] * g.ps[None, :]
    return np.diff(p_int, axis=0) / P.GRAV


def test_off_by_default_and_continuous(oracle, grid, base):
    d0, s0 = base
    d1, s1 = _run(oracle, grid, 0.0)
    for a, b in ((d0, d1), (s0, s1)):
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    _, s2 = _run(oracle, grid, 1e-12)
    act = _act(s0, oracle)
    assert np.all(np.abs(s2["prec"] - s0["prec"])[act] <= 1e-8 * s0["prec"][act] + 1e-300)


@pytest.mark.parametrize("k", [0.05, 0.2, 1.0])
def test_moves_water_and_heat_only(oracle, grid, base, k):
    d0, s0 = base
    d1, s1 = _run(oracle, grid, k)
    for key in d0:  # the deep scheme and every decision are untouched
        assert np.array_equal(d0[key], d1[key]), key
    for key in ("flags", "kb", "klcl", "ktop", "kaux", "cape", "mb"):
        assert np.array_equal(s0[key], s1[key]), key
    act = _act(s0, oracle)
    assert act.sum() > 50
    m = _layer_mass(grid)
    ddq = (s1["dqdt"] - s0["dqdt"])[:, act]
    ddT = (s1["dTdt"] - s0["dTdt"])[:, act]
    scale = np.abs(s0["dqdt"][:, act]).max(axis=0)
    assert np.all(ddq >= -1e-15 * scale) and np.all(ddT <= 1e-15 * P.LV / P.CP * scale)
    assert np.abs(P.CP * ddT + P.LV * ddq).max() <= 1e-12 * P.LV * scale.max()
    lost = s0["prec"][act] - s1["prec"][act]
    assert np.all(s1["prec"][act] >= 0.0) and np.all(lost >= -1e-15 * s0["prec"][act])
    evap = np.sum(m[:, act] * ddq, axis=0)
    assert np.allclose(evap, lost, rtol=1e-9, atol=1e-12 * s0["prec"][act].max())
    assert s1["cons_err"][act].max() <= 1e-12
    assert lost.sum() > 0.05 * s0["prec"][act].sum()  # the variant does something


def test_monotone_in_k(oracle, grid, base):
    _, s0 = base
    ps = [s0["prec"]] + [_run(oracle, grid, k)[1]["prec"] for k in (0.05, 0.2, 1.0)]
    for a, b in zip(ps, ps[1:]):
        assert np.all(b <= a * (1 + 1e-15))


def test_everything_evaporates_in_the_limit(oracle, grid):
    """Deep scheme off, so the shallow scheme sees the original state: where
    every layer from below the plume top to the surface is unsaturated, an
    unbounded coefficient leaves no precipitation and the evaporated water is
    all the rain."""
    g = grid
    dpar = oracle.deep_params(capelmt=1e30)
    _, s0 = _run(oracle, g, 0.0, dpar=dpar)
    _, s1 = _run(oracle, g, 1e12, dpar=dpar)
    m = _layer_mass(g)
    checked = 0
    for i in np.flatnonzero(_act(s0, oracle) & (s0["prec"] > 0)):
        kt = s0["ktop"][i]
        p_int, p_mid = oracle.levels(g.pver, g.hyai, g.hybi, g.ps[i])
        qs = np.array([oracle.qs(g.T[j, i], p_mid[j]) for j in range(g.pver)])
        if np.all(qs[kt + 1:] > g.q[kt + 1:, i]):
            assert s1["prec"][i] == 0.0
            evap = np.sum(m[:, i] * (s1["dqdt"][:, i] - s0["dqdt"][:, i]))
            assert evap == pytest.approx(s0["prec"][i], rel=1e-9)
            checked += 1
    assert checked > 20


def test_first_order_loss(oracle, grid):
    """(P(0) - P(k)) / k -> sum_j G_j (qs_j - q_j)^+ dz_j as k -> 0, with G_j the
    rain made in the plume layers above j (kts < layer < j): rain leaves the
    layer that makes it before it can evaporate."""
    g = grid
    dpar = oracle.deep_params(capelmt=1e30)
    _, s0 = _run(oracle, g, 0.0, dpar=dpar)
    k = 1e-7
    _, s1 = _run(oracle, g, k, dpar=dpar)
    cols = np.flatnonzero(_act(s0, oracle) & (s0["prec"] > 0))[:40]
    assert cols.size >= 20
    for i in cols:
        d = oracle.shallow_column_diag(g.pver, g.hyai, g.hybi, g.T[:, i], g.q[:, i], g.ps[i],
                                       par=oracle.shallow_params(ql_crit=QL))
        kt, ks = d.kts, g.pver - 1
        assert d.kts == s0["ktop"][i]
        want = 0.0
        for j in range(kt + 1, ks + 1):
            G = d.mb * sum(d.rf[kk] for kk in range(kt + 1, j))
            dz = d.z_int[j] - d.z_int[j + 1]
            dfc = max(oracle.qs(g.T[j, i], d.p_mid[j]) - g.q[j, i], 0.0)
            want += G * dfc * dz
        got = (s0["prec"][i] - s1["prec"][i]) / k
        assert got == pytest.approx(want, rel=1e-4), i


def test_no_evaporation_into_saturated_air(oracle, grid):
    """Deep scheme off.  In the raining columns, every layer from below the plume
    top to the surface is moistened to 1% above saturation; where the plume top
    stays put, the saturation deficit is clamped at zero in every layer the rain
    falls through, so a large coefficient evaporates nothing: identical
    tendencies, and the same precipitation up to the order of its sum."""
    g = grid
    dpar = oracle.deep_params(capelmt=1e30)
    _, s0 = _run(oracle, g, 0.0, dpar=dpar)
    rain = _act(s0, oracle) & (s0["prec"] > 0)
    g2 = copy.deepcopy(g)
    for i in np.flatnonzero(rain):
        _, p_mid = oracle.levels(g.pver, g.hyai, g.hybi, g.ps[i])
        for j in range(s0["ktop"][i] + 1, g.pver):
            g2.q[j, i] = max(g.q[j, i], 1.01 * oracle.qs(g.T[j, i], p_mid[j]))
    _, a = _run(oracle, g2, 0.0, dpar=dpar)
    _, b = _run(oracle, g2, 1.0, dpar=dpar)
    checked = 0
    for i in np.flatnonzero(rain & _act(a, oracle) & (a["prec"] > 0)):
        kt = a["ktop"][i]
        _, p_mid = oracle.levels(g.pver, g.hyai, g.hybi, g.ps[i])
        if any(g2.q[j, i] < oracle.qs(g2.T[j, i], p_mid[j]) for j in range(kt + 1, g.pver)):
            continue  # the plume top moved up into air left unsaturated
        assert np.array_equal(a["dqdt"][:, i], b["dqdt"][:, i]), i
        assert np.array_equal(a["dTdt"][:, i], b["dTdt"][:, i]), i
        assert b["prec"][i] == pytest.approx(a["prec"][i], rel=1e-14, abs=0.0), i
        checked += 1
    assert checked > 50
