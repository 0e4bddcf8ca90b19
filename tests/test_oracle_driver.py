"""Pins of the oracle's multi-step column driver: the state advance against the
closed form of Newtonian relaxation, and one full step against the column
energy and water budgets of the two schemes."""
import numpy as np

from paper_1711_00289_gb300 import soundings as S
from tests import physics_ref as P


def test_relaxation_closed_form(oracle):
    g = S.column_set(64)
    zero = {"dTdt": np.zeros_like(g.T), "dqdt": np.zeros_like(g.q)}
    Tr, qr = g.T.copy(), g.q.copy()
    T, q = g.T + 1.5, g.q * 0.9
    dt, tau, n = 1800.0, 86400.0, 40
    for _ in range(n):
        T, q = oracle.advance(T, q, zero, zero, dt, Tr, qr, tau)
    f = (1.0 - dt / tau) ** n
    np.testing.assert_allclose(T - Tr, 1.5 * f, rtol=1e-9)
    np.testing.assert_allclose(q - qr, -0.1 * g.q * f, rtol=1e-9, atol=1e-18)


def test_step_conserves_column_energy_and_water(oracle):
    """Without relaxation, one step changes column enthalpy by Lv times the
    precipitated water and column water by minus it (both schemes conserve
    both, Sec. II-A's tendencies in flux form), wherever no q floor binds."""
    g = S.latlon_grid(24, 36)
    recs = []
    oracle.column_model(g, 1, tau_relax=0.0,
                        record=lambda s, T, q, d, sh: recs.append((T, q, d, sh)))
    T1, q1, d, sh = recs[0]
    p_int = g.hyai[:, None] * 1e5 + g.hybi[:, None] * g.ps[None, :]
    m = np.diff(p_int, axis=0) / P.GRAV
    rain = (d["prec"] + sh["prec"]) * g.dt
    dE = (m * P.CP * (T1 - g.T)).sum(axis=0)
    dW = (m * (q1 - g.q)).sum(axis=0)
    floored = np.any(q1 == 0.0, axis=0)
    act = (((d["flags"] | sh["flags"]) & oracle.F_ACTIVE) > 0) & ~floored
    assert act.sum() > 100
    scale = (m * P.CP * np.abs(T1 - g.T)).sum(axis=0)[act]
    assert np.all(np.abs(dE[act] - P.LV * rain[act]) <= 1e-9 * scale)
    assert np.all(np.abs(dW[act] + rain[act]) <= 1e-9 * scale / P.LV)
