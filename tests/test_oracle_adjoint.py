"""Pins of the oracle's deep-scheme gradients (tangent mode) against central
finite differences of the FP64 oracle and against exact identities."""
import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S
from tests import physics_ref as P


@pytest.fixture(scope="module")
def grid():
    g = S.latlon_grid(24, 36, tau_range=(1800.0, 7200.0))
    g.lam = np.full(g.n_cols, 1e-3)
    return g


def _J(oracle, g, T, q, lam, tau, gP, gH, w):
    sub = S.Columns("c", g.pver, T, q, g.ps[:1].copy(), g.hyai, g.hybi,
                    np.array([lam]), np.array([tau]), g.dt)
    o = oracle.deep(sub)
    p_int, p_mid = P.levels(g.hyai, g.hybi, sub.ps[0])
    m = np.diff(p_int) / P.GRAV
    wk = p_mid / sub.ps[0] if w is None else w
    return gP * o["prec"][0] + gH * np.sum(wk * m * P.CP * o["dTdt"][:, 0]), o


def _decisions(o):
    return tuple(int(o[k][0]) for k in ("flags", "kb", "klcl", "ktop", "kaux"))


def _select(oracle, g, n):
    od = oracle.deep(g, threads=4)
    act = np.where((od["flags"] & oracle.F_ACTIVE) > 0)[0]
    far = act[np.abs(od["cape"][act] - 70.0) >= 5.0]
    return far[:: max(1, len(far) // n)][:n]


@pytest.mark.parametrize("gP,gH", [(1.0, 0.0), (0.0, 1e-3), (0.7, -2e-4)])
def test_tangent_matches_central_differences(oracle, grid, gP, gH):
    cols = _select(oracle, grid, 6)
    assert len(cols) >= 4
    gPv = np.full(grid.n_cols, gP)
    gHv = np.full(grid.n_cols, gH)
    gT, gq, gl, gt = oracle.deep_adjoint(grid, gPv, gHv, threads=4)
    checked = 0
    for i in cols:
        T0, q0 = grid.T[:, i].copy(), grid.q[:, i].copy()
        lam0, tau0 = grid.lam[i], grid.tau[i]
        _, o0 = _J(oracle, grid, T0[:, None], q0[:, None], lam0, tau0, gP, gH, None)
        dec0 = _decisions(o0)
        fd = []
        an = []
        ok = True
        for v in range(2 * grid.pver + 2):
            T, q, lam, tau = T0.copy(), q0.copy(), lam0, tau0
            if v < grid.pver:
                h = 1e-6 * T0[v]
                vals = [(T0[v] + s * h) for s in (1, -1)]
            elif v < 2 * grid.pver:
                h = 1e-6 * max(q0[v - grid.pver], 1e-7)
                vals = [(q0[v - grid.pver] + s * h) for s in (1, -1)]
            elif v == 2 * grid.pver:
                h = 1e-6 * lam0
                vals = [lam0 + h, lam0 - h]
            else:
                h = 1e-6 * tau0
                vals = [tau0 + h, tau0 - h]
            Js = []
            for x in vals:
                T, q, lam, tau = T0.copy(), q0.copy(), lam0, tau0
                if v < grid.pver:
                    T[v] = x
                elif v < 2 * grid.pver:
                    q[v - grid.pver] = x
                elif v == 2 * grid.pver:
                    lam = x
                else:
                    tau = x
                J, o = _J(oracle, grid, T[:, None], q[:, None], lam, tau, gP, gH, None)
                if _decisions(o) != dec0:
                    ok = False
                Js.append(J)
            fd.append((Js[0] - Js[1]) / (2 * h))
            if v < grid.pver:
                an.append(gT[v, i])
            elif v < 2 * grid.pver:
                an.append(gq[v - grid.pver, i])
            elif v == 2 * grid.pver:
                an.append(gl[i])
            else:
                an.append(gt[i])
        if not ok:
            continue
        fd, an = np.array(fd), np.array(an)
        # scale each entry by the input it perturbs so T, q, lambda, tau are comparable
        xs = np.concatenate([T0, np.maximum(q0, 1e-7), [lam0, tau0]])
        err = np.abs(fd - an) * xs
        assert err.max() <= 1e-6 * np.abs(an * xs).max(), (i, err.max(), np.abs(an * xs).max())
        checked += 1
    assert checked >= 3


def test_dP_dtau_identity(oracle, grid):
    """P is proportional to 1/tau when the limiter is off: dP/dtau = -P/tau."""
    od = oracle.deep(grid, threads=4)
    act = ((od["flags"] & oracle.F_ACTIVE) > 0) & ((od["flags"] & oracle.F_LIMITED) == 0)
    assert act.sum() > 5
    one = np.ones(grid.n_cols)
    _, _, _, gt = oracle.deep_adjoint(grid, one, 0 * one, threads=4)
    np.testing.assert_allclose(gt[act], -od["prec"][act] / grid.tau[act], rtol=1e-10)


def test_heating_gradient_equals_lv_precip_gradient_for_unit_weights(oracle, grid):
    """With w = 1 column heating equals Lv P exactly, so the gradients agree."""
    one = np.ones(grid.n_cols)
    w = np.ones(grid.pver)
    a = oracle.deep_adjoint(grid, one, 0 * one, threads=4)
    b = oracle.deep_adjoint(grid, 0 * one, one, w_heat=w, threads=4)
    for x, y in zip(a, b):
        np.testing.assert_allclose(y, P.LV * x, rtol=1e-10, atol=1e-12 * np.abs(P.LV * x).max())


def test_zero_gradient_off_trigger(oracle, grid):
    od = oracle.deep(grid, threads=4)
    off = (od["flags"] & oracle.F_ACTIVE) == 0
    one = np.ones(grid.n_cols)
    gT, gq, gl, gt = oracle.deep_adjoint(grid, one, one, threads=4)
    assert np.all(gT[:, off] == 0) and np.all(gq[:, off] == 0)
    assert np.all(gl[off] == 0) and np.all(gt[off] == 0)
