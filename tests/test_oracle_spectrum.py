"""Pins of the oracle's plume-spectrum variant of the deep scheme: n plumes with
entrainment rates lambda * spread^(i/(n-1) - 1/2), each carrying 1/n of the
cloud-base mass flux and detraining at its own top; the ensemble's top starts
the downdraft.

Pinned against what the mathematics fixes: one plume is the bulk scheme
exactly; a spectrum of identical plumes (spread 1) is the bulk scheme up to
rounding; without a downdraft the ensemble's unit tendencies and rain are the
mass-weighted sums of single-plume runs at the member rates (superposition),
its top is the highest member top; column enthalpy and water still close."""
import math

import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S


@pytest.fixture(scope="module")
def grid():
    return S.latlon_grid(24, 36)


def _act(o, oracle):
    return (o["flags"] & oracle.F_ACTIVE) > 0


def test_one_plume_is_the_bulk_scheme(oracle, grid):
    a = oracle.deep_shallow(grid, threads=4)
    b = oracle.deep_shallow(grid, dpar=oracle.deep_params(n_plumes=1, plume_spread=9.0),
                            threads=4)
    for x, y in zip(a, b):
        for k in x:
            assert np.array_equal(x[k], y[k]), k


@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_identical_members_reproduce_the_bulk_plume(oracle, grid, n):
    a, _ = oracle.deep_shallow(grid, threads=4)
    b, _ = oracle.deep_shallow(grid, dpar=oracle.deep_params(n_plumes=n, plume_spread=1.0),
                               threads=4)
    for k in ("flags", "kb", "klcl", "ktop", "kaux"):
        assert np.array_equal(a[k], b[k]), k
    act = _act(a, oracle)
    assert act.sum() > 100
    for k in ("dTdt", "dqdt"):
        den = np.abs(a[k]).max(axis=0)[act]
        assert (np.abs(a[k] - b[k]).max(axis=0)[act] / den).max() <= 1e-12, k
    assert np.allclose(a["prec"], b["prec"], rtol=1e-12, atol=0.0)


@pytest.mark.parametrize("n", [2, 4])
def test_superposition_without_downdraft(oracle, grid, n):
    g = grid
    spread, lam, tau = 4.0, 1e-3, 3600.0
    par_e = oracle.deep_params(n_plumes=n, plume_spread=spread, alpha_dd=0.0)
    checked = 0
    for i in range(0, g.n_cols, 7):
        T, q, ps = g.T[:, i], g.q[:, i], g.ps[i]
        e = oracle.deep_column_diag(g.pver, g.hyai, g.hybi, T, q, ps, lam, tau, par_e, g.dt)
        if not e.triggered or e.jt < 0:
            continue
        dh = np.zeros(g.pver)
        dq = np.zeros(g.pver)
        sumR, tops = 0.0, []
        for ip in range(n):
            li = lam * spread ** (ip / (n - 1) - 0.5)
            d = oracle.deep_column_diag(g.pver, g.hyai, g.hybi, T, q, ps, li, tau,
                                        oracle.deep_params(alpha_dd=0.0), g.dt)
            if d.jt < 0 or d.jt >= d.klcl:
                continue  # this member has no cloud above the LCL
            dh += np.array(d.dh[:g.pver]) / n
            dq += np.array(d.dq[:g.pver]) / n
            sumR += d.sumR / n
            tops.append(d.jt)
        assert e.jt == min(tops)
        sc = np.abs(dh).max()
        assert np.abs(np.array(e.dh[:g.pver]) - dh).max() <= 1e-12 * sc
        assert np.abs(np.array(e.dq[:g.pver]) - dq).max() <= 1e-12 * np.abs(dq).max()
        assert e.sumR == pytest.approx(sumR, rel=1e-12)
        checked += 1
    assert checked > 15


@pytest.mark.parametrize("n", [2, 3, 4])
def test_ensemble_conserves_and_reaches_the_least_entraining_top(oracle, grid, n):
    g = grid
    a, _ = oracle.deep_shallow(g, threads=4)
    b, _ = oracle.deep_shallow(g, dpar=oracle.deep_params(n_plumes=n), threads=4)
    act = _act(b, oracle)
    assert act.sum() > 100
    assert b["cons_err"][act].max() <= 1e-12
    # decisions of the trigger stage do not depend on the plumes
    for k in ("kb", "klcl"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["flags"] & 1, b["flags"] & 1)
    # the top of the ensemble is the top of its least-entraining member
    c, _ = oracle.deep_shallow(g, lam=np.full(g.n_cols, 1e-3 / math.sqrt(4.0)), threads=4)
    both = act & _act(c, oracle)
    assert both.sum() > 100
    assert np.array_equal(b["ktop"][both], c["ktop"][both])
