"""Pins of the oracle's convective tracer transport and mass-flux profiles.

Each scheme mixes a passive tracer as it mixes its conserved moist static
energy, with no source term.  Pinned here against what the mathematics fixes:
a uniform tracer is left unchanged (exactly); column tracer mass is conserved;
the transport matrix of an upwind flux-form scheme with non-negative mass
fluxes has non-negative off-diagonal entries; transporting the column's own
moist static energy reproduces each scheme's MSE tendency cp dT/dt + Lv dq/dt,
computed by the schemes' separate (and separately pinned) code; and the
mass-flux profiles close the plume's mass budget."""
import math

import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S
from tests import physics_ref as P


@pytest.fixture(scope="module")
def grid():
    return S.latlon_grid(24, 36)


@pytest.fixture(scope="module")
def runs(oracle, grid):
    g = grid
    od, os_ = oracle.deep_shallow(g, threads=4)
    return od, os_


@pytest.fixture(scope="module")
def off(oracle, grid):
    """Deep scheme switched off (CAPE threshold out of reach): the shallow scheme
    then sees the original state and tracers in every column."""
    dpar = oracle.deep_params(capelmt=1e30)
    od, os_ = oracle.deep_shallow(grid, dpar=dpar, threads=4)
    assert not np.any(_active(od, oracle))
    return dpar, os_


def _active(o, oracle):
    return (o["flags"] & oracle.F_ACTIVE) > 0


def _layer_mass(g):
    p_int = g.hyai[:, None] * 1e5 + g.hybi[:, None] * g.ps[None, :]
    return np.diff(p_int, axis=0) / P.GRAV


def _mse(oracle, g, cols):
    """Moist static energy cp T + g z + Lv q of the given columns ([pver][len])."""
    h = np.zeros((g.pver, len(cols)))
    for j, i in enumerate(cols):
        p_int, p_mid = oracle.levels(g.pver, g.hyai, g.hybi, g.ps[i])
        _, z_mid = oracle.heights(g.T[:, i], g.q[:, i], p_int, p_mid)
        h[:, j] = P.CP * g.T[:, i] + P.GRAV * z_mid + P.LV * g.q[:, i]
    return h


def test_uniform_tracer_is_unchanged(oracle, grid, runs):
    g = grid
    od, os_ = runs
    assert _active(od, oracle).sum() > 20 and _active(os_, oracle).sum() > 20
    c = np.array([1.0, 3.7e-9])
    tr = np.ones((2, g.pver, g.n_cols)) * c[:, None, None]
    td, ts, fd, fs = oracle.deep_shallow_tracers(g, tr, threads=4)
    m = _layer_mass(g)
    for t, f in ((td, fd), (ts, fs)):
        # the plume of a uniform tracer carries the same value (weighted means of
        # equal values): zero up to the rounding of those means
        rate = (f["mu"] + f["du"] + f["md"]).max(axis=0) / m.min(axis=0)
        assert np.all(np.abs(t) <= 1e-14 * c[:, None, None] * rate[None, None, :])
    # the subsidence terms alone are exact: nothing moves below the plume tops
    assert np.all(td[:, -1][:, ~_active(od, oracle)] == 0.0)


def test_column_tracer_mass_is_conserved(oracle, grid, runs):
    g = grid
    rng = np.random.default_rng(11)
    tr = rng.uniform(0.0, 1.0, (3, g.pver, g.n_cols)) * np.array([1.0, 1e-6, 1e-9])[:, None, None]
    td, ts, _, _ = oracle.deep_shallow_tracers(g, tr, threads=4)
    m = _layer_mass(g)
    for t in (td, ts):
        net = np.abs(np.sum(m[None] * t, axis=1))
        scale = np.sum(m[None] * np.abs(t), axis=1) + 1e-300
        assert (net / scale).max() <= 1e-13, (net / scale).max()


def test_mse_transport_reproduces_scheme_tendencies(oracle, grid, runs, off):
    """Deep: on every active column.  Shallow: with the deep scheme off, so that
    it sees the original state and tracer."""
    g = grid
    od, _ = runs
    dpar_off, os_ = off
    h = _mse(oracle, g, np.arange(g.n_cols))
    td, _, _, _ = oracle.deep_shallow_tracers(g, h[None], threads=4)
    _, ts, _, _ = oracle.deep_shallow_tracers(g, h[None], dpar=dpar_off, threads=4)
    ad, as_ = _active(od, oracle), _active(os_, oracle)
    assert ad.sum() > 20 and as_.sum() > 20
    for t, o, sel in ((td[0], od, ad), (ts[0], os_, as_)):
        want = P.CP * o["dTdt"] + P.LV * o["dqdt"]
        err = np.abs(t - want)[:, sel].max(axis=0)
        scale = np.abs(want)[:, sel].max(axis=0)
        assert (err / scale).max() <= 1e-9, (err / scale).max()
        # no tendency where the scheme is inactive
        assert np.all(t[:, ~sel] == 0.0)


def test_transport_matrix_is_upwind_monotone(oracle, grid, runs, off):
    """Unit tracers e_j give the columns of each column's transport matrix A:
    A 1 = 0, m^T A = 0 and A[k, j] >= 0 for k != j."""
    g = grid
    od, _ = runs
    dpar_off, os_ = off
    ad, as_ = _active(od, oracle), _active(os_, oracle)
    tr = np.zeros((g.pver, g.pver, g.n_cols))
    for j in range(g.pver):
        tr[j, j, :] = 1.0
    td, _, _, _ = oracle.deep_shallow_tracers(g, tr, threads=4)
    _, ts, _, _ = oracle.deep_shallow_tracers(g, tr, dpar=dpar_off, threads=4)
    m = _layer_mass(g)
    checked = 0
    for t, sel in ((td, ad), (ts, as_)):
        for i in np.flatnonzero(sel):
            A = t[:, :, i].T  # A[k, j] = tendency at k of unit tracer at j
            scale = np.abs(A).max()
            assert scale > 0.0
            off = A - np.diag(np.diag(A))
            assert off.min() >= -1e-14 * scale, off.min() / scale
            assert np.abs(A.sum(axis=1)).max() <= 1e-12 * scale
            assert np.abs(m[:, i] @ A).max() <= 1e-12 * scale * m[:, i].max()
            checked += 1
    assert checked > 40


def test_mass_flux_profiles_close_the_plume_budget(oracle, grid, runs, off):
    g = grid
    od, os_ = runs
    _, _, fd, fs = oracle.deep_shallow_tracers(g, np.zeros((0, g.pver, g.n_cols)), threads=4)
    ad, as_ = _active(od, oracle), _active(os_, oracle)
    assert ad.sum() > 20 and as_.sum() > 20
    for f in (fd, fs):
        for v in f.values():
            assert v.min() >= 0.0
    for f, o, act in ((fd, od, ad), (fs, os_, as_)):
        for v in f.values():
            assert np.all(v[:, ~act] == 0.0)
        for i in np.flatnonzero(act):
            kb, kt = o["kb"][i], o["ktop"][i]
            mu, du = f["mu"][:, i], f["du"][:, i]
            assert np.all(mu[: kt + 1] == 0.0) and np.all(mu[kb + 1:] == 0.0)
            assert np.all(mu[kt + 1: kb + 1] > 0.0)
            assert mu[kb] == pytest.approx(o["mb"][i], rel=1e-15)  # eta = 1 at the launch layer
            assert du[kt] == mu[kt + 1]  # everything left detrains at the top
    # deep: entrainment eu = mu[k] - mu[k+1] >= 0 below the top (no detrainment there),
    # and the updraft grows as exp(lambda (z - z_b)) capped by the entrainment scale
    for i in np.flatnonzero(ad)[:30]:
        kb, kt = od["kb"][i], od["ktop"][i]
        mu = fd["mu"][:, i]
        assert np.all(np.diff(mu[kt + 1: kb + 1]) <= 0.0)  # mu grows upwards
        assert np.all(fd["du"][kt + 1:, i] == 0.0)
    # shallow (deep off: its input is the original state): constant mass flux
    # M_b and detrainment fraction 1 - exp(-eps dz)
    dpar_off, os0 = off
    _, _, _, fs = oracle.deep_shallow_tracers(g, np.zeros((0, g.pver, g.n_cols)), dpar=dpar_off,
                                              threads=4)
    eps = oracle.shallow_params().eps_s
    for i in np.flatnonzero(_active(os0, oracle))[:30]:
        kt, klcl = os0["ktop"][i], os0["klcl"][i]
        mb = os0["mb"][i]
        mu, du = fs["mu"][:, i], fs["du"][:, i]
        assert np.all(mu[kt + 1:] == mb)
        p_int, p_mid = oracle.levels(g.pver, g.hyai, g.hybi, g.ps[i])
        z_int, _ = oracle.heights(g.T[:, i], g.q[:, i], p_int, p_mid)
        for k in range(kt + 1, g.pver - 1):
            want = mb * (-math.expm1(-eps * (z_int[k] - z_int[k + 1]))) if k < klcl else 0.0
            assert du[k] == pytest.approx(want, rel=1e-12, abs=1e-300)
    assert np.all(fd["md"][:, ad].sum(axis=0) >= 0.0)


def _budget_tendency(mu, du, md, kb, kt, jd, m, c):
    """One column's tracer tendency from its mass-flux profiles alone, as the
    budget of what crosses each environment layer's boundaries:

      subsidence    mu[k] down through the top of layer k, carrying c[k-1];
      ascent        md[k] up through the bottom of layer k (it replaces the
                    downdraft air leaving k), carrying c[k+1];
      updraft       entrains e[k] = mu[k] - mu[k+1] + du[k] of c[k] and detrains
                    du[k] of the value cu[k+1] arriving from below, its own value
                    following from its mass budget
                    mu[k] cu[k] = (mu[k+1] - du[k]) cu[k+1] + e[k] c[k];
      downdraft     entrains md[k] - md[k-1] of c[k] on jd..kb-1
                    (md[k] cd[k] = md[k-1] cd[k-1] + (md[k] - md[k-1]) c[k]) and
                    detrains md[kb-1] of cd[kb-1] into the launch layer kb.

    Written as inflow minus outflow (conservative form), not as the upwind
    differences the schemes use."""
    n = len(c)
    mu_ = np.append(mu, 0.0)  # nothing rises into the lowest layer from below
    md_up = np.concatenate(([0.0], md))  # md_up[k] = md[k-1]: crosses the top of layer k
    cu = np.zeros(n + 1)
    for k in range(kb, kt, -1):
        e = mu_[k] - mu_[k + 1] + du[k]
        cu[k] = ((mu_[k + 1] - du[k]) * cu[k + 1] + e * c[k]) / mu_[k]
    cd = np.zeros(n)
    if jd >= 0:
        for k in range(jd, kb):
            if md[k] > 0.0:
                cd[k] = (md_up[k] * (cd[k - 1] if k > jd else 0.0) + (md[k] - md_up[k]) * c[k]) / md[k]
    t = np.zeros(n)
    for k in range(kt, kb + 1):
        above = c[k - 1] if k > 0 else 0.0
        below = c[k + 1] if k + 1 < n else 0.0
        flow = mu_[k] * above - mu_[k + 1] * c[k]  # subsidence in, out
        flow += md[k] * below - md_up[k] * c[k]  # compensating ascent in, out
        e = mu_[k] - mu_[k + 1] + du[k]
        flow += du[k] * cu[k + 1] - e * c[k]  # updraft detrainment, entrainment
        if jd >= 0 and jd <= k <= kb - 1:
            flow -= (md[k] - md_up[k]) * c[k]  # downdraft entrainment
        if jd >= 0 and k == kb:
            flow += md[kb - 1] * cd[kb - 1]  # downdraft detrainment into the launch layer
        t[k] = flow / m[k]
    return t


def test_flux_profiles_reproduce_the_transport(oracle, grid, runs):
    """The profiles mu, du, md the oracle reports carry exactly the transport its
    schemes apply: the budget above, fed the profiles, reproduces the deep
    tendencies and the shallow tendencies of the deep-updated tracer
    (max(c + dt tend_deep, 0)) on every active column, and the downdraft flux
    vanishes outside kaux..kb-1."""
    g = grid
    od, os_ = runs
    rng = np.random.default_rng(5)
    tr = rng.uniform(0.0, 1.0, (2, g.pver, g.n_cols)) * np.array([1.0, 1e-8])[:, None, None]
    td, ts, fd, fs = oracle.deep_shallow_tracers(g, tr, threads=4)
    m = _layer_mass(g)
    checked = 0
    for t_all, f, o, deep in ((td, fd, od, True), (ts, fs, os_, False)):
        act = _active(o, oracle)
        assert act.sum() > 20
        for i in np.flatnonzero(act):
            kb, kt = int(o["kb"][i]), int(o["ktop"][i])
            jd = int(o["kaux"][i]) if deep else -1
            md = f["md"][:, i]
            if deep and jd >= 0:
                assert np.all(md[:jd] == 0.0) and np.all(md[kb:] == 0.0)
            else:
                assert np.all(md == 0.0)
            for n in range(tr.shape[0]):
                c = tr[n, :, i] if deep else np.maximum(tr[n, :, i] + g.dt * td[n, :, i], 0.0)
                want = _budget_tendency(f["mu"][:, i], f["du"][:, i], md, kb, kt, jd, m[:, i], c)
                got = t_all[n, :, i]
                assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max(), (deep, i, n)
            checked += 1
    assert checked > 100
