"""Pins of the oracle's convective momentum transport.

A wind component is carried by the plumes like a tracer, with the plumes'
convective-scale pressure-gradient term (coefficients c_up, c_down) pushing the
plume's momentum towards the environment's by that fraction of the wind change
it crosses, and the environment's tendency the divergence of the interface eddy
fluxes.  Pinned against what the mathematics fixes:
* with both coefficients 0 it is the tracer transport (a separate, separately
  pinned code path);
* column momentum is conserved and a uniform wind is left unchanged, whatever
  the coefficients; the transport is linear (its matrix annihilates a uniform
  wind and conserves momentum);
* with both coefficients 1 every plume's momentum equals the environment's at
  every layer it crosses, so the tendency has a closed form in the mass-flux
  profiles alone: m_k du_k/dt = (F_k+1 - F_k) + (G_k - G_k+1) with
  F_k = mu_k (u_k - u_k-1) and G_k+1 = md_k (u_k - u_k+1);
* for any coefficients it equals an independent budget of the mass-flux
  profiles (the tracer budget of inflow and outflow with the plume recurrence
  written on mu, du, md, minus the pressure force in each layer crossed).
The shallow pins run with the deep scheme off, so the shallow scheme sees the
grid's own state and wind."""
import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S
from tests import physics_ref as P


@pytest.fixture(scope="module")
def grid():
    return S.latlon_grid(24, 36)


def _layer_mass(g):
    p_int = g.hyai[:, None] * 1e5 + g.hybi[:, None] * g.ps[None, :]
    return np.diff(p_int, axis=0) / P.GRAV


def _wind(g, seed, positive=False):
    """A sheared wind with random structure: [2][pver][n]."""
    rng = np.random.default_rng(seed)
    k = np.arange(g.pver)[:, None]
    base = np.stack([10.0 + 20.0 * (1 - k / g.pver), -5.0 + 8.0 * np.sin(k / 4.0)])
    uv = base + rng.normal(0.0, 3.0, (2, g.pver, g.n_cols))
    if positive:
        uv = np.abs(uv) + 1.0
    return uv


def _scale(f, m):
    """Each column's transport rate: max over levels of (mu + du + md) / m."""
    return ((f["mu"] + f["du"] + f["md"]) / m).max(axis=0)


@pytest.fixture(scope="module")
def deep_off(oracle):
    return oracle.deep_params(capelmt=1e30)


def test_zero_coefficients_are_the_tracer_transport(oracle, grid):
    g = grid
    uv = _wind(g, 1, positive=True)  # positive: the tracer path's floor at 0 never binds
    td, ts = oracle.deep_shallow_momentum(g, uv, 0.0, 0.0, threads=4)
    rd, rs, fd, fs = oracle.deep_shallow_tracers(g, uv, threads=4)
    m = _layer_mass(g)
    for a, b, f in ((td, rd, fd), (ts, rs, fs)):
        assert np.abs(b).max() > 0
        tol = 1e-12 * np.abs(uv).max() * _scale(f, m)
        assert np.all(np.abs(a - b) <= tol[None, None, :])


@pytest.mark.parametrize("cu,cd", [(0.7, 0.7), (0.3, 0.9), (1.0, 0.0)])
def test_conservation_and_uniform_wind(oracle, grid, cu, cd):
    g = grid
    m = _layer_mass(g)
    uv = _wind(g, 2)
    td, ts = oracle.deep_shallow_momentum(g, uv, cu, cd, threads=4)
    _, _, fd, fs = oracle.deep_shallow_tracers(g, np.ones((1, g.pver, g.n_cols)), threads=4)
    for t, f in ((td, fd), (ts, fs)):
        colsum = np.abs((m[None] * t).sum(axis=1))
        scale = (m[None] * np.abs(t)).sum(axis=1) + 1e-300
        assert np.all(colsum <= 1e-12 * scale)
        assert np.count_nonzero(t) > 100
    uni = np.ones((2, g.pver, g.n_cols)) * np.array([7.0, -3.0])[:, None, None]
    td, ts = oracle.deep_shallow_momentum(g, uni, cu, cd, threads=4)
    for t, f in ((td, fd), (ts, fs)):
        assert np.all(np.abs(t) <= 1e-13 * 7.0 * _scale(f, m)[None, None, :])


def test_linear_transport_matrix(oracle, grid):
    """The transport of one column is linear in the wind: build its matrix from
    unit profiles; it annihilates a uniform wind (A 1 = 0) and conserves
    momentum (m^T A = 0); a random wind's tendency is A u."""
    g = grid
    od, _ = oracle.deep_shallow(g, threads=4)
    i = int(np.where((od["flags"] & 2) > 0)[0][3])
    col = S.Columns(g.name, g.pver, g.T[:, [i]].copy(), g.q[:, [i]].copy(), g.ps[[i]].copy(),
                    g.hyai, g.hybi)
    pver = g.pver
    A = np.zeros((pver, pver))
    for j in range(pver):
        e = np.zeros((2, pver, 1))
        e[0, j, 0] = 1.0
        td, _ = oracle.deep_shallow_momentum(col, e, 0.6, 0.4)
        A[:, j] = td[0, :, 0]
    m = _layer_mass(col)[:, 0]
    s = np.abs(A).max()
    assert s > 0
    assert np.abs(A.sum(axis=1)).max() <= 1e-12 * s
    assert np.abs(m @ A).max() <= 1e-12 * s * m.max()
    u = _wind(col, 3)
    td, _ = oracle.deep_shallow_momentum(col, u, 0.6, 0.4)
    assert np.allclose(td[0, :, 0], A @ u[0, :, 0], rtol=0, atol=1e-12 * s * np.abs(u).max())


def _closed_form_c1(u, f):
    """Tendency with both coefficients 1, from the mass-flux profiles alone."""
    mu, md = f["mu"], f["md"]
    pver = u.shape[0]
    F = np.zeros((pver + 1,) + u.shape[1:])
    G = np.zeros_like(F)
    F[1:pver] = mu[1:] * (u[1:] - u[:-1])
    G[1:pver] = md[:-1] * (u[:-1] - u[1:])
    return (F[1:] - F[:-1]) + (G[:-1] - G[1:])


def test_unit_coefficients_closed_form(oracle, grid, deep_off):
    g = grid
    m = _layer_mass(g)
    uv = _wind(g, 4)
    # deep scheme on the grid's state
    td, _ = oracle.deep_shallow_momentum(g, uv, 1.0, 1.0, threads=4)
    _, _, fd, _ = oracle.deep_shallow_tracers(g, np.ones((1, g.pver, g.n_cols)), threads=4)
    for n in range(2):
        want = _closed_form_c1(uv[n], fd) / m
        tol = 1e-11 * np.abs(uv).max() * _scale(fd, m)
        assert np.all(np.abs(td[n] - want) <= tol[None, :])
    # shallow scheme, the deep scheme off (it sees the grid's own wind)
    _, ts = oracle.deep_shallow_momentum(g, uv, 1.0, 1.0, dpar=deep_off, threads=4)
    _, _, _, fs = oracle.deep_shallow_tracers(g, np.ones((1, g.pver, g.n_cols)), dpar=deep_off,
                                              threads=4)
    assert np.count_nonzero(fs["mu"]) > 100
    for n in range(2):
        want = _closed_form_c1(uv[n], fs) / m
        tol = 1e-11 * np.abs(uv).max() * _scale(fs, m)
        assert np.all(np.abs(ts[n] - want) <= tol[None, :])


def _profile_budget(u, f, m, c_up, c_down, kb, kt, jd):
    """One column's tendency from its mass-flux profiles: the plume recurrences
    written on mu, du, md (plume leaving layer k: mu_k u_k = (mu_k+1 - du_k)
    (u_k+1 + c_up (u_k - u_k+1)) + e_k u_k, e_k = mu_k - mu_k+1 + du_k; downdraft
    leaving k: md_k d_k = md_k-1 (d_k-1 + c_down (u_k - u_k-1)) + (md_k - md_k-1)
    u_k), the tracer budget of inflow and outflow of each layer, and the
    pressure force each plume exerts in each layer it crosses."""
    mu, du, md = f["mu"], f["du"], f["md"]
    pver = u.size
    t = np.zeros(pver)
    if kt < 0:
        return t
    up = np.zeros(pver)
    pf = np.zeros(pver)
    prev = 0.0
    for k in range(kb, kt - 1, -1):
        cont = (mu[k + 1] if k + 1 < pver else 0.0) - du[k]
        ubelow = up[k + 1] if k + 1 < pver else 0.0
        gain = c_up * cont * (u[k] - (u[k + 1] if k + 1 < pver else u[k]))
        pf[k] += gain
        e = mu[k] - (mu[k + 1] if k + 1 < pver else 0.0) + du[k]
        if mu[k] > 0:
            up[k] = (cont * ubelow + gain + e * u[k]) / mu[k]
        prev = mu[k]
    dn = np.zeros(pver)
    if jd >= 0:
        for k in range(jd, kb):
            mdp = md[k - 1] if k > jd else 0.0
            dprev = dn[k - 1] if k > jd else 0.0
            gain = c_down * mdp * (u[k] - (u[k - 1] if k > jd else u[k]))
            pf[k] += gain
            dn[k] = (mdp * dprev + gain + (md[k] - mdp) * u[k]) / md[k]
    for k in range(kt, kb + 1):
        # inflow: plume air detrained here from below, environment subsiding from
        # above, environment rising from below with the downdraft's compensation,
        # the downdraft detraining into the launch layer; outflow: this layer's air
        # entrained into the plumes and carried away
        inflow = du[k] * (up[k + 1] if k + 1 < pver else 0.0) + mu[k] * u[k - 1] \
            if k > 0 else du[k] * up[k + 1]
        outflow = (du[k] + mu[k]) * u[k]
        if jd >= 0 and jd <= k <= kb - 1:
            inflow += md[k] * u[k + 1]
            outflow += md[k] * u[k]
        if jd >= 0 and k == kb:
            inflow += md[kb - 1] * dn[kb - 1]
            outflow += md[kb - 1] * u[kb]
        t[k] = (inflow - outflow - pf[k]) / m[k]
    return t


@pytest.mark.parametrize("cu,cd", [(0.7, 0.7), (0.25, 0.9)])
def test_profile_budget(oracle, grid, deep_off, cu, cd):
    g = grid
    m = _layer_mass(g)
    uv = _wind(g, 5)
    td, _ = oracle.deep_shallow_momentum(g, uv, cu, cd, threads=4)
    od, _ = oracle.deep_shallow(g, threads=4)
    _, _, fd, _ = oracle.deep_shallow_tracers(g, np.ones((1, g.pver, g.n_cols)), threads=4)
    _, ts = oracle.deep_shallow_momentum(g, uv, cu, cd, dpar=deep_off, threads=4)
    _, os_ = oracle.deep_shallow(g, dpar=deep_off, threads=4)
    _, _, _, fs = oracle.deep_shallow_tracers(g, np.ones((1, g.pver, g.n_cols)), dpar=deep_off,
                                              threads=4)
    done = 0
    for i in range(g.n_cols):
        fcol = {k: v[:, i] for k, v in fd.items()}
        scol = {k: v[:, i] for k, v in fs.items()}
        for n in range(2):
            if od["flags"][i] & 2:
                want = _profile_budget(uv[n, :, i], fcol, m[:, i], cu, cd, int(od["kb"][i]),
                                       int(od["ktop"][i]), int(od["kaux"][i]))
                tol = 1e-11 * np.abs(uv).max() * _scale(fd, m)[i]
                assert np.all(np.abs(td[n, :, i] - want) <= tol), (i, n)
                done += 1
            if os_["flags"][i] & 2:
                want = _profile_budget(uv[n, :, i], scol, m[:, i], cu, cd, g.pver - 1,
                                       int(os_["ktop"][i]), -1)
                tol = 1e-11 * np.abs(uv).max() * _scale(fs, m)[i]
                assert np.all(np.abs(ts[n, :, i] - want) <= tol), (i, n)
                done += 1
    assert done > 200
