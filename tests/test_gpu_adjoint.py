"""Deep-scheme adjoint on the GPU (conv_deep_adjoint, FP64) and its
torch.autograd.Function: equality with the oracle's forward-mode tangent,
central finite differences of the GPU forward scheme, exact identities of the
scheme (tau enters only through M_b = -CAPE/(tau F); column energy balance
H(w = 1) = Lv P), zero gradients where the scheme is inactive, and autograd
backward equal to the direct call."""
import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S
from tests.gpu_util import THREADS, to_device

pytestmark = pytest.mark.gpu

LV = 2.501e6
CP = 1004.64
GRAV = 9.80616


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _grid(nlat=96, nlon=144):
    """Lat-lon grid of 13,824 x 30 columns at the default size, with a per-column
    CAPE relaxation time and entrainment rate."""
    g = S.latlon_grid(nlat, nlon, tau_range=(1800.0, 7200.0))
    g.lam = 5e-4 + 1.5e-3 * S.uniform(20171104, 0, np.arange(g.n_cols), 0)
    return g


def _seeds(n, seed=7):
    c = np.arange(n)
    return 2.0 * S.uniform(seed, 0, c, 0) - 1.0, 2.0 * S.uniform(seed, 0, c, 1) - 1.0


def _gpu_adjoint(g, gP, gH, w_heat=None, ld=None, objective=False, gradient=True, T=None,
                 q=None):
    import torch

    from paper_1711_00289_gb300 import api

    n = g.n_cols
    ld = n if ld is None else ld
    T0, q0, ps, lam, tau = to_device(g, "fp64", ld)
    T = T0 if T is None else T
    q = q0 if q is None else q
    pad = lambda a: torch.tensor(S.to_ld(np.asarray(a, dtype=np.float64), ld), device="cuda")
    r = api.deep_adjoint(T, q, ps, api.VerticalGrid(g.hyai, g.hybi), gP=pad(gP), gH=pad(gH),
                         w_heat=w_heat, dt=g.dt, lam=lam, tau=tau, n_cols=n,
                         objective=objective, gradient=gradient)
    torch.cuda.synchronize()
    out = {}
    for k, v in r.items():
        a = v.cpu().numpy()
        out[k] = a[..., :n]
    return out


def _col_rel(x, y):
    """Per-column max-norm relative difference of [pver, n] (or [n]) arrays."""
    x, y = np.atleast_2d(x), np.atleast_2d(y)
    den = np.abs(y).max(axis=0)
    return np.abs(x - y).max(axis=0) / np.where(den > 0, den, 1.0), den


@pytest.mark.parametrize("weights", ["p_over_ps", "given"])
def test_gpu_adjoint_equals_oracle_tangent(oracle, weights):
    g = _grid()
    n = g.n_cols
    gP, gH = _seeds(n)
    w = None if weights == "p_over_ps" else np.linspace(0.2, 1.0, g.pver)
    got = _gpu_adjoint(g, gP, gH, w_heat=w, ld=S.pad_ld(n) + 32)
    ref = dict(zip(("gT", "gq", "glambda", "gtau"),
                   oracle.deep_adjoint(g, gP, gH, w_heat=w, threads=THREADS)))
    d = oracle.deep(g, threads=THREADS)
    active = (d["flags"] & 2) > 0
    assert active.sum() > 500 and (~active).sum() > 500
    for k in ("gT", "gq", "glambda", "gtau"):
        rel, den = _col_rel(got[k], ref[k])
        nz = den > 0
        assert rel[nz].max() <= 1e-10, f"{k}: max column-relative error {rel[nz].max():.3e}"
        assert np.all(got[k][..., ~nz] == 0.0), f"{k}: non-zero where the oracle's is zero"
    # columns where the scheme is inactive have exactly zero gradient
    for k in ("gT", "gq", "glambda", "gtau"):
        assert np.all(np.atleast_2d(got[k])[:, ~active] == 0.0)


def test_objective_values_match_forward_scheme(oracle):
    g = _grid(48, 72)
    n = g.n_cols
    w = np.linspace(0.5, 1.0, g.pver)
    got = _gpu_adjoint(g, np.zeros(n), np.zeros(n), w_heat=w, objective=True, gradient=False)
    d = oracle.deep(g, threads=THREADS)
    pi = g.hyai[:, None] * 1e5 + g.hybi[:, None] * g.ps[None, :]  # interface pressures
    m = (pi[1:] - pi[:-1]) / GRAV
    H_ref = (w[:, None] * m * CP * d["dTdt"]).sum(axis=0)
    np.testing.assert_allclose(got["P"], d["prec"], rtol=1e-10, atol=1e-12 * d["prec"].max())
    np.testing.assert_allclose(got["H"], H_ref, rtol=1e-10, atol=1e-10 * np.abs(H_ref).max())


def test_dP_dtau_is_minus_P_over_tau_when_unlimited(oracle):
    g = _grid(48, 72)
    n = g.n_cols
    got = _gpu_adjoint(g, np.ones(n), np.zeros(n), objective=True)
    d = oracle.deep(g, threads=THREADS)
    active = (d["flags"] & 2) > 0
    free = active & ((d["flags"] & 4) == 0)
    assert free.sum() > 50
    P, tau = got["P"][free], g.tau[free]
    np.testing.assert_allclose(got["gtau"][free], -P / tau, rtol=1e-12, atol=0)
    # the limiter fixes M_b independently of tau
    assert np.all(got["gtau"][active & ~free] == 0.0)


def test_energy_balance_of_gradients(oracle):
    """With w = 1, H = sum m cp dTdt equals Lv P identically (column energy
    balance of the flux-form tendencies), so grad H = Lv grad P."""
    g = _grid(48, 72)
    n = g.n_cols
    w1 = np.ones(g.pver)
    aP = _gpu_adjoint(g, np.ones(n), np.zeros(n), w_heat=w1, objective=True)
    aH = _gpu_adjoint(g, np.zeros(n), np.ones(n), w_heat=w1)
    active = aP["P"] > 0
    assert active.sum() > 100
    np.testing.assert_allclose(aP["H"][active], LV * aP["P"][active], rtol=1e-12)
    for k in ("gT", "gq", "glambda", "gtau"):
        rel, den = _col_rel(aH[k], LV * np.asarray(aP[k]))
        assert rel[den > 0].max() <= 1e-11, f"{k}: {rel[den > 0].max():.3e}"


def _forward(g, T, q, lam=None, tau=None):
    """GPU objective (P, H) and visible decisions at the given device state."""
    import torch

    from paper_1711_00289_gb300 import api

    n = g.n_cols
    _, _, ps, lam0, tau0 = to_device(g, "fp64")
    lam = lam0 if lam is None else lam
    tau = tau0 if tau is None else tau
    vg = api.VerticalGrid(g.hyai, g.hybi)
    r = api.deep_adjoint(T, q, ps, vg, dt=g.dt, lam=lam, tau=tau, objective=True,
                         gradient=False)
    o = api.deep(T, q, ps, vg, dt=g.dt, precision="fp64", lam=lam, tau=tau, path="plain")
    torch.cuda.synchronize()
    dec = np.stack([o[k].cpu().numpy() for k in ("flags", "kb", "klcl", "ktop", "kaux")])
    return r["P"].cpu().numpy()[:n], r["H"].cpu().numpy()[:n], dec


def test_gpu_adjoint_matches_central_differences(oracle):
    """Central differences of the GPU forward scheme, one input at a time over
    all columns at once (columns are independent), step 1e-6 of the variable's
    scale (T: 300 K; q: 0.02, on levels where q > 1e-6 so that q - h stays
    valid; lambda: 1e-3 1/m; tau: 3600 s).  Compared on columns whose CAPE is
    at least 5 J/kg from the trigger threshold and whose discrete decisions are
    unchanged at +-h: levels and flags are compared directly; hidden switches
    (highest buoyant layer, saturation of a plume level, downdraft cap, limiter
    level) show up as one-sided differences that disagree, and such columns
    are left out.  Bound: 1e-6 relative."""
    import torch

    g = _grid(24, 36)
    n = g.n_cols
    gP, gH = _seeds(n, seed=11)
    ad = _gpu_adjoint(g, gP, gH)
    T0, q0, ps, lam0, tau0 = to_device(g, "fp64")
    P0, H0, dec0 = _forward(g, T0, q0)
    J = lambda P, H: gP * P + gH * H
    d = oracle.deep(g, threads=THREADS)
    ok = ((d["flags"] & 2) > 0) & (np.abs(d["cape"] - 70.0) >= 5.0)
    kinked = np.zeros(n, bool)
    fd = {"gT": np.zeros((g.pver, n)), "gq": np.zeros((g.pver, n)), "glambda": np.zeros(n),
          "gtau": np.zeros(n)}
    cmp = {"gT": np.ones((g.pver, n), bool), "gq": g.q > 1e-6, "glambda": np.ones(n, bool),
           "gtau": np.ones(n, bool)}
    pert = [("gT", k) for k in range(g.pver)] + [("gq", k) for k in range(g.pver)] + \
        [("glambda", None), ("gtau", None)]
    J0 = J(P0, H0)
    for var, k in pert:
        if var == "gT":
            h = np.full(n, 1e-6 * 300.0)
        elif var == "gq":
            h = np.where(cmp["gq"][k], 1e-6 * 0.02, 0.0)
        elif var == "glambda":
            h = np.full(n, 1e-6 * 1e-3)
        else:
            h = np.full(n, 1e-6 * 3600.0)
        ht = torch.tensor(h, device="cuda")
        res = []
        for sgn in (1.0, -1.0):
            T, q, lam, tau = T0.clone(), q0.clone(), lam0.clone(), tau0.clone()
            {"gT": lambda: T[k].add_(sgn * ht), "gq": lambda: q[k].add_(sgn * ht),
             "glambda": lambda: lam.add_(sgn * ht), "gtau": lambda: tau.add_(sgn * ht)}[var]()
            P, H, dec = _forward(g, T, q, lam, tau)
            ok &= np.all(dec == dec0, axis=0)
            res.append(J(P, H))
        Jp, Jm = res
        hs = np.where(h > 0, h, 1.0)
        fwd, bwd = (Jp - J0) / hs, (J0 - Jm) / hs
        scale = np.maximum(np.abs(np.atleast_2d(ad[var])).max(axis=0), 1e-300)
        kinked |= (np.abs(fwd - bwd) > 1e-3 * scale) & (h > 0)
        c = (Jp - Jm) / (2 * hs)
        if k is None:
            fd[var] = c
        else:
            fd[var][k] = c
    use = ok & ~kinked
    assert use.sum() >= 0.8 * ok.sum() and use.sum() > 50, (use.sum(), ok.sum())
    # error relative to the column's gradient, or to |J| / (variable scale) where
    # that is larger (a gradient that nearly cancels is only as accurate as the
    # rounding noise of J allows a difference quotient to be)
    xs = {"gT": 300.0, "gq": 0.02, "glambda": 1e-3, "gtau": 3600.0}
    for var in fd:
        a = np.atleast_2d(np.asarray(ad[var]))
        den = np.maximum(np.abs(a).max(axis=0), np.abs(J0) / xs[var])
        err = np.where(np.atleast_2d(cmp[var]), np.abs(np.atleast_2d(fd[var]) - a), 0.0)
        rel = err.max(axis=0)[use] / den[use]
        assert rel.max() <= 1e-6, f"{var}: central difference vs adjoint {rel.max():.3e}"


def test_autograd_function_backward_equals_direct_call(oracle):
    import torch

    from paper_1711_00289_gb300 import api

    g = _grid(24, 36)
    n = g.n_cols
    T, q, ps, lam, tau = to_device(g, "fp64")
    vg = api.VerticalGrid(g.hyai, g.hybi)
    T.requires_grad_(True)
    q.requires_grad_(True)
    lam.requires_grad_(True)
    tau.requires_grad_(True)
    P, H = api.deep_precip_heating(T, q, ps, vg, lam=lam, tau=tau, dt=g.dt)
    a, b = _seeds(n, seed=5)
    ta, tb = torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda")
    loss = (ta * P).sum() + (tb * H).sum()
    loss.backward()
    direct = api.deep_adjoint(T.detach(), q.detach(), ps, vg, gP=ta, gH=tb, dt=g.dt,
                              lam=lam.detach(), tau=tau.detach())
    torch.cuda.synchronize()
    assert torch.equal(T.grad, direct["gT"]) and torch.equal(q.grad, direct["gq"])
    assert torch.equal(lam.grad, direct["glambda"]) and torch.equal(tau.grad, direct["gtau"])
    # forward values are the scheme's precipitation
    d = oracle.deep(g, threads=THREADS)
    np.testing.assert_allclose(P.detach().cpu().numpy(), d["prec"], rtol=1e-10,
                               atol=1e-12 * d["prec"].max())


def test_adjoint_of_empty_and_bad_columns():
    import torch

    from paper_1711_00289_gb300 import api

    g = _grid(8, 16)
    n = g.n_cols
    T, q, ps, lam, tau = to_device(g, "fp64")
    T[:, 3] = 500.0  # outside (100, 400) K: bad input
    vg = api.VerticalGrid(g.hyai, g.hybi)
    ones = torch.ones(n, dtype=torch.float64, device="cuda")
    r = api.deep_adjoint(T, q, ps, vg, gP=ones, gH=ones, dt=g.dt, lam=lam, tau=tau,
                         objective=True)
    torch.cuda.synchronize()
    assert torch.all(r["gT"][:, 3] == 0) and torch.all(r["gq"][:, 3] == 0)
    assert r["P"][3].item() == 0.0 and r["glambda"][3].item() == 0.0
    e = api.deep_adjoint(T, q, ps, vg, gP=ones, gH=ones, dt=g.dt, n_cols=0)
    torch.cuda.synchronize()
    assert e["gT"].shape == (g.pver, n)
    with pytest.raises(Exception):
        api.deep_adjoint(T.float(), q.float(), ps, vg, gP=ones, gH=ones)
