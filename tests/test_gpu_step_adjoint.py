"""Adjoint of the fused deep -> shallow step on the GPU
(conv_deep_shallow_adjoint, FP64) and its torch.autograd.Function: equality
with the oracle's forward-mode tangent of the step, central differences of the
GPU forward step, consistency with the deep-only adjoint, the shallow energy
balance, and autograd backward equal to the direct call."""
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
    """Lat-lon grid (13,824 x 30 at the default size) with per-column CAPE
    relaxation time and entrainment rate."""
    g = S.latlon_grid(nlat, nlon, tau_range=(1800.0, 7200.0))
    g.lam = 5e-4 + 1.5e-3 * S.uniform(20171106, 0, np.arange(g.n_cols), 0)
    return g


def _seeds(n, seed):
    c = np.arange(n)
    return [2.0 * S.uniform(seed, 0, c, j) - 1.0 for j in range(4)]


def _gpu(g, seeds, ld=None, w_heat=None, gradient=True, objective=False, T=None, q=None,
         lam=None, tau=None):
    import torch

    from paper_1711_00289_gb300 import api

    n = g.n_cols
    ld = n if ld is None else ld
    T0, q0, ps, lam0, tau0 = to_device(g, "fp64", ld)
    pad = lambda a: None if a is None else torch.tensor(
        S.to_ld(np.asarray(a, dtype=np.float64), ld), device="cuda")
    r = api.deep_shallow_adjoint(
        T0 if T is None else T, q0 if q is None else q, ps, api.VerticalGrid(g.hyai, g.hybi),
        gPd=pad(seeds[0]), gHd=pad(seeds[1]), gPs=pad(seeds[2]), gHs=pad(seeds[3]),
        w_heat=w_heat, dt=g.dt, lam=lam0 if lam is None else lam,
        tau=tau0 if tau is None else tau, n_cols=n, gradient=gradient, objective=objective)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy()[..., :n] for k, v in r.items()}


def _col_rel(x, y):
    x, y = np.atleast_2d(x), np.atleast_2d(y)
    den = np.abs(y).max(axis=0)
    return np.abs(x - y).max(axis=0) / np.where(den > 0, den, 1.0), den


@pytest.mark.parametrize("which", ["all", "shallow_only"])
def test_gpu_step_adjoint_equals_oracle_tangent(oracle, which):
    g = _grid()
    n = g.n_cols
    seeds = _seeds(n, 13)
    if which == "shallow_only":
        seeds[0] = seeds[1] = None
    got = _gpu(g, seeds, ld=S.pad_ld(n) + 32)
    ref = dict(zip(("gT", "gq", "glambda", "gtau"),
                   oracle.deep_shallow_adjoint(g, *seeds, threads=THREADS)))
    for k in ref:
        rel, den = _col_rel(got[k], ref[k])
        nz = den > 0
        assert nz.sum() > 200
        assert rel[nz].max() <= 1e-10, f"{k}: max column-relative error {rel[nz].max():.3e}"
        assert np.all(np.atleast_2d(got[k])[:, ~nz] == 0.0), f"{k}: non-zero off the schemes"


def test_step_objective_matches_forward(oracle):
    g = _grid(48, 72)
    n = g.n_cols
    got = _gpu(g, [None] * 4, gradient=False, objective=True)["obj"]
    od, os_ = oracle.deep_shallow(g, threads=THREADS)
    pi = g.hyai[:, None] * 1e5 + g.hybi[:, None] * g.ps[None, :]
    pm = 0.5 * (pi[1:] + pi[:-1])
    wm = pm / g.ps[None, :] * (pi[1:] - pi[:-1]) / GRAV
    ref = [od["prec"], CP * (wm * od["dTdt"]).sum(axis=0), os_["prec"],
           CP * (wm * os_["dTdt"]).sum(axis=0)]
    for j in range(4):
        scale = np.abs(ref[j]).max()
        np.testing.assert_allclose(got[j], ref[j], rtol=1e-10, atol=1e-10 * scale)


def test_deep_seeds_equal_deep_adjoint(oracle):
    import torch

    from paper_1711_00289_gb300 import api

    g = _grid(48, 72)
    n = g.n_cols
    gPd, gHd, _, _ = _seeds(n, 17)
    a = _gpu(g, [gPd, gHd, None, None])
    T, q, ps, lam, tau = to_device(g, "fp64")
    b = api.deep_adjoint(T, q, ps, api.VerticalGrid(g.hyai, g.hybi),
                         gP=torch.tensor(gPd, device="cuda"), gH=torch.tensor(gHd, device="cuda"),
                         dt=g.dt, lam=lam, tau=tau)
    torch.cuda.synchronize()
    for k in ("gT", "gq", "glambda", "gtau"):
        rel, den = _col_rel(a[k], b[k].cpu().numpy())
        assert rel[den > 0].max() <= 1e-12, f"{k}: {rel[den > 0].max():.3e}"


def test_shallow_energy_balance_of_gradients(oracle):
    g = _grid(48, 72)
    n = g.n_cols
    w1 = np.ones(g.pver)
    aP = _gpu(g, [None, None, np.ones(n), None], w_heat=w1, objective=True)
    aH = _gpu(g, [None, None, None, np.ones(n)], w_heat=w1)
    rain = aP["obj"][2] > 0
    assert rain.sum() > 20
    np.testing.assert_allclose(aP["obj"][3][rain], LV * aP["obj"][2][rain], rtol=1e-11)
    for k in ("gT", "gq", "glambda", "gtau"):
        rel, den = _col_rel(np.atleast_2d(aH[k])[:, rain], LV * np.atleast_2d(aP[k])[:, rain])
        assert rel.max() <= 1e-10, f"{k}: {rel.max():.3e}"


def test_gpu_step_adjoint_matches_central_differences(oracle):
    """Central differences of the GPU forward step (the step objective of
    conv_deep_shallow_adjoint, checked against the forward kernels above), one
    input at a time over all columns at once, step 1e-6 of each variable's
    scale, on columns where both schemes are active, CAPE is >= 5 J/kg from the
    trigger threshold, the decisions of both schemes (conv_deep_shallow_run
    outputs) are unchanged at +-h and the one-sided differences agree (no hidden
    switch in between).  Bound: 1e-6 relative."""
    import torch

    from paper_1711_00289_gb300 import api

    g = _grid(24, 36)
    n = g.n_cols
    seeds = _seeds(n, 19)
    ad = _gpu(g, seeds)
    T0, q0, ps, lam0, tau0 = to_device(g, "fp64")
    vg = api.VerticalGrid(g.hyai, g.hybi)

    def fwd(T, q, lam, tau):
        r = api.deep_shallow_adjoint(T, q, ps, vg, dt=g.dt, lam=lam, tau=tau, gradient=False,
                                     objective=True)
        od, os_ = api.deep_shallow(T, q, ps, vg, dt=g.dt, precision="fp64", lam=lam, tau=tau,
                                   path="plain")
        torch.cuda.synchronize()
        o = r["obj"].cpu().numpy()
        J = sum(seeds[j] * o[j] for j in range(4))
        dec = np.stack([x[k].cpu().numpy() for x in (od, os_)
                        for k in ("flags", "kb", "klcl", "ktop", "kaux")])
        return J, dec, od, os_

    J0, dec0, od, os_ = fwd(T0, q0, lam0, tau0)
    dflags, sflags = od["flags"].cpu().numpy(), os_["flags"].cpu().numpy()
    ok = ((dflags & 2) > 0) & ((sflags & 2) > 0) & (np.abs(od["cape"].cpu().numpy() - 70) >= 5)
    assert ok.sum() >= 20
    kinked = np.zeros(n, bool)
    fd = {"gT": np.zeros((g.pver, n)), "gq": np.zeros((g.pver, n)), "glambda": np.zeros(n),
          "gtau": np.zeros(n)}
    cmp = {"gT": np.ones((g.pver, n), bool), "gq": g.q > 1e-6, "glambda": np.ones(n, bool),
           "gtau": np.ones(n, bool)}
    for var, k in ([("gT", k) for k in range(g.pver)] + [("gq", k) for k in range(g.pver)]
                   + [("glambda", None), ("gtau", None)]):
        h = {"gT": np.full(n, 3e-4), "glambda": np.full(n, 1e-9),
             "gtau": np.full(n, 3.6e-3)}.get(var)
        if var == "gq":
            h = np.where(cmp["gq"][k], 2e-8, 0.0)
        ht = torch.tensor(h, device="cuda")
        res = []
        for sgn in (1.0, -1.0):
            T, q, lam, tau = T0.clone(), q0.clone(), lam0.clone(), tau0.clone()
            {"gT": lambda: T[k].add_(sgn * ht), "gq": lambda: q[k].add_(sgn * ht),
             "glambda": lambda: lam.add_(sgn * ht), "gtau": lambda: tau.add_(sgn * ht)}[var]()
            J, dec, _, _ = fwd(T, q, lam, tau)
            ok &= np.all(dec == dec0, axis=0)
            res.append(J)
        hs = np.where(h > 0, h, 1.0)
        f, b = (res[0] - J0) / hs, (J0 - res[1]) / hs
        scale = np.maximum(np.abs(np.atleast_2d(ad[var])).max(axis=0), 1e-300)
        kinked |= (np.abs(f - b) > 1e-3 * scale) & (h > 0)
        c = (res[0] - res[1]) / (2 * hs)
        if k is None:
            fd[var] = c
        else:
            fd[var][k] = c
    use = ok & ~kinked
    assert use.sum() >= 0.7 * ok.sum() and use.sum() >= 15, (use.sum(), ok.sum())
    xs = {"gT": 300.0, "gq": 0.02, "glambda": 1e-3, "gtau": 3600.0}
    for var in fd:
        a = np.atleast_2d(np.asarray(ad[var]))
        den = np.maximum(np.abs(a).max(axis=0), np.abs(J0) / xs[var])
        err = np.where(np.atleast_2d(cmp[var]), np.abs(np.atleast_2d(fd[var]) - a), 0.0)
        rel = err.max(axis=0)[use] / den[use]
        assert rel.max() <= 1e-6, f"{var}: central difference vs adjoint {rel.max():.3e}"


def test_step_autograd_backward_equals_direct_call(oracle):
    import torch

    from paper_1711_00289_gb300 import api

    g = _grid(24, 36)
    n = g.n_cols
    T, q, ps, lam, tau = to_device(g, "fp64")
    vg = api.VerticalGrid(g.hyai, g.hybi)
    for t in (T, q, lam, tau):
        t.requires_grad_(True)
    outs = api.deep_shallow_step(T, q, ps, vg, lam=lam, tau=tau, dt=g.dt)
    seeds = [torch.tensor(s, device="cuda") for s in _seeds(n, 23)]
    loss = sum((s * o).sum() for s, o in zip(seeds, outs))
    loss.backward()
    direct = api.deep_shallow_adjoint(T.detach(), q.detach(), ps, vg, gPd=seeds[0],
                                      gHd=seeds[1], gPs=seeds[2], gHs=seeds[3], dt=g.dt,
                                      lam=lam.detach(), tau=tau.detach())
    torch.cuda.synchronize()
    assert torch.equal(T.grad, direct["gT"]) and torch.equal(q.grad, direct["gq"])
    assert torch.equal(lam.grad, direct["glambda"]) and torch.equal(tau.grad, direct["gtau"])
