"""Convective momentum transport on the GPU (conv_momentum_transport) against
the FP64 oracle, through the C ABI.

Tolerances are relative to each column's natural scale of the transport terms,
max_k |u| * max_k (mu + du + md) / m_k: FP64 1e-10 (FP64 throughout, a different
formulation of the same fluxes: the kernel writes the tracer budget minus the
pressure forces on the mass-flux profiles, the oracle the divergence of the
interface eddy fluxes), mixed 1e-3 on columns whose decisions agree (the
plume's M_b carries the mixed closure's error), 1e-5 for the FP32 kernel fed the
oracle's own profiles.  Column momentum must be conserved and a uniform wind
left unchanged; with both coefficients 0 the kernel is the tracer kernel."""
import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S
from tests.gpu_util import THREADS, layer_mass, same_decisions, to_device

pytestmark = pytest.mark.gpu

FLUX = ("mu", "du", "md")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _wind(g, ld, seed=9):
    """A sheared wind with random structure, [2][pver][ld]."""
    n = g.n_cols
    c = np.arange(n)
    k = np.arange(g.pver)[:, None]
    noise = np.stack([np.stack([S.uniform(seed, 2 * kk + j, c, 0) for kk in range(g.pver)])
                      for j in range(2)])
    base = np.stack([10.0 + 20.0 * (1 - k / g.pver) + 0 * c,
                     -5.0 + 8.0 * np.sin(k / 4.0) + 0 * c])
    uv = base + 6.0 * (noise - 0.5)
    return np.stack([S.to_ld(w, ld) for w in uv])


def _scale(uv, flux, g):
    m = layer_mass(g)
    rate = ((flux["mu"] + flux["du"] + flux["md"]) / m).max(axis=0)
    return np.abs(uv).max(axis=1) * rate[None, :] + 1e-300


def _gpu(g, precision, path, ld, uv_np, cu, cd):
    import torch

    from paper_1711_00289_gb300 import api

    n = g.n_cols
    T, q, ps, lam, tau = to_device(g, precision, ld)
    vg = api.VerticalGrid(g.hyai, g.hybi)
    rd = api.real_dtype(precision)
    od = api.new_outputs(g.pver, ld, precision, flux=True)
    os_ = api.new_outputs(g.pver, ld, precision, flux=True)
    api.deep_shallow(T, q, ps, vg, dt=g.dt, precision=precision, lam=lam, tau=tau, path=path,
                     n_cols=n, out_deep=od, out_shallow=os_)
    uv = torch.tensor(uv_np, device="cuda").to(rd).contiguous()
    td, ts = api.momentum_transport(uv, ps, vg, deep_out=od, shallow_out=os_, dt=g.dt,
                                    precision=precision, cp_up=cu, cp_down=cd, n_cols=n)
    torch.cuda.synchronize()

    def cut(v):
        h = v[..., :n].cpu().numpy()
        return h.astype(np.float64) if h.dtype == np.float32 else h

    return ({k: cut(v) for k, v in od.items()}, {k: cut(v) for k, v in os_.items()}, cut(td),
            cut(ts))


@pytest.mark.parametrize("path,cu,cd", [("plain", 0.7, 0.7), ("compact", 0.7, 0.7),
                                        ("compact", 0.2, 1.0), ("compact", 1.0, 0.0)])
def test_fp64_matches_oracle(oracle, path, cu, cd):
    g = S.clustered_grid(0.3, 96, 144)
    n = g.n_cols
    ld = S.pad_ld(n) + 32
    uv = _wind(g, ld)
    gd, gs, td, ts = _gpu(g, "fp64", path, ld, uv, cu, cd)
    rtd, rts = oracle.deep_shallow_momentum(g, uv[:, :, :n], cu, cd, threads=THREADS)
    _, _, rfd, rfs = oracle.deep_shallow_tracers(g, np.ones((1, g.pver, n)), threads=THREADS)
    assert (rfd["mu"] > 0).any(axis=0).sum() > 500 and (rfs["mu"] > 0).any(axis=0).sum() > 200
    for got, ref, f, tag in ((td, rtd, rfd, "deep"), (ts, rts, rfs, "shallow")):
        err = np.abs(got - ref).max(axis=1) / _scale(uv[:, :, :n], f, g)
        assert err.max() <= 1e-10, f"{tag}: {err.max():.3g}"
        inactive = (f["mu"] == 0).all(axis=0)
        assert np.all(got[:, :, inactive] == 0.0)


def test_zero_coefficients_are_the_tracer_kernel():
    import torch

    from paper_1711_00289_gb300 import api

    g = S.clustered_grid(0.3, 96, 144)
    n = g.n_cols
    T, q, ps, lam, tau = to_device(g, "mixed")
    vg = api.VerticalGrid(g.hyai, g.hybi)
    od = api.new_outputs(g.pver, n, "mixed", flux=True)
    api.deep_shallow(T, q, ps, vg, dt=g.dt, precision="mixed", out_deep=od,
                     out_shallow=api.new_outputs(g.pver, n, "mixed", flux=True))
    uv = torch.tensor(np.abs(_wind(g, n)) + 1.0, device="cuda").float()
    md, _ = api.momentum_transport(uv, ps, vg, deep_out=od, precision="mixed", cp_up=0.0,
                                   cp_down=0.0)
    tdr, _ = api.tracer_transport(uv, ps, vg, deep_out=od, precision="mixed")
    torch.cuda.synchronize()
    assert bool((md != 0).any())
    # the same FP32 arithmetic in two instantiations (2 and 4 tracers per thread):
    # equal up to the compiler's different fusing of multiply-adds
    scale = float(md.abs().max())
    assert float((md - tdr).abs().max()) <= 1e-6 * scale


def test_mixed_within_budget(oracle):
    g = S.clustered_grid(0.3, 96, 144)
    n = g.n_cols
    uv = _wind(g, n)
    gd, gs, td, ts = _gpu(g, "mixed", "compact", n, uv, 0.7, 0.7)
    rtd, rts = oracle.deep_shallow_momentum(g, uv, 0.7, 0.7, threads=THREADS)
    _, _, rfd, rfs = oracle.deep_shallow_tracers(g, np.ones((1, g.pver, n)), threads=THREADS)
    rd, rs = oracle.deep_shallow(g, threads=THREADS)
    sd = same_decisions(gd, rd)
    ss = sd & same_decisions(gs, rs)
    assert (~sd).sum() <= 1e-3 * n and (~ss).sum() <= 2e-3 * n
    for got, ref, f, same, tag in ((td, rtd, rfd, sd, "deep"), (ts, rts, rfs, ss, "shallow")):
        err = (np.abs(got - ref).max(axis=1) / _scale(uv, f, g))[:, same]
        assert err.max() <= 1e-3, f"{tag}: {err.max():.3g}"


def test_fp32_kernel_on_oracle_profiles(oracle):
    """The kernel alone: FP32 arithmetic on the oracle's decisions and mass-flux
    profiles against the oracle's FP64 momentum transport, stage by stage."""
    import torch

    from paper_1711_00289_gb300 import api

    g = S.clustered_grid(0.3, 96, 144)
    n = g.n_cols
    uv = _wind(g, n)
    cu, cd = 0.6, 0.8
    rtd, rts = oracle.deep_shallow_momentum(g, uv, cu, cd, threads=THREADS)
    _, _, rfd, rfs = oracle.deep_shallow_tracers(g, np.ones((1, g.pver, n)), threads=THREADS)
    rd, rs = oracle.deep_shallow(g, threads=THREADS)
    outs = []
    for r, f in ((rd, rfd), (rs, rfs)):
        o = {k: torch.tensor(r[k], device="cuda") for k in ("flags", "kb", "ktop", "kaux")}
        o.update({k: torch.tensor(f[k], device="cuda").float() for k in FLUX})
        o["dTdt"] = o["dqdt"] = torch.zeros((g.pver, n), device="cuda")
        outs.append(o)
    ps = torch.tensor(g.ps, device="cuda")
    vg = api.VerticalGrid(g.hyai, g.hybi)
    uv2 = uv + g.dt * rtd  # the shallow stage sees the deep-updated wind
    td, _ = api.momentum_transport(torch.tensor(uv, device="cuda").float(), ps, vg,
                                   deep_out=outs[0], precision="mixed", cp_up=cu, cp_down=cd)
    _, ts = api.momentum_transport(torch.tensor(uv2, device="cuda").float(), ps, vg,
                                   shallow_out=outs[1], precision="mixed", cp_up=cu, cp_down=cd)
    torch.cuda.synchronize()
    for got, ref, f, c, tag in ((td, rtd, rfd, uv, "deep"), (ts, rts, rfs, uv2, "shallow")):
        err = np.abs(got.double().cpu().numpy() - ref).max(axis=1) / _scale(c, f, g)
        assert err.max() <= 1e-5, f"{tag}: {err.max():.3g}"


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_resolution(oracle, precision):
    """884,736 columns x 30 levels, the benchmark's launch configuration: every
    column against the oracle (FP64 1e-10 of the natural scale; mixed 1e-3 where
    decisions agree), column momentum conserved, a uniform wind unchanged,
    inactive columns exact zeros."""
    import torch

    from paper_1711_00289_gb300 import api

    g = S.clustered_grid(0.3)
    n = g.n_cols
    uv_np = _wind(g, n)
    gd, gs, td, ts = _gpu(g, precision, "compact", n, uv_np, 0.7, 0.7)
    m = layer_mass(g)
    rtd, rts = oracle.deep_shallow_momentum(g, uv_np, 0.7, 0.7, threads=THREADS)
    _, _, rfd, rfs = oracle.deep_shallow_tracers(g, np.ones((1, g.pver, n)), threads=THREADS)
    rd, rs = oracle.deep_shallow(g, threads=THREADS)
    if precision == "fp64":
        same_d = np.ones(n, bool)
        same_s = same_d
        tol = 1e-10
    else:
        same_d = same_decisions(gd, rd)
        same_s = same_d & same_decisions(gs, rs)
        assert (~same_s).sum() <= 2e-3 * n
        tol = 1e-3
    for got, ref, f, o, same, tag in ((td, rtd, rfd, gd, same_d, "deep"),
                                      (ts, rts, rfs, gs, same_s, "shallow")):
        act = (o["flags"] & 2) > 0
        assert act.sum() > 10000
        err = np.abs(got - ref).max(axis=1) / _scale(uv_np, f, g)
        assert err[:, same].max() <= tol, f"{tag}: {err[:, same].max():.3g}"
        net = np.abs((m[None] * got).sum(axis=1))
        tot = (m[None] * np.abs(got)).sum(axis=1) + 1e-300
        assert (net / tot)[:, act].max() <= (1e-12 if precision == "fp64" else 1e-4), tag
        assert np.all(got[:, :, ~act] == 0.0), tag
    # a uniform wind: zero up to the rounding of the plumes' weighted means
    uni = np.ones((2, g.pver, n)) * np.array([7.0, -3.0])[:, None, None]
    _, _, tu, su = _gpu(g, precision, "compact", n, uni, 0.7, 0.7)
    for t, o in ((tu, gd), (su, gs)):
        rate = ((o["mu"] + o["du"] + o["md"]) / m).max(axis=0)
        bound = (1e-13 if precision == "fp64" else 1e-5) * 7.0 * rate
        assert np.all(np.abs(t) <= bound[None, None, :])
    _ = torch


def test_argument_checks():
    import torch

    from paper_1711_00289_gb300 import _lib as L
    from paper_1711_00289_gb300 import api

    g = S.clustered_grid(0.5, 4, 5)
    n = g.n_cols
    T, q, ps, _, _ = to_device(g, "fp64")
    vg = api.VerticalGrid(g.hyai, g.hybi)
    od = api.new_outputs(g.pver, n, "fp64", flux=True)
    api.deep_shallow(T, q, ps, vg, dt=g.dt, precision="fp64", out_deep=od,
                     out_shallow=api.new_outputs(g.pver, n, "fp64", flux=True))
    uv = torch.zeros((2, g.pver, n), dtype=torch.float64, device="cuda")
    for cu, cd in ((-0.1, 0.5), (0.5, 1.5), (float("nan"), 0.5)):
        with pytest.raises(L.ConvError):
            api.momentum_transport(uv, ps, vg, deep_out=od, cp_up=cu, cp_down=cd)
    with pytest.raises(TypeError):
        api.momentum_transport(uv[:1].contiguous(), ps, vg, deep_out=od)
