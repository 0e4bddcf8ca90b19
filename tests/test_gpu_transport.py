"""Convective tracer transport on the GPU (conv_tracer_transport) and the
mass-flux profiles the scheme kernels write, against the FP64 oracle.

Tolerances are relative to each column's natural scale of the transport terms,
max_k |c| * max_k (mu + du + md) / m_k (the largest flux difference a layer can
see): FP64 1e-10 (FP64 throughout, different rounding order), mixed 1e-3 on
columns whose decisions agree (the plume's M_b carries the mixed path's
closure error), and 1e-5 for the FP32 kernel fed the oracle's own profiles (FP32
recurrences over at most 32 levels)."""
import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S
from tests.gpu_util import THREADS, assert_fp64_parity, layer_mass, same_decisions, to_device

pytestmark = pytest.mark.gpu

FLUX = ("mu", "du", "md")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _tracers(g, ld, seed=5):
    """Four tracers: O(1) uniform noise, a 1e-9 trace gas with a vertical
    gradient, humidity itself, and a layer of 1 between 2 and 4 km high."""
    n = g.n_cols
    c = np.arange(n)
    u = np.stack([S.uniform(seed, k, c, 0) for k in range(g.pver)])
    grad = 1e-9 * (1.0 + np.linspace(0.0, 2.0, g.pver))[:, None] * (0.5 + u)
    lay = np.zeros((g.pver, n))
    lay[g.pver // 3: g.pver // 2] = 1.0
    tr = np.stack([u, grad, g.q, lay])
    return np.stack([S.to_ld(t, ld) for t in tr])


def _scale(tr, flux, g):
    m = layer_mass(g)
    rate = ((flux["mu"] + flux["du"] + flux["md"]) / m).max(axis=0)
    return np.abs(tr).max(axis=1) * rate[None, :] + 1e-300


def _gpu_step(g, precision, path, ld, tr_np):
    import torch

    from paper_1711_00289_gb300 import api

    n = g.n_cols
    T, q, ps, lam, tau = to_device(g, precision, ld)
    vg = api.VerticalGrid(g.hyai, g.hybi)
    rd = api.real_dtype(precision)
    tr = torch.tensor(tr_np, device="cuda").to(rd).contiguous()
    od, os_, td, ts = api.deep_shallow_tracers(T, q, ps, tr, vg, dt=g.dt, precision=precision,
                                              lam=lam, tau=tau, path=path, n_cols=n)
    torch.cuda.synchronize()

    def cut(v):
        h = v[..., :n].cpu().numpy()
        return h.astype(np.float64) if h.dtype == np.float32 else h

    host = [{k: cut(v) for k, v in o.items()} for o in (od, os_)]
    return host[0], host[1], cut(td), cut(ts), (td, ts, tr, od, os_)


def _flux_err(got, ref):
    den = np.maximum(np.abs(ref["mu"]).max(axis=0), 1e-300)
    return max(float((np.abs(got[k] - ref[k]).max(axis=0) / den).max()) for k in FLUX)


@pytest.mark.parametrize("path", ["plain", "compact"])
def test_fp64_profiles_and_tendencies_match_oracle(oracle, path):
    g = S.clustered_grid(0.3, 96, 144)
    n = g.n_cols
    ld = S.pad_ld(n) + 32
    tr = _tracers(g, ld)
    gd, gs, td, ts, _ = _gpu_step(g, "fp64", path, ld, tr)
    rtd, rts, rfd, rfs = oracle.deep_shallow_tracers(g, tr[:, :, :n], threads=THREADS)
    rd, rs = oracle.deep_shallow(g, threads=THREADS)
    assert_fp64_parity(gd, rd, what=f"deep {path}")
    assert_fp64_parity(gs, rs, what=f"shallow {path}")
    assert ((rd["flags"] & 2) > 0).sum() > 500 and ((rs["flags"] & 2) > 0).sum() > 200
    assert _flux_err(gd, rfd) <= 1e-12 and _flux_err(gs, rfs) <= 1e-12
    for got, ref, f, tag in ((td, rtd, rfd, "deep"), (ts, rts, rfs, "shallow")):
        err = np.abs(got - ref).max(axis=1) / _scale(tr[:, :, :n], f, g)
        assert err.max() <= 1e-10, f"{tag}: {err.max():.3g}"
        inactive = (f["mu"] == 0).all(axis=0)
        assert np.all(got[:, :, inactive] == 0.0)


def test_mixed_tendencies_within_budget(oracle):
    g = S.clustered_grid(0.3, 96, 144)
    n = g.n_cols
    tr = _tracers(g, n)
    gd, gs, td, ts, _ = _gpu_step(g, "mixed", "compact", n, tr)
    rtd, rts, rfd, rfs = oracle.deep_shallow_tracers(g, tr, threads=THREADS)
    rd, rs = oracle.deep_shallow(g, threads=THREADS)
    sd = same_decisions(gd, rd)
    ss = sd & same_decisions(gs, rs)
    assert (~sd).sum() <= 1e-3 * n and (~ss).sum() <= 2e-3 * n
    for got, ref, gf, f, same, tag in ((td, rtd, gd, rfd, sd, "deep"),
                                       (ts, rts, gs, rfs, ss, "shallow")):
        err = (np.abs(got - ref).max(axis=1) / _scale(tr, f, g))[:, same]
        assert err.max() <= 1e-3, f"{tag}: {err.max():.3g}"
        den = np.maximum(np.abs(f["mu"]).max(axis=0), 1e-300)
        for k in FLUX:
            ferr = (np.abs(gf[k] - f[k]).max(axis=0) / den)[same].max()
            assert ferr <= 1e-3, f"{tag} {k}: {ferr:.3g}"


def test_fp32_kernel_on_oracle_profiles(oracle):
    """The transport kernel alone: FP32 arithmetic on the oracle's decisions and
    mass-flux profiles against the oracle's FP64 transport."""
    import torch

    from paper_1711_00289_gb300 import api

    g = S.clustered_grid(0.3, 96, 144)
    n = g.n_cols
    tr = _tracers(g, n)
    rtd, rts, rfd, rfs = oracle.deep_shallow_tracers(g, tr, threads=THREADS)
    rd, rs = oracle.deep_shallow(g, threads=THREADS)
    outs = []
    for r, f in ((rd, rfd), (rs, rfs)):
        o = {k: torch.tensor(r[k], device="cuda") for k in ("flags", "kb", "ktop", "kaux")}
        o.update({k: torch.tensor(f[k], device="cuda").float() for k in FLUX})
        o["dTdt"] = o["dqdt"] = torch.zeros((g.pver, n), device="cuda")
        outs.append(o)
    ps = torch.tensor(g.ps, device="cuda")
    # deep and shallow stages separately: each against the oracle's stage on the
    # same input (the shallow stage gets the oracle's deep-updated tracer)
    trd = torch.tensor(tr, device="cuda").float()
    tr2 = np.maximum(tr + g.dt * rtd, 0.0)
    tr2d = torch.tensor(tr2, device="cuda").float()
    vg = api.VerticalGrid(g.hyai, g.hybi)
    td, _ = api.tracer_transport(trd, ps, vg, deep_out=outs[0], precision="mixed")
    _, ts = api.tracer_transport(tr2d, ps, vg, shallow_out=outs[1], precision="mixed")
    torch.cuda.synchronize()
    for got, ref, f, c, tag in ((td, rtd, rfd, tr, "deep"), (ts, rts, rfs, tr2, "shallow")):
        err = np.abs(got.double().cpu().numpy() - ref).max(axis=1) / _scale(c, f, g)
        assert err.max() <= 1e-5, f"{tag}: {err.max():.3g}"


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_profile_outputs_leave_the_step_unchanged(precision):
    """Writing the mass-flux profiles selects separate kernel instantiations;
    the step's own outputs stay the same (FP64: to rounding; mixed: decisions
    identical in all but a handful of columns, real outputs to FP32 rounding)."""
    from tests.gpu_util import run_gpu

    import torch

    from paper_1711_00289_gb300 import api

    g = S.clustered_grid(0.3, 96, 144)
    n = g.n_cols
    a = run_gpu(g, precision, "compact")
    T, q, ps, lam, tau = to_device(g, precision)
    vg = api.VerticalGrid(g.hyai, g.hybi)
    od = api.new_outputs(g.pver, n, precision, flux=True)
    os_ = api.new_outputs(g.pver, n, precision, flux=True)
    api.deep_shallow(T, q, ps, vg, dt=g.dt, precision=precision, lam=lam, tau=tau,
                     path="compact", out_deep=od, out_shallow=os_)
    torch.cuda.synchronize()
    b = [{k: (v.cpu().numpy().astype(np.float64) if v.dtype == torch.float32 else
              v.cpu().numpy()) for k, v in o.items()} for o in (od, os_)]
    for x, y, tag in zip(b, a, ("deep", "shallow")):
        if precision == "fp64":
            assert_fp64_parity(x, y, tol=1e-12, what=tag)
        else:
            same = same_decisions(x, y)
            assert (~same).sum() <= 5, tag
            for k in ("dTdt", "dqdt"):
                den = np.maximum(np.abs(y[k]).max(axis=0), 1e-30)
                assert (np.abs(x[k] - y[k]).max(axis=0) / den)[same].max() <= 1e-5


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_resolution_against_oracle(oracle, precision):
    """884,736 columns x 30 levels, the launch configuration of the benchmark
    (compacted step, then one transport launch), 2 tracers: every column against
    the oracle (FP64: within 1e-10 of the natural scale; mixed: 1e-3 on columns
    whose decisions agree), plus the exact properties -- a uniform tracer stays
    unchanged, tracer mass is conserved, inactive columns get exact zeros."""
    import torch

    from paper_1711_00289_gb300 import api

    g = S.clustered_grid(0.3)
    n = g.n_cols
    T, q, ps, lam, tau = to_device(g, precision)
    vg = api.VerticalGrid(g.hyai, g.hybi)
    rd = api.real_dtype(precision)
    tr_np = np.stack([np.ones((g.pver, n)), g.q])
    tr = torch.tensor(tr_np, device="cuda").to(rd)
    od, os_, td, ts = api.deep_shallow_tracers(T, q, ps, tr, vg, dt=g.dt, precision=precision,
                                              lam=lam, tau=tau)
    torch.cuda.synchronize()
    m = torch.tensor(layer_mass(g), device="cuda")
    for o, t, tag in ((od, td, "deep"), (os_, ts, "shallow")):
        act = (o["flags"] & 2) > 0
        assert int(act.sum()) > 10000
        rate = ((o["mu"] + o["du"] + o["md"]).double() / m).amax(dim=0)
        uni = float((t[0].double().abs().amax(dim=0) / (rate + 1e-300))[act].max())
        assert uni <= (1e-13 if precision == "fp64" else 1e-5), (tag, uni)
        net = (m * t[1].double()).sum(dim=0).abs()
        tot = (m * t[1].double().abs()).sum(dim=0) + 1e-300
        assert float((net / tot)[act].max()) <= (1e-12 if precision == "fp64" else 1e-4), tag
        assert bool((t[:, :, ~act] == 0).all()), tag
    rtd, rts, rfd, rfs = oracle.deep_shallow_tracers(g, tr_np, threads=THREADS)
    gd = {k: v.cpu().numpy() for k, v in od.items()}
    gs = {k: v.cpu().numpy() for k, v in os_.items()}
    rdo, rso = oracle.deep_shallow(g, threads=THREADS)
    if precision == "fp64":
        same_d = np.ones(n, bool)
        same_s = same_d
        for k in ("flags", "kb", "ktop", "kaux"):
            assert np.array_equal(gd[k], rdo[k]) and np.array_equal(gs[k], rso[k]), k
        tol = 1e-10
    else:
        same_d = same_decisions(gd, rdo)
        same_s = same_d & same_decisions(gs, rso)
        assert (~same_s).sum() <= 2e-3 * n
        tol = 1e-3
    for got, ref, f, same, tag in ((td, rtd, rfd, same_d, "deep"),
                                   (ts, rts, rfs, same_s, "shallow")):
        err = (np.abs(got.double().cpu().numpy() - ref).max(axis=1) / _scale(tr_np, f, g))
        assert err[:, same].max() <= tol, f"{tag}: {err[:, same].max():.3g}"


@pytest.mark.parametrize("pver", [8, 32])
def test_other_level_counts(oracle, pver):
    """Fewest and most levels the library takes a tile of (32 = the maximum)."""
    g = S.clustered_grid(0.4, 24, 36, pver=pver)
    n = g.n_cols
    tr = _tracers(g, n)
    gd, gs, td, ts, _ = _gpu_step(g, "fp64", "compact", n, tr)
    rtd, rts, rfd, rfs = oracle.deep_shallow_tracers(g, tr, threads=THREADS)
    for got, ref, f, tag in ((td, rtd, rfd, "deep"), (ts, rts, rfs, "shallow")):
        err = np.abs(got - ref).max(axis=1) / _scale(tr, f, g)
        assert err.max() <= 1e-10, f"{tag} pver={pver}: {err.max():.3g}"


def test_edge_cases(oracle):
    """No tracers (no launch), one scheme at a time, ragged tails with padding
    left untouched, and a single column."""
    import torch

    from paper_1711_00289_gb300 import api

    g = S.clustered_grid(0.5, 4, 5)  # 20 columns
    n = g.n_cols
    ld = n + 13
    T, q, ps, lam, tau = to_device(g, "fp64", ld)
    vg = api.VerticalGrid(g.hyai, g.hybi)
    od = api.new_outputs(g.pver, ld, "fp64", flux=True)
    os_ = api.new_outputs(g.pver, ld, "fp64", flux=True)
    api.deep_shallow(T, q, ps, vg, dt=g.dt, precision="fp64", lam=lam, tau=tau, n_cols=n,
                     out_deep=od, out_shallow=os_)
    empty = torch.empty((0, g.pver, ld), dtype=torch.float64, device="cuda")
    td, ts = api.tracer_transport(empty, ps, vg, deep_out=od, shallow_out=os_, n_cols=n)
    assert td.numel() == 0 and ts.numel() == 0
    tr = torch.tensor(_tracers(g, ld), device="cuda")
    sent = torch.full_like(tr, -7.0)
    td, _ = api.tracer_transport(tr, ps, vg, deep_out=od, n_cols=n, tend_deep=sent.clone())
    _, ts = api.tracer_transport(tr, ps, vg, shallow_out=os_, n_cols=n, tend_shallow=sent.clone())
    torch.cuda.synchronize()
    assert bool((td[:, :, n:] == -7.0).all()) and bool((ts[:, :, n:] == -7.0).all())
    both_d, both_s = api.tracer_transport(tr, ps, vg, deep_out=od, shallow_out=os_, n_cols=n)
    # the deep stage does not depend on the shallow one
    assert torch.equal(both_d[:, :, :n], td[:, :, :n])
    # deep only against the oracle's deep stage
    rtd, _, rfd, _ = oracle.deep_shallow_tracers(g, tr[:, :, :n].cpu().numpy(), threads=1)
    err = np.abs(td[:, :, :n].cpu().numpy() - rtd).max(axis=1) / _scale(
        tr[:, :, :n].cpu().numpy(), rfd, g)
    assert err.max() <= 1e-10
    # one column
    g1 = S.clustered_grid(1.0, 1, 1)
    gd, gs, td1, ts1, _ = _gpu_step(g1, "fp64", "compact", 1, _tracers(g1, 1))
    r1d, r1s, _, _ = oracle.deep_shallow_tracers(g1, _tracers(g1, 1), threads=1)
    assert np.allclose(td1, r1d, rtol=1e-10, atol=1e-25)
    assert np.allclose(ts1, r1s, rtol=1e-10, atol=1e-25)
