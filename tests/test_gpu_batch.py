"""Batched ensembles (members of uneven column and level counts in one trigger
launch and one persistent plume launch): per-member equality with unbatched
runs, FP64 parity with the oracle, CUDA-graph capture and the autotuner."""
import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S
from tests.gpu_util import THREADS, assert_fp64_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _members(precision, n_members=8, seed=42):
    import torch

    from paper_1711_00289_gb300 import api

    ens = S.ensemble(n_members, seed=seed, n_min=1, n_max=6000)
    ens.append(S.column_set(0, pver=30))  # an empty member
    ens.append(S.column_set(1, seed=3, pver=26))
    rd = api.real_dtype(precision)
    mem = []
    for g in ens:
        ld = S.pad_ld(max(g.n_cols, 1))
        mem.append(dict(T=torch.tensor(S.to_ld(g.T, ld), device="cuda").to(rd),
                        q=torch.tensor(S.to_ld(g.q, ld), device="cuda").to(rd),
                        ps=torch.tensor(np.where(np.arange(ld) < g.n_cols, S.to_ld(g.ps, ld), 1e5),
                                        device="cuda"),
                        lam=(None if g.lam is None else
                             torch.tensor(S.to_ld(g.lam, ld), device="cuda")),
                        vgrid=api.VerticalGrid(g.hyai, g.hybi), n_cols=g.n_cols, dt=g.dt))
    return ens, mem


def _host(o, n):
    return {k: (v[:, :n] if v.dim() == 2 else v[:n]).double().cpu().numpy()
            if v.dtype != __import__("torch").int32 else
            (v[:, :n] if v.dim() == 2 else v[:n]).cpu().numpy() for k, v in o.items()}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_unbatched_runs(precision):
    import torch

    from paper_1711_00289_gb300 import api

    ens, mem = _members(precision)
    b = api.Batch(mem, precision)
    b.set_config("thread", 128, 128)  # the single-grid runs' mapping (see below)
    outs = b.run()
    torch.cuda.synchronize()
    for g, m, (od, os_) in zip(ens, mem, outs):
        n = g.n_cols
        if n == 0:
            continue
        rd, rs = api.deep_shallow(m["T"], m["q"], m["ps"], m["vgrid"], dt=g.dt,
                                  precision=precision, lam=m["lam"], path="compact", n_cols=n)
        torch.cuda.synchronize()
        for got, want in ((od, rd), (os_, rs)):
            a, w = _host(got, n), _host(want, n)
            for k in a:
                assert np.array_equal(a[k], w[k]), (g.name, k)
    b.close()


def test_batch_fp64_matches_oracle(oracle):
    import torch

    from paper_1711_00289_gb300 import api

    ens, mem = _members("fp64", seed=7)
    b = api.Batch(mem, "fp64")
    outs = b.run()
    torch.cuda.synchronize()
    for g, (od, os_) in zip(ens, outs):
        if g.n_cols == 0:
            continue
        rd, rs = oracle.deep_shallow(g, threads=THREADS)
        assert_fp64_parity(_host(od, g.n_cols), rd, what=f"deep {g.name} pver={g.pver}")
        assert_fp64_parity(_host(os_, g.n_cols), rs, what=f"shallow {g.name}")
    b.close()


def test_batch_graph_capture_and_autotune():
    import torch

    from paper_1711_00289_gb300 import api

    ens, mem = _members("mixed", seed=11)
    b = api.Batch(mem, "mixed")
    before = [tuple(_host(o, g.n_cols) for o in pair) for g, pair in zip(ens, b.run())]
    torch.cuda.synchronize()
    cfg = b.autotune(reps=2)
    assert cfg["trigger_block"] in (64, 128, 256) and cfg["plume_block"] in (64, 128, 256)
    assert cfg["plume_grid"] > 0
    ref = [tuple(_host(o, g.n_cols) for o in pair) for g, pair in zip(ens, b.run())]
    torch.cuda.synchronize()
    if cfg["trigger_mapping"] == "thread":
        # block shapes and the plume pass's slot order change no column's arithmetic
        # (the warp mapping sums CAPE in another order, so it is compared only to itself)
        for g, got, want in zip(ens, ref, before):
            for o, w in zip(got, want):
                for k in o:
                    assert np.array_equal(o[k], w[k]), (g.name, k, cfg)
    b.ws.get(b.workspace_bytes())  # workspace exists before capture
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    for pair in b.outputs:  # the replay must rewrite every output
        for o in pair:
            for v in o.values():
                v.fill_(-5)
    with torch.cuda.graph(graph, stream=s):
        b.run(stream=s)
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    for g, pair, want in zip(ens, b.outputs, ref):
        for o, w in zip(pair, want):
            h = _host(o, g.n_cols)
            for k in h:
                assert np.array_equal(h[k], w[k]), (g.name, k, cfg)
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_members_with_their_own_parameters(precision):
    """Each member's own deep and shallow parameters, time step and relaxation
    times reach its columns: every member equals its unbatched run."""
    import torch

    from paper_1711_00289_gb300 import _lib as L
    from paper_1711_00289_gb300 import api

    ens, mem = _members(precision, n_members=6, seed=7)
    settings = []
    for j, (g, m) in enumerate(zip(ens, mem)):
        dp, sp = L.deep_defaults(), L.shallow_defaults()
        dp.capelmt = 30.0 + 20.0 * (j % 4)
        dp.c0 = 1e-3 * (1 + j % 3)
        dp.alpha_dd = 0.1 + 0.1 * (j % 3)
        sp.c_m = 0.02 + 0.01 * (j % 3)
        sp.cin_max = 30.0 + 15.0 * (j % 4)
        m["deep_params"], m["shallow_params"] = dp, sp
        m["dt"] = 900.0 * (1 + j % 3)
        ld = m["T"].shape[1]
        tau = 1800.0 + 600.0 * (np.arange(ld) % 7) + 100.0 * j
        m["tau"] = torch.tensor(tau, device="cuda")
        settings.append((dp, sp))
    b = api.Batch(mem, precision)
    # the single-grid runs below take one column per thread; a plan made after
    # another batch's autotune may have inherited the warp mapping, which sums
    # CAPE in another order (mixed results then agree only to rounding)
    b.set_config("thread", 128, 128)
    outs = b.run()
    torch.cuda.synchronize()
    checked = 0
    for g, m, (od, os_) in zip(ens, mem, outs):
        n = g.n_cols
        if n == 0:
            continue
        rd, rs = api.deep_shallow(m["T"], m["q"], m["ps"], m["vgrid"], dt=m["dt"],
                                  precision=precision, lam=m["lam"], tau=m["tau"],
                                  deep_params=m["deep_params"],
                                  shallow_params=m["shallow_params"], path="compact", n_cols=n)
        torch.cuda.synchronize()
        for got, want in ((od, rd), (os_, rs)):
            a, w = _host(got, n), _host(want, n)
            for k in a:
                assert np.array_equal(a[k], w[k]), (g.name, k)
        checked += n
    assert checked > 1000
    b.close()
