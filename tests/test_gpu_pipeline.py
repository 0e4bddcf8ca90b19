"""The host pipeline (conv_pipeline_*): chunked, overlapped runs on host buffers
give bit-identical results to one device-resident conv_deep_shallow_run, for
both precisions, a ragged last chunk and a padded leading dimension."""
import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_pipeline_equals_device_run(precision):
    import torch

    from paper_1711_00289_gb300 import api

    g = S.clustered_grid(0.3, 96, 144)
    n = g.n_cols
    ld = S.pad_ld(n) + 64
    rd = api.real_dtype(precision)
    vg = api.VerticalGrid(g.hyai, g.hybi)
    hT = torch.tensor(S.to_ld(g.T, ld)).to(rd).pin_memory()
    hq = torch.tensor(S.to_ld(g.q, ld)).to(rd).pin_memory()
    ps_np = S.to_ld(g.ps, ld)
    ps_np[n:] = 1e5
    hps = torch.tensor(ps_np).pin_memory()
    hd, hs = api.new_host_outputs(g.pver, ld, precision), api.new_host_outputs(g.pver, ld, precision)
    pipe = api.HostPipeline(vg, n, ld, precision, chunk_cols=3000)  # 5 chunks, ragged last
    pipe.run(hT, hq, hps, hd, hs, dt=g.dt)
    torch.cuda.synchronize()
    d, s = api.deep_shallow(hT.cuda(), hq.cuda(), hps.cuda(), vg, dt=g.dt, precision=precision,
                            n_cols=n)
    torch.cuda.synchronize()
    for host, dev in ((hd, d), (hs, s)):
        for k in host:
            a = host[k].numpy()[..., :n]
            b = dev[k].cpu().numpy()[..., :n]
            assert np.array_equal(a, b, equal_nan=True), k
    pipe.close()


def test_pipeline_with_per_column_lambda_tau_and_params():
    """Per-column entrainment rates and relaxation times travel chunk by chunk
    with the profiles; non-default scheme parameters reach every chunk."""
    import torch

    from paper_1711_00289_gb300 import _lib as L
    from paper_1711_00289_gb300 import api

    g = S.latlon_grid(48, 72, tau_range=(1800.0, 7200.0))
    n = g.n_cols
    lam = 5e-4 + 1.5e-3 * S.uniform(4242, 0, np.arange(n), 0)
    vg = api.VerticalGrid(g.hyai, g.hybi)
    hT = torch.tensor(g.T).float().pin_memory()
    hq = torch.tensor(g.q).float().pin_memory()
    hps = torch.tensor(g.ps).pin_memory()
    hlam = torch.tensor(lam).pin_memory()
    htau = torch.tensor(g.tau).pin_memory()
    dp, sp = L.deep_defaults(), L.shallow_defaults()
    dp.capelmt, sp.c_m = 40.0, 0.05
    hd, hs = api.new_host_outputs(g.pver, n, "mixed"), api.new_host_outputs(g.pver, n, "mixed")
    pipe = api.HostPipeline(vg, n, n, "mixed", chunk_cols=1000)  # 4 chunks, ragged last
    pipe.run(hT, hq, hps, hd, hs, dt=g.dt, lam=hlam, tau=htau, deep_params=dp,
             shallow_params=sp)
    torch.cuda.synchronize()
    d, s = api.deep_shallow(hT.cuda(), hq.cuda(), hps.cuda(), vg, dt=g.dt, precision="mixed",
                            lam=hlam.cuda(), tau=htau.cuda(), deep_params=dp, shallow_params=sp)
    torch.cuda.synchronize()
    for host, dev in ((hd, d), (hs, s)):
        for k in host:
            assert np.array_equal(host[k].numpy(), dev[k].cpu().numpy(), equal_nan=True), k
    assert ((hd["flags"] & 2) > 0).sum() > 100
    pipe.close()
