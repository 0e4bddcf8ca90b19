"""Shallow rain evaporation (a scheme variant, off by default) on the GPU against
the oracle with the same parameters: FP64 within 1e-10 on both paths, on the
13,824-column lat-lon grid and on every column of the 884,736-column grid; the
mixed path within its error budget; decisions and the deep scheme unchanged by
the variant; column budgets closed."""
import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S
from tests.gpu_util import (THREADS, assert_fp64_parity, check_mixed, layer_mass, mixed_report,
                            run_gpu, same_decisions)

pytestmark = pytest.mark.gpu

# a lower autoconversion threshold than the default makes most shallow plumes rain
QL, KE = 1e-4, 0.05


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _spar(k=KE):
    from paper_1711_00289_gb300 import _lib as L

    sp = L.shallow_defaults()
    sp.ql_crit, sp.evap_k = QL, k
    return sp


def _oracle(oracle, g, k=KE):
    return oracle.deep_shallow(g, spar=oracle.shallow_params(ql_crit=QL, evap_k=k),
                               threads=THREADS)


@pytest.mark.parametrize("path", ["plain", "compact"])
def test_fp64_matches_oracle(oracle, path):
    g = S.latlon_grid(96, 144)
    rd, rs = _oracle(oracle, g)
    gd, gs = run_gpu(g, "fp64", path, ld=S.pad_ld(g.n_cols) + 32, shallow_params=_spar())
    assert_fp64_parity(gd, rd, what=f"deep {path}")
    assert_fp64_parity(gs, rs, what=f"shallow {path}")
    _, r0 = _oracle(oracle, g, 0.0)
    act = (rs["flags"] & 2) > 0
    assert act.sum() > 300
    lost = (r0["prec"] - rs["prec"])[act].sum() / r0["prec"][act].sum()
    assert lost > 0.05  # the variant does something on this grid
    assert gs["cons_err"][act].max() <= 1e-12


def test_variant_changes_only_the_shallow_tendencies_and_rain(oracle):
    g = S.latlon_grid(96, 144)
    a = run_gpu(g, "fp64", "compact", shallow_params=_spar(0.0))
    b = run_gpu(g, "fp64", "compact", shallow_params=_spar())
    for k in a[0]:
        assert np.array_equal(a[0][k], b[0][k]), k
    for k in ("flags", "kb", "klcl", "ktop", "kaux", "cape", "mb"):
        assert np.array_equal(a[1][k], b[1][k]), k
    m = layer_mass(g)
    act = (a[1]["flags"] & 2) > 0
    ddq = (b[1]["dqdt"] - a[1]["dqdt"])[:, act]
    evap = np.sum(m[:, act] * ddq, axis=0)
    lost = (a[1]["prec"] - b[1]["prec"])[act]
    assert np.all(ddq >= -1e-18) and np.all(lost >= -1e-18)
    assert np.allclose(evap, lost, rtol=1e-9, atol=1e-12 * a[1]["prec"].max())


def test_mixed_within_budget(oracle):
    g = S.latlon_grid(96, 144)
    rd, rs = _oracle(oracle, g)
    gd, gs = run_gpu(g, "mixed", "compact", shallow_params=_spar())
    m = layer_mass(g)
    deep_same = same_decisions(gd, rd)
    psurf = rd["prec"] + rs["prec"]
    for tag, got, ref, up in (("deep", gd, rd, None), ("shallow", gs, rs, deep_same)):
        r = mixed_report(got, ref, m, up, psurf)
        check_mixed(r, tag)


def test_full_resolution_fp64(oracle):
    """Every column of the 884,736-column grid, compacted FP64 path."""
    g = S.clustered_grid(0.3)
    rd, rs = _oracle(oracle, g)
    gd, gs = run_gpu(g, "fp64", "compact", shallow_params=_spar())
    assert_fp64_parity(gd, rd, what="deep")
    assert_fp64_parity(gs, rs, what="shallow")


def test_with_profile_outputs_and_transport(oracle):
    """The variant and the mass-flux profiles in one extended run: the
    tendencies are those of the variant alone and the transport is that of the
    step without evaporation (evaporation moves no tracer)."""
    import torch

    from paper_1711_00289_gb300 import api
    from tests.gpu_util import to_device

    g = S.latlon_grid(48, 72)
    n = g.n_cols
    T, q, ps, lam, tau = to_device(g, "fp64")
    vg = api.VerticalGrid(g.hyai, g.hybi)
    tr = torch.tensor(np.stack([g.q, np.ones_like(g.q)]), device="cuda")
    od, os_, td, ts = api.deep_shallow_tracers(T, q, ps, tr, vg, dt=g.dt, precision="fp64",
                                              lam=lam, tau=tau, shallow_params=_spar())
    od0, os0, td0, ts0 = api.deep_shallow_tracers(T, q, ps, tr, vg, dt=g.dt, precision="fp64",
                                                 lam=lam, tau=tau, shallow_params=_spar(0.0))
    torch.cuda.synchronize()
    assert torch.equal(td, td0) and torch.equal(ts, ts0)
    rd, rs = _oracle(oracle, g)
    got = {k: v.cpu().numpy() for k, v in os_.items()}
    assert_fp64_parity(got, rs, what="shallow with profiles")
    assert n > 0
