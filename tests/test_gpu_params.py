"""FP64 parity with the oracle away from the default parameters: every deep and
shallow parameter of the C ABI is moved (trigger threshold, entrainment,
rain-out, downdraft strength, launch and top limits, limiter floor, Newton
counts, the shallow plume's mixing, TKE closure, CIN limits, w2 coefficients,
autoconversion threshold), on both paths, through the same comparison as the
default-parameter tests (flags and level indices bit-exact, tendencies within
1e-10)."""
import pytest

from paper_1711_00289_gb300 import soundings as S
from tests.gpu_util import THREADS, assert_fp64_parity, run_gpu

pytestmark = pytest.mark.gpu

DEEP = [
    dict(capelmt=20.0, lambda_default=5e-4, tau_default=1800.0, c0=4e-3, alpha_dd=0.1),
    dict(capelmt=150.0, c0=1e-3, alpha_dd=0.5, p_launch_min=70000.0, p_top_lim=10000.0),
    dict(q_min=1e-8, ent_zscale=500.0, n_newton_lcl=3, n_newton_h=2, tau_default=7200.0),
]
SHALLOW = [
    dict(eps_s=1e-3, tke=2.0, c_m=0.05, cin_scale=5.0, cin_max=80.0),
    dict(a_w=0.5, b_w=0.0, ql_crit=5e-4, p_lcl_min=75000.0, p_lfc_min=60000.0),
    dict(p_top_lim=10000.0, n_newton_lcl=3, n_newton_h=2, b_w=4.0),
]


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def grid():
    return S.latlon_grid(48, 72)


@pytest.mark.parametrize("path", ["plain", "compact"])
@pytest.mark.parametrize("case", range(3))
def test_fp64_parity_off_default(oracle, grid, path, case):
    from paper_1711_00289_gb300 import _lib as L

    dp, sp = L.deep_defaults(), L.shallow_defaults()
    for k, v in DEEP[case].items():
        setattr(dp, k, v)
    for k, v in SHALLOW[case].items():
        setattr(sp, k, v)
    g = grid
    rd, rs = oracle.deep_shallow(g, dpar=oracle.deep_params(**DEEP[case]),
                                 spar=oracle.shallow_params(**SHALLOW[case]), threads=THREADS)
    act = ((rd["flags"] & 2) > 0).sum() + ((rs["flags"] & 2) > 0).sum()
    assert act > 50
    gd, gs = run_gpu(g, "fp64", path, ld=S.pad_ld(g.n_cols) + 32, deep_params=dp,
                     shallow_params=sp)
    assert_fp64_parity(gd, rd, what=f"deep case {case} {path}")
    assert_fp64_parity(gs, rs, what=f"shallow case {case} {path}")


@pytest.mark.parametrize("case", [0, 1])
def test_mixed_budget_off_default(oracle, grid, case):
    """The mixed compacted path within its error budget at converged off-default
    parameter sets (case 2 cuts the Newton counts, where the two precisions'
    convergence flags are defined differently)."""
    from paper_1711_00289_gb300 import _lib as L
    from tests.gpu_util import check_mixed, layer_mass, mixed_report, same_decisions

    dp, sp = L.deep_defaults(), L.shallow_defaults()
    for k, v in DEEP[case].items():
        setattr(dp, k, v)
    for k, v in SHALLOW[case].items():
        setattr(sp, k, v)
    g = grid
    rd, rs = oracle.deep_shallow(g, dpar=oracle.deep_params(**DEEP[case]),
                                 spar=oracle.shallow_params(**SHALLOW[case]), threads=THREADS)
    gd, gs = run_gpu(g, "mixed", "compact", deep_params=dp, shallow_params=sp)
    m = layer_mass(g)
    deep_same = same_decisions(gd, rd)
    psurf = rd["prec"] + rs["prec"]
    for tag, got, ref, up in (("deep", gd, rd, None), ("shallow", gs, rs, deep_same)):
        r = mixed_report(got, ref, m, up, psurf)
        check_mixed(r, tag, 2e-3)


@pytest.mark.parametrize("case", [0, 1])
def test_adjoints_off_default(oracle, grid, case):
    """Both FP64 adjoints against the oracle's forward-mode tangent at converged
    off-default parameter sets (gradients within 1e-10 of each column's largest)."""
    import numpy as np
    import torch

    from paper_1711_00289_gb300 import _lib as L
    from paper_1711_00289_gb300 import api
    from tests.gpu_util import to_device

    dp, sp = L.deep_defaults(), L.shallow_defaults()
    for k, v in DEEP[case].items():
        setattr(dp, k, v)
    for k, v in SHALLOW[case].items():
        setattr(sp, k, v)
    g = grid
    n = g.n_cols
    c = np.arange(n)
    seeds = [2.0 * S.uniform(31 + case, 0, c, j) - 1.0 for j in range(4)]
    T, q, ps, lam, tau = to_device(g, "fp64")
    vg = api.VerticalGrid(g.hyai, g.hybi)
    dev = [torch.tensor(x, device="cuda") for x in seeds]
    od = oracle.deep_params(**DEEP[case])
    osp = oracle.shallow_params(**SHALLOW[case])

    def close(got, ref, what):
        for x, y, k in zip(got, ref, ("gT", "gq", "glambda", "gtau")):
            x, y = np.atleast_2d(x), np.atleast_2d(y)
            den = np.maximum(np.abs(y).max(axis=0), 1e-300)
            err = (np.abs(x - y).max(axis=0) / den)[np.abs(y).max(axis=0) > 0]
            assert err.size == 0 or err.max() <= 1e-10, f"{what} {k}: {err.max():.3g}"

    r = api.deep_adjoint(T, q, ps, vg, gP=dev[0], gH=dev[1], dt=g.dt, lam=lam, tau=tau,
                         params=dp)
    torch.cuda.synchronize()
    got = [r[k].cpu().numpy() for k in ("gT", "gq", "glambda", "gtau")]
    close(got, oracle.deep_adjoint(g, seeds[0], seeds[1], par=od, threads=THREADS), "deep")
    r = api.deep_shallow_adjoint(T, q, ps, vg, gPd=dev[0], gHd=dev[1], gPs=dev[2], gHs=dev[3],
                                 dt=g.dt, lam=lam, tau=tau, deep_params=dp, shallow_params=sp)
    torch.cuda.synchronize()
    got = [r[k].cpu().numpy() for k in ("gT", "gq", "glambda", "gtau")]
    ref = oracle.deep_shallow_adjoint(g, *seeds, dpar=od, spar=osp, threads=THREADS)
    close(got, ref, "step")
