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
