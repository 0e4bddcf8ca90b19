"""The plume-spectrum variant of the deep scheme (n_plumes > 1) on the GPU
against the oracle with the same parameters: FP64 within 1e-10 on both paths,
on the 13,824-column lat-lon grid and on every column of the 884,736-column
grid; the mixed path within its error budget; one plume is the default kernels'
result bit for bit; the variant together with shallow rain evaporation."""
import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S
from tests.gpu_util import (THREADS, assert_fp64_parity, check_mixed, layer_mass, mixed_report,
                            run_gpu, same_decisions)

pytestmark = pytest.mark.gpu

NP, SPREAD = 3, 4.0


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _dpar(n=NP):
    from paper_1711_00289_gb300 import _lib as L

    dp = L.deep_defaults()
    dp.n_plumes, dp.plume_spread = n, SPREAD
    return dp


def _oracle(oracle, g, n=NP, **kw):
    return oracle.deep_shallow(g, dpar=oracle.deep_params(n_plumes=n, plume_spread=SPREAD),
                               threads=THREADS, **kw)


@pytest.mark.parametrize("path", ["plain", "compact"])
def test_fp64_matches_oracle(oracle, path):
    g = S.latlon_grid(96, 144)
    rd, rs = _oracle(oracle, g)
    gd, gs = run_gpu(g, "fp64", path, ld=S.pad_ld(g.n_cols) + 32, deep_params=_dpar())
    assert_fp64_parity(gd, rd, what=f"deep {path}")
    assert_fp64_parity(gs, rs, what=f"shallow {path}")
    # the variant changes the result: the ensemble reaches higher than the bulk plume
    r1, _ = oracle.deep_shallow(g, threads=THREADS)
    act = (rd["flags"] & 2) > 0
    assert act.sum() > 1000
    assert (rd["ktop"][act] < r1["ktop"][act]).mean() > 0.2


@pytest.mark.parametrize("n", [2, 8])
def test_member_count_edges(oracle, n):
    """Two members (the rate exponent's denominator n - 1 = 1) and the most the
    interface allows (CONV_MAX_PLUMES = 8): FP64 on the compacted path and the
    mixed path within its budget."""
    g = S.latlon_grid(48, 72)
    rd, rs = _oracle(oracle, g, n)
    gd, gs = run_gpu(g, "fp64", "compact", ld=S.pad_ld(g.n_cols) + 32, deep_params=_dpar(n))
    assert_fp64_parity(gd, rd, what=f"deep n={n}")
    assert_fp64_parity(gs, rs, what=f"shallow n={n}")
    md, ms = run_gpu(g, "mixed", "compact", deep_params=_dpar(n))
    m = layer_mass(g)
    psurf = rd["prec"] + rs["prec"]
    for tag, got, ref, up in (("deep", md, rd, None), ("shallow", ms, rs, same_decisions(md, rd))):
        r = mixed_report(got, ref, m, up, psurf)
        check_mixed(r, tag, 3e-3)


def test_one_plume_is_the_default(oracle):
    g = S.latlon_grid(48, 72)
    a = run_gpu(g, "mixed", "compact")
    b = run_gpu(g, "mixed", "compact", deep_params=_dpar(1))
    for x, y in zip(a, b):
        for k in x:
            assert np.array_equal(x[k], y[k]), k


def test_mixed_within_budget(oracle):
    g = S.latlon_grid(96, 144)
    rd, rs = _oracle(oracle, g)
    gd, gs = run_gpu(g, "mixed", "compact", deep_params=_dpar())
    m = layer_mass(g)
    deep_same = same_decisions(gd, rd)
    psurf = rd["prec"] + rs["prec"]
    for tag, got, ref, up in (("deep", gd, rd, None), ("shallow", gs, rs, deep_same)):
        r = mixed_report(got, ref, m, up, psurf)
        check_mixed(r, tag)


def test_full_resolution_fp64(oracle):
    g = S.clustered_grid(0.3)
    rd, rs = _oracle(oracle, g)
    gd, gs = run_gpu(g, "fp64", "compact", deep_params=_dpar())
    assert_fp64_parity(gd, rd, what="deep")
    assert_fp64_parity(gs, rs, what="shallow")


def test_with_rain_evaporation(oracle):
    from paper_1711_00289_gb300 import _lib as L

    g = S.latlon_grid(96, 144)
    sp = L.shallow_defaults()
    sp.ql_crit, sp.evap_k = 1e-4, 0.05
    rd, rs = _oracle(oracle, g, spar=oracle.shallow_params(ql_crit=1e-4, evap_k=0.05))
    gd, gs = run_gpu(g, "fp64", "compact", deep_params=_dpar(), shallow_params=sp)
    assert_fp64_parity(gd, rd, what="deep")
    assert_fp64_parity(gs, rs, what="shallow")
