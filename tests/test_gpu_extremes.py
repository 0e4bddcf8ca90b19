"""Parity on physically extreme columns, where the rarely taken branches run:
very dry air (no LCL in reach), saturated and supersaturated low levels (the
LCL at the launch point, the q_s clamp), columns 30 K colder than the grid
(moist inversions started far from their roots), mountain surface pressures of
500-900 hPa, hot, moist columns, and superadiabatic surface layers (a dry-lifted
parcel buoyant below its LCL, where the shallow LFC must not be placed).  With
rain evaporation switched on, the (super)saturated low levels are layers the
rain falls through without evaporating.  FP64 against the oracle on both paths
(decisions bit-exact, values within 1e-10); the mixed path within its budget,
its convergence flag left out of the decision comparison (the two precisions
define it differently)."""
import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S
from tests.gpu_util import (THREADS, assert_fp64_parity, check_mixed, layer_mass, mixed_report,
                            run_gpu)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def extremes(oracle):
    g = S.latlon_grid(48, 72)
    n = g.n_cols
    c = np.arange(n)
    u = S.uniform(777, 0, c, 0)
    T, q, ps = g.T.copy(), g.q.copy(), g.ps.copy()
    kind = c % 6
    q[:, kind == 0] *= 0.05                                   # dry
    p_int = g.hyai[:, None] * 1e5 + g.hybi[:, None] * ps[None, :]
    pm = 0.5 * (p_int[1:] + p_int[:-1])
    qs = np.vectorize(oracle.qs)(T, pm)
    sel = kind == 1                                           # (super)saturated low levels
    q[-4:, sel] = qs[-4:, sel] * (1.0 + 0.05 * u[sel])
    T[:, kind == 2] -= 30.0                                   # cold
    ps[kind == 3] = 5e4 + 4e4 * u[kind == 3]                  # mountains
    T[:, kind == 4] += 8.0                                    # hot and moist
    q[:, kind == 4] *= 1.3
    sel = kind == 5                                           # superadiabatic surface layer
    T[-1, sel] += 2.0 + 2.0 * u[sel]
    return S.Columns("extremes-48x72", g.pver, T, q, ps, g.hyai, g.hybi, None, None, g.dt)


@pytest.mark.parametrize("path", ["plain", "compact"])
def test_fp64(oracle, extremes, path):
    g = extremes
    rd, rs = oracle.deep_shallow(g, threads=THREADS)
    # the cold columns' solves start far from their roots; the convergence test
    # still ends every one of them converged
    assert not ((rd["flags"] | rs["flags"]) & 8).any()
    gd, gs = run_gpu(g, "fp64", path, ld=S.pad_ld(g.n_cols) + 32)
    assert_fp64_parity(gd, rd, what=f"deep {path}")
    assert_fp64_parity(gs, rs, what=f"shallow {path}")


def test_superadiabatic_columns_reach_the_dry_branch(oracle, extremes):
    g = extremes
    idx = np.flatnonzero(np.arange(g.n_cols) % 6 == 5)[:100]
    dry = 0
    for i in idx:
        d = oracle.shallow_column_diag(g.pver, g.hyai, g.hybi, g.T[:, i], g.q[:, i],
                                       float(g.ps[i]))
        dry += d.exit_code != 1 and any(d.b[k] > 0 for k in range(d.klcl + 1, g.pver))
    assert dry > 50


def _spar_evap():
    from paper_1711_00289_gb300 import _lib as L

    sp = L.shallow_defaults()
    sp.ql_crit, sp.evap_k = 1e-4, 0.05
    return sp


@pytest.mark.parametrize("path", ["plain", "compact"])
def test_fp64_with_rain_evaporation(oracle, extremes, path):
    g = extremes
    rd, rs = oracle.deep_shallow(g, spar=oracle.shallow_params(ql_crit=1e-4, evap_k=0.05),
                                 threads=THREADS)
    sat = (np.arange(g.n_cols) % 6 == 1) & ((rs["flags"] & 2) > 0) & (rs["prec"] > 0)
    assert sat.sum() > 100  # raining columns whose low levels are (super)saturated
    gd, gs = run_gpu(g, "fp64", path, ld=S.pad_ld(g.n_cols) + 32, shallow_params=_spar_evap())
    assert_fp64_parity(gd, rd, what=f"deep {path}")
    assert_fp64_parity(gs, rs, what=f"shallow {path}")


def _mixed_check(g, gd, gs, rd, rs):
    for o in (rd, rs, gd, gs):
        o["flags"] = o["flags"] & ~8
    m = layer_mass(g)
    from tests.gpu_util import same_decisions

    deep_same = same_decisions(gd, rd)
    psurf = rd["prec"] + rs["prec"]
    for tag, got, ref, up in (("deep", gd, rd, None), ("shallow", gs, rs, deep_same)):
        r = mixed_report(got, ref, m, up, psurf)
        check_mixed(r, tag, 3e-3)


def test_mixed(oracle, extremes):
    g = extremes
    rd, rs = oracle.deep_shallow(g, threads=THREADS)
    gd, gs = run_gpu(g, "mixed", "compact")
    _mixed_check(g, gd, gs, rd, rs)


def test_mixed_with_rain_evaporation(oracle, extremes):
    g = extremes
    rd, rs = oracle.deep_shallow(g, spar=oracle.shallow_params(ql_crit=1e-4, evap_k=0.05),
                                 threads=THREADS)
    gd, gs = run_gpu(g, "mixed", "compact", shallow_params=_spar_evap())
    _mixed_check(g, gd, gs, rd, rs)
