"""Parity on randomly perturbed soundings (inversions, superadiabatic, moist and
dry layers, surface pressures of 600-1040 hPa, random entrainment rates and
closure times).

FP64 against the oracle on both paths: decisions bit-exact, values within
1e-10.  On these columns a parcel can lie 10-50 K from the environment
temperature its moist inversion starts from; the inversions test convergence
for termination, so every solve of both sides converges.

The mixed path against the same default oracle, within its full budget:
trigger flips and decision mismatches on at most 0.1% of the columns, tendency
column integrals within 1e-4 and precipitation within 1e-3 where decisions
agree.  Trace drizzle -- a shallow plume barely above the autoconversion
threshold -- is where FP32 rounding of the saturation temperature would be a
large part of the rain; the mixed path refines it in FP64 there."""
import pytest

from paper_1711_00289_gb300 import soundings as S
from tests.gpu_util import (THREADS, assert_fp64_parity, check_mixed, layer_mass, mixed_report,
                            run_gpu, same_decisions)
from tests.test_oracle_random import _random_columns

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def grid():
    return _random_columns(7, n=3000)


@pytest.fixture(scope="module")
def reference(oracle, grid):
    rd, rs = oracle.deep_shallow(grid, threads=THREADS)
    assert not ((rd["flags"] | rs["flags"]) & 8).any()  # every reference solve converged
    return rd, rs


@pytest.fixture(scope="module")
def mixed(reference, grid):
    rd, rs = reference
    gd, gs = run_gpu(grid, "mixed", "compact")
    m = layer_mass(grid)
    psurf = rd["prec"] + rs["prec"]
    rep = {tag: mixed_report(got, ref, m, up, psurf)
           for tag, got, ref, up in (("deep", gd, rd, None),
                                     ("shallow", gs, rs, same_decisions(gd, rd)))}
    print(rep)
    return rep


@pytest.mark.parametrize("path", ["plain", "compact"])
def test_fp64(reference, grid, path):
    rd, rs = reference
    gd, gs = run_gpu(grid, "fp64", path, ld=S.pad_ld(grid.n_cols) + 32)
    assert_fp64_parity(gd, rd, what=f"deep {path}")
    assert_fp64_parity(gs, rs, what=f"shallow {path}")


def test_mixed_budget(mixed):
    for tag, r in mixed.items():
        assert r["active"] > 300, f"{tag} {r}"
        check_mixed(r, tag)
