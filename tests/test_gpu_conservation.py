"""Column energy and water conservation of both schemes' outputs (cons_err,
the residual ratio (|E_s - Lv P| + Lv |E_w + P|) / (cp sum m |dT| + Lv P) of a
column's tendencies and precipitation), through the C ABI.

FP64: at the rounding of FP64 sums (below 1e-12).  Mixed: at the rounding of
the FP32 tendencies, which the schemes build to conserve exactly in exact
arithmetic: below 1e-5 on every column where a scheme is active, on the
clustered grid at the three convecting fractions and on randomly perturbed
soundings.  The mixed ratio is evaluated in FP32 with error-free
transformations; a lost term or a sign error in it reads as O(1)."""
import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S
from tests.gpu_util import run_gpu
from tests.test_oracle_random import _random_columns

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


GRIDS = {
    "clustered-0.1": lambda: S.clustered_grid(0.1, 192, 288),
    "clustered-0.3": lambda: S.clustered_grid(0.3, 192, 288),
    "clustered-0.6": lambda: S.clustered_grid(0.6, 192, 288),
    "random": lambda: _random_columns(7, n=3000),
}


def _worst(out):
    act = (out["flags"] & 2) > 0
    assert act.sum() > 100
    c = out["cons_err"][act]
    assert np.all(np.isfinite(c))
    return float(c.max())


@pytest.mark.parametrize("name", sorted(GRIDS))
def test_mixed_conserves_to_fp32_rounding(name):
    g = GRIDS[name]()
    gd, gs = run_gpu(g, "mixed", "compact")
    wd, ws = _worst(gd), _worst(gs)
    print(name, "mixed cons_err max: deep", wd, "shallow", ws)
    assert wd <= 1e-5 and ws <= 1e-5, (wd, ws)


@pytest.mark.parametrize("name", ["clustered-0.3", "random"])
def test_fp64_conserves_to_fp64_rounding(name):
    g = GRIDS[name]()
    gd, gs = run_gpu(g, "fp64", "compact")
    assert _worst(gd) <= 1e-12 and _worst(gs) <= 1e-12


def test_mixed_plain_and_compact_agree():
    """The plain and compacted kernels evaluate the same ratio."""
    g = GRIDS["clustered-0.3"]()
    a = run_gpu(g, "mixed", "plain")
    b = run_gpu(g, "mixed", "compact")
    for x, y in zip(a, b):
        act = (x["flags"] & 2) > 0
        assert np.allclose(x["cons_err"][act], y["cons_err"][act], rtol=0, atol=1e-6)
