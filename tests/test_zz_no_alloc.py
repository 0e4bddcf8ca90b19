"""conv_deep_shallow_run_noalloc: the fused run for callers that cannot allocate
device memory (its scratch is a library-owned static device array).  Its
outputs must equal those of conv_deep_shallow_run with a caller workspace, on
two calls in a row (the shared scratch keeps the previous call's contents).
Collected last on purpose, and independent of every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run_noalloc(L, api, vg, T, q, ps, n, precision, dt):
    od, os_ = api.new_outputs(30, n, precision), api.new_outputs(30, n, precision)
    grid = vg.struct(n, n)
    inp = L.In(T.data_ptr(), q.data_ptr(), ps.data_ptr(), None, None)
    st = L.lib().conv_deep_shallow_run_noalloc(
        C.byref(grid), C.byref(inp), C.byref(L.deep_defaults()), C.byref(L.shallow_defaults()),
        dt, api._PREC[precision], C.byref(api._out_struct(od, 30, n, precision)),
        C.byref(api._out_struct(os_, 30, n, precision)), api._stream(None))
    L.check(st, "conv_deep_shallow_run_noalloc")
    return od, os_


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_workspace_entry_point(precision):
    import torch

    from paper_1711_00289_gb300 import _lib as L
    from paper_1711_00289_gb300 import api

    g = S.latlon_grid()
    n = g.n_cols
    assert n <= L.NOALLOC_MAX_COLS
    rd = api.real_dtype(precision)
    T = torch.tensor(g.T, device="cuda").to(rd)
    q = torch.tensor(g.q, device="cuda").to(rd)
    ps = torch.tensor(g.ps, device="cuda")
    vg = api.VerticalGrid(g.hyai, g.hybi)
    ref = api.deep_shallow(T, q, ps, vg, dt=g.dt, precision=precision, path="compact")
    outs = [_run_noalloc(L, api, vg, T, q, ps, n, precision, g.dt) for _ in range(2)]
    torch.cuda.synchronize()
    for call in outs:
        for got, want in zip(call, ref):
            for k in want:
                a, b = got[k].cpu().numpy(), want[k].cpu().numpy()
                if a.dtype.kind == "i":
                    assert np.array_equal(a, b), k
                else:
                    den = np.maximum(np.abs(b), 1e-300)
                    assert np.all(np.abs(a - b) <= 1e-10 * den), k


def test_noalloc_rejects_more_columns_than_its_scratch():
    import torch

    from paper_1711_00289_gb300 import _lib as L
    from paper_1711_00289_gb300 import api

    n = L.NOALLOC_MAX_COLS + 1  # buffers really have n columns: nothing here is out of bounds
    a, b = S.hybrid_coefficients(30)
    vg = api.VerticalGrid(a, b)
    T = torch.full((30, n), 280.0, device="cuda", dtype=torch.float64)
    q = torch.full((30, n), 1e-3, device="cuda", dtype=torch.float64)
    ps = torch.full((n,), 1e5, device="cuda", dtype=torch.float64)
    with pytest.raises(L.ConvError) as ei:
        _run_noalloc(L, api, vg, T, q, ps, n, "fp64", 1800.0)
    assert ei.value.status == L.CONV_ERR_ARG
