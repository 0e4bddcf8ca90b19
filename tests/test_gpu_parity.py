"""CUDA path vs the FP64 CPU oracle, through the C ABI, on seeded soundings.

FP64 bar: flags and cloud-base/top level indices bit-exact, tendencies within
1e-10 of each column's largest reference tendency, column scalars within 1e-10.
Mixed bar: decision mismatches and trigger flips <= 0.1% of columns; over
columns with identical decisions, tendency column integrals within 1e-4 and
precipitation within 1e-3 (relative).
"""
import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S
from tests.gpu_util import (THREADS, assert_fp64_parity, check_mixed, layer_mass, mixed_report,
                            run_gpu, same_decisions, to_device)

pytestmark = pytest.mark.gpu

PATHS = ["plain", "compact"]


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def latlon():
    return S.latlon_grid()


@pytest.mark.parametrize("path", PATHS)
def test_column_set_fp64(oracle, path):
    g = S.column_set(64)
    rd, rs = oracle.deep_shallow(g)
    gd, gs = run_gpu(g, "fp64", path)
    assert_fp64_parity(gd, rd, what="deep")
    assert_fp64_parity(gs, rs, what="shallow")
    assert ((rd["flags"] & 2) > 0).sum() > 5


@pytest.mark.parametrize("path", PATHS)
def test_latlon_fp64_deep_shallow(oracle, latlon, path):
    rd, rs = oracle.deep_shallow(latlon, threads=THREADS)
    gd, gs = run_gpu(latlon, "fp64", path)
    assert_fp64_parity(gd, rd, what="deep")
    assert_fp64_parity(gs, rs, what="shallow")
    frac = ((rd["flags"] & 1) > 0).mean()
    assert 0.2 < frac < 0.3


@pytest.mark.parametrize("path", PATHS)
def test_separate_entry_points_fp64(oracle, path):
    g = S.latlon_grid(24, 36)
    (gd,) = run_gpu(g, "fp64", path, scheme="deep")
    assert_fp64_parity(gd, oracle.deep(g), what="deep-only")
    (gs,) = run_gpu(g, "fp64", path, scheme="shallow")
    assert_fp64_parity(gs, oracle.shallow(g), what="shallow-only")


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("n,pad", [(1, 0), (31, 1), (33, 31), (129, 0), (1000, 24), (4099, 61)])
def test_ragged_sizes_and_padding_untouched(oracle, path, n, pad):
    g = S.column_set(n, seed=777 + n)
    ld = n + pad
    (gd, gs), (hd, hs) = run_gpu(g, "fp64", path, ld=ld, sentinel=True)
    rd, rs = oracle.deep_shallow(g, threads=THREADS)
    assert_fp64_parity(gd, rd, what=f"deep n={n}")
    assert_fp64_parity(gs, rs, what=f"shallow n={n}")
    for h in (hd, hs):
        for k, v in h.items():
            tail = v[:, n:] if v.ndim == 2 else v[n:]
            assert np.all(tail == -7), f"padding of {k} written"


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("pver", [4, 8, 26, 32])
def test_other_level_counts(oracle, path, pver):
    g = S.column_set(512, seed=99 + pver, pver=pver)
    g.lam = np.full(g.n_cols, 1.7e-3)
    rd, rs = oracle.deep_shallow(g, threads=THREADS)
    gd, gs = run_gpu(g, "fp64", path)
    assert_fp64_parity(gd, rd, what=f"deep pver={pver}")
    assert_fp64_parity(gs, rs, what=f"shallow pver={pver}")


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("pver", [4, 8, 26, 32])
def test_mixed_other_level_counts(oracle, path, pver):
    """The mixed path at the level counts the ABI accepts besides 30 (its level
    arrays, in shared memory in the trigger pass, are sized by the level count;
    on 8 levels a warm-started moist inversion needs up to four Newton steps),
    within the mixed budget against the FP64 oracle on the mixed path's own
    FP32 inputs (trace deep precipitation on 8 levels moves by up to 7.9e-4
    when the oracle's inputs alone are rounded to FP32)."""
    import copy

    g = S.column_set(4096, seed=7 + pver, pver=pver)
    g32 = copy.copy(g)
    g32.T = g.T.astype(np.float32).astype(np.float64)
    g32.q = g.q.astype(np.float32).astype(np.float64)
    rd, rs = oracle.deep_shallow(g32, threads=THREADS)
    md, ms_ = run_gpu(g, "mixed", path)
    m = layer_mass(g32)
    psurf = rd["prec"] + rs["prec"]
    check_mixed(mixed_report(md, rd, m, None, psurf), f"deep pver={pver}")
    check_mixed(mixed_report(ms_, rs, m, same_decisions(md, rd), psurf), f"shallow pver={pver}")


@pytest.mark.parametrize("path", PATHS)
def test_bad_inputs_flagged_and_zeroed(oracle, path):
    g = S.column_set(64, seed=5)
    g.T[3, 1] = np.nan
    g.q[29, 2] = -1e-6
    g.ps[3] = 4.0e4
    g.T[0, 4] = 450.0
    g.q[10, 5] = np.inf
    rd, rs = oracle.deep_shallow(g)
    gd, gs = run_gpu(g, "fp64", path)
    for c in range(1, 6):
        assert gd["flags"][c] == 16 and gs["flags"][c] == 16
        assert np.all(gd["dTdt"][:, c] == 0) and np.all(gs["dqdt"][:, c] == 0)
    assert_fp64_parity(gd, rd, what="deep")
    assert_fp64_parity(gs, rs, what="shallow")


@pytest.mark.parametrize("path", PATHS)
def test_zero_columns_is_a_noop(path):
    import torch

    from paper_1711_00289_gb300 import api

    g = S.column_set(32)
    vg = api.VerticalGrid(g.hyai, g.hybi)
    T = torch.tensor(g.T, device="cuda")
    q = torch.tensor(g.q, device="cuda")
    ps = torch.tensor(g.ps, device="cuda")
    od = api.new_outputs(30, 32, "fp64")
    od["flags"].fill_(-3)
    api.deep(T, q, ps, vg, n_cols=0, out=od, path=path)
    torch.cuda.synchronize()
    assert torch.all(od["flags"] == -3)


@pytest.mark.parametrize("path", PATHS)
def test_deterministic_and_permutation_invariant(path):
    g = S.latlon_grid(48, 72)
    a = run_gpu(g, "fp64", path)
    b = run_gpu(g, "fp64", path)
    perm = np.random.default_rng(3).permutation(g.n_cols)
    gp = S.Columns("perm", g.pver, g.T[:, perm], g.q[:, perm], g.ps[perm], g.hyai, g.hybi)
    c = run_gpu(gp, "fp64", path)
    for x, y, z in zip(a, b, c):
        for k in x:
            assert np.array_equal(x[k], y[k], equal_nan=True), k
            zz = z[k]
            xx = x[k][:, perm] if x[k].ndim == 2 else x[k][perm]
            assert np.array_equal(xx, zz, equal_nan=True), k


@pytest.mark.parametrize("path", PATHS)
def test_mixed_precision_budget(oracle, latlon, path):
    rd, rs = oracle.deep_shallow(latlon, threads=THREADS)
    gd, gs = run_gpu(latlon, "mixed", path)
    m = layer_mass(latlon)
    deep_same = same_decisions(gd, rd)
    psurf = rd["prec"] + rs["prec"]
    for tag, got, ref, up in (("deep", gd, rd, None), ("shallow", gs, rs, deep_same)):
        r = mixed_report(got, ref, m, up, psurf)
        check_mixed(r, tag)


@pytest.mark.parametrize("frac", [0.1, 0.3, 0.6])
def test_full_resolution_grid(oracle, frac):
    """884,736 columns x 30 levels, the launches the benchmark times: every column
    of the FP64 paths against the oracle, the mixed compacted path against its
    error budget."""
    g = S.clustered_grid(frac)
    rd, rs = oracle.deep_shallow(g, threads=THREADS)
    for path in PATHS:
        gd, gs = run_gpu(g, "fp64", path)
        assert_fp64_parity(gd, rd, what=f"deep f={frac} {path}")
        assert_fp64_parity(gs, rs, what=f"shallow f={frac} {path}")
    trig = ((rd["flags"] & 1) > 0).mean()
    assert abs(trig - frac) < 0.02
    m = layer_mass(g)
    gd, gs = run_gpu(g, "mixed", "compact")
    deep_same = same_decisions(gd, rd)
    psurf = rd["prec"] + rs["prec"]
    for tag, got, ref, up in (("deep", gd, rd, None), ("shallow", gs, rs, deep_same)):
        r = mixed_report(got, ref, m, up, psurf)
        check_mixed(r, tag)


def test_compact_fp64_matches_plain_fp64():
    """The compacted FP64 path runs the same column code as the plain kernel (the
    shallow scheme reuses the deep LCL and parcel only when they are the same
    computation): decisions and integer outputs are identical, and real outputs
    agree to rounding -- the two kernels are compiled separately, so the
    compiler may contract a multiply-add differently in each."""
    g = S.latlon_grid()
    a = run_gpu(g, "fp64", "plain")
    b = run_gpu(g, "fp64", "compact")
    for x, y, tag in zip(a, b, ("deep", "shallow")):
        assert_fp64_parity(y, x, tol=1e-12, what=f"compact vs plain {tag}")


def test_workspace_errors():
    """Missing, short or misaligned workspaces are rejected on the host.  n_cols is
    0, so even a wrongly accepted call would launch nothing."""
    import ctypes as C

    import torch

    from paper_1711_00289_gb300 import _lib as L
    from paper_1711_00289_gb300 import api

    g = S.column_set(64)
    vg = api.VerticalGrid(g.hyai, g.hybi)
    T, q, ps = (torch.tensor(x, device="cuda") for x in (g.T, g.q, g.ps))
    out = api.new_outputs(30, 64, "fp64")
    grid = vg.struct(0, 64)
    inp = L.In(T.data_ptr(), q.data_ptr(), ps.data_ptr(), None, None)
    o = api._out_struct(out, 30, 64, "fp64")
    lc = L.Launch(L.CONV_PATH_COMPACT, 0, 0, 0, None)
    dp = L.deep_defaults()
    need = L.lib().conv_workspace_bytes(C.byref(grid), L.CONV_FP64, C.byref(lc))
    assert need >= 256
    buf = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    base = buf.data_ptr() + ((-buf.data_ptr()) % 256)
    run = L.lib().conv_deep_run
    args = (C.byref(grid), C.byref(inp), C.byref(dp), 1800.0, L.CONV_FP64, C.byref(o),
            C.byref(lc))
    assert run(*args, None, need, None) == L.CONV_ERR_WORKSPACE
    assert run(*args, C.c_void_p(base), need - 1, None) == L.CONV_ERR_WORKSPACE
    assert run(*args, C.c_void_p(base + 8), need, None) == L.CONV_ERR_WORKSPACE
    assert run(*args, C.c_void_p(base), need, None) == L.CONV_OK
    torch.cuda.synchronize()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_prepared_step_matches_call(precision):
    """api.PreparedStep (arguments marshalled once) gives bit-identical outputs to
    api.deep_shallow, with and without stage events, call after call."""
    import torch

    from paper_1711_00289_gb300 import api

    g = S.clustered_grid(0.3, 48, 72)
    T, q, ps, lam, tau = to_device(g, precision)
    vg = api.VerticalGrid(g.hyai, g.hybi)
    a = api.deep_shallow(T, q, ps, vg, dt=g.dt, precision=precision, lam=lam, tau=tau,
                         path="compact")
    run = api.PreparedStep(T, q, ps, vg, dt=g.dt, precision=precision, lam=lam, tau=tau,
                           path="compact")
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for launch in (None, run.launch_struct(evs), None):
        b = run(launch)
        torch.cuda.synchronize()
        for x, y in zip(a, b):
            for k in x:
                assert torch.equal(x[k], y[k]), k
    assert evs[0].elapsed_time(evs[2]) > 0.0


@pytest.mark.parametrize("path", PATHS)
def test_every_column_convecting(oracle, path):
    """The degenerate load the compaction exists for, inverted: every column
    triggers (the queue holds the whole grid)."""
    g = S.clustered_grid(1.0, 48, 72)
    rd, rs = oracle.deep_shallow(g, threads=THREADS)
    assert ((rd["flags"] & 1) > 0).mean() > 0.99
    gd, gs = run_gpu(g, "fp64", path)
    assert_fp64_parity(gd, rd, what="deep")
    assert_fp64_parity(gs, rs, what="shallow")
    md, ms_ = run_gpu(g, "mixed", path)
    r = mixed_report(md, rd, layer_mass(g), None, rd["prec"] + rs["prec"])
    check_mixed(r, "deep", 2e-3)


@pytest.mark.parametrize("path", PATHS)
def test_no_column_convecting(oracle, path):
    """The other degenerate load: no column triggers the deep scheme (a CAPE
    threshold no column reaches), so the compacted path's queue stays empty and
    the plume pass has nothing to do; the shallow scheme then runs on every
    column's own state in the trigger pass, plumes included.

    FP64 against the oracle as everywhere.  Mixed: against the oracle on the
    mixed path's own inputs (the FP32 profiles, exactly converted): shallow-only
    trace rain here is conditioned so that rounding the inputs to FP32 alone
    moves the FP64 definition's precipitation by up to 7.5e-4, half the total
    difference from the unrounded oracle; the budget measures the arithmetic."""
    import copy

    from paper_1711_00289_gb300 import _lib as L
    from tests.test_oracle_random import _random_columns

    g = _random_columns(5, n=4000)
    dpar = oracle.deep_params(capelmt=1e9)
    rd, rs = oracle.deep_shallow(g, dpar=dpar, threads=THREADS)
    assert not ((rd["flags"] & 1) > 0).any()
    assert ((rs["flags"] & 2) > 0).sum() > 100  # active shallow plumes
    dp = L.deep_defaults()
    dp.capelmt = 1e9
    gd, gs = run_gpu(g, "fp64", path, deep_params=dp)
    assert_fp64_parity(gd, rd, what="deep")
    assert_fp64_parity(gs, rs, what="shallow")
    assert not gd["dTdt"].any() and not gd["dqdt"].any() and not gd["prec"].any()
    g32 = copy.copy(g)
    g32.T = g.T.astype(np.float32).astype(np.float64)
    g32.q = g.q.astype(np.float32).astype(np.float64)
    r32d, r32s = oracle.deep_shallow(g32, dpar=dpar, threads=THREADS)
    md, ms_ = run_gpu(g, "mixed", path, deep_params=dp)
    r = mixed_report(ms_, r32s, layer_mass(g32), same_decisions(md, r32d),
                     r32d["prec"] + r32s["prec"])
    check_mixed(r, "shallow")
