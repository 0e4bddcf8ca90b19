"""Sharding by convective work on the GPU (one device): the per-block count of
triggered columns (conv_count_triggered) against a count on the host, runs of
column ranges (the inputs and outputs offset by the range's first column) that
put together equal the whole-grid run bit for bit, and three ranks' steps taken
one after the other on this device (their kernels do not wait on each other),
whose ranges after a rebalance are those the grid's counts give and whose
outputs together equal the whole-grid run."""
import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def grid():
    return S.clustered_grid(0.3, 96, 144)


def _inputs(g, precision):
    from tests.gpu_util import to_device

    T, q, ps, _, _ = to_device(g, precision)
    return T, q, ps


def _whole(g, precision, path):
    import torch

    from paper_1711_00289_gb300 import api

    T, q, ps = _inputs(g, precision)
    od, os_ = api.deep_shallow(T, q, ps, api.VerticalGrid(g.hyai, g.hybi), dt=g.dt,
                               precision=precision, path=path)
    torch.cuda.synchronize()
    return od, os_


@pytest.mark.parametrize("block", [1024, 100, 32, 7])
def test_count_triggered(grid, block):
    from paper_1711_00289_gb300 import shard

    od, _ = _whole(grid, "mixed", "compact")
    n = grid.n_cols - 5  # a ragged last block
    got = shard.count_triggered(od["flags"], n, 0, block).cpu().numpy()
    trig = (od["flags"].cpu().numpy()[:n] & 1) > 0
    want = np.array([trig[j * block:(j + 1) * block].sum() for j in range(-(-n // block))])
    assert np.array_equal(got, want)
    # a block-aligned range of the grid
    c0 = 3 * block
    got2 = shard.count_triggered(od["flags"], n - c0, c0, block).cpu().numpy()
    assert np.array_equal(got2, want[3:])


@pytest.mark.parametrize("precision,path", [("mixed", "compact"), ("fp64", "plain"),
                                            ("fp64", "compact")])
def test_ranges_equal_the_whole_grid(grid, precision, path):
    import torch

    from paper_1711_00289_gb300 import api

    ref_d, ref_s = _whole(grid, precision, path)
    T, q, ps = _inputs(grid, precision)
    vg = api.VerticalGrid(grid.hyai, grid.hybi)
    n = grid.n_cols
    od = api.new_outputs(grid.pver, n, precision)
    os_ = api.new_outputs(grid.pver, n, precision)
    for c0, c1 in ((0, 4000), (4000, 4001), (4001, 9000), (9000, n)):
        api.deep_shallow(T, q, ps, vg, dt=grid.dt, precision=precision, path=path, col0=c0,
                         n_cols=c1 - c0, out_deep=od, out_shallow=os_)
    torch.cuda.synchronize()
    for a, b in ((od, ref_d), (os_, ref_s)):
        for k in a:
            assert torch.equal(a[k], b[k]), k


def test_three_ranks_one_after_the_other(grid):
    import torch

    from paper_1711_00289_gb300 import api, shard

    n = grid.n_cols
    ref_d, ref_s = _whole(grid, "mixed", "compact")
    T, q, ps = _inputs(grid, "mixed")
    vg = api.VerticalGrid(grid.hyai, grid.hybi)
    od = api.new_outputs(grid.pver, n, "mixed")
    os_ = api.new_outputs(grid.pver, n, "mixed")
    W = 3
    ranks = [shard.ShardedStep(T, q, ps, vg, rank=r, world=W, dt=grid.dt, precision="mixed",
                               out_deep=od, out_shallow=os_, path="compact") for r in range(W)]
    assert ranks[0].range[0] == 0 and ranks[-1].range[1] == n
    assert all(ranks[r].range[1] == ranks[r + 1].range[0] for r in range(W - 1))
    for step in range(2):
        for r in ranks:
            r.run()
        torch.cuda.synchronize()
        for a, b in ((od, ref_d), (os_, ref_s)):
            for k in a:
                assert torch.equal(a[k], b[k]), (step, k)
        # rebalance: every rank's counts of its own range, summed
        cnt = np.zeros(-(-n // shard.BLOCK), np.int64)
        for r in ranks:
            c0, c1 = r.range
            loc = shard.count_triggered(od["flags"], c1 - c0, c0).cpu().numpy()
            cnt[c0 // shard.BLOCK:c0 // shard.BLOCK + loc.size] += loc
        bounds = shard.partition(cnt, n, W)
        trig = (ref_d["flags"].cpu().numpy() & 1) > 0
        want = np.array([trig[j * shard.BLOCK:(j + 1) * shard.BLOCK].sum()
                         for j in range(cnt.size)])
        assert np.array_equal(cnt, want)
        for r in ranks:
            r.bounds = bounds
    # on this grid (convection in the middle third) the balanced split differs
    # from the even one
    assert not np.array_equal(ranks[0].bounds, shard.even_bounds(n, W))
