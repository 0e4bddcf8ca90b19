"""Splitting a grid's columns over ranks by convective work (the proportional
partitioning of Sec. IV-D, by triggered columns instead of device speeds), on
the CPU: the partitioner's ranges (contiguous, block-aligned, the cost split as
evenly as block boundaries allow, against brute force), its argument checks,
and a two-rank gloo job in which the ranks sum their per-block counts, compute
identical ranges, and their ranges' outputs put together equal a one-rank run
(the oracle computes each range: the columns are independent).  Not measured on
several GPUs: every GPU run available to this project has one GPU."""
import os
import socket
import sys

import numpy as np
import pytest

from paper_1711_00289_gb300 import shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cost(counts, n, block, w_all, w_act):
    cols = np.full(counts.size, block, dtype=np.float64)
    cols[-1] = n - block * (counts.size - 1)
    return w_all * cols + w_act * counts


@pytest.mark.parametrize("seed,n,block,parts", [(1, 10000, 128, 2), (2, 884736, 1024, 4),
                                                (3, 5000, 100, 3), (4, 257, 32, 8)])
def test_partition_ranges(seed, n, block, parts):
    rng = np.random.default_rng(seed)
    nb = -(-n // block)
    cols = np.full(nb, block)
    cols[-1] = n - block * (nb - 1)
    # clustered convection: a few patches of busy blocks
    busy = np.zeros(nb)
    for c in rng.integers(0, nb, 3):
        busy[max(0, c - nb // 10):c + nb // 10] = 1
    counts = np.minimum(cols, (busy * rng.uniform(0.5, 1.0, nb) * cols).astype(np.int32))
    b = shard.partition(counts, n, parts, block=block)
    assert b[0] == 0 and b[-1] == n and np.all(np.diff(b) >= 0)
    assert np.all((b[1:-1] % block == 0) | (b[1:-1] == n))
    # each inner bound is the block boundary closest to its share of the cost
    pre = np.concatenate([[0.0], np.cumsum(_cost(counts, n, block, 1.0, 3.0))])
    for r in range(1, parts):
        target = pre[-1] * r / parts
        j = b[r] // block if b[r] < n else nb
        best = np.min(np.abs(pre - target))
        assert abs(pre[j] - target) <= best + 1e-9 * pre[-1]
    # the work of the busiest range is within one block of the ideal share
    cmax = _cost(counts, n, block, 1.0, 3.0).max()
    part_cost = [pre[(b[r + 1] // block if b[r + 1] < n else nb)]
                 - pre[(b[r] // block if b[r] < n else nb)] for r in range(parts)]
    assert max(part_cost) <= pre[-1] / parts + cmax + 1e-9
    # deterministic
    assert np.array_equal(b, shard.partition(counts.copy(), n, parts, block=block))


def test_partition_balances_better_than_an_even_split():
    n, block = 65536, 512
    nb = n // block
    counts = np.zeros(nb, np.int32)
    counts[: nb // 4] = block  # the first quarter convects everywhere
    even = shard.even_bounds(n, 2, block)
    bal = shard.partition(counts, n, 2, block=block)
    c = _cost(counts, n, block, shard.W_ALL, shard.W_ACTIVE)
    work = lambda b: [c[b[r] // block:b[r + 1] // block].sum() for r in range(2)]  # noqa: E731
    assert even[1] == n // 2
    assert max(work(bal)) < 0.8 * max(work(even))
    assert abs(work(bal)[0] - work(bal)[1]) <= c.max()


@pytest.mark.parametrize("n,block,parts", [(1000, 128, 4), (884736, 1024, 8), (100, 128, 4),
                                          (0, 128, 2), (1024, 128, 8), (1024, 128, 16)])
def test_partition_degenerate_cases(n, block, parts):
    """No convection anywhere: the split is by columns alone, each bound the
    block boundary nearest its share.  More ranks than blocks, or no columns:
    the ranges still tile [0, n) in order, the surplus ranks empty."""
    nb = -(-n // block)
    b = shard.partition(np.zeros(nb, np.int32), n, parts, block=block)
    assert b.shape == (parts + 1,) and b[0] == 0 and b[-1] == n and np.all(np.diff(b) >= 0)
    assert np.all((b[1:-1] % block == 0) | (b[1:-1] == n))
    edges = np.minimum(np.arange(nb + 1) * block, n)
    for r in range(1, parts):
        target = n * r / parts
        assert abs(b[r] - target) <= np.min(np.abs(edges - target)) + 1e-9
    assert int(np.count_nonzero(np.diff(b))) <= nb
    if n % block == 0 and nb % parts == 0:  # an exact split: equal ranges
        assert np.all(np.diff(b) == n // parts)


@pytest.mark.parametrize("kw", [dict(n_cols=-1), dict(block=0), dict(n_parts=0),
                                dict(w_all=0.0, w_active=0.0), dict(w_all=-1.0),
                                dict(count=200), dict(count=-1)])
def test_partition_rejects_bad_arguments(kw):
    import ctypes as C

    from paper_1711_00289_gb300 import _lib as L

    n, block = kw.get("n_cols", 1000), kw.get("block", 128)
    nb = max(1, -(-max(n, 1) // max(block, 1)))
    counts = np.zeros(nb, np.int32)
    if "count" in kw:
        counts[0] = kw["count"]
    bounds = np.full(kw.get("n_parts", 2) + 1 if kw.get("n_parts", 2) > 0 else 1, -7, np.int32)
    st = L.lib().conv_partition_columns(n, block, counts.ctypes.data, kw.get("w_all", 1.0),
                                        kw.get("w_active", 3.0), kw.get("n_parts", 2),
                                        bounds.ctypes.data)
    assert st == L.CONV_ERR_ARG
    assert np.all(bounds == -7)
    _ = C


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _grid():
    from paper_1711_00289_gb300 import soundings as S

    return S.clustered_grid(0.3, 48, 72)


def _sub(g, c0, c1):
    from paper_1711_00289_gb300 import soundings as S

    return S.Columns(g.name, g.pver, np.ascontiguousarray(g.T[:, c0:c1]),
                     np.ascontiguousarray(g.q[:, c0:c1]), g.ps[c0:c1].copy(), g.hyai, g.hybi)


def _rank(rank, world, port, block, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    from paper_1711_00289_gb300 import shard as SH

    g = _grid()
    n = g.n_cols
    b0 = SH.even_bounds(n, world, block)
    res = []
    for bounds in (b0, None):
        if bounds is None:  # second step: ranges from the first step's triggers
            bounds = SH.partition(cnt, n, world, block=block)
        c0, c1 = int(bounds[rank]), int(bounds[rank + 1])
        d, s = O.deep_shallow(_sub(g, c0, c1))
        nb = -(-(c1 - c0) // block)
        trig = (d["flags"] & O.F_TRIGGERED) > 0
        loc = np.array([trig[j * block:(j + 1) * block].sum() for j in range(nb)], np.int32)
        cnt = SH.global_counts(loc, c0, n, block)
        outs = [None] * world
        dist.all_gather_object(outs, (c0, c1, d, s))
        res.append((bounds.tolist(), cnt.tolist(), outs))
    out.put((rank, res))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo(oracle):
    import torch.multiprocessing as mp

    block = 128
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, block, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    g = _grid()
    n = g.n_cols
    ref_d, ref_s = oracle.deep_shallow(g)
    trig = (ref_d["flags"] & oracle.F_TRIGGERED) > 0
    want = np.array([trig[j * block:(j + 1) * block].sum() for j in range(-(-n // block))])
    for step in range(2):
        (b_a, c_a, o_a), (b_b, c_b, o_b) = res[0][step], res[1][step]
        assert b_a == b_b and c_a == c_b  # every rank computes the same ranges
        assert np.array_equal(c_a, want)  # the summed counts are the grid's
        # the ranks' ranges put together are the one-rank run, bit for bit
        for k in ref_d:
            got_d = np.concatenate([o[2][k] for o in o_a], axis=-1)
            got_s = np.concatenate([o[3][k] for o in o_a], axis=-1)
            assert np.array_equal(got_d, ref_d[k]) and np.array_equal(got_s, ref_s[k]), k
    # the second step's ranges balance the work better than the even first split
    c = _cost(want, n, block, shard.W_ALL, shard.W_ACTIVE)
    b1 = np.array(res[0][1][0])
    b0 = np.array(res[0][0][0])
    work = lambda b: [c[b[r] // block:-(-b[r + 1] // block)].sum() for r in range(2)]  # noqa: E731
    assert max(work(b1)) <= max(work(b0))
    assert abs(work(b1)[0] - work(b1)[1]) <= c.max()
