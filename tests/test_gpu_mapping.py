"""The trigger pass with one column per warp (conv_launch.mapping =
CONV_MAP_WARP; lane k takes level k) against the FP64 oracle and against the
default one-column-per-thread mapping, single grids and batched ensembles,
through the C ABI.

FP64: decisions bit-exact and values within 1e-10 of the oracle, and the same
against the thread mapping (the warp's height scan sums in another order, which
moves a near-cancelling CAPE or CIN sum by up to ~2e-11 relative; tendencies
agree far closer).  Mixed: within the mixed path's budget (its parcel
inversions start from the environment on every level instead of from the level
below).  Batches: the warp mapping set by hand equals the oracle (FP64) and the
autotuner's record times both mappings."""
import numpy as np
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


GRIDS = {
    "latlon": lambda: S.latlon_grid(96, 144, tau_range=(1800.0, 7200.0)),
    "clustered": lambda: S.clustered_grid(0.3, 96, 144),
    "random": lambda: _random_columns(7, n=3000),
    "levels26": lambda: S.clustered_grid(0.4, 24, 37, pver=26),
    "levels32": lambda: S.clustered_grid(0.4, 24, 37, pver=32),
}


@pytest.mark.parametrize("name", sorted(GRIDS))
def test_fp64_warp_mapping_matches_oracle(oracle, name):
    g = GRIDS[name]()
    rd, rs = oracle.deep_shallow(g, threads=THREADS)
    gd, gs = run_gpu(g, "fp64", "compact", ld=S.pad_ld(g.n_cols) + 32, mapping="warp")
    assert ((rd["flags"] & 2) > 0).sum() > 20
    assert_fp64_parity(gd, rd, what=f"deep warp {name}")
    assert_fp64_parity(gs, rs, what=f"shallow warp {name}")
    td, ts = run_gpu(g, "fp64", "compact", mapping="thread")
    assert_fp64_parity(gd, td, what=f"deep warp/thread {name}")
    assert_fp64_parity(gs, ts, what=f"shallow warp/thread {name}")


@pytest.mark.parametrize("name", ["clustered", "random"])
def test_mixed_warp_mapping_within_budget(oracle, name):
    g = GRIDS[name]()
    rd, rs = oracle.deep_shallow(g, threads=THREADS)
    gd, gs = run_gpu(g, "mixed", "compact", mapping="warp")
    for o in (rd, rs, gd, gs):
        o["flags"] = o["flags"] & ~8
    m = layer_mass(g)
    psurf = rd["prec"] + rs["prec"]
    for tag, got, ref, up in (("deep", gd, rd, None), ("shallow", gs, rs, same_decisions(gd, rd))):
        r = mixed_report(got, ref, m, up, psurf)
        check_mixed(r, f"{tag} warp {name}")


def test_full_resolution_fp64(oracle):
    """Every column of the 884,736-column benchmark grid, FP64, warp mapping."""
    g = S.clustered_grid(0.3)
    rd, rs = oracle.deep_shallow(g, threads=THREADS)
    gd, gs = run_gpu(g, "fp64", "compact", mapping="warp")
    assert_fp64_parity(gd, rd, what="deep warp full")
    assert_fp64_parity(gs, rs, what="shallow warp full")


def test_ragged_and_padding():
    """Column counts that leave the last block's warps idle, padded ld untouched."""
    for n in (1, 7, 9, 4099):
        g = S.column_set(n, seed=n)
        ld = S.pad_ld(n) + 32
        (gd, gs), (hd, hs) = run_gpu(g, "fp64", "compact", ld=ld, mapping="warp", sentinel=True)
        td, ts = run_gpu(g, "fp64", "compact", ld=ld, mapping="thread")
        assert_fp64_parity(gd, td, what=f"n={n}")
        assert_fp64_parity(gs, ts, what=f"n={n}")
        for h in (hd, hs):
            for k, v in h.items():
                tail = v[..., n:]
                assert np.all(tail == -7), (n, k)


def _members(precision, seed=42, n_members=8):
    import torch

    from paper_1711_00289_gb300 import api

    ens = S.ensemble(n_members, seed=seed, n_min=1, n_max=6000)
    rd = api.real_dtype(precision)
    mem = []
    for g in ens:
        mem.append(dict(T=torch.tensor(g.T, device="cuda").to(rd),
                        q=torch.tensor(g.q, device="cuda").to(rd),
                        ps=torch.tensor(g.ps, device="cuda"),
                        lam=torch.tensor(g.lam, device="cuda"),
                        vgrid=api.VerticalGrid(g.hyai, g.hybi), dt=g.dt))
    return ens, mem


def test_batch_warp_mapping(oracle):
    import torch

    from paper_1711_00289_gb300 import api

    ens, mem = _members("fp64", seed=7)
    b = api.Batch(mem, "fp64")
    assert b.set_config("warp", 128, 128)["trigger_mapping"] == "warp"
    outs = b.run()
    torch.cuda.synchronize()
    for g, (od, os_) in zip(ens, outs):
        rd, rs = oracle.deep_shallow(g, threads=THREADS, lam=g.lam)
        got = [{k: v.cpu().numpy() for k, v in o.items()} for o in (od, os_)]
        assert_fp64_parity(got[0], rd, what=f"batch deep {g.name}")
        assert_fp64_parity(got[1], rs, what=f"batch shallow {g.name}")
    b.close()


def test_autotuner_times_both_mappings():
    import torch

    from paper_1711_00289_gb300 import api

    _, mem = _members("mixed", seed=3)
    b = api.Batch(mem, "mixed")
    cfg = b.autotune(reps=2)
    rec = b.tune_record()
    assert cfg["trigger_mapping"] in ("thread", "warp")
    assert all(v > 0 for v in rec.values()), rec
    best_trigger = min(rec["trigger_thread_block_64"], rec["trigger_thread_block_128"],
                       rec["trigger_thread_block_256"], rec["trigger_warp_per_column"])
    chosen = (rec["trigger_warp_per_column"] if cfg["trigger_mapping"] == "warp" else
              rec[f"trigger_thread_block_{cfg['trigger_block']}"])
    assert chosen == best_trigger
    torch.cuda.synchronize()
    b.close()
