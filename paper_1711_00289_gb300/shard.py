"""One grid's columns over several GPUs, split by convective work.

The GPU counterpart of the paper's proportional partitioning of the column
computations between devices (Sec. IV-D).  The columns are independent, so each
rank runs the fused step on its own contiguous range of the grid, with no
exchange on the data path.  What differs between ranges is the work: the trigger
pass costs about the same on every column, the plume pass runs only where the
deep scheme triggers, and triggering columns cluster (ITCZ, storm systems).  So
after a step each rank counts the triggered columns of its range per block of
columns (conv_count_triggered), the ranks sum the counts (one small integer
all-reduce on the control path), and every rank computes the same new ranges
(conv_partition_columns) for the next step: contiguous, block-aligned, of
near-equal cost  w_all * columns + w_active * triggered columns.

Every rank keeps the whole grid's inputs and outputs here (a rank touches only
its range); a model that distributes its state would move the columns whose
owner changed.  The C-ABI calls do the arithmetic; this module only marshals
arguments and calls torch.distributed.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L

# Block of columns the counts and the range bounds are taken in.
BLOCK = 1024
# Cost of a triggered column's plume pass relative to one column's trigger pass:
# on the 884,736-column benchmark grid (mixed precision) the trigger pass takes
# 0.50 ms over all columns and the plume pass 0.46 ms over 265,421 triggered
# ones, i.e. 0.57 and 1.73 ns per column.
W_ALL, W_ACTIVE = 1.0, 3.0


def partition(block_triggered, n_cols: int, n_parts: int, *, block: int = BLOCK,
              w_all: float = W_ALL, w_active: float = W_ACTIVE) -> np.ndarray:
    """Range bounds [n_parts + 1] (host int32) from per-block triggered counts."""
    cnt = np.ascontiguousarray(block_triggered, dtype=np.int32)
    nb = -(-int(n_cols) // int(block))
    if cnt.shape != (nb,):
        raise ValueError(f"need {nb} block counts, got {cnt.shape}")
    bounds = np.zeros(int(n_parts) + 1, dtype=np.int32)
    st = L.lib().conv_partition_columns(int(n_cols), int(block), cnt.ctypes.data, float(w_all),
                                        float(w_active), int(n_parts), bounds.ctypes.data)
    L.check(st, "conv_partition_columns")
    return bounds


def even_bounds(n_cols: int, n_parts: int, block: int = BLOCK) -> np.ndarray:
    """The first step's ranges, before any trigger count is known: equal block
    counts."""
    return partition(np.zeros(-(-int(n_cols) // int(block)), np.int32), n_cols, n_parts,
                     block=block, w_all=1.0, w_active=0.0)


def count_triggered(flags, n_cols: int, col0: int = 0, block: int = BLOCK, out=None,
                    stream=None):
    """Per-block triggered counts of the deep flags of columns col0 .. col0 +
    n_cols - 1 (a CUDA int32 tensor of the grid, col0 a multiple of block): a
    CUDA int32 tensor of ceil(n_cols / block) entries."""
    import torch

    if not (flags.is_cuda and flags.dtype == torch.int32 and flags.is_contiguous()):
        raise TypeError("flags must be a contiguous CUDA int32 tensor")
    if col0 % block or col0 < 0 or col0 + n_cols > flags.numel():
        raise ValueError("range outside flags or not block-aligned")
    nb = -(-int(n_cols) // int(block))
    if out is None:
        out = torch.empty(nb, dtype=torch.int32, device=flags.device)
    s = torch.cuda.current_stream() if stream is None else stream
    st = L.lib().conv_count_triggered(C.c_void_p(flags.data_ptr() + 4 * col0), int(n_cols),
                                      int(block), C.c_void_p(out.data_ptr()),
                                      C.c_void_p(s.cuda_stream))
    L.check(st, "conv_count_triggered")
    return out


def global_counts(local_counts, col0: int, n_cols: int, block: int = BLOCK, group=None,
                  device=None):
    """Sum every rank's per-block counts of its own (block-aligned) range into the
    grid's per-block counts (an all-reduce of ceil(n_cols / block) int32s; the
    ranges are disjoint, so the sum places each rank's counts).  Returns a host
    numpy array, identical on every rank."""
    import torch
    import torch.distributed as dist

    nb = -(-int(n_cols) // int(block))
    dev = device if device is not None else (
        local_counts.device if isinstance(local_counts, torch.Tensor) else torch.device("cpu"))
    full = torch.zeros(nb, dtype=torch.int32, device=dev)
    loc = torch.as_tensor(local_counts, dtype=torch.int32, device=dev)
    j0 = col0 // block
    full[j0:j0 + loc.numel()] = loc
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(full, op=dist.ReduceOp.SUM, group=group)
    return full.cpu().numpy()


class ShardedStep:
    """The fused step on this rank's range of a grid split over the ranks of a
    process group (one GPU per rank).  ``run()`` advances the rank's range;
    ``rebalance()`` (between steps) recomputes every rank's range from the
    triggered columns of the last run."""

    def __init__(self, T, q, ps, vgrid, *, rank: int, world: int, dt: float = 1800.0,
                 precision: str = "mixed", out_deep=None, out_shallow=None, group=None,
                 block: int = BLOCK, **kw):
        from . import api

        self.api = api
        self.T, self.q, self.ps, self.vgrid = T, q, ps, vgrid
        self.n = T.shape[1]
        self.rank, self.world, self.group, self.block = rank, world, group, block
        self.dt, self.precision, self.kw = dt, precision, kw
        pver = T.shape[0]
        self.out_deep = out_deep if out_deep is not None else api.new_outputs(
            pver, self.n, precision, T.device)
        self.out_shallow = out_shallow if out_shallow is not None else api.new_outputs(
            pver, self.n, precision, T.device)
        self.bounds = even_bounds(self.n, world, block)

    @property
    def range(self):
        return int(self.bounds[self.rank]), int(self.bounds[self.rank + 1])

    def run(self, stream=None):
        c0, c1 = self.range
        if c1 > c0:
            self.api.deep_shallow(self.T, self.q, self.ps, self.vgrid, dt=self.dt,
                                  precision=self.precision, col0=c0, n_cols=c1 - c0,
                                  out_deep=self.out_deep, out_shallow=self.out_shallow,
                                  stream=stream, **self.kw)
        return self.out_deep, self.out_shallow

    def rebalance(self):
        c0, c1 = self.range
        loc = count_triggered(self.out_deep["flags"], c1 - c0, c0, self.block)
        cnt = global_counts(loc, c0, self.n, self.block, self.group, device=loc.device)
        self.bounds = partition(cnt, self.n, self.world, block=self.block)
        return self.bounds
