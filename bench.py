"""Benchmark: deep + shallow column convection over 884,736 columns x 30 levels.

One step = one call of the fused deep->shallow path over the whole grid (the
768 x 1152 resolution of the paper's R3 grid, Sec. V-A, with a clustered 30%
convecting fraction), inputs resident in HBM (202 MB of FP32 / 405 MB of FP64
profiles, larger than the 129 MB L2, so no L2 flush is needed between steps).
Default: the mixed-precision compacted path; the plain FP64 kernel is timed
beside it (the metric's reference point).

Arms:
  default              the CUDA library (libconvgb.so) through the C ABI;
  --impl reference     the FP64 CPU oracle on this machine's cores (OpenMP,
                       dynamic schedule) over a bounded sample of the grid.

Prints one JSON line (rank 0).  Multi-GPU (torchrun): every rank processes its
own full grid, no collective on the data path ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "convection columns/s (deep+shallow, 884,736x30)"
UNIT = "columns/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    p.add_argument("--path", default="compact", choices=["plain", "compact"])
    p.add_argument("--no-baseline", action="store_true",
                   help="skip timing the plain FP64 kernel beside the measured path")
    p.add_argument("--frac", type=float, default=0.30)
    p.add_argument("--nlat", type=int, default=768)
    p.add_argument("--nlon", type=int, default=1152)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-transport", action="store_true",
                   help="skip the tracer-transport measurement")
    p.add_argument("--no-driver", action="store_true",
                   help="skip the multi-step driver measurement")
    p.add_argument("--no-adjoint", action="store_true",
                   help="skip the deep-adjoint timing")
    p.add_argument("--no-sweep", action="store_true",
                   help="skip the 10/30/60%% convecting-fraction sweep")
    p.add_argument("--no-ensemble", action="store_true",
                   help="skip the batched 64-member ensemble measurement")
    return p.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ roofline
def op_counts(frac: float):
    """Per-column algorithmic operation counts (oracle counting instantiation,
    oracle/op_counts.json) of the clustered workload with this convecting
    fraction; per-column counts do not depend on the grid size."""
    path = os.path.join(ROOT, "oracle", "op_counts.json")
    with open(path) as fh:
        w = json.load(fh)["workloads"]
    key = min((k for k in w if k.startswith("clustered")),
              key=lambda k: abs(float(k.rsplit("-f", 1)[1]) - frac))
    return w[key], key


def device_rates(L):
    """Measured evaluations/s per operation class on this device."""
    r = {}
    for name, arith in (("fp64", L.CONV_ARITH_FP64), ("fp32", L.CONV_ARITH_FP32_FAST)):
        for op, k in ((L.CONV_OP_FMA, "fma"), (L.CONV_OP_EXP, "exp"), (L.CONV_OP_LOG, "log"),
                      (L.CONV_OP_DIV, "div"), (L.CONV_OP_POW, "pow")):
            r[f"{name}_{k}"] = L.op_rate(op, arith)
    return r


def t_ops(c, r, pfx):
    """Lower-bound time of an operation mix at measured rates (adds and multiplies
    paired into FMAs, each other class at its own measured throughput)."""
    return (max(c["add"], c["mul"]) / r[pfx + "fma"] + c["div"] / r[pfx + "div"]
            + c["exp"] / r[pfx + "exp"] + c["log"] / r[pfx + "log"] + c["pow"] / r[pfx + "pow"])


# FP64 work of one FP64 LCL correction of the mixed design (residual, relative
# humidity and LCL pressure): 1 log, 1 exp, 4 div, 27 FMA.  It runs only for LCL
# solves whose FP32 pressure lies within the decision band of a layer or of the
# E1 threshold (fp64_lcl_corrections, counted from the oracle's LCL pressures by
# oracle/count_ops.py).  One FP64 drizzle correction (q_s and dq_s/dT at the FP32
# saturation temperature, one Newton correction, q_s at the result): 2 exp,
# 6 div, 24 FMA, on the saturated shallow plume layers whose rain lies within
# 1e-4 kg/kg of zero (fp64_drizzle).  The CAPE, CIN and conservation sums keep
# their accuracy as compensated FP32 sums; their terms are FP32 work, already in
# the oracle's operation counts (one add per term; the compensation's extra adds
# are not counted as work).
def t_fp64_islands(c, r):
    lcl = (1 / r["fp64_log"] + 1 / r["fp64_exp"] + 4 / r["fp64_div"] + 27 / r["fp64_fma"])
    drizzle = 2 / r["fp64_exp"] + 6 / r["fp64_div"] + 24 / r["fp64_fma"]
    return c["fp64_lcl_corrections"] * lcl + c.get("fp64_drizzle", 0.0) * drizzle


# Nominal ALU peaks from unit counts and clocks: 152 SMs at the 2070 MHz maximum
# SM clock; per SM and clock 128 FP32 FMA lanes and 2 FP64 FMA units (the
# latter give 1.26 TFLOP/s, GB300's quoted FP64 rate).
SMS, SM_MHZ = 152, 2070.0
FMA_PER_SM_CLOCK = {"fp32": 128, "fp64": 2}


def nominal_fma_rate(pipe):
    """FMAs per second of a pipe at the maximum SM clock."""
    return SMS * FMA_PER_SM_CLOCK[pipe] * SM_MHZ * 1e6


def kernel_roofline(counts, precision, kernel_s, n_cols, r):
    """Arithmetic roofline of one kernel.  Its algorithmic work is weighed in
    FMA-equivalents on the binding pipe (each operation class at its cost
    relative to an FMA, from the measured per-operation throughputs r); the
    achieved rate of that work is compared with the pipe's nominal FMA peak
    (unit counts x clock), and with its measured FMA rate beside it.  FP64 path:
    every operation on the FP64 pipe.  Mixed path: the bulk on the FP32 pipes
    (fast intrinsic rates, the lowest bound) and the FP64 islands on the FP64
    pipe; the larger of the two binds."""
    if precision == "fp64":
        t64, t32 = t_ops(counts, r, "fp64_") * n_cols, 0.0
    else:
        t64, t32 = t_fp64_islands(counts, r) * n_cols, t_ops(counts, r, "fp32_") * n_cols
    fp64_binds = t64 >= t32
    pipe = "fp64" if fp64_binds else "fp32"
    t_bound = t64 if fp64_binds else t32  # the work's time at the measured rates
    measured = 2.0 * r[pipe + "_fma"]  # FLOP/s
    peak = 2.0 * nominal_fma_rate(pipe)
    achieved = measured * t_bound / kernel_s  # FMA-equivalent FLOP/s of the work
    return {"bound": "alu", "binding_pipe": pipe,
            "achieved": achieved / 1e12, "peak": peak / 1e12,
            "unit": "TFLOP/s (FMA-equivalent on the binding pipe)",
            "frac": achieved / peak, "peak_measured": measured / 1e12,
            "frac_of_measured": t_bound / kernel_s,
            "t_bound_fp64_ms": t64 * 1e3, "t_bound_fp32_ms": t32 * 1e3,
            "t_bound_ms": t_bound * 1e3, "kernel_ms": kernel_s * 1e3, "traffic": None,
            "peak_source": (f"{SMS} SMs x {FMA_PER_SM_CLOCK[pipe]} {pipe.upper()} FMA per "
                            f"clock x 2 FLOP x {SM_MHZ:.0f} MHz (unit counts and maximum SM "
                            "clock); peak_measured: this device's FMA rate "
                            "(conv_bench_op_rate)")}


def hbm_bytes_per_column(pver, real_bytes):
    # read T, q, ps; write deep and shallow dTdt, dqdt; 4 doubles + 5 int32 per scheme
    return 2 * pver * real_bytes + 8 + 4 * pver * real_bytes + 2 * (4 * 8 + 5 * 4)


OP_CATS = ("add", "mul", "div", "exp", "log", "pow", "sqrt")


def path_rooflines(counts, prec, path, kern_ms, n, r):
    """Per-kernel arithmetic rooflines of one measured step.  Plain path: one
    kernel doing the whole step.  Compacted path: the trigger pass (all columns)
    and the plume pass (queued columns).  The trigger pass's headline work leaves
    out the shallow LFC search of the columns that end at exit E2, which the
    kernel settles by bounds instead (trigger_pass_e2_search_per_column); the
    figure with that search counted is reported beside it."""
    kernels = {}
    if path == "plain":
        tot = {c: counts["trigger_pass_per_column"][c] + counts["plume_pass_per_column"][c]
               for c in counts["trigger_pass_per_column"]}
        if prec == "fp64":
            tot.update(counts["total_per_column"])
        kernels["k_plain"] = kernel_roofline(tot, prec, kern_ms[0] * 1e-3, n, r)
        kernels["k_plain"]["share"] = 1.0
        return kernels
    kt, kp = kern_ms
    trig = dict(counts["trigger_pass_per_column"])
    e2 = counts.get("trigger_pass_e2_search_per_column", {})
    net = {c: (trig[c] - e2.get(c, 0.0)) if c in OP_CATS else trig[c] for c in trig}
    kernels["k_trigger"] = kernel_roofline(net, prec, kt * 1e-3, n, r)
    gross = kernel_roofline(trig, prec, kt * 1e-3, n, r)
    kernels["k_trigger"]["with_e2_search_counted"] = {
        k: gross[k] for k in ("frac", "frac_of_measured", "t_bound_ms")}
    kernels["k_plume"] = kernel_roofline(counts["plume_pass_per_column"], prec, kp * 1e-3, n, r)
    kernels["k_trigger"]["share"] = kt / (kt + kp)
    kernels["k_plume"]["share"] = kp / (kt + kp)
    return kernels


def step_roofline(kernels, step_ms):
    """The whole step against the same arithmetic roofline: the kernels' bound
    times summed, over the measured step time (gaps and small launches between
    the kernels included)."""
    t_bound = sum(k["t_bound_ms"] for k in kernels.values())
    achieved_nominal = sum(k["t_bound_ms"] * k["peak_measured"] / k["peak"]
                           for k in kernels.values()) / step_ms
    return {"t_bound_ms": t_bound, "step_ms": step_ms, "frac_of_measured": t_bound / step_ms,
            "frac": achieved_nominal,
            "note": "sum of the kernels' bound times at measured rates / step time "
                    "(frac: the same at nominal FMA peaks)"}


# ------------------------------------------------------------------ CPU oracle
def cpu_oracle_rate(g, budget_s):
    """Columns/s of the FP64 oracle on all host cores over a strided sample of g."""
    from oracle import oracle as O
    from paper_1711_00289_gb300 import soundings as S

    threads = os.cpu_count() or 1

    def sample(stride):
        return S.Columns(g.name, g.pver, np.ascontiguousarray(g.T[:, ::stride]),
                         np.ascontiguousarray(g.q[:, ::stride]), g.ps[::stride].copy(),
                         g.hyai, g.hybi)

    probe = sample(max(1, g.n_cols // 20000))
    t0 = time.perf_counter()
    O.deep_shallow(probe, threads=threads)
    rate = probe.n_cols / (time.perf_counter() - t0)
    want = min(g.n_cols, max(probe.n_cols, int(rate * budget_s)))
    sub = sample(max(1, g.n_cols // want))
    # repeat the sample until the time budget is spent (the whole grid may take
    # well under it on a many-core host)
    done, t0 = 0, time.perf_counter()
    while True:
        O.deep_shallow(sub, threads=threads)
        done += sub.n_cols
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return done / el, done, threads, el


def cpu_model():
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ------------------------------------------------------------------ arms
def max_over_ranks(x, world, dev):
    """The largest of a value over all ranks (the slowest rank's time): an
    all-reduce MAX on the process group (NCCL on GPUs, gloo on CPU)."""
    if world <= 1:
        return x
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, n_cols, ms):
    """Columns per second of the whole job: every rank advances its own copy of
    the grid (replicas, weak scaling), timed by the slowest rank."""
    return world * n_cols / (ms * 1e-3)


def reference_arm(args, rank):
    from oracle import oracle as O  # noqa: F401  (reference arm = the oracle)
    from paper_1711_00289_gb300 import soundings as S

    if rank != 0:
        return
    g = S.clustered_grid(args.frac, args.nlat, args.nlon)
    per_step = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    vals = []
    for i in range(args.warmup + args.steps):
        rate, ncols, threads, el = cpu_oracle_rate(g, per_step)
        if i >= args.warmup:
            vals.append(rate)
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * g.n_cols / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": g.name, "columns": g.n_cols, "levels": g.pver,
                       "convecting_fraction": args.frac, "dt_s": g.dt},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{ncols} column evaluations per step (strided sample of the grid, "
                                       f"repeated), OpenMP dynamic(8) on {threads} threads, "
                                       f"{cpu_model()}"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def ours_arm(args, rank, world, local_rank):
    import torch

    from paper_1711_00289_gb300 import _lib as L
    from paper_1711_00289_gb300 import api
    from paper_1711_00289_gb300 import soundings as S

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    g = S.clustered_grid(args.frac, args.nlat, args.nlon)
    n, pver = g.n_cols, g.pver
    vg = api.VerticalGrid(g.hyai, g.hybi)
    stream = torch.cuda.current_stream(dev)
    ws = api.Workspace(dev)
    bufs = {}

    def setup(grid, prec):
        key = (grid.name, prec)
        if key not in bufs:
            rd = api.real_dtype(prec)
            bufs[key] = (torch.tensor(grid.T, device=dev).to(rd),
                         torch.tensor(grid.q, device=dev).to(rd),
                         torch.tensor(grid.ps, device=dev),
                         api.new_outputs(grid.pver, grid.n_cols, prec, dev),
                         api.new_outputs(grid.pver, grid.n_cols, prec, dev))
        return bufs[key]

    preps = {}

    def prepared(grid, prec, path, mapping="auto"):
        # the step's C-ABI arguments marshalled once (api.PreparedStep): a timed
        # step is one library call, so the loop measures the GPU, not Python
        key = (grid.name, prec, path, mapping)
        if key not in preps:
            T, q, ps, od, os_ = setup(grid, prec)
            preps[key] = api.PreparedStep(T, q, ps, api.VerticalGrid(grid.hyai, grid.hybi),
                                          dt=grid.dt, precision=prec, path=path, out_deep=od,
                                          out_shallow=os_, workspace=ws, stream=stream,
                                          mapping=mapping)
        return preps[key]

    def timed(grid, prec, path, steps, warmup, per_kernel, mapping="auto"):
        run = prepared(grid, prec, path, mapping)
        for _ in range(warmup):
            run()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        if per_kernel:
            for e3 in evs:  # materialise the CUDA events outside the timed region
                for e in e3:
                    e.record(stream)
        lcs = [run.launch_struct(evs[s_] if per_kernel else None) for s_ in range(steps)]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        e0.record(stream)
        for s_ in range(steps):
            run(lcs[s_])
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        kern = None
        if per_kernel:
            kern = (statistics.mean(e[0].elapsed_time(e[1]) for e in evs),
                    statistics.mean(e[1].elapsed_time(e[2]) for e in evs))
        return ms, kern

    def soak(grid, prec, path, seconds):
        # the step run untimed for `seconds` right before the timed steps, so
        # that the clock samples (nvidia-smi every 100 ms, longer than a short
        # timed region) see the GPU under this load; returns the steps run
        run = prepared(grid, prec, path)
        n = 0
        t_end = time.perf_counter() + seconds
        while time.perf_counter() < t_end:
            for _ in range(20):
                run()
            torch.cuda.synchronize()
            n += 20
        return n

    prec, path = args.precision, args.path
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    n_soak = soak(g, prec, path, 0.6)
    ms, kern = timed(g, prec, path, args.steps, args.warmup, True)
    clk = clocks.stop()
    clk["window"] = ("nvidia-smi every 100 ms from 0.3 s before a 0.6 s untimed run "
                     f"of the same step ({n_soak} steps) through the warm-up and timed steps")
    ms = max_over_ranks(ms, world, dev)
    value = whole_job_value(world, n, ms)
    od = setup(g, prec)[3]
    act = int(((od["flags"] & 2) > 0).sum().item())

    # the plain FP64 kernel, the reference point of the metric
    base = None
    bkern = None
    if not args.no_baseline and not (prec == "fp64" and path == "plain"):
        bms, bkern = timed(g, "fp64", "plain", max(2, min(args.steps, 5)), 2, True)
        bms = max_over_ranks(bms, world, dev)
        base = {"value": whole_job_value(world, n, bms), "unit": UNIT, "ms_per_step": bms,
                "path": "plain", "precision": "fp64"}

    # the same path at the other convecting fractions of the 884,736-column
    # workload (each its own grid; the headline value stays at args.frac)
    sweep = []
    if not args.no_sweep:
        for f in (0.10, 0.30, 0.60):
            if abs(f - args.frac) < 1e-9:
                sweep.append({"convecting_fraction": f, "ms_per_step": ms, "kern_ms": kern,
                              "deep_active_columns": act, "columns": n})
                continue
            gf = S.clustered_grid(f, args.nlat, args.nlon)
            msf, kf = timed(gf, prec, path, args.steps, args.warmup, True)
            msf = max_over_ranks(msf, world, dev)
            actf = int(((setup(gf, prec)[3]["flags"] & 2) > 0).sum().item())
            sweep.append({"convecting_fraction": f, "ms_per_step": msf, "kern_ms": kf,
                          "deep_active_columns": actf, "columns": gf.n_cols})
            del bufs[(gf.name, prec)], preps[(gf.name, prec, path, "auto")]
            torch.cuda.empty_cache()

    # the trigger pass's other mapping (one column per warp) on the same step
    alt = None
    if path == "compact" and not args.no_sweep:
        msw, kw_ = timed(g, prec, path, args.steps, args.warmup, True, mapping="warp")
        alt = {"thread_per_column": {"ms_per_step": ms, "k_trigger_ms": kern[0]},
               "warp_per_column": {"ms_per_step": msw, "k_trigger_ms": kw_[0]},
               "chosen": "thread_per_column" if ms <= msw else "warp_per_column"}

    # end to end through the public API from pinned host buffers: the host
    # pipeline (conv_pipeline_run) copies the inputs in, runs the fused step and
    # copies every output back, chunk by chunk with the copies overlapping
    e2e = None
    if not args.no_e2e:
        T, q, ps, od_, os__ = setup(g, prec)
        hT, hq, hps = (x.cpu().pin_memory() for x in (T, q, ps))
        hd, hs = api.new_host_outputs(pver, n, prec), api.new_host_outputs(pver, n, prec)
        pipe = api.HostPipeline(vg, n, n, prec)

        def e2e_step():
            pipe.run(hT, hq, hps, hd, hs, dt=g.dt, stream=stream)

        for _ in range(max(3, args.warmup)):
            e2e_step()
        k2 = args.steps
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(k2 + 1)]
        for e in ev:  # materialise the events outside the timed region
            e.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ev[0].record(stream)
        for s_ in range(k2):
            e2e_step()
            ev[s_ + 1].record(stream)
        torch.cuda.synchronize()
        ms2 = max_over_ranks(ev[0].elapsed_time(ev[-1]) / k2, world, dev)
        per = [ev[i].elapsed_time(ev[i + 1]) for i in range(k2)]
        h2d = sum(x.numel() * x.element_size() for x in (hT, hq, hps))
        d2h = sum(v.numel() * v.element_size() for o in (hd, hs) for v in o.values())
        e2e = {"value": whole_job_value(world, n, ms2), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": ms2,
               "ms_median": statistics.median(per), "ms_min": min(per), "ms_max": max(per),
               "ms_steps": per,
               "path": "conv_pipeline_run (host buffers, chunked copies overlapping compute)"}
        pipe.close()

    if rank != 0:
        return
    counts, key = op_counts(args.frac)
    r = device_rates(L)
    kernels = path_rooflines(counts, prec, path, kern, n, r)
    traffic = ncu_traffic(g.name)
    for k in kernels:
        kernels[k]["traffic"] = traffic.get(k)
    dom = max(kernels, key=lambda k: kernels[k]["share"])
    roof = dict(kernels[dom])
    roof["kernel"] = dom
    roof["op_counts_workload"] = key
    roof["step"] = step_roofline(kernels, ms)
    rb = 8 if prec == "fp64" else 4
    roof["hbm_algorithmic_bytes_per_column"] = hbm_bytes_per_column(pver, rb)
    hbm_peak, hbm_src = measured_hbm()
    roof["hbm_frac_of_measured_path"] = (hbm_bytes_per_column(pver, rb) * n / (ms * 1e-3) / 1e9
                                         / hbm_peak)
    roof["hbm_peak_source"] = hbm_src
    if base is not None:
        bk = path_rooflines(counts, "fp64", "plain", bkern, n, r)
        base["roofline"] = dict(bk["k_plain"], kernel="k_plain", op_counts_workload=key,
                                step=step_roofline(bk, base["ms_per_step"]))
        base["roofline"]["traffic"] = traffic.get("k_plain_fp64")
    for row in sweep:
        cf, kf_ = op_counts(row["convecting_fraction"])
        kk = path_rooflines(cf, prec, path, row.pop("kern_ms"), row["columns"], r)
        row["value"] = whole_job_value(world, row["columns"], row["ms_per_step"])
        row["unit"] = UNIT
        row["op_counts_workload"] = kf_
        row["kernels"] = {k: {x: v[x] for x in ("kernel_ms", "frac", "frac_of_measured",
                                                 "t_bound_ms", "binding_pipe")}
                          for k, v in kk.items()}
        row["step"] = step_roofline(kk, row["ms_per_step"])
    ens = None if args.no_ensemble else ensemble_bench(args, dev, r)
    adj = None if args.no_adjoint else adjoint_bench(args, dev, g)
    trn = None if args.no_transport else transport_bench(args, dev, g)
    drv = None if args.no_driver else driver_bench(args, dev, g)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        rate, ncols, threads, el = cpu_oracle_rate(g, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{ncols} column evaluations of this grid (strided sample, repeated) "
                         f"in {el:.1f} s, FP64 oracle, OpenMP dynamic(8) on {threads} threads, "
                         f"{cpu_model()}"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": g.name, "columns": n, "levels": pver,
                       "convecting_fraction": args.frac, "deep_active_columns": act,
                       "precision": prec, "path": path, "dt_s": g.dt,
                       "l2": l2_note(prec, n, pver), "parallelism": f"replicas x{world}"},
            "baseline_fp64_plain": base,
            "speedup_vs_fp64_plain": (value / base["value"]) if base else None,
            "roofline": roof, "kernels": kernels, "convecting_fraction_sweep": sweep,
            "trigger_mapping": alt,
            "batched_ensemble": ens, "deep_adjoint": adj,
            "tracer_transport": trn, "column_driver": drv,
            "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clk, "gpu_launches": (1 if path == "plain" else 2) * args.steps,
            "op_rates_per_s": r}
    print(json.dumps(line), flush=True)


def ensemble_bench(args, dev, rates=None):
    """64 members, log-uniform 1,000-200,000 columns, 26/30/32 levels, member
    surface-T offsets and entrainment rates: one batched run (trigger launch +
    persistent plume launch), autotuned, captured in a CUDA graph and replayed.
    Its arithmetic roofline: the ensemble's counted work (oracle/op_counts.json,
    workload ensemble-64) against the two kernels' times from eager runs with
    stage events, and against the graph-replayed step."""
    import torch

    from paper_1711_00289_gb300 import api
    from paper_1711_00289_gb300 import soundings as S

    ens = S.ensemble(64)
    mem = []
    for g in ens:
        mem.append(dict(T=torch.tensor(g.T, device=dev).float(),
                        q=torch.tensor(g.q, device=dev).float(),
                        ps=torch.tensor(g.ps, device=dev),
                        lam=torch.tensor(g.lam, device=dev), vgrid=api.VerticalGrid(g.hyai, g.hybi),
                        dt=g.dt))
    b = api.Batch(mem, "mixed", device=dev)
    cfg = b.autotune(reps=2)
    tune = b.tune_record()
    b.ws.get(b.workspace_bytes())
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        b.run(stream=s)
    for _ in range(max(3, args.warmup)):
        graph.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cur = torch.cuda.current_stream(dev)
    e0.record(cur)
    for _ in range(args.steps):
        graph.replay()
    e1.record(cur)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    total = sum(g.n_cols for g in ens)
    active = sum(int(((o[0]["flags"] & 2) > 0).sum().item()) for o in b.outputs)
    # per-kernel times: eager runs on the same stream with stage events
    kev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    for e3 in kev:
        for e in e3:
            e.record(s)
    torch.cuda.synchronize()
    for e3 in kev:
        b.run(stream=s, stage_events=e3)
    torch.cuda.synchronize()
    kt = statistics.mean(e[0].elapsed_time(e[1]) for e in kev)
    kp = statistics.mean(e[1].elapsed_time(e[2]) for e in kev)
    b.close()
    roof = None
    if rates is not None:
        with open(os.path.join(ROOT, "oracle", "op_counts.json")) as fh:
            cnt = json.load(fh)["workloads"].get("ensemble-64")
        if cnt is not None:
            kk = path_rooflines(cnt, "mixed", "compact", (kt, kp), total, rates)
            kk = {"k_batch_trigger": kk["k_trigger"], "k_batch_plume": kk["k_plume"]}
            dom = max(kk, key=lambda k: kk[k]["share"])
            roof = dict(kk[dom], kernel=dom, op_counts_workload="ensemble-64",
                        kernels={k: {x: v[x] for x in ("kernel_ms", "frac", "frac_of_measured",
                                                        "t_bound_ms", "share")}
                                 for k, v in kk.items()},
                        step=step_roofline(kk, ms))
    # the same members one after another through the single-grid compacted
    # kernels (three launches each), also replayed from a CUDA graph
    runs = []
    for m in mem:
        w = api.Workspace(dev)
        out = (api.new_outputs(m["T"].shape[0], m["T"].shape[1], "mixed", dev),
               api.new_outputs(m["T"].shape[0], m["T"].shape[1], "mixed", dev))
        runs.append((m, w, out))
        api.deep_shallow(m["T"], m["q"], m["ps"], m["vgrid"], dt=m["dt"], precision="mixed",
                         lam=m["lam"], path="compact", workspace=w, out_deep=out[0],
                         out_shallow=out[1])
    torch.cuda.synchronize()
    graph2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph2, stream=s):
        for m, w, out in runs:
            api.deep_shallow(m["T"], m["q"], m["ps"], m["vgrid"], dt=m["dt"], precision="mixed",
                             lam=m["lam"], path="compact", workspace=w, out_deep=out[0],
                             out_shallow=out[1], stream=s)
    for _ in range(3):
        graph2.replay()
    torch.cuda.synchronize()
    e0.record(cur)
    for _ in range(args.steps):
        graph2.replay()
    e1.record(cur)
    torch.cuda.synchronize()
    ms_sep = e0.elapsed_time(e1) / args.steps
    return {"members": len(ens), "columns": total, "levels": sorted({g.pver for g in ens}),
            "deep_active_columns": active, "precision": "mixed", "ms_per_step": ms,
            "value": total / (ms * 1e-3), "unit": UNIT, "launch": "CUDA graph replay",
            "autotuned_shape": cfg, "autotune_ms_per_run": tune, "gpu_launches_per_step": 2,
            "members_one_after_another_ms": ms_sep, "roofline": roof}


def adjoint_bench(args, dev, g_full):
    """Deep-scheme adjoint (FP64): gradient of J = P + H w.r.t. T, q, lambda, tau
    against the FP64 forward deep scheme on the same columns (plain kernel), and
    the fused deep -> shallow step adjoint against the FP64 forward step, on the
    13,824 x 30 lat-lon grid and on the benchmark grid."""
    import torch

    from paper_1711_00289_gb300 import api
    from paper_1711_00289_gb300 import soundings as S

    def ev_time(fn, reps):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        cur = torch.cuda.current_stream(dev)
        e0.record(cur)
        for _ in range(reps):
            fn()
        e1.record(cur)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    res = {}
    for name, g, reps in (("latlon-96x144x30", S.latlon_grid(96, 144, tau_range=(1800.0, 7200.0)),
                           max(3, args.steps)),
                          (g_full.name, g_full, 2)):
        n = g.n_cols
        T = torch.tensor(g.T, device=dev)
        q = torch.tensor(g.q, device=dev)
        ps = torch.tensor(g.ps, device=dev)
        tau = None if g.tau is None else torch.tensor(g.tau, device=dev)
        vg = api.VerticalGrid(g.hyai, g.hybi)
        one = torch.ones(n, dtype=torch.float64, device=dev)
        out = api.new_outputs(g.pver, n, "fp64", dev)
        fwd = ev_time(lambda: api.deep(T, q, ps, vg, dt=g.dt, precision="fp64", tau=tau,
                                       path="plain", out=out), reps)
        adj = ev_time(lambda: api.deep_adjoint(T, q, ps, vg, gP=one, gH=one, dt=g.dt, tau=tau),
                      reps)
        active = int(((out["flags"] & 2) > 0).sum().item())
        # fused deep -> shallow step: adjoint against the FP64 plain forward step
        od, os_ = api.new_outputs(g.pver, n, "fp64", dev), api.new_outputs(g.pver, n, "fp64", dev)
        fwd2 = ev_time(lambda: api.deep_shallow(T, q, ps, vg, dt=g.dt, precision="fp64", tau=tau,
                                                path="plain", out_deep=od, out_shallow=os_), reps)
        adj2 = ev_time(lambda: api.deep_shallow_adjoint(T, q, ps, vg, gPd=one, gHd=one, gPs=one,
                                                        gHs=one, dt=g.dt, tau=tau), reps)
        res[name] = {"columns": n, "deep_active_columns": active, "ms_adjoint": adj,
                     "ms_forward_fp64_plain": fwd, "adjoint_over_forward": adj / fwd,
                     "value": n / (adj * 1e-3), "unit": UNIT, "gpu_launches_per_call": 1,
                     "step": {"ms_adjoint": adj2, "ms_forward_fp64_plain": fwd2,
                              "adjoint_over_forward": adj2 / fwd2,
                              "value": n / (adj2 * 1e-3), "unit": UNIT}}
    return res


def transport_bench(args, dev, g, ntr=25):
    """Convective tracer transport of ``ntr`` tracers by the fused step's plumes
    (mixed precision, FP32 tracers) on the benchmark grid: the transport kernel
    timed alone with CUDA events, its algorithmic HBM bytes counted from the
    plumes' extents (tendencies written everywhere; tracers read on the levels
    a plume touches; mass-flux profiles, flags and levels once per column), and
    the fused step with and without the profile outputs and with the scheme
    variants (shallow rain evaporation, deep plume spectrum)."""
    import torch

    from paper_1711_00289_gb300 import _lib as L
    from paper_1711_00289_gb300 import api

    n, pver = g.n_cols, g.pver
    vg = api.VerticalGrid(g.hyai, g.hybi)
    T = torch.tensor(g.T, device=dev).float()
    q = torch.tensor(g.q, device=dev).float()
    ps = torch.tensor(g.ps, device=dev)
    tau = None if g.tau is None else torch.tensor(g.tau, device=dev)
    ws = api.Workspace(dev)
    od = api.new_outputs(pver, n, "mixed", dev, flux=True)
    os_ = api.new_outputs(pver, n, "mixed", dev, flux=True)
    od0 = api.new_outputs(pver, n, "mixed", dev)
    os0 = api.new_outputs(pver, n, "mixed", dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(20171106)
    tr = torch.rand((ntr, pver, n), device=dev, generator=gen)
    td, ts = torch.empty_like(tr), torch.empty_like(tr)
    cur = torch.cuda.current_stream(dev)

    def ev_time(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        for _ in range(reps):
            fn()
        e1.record(cur)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    reps = max(3, args.steps)
    step_flux = ev_time(api.PreparedStep(T, q, ps, vg, dt=g.dt, precision="mixed", tau=tau,
                                         out_deep=od, out_shallow=os_, workspace=ws), reps)
    step_plain = ev_time(api.PreparedStep(T, q, ps, vg, dt=g.dt, precision="mixed", tau=tau,
                                          out_deep=od0, out_shallow=os0, workspace=ws), reps)
    # the shallow rain-evaporation variant (extended kernels), coefficient 0.05
    sp = L.shallow_defaults()
    sp.evap_k = 0.05
    od1 = api.new_outputs(pver, n, "mixed", dev)
    os1 = api.new_outputs(pver, n, "mixed", dev)
    step_evap = ev_time(api.PreparedStep(T, q, ps, vg, dt=g.dt, precision="mixed", tau=tau,
                                         shallow_params=sp, out_deep=od1, out_shallow=os1,
                                         workspace=ws), reps)
    p_off, p_on = float(os0["prec"].sum()), float(os1["prec"].sum())
    # the deep plume-spectrum variant (extended kernels): 3 plumes, spread 4
    dpv = L.deep_defaults()
    dpv.n_plumes, dpv.plume_spread = 3, 4.0
    od2 = api.new_outputs(pver, n, "mixed", dev)
    os2 = api.new_outputs(pver, n, "mixed", dev)
    step_spec = ev_time(api.PreparedStep(T, q, ps, vg, dt=g.dt, precision="mixed", tau=tau,
                                         deep_params=dpv, out_deep=od2, out_shallow=os2,
                                         workspace=ws), reps)
    d_off, d_on = float(od0["prec"].sum()), float(od2["prec"].sum())
    ms = ev_time(lambda: api.tracer_transport(tr, ps, vg, deep_out=od, shallow_out=os_, dt=g.dt,
                                              precision="mixed", tend_deep=td, tend_shallow=ts),
                 reps)
    # momentum transport of (u, v) by the same plumes (pressure-gradient
    # coefficients 0.7): one launch, timed alone
    k = torch.arange(pver, device=dev, dtype=torch.float32)[:, None]
    uv = torch.stack([10.0 + 20.0 * (1 - k / pver) + 3.0 * torch.rand((pver, n), device=dev,
                                                                     generator=gen),
                      -5.0 + 8.0 * torch.sin(k / 4.0) + 3.0 * torch.rand((pver, n), device=dev,
                                                                         generator=gen)])
    ud, us = torch.empty_like(uv), torch.empty_like(uv)
    ms_mom = ev_time(lambda: api.momentum_transport(uv, ps, vg, deep_out=od, shallow_out=os_,
                                                    dt=g.dt, precision="mixed", cp_up=0.7,
                                                    cp_down=0.7, tend_deep=ud, tend_shallow=us),
                     reps)
    # algorithmic bytes of one launch
    ad = (od["flags"] & 2) > 0
    as_ = (os_["flags"] & 2) > 0
    jt, kb = od["ktop"].long(), od["kb"].long()
    kts = os_["ktop"].long()
    ld_ = torch.where(ad, kb - jt + 1, torch.zeros_like(kb))
    ls_ = torch.where(as_, pver - kts, torch.zeros_like(kts))
    ov = torch.clamp(torch.minimum(kb, torch.full_like(kb, pver - 1)) - torch.maximum(jt, kts) + 1,
                     min=0)
    both = ad & as_
    read_levels = ld_ + ls_ - torch.where(both, ov, torch.zeros_like(ov))
    jd = od["kaux"].long()
    dd_levels = torch.where(ad & (jd >= 0), kb - jd, torch.zeros_like(kb))
    es = 4
    per_col_prof = (2 * ld_ + dd_levels + 2 * ls_) * es + 7 * 4 + 8  # profiles, ints, ps
    tracer_bytes = ntr * (2 * pver * n * es + int(read_levels.sum()) * es)
    alg = tracer_bytes + int(per_col_prof.sum())
    achieved = alg / (ms * 1e-3) / 1e9
    peak, peak_src = measured_hbm()
    alg_mom = 2 * (2 * pver * n * es + int(read_levels.sum()) * es) + int(per_col_prof.sum())
    mom = {"components": 2, "cp_up": 0.7, "cp_down": 0.7, "ms_transport": ms_mom,
           "value": n / (ms_mom * 1e-3), "unit": UNIT, "gpu_launches_per_call": 1,
           "roofline": {"bound": "hbm", "achieved": alg_mom / (ms_mom * 1e-3) / 1e9,
                        "peak": peak, "unit": "GB/s",
                        "frac": alg_mom / (ms_mom * 1e-3) / 1e9 / peak,
                        "algorithmic_bytes": alg_mom, "traffic": None, "peak_source": peak_src}}
    return {"tracers": ntr, "columns": n, "levels": pver, "precision": "mixed",
            "ms_transport": ms, "value": ntr * n / (ms * 1e-3), "unit": "tracer-columns/s",
            "ms_step_with_profiles": step_flux, "ms_step_without_profiles": step_plain,
            "shallow_evaporation": {"evap_k": 0.05, "ms_step": step_evap,
                                    "shallow_rain_evaporated": 1.0 - p_on / max(p_off, 1e-300)},
            "deep_plume_spectrum": {"n_plumes": 3, "plume_spread": 4.0, "ms_step": step_spec,
                                    "deep_precip_ratio": d_on / max(d_off, 1e-300)},
            "gpu_launches_per_call": 1, "momentum_transport": mom,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "algorithmic_bytes": alg,
                         "traffic": ncu_traffic(g.name + "-tracers25", "transport").get(
                             "k_transport"),
                         "peak_source": peak_src}}


def driver_bench(args, dev, g):
    """The multi-step column driver (api.ColumnModel: fused step + state advance
    with relaxation) on the benchmark grid, mixed precision: per-step time of
    eager steps (Python marshalling every step) and of CUDA-graph replays."""
    import torch

    from paper_1711_00289_gb300 import api

    vg = api.VerticalGrid(g.hyai, g.hybi)
    T = torch.tensor(g.T, device=dev).float()
    q = torch.tensor(g.q, device=dev).float()
    ps = torch.tensor(g.ps, device=dev)
    tau = None if g.tau is None else torch.tensor(g.tau, device=dev)
    m = api.ColumnModel(T, q, ps, vg, precision="mixed", dt=g.dt, tau=tau)
    k = max(3, args.steps)
    res = {}
    for mode in ("eager", "graph"):
        run = (lambda n: m.step(n)) if mode == "eager" else (lambda n: m.run_graph(n))
        run(2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run(k)
        e1.record()
        torch.cuda.synchronize()
        res[f"ms_per_step_{mode}"] = e0.elapsed_time(e1) / k
    res.update({"columns": g.n_cols, "precision": "mixed", "steps_timed": k,
                "gpu_launches_per_step": 4})
    return res


def l2_note(prec, n, pver):
    mb = 2 * pver * n * (8 if prec == "fp64" else 4) / 2**20
    if mb > 129:
        return f"profile inputs ({mb:.0f} MB) larger than the 129 MB L2; no flush"
    return (f"profile inputs ({mb:.0f} MB) fit in L2: timings of this small case are not "
            f"HBM-representative")


# the sources each measured kernel is compiled from (an ncu capture stays valid
# while none of them changes); "step" covers k_trigger, k_plume and the FP64
# plain kernel k_plain of the baseline line
KERNEL_SOURCES = {
    "step": ("paper_1711_00289_gb300/csrc/column.cuh", "paper_1711_00289_gb300/csrc/compact.cu",
             "paper_1711_00289_gb300/csrc/compact.h", "paper_1711_00289_gb300/csrc/launch.h",
             "paper_1711_00289_gb300/csrc/plain.cu", "include/conv.h"),
    "transport": ("paper_1711_00289_gb300/csrc/transport.cu", "paper_1711_00289_gb300/csrc/column.cuh",
                  "paper_1711_00289_gb300/csrc/launch.h", "include/conv.h"),
}


def kernel_sources_sha256(group="step"):
    """Digest of the CUDA sources of a kernel group, to match an ncu capture to
    the kernels it measured."""
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[group]:
        h.update(rel.encode())
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def ncu_traffic(workload, group="step"):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of each
    kernel from the ncu capture summarised under profiles/, if it was taken of
    these sources on this workload; otherwise {} (traffic is then reported null).
    Records are lines `traffic-record: sha256=<digest> workload=<name>
    <kernel>=<bytes> ...`."""
    d = os.path.join(ROOT, "profiles")
    want = kernel_sources_sha256(group)
    out = {}
    for name in sorted(os.listdir(d)) if os.path.isdir(d) else []:
        if not name.endswith(".md"):
            continue
        with open(os.path.join(d, name)) as fh:
            for line in fh:
                if not line.startswith("traffic-record:"):
                    continue
                f = dict(t.split("=", 1) for t in line.split()[1:] if "=" in t)
                if f.get("sha256") == want and f.get("workload") == workload:
                    out.update({k: float(v) for k, v in f.items()
                                if k not in ("sha256", "workload")})
    return out


def measured_hbm():
    """HBM copy bandwidth in GB/s and where it comes from: the figure measured on
    this machine's GPUs (MEASURED_PEAKS.json), else 6.8 TB/s, one earlier copy
    measurement on a GB300."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except (OSError, KeyError, ValueError, TypeError):
        return 6800.0, "6.8 TB/s from an earlier GB300 copy measurement (of fallback)"


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank)
        return
    if world > 1:
        import torch

        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    ours_arm(args, rank, world, local_rank)
    if world > 1:
        import torch

        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
