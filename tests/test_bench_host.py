"""Host-side arithmetic of bench.py's JSON line, without a GPU: the ALU roofline
fields, the nominal peaks from unit counts and clocks, the algorithmic bytes per
column, and the rule that an ncu traffic record applies only to the sources and
workload it was captured on."""
import os
import shutil

import pytest

import bench


def _rates(fp32_fma=35.7e12, fp64_fma=5.3e11):
    r = {}
    for pipe, fma in (("fp32", fp32_fma), ("fp64", fp64_fma)):
        r.update({f"{pipe}_fma": fma, f"{pipe}_exp": fma / 8, f"{pipe}_log": fma / 8,
                  f"{pipe}_div": fma / 10, f"{pipe}_pow": fma / 30})
    return r


def test_nominal_peaks_from_unit_counts_and_clock():
    # 152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz; 152 x 2 FP64 units x 2 x 2.07 GHz
    assert 2 * bench.nominal_fma_rate("fp32") == pytest.approx(80.5478e12, rel=1e-5)
    assert 2 * bench.nominal_fma_rate("fp64") == pytest.approx(1.258560e12, rel=1e-6)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_alu_roofline_fields(precision):
    counts = dict(add=900.0, mul=700.0, div=40.0, exp=30.0, log=20.0, pow=2.0,
                  fp64_lcl_corrections=0.001)
    r = _rates()
    n, t = 884736, 0.5e-3
    x = bench.kernel_roofline(counts, precision, t, n, r)
    pipe = "fp64" if precision == "fp64" else "fp32"
    assert x["bound"] == "alu" and x["binding_pipe"] == pipe
    # the work at the measured rates, in seconds, from the operation mix by hand
    pfx = pipe + "_"
    t_bound = n * (900 / r[pfx + "fma"] + 40 / r[pfx + "div"] + 30 / r[pfx + "exp"]
                   + 20 / r[pfx + "log"] + 2 / r[pfx + "pow"])
    assert x["frac_of_measured"] == pytest.approx(t_bound / t, rel=1e-12)
    assert x["peak"] == pytest.approx(2 * bench.nominal_fma_rate(pipe) / 1e12, rel=1e-12)
    assert x["peak_measured"] == pytest.approx(2 * r[pfx + "fma"] / 1e12, rel=1e-12)
    assert x["frac"] == pytest.approx(x["achieved"] / x["peak"], rel=1e-12)
    assert x["frac"] == pytest.approx(x["frac_of_measured"] * x["peak_measured"] / x["peak"],
                                      rel=1e-12)
    assert x["traffic"] is None and "unit counts" in x["peak_source"]


def test_fp64_islands_bind_when_the_fp32_work_is_tiny():
    counts = dict(add=1.0, mul=1.0, div=0.0, exp=0.0, log=0.0, pow=0.0,
                  fp64_lcl_corrections=100.0)
    x = bench.kernel_roofline(counts, "mixed", 1e-3, 1000, _rates())
    assert x["binding_pipe"] == "fp64"
    assert x["peak"] == pytest.approx(2 * bench.nominal_fma_rate("fp64") / 1e12)


def test_algorithmic_bytes_per_column():
    # read T, q (pver each) and ps; write dT/dt, dq/dt of both schemes and
    # 4 doubles + 5 int32 per scheme
    assert bench.hbm_bytes_per_column(30, 4) == 832
    assert bench.hbm_bytes_per_column(30, 8) == 1552


def test_traffic_record_applies_only_to_its_sources_and_workload(tmp_path, monkeypatch):
    root = tmp_path
    for rel in set(bench.KERNEL_SOURCES["step"]):
        os.makedirs(root / os.path.dirname(rel), exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, rel), root / rel)
    monkeypatch.setattr(bench, "ROOT", str(root))
    sha = bench.kernel_sources_sha256("step")
    os.makedirs(root / "profiles")
    (root / "profiles" / "k.md").write_text(
        "summary\n"
        f"traffic-record: sha256={sha} workload=w1 k_trigger=100 k_plume=50\n"
        f"traffic-record: sha256={'0' * 64} workload=w1 k_trigger=999\n")
    assert bench.ncu_traffic("w1") == {"k_trigger": 100.0, "k_plume": 50.0}
    assert bench.ncu_traffic("w2") == {}
    with open(root / bench.KERNEL_SOURCES["step"][0], "a") as fh:
        fh.write("\n// changed\n")
    assert bench.kernel_sources_sha256("step") != sha
    assert bench.ncu_traffic("w1") == {}


def test_hbm_peak_source_is_named(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    v, src = bench.measured_hbm()
    assert v == 6800.0 and "fallback" in src
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6777.0}')
    v, src = bench.measured_hbm()
    assert v == 6777.0 and "measured" in src


def _pass_counts():
    base = dict(add=900.0, mul=700.0, div=40.0, exp=30.0, log=20.0, pow=2.0, sqrt=0.0,
                fp64_lcl_corrections=0.001, fp64_drizzle=0.02)
    plume = {k: v / 3 for k, v in base.items()}
    e2 = dict(add=100.0, mul=80.0, div=10.0, exp=5.0, log=0.0, pow=0.0, sqrt=0.0)
    return {"trigger_pass_per_column": base, "plume_pass_per_column": plume,
            "trigger_pass_e2_search_per_column": e2,
            "total_per_column": {k: base[k] + plume[k] for k in bench.OP_CATS}}


def test_trigger_pass_work_leaves_out_the_e2_search():
    c, r, n = _pass_counts(), _rates(), 884736
    k = bench.path_rooflines(c, "mixed", "compact", (0.5, 0.4), n, r)
    net = {x: c["trigger_pass_per_column"][x] - c["trigger_pass_e2_search_per_column"].get(x, 0)
           for x in bench.OP_CATS}
    net.update(fp64_lcl_corrections=0.001, fp64_drizzle=0.02)
    ref = bench.kernel_roofline(net, "mixed", 0.5e-3, n, r)
    gross = bench.kernel_roofline(c["trigger_pass_per_column"], "mixed", 0.5e-3, n, r)
    assert k["k_trigger"]["frac"] == pytest.approx(ref["frac"], rel=1e-12)
    assert k["k_trigger"]["with_e2_search_counted"]["frac"] == pytest.approx(gross["frac"])
    assert k["k_trigger"]["frac"] < gross["frac"]
    assert k["k_trigger"]["share"] + k["k_plume"]["share"] == pytest.approx(1.0)


def test_step_roofline_sums_the_kernels_bound_times():
    c, r, n = _pass_counts(), _rates(), 884736
    k = bench.path_rooflines(c, "mixed", "compact", (0.5, 0.4), n, r)
    st = bench.step_roofline(k, 1.0)
    tb = k["k_trigger"]["t_bound_ms"] + k["k_plume"]["t_bound_ms"]
    assert st["frac_of_measured"] == pytest.approx(tb / 1.0, rel=1e-12)
    # kernels alone (0.9 ms of the 1.0 ms step): the step's fraction is lower
    kt = bench.step_roofline(k, 0.9)
    assert st["frac"] == pytest.approx(kt["frac"] * 0.9, rel=1e-12)
    assert st["frac"] == pytest.approx(st["frac_of_measured"] * 2 * 35.7 / 80.5478, rel=1e-4)


def test_drizzle_corrections_cost_fp64_work():
    r = _rates()
    a = bench.t_fp64_islands(dict(fp64_lcl_corrections=0.0, fp64_drizzle=1.0), r)
    assert a == pytest.approx(2 / r["fp64_exp"] + 6 / r["fp64_div"] + 24 / r["fp64_fma"])
