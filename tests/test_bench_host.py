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
