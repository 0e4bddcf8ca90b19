"""Planted mistakes in a copy of the oracle must each fail a pin test.

Every mutant below is a plausible slip (an index off by one, a dropped factor,
a flipped sign, a swapped operand) in one step of the column schemes.  The
mutant is compiled from a patched copy of conv_oracle.cpp in a temporary
directory and the pin suites are run against it in a subprocess.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "conv_oracle.cpp")

MUTANTS = {
    "updraft detrainment uses eta_jt": (
        "s.dh[jt_i] = s.dh[jt_i] + (w * s.eta[jt_i + 1]) * (s.hu[jt_i + 1] - s.h[jt_i]);",
        "s.dh[jt_i] = s.dh[jt_i] + (w * s.eta[jt_i]) * (s.hu[jt_i + 1] - s.h[jt_i]);"),
    "subsidence upwinds from below": (
        "s.dh[k] = s.dh[k] + (w * s.eta[k]) * (s.h[k - 1] - s.h[k]);",
        "s.dh[k] = s.dh[k] + (w * s.eta[k]) * (s.h[k + 1] - s.h[k]);"),
    "downdraft detrains level above": (
        "s.dq[kb] = s.dq[kb] + D * (s.qd[kb - 1] - q[kb]);",
        "s.dq[kb] = s.dq[kb] + D * (s.qd[kb - 2] - q[kb]);"),
    "CAPE sum skips the EL": (
        "for (int k = klcl; k >= kel; --k) cape = cape + RD * s.b[k] * s.dlnp[k];",
        "for (int k = klcl; k > kel; --k) cape = cape + RD * s.b[k] * s.dlnp[k];"),
    "closure sign of environment term": (
        "F = F + RD * s.dlnp[k] * (dTvp * s.dh[kb] - dTv);",
        "F = F + RD * s.dlnp[k] * (dTvp * s.dh[kb] + dTv);"),
    "dqs/dT drops p/D": (
        "dqs = qs * (p / D) * dlnes;", "dqs = qs * dlnes;"),
    "LCL exponent inverted": (
        "pL = pb * pow(TL / Tb, INV_KAPPA);", "pL = pb * pow(TL / Tb, KAPPA);"),
    "mid-layer height from the wrong interface": (
        "z_mid[k] = z_int[k + 1] + scale * log(p_int[k + 1] / p_mid[k]);",
        "z_mid[k] = z_int[k + 1] + scale * log(p_int[k] / p_mid[k]);"),
    "shallow outflow uses post-rain water": (
        "s.dq[k] = mb * ((s.qtu[k + 1] - s.qtpre[k]) + (q[k - 1] - q[k]));",
        "s.dq[k] = mb * ((s.qtu[k + 1] - s.qtu[k]) + (q[k - 1] - q[k]));"),
    "rain not implicit": (
        "s.rain[k] = s.eta[k] * P.c0 * dz * l / (1.0 + P.c0 * dz);",
        "s.rain[k] = s.eta[k] * P.c0 * dz * l;"),
    "evaporation sign": (
        "s.E1[jd] = s.etad[jd] * (s.qd[jd] - q[jd]);",
        "s.E1[jd] = s.etad[jd] * (q[jd] - s.qd[jd]);"),
    "entrainment exponent": (
        "return exp(lambda * z_e * log(1.0 + dz / z_e));",
        "return exp(lambda * log(1.0 + dz / z_e));"),
    "launch tie keeps the upper level": (
        "if (val(s.h[k]) > val(s.h[kb])) kb = k;",
        "if (val(s.h[k]) >= val(s.h[kb])) kb = k;"),
    "virtual temperature factor": (
        "Tv[k] = T[k] * (1.0 + ZVIR * q[k]);", "Tv[k] = T[k] * (1.0 + EPS * q[k]);"),
    "LCL level off by one": (
        "if (val(p_mid[k]) <= val(pL)) return k;", "if (val(p_mid[k]) <= val(pL)) return k - 1;"),
    "CIN thickness of the layer above": (
        "cin = cin + RD * neg * s.dlnp[k];", "cin = cin + RD * neg * s.dlnp[k - 1];"),
    "w2 drag decay sign": (
        "const R decay = exp(-2.0 * beps * dz);", "const R decay = exp(2.0 * beps * dz);"),
    "w2 buoyancy work halved": (
        "s.w2[k] = s.w2[k + 1] + 2.0 * P.a_w * B * dz;", "s.w2[k] = s.w2[k + 1] + P.a_w * B * dz;"),
    "es constants swapped": (
        "return ES0 * exp(ESA * (T - EST0) / (T - EST1));",
        "return ES0 * exp(ESA * (T - EST1) / (T - EST0));"),
}

PIN_FILES = ["tests/test_oracle_pins.py", "tests/test_oracle_adjoint.py"]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found once: {name}"
    mpath = tmp_path / "conv_oracle.cpp"
    mpath.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    "-std=c++17", "-I", os.path.join(ROOT, "oracle"), "-o", str(lib),
                    str(mpath)], check=True)
    env = dict(os.environ, CONV_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        *PIN_FILES], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode != 0, f"mutant survived the pins: {name}\n{r.stdout[-2000:]}"
