"""Planted mistakes in a copy of the oracle must each fail a pin test.

Every mutant below is a plausible slip (an index off by one, a dropped factor,
a flipped sign, a swapped operand) in one step of the column schemes.  The
mutant is compiled from a patched copy of conv_oracle.cpp in a temporary
directory and the pin suites are run against it in a subprocess; the mutants
are built and checked several at a time, each in its own directory.
"""
import concurrent.futures as cf
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
    "moisture limiter keeps the larger flux": (
        "if (val(ml) < val(mb)) {", "if (val(ml) > val(mb)) {"),
    "moisture limiter ignores q_min": (
        "const R ml = (q[k] - P.q_min) / (-dt * s.dq[k]);",
        "const R ml = q[k] / (-dt * s.dq[k]);"),
    "precipitation ignores downdraft evaporation": (
        "R net = sumR - alpha * sumE;", "R net = sumR;"),
    "closure drops tau": ("R mb = -cape / (tau * F);", "R mb = -cape / F;"),
    "closure drops the moisture part of dTv": (
        "const R dTv = (1.0 + ZVIR * q[k]) * s.dT[k] + ZVIR * T[k] * s.dq[k];",
        "const R dTv = (1.0 + ZVIR * q[k]) * s.dT[k];"),
    "shallow closure density from the dry temperature": (
        "const R rho = psrc / (RD * s.Tv[ks]);", "const R rho = psrc / (RD * Ts);"),
    "shallow w2 starts at tke": (
        "const double w2_0 = 2.0 / 3.0 * P.tke;", "const double w2_0 = P.tke;"),
    "shallow rain from total water": ("R r = l - P.ql_crit;", "R r = qt - P.ql_crit;"),
    "unsaturated plume temperature from qs": (
        "Tu = (s.hu[k] - gz - LV * qt) / CP;", "Tu = (s.hu[k] - gz - LV * qsu) / CP;"),
    "shallow top at the layer where w2 runs out": (
        "if (!(val(s.w2[k]) > 0.0)) { kts = k + 1; break; }",
        "if (!(val(s.w2[k]) > 0.0)) { kts = k; break; }"),
    "LFC allowed below the LCL": (
        "if (k <= klcl && val(s.b[k]) > 0.0) { klfc = k; break; }",
        "if (val(s.b[k]) > 0.0) { klfc = k; break; }"),
    "mid-layer pressure at the bottom interface": (
        "p_mid[k] = 0.5 * (p_int[k] + p_int[k + 1]);", "p_mid[k] = p_int[k + 1];"),
    "shallow dry parcel pressure ratio inverted": (
        "Tp = Ts * pow(s.p_mid[k] / psrc, KAPPA);", "Tp = Ts * pow(psrc / s.p_mid[k], KAPPA);"),
    "Newton step sign": (
        "    T = T - step;\n    if (last_step)", "    T = T + step;\n    if (last_step)"),
    "EL scanned upwards from the LCL": (
        "for (int k = ktl; k <= klcl; ++k)\n    if (val(s.b[k]) > 0.0) { kel = k; break; }",
        "for (int k = klcl; k >= ktl; --k)\n    if (val(s.b[k]) > 0.0) { kel = k; break; }"),
    "h* from the environment's own humidity": (
        "s.hs[k] = sdry + LV * qsk;", "s.hs[k] = sdry + LV * q[k];"),
    "CIN sign": ("R neg = -s.b[k];", "R neg = s.b[k];"),
}

PIN_FILES = ["tests/test_oracle_pins.py", "tests/test_oracle_adjoint.py"]

# Mistakes in the tracer transport, the mass-flux profiles and the two scheme
# variants, each with the pin suite that covers that part.
TRANSPORT = "tests/test_oracle_transport.py"
EVAPORATION = "tests/test_oracle_evaporation.py"
SPECTRUM = "tests/test_oracle_spectrum.py"
ADJOINT = "tests/test_oracle_adjoint.py"
COUNTS = "tests/test_oracle_counts.py"
MOMENTUM = "tests/test_oracle_momentum.py"
# The forward-mode type's rules for pow and sqrt are left out: no derivative
# that reaches an output passes through them (pow's differentiated argument is
# the LCL pressure, which only places levels; sqrt takes a constant), so a slip
# there changes nothing a pin could see.
EXT_MUTANTS = {
    # the counting instantiation (numerator of the arithmetic roofline)
    "subtraction not counted": (
        "inline Cnt operator-(const Cnt& a, const Cnt& b) { g_count[C_ADD] += 1; return Cnt(a.v - b.v); }",
        "inline Cnt operator-(const Cnt& a, const Cnt& b) { return Cnt(a.v - b.v); }", COUNTS),
    "division counted as a multiplication": (
        "inline Cnt operator/(const Cnt& a, const Cnt& b) { g_count[C_DIV] += 1;",
        "inline Cnt operator/(const Cnt& a, const Cnt& b) { g_count[C_MUL] += 1;", COUNTS),
    "counted power squares its base": (
        "g_count[C_POW] += 1; return Cnt(std::pow(a.v, e));",
        "g_count[C_POW] += 1; return Cnt(a.v * a.v);", COUNTS),
    "trigger-pass mark before the CAPE sum": (
        "  s.cape = cape;\n  mark_trigger_end<R>();", "  s.cape = cape;", COUNTS),
    "LFC-search tally from the start of the column": (
        "  mark_lfc_search<R>(false);\n", "", COUNTS),
    # the momentum transport
    "updraft pressure term pushes away from the environment": (
        "cu[k] = (s.eta[k + 1] * (cu[k + 1] + c_up * (c[k] - c[k + 1])) +",
        "cu[k] = (s.eta[k + 1] * (cu[k + 1] - c_up * (c[k] - c[k + 1])) +", MOMENTUM),
    "downdraft pressure term from the layer below": (
        "cd[k] = (s.etad[k - 1] * (cd[k - 1] + c_down * (c[k] - c[k - 1])) +",
        "cd[k] = (s.etad[k - 1] * (cd[k - 1] + c_down * (c[k] - c[k + 1])) +", MOMENTUM),
    "shallow plume skips the pressure term below its LCL": (
        "      cu[k] = ustar;\n", "      cu[k] = cu[k + 1];\n", MOMENTUM),
    "updraft eddy flux upwinded from its own layer": (
        "for (int k = jt + 1; k <= kb; ++k) F[k] = s.eta[k] * (cu[k] - c[k - 1]);",
        "for (int k = jt + 1; k <= kb; ++k) F[k] = s.eta[k] * (cu[k] - c[k]);", MOMENTUM),
    "downdraft eddy flux without its limiter": (
        "G[k + 1] = s.alpha * s.etad[k] * (cd[k] - c[k + 1]);",
        "G[k + 1] = s.etad[k] * (cd[k] - c[k + 1]);", MOMENTUM),
    "shallow eddy flux through the wrong interface": (
        "for (int k = kts + 1; k <= ks; ++k) F[k] = s.mb * (cu[k] - c[k - 1]);",
        "for (int k = kts + 1; k <= ks; ++k) F[k] = s.mb * (cu[k - 1] - c[k - 1]);", MOMENTUM),
    "drizzle band ten times wider": (
        "std::fabs(val(l) - P.ql_crit) < 1e-4", "std::fabs(val(l) - P.ql_crit) < 1e-3", COUNTS),
    "tangent quotient rule sign": (
        "r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v;", "r.d[i] = (a.d[i] + r.v * b.d[i]) / b.v;",
        ADJOINT),
    "tangent product rule drops a term": (
        "r.d[i] = a.d[i] * b.v + a.v * b.d[i];", "r.d[i] = a.d[i] * b.v;", ADJOINT),
    "tangent of log": (
        "for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] / a.v;",
        "for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * a.v;", ADJOINT),
    "tangent of exp": (
        "for (int i = 0; i < ND; ++i) r.d[i] = r.v * a.d[i];",
        "for (int i = 0; i < ND; ++i) r.d[i] = a.d[i];", ADJOINT),
    "tracer updraft entrains the layer below": (
        "cu[k] = (s.eta[k + 1] * cu[k + 1] + (s.eta[k] - s.eta[k + 1]) * c[k]) / s.eta[k];",
        "cu[k] = (s.eta[k + 1] * cu[k + 1] + (s.eta[k] - s.eta[k + 1]) * c[k + 1]) / s.eta[k];",
        TRANSPORT),
    "tracer subsidence upwinds from below": (
        "for (int k = jt + 1; k <= kb; ++k) dc[k] = dc[k] + s.eta[k] * (c[k - 1] - c[k]);",
        "for (int k = jt + 1; k <= kb; ++k) dc[k] = dc[k] + s.eta[k] * (c[k + 1] - c[k]);",
        TRANSPORT),
    "tracer downdraft detrains the level above": (
        "dc[kb] = dc[kb] + s.alpha * s.etad[kb - 1] * (cd[kb - 1] - c[kb]);",
        "dc[kb] = dc[kb] + s.alpha * s.etad[kb - 1] * (cd[kb - 2] - c[kb]);",
        TRANSPORT),
    "shallow tracer plume mixes in the LCL layer": (
        "    if (k >= s.klcl) {\n      cu[k] = cu[k + 1];",
        "    if (k > s.klcl) {\n      cu[k] = cu[k + 1];",
        TRANSPORT),
    "downdraft flux profile drops alpha": (
        "md[k] = s.mb * s.alpha * s.etad[k];", "md[k] = s.mb * s.etad[k];", TRANSPORT),
    "top detrainment flux from the top layer's eta": (
        "du[s.jt] = s.mb * s.eta[s.jt + 1];", "du[s.jt] = s.mb * s.eta[s.jt];", TRANSPORT),
    "shallow detrainment flux in the LCL layer": (
        "for (int k = s.kts + 1; k <= s.klcl - 1 && k <= ks - 1; ++k) {",
        "for (int k = s.kts + 1; k <= s.klcl && k <= ks - 1; ++k) {",
        TRANSPORT),
    "evaporated fraction without the layer depth": (
        "const R E = F * (1.0 - exp(-P.evap_k * def * dz));",
        "const R E = F * (1.0 - exp(-P.evap_k * def));",
        EVAPORATION),
    "evaporation warms the layer": (
        "s.dT[j] = s.dT[j] - LV * E / (CP * s.m[j]);",
        "s.dT[j] = s.dT[j] + LV * E / (CP * s.m[j]);",
        EVAPORATION),
    "rain evaporates in the layer that makes it": (
        "      const R E = F * (1.0 - exp(-P.evap_k * def * dz));\n"
        "      F = F - E;\n"
        "      s.dq[j] = s.dq[j] + E / s.m[j];\n"
        "      s.dT[j] = s.dT[j] - LV * E / (CP * s.m[j]);\n"
        "      if (j < ks) F = F + mb * s.rf[j];\n",
        "      if (j < ks) F = F + mb * s.rf[j];\n"
        "      const R E = F * (1.0 - exp(-P.evap_k * def * dz));\n"
        "      F = F - E;\n"
        "      s.dq[j] = s.dq[j] + E / s.m[j];\n"
        "      s.dT[j] = s.dT[j] - LV * E / (CP * s.m[j]);\n",
        EVAPORATION),
    "saturation deficit not clamped": (
        "      if (val(def) < 0.0) def = R(0.0);\n      const R E",
        "      const R E",
        EVAPORATION),
    "spectrum rates centred on the wrong member": (
        "lambda * std::pow(P.plume_spread, (double)ip / (NP - 1) - 0.5);",
        "lambda * std::pow(P.plume_spread, (double)ip / NP - 0.5);",
        SPECTRUM),
    "member share 1/(n-1)": ("w = 1.0 / NP;", "w = 1.0 / (NP - 1);", SPECTRUM),
    "ensemble top from the most entraining member": (
        "if (jt < 0 || jt_i < jt) jt = jt_i;", "if (jt < 0 || jt_i > jt) jt = jt_i;", SPECTRUM),
    "member rain not weighted by its share": (
        "sumR = sumR + w * sumR_i;", "sumR = sumR + sumR_i;", SPECTRUM),
}

CASES = {**{k: (o, n, PIN_FILES) for k, (o, n) in MUTANTS.items()},
         **{k: (o, n, [f]) for k, (o, n, f) in EXT_MUTANTS.items()}}


def _check(name, d):
    """Build mutant `name` in directory d and run its pin suites; returns the
    pytest exit code and the end of its output."""
    old, new, files = CASES[name]
    src = open(SRC).read()
    if src.count(old) != 1:
        return None, f"mutation anchor not found once: {name}"
    mpath = os.path.join(d, "conv_oracle.cpp")
    with open(mpath, "w") as f:
        f.write(src.replace(old, new))
    lib = os.path.join(d, "libmutant.so")
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    "-std=c++17", "-I", os.path.join(ROOT, "oracle"), "-o", lib, mpath],
                   check=True)
    env = dict(os.environ, CONV_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        *files], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    workers = max(1, min(6, (os.cpu_count() or 2) // 2))
    with cf.ThreadPoolExecutor(workers) as ex:
        futs = {name: ex.submit(_check, name, str(tmp_path_factory.mktemp("mutant")))
                for name in sorted(CASES)}
        return {name: f.result() for name, f in futs.items()}


@pytest.mark.parametrize("name", sorted(CASES))
def test_mutant_is_caught(name, outcomes):
    rc, out = outcomes[name]
    assert rc is not None, out
    assert rc != 0, f"mutant survived the pins: {name}\n{out}"
    # a failed pin (1) or a crash (killed by a signal), not a usage error or an
    # empty collection
    assert rc == 1 or rc < 0, f"pin run did not execute: {name} (exit {rc})\n{out}"
