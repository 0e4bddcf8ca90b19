"""Independent checking helpers for the pin tests (test infrastructure only).

Constants restate the values the schemes are defined with; the root finders are
bisections on the *defining* equations, deliberately a different algorithm from
the Newton iterations used by the oracle and the CUDA kernels.
"""
import math

import numpy as np

GRAV = 9.80616
RD = 287.04
RV = 461.5
CP = 1004.64
LV = 2.501e6
EPS = RD / RV
ZVIR = RV / RD - 1.0
KAPPA = RD / CP


def bisect(f, lo, hi, iters=200):
    flo = f(lo)
    assert flo * f(hi) <= 0.0, (lo, hi, flo, f(hi))
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        fm = f(mid)
        if (fm < 0) == (flo < 0):
            lo, flo = mid, fm
        else:
            hi = mid
        if hi - lo <= 1e-13 * max(1.0, abs(mid)):
            break
    return 0.5 * (lo + hi)


def saturated_temperature(O, h, gz, p):
    """T solving cp T + gz + Lv qs(T, p) = h by bisection (qs from the oracle)."""
    return bisect(lambda T: CP * T + gz + LV * O.qs(T, p) - h, 40.0, 400.0)


def lcl_by_bisection(O, Tb, qb, pb):
    """T_L solving qs(T, pb (T/Tb)^(cp/Rd)) = qb on the dry adiabat."""
    return bisect(lambda T: O.qs(T, pb * (T / Tb) ** (1.0 / KAPPA)) - qb, 150.0, Tb)


def bolton_tl(Tb, rh):
    """Bolton (1980) eq. 22 LCL temperature (K) from temperature and RH (fraction)."""
    return 1.0 / (1.0 / (Tb - 55.0) - math.log(rh) / 2840.0) + 55.0


def levels(hyai, hybi, ps, p0=1e5):
    p_int = np.asarray(hyai) * p0 + np.asarray(hybi) * ps
    return p_int, 0.5 * (p_int[:-1] + p_int[1:])
