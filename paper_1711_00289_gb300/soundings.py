"""Seeded synthetic soundings shaped like the paper's CAM5 workloads.

This module only makes inputs: hybrid level coefficients, temperature and
humidity profiles, surface pressure and per-column scheme parameters.  It
contains none of the convection arithmetic (its humidity uses its own Magnus
formula, not the schemes' saturation function), so the CPU oracle and the CUDA
path can both be fed from it.

Workloads (Sec. V-A, resolutions table: 30 levels; R1 = 96 x 144 = 13,824
columns, R3 = 768 x 1152 = 884,736 columns):

* ``column_set``  -- 64 independent columns (surface T ~ U(280, 305) K,
  surface RH ~ U(0.40, 0.95)).
* ``latlon_grid`` -- a lat-lon grid with surface T/RH varying with latitude and a
  moist band centred at 5 N, so convecting columns are spatially clustered.
* ``clustered_grid`` -- a grid with a clustered convecting mask from a sum of
  64 random Gaussian blobs (periodic in longitude) thresholded at its
  (1 - f) quantile.
* ``ensemble`` -- members of log-uniform column counts and mixed level counts.

Random numbers: SplitMix64 (Steele, Lea & Flood 2014) keyed by
(seed, member, column, stream), so every value is independent of ordering and
layout.
"""
from __future__ import annotations

import dataclasses

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)

P_TOP = 300.0  # Pa, model top (3 hPa)
P_SURF_REF = 1.0e5  # Pa
P0 = 1.0e5  # Pa, reference pressure multiplying the A coefficients


def _splitmix(x: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (x + _GOLDEN) & _M64
        z = ((z ^ (z >> np.uint64(30))) * _MIX1) & _M64
        z = ((z ^ (z >> np.uint64(27))) * _MIX2) & _M64
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, member: int, column, stream: int) -> np.ndarray:
    """U[0,1) per (seed, member, column, stream); ``column`` may be an array."""
    col = np.asarray(column, dtype=np.uint64)
    k = _splitmix(np.full(col.shape, np.uint64(seed), dtype=np.uint64))
    k = _splitmix(k ^ np.uint64(member))
    k = _splitmix(k ^ col)
    k = _splitmix(k ^ np.uint64(stream))
    return (k >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def hybrid_coefficients(pver: int):
    """Interface coefficients (A, B), pver+1 each, top (index 0) to surface.

    Reference interface pressure p_i = p_top + (p_s,ref - p_top) (i/pver)^1.6;
    B_i = max(0, (p_i/p_s,ref - 0.2)/0.8), A_i p0 = p_i - B_i p_s,ref, so the
    model top is 3 hPa and the grid is pure pressure above 200 hPa.
    """
    i = np.arange(pver + 1, dtype=np.float64)
    p_ref = P_TOP + (P_SURF_REF - P_TOP) * (i / pver) ** 1.6
    b = np.maximum(0.0, (p_ref / P_SURF_REF - 0.2) / 0.8)
    b[-1] = 1.0
    a = (p_ref - b * P_SURF_REF) / P0
    a[-1] = 0.0
    return a, b


# --- sounding shape (input recipe; generator-only constants) -----------------
_R_GEN = 287.0
_G_GEN = 9.81
_LAPSE = 6.5e-3  # K/m up to the tropopause
_P_TROP = 2.0e4  # Pa, isothermal above
_P_RH = 5.0e4  # Pa, RH decays as (p/5e4)^3 above


def _magnus_es(T):
    """Alduchov & Eskridge (1996) Magnus form over water, Pa (input recipe only)."""
    tc = T - 273.15
    return 610.94 * np.exp(17.625 * tc / (tc + 243.04))


def profiles(pver: int, t_surf, rh_surf, ps=None):
    """Temperature and specific humidity, shape [pver, n], for surface T and RH.

    T(p) = T_s (p/ps)^(R Gamma/g) for p >= 200 hPa and isothermal above;
    RH(p) = RH_s for p >= 500 hPa, RH_s (p/500 hPa)^3 above;
    q = 0.622 RH e_s(T)/p with the generator's Magnus e_s.
    """
    t_surf = np.asarray(t_surf, dtype=np.float64)
    rh_surf = np.asarray(rh_surf, dtype=np.float64)
    n = t_surf.shape[0]
    if ps is None:
        ps = np.full(n, P_SURF_REF)
    a, b = hybrid_coefficients(pver)
    p_int = a[:, None] * P0 + b[:, None] * ps[None, :]
    p_mid = 0.5 * (p_int[:-1] + p_int[1:])
    expo = _R_GEN * _LAPSE / _G_GEN
    t = t_surf[None, :] * (np.maximum(p_mid, _P_TROP) / ps[None, :]) ** expo
    rh = np.where(p_mid >= _P_RH, rh_surf[None, :], rh_surf[None, :] * (p_mid / _P_RH) ** 3)
    q = 0.622 * rh * _magnus_es(t) / p_mid
    return np.ascontiguousarray(t), np.ascontiguousarray(q), np.ascontiguousarray(ps)


@dataclasses.dataclass
class Columns:
    """One grid of columns, level-major [pver][n] float64 arrays."""

    name: str
    pver: int
    T: np.ndarray
    q: np.ndarray
    ps: np.ndarray
    hyai: np.ndarray
    hybi: np.ndarray
    lam: np.ndarray | None = None
    tau: np.ndarray | None = None
    dt: float = 1800.0

    @property
    def n_cols(self) -> int:
        return int(self.T.shape[1])


def _grid(name, pver, ts, rh, lam=None, tau=None):
    t, q, ps = profiles(pver, ts, rh)
    a, b = hybrid_coefficients(pver)
    return Columns(name, pver, t, q, ps, a, b, lam, tau)


def column_set(n: int = 64, seed: int = 20171101, pver: int = 30) -> Columns:
    """Independent columns: T_s ~ U(280, 305) K, RH_s ~ U(0.40, 0.95)."""
    c = np.arange(n)
    ts = 280.0 + 25.0 * uniform(seed, 0, c, 0)
    rh = 0.40 + 0.55 * uniform(seed, 0, c, 1)
    return _grid(f"columns-{n}x{pver}", pver, ts, rh)


ITCZ_HALF_WIDTH_DEG = 19.0  # e-folding half width of the moist band (gives ~25% deep-convecting columns)


def latlon_grid(nlat: int = 96, nlon: int = 144, seed: int = 20171102, pver: int = 30,
                band_deg: float = ITCZ_HALF_WIDTH_DEG, tau_range=None) -> Columns:
    """Lat-lon grid (column index = j*nlon + i): T_s = 280 + 25 cos^2(lat) + U(-1,1),
    RH_s = 0.40 + 0.55 exp(-((lat-5)/band)^2) + U(-0.03, 0.03) clipped to [0.40, 0.95].
    ``tau_range`` draws a per-column CAPE relaxation time uniformly in it."""
    j = np.repeat(np.arange(nlat), nlon)
    c = np.arange(nlat * nlon)
    lat = -90.0 + (j + 0.5) * 180.0 / nlat
    ts = 280.0 + 25.0 * np.cos(np.deg2rad(lat)) ** 2 + (2.0 * uniform(seed, 0, c, 0) - 1.0)
    rh = 0.40 + 0.55 * np.exp(-(((lat - 5.0) / band_deg) ** 2))
    rh = np.clip(rh + 0.03 * (2.0 * uniform(seed, 0, c, 1) - 1.0), 0.40, 0.95)
    tau = None
    if tau_range is not None:
        lo, hi = tau_range
        tau = lo + (hi - lo) * uniform(seed, 0, c, 2)
    return _grid(f"latlon-{nlat}x{nlon}x{pver}", pver, ts, rh, tau=tau)


def blob_field(nlat: int, nlon: int, seed: int, n_blobs: int = 64) -> np.ndarray:
    """Sum of Gaussian blobs (sigma 10-40 cells, periodic in longitude), [nlat, nlon]."""
    b = np.arange(n_blobs)
    cy = uniform(seed, 1, b, 0) * nlat
    cx = uniform(seed, 1, b, 1) * nlon
    sig = 10.0 + 30.0 * uniform(seed, 1, b, 2)
    amp = 0.5 + 0.5 * uniform(seed, 1, b, 3)
    y = np.arange(nlat, dtype=np.float64)[:, None]
    x = np.arange(nlon, dtype=np.float64)[None, :]
    f = np.zeros((nlat, nlon))
    for k in range(n_blobs):
        dx = np.abs(x - cx[k])
        dx = np.minimum(dx, nlon - dx)
        dy = y - cy[k]
        f += amp[k] * np.exp(-(dx * dx + dy * dy) / (2.0 * sig[k] ** 2))
    return f


def clustered_grid(frac: float = 0.30, nlat: int = 768, nlon: int = 1152,
                   seed: int = 20171103, pver: int = 30) -> Columns:
    """Clustered convecting patches covering ``frac`` of the grid.

    Inside the mask: T_s ~ U(298, 305) K, RH_s ~ U(0.80, 0.95);
    outside: T_s ~ U(280, 292) K, RH_s ~ U(0.40, 0.60).
    """
    f = blob_field(nlat, nlon, seed).ravel()
    thr = np.quantile(f, 1.0 - frac)
    inside = f > thr
    c = np.arange(nlat * nlon)
    u0 = uniform(seed, 0, c, 0)
    u1 = uniform(seed, 0, c, 1)
    ts = np.where(inside, 298.0 + 7.0 * u0, 280.0 + 12.0 * u0)
    rh = np.where(inside, 0.80 + 0.15 * u1, 0.40 + 0.20 * u1)
    g = _grid(f"clustered-{nlat}x{nlon}x{pver}-f{frac:.2f}", pver, ts, rh)
    g.mask = inside  # type: ignore[attr-defined]
    return g


def ensemble(n_members: int = 64, seed: int = 20171104, n_min: int = 1000,
             n_max: int = 200000, scale: float = 1.0):
    """Members with n_cols = round(exp(U(ln n_min, ln n_max))) * scale, pver from
    {26, 30, 32}, a member surface-T offset U(-3, 3) K added to a ``column_set``
    style draw, and a member entrainment rate lambda ~ U(0.5e-3, 2.0e-3) 1/m."""
    m = np.arange(n_members)
    un = uniform(seed, 2, m, 0)
    n_cols = np.maximum(1, np.round(np.exp(np.log(n_min) + (np.log(n_max) - np.log(n_min)) * un)
                                    * scale)).astype(np.int64)
    pvers = np.array([26, 30, 32])[np.minimum(2, (3.0 * uniform(seed, 2, m, 1)).astype(int))]
    offs = -3.0 + 6.0 * uniform(seed, 2, m, 2)
    lams = 0.5e-3 + 1.5e-3 * uniform(seed, 2, m, 3)
    out = []
    for i in range(n_members):
        c = np.arange(int(n_cols[i]))
        ts = 280.0 + 25.0 * uniform(seed, 3 + i, c, 0) + offs[i]
        rh = 0.40 + 0.55 * uniform(seed, 3 + i, c, 1)
        g = _grid(f"member-{i}", int(pvers[i]), ts, rh, lam=np.full(c.shape[0], lams[i]))
        out.append(g)
    return out


def pad_ld(n: int, align: int = 32) -> int:
    """Leading dimension: n rounded up to a multiple of ``align`` columns."""
    return ((n + align - 1) // align) * align


def to_ld(a: np.ndarray, ld: int) -> np.ndarray:
    """Copy [pver][n] (or [n]) into a zero-padded [pver][ld] (or [ld]) array."""
    if a.ndim == 1:
        out = np.zeros(ld, dtype=a.dtype)
        out[: a.shape[0]] = a
        return out
    out = np.zeros((a.shape[0], ld), dtype=a.dtype)
    out[:, : a.shape[1]] = a
    return out
