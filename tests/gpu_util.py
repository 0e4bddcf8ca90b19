"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
on a soundings grid and compare with the FP64 oracle."""
import os

import numpy as np

from paper_1711_00289_gb300 import soundings as S

INDEX_KEYS = ("flags", "kb", "klcl", "ktop", "kaux")
THREADS = os.cpu_count() or 1


def to_device(g, precision, ld=None, dev="cuda"):
    import torch

    from paper_1711_00289_gb300 import api

    n = g.n_cols
    ld = n if ld is None else ld
    rd = api.real_dtype(precision)
    T = torch.tensor(S.to_ld(g.T, ld), device=dev).to(rd)
    q = torch.tensor(S.to_ld(g.q, ld), device=dev).to(rd)
    ps_np = S.to_ld(g.ps, ld)
    ps_np[n:] = 1e5
    ps = torch.tensor(ps_np, device=dev)
    lam = None if g.lam is None else torch.tensor(S.to_ld(g.lam, ld), device=dev)
    tau = None if g.tau is None else torch.tensor(S.to_ld(g.tau, ld), device=dev)
    return T, q, ps, lam, tau


def run_gpu(g, precision="fp64", path="plain", ld=None, scheme="deep_shallow", sentinel=False,
            **kw):
    """Returns numpy dicts trimmed to n_cols (and the raw padded tails if sentinel)."""
    import torch

    from paper_1711_00289_gb300 import api

    n = g.n_cols
    ld = n if ld is None else ld
    T, q, ps, lam, tau = to_device(g, precision, ld)
    vg = api.VerticalGrid(g.hyai, g.hybi)
    outs = [api.new_outputs(g.pver, ld, precision) for _ in range(2)]
    if sentinel:
        for o in outs:
            for k, v in o.items():
                v.fill_(-7)
    if scheme == "deep_shallow":
        api.deep_shallow(T, q, ps, vg, dt=g.dt, precision=precision, lam=lam, tau=tau, path=path,
                         n_cols=n, out_deep=outs[0], out_shallow=outs[1], **kw)
        res = outs
    elif scheme == "deep":
        api.deep(T, q, ps, vg, dt=g.dt, precision=precision, lam=lam, tau=tau, path=path,
                 n_cols=n, out=outs[0], **kw)
        res = [outs[0]]
    else:
        api.shallow(T, q, ps, vg, precision=precision, path=path, n_cols=n, out=outs[0], **kw)
        res = [outs[0]]
    torch.cuda.synchronize()
    host = []
    for o in res:
        h = {k: v.cpu().numpy() for k, v in o.items()}
        host.append(h)
    trimmed = [{k: (v[:, :n] if v.ndim == 2 else v[:n]).astype(
        np.float64 if v.dtype == np.float32 else v.dtype) for k, v in h.items()} for h in host]
    if sentinel:
        return trimmed, host
    return trimmed


def assert_fp64_parity(got, ref, tol=1e-10, what=""):
    """Flags and level indices bit-exact; tendencies per column within tol of the
    column's max |reference|; column scalars within tol relative."""
    for k in INDEX_KEYS:
        bad = np.where(got[k] != ref[k])[0]
        assert bad.size == 0, f"{what} {k} differs in {bad.size} columns, first {bad[:5]}"
    for k in ("dTdt", "dqdt"):
        den = np.maximum(np.abs(ref[k]).max(axis=0), 1e-300)
        err = np.abs(got[k] - ref[k]).max(axis=0) / den
        assert np.all(err <= tol), f"{what} {k} rel err {err.max():.3g} at column {err.argmax()}"
    # column scalars.  Precipitation is a difference (rain minus evaporation, or
    # liquid above a threshold) and is compared against M_b x 1 g/kg, the water
    # flux scale of the column, so cancellation at trace rain does not count.
    # CAPE / CIN below 0.05 J/kg are sums over layers of near-zero buoyancy: one
    # last-bit change of the state moves such a CIN by ~1e-12 J/kg (measured: a
    # 1e-15 relative change of T moves a 5.6e-4 J/kg CIN by 2.7e-12 J/kg), so
    # they are compared against 0.05 J/kg.
    pscale = np.maximum(np.abs(ref["prec"]), 1e-3 * np.abs(ref["mb"]))
    for k, den in (("prec", np.maximum(pscale, 1e-300)),
                   ("cape", np.maximum(np.abs(ref["cape"]), 0.05)),
                   ("mb", np.maximum(np.abs(ref["mb"]), 1e-300))):
        err = np.abs(got[k] - ref[k]) / den
        err[(got[k] == 0) & (ref[k] == 0)] = 0
        assert np.all(err <= tol), f"{what} {k} rel err {err.max():.3g} at {err.argmax()}"


def same_decisions(got, ref):
    same = np.ones(ref["flags"].shape[0], bool)
    for k in INDEX_KEYS:
        same &= got[k] == ref[k]
    return same


def mixed_report(got, ref, m, upstream_same=None, p_surface=None):
    """Mixed-precision error budget.  Decisions: any of flags/kb/klcl/ktop/kaux
    differing.  Errors over columns active in both with identical decisions:
    tendency column integral |sum m (x - y)| / sum m |y|; precipitation
    |P - P_ref| / max(P_ref, 1e-3 * median nonzero surface precipitation), the
    surface precipitation being deep + shallow of the oracle (p_surface; the
    scheme's own P when not given), so trace drizzle -- liquid a hair above the
    autoconversion threshold, whose FP32 rounding is relatively large -- is
    measured against the precipitation scale of the grid.  upstream_same: for
    the shallow scheme, the columns whose deep decisions agree -- a deep
    decision flip changes the shallow scheme's input state, and is already
    counted against the deep scheme."""
    same = same_decisions(got, ref)
    if upstream_same is not None:
        same_own = same.copy()
        same &= upstream_same
    trig_flips = int(np.sum((got["flags"] & 1) != (ref["flags"] & 1)))
    act = same & ((ref["flags"] & 2) > 0)
    if upstream_same is not None:
        # flips of the shallow scheme on columns whose deep decisions agree
        trig_flips = int(np.sum(((got["flags"] & 1) != (ref["flags"] & 1)) & upstream_same))
        same_for_count = same_own | ~upstream_same
    else:
        same_for_count = same
    by_key = {k: int(np.sum(got[k] != ref[k])) for k in INDEX_KEYS}
    x = got["flags"] ^ ref["flags"]
    bits = {b: int(np.sum((x >> b) & 1)) for b in range(12) if np.any((x >> b) & 1)}
    out = dict(n=int(same.size), decision_mismatch=int((~same_for_count).sum()),
               trigger_flips=trig_flips, active=int(act.sum()), mismatch_by_key=by_key,
               flag_bits_differing=bits)
    for k in ("dTdt", "dqdt"):
        num = np.abs(np.sum(m * (got[k] - ref[k]), axis=0))
        den = np.maximum(np.sum(m * np.abs(ref[k]), axis=0), 1e-300)
        e = (num / den)[act]
        out[k + "_colint_max"] = float(e.max()) if e.size else 0.0
    pr = ref["prec"]
    ps_ = pr if p_surface is None else p_surface
    for key, src in (("prec_max", ps_), ("prec_max_own", pr)):
        nz = src[src > 0]
        floor = 1e-3 * (np.median(nz) if nz.size else 1.0)
        e = (np.abs(got["prec"] - pr) / np.maximum(pr, floor))[act]
        out[key] = float(e.max()) if e.size else 0.0
    return out


def check_mixed(r, tag="", mismatch=1e-3):
    """The mixed path's error budget against the FP64 oracle (a mixed_report):
    trigger flips on at most 0.1% of the columns; decision mismatches of any
    kind (level indices, exit codes, flag bits) on at most `mismatch` of them;
    on the columns whose decisions agree, tendency column integrals within 1e-4
    and precipitation within 1e-3 (prec_max: against the floor of 1e-3 x the
    median nonzero surface precipitation; prec_max_own, the floor from the
    scheme's own median, is reported beside it)."""
    assert r["trigger_flips"] <= 1e-3 * r["n"], f"{tag} {r}"
    assert r["decision_mismatch"] <= mismatch * r["n"], f"{tag} {r}"
    assert r["dTdt_colint_max"] <= 1e-4 and r["dqdt_colint_max"] <= 1e-4, f"{tag} {r}"
    assert r["prec_max"] <= 1e-3, f"{tag} {r}"


def layer_mass(g):
    p_int = g.hyai[:, None] * 1e5 + g.hybi[:, None] * g.ps[None, :]
    return np.diff(p_int, axis=0) / 9.80616
