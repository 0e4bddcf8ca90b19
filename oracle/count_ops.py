"""Writes oracle/op_counts.json: the algorithmic floating-point operation counts
of the deep+shallow path per column, by category, for the benchmark workloads,
counted by the oracle's counting instantiation.  These are the numerators of the
benchmark's arithmetic roofline.  Run: python -m oracle.count_ops
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1711_00289_gb300 import soundings as S  # noqa: E402

CATS = ["add", "mul", "div", "exp", "log", "pow", "sqrt"]
PASS_CATS = CATS + ["unused", "fp64_lcl", "fp64_cape_terms", "fp64_cin_terms",
                    "fp64_cons_terms", "fp64_drizzle"]


# Relative half-width of the band around the FP32 LCL pressure within which the
# mixed GPU path applies its FP64 LCL correction (a layer mid-point or the
# shallow E1 threshold inside the band).
LCL_BAND = 2e-5


def _near(pL, kstart, pm, guard):
    k = kstart
    while k >= 0 and not pm[k] <= pL:
        k -= 1
    lo, hi = pL * (1 - LCL_BAND), pL * (1 + LCL_BAND)
    return ((k >= 0 and pm[k] > lo) or (k < kstart and pm[k + 1] <= hi)
            or (guard > 0 and abs(guard - pL) <= LCL_BAND * pL))


def lcl_corrections(sub, dpar=None):
    """FP64 LCL corrections per column of the mixed design, by pass: LCL solves
    whose pressure (the oracle's) lies within LCL_BAND of a layer mid-point or
    of the E1 threshold.  Trigger pass: the deep LCL of every valid column and
    the shallow LCL of non-triggered ones (reused from the deep solve when the
    launch layer is the lowest); plume pass: the shallow LCL of triggered
    columns on the deep-updated state."""
    od, _ = O.deep_shallow(sub, dpar=dpar, threads=os.cpu_count() or 1)
    guard = O.shallow_params().p_lcl_min
    pi = sub.hyai[:, None] * 1e5 + sub.hybi[:, None] * sub.ps[None, :]
    pm = 0.5 * (pi[1:] + pi[:-1])
    ks = sub.pver - 1
    trig = (od["flags"] & 1) > 0
    bad = (od["flags"] & 16) > 0
    a = b = 0
    for i in range(sub.n_cols):
        if bad[i]:
            continue
        col = pm[:, i]
        kb = int(od["kb"][i])
        _, pL, _ = O.lcl(sub.T[kb, i], sub.q[kb, i], col[kb])
        exact = pL == col[kb]
        if not exact and _near(pL, kb, col, -1.0):
            a += 1
            exact = True
        if not trig[i]:
            if kb == ks:
                a += int(not exact and abs(guard - pL) <= LCL_BAND * pL)
            else:
                _, p2, _ = O.lcl(sub.T[ks, i], sub.q[ks, i], col[ks])
                a += int(p2 != col[ks] and _near(p2, ks, col, guard))
        else:
            T2 = sub.T[ks, i] + sub.dt * od["dTdt"][ks, i]
            q2 = max(sub.q[ks, i] + sub.dt * od["dqdt"][ks, i], 0.0)
            _, p2, _ = O.lcl(T2, q2, col[ks])
            b += int(p2 != col[ks] and _near(p2, ks, col, guard))
    return a / sub.n_cols, b / sub.n_cols


def counts(g, stride=1):
    sub = S.Columns(g.name, g.pver, g.T[:, ::stride].copy(), g.q[:, ::stride].copy(),
                    g.ps[::stride].copy(), g.hyai, g.hybi)
    cd, ct = O.count_ops(sub)
    a, b, nt, e2 = O.count_ops_by_pass(sub, e2=True)
    ca, cb = lcl_corrections(sub)
    n = sub.n_cols
    trig = {c: a[i] / n for i, c in enumerate(PASS_CATS) if c != "unused"}
    plume = {c: b[i] / n for i, c in enumerate(PASS_CATS) if c != "unused"}
    trig["fp64_lcl_corrections"] = ca
    plume["fp64_lcl_corrections"] = cb
    return {"columns_counted": n, "triggered_fraction": nt / n,
            "deep_per_column": {c: cd[i] / n for i, c in enumerate(CATS)},
            "total_per_column": {c: ct[i] / n for i, c in enumerate(CATS)},
            # per column of the whole grid, split by pass of the compacted path
            "trigger_pass_per_column": trig, "plume_pass_per_column": plume,
            # part of the trigger pass: the shallow LFC search of columns that
            # end at exit E2, which the GPU may settle by bounds instead
            "trigger_pass_e2_search_per_column": {c: e2[i] / n for i, c in enumerate(CATS)}}


def ensemble_counts(per_member=1500):
    """The 64-member batched ensemble (26/30/32 levels, member entrainment
    rates): trigger- and plume-pass counts per column of the whole ensemble, each
    member counted on a strided sample and weighted by its column count."""
    ens = S.ensemble(64)
    total = sum(g.n_cols for g in ens)
    trig, plume, e2s, ntrig = {}, {}, {}, 0.0
    counted = 0
    for g in ens:
        st = max(1, g.n_cols // per_member)
        sub = S.Columns(g.name, g.pver, g.T[:, ::st].copy(), g.q[:, ::st].copy(),
                        g.ps[::st].copy(), g.hyai, g.hybi)
        dpar = O.deep_params(lambda_default=float(g.lam[0]))
        a, b, nt, e2 = O.count_ops_by_pass(sub, dpar=dpar, e2=True)
        ca, cb = lcl_corrections(sub, dpar)
        w = g.n_cols / total
        for i, c in enumerate(PASS_CATS):
            if c != "unused":
                trig[c] = trig.get(c, 0.0) + w * a[i] / sub.n_cols
                plume[c] = plume.get(c, 0.0) + w * b[i] / sub.n_cols
        for i, c in enumerate(CATS):
            e2s[c] = e2s.get(c, 0.0) + w * e2[i] / sub.n_cols
        trig["fp64_lcl_corrections"] = trig.get("fp64_lcl_corrections", 0.0) + w * ca
        plume["fp64_lcl_corrections"] = plume.get("fp64_lcl_corrections", 0.0) + w * cb
        ntrig += w * nt / sub.n_cols
        counted += sub.n_cols
    return {"columns_counted": counted, "columns": total, "triggered_fraction": ntrig,
            "trigger_pass_per_column": trig, "plume_pass_per_column": plume,
            "trigger_pass_e2_search_per_column": e2s}


def main():
    out = {"source": "oracle/conv_oracle.cpp counting instantiation (R = Cnt)",
           "categories": CATS, "workloads": {}}
    for f in (0.1, 0.3, 0.6):
        g = S.clustered_grid(f)
        out["workloads"][f"clustered-768x1152x30-f{f:.2f}"] = counts(g, stride=7)
    g = S.latlon_grid()
    out["workloads"]["latlon-96x144x30"] = counts(g)
    out["workloads"]["ensemble-64"] = ensemble_counts()
    path = os.path.join(ROOT, "oracle", "op_counts.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
    print(path)


if __name__ == "__main__":
    main()
