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
                    "fp64_cons_terms"]


def counts(g, stride=1):
    sub = S.Columns(g.name, g.pver, g.T[:, ::stride].copy(), g.q[:, ::stride].copy(),
                    g.ps[::stride].copy(), g.hyai, g.hybi)
    cd, ct = O.count_ops(sub)
    a, b, nt = O.count_ops_by_pass(sub)
    n = sub.n_cols
    return {"columns_counted": n, "triggered_fraction": nt / n,
            "deep_per_column": {c: cd[i] / n for i, c in enumerate(CATS)},
            "total_per_column": {c: ct[i] / n for i, c in enumerate(CATS)},
            # per column of the whole grid, split by pass of the compacted path
            "trigger_pass_per_column": {c: a[i] / n for i, c in enumerate(PASS_CATS)
                                        if c != "unused"},
            "plume_pass_per_column": {c: b[i] / n for i, c in enumerate(PASS_CATS)
                                      if c != "unused"}}


def main():
    out = {"source": "oracle/conv_oracle.cpp counting instantiation (R = Cnt)",
           "categories": CATS, "workloads": {}}
    for f in (0.1, 0.3, 0.6):
        g = S.clustered_grid(f)
        out["workloads"][f"clustered-768x1152x30-f{f:.2f}"] = counts(g, stride=7)
    g = S.latlon_grid()
    out["workloads"]["latlon-96x144x30"] = counts(g)
    path = os.path.join(ROOT, "oracle", "op_counts.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
    print(path)


if __name__ == "__main__":
    main()
