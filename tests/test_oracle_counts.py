"""Pins of the oracle's counting instantiation, whose operation counts are the
numerator of the benchmark's arithmetic roofline.

* The counting instantiation computes the oracle: its outputs equal the plain
  FP64 oracle's bit for bit.
* Every operator counts: on dry columns (the deep scheme stops at its LCL, the
  shallow scheme at exit E1) the per-category counts equal a count made by hand
  from the formulas each stage evaluates, at 4 and 7 levels (which separates the
  per-level work from the fixed work).
* The split between the trigger pass and the plume pass: the two passes sum to
  the whole step; a column that triggers puts into the trigger pass exactly the
  work the deep scheme does up to its trigger decision (the same column with an
  unreachable CAPE threshold stops there); nothing goes to the plume pass when
  no column triggers.
* The tallies beside the counts: the E2 LFC-search work of a column that ends
  at exit E2 equals the work that column loses when its search limit is moved
  below the source (no layer searched); the FP64 drizzle-island tally equals a
  brute-force count of saturated plume layers whose rain lies within 1e-4
  kg/kg of zero.
tests/test_oracle_mutants.py plants slips in the counting (an operator that does
not count, a division counted as a multiplication, a wrong value, a misplaced
pass mark or search mark, a wider island band); each fails one of these pins."""
import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S

CATS = ["add", "mul", "div", "exp", "log", "pow", "sqrt"]


def _cols(g, idx):
    return S.Columns(g.name, g.pver, np.ascontiguousarray(g.T[:, idx]),
                     np.ascontiguousarray(g.q[:, idx]), g.ps[idx].copy(), g.hyai, g.hybi)


def test_counting_instantiation_equals_the_oracle(oracle):
    for g in (S.latlon_grid(24, 36), S.clustered_grid(0.5, 24, 24)):
        rd, rs = oracle.deep_shallow(g, threads=4)
        cd, cs = oracle.deep_shallow_counted(g)
        assert ((rd["flags"] & 2) > 0).sum() > 20 and ((rs["flags"] & 2) > 0).sum() > 20
        for a, b in ((rd, cd), (rs, cs)):
            for k in a:
                assert np.array_equal(a[k], b[k]), k


def _dry_grid(pver, n=3):
    a, b = S.hybrid_coefficients(pver)
    ts = np.array([290.0, 300.0, 305.0])[:n]
    T, q, ps = S.profiles(pver, ts, np.full(n, 0.1), np.full(n, 1e5))
    return S.Columns(f"dry-{pver}", pver, T, q, ps, a, b)


def _hand_count(pver):
    """Operations of one dry column, counted from the formulas each stage evaluates.

    levels: p_i = A_i p0 + B_i ps (1 mul, 1 add per interface; A_i p0 is a
      constant) and p_k = 0.5 (p_k + p_k+1) (1 add, 1 mul per layer);
    heights, per layer: Tv = T (1 + zv q) 2 mul 1 add; Rd Tv / g 1 mul 1 div;
      dln p = ln(p_k+1 / p_k) 1 div 1 log; z_int 1 mul 1 add; z_mid 1 div 1 log
      1 mul 1 add;
    qs(T, p): es = 611.2 exp(17.67 (T - T0)/(T - T1)) 2 add 2 mul 1 div 1 exp;
      D = p - (1-eps) es 1 mul 1 add; 1e-3 p 1 mul; eps es / D 1 mul 1 div;
    deep, per layer: m = dp/g 1 add 1 div; qs; cp T + g z 2 mul 1 add;
      h, h* 1 mul 1 add each;
    shallow, per layer: m 1 add 1 div; h = cp T + g z + Lv q 3 mul 2 add;
    LCL of an unsaturated parcel: qs at the launch point; e_b = q p/(eps +
      (1-eps) q) 2 mul 1 add 1 div; RH = e_b / es 1 div plus es; Bolton's first
      guess 3 add 3 div 1 log; ln e_b 1 log; 6 Newton steps of 9 add 3 mul 5 div
      1 log; p_L = p_b (T_L/T_b)^(cp/Rd) 1 div 1 pow 1 mul;
    the deep-updated state passed to the shallow scheme: 2 add per layer."""
    n = pver
    qs = dict(add=3, mul=5, div=2, exp=1)
    es = dict(add=2, mul=2, div=1, exp=1)
    newton = dict(add=9, mul=3, div=5, log=1)
    lcl = {c: qs.get(c, 0) + es.get(c, 0) + 6 * newton.get(c, 0) for c in CATS}
    for c, v in dict(mul=2, add=1, div=1).items():  # e_b
        lcl[c] += v
    lcl["div"] += 1  # RH
    for c, v in dict(add=3, div=3, log=1).items():  # Bolton eq. 22
        lcl[c] += v
    lcl["log"] += 1  # ln e_b
    for c, v in dict(div=1, pow=1, mul=1).items():  # p_L
        lcl[c] += v
    prof = {c: 0 for c in CATS}  # levels + heights
    for c, v in dict(mul=1, add=1).items():
        prof[c] += v * (n + 1)
    for c, v in dict(add=1, mul=1).items():
        prof[c] += v * n
    for c, v in dict(mul=5, add=3, div=3, log=2).items():
        prof[c] += v * n
    deep = {c: prof[c] + lcl[c] for c in CATS}
    for c in CATS:
        deep[c] += n * (qs.get(c, 0) + dict(add=1 + 1 + 1 + 1, mul=2 + 1 + 1, div=1).get(c, 0))
    shal = {c: prof[c] + lcl[c] for c in CATS}
    for c, v in dict(add=1 + 2, mul=3, div=1).items():
        shal[c] += n * v
    total = {c: deep[c] + shal[c] + (2 * n if c == "add" else 0) for c in CATS}
    return deep, total


@pytest.mark.parametrize("pver", [4, 7])
def test_hand_count_of_a_dry_column(oracle, pver):
    g = _dry_grid(pver)
    dpar = oracle.deep_params(p_top_lim=95000.0)  # no layer above the LCL is admitted
    d, s = oracle.deep_shallow(g, dpar=dpar)
    assert np.all((d["flags"] & 1) == 0) and np.all(d["klcl"] < pver - 1)
    assert np.all(((s["flags"] >> oracle.EXIT_SHIFT) & 7) == 1)  # exit E1
    cd, ct = oracle.count_ops(g, dpar=dpar)
    deep, total = _hand_count(pver)
    for i, c in enumerate(CATS):
        assert cd[i] == g.n_cols * deep[c], (c, cd[i] / g.n_cols, deep[c])
        assert ct[i] == g.n_cols * total[c], (c, ct[i] / g.n_cols, total[c])


def test_pass_split(oracle):
    g = S.clustered_grid(0.3, 24, 36)
    cd, ct = oracle.count_ops(g)
    a, b, nt, e2 = oracle.count_ops_by_pass(g, e2=True)
    assert 0 < nt < g.n_cols
    for i in range(len(CATS)):
        assert a[i] + b[i] == pytest.approx(ct[i], rel=1e-15, abs=0)
        assert 0 <= e2[i] <= a[i]
    assert e2[0] > 0 and b[0] > 0
    # the trigger pass of a triggered column is the deep work up to the trigger
    # decision, plus nothing of its shallow scheme
    rd, _ = oracle.deep_shallow(g)
    trig = np.where((rd["flags"] & 1) > 0)[0][:12]
    stop = oracle.deep_params(capelmt=1e30)
    for i in trig:
        one = _cols(g, [i])
        ai, bi, nti = oracle.count_ops_by_pass(one)
        assert nti == 1.0
        cdi, _ = oracle.count_ops(one, dpar=stop)
        for c in range(len(CATS)):
            assert ai[c] == cdi[c], (i, CATS[c], ai[c], cdi[c])
    # the E2 tally of a column that ends at exit E2 without triggering is the work
    # its LFC search adds: the same column with the search limit below the
    # source (no layer searched) does everything else
    nolfc = oracle.shallow_params(p_lfc_min=2.0e5)
    _, rs = oracle.deep_shallow(g)
    e2cols = np.where(((rs["flags"] >> oracle.EXIT_SHIFT) & 7 == 2)
                      & ((rd["flags"] & 1) == 0))[0][:12]
    assert e2cols.size > 5
    for i in e2cols:
        one = _cols(g, [i])
        _, _, _, e2i = oracle.count_ops_by_pass(one, e2=True)
        _, t_full = oracle.count_ops(one)
        _, t_none = oracle.count_ops(one, spar=nolfc)
        for c in range(len(CATS)):
            assert e2i[c] == t_full[c] - t_none[c], (i, CATS[c])
    # nothing triggers: no plume pass
    a0, b0, nt0 = oracle.count_ops_by_pass(g, dpar=stop)
    assert nt0 == 0 and not b0.any() and a0[0] > 0


def test_drizzle_island_tally(oracle):
    """Saturated shallow plume layers with |qt - qs(T_sat) - ql_crit| < 1e-4
    kg/kg, counted by brute force from the scheme's internals (deep scheme off,
    so the shallow scheme sees the columns' own state), on randomly perturbed
    soundings whose moist layers make such drizzle."""
    from tests.test_oracle_random import _random_columns

    g = _random_columns(3, n=600)
    stop = oracle.deep_params(capelmt=1e30)
    spar = oracle.shallow_params()
    a, b, _ = oracle.count_ops_by_pass(g, dpar=stop)
    want = 0
    for i in range(g.n_cols):
        d = oracle.shallow_column_diag(g.pver, g.hyai, g.hybi, g.T[:, i], g.q[:, i],
                                       float(g.ps[i]), par=spar)
        if d.exit_code in (1, 2, 3):
            continue
        # the plume layers that evaluate their rain: up to the top layer when the
        # plume stopped there on w2 <= 0 one layer higher, below it when the
        # plume reached the top limit
        lo = d.kts + 1 if d.kts == d.k_top_lim else d.kts
        for k in range(lo, g.pver - 1):
            qsu = oracle.qs(d.Tu[k], d.p_mid[k])
            if d.qtpre[k] >= qsu and abs(d.qtpre[k] - qsu - spar.ql_crit) < 1e-4:
                want += 1
    assert want > 0
    assert a[12] + b[12] == want
