"""Seeded input generator: determinism, order independence, recipe shape."""
import numpy as np

from paper_1711_00289_gb300 import soundings as S


def test_uniform_is_counter_based():
    a = S.uniform(7, 3, np.arange(1000), 2)
    b = np.array([S.uniform(7, 3, i, 2) for i in (999, 5, 0)])
    assert np.array_equal(b, a[[999, 5, 0]])
    assert np.all((a >= 0) & (a < 1))
    assert abs(a.mean() - 0.5) < 0.03
    assert not np.array_equal(a, S.uniform(8, 3, np.arange(1000), 2))
    assert not np.array_equal(a, S.uniform(7, 3, np.arange(1000), 1))


def test_splitmix_reference_value():
    # SplitMix64 of state 0 (first output of the generator seeded with 0):
    # published test value 0xE220A8397B1DCDAF.
    out = S._splitmix(np.array([0], dtype=np.uint64))[0]
    assert int(out) == 0xE220A8397B1DCDAF


def test_hybrid_grid_shape():
    for pver in (26, 30, 32):
        a, b = S.hybrid_coefficients(pver)
        p = a * S.P0 + b * 1e5
        assert p[0] == 300.0 and p[-1] == 1e5
        assert np.all(np.diff(p) > 0)
        assert np.all(b[p < 2e4] == 0.0)


def test_profiles_recipe():
    t, q, ps = S.profiles(30, np.array([300.0, 285.0]), np.array([0.9, 0.5]))
    a, b = S.hybrid_coefficients(30)
    p_int = a[:, None] * S.P0 + b[:, None] * ps[None, :]
    p_mid = 0.5 * (p_int[:-1] + p_int[1:])
    top = p_mid[:, 0] < 2e4
    assert np.allclose(t[top, 0], t[top, 0][-1])  # isothermal above 200 hPa
    assert np.all(np.diff(t[~top, 0]) > 0)  # warmer downwards below
    assert np.all(q > 0) and np.all(q < 0.05)


def test_grids_deterministic_and_sized():
    g1 = S.latlon_grid(12, 18)
    g2 = S.latlon_grid(12, 18)
    assert g1.n_cols == 216 and np.array_equal(g1.T, g2.T) and np.array_equal(g1.q, g2.q)
    g = S.clustered_grid(0.3, 48, 72)
    assert abs(g.mask.mean() - 0.3) < 0.01
    ens = S.ensemble(8, scale=0.01)
    assert len(ens) == 8 and {m.pver for m in ens} <= {26, 30, 32}
    assert all(5e-4 <= m.lam[0] <= 2e-3 for m in ens)
