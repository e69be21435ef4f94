"""Seeded synthetic inputs: recipes, determinism and the B-spline invariants (CPU only)."""

import numpy as np

import synthetic_inputs as S


def test_bspline_partition_of_unity_and_endpoints():
    w = np.linspace(0.0, 1.0, 101)
    b = S.bspline4_weights(w)
    assert np.allclose(b.sum(axis=-1), 1.0, atol=1e-15)
    assert np.all(b >= -1e-17)
    # w = 0: the cubic B-spline at integer knots is (1/6, 2/3, 1/6, 0)
    assert np.allclose(b[0], [1 / 6, 2 / 3, 1 / 6, 0.0], atol=1e-15)
    # symmetry: b_i(w) = b_{3-i}(1 - w)
    assert np.allclose(b, S.bspline4_weights(1.0 - w)[..., ::-1], atol=1e-15)


def test_white_noise_recipe():
    x = S.white_noise((4, 5, 6), 0)
    assert x.dtype == np.complex64 and x.shape == (4, 5, 6)
    a = np.random.default_rng(0).uniform(-1.0, 1.0, (4, 5, 6, 2))
    assert np.array_equal(x, (a[..., 0] + 1j * a[..., 1]).astype(np.complex64))
    assert np.array_equal(x, S.white_noise((4, 5, 6), 0))


def test_pme_grid_properties():
    rng = np.random.default_rng(1)
    pos = rng.random((2000, 3))
    q = rng.permutation(np.concatenate([np.ones(1000), -np.ones(1000)]))
    g = S.spread_charges((12, 10, 8), pos, q, chunk=333)
    assert g.shape == (12, 10, 8)
    assert abs(g.sum()) < 1e-10                     # net zero charge
    g1 = S.spread_charges((12, 10, 8), pos, np.ones(2000), chunk=2000)
    assert abs(g1.sum() - 2000.0) < 1e-9            # every charge deposits weight 1
    # one charge: separable product of the axis weights, wrapped periodically
    one = S.spread_charges((8, 8, 8), np.array([[0.01, 0.5, 0.99]]), np.array([1.0]))
    # y sits exactly on a mesh point (w = 0), where the fourth weight w^3/6 vanishes: 4 * 3 * 4 points
    assert np.count_nonzero(one) == 48
    assert abs(one.sum() - 1.0) < 1e-14
    assert one[7, 3, 6] > 0 and one[0, 4, 0] > 0   # i0-1 wraps for x, i0+2 wraps for z


def test_pme_grid_deterministic_and_complex64():
    a = S.pme_charge_grid((16, 12, 10), 5000, np.random.default_rng(7))
    b = S.pme_charge_grid((16, 12, 10), 5000, np.random.default_rng(7))
    assert a.dtype == np.complex64
    assert np.array_equal(a, b)
    assert np.all(a.imag == 0)


def test_pme_batch_recipe():
    dims, grids = S.pme_batch(count=4, seed=3)
    rng = np.random.default_rng(3)
    d = rng.choice(np.asarray(S.BATCH_AXIS_CHOICES), size=(4, 3))
    assert [tuple(r) for r in d.tolist()] == dims
    for dd, g in zip(dims, grids):
        assert g.shape == dd and g.dtype == np.complex64
