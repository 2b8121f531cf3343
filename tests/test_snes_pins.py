"""Pins of the training-loop oracle (SNES, Sec. II.D) against facts other
than its own formulas: the library Philox generator, the normal
distribution, closed forms, invariances of the evolution strategy and its
behaviour on functions whose minimiser is known."""

import numpy as np
import pytest
from scipy import stats

import oracle


def test_philox_matches_library_generator():
    # numpy's Philox bit generator is Philox4x64-10; it advances the counter
    # before each block, so its first block belongs to counter + 1.
    rng = np.random.default_rng(7)
    for _ in range(5):
        key = rng.integers(0, 2 ** 63, size=2, dtype=np.uint64)
        ctr = rng.integers(1, 2 ** 63, size=4, dtype=np.uint64)
        prev = ctr.copy()
        prev[0] -= np.uint64(1)
        lib = np.random.Philox(key=key, counter=prev).random_raw(4)
        ours = oracle.philox4x64_10(ctr[None, :], key)[0]
        assert np.array_equal(lib, ours)


def test_normals_are_standard_normal():
    s = oracle.snes_normals(2312005233, 3, 64, 4099).ravel()
    n = s.size
    assert abs(s.mean()) < 5 / np.sqrt(n)
    assert abs(s.var() - 1) < 5 * np.sqrt(2 / n)
    assert stats.kstest(s, "norm").pvalue > 1e-3
    # neighbours in a Box-Muller pair and across blocks are uncorrelated
    pairs = s[: n // 2 * 2].reshape(-1, 2)
    assert abs(np.corrcoef(pairs[:, 0], pairs[:, 1])[0, 1]) < 5 / np.sqrt(len(pairs))


def test_normals_depend_on_every_counter_word():
    base = oracle.snes_normals(11, 0, 3, 9)
    assert not np.array_equal(base, oracle.snes_normals(12, 0, 3, 9))  # key
    assert not np.array_equal(base, oracle.snes_normals(11, 1, 3, 9))  # generation
    assert not np.array_equal(base[0], base[1])  # individual
    assert not np.array_equal(base[0, :4], base[0, 4:8])  # block
    # a longer vector extends, not reshuffles, the shorter one
    assert np.array_equal(base, oracle.snes_normals(11, 0, 3, 13)[:, :9])


def test_utilities_closed_forms():
    # lambda = 2: weights (ln 2, 0) -> (1, 0) - 1/2
    np.testing.assert_allclose(oracle.snes_utilities(2), [0.5, -0.5], atol=1e-15)
    for lam in (2, 3, 8, 50, 1024):
        u = oracle.snes_utilities(lam)
        assert abs(u.sum()) < 1e-13
        assert np.all(np.diff(u) <= 0)
        # only ranks below lambda/2 + 1 get a positive share; all others -1/lambda
        r = np.arange(1, lam + 1)
        assert np.allclose(u[r >= lam / 2 + 1], -1.0 / lam)


def test_regularization_closed_form():
    z = np.full(7, -0.3)
    assert oracle.regularization(z, 0.2, 0.5) == pytest.approx(0.2 * 0.3 + 0.5 * 0.3)
    z = np.array([3.0, 4.0, 0.0, 0.0])
    assert oracle.regularization(z, 1.0, 0.0) == pytest.approx(7 / 4)
    assert oracle.regularization(z, 0.0, 1.0) == pytest.approx(np.sqrt(25 / 4))


def _run(f, mu, sigma, gens, n_pop, seed=5):
    for g in range(gens):
        mu, sigma, _, _ = oracle.snes_generation(mu, sigma, g, seed, n_pop, f)
    return mu, sigma


def test_converges_on_separable_quadratic():
    rng = np.random.default_rng(1)
    d = 8
    a = rng.uniform(0.5, 5.0, d)
    c = rng.uniform(-2, 2, d)
    f = lambda z: float(np.sum(a * (z - c) ** 2))
    mu, sigma = _run(f, np.zeros(d), np.full(d, 1.0), 500, 12)
    assert np.max(np.abs(mu - c)) < 1e-3
    assert np.all(sigma < 1e-2)


def test_mean_moves_downhill_and_sigma_grows_on_a_slope():
    d = 6
    g = np.array([1.0, -2.0, 0.5, 3.0, -1.0, 0.25])
    f = lambda z: float(g @ z)
    mu, sigma = _run(f, np.zeros(d), np.full(d, 1e-3), 30, 10)
    assert f(mu) < -1e-3 * 5 and np.all(np.sign(mu) == -np.sign(g))
    # in one dimension the ranking is fixed by s alone: consistent
    # improvement along the slope must widen the search distribution
    mu1, sigma1 = _run(lambda z: float(-2.0 * z[0]), np.zeros(1), np.full(1, 1e-3), 60, 10)
    assert mu1[0] > 0 and sigma1[0] > 1e-1


def test_rank_based_invariant_to_monotone_loss_transform():
    rng = np.random.default_rng(2)
    c = rng.normal(size=5)
    f = lambda z: float(np.sum((z - c) ** 2))
    h = lambda z: float(np.exp(0.1 * f(z)) - 3.0)
    m1, s1 = _run(f, np.zeros(5), np.ones(5), 20, 8)
    m2, s2 = _run(h, np.zeros(5), np.ones(5), 20, 8)
    assert np.array_equal(m1, m2) and np.array_equal(s1, s2)


def test_translation_and_axis_scale_invariance():
    rng = np.random.default_rng(3)
    d = 5
    c = rng.normal(size=d)
    delta = rng.normal(size=d)
    scale = rng.uniform(0.1, 10.0, d)
    f = lambda z: float(np.sum((z - c) ** 2 * np.arange(1, d + 1)))
    m0, s0 = _run(f, np.zeros(d), np.ones(d), 15, 8)
    m1, s1 = _run(lambda z: f(z - delta), delta.copy(), np.ones(d), 15, 8)
    np.testing.assert_allclose(m1, m0 + delta, rtol=0, atol=1e-12)
    np.testing.assert_allclose(s1, s0, rtol=1e-12)
    m2, s2 = _run(lambda z: f(z / scale), np.zeros(d), scale.copy(), 15, 8)
    np.testing.assert_allclose(m2, m0 * scale, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(s2, s0 * scale, rtol=1e-12)


def test_update_reduces_to_plain_evolution_step_for_two_individuals():
    # lambda = 2, utilities (+1/2, -1/2): mu moves half a step from the loser
    # towards the winner, sigma grows where they differed by more than 1 sigma
    mu, sigma = np.array([0.0, 1.0]), np.array([1.0, 2.0])
    s = np.array([[1.0, -0.5], [-1.0, 2.0]])
    loss = np.array([3.0, 1.0])  # individual 1 wins
    eta_s = 0.4
    mu1, sg1 = oracle.snes_update(mu, sigma, s, loss, 1.0, eta_s)
    np.testing.assert_allclose(mu1, mu + sigma * 0.5 * (s[1] - s[0]))
    np.testing.assert_allclose(sg1, sigma * np.exp(0.5 * eta_s * 0.5 * (s[1] ** 2 - s[0] ** 2)))
