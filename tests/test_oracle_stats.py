"""Pins of the oracle's ensemble statistics (mean and quantile bands of the
receiver traces over the realizations, Sec. 4.5.2) against numpy's
quantile, hand-computed order statistics and invariances."""
import numpy as np

import oracle


def test_hand_example():
    # 4 realizations of one receiver at one record: sorted 1, 2, 3, 4
    x = np.array([3.0, 1.0, 4.0, 2.0]).reshape(1, 4, 1)
    mean, q = oracle.trace_stats(x, [0.0, 0.5, 1.0, 1.0 / 3.0, 0.25])
    assert mean[0, 0] == 2.5
    # h = 3p: p = 1/2 -> halfway between x(1) = 2 and x(2) = 3; p = 1/3 -> h = 1,
    # x(1) = 2; p = 1/4 -> h = 0.75, three quarters from x(0) = 1 to x(1) = 2
    np.testing.assert_array_equal(q[:, 0, 0], [1.0, 2.5, 4.0, 2.0, 1.75])


def test_matches_numpy_quantile_bitwise():
    rng = np.random.default_rng(3)
    ps = [0.05, 0.5, 0.95, 0.0, 1.0, 0.1234567]
    for M in (1, 2, 3, 64, 513):
        x = rng.standard_normal((4, M, 5)).astype(np.float32)
        mean, q = oracle.trace_stats(x, ps)
        ref = np.quantile(x.astype(np.float64), ps, axis=1, method="linear")
        np.testing.assert_array_equal(q, ref)
        np.testing.assert_allclose(mean, x.astype(np.float64).mean(axis=1), rtol=1e-14, atol=1e-15)


def test_permutation_invariance_and_constants():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((3, 50, 2))
    perm = rng.permutation(50)
    m1, q1 = oracle.trace_stats(x, [0.05, 0.95])
    m2, q2 = oracle.trace_stats(x[:, perm, :], [0.05, 0.95])
    np.testing.assert_array_equal(q1, q2)
    np.testing.assert_allclose(m1, m2, rtol=1e-14)
    c = np.full((2, 7, 3), 1.25)
    m, q = oracle.trace_stats(c, [0.0, 0.3, 1.0])
    assert np.all(m == 1.25) and np.all(q == 1.25)


def test_quantiles_are_monotone_and_bracket_the_mean_band():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((6, 101, 4))
    _, q = oracle.trace_stats(x, [0.05, 0.25, 0.5, 0.75, 0.95])
    assert np.all(np.diff(q, axis=0) >= 0)
    # for 101 values h = 100 p is an integer for these p: the order statistics themselves
    xs = np.sort(x, axis=1)
    np.testing.assert_array_equal(q[0], xs[:, 5, :])
    np.testing.assert_array_equal(q[4], xs[:, 95, :])
