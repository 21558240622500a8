"""Posterior products (per-bin phi summaries, P(k), Delta^2(k)) pinned to
closed forms and to a known distribution."""

import math

import numpy as np
import pytest

from paper_2501_12928_gb300.posterior import (delta_squared, injected_within, log_bayes_factor,
                                              point_null_logz, power_spectrum_posterior, weighted_quantiles)


def test_equal_weights_are_hazen_quantiles():
    x = np.random.default_rng(0).standard_normal(101)
    qs = [0.05, 0.16, 0.5, 0.84, 0.95]
    got = weighted_quantiles(x, np.ones_like(x), qs)
    assert np.allclose(got, np.quantile(x, qs, method="hazen"), rtol=0, atol=1e-14)
    # invariant to the scale of the weights
    assert np.allclose(weighted_quantiles(x, np.full_like(x, 7.5), qs), got, rtol=0, atol=1e-14)


def test_importance_weights_recover_a_normal():
    """x ~ U(-6, 6) weighted by the standard normal density: the weighted
    quantiles are those of N(0, 1) (a swapped or inverted weight fails)."""
    g = np.random.default_rng(1)
    x = g.uniform(-6, 6, 400_000)
    w = np.exp(-0.5 * x * x)
    qs = np.array([0.02275, 0.15866, 0.5, 0.84134, 0.97725])      # Phi(-2), Phi(-1), ..., Phi(2)
    got = weighted_quantiles(x, w, qs)
    assert np.allclose(got, [-2, -1, 0, 1, 2], atol=0.02)


def test_delta_squared_closed_forms():
    # P = A k^-3 gives a flat Delta^2 = A / (2 pi^2)
    k = np.array([0.1, 1.0, 3.0, 40.0])
    assert np.allclose(delta_squared(k, 5.0 * k ** -3.0), 5.0 / (2 * math.pi ** 2), rtol=1e-15)
    assert delta_squared(1.0, 2 * math.pi ** 2) == pytest.approx(1.0, rel=1e-15)
    assert delta_squared(2.0, 1.0) == pytest.approx(8.0 / (2 * math.pi ** 2), rel=1e-15)


def test_power_spectrum_posterior_gaussian_bins():
    g = np.random.default_rng(2)
    mu = np.array([-1.0, 0.3, 1.2])
    sd = np.array([0.05, 0.2, 0.4])
    s = mu + sd * g.standard_normal((200_000, 3))
    k = np.array([0.5, 1.0, 2.0])
    summ = power_spectrum_posterior(s, np.ones(len(s)), k)
    for b, m, d, kk in zip(summ, mu, sd, k):
        assert b.phi_mean == pytest.approx(m, abs=3e-3)
        assert b.phi_std == pytest.approx(d, rel=1e-2)
        assert b.phi_q[1] == pytest.approx(m, abs=4e-3)
        assert np.allclose(b.p_q, 10.0 ** b.phi_q, rtol=1e-14)
        assert np.allclose(b.delta2_q, kk ** 3 * b.p_q / (2 * math.pi ** 2), rtol=1e-14)
    assert injected_within(summ, mu).all()
    assert not injected_within(summ, mu + 10 * sd).any()


def test_bad_inputs_raise():
    with pytest.raises(ValueError):
        weighted_quantiles([], [], [0.5])
    with pytest.raises(ValueError):
        weighted_quantiles([1.0, 2.0], [1.0, -1.0], [0.5])
    with pytest.raises(ValueError):
        power_spectrum_posterior(np.zeros((4, 2)), np.ones(4), [1.0, 2.0, 3.0])


def test_bayes_factor_and_point_null():
    assert log_bayes_factor(10.0, 4.5) == 5.5
    # a point-null model's evidence is its likelihood at the fixed parameters
    calls = []

    def loglike(x):
        calls.append(x.copy())
        return -0.5 * np.sum(x * x, axis=1)

    assert point_null_logz(loglike, [1.0, 2.0]) == pytest.approx(-2.5)
    assert calls[0].shape == (1, 2)
