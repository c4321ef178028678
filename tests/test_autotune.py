"""Thompson-sampling tuner (host logic, no GPU): posterior updates against
their closed forms, and the sampler concentrating on the fastest candidate."""
import math

import numpy as np
import pytest

from paper_2605_00219_gb300.autotune import NIGPosterior, ThompsonTuner


def test_nig_posterior_closed_form():
    xs = [1.0, 1.2, 0.9, 1.1, 1.05]
    p = NIGPosterior()
    for x in xs:
        p.update(x)
    # after the first observation (prior kappa=1, mu=x0), the standard
    # Normal-Inverse-Gamma update gives mu_n = mean of all observations
    # weighted by kappa: (x0 + sum(xs)) / (1 + n)
    n = len(xs)
    assert p.kappa == pytest.approx(n)
    assert p.mu == pytest.approx((xs[0] + sum(xs[1:])) / n)
    assert p.alpha == pytest.approx(1.0 + 0.5 * (n - 1))
    # beta grows by the kappa-weighted squared innovations
    mu, kappa, beta = xs[0], 1.0, (0.1 * xs[0]) ** 2 + 1e-12
    for x in xs[1:]:
        beta += 0.5 * kappa * (x - mu) ** 2 / (kappa + 1)
        mu = (kappa * mu + x) / (kappa + 1)
        kappa += 1
    assert p.beta == pytest.approx(beta)


def test_thompson_prefers_fastest():
    rng = np.random.default_rng(0)
    means = [1.0, 1.3, 0.8, 1.1]
    tuner = ThompsonTuner(list(range(4)), seed=1)
    best = tuner.run(lambda c: rng.normal(means[c], 0.05), rounds=120)
    assert best == 2
    assert tuner.pulls[2] > 0.6 * sum(tuner.pulls)
    assert all(p >= 1 for p in tuner.pulls)   # every candidate was tried


def test_thompson_close_candidates():
    """Two candidates 3% apart with 2% noise: the better one is picked."""
    rng = np.random.default_rng(5)
    means = [1.03, 1.0]
    tuner = ThompsonTuner([0, 1], seed=2)
    assert tuner.run(lambda c: rng.normal(means[c], 0.02), rounds=200) == 1
