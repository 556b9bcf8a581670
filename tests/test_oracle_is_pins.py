"""Pins of the learned-proposal oracle (MLP, Adam, proposal, sampler,
importance-sampling estimator) against closed forms, finite differences and
exact statistical facts."""
import math

import numpy as np
import pytest

NP = 9156


def _random_params(seed, scale=0.4):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, NP)


def test_parameter_count(oracle):
    assert oracle.lib().oracle_mlp_num_params() == NP == 8 * 64 + 64 + 2 * (64 * 64 + 64) + 4 * 64 + 4


def test_loss_gradient_matches_finite_differences(oracle):
    rng = np.random.default_rng(1)
    p = _random_params(2)
    x = rng.normal(0, 1, (24, 8))
    lab = rng.integers(0, 6, 24).astype(np.int32)    # 4, 5 (AMBIG, FAIL) are skipped
    loss, g = oracle.mlp_loss_grad(p, x, lab)
    idx = np.concatenate([rng.choice(np.arange(a, b), min(6, b - a), replace=False) for a, b in
                          [(0, 512), (512, 576), (576, 4672), (4672, 4736), (4736, 8832),
                           (8832, 8896), (8896, 9152), (9152, 9156)]])
    for i in idx:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (oracle.mlp_loss_grad(pp, x, lab)[0] - oracle.mlp_loss_grad(pm, x, lab)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_zero_network_closed_form(oracle):
    """All parameters zero: logits 0, softmax uniform, loss = ln 4, and the
    output-bias gradient is the mean of (1/4 - one-hot)."""
    p = np.zeros(NP)
    lab = np.array([0, 1, 1, 3, 2, 5], np.int32)
    x = np.random.default_rng(0).normal(0, 1, (6, 8))
    loss, g = oracle.mlp_loss_grad(p, x, lab)
    assert loss == pytest.approx(5 * math.log(4) / 6, rel=1e-15)
    want = np.array([0.25 * 5 - 1, 0.25 * 5 - 2, 0.25 * 5 - 1, 0.25 * 5 - 1]) / 6
    assert np.allclose(g[9152:9156], want, rtol=1e-14, atol=1e-16)
    assert np.all(g[:9152] == 0.0)


def test_adam_first_step_closed_form(oracle):
    """t = 1: m_hat = g, v_hat = g^2, so each parameter moves by -lr g/(|g| + eps)."""
    rng = np.random.default_rng(3)
    p = rng.normal(0, 1, 50)
    g = rng.normal(0, 1e-2, 50)
    p1, m, v = oracle.adam_step(p, np.zeros(50), np.zeros(50), g, 1, 1e-3)
    assert np.allclose(p1 - p, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-18)
    assert np.allclose(m, 0.1 * g, rtol=1e-15) and np.allclose(v, 0.001 * g * g, rtol=1e-15)


def test_proposal_normalisation_and_uniform_limit(oracle):
    dims = (4, 3, 2, 2, 2)
    x = oracle.proposal_grid(dims, 100.0, 0.1, 2, 3, np.zeros(8), np.ones(8))
    q = oracle.proposal(_random_params(4, 0.3), x, 1e-3, 0.2)
    N = int(np.prod(dims))
    assert abs(q.sum() - 1.0) < 1e-14 and np.all(q >= 0.2 / N * (1 - 1e-15))
    # constant reactive probability (zero weights, output bias fixes softmax
    # = (1/6, 1/3, 1/3, 1/6)) gives the uniform proposal
    p = np.zeros(NP)
    p[9153] = p[9154] = math.log(2.0)
    qu = oracle.proposal(p, x, 1e-3, 0.2)
    assert np.allclose(qu, 1.0 / N, rtol=1e-14)
    # grid centres: b = sqrt(b2max (i + 1/2)/n), cos theta centres, angles
    b_centres = np.unique(np.round(x[:, 1], 12))
    assert np.allclose(b_centres, np.sqrt(100.0 * (np.arange(4) + 0.5) / 4))


def test_sampler_frequencies_positions_and_weights(oracle):
    from scipy.stats import chisquare, kstest
    dims = (4, 2, 2, 2, 2)
    N = int(np.prod(dims))
    rng = np.random.default_rng(5)
    q = rng.uniform(0.2, 3.0, N)
    q /= q.sum()
    qfix, cdf = oracle.proposal_cdf(q)
    assert cdf[-1] == qfix.sum() and np.all(qfix == np.rint(q * 2.0 ** 40))
    n = 200_000
    b, u, w, cell = oracle.sample_proposal(dims, 100.0, qfix, cdf, n, seed=11)
    counts = np.bincount(cell, minlength=N)
    assert chisquare(counts, qfix / qfix.sum() * n).pvalue > 1e-3
    assert np.allclose(w, (cdf[-1] / N) / qfix[cell], rtol=1e-15)
    # decoded positions lie inside the drawn cell and are uniform there
    i_b2 = cell // 16
    frac_b2 = (b * b / 100.0) * dims[0] - i_b2
    assert np.all((frac_b2 >= 0) & (frac_b2 < 1))
    assert kstest(frac_b2, "uniform").pvalue > 1e-3
    i_cth = (cell // 8) % 2
    frac_c = u[:, 0] * dims[1] - i_cth
    assert np.all((frac_c >= 0) & (frac_c < 1))


def test_importance_sampling_is_unbiased_on_a_known_integral(oracle):
    """f = 1[b^2 < 25] 1[cos theta > 0.5] has uniform-measure mean
    (25/100) ((1 - 0.5)/2) = 0.0625; the weighted estimate from a skewed
    proposal falls within 3 standard errors for every seed."""
    dims = (8, 4, 2, 2, 2)
    N = int(np.prod(dims))
    rng = np.random.default_rng(6)
    q = rng.uniform(0.05, 2.0, N)
    q /= q.sum()
    qfix, cdf = oracle.proposal_cdf(q)
    for seed in range(5):
        b, u, w, cell = oracle.sample_proposal(dims, 100.0, qfix, cdf, 100_000, seed=seed)
        f = ((b * b < 25.0) & (2 * u[:, 0] - 1 > 0.5)).astype(float)
        mean, se = oracle.is_mean(w, f)
        assert abs(mean - 0.0625) <= 3 * se, (seed, mean, se)
        assert se < 0.002
