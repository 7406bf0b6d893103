"""Pins of the PPO oracle: the Gaussian log-density against scipy, GAE against
its closed forms (lambda = 1: discounted return minus value; lambda = 0: the
TD residual; episode ends cut both), the loss gradient against central finite
differences, the Gaussian KL against numerical integration, and the
learning-rate rule's cases."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import ppo as PO


def test_logp_matches_scipy():
    rng = np.random.default_rng(1)
    mu = rng.normal(0, 1, (50, 3))
    s = np.array([-0.5, 0.2, -1.1])
    a = mu + np.exp(s) * rng.normal(0, 1, (50, 3))
    ref = stats.norm.logpdf(a, mu, np.exp(s)).sum(1)
    np.testing.assert_allclose(PO.gaussian_logp(a, mu, s), ref, rtol=1e-12, atol=1e-12)


def test_gae_closed_forms():
    rng = np.random.default_rng(2)
    T, A = 12, 5
    r = rng.normal(0, 1, (T, A))
    v = rng.normal(0, 1, (T, A))
    last = rng.normal(0, 1, A)
    d = np.zeros((T, A))
    g = 0.97
    # lambda = 1: A_t = sum_k g^k r_{t+k} + g^{T-t} V_T - V_t
    adv, ret = PO.gae(r, v, d, last, g, 1.0)
    for t in range(T):
        disc = sum(g ** k * r[t + k] for k in range(T - t)) + g ** (T - t) * last
        np.testing.assert_allclose(adv[t], disc - v[t], atol=1e-12)
        np.testing.assert_allclose(ret[t], disc, atol=1e-12)
    # lambda = 0: the TD residual
    adv0, _ = PO.gae(r, v, d, last, g, 0.0)
    nxt = np.vstack([v[1:], last[None]])
    np.testing.assert_allclose(adv0, r + g * nxt - v, atol=1e-12)
    # an episode end at t = 5 cuts the sums: agent 0's A_5 only sees r_5 - V_5
    d[5, 0] = 1.0
    adv1, _ = PO.gae(r, v, d, last, g, 1.0)
    assert abs(adv1[5, 0] - (r[5, 0] - v[5, 0])) < 1e-12
    disc4 = r[4, 0] + g * r[5, 0]
    assert abs(adv1[4, 0] - (disc4 - v[4, 0])) < 1e-12


@pytest.mark.parametrize("seed", [3, 4])
def test_loss_gradient_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    B = 40
    mu = rng.normal(0, 0.5, (B, 3))
    s = rng.normal(-0.5, 0.2, 3)
    val = rng.normal(0, 1, B)
    a = mu + np.exp(s) * rng.normal(0, 1, (B, 3))
    # old log-probs spread so that some ratios fall outside the clip range
    lpo = PO.gaussian_logp(a, mu, s) + rng.normal(0, 0.3, B)
    adv = rng.normal(0, 1, B)
    ret = rng.normal(0, 1, B)
    args = (0.15, 1.0, 3e-5)
    d_mu, d_s, d_v = PO.ppo_grads(mu, s, val, a, lpo, adv, ret, *args)
    f = lambda mu_, s_, v_: PO.ppo_loss(mu_, s_, v_, a, lpo, adv, ret, *args)[0]
    h = 1e-6
    for idx in [(0, 0), (7, 2), (19, 1), (33, 0)]:
        e = np.zeros_like(mu); e[idx] = h
        fd = (f(mu + e, s, val) - f(mu - e, s, val)) / (2 * h)
        assert abs(fd - d_mu[idx]) < 1e-7 * max(1, abs(fd)), (idx, fd, d_mu[idx])
    for i in range(3):
        e = np.zeros(3); e[i] = h
        fd = (f(mu, s + e, val) - f(mu, s - e, val)) / (2 * h)
        assert abs(fd - d_s[i]) < 1e-7 * max(1, abs(fd))
    for j in [0, 11, 39]:
        e = np.zeros(B); e[j] = h
        fd = (f(mu, s, val + e) - f(mu, s, val - e)) / (2 * h)
        assert abs(fd - d_v[j]) < 1e-8
    # some rows are clipped (zero surrogate gradient), some are not
    ratio = np.exp(PO.gaussian_logp(a, mu, s) - lpo)
    out = (ratio < 0.85) | (ratio > 1.15)
    assert out.any() and (~out).any()


def test_gaussian_kl_matches_numerical_integration():
    mo, so, mn, sn = 0.3, -0.2, -0.1, 0.25
    p = lambda x: stats.norm.pdf(x, mo, math.exp(so))
    q = lambda x: stats.norm.pdf(x, mn, math.exp(sn))
    num, _ = integrate.quad(lambda x: p(x) * (math.log(p(x)) - math.log(q(x))), -12, 12)
    kl = PO.gaussian_kl(np.array([[mo]]), np.array([so]), np.array([[mn]]), np.array([sn]))
    assert abs(kl - num) < 1e-9
    assert PO.gaussian_kl(np.ones((4, 3)), np.zeros(3), np.ones((4, 3)), np.zeros(3)) == 0.0


def test_adaptive_lr_rule():
    assert PO.adapt_lr(2e-4, 0.03, 0.01) == 1e-4
    assert PO.adapt_lr(2e-4, 0.004, 0.01) == 4e-4
    assert PO.adapt_lr(2e-4, 0.01, 0.01) == 2e-4
    assert PO.adapt_lr(8e-3, 0.0, 0.01) == 1e-2
