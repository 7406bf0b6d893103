"""FP64 oracle of the on-device PPO pieces (SceneFactory App. L, Tab.
app_ppo_hparams; the training loop of Alg. 1).

TEST INFRASTRUCTURE ONLY: used by tests/ and never by the product path.

Definitions (per agent, per rollout step t of a horizon T):
  diagonal Gaussian policy with mean mu (the actor's output) and a state-free
  log standard deviation s:  log pi(a) = sum_i -(a_i - mu_i)^2 / (2 e^{2 s_i}) - s_i - log(2 pi) / 2
  TD residual      delta_t = r_t + gamma (1 - d_t) V_{t+1} - V_t
  GAE              A_t = delta_t + gamma lambda (1 - d_t) A_{t+1},   A_T = 0
  return           R_t = A_t + V_t
  (d_t = 1 when the step ended the agent's episode; V_T is the critic's value
  of the state after the last step.)  Advantages are normalised over the
  rollout: (A - mean) / (std + 1e-8).
  PPO loss of a minibatch of B rows (clip eps, value coef c_v, entropy coef c_e):
    ratio = exp(log pi_new(a) - log pi_old(a))
    L = mean(-min(ratio A, clip(ratio, 1 - eps, 1 + eps) A)) + c_v mean((V - R)^2) - c_e H
    H = sum_i (s_i + log(2 pi e) / 2)                     (Gaussian entropy)
  KL(old || new) = sum_i [s_new - s_old + (e^{2 s_old} + (mu_old - mu_new)^2) / (2 e^{2 s_new}) - 1/2],
  averaged over the minibatch.
  Adaptive learning rate (App. L: "halves or doubles the rate to maintain the
  per-update KL near 0.01"): after each minibatch update, kl > 2 target ->
  lr / 2, kl < target / 2 -> lr * 2, clamped to [1e-6, 1e-2].
  Gradients are clipped to a global 2-norm of max_grad_norm before Adam.
"""
from __future__ import annotations

import math

import numpy as np


def gaussian_logp(a, mu, log_std):
    a, mu = np.asarray(a, np.float64), np.asarray(mu, np.float64)
    s = np.asarray(log_std, np.float64)
    return np.sum(-(a - mu) ** 2 / (2 * np.exp(2 * s)) - s - 0.5 * math.log(2 * math.pi), axis=-1)


def gae(rewards, values, dones, last_value, gamma, lam):
    """rewards, values, dones [T, A]; last_value [A].  Returns (advantages, returns) [T, A]."""
    r = np.asarray(rewards, np.float64)
    v = np.asarray(values, np.float64)
    d = np.asarray(dones, np.float64)
    T = r.shape[0]
    adv = np.zeros_like(r)
    nxt_v = np.asarray(last_value, np.float64)
    nxt_a = np.zeros_like(nxt_v)
    for t in range(T - 1, -1, -1):
        delta = r[t] + gamma * (1 - d[t]) * nxt_v - v[t]
        nxt_a = delta + gamma * lam * (1 - d[t]) * nxt_a
        adv[t] = nxt_a
        nxt_v = v[t]
    return adv, adv + v


def normalise(adv):
    adv = np.asarray(adv, np.float64)
    return (adv - adv.mean()) / (adv.std() + 1e-8)


def ppo_loss(mu, log_std, value, a, logp_old, adv, ret, clip, vf_coef, ent_coef):
    """Loss of one minibatch (scalar) and its parts."""
    lp = gaussian_logp(a, mu, log_std)
    ratio = np.exp(lp - np.asarray(logp_old, np.float64))
    adv = np.asarray(adv, np.float64)
    surr = np.minimum(ratio * adv, np.clip(ratio, 1 - clip, 1 + clip) * adv)
    pol = -np.mean(surr)
    vl = np.mean((np.asarray(value, np.float64) - np.asarray(ret, np.float64)) ** 2)
    ent = float(np.sum(np.asarray(log_std, np.float64) + 0.5 * math.log(2 * math.pi * math.e)))
    return pol + vf_coef * vl - ent_coef * ent, pol, vl, ent


def ppo_grads(mu, log_std, value, a, logp_old, adv, ret, clip, vf_coef, ent_coef):
    """Analytic gradient of ppo_loss with respect to mu [B, 3], log_std [3] and value [B].
    Where the clipped term is the smaller one and the ratio lies outside the
    clip range the surrogate's gradient is zero; at a tie the unclipped branch
    is taken."""
    mu = np.asarray(mu, np.float64)
    s = np.asarray(log_std, np.float64)
    a = np.asarray(a, np.float64)
    adv = np.asarray(adv, np.float64)
    B = mu.shape[0]
    lp = gaussian_logp(a, mu, s)
    ratio = np.exp(lp - np.asarray(logp_old, np.float64))
    unclipped = ratio * adv
    clipped = np.clip(ratio, 1 - clip, 1 + clip) * adv
    active = (unclipped <= clipped) | ((ratio >= 1 - clip) & (ratio <= 1 + clip))
    g_ratio = np.where(active, -adv / B, 0.0)             # d loss / d ratio
    g_lp = g_ratio * ratio                                # d loss / d log pi
    var = np.exp(2 * s)
    d_mu = g_lp[:, None] * (a - mu) / var
    d_s = np.sum(g_lp[:, None] * ((a - mu) ** 2 / var - 1.0), axis=0) - ent_coef
    d_v = 2 * vf_coef * (np.asarray(value, np.float64) - np.asarray(ret, np.float64)) / B
    return d_mu, d_s, d_v


def gaussian_kl(mu_old, log_std_old, mu_new, log_std_new):
    """Mean over rows of KL(N(mu_old, e^{2 s_old}) || N(mu_new, e^{2 s_new}))."""
    so, sn = np.asarray(log_std_old, np.float64), np.asarray(log_std_new, np.float64)
    mo, mn = np.asarray(mu_old, np.float64), np.asarray(mu_new, np.float64)
    kl = sn - so + (np.exp(2 * so) + (mo - mn) ** 2) / (2 * np.exp(2 * sn)) - 0.5
    return float(np.mean(np.sum(kl, axis=-1)))


def adapt_lr(lr, kl, target, lo=1e-6, hi=1e-2):
    if kl > 2 * target:
        return max(lo, lr / 2)
    if kl < target / 2:
        return min(hi, lr * 2)
    return lr
