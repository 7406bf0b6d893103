"""GPU parity of the on-device PPO (App. L) against the FP64 oracle
(oracle/ppo.py).

Tolerances: the rollout's log-probabilities are FP32 evaluations of the
Gaussian density (|d| <= 1e-4 on values of order 1-10); GAE is an FP32
recursion over the horizon (|d| <= 2e-4 after normalisation); the loss
gradients and KL are FP32 per-row formulas fed the GPU's own actor / critic
outputs (relative 1e-4 of the largest entry, sums over rows 1e-3 relative).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ppo as PO
from paper_2605_08528_b300 import sf, synth

pytestmark = pytest.mark.gpu


def setup(horizon=16, minibatches=4, epochs=2, worlds=4, seed=3):
    sc = synth.procedural_scene(worlds, 16, seed_base=1700)
    stream = torch.cuda.Stream()
    W = sf.World(sc, seed=seed, flags=sf.FLAG_AUTO_RESET, stream=stream)
    with torch.cuda.stream(stream):
        sf.sf_reset(W.h, torch.ones(W.A, dtype=torch.uint8, device="cuda"))
    actor = sf.init_policy(seed=seed, stream=stream, out_scale=0.1)
    critic = sf.init_value(seed=seed + 1, stream=stream)
    cfg = sf.sf_ppo_default_config(horizon=horizon, minibatches=minibatches, epochs=epochs, init_log_std=-0.5)
    p = sf.sf_ppo_create(W.h, actor, critic, cfg)
    return W, actor, critic, p, cfg, stream


def view(ptr, shape, dtype="float32"):
    return sf.device_view(ptr, shape, dtype).cpu().numpy()


def rollout_arrays(p):
    r = sf.sf_ppo_rollout_ptrs(p)
    T, A = r.horizon, r.num_agents
    return dict(T=T, A=A, B=r.minibatch_rows, obs=view(r.obs, (T, A, 320)), act=view(r.actions, (T, A, 3)),
                mean=view(r.mean, (T, A, 3)), logp=view(r.logp, (T, A)), value=view(r.value, (T + 1, A)),
                reward=view(r.reward, (T, A)), done=view(r.done, (T, A), "uint8"), adv=view(r.advantage, (T, A)),
                ret=view(r.ret, (T, A)), raw=r)


def test_rollout_sampling_and_values():
    W, actor, critic, p, cfg, stream = setup()
    sf.sf_ppo_collect(p)
    torch.cuda.synchronize()
    R = rollout_arrays(p)
    s = sf.sf_ppo_log_std(p)
    np.testing.assert_allclose(s, -0.5)
    ref = PO.gaussian_logp(R["act"], R["mean"], s)
    assert np.abs(R["logp"] - ref).max() <= 1e-4
    z = (R["act"] - R["mean"]) / np.exp(s)
    print("standard normal draws: mean %.3f std %.3f over %d" % (z.mean(), z.std(), z.size))
    assert abs(z.mean()) < 0.08 and abs(z.std() - 1.0) < 0.06
    # the stored values are the critic's outputs on the stored observations
    T, A = R["T"], R["A"]
    v = torch.zeros((A, 1), device="cuda")
    for t in (0, T // 2, T - 1):
        sf.sf_mlp_forward(critic, torch.as_tensor(R["obs"][t]).cuda(), A, v)
        sf.sf_mlp_sync(critic)
        assert np.abs(v.cpu().numpy()[:, 0] - R["value"][t]).max() <= 1e-5
    assert np.isfinite(R["reward"]).all() and set(np.unique(R["done"])) <= {0, 1}
    sf.sf_ppo_destroy(p)
    W.close()


def test_gae_and_loss_gradients_match_the_oracle():
    W, actor, critic, p, cfg, stream = setup()
    sf.sf_ppo_collect(p)
    stats = sf.sf_ppo_update(p)
    R = rollout_arrays(p)
    adv, ret = PO.gae(R["reward"], R["value"][:-1], R["done"], R["value"][-1], cfg.gamma, cfg.lam)
    assert np.abs(R["ret"] - ret).max() <= 2e-4 * max(1.0, np.abs(ret).max())
    assert np.abs(R["adv"] - PO.normalise(adv)).max() <= 2e-4
    print("update stats (reward, policy loss, value loss, kl, lr, grad norm):", stats)
    assert np.isfinite(stats).all() and 1e-6 <= stats[4] <= 1e-2
    # loss gradients of the first minibatch-sized block of rows, with the current parameters
    n = R["B"]
    rows = np.arange(n)
    t, a = rows // R["A"], rows % R["A"]
    small = np.zeros((n, 12), np.float32)
    small[:, 0:3] = R["act"][t, a]
    small[:, 3:6] = R["mean"][t, a]
    small[:, 6] = R["logp"][t, a]
    small[:, 7] = R["adv"][t, a]
    small[:, 8] = R["ret"][t, a]
    obs = torch.as_tensor(np.ascontiguousarray(R["obs"][t, a])).cuda()
    d_small = torch.as_tensor(small).cuda()
    mu = torch.zeros((n, 3), device="cuda"); v = torch.zeros(n, device="cuda")
    dmu = torch.zeros((n, 3), device="cuda"); dv = torch.zeros(n, device="cuda")
    out = sf.sf_ppo_loss_grads(p, obs, d_small, n, mu, v, dmu, dv)
    mu, v, dmu, dv = mu.cpu().numpy(), v.cpu().numpy(), dmu.cpu().numpy(), dv.cpu().numpy()
    s = sf.sf_ppo_log_std(p)
    g_mu, g_s, g_v = PO.ppo_grads(mu, s, v, small[:, 0:3], small[:, 6], small[:, 7], small[:, 8], cfg.clip,
                                  cfg.vf_coef, cfg.ent_coef)
    assert np.abs(dmu - g_mu).max() <= 1e-4 * np.abs(g_mu).max() + 1e-9
    assert np.abs(dv - g_v).max() <= 1e-4 * np.abs(g_v).max() + 1e-9
    assert np.abs(out[:3] - g_s).max() <= 1e-3 * np.abs(g_s).max() + 1e-7
    loss, pol, vl, ent = PO.ppo_loss(mu, s, v, small[:, 0:3], small[:, 6], small[:, 7], small[:, 8], cfg.clip,
                                     cfg.vf_coef, cfg.ent_coef)
    assert abs(out[3] - pol) <= 1e-3 * max(1.0, abs(pol)) and abs(out[4] - vl) <= 1e-3 * max(1.0, vl)
    kl = PO.gaussian_kl(small[:, 3:6], np.full(3, -0.5), mu, s)
    assert abs(out[5] - kl) <= 1e-3 * max(kl, 1e-3)
    sf.sf_ppo_destroy(p)
    W.close()


def test_training_fits_the_value_function():
    W, actor, critic, p, cfg, stream = setup(horizon=32, minibatches=4, epochs=5, worlds=8)
    vals = []
    for it in range(6):
        sf.sf_ppo_collect(p)
        st = sf.sf_ppo_update(p)
        vals.append(float(st[2]))
        assert np.isfinite(st).all()
    print("value loss per update:", vals, "log std:", sf.sf_ppo_log_std(p))
    assert min(vals[3:]) < vals[0]
    sf.sf_ppo_destroy(p)
    W.close()


def test_updates_are_deterministic():
    """Two PPO runs from the same seeds give bit-identical statistics, log
    standard deviations and weights: every reduction of the update (GAE
    moments, loss sums, split-K weight gradients, bias gradients, the gradient
    norm) runs in a fixed order."""
    out = []
    for _ in range(2):
        W, actor, critic, p, cfg, stream = setup(horizon=16, minibatches=4, epochs=2, worlds=4)
        stats = []
        for it in range(2):
            sf.sf_ppo_collect(p)
            stats.append(np.asarray(sf.sf_ppo_update(p)))
        torch.cuda.synchronize()
        weights = [sf.sf_mlp_get_layer(m, l, o, i)[0]
                   for m, dims in ((actor, (320, 512, 512, 3)), (critic, (320, 512, 512, 1)))
                   for l, (i, o) in enumerate(zip(dims[:-1], dims[1:]))]
        out.append((np.stack(stats), np.asarray(sf.sf_ppo_log_std(p)), weights))
        sf.sf_ppo_destroy(p)
        sf.sf_mlp_destroy(actor)
        sf.sf_mlp_destroy(critic)
        W.close()
    (s1, l1, w1), (s2, l2, w2) = out
    assert np.array_equal(s1, s2) and np.array_equal(l1, l2)
    assert all(np.array_equal(a, b) for a, b in zip(w1, w2))
