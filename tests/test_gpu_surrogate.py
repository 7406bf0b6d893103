"""GPU tests of the learned dynamics surrogate against the oracle.

* collected training rows: features and targets of every gated agent equal
  the FP64 oracle's definitions evaluated on the GPU's own FP32 states
  (features to 1e-5 relative, targets to 5e-5 m or m/s absolute: they are
  differences of FP32 states), and the gate selects the same agents;
* agents the gate leaves to the physics evolve bit-identically to a plain step;
* the trained surrogate's 1 s (30-step) rollout position error against the
  FP64 oracle physics: mean <= 1 cm (the target), p90 / p99 / max printed;
* a seeded collection gives the same rows on every run, a cap keeps the first
  rows, and training on the same rows gives the same loss and weights.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from oracle import surrogate as OS
from paper_2605_08528_b300 import sf, synth

pytestmark = pytest.mark.gpu
DT = 1.0 / 30.0


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def oracle_gate(F, I, sc):
    """The gate from FP32 state rows: alive, mu >= 0.3, speed <= 35, tilt < 10 deg,
    no other alive centre within 4.8466 + 2 + |dv| dt."""
    A = len(F)
    g = np.zeros(A, bool)
    alive = (I[:, O.I_STATUS] & O.ALIVE) != 0
    for w in range(sc.num_worlds):
        a0, a1 = sc.agent_off[w], sc.agent_off[w + 1]
        for i in range(a0, a1):
            f = F[i].astype(np.float64)
            if not alive[i] or f[O.F_MU] < 0.3 or np.linalg.norm(f[7:10]) > 35:
                continue
            if 1 - 2 * (f[4] ** 2 + f[5] ** 2) < math.cos(math.radians(10)):
                continue
            ok = True
            for j in range(a0, a1):
                if j == i or not alive[j]:
                    continue
                reach = 4.8466483 + 2.0 + np.linalg.norm(F[j, 7:9].astype(np.float64) - f[7:9]) * DT
                if np.linalg.norm(F[j, :2].astype(np.float64) - f[:2]) <= reach:
                    ok = False
            g[i] = ok
    return g


def test_collected_rows_match_the_oracle():
    sc = synth.procedural_scene(12, 4, seed_base=900)
    W = sf.World(sc, seed=3, flags=sf.FLAG_AUTO_RESET)
    sf.sf_reset(W.h, dev(np.ones(W.A, np.uint8)))
    s = sf.sf_surrogate_create()
    cap = 10000
    dx = torch.zeros((cap, 30), device="cuda")
    dy = torch.zeros((cap, 16), device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    acts = synth.ou_actions(W.A, 8, seed=5)
    checked = 0
    for t in range(8):
        F0, I0, _ = sf.sf_get_state(W.h)
        before = int(cnt.item())
        sf.sf_surrogate_collect(W.h, s, dev(acts[t]), dx, dy, cap, cnt)
        F1, I1, _ = sf.sf_get_state(W.h)
        n = int(cnt.item()) - before
        g = oracle_gate(F0, I0, sc)
        ev = I1[:, O.I_EVENTS]
        keep = g & ((ev & (O.EV["respawned"] | O.EV["nonfinite"] | O.EV["collision"] | O.EV["crash"])) == 0)
        keep &= (I1[:, O.I_STATUS] & O.ALIVE) != 0
        assert abs(n - int(keep.sum())) <= 1, (t, n, int(keep.sum()))     # a gate decision within rounding
        X = dx[before:before + n].cpu().numpy()
        Y = dy[before:before + n].cpu().numpy()
        rows = []
        for a in np.nonzero(keep)[0]:
            xo = OS.features(F0[a], acts[t][a])
            yo = OS.targets(F0[a], F1[a], DT)
            k = int(np.argmin(np.abs(X - xo).sum(1)))
            rows.append(k)
            assert np.abs(X[k] - xo).max() <= 1e-5 * max(1.0, np.abs(xo).max()), (t, a)
            assert np.abs(Y[k] - yo).max() <= 5e-5, (t, a, float(np.abs(Y[k] - yo).max()))
            checked += 1
        if n == int(keep.sum()):
            assert rows == list(range(n)), t       # one call's rows follow the agents' order
    assert checked > 50
    sf.sf_surrogate_destroy(s)


def collect(sc, steps, cap, seed=3):
    W = sf.World(sc, seed=seed, flags=sf.FLAG_AUTO_RESET)
    sf.sf_reset(W.h, dev(np.ones(W.A, np.uint8)))
    s = sf.sf_surrogate_create()
    dx = torch.zeros((cap, 30), device="cuda")
    dy = torch.zeros((cap, 16), device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    acts = dev(synth.ou_actions(W.A, steps, seed=7))
    for t in range(steps):
        sf.sf_surrogate_collect(W.h, s, acts[t], dx, dy, cap, cnt)
    torch.cuda.synchronize()
    out = int(cnt.item()), dx.cpu().numpy(), dy.cpu().numpy()
    sf.sf_surrogate_destroy(s)
    W.close()
    return out


def test_collection_repeats_and_cap_keeps_the_first_rows():
    """Two collections from the same seeded worlds give the same rows bit for
    bit (the training set, its normalisation and the trained weights repeat
    from run to run); a collection cut at a small cap keeps exactly the first
    rows of the uncut one, and its counter still counts every transition."""
    sc = synth.procedural_scene(40, 16, seed_base=910)       # 640 agents: two 512-agent chunks
    n1, x1, y1 = collect(sc, 24, 20000)
    n2, x2, y2 = collect(sc, 24, 20000)
    assert n1 == n2 and 1000 < n1 <= 20000
    assert np.array_equal(x1.view(np.uint32), x2.view(np.uint32))
    assert np.array_equal(y1.view(np.uint32), y2.view(np.uint32))
    cap = 777
    n3, x3, y3 = collect(sc, 24, cap)
    assert n3 == n1
    assert np.array_equal(x3.view(np.uint32), x1[:cap].view(np.uint32))
    assert np.array_equal(y3.view(np.uint32), y1[:cap].view(np.uint32))
    # training on the same rows with the same seed gives the same loss, statistics and weights
    dims = [30, 256, 256, 256, 16]
    got = []
    for _ in range(2):
        s = sf.sf_surrogate_create()
        loss = sf.sf_surrogate_train(s, dev(x1[:n1]), dev(y1[:n1]), n1, batch=1024, steps=200, lr=3e-3, seed=11)
        m = sf.sf_surrogate_mlp(s)
        got.append([np.array([loss], np.float32), sf.sf_surrogate_stats(s)] +
                   [a for l in range(4) for a in sf.sf_mlp_get_layer(m, l, dims[l + 1], dims[l])[:2]])
        sf.sf_surrogate_destroy(s)
    for a, b in zip(*got):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_ungated_agents_follow_the_physics_exactly():
    sc = synth.procedural_scene(8, 16, seed_base=950, weather="uniform")
    s = sf.sf_surrogate_create()
    W1 = sf.World(sc, seed=2, flags=sf.FLAG_AUTO_RESET)
    W2 = sf.World(sc, seed=2, flags=sf.FLAG_AUTO_RESET)
    for W in (W1, W2):
        sf.sf_reset(W.h, dev(np.ones(W.A, np.uint8)))
    act = dev(synth.ou_actions(W1.A, 1, seed=1)[0])
    F0, I0, _ = sf.sf_get_state(W1.h)
    g = oracle_gate(F0, I0, sc)
    sf.sf_step(W1.h, act)
    sf.sf_step_surrogate(W2.h, s, act)
    F1, I1, _ = sf.sf_get_state(W1.h)
    F2, I2, _ = sf.sf_get_state(W2.h)
    _, used = sf.sf_surrogate_audit(W2.h)
    assert abs(used - int(g.sum())) <= 1
    resp = ((I1[:, O.I_EVENTS] | I2[:, O.I_EVENTS]) & O.EV["respawned"]) != 0
    same = ~g & ~resp                       # respawn spacing sees every agent's new position
    assert same.sum() > 10
    bad = np.nonzero(same & (F1[:, :19] != F2[:, :19]).any(1))[0]
    for a in bad[:4]:
        cols = np.nonzero(F1[a, :19] != F2[a, :19])[0]
        print("agent", a, "columns", cols, "max |d|", float(np.abs(F1[a, :19] - F2[a, :19]).max()))
    assert np.array_equal(F1[same][:, :19], F2[same][:, :19])
    sf.sf_surrogate_destroy(s)


def test_trained_surrogate_rollout_error_against_the_oracle():
    from paper_2605_08528_b300 import surrogate as SU
    s, n, loss = SU.collect_and_train(synth.procedural_scene(128, 16, seed_base=3000), transitions=4_000_000,
                                      train_steps=40000, seed=31)
    print("training rows", n, "final normalised loss %.4f" % loss)
    assert n > 1_000_000 and loss < 0.1
    # 1 s rollouts of lone agents (one per world, mu >= 0.3 cells only) against the FP64 physics
    scw = synth.procedural_scene(96, 1, seed_base=3500)
    scw.precip[:] = np.minimum(scw.precip, 2)                  # keep mu >= 0.3 (no snow)
    W = sf.World(scw, seed=21, flags=sf.FLAG_INVINCIBLE)
    sf.sf_reset(W.h, dev(np.ones(W.A, np.uint8)))
    warm = synth.ou_actions(W.A, 40, seed=31)
    for t in range(10):
        sf.sf_step(W.h, dev(warm[t]))
    F0, I0, _ = sf.sf_get_state(W.h)
    orc = O.Oracle(scw)
    Fo, Io = F0.astype(np.float64), I0.copy()
    used_total = 0
    for t in range(30):
        a = warm[10 + t]
        sf.sf_step_surrogate(W.h, s, dev(a))
        _, used = sf.sf_surrogate_audit(W.h)
        used_total += used
        orc.step(Fo, Io, a.astype(np.float64), flags=O.FLAG_INVINCIBLE, want_obs=False)
    F1, _, _ = sf.sf_get_state(W.h)
    err = np.linalg.norm(F1[:, :3] - Fo[:, :3], axis=1)
    print("surrogate 1 s rollout position error vs FP64 oracle: mean %.4f m, p90 %.4f m, p99 %.4f m, max %.4f m "
          "(agent-steps on the surrogate %d of %d)" % (err.mean(), np.percentile(err, 90), np.percentile(err, 99),
                                                       err.max(), used_total, 30 * W.A))
    assert used_total > 0.8 * 30 * W.A
    assert np.isfinite(err).all() and err.mean() <= 1e-2
    # the audit measures the same kind of error on one step
    sf.sf_step_surrogate(W.h, s, dev(warm[0]), audit=True)
    e1, used = sf.sf_surrogate_audit(W.h)
    print("audit: max one-step position error %.5f m" % e1)
    assert used == 0 and 0.0 < e1 < 0.5
    sf.sf_surrogate_destroy(s)
