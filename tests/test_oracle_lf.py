"""Pins of the late-fusion actor-critic oracle (App. E).

The masked max-pool is pinned by the properties that define a set encoder:
invariance to the order of the valid slots, to the contents of padded slots and
to a duplicated slot; the whole network by a second formulation written as
plain loops over the valid slots only (no padding, no -inf), including empty
groups; and the actor / critic split by their independence.
"""
import numpy as np
import pytest

from oracle import lf as LF


def params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    P = []
    for net in ("actor", "critic"):
        for _, o, i in LF.net_layers(net):
            P.append(rng.normal(0, scale / np.sqrt(i), o * i))
            P.append(rng.normal(0, 0.1, o))
    P.append(np.full(3, -0.5))
    return np.concatenate(P)


def observations(seed, A, n_road, n_veh):
    rng = np.random.default_rng(seed)
    obs = rng.normal(0, 1, (A, LF.OBS))
    for a in range(A):   # padding slots are zero, as the observation writes them
        obs[a, LF.ROAD0 + n_road[a] * LF.PT:LF.VEH0] = 0
        obs[a, LF.VEH0 + n_veh[a] * LF.NB:] = 0
    return obs


def test_parameter_count():
    per = lambda out: (11 * 64 + 64 + 64 * 64 + 64 + 5 * 96 + 96 + 96 * 96 + 96 + 7 * 96 + 96 + 96 * 96 + 96
                       + 256 * 128 + 128 + 128 * 64 + 64 + 64 * out + out)
    assert LF.num_params() == per(3) + per(1) + 3


def test_loop_formulation_agrees_including_empty_groups():
    p = params(1)
    n_road = np.array([0, 1, 3, 7])
    n_veh = np.array([2, 0, 1, 24])
    obs = observations(2, 4, n_road, n_veh)
    mean, value = LF.forward(p, obs, n_road, n_veh)
    for a in range(4):
        m, v = LF.forward_loops(p, obs[a], int(n_road[a]), int(n_veh[a]))
        np.testing.assert_allclose(mean[a], m, rtol=1e-12, atol=1e-12)
        assert abs(value[a] - v) < 1e-12


def test_set_invariances():
    p = params(3)
    rng = np.random.default_rng(4)
    n_road = np.array([40, 350, 5])
    n_veh = np.array([15, 3, 24])
    obs = observations(5, 3, n_road, n_veh)
    mean, value = LF.forward(p, obs, n_road, n_veh)
    # order of the valid slots
    o2 = obs.copy()
    for a in range(3):
        r = o2[a, LF.ROAD0:LF.VEH0].reshape(LF.KR, LF.PT)
        r[:n_road[a]] = r[rng.permutation(n_road[a])]
        v = o2[a, LF.VEH0:].reshape(LF.KV, LF.NB)
        v[:n_veh[a]] = v[rng.permutation(n_veh[a])]
    m2, v2 = LF.forward(p, o2, n_road, n_veh)
    np.testing.assert_allclose(m2, mean, atol=1e-12)
    np.testing.assert_allclose(v2, value, atol=1e-12)
    # contents of the padded slots
    o3 = obs.copy()
    for a in range(3):
        o3[a, LF.ROAD0 + n_road[a] * LF.PT:LF.VEH0] = rng.normal(0, 50, (LF.KR - n_road[a]) * LF.PT)
        o3[a, LF.VEH0 + n_veh[a] * LF.NB:] = rng.normal(0, 50, (LF.KV - n_veh[a]) * LF.NB)
    m3, v3 = LF.forward(p, o3, n_road, n_veh)
    np.testing.assert_allclose(m3, mean, atol=1e-12)
    np.testing.assert_allclose(v3, value, atol=1e-12)
    # a duplicated valid slot (max is idempotent)
    o4 = obs.copy()
    o4[2, LF.ROAD0 + 5 * LF.PT:LF.ROAD0 + 6 * LF.PT] = o4[2, LF.ROAD0:LF.ROAD0 + LF.PT]
    n4 = n_road.copy(); n4[2] = 6
    m4, v4 = LF.forward(p, o4, n4, n_veh)
    np.testing.assert_allclose(m4, mean, atol=1e-12)
    # ... while a new, different slot does change the output
    o4[2, LF.ROAD0 + 5 * LF.PT:LF.ROAD0 + 6 * LF.PT] = [3.0, -3.0, 1.0, 0.0, 1.0]
    m5, _ = LF.forward(p, o4, n4, n_veh)
    assert np.abs(m5[2] - mean[2]).max() > 1e-6


def test_actor_and_critic_are_independent():
    p = params(6)
    n_road, n_veh = np.array([10, 0]), np.array([4, 1])
    obs = observations(7, 2, n_road, n_veh)
    mean, value = LF.forward(p, obs, n_road, n_veh)
    half = sum(o * i + o for _, o, i in LF.net_layers("actor"))
    pa, pc = p.copy(), p.copy()
    pa[:half] += 0.3           # actor changed
    pc[half:-3] += 0.3         # critic changed
    ma, va = LF.forward(pa, obs, n_road, n_veh)
    mc, vc = LF.forward(pc, obs, n_road, n_veh)
    np.testing.assert_array_equal(va, value)
    np.testing.assert_array_equal(mc, mean)
    assert np.abs(ma - mean).max() > 1e-3 and np.abs(vc - value).max() > 1e-3


def test_gradients_match_central_differences():
    """The analytic gradient of L = sum(dmean * mean) + sum(dvalue * value)
    against central differences of the forward pass, on 20 parameters drawn
    from every layer of both networks (3 agents: full groups, a partly filled
    road group, an empty vehicle group)."""
    n_road, n_veh = [4, 2, 3], [3, 0, 1]
    P = params(11)
    obs = observations(12, 3, n_road, n_veh)
    rng = np.random.default_rng(13)
    dmean, dvalue = rng.normal(0, 1, (3, 3)), rng.normal(0, 1, 3)
    G = LF.gradients(P, obs, n_road, n_veh, dmean, dvalue)
    assert G.shape == P.shape

    def L(q):
        m, v = LF.forward(q, obs, n_road, n_veh)
        return float((m * dmean).sum() + (v * dvalue).sum())

    k, checked, expected = 0, 0, 0
    for net in ("actor", "critic"):
        for _, o, i in LF.net_layers(net):
            nw, nb = min(15, o * i), min(5, o)
            picks = [k + int(t) for t in rng.choice(o * i, nw, replace=False)]
            picks += [k + o * i + int(t) for t in rng.choice(o, nb, replace=False)]
            for j in picks:
                e = 1e-6
                qp, qm = P.copy(), P.copy()
                qp[j] += e
                qm[j] -= e
                fd = (L(qp) - L(qm)) / (2 * e)
                assert abs(fd - G[j]) <= 1e-6 + 1e-5 * abs(fd), (net, j, fd, G[j])
                checked += 1
            expected += nw + nb
            k += o * i + o
    assert checked == expected
    assert np.all(G[-3:] == 0)


def test_gradient_of_a_pool_reaches_only_its_argmax_slot():
    """A feature's pooled gradient reaches the encoder through one slot: the
    layer-1 weight gradient of a road encoder vanishes when every valid slot
    but the maximising ones is changed (their inputs matter to the gradient
    only through the max)."""
    n_road, n_veh = [3], [0]
    P = params(21)
    obs = observations(22, 1, n_road, n_veh)
    dmean = np.array([[1.0, -0.5, 0.25]])
    G = LF.gradients(P, obs, n_road, n_veh, dmean, np.zeros(1))
    # a copy of the first road slot appended as a fourth (tied) slot changes nothing
    obs2 = obs.copy()
    obs2[0, LF.ROAD0 + 3 * LF.PT:LF.ROAD0 + 4 * LF.PT] = obs[0, LF.ROAD0:LF.ROAD0 + LF.PT]
    G2 = LF.gradients(P, obs2, [4], n_veh, dmean, np.zeros(1))
    assert np.allclose(G, G2, rtol=0, atol=1e-12)


def test_gradient_with_a_given_maximising_slot():
    """The slot choice of the max-pool's gradient can be given: the natural
    choice reproduces the default, and a tied duplicate slot gives the same
    gradient as the slot it copies."""
    n_road, n_veh = [3, 2], [2, 1]
    P = params(31)
    obs = observations(32, 2, n_road, n_veh)
    rng = np.random.default_rng(33)
    dmean, dvalue = rng.normal(0, 1, (2, 3)), rng.normal(0, 1, 2)
    G = LF.gradients(P, obs, n_road, n_veh, dmean, dvalue)
    U = LF.unpack(P)

    def first_max(h2, cnts):   # [A, 96] first maximising valid slot per feature
        K = h2.shape[1]
        return np.where(np.arange(K)[None, :, None] < np.asarray(cnts)[:, None, None], h2, -np.inf).argmax(axis=1)

    arg = [[first_max(LF.slot_outputs(U[net], obs, grp), cnts)
            for grp, cnts in (("road", n_road), ("vehicles", n_veh))] for net in ("actor", "critic")]
    assert np.array_equal(LF.gradients(P, obs, n_road, n_veh, dmean, dvalue, arg=arg), G)
    # agent 0's road slot 0 duplicated as slot 3: pointing every feature held by slot 0 at slot 3 changes nothing
    obs2 = obs.copy()
    obs2[0, LF.ROAD0 + 3 * LF.PT:LF.ROAD0 + 4 * LF.PT] = obs[0, LF.ROAD0:LF.ROAD0 + LF.PT]
    arg2 = [[a.copy() for a in row] for row in arg]
    for ni in range(2):
        arg2[ni][0][0] = np.where(arg[ni][0][0] == 0, 3, arg[ni][0][0])
    G2 = LF.gradients(P, obs2, [4, 2], n_veh, dmean, dvalue, arg=arg2)
    assert np.allclose(G2, G, rtol=0, atol=1e-12)
