"""FP64 oracle of the paper's late-fusion actor-critic network (App. E).

TEST INFRASTRUCTURE ONLY: used by tests/ and never by the product path.

Each of the two networks (actor, critic; no weight sharing) splits the
1,929-value observation (App. D) into its groups and encodes them separately:
  ego      11 -> 64 -> 64                     (ELU after each layer)
  road     5 -> 96 -> 96 on each of the 350 slots, then a masked max-pool
  vehicles 7 -> 96 -> 96 on each of the 24 slots, then a masked max-pool
The masked max-pool fills padded slots with -inf before the maximum (App. E
modification (i)).  The three embeddings are concatenated in that order
(64 + 96 + 96 = 256) and pass the trunk 256 -> 128 -> 64 (ELU); the actor head
projects to the 3 action means, the critic head to one value (both linear).
The diagonal Gaussian's log standard deviation is a free 3-vector.

Readings: a slot is padding when its index is at or beyond the group's count
(the observation fills a prefix of the slots); a group with no valid slot
pools to zeros (the -inf of an empty maximum is not a usable input).

Parameters are a flat float vector: for the actor then the critic, each layer's
weight [out][in] row-major followed by its bias [out], layers in the order of
LAYERS; then log_std[3].
"""
from __future__ import annotations

import numpy as np

from oracle import mlp as MO

EGO, KR, PT, KV, NB = 11, 350, 5, 24, 7
OBS = EGO + KR * PT + KV * NB          # 1929
ROAD0, VEH0 = EGO, EGO + KR * PT

# (name, out, in) of one network, in parameter order
LAYERS = [("ego0", 64, 11), ("ego1", 64, 64), ("road0", 96, 5), ("road1", 96, 96), ("veh0", 96, 7),
          ("veh1", 96, 96), ("trunk0", 128, 256), ("trunk1", 64, 128), ("head", None, 64)]
HEAD_OUT = {"actor": 3, "critic": 1}


def net_layers(net):
    return [(n, HEAD_OUT[net] if o is None else o, i) for n, o, i in LAYERS]


def num_params() -> int:
    return sum(o * i + o for net in ("actor", "critic") for _, o, i in net_layers(net)) + 3


def unpack(flat):
    """Flat vector -> {"actor": {layer: (W, b)}, "critic": {...}, "log_std": [3]} (float64)."""
    flat = np.asarray(flat, np.float64)
    assert flat.shape == (num_params(),)
    out, k = {}, 0
    for net in ("actor", "critic"):
        d = {}
        for n, o, i in net_layers(net):
            W = flat[k:k + o * i].reshape(o, i); k += o * i
            b = flat[k:k + o]; k += o
            d[n] = (W, b)
        out[net] = d
    out["log_std"] = flat[k:k + 3]
    return out


def _dense(x, Wb):
    W, b = Wb
    return x @ W.T + b


def _set_encoder(p, l0, l1, slots, count):
    """slots [A, K, F], count [A] -> masked max over the valid slots [A, 96]."""
    h = MO.act(_dense(slots, p[l0]), MO.ELU)
    h = MO.act(_dense(h, p[l1]), MO.ELU)                       # [A, K, 96]
    K = slots.shape[1]
    valid = np.arange(K)[None, :] < np.asarray(count)[:, None]
    h = np.where(valid[:, :, None], h, -np.inf)
    pooled = h.max(axis=1)
    return np.where(np.isfinite(pooled), pooled, 0.0)         # empty group -> zeros


def embeddings(p, obs, n_road, n_veh):
    """The 256-value trunk input of one network: [ego 64 | road 96 | vehicles 96]."""
    obs = np.asarray(obs, np.float64)
    A = obs.shape[0]
    ego = MO.act(_dense(MO.act(_dense(obs[:, :EGO], p["ego0"]), MO.ELU), p["ego1"]), MO.ELU)
    road = _set_encoder(p, "road0", "road1", obs[:, ROAD0:VEH0].reshape(A, KR, PT), n_road)
    veh = _set_encoder(p, "veh0", "veh1", obs[:, VEH0:].reshape(A, KV, NB), n_veh)
    return np.concatenate([ego, road, veh], axis=1)


def forward(params, obs, n_road, n_veh):
    """Action means [A, 3] and values [A] of the actor-critic pair."""
    P = unpack(params) if not isinstance(params, dict) else params
    outs = []
    for net in ("actor", "critic"):
        p = P[net]
        z = embeddings(p, obs, n_road, n_veh)
        z = MO.act(_dense(z, p["trunk0"]), MO.ELU)
        z = MO.act(_dense(z, p["trunk1"]), MO.ELU)
        outs.append(_dense(z, p["head"]))
    return outs[0], outs[1][:, 0]


def forward_loops(params, obs_row, n_road, n_veh):
    """The same network for one agent written as plain loops over the valid
    slots only (no padding, no -inf): a second formulation for small cases."""
    P = unpack(params) if not isinstance(params, dict) else params
    x = [float(v) for v in obs_row]

    def elu(v):
        return v if v > 0 else float(np.expm1(v))

    def layer(Wb, v, act=True):
        W, b = Wb
        out = []
        for o in range(W.shape[0]):
            s = float(b[o])
            for i in range(W.shape[1]):
                s += float(W[o, i]) * v[i]
            out.append(elu(s) if act else s)
        return out

    res = []
    for net in ("actor", "critic"):
        p = P[net]
        ego = layer(p["ego1"], layer(p["ego0"], x[:EGO]))
        pools = []
        for (l0, l1, base, F, n) in (("road0", "road1", ROAD0, PT, n_road), ("veh0", "veh1", VEH0, NB, n_veh)):
            best = [0.0] * 96
            for s in range(n):
                h = layer(p[l1], layer(p[l0], x[base + s * F: base + (s + 1) * F]))
                best = h if s == 0 else [max(u, v) for u, v in zip(best, h)]
            pools.append(best)
        z = ego + pools[0] + pools[1]
        z = layer(p["trunk1"], layer(p["trunk0"], z))
        res.append(layer(p["head"], z, act=False))
    return np.array(res[0]), res[1][0]


def _elu_grad(z):
    return np.where(z > 0, 1.0, np.exp(np.minimum(z, 0.0)))


def _dense_back(x, W, dz):
    """Gradients of z = x W^T + b (rows of x summed over): dW, db, dx."""
    return dz.T @ x, dz.sum(axis=0), dz @ W


def slot_outputs(p, obs, group):
    """Every slot's encoder output h2 [A, K, 96] of one network's group
    ("road" or "vehicles"), padded slots included."""
    obs = np.asarray(obs, np.float64)
    A = obs.shape[0]
    l0, l1, lo, hi, F = (("road0", "road1", ROAD0, VEH0, PT) if group == "road" else ("veh0", "veh1", VEH0, OBS, NB))
    slots = obs[:, lo:hi].reshape(A, -1, F)
    return MO.act(_dense(MO.act(_dense(slots, p[l0]), MO.ELU), p[l1]), MO.ELU)


def gradients(params, obs, n_road, n_veh, dmean, dvalue, arg=None):
    """Gradient of L = sum(dmean * mean) + sum(dvalue * value) with respect to
    every parameter, as a flat vector in the parameter layout (the log_std
    entries are zero: the forward does not use them).

    Back-propagation through the layers of `forward` in reverse order; the
    masked max-pool passes each feature's gradient to the valid slot holding
    the maximum, the first one (lowest slot) when several do (a subgradient:
    the maximum is not differentiable where slots tie).  A group without a
    valid slot outputs constant zeros and receives no gradient.  arg, when
    given, fixes that choice: arg[net][group] ([A, 96] slot indices, net 0
    actor / 1 critic, group 0 road / 1 vehicles) replaces the first maximum
    (any maximising slot gives a valid subgradient)."""
    P = unpack(params) if not isinstance(params, dict) else params
    obs = np.asarray(obs, np.float64)
    A = obs.shape[0]
    grads = []
    for ni, (net, g_out) in enumerate((("actor", np.asarray(dmean, np.float64).reshape(A, -1)),
                                       ("critic", np.asarray(dvalue, np.float64).reshape(A, 1)))):
        p = P[net]
        G = {}
        # forward, keeping the pre-activations
        xe = obs[:, :EGO]
        a0 = _dense(xe, p["ego0"]); h0 = MO.act(a0, MO.ELU)
        a1 = _dense(h0, p["ego1"]); ego = MO.act(a1, MO.ELU)
        sets = []
        for gi, (l0, l1, lo, hi, F, cnt) in enumerate((("road0", "road1", ROAD0, VEH0, PT, n_road),
                                                       ("veh0", "veh1", VEH0, OBS, NB, n_veh))):
            slots = obs[:, lo:hi].reshape(A, -1, F)
            K = slots.shape[1]
            z1 = _dense(slots, p[l0]); h1 = MO.act(z1, MO.ELU)
            z2 = _dense(h1, p[l1]); h2 = MO.act(z2, MO.ELU)
            cnt = np.asarray(cnt)
            valid = np.arange(K)[None, :] < cnt[:, None]
            masked = np.where(valid[:, :, None], h2, -np.inf)
            am = masked.argmax(axis=1)                           # first maximum along the slots
            if arg is not None:
                am = np.where(cnt[:, None] > 0, np.asarray(arg[ni][gi], np.int64), am)
            pooled = np.where(cnt[:, None] > 0, np.take_along_axis(h2, am[:, None, :], axis=1)[:, 0, :], 0.0)
            sets.append((l0, l1, slots, z1, h1, z2, am, cnt, pooled))
        x = np.concatenate([ego, sets[0][8], sets[1][8]], axis=1)
        t0 = _dense(x, p["trunk0"]); u0 = MO.act(t0, MO.ELU)
        t1 = _dense(u0, p["trunk1"]); u1 = MO.act(t1, MO.ELU)
        # backward
        G["head"] = _dense_back(u1, p["head"][0], g_out)
        dt1 = G["head"][2] * _elu_grad(t1)
        G["trunk1"] = _dense_back(u0, p["trunk1"][0], dt1)
        dt0 = G["trunk1"][2] * _elu_grad(t0)
        G["trunk0"] = _dense_back(x, p["trunk0"][0], dt0)
        dx = G["trunk0"][2]
        da1 = dx[:, :64] * _elu_grad(a1)
        G["ego1"] = _dense_back(h0, p["ego1"][0], da1)
        da0 = G["ego1"][2] * _elu_grad(a0)
        G["ego0"] = _dense_back(xe, p["ego0"][0], da0)
        for (l0, l1, slots, z1, h1, z2, am, cnt, _), c0 in zip(sets, (64, 160)):
            K = slots.shape[1]
            dpool = np.where(cnt[:, None] > 0, dx[:, c0:c0 + 96], 0.0)
            dh2 = np.zeros((A, K, 96))
            np.put_along_axis(dh2, am[:, None, :], dpool[:, None, :], axis=1)
            dz2 = (dh2 * _elu_grad(z2)).reshape(A * K, 96)
            W2, W1 = p[l1][0], p[l0][0]
            dW2, db2, dh1 = _dense_back(h1.reshape(A * K, 96), W2, dz2)
            dz1 = dh1 * _elu_grad(z1.reshape(A * K, 96))
            dW1, db1, _ = _dense_back(slots.reshape(A * K, -1), W1, dz1)
            G[l1] = (dW2, db2)
            G[l0] = (dW1, db1)
        for n, o, i in net_layers(net):
            grads.append(G[n][0].reshape(-1))
            grads.append(G[n][1].reshape(-1))
    grads.append(np.zeros(3))
    return np.concatenate(grads)
