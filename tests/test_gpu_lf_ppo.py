"""PPO on the paper's late-fusion network (Alg. 1 with App. E and App. L).

Gradients: the engine's gradient of L = sum(dmean * mean) + sum(dvalue * value)
with respect to every parameter, on full observations of a procedural world,
against the FP64 oracle's back-propagation (oracle/lf.py, pinned by central
differences) fed the same bf16-rounded weights and observation values.  The
tensor cores round every hidden activation, the trunk inputs and the
backward's dZ to bf16, and the set encoders' ELU runs in bf16, so each
gradient tensor agrees to 3e-2 of its norm, element by element to 5e-2 of the
element plus 5e-2 of the tensor's RMS (the MLP gradient tests' bounds; the floor covers sums of cancelling
terms; a dropped term, a wrong slot or a transposed operand is off by about
the RMS itself).  The max-pool's arg-max can differ from the oracle's only
where two slots tie within the bf16 rounding, and real observations hold many
such near-ties (neighbouring road points): the test checks that every slot the
engine chose holds a maximum within 2e-2 of its scale, then compares with the
oracle's gradient for the same choice of slots (any maximising slot gives a
valid subgradient).

Training: updates run, stay finite, change the weights, write them back into
the rollout's network, and repeat bit for bit from the same start.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lf as LF
from paper_2605_08528_b300 import sf, synth

pytestmark = pytest.mark.gpu

TOL_NORM = 3e-2
TOL_ELEM = 5e-2


def bf16(x):
    return torch.as_tensor(np.asarray(x, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def oracle_params(p):
    P = LF.unpack(p.astype(np.float64))
    for net in ("actor", "critic"):
        for k, (W, b) in P[net].items():
            P[net][k] = (bf16(W), b)
    return P


def lf_setup(worlds=4, seed=5, horizon=8, minibatches=2, epochs=1, pseed=11):
    sc = synth.procedural_scene(worlds, 16, seed_base=1900)
    stream = torch.cuda.Stream()
    W = sf.World(sc, seed=seed, flags=sf.FLAG_AUTO_RESET, stream=stream)
    with torch.cuda.stream(stream):
        sf.sf_reset(W.h, torch.ones(W.A, dtype=torch.uint8, device="cuda"))
    p0 = sf.init_lf(seed=pseed)
    lf = sf.sf_lf_create(stream)
    sf.sf_lf_set_params(lf, p0)
    cfg = sf.sf_ppo_default_config(horizon=horizon, minibatches=minibatches, epochs=epochs)
    ppo = sf.sf_ppo_create_lf(W.h, lf, cfg)
    return W, lf, ppo, p0, stream


def full_obs(W, stream):
    A = W.A
    obs = torch.zeros((A, sf.FULL_OBS_DIM), device="cuda")
    nr = torch.zeros(A, dtype=torch.int32, device="cuda")
    nv = torch.zeros_like(nr)
    with torch.cuda.stream(stream):
        sf.sf_observe_full(W.h, obs, nr, nv)
    torch.cuda.synchronize()
    return obs, nr, nv


@pytest.mark.parametrize("worlds", [4, 24])
def test_lf_gradients_against_fp64(worlds):
    """24 worlds: about 7,000 rows in the set encoders' backward products (many split-K
    partials and tiles)."""
    W, lf, ppo, p0, stream = lf_setup(worlds=worlds)
    obs, nr, nv = full_obs(W, stream)
    A = W.A
    rng = np.random.default_rng(7)
    dmean = rng.normal(0, 1, (A, 3)).astype(np.float32)
    dvalue = rng.normal(0, 1, A).astype(np.float32)
    mean = torch.full((A, 3), float("nan"), device="cuda")
    value = torch.full((A,), float("nan"), device="cuda")
    amax = torch.zeros((2, 2, A, 96), dtype=torch.int16, device="cuda")
    g = sf.sf_ppo_lf_grads(ppo, obs, nr, nv, A, torch.as_tensor(dmean).cuda(), torch.as_tensor(dvalue).cuda(),
                           mean, value, amax)
    ob, n_r, n_v = obs.cpu().numpy(), nr.cpu().numpy(), nv.cpu().numpy()
    assert (n_r > 0).all() and (n_v > 0).any()
    P = oracle_params(p0)
    # the slot each pooled feature's gradient went to must hold a maximum: within the
    # rounding of the bf16 encoder of the oracle's largest valid output (2e-2 of its scale)
    am = amax.cpu().numpy().view(np.uint16).astype(np.int64)
    arg = [[None, None], [None, None]]
    differ = total = 0
    for gi, (grp, cnt) in enumerate((("road", n_r), ("vehicles", n_v))):
        for ni, net in enumerate(("actor", "critic")):
            h2 = LF.slot_outputs(P[net], bf16(ob), grp)
            K = h2.shape[1]
            valid = np.arange(K)[None, :, None] < cnt[:, None, None]
            hm = np.where(valid, h2, -np.inf)
            best, first = hm.max(axis=1), hm.argmax(axis=1)
            full = cnt > 0
            ch = am[gi, ni]
            assert np.all(ch[~full] == 0xFFFF) and np.all(ch[full] < cnt[full, None])
            got = np.take_along_axis(h2, np.where(full[:, None], ch, 0)[:, None, :], axis=1)[:, 0, :]
            gap = (best - got)[full] / np.maximum(1.0, np.abs(best[full]))
            assert gap.max() <= 2e-2, (grp, net, float(gap.max()))
            differ += int((ch != first)[full].sum())
            total += int(full.sum()) * 96
            arg[ni][gi] = ch
    print("pooled features whose slot differs from the oracle's first maximum (near-ties): %d of %d" % (differ, total))
    ref = LF.gradients(P, bf16(ob), n_r, n_v, dmean.astype(np.float64), dvalue.astype(np.float64), arg=arg)
    # the training forward's outputs match the oracle's forward (the same check as the inference network's)
    rm, rv = LF.forward(P, bf16(ob), n_r, n_v)
    em = np.abs(mean.cpu().numpy() - rm).max() / max(1.0, float(np.abs(rm).max()))
    ev = np.abs(value.cpu().numpy() - rv).max() / max(1.0, float(np.abs(rv).max()))
    assert em < 3e-2 and ev < 3e-2, (em, ev)
    assert np.isfinite(g).all() and np.all(g[-3:] == 0)
    k, bad = 0, []
    for net in ("actor", "critic"):
        for name, o, i in LF.net_layers(net):
            for part, n in (("W", o * i), ("b", o)):
                a, r = g[k:k + n].astype(np.float64), ref[k:k + n]
                k += n
                rms = np.sqrt(np.mean(r ** 2))
                en = np.linalg.norm(a - r) / max(np.linalg.norm(r), 1e-30)
                ee = (np.abs(a - r) / (TOL_ELEM * np.abs(r) + TOL_ELEM * rms + 1e-30)).max()
                print("%s %-6s %s: norm error %.2e, element-wise worst %.2f of the bound" % (net, name, part, en, ee))
                if not (en < TOL_NORM and ee <= 1.0):
                    bad.append((net, name, part, float(en), float(ee)))
    assert k == len(g) - 3
    assert not bad, bad
    sf.sf_ppo_destroy(ppo)
    sf.sf_lf_destroy(lf)
    W.close()


def run_lf_ppo(iters=2):
    W, lf, ppo, p0, stream = lf_setup()
    stats = []
    for _ in range(iters):
        sf.sf_ppo_collect(ppo)
        stats.append(sf.sf_ppo_update(ppo))
    params = sf.sf_ppo_lf_params(ppo)
    obs, nr, nv = full_obs(W, stream)
    A = W.A
    mean = torch.zeros((A, 3), device="cuda")
    value = torch.zeros(A, device="cuda")
    sf.sf_lf_forward(lf, obs, nr, nv, A, mean, value)
    sf.sf_lf_sync(lf)
    out = dict(stats=np.array(stats), params=params, p0=p0, mean=mean.cpu().numpy(), value=value.cpu().numpy(),
               obs=obs.cpu().numpy(), nr=nr.cpu().numpy(), nv=nv.cpu().numpy())
    sf.sf_ppo_destroy(ppo)
    sf.sf_lf_destroy(lf)
    W.close()
    return out


def test_lf_ppo_trains_and_publishes():
    r = run_lf_ppo()
    st, p, p0 = r["stats"], r["params"], r["p0"]
    print("stats (reward, policy loss, value loss, KL, lr, grad norm):", st)
    assert np.isfinite(st).all() and np.isfinite(p).all()
    assert (st[:, 3] >= 0).all() and (st[:, 5] > 0).all()
    # every layer of both networks moved
    k = 0
    for net in ("actor", "critic"):
        for name, o, i in LF.net_layers(net):
            assert np.abs(p[k:k + o * i] - p0[k:k + o * i]).max() > 0, (net, name)
            k += o * i + o
    # the rollout's (inference) network holds the trained weights: its outputs are the oracle's on them
    P = oracle_params(p)
    rm, rv = LF.forward(P, bf16(r["obs"]), r["nr"], r["nv"])
    em = np.abs(r["mean"] - rm).max() / max(1.0, float(np.abs(rm).max()))
    ev = np.abs(r["value"] - rv).max() / max(1.0, float(np.abs(rv).max()))
    print("inference network vs oracle on the trained weights: mean %.2e, value %.2e" % (em, ev))
    assert em < 3e-2 and ev < 3e-2


def test_lf_ppo_is_deterministic():
    a, b = run_lf_ppo(), run_lf_ppo()
    assert np.array_equal(a["params"].view(np.uint32), b["params"].view(np.uint32))
    assert np.array_equal(a["stats"].view(np.uint32), b["stats"].view(np.uint32))
