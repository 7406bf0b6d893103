"""GPU parity of the late-fusion actor-critic network (App. E) against the
FP64 oracle.

The oracle is fed the same bf16-rounded weights and observation values the
tensor cores see (biases stay fp32), so the remaining differences are the bf16
rounding of the hidden activations (relative 2^-9 each), the bf16 trunk inputs
and fp32 accumulation: the pooled embeddings agree to 2e-2 of their scale and
the outputs to 3e-2 of max(1, |output|).  A wrong pooling boundary (a slot
counted for the wrong agent, a padded slot taken into the max) changes an
embedding by O(1) and fails these bounds.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lf as LF
from oracle import oracle as O
from paper_2605_08528_b300 import sf, synth

pytestmark = pytest.mark.gpu


def bf16(x):
    return torch.as_tensor(np.asarray(x, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def oracle_params(p):
    """bf16-rounded weights, fp32 biases, in the oracle's structure."""
    P = LF.unpack(p.astype(np.float64))
    for net in ("actor", "critic"):
        for k, (W, b) in P[net].items():
            P[net][k] = (bf16(W), b)
    return P


def run(m, obs, nr, nv):
    A = len(obs)
    d_obs = torch.as_tensor(np.ascontiguousarray(obs, np.float32)).cuda()
    d_nr = torch.as_tensor(np.asarray(nr, np.int32)).cuda()
    d_nv = torch.as_tensor(np.asarray(nv, np.int32)).cuda()
    mean = torch.full((A, 3), float("nan"), device="cuda")
    value = torch.full((A,), float("nan"), device="cuda")
    emb = torch.full((A, 512), float("nan"), device="cuda")
    sf.sf_lf_forward(m, d_obs, d_nr, d_nv, A, mean, value, emb)
    sf.sf_lf_sync(m)
    return mean.cpu().numpy(), value.cpu().numpy(), emb.cpu().numpy()


def check(p, obs, nr, nv, got):
    P = oracle_params(p)
    ob = bf16(obs)
    mean, value, emb = got
    for h, net in enumerate(("actor", "critic")):
        ref = LF.embeddings(P[net], ob, nr, nv)
        scale = max(1.0, float(np.abs(ref).max()))
        err = np.abs(emb[:, 256 * h:256 * (h + 1)] - ref).max() / scale
        print(net, "embedding max error / scale: %.2e" % err)
        assert err < 2e-2
        empty_r = np.asarray(nr) == 0
        assert not emb[empty_r, 256 * h + 64:256 * h + 160].any()   # empty road group pools to zeros
    rm, rv = LF.forward(P, ob, nr, nv)
    em = np.abs(mean - rm).max() / max(1.0, float(np.abs(rm).max()))
    ev = np.abs(value - rv).max() / max(1.0, float(np.abs(rv).max()))
    print("mean error %.2e, value error %.2e" % (em, ev))
    assert np.isfinite(mean).all() and np.isfinite(value).all()
    assert em < 3e-2 and ev < 3e-2


def random_obs(seed, A):
    rng = np.random.default_rng(seed)
    nr = rng.integers(0, LF.KR + 1, A)
    nr[::7] = 0
    nr[1::11] = LF.KR
    nv = rng.integers(0, LF.KV + 1, A)
    nv[2::5] = 0
    obs = rng.normal(0, 1, (A, LF.OBS)).astype(np.float32)
    for a in range(A):
        obs[a, LF.ROAD0 + nr[a] * LF.PT:LF.VEH0] = 0
        obs[a, LF.VEH0 + nv[a] * LF.NB:] = 0
    return obs, nr, nv


@pytest.mark.parametrize("A", [1, 31, 1000])
def test_lf_forward_random_observations(A):
    p = sf.init_lf(seed=A)
    m = sf.sf_lf_create()
    sf.sf_lf_set_params(m, p)
    assert np.array_equal(sf.sf_lf_get_params(m), p)
    obs, nr, nv = random_obs(A, A)
    check(p, obs, nr, nv, run(m, obs, nr, nv))
    sf.sf_lf_destroy(m)


def test_lf_empty_items_between_full_ones():
    """Items (32 consecutive agents) whose groups have no filled slot at all,
    among full ones, with more items than the set encoder's persistent CTAs
    (150 items, one CTA per SM and network): CTAs 0 and 1 take an empty item
    and then a full one, whose tiles must not see barrier phases or pool
    entries left by the empty one.  Every output against the oracle."""
    A = 150 * 32
    obs, nr, nv = random_obs(11, A)
    for it in [0, 1] + list(range(7, 150, 7)):
        nr[32 * it:32 * it + 32] = 0
        nv[32 * it:32 * it + 32] = 0
        obs[32 * it:32 * it + 32, LF.ROAD0:] = 0
    p = sf.init_lf(seed=11)
    m = sf.sf_lf_create()
    sf.sf_lf_set_params(m, p)
    check(p, obs, nr, nv, run(m, obs, nr, nv))
    sf.sf_lf_destroy(m)


def test_lf_forward_on_full_observations():
    """The network on the library's own full observations: paper-shaped worlds,
    a ragged batch (up to 32 agents and 5,000 points a world) and parked agents."""
    p = sf.init_lf(seed=7)
    m = sf.sf_lf_create()
    sf.sf_lf_set_params(m, p)
    for sc, flags in ((synth.procedural_scene(8, 16, seed_base=1000), sf.FLAG_AUTO_RESET),
                      (synth.ragged_scene(40, seed_base=2000), 0)):
        W = sf.World(sc, seed=2, flags=flags)
        sf.sf_reset(W.h, torch.ones(W.A, dtype=torch.uint8, device="cuda"))
        acts = synth.ou_actions(W.A, 30, seed=1, sigma=0.6)
        for t in range(30):
            sf.sf_step(W.h, torch.as_tensor(acts[t]).cuda())
        g = W.full_obs()
        parked = (g["n_veh"] == 0) & (g["n_road"] == 0)
        print("agents", W.A, "parked or isolated", int(parked.sum()), "mean road slots", g["n_road"].mean())
        check(p, g["obs"], g["n_road"], g["n_veh"], run(m, g["obs"], g["n_road"], g["n_veh"]))
        W.close()
    sf.sf_lf_destroy(m)


def test_lf_rejects_bad_arguments():
    m = sf.sf_lf_create()
    with pytest.raises(sf.SFError):
        sf.sf_lf_set_params(m, np.zeros(5, np.float32))
    bad = sf.init_lf(1)
    bad[10] = np.nan
    with pytest.raises(sf.SFError):
        sf.sf_lf_set_params(m, bad)
    with pytest.raises(sf.SFError):
        sf.sf_lf_forward(m, None, None, None, 4, None)
    sf.sf_lf_destroy(m)


def lf_world(sc, stream, seed=5):
    W = sf.World(sc, seed=seed, flags=sf.FLAG_AUTO_RESET, stream=stream)
    with torch.cuda.stream(stream):
        sf.sf_reset(W.h, torch.ones(W.A, dtype=torch.uint8, device="cuda"))
    return W


def test_lf_policy_step_and_its_graph_match_the_individual_calls():
    """sf_step_lf = full observation -> actor means -> sf_step, and its captured
    graph (with a reset mask) replays bit-identically to those calls."""
    sc = synth.procedural_scene(6, 16, seed_base=900)
    s1, s2, s3 = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    W1, W2, W3 = lf_world(sc, s1), lf_world(sc, s2), lf_world(sc, s3)
    p = sf.init_lf(seed=11)
    lf1, lf2, lf3 = sf.sf_lf_create(s1), sf.sf_lf_create(s2), sf.sf_lf_create(s3)
    for m in (lf1, lf2, lf3):
        sf.sf_lf_set_params(m, p)
    A = W1.A
    obs = torch.zeros((A, sf.FULL_OBS_DIM), device="cuda")
    nr = torch.zeros(A, dtype=torch.int32, device="cuda")
    nv = torch.zeros_like(nr)
    mean = torch.zeros((A, 3), device="cuda")
    val = torch.zeros(A, device="cuda")
    mask = torch.zeros(A, dtype=torch.uint8, device="cuda")
    masks = torch.as_tensor(np.stack([synth.reset_mask(A, t, 0.2) for t in range(8)]), device="cuda")
    torch.cuda.synchronize()
    g = sf.sf_graph_capture_lf(W3.h, lf3, d_reset_mask=mask)
    for t in range(8):
        with torch.cuda.stream(s1):
            sf.sf_step_lf(W1.h, lf1)
            sf.sf_reset(W1.h, masks[t])
        with torch.cuda.stream(s2):
            sf.sf_observe_full(W2.h, obs, nr, nv)
            sf.sf_lf_forward(lf2, obs, nr, nv, A, mean, val)
            sf.sf_step(W2.h, mean)
            sf.sf_reset(W2.h, masks[t])
        with torch.cuda.stream(s3):
            mask.copy_(masks[t])
            sf.sf_graph_launch(g)
        torch.cuda.synchronize()
    o = sf.sf_lf_step_outputs(W3.h)
    F1, I1, _ = sf.sf_get_state(W1.h)
    F2, I2, _ = sf.sf_get_state(W2.h)
    F3, I3, _ = sf.sf_get_state(W3.h)
    assert np.array_equal(F1, F2) and np.array_equal(I1, I2)
    assert np.array_equal(F1, F3) and np.array_equal(I1, I3)
    assert o.num_agents == A and o.value and o.actions
    v3 = sf.device_view(o.value, (A,)).clone()
    a3 = sf.device_view(o.actions, (A, 3)).clone()
    assert torch.isfinite(v3).all()
    assert torch.equal(v3, val) and torch.equal(a3, mean)   # the last step's critic values and actions
    sf.sf_graph_destroy(g)
    for m in (lf1, lf2, lf3):
        sf.sf_lf_destroy(m)
