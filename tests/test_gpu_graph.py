"""The policy in the loop and the captured step graph: replaying the graph must
give bit-identical states to issuing the same calls one by one, and the policy
step must equal the policy's forward followed by a plain step."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_08528_b300 import sf, synth

pytestmark = pytest.mark.gpu


def world(sc, stream, seed=5, **shape):
    W = sf.World(sc, seed=seed, flags=sf.FLAG_AUTO_RESET, stream=stream, **shape)
    with torch.cuda.stream(stream):
        sf.sf_reset(W.h, torch.ones(W.A, dtype=torch.uint8, device="cuda"))
    return W


def test_policy_step_equals_forward_then_step():
    sc = synth.procedural_scene(8, 16, seed_base=700)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    W1, W2 = world(sc, s1), world(sc, s2)
    pol = sf.init_policy(seed=3)
    act = torch.zeros((W1.A, 3), device="cuda")
    for t in range(10):
        sf.sf_step_policy(W1.h, pol)
        obs = W2.outputs()[0]
        torch.cuda.synchronize()
        sf.sf_mlp_forward(pol, obs, W2.A, act)
        sf.sf_mlp_sync(pol)
        with torch.cuda.stream(s2):
            sf.sf_step(W2.h, act)
    F1, I1, _ = sf.sf_get_state(W1.h)
    F2, I2, _ = sf.sf_get_state(W2.h)
    assert np.array_equal(F1, F2) and np.array_equal(I1, I2)
    assert np.abs(act.cpu().numpy()).max() <= 1.0
    sf.sf_mlp_destroy(pol)


@pytest.mark.parametrize("with_policy,with_reset", [(False, False), (True, False), (False, True)])
def test_graph_replay_matches_individual_calls(with_policy, with_reset):
    sc = synth.procedural_scene(6, 16, seed_base=800)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    W1, W2 = world(sc, s1), world(sc, s2)
    pol = sf.init_policy(seed=4) if with_policy else None
    acts = torch.as_tensor(synth.ou_actions(W1.A, 12, seed=9), device="cuda")
    masks = torch.as_tensor(np.stack([synth.reset_mask(W1.A, t, 0.2) for t in range(12)]), device="cuda")
    act_buf = torch.zeros((W1.A, 3), device="cuda")
    mask = torch.zeros(W1.A, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    g = sf.sf_graph_capture(W1.h, policy=pol, d_actions=act_buf, d_reset_mask=mask if with_reset else None)
    for t in range(12):
        m = masks[t]
        with torch.cuda.stream(s1):
            act_buf.copy_(acts[t])
            mask.copy_(m)
            sf.sf_graph_launch(g)
        with torch.cuda.stream(s2):
            if with_policy:
                sf.sf_step_policy(W2.h, pol)
            else:
                sf.sf_step(W2.h, acts[t])
            if with_reset:
                sf.sf_reset(W2.h, m)
    F1, I1, _ = sf.sf_get_state(W1.h)
    F2, I2, _ = sf.sf_get_state(W2.h)
    o1, o2 = W1.outputs()[0].cpu().numpy(), W2.outputs()[0].cpu().numpy()
    assert np.array_equal(F1, F2) and np.array_equal(I1, I2) and np.array_equal(o1, o2)
    sf.sf_graph_destroy(g)
    if pol is not None:
        sf.sf_mlp_destroy(pol)


def test_graph_with_surrogate_matches_individual_calls():
    sc = synth.procedural_scene(6, 8, seed_base=820)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    W1, W2 = world(sc, s1), world(sc, s2)
    sur = sf.sf_surrogate_create(s1)
    acts = torch.as_tensor(synth.ou_actions(W1.A, 8, seed=2), device="cuda")
    act_buf = torch.zeros((W1.A, 3), device="cuda")
    torch.cuda.synchronize()
    g = sf.sf_graph_capture(W1.h, d_actions=act_buf, surrogate=sur)
    # one surrogate object: its MLP's activation buffers serve one stream at a time
    for t in range(8):
        with torch.cuda.stream(s1):
            act_buf.copy_(acts[t])
            sf.sf_graph_launch(g)
    torch.cuda.synchronize()
    for t in range(8):
        with torch.cuda.stream(s2):
            sf.sf_step_surrogate(W2.h, sur, acts[t])
    torch.cuda.synchronize()
    F1, I1, _ = sf.sf_get_state(W1.h)
    F2, I2, _ = sf.sf_get_state(W2.h)
    assert np.array_equal(F1, F2) and np.array_equal(I1, I2)
    assert sf.sf_surrogate_audit(W1.h)[1] == sf.sf_surrogate_audit(W2.h)[1] > 0
    sf.sf_graph_destroy(g)
    sf.sf_surrogate_destroy(sur)


@pytest.mark.parametrize("shape", [dict(), dict(warps_per_block=8, stage_bytes=49152), dict(split_step=1)],
                         ids=["fused", "fused-staged", "split"])
def test_step_from_host_buffers_equals_device_step(shape):
    """sf_step_host (copy in, step, copies out, one captured graph for
    page-locked buffers) gives the device step's rewards, done flags and state
    bit for bit: replays, a ring of page-locked action buffers (the graph's
    transfers are retargeted: with the fused step the world kernel's own
    arguments), pageable numpy buffers (no graph) and a re-capture after
    sf_autotune; in each launch shape."""
    sc = synth.procedural_scene(6, 16, seed_base=720)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    W1, W2 = world(sc, s1, **shape), world(sc, s2, **shape)
    A = W1.A
    acts = synth.ou_actions(A, 24, seed=6)
    ring = [torch.as_tensor(acts[t]).pin_memory() for t in range(3)]
    rew_h = torch.empty(A, dtype=torch.float32).pin_memory()
    done_h = torch.empty(A, dtype=torch.uint8).pin_memory()
    rew_np, done_np = np.zeros(A, np.float32), np.zeros(A, np.uint8)
    act_dev = torch.empty((A, 3), device="cuda")
    rew_dev = torch.empty(A, device="cuda")
    done_dev = torch.empty(A, dtype=torch.uint8, device="cuda")
    for t in range(24):
        if t == 12:
            with torch.cuda.stream(s2):
                sf.sf_autotune(W2.h, torch.zeros((A, 3), device="cuda"), iters=2)
            torch.cuda.synchronize()
        if t < 16:
            a_h = ring[t % 3]
            a_h.copy_(torch.as_tensor(acts[t]))
            sf.sf_step_host(W2.h, a_h, rew_h, done_h)
            r2, d2 = rew_h.numpy().copy(), done_h.numpy().copy()
        else:
            sf.sf_step_host(W2.h, np.ascontiguousarray(acts[t]), rew_np, done_np)
            r2, d2 = rew_np.copy(), done_np.copy()
        with torch.cuda.stream(s1):
            act_dev.copy_(torch.as_tensor(acts[t]))
            sf.sf_step(W1.h, act_dev)
            sf.sf_get_obs(W1.h, None, rew_dev, done_dev, None)
        torch.cuda.synchronize()
        assert np.array_equal(rew_dev.cpu().numpy(), r2), t
        assert np.array_equal(done_dev.cpu().numpy(), d2), t
    F1, I1, _ = sf.sf_get_state(W1.h)
    F2, I2, _ = sf.sf_get_state(W2.h)
    assert np.array_equal(F1, F2) and np.array_equal(I1, I2)


def test_step_from_host_buffers_with_observations():
    """sf_step_host_obs also delivers the step's observations to the host: they
    equal the device step's (sf_get_obs) bit for bit, through replays, a
    retargeted observation buffer, a switch back to sf_step_host (re-capture)
    and pageable buffers (no graph)."""
    sc = synth.procedural_scene(4, 16, seed_base=730)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    W1, W2 = world(sc, s1), world(sc, s2)
    A = W1.A
    acts = synth.ou_actions(A, 12, seed=7)
    a_h = torch.empty((A, 3), dtype=torch.float32).pin_memory()
    obs_ring = [torch.empty((A, sf.OBS_DIM), dtype=torch.float32).pin_memory() for _ in range(2)]
    rew_h = torch.empty(A, dtype=torch.float32).pin_memory()
    done_h = torch.empty(A, dtype=torch.uint8).pin_memory()
    act_dev = torch.empty((A, 3), device="cuda")
    obs_dev = torch.empty((A, sf.OBS_DIM), device="cuda")
    for t in range(12):
        a_h.copy_(torch.as_tensor(acts[t]))
        if t == 6:
            sf.sf_step_host(W2.h, a_h, rew_h, done_h)          # without the observation
            o2 = None
        elif t >= 10:
            o_np = np.zeros((A, sf.OBS_DIM), np.float32)
            sf.sf_step_host_obs(W2.h, np.ascontiguousarray(acts[t]), o_np, np.zeros(A, np.float32),
                                np.zeros(A, np.uint8))
            o2 = o_np
        else:
            o = obs_ring[t % 2]
            sf.sf_step_host_obs(W2.h, a_h, o, rew_h, done_h)
            o2 = o.numpy().copy()
        with torch.cuda.stream(s1):
            act_dev.copy_(torch.as_tensor(acts[t]))
            sf.sf_step(W1.h, act_dev)
            sf.sf_get_obs(W1.h, obs_dev, None, None, None)
        torch.cuda.synchronize()
        if o2 is not None:
            assert np.array_equal(obs_dev.cpu().numpy().view(np.uint32), o2.view(np.uint32)), t
    with pytest.raises(sf.SFError) as e:
        sf.sf_step_host_obs(W2.h, a_h, None, rew_h, done_h)
    assert e.value.status == sf.SF_ERR_INVALID_ARG
    W1.close()
    W2.close()
