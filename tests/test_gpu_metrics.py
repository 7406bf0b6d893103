"""Episode metrics of Sec. 4 (SR, CR, mean episode-maximum DRAC) counted on the
device with SF_FLAG_METRICS, against the same counts made on the host from the
per-step outputs the step already exposes (events, done flags and the step
DRAC): per agent the running maximum DRAC and the union of event bits, an
episode added at its done step, a masked reset dropping the interrupted
episodes.  The counters are integers (the DRAC sum in units of 1e-6 m/s^2), so
the two must agree exactly; through plain steps, a masked reset, a captured
graph and the host-buffer step (whose retargeting must leave the metrics
kernel alone)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_08528_b300 import sf, synth

pytestmark = pytest.mark.gpu

# the SF_EV_* event bits of include/sf.h
EV = {"goals": 1, "collisions": 2, "crashes": 4, "lane_forbidden": 8, "offroad": 16, "idle": 32, "timeouts": 64,
      "nonfinite": 128}


class HostMetrics:
    def __init__(self, A):
        self.epmax = np.zeros(A, np.float32)
        self.epev = np.zeros(A, np.uint32)
        self.c = {k: 0 for k in list(EV) + ["episodes", "drac_over"]}
        self.micro = 0

    def step(self, events, done, drac):
        m = np.where(drac > self.epmax, drac, self.epmax).astype(np.float32)
        e = self.epev | events.astype(np.uint32)
        d = done != 0
        self.c["episodes"] += int(d.sum())
        for k, bit in EV.items():
            self.c[k] += int(((e & bit) != 0)[d].sum())
        self.c["drac_over"] += int((m[d] > np.float32(3.4)).sum())
        capped = np.minimum(m[d], np.float32(1e6)).astype(np.float64)
        self.micro += int(np.rint(capped * 1e6).astype(np.int64).sum())
        self.epmax = np.where(d, np.float32(0), m).astype(np.float32)
        self.epev = np.where(d, np.uint32(0), e).astype(np.uint32)

    def reset(self, mask):
        self.epmax[mask != 0] = 0
        self.epev[mask != 0] = 0

    def check(self, got):
        for k, v in self.c.items():
            assert got[k] == v, (k, got[k], v)
        n = self.c["episodes"]
        if n:
            assert got["success_rate"] == self.c["goals"] / n
            assert got["collision_rate"] == self.c["collisions"] / n
            assert abs(got["mean_episode_max_drac"] - self.micro * 1e-6 / n) <= 1e-12 * max(1.0, self.micro * 1e-6 / n)


def outputs(W, stream):
    A = W.A
    ev = torch.zeros(A, dtype=torch.int32, device="cuda")
    dn = torch.zeros(A, dtype=torch.uint8, device="cuda")
    dr = torch.zeros(A, device="cuda")
    with torch.cuda.stream(stream):
        sf.sf_get_obs(W.h, None, None, dn, ev)
        sf.sf_get_indices(W.h, None, None, None, dr)
    torch.cuda.synchronize()
    return ev.cpu().numpy().view(np.uint32), dn.cpu().numpy(), dr.cpu().numpy()


@pytest.mark.parametrize("split", [0, 1], ids=["fused", "split"])
def test_metrics_match_host_counts(split):
    sc = synth.procedural_scene(8, 16, seed_base=940)
    stream = torch.cuda.Stream()
    W = sf.World(sc, seed=3, flags=sf.FLAG_AUTO_RESET | sf.FLAG_METRICS, stream=stream, split_step=split)
    A = W.A
    with torch.cuda.stream(stream):
        sf.sf_reset(W.h, torch.ones(A, dtype=torch.uint8, device="cuda"))
    H = HostMetrics(A)
    acts = synth.ou_actions(A, 240, seed=21)
    act_dev = torch.empty((A, 3), device="cuda")
    rng = np.random.default_rng(5)
    for t in range(160):                         # plain steps, with a masked reset at t = 80
        with torch.cuda.stream(stream):
            act_dev.copy_(torch.as_tensor(acts[t]))
            sf.sf_step(W.h, act_dev)
        H.step(*outputs(W, stream))
        if t == 80:
            mask = (rng.random(A) < 0.3).astype(np.uint8)
            with torch.cuda.stream(stream):
                sf.sf_reset(W.h, torch.as_tensor(mask).cuda())
            torch.cuda.synchronize()
            H.reset(mask)
    got = sf.sf_get_metrics(W.h)
    print("after 160 steps:", got)
    assert got["episodes"] > 0
    H.check(got)
    # a captured graph of the step
    g = sf.sf_graph_capture(W.h, d_actions=act_dev)
    for t in range(160, 200):
        with torch.cuda.stream(stream):
            act_dev.copy_(torch.as_tensor(acts[t]))
            sf.sf_graph_launch(g)
        H.step(*outputs(W, stream))
    sf.sf_graph_destroy(g)
    H.check(sf.sf_get_metrics(W.h))
    # the host-buffer step: a ring of page-locked action buffers retargets the graph every call
    ring = [torch.empty((A, 3), dtype=torch.float32).pin_memory() for _ in range(3)]
    rew_h = torch.empty(A, dtype=torch.float32).pin_memory()
    done_h = torch.empty(A, dtype=torch.uint8).pin_memory()
    for t in range(200, 240):
        a_h = ring[t % 3]
        a_h.copy_(torch.as_tensor(acts[t]))
        sf.sf_step_host(W.h, a_h, rew_h, done_h)
        ev, dn, dr = outputs(W, stream)
        assert np.array_equal(dn, done_h.numpy())
        H.step(ev, dn, dr)
    H.check(sf.sf_get_metrics(W.h))
    # clearing the counters: episodes under way count when they end
    sf.sf_reset_metrics(W.h)
    H.c = {k: 0 for k in H.c}
    H.micro = 0
    for t in range(40):
        with torch.cuda.stream(stream):
            act_dev.copy_(torch.as_tensor(acts[t]))
            sf.sf_step(W.h, act_dev)
        H.step(*outputs(W, stream))
    H.check(sf.sf_get_metrics(W.h))
    W.close()


def test_metrics_need_the_flag():
    sc = synth.procedural_scene(2, 4, seed_base=950)
    W = sf.World(sc, seed=1, flags=sf.FLAG_AUTO_RESET, stream=torch.cuda.Stream())
    with pytest.raises(sf.SFError) as e:
        sf.sf_get_metrics(W.h)
    assert e.value.status == sf.SF_ERR_STATE
    with pytest.raises(sf.SFError) as e:
        sf.sf_reset_metrics(W.h)
    assert e.value.status == sf.SF_ERR_STATE
    W.close()
