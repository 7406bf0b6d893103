"""GPU parity of the kinematic bicycle backend (SF_DYN_BICYCLE, Sec. 4.4)
against the FP64 oracle's bicycle step.

Tolerances: one update per control step in FP32 (sin, cos, atan, tan of the
CUDA math library and ~1e-5 m position rounding at |p| ~ 100 m): a single step
matches the oracle fed the same FP32 state to 1e-5 relative per state block;
100-step contact-free rollouts stay within 1e-3 m and 1e-3 m/s (the bound the
raycast vehicle meets).  Events, rewards and observations are the shared
kernels: their flags and indices are bit-exact up to counted near-ties.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2605_08528_b300 import sf, synth
from tests.helpers import block_errors

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def test_bicycle_single_step_parity_and_rollout():
    sc = synth.straight_road(num_agents=4)
    W = sf.World(sc, seed=1, flags=sf.FLAG_INVINCIBLE, dynamics=sf.DYN_BICYCLE)
    place = synth.straight_road_placements(seed=1).astype(np.float32)
    sf.sf_place_agents(W.h, place)
    orc = O.Oracle(sc)
    Fo, Io = orc.empty_state()
    for a in range(4):
        orc.place(Fo, Io, a, *[float(v) for v in place[a]])
    acts = synth.uniform_actions(4, 100, seed=2)
    worst = 0.0
    for t in range(100):
        F0, I0, _ = sf.sf_get_state(W.h)
        sf.sf_step(W.h, dev(acts[t]))
        F1, I1, _ = sf.sf_get_state(W.h)
        # single step from the GPU's own state
        Fs, Is = F0.astype(np.float64), I0.copy()
        orc.step(Fs, Is, acts[t].astype(np.float64), flags=O.FLAG_INVINCIBLE | O.FLAG_BICYCLE, want_obs=False)
        alive = (I1[:, O.I_STATUS] & O.ALIVE) != 0
        errs = block_errors(F1, Fs, np.nonzero(alive)[0])
        for k, e in errs.items():
            if len(e):
                worst = max(worst, float(e.max()))
                assert e.max() <= 1e-5, (t, k, float(e.max()))
        # the free-running oracle rollout
        orc.step(Fo, Io, acts[t].astype(np.float64), flags=O.FLAG_INVINCIBLE | O.FLAG_BICYCLE, want_obs=False)
    F, I, _ = sf.sf_get_state(W.h)
    dp = np.abs(F[:, :2] - Fo[:, :2]).max()
    dv = np.abs(F[:, 7:9] - Fo[:, 7:9]).max()
    print("bicycle single-step worst relative error %.2e; 100-step |dp| %.2e m, |dv| %.2e m/s" % (worst, dp, dv))
    assert dp <= 1e-3 and dv <= 1e-3
    # level chassis, wheels rolling, steer within 30 degrees
    assert np.allclose(F[:, 2], F[0, 2]) and np.abs(F[:, 4:6]).max() == 0.0
    assert np.abs(F[:, O.F_DELTA]).max() <= np.radians(30) + 1e-6
    W.close()


def test_bicycle_events_and_observations_on_paper_worlds():
    sc = synth.procedural_scene(4, 16, seed_base=1500)
    W = sf.World(sc, seed=4, flags=sf.FLAG_RECORD_INDICES, dynamics=sf.DYN_BICYCLE)
    sf.sf_reset(W.h, dev(np.ones(W.A, np.uint8)))
    orc = O.Oracle(sc)
    acts = synth.ou_actions(W.A, 20, seed=3, sigma=0.5)
    mism = 0
    for t in range(20):
        F0, I0, _ = sf.sf_get_state(W.h)
        sf.sf_step(W.h, dev(acts[t]))
        F1, I1, _ = sf.sf_get_state(W.h)
        obs = W.outputs()[0].cpu().numpy()
        oo = orc.observe(F1.astype(np.float64), I1)
        ix = W.indices()
        for a in range(W.A):
            if not I1[a, O.I_STATUS] & O.ALIVE:
                assert not obs[a].any()
                continue
            if not (np.array_equal(ix["knn_pts"][a], oo["knn_pts"][a]) and ix["lane_seg"][a] == oo["lane_seg"][a]
                    and np.array_equal(ix["knn_agents"][a], oo["knn_agents"][a])):
                mism += 1          # near-ties, as in the vehicle parity test
                continue
            d = np.abs(obs[a] - oo["obs"][a])
            for k in range(8):
                c = 16 + 10 * k + 4
                d[c] = min(d[c], abs(2.0 - d[c]))
            ttc = [16 + 10 * k + 8 for k in range(8)]
            assert np.delete(d, ttc).max() <= 2e-5, (t, a)
    print("index near-ties:", mism)
    assert mism <= 0.01 * 20 * W.A + 2
    W.close()


def test_bicycle_rejects_the_surrogate_and_bad_dynamics():
    sc = synth.straight_road(num_agents=2)
    with pytest.raises(sf.SFError):
        sf.sf_create(dynamics=7)
    W = sf.World(sc, dynamics=sf.DYN_BICYCLE)
    s = sf.sf_surrogate_create()
    with pytest.raises(sf.SFError) as e:
        sf.sf_step_surrogate(W.h, s, torch.zeros((2, 3), device="cuda"))
    assert e.value.status == sf.SF_ERR_STATE
    sf.sf_surrogate_destroy(s)
    W.close()
