"""GPU parity of the modified ALL weather-to-friction model (Sec. 3.3, App. B)
through the C-ABI against the FP64 oracle.

With SF_WEATHER_ALL every agent has a road surface (AC, SMA, OGFC) and a water
film; its friction coefficient is the model's static friction at 13.89 m/s
(the printed curve points joined linearly, the 1e-3 floor from 0.85 mm), and
the ego group's weather token is Eq. weather_obs.  Tolerances: mu within 1e-6
(FP32 interpolation of the same points), spawns bit-exact, the state of a
step and the observation as in the other parity tests (1e-5 relative per
state block, 2e-5 absolute per observation feature).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2605_08528_b300 import sf, synth
from tests.helpers import block_errors
from tests.test_gpu_parity import lane_tie

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def all_params():
    P = O.default_params()
    P.weather_model = O.WEATHER_ALL
    return P


def test_all_model_mu_token_and_step_parity():
    sc = synth.with_water_films(synth.procedural_scene(6, 16, seed_base=1700), seed=5)
    W = sf.World(sc, seed=12, flags=sf.FLAG_INVINCIBLE, weather_model=sf.WEATHER_ALL)
    orc = O.Oracle(sc, all_params())
    Fo, Io = orc.empty_state()
    Io[:, O.I_PRECIP], Io[:, O.I_SURFACE] = synth.film_code(sc.film_mm), sc.surface
    sf.sf_reset(W.h, dev(np.ones(W.A, np.uint8)))
    orc.reset(Fo, Io, np.ones(W.A, np.uint8), seed=12)
    F, I, _ = sf.sf_get_state(W.h)
    assert np.array_equal(F[:, :2].astype(np.float64), Fo[:, :2])            # same spawn points
    assert np.array_equal(I[:, :2], Io[:, :2])
    mu = F[:, O.F_MU].astype(np.float64)
    assert np.abs(mu - Fo[:, O.F_MU]).max() <= 1e-6
    films = synth.film_code(sc.film_mm)
    assert (mu[films >= 85] == np.float32(1e-3)).all() and (films >= 85).sum() > 5     # aquaplaning agents
    assert mu.max() > 1.2                                                               # dry OGFC
    # the ego group's weather token and the rest of the observation
    obs = W.outputs()[0].cpu().numpy()
    oo = orc.observe(F.astype(np.float64), I)
    np.testing.assert_allclose(obs[:, 7], films * 0.01, atol=2e-6)
    assert np.array_equal(obs[:, 8:11], np.eye(3)[sc.surface])
    assert np.abs(obs[:, :14] - oo["obs"][:, :14]).max() <= 2e-5
    # the lane features (14, 15) too, except where the nearest lane is a near-tie:
    # an agent spawned on a lane vertex is at distance 0 from the segments that
    # end and start there (counted, as in the other parity tests)
    ties = 0
    for a in range(W.A):
        if np.abs(obs[a, 14:16] - oo["obs"][a, 14:16]).max() > 2e-5:
            w = int(np.searchsorted(sc.agent_off, a, side="right") - 1)
            assert lane_tie(orc, sc, w, F[a, :2].astype(np.float64)), a
            ties += 1
    print("lane near-ties at the spawn points:", ties)
    # the full observation's 11-value ego group carries Eq. weather_obs
    full = W.full_obs()
    fo = orc.observe_full(F.astype(np.float64), I)
    assert np.abs(full["obs"][:, :11] - fo["obs"][:, :11]).max() <= 2e-5
    # steps: state parity of the physics over the whole friction range
    acts = synth.ou_actions(W.A, 10, seed=3)
    worst = {}
    for t in range(10):
        F0, I0, _ = sf.sf_get_state(W.h)
        sf.sf_step(W.h, dev(acts[t]))
        F1, _, _ = sf.sf_get_state(W.h)
        Fe, Ie = F0.astype(np.float64), I0.copy()
        orc.step(Fe, Ie, acts[t].astype(np.float64), flags=O.FLAG_INVINCIBLE, want_obs=False)
        rows = np.nonzero(Ie[:, O.I_STATUS] & O.ALIVE)[0]
        for k, e in block_errors(F1, Fe, rows).items():
            worst[k] = max(worst.get(k, 0.0), float(e.max()))
    print("ALL model single-step worst relative errors:", worst)
    for k, e in worst.items():
        assert e <= 5e-5, (k, e)          # contact pairs included (see the contact tolerance)
    W.close()


def test_all_model_rejects_bad_films():
    sc = synth.with_water_films(synth.straight_road(num_agents=2), seed=1)
    for bad in (-0.1, float("nan"), float("inf")):
        s2 = synth.with_water_films(synth.straight_road(num_agents=2), seed=1)
        s2.film_mm = s2.film_mm.copy()
        s2.film_mm[1] = bad
        h = sf.sf_create(weather_model=sf.WEATHER_ALL)
        try:
            with pytest.raises(sf.SFError) as e:
                sf.sf_load_roads(h, s2)
            assert e.value.status == sf.SF_ERR_INVALID_ARG
        finally:
            sf.sf_destroy(h)
    s3 = synth.straight_road(num_agents=2)                 # no films at all
    h = sf.sf_create(weather_model=sf.WEATHER_ALL)
    try:
        with pytest.raises(sf.SFError):
            sf.sf_load_roads(h, s3)
        sf.sf_load_roads(h, sc)
    finally:
        sf.sf_destroy(h)
