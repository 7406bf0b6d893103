"""Pins of the surrogate's feature / target oracle: constant-velocity motion
has zero targets, targets and their inverse round-trip, level cars have an
identity tilt and the static sag as compression."""
import math

import numpy as np

from oracle import oracle as O
from oracle import surrogate as S


def placed(psi=0.7, v0=12.0):
    sc_f = np.zeros((1, O.NF)); sc_i = np.zeros((1, O.NI), np.int32)
    P = O.default_params()
    from paper_2605_08528_b300 import synth
    orc = O.Oracle(synth.straight_road(num_agents=1))
    orc.place(sc_f, sc_i, 0, 3.0, -2.0, psi, v0, 50.0, 0.0)
    return sc_f[0]


def test_level_car_features():
    f = placed(psi=0.7, v0=12.0)
    x = S.features(f, [0.5, -0.2, 0.0])
    assert abs(x[0] - 0.774893) < 1e-6
    assert np.allclose(x[1:5], [1, 0, 0, 0], atol=1e-12)            # no tilt
    assert np.allclose(x[5:8], [12.0, 0, 0], atol=1e-12)            # speed along the heading
    assert np.allclose(x[15:19], 1500 * 9.81 / (4 * 35000), atol=1e-9)   # static sag on every wheel
    assert np.allclose(x[19:23], 0, atol=1e-12)
    assert np.allclose(x[25:28], [0.5, -0.09, 0.0], atol=1e-12)
    assert x[28] == 0.9 and x[29] == 0.0


def test_constant_velocity_motion_has_zero_targets():
    f0 = placed(psi=-2.1, v0=8.0)
    f0[O.F_WZ] = 0.3                        # yaw rate about the (vertical) body z
    dt = 1 / 30
    f1 = f0.copy()
    f1[0:3] = f0[0:3] + f0[7:10] * dt
    yaw = 0.3 * dt
    q = S.quat_mul(f0[3:7], [math.cos(yaw / 2), 0, 0, math.sin(yaw / 2)])
    f1[3:7] = q
    assert np.abs(S.targets(f0, f1, dt)).max() < 1e-12


def test_targets_and_apply_round_trip():
    rng = np.random.default_rng(2)
    for _ in range(200):
        f0 = np.zeros(O.NF)
        f0[0:3] = rng.normal(0, 30, 3); f0[2] = 0.77 + rng.normal(0, 0.02)
        q = rng.normal(0, 1, 4); q[0] += 4; f0[3:7] = q / np.linalg.norm(q)
        f0[7:13] = rng.normal(0, 3, 6); f0[13:17] = rng.normal(30, 5, 4)
        f1 = f0.copy()
        f1[0:3] += rng.normal(0, 0.5, 3)
        q1 = S.quat_mul(f0[3:7], [1, *rng.normal(0, 0.05, 3)]); f1[3:7] = q1 / np.linalg.norm(q1)
        f1[7:13] += rng.normal(0, 0.5, 6); f1[13:17] += rng.normal(0, 1, 4)
        g = S.apply(f0, S.targets(f0, f1, 1 / 30), 1 / 30)
        assert np.abs(g[0:3] - f1[0:3]).max() < 1e-9
        assert min(np.abs(g[3:7] - f1[3:7]).max(), np.abs(g[3:7] + f1[3:7]).max()) < 1e-9
        assert np.abs(g[7:17] - f1[7:17]).max() < 1e-9


def test_rotation_vector_of_a_known_rotation():
    ax = np.array([1.0, 2.0, -2.0]) / 3.0
    q = np.concatenate([[math.cos(0.4)], math.sin(0.4) * ax])
    assert np.allclose(S.rotvec(q), 0.8 * ax, atol=1e-14)
    assert np.allclose(S.rotvec(-q), 0.8 * ax, atol=1e-14)      # sign of the quaternion does not matter
