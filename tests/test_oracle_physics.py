"""Pins of the FP64 oracle's vehicle step against closed forms and invariants.

Each test fixes one part of the substep so that a plausible slip (a dropped
term, a wrong sign, a swapped operand) fails: static suspension sag, free fall,
friction-limited stopping distance, the friction circle, the kinematic yaw
rate, coasting, the steering recurrence and fixed-axis rotation.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_08528_b300 import synth

G, M, K, R_W, L0 = 9.81, 1500.0, 35000.0, 0.33, 0.3
Z_STAR = 0.25 + R_W + (L0 - M * G / (4 * K))   # hardpoint depth + wheel + compressed spring


def one_agent(x=0.0, y=0.0, psi=0.0, v0=0.0, precip=0, surface=0, params=None):
    sc = synth.straight_road(num_agents=1, length=400.0, spacing=2.0)
    orc = O.Oracle(sc, params)
    F, I = orc.empty_state()
    orc.place(F, I, 0, x, y, psi, v0, x + 1000.0, y, precip, surface)
    return orc, F, I


def run(orc, F, I, act, steps, flags=O.FLAG_INVINCIBLE):
    act = np.asarray(act, np.float64).reshape(1, 3)
    hist = []
    for _ in range(steps):
        orc.step(F, I, act, flags=flags, want_obs=False)
        hist.append(F[0].copy())
    return np.asarray(hist)


def test_static_sag_value():
    # m g / (4 k) for the 1500 kg, 35 kN/m car
    assert abs(M * G / (4 * K) - 0.105107) < 1e-6
    assert abs(Z_STAR - 0.774893) < 1e-6


def test_equilibrium_is_exact():
    orc, F, I = one_agent()
    assert abs(F[0, O.F_PZ] - Z_STAR) < 1e-12
    h = run(orc, F, I, [0, 0, 0], 300)
    assert np.abs(h[:, O.F_PZ] - Z_STAR).max() < 1e-9
    assert np.abs(h[:, O.F_VX:O.F_WZ + 1]).max() < 1e-9


def test_settles_to_static_sag():
    orc, F, I = one_agent()
    F[0, O.F_PZ] += 0.05
    h = run(orc, F, I, [0, 0, 0], 300)
    assert abs(h[-1, O.F_PZ] - Z_STAR) < 1e-6
    # it really moved: the first steps are away from equilibrium
    assert abs(h[0, O.F_PZ] - Z_STAR) > 1e-2


def test_free_fall_recurrence():
    orc, F, I = one_agent()
    z0 = 10.0
    F[0, O.F_PZ] = z0
    h = 1.0 / 120.0
    act = np.zeros((1, 3))
    for n in range(1, 41):
        orc.substep_world(0, F, I, act, h)
        exact = z0 - G * h * h * n * (n + 1) / 2.0     # symplectic Euler: v first, then z
        assert abs(F[0, O.F_PZ] - exact) < 1e-12
        assert abs(F[0, O.F_VZ] + G * h * n) < 1e-12


@pytest.mark.parametrize("precip,surface,mu,brake_scale", [(2, 0, 0.5, 1.0), (3, 2, 0.2, 1.0), (0, 0, 0.9, 5.0)])
def test_locked_wheel_stopping_distance(precip, surface, mu, brake_scale):
    P = O.default_params()
    P.tau_brk_f *= brake_scale
    P.tau_brk_r *= brake_scale
    v0 = 20.0
    orc, F, I = one_agent(v0=v0, precip=precip, surface=surface, params=P)
    assert F[0, O.F_MU] == mu
    x0 = F[0, O.F_PX]
    for _ in range(900):
        orc.step(F, I, np.array([[-1.0, 0.0, 1.0]]), flags=O.FLAG_INVINCIBLE, want_obs=False)
        if math.hypot(F[0, O.F_VX], F[0, O.F_VY]) < 1e-6:
            break
    d = F[0, O.F_PX] - x0
    expect = v0 * v0 / (2 * mu * G)
    assert abs(d - expect) / expect < 0.01, (d, expect)
    assert abs(F[0, O.F_PY]) < 1e-6          # straight line
    assert np.abs(F[0, O.F_S0:O.F_S0 + 4]).max() < 1e-9   # wheels locked at rest


@pytest.mark.parametrize("act,binding", [([0.3, 1.0, 0.0], 0.9), ([1.0, 0.6, 0.0], 0.9), ([0.0, 1.0, 0.6], 0.999)])
def test_friction_circle_caps_planar_acceleration(act, binding):
    """Friction circle, per wheel |J| <= mu N h, hence for the chassis
    |sum J| <= mu h sum N.  With lambda_lat = 0 the tyre impulses are the only
    planar force (suspension loads act along the ground normal +z, the yaw
    damping wrench is a torque), so per substep
    |dv_xy| / h <= mu (sum N) / m, and sum N / m = dv_z / h + g.  The bound holds
    to rounding; with the wheels locked in a braking turn the car slides and
    the bound is reached (a cap per component instead of on |J| would allow
    up to sqrt(2) times the circle)."""
    mu = 0.5
    orc, F, I = one_agent(v0=20.0, precip=2, surface=0)
    hh = 1.0 / 120.0
    ratio = []
    for _ in range(960):
        v0 = F[0, O.F_VX:O.F_VZ + 1].copy()
        orc.substep_world(0, F, I, np.array([act], np.float64), hh)
        dv = F[0, O.F_VX:O.F_VZ + 1] - v0
        a_xy = math.hypot(dv[0], dv[1]) / hh
        ratio.append(a_xy / (mu * (dv[2] / hh + G)))
    ratio = np.asarray(ratio)
    assert ratio.max() <= 1.0 + 1e-9, ratio.max()
    assert ratio.max() >= binding, ratio.max()


def test_kinematic_yaw_rate_low_speed():
    delta = 0.1
    orc, F, I = one_agent(v0=2.0)
    for _ in range(150):
        orc.step(F, I, np.array([[0.0, delta / 0.45, 0.0]]), flags=O.FLAG_INVINCIBLE, want_obs=False)
    v = math.hypot(F[0, O.F_VX], F[0, O.F_VY])
    assert abs(F[0, O.F_DELTA] - delta) < 1e-6
    expect = v * math.tan(delta) / 2.6
    assert abs(F[0, O.F_WZ] - expect) / expect < 0.02, (F[0, O.F_WZ], expect)


def test_coasting_conserves_speed():
    orc, F, I = one_agent(v0=15.0, psi=0.3)
    h = run(orc, F, I, [0, 0, 0], 100)
    sp = np.hypot(h[:, O.F_VX], h[:, O.F_VY])
    assert np.abs(sp - 15.0).max() / 15.0 < 1e-10
    assert np.abs(h[:, O.F_PZ] - Z_STAR).max() < 1e-9


def test_steering_recurrence_matches_matrix_power():
    P = O.default_params()
    orc, F, I = one_agent()
    F[0, O.F_PZ] = 50.0                        # in the air: steering is decoupled
    target = 0.2
    hh = 1.0 / 120.0
    a = hh * P.kd / P.steer_inertia
    b = hh * P.kp / P.steer_inertia
    Mx = np.array([[1 - a, -b], [hh * (1 - a), 1 - hh * b]])
    c = np.array([b * target, hh * b * target])
    x = np.zeros(2)
    act = np.array([[0.0, target / 0.45, 0.0]])
    for n in range(1, 60):
        orc.substep_world(0, F, I, act, hh)
        x = Mx @ x + c
        assert abs(F[0, O.F_DELTA] - x[1]) < 1e-12
        assert abs(F[0, O.F_DDELTA] - x[0]) < 1e-10
    # closed form via the matrix power, not the loop
    Mn = np.linalg.matrix_power(Mx, 59)
    xs = np.linalg.solve(np.eye(2) - Mx, c)
    assert abs((xs + Mn @ (np.zeros(2) - xs))[1] - F[0, O.F_DELTA]) < 1e-12


def test_steering_torque_and_angle_clamps():
    P = O.default_params()
    orc, F, I = one_agent()
    F[0, O.F_PZ] = 50.0
    F[0, O.F_DELTA] = -0.45
    orc.substep_world(0, F, I, np.array([[0.0, 1.0, 0.0]]), 1.0 / 120.0)
    # Kp * 0.9 = 1655 N m exceeds the 1200 N m clamp
    assert abs(F[0, O.F_DDELTA] - (1.0 / 120.0) * P.tau_steer_max / P.steer_inertia) < 1e-12
    for _ in range(400):
        orc.substep_world(0, F, I, np.array([[0.0, 5.0, 0.0]]), 1.0 / 120.0)
        assert F[0, O.F_DELTA] <= 0.45 + 1e-15


@pytest.mark.parametrize("axis", [0, 2])
def test_fixed_axis_rotation(axis):
    P = O.default_params()
    P.lambda_yaw = 0.0                          # the yaw damping wrench is pinned below
    orc, F, I = one_agent(params=P)
    F[0, O.F_PZ] = 500.0
    w = 0.5
    F[0, O.F_WX + axis] = w
    hh = 1.0 / 120.0
    for _ in range(120):
        orc.substep_world(0, F, I, np.zeros((1, 3)), hh)
    q = F[0, O.F_QW:O.F_QZ + 1]
    ang = 2 * math.atan2(np.linalg.norm(q[1:]), q[0])
    assert abs(ang - w * 1.0) < 1e-6
    assert abs(q[1 + axis] / np.linalg.norm(q[1:]) - 1.0) < 1e-12
    assert abs(F[0, O.F_WX + axis] - w) < 1e-12          # principal axis: no precession


def test_gravity_sign_and_wheel_drive():
    # throttle accelerates forward (FWD), brake from rest does nothing
    orc, F, I = one_agent(v0=0.0)
    run(orc, F, I, [1.0, 0.0, 0.0], 30)
    assert F[0, O.F_VX] > 1.0 and F[0, O.F_S0] > 0 and F[0, O.F_S0 + 2] > 0
    orc2, F2, I2 = one_agent(v0=0.0)
    run(orc2, F2, I2, [-1.0, 0.0, 1.0], 30)
    assert abs(F2[0, O.F_VX]) < 1e-12


def test_rest_state_no_drift_under_brake_and_steer():
    orc, F, I = one_agent(v0=0.0)
    h = run(orc, F, I, [0.0, 0.5, 1.0], 60)
    assert np.abs(h[-1, O.F_PX:O.F_PY + 1]).max() < 1e-9


def test_yaw_damping_wrench_decay():
    P = O.default_params()
    orc, F, I = one_agent()
    F[0, O.F_PZ] = 500.0
    F[0, O.F_WZ] = 0.5
    hh = 1.0 / 120.0
    for n in range(1, 121):
        orc.substep_world(0, F, I, np.zeros((1, 3)), hh)
        assert abs(F[0, O.F_WZ] - 0.5 * (1 - hh * P.lambda_yaw / P.inertia[2]) ** n) < 1e-14
