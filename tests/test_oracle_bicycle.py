"""Pins of the oracle's kinematic bicycle backend (Sec. 4.4 vehicle dynamics
ablation: front-wheel steering, wheelbase 2.6 m, steering limit 30 degrees, no
suspension, contact response or lateral slip).

Closed forms: constant throttle on a straight line (discrete sum of the
velocity recurrence), braking to rest without reversing, a constant steer at
constant speed tracing a regular polygon inscribed in one circle, the yaw rate
v tan(delta) / (WB sqrt(1 + tan^2(delta) / 4)) of the centre-of-mass model,
and the 30 degree steering limit.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_08528_b300 import synth

P = O.default_params()
DT = 1.0 / 30.0
WB = 2.6


def row(x=0.0, y=0.0, psi=0.0, v=10.0):
    sc = synth.straight_road(num_agents=1)
    orc = O.Oracle(sc)
    F, I = orc.empty_state()
    orc.place(F, I, 0, x, y, psi, v, 1e3, 0.0)
    return F[0].copy()


def test_actuator_accelerations_and_steer_limit():
    assert abs(P.bike_theta_max - math.radians(30)) < 1e-15
    assert abs(P.bike_a_drive - 2 * 600.7 / (0.33 * 1500)) < 1e-12
    assert abs(P.bike_a_brake - 2 * (1090.5 + 980.7) / (0.33 * 1500)) < 1e-12
    f = row()
    O.bicycle_agent(f, [0.0, 1.0, 0.0])
    assert abs(f[O.F_DELTA] - math.radians(30)) < 1e-15
    f = row()
    O.bicycle_agent(f, [0.0, -3.0, 0.0])          # clamped to the limit
    assert abs(f[O.F_DELTA] + math.radians(30)) < 1e-15


def test_straight_line_constant_throttle_closed_form():
    f = row(x=-50.0, v=5.0)
    a = P.bike_a_drive
    n = 90
    for _ in range(n):
        O.bicycle_agent(f, [1.0, 0.0, 0.0], DT)
    # v_k = v0 + k a dt;  x_n = x0 + dt sum_{k=1..n} v_k
    x_ref = -50.0 + n * 5.0 * DT + a * DT * DT * n * (n + 1) / 2
    assert abs(f[O.F_PX] - x_ref) < 1e-9
    assert abs(f[O.F_PY]) < 1e-12 and abs(f[O.F_VX] - (5.0 + n * a * DT)) < 1e-9
    assert abs(f[O.F_S0] - f[O.F_VX] / 0.33) < 1e-9


def test_braking_stops_without_reversing():
    f = row(v=12.0)
    ab = P.bike_a_brake
    xs = [f[O.F_PX]]
    for _ in range(60):
        O.bicycle_agent(f, [0.0, 0.0, 1.0], DT)
        xs.append(f[O.F_PX])
    assert f[O.F_VX] == 0.0 and f[O.F_VY] == 0.0
    assert np.all(np.diff(xs) >= 0)
    # steps until rest and the distance: sum of max(0, v0 - k ab dt) dt
    ks = np.arange(1, 61)
    d_ref = float(np.sum(np.maximum(0.0, 12.0 - ks * ab * DT)) * DT)
    assert abs(xs[-1] - d_ref) < 1e-9


@pytest.mark.parametrize("steer", [0.2, -0.7, 1.0])
def test_constant_steer_traces_a_regular_polygon(steer):
    v = 8.0
    f = row(v=v)
    O.bicycle_agent(f, [0.0, steer, 0.0], DT)       # first step sets delta; speed stays v
    delta = P.bike_theta_max * steer
    beta = math.atan(0.5 * math.tan(delta))
    rate = v * math.tan(delta) / (WB * math.sqrt(1 + math.tan(delta) ** 2 / 4))
    assert abs(f[O.F_WZ] - rate) < 1e-12
    assert abs(rate - v / (WB / 2) * math.sin(beta)) < 1e-12
    pts = []
    for _ in range(40):
        O.bicycle_agent(f, [0.0, steer, 0.0], DT)
        pts.append(f[:2].copy())
    pts = np.array(pts)
    # side v dt, exterior angle rate dt: circumradius v dt / (2 sin(rate dt / 2))
    R = v * DT / (2 * math.sin(abs(rate) * DT / 2))
    (ax, ay), (bx, by), (cx, cy) = pts[0], pts[13], pts[27]
    dd = 2 * (ax * (by - cy) + bx * (cy - ay) + cx * (ay - by))
    ux = ((ax * ax + ay * ay) * (by - cy) + (bx * bx + by * by) * (cy - ay) + (cx * cx + cy * cy) * (ay - by)) / dd
    uy = ((ax * ax + ay * ay) * (cx - bx) + (bx * bx + by * by) * (ax - cx) + (cx * cx + cy * cy) * (bx - ax)) / dd
    r = np.hypot(pts[:, 0] - ux, pts[:, 1] - uy)
    assert np.abs(r - R).max() < 1e-8
    assert np.abs(np.hypot(*np.diff(pts, axis=0).T) - v * DT).max() < 1e-12
    # the centre lies on the side the car turns to
    assert np.sign(uy) == np.sign(steer)


def test_level_state_and_events_through_the_step():
    sc = synth.straight_road(num_agents=1)
    orc = O.Oracle(sc)
    F, I = orc.empty_state()
    orc.place(F, I, 0, 0.0, -1.8, 0.0, 15.0, 20.0, -1.8)
    zstar = F[0, O.F_PZ]
    out = None
    for t in range(60):
        out = orc.step(F, I, np.array([[0.3, 0.0, 0.0]]), flags=O.FLAG_BICYCLE)
        if out["events"][0] & O.EV["goal"]:
            break
    assert out["events"][0] & O.EV["goal"]                # 17 m (3 m goal radius) at ~15 m/s: ~34 steps
    assert 30 <= t <= 36
    assert abs(F[0, O.F_PZ] - zstar) < 1e-12 or not (I[0, O.I_STATUS] & O.ALIVE)
