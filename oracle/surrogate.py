"""FP64 oracle of the dynamics surrogate's inputs, targets and their inverse.

TEST INFRASTRUCTURE ONLY: used by tests/ and bench.py's CPU legs, never by the
product path.

State rows use the exchange layout (position 0-2, quaternion 3-6 (w, x, y, z),
velocity 7-9, angular velocity 10-12, wheel spins 13-16, steer 17, steer rate
18, ..., mu 23).  The heading frame at t rotates by psi about z, psi the angle
of the body x axis projected on the road plane.

inputs (30): z, tilt quaternion q_psi^-1 q (4), v and w in the heading frame
(3 + 3), wheel spins (4), suspension compressions (4) and rates (4), steer
angle and rate, decoded action (throttle, steer target, brake), mu, 0.
targets (16): heading-frame displacement - v_h dt (3), body rotation vector of
q_t^-1 q_t+1 - w_body dt (3), heading-frame velocity change (3), angular
velocity change (3), wheel spin change (4).
"""
from __future__ import annotations

import math

import numpy as np

HARD = [(1.3, 0.8), (1.3, -0.8), (-1.3, 0.8), (-1.3, -0.8)]
HARD_Z, WHEEL_R, REST, UZ_MIN, THETA_MAX = -0.25, 0.33, 0.3, 0.05, 0.45


def quat_mat(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def quat_mul(a, b):
    a0, av = a[0], np.asarray(a[1:])
    b0, bv = b[0], np.asarray(b[1:])
    return np.concatenate([[a0 * b0 - av @ bv], a0 * bv + b0 * av + np.cross(av, bv)])


def heading(q):
    R = quat_mat(q)
    n = math.hypot(R[0, 0], R[1, 0])
    return (R[0, 0] / n, R[1, 0] / n) if n > 0 else (1.0, 0.0)


def rot_z(c, s, v):
    """world -> heading frame"""
    return np.array([c * v[0] + s * v[1], -s * v[0] + c * v[1], v[2]])


def features(f, action):
    f = np.asarray(f, np.float64)
    q = f[3:7]
    c, s = heading(q)
    psi = math.atan2(s, c)
    qpsi_inv = np.array([math.cos(psi / 2), 0.0, 0.0, -math.sin(psi / 2)])
    tilt = quat_mul(qpsi_inv, q)
    R = quat_mat(q)
    u = R[:, 2]
    comp, rate = np.zeros(4), np.zeros(4)
    for i, (bx, by) in enumerate(HARD):
        rb = R @ np.array([bx, by, HARD_Z])
        if u[2] > UZ_MIN:
            t = (f[2] + rb[2]) / u[2]
            l = t - WHEEL_R
            if l < REST:
                comp[i] = REST - max(l, 0.0)
                rate[i] = -(f[9] + np.cross(f[10:13], rb)[2]) / u[2]
    a = np.asarray(action, np.float64)
    dec = [min(max(a[0], 0), 1), THETA_MAX * min(max(a[1], -1), 1), min(max(a[2], 0), 1)]
    return np.concatenate([[f[2]], tilt, rot_z(c, s, f[7:10]), rot_z(c, s, f[10:13]), f[13:17], comp, rate,
                           f[17:19], dec, [f[23], 0.0]])


def rotvec(q):
    q = np.asarray(q, np.float64)
    if q[0] < 0:
        q = -q
    n = np.linalg.norm(q[1:])
    ang = 2 * math.atan2(n, q[0])
    return q[1:] * (ang / n) if n > 1e-300 else 2 * q[1:]


def targets(f0, f1, dt):
    f0 = np.asarray(f0, np.float64)
    f1 = np.asarray(f1, np.float64)
    c, s = heading(f0[3:7])
    vh0 = rot_z(c, s, f0[7:10])
    dp = rot_z(c, s, f1[0:3] - f0[0:3]) - vh0 * dt
    q0inv = f0[3:7] * np.array([1, -1, -1, -1])
    th = rotvec(quat_mul(q0inv, f1[3:7])) - quat_mat(f0[3:7]).T @ f0[10:13] * dt
    dv = rot_z(c, s, f1[7:10]) - vh0
    dw = rot_z(c, s, f1[10:13]) - rot_z(c, s, f0[10:13])
    return np.concatenate([dp, th, dv, dw, f1[13:17] - f0[13:17]])


def apply(f0, d, dt):
    """chassis state after one step from f0 given targets d (inverse of targets)"""
    f0 = np.asarray(f0, np.float64)
    d = np.asarray(d, np.float64)
    c, s = heading(f0[3:7])
    back = lambda v: np.array([c * v[0] - s * v[1], s * v[0] + c * v[1], v[2]])
    vh0 = rot_z(c, s, f0[7:10])
    wh0 = rot_z(c, s, f0[10:13])
    out = f0.copy()
    out[0:3] = f0[0:3] + back(d[0:3] + vh0 * dt)
    th = d[3:6] + quat_mat(f0[3:7]).T @ f0[10:13] * dt
    ang = np.linalg.norm(th)
    e = np.concatenate([[math.cos(ang / 2)], th * (math.sin(ang / 2) / ang if ang > 0 else 0.5)])
    q = quat_mul(f0[3:7], e)
    out[3:7] = q / np.linalg.norm(q)
    out[7:10] = back(vh0 + d[6:9])
    out[10:13] = back(wh0 + d[9:12])
    out[13:17] = f0[13:17] + d[12:16]
    return out
