"""Shared helpers of the GPU parity tests: sub-scenes, state conversion and the
per-block error measures used against the FP64 oracle."""
from __future__ import annotations

import math

import numpy as np

from paper_2605_08528_b300 import synth

# state blocks of the exchange layout and the floor of each relative error
BLOCKS = {
    "position": (slice(0, 3), 1.0),
    "velocity": (slice(7, 10), 1.0),
    "angular_velocity": (slice(10, 13), 1.0),
    "wheel_spin": (slice(13, 17), 1.0),
    "steer": (slice(17, 18), 1e-2),
    "steer_rate": (slice(18, 19), 1.0),
}
# FP32 holds a unit quaternion to ~6e-8 per component, so the attitude error is
# measured as a rotation angle relative to max(attitude angle, 0.1 rad)
ATT_FLOOR = 0.1


def quat_angle(q):
    q = np.asarray(q, np.float64)
    return 2 * np.arctan2(np.linalg.norm(q[..., 1:], axis=-1), np.abs(q[..., 0]))


def quat_err(qa, qb):
    """Angle of qa * conj(qb) per row."""
    qa = np.asarray(qa, np.float64); qb = np.asarray(qb, np.float64)
    w1, x1, y1, z1 = qa.T
    w2, x2, y2, z2 = qb.T
    # qa * conj(qb)
    w = w1 * w2 + x1 * x2 + y1 * y2 + z1 * z2
    x = -w1 * x2 + x1 * w2 - y1 * z2 + z1 * y2
    y = -w1 * y2 + y1 * w2 - z1 * x2 + x1 * z2
    z = -w1 * z2 + z1 * w2 - x1 * y2 + y1 * x2
    return 2 * np.arctan2(np.sqrt(x * x + y * y + z * z), np.abs(w))


def block_errors(F_gpu, F_ref, rows=None):
    """Relative error per state block, per agent: ||d|| / max(||x||, floor)."""
    G = np.asarray(F_gpu, np.float64)
    R = np.asarray(F_ref, np.float64)
    if rows is not None:
        G, R = G[rows], R[rows]
    out = {}
    for name, (sl, floor) in BLOCKS.items():
        d = np.linalg.norm(G[:, sl] - R[:, sl], axis=1)
        out[name] = d / np.maximum(np.linalg.norm(R[:, sl], axis=1), floor)
    out["attitude"] = quat_err(G[:, 3:7], R[:, 3:7]) / np.maximum(quat_angle(R[:, 3:7]), ATT_FLOOR)
    return out


subscene = synth.subscene


def point_offset_map(scene, worlds):
    """Global point index in `scene` of each point index of subscene(scene, worlds)."""
    m = []
    for w in worlds:
        m.extend(range(scene.point_off[scene.poly_off[w]], scene.point_off[scene.poly_off[w + 1]]))
    return np.asarray(m, int)


def lex_margin_points(scene, w, p, idx_list, L=32):
    """Distance margin of the k-NN selection of point p (float64): min over the
    boundary between rank L-1 and L of |d_L - d_(L-1)| and between adjacent ranks."""
    q0, q1 = scene.point_off[scene.poly_off[w]], scene.point_off[scene.poly_off[w + 1]]
    d = np.hypot(scene.px[q0:q1].astype(np.float64) - p[0], scene.py[q0:q1].astype(np.float64) - p[1])
    ds = np.sort(d)
    k = min(L + 1, len(ds))
    if k < 2:
        return math.inf
    return float(np.diff(ds[:k]).min())


def in_contact(F, I, scene):
    """Per agent: footprint overlap with another alive agent of its world (FP64 SAT)."""
    from oracle import oracle as O
    out = np.zeros(len(F), bool)
    alive = (I[:, O.I_STATUS] & O.ALIVE) != 0
    psi = 2 * np.arctan2(F[:, O.F_QZ], F[:, O.F_QW])
    for w in range(scene.num_worlds):
        a0, a1 = scene.agent_off[w], scene.agent_off[w + 1]
        for i in range(a0, a1):
            if not alive[i]:
                continue
            for j in range(i + 1, a1):
                if not alive[j] or np.hypot(*(F[j, :2] - F[i, :2])) > 4.85:
                    continue
                d, _ = O.sat(F[i, :2], [np.cos(psi[i]), np.sin(psi[i])], F[j, :2], [np.cos(psi[j]), np.sin(psi[j])])
                if d > 0:
                    out[i] = out[j] = True
    return out


TIE = 1e-5


def heading(F, a):
    """Unit heading (x, y) of agent a: the body x axis projected on the road plane."""
    from oracle import oracle as O
    qw, qx, qy, qz = (float(F[a, k]) for k in (O.F_QW, O.F_QX, O.F_QY, O.F_QZ))
    hx, hy = 1.0 - 2.0 * (qy * qy + qz * qz), 2.0 * (qx * qy + qw * qz)
    n = math.hypot(hx, hy)
    return np.array([hx / n, hy / n]) if n > 0 else np.array([1.0, 0.0])


def agent_tie(scene, F, I, w, a_local, p, K=8):
    """True if the selection of the K nearest alive other agents of p has a near-tie."""
    from oracle import oracle as O
    a0, a1 = scene.agent_off[w], scene.agent_off[w + 1]
    d = [np.hypot(F[j, 0] - p[0], F[j, 1] - p[1]) for j in range(a0, a1)
         if j != a_local and I[j, O.I_STATUS] & O.ALIVE]
    ds = np.sort(np.asarray(d, np.float64))[:K + 1]
    return len(ds) > 1 and np.diff(ds).min() < TIE


def ttc_tie(F, a, j, gpu_feature, tol, trials=200, eps=1e-5):
    """True if the FP64 TTC of pair (a, j) comes within tol of the GPU's TTC
    feature (TTC / 10 s) for some perturbation of the pair's positions and
    velocities by ~eps (m, m/s) and headings by ~eps rad: the quadratic's root
    is ill-conditioned there (a grazing closest approach, or the choice
    between no root and a root).  A genuine discrepancy matches none."""
    from oracle import oracle as O
    rng = np.random.default_rng(1000 * a + j)
    pi, vi, hi = F[a, 0:2].astype(np.float64), F[a, 7:9].astype(np.float64), heading(F, a)
    pj, vj, hj = F[j, 0:2].astype(np.float64), F[j, 7:9].astype(np.float64), heading(F, j)

    def rot(h, e):
        c, s = math.cos(e), math.sin(e)
        return np.array([c * h[0] - s * h[1], s * h[0] + c * h[1]])

    for _ in range(trials):
        e = rng.normal(0, eps, 10)
        t = O.ttc(pi + e[0:2], rot(hi, e[8]), vi + e[2:4], pj + e[4:6], rot(hj, e[9]), vj + e[6:8])
        if abs(t / 10.0 - gpu_feature) <= tol:
            return True
    return False
