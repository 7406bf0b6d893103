"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds input data only: road polylines shaped like the paper's
z-flattened, re-centred scenes (SceneFactory App. C: lane centrelines and road
edges inside a 200 m box, Waymo type codes), agent categories, placements and
action sequences.  It contains none of the method's arithmetic (no vehicle
physics, no spawn rule, no observation or reward); the CUDA library and the
FP64 oracle each implement those from the paper on their own.

Waymo type codes used: 1 freeway lane, 2 surface-street lane, 15 road-edge
boundary, 16 road-edge median.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

LANE_WIDTH = 3.6
BOX_HALF = 100.0


@dataclass
class Scene:
    """Worlds as CSR: world -> agents, world -> polylines -> points."""
    agent_off: np.ndarray   # int32 [W+1]
    poly_off: np.ndarray    # int32 [W+1]
    point_off: np.ndarray   # int32 [NPoly+1]
    poly_type: np.ndarray   # uint8 [NPoly]
    px: np.ndarray          # float32 [NPt]
    py: np.ndarray          # float32 [NPt]
    precip: np.ndarray      # uint8 [A]  0 dry, 1 light rain, 2 heavy rain, 3 snow
    surface: np.ndarray     # uint8 [A]  0 asphalt, 1 concrete, 2 gravel (ALL model: 0 AC, 1 SMA, 2 OGFC)
    film_mm: np.ndarray = None   # float32 [A] water film [mm] (the ALL weather model only)

    @property
    def num_worlds(self) -> int:
        return len(self.agent_off) - 1

    @property
    def num_agents(self) -> int:
        return int(self.agent_off[-1])

    @property
    def num_points(self) -> int:
        return int(self.point_off[-1])

    def world_points(self, w: int) -> int:
        return int(self.point_off[self.poly_off[w + 1]] - self.point_off[self.poly_off[w]])


def _assemble(worlds, agent_counts, precip, surface) -> Scene:
    """worlds: list (per world) of list of (type, xy[n,2]) polylines."""
    poly_off, point_off, types, xs, ys = [0], [0], [], [], []
    for polys in worlds:
        for t, xy in polys:
            types.append(t)
            xs.append(xy[:, 0])
            ys.append(xy[:, 1])
            point_off.append(point_off[-1] + len(xy))
        poly_off.append(len(types))
    agent_off = np.concatenate([[0], np.cumsum(agent_counts)]).astype(np.int32)
    cat = (lambda v: np.concatenate(v).astype(np.float32)) if xs else (lambda v: np.zeros(0, np.float32))
    return Scene(agent_off, np.asarray(poly_off, np.int32), np.asarray(point_off, np.int32),
                 np.asarray(types, np.uint8), cat(xs), cat(ys), np.asarray(precip, np.uint8),
                 np.asarray(surface, np.uint8))


# --------------------------------------------------------------------------- straight road
def straight_road(num_agents: int = 4, length: float = 200.0, spacing: float = 1.0):
    """One world: a straight two-lane two-way road along x, lanes at y = -1.8
    (eastbound) and y = +1.8 (westbound), road edges at y = +-3.6, points every
    ``spacing`` metres.  Dry asphalt for every agent."""
    n = int(round(length / spacing)) + 1
    x = np.linspace(-length / 2, length / 2, n)
    polys = [
        (2, np.stack([x, np.full(n, -LANE_WIDTH / 2)], 1)),
        (2, np.stack([x[::-1], np.full(n, LANE_WIDTH / 2)], 1)),
        (15, np.stack([x, np.full(n, -LANE_WIDTH)], 1)),
        (15, np.stack([x, np.full(n, LANE_WIDTH)], 1)),
    ]
    return _assemble([polys], [num_agents], np.zeros(num_agents), np.zeros(num_agents))


def straight_road_placements(seed: int = 1, xs=(-60.0, -20.0, 20.0, 60.0), goal_ahead: float = 100.0):
    """Agent placements on the straight road: x positions, alternating lanes,
    heading along the lane, initial speed uniform in [5, 20] m/s, goal
    ``goal_ahead`` metres ahead along the lane (clipped to the road end).
    Returns an array [n, 6] = (x, y, psi, v0, goal_x, goal_y)."""
    rng = np.random.default_rng(seed)
    out = []
    for i, x in enumerate(xs):
        east = i % 2 == 0
        y = -LANE_WIDTH / 2 if east else LANE_WIDTH / 2
        psi = 0.0 if east else math.pi
        v0 = rng.uniform(5.0, 20.0)
        gx = min(x + goal_ahead, 100.0) if east else max(x - goal_ahead, -100.0)
        out.append((x, y, psi, v0, gx, y))
    return np.asarray(out, np.float64)


def uniform_actions(num_agents: int, steps: int, seed: int = 2, steer_rad: float = 0.4,
                    theta_max: float = 0.45) -> np.ndarray:
    """Seeded actions [steps, A, 3] = (throttle, steer, brake) in the policy's
    [-1, 1] convention: one combined throttle/brake axis u ~ U[-1, 1] drives
    throttle = u and brake = -u (each rectified by the method), and a steering
    angle ~ U[-steer_rad, steer_rad] rad expressed as a fraction of theta_max."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1.0, 1.0, (steps, num_agents))
    s = rng.uniform(-steer_rad, steer_rad, (steps, num_agents)) / theta_max
    return np.stack([u, s, -u], -1).astype(np.float32)


def ou_actions(num_agents: int, steps: int, seed: int, theta: float = 0.15, sigma: float = 0.3) -> np.ndarray:
    """Smooth random actions: an Ornstein-Uhlenbeck process per channel, clipped to [-1, 1]."""
    rng = np.random.default_rng(seed)
    a = np.zeros((steps, num_agents, 3), np.float32)
    x = rng.uniform(-0.5, 0.5, (num_agents, 3))
    for t in range(steps):
        x = x - theta * x + sigma * rng.standard_normal((num_agents, 3))
        a[t] = np.clip(x, -1, 1)
    return a


def reset_mask(num_agents: int, step: int, frac: float = 0.2, seed: int = 7) -> np.ndarray:
    """Random per-step reset mask: each agent independently with probability ``frac``."""
    rng = np.random.default_rng([seed, step])
    return (rng.random(num_agents) < frac).astype(np.uint8)


# --------------------------------------------------------------------------- procedural roads
def _integrate_centerline(rng, start, heading, length, kmax, ds=0.25):
    """Dense centreline from straight / arc / clothoid pieces with |kappa| <= kmax.
    Returns xy [n, 2] and the tangent angle [n]."""
    x, y, th, k = float(start[0]), float(start[1]), float(heading), 0.0
    xs, ys, ths = [x], [y], [th]
    s = 0.0
    while s < length:
        kind = rng.integers(3)
        L = rng.uniform(15.0, 50.0)
        if kind == 0:
            k0 = k1 = 0.0
        elif kind == 1:
            k0 = k1 = rng.uniform(-kmax, kmax)
        else:
            k0, k1 = k, rng.uniform(-kmax, kmax)
        n = max(1, int(L / ds))
        for i in range(n):
            kk = k0 + (k1 - k0) * (i + 0.5) / n
            th += kk * ds
            x += ds * math.cos(th)
            y += ds * math.sin(th)
            xs.append(x); ys.append(y); ths.append(th)
            s += ds
            if s >= length:
                break
        k = k1
    return np.stack([xs, ys], 1), np.asarray(ths)


def _resample(xy, th, spacing):
    seg = np.hypot(np.diff(xy[:, 0]), np.diff(xy[:, 1]))
    s = np.concatenate([[0.0], np.cumsum(seg)])
    n = max(2, int(s[-1] / spacing) + 1)
    t = np.linspace(0.0, s[-1], n)
    return np.stack([np.interp(t, s, xy[:, 0]), np.interp(t, s, xy[:, 1])], 1), np.interp(t, s, th)


def _split_inside(xy, keep):
    """Split a polyline into runs of consecutive kept points (runs of >= 2 points)."""
    runs, cur = [], []
    for p, k in zip(xy, keep):
        if k:
            cur.append(p)
        elif cur:
            runs.append(np.asarray(cur)); cur = []
    if cur:
        runs.append(np.asarray(cur))
    return [r for r in runs if len(r) >= 2]


def _min_dist_to(points, poly):
    d = np.full(len(points), np.inf)
    for i in range(0, len(poly), 256):
        blk = poly[i:i + 256]
        dd = np.hypot(points[:, None, 0] - blk[None, :, 0], points[:, None, 1] - blk[None, :, 1]).min(1)
        d = np.minimum(d, dd)
    return d


def procedural_world(seed: int, points_range=(400, 1200), lanes_range=(4, 12), max_intersections=2,
                     kmax: float = 0.05):
    """One procedural road graph: 4-12 lanes on 1-3 corridors, the first built
    from straight/arc/clothoid pieces (|kappa| <= 0.05 1/m), the others straight
    corridors crossing it (0-2 four-way intersections); road edges half a lane
    outside the outer lanes, cut where another corridor crosses; every point
    inside the +-100 m box; about U[400, 1200] points in total."""
    rng = np.random.default_rng(seed)
    n_int = int(rng.integers(0, max_intersections + 1))
    n_corr = 1 + n_int
    n_lanes = int(rng.integers(lanes_range[0], lanes_range[1] + 1))
    n_lanes = max(n_lanes, 2 * n_corr)
    per = [n_lanes // n_corr + (1 if i < n_lanes % n_corr else 0) for i in range(n_corr)]
    target_pts = int(rng.integers(points_range[0], points_range[1] + 1))
    n_poly = n_lanes + 2 * n_corr
    corr_len = float(rng.uniform(150.0, 190.0))
    spacing = n_poly * corr_len / target_pts
    if spacing > 2.5:
        spacing = 2.5
        corr_len = spacing * target_pts / n_poly
    spacing = max(spacing, 0.5)
    lim = BOX_HALF - 1.0

    corridors = []  # (centre dense xy, theta dense, lanes)
    half0 = per[0] * LANE_WIDTH / 2
    k_c = min(kmax, 0.5 / (half0 + LANE_WIDTH))
    phi = rng.uniform(-math.pi, math.pi)
    start = np.array([-corr_len / 2 * math.cos(phi), -corr_len / 2 * math.sin(phi)])
    xy, th = _integrate_centerline(rng, start, phi + rng.uniform(-0.2, 0.2), corr_len, k_c)
    corridors.append((xy, th, per[0]))
    for c in range(1, n_corr):
        i0 = int(rng.uniform(0.3, 0.7) * (len(xy) - 1))
        cx, cy, ct = xy[i0, 0], xy[i0, 1], th[i0] + math.pi / 2 + rng.uniform(-0.15, 0.15)
        st = np.array([cx - corr_len / 2 * math.cos(ct), cy - corr_len / 2 * math.sin(ct)])
        n = int(corr_len / 0.25) + 1
        s = np.linspace(0.0, corr_len, n)
        cxy = np.stack([st[0] + s * math.cos(ct), st[1] + s * math.sin(ct)], 1)
        corridors.append((cxy, np.full(n, ct), per[c]))

    polys = []
    for ci, (cxy, cth, nl) in enumerate(corridors):
        rxy, rth = _resample(cxy, cth, spacing)
        nrm = np.stack([-np.sin(rth), np.cos(rth)], 1)
        others = [o for oj, o in enumerate(corridors) if oj != ci]
        for j in range(nl):
            off = (j - (nl - 1) / 2) * LANE_WIDTH
            lxy = rxy + off * nrm
            if off > 0:
                lxy = lxy[::-1]          # left-hand lanes run the other way
            keep = (np.abs(lxy) <= lim).all(1)
            for run in _split_inside(lxy, keep):
                polys.append((2, run))
        for side, t in ((-1, 16), (1, 15)):
            exy = rxy + side * (nl / 2) * LANE_WIDTH * nrm
            keep = (np.abs(exy) <= lim).all(1)
            for oxy, _, onl in others:
                keep &= _min_dist_to(exy, oxy) > onl * LANE_WIDTH / 2 + 1.0
            for run in _split_inside(exy, keep):
                polys.append((t, run))
    return polys


def procedural_scene(num_worlds: int, agents_per_world, seed_base: int = 1000, points_range=(400, 1200),
                     weather: str = "uniform", weather_seed: int = 99):
    """Worlds from ``procedural_world(seed_base + w)``.  ``agents_per_world`` is an
    int or a per-world sequence.  weather: "uniform" draws precipitation and
    surface uniformly per agent; "wet_mix" gives half the agents heavy rain on
    asphalt and half dry asphalt."""
    counts = (np.full(num_worlds, agents_per_world) if np.isscalar(agents_per_world)
              else np.asarray(agents_per_world))
    worlds = [procedural_world(seed_base + w, points_range) for w in range(num_worlds)]
    A = int(counts.sum())
    rng = np.random.default_rng(weather_seed)
    if weather == "uniform":
        precip, surface = rng.integers(0, 4, A), rng.integers(0, 3, A)
    elif weather == "wet_mix":
        precip, surface = np.where(rng.random(A) < 0.5, 2, 0), np.zeros(A, int)
    else:
        raise ValueError(weather)
    return _assemble(worlds, counts, precip, surface)


def ragged_scene(num_worlds: int = 1024, seed_base: int = 2000, max_agents: int = 32,
                 points_lo: int = 100, points_hi: int = 5000):
    """Ragged batch: per world, agents floor(exp(U[0, ln 32])) in [1, 32] and a
    road point budget exp(U[ln 100, ln 5000])."""
    rng = np.random.default_rng(seed_base)
    counts = np.clip(np.floor(np.exp(rng.uniform(0.0, math.log(max_agents), num_worlds))), 1, max_agents)
    pts = np.exp(rng.uniform(math.log(points_lo), math.log(points_hi), num_worlds)).astype(int)
    worlds = []
    for w in range(num_worlds):
        p = int(pts[w])
        lanes = (2, 4) if p < 300 else (4, 12)
        worlds.append(procedural_world(seed_base + 1 + w, (p, p), lanes_range=lanes,
                                       max_intersections=0 if p < 300 else 2))
    A = int(counts.sum())
    precip, surface = rng.integers(0, 4, A), rng.integers(0, 3, A)
    return _assemble(worlds, counts.astype(int), precip, surface)


def subscene(scene: Scene, worlds):
    """The scene restricted to the given worlds (renumbered CSR, the exact float32
    coordinates) and the indices of the agent rows kept."""
    worlds = list(worlds)
    polys, counts, rows = [], [], []
    for w in worlds:
        pl = []
        for p in range(scene.poly_off[w], scene.poly_off[w + 1]):
            k0, k1 = scene.point_off[p], scene.point_off[p + 1]
            pl.append((int(scene.poly_type[p]), np.stack([scene.px[k0:k1], scene.py[k0:k1]], 1)))
        polys.append(pl)
        a0, a1 = scene.agent_off[w], scene.agent_off[w + 1]
        counts.append(a1 - a0)
        rows.extend(range(a0, a1))
    rows = np.asarray(rows, int)
    return _assemble(polys, counts, scene.precip[rows], scene.surface[rows]), rows


def with_water_films(scene: Scene, seed: int, h_max: float = 1.2) -> Scene:
    """The scene with the ALL weather model's inputs (Sec. 3.3, App. B): a road
    surface 0 AC, 1 SMA, 2 OGFC and a water film depth uniform in [0, h_max] mm
    per agent (h_max 1.2 mm spans dry road to full aquaplaning)."""
    rng = np.random.default_rng(seed)
    A = scene.num_agents
    out = Scene(scene.agent_off, scene.poly_off, scene.point_off, scene.poly_type, scene.px, scene.py,
                scene.precip, rng.integers(0, 3, A).astype(np.uint8),
                (rng.random(A) * h_max).astype(np.float32))
    return out


def film_code(film_mm) -> np.ndarray:
    """The water film in hundredths of a millimetre, held to 2.55 mm, as the
    library stores it in the agent's weather byte (and the oracle's precip column)."""
    return np.minimum(255, np.rint(np.asarray(film_mm, np.float64) * 100.0)).astype(np.int32)
