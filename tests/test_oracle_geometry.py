"""Pins of the oracle's pair geometry, road queries, observations, events and
resets: brute force on tiny inputs, polygon clipping, hand-built cases, the
paper's printed TTC circle geometry and the published SplitMix64 outputs."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_08528_b300 import synth

HL, HW = 2.25, 0.9


# ----------------------------------------------------------------------------- SAT
def box_poly(c, h):
    ax, ay = np.array(h), np.array([-h[1], h[0]])
    c = np.asarray(c)
    return [c + HL * ax + HW * ay, c - HL * ax + HW * ay, c - HL * ax - HW * ay, c + HL * ax - HW * ay]


def clip_area(subject, clipper):
    """Sutherland-Hodgman clip of convex polygons (both counter-clockwise); returns the area."""
    def inside(p, a, b):
        return (b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0]) >= 0

    def inter(p, q, a, b):
        r, s = q - p, b - a
        den = r[0] * s[1] - r[1] * s[0]
        t = ((a[0] - p[0]) * s[1] - (a[1] - p[1]) * s[0]) / den
        return p + t * r

    out = list(subject)
    for i in range(len(clipper)):
        a, b = clipper[i], clipper[(i + 1) % len(clipper)]
        inp, out = out, []
        if not inp:
            break
        for j in range(len(inp)):
            p, q = inp[j - 1], inp[j]
            if inside(q, a, b):
                if not inside(p, a, b):
                    out.append(inter(p, q, a, b))
                out.append(q)
            elif inside(p, a, b):
                out.append(inter(p, q, a, b))
    if len(out) < 3:
        return 0.0
    x = np.array([p[0] for p in out]); y = np.array([p[1] for p in out])
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


def rand_pair(rng):
    ci = rng.uniform(-3, 3, 2); cj = rng.uniform(-3, 3, 2)
    a, b = rng.uniform(-math.pi, math.pi, 2)
    return ci, np.array([math.cos(a), math.sin(a)]), cj, np.array([math.cos(b), math.sin(b)])


def test_sat_matches_polygon_clipping():
    rng = np.random.default_rng(5)
    hits = 0
    for _ in range(20000):
        ci, hi, cj, hj = rand_pair(rng)
        d, _ = O.sat(ci, hi, cj, hj)
        area = clip_area(box_poly(ci, hi), box_poly(cj, hj))
        if area > 1e-9:
            assert d > 0
            hits += 1
        elif area == 0.0:
            assert d <= 1e-9
    assert 2000 < hits < 18000


def test_sat_depth_is_minimum_translation():
    rng = np.random.default_rng(6)
    n = 0
    while n < 3000:
        ci, hi, cj, hj = rand_pair(rng)
        d, nv = O.sat(ci, hi, cj, hj)
        if d <= 1e-3:
            continue
        n += 1
        assert abs(np.linalg.norm(nv) - 1) < 1e-12
        assert np.dot(nv, cj - ci) >= -1e-12             # normal points from i to j
        eps = 1e-6
        d_out, _ = O.sat(ci, hi, cj + (d + eps) * nv, hj)
        d_in, _ = O.sat(ci, hi, cj + (d - eps) * nv, hj)
        assert d_out == 0.0 and d_in > 0


# ----------------------------------------------------------------------------- roads
def tiny_scene(rng, n_poly=5, gap=True):
    polys = []
    for p in range(n_poly):
        n = int(rng.integers(2, 12))
        start = rng.uniform(-20, 20, 2)
        steps = rng.uniform(0.4, 2.5, (n, 2)) * rng.choice([-1, 1], 2)
        xy = start + np.cumsum(steps, 0)
        if gap and p == 0 and n > 4:
            xy[n // 2:] += 5.0                        # a > 3 m discontinuity inside the polyline
        polys.append((int(rng.choice([1, 2, 15, 16, 3])), xy))
    polys[0] = (2, polys[0][1])
    return synth._assemble([polys], [3], [0, 0, 0], [0, 0, 0])


def brute_nearest_lane(sc, q):
    best = (math.inf, -1)
    for p in range(sc.poly_off[0], sc.poly_off[1]):
        if sc.poly_type[p] not in (1, 2):
            continue
        for k in range(sc.point_off[p], sc.point_off[p + 1] - 1):
            a = np.array([sc.px[k], sc.py[k]], float); b = np.array([sc.px[k + 1], sc.py[k + 1]], float)
            if np.linalg.norm(b - a) > 3.0:
                continue
            # minimise over a dense sampling + the exact endpoints: the projection
            # formula is not re-used here
            ts = np.concatenate([np.linspace(0, 1, 2001), [0.0, 1.0]])
            pts = a[None] + ts[:, None] * (b - a)[None]
            d2 = ((pts - q[None]) ** 2).sum(1).min()
            if d2 < best[0] - 1e-9:
                best = (d2, k)
    return best


def test_nearest_lane_brute_force():
    rng = np.random.default_rng(11)
    for trial in range(40):
        sc = tiny_scene(rng)
        orc = O.Oracle(sc)
        for _ in range(10):
            q = rng.uniform(-25, 25, 2)
            k, dist, lat, tan = orc.nearest_lane(0, q)
            d2, kb = brute_nearest_lane(sc, q)
            if kb < 0:
                assert k == -1
                continue
            assert abs(dist * dist - d2) < 1e-5 * max(1.0, d2)
            if k != kb:     # only an (almost) exact tie may pick another segment
                assert abs(dist * dist - d2) < 1e-6
            # lateral: left of the segment direction is positive
            a = np.array([sc.px[k], sc.py[k]], float)
            assert abs(lat - (tan[0] * (q[1] - a[1]) - tan[1] * (q[0] - a[0]))) < 1e-12
            assert abs(abs(lat) - dist) < 1e-9 or abs(lat) < dist


def test_segment_gap_and_box_rules():
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [5.0, 0.0], [6.0, 0.0]])       # 4 m gap between 1 and 2
    sc = synth._assemble([[(2, xy)]], [1], [0], [0])
    orc = O.Oracle(sc)
    k, dist, _, _ = orc.nearest_lane(0, np.array([3.0, 0.5]))
    assert k in (0, 2) and abs(dist - math.hypot(2.0, 0.5)) < 1e-12
    xy2 = np.array([[99.5, 0.0], [100.5, 0.0], [101.0, 0.0]])              # outside the 200 m box
    sc2 = synth._assemble([[(2, xy2)]], [1], [0], [0])
    assert O.Oracle(sc2).nearest_lane(0, np.array([100.0, 0.0]))[0] == -1


def test_knn_points_and_agents_brute_force():
    rng = np.random.default_rng(3)
    sc = synth.procedural_scene(2, 12, seed_base=50)
    orc = O.Oracle(sc)
    F, I = orc.empty_state()
    orc.reset(F, I, np.ones(sc.num_agents, np.uint8), seed=9)
    # jitter positions so the query points are generic
    F[:, O.F_PX] += rng.uniform(-2, 2, sc.num_agents)
    F[:, O.F_PY] += rng.uniform(-2, 2, sc.num_agents)
    out = orc.observe(F, I)
    for w in range(sc.num_worlds):
        q0, q1 = sc.point_off[sc.poly_off[w]], sc.point_off[sc.poly_off[w + 1]]
        pts = np.stack([sc.px[q0:q1], sc.py[q0:q1]], 1).astype(float)
        for a in range(sc.agent_off[w], sc.agent_off[w + 1]):
            p = F[a, :2]
            d2 = ((pts - p) ** 2).sum(1)
            order = np.lexsort((np.arange(q0, q1), d2))[:32] + q0
            assert np.array_equal(out["knn_pts"][a], order)
            others = [j for j in range(sc.agent_off[w], sc.agent_off[w + 1]) if j != a]
            dd = np.array([((F[j, :2] - p) ** 2).sum() for j in others])
            o2 = np.array(others)[np.lexsort((others, dd))][:8]
            assert np.array_equal(out["knn_agents"][a][:len(o2)], o2)


def test_knn_pads_when_few():
    sc = synth._assemble([[(2, np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0]]))]], [2], [0, 0], [0, 0])
    orc = O.Oracle(sc)
    F, I = orc.empty_state()
    orc.place(F, I, 0, 0.5, 0.2, 0.0, 5.0, 50.0, 0.0)
    orc.place(F, I, 1, 30.0, 0.0, 0.0, 5.0, 80.0, 0.0)
    out = orc.observe(F, I)
    assert list(out["knn_pts"][0][:3]) == [0, 1, 2] and (out["knn_pts"][0][3:] == -1).all()
    assert out["knn_agents"][0][0] == 1 and (out["knn_agents"][0][1:] == -1).all()
    obs = out["obs"][0]
    assert obs[16 + 9] == 1.0 and obs[16 + 10 + 9] == 0.0          # neighbour valid flags
    assert obs[96 + 2 * 7 + 6] == 1.0 and obs[96 + 3 * 7 + 6] == 0.0  # road point valid flags
    assert np.all(obs[96 + 3 * 7:] == 0.0)


# ----------------------------------------------------------------------------- TTC, DRAC, shaping
def test_ttc_circle_geometry_matches_paper_example():
    r, d = O.ttc_circles(4.0, 2.0, 2.6)        # App. D: r ~ 1.10 m, d ~ 1.12 m
    assert abs(r - 1.10) < 5e-3 and abs(d - 1.12) < 5e-3
    r, d = O.ttc_circles(4.5, 1.8, 2.6)
    assert abs(r - 0.99) < 1e-12 and abs(d - 1.3) < 1e-12          # d capped at WB/2


def test_ttc_head_on_closed_form():
    r, d = O.ttc_circles(4.5, 1.8, 2.6)
    for D, V in [(30.0, 10.0), (12.0, 4.0), (50.0, 25.0)]:
        t = O.ttc([0, 0], [1, 0], [V / 2, 0], [D, 0], [-1, 0], [-V / 2, 0])
        expect = (D - 2 * d - 2 * r) / V
        assert abs(t - min(expect, 10.0)) < 1e-12
    # behind the ego, separating, parallel miss, already overlapping
    assert O.ttc([0, 0], [1, 0], [0, 0], [-20, 0], [1, 0], [5, 0]) == 10.0
    assert O.ttc([0, 0], [1, 0], [0, 0], [20, 0], [1, 0], [5, 0]) == 10.0
    assert O.ttc([0, 0], [1, 0], [10, 0], [20, 5], [1, 0], [0, 0]) == 10.0
    assert O.ttc([0, 0], [1, 0], [10, 0], [2.0, 0.5], [1, 0], [0, 0]) == 0.0


def test_ttc_lateral_offset_closed_form():
    # j crosses in front of i: moving along -y at x = D; first touch of circle pairs
    r, d = O.ttc_circles(4.5, 1.8, 2.6)
    D, y0, V = 2.5, 20.0, 5.0
    t = O.ttc([0, 0], [1, 0], [0, 0], [D, y0], [0, -1], [0, -V])
    # only i's front circle is within 2r of j's track; j's leading circle touches first
    dx = D - d
    assert dx < 2 * r < D
    expect = ((y0 - d) - math.sqrt((2 * r) ** 2 - dx * dx)) / V
    assert abs(t - expect) < 1e-12
    # far to the side: the track misses every circle
    assert O.ttc([0, 0], [1, 0], [0, 0], [8.0, y0], [0, -1], [0, -V]) == 10.0


def test_drac_hand_cases():
    # closing 10 m/s, gap 10 m (centres 14.5 m apart, two 4.5 m cars in line) -> 5.0 m/s^2
    assert abs(O.drac([0, 0], [10, 0], [14.5, 0], [0, 0]) - 5.0) < 1e-12
    assert O.drac([0, 0], [0, 0], [14.5, 0], [10, 0]) == 0.0             # opening
    assert abs(O.drac([0, 0], [2, 0], [4.0, 0], [0, 0]) - 4.0 / 0.2) < 1e-12   # gap floored at 0.1 m
    # only the radial component closes
    assert abs(O.drac([0, 0], [0, 10], [14.5, 0], [0, 0])) < 1e-12
    # side by side on adjacent lanes (3.6 m apart): the gap is 3.6 - 2 * 0.9 = 1.8 m
    assert abs(O.drac([0, 0], [0, 1.0], [0, 3.6], [0, 0]) - 1.0 / (2 * 1.8)) < 1e-12
    # crossing at right angles: 2.25 + 0.9 of reach along the line of centres
    assert abs(O.drac([0, 0], [5.0, 0], [10.0, 0], [0, 0], hj=(0.0, 1.0)) - 25.0 / (2 * (10 - 3.15))) < 1e-12


def test_lane_keep_score_and_penalty():
    assert abs(O.lane_keep_q(0.0, 1.0) - 1.0) < 1e-15
    assert abs(O.lane_keep_q(1.75, 1.0) - math.exp(-1)) < 1e-15
    assert abs(O.lane_keep_q(0.0, 0.0) - 0.2) < 1e-15
    assert abs(O.lane_keep_q(0.0, -1.0) - 0.2) < 1e-15
    assert abs(O.penalty(0.10, 0.1, 0.5, 0.35) - 0.2) < 1e-15
    assert abs(O.penalty(0.10, 0.2, 0.5, 0.15) - 0.15) < 1e-15
    assert abs(O.penalty(0.07, 1.0, 0.5, 0.40) - 0.07) < 1e-15


def test_splitmix64_published_outputs():
    # Vigna's splitmix64.c: state 0, first three outputs
    g = 0x9E3779B97F4A7C15
    assert O.splitmix64(0) == 0xE220A8397B1DCDAF
    assert O.splitmix64(g) == 0x6E789E6AA1B965F4
    assert O.splitmix64((2 * g) & 0xFFFFFFFFFFFFFFFF) == 0x06C45D188009454F


def test_obs_dimension():
    assert O.OBS == 16 + 8 * 10 + 32 * 7 == 320


# ----------------------------------------------------------------------------- events
def road_world(n=2):
    sc = synth.straight_road(num_agents=n)
    orc = O.Oracle(sc)
    F, I = orc.empty_state()
    return sc, orc, F, I


def test_ego_features_hand_case():
    sc, orc, F, I = road_world(1)
    orc.place(F, I, 0, 0.0, -1.8, 0.0, 10.0, 50.0, -1.8, precip=1, surface=2)
    o = orc.observe(F, I)["obs"][0]
    assert np.allclose(o[:8], [0.5, 0.0, 0.0, 1.0, 0.5, 1.0, 0.0, 1 / 3], atol=1e-12)
    assert list(o[8:11]) == [0, 0, 1]
    assert abs(o[13] - 0.5) < 1e-12                # light rain on gravel
    assert abs(o[14]) < 1e-7 and abs(o[15]) < 1e-12    # on the (float32) lane centre, aligned


def test_goal_crash_offroad_events():
    sc, orc, F, I = road_world(1)
    orc.place(F, I, 0, 10.0, -1.8, 0.0, 10.0, 12.0, -1.8)
    prev = F[:, :2].copy()
    ev = orc.events(F, I, prev)["events"][0]
    assert ev & O.EV["goal"]
    # tilt: rotate 90 degrees about x -> body z horizontal -> crash
    sc, orc, F, I = road_world(1)
    orc.place(F, I, 0, 10.0, -1.8, 0.0, 10.0, 80.0, -1.8)
    F[0, O.F_QW:O.F_QZ + 1] = [math.cos(math.pi / 4), math.sin(math.pi / 4), 0, 0]
    assert orc.events(F, I, F[:, :2].copy())["events"][0] & O.EV["crash"]
    # 3.3 m off the lane centre, 1.5 m beyond the edge line -> off-road, no edge overlap
    sc, orc, F, I = road_world(1)
    orc.place(F, I, 0, 10.0, -1.8 - 3.3, 0.0, 10.0, 80.0, -1.8)
    ev = orc.events(F, I, F[:, :2].copy())["events"][0]
    assert ev & O.EV["offroad"] and not ev & O.EV["lane_forbidden"]
    # 0.6 m from the edge line: the 0.99 m circles (+0.05 m half width) overlap it
    sc, orc, F, I = road_world(1)
    orc.place(F, I, 0, 10.0, -3.0, 0.0, 10.0, 80.0, -1.8)
    ev = orc.events(F, I, F[:, :2].copy())["events"][0]
    assert ev & O.EV["lane_forbidden"] and not ev & O.EV["offroad"]
    sc, orc, F, I = road_world(1)
    orc.place(F, I, 0, 10.0, -3.6 + 1.05, 0.0, 10.0, 80.0, -1.8)
    assert not orc.events(F, I, F[:, :2].copy())["events"][0] & O.EV["lane_forbidden"]
    sc, orc, F, I = road_world(1)
    orc.place(F, I, 0, 10.0, -1.8 + 0.7, 0.0, 10.0, 80.0, -1.8)
    ev = orc.events(F, I, F[:, :2].copy())["events"][0]
    assert not ev & (O.EV["offroad"] | O.EV["lane_forbidden"])


def test_collision_warmup_and_reward():
    sc, orc, F, I = road_world(2)
    orc.place(F, I, 0, 0.0, -1.8, 0.0, 0.5, 80.0, -1.8)
    orc.place(F, I, 1, 3.0, -1.8, 0.0, 0.5, 80.0, -1.8)        # overlapping footprints
    out = orc.events(F, I, F[:, :2].copy())
    assert not out["events"][0] & O.EV["collision"]             # step 1 <= 24-step warm-up
    I[:, O.I_STEP] = 30
    out = orc.events(F, I, F[:, :2].copy())
    assert out["events"][0] & O.EV["collision"] and out["events"][1] & O.EV["collision"]
    assert out["reward"][0] < -5.0


def test_ttc_penalty_on_the_minimum_neighbour_ttc():
    """App. G: r_ttc = -p(min over neighbours of TTC), p(tau) = min(0.10 / max(tau, 0.5), 0.35),
    with TTC = tau_max = 10 s for a neighbour behind the ego or on no collision
    course (App. D).  So one harmless neighbour costs exactly 0.10 / 10 = 0.01."""
    def reward_of_agent0(others):
        sc, orc, F, I = road_world(1 + len(others))
        orc.place(F, I, 0, 0.0, -1.8, 0.0, 10.0, 80.0, -1.8)
        for k, (x, y, v) in enumerate(others):
            orc.place(F, I, 1 + k, x, y, 0.0, v, 80.0, y)
        return orc.events(F, I, F[:, :2].copy())["reward"][0]

    alone = reward_of_agent0([])
    # same speed on the other lane, 30 m ahead: no collision course
    assert abs((alone - reward_of_agent0([(30.0, 1.8, 10.0)])) - 0.01) < 1e-12
    # behind the ego, closing: still TTC = tau_max for the ego
    assert abs((alone - reward_of_agent0([(-30.0, -1.8, 20.0)])) - 0.01) < 1e-12
    # stopped 20 m ahead in the same lane: the front circle of the ego (+1.3 m)
    # meets the rear circle of the other (-1.3 m) when their gap 17.4 m has
    # shrunk to 2 r = 1.98 m, at 10 m/s: tau = 1.542 s
    tau = (20.0 - 2 * 1.3 - 2 * 0.99) / 10.0
    closing = reward_of_agent0([(20.0, -1.8, 0.0)])
    assert abs((alone - closing) - 0.10 / tau) < 1e-12
    # the minimum over the neighbours decides, not the sum
    both = reward_of_agent0([(30.0, 1.8, 10.0), (20.0, -1.8, 0.0)])
    assert abs((alone - both) - 0.10 / tau) < 1e-12
    # 5.5 m ahead (footprints 1 m apart), closing at 10 m/s: tau = (2.9 - 1.98) / 10
    # = 0.092 s is floored at 0.5 s, p = 0.10 / 0.5 = 0.2 (below the 0.35 cap);
    # DRAC = 10^2 / (2 * 1.0) = 50 m/s^2 adds 0.01 * (50 - 3.4)
    near = reward_of_agent0([(5.5, -1.8, 0.0)])
    assert abs((alone - near) - (0.2 + 0.01 * (50.0 - 3.4))) < 1e-12


def test_progress_reward_sign():
    sc, orc, F, I = road_world(1)
    orc.place(F, I, 0, 0.0, -1.8, 0.0, 10.0, 80.0, -1.8)
    prev = F[:, :2].copy() - np.array([[0.5, 0.0]])             # moved +0.5 m toward the goal
    r1 = orc.events(F, I, prev)["reward"][0]
    prev = F[:, :2].copy() + np.array([[0.5, 0.0]])
    r2 = orc.events(F, I, prev)["reward"][0]
    assert abs((r1 - r2) - 2.0 * 1.0) < 1e-12


# ----------------------------------------------------------------------------- resets
def test_reset_spawn_rules():
    sc = synth.procedural_scene(4, 16, seed_base=70)
    orc = O.Oracle(sc)
    F, I = orc.empty_state()
    I[:, O.I_PRECIP], I[:, O.I_SURFACE] = sc.precip, sc.surface
    F2, I2 = F.copy(), I.copy()
    orc.reset(F, I, np.ones(sc.num_agents, np.uint8), seed=123)
    orc.reset(F2, I2, np.ones(sc.num_agents, np.uint8), seed=123)
    assert np.array_equal(F, F2) and np.array_equal(I, I2)       # deterministic
    z_star = 0.25 + 0.33 + 0.3 - 1500 * 9.81 / (4 * 35000)
    assert np.allclose(F[:, O.F_PZ], z_star)
    sp = np.hypot(F[:, O.F_VX], F[:, O.F_VY])
    assert (sp >= 5.0).all() and (sp <= 20.0).all()
    assert np.allclose(F[:, O.F_S0], sp / 0.33)
    assert (I[:, O.I_STATUS] == O.ALIVE).all() and (I[:, O.I_EPISODE] == 1).all()
    lanes = set()
    for w in range(sc.num_worlds):
        for p in range(sc.poly_off[w], sc.poly_off[w + 1]):
            if sc.poly_type[p] in (1, 2):
                lanes.update((float(x), float(y)) for x, y in zip(sc.px[sc.point_off[p]:sc.point_off[p + 1]],
                                                                  sc.py[sc.point_off[p]:sc.point_off[p + 1]]))
        a0, a1 = sc.agent_off[w], sc.agent_off[w + 1]
        for a in range(a0, a1):
            assert (float(F[a, 0]), float(F[a, 1])) in lanes
            assert (float(F[a, O.F_GX]), float(F[a, O.F_GY])) in lanes
            g = math.hypot(F[a, O.F_GX] - F[a, 0], F[a, O.F_GY] - F[a, 1])
            assert 3.0 < g <= 150.0 + 1e-9
        d = np.hypot(*(F[a0:a1, None, :2] - F[None, a0:a1, :2]).transpose(2, 0, 1))
        d[np.eye(a1 - a0, dtype=bool)] = np.inf
        assert (d.min() >= 10.0 - 1e-9) or (d.min() > 0)
    P = O.default_params()
    for a in range(sc.num_agents):
        assert F[a, O.F_MU] == P.mu_table[int(sc.precip[a])][int(sc.surface[a])]
    assert len(set(F[:, O.F_MU])) > 3


def test_friction_table_anchors():
    P = O.default_params()
    tab = np.array([[P.mu_table[i][j] for j in range(3)] for i in range(4)])
    assert tab[0, 0] == 0.9 and tab[2, 0] == 0.5           # dry / heavy-rain asphalt
    assert tab.min() >= 0.2 and tab.max() <= 0.9
    assert (np.diff(tab, axis=0) < 0).all()                 # wetter -> lower friction


def test_auto_reset_and_parking():
    sc, orc, F, I = road_world(1)
    orc.place(F, I, 0, 10.0, -1.8, 0.0, 10.0, 11.0, -1.8)     # goal within reach
    out = orc.step(F, I, np.zeros((1, 3)), flags=0)
    assert out["done"][0] == 1 and I[0, O.I_STATUS] == O.PARKED and F[0, O.F_PX] == 1000.0
    assert not out["obs"][0].any()
    sc, orc, F, I = road_world(1)
    orc.place(F, I, 0, 10.0, -1.8, 0.0, 10.0, 11.0, -1.8)
    out = orc.step(F, I, np.zeros((1, 3)), flags=O.FLAG_AUTO_RESET, seed=4)
    assert out["done"][0] == 1 and I[0, O.I_STATUS] == O.ALIVE and out["events"][0] & O.EV["respawned"]
    assert I[0, O.I_EPISODE] == 1 and I[0, O.I_STEP] == 0
    sc, orc, F, I = road_world(1)
    orc.place(F, I, 0, 10.0, -1.8, 0.0, 10.0, 11.0, -1.8)
    out = orc.step(F, I, np.zeros((1, 3)), flags=O.FLAG_INVINCIBLE)
    assert out["done"][0] == 0 and out["events"][0] & O.EV["goal"]


def test_timeout():
    sc, orc, F, I = road_world(1)
    orc.place(F, I, 0, 0.0, -1.8, 0.0, 0.0, 80.0, -1.8)
    I[0, O.I_STEP] = 1498
    assert orc.step(F, I, np.zeros((1, 3)))["done"][0] == 0
    out = orc.step(F, I, np.zeros((1, 3)))
    assert out["done"][0] == 1 and out["events"][0] & O.EV["timeout"]
