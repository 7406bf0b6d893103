"""Pins of the oracle's full observation (App. D, 1,929 values per agent).

The road group is pinned by a closed-form count on a straight road, by the
350-slot cap and polyline ordering on a dense synthetic map, by the segment gap
rule and by invariance under a rigid motion of the whole world; the neighbour
group by its agreement with the independently written neighbour slots of the
320-value observation (same features, other code path) and by its count.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_08528_b300 import synth

EGO, KR, PT, KV, NB = O.FULL_EGO, O.FULL_KR, O.FULL_PT, O.FULL_KV, O.FULL_NB
R0, V0 = O.FULL_ROAD0, O.FULL_VEH0


def placed(scene, rows):
    orc = O.Oracle(scene)
    F, I = orc.empty_state()
    for a, r in enumerate(rows):
        orc.place(F, I, a, *r)
    return orc, F, I


def test_layout_is_1929():
    assert O.FULL_OBS == 1929 == 11 + 350 * 5 + 24 * 7


def test_straight_road_count_and_features_closed_form():
    # lanes at y = -1.8 (east), +1.8 (west), edges at -3.6, +3.6; points every 1 m,
    # so segment midpoints sit at x = k + 0.5.  An agent at (0.3, -1.8) heading +x
    # sees every midpoint with (x - 0.3)^2 + dy^2 <= 100.
    sc = synth.straight_road(num_agents=1)
    orc, F, I = placed(sc, [(0.3, -1.8, 0.0, 10.0, 50.0, -1.8)])
    out = orc.observe_full(F, I)
    n = int(out["n_road"][0])
    xs = np.arange(-100, 100) + 0.5
    expect = []
    ys = [-1.8, 1.8, -3.6, 3.6]
    for pl, y in enumerate(ys):
        dy = y - (-1.8)
        order = xs if pl != 1 else xs[::-1]           # the westbound lane runs from +100 to -100
        for x in order:
            if (x - 0.3) ** 2 + dy ** 2 <= 100.0:
                expect.append((x, dy, pl))
    assert n == len(expect) == 20 + 19 + 20 + 17      # |x - 0.3| <= sqrt(100 - dy^2) per line
    road = out["obs"][0, R0:R0 + KR * PT].reshape(KR, PT)
    types = [2, 2, 15, 15]
    for t, (x, dy, pl) in enumerate(expect):
        dirx = -1.0 if pl == 1 else 1.0
        np.testing.assert_allclose(road[t], [(x - 0.3) / 10, dy / 10, types[pl] / 20, dirx, 0.0], atol=1e-7)   # float32 road y
    assert not road[n:].any()
    # ego: goal 49.7 m ahead, moving forward at 10 m/s, dry asphalt
    np.testing.assert_allclose(out["obs"][0, :EGO], [0.497, 0, 0, 1, 0.497, 1.0, 0, 0, 1, 0, 0], atol=1e-9)


def dense_scene(spacing=0.5, half=12.0, gap_poly=None):
    """Short parallel polylines every `spacing` m in a square: far more than 350
    segment midpoints lie within 10 m of the centre."""
    polys = []
    ys = np.arange(-half, half + 1e-9, spacing)
    for i, y in enumerate(ys):
        x = np.arange(-half, half + 1e-9, spacing)
        polys.append((2 if i % 3 else 16, np.stack([x, np.full_like(x, y)], 1)))
    if gap_poly is not None:
        polys.append(gap_poly)
    return synth._assemble([polys], [2], [1, 0], [2, 0])


def test_cap_and_polyline_order_on_dense_map():
    sc = dense_scene()
    orc, F, I = placed(sc, [(0.1, 0.2, 0.3, 5.0, 40.0, 0.0), (30.0, 30.0, 0.0, 5.0, 0.0, 0.0)])
    out = orc.observe_full(F, I)
    idx = out["road_idx"][0]
    assert out["n_road"][0] == KR
    assert np.all(np.diff(idx) > 0)                  # ascending segment index = polyline order
    # every segment midpoint within 10 m that is not selected comes after the last selected one
    px, py = sc.px.astype(np.float64), sc.py.astype(np.float64)
    inside = []
    for p in range(len(sc.poly_type)):
        for k in range(sc.point_off[p], sc.point_off[p + 1] - 1):
            mx, my = (px[k] + px[k + 1]) / 2, (py[k] + py[k + 1]) / 2
            if (mx - 0.1) ** 2 + (my - 0.2) ** 2 <= 100:
                inside.append(k)
    assert len(inside) > KR
    assert list(idx) == inside[:KR]
    # agent 1 is 42 m away from every segment: no road context, but it sees agent 0
    assert out["n_road"][1] == 0 and not out["obs"][1, R0:V0].any()
    assert out["n_veh"][1] == 1 and out["veh_idx"][1, 0] == 0


def test_gap_rule_excludes_long_segments():
    gap = (2, np.array([[-2.0, 1.3], [2.0, 1.3], [2.5, 1.3]]))    # 4 m gap, then a 0.5 m segment
    sc = synth._assemble([[gap]], [1], [0], [0])
    orc, F, I = placed(sc, [(0.0, 0.0, 0.0, 5.0, 50.0, 0.0)])
    out = orc.observe_full(F, I)
    assert out["n_road"][0] == 1 and out["road_idx"][0, 0] == 1


@pytest.mark.parametrize("theta,shift", [(0.7, (3.0, -2.0)), (-2.2, (-1.5, 4.0)), (math.pi, (0.0, 0.0))])
def test_rigid_motion_invariance(theta, shift):
    sc = synth.procedural_scene(1, 12, seed_base=1000, weather="uniform")
    orc = O.Oracle(sc)
    F, I = orc.empty_state()
    rng = np.random.default_rng(4)
    orc.reset(F, I, np.ones(12, np.uint8), seed=5)     # agents on lanes
    F[:, O.F_VY] += rng.normal(0, 1, 12)              # some sideslip, so velocities are not along the heading
    base = orc.observe_full(F, I)

    c, s = math.cos(theta), math.sin(theta)
    rot = lambda x, y: (c * x - s * y + shift[0], s * x + c * y + shift[1])
    px, py = rot(sc.px.astype(np.float64), sc.py.astype(np.float64))
    sc2 = synth.Scene(sc.agent_off, sc.poly_off, sc.point_off, sc.poly_type, px, py, sc.precip, sc.surface)
    orc2 = O.Oracle(sc2)
    F2, I2 = F.copy(), I.copy()
    F2[:, 0], F2[:, 1] = rot(F[:, 0], F[:, 1])
    F2[:, O.F_GX], F2[:, O.F_GY] = rot(F[:, O.F_GX], F[:, O.F_GY])
    F2[:, O.F_VX], F2[:, O.F_VY] = c * F[:, O.F_VX] - s * F[:, O.F_VY], s * F[:, O.F_VX] + c * F[:, O.F_VY]
    # attitude: pre-multiply by the yaw rotation about z
    hw, hz = math.cos(theta / 2), math.sin(theta / 2)
    qw, qx, qy, qz = F[:, 3], F[:, 4], F[:, 5], F[:, 6]
    F2[:, 3], F2[:, 4], F2[:, 5], F2[:, 6] = hw * qw - hz * qz, hw * qx - hz * qy, hw * qy + hz * qx, hw * qz + hz * qw
    moved = orc2.observe_full(F2, I2)
    # segments near the corners of the 200 m box may leave it: compare the agents
    # whose 10 m disc stays well inside the box after the motion
    near = np.hypot(F[:, 0], F[:, 1]) < 85.0
    assert near.sum() >= 6 and base["n_road"][near].min() > 0
    assert np.array_equal(base["n_road"][near], moved["n_road"][near])
    assert np.array_equal(base["road_idx"][near], moved["road_idx"][near])
    assert np.array_equal(base["veh_idx"], moved["veh_idx"])
    np.testing.assert_allclose(moved["obs"][near], base["obs"][near], atol=1e-9)
    np.testing.assert_allclose(moved["obs"][:, O.FULL_VEH0:], base["obs"][:, O.FULL_VEH0:], atol=1e-9)


def test_neighbour_group_matches_the_320_value_observation():
    sc = synth.procedural_scene(2, 16, seed_base=1003, weather="uniform")
    orc = O.Oracle(sc)
    F, I = orc.empty_state()
    orc.reset(F, I, np.ones(sc.num_agents, np.uint8), seed=9)
    I[3, O.I_STATUS] = O.PARKED                       # one dead agent: nobody sees it
    full = orc.observe_full(F, I)
    small = orc.observe(F, I)
    for a in range(sc.num_agents):
        if a == 3:
            assert full["n_veh"][a] == 0 and full["n_road"][a] == 0 and not full["obs"][a].any()
            continue
        others = 14 if a < 16 else 15                 # 16 agents a world, minus self (and the parked one)
        assert full["n_veh"][a] == others
        assert 3 not in full["veh_idx"][a]
        np.testing.assert_array_equal(full["veh_idx"][a, :8], small["knn_agents"][a])
        for t in range(8):
            s = small["obs"][a, 16 + 10 * t:16 + 10 * t + 10]
            f = full["obs"][a, V0 + NB * t:V0 + NB * t + NB]
            np.testing.assert_allclose(f, s[[0, 1, 2, 3, 4, 5, 8]], atol=1e-12)
        np.testing.assert_allclose(full["obs"][a, :7], small["obs"][a, :7], atol=1e-12)
        np.testing.assert_allclose(full["obs"][a, 7:11], small["obs"][a, 7:11], atol=1e-12)
        d = np.hypot(*(F[full["veh_idx"][a, :others], :2] - F[a, :2]).T)
        assert np.all(np.diff(d) >= 0)
