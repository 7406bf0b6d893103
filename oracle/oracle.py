"""ctypes wrapper of the FP64 CPU oracle (sf_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this module.  It
shares no code with the CUDA library: it compiles and loads its own C file.

All arrays are float64 / int32 numpy arrays in the oracle's row-per-agent
layout (``NF`` float columns and ``NI`` int columns per agent, see
``sf_oracle.h``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sf_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

NF, NI = 25, 6
F_PX, F_PY, F_PZ, F_QW, F_QX, F_QY, F_QZ = 0, 1, 2, 3, 4, 5, 6
F_VX, F_VY, F_VZ, F_WX, F_WY, F_WZ = 7, 8, 9, 10, 11, 12
F_S0, F_DELTA, F_DDELTA, F_GX, F_GY, F_SX, F_SY, F_MU, F_PEAK_DRAC = 13, 17, 18, 19, 20, 21, 22, 23, 24
I_PRECIP, I_SURFACE, I_STEP, I_EPISODE, I_STATUS, I_EVENTS = range(6)
ALIVE, PARKED = 1, 2
EV = dict(goal=1, collision=2, crash=4, lane_forbidden=8, offroad=16, idle=32, timeout=64,
          nonfinite=128, respawned=256)
FLAG_INVINCIBLE, FLAG_AUTO_RESET, FLAG_BICYCLE = 1, 2, 4
WEATHER_TABLE, WEATHER_ALL = 0, 1
K_AGENTS, L_POINTS, OBS = 8, 32, 320
FULL_EGO, FULL_KR, FULL_PT, FULL_KV, FULL_NB = 11, 350, 5, 24, 7
FULL_OBS = FULL_EGO + FULL_KR * FULL_PT + FULL_KV * FULL_NB   # 1929 (App. D)
FULL_ROAD0, FULL_VEH0 = FULL_EGO, FULL_EGO + FULL_KR * FULL_PT
FULL_RADIUS = 10.0


def build(force: bool = False) -> str:
    """Compile sf_oracle.c with gcc (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "sf_oracle.h"))):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class Params(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "g", "mass", "half_len", "half_wid", "half_hgt")] + [("inertia", C.c_double * 3)] + [
        (n, C.c_double) for n in (
            "hard_x", "hard_y", "hard_z", "wheel_r", "k_susp", "c_susp", "rest_len", "wheel_inertia",
            "steer_inertia", "theta_max", "kp", "kd", "tau_steer_max", "tau_drive", "tau_brk_f",
            "tau_brk_r", "lambda_yaw", "lambda_lat", "u_z_min", "k_contact", "c_contact", "damp_ramp", "wheelbase",
            "goal_radius", "w_goal", "w_collision", "w_crash", "w_lane_forb", "w_progress",
            "progress_clip", "w_lane", "lane_sigma", "lane_wh", "w_offroad", "offroad_lat",
            "offroad_dist", "w_idle", "idle_speed", "ttc_alpha_v", "ttc_pmax_v", "ttc_floor",
            "ttc_max", "ttc_alpha_e", "ttc_pmax_e", "edge_horizon", "drac_thresh", "w_drac",
            "drac_gap_floor", "drift_max", "tilt_gz", "seg_gap_max", "scene_half",
            "edge_half_width")] + [("warmup_steps", C.c_int), ("max_steps", C.c_int)] + [
        (n, C.c_double) for n in (
            "spawn_goal_min", "spawn_goal_max", "spawn_v_min", "spawn_v_max", "spawn_spacing",
            "park_x")] + [("spawn_tries", C.c_int), ("mu_table", (C.c_double * 3) * 4)] + [
        (n, C.c_double) for n in ("bike_theta_max", "bike_a_drive", "bike_a_brake")] + [
        ("weather_model", C.c_int), ("all_mu", (C.c_double * 9) * 3), ("all_h_cut", C.c_double),
        ("all_floor", C.c_double), ("all_theta", C.c_double * 3), ("all_td", C.c_double * 3),
        ("h_norm", C.c_double), ("stribeck_b", C.c_double * 4)]


class _Scene(C.Structure):
    _fields_ = [("num_worlds", C.c_int), ("agent_off", C.c_void_p), ("poly_off", C.c_void_p),
                ("point_off", C.c_void_p), ("poly_type", C.c_void_p), ("px", C.c_void_p),
                ("py", C.c_void_p)]


class _Out(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in (
        "obs", "reward", "done", "events", "lane_seg", "knn_pts", "knn_agents", "drac")]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        vp, d, i, u64 = C.c_void_p, C.c_double, C.c_int, C.c_uint64
        L.or_default_params.argtypes = [vp]
        L.or_splitmix64.argtypes = [u64]
        L.or_splitmix64.restype = u64
        L.or_substep_world.argtypes = [vp, vp, i, vp, vp, vp, d]
        L.or_step.argtypes = [vp, vp, vp, vp, vp, d, i, u64, i, vp]
        L.or_step.restype = i
        L.or_events.argtypes = [vp, vp, vp, vp, vp, i, vp]
        L.or_observe.argtypes = [vp, vp, vp, vp, vp]
        L.or_observe_full.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.or_reset.argtypes = [vp, vp, vp, vp, vp, u64, vp]
        L.or_place_agent.argtypes = [vp, vp, vp, i, d, d, d, d, d, d, i, i]
        L.or_bicycle_agent.argtypes = [vp, vp, vp, d]
        L.or_sat.argtypes = [vp, vp, vp, vp, vp, vp]
        L.or_sat.restype = d
        L.or_nearest_lane.argtypes = [vp, vp, i, vp, vp, vp, vp]
        L.or_nearest_lane.restype = i
        L.or_ttc.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.or_ttc.restype = d
        L.or_drac.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.or_drac.restype = d
        L.or_lane_keep_q.argtypes = [vp, d, d]
        L.or_lane_keep_q.restype = d
        L.or_ttc_circles.argtypes = [d, d, d, vp, vp]
        L.or_penalty.argtypes = [d, d, d, d]
        L.or_penalty.restype = d
        L.or_all_mu_static.argtypes = [vp, i, i]
        L.or_all_mu_static.restype = d
        L.or_stribeck_vs.argtypes = [vp, d]
        L.or_stribeck_vs.restype = d
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data if a is not None else None


def default_params() -> Params:
    P = Params()
    lib().or_default_params(C.byref(P))
    return P


def splitmix64(x: int) -> int:
    return int(lib().or_splitmix64(C.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


class Oracle:
    """Holds one scene (float64 copies of the roads) and calls the C oracle on it."""

    def __init__(self, scene, params: Params | None = None):
        self.P = params if params is not None else default_params()
        self.agent_off = np.ascontiguousarray(scene.agent_off, dtype=np.int32)
        self.poly_off = np.ascontiguousarray(scene.poly_off, dtype=np.int32)
        self.point_off = np.ascontiguousarray(scene.point_off, dtype=np.int32)
        self.poly_type = np.ascontiguousarray(scene.poly_type, dtype=np.int32)
        self.px = np.ascontiguousarray(scene.px, dtype=np.float64)
        self.py = np.ascontiguousarray(scene.py, dtype=np.float64)
        self.W = len(self.agent_off) - 1
        self.A = int(self.agent_off[-1])
        self.S = _Scene(self.W, _p(self.agent_off), _p(self.poly_off), _p(self.point_off),
                        _p(self.poly_type), _p(self.px), _p(self.py))

    # -- state helpers ------------------------------------------------------------
    def empty_state(self):
        return np.zeros((self.A, NF), np.float64), np.zeros((self.A, NI), np.int32)

    def _outs(self, want_obs=True):
        A = self.A
        o = dict(obs=np.zeros((A, OBS)) if want_obs else None, reward=np.zeros(A), done=np.zeros(A, np.uint8),
                 events=np.zeros(A, np.uint32), lane_seg=np.zeros(A, np.int32),
                 knn_pts=np.zeros((A, L_POINTS), np.int32), knn_agents=np.zeros((A, K_AGENTS), np.int32),
                 drac=np.zeros(A))
        s = _Out(*[_p(o[k]) for k in ("obs", "reward", "done", "events", "lane_seg", "knn_pts",
                                        "knn_agents", "drac")])
        return o, s

    @staticmethod
    def _chk(F, I):
        assert F.dtype == np.float64 and F.flags.c_contiguous and F.shape[1] == NF
        assert I.dtype == np.int32 and I.flags.c_contiguous and I.shape[1] == NI

    # -- method calls ---------------------------------------------------------------
    def step(self, F, I, actions, dt=1.0 / 30.0, substeps=4, seed=0, flags=0, want_obs=True):
        self._chk(F, I)
        act = np.ascontiguousarray(actions, dtype=np.float64)
        o, s = self._outs(want_obs)
        bad = lib().or_step(C.byref(self.P), C.byref(self.S), _p(F), _p(I), _p(act), float(dt), int(substeps),
                            C.c_uint64(seed), int(flags), C.byref(s))
        o["nonfinite"] = bad
        return o

    def substep_world(self, w, F, I, actions, h):
        self._chk(F, I)
        act = np.ascontiguousarray(actions, dtype=np.float64)
        lib().or_substep_world(C.byref(self.P), C.byref(self.S), int(w), _p(F), _p(I), _p(act), float(h))

    def events(self, F, I, prev_xy, flags=0):
        self._chk(F, I)
        prev = np.ascontiguousarray(prev_xy, dtype=np.float64)
        o, s = self._outs(False)
        lib().or_events(C.byref(self.P), C.byref(self.S), _p(F), _p(I), _p(prev), int(flags), C.byref(s))
        return o

    def observe(self, F, I):
        self._chk(F, I)
        o, s = self._outs(True)
        lib().or_observe(C.byref(self.P), C.byref(self.S), _p(F), _p(I), C.byref(s))
        return o

    def observe_full(self, F, I):
        """The paper's 1,929-value observation of every agent (App. D) with the
        filled-slot counts and the selected segment / agent indices."""
        self._chk(F, I)
        A = self.A
        o = dict(obs=np.zeros((A, FULL_OBS)), n_road=np.zeros(A, np.int32), n_veh=np.zeros(A, np.int32),
                 road_idx=np.zeros((A, FULL_KR), np.int32), veh_idx=np.zeros((A, FULL_KV), np.int32))
        lib().or_observe_full(C.byref(self.P), C.byref(self.S), _p(F), _p(I), _p(o["obs"]), _p(o["n_road"]),
                              _p(o["n_veh"]), _p(o["road_idx"]), _p(o["veh_idx"]))
        return o

    def reset(self, F, I, mask, seed=0):
        self._chk(F, I)
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        o, s = self._outs(True)
        lib().or_reset(C.byref(self.P), C.byref(self.S), _p(F), _p(I), _p(m), C.c_uint64(seed), C.byref(s))
        return o

    def place(self, F, I, a, x, y, psi, v0, gx, gy, precip=0, surface=0):
        lib().or_place_agent(C.byref(self.P), _p(F), _p(I), int(a), float(x), float(y), float(psi), float(v0),
                             float(gx), float(gy), int(precip), int(surface))

    def nearest_lane(self, w, q):
        qq = np.asarray(q, np.float64)
        dist, lat = C.c_double(), C.c_double()
        tan = np.zeros(2)
        k = lib().or_nearest_lane(C.byref(self.P), C.byref(self.S), int(w), _p(qq), C.byref(dist),
                                  C.byref(lat), _p(tan))
        return k, dist.value, lat.value, tan


def bicycle_agent(f_row, action, dt=1.0 / 30.0, params=None):
    """One kinematic-bicycle control step of one state row (modified in place)."""
    P = params or default_params()
    assert f_row.dtype == np.float64 and f_row.flags.c_contiguous and f_row.shape == (NF,)
    act = np.ascontiguousarray(action, dtype=np.float64)
    lib().or_bicycle_agent(C.byref(P), _p(f_row), _p(act), float(dt))


# -- free functions on the pair geometry ---------------------------------------------------
def sat(ci, hi, cj, hj, params=None):
    P = params or default_params()
    a = [np.asarray(x, np.float64) for x in (ci, hi, cj, hj)]
    n = np.zeros(2)
    d = lib().or_sat(C.byref(P), *[_p(x) for x in a], _p(n))
    return d, n


def ttc(pi, hi, vi, pj, hj, vj, params=None):
    P = params or default_params()
    a = [np.asarray(x, np.float64) for x in (pi, hi, vi, pj, hj, vj)]
    return lib().or_ttc(C.byref(P), *[_p(x) for x in a])


def drac(pi, vi, pj, vj, hi=(1.0, 0.0), hj=(1.0, 0.0), params=None):
    P = params or default_params()
    a = [np.asarray(x, np.float64) for x in (pi, hi, vi, pj, hj, vj)]
    return lib().or_drac(C.byref(P), *[_p(x) for x in a])


def lane_keep_q(lateral, cos_dpsi, params=None):
    P = params or default_params()
    return lib().or_lane_keep_q(C.byref(P), float(lateral), float(cos_dpsi))


def ttc_circles(L, W, WB):
    r, d = C.c_double(), C.c_double()
    lib().or_ttc_circles(float(L), float(W), float(WB), C.byref(r), C.byref(d))
    return r.value, d.value


def penalty(alpha, tau, tau_floor, pmax):
    return lib().or_penalty(float(alpha), float(tau), float(tau_floor), float(pmax))


def all_mu_static(surface, film_cmm, params=None):
    """Static friction of the modified ALL model (App. B) of surface 0 AC,
    1 SMA, 2 OGFC at a water film of film_cmm hundredths of a millimetre."""
    P = params or default_params()
    return lib().or_all_mu_static(C.byref(P), int(surface), int(film_cmm))


def stribeck_vs(h_m, params=None):
    """Stribeck speed [m/s] at a water film of h_m metres (Eq. app_stribeck_speed)."""
    P = params or default_params()
    return lib().or_stribeck_vs(C.byref(P), float(h_m))
