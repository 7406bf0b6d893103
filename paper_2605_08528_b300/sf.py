"""Thin ctypes binding of the C-ABI in include/sf.h (argument marshalling only).

Every computation of the vehicle step runs in the CUDA kernels of libsf.so;
this module only converts Python / numpy / torch arguments into the pointers
and sizes the C functions take.  It never falls back to a CPU path: if the
library is missing or no CUDA device is usable, the calls raise.

The function names are those of the C-ABI (sf_create, sf_load_roads, sf_step,
sf_get_obs, sf_reset, ...).  ``World`` bundles a handle with its roads for
convenience.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsf.so")

SF_OK, SF_ERR_INVALID_ARG, SF_ERR_CUDA, SF_ERR_OOM, SF_ERR_NONFINITE, SF_ERR_TIMEOUT, SF_ERR_STATE = range(7)
STATUS_NAMES = {0: "SF_OK", 1: "SF_ERR_INVALID_ARG", 2: "SF_ERR_CUDA", 3: "SF_ERR_OOM", 4: "SF_ERR_NONFINITE",
                5: "SF_ERR_TIMEOUT", 6: "SF_ERR_STATE"}
NF, NI, OBS_DIM, K_AGENTS, L_POINTS = 25, 6, 320, 8, 32
FULL_EGO, FULL_KR, FULL_PT, FULL_KV, FULL_NB = 11, 350, 5, 24, 7
FULL_OBS_DIM = FULL_EGO + FULL_KR * FULL_PT + FULL_KV * FULL_NB   # 1929
FLAG_INVINCIBLE, FLAG_AUTO_RESET, FLAG_RECORD_INDICES, FLAG_METRICS = 1, 2, 4, 8
DYN_VEHICLE, DYN_BICYCLE = 0, 1
WEATHER_TABLE, WEATHER_ALL = 0, 1
ACT_NONE, ACT_ELU, ACT_SILU, ACT_TANH = 0, 1, 2, 3


class SFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class sf_metrics(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("episodes", "goals", "collisions", "crashes", "offroad", "lane_forbidden",
                                          "idle", "timeouts", "nonfinite", "drac_over")] + \
               [(n, C.c_double) for n in ("success_rate", "collision_rate", "mean_episode_max_drac", "drac_over_rate")]


class sf_config(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("flags", C.c_int32), ("warps_per_block", C.c_int32),
                ("pack_agents", C.c_int32), ("stage_bytes", C.c_int32), ("split_step", C.c_int32),
                ("dynamics", C.c_int32), ("world_begin", C.c_int32), ("world_end", C.c_int32),
                ("weather_model", C.c_int32), ("reserved", C.c_int32 * 1)]


class sf_roads(C.Structure):
    _fields_ = [("num_worlds", C.c_int32), ("num_polylines", C.c_int32), ("num_points", C.c_int32),
                ("agent_off", C.c_void_p), ("poly_off", C.c_void_p), ("point_off", C.c_void_p),
                ("poly_type", C.c_void_p), ("px", C.c_void_p), ("py", C.c_void_p), ("precip", C.c_void_p),
                ("surface", C.c_void_p), ("film_mm", C.c_void_p)]


class sf_outputs(C.Structure):
    _fields_ = [("obs", C.c_void_p), ("reward", C.c_void_p), ("done", C.c_void_p), ("events", C.c_void_p),
                ("lane_seg", C.c_void_p), ("knn_points", C.c_void_p), ("knn_agents", C.c_void_p),
                ("drac", C.c_void_p), ("num_agents", C.c_int32)]


_lib = None


def lib():
    """Load libsf.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsf.so is missing: build it with `python -m paper_2605_08528_b300.build`")
        L = C.CDLL(LIB_PATH)
        vp, i32, f32 = C.c_void_p, C.c_int32, C.c_float
        sig = {
            "sf_create": ([vp, vp, vp], i32), "sf_destroy": ([vp], i32), "sf_load_roads": ([vp, vp], i32),
            "sf_step": ([vp, vp, f32, C.c_int], i32), "sf_get_obs": ([vp, vp, vp, vp, vp], i32),
            "sf_step_host": ([vp, vp, vp, vp, f32, C.c_int], i32),
            "sf_step_host_obs": ([vp, vp, vp, vp, vp, f32, C.c_int], i32),
            "sf_fp32_fma_peak": ([vp, C.c_int, C.POINTER(C.c_double)], i32),
            "sf_output_ptrs": ([vp, vp], i32), "sf_observe_full": ([vp, vp, vp, vp, vp, vp], i32), "sf_get_indices": ([vp, vp, vp, vp, vp], i32),
            "sf_get_metrics": ([vp, vp], i32), "sf_reset_metrics": ([vp], i32), "sf_reset": ([vp, vp], i32), "sf_place_agents": ([vp, vp], i32),
            "sf_get_state": ([vp, vp, vp], i32), "sf_set_state": ([vp, vp, vp], i32),
            "sf_save_state": ([vp, C.c_char_p], i32), "sf_load_state": ([vp, C.c_char_p], i32),
            "sf_sync": ([vp], i32), "sf_set_wait_limit": ([vp, C.c_ulonglong, C.c_int], i32),
            "sf_mlp_set_wait_limit": ([vp, C.c_ulonglong, C.c_int], i32), "sf_autotune": ([vp, vp, f32, C.c_int, C.c_int, vp, vp], i32), "sf_num_agents": ([vp], i32), "sf_num_worlds": ([vp], i32),
            "sf_last_error": ([vp], C.c_char_p), "sf_version": ([], C.c_char_p),
            "sf_mlp_create": ([C.c_int, vp, C.c_int, C.c_int, vp, vp], i32), "sf_mlp_destroy": ([vp], i32),
            "sf_mlp_last_error": ([vp], C.c_char_p), "sf_mlp_set_layer": ([vp, C.c_int, vp, vp], i32),
            "sf_mlp_get_layer": ([vp, C.c_int, vp, vp, vp, vp], i32),
            "sf_mlp_forward": ([vp, vp, C.c_int, C.c_int, vp, C.c_int], i32),
            "sf_mlp_train_step": ([vp, vp, vp, C.c_int, f32, C.c_int, vp], i32), "sf_mlp_sync": ([vp], i32),
            "sf_mlp_forward_static": ([vp, vp, C.c_int, C.c_int, vp, C.c_int], i32),
            "sf_mlp_static_scratch_bytes": ([], C.c_size_t),
            "sf_gemm_bf16": ([vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp, C.c_int, C.c_int,
                              C.c_int, vp, vp], i32),
            "sf_step_policy": ([vp, vp, f32, C.c_int], i32),
            "sf_graph_capture": ([vp, vp, vp, vp, vp, f32, C.c_int, vp], i32), "sf_graph_launch": ([vp], i32),
            "sf_graph_destroy": ([vp], i32),
            "sf_surrogate_create": ([vp, vp], i32), "sf_surrogate_destroy": ([vp], i32),
            "sf_surrogate_collect": ([vp, vp, vp, f32, C.c_int, vp, vp, C.c_uint64, vp], i32),
            "sf_surrogate_train": ([vp, vp, vp, C.c_uint64, C.c_int, C.c_int, f32, C.c_uint64, vp], i32),
            "sf_surrogate_mlp": ([vp], vp), "sf_surrogate_stats": ([vp, vp], i32),
            "sf_surrogate_set_stats": ([vp, vp], i32),
            "sf_step_surrogate": ([vp, vp, vp, f32, C.c_int, C.c_int], i32),
            "sf_surrogate_audit": ([vp, vp, vp], i32),
            "sf_lf_num_params": ([], C.c_size_t), "sf_lf_create": ([vp, vp], i32), "sf_lf_destroy": ([vp], i32),
            "sf_lf_last_error": ([vp], C.c_char_p), "sf_lf_set_params": ([vp, vp, C.c_size_t], i32),
            "sf_lf_get_params": ([vp, vp, C.c_size_t], i32),
            "sf_lf_forward": ([vp, vp, vp, vp, C.c_int, vp, vp, vp], i32), "sf_lf_sync": ([vp], i32),
            "sf_step_lf": ([vp, vp, f32, C.c_int], i32), "sf_lf_step_outputs": ([vp, vp], i32),
            "sf_graph_capture_lf": ([vp, vp, vp, f32, C.c_int, vp], i32),
            "sf_ppo_default_config": ([vp], None), "sf_ppo_create": ([vp, vp, vp, vp, vp], i32),
            "sf_ppo_destroy": ([vp], i32), "sf_ppo_last_error": ([vp], C.c_char_p), "sf_ppo_collect": ([vp], i32),
            "sf_ppo_update": ([vp, vp], i32), "sf_ppo_log_std": ([vp, vp], i32),
            "sf_ppo_rollout_ptrs": ([vp, vp], i32),
            "sf_ppo_loss_grads": ([vp, vp, vp, C.c_int, vp, vp, vp, vp, vp], i32),
            "sf_ppo_create_lf": ([vp, vp, vp, vp], i32),
            "sf_ppo_lf_grads": ([vp, vp, vp, vp, C.c_int, vp, vp, vp, vp, vp, vp, C.c_size_t], i32),
            "sf_ppo_lf_params": ([vp, vp, C.c_size_t], i32),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(status, h=None, allow=()):
    if status != SF_OK and status not in allow:
        raise SFError(status, lib().sf_last_error(h).decode())
    return status


def _ptr(x):
    """Device or host pointer of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


# --------------------------------------------------------------------------- C-ABI names
def sf_version() -> str:
    return lib().sf_version().decode()


def sf_create(seed=0, flags=0, warps_per_block=0, stream=None, pack_agents=0, stage_bytes=0, split_step=0,
              dynamics=DYN_VEHICLE, world_range=(0, 0), weather_model=WEATHER_TABLE):
    cfg = sf_config(seed, flags, warps_per_block, pack_agents, stage_bytes, split_step, dynamics,
                    int(world_range[0]), int(world_range[1]), int(weather_model))
    h = C.c_void_p()
    st = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(lib().sf_create(C.byref(cfg), C.c_void_p(st), C.byref(h)))
    return h


def sf_destroy(h):
    _check(lib().sf_destroy(h), h)


def sf_load_roads(h, scene):
    arrs = dict(agent_off=np.ascontiguousarray(scene.agent_off, np.int32),
                poly_off=np.ascontiguousarray(scene.poly_off, np.int32),
                point_off=np.ascontiguousarray(scene.point_off, np.int32),
                poly_type=np.ascontiguousarray(scene.poly_type, np.uint8),
                px=np.ascontiguousarray(scene.px, np.float32), py=np.ascontiguousarray(scene.py, np.float32),
                precip=np.ascontiguousarray(scene.precip, np.uint8),
                surface=np.ascontiguousarray(scene.surface, np.uint8))
    film = getattr(scene, "film_mm", None)
    arrs["film_mm"] = None if film is None else np.ascontiguousarray(film, np.float32)
    r = sf_roads(len(arrs["agent_off"]) - 1, len(arrs["poly_type"]), len(arrs["px"]),
                 *[_ptr(arrs[k]) for k in ("agent_off", "poly_off", "point_off", "poly_type", "px", "py", "precip",
                                           "surface", "film_mm")])
    _check(lib().sf_load_roads(h, C.byref(r)), h)


def sf_step(h, d_actions, dt=1.0 / 30.0, substeps=4):
    _check(lib().sf_step(h, _ptr(d_actions), float(dt), int(substeps)), h)


def sf_step_host(h, h_actions, h_reward, h_done, dt=1.0 / 30.0, substeps=4):
    """One step end to end from host buffers (numpy arrays or CPU tensors,
    page-locked for the captured-graph path): actions in, rewards and done
    flags out; returns when they are in host memory."""
    _check(lib().sf_step_host(h, _ptr(h_actions), _ptr(h_reward), _ptr(h_done), float(dt), int(substeps)), h)


def sf_step_host_obs(h, h_actions, h_obs, h_reward, h_done, dt=1.0 / 30.0, substeps=4):
    """sf_step_host that also copies the step's observations [A][320] into h_obs."""
    _check(lib().sf_step_host_obs(h, _ptr(h_actions), _ptr(h_obs), _ptr(h_reward), _ptr(h_done), float(dt),
                                  int(substeps)), h)


def sf_fp32_fma_peak(stream=None, iters=20000):
    """Measured FP32 FMA throughput of the device in TFLOP/s."""
    out = C.c_double(0.0)
    st = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    s = lib().sf_fp32_fma_peak(st or None, int(iters), C.byref(out))
    if s != SF_OK:
        raise SFError(s, "sf_fp32_fma_peak")
    return out.value


def sf_get_obs(h, d_obs=None, d_reward=None, d_done=None, d_events=None):
    _check(lib().sf_get_obs(h, _ptr(d_obs), _ptr(d_reward), _ptr(d_done), _ptr(d_events)), h)


def sf_get_metrics(h):
    """The episode metrics of a handle created with FLAG_METRICS, as a dict."""
    m = sf_metrics()
    _check(lib().sf_get_metrics(h, C.byref(m)), h)
    return {n: getattr(m, n) for n, _ in sf_metrics._fields_}


def sf_reset_metrics(h):
    _check(lib().sf_reset_metrics(h), h)


def sf_get_indices(h, d_lane_seg=None, d_knn_points=None, d_knn_agents=None, d_drac=None):
    _check(lib().sf_get_indices(h, _ptr(d_lane_seg), _ptr(d_knn_points), _ptr(d_knn_agents), _ptr(d_drac)), h)


def sf_observe_full(h, d_obs, d_n_road=None, d_n_veh=None, d_road_idx=None, d_veh_idx=None):
    _check(lib().sf_observe_full(h, _ptr(d_obs), _ptr(d_n_road), _ptr(d_n_veh), _ptr(d_road_idx), _ptr(d_veh_idx)),
           h)


def sf_output_ptrs(h) -> sf_outputs:
    o = sf_outputs()
    _check(lib().sf_output_ptrs(h, C.byref(o)), h)
    return o


def sf_reset(h, d_mask):
    _check(lib().sf_reset(h, _ptr(d_mask)), h)


def sf_place_agents(h, place):
    p = np.ascontiguousarray(place, np.float32)
    _check(lib().sf_place_agents(h, _ptr(p)), h)


def sf_get_state(h, allow_nonfinite=True):
    A = lib().sf_num_agents(h)
    F = np.zeros((A, NF), np.float32)
    I = np.zeros((A, NI), np.int32)
    s = _check(lib().sf_get_state(h, _ptr(F), _ptr(I)), h, allow=(SF_ERR_NONFINITE,) if allow_nonfinite else ())
    return F, I, s


def sf_set_state(h, F, I):
    F = np.ascontiguousarray(F, np.float32)
    I = np.ascontiguousarray(I, np.int32)
    _check(lib().sf_set_state(h, _ptr(F), _ptr(I)), h)


def sf_save_state(h, path):
    _check(lib().sf_save_state(h, path.encode()), h, allow=(SF_ERR_NONFINITE,))


def sf_load_state(h, path):
    _check(lib().sf_load_state(h, path.encode()), h)


def sf_sync(h, allow=()):
    return _check(lib().sf_sync(h), h, allow=allow)


def sf_set_wait_limit(h, limit_ns=1_000_000_000, withhold_producer=False):
    """Limit of the step kernels' bounded staging wait (and the test switch that issues no copy)."""
    _check(lib().sf_set_wait_limit(h, int(limit_ns), int(bool(withhold_producer))), h)


def sf_mlp_set_wait_limit(m, limit_ns=1_000_000_000, withhold_producer=False):
    """Limit of the MLP GEMMs' bounded operand waits (and the test switch that issues no load)."""
    _mcheck(lib().sf_mlp_set_wait_limit(m, int(limit_ns), int(bool(withhold_producer))), m)


AUTOTUNE_SHAPES = 38


def sf_autotune(h, d_actions, dt=1.0 / 30.0, substeps=4, iters=20):
    """Pick the fastest launch shape of the step; returns ((warps per block, pack agents,
    stage bytes, split step), ms per shape: s < 32 the fused kernel with 1 << (s & 3) warps,
    packed if s & 4, staging budget s >> 3; s = 32 + k the split step with 2 << (k % 3)
    warps per query block, packed if k >= 3)."""
    best = (C.c_int32 * 4)()
    ms = (C.c_float * AUTOTUNE_SHAPES)()
    _check(lib().sf_autotune(h, _ptr(d_actions), float(dt), int(substeps), int(iters), best, ms), h)
    return (int(best[0]), int(best[1]), int(best[2]), int(best[3])), list(ms)


def sf_num_agents(h) -> int:
    return int(lib().sf_num_agents(h))


def sf_num_worlds(h) -> int:
    return int(lib().sf_num_worlds(h))


# --------------------------------------------------------------------------- convenience
class World:
    """A handle plus its roads, with torch views of the library-owned outputs."""

    def __init__(self, scene, seed=0, flags=0, warps_per_block=0, stream=None, pack_agents=0, stage_bytes=0,
                 split_step=0, dynamics=DYN_VEHICLE, world_range=(0, 0), weather_model=WEATHER_TABLE):
        import torch
        self.torch = torch
        self.scene = scene
        self.h = sf_create(seed, flags, warps_per_block, stream, pack_agents, stage_bytes, split_step, dynamics,
                           world_range, weather_model)
        sf_load_roads(self.h, scene)
        self.A = sf_num_agents(self.h)
        self.W = sf_num_worlds(self.h)

    def close(self):
        if self.h is not None:
            sf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def outputs(self):
        """Copies (torch, on the device) of the last outputs."""
        t = self.torch
        dev = t.device("cuda")
        obs = t.empty((self.A, OBS_DIM), dtype=t.float32, device=dev)
        rew = t.empty(self.A, dtype=t.float32, device=dev)
        done = t.empty(self.A, dtype=t.uint8, device=dev)
        ev = t.empty(self.A, dtype=t.int32, device=dev)
        sf_get_obs(self.h, obs, rew, done, ev)
        return obs, rew, done, ev

    def full_obs(self):
        """Host copies of the paper's full observation (sf_observe_full) of the
        current state: obs [A][1929], n_road, n_veh [A], road_idx [A][350],
        veh_idx [A][24]."""
        t = self.torch
        obs = t.empty((self.A, FULL_OBS_DIM), dtype=t.float32, device="cuda")
        nr = t.empty(self.A, dtype=t.int32, device="cuda")
        nv = t.empty(self.A, dtype=t.int32, device="cuda")
        ri = t.empty((self.A, FULL_KR), dtype=t.int32, device="cuda")
        vi = t.empty((self.A, FULL_KV), dtype=t.int32, device="cuda")
        sf_observe_full(self.h, obs, nr, nv, ri, vi)
        sf_sync(self.h, allow=(SF_ERR_NONFINITE,))
        return dict(obs=obs.cpu().numpy(), n_road=nr.cpu().numpy(), n_veh=nv.cpu().numpy(),
                    road_idx=ri.cpu().numpy(), veh_idx=vi.cpu().numpy())

    def indices(self):
        """Host copies of the recorded nearest-lane / k-NN indices (SF_FLAG_RECORD_INDICES) and step DRAC."""
        t = self.torch
        lane = t.empty(self.A, dtype=t.int32, device="cuda")
        pts = t.empty((self.A, L_POINTS), dtype=t.int32, device="cuda")
        nbr = t.empty((self.A, K_AGENTS), dtype=t.int32, device="cuda")
        drac = t.empty(self.A, dtype=t.float32, device="cuda")
        sf_get_indices(self.h, lane, pts, nbr, drac)
        sf_sync(self.h, allow=(SF_ERR_NONFINITE,))
        return dict(lane_seg=lane.cpu().numpy(), knn_pts=pts.cpu().numpy(), knn_agents=nbr.cpu().numpy(),
                    drac=drac.cpu().numpy())


# --------------------------------------------------------------------------- MLPs
def _mcheck(status, m):
    if status != SF_OK:
        raise SFError(status, lib().sf_mlp_last_error(m).decode() if m else "")
    return status


def sf_mlp_create(dims, hidden_act, out_act, stream=None):
    d = (C.c_int32 * len(dims))(*dims)
    h = C.c_void_p()
    st = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _mcheck(lib().sf_mlp_create(len(dims) - 1, d, int(hidden_act), int(out_act), C.c_void_p(st), C.byref(h)), None)
    return h


def sf_mlp_destroy(m):
    _mcheck(lib().sf_mlp_destroy(m), None)


def sf_mlp_set_layer(m, layer, w, b):
    w = np.ascontiguousarray(w, np.float32)
    b = np.ascontiguousarray(b, np.float32)
    _mcheck(lib().sf_mlp_set_layer(m, int(layer), _ptr(w), _ptr(b)), m)


def sf_mlp_get_layer(m, layer, out_dim, in_dim):
    w = np.zeros((out_dim, in_dim), np.float32)
    b = np.zeros(out_dim, np.float32)
    gw = np.zeros((out_dim, in_dim), np.float32)
    gb = np.zeros(out_dim, np.float32)
    _mcheck(lib().sf_mlp_get_layer(m, int(layer), _ptr(w), _ptr(b), _ptr(gw), _ptr(gb)), m)
    return w, b, gw, gb


def sf_mlp_forward(m, d_x, batch, d_y, ldx=None, ldy=None):
    ldx = d_x.shape[-1] if ldx is None else ldx
    ldy = d_y.shape[-1] if ldy is None else ldy
    _mcheck(lib().sf_mlp_forward(m, _ptr(d_x), int(ldx), int(batch), _ptr(d_y), int(ldy)), m)


def sf_mlp_forward_static(m, d_x, batch, d_y, ldx=None, ldy=None):
    """sf_mlp_forward without any device allocation (fixed 4 MiB scratch inside the library)."""
    ldx = d_x.shape[-1] if ldx is None else ldx
    ldy = d_y.shape[-1] if ldy is None else ldy
    _mcheck(lib().sf_mlp_forward_static(m, _ptr(d_x), int(ldx), int(batch), _ptr(d_y), int(ldy)), m)


def sf_mlp_static_scratch_bytes() -> int:
    return int(lib().sf_mlp_static_scratch_bytes())


def sf_mlp_train_step(m, d_x, d_t, batch, lr, update=True, want_loss=True):
    loss = np.zeros(1, np.float32)
    _mcheck(lib().sf_mlp_train_step(m, _ptr(d_x), _ptr(d_t), int(batch), float(lr), int(bool(update)),
                                    _ptr(loss) if want_loss else None), m)
    return float(loss[0])


def sf_mlp_sync(m):
    return _mcheck(lib().sf_mlp_sync(m), m)


def sf_gemm_bf16(d_a, d_b, d_bias, M, N, K, act=ACT_NONE, d_out_f32=None, d_out_bf16=None, d_out_bf16_t=None,
                 ldc=None, ldt=None, tile_n=128, d_err=None, stream=None):
    ldc = N if ldc is None else ldc
    ldt = M if ldt is None else ldt
    st = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    s = lib().sf_gemm_bf16(_ptr(d_a), _ptr(d_b), _ptr(d_bias), int(M), int(N), int(K), int(act), _ptr(d_out_f32),
                           _ptr(d_out_bf16), _ptr(d_out_bf16_t), int(ldc), int(ldt), int(tile_n), _ptr(d_err),
                           C.c_void_p(st))
    if s != SF_OK:
        raise SFError(s, "sf_gemm_bf16")


# --------------------------------------------------------------------------- policy loop and graphs
def sf_step_policy(h, policy, dt=1.0 / 30.0, substeps=4):
    _check(lib().sf_step_policy(h, policy, float(dt), int(substeps)), h)


def sf_graph_capture(h, policy=None, d_actions=None, d_reset_mask=None, dt=1.0 / 30.0, substeps=4, surrogate=None):
    g = C.c_void_p()
    _check(lib().sf_graph_capture(h, policy, surrogate, _ptr(d_actions), _ptr(d_reset_mask), float(dt),
                                  int(substeps), C.byref(g)), h)
    return g


def sf_graph_launch(g):
    s = lib().sf_graph_launch(g)
    if s != SF_OK:
        raise SFError(s, "sf_graph_launch")


def sf_graph_destroy(g):
    lib().sf_graph_destroy(g)


def init_policy(seed=0, dims=(320, 512, 512, 3), stream=None, out_act=ACT_TANH, out_scale=1.0):
    """A policy MLP with seeded random (untrained) weights: ELU hidden layers,
    tanh actions (or out_act); the last layer's weights scaled by out_scale."""
    m = sf_mlp_create(list(dims), ACT_ELU, out_act, stream)
    rng = np.random.default_rng(seed)
    for l, (i, o) in enumerate(zip(dims[:-1], dims[1:])):
        w = rng.normal(0, 1 / np.sqrt(i), (o, i)) * (out_scale if l == len(dims) - 2 else 1.0)
        sf_mlp_set_layer(m, l, w, np.zeros(o))
    return m


# --------------------------------------------------------------------------- dynamics surrogate
SURR_IN, SURR_OUT = 30, 16


def sf_surrogate_create(stream=None):
    h = C.c_void_p()
    st = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    s = lib().sf_surrogate_create(C.c_void_p(st), C.byref(h))
    if s != SF_OK:
        raise SFError(s, "sf_surrogate_create")
    return h


def sf_surrogate_destroy(s):
    lib().sf_surrogate_destroy(s)


def sf_surrogate_collect(h, s, d_actions, d_x, d_y, cap, d_count, dt=1.0 / 30.0, substeps=4):
    _check(lib().sf_surrogate_collect(h, s, _ptr(d_actions), float(dt), int(substeps), _ptr(d_x), _ptr(d_y),
                                      int(cap), _ptr(d_count)), h)


def sf_surrogate_train(s, d_x, d_y, n, batch=4096, steps=2000, lr=1e-3, seed=1):
    loss = C.c_float()
    st = lib().sf_surrogate_train(s, _ptr(d_x), _ptr(d_y), int(n), int(batch), int(steps), float(lr), int(seed),
                                  C.byref(loss))
    if st != SF_OK:
        raise SFError(st, "sf_surrogate_train")
    return float(loss.value)


def sf_surrogate_mlp(s):
    return C.c_void_p(lib().sf_surrogate_mlp(s))


def sf_surrogate_stats(s):
    out = np.zeros(2 * (SURR_IN + SURR_OUT), np.float32)
    if lib().sf_surrogate_stats(s, _ptr(out)) != SF_OK:
        raise SFError(SF_ERR_CUDA, "sf_surrogate_stats")
    return out


def sf_surrogate_set_stats(s, stats):
    a = np.ascontiguousarray(stats, np.float32)
    if lib().sf_surrogate_set_stats(s, _ptr(a)) != SF_OK:
        raise SFError(SF_ERR_CUDA, "sf_surrogate_set_stats")


def sf_step_surrogate(h, s, d_actions, dt=1.0 / 30.0, substeps=4, audit=False):
    _check(lib().sf_step_surrogate(h, s, _ptr(d_actions), float(dt), int(substeps), int(bool(audit))), h)


def sf_surrogate_audit(h):
    e = C.c_float()
    n = C.c_uint64()
    _check(lib().sf_surrogate_audit(h, C.byref(e), C.byref(n)), h)
    return float(e.value), int(n.value)


# --------------------------------------------------------------------------- late-fusion actor-critic (App. E)
def _lcheck(status, m):
    if status != SF_OK:
        raise SFError(status, lib().sf_lf_last_error(m).decode())
    return status


def sf_lf_num_params() -> int:
    return int(lib().sf_lf_num_params())


def sf_lf_create(stream=None):
    m = C.c_void_p()
    st = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(lib().sf_lf_create(C.c_void_p(st), C.byref(m)))
    return m


def sf_lf_destroy(m):
    _lcheck(lib().sf_lf_destroy(m), m)


def sf_lf_set_params(m, params):
    p = np.ascontiguousarray(params, np.float32)
    _lcheck(lib().sf_lf_set_params(m, p.ctypes.data, p.size), m)


def sf_lf_get_params(m):
    p = np.zeros(sf_lf_num_params(), np.float32)
    _lcheck(lib().sf_lf_get_params(m, p.ctypes.data, p.size), m)
    return p


def sf_lf_forward(m, d_obs, d_n_road, d_n_veh, num_agents, d_mean, d_value=None, d_embed=None):
    _lcheck(lib().sf_lf_forward(m, _ptr(d_obs), _ptr(d_n_road), _ptr(d_n_veh), int(num_agents), _ptr(d_mean),
                                _ptr(d_value), _ptr(d_embed)), m)


def sf_lf_sync(m):
    _lcheck(lib().sf_lf_sync(m), m)


class sf_lf_outputs(C.Structure):
    _fields_ = [("obs", C.c_void_p), ("n_road", C.c_void_p), ("n_veh", C.c_void_p), ("actions", C.c_void_p),
                ("value", C.c_void_p), ("num_agents", C.c_int32)]


class _DevArray:
    """A library-owned device buffer exposed through __cuda_array_interface__."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = dict(shape=tuple(shape), typestr=typestr, data=(int(ptr), False),
                                             version=2, strides=None)


def device_view(ptr, shape, dtype="float32"):
    """Zero-copy torch view of a library-owned device buffer (e.g. a pointer
    from sf_output_ptrs or sf_lf_step_outputs)."""
    import torch
    typestr = {"float32": "<f4", "int32": "<i4", "uint8": "|u1", "uint32": "<u4"}[dtype]
    return torch.as_tensor(_DevArray(ptr, shape, typestr), device="cuda")


def sf_step_lf(h, lf, dt=1.0 / 30.0, substeps=4):
    _check(lib().sf_step_lf(h, lf, dt, substeps), h)


def sf_lf_step_outputs(h) -> sf_lf_outputs:
    o = sf_lf_outputs()
    _check(lib().sf_lf_step_outputs(h, C.byref(o)), h)
    return o


def sf_graph_capture_lf(h, lf, d_reset_mask=None, dt=1.0 / 30.0, substeps=4):
    g = C.c_void_p()
    _check(lib().sf_graph_capture_lf(h, lf, _ptr(d_reset_mask), dt, substeps, C.byref(g)), h)
    return g


# layer shapes (out, in) of one network in parameter order; the head has 3
# outputs in the actor and 1 in the critic
LF_LAYERS = [(64, 11), (64, 64), (96, 5), (96, 96), (96, 7), (96, 96), (128, 256), (64, 128), (None, 64)]


def init_lf(seed=0, log_std=-0.5):
    """Seeded initial parameters of the late-fusion network: weights
    N(0, 1/fan_in), biases N(0, 0.05^2), log standard deviations log_std."""
    rng = np.random.default_rng(seed)
    out = []
    for head in (3, 1):
        for o, i in LF_LAYERS:
            o = head if o is None else o
            out.append(rng.normal(0, 1 / np.sqrt(i), o * i))
            out.append(rng.normal(0, 0.05, o))
    out.append(np.full(3, log_std))
    p = np.concatenate(out).astype(np.float32)
    assert p.size == sf_lf_num_params()
    return p


# --------------------------------------------------------------------------- on-device PPO (App. L)
class sf_ppo_config(C.Structure):
    _fields_ = [("horizon", C.c_int32), ("minibatches", C.c_int32), ("epochs", C.c_int32), ("lr", C.c_float),
                ("kl_target", C.c_float), ("gamma", C.c_float), ("lam", C.c_float), ("clip", C.c_float),
                ("ent_coef", C.c_float), ("vf_coef", C.c_float), ("max_grad_norm", C.c_float),
                ("init_log_std", C.c_float), ("dt", C.c_float), ("substeps", C.c_int32), ("seed", C.c_uint64)]


class sf_ppo_rollout(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("obs", "actions", "mean", "logp", "value", "reward", "done", "advantage",
                                          "ret")] + [("horizon", C.c_int32), ("num_agents", C.c_int32),
                                                     ("minibatch_rows", C.c_int32)]


def _pcheck(status, p):
    if status != SF_OK:
        raise SFError(status, lib().sf_ppo_last_error(p).decode() if p else "sf_ppo")
    return status


def sf_ppo_default_config(**overrides):
    c = sf_ppo_config()
    lib().sf_ppo_default_config(C.byref(c))
    for k, v in overrides.items():
        setattr(c, k, v)
    return c


def sf_ppo_create(h, actor, critic, cfg=None):
    cfg = cfg if cfg is not None else sf_ppo_default_config()
    p = C.c_void_p()
    _check(lib().sf_ppo_create(h, actor, critic, C.byref(cfg), C.byref(p)), h)
    return p


def sf_ppo_create_lf(h, lf, cfg=None):
    """PPO on the late-fusion network lf (the full observation); lf is trained in place."""
    cfg = cfg if cfg is not None else sf_ppo_default_config()
    p = C.c_void_p()
    _check(lib().sf_ppo_create_lf(h, lf, C.byref(cfg), C.byref(p)), h)
    return p


def sf_ppo_lf_grads(p, d_obs, d_n_road, d_n_veh, rows, d_dmean, d_dvalue, d_mean=None, d_value=None,
                    d_argmax=None):
    """Flat gradient (sf_lf_set_params layout) of sum(dmean * mean) + sum(dvalue * value)."""
    g = np.zeros(sf_lf_num_params(), np.float32)
    _pcheck(lib().sf_ppo_lf_grads(p, _ptr(d_obs), _ptr(d_n_road), _ptr(d_n_veh), int(rows), _ptr(d_dmean),
                                  _ptr(d_dvalue), _ptr(d_mean), _ptr(d_value), _ptr(d_argmax), g.ctypes.data,
                                  C.c_size_t(g.size)), p)
    return g


def sf_ppo_lf_params(p):
    q = np.zeros(sf_lf_num_params(), np.float32)
    _pcheck(lib().sf_ppo_lf_params(p, q.ctypes.data, C.c_size_t(q.size)), p)
    return q


def sf_ppo_destroy(p):
    _pcheck(lib().sf_ppo_destroy(p), p)


def sf_ppo_collect(p):
    _pcheck(lib().sf_ppo_collect(p), p)


def sf_ppo_update(p, want_stats=True):
    """Returns (mean reward, policy loss, value loss, KL, learning rate, gradient norm) when want_stats."""
    st = np.zeros(6, np.float32)
    _pcheck(lib().sf_ppo_update(p, st.ctypes.data if want_stats else None), p)
    return st if want_stats else None


def sf_ppo_log_std(p):
    s = np.zeros(3, np.float32)
    _pcheck(lib().sf_ppo_log_std(p, s.ctypes.data), p)
    return s


def sf_ppo_rollout_ptrs(p) -> sf_ppo_rollout:
    r = sf_ppo_rollout()
    _pcheck(lib().sf_ppo_rollout_ptrs(p, C.byref(r)), p)
    return r


def sf_ppo_loss_grads(p, d_obs, d_small, rows, d_mean=None, d_value=None, d_dmean=None, d_dvalue=None):
    out = np.zeros(6, np.float32)
    _pcheck(lib().sf_ppo_loss_grads(p, _ptr(d_obs), _ptr(d_small), int(rows), _ptr(d_mean), _ptr(d_value),
                                    _ptr(d_dmean), _ptr(d_dvalue), out.ctypes.data), p)
    return out


def init_value(seed=0, dims=(320, 512, 512, 1), stream=None):
    """A critic MLP with seeded weights (ELU hidden layers, linear output)."""
    return init_policy(seed=seed, dims=dims, stream=stream, out_act=ACT_NONE, out_scale=0.1)
