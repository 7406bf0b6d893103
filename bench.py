"""Benchmark of the batched multi-world vehicle step (CASPS on one B300).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  ``value`` is controlled-agent steps per second (CASPS,
SceneFactory Sec. 4.2: agents completing one 30 Hz control step per
wall-clock second) over all ranks for the 256 worlds x 16 agents workload on
synthetic paper-shaped road graphs; the same line carries the 4096 x 16
workload, the end-to-end number through the C-ABI with host buffers, the
roofline of the world kernel and the FP64 oracle timed on the host cores.

A step is one ``sf_step``: four 120 Hz substeps with footprint contact, events,
rewards, automatic respawns of done agents and the 320-float observations of
every agent.  Inputs are resident on the device; L2 is flushed (a 256 MB
write) before every timed step, whose duration is taken by CUDA events on the
stream the kernel runs on.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2605_08528_b300 import synth  # noqa: E402

WORKLOADS = {
    # name: (worlds, agents per world, road seed base, weather)
    "256x16": (256, 16, 1000, "uniform"),
    "4096x16": (4096, 16, 4000, "wet_mix"),
}
METRIC = "CASPS at 256x16 and 4096x16; surrogate vs plain physics at matched error"
FLUSH_BYTES = 256 << 20


RAGGED = (1024, 2000, 0.2)   # worlds, road seed base, per-step reset fraction
PROFILE_STEPS = False        # --profile-steps: the timed steps bracketed by cudaProfilerStart / Stop


def make_scene(name: str, rank: int = 0):
    if name == "ragged1024":
        return synth.ragged_scene(RAGGED[0], seed_base=RAGGED[1] + rank * RAGGED[0])
    worlds, apw, seed, weather = WORKLOADS[name]
    return synth.procedural_scene(worlds, apw, seed_base=seed + rank * worlds, weather=weather,
                                  weather_seed=seed + 17 + rank)


def algorithmic_bytes(scene) -> dict:
    """Bytes one step must move at minimum: agent state read and written
    (6 float4 + 4 words = 112 B each way), actions (12 B), the observation row
    (1280 B), reward/done/events/DRAC (13 B) per agent, and every world's road
    points (float4 point + 4 B meta = 20 B) read once."""
    A = scene.num_agents
    per_agent = 2 * 112 + 12 + 320 * 4 + 13
    roads = 20 * scene.num_points
    return dict(per_agent=per_agent, roads=roads, total=A * per_agent + roads)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def load_bf16_peak():
    """Dense bf16 TFLOP/s for a kernel timed alone (burst), measured, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:
        return 1800.0


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join("/tmp", "sf_clocks_%d_%d.csv" % (os.getpid(), device_index))

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"], samples=0)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                c = [x.strip() for x in line.split(",")]
                if len(c) < 9:
                    continue
                try:
                    sm.append(float(c[1])); smax.append(float(c[2]))
                except ValueError:
                    continue
                for n, v in zip(names, c[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        return dict(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(smax) if smax else None,
                    reasons=sorted(reasons), samples=len(sm))


# --------------------------------------------------------------------------- our arm
def combine_over_ranks(t_seconds, e2e_seconds, alive, steps, e2e_steps, dist, torch, device):
    """Whole-job CASPS over all ranks: the agents every rank stepped, summed,
    over the slowest rank's time (the max over ranks of each timed region).
    dist is torch.distributed (initialised) or None for one rank."""
    tt = torch.tensor([t_seconds, e2e_seconds], dtype=torch.float64, device=device)
    n = torch.tensor([float(alive)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(n[0]) * steps / float(tt[0]), float(n[0]) * e2e_steps / float(tt[1])


def run_workload(name, steps, warmup, rank, torch, sf, stream, e2e=True, nw=0, policy_seed=None, surrogate=None,
                 pack=0, reset_frac=0.0, stage=0, split=0, dynamics=0):
    """Time `steps` replays of the captured step graph (policy forward + step
    when policy_seed is given) on the workload `name`."""
    scene = make_scene(name, rank)
    W = sf.World(scene, seed=4242 + rank, flags=sf.FLAG_AUTO_RESET, warps_per_block=nw, stream=stream,
                 pack_agents=pack, stage_bytes=stage, split_step=split, dynamics=dynamics)
    A = W.A
    dev = torch.device("cuda")
    policy = sf.init_policy(seed=policy_seed, stream=stream) if policy_seed is not None else None
    with torch.cuda.stream(stream):
        sf.sf_reset(W.h, torch.ones(A, dtype=torch.uint8, device=dev))
        ring = 64
        acts_h = synth.ou_actions(A, ring, seed=11 + rank)
        acts = torch.as_tensor(acts_h, device=dev)
        act_cur = torch.zeros((A, 3), dtype=torch.float32, device=dev)
        flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        masks = mask_cur = None
        if reset_frac > 0:                                # a random mask per step, reset inside the graph
            masks = torch.as_tensor(np.stack([synth.reset_mask(A, t, reset_frac, seed=7 + rank) for t in range(ring)]),
                                    device=dev)
            mask_cur = torch.zeros(A, dtype=torch.uint8, device=dev)
        tuned = None
        if nw == 0:                                       # setup: pick the launch shape (state restored)
            tuned = sf.sf_autotune(W.h, acts[0], iters=10)
        graph = sf.sf_graph_capture(W.h, policy=policy, d_actions=act_cur, d_reset_mask=mask_cur,
                                    surrogate=surrogate)
        if surrogate is not None:
            sf.sf_surrogate_audit(W.h)                    # reset the usage counter
        for t in range(warmup):
            act_cur.copy_(acts[t % ring])
            if masks is not None:
                mask_cur.copy_(masks[t % ring])
            sf.sf_graph_launch(graph)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        torch.cuda.synchronize()
        if PROFILE_STEPS:                                 # an external profiler captures the timed steps only
            torch.cuda.profiler.start()
        t0 = time.perf_counter()
        for t in range(steps):
            act_cur.copy_(acts[(warmup + t) % ring])      # stage this step's actions (untimed)
            if masks is not None:
                mask_cur.copy_(masks[(warmup + t) % ring])
            flush.fill_(float(t))                         # evict the working set from L2
            starts[t].record(stream)
            sf.sf_graph_launch(graph)
            ends[t].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if PROFILE_STEPS:
            torch.cuda.profiler.stop()
    st = sf.sf_sync(W.h, allow=(sf.SF_ERR_NONFINITE,))
    ms = np.array([s.elapsed_time(e) for s, e in zip(starts, ends)])
    surr_used = sf.sf_surrogate_audit(W.h)[1] if surrogate is not None else 0
    F, I, _ = sf.sf_get_state(W.h)
    alive = int(((I[:, 4] & 1) != 0).sum())
    peak_drac = float(F[(I[:, 4] & 1) != 0, 24].mean()) if alive else 0.0
    sf.sf_graph_destroy(graph)
    if policy is not None:
        sf.sf_mlp_destroy(policy)
    if not e2e:
        W.close()
        return dict(scene=scene, A=A, alive=alive, ms=ms, wall=wall, status=st, e2e_wall=float("nan"),
                    e2e_steps=1, h2d=A * 12, d2h=A * 5, tuned=tuned, peak_drac=peak_drac,
                    surr_frac=surr_used / float((warmup + steps) * A), e2e_obs_wall=float("nan"), d2h_obs=0)
    # end to end through the C-ABI (sf_step_host): page-locked host actions in (a
    # ring of action sets), host rewards / done flags out, every step
    acts_pin = [torch.as_tensor(acts_h[k]).pin_memory() for k in range(ring)]
    rew_h = torch.empty(A, dtype=torch.float32).pin_memory()
    done_h = torch.empty(A, dtype=torch.uint8).pin_memory()
    rew_np = rew_h.numpy()                               # host views of the page-locked results
    e2e_steps = max(50, steps // 4)
    sf.sf_step_host(W.h, acts_pin[0], rew_h, done_h)   # capture outside the timed region
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for t in range(e2e_steps):
        sf.sf_step_host(W.h, acts_pin[t % ring], rew_h, done_h)
        float(rew_np[0])                                 # the host consumes the result
    e2e_wall = time.perf_counter() - t0
    # the same with the 320-value observation delivered to the host every step
    # (sf_step_host_obs: one more copy node in the graph, 1,280 B per agent)
    obs_h = torch.empty((A, sf.OBS_DIM), dtype=torch.float32).pin_memory()
    obs_np = obs_h.numpy()
    sf.sf_step_host_obs(W.h, acts_pin[0], obs_h, rew_h, done_h)   # capture outside the timed region
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for t in range(e2e_steps):
        sf.sf_step_host_obs(W.h, acts_pin[t % ring], obs_h, rew_h, done_h)
        float(rew_np[0]) + float(obs_np[0, 0])           # the host consumes the results
    e2e_obs_wall = time.perf_counter() - t0
    W.close()
    return dict(scene=scene, A=A, alive=alive, ms=ms, wall=wall, status=st, e2e_wall=e2e_wall,
                e2e_steps=e2e_steps, h2d=A * 12, d2h=A * 5, tuned=tuned, peak_drac=peak_drac, surr_frac=0.0,
                e2e_obs_wall=e2e_obs_wall, d2h_obs=A * (5 + sf.OBS_DIM * 4))


def time_mlp_forward(m, rows, torch, sf, stream, reps=20):
    """Mean time [ms] of one forward of MLP m over `rows` rows of 30 inputs
    (CUDA events on the MLP's stream after a warm-up; the surrogate MLP of the
    step alone, for the phase-level comparison with the physics)."""
    with torch.cuda.stream(stream):
        x = torch.randn((rows, sf.SURR_IN), device="cuda")
        y = torch.empty((rows, sf.SURR_OUT), device="cuda")
        for _ in range(3):
            sf.sf_mlp_forward(m, x, rows, y)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            sf.sf_mlp_forward(m, x, rows, y)
        t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / reps


def lf_flops(n_road, n_veh):
    """Algorithmic FLOPs of one late-fusion forward (actor and critic, App. E):
    the set encoders on every filled slot, ego, trunk and heads per agent."""
    per_road = 2 * (5 * 96 + 96 * 96)
    per_veh = 2 * (7 * 96 + 96 * 96)
    per_agent = 2 * (11 * 64 + 64 * 64 + 256 * 128 + 128 * 64)
    return 2 * (per_road * float(np.sum(n_road)) + per_veh * float(np.sum(n_veh)) + per_agent * len(n_road)) + \
        2 * 64 * 4 * len(n_road)


def run_paper_loop(name, steps, warmup, rank, torch, sf, stream, nw=0, pack=0, stage=0, split=0):
    """The paper's control loop on the full observation: sf_observe_full ->
    late-fusion actor-critic (seeded random weights) -> sf_step, captured in one
    graph, auto-reset; plus the observation and network timed alone."""
    scene = make_scene(name, rank)
    W = sf.World(scene, seed=4242 + rank, flags=sf.FLAG_AUTO_RESET, stream=stream, warps_per_block=nw,
                 pack_agents=pack, stage_bytes=stage, split_step=split)
    A = W.A
    dev = torch.device("cuda")
    lf = sf.sf_lf_create(stream)
    sf.sf_lf_set_params(lf, sf.init_lf(seed=4000 + rank))
    with torch.cuda.stream(stream):
        sf.sf_reset(W.h, torch.ones(A, dtype=torch.uint8, device=dev))
        if nw == 0:                                   # setup: pick the step's launch shape (state restored)
            sf.sf_autotune(W.h, torch.zeros((A, 3), device=dev), iters=10)
        flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        graph = sf.sf_graph_capture_lf(W.h, lf)
        for t in range(warmup):
            sf.sf_graph_launch(graph)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        torch.cuda.synchronize()
        for t in range(steps):
            flush.fill_(float(t))
            starts[t].record(stream)
            sf.sf_graph_launch(graph)
            ends[t].record(stream)
        torch.cuda.synchronize()
        ms = np.array([a.elapsed_time(b) for a, b in zip(starts, ends)])
        o = sf.sf_lf_step_outputs(W.h)
        obs = sf.device_view(o.obs, (A, sf.FULL_OBS_DIM))
        nr = sf.device_view(o.n_road, (A,), "int32")
        nv = sf.device_view(o.n_veh, (A,), "int32")
        mean = torch.empty((A, 3), device=dev)
        val = torch.empty(A, device=dev)

        def alone(fn, n=30):
            ts = []
            for i in range(n + 3):
                flush.fill_(float(i))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                torch.cuda.synchronize()
                if i >= 3:
                    ts.append(a.elapsed_time(b))
            return float(np.mean(ts))
        obs_ms = alone(lambda: sf.sf_observe_full(W.h, obs, nr, nv))
        lf_ms = alone(lambda: sf.sf_lf_forward(lf, obs, nr, nv, A, mean, val))
        n_road, n_veh = nr.cpu().numpy(), nv.cpu().numpy()
    sf.sf_sync(W.h, allow=(sf.SF_ERR_NONFINITE,))
    sf.sf_lf_sync(lf)
    sf.sf_graph_destroy(graph)
    sf.sf_lf_destroy(lf)
    W.close()
    obs_bytes = A * (sf.FULL_OBS_DIM * 4 + 8 + 68) + scene.num_points * 17
    return dict(A=A, ms=ms, obs_ms=obs_ms, lf_ms=lf_ms, obs_bytes=obs_bytes, flops=lf_flops(n_road, n_veh),
                mean_road=float(n_road.mean()), mean_veh=float(n_veh.mean()))


def run_ppo(name, iters, rank, torch, sf, stream, profile_update=False, net="mlp", stat_iters=3):
    """On-device PPO with the paper's hyperparameters (App. L: horizon 128, 16
    minibatches, 5 epochs): per iteration one rollout (policy and value forward,
    Gaussian sampling, the step) and one update (GAE and 80 minibatch steps),
    timed with CUDA events; the training CASPS counts the rollout's agent-steps
    over the whole iteration, as the paper's CASPS includes the PPO update.
    net "mlp": actor / critic MLPs on the 320-value observation; "lf": the
    paper's late-fusion actor-critic (App. E) on the full observation."""
    scene = make_scene(name, rank)
    W = sf.World(scene, seed=4242 + rank, flags=sf.FLAG_AUTO_RESET, stream=stream)
    A = W.A
    with torch.cuda.stream(stream):
        sf.sf_reset(W.h, torch.ones(A, dtype=torch.uint8, device="cuda"))
        sf.sf_autotune(W.h, torch.zeros((A, 3), device="cuda"), iters=10)
    actor = critic = lf = None
    if net == "lf":
        lf = sf.sf_lf_create(stream)
        sf.sf_lf_set_params(lf, sf.init_lf(seed=5000 + rank, log_std=-0.5))
        cfg = sf.sf_ppo_default_config(seed=77 + rank)
        ppo = sf.sf_ppo_create_lf(W.h, lf, cfg)
    else:
        actor = sf.init_policy(seed=5000 + rank, stream=stream, out_scale=0.1)
        critic = sf.init_value(seed=6000 + rank, stream=stream)
        cfg = sf.sf_ppo_default_config(init_log_std=-0.5, seed=77 + rank)
        ppo = sf.sf_ppo_create(W.h, actor, critic, cfg)
    sf.sf_ppo_collect(ppo)                        # warm-up iteration (buffers, kernel attributes)
    sf.sf_ppo_update(ppo)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(iters)]
    stats = []
    torch.cuda.synchronize()
    for i in range(iters):
        ev[i][0].record(stream)
        sf.sf_ppo_collect(ppo)
        ev[i][1].record(stream)
        if profile_update:                        # an external profiler captures this update only
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
        sf.sf_ppo_update(ppo, want_stats=False)
        ev[i][2].record(stream)
        if profile_update:
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
    torch.cuda.synchronize()
    collect_ms = np.array([e[0].elapsed_time(e[1]) for e in ev])
    update_ms = np.array([e[1].elapsed_time(e[2]) for e in ev])
    for i in range(stat_iters):                   # learning statistics (untimed iterations)
        sf.sf_ppo_collect(ppo)
        stats.append(sf.sf_ppo_update(ppo).tolist())
    log_std = sf.sf_ppo_log_std(ppo).tolist()
    sf.sf_ppo_destroy(ppo)
    if lf is not None:
        sf.sf_lf_destroy(lf)
    else:
        sf.sf_mlp_destroy(actor)
        sf.sf_mlp_destroy(critic)
    W.close()
    steps = A * cfg.horizon
    return dict(A=A, horizon=cfg.horizon, collect_ms=float(collect_ms.mean()), update_ms=float(update_ms.mean()),
                casps_train=steps / ((collect_ms + update_ms).mean() / 1e3),
                casps_collect=steps / (collect_ms.mean() / 1e3), stats=stats, log_std=log_std)


def cpu_baseline(name, seconds=12.0):
    """The FP64 oracle as it stands, single thread, on a bounded sample of the
    workload: the first worlds of the same scene, stepped until ~`seconds`."""
    from oracle import oracle as O
    scene = make_scene(name)
    worlds = list(range(8))
    sub, rows = synth.subscene(scene, worlds)
    orc = O.Oracle(sub)
    F, I = orc.empty_state()
    I[:, O.I_PRECIP], I[:, O.I_SURFACE] = sub.precip, sub.surface
    orc.reset(F, I, np.ones(sub.num_agents, np.uint8), seed=4242)
    acts = synth.ou_actions(sub.num_agents, 64, seed=11).astype(np.float64)
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < seconds:
        orc.step(F, I, acts[n % 64], flags=O.FLAG_AUTO_RESET, seed=4242)
        n += 1
    dt = time.perf_counter() - t0
    return dict(value=sub.num_agents * n / dt, unit="CASPS", cores=1, kind="oracle", cpu_model=host_cpu_model(),
                sample="%d of %d worlds (%d agents) x %d steps of the %s workload, FP64, 1 thread" % (
                    len(worlds), scene.num_worlds, sub.num_agents, n, name))


def _oracle_worker(job):
    """One host process of the all-cores oracle timing: worlds [w0, w0 + nw) of
    the workload, `warmup` untimed steps, then `steps` timed steps (or as many
    as fit in `seconds` when steps is None); returns (agents, steps, elapsed)."""
    name, w0, nw, warmup, steps, seconds = job
    from oracle import oracle as O
    scene = make_scene(name)
    sub, _ = synth.subscene(scene, list(range(w0, w0 + nw)))
    orc = O.Oracle(sub)
    F, I = orc.empty_state()
    I[:, O.I_PRECIP], I[:, O.I_SURFACE] = sub.precip, sub.surface
    orc.reset(F, I, np.ones(sub.num_agents, np.uint8), seed=4242)
    acts = synth.ou_actions(sub.num_agents, 64, seed=11 + w0).astype(np.float64)
    for t in range(warmup):
        orc.step(F, I, acts[t % 64], flags=O.FLAG_AUTO_RESET, seed=4242)
    t0 = time.perf_counter()
    n = 0
    while (n < steps) if steps is not None else (time.perf_counter() - t0 < seconds):
        orc.step(F, I, acts[(warmup + n) % 64], flags=O.FLAG_AUTO_RESET, seed=4242)
        n += 1
    return sub.num_agents, n, time.perf_counter() - t0


def oracle_on_all_cores(name, warmup=0, steps=None, seconds=12.0):
    """The oracle on every host core: one process per core (started with
    spawn), each on its own consecutive worlds of the workload (8, or fewer
    when the cores outnumber the worlds / 8); returns (agent-steps per second
    over the slowest process, processes, agents, worlds per process)."""
    import multiprocessing as mp
    worlds = WORKLOADS[name][0]
    cores = os.cpu_count() or 1
    per = max(1, min(8, worlds // cores))
    procs = min(cores, worlds // per)
    jobs = [(name, per * k, per, warmup, steps, seconds) for k in range(procs)]
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_worker, jobs)
    agent_steps = sum(a * n for a, n, _ in res)
    return agent_steps / max(t for _, _, t in res), procs, sum(a for a, _, _ in res), per


def host_cpu_model():
    """The host CPU's model name (Linux), or the platform's processor string."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or "unknown"


def cpu_baseline_all_cores(name, seconds=12.0):
    """The same oracle on every host core (after the GPU work), each process on
    its own 8 worlds of the workload."""
    v, cores, agents, per = oracle_on_all_cores(name, seconds=seconds)
    return dict(value=v, unit="CASPS", cores=cores, kind="oracle", cpu_model=host_cpu_model(),
                sample="%d processes x %d worlds (%d agents in all) of the %s workload, FP64, %.0f s each" % (
                    cores, per, agents, name, seconds))


def main_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2605_08528_b300 import sf
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    peak, peak_kind = load_peaks()
    bf16_peak = load_bf16_peak()

    clocks = ClockSampler(local)
    clocks.start()
    res = {}
    names = [args.only] if args.only else list(WORKLOADS) + ["ragged1024"]
    for name in names:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if name in ("ppo", "ppo_lf"):                 # profiling target: a PPO leg alone
            r = run_ppo("256x16", 1 if args.profile_update else (3 if name == "ppo" else 2), rank, torch, sf, stream,
                        profile_update=args.profile_update, net="lf" if name == "ppo_lf" else "mlp",
                        stat_iters=3 if name == "ppo" else 1)
            if rank == 0:
                print(json.dumps({"profile_run": name, "rollout_ms": r["collect_ms"], "update_ms": r["update_ms"]}))
            clocks.stop()
            return
        if name.startswith("paper"):                  # profiling target: the paper loop alone
            r = run_paper_loop(name[5:], args.steps, args.warmup, rank, torch, sf, stream, nw=args.nw, pack=args.pack,
                               stage=args.stage, split=args.split)
            if rank == 0:
                print(json.dumps({"profile_run": name, "ms_per_step": float(r["ms"].mean()), "agents": r["A"],
                                  "observation_ms": r["obs_ms"], "network_ms": r["lf_ms"]}))
            clocks.stop()
            return
        if name.endswith("+surrogate"):               # profiling target: the surrogate step graph alone
            from paper_2605_08528_b300 import surrogate as SU
            base = name[:-len("+surrogate")]
            surr, rows, loss = SU.collect_and_train(make_scene("256x16", rank), transitions=args.surr_rows,
                                                    train_steps=args.surr_steps, seed=31 + rank, stream=stream)
            r = run_workload(base, args.steps, args.warmup, rank, torch, sf, stream, e2e=False, nw=args.nw,
                             surrogate=surr, pack=args.pack, stage=args.stage, split=args.split)
            sf.sf_surrogate_destroy(surr)
            if rank == 0:
                print(json.dumps({"profile_run": name, "ms_per_step": float(r["ms"].mean()), "agents": r["A"],
                                  "gated_fraction": r["surr_frac"], "training_rows": rows}))
            clocks.stop()
            return
        if name == "4096x16+policy":                  # profiling target: the policy + step graph alone
            res[name] = run_workload("4096x16", args.steps, args.warmup, rank, torch, sf, stream, e2e=False,
                                     nw=args.nw, policy_seed=4000, pack=args.pack, stage=args.stage,
                                     split=args.split)
        elif name == "ragged1024":
            res[name] = run_workload(name, args.steps, args.warmup, rank, torch, sf, stream, e2e=False, nw=args.nw,
                                     pack=args.pack, reset_frac=RAGGED[2], stage=args.stage,
                                     split=args.split)
        else:
            res[name] = run_workload(name, args.steps, args.warmup, rank, torch, sf, stream,
                                     e2e=not args.skip_e2e, nw=args.nw, pack=args.pack, stage=args.stage,
                                     split=args.split)
    surr = None
    surr_info = None
    if not args.only and not args.skip_surrogate:
        from paper_2605_08528_b300 import surrogate as SU
        t0 = time.perf_counter()
        surr, rows, loss = SU.collect_and_train(make_scene("256x16", rank), transitions=args.surr_rows,
                                                train_steps=args.surr_steps, seed=31 + rank, stream=stream)
        t_train = time.perf_counter() - t0
        lone = synth.procedural_scene(2048, 1, seed_base=9000 + 2048 * rank)
        lone.precip[:] = np.minimum(lone.precip, 2)       # mu >= 0.3 cells (the gate's range)
        err, frac = SU.rollout_error(surr, lone, stream=stream, segments=5)    # 10,240 held-out start states
        surr_info = dict(rows=rows, train_steps=args.surr_steps, final_loss=loss, train_s=t_train,
                         err_mean_m=float(err.mean()), err_p90_m=float(np.percentile(err, 90)),
                         err_p99_m=float(np.percentile(err, 99)),
                         err_max_m=float(err.max()), eval_states=int(err.size), gated_fraction_lone=frac)
        for name in ("256x16", "4096x16"):
            if world > 1:
                dist.barrier()
            res[name + "+surrogate"] = run_workload(name, args.steps, args.warmup, rank, torch, sf, stream,
                                                    e2e=False, nw=args.nw, surrogate=surr, pack=args.pack,
                                                    stage=args.stage, split=args.split)
            surr_info["mlp_forward_ms_" + name] = time_mlp_forward(sf.sf_surrogate_mlp(surr),
                                                                   res[name + "+surrogate"]["A"], torch, sf, stream)
    if not args.only and not args.skip_policy:
        if world > 1:
            dist.barrier()
        res["4096x16+policy"] = run_workload("4096x16", args.steps, args.warmup, rank, torch, sf, stream, e2e=False,
                                             nw=args.nw, policy_seed=4000, surrogate=surr, pack=args.pack,
                                             stage=args.stage, split=args.split)
    if surr is not None:
        sf.sf_surrogate_destroy(surr)
    bikes = {}
    if not args.only and not args.skip_bicycle:
        for name in ("256x16", "4096x16"):
            if world > 1:
                dist.barrier()
            bikes[name] = run_workload(name, max(args.steps // 4, 50), args.warmup, rank, torch, sf, stream,
                                       e2e=False, nw=args.nw, pack=args.pack, stage=args.stage, split=args.split,
                                       dynamics=sf.DYN_BICYCLE)
    ppo = ppo_lf = None
    if not args.only and not args.skip_ppo:
        if world > 1:
            dist.barrier()
        ppo = run_ppo("256x16", 3, rank, torch, sf, stream)
        if world > 1:
            dist.barrier()
        ppo_lf = run_ppo("256x16", 2, rank, torch, sf, stream, net="lf", stat_iters=2)
    loops = {}
    if not args.only and not args.skip_paper_loop:
        for name in ("256x16", "4096x16"):
            if world > 1:
                dist.barrier()
            loops[name] = run_paper_loop(name, max(args.steps // 4, 50), args.warmup, rank, torch, sf, stream)
    clk = clocks.stop()
    if args.only:          # profiling run: one workload, no report line
        if rank == 0:
            r = res[args.only]
            print(json.dumps({"profile_run": args.only, "ms_per_step": float(r["ms"].mean()), "agents": r["A"]}))
        return

    def agg(name):
        r = res[name]
        casps, e2e_casps = combine_over_ranks(float(r["ms"].sum()) / 1e3, r["e2e_wall"], r["alive"], args.steps,
                                              r["e2e_steps"], dist if world > 1 else None, torch, "cuda")
        _, e2e_obs = combine_over_ranks(float(r["ms"].sum()) / 1e3, r["e2e_obs_wall"], r["alive"], args.steps,
                                        r["e2e_steps"], dist if world > 1 else None, torch, "cuda")
        ab = algorithmic_bytes(r["scene"])
        mean_s = float(r["ms"].mean()) / 1e3
        ach = ab["total"] / mean_s / 1e9
        return dict(casps=casps, e2e=e2e_casps, e2e_obs=e2e_obs, d2h_obs=r["d2h_obs"], ms=float(r["ms"].mean()), p50=float(np.percentile(r["ms"], 50)),
                    p99=float(np.percentile(r["ms"], 99)), bytes=ab, achieved=ach, A=r["A"], alive=r["alive"],
                    h2d=r["h2d"], d2h=r["d2h"], tuned=r["tuned"], peak_drac=r["peak_drac"], surr_frac=r["surr_frac"])

    a256, a4096 = agg("256x16"), agg("4096x16")
    apol = agg("4096x16+policy") if "4096x16+policy" in res else None
    arag = agg("ragged1024") if "ragged1024" in res else None
    asur = {k: agg(k + "+surrogate") for k in ("256x16", "4096x16") if k + "+surrogate" in res}
    if rank == 0:
        base = cpu_baseline("256x16") if (world == 1 and not args.skip_cpu) else None
        base_all = cpu_baseline_all_cores("256x16") if (world == 1 and not args.skip_cpu) else None
        fp32_peak = sf.sf_fp32_fma_peak(stream)
        traffic = load_traffic()
        line = {
            "metric": METRIC, "value": a256["casps"], "unit": "CASPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": a256["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "256 worlds x 16 agents, paper-shaped procedural roads (4-12 lanes, 0-2 "
                                   "intersections, 400-1200 points/world), per-agent weather table mu, auto-reset",
                       "worlds": 256 * world, "agents": a256["A"] * world, "dt": 1 / 30, "substeps": 4,
                       "K_agents": 8, "L_points": 32, "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": "worlds sharded, no data-path collective" if world > 1 else "1 GPU",
                       "autotune": a256["tuned"]},
            "p50_ms": a256["p50"], "p99_ms": a256["p99"],
            "e2e": {"value": a256["e2e"], "unit": "CASPS", "h2d_bytes_per_step": a256["h2d"],
                    "d2h_bytes_per_step": a256["d2h"],
                    "what": "sf_step_host: actions in, rewards and done flags out each step; the observation "
                            "stays on the device (a policy on the GPU reads it there)"},
            "e2e_with_observation": {"value": a256["e2e_obs"], "unit": "CASPS", "h2d_bytes_per_step": a256["h2d"],
                                     "d2h_bytes_per_step": a256["d2h_obs"],
                                     "what": "sf_step_host_obs: the same plus the 320-value observation of every "
                                             "agent copied to page-locked host memory each step"},
            "gpu_launches": args.steps,
            "graph": "each timed step is one CUDA-graph replay",
            "roofline": {"bound": "hbm", "kernel": step_kernels(a256["tuned"]), "achieved": a256["achieved"],
                         "peak": peak, "unit": "GB/s", "frac": a256["achieved"] / peak,
                         "peak_source": peak_kind, "algorithmic_bytes_per_launch": a256["bytes"]["total"],
                         "traffic": traffic_of(traffic, "256x16", a256["tuned"])},
            "scale_4096x16": {"value": a4096["casps"], "unit": "CASPS", "ms_per_step": a4096["ms"],
                              "p50_ms": a4096["p50"], "p99_ms": a4096["p99"],
                              "agents": a4096["A"] * world, "autotune": a4096["tuned"],
                              "e2e": {"value": a4096["e2e"], "unit": "CASPS", "h2d_bytes_per_step": a4096["h2d"],
                                      "d2h_bytes_per_step": a4096["d2h"]},
                              "e2e_with_observation": {"value": a4096["e2e_obs"], "unit": "CASPS",
                                                       "h2d_bytes_per_step": a4096["h2d"],
                                                       "d2h_bytes_per_step": a4096["d2h_obs"]},
                              "roofline": {"bound": "hbm", "kernel": step_kernels(a4096["tuned"]),
                                           "achieved": a4096["achieved"], "peak": peak,
                                           "unit": "GB/s", "frac": a4096["achieved"] / peak,
                                           "algorithmic_bytes_per_launch": a4096["bytes"]["total"],
                                           "traffic": traffic_of(traffic, "4096x16", a4096["tuned"])},
                              "mean_peak_drac": a4096["peak_drac"]},
            "scale_ragged1024": None if arag is None else {
                "value": arag["casps"], "unit": "CASPS", "ms_per_step": arag["ms"], "p50_ms": arag["p50"],
                "p99_ms": arag["p99"], "agents": arag["A"] * world, "autotune": arag["tuned"],
                "workload": "1024 worlds, agents floor(exp(U[0, ln 32])), road points exp(U[ln 100, ln 5000]), "
                            "CSR; a random 20% reset mask every step inside the graph",
                "roofline": {"bound": "hbm", "kernel": step_kernels(arag["tuned"]), "achieved": arag["achieved"],
                             "peak": peak, "unit": "GB/s",
                             "frac": arag["achieved"] / peak,
                             "algorithmic_bytes_per_launch": arag["bytes"]["total"]}},
            "scale_4096x16_policy": None if apol is None else {
                "value": apol["casps"], "unit": "CASPS", "ms_per_step": apol["ms"], "p50_ms": apol["p50"],
                "p99_ms": apol["p99"], "mean_peak_drac": apol["peak_drac"],
                "surrogate_fraction": apol["surr_frac"],
                "graph": "BF16 tcgen05 policy 320-512-512-3 (ELU, tanh; seeded random weights) + surrogate "
                         "features + BF16 surrogate MLP + world step (surrogate for gated agents, physics fallback)",
                "wet_mix": "50% heavy-rain asphalt mu 0.5, 50% dry asphalt mu 0.9"},
            "surrogate": None if surr_info is None else dict(
                surr_info,
                error_reference="FP32 physics path (parity with the FP64 oracle <= 4.3e-5 m over 100 steps)",
                **{"casps_" + k: v["casps"] for k, v in asur.items()},
                **{"speedup_vs_physics_" + k: v["casps"] / (a256 if k == "256x16" else a4096)["casps"]
                   for k, v in asur.items()},
                **{"gated_fraction_" + k: v["surr_frac"] for k, v in asur.items()}),
            "bicycle": {k: {
                "value": v["alive"] * world * len(v["ms"]) / (float(v["ms"].sum()) / 1e3), "unit": "CASPS",
                "ms_per_step": float(v["ms"].mean()), "p50_ms": float(np.percentile(v["ms"], 50)),
                "p99_ms": float(np.percentile(v["ms"], 99)), "agents": v["A"] * world, "autotune": v["tuned"],
                "dynamics": "kinematic bicycle (Sec. 4.4 ablation backend): one update per control step, same "
                            "events, rewards, observations and resets"}
                for k, v in bikes.items()} or None,
            "ppo": None if ppo is None else {
                "value": ppo["casps_train"] * world, "unit": "CASPS (training: rollout + PPO update)",
                "workload": "256 worlds x 16 agents, App. L hyperparameters (horizon 128, 16 minibatches, 5 epochs, "
                            "clip 0.15, gamma 0.99, lambda 0.98, adaptive KL 0.01); actor 320-512-512-3 and critic "
                            "320-512-512-1 BF16 tcgen05 MLPs",
                "rollout_ms": ppo["collect_ms"], "update_ms": ppo["update_ms"],
                "rollout_casps": ppo["casps_collect"] * world,
                "stats_columns": ["mean reward", "policy loss", "value loss", "kl", "lr", "grad norm"],
                "stats_last_iterations": ppo["stats"], "log_std": ppo["log_std"],
                "paper_context": "19,250 CASPS during PPO training at 256 x 16 (RTX PRO 6000, Isaac Sim/PhysX)"},
            "ppo_lf": None if ppo_lf is None else {
                "value": ppo_lf["casps_train"] * world, "unit": "CASPS (training: rollout + PPO update)",
                "workload": "256 worlds x 16 agents, App. L hyperparameters, the paper's late-fusion actor-critic "
                            "(App. E) on the full 1929-value observation (App. D): tensor-core set encoders with "
                            "masked max-pool, trunk and heads; backward through the max-pool as tensor-core products over "
                            "each sample's distinct maximising slots",
                "rollout_ms": ppo_lf["collect_ms"], "update_ms": ppo_lf["update_ms"],
                "rollout_casps": ppo_lf["casps_collect"] * world,
                "stats_columns": ["mean reward", "policy loss", "value loss", "kl", "lr", "grad norm"],
                "stats_last_iterations": ppo_lf["stats"], "log_std": ppo_lf["log_std"]},
            "paper_loop": {k: {
                "value": v["A"] * world * len(v["ms"]) / (float(v["ms"].sum()) / 1e3), "unit": "CASPS",
                "ms_per_step": float(v["ms"].mean()), "p50_ms": float(np.percentile(v["ms"], 50)),
                "p99_ms": float(np.percentile(v["ms"], 99)), "agents": v["A"] * world,
                "graph": "full 1929-value observation (App. D) + late-fusion actor-critic (App. E, BF16 tcgen05, "
                         "seeded random weights) + step, one CUDA graph, auto-reset",
                "mean_filled_slots": {"road": v["mean_road"], "vehicles": v["mean_veh"]},
                "observation_kernel": {"bound": "hbm", "ms": v["obs_ms"], "algorithmic_bytes": v["obs_bytes"],
                                       "achieved": v["obs_bytes"] / v["obs_ms"] / 1e6, "peak": peak,
                                       "unit": "GB/s", "frac": v["obs_bytes"] / v["obs_ms"] / 1e6 / peak},
                "network": {"bound": "tensor", "ms": v["lf_ms"], "algorithmic_flops": v["flops"],
                            "achieved": v["flops"] / v["lf_ms"] / 1e9, "peak": bf16_peak, "unit": "TFLOP/s",
                            "frac": v["flops"] / v["lf_ms"] / 1e9 / bf16_peak}}
                for k, v in loops.items()} or None,
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"],
                       "samples": clk["samples"]},
            "paper_context": "19,250 CASPS at 256x16 on an RTX PRO 6000 (Isaac Sim/PhysX + PPO), context only",
        }
        if base is not None:
            line["cpu_baseline"] = base
        if base_all is not None:
            line["cpu_baseline_all_cores"] = base_all
        # the denominator of the step's ALU roofline (its FP32 pipe use is in profiles/)
        line["fp32_fma_peak"] = {"value": fp32_peak, "unit": "TFLOP/s", "kind": "measured",
                                 "nominal": 2.0 * 128 * torch.cuda.get_device_properties(0).multi_processor_count
                                 * clk["sm_max_mhz"] * 1e6 / 1e12 if clk["sm_max_mhz"] else None}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def step_kernels(tuned) -> str:
    """The kernels one timed step launches, from the autotuned launch shape."""
    if not tuned:
        return "world_kernel<step>"
    nw, pack, stage, split = tuned[0]
    if split:
        return "split step: phys, query<%d>, events, fix kernels (pack %d)" % (nw, pack)
    return "world_kernel<step, %d warps> (pack %d, staged %d B)" % (nw, pack, stage)


def kernel_source_tag():
    """First 12 hex digits of the SHA-1 of the step kernels' code (sf_world.cu
    then sf_internal.cuh, comments dropped and white space collapsed): a DRAM
    traffic figure holds only for the code it was captured on."""
    import hashlib
    import re
    h = hashlib.sha1()
    for f in ("sf_world.cu", "sf_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2605_08528_b300", "csrc", f)) as fh:
            code = re.sub(r"/\*.*?\*/", " ", fh.read(), flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(re.sub(r"\s+", " ", code).strip().encode())
    return h.hexdigest()[:12]


def load_traffic():
    """DRAM bytes per launch of the kernel a roofline describes, from the
    committed ncu summary (lines "workload bytes shape source-tag ..."); an
    entry captured on another source than the current one is dropped."""
    out = {}
    try:
        tag = kernel_source_tag()
        with open(os.path.join(ROOT, "profiles", "world_kernel_traffic.txt")) as f:
            for line in f:
                parts = line.split()
                if parts and not parts[0].startswith("#") and len(parts) >= 4 and parts[3] == tag:
                    out[parts[0]] = (int(parts[1]), [int(x) for x in parts[2].split(",")])
    except (OSError, ValueError):
        pass
    return out


def traffic_of(traffic, name, tuned):
    """Captured DRAM bytes per launch for this workload when the timed launch
    shape and the kernel source are the captured ones, else None."""
    t = traffic.get(name)
    if t is None or not tuned or list(tuned[0]) != t[1]:
        return None
    return t[0]


# --------------------------------------------------------------------------- reference arm
def main_reference(args):
    """The FP64 oracle as it stands on the host cores, for the same metric and
    workload: one process per core, each stepping its own 8 of the 256 worlds."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    v, cores, agents, per = oracle_on_all_cores("256x16", warmup=args.warmup, steps=args.steps)
    dt = agents * args.steps / v

    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "CASPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "256 worlds x 16 agents (sample: %d worlds per host process, %d agents per "
                                   "step)" % (per, agents)},
            "cpu_baseline": {"value": v, "unit": "CASPS", "cores": cores, "kind": "oracle",
                             "cpu_model": host_cpu_model(), "sample": "%d processes x %d of the 256 worlds (%d agents in all) per step, FP64" % (
                                 cores, per, agents)},
            "e2e": {"value": v, "unit": "CASPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--only", default=None,
                    choices=list(WORKLOADS) + ["ragged1024", "4096x16+policy", "256x16+surrogate", "4096x16+surrogate",
                                               "paper256x16", "paper4096x16", "ppo", "ppo_lf"],
                    help="profiling: run one workload only (*+surrogate: a surrogate trained with --surr-rows / "
                         "--surr-steps, then its step graph; paper*: the full-observation + late-fusion loop; "
                         "ppo: the on-device PPO leg)")
    ap.add_argument("--profile-update", action="store_true",
                    help="with --only ppo: one iteration, its update bracketed by cudaProfilerStart / Stop")
    ap.add_argument("--profile-steps", action="store_true",
                    help="profiling: the timed steps of each leg bracketed by cudaProfilerStart / Stop "
                         "(for ncu --profile-from-start off)")
    ap.add_argument("--skip-e2e", action="store_true", help="profiling: no end-to-end leg")
    ap.add_argument("--skip-cpu", action="store_true", help="no oracle CPU baseline")
    ap.add_argument("--nw", type=int, default=0, help="warps per block (1, 2, 4, 8; 0 = autotuned)")
    ap.add_argument("--pack", type=int, default=0, help="with --nw: agents per packed block (0 = one world)")
    ap.add_argument("--stage", type=int, default=0, help="with --nw: road staging bytes per block (0 = off)")
    ap.add_argument("--split", type=int, default=0, help="with --nw: 1 = the step as four kernels")
    ap.add_argument("--skip-policy", action="store_true", help="no 4096x16 + policy leg")
    ap.add_argument("--skip-surrogate", action="store_true", help="no surrogate training / legs")
    ap.add_argument("--skip-paper-loop", action="store_true", help="no full-observation + late-fusion legs")
    ap.add_argument("--skip-bicycle", action="store_true", help="no kinematic-bicycle legs")
    ap.add_argument("--skip-ppo", action="store_true", help="no on-device PPO leg")
    ap.add_argument("--surr-rows", type=int, default=10_000_000, help="surrogate training transitions")
    ap.add_argument("--surr-steps", type=int, default=60000, help="surrogate Adam steps")
    args = ap.parse_args()
    global PROFILE_STEPS
    PROFILE_STEPS = args.profile_steps
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        main_reference(args)
    else:
        main_ours(args)


if __name__ == "__main__":
    main()
