"""Benchmark of one explicit lattice step on the large hollow ball drop
(spherical shell of outer radius 100 voxels and thickness 8: 926,584 voxels,
E 0.5 MPa, rho 1100, nu 0.45, dropped at 2 m/s from 5 voxels above the floor,
floor contact and surface-voxel self-collision on, anchor-offset FP32 state).

One bench "step" is one simulation step of the whole lattice: the fused step
kernel (bonds, gather, voxel contacts, floor, integration, collision horizon)
and the candidate-rebuild launch (which rebuilds when the horizon says so and
otherwise returns at once).  The drop is first advanced untimed to step 350,
just before the impact (about step 370), so that the warm-up and timed steps
cover the impact, the contacts and the rebuilds.  The state is close to the
L2 size, so the timed loop writes a 256 MB buffer between steps (L2 flush)
and times every step with CUDA events on the simulator's stream; `value` is
voxel-steps per second over the K timed steps.  The line also carries the
same kind of measurement on the heterogeneous actuated block and on a
lattice larger than L2 (hollow shell R 200, t 8), and the step forms.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload instead.  Under torchrun every rank runs
an independent replica (the plain step of one lattice is not sharded across
GPUs).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1212_2845_gb300 import scenes  # noqa: E402

METRIC = "voxel-steps/s"
WORKLOAD = "hollow_ball_R100_t8 drop (floor + self-collision, anchor-offset FP32 state)"
B_ALG = 108  # algorithmic bytes per voxel-step for this workload (state r/w 104, flags 2, material 1,
             # bond mask 1); bond results and candidate lists are not algorithmic traffic
PRE_STEPS = 350  # untimed set-up: the drop advanced to just before the impact (about step 370)


KERNEL_SOURCES = ("paper_1212_2845_gb300/csrc/vx_pipe.cu", "paper_1212_2845_gb300/csrc/vx_dev.cuh")


def kernel_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(workload_key):
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    or None when the kernel sources changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(workload_key)
    if not e or e.get("kernel_hash") != kernel_hash():
        return None
    return e["dram_bytes_per_launch"]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.times = []
        self.proc = None
        self.w0, self.w1 = None, None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])
            self.times.append(time.perf_counter())

    def start_window(self, timeout=2.0):
        """Waits (up to timeout s) for the sampler's first row, then opens the
        window whose rows the summary keeps."""
        t0 = time.perf_counter()
        while self.proc and not self.rows and time.perf_counter() - t0 < timeout:
            time.sleep(0.01)
        self.w0 = time.perf_counter()

    def end_window(self):
        self.w1 = time.perf_counter()

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.t.join(timeout=2)

    def summary(self):
        rows = self.rows
        if self.w0 is not None and self.w1 is not None:  # rows taken while the timed region ran
            rows = [r for r, t in zip(self.rows, self.times) if self.w0 <= t <= self.w1 + 0.1]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), ws


def host_cpu():
    """Model name and online core count of the host (reported beside the oracle timing)."""
    model = platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"model": model, "nproc": os.cpu_count()}


def cpu_baseline(sc, steps=20):
    """The FP64 oracle (single thread) on a bounded sample of the same
    workload: the first `steps` steps of the full ball drop from rest."""
    from oracle import Oracle
    o = Oracle(sc)
    t0 = time.perf_counter()
    o.step(steps)
    t = time.perf_counter() - t0
    return {"value": o.N * steps / t, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"{WORKLOAD}: the first {steps} steps from rest of the full {o.N}-voxel ball, FP64, "
                      f"1 thread, {t:.1f} s (creation and the initial candidate search not timed)",
            "host": host_cpu()}


def oracle_per_config(seconds=4.0):
    """The oracle (single thread) on a bounded sample of each other
    configuration: the cantilever, the heterogeneous block, a 64-body subset
    of the population and one design body."""
    from oracle import Oracle
    out = {}
    for name, sc in (("cantilever_10x10x10", scenes.cantilever()),
                     ("hetero_block_64x64x32", scenes.hetero_block()),
                     ("population_64", scenes.population(n_bodies=64)),
                     ("design_population_1x12^3", scenes.design_population(n_bodies=1))):
        o = Oracle(sc)
        n = 0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < seconds:
            o.step(1)
            n += 1
        t = time.perf_counter() - t0
        out[name] = {"voxels": o.N, "steps": n, "value": o.N * n / t, "unit": METRIC, "steps_per_s": n / t}
    return out


# Each step of the reference arm: one oracle step of a bounded sample of the
# workload, a hollow ball of outer radius 8 and thickness 4 built by the same
# recipe (material, drop height and speed, floor, self-collision), so that the
# requested steps end within seconds to a few minutes at the oracle's rate
# (which hardly depends on the size).
REF_SAMPLE = {"R": 8, "t": 4}


def run_reference(args):
    rank, _, ws = dist_env()
    if rank != 0:
        return
    from oracle import Oracle
    o = Oracle(scenes.hollow_ball(**REF_SAMPLE))
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(1)
    t = time.perf_counter() - t0
    v = o.N * args.steps / t
    sample = (f"each step: one FP64 oracle step of a hollow ball R{REF_SAMPLE['R']} t{REF_SAMPLE['t']} of the same "
              f"recipe ({o.N} voxels, floor + self-collision); {args.steps} steps after {args.warmup} warm-up, 1 thread")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_voxels": o.N, "sample_bonds": o.n_bonds},
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": sample,
                             "host": host_cpu()},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(x, device):
    """The largest x over the ranks of the process group (x itself with one
    rank): the job's time is its slowest replica's.  Ends with a barrier."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def time_steps(sim, stream, steps, warmup, flush=None):
    """Per-step CUDA-event times (s) of `steps` single-step launches."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            if flush is not None:
                flush.fill_(0.0)
            sim.step_async(1, stream)
    stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for i in range(steps):
            if flush is not None:
                flush.fill_(float(i & 1))      # evicts the lattice from L2 between steps
            ev[i][0].record(stream)
            sim.step_async(1, stream)
            ev[i][1].record(stream)
    stream.synchronize()
    st, _, _ = sim.status(stream)
    if st != 0:
        raise RuntimeError(f"simulation reported status {st}")
    return np.array([a.elapsed_time(b) for a, b in ev]) * 1e-3


def large_lattice(stream, peak, steps=200, warmup=5, R=200, tile=0):
    """Plain step on a hollow shell of outer radius R (200: 3.86M voxels, state
    ~400 MB per step, larger than L2) and thickness 8 voxels, on the floor."""
    from paper_1212_2845_gb300 import vx
    sc = scenes.hollow_ball(R=R, t=8, collide=False)
    sim = vx.Sim(sc)
    if tile:
        sim.set_step_form(vx.FORM_PIPELINED, tile)
    t = time_steps(sim, stream, steps, warmup)
    avg = float(t.mean())
    b_alg = 108  # state r/w 104, flags 2, material 1, bond mask 1
    out = {"workload": f"hollow_shell_R{R}_t8 (plain step, fused kernel, no self-collision)", "voxels": sim.N,
           "bonds": sim.n_bonds, "value": sim.N / avg, "unit": METRIC, "ms_per_step": avg * 1e3,
           "bond_steps_per_s": sim.n_bonds / avg,
           "l2": "inputs larger than L2",
           "roofline": {"bound": "hbm", "achieved": b_alg * sim.N / avg / 1e9, "peak": peak, "unit": "GB/s",
                        "frac": b_alg * sim.N / avg / 1e9 / peak, "bytes_per_voxel_step": b_alg,
                        "kernel": "fused_pipe<256, 1> (lean: one body, no contacts)",
                        "traffic": measured_traffic("hollow_shell_R200_t8") if R == 200 else None}}
    sim.close()
    return out


def _events_time(stream, fn):
    """Seconds taken on `stream` by what fn() enqueues (CUDA events)."""
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    fn()
    b.record(stream)
    stream.synchronize()
    return a.elapsed_time(b) * 1e-3


def batched_form(stream, peak, n_bodies=4096, steps=200, warmup=5):
    """Population of independent bodies (edges U{4..24}, seed 4): the plain
    per-step launches against the autotuned batched form replayed as one
    captured launch of `steps` steps.  State ~0.47 GB: larger than L2."""
    from paper_1212_2845_gb300 import vx
    sc = scenes.population(n_bodies=n_bodies)
    sim = vx.Sim(sc)
    N = sim.N
    b_alg = 112
    sim.step(warmup)
    t_plain = _events_time(stream, lambda: sim.step_async(steps, stream))
    st0 = sim.status(stream)[0]
    tm, gv, rate = sim.autotune_batching(20, stream)
    if gv <= 0:                      # per-step launches or the resident form won: time the batched launch too
        sim.set_batching(4096)
    sim.graph_capture(steps, stream)
    sim.graph_launch(stream)         # warm-up replay
    t_graph = _events_time(stream, lambda: sim.graph_launch(stream))
    st1 = sim.status(stream)[0]
    t_res = None
    try:
        sim.set_batching(vx.GROUPS_RESIDENT)
        sim.graph_capture(steps, stream)
        sim.graph_launch(stream)
        t_res = _events_time(stream, lambda: sim.graph_launch(stream))
        st1 = st1 or sim.status(stream)[0]
    except vx.VxError:
        pass
    if st0 or st1:
        raise RuntimeError("population became unstable")
    out = {"workload": f"population_{n_bodies} (edges U{{4..24}}, seed 4)", "voxels": N, "bonds": sim.n_bonds,
           "steps": steps, "l2": "inputs larger than L2", "bytes_per_voxel_step": b_alg,
           "per_step": {"value": N * steps / t_plain, "unit": METRIC, "ms_per_step": 1e3 * t_plain / steps,
                        "bond_steps_per_s": sim.n_bonds * steps / t_plain,
                        "frac": b_alg * N * steps / t_plain / 1e9 / peak, "kernel": "fused_pipe<256, 5-8> (lean: actuated, per-voxel phase)"},
           "batched": {"value": N * steps / t_graph, "unit": METRIC, "ms_per_step": 1e3 * t_graph / steps,
                       "bond_steps_per_s": sim.n_bonds * steps / t_graph,
                       "frac": b_alg * N * steps / t_graph / 1e9 / peak, "kernel": f"batched_pipe<{sim.tiling()['tile_max']}>",
                       "launch": "one captured CUDA graph replay", "group_voxels": gv if gv else 4096},
           "autotune": {"tile_max": tm, "group_voxels": gv, "sample_voxel_steps_per_s": rate, "sample_steps": 20}}
    if t_res is not None:
        out["resident"] = {"value": N * steps / t_res, "unit": METRIC, "ms_per_step": 1e3 * t_res / steps,
                           "frac": b_alg * N * steps / t_res / 1e9 / peak, "kernel": "res_pipe (thread per voxel)",
                           "launch": "one captured CUDA graph replay"}
    sim.close()
    return out


def adjoint_form(stream, peak, n_bodies=1024, steps=2000, K=100):
    """Design population (n_bodies x 12^3, per-voxel log E and phase, seed 5):
    the plain per-step launches against the adjoint rollout (forward with
    checkpoints every K steps + backward with recomputation) over `steps`."""
    import torch
    from paper_1212_2845_gb300 import vx
    sc = scenes.design_population(n_bodies=n_bodies, steps=steps)
    sim = vx.Sim(sc)
    N = sim.N
    sim.step(5)
    t_plain = _events_time(stream, lambda: sim.step_async(200, stream)) / 200 * steps
    sim.set_batching(vx.GROUPS_RESIDENT)
    sim.step_async(200, stream)
    t_res = _events_time(stream, lambda: sim.step_async(200, stream)) / 200 * steps
    sim.set_batching(0)
    sim.reset(sc["v0"])
    gE = torch.empty(N, device="cuda")
    gP = torch.empty(N, device="cuda")
    with torch.cuda.stream(stream):
        sim.rollout_forward(steps, K, stream)          # warm-up: allocations, kernel preparation
        sim.rollout_backward(gE, gP, stream=stream)
        sim.reset(sc["v0"])
        t_fwd = _events_time(stream, lambda: sim.rollout_forward(steps, K, stream))
        t_bwd = _events_time(stream, lambda: sim.rollout_backward(gE, gP, stream=stream))
    b_fwd, b_bwd = 116, 290
    out = {"workload": f"design_population_{n_bodies}x12^3 (log E, phase per voxel, seed 5)", "voxels": N,
           "bonds": sim.n_bonds, "steps": steps, "checkpoint_every": K, "l2": "inputs larger than L2",
           "plain_step": {"value": N * steps / t_plain, "unit": METRIC, "ms_per_step": 1e3 * t_plain / steps,
                          "bond_steps_per_s": sim.n_bonds * steps / t_plain,
                          "frac": b_fwd * N * steps / t_plain / 1e9 / peak},
           "resident_step": {"value": N * steps / t_res, "unit": METRIC, "ms_per_step": 1e3 * t_res / steps,
                             "frac": b_fwd * N * steps / t_res / 1e9 / peak,
                             "kernel": "res_pipe (thread per voxel, 200 steps per launch)"},
           "rollout_forward": {"value": N * steps / t_fwd, "unit": METRIC, "s": t_fwd},
           "backward": {"value": N * steps / t_bwd, "unit": METRIC, "s": t_bwd,
                        "bond_steps_per_s": sim.n_bonds * steps / t_bwd,
                        "bytes_per_voxel_step": b_bwd, "frac": b_bwd * N * steps / t_bwd / 1e9 / peak,
                        "kernels": "fused_pipe<256> (recompute) + finish_adj + adj_tile<256>"},
           "gradient": {"value": N * steps / (t_fwd + t_bwd), "unit": METRIC,
                        "cost_vs_plain_rollout": (t_fwd + t_bwd) / t_plain}}
    sim.close()
    return out


def collision_form(stream, steps=600):
    """Hollow ball drop (shell R 100, t 8: 926,584 voxels) with floor contact
    and surface-voxel self-collision on, from the start through the impact
    (about step 370): per-step launches including the horizon update, the
    device-flagged candidate rebuilds and the voxel contacts; the cost of one
    forced rebuild is timed on its own."""
    from paper_1212_2845_gb300 import vx
    sc = scenes.hollow_ball(R=100, t=8)
    sim = vx.Sim(sc)
    N = sim.N
    n0, _ = sim.collision_stats()
    t_run = _events_time(stream, lambda: sim.step_async(steps, stream))
    if sim.status(stream)[0]:
        raise RuntimeError("ball drop reported a bad status")
    n1, _ = sim.collision_stats()
    pairs = len(sim.collision_pairs())
    sim.rebuild_collisions(stream)
    t_reb = _events_time(stream, lambda: sim.rebuild_collisions(stream))
    out = {"workload": "hollow_ball_R100_t8 drop (floor + self-collision)", "voxels": N, "bonds": sim.n_bonds,
           "surface_voxels": sim.n_surface, "steps": steps, "value": N * steps / t_run, "unit": METRIC,
           "bond_steps_per_s": sim.n_bonds * steps / t_run,
           "us_per_step": 1e6 * t_run / steps, "rebuilds_in_run": n1 - n0,
           "us_per_forced_rebuild": 1e6 * t_reb, "candidate_pairs_at_end": pairs,
           "bytes_per_voxel_step": 108, "l2": "inputs larger than L2"}
    sim.close()
    return out


def rebuild_sizes(stream, reps=20):
    """Forced candidate rebuilds (flag every body, rebuild, wait) on lattices
    from the clapper to the R100 ball: the query runs one warp per searched
    voxel while the grid has a warp for every 8 of them, else one thread."""
    from paper_1212_2845_gb300 import vx
    out = {}
    for name, mk, all_v in (("clapper_surface", scenes.clapper, False), ("clapper_all_voxels", scenes.clapper, True),
                            ("shell_R12_t3", lambda: scenes.hollow_ball(R=12, t=3), False),
                            ("shell_R20_t4", lambda: scenes.hollow_ball(R=20, t=4), False),
                            ("shell_R40_t4", lambda: scenes.hollow_ball(R=40, t=4), False),
                            ("shell_R100_t8", lambda: scenes.hollow_ball(R=100, t=8), False)):
        sim = vx.Sim(mk())
        sim.set_collision_scheme(all_v, False)
        sim.rebuild_collisions(stream)
        t = _events_time(stream, lambda: [sim.rebuild_collisions(stream) for _ in range(reps)]) / reps
        out[name] = {"searched_voxels": sim.N if all_v else sim.n_surface, "us_per_rebuild": 1e6 * t}
        sim.close()
    return out


def collision_schemes(stream, steps=2000):
    """The paper's comparison of collision schemes on a synthetic clapper
    (880 voxels, arms closing and touching during the run): candidates among
    all voxels or surface voxels only, rebuilt every step or when the horizon
    accumulator requires it.  Iteration rate of each scheme over the same
    steps (per-step launches)."""
    from paper_1212_2845_gb300 import vx
    sc = scenes.clapper()
    out = {"workload": "clapper (880 voxels, 2 bilayer arms, +-10 K, contact during the run)", "steps": steps}
    for name, all_voxels, every in (("all+every", True, True), ("surf+every", False, True),
                                    ("all+horizon", True, False), ("surf+horizon", False, False)):
        sim = vx.Sim(sc)
        sim.set_collision_scheme(all_voxels, every)
        n0, _ = sim.collision_stats()
        t = _events_time(stream, lambda: sim.step_async(steps, stream))
        if sim.status(stream)[0]:
            raise RuntimeError("clapper reported a bad status")
        n1, _ = sim.collision_stats()
        out[name] = {"steps_per_s": steps / t, "us_per_step": 1e6 * t / steps, "rebuilds": n1 - n0}
        sim.close()
    return out


def small_lattice(stream, steps=1000):
    """Cantilever 10x10x10 (1,000 voxels, 4 tiles): latency-bound.  Per-step
    launches, one cooperative multi-step launch (grid barrier between steps),
    the resident form (the lattice in the shared memory of a cluster of 8
    CTAs for all steps of the launch; the default for vx_step(n > 1) at this
    size) and one captured persistent batched launch (the body in one CTA)."""
    from paper_1212_2845_gb300 import vx
    sc = scenes.cantilever()
    sim = vx.Sim(sc)
    sim.step(10)
    sim.set_multistep(0)
    t_plain = _events_time(stream, lambda: sim.step_async(steps, stream))
    sim.set_multistep(2)
    sim.step_async(steps, stream)
    t_multi = _events_time(stream, lambda: sim.step_async(steps, stream))
    sim.set_multistep(1)
    sim.step_async(steps, stream)
    t_res = _events_time(stream, lambda: sim.step_async(steps, stream))
    sim.set_batching(1 << 20)
    sim.graph_capture(steps, stream)
    sim.graph_launch(stream)
    t_graph = _events_time(stream, lambda: sim.graph_launch(stream))
    if sim.status(stream)[0]:
        raise RuntimeError("cantilever became unstable")
    out = {"workload": "cantilever_10x10x10", "voxels": sim.N, "steps": steps,
           "per_step_launches": {"steps_per_s": steps / t_plain, "us_per_step": 1e6 * t_plain / steps},
           "multi_step_launch": {"steps_per_s": steps / t_multi, "us_per_step": 1e6 * t_multi / steps},
           "resident_launch": {"steps_per_s": steps / t_res, "us_per_step": 1e6 * t_res / steps,
                               "kernel": "res_pipe (cluster of 8 CTAs, thread per bond)"},
           "captured_batched_launch": {"steps_per_s": steps / t_graph, "us_per_step": 1e6 * t_graph / steps}}
    sim.close()
    return out


def multi_step_line(sim, stream, flush, steps=500):
    """The same lattice stepped by one call of `steps` steps (one cooperative
    launch on this size), L2 flushed before the call."""
    sim.set_multistep(2)
    sim.step_async(steps, stream)
    flush.fill_(3.0)
    t = _events_time(stream, lambda: sim.step_async(steps, stream))
    if sim.status(stream)[0]:
        raise RuntimeError("simulation reported a bad status")
    return {"us_per_step": 1e6 * t / steps, "value": sim.N * steps / t, "unit": METRIC, "steps_per_call": steps,
            "l2": "flushed before each call; the lattice stays in L2 across the steps of a call"}


def hetero_block_line(stream, peak, flush, steps=2000, warmup=10):
    """The heterogeneous actuated block (64 x 64 x 32 sites, seed 2; 117,907
    voxels, about 13 MB of state): per-step launches with the L2 flushed
    between steps, then the same lattice stepped by one call of 500 steps."""
    from paper_1212_2845_gb300 import vx
    sim = vx.Sim(scenes.hetero_block())
    t = time_steps(sim, stream, steps, warmup, flush)
    avg = float(t.mean())
    b_alg = 112  # state r/w 104, flags 2, material 1, bond mask 1, phase 4
    out = {"workload": "hetero_block_64x64x32 (plain step, floor, actuation)", "voxels": sim.N,
           "bonds": sim.n_bonds, "value": sim.N / avg, "unit": METRIC, "ms_per_step": avg * 1e3,
           "bond_steps_per_s": sim.n_bonds / avg, "l2": "flushed between steps",
           "roofline": {"bound": "hbm", "achieved": b_alg * sim.N / avg / 1e9, "peak": peak, "unit": "GB/s",
                        "frac": b_alg * sim.N / avg / 1e9 / peak, "bytes_per_voxel_step": b_alg,
                        "kernel": "fused_pipe<256, 5-8> (lean: actuated, per-voxel phase)", "traffic": measured_traffic("hetero_block_64x64x32")},
           "multi_step_call": multi_step_line(sim, stream, flush)}
    sim.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--only-large", action="store_true",
                    help="time only the large-shell plain step (profiling aid)")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched / adjoint / small-lattice lines")
    ap.add_argument("--only-adjoint", action="store_true", help="time only the adjoint form (profiling aid)")
    ap.add_argument("--only-batched", action="store_true", help="time only the batched form (profiling aid)")
    ap.add_argument("--only-collisions", action="store_true", help="time only the ball drop with collisions")
    ap.add_argument("--only-small", action="store_true", help="time only the small-lattice forms")
    ap.add_argument("--only-hetero", action="store_true", help="time only the heterogeneous block (profiling aid)")
    ap.add_argument("--tile", type=int, default=0, help="tile size of the pipelined step (profiling aid; 0: default)")
    ap.add_argument("--pre-steps", type=int, default=PRE_STEPS,
                    help="untimed steps of the drop before the warm-up (profiling aid: 0 starts in the free fall)")
    ap.add_argument("--bodies", type=int, default=0, help="bodies for --only-adjoint / --only-batched")
    ap.add_argument("--shell-radius", type=int, default=200, help="outer radius of the --only-large shell")
    ap.add_argument("--form-steps", type=int, default=0, help="steps for --only-adjoint / --only-batched")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    rank, local_rank, ws = dist_env()
    torch.cuda.set_device(local_rank)
    if args.only_large:
        peak, _ = load_peaks()
        print(json.dumps(large_lattice(torch.cuda.Stream(), peak, steps=args.steps, warmup=args.warmup,
                                       R=args.shell_radius, tile=args.tile)))
        return
    if args.only_adjoint:
        peak, _ = load_peaks()
        print(json.dumps(adjoint_form(torch.cuda.Stream(), peak, n_bodies=args.bodies or 1024,
                                      steps=args.form_steps or 2000)))
        return
    if args.only_collisions:
        st = torch.cuda.Stream()
        print(json.dumps({"ball": collision_form(st, steps=args.form_steps or 600),
                          "schemes": collision_schemes(st), "rebuilds": rebuild_sizes(st)}))
        return
    if args.only_batched:
        peak, _ = load_peaks()
        print(json.dumps(batched_form(torch.cuda.Stream(), peak, n_bodies=args.bodies or 4096,
                                      steps=args.form_steps or 200)))
        return
    if args.only_small:
        print(json.dumps(small_lattice(torch.cuda.Stream())))
        return
    if args.only_hetero:
        peak, _ = load_peaks()
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        print(json.dumps(hetero_block_line(torch.cuda.Stream(), peak, flush, steps=args.steps, warmup=args.warmup)))
        return
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1212_2845_gb300 import vx

    sc = scenes.hollow_ball()
    sim = vx.Sim(sc)
    if args.tile:
        sim.set_step_form(vx.FORM_PIPELINED, args.tile)
    stream = torch.cuda.Stream()
    sim.step(args.pre_steps, stream)          # untimed set-up: the drop to just before the impact
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    reb0 = sim.collision_stats()[0]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        clk.start_window()
        t_wall0 = time.perf_counter()
        times = time_steps(sim, stream, args.steps, args.warmup, flush)
        t_wall = time.perf_counter() - t_wall0
        torch.cuda.synchronize()
        clk.end_window()
    rebuilds = sim.collision_stats()[0] - reb0
    t_steps = max_over_ranks(float(times.sum()), "cuda")
    value = ws * sim.N * args.steps / t_steps
    avg = t_steps / args.steps

    # end to end through the C ABI with host buffers: state in, one step, state out
    N = sim.N
    pin = {k: torch.empty(shape, dtype=dt).pin_memory() for k, shape, dt in
           (("offset", (N, 3), torch.float32), ("quat", (N, 4), torch.float32), ("vel", (N, 3), torch.float32),
            ("angvel", (N, 3), torch.float32), ("flags", (N,), torch.uint8))}
    sim.read_state_into(**pin, stream=stream, on_device=False)
    nb = sum(t.numel() * t.element_size() for t in pin.values())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        sim.write_state_from(**pin, stream=stream, on_device=False, wait=False)
        sim.step_async(1, stream)              # the read below waits for the upload and the step
        sim.read_state_into(**pin, stream=stream, on_device=False)
    t_e2e = time.perf_counter() - t0
    if sim.status(stream)[0] != 0:
        raise RuntimeError("end-to-end run reported an unstable state")

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    peak, peak_kind = load_peaks()
    achieved = B_ALG * N / avg / 1e9
    p0 = args.pre_steps
    window = (f"steps {p0 + args.warmup}..{p0 + args.warmup + args.steps} of the 20,000-step drop "
              f"(steps 0..{p0} untimed set-up, then {args.warmup} warm-up; impact near step 370)")
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": avg * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "voxels": N, "bonds": sim.n_bonds, "surface_voxels": sim.n_surface,
                   "window": window, "candidate_rebuilds_in_window": rebuilds, "l2": "flushed between steps",
                   "parallelism": "replicas" if ws > 1 else "single",
                   "bond_steps_per_s": ws * sim.n_bonds * args.steps / t_steps, "wall_s": t_wall},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": measured_traffic("hollow_ball_R100_t8"),
                     "traffic_source": "stored ncu capture of the same kernel source (null when it changed)",
                     "kernel": "fused_pipe<256, 2> (lean: contacts, one body) + rebuild_all (every launch of a step, rebuilds included)",
                     "bytes_per_voxel_step": B_ALG, "peak_kind": peak_kind},
        "e2e": {"value": N * args.e2e_steps / t_e2e, "unit": METRIC, "h2d_bytes_per_step": nb,
                "d2h_bytes_per_step": nb, "steps": args.e2e_steps},
        "gpu_launches": 2 * (args.steps + args.warmup),
        "clocks": clk.summary(),
    }
    if not args.no_large:
        line["large_lattice"] = large_lattice(stream, peak)
    if not args.no_forms:
        line["forms"] = {"hetero_block": hetero_block_line(stream, peak, flush),
                         "batched": batched_form(stream, peak), "adjoint": adjoint_form(stream, peak),
                         "collisions": collision_form(stream),
                         "collision_schemes": collision_schemes(stream),
                         "collision_rebuilds": rebuild_sizes(stream),
                         "small_lattice": small_lattice(stream)}
    sim.close()
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sc)
        if not args.no_forms:
            line["cpu_baseline"]["other_configs"] = oracle_per_config()
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
