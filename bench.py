#!/usr/bin/env python3
"""Benchmark of batched HJCD-IK (arXiv 2510.07514) on GB300.

One step = the whole method over one batch: seeds -> PO-CCD -> top-K and
duplication -> PJ-IK -> collision filter -> ranking (one launch per phase),
for 1000 target poses x 1000 seeds of the 7-DoF Panda with 60 link spheres in
a scene of 200 spheres and 20 boxes.  Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hjcd|reference]

`--impl reference` times the FP64 CPU oracle (the reference of this build) on
the host cores for the same metric, each step a bounded sample of targets.
Under torchrun every rank runs its own replica; rank 0 prints.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "IK solves/s and candidates/s at 1 mm/0.01 rad; p50/p99 latency, served vs plain"
UNIT = "solves/s"
WORKLOAD = ("Panda 7-DoF (modified DH), 1000 targets x 1000 seeds in one batched launch per phase; "
            "60 link spheres (r 0.04-0.08 m); scene of 200 spheres (r 0.02-0.15 m) + 20 boxes in a 1.5 m cube; "
            "targets = FK of uniform in-limit samples kept collision-free; FP32")
DATA = "synthetic: seeded generators (no datasets or trained weights involved)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("hjcd", "reference"), default="hjcd")
    ap.add_argument("--targets", type=int, default=1000)
    ap.add_argument("--seeds", type=int, default=1000)
    ap.add_argument("--top-k", type=int, default=1)
    ap.add_argument("--cpu-sample", type=int, default=96, help="targets in the timed oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--uneven-steps", type=int, default=3, help="timed steps of the uneven 8-chain batch (0: skip)")
    ap.add_argument("--large-steps", type=int, default=2,
                    help="timed steps of the large case, 10000 targets x 4096 seeds (0: skip)")
    ap.add_argument("--large-budget-gb", type=float, default=2.0, help="workspace budget of the large case (waves)")
    ap.add_argument("--large-targets", type=int, default=10000, help="targets of the large case (profiling: fewer)")
    ap.add_argument("--dof-scaling", type=int, default=1, help="run the 7/12/18/24-DoF leg (0: skip)")
    ap.add_argument("--ccd-baseline", type=int, default=1,
                    help="also time the main workload with the position-only CCD initialiser (0: skip)")
    ap.add_argument("--tracking-frames", type=int, default=200, help="frames of the tracking loop (0: skip)")
    ap.add_argument("--latency", type=int, default=1, help="single-target latency leg (0: skip)")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the served Poisson trace at 2000 req/s (0: skip the serving comparison)")
    ap.add_argument("--serve-repeats", type=int, default=3,
                    help="repeats of the plain path's sweep around the served p99")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# distributed plumbing (replicas: one process per GPU, no data-path collective)

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, backend):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend)
    return dist


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device])
        else:
            dist.barrier()


def max_over_ranks(dist, value, device):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        # nvidia-smi takes a moment to start: the timed region begins after its first sample
        t0 = time.perf_counter()
        while not self.lines and time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
            time.sleep(0.01)
        self.lines.clear()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
# algorithmic FP32 work per unit (FMA = 2 flops), counted from the kernels'
# arithmetic for an n-joint chain; see the design notes for the derivation

def flops_ccd_iter(n):
    # per joint: the kinematics step 49 and both trials 203; per iteration: the flange, error
    # quaternion and residual 120, the acceptance's two-joint composition 178, the update 3
    # (ncu's FP32 instruction counters give 2054 per Panda iteration against the 2065 counted)
    return 252 * n + 301


def flops_lm_iter(n):
    return 173 * n + 410


def flops_fk_trial(n):
    return 56 * n + 166


FLOPS_COORD_TRIAL = 108  # PJ-IK single-coordinate trial in closed form (rotation about one axis)
FLOPS_SPHERE_TEST = 10
FLOPS_BOX_TEST = 8


def flops_collide_cand(n, n_sph):
    return 18 * n_sph + 54 * n + 63


def _strip_comments(src: str) -> str:
    """C++ source without its comments, trailing blanks and blank lines (the kernel sources hold
    no comment markers inside string literals)."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


def kernel_source_hash():
    """sha256 of the device code (csrc/k_*.cu and the shared *.cuh, comments and blank lines
    removed), first 12 hex digits: a committed ncu figure counts only while it matches."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2510_07514_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if (f.startswith("k_") and f.endswith(".cu")) or f.endswith(".cuh"):
            h.update(f.encode() + b"\0")
            h.update(_strip_comments(open(os.path.join(csrc, f), encoding="utf-8").read()).encode())
    return h.hexdigest()[:12]


def recorded_fp32_ops(kernel: str):
    """FP32 flops per iteration that ncu's instruction counters measured for the kernel, if taken
    on the current kernel sources (Panda, the 320-target case)."""
    path = os.path.join(ROOT, "profiles", "fp32_ops.txt")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash()
    for ln in open(path):
        f = ln.split()
        if len(f) >= 4 and not ln.startswith("#") and f[0] == kernel and f[3] == src:
            return float(f[1])
    return None


def recorded_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash()
    for ln in open(path):
        f = ln.split()
        if len(f) >= 3 and not ln.startswith("#") and f[0] == kernel and f[2] == src:
            return float(f[1])
    return None


# ----------------------------------------------------------------------------

def step_config(args, world: int) -> dict:
    """The workload of one step, the same for both arms (the reference arm times a bounded sample
    of it and says so in its cpu_baseline)."""
    return {"workload": WORKLOAD, "targets": args.targets, "seeds_per_target": args.seeds, "top_k": args.top_k,
            "tolerance": "1 mm / 0.01 rad", "l2": "flushed between timed steps (256 MB write)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def cpu_baseline(sample_targets: int, seeds: int) -> dict:
    """The FP64 oracle, as it stands, on the host cores: a bounded sample of
    the same workload (its own FK and collision checks choose the targets)."""
    import oracle as orc
    from paper_2510_07514_gb300 import inputs
    wl = inputs.cfg2(sample_targets, seeds)
    rob, sc = orc.Robot(wl.robot), orc.Scene(wl.scene)
    pool = wl.theta_gen.astype(np.float32).astype(np.float64)
    hit, _ = orc.collide(rob, sc, pool)
    keep = pool[~hit][:sample_targets]
    tg = orc.pose(rob, keep).astype(np.float32).astype(np.float64)
    P = orc.make_params(wl.eps_pos, wl.eps_ori, seed=wl.seed)
    t0 = time.perf_counter()
    o = orc.solve(rob, sc, P, tg, seeds, 1)
    dt = time.perf_counter() - t0
    succ = float(np.mean((o["count"] > 0) & (o["err"][:, 0, 0] <= wl.eps_pos) & (o["err"][:, 0, 1] <= wl.eps_ori)))
    return {"value": len(tg) / dt, "unit": UNIT, "cores": orc.threads(), "kind": "oracle",
            "sample": f"{len(tg)} targets x {seeds} seeds of the same workload, FP64, OpenMP over candidates",
            "seconds": dt, "success_rate": succ}


def reference_arm(args):
    world, rank, _ = dist_env()
    dist = dist_init(world, "gloo")
    if rank != 0:
        barrier(dist)
        return
    import oracle as orc
    from paper_2510_07514_gb300 import inputs
    sample = max(1, min(args.cpu_sample // 4, args.targets))
    wl = inputs.cfg2(sample * (args.steps + args.warmup), args.seeds)
    rob, sc = orc.Robot(wl.robot), orc.Scene(wl.scene)
    pool = wl.theta_gen.astype(np.float32).astype(np.float64)
    hit, _ = orc.collide(rob, sc, pool)
    keep = pool[~hit]
    tg_all = orc.pose(rob, keep[: sample * (args.steps + args.warmup)]).astype(np.float32).astype(np.float64)
    P = orc.make_params(wl.eps_pos, wl.eps_ori, seed=wl.seed)
    times, succ = [], []
    for s in range(args.warmup + args.steps):
        tg = tg_all[s * sample:(s + 1) * sample]
        t0 = time.perf_counter()
        o = orc.solve(rob, sc, P, tg, args.seeds, args.top_k)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            succ.append(np.mean((o["count"] > 0) & (o["err"][:, 0, 0] <= wl.eps_pos) & (o["err"][:, 0, 1] <= wl.eps_ori)))
    value = sample * len(times) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": DATA,
        "config": step_config(args, world),
        "success_rate": float(np.mean(succ)),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": orc.threads(), "kind": "oracle",
                         "sample": f"{sample} of the {args.targets} targets x {args.seeds} seeds per step "
                                   "(a bounded sample of the workload; value scaled to solves/s)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    barrier(dist)


def collision_free_targets(ctx, rid, sid, rob, pool, count, dev):
    """FK of the first `count` joint samples of `pool` the library finds collision-free."""
    import torch
    th = torch.as_tensor(np.ascontiguousarray(pool.T), dtype=torch.float32, device=dev)
    hit = ctx.collide(rid, sid, th).bool() if len(rob.sph_body) else torch.zeros(th.shape[1], dtype=torch.bool,
                                                                                  device=dev)
    keep = th[:, ~hit][:, :count].contiguous()
    return ctx.fk(rid, keep).contiguous(), int(keep.shape[1]), float((~hit).float().mean())


def uneven_leg(ctx, args, dev, stream):
    """The uneven batch: 8 random chains x 500 targets, per-target seed counts
    log-uniform in [32, 4096], one scene, packed into one launch per phase."""
    import torch
    from paper_2510_07514_gb300 import hjcd, inputs
    wl = inputs.cfg3()
    sid = ctx.set_scene(wl.scene)
    items, outs, accept = [], [], []
    for i, rob in enumerate(wl.robots):
        rid = ctx.add_robot(rob)
        tg, got, acc = collision_free_targets(ctx, rid, sid, rob, wl.pools[i], wl.n_targets, dev)
        accept.append(acc)
        if got < wl.n_targets:
            return {"skipped": f"chain {i}: only {got} collision-free samples of {len(wl.pools[i])}"}
        it, out = ctx.batch_item(rid, sid, tg, 1, 1, wl.seed + i, rob.n, wl.eps_pos, wl.eps_ori,
                                 samples_per_target=wl.samples[i])
        items.append(it)
        outs.append(out)
    C = int(sum(int(s.sum()) for s in wl.samples))
    T = wl.n_targets * len(wl.robots)
    for _ in range(2):
        ctx.solve_batch(items, stream=stream)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.uneven_steps):
        ctx.solve_batch(items, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.uneven_steps
    # the same batch captured as one CUDA graph; host wall time per step, direct call vs replay
    g = hjcd.hjcd_graph_create(ctx.h, items)
    try:
        hjcd.hjcd_graph_launch(ctx.h, g, stream)
        torch.cuda.synchronize(dev)
        wall = {"direct": [], "graph": []}
        for _ in range(args.uneven_steps):
            t0 = time.perf_counter()
            l0 = hjcd.hjcd_launch_count(ctx.h)
            ctx.solve_batch(items, stream=stream)
            launches_step = hjcd.hjcd_launch_count(ctx.h) - l0
            torch.cuda.synchronize(dev)
            wall["direct"].append(time.perf_counter() - t0)
            t0 = time.perf_counter()
            hjcd.hjcd_graph_launch(ctx.h, g, stream)
            torch.cuda.synchronize(dev)
            wall["graph"].append(time.perf_counter() - t0)
        hjcd.hjcd_graph_check(ctx.h, g)
    finally:
        hjcd.hjcd_graph_destroy(g)
    succ = []
    for out in outs:
        c, e = out[2].cpu().numpy(), out[1].cpu().numpy()
        succ.append((c > 0) & (e[:, 0, 0] <= wl.eps_pos) & (e[:, 0, 1] <= wl.eps_ori))
    # autotuned: launch configuration and iteration caps from a calibration batch (the first 48
    # targets of each chain, other seeds), then the whole batch again, timed, with the picks
    cal = []
    for i, it in enumerate(items):
        c_it = hjcd.hjcd_batch_item.from_buffer_copy(it)
        c_it.n_targets = 48
        c_it.opts.seed = wl.seed + 1000 + i
        cal.append(c_it)
    t0 = time.perf_counter()
    tuned, rep = hjcd.hjcd_autotune(ctx.h, cal, None, 0.01, 3)
    tune_s = time.perf_counter() - t0
    items_t = []
    for it in items:
        t_it = hjcd.hjcd_batch_item.from_buffer_copy(it)
        t_it.opts.params = hjcd.ct.pointer(tuned)
        items_t.append(t_it)
    ctx.solve_batch(items_t, stream=stream)
    e0.record(stream)
    for _ in range(args.uneven_steps):
        ctx.solve_batch(items_t, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_t = e0.elapsed_time(e1) / args.uneven_steps
    succ_t = []
    for out in outs:
        c, e = out[2].cpu().numpy(), out[1].cpu().numpy()
        succ_t.append((c > 0) & (e[:, 0, 0] <= wl.eps_pos) & (e[:, 0, 1] <= wl.eps_ori))
    hjcd.hjcd_set_launch_config(ctx.h, 64, 8)  # the defaults
    tuned_line = {"ccd_block": rep.ccd_block, "lm_warps": rep.lm_warps, "cd_max_iters": rep.cd_max_iters,
                  "lm_max_iters": rep.lm_max_iters, "calibration_success": rep.success_rate,
                  "calibration_best_success": rep.best_success_rate, "trials": rep.trials, "tune_s": tune_s,
                  "ms_per_step": ms_t, "solves_per_s": (wl.n_targets * len(wl.robots)) / (ms_t * 1e-3),
                  "success_rate": float(np.mean(np.concatenate(succ_t)))}
    return {"workload": wl.name, "dofs": [r.n for r in wl.robots], "link_spheres": [len(r.sph_body) for r in wl.robots],
            "targets": T, "seeds": C, "ms_per_step": ms, "solves_per_s": T / (ms * 1e-3),
            "candidates_per_s": C / (ms * 1e-3), "success_rate": float(np.mean(np.concatenate(succ))),
            "collision_free_fraction_of_samples": accept,
            "wall_ms_direct": 1e3 * float(np.median(wall["direct"])),
            "wall_ms_graph_replay": 1e3 * float(np.median(wall["graph"])),
            "launches_per_step": int(launches_step), "autotuned": tuned_line}


def large_leg(ctx, args, dev, stream):
    """10 000 targets x 4096 seeds of the Panda with 60 link spheres, top-16,
    against 5000 obstacle spheres on a jittered grid carved (by the library's
    contact query) around the target configurations; memory-admitted waves."""
    import torch
    from paper_2510_07514_gb300 import hjcd, inputs
    wl = inputs.cfg5(n_targets=args.large_targets)
    rob = wl.robot
    rid = ctx.add_robot(rob)
    pool = torch.as_tensor(np.ascontiguousarray(wl.target_pool.T), dtype=torch.float32, device=dev)
    self_hit = ctx.collide(rid, -1, pool).bool()
    keep = pool[:, ~self_hit][:, :wl.n_targets].contiguous()
    T = int(keep.shape[1])
    nodes_sid = ctx.set_scene(inputs.Scene(wl.nodes, np.zeros((0, 6))))
    touched = torch.empty(len(wl.nodes), dtype=torch.uint8, device=dev)
    hjcd.hjcd_scene_contacts(ctx.h, rid, nodes_sid, T, keep, keep.stride(0), touched)
    free = wl.nodes[~touched.bool().cpu().numpy()][:wl.n_obstacles]
    sid = ctx.set_scene(inputs.Scene(free, np.zeros((0, 6))))
    tg = ctx.fk(rid, keep).contiguous()
    K, S = wl.top_k, wl.n_samples
    out = (torch.empty((T, K, rob.n), device=dev), torch.empty((T, K, 2), device=dev),
           torch.empty((T,), dtype=torch.int32, device=dev))
    budget = int(args.large_budget_gb * 2 ** 30)
    hjcd.hjcd_set_memory_budget(ctx.h, budget)
    try:
        ctx.solve(rid, sid, tg, S, K, wl.seed, rob.n, stream=stream, out=out)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        hjcd.hjcd_counters(ctx.h, reset=True)
        e0.record(stream)
        for _ in range(args.large_steps):
            ctx.solve(rid, sid, tg, S, K, wl.seed, rob.n, stream=stream, out=out)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        cnt = hjcd.hjcd_counters(ctx.h, reset=True)
    finally:
        hjcd.hjcd_set_memory_budget(ctx.h, 0)
    ms = e0.elapsed_time(e1) / args.large_steps
    c, e = out[2].cpu().numpy(), out[1].cpu().numpy()
    succ = (c > 0) & (e[:, 0, 0] <= wl.eps_pos) & (e[:, 0, 1] <= wl.eps_ori)
    # phase split: the same solve in one wave (its whole workspace, about 2.6 GB, fits the device)
    # with the phases' events recorded; the roofline of its dominant kernel from the work counters
    hjcd.hjcd_set_profiling(ctx.h, True)
    ctx.solve(rid, sid, tg, S, K, wl.seed, rob.n, stream=stream, out=out)
    torch.cuda.synchronize(dev)
    hjcd.hjcd_counters(ctx.h, reset=True)
    w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0.record(stream)
    ctx.solve(rid, sid, tg, S, K, wl.seed, rob.n, stream=stream, out=out)
    w1.record(stream)
    torch.cuda.synchronize(dev)
    ph = np.asarray(hjcd.hjcd_phase_times(ctx.h), dtype=float)
    cw = hjcd.hjcd_counters(ctx.h, reset=True)
    names = ["po_ccd", "topk_dup", "pjik", "collide", "rank"]
    ph_c = ph.copy()
    ph_c[3] += ph_c[4]  # the ranked collision filter runs in the rank phase
    ph_c[4] = 0.0
    n, n_sph = rob.n, len(rob.sph_body)
    fl = {"po_ccd": cw[0] * flops_ccd_iter(n),
          "pjik": cw[1] * flops_lm_iter(n) + (cw[2] - cw[1]) * flops_fk_trial(n) + cw[7] * FLOPS_COORD_TRIAL,
          "collide": cw[3] * FLOPS_SPHERE_TEST + cw[6] * FLOPS_BOX_TEST + cw[4] * flops_collide_cand(n, n_sph)}
    sm_max = 2070.0
    props = torch.cuda.get_device_properties(dev)
    peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    dom = max(fl, key=lambda k: ph_c[names.index(k)])
    dom_ms = ph_c[names.index(dom)]
    achieved = fl[dom] / (dom_ms * 1e-3) / 1e12
    roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None,
            "peak_note": f"FP32 CUDA-core peak from unit counts: {props.multi_processor_count} SMs x 128 lanes x 2 "
                         f"x {sm_max:.0f} MHz",
            "per_kernel": {k: {"ms": float(ph_c[names.index(k)]), "gflop": fl[k] / 1e9,
                               "tflops": fl[k] / max(ph_c[names.index(k)] * 1e-3, 1e-12) / 1e12} for k in fl}}
    # end to end with host buffers (pinned), within the workspace budget (waves), copies inside
    tg_h = tg.cpu().pin_memory()
    hout = (torch.empty((T, K, rob.n)).pin_memory(), torch.empty((T, K, 2)).pin_memory(),
            torch.empty((T,), dtype=torch.int32).pin_memory())
    hjcd.hjcd_set_memory_budget(ctx.h, budget)
    try:
        e2e = []
        for i in range(2):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            ctx.solve(rid, sid, tg_h, S, K, wl.seed, rob.n, stream=stream, out=hout)
            e2e.append(time.perf_counter() - t0)
    finally:
        hjcd.hjcd_set_memory_budget(ctx.h, 0)
    e2e_s = min(e2e)
    return {"workload": f"Panda + 60 link spheres, {T} targets x {S} seeds, top-{K}; {len(free)} obstacle spheres "
                        f"(jittered grid carved around the target configurations, uniform grid broadphase)",
            "candidates": T * S, "ms_per_step": ms, "solves_per_s": T / (ms * 1e-3),
            "candidates_per_s": T * S / (ms * 1e-3), "success_rate": float(succ.mean()),
            "mean_solutions_per_target": float(c.mean()), "workspace_budget_bytes": budget,
            "sphere_tests_per_candidate": cnt[3] / args.large_steps / max(cnt[4] / args.large_steps, 1),
            "one_wave": {"ms_per_step": w0.elapsed_time(w1),
                         "phase_ms": {nm: float(v) for nm, v in zip(names + ["step"], ph)},
                         "work": {"ccd_iters": cw[0], "lm_iters": cw[1], "lm_fk_passes": cw[2],
                                  "lm_coord_trials": cw[7], "sphere_tests": cw[3], "box_tests": cw[6],
                                  "collide_candidates": cw[4]}},
            "roofline": roof,
            "e2e": {"value": T / e2e_s, "unit": UNIT, "ms_per_step": 1e3 * e2e_s,
                    "h2d_bytes_per_step": T * 7 * 4, "d2h_bytes_per_step": T * K * (rob.n + 2) * 4 + T * 4,
                    "note": "host targets and outputs (pinned), waves within the workspace budget"}}


def dof_scaling_leg(ctx, args, dev, stream):
    """The Panda and its 12/18/24-DoF chained variants in an open world, B = 1000
    seeds per target: single-target latency (one target per call, end to end
    through hjcd_solve with pinned host buffers, median of 30) and batched
    throughput (1000 targets x 1000 seeds, one launch per phase)."""
    import torch
    from paper_2510_07514_gb300 import inputs
    rng = np.random.default_rng(inputs.CFG_SEED[1] + 77)
    out = {}
    for dof in inputs.DOF_SCALING:
        rob = inputs.dof_scaling_robot(dof)
        rid = ctx.add_robot(rob)
        th = torch.as_tensor(np.ascontiguousarray(rng.uniform(rob.lo, rob.hi, (1000, dof)).T), dtype=torch.float32,
                             device=dev)
        tg = ctx.fk(rid, th).contiguous()
        tg_h = tg.cpu().pin_memory()
        h1 = (torch.empty((1, 1, dof)).pin_memory(), torch.empty((1, 1, 2)).pin_memory(),
              torch.empty((1,), dtype=torch.int32).pin_memory())
        lat = []
        for i in range(35):
            t0 = time.perf_counter()
            ctx.solve(rid, -1, tg_h[i % 100:i % 100 + 1], 1000, 1, 1000 + i, dof, out=h1)
            if i >= 5:
                lat.append(1e3 * (time.perf_counter() - t0))
        outs = (torch.empty((1000, 1, dof), device=dev), torch.empty((1000, 1, 2), device=dev),
                torch.empty((1000,), dtype=torch.int32, device=dev))
        ctx.solve(rid, -1, tg, 1000, 1, 7, dof, stream=stream, out=outs)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            ctx.solve(rid, -1, tg, 1000, 1, 7, dof, stream=stream, out=outs)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / 3
        c, e = outs[2].cpu().numpy(), outs[1].cpu().numpy()
        succ = (c > 0) & (e[:, 0, 0] <= 1e-3) & (e[:, 0, 1] <= 1e-2)
        out[str(dof)] = {"single_target_latency_ms_p50": float(np.median(lat)),
                         "single_target_latency_ms_p90": float(np.percentile(lat, 90)),
                         "batch_1000x1000_ms": ms, "solves_per_s": 1000 / (ms * 1e-3),
                         "success_rate": float(succ.mean()),
                         "median_pos_err_m": float(np.median(e[succ, 0, 0])) if succ.any() else None,
                         "median_ori_err_rad": float(np.median(e[succ, 0, 1])) if succ.any() else None}
    return out


def tracking_leg(ctx, args, dev):
    """The tracking loop: every frame the obstacles move (the resident scene is
    rewritten), the target moves along a circle, and one target x 1000 seeds is
    solved with the solutions ranked nearest to the current configuration
    (hjcd_solve_nearest); the arm moves to the first one.  Frame latency is host
    wall time of scene update + solve with pinned host buffers.  The same frames
    ranked by score show how much the nearest ranking smooths the motion."""
    import torch
    from paper_2510_07514_gb300 import inputs
    rob = inputs.panda_with_spheres(np.random.default_rng(inputs.CFG_SEED[2]))
    rid = ctx.add_robot(rob)
    rng = np.random.default_rng(inputs.CFG_SEED[2] + 5)
    q_home = np.array([0.0, -0.4, 0.0, -2.0, 0.0, 1.8, 0.8])
    home = ctx.fk(rid, torch.as_tensor(q_home[:, None], dtype=torch.float32, device=dev)).cpu().numpy()[0]
    ang = rng.uniform(0, 2 * np.pi, 24)
    base = np.stack([0.75 * np.cos(ang), 0.75 * np.sin(ang), rng.uniform(0.2, 1.1, 24),
                     rng.uniform(0.04, 0.08, 24)], 1)
    sid = ctx.set_scene(inputs.Scene(base, np.zeros((0, 6))))
    F = args.tracking_frames
    res = {}
    for mode in ("nearest", "score"):
        q_cur = torch.as_tensor(q_home[None], dtype=torch.float32).pin_memory()
        tgt = torch.empty((1, 7)).pin_memory()
        out = (torch.empty((1, 1, 7)).pin_memory(), torch.empty((1, 1, 2)).pin_memory(),
               torch.empty((1,), dtype=torch.int32).pin_memory())
        lat, steps, ok = [], [], 0
        for f in range(F):
            ph = 2 * np.pi * f / F
            obs = base.copy()
            obs[:, 2] += 0.05 * np.sin(ph * 3 + np.arange(24))
            pose = home.copy()
            pose[0] += 0.12 * np.cos(ph) - 0.12
            pose[1] += 0.12 * np.sin(ph)
            tgt[0] = torch.as_tensor(pose)
            t0 = time.perf_counter()
            ctx.set_scene(inputs.Scene(obs, np.zeros((0, 6))), sid)
            ctx.solve(rid, sid, tgt, 1000, 1, 100 + f, 7, out=out, q_current=q_cur if mode == "nearest" else None)
            lat.append(1e3 * (time.perf_counter() - t0))
            c, e = int(out[2][0]), out[1][0, 0].numpy()
            if c > 0 and e[0] <= 1e-3 and e[1] <= 1e-2:
                ok += 1
                steps.append(float(torch.max(torch.abs(out[0][0, 0] - q_cur[0]))))
                q_cur[0] = out[0][0, 0]
        res[mode] = {"frame_ms_p50": float(np.median(lat[5:])), "frame_ms_p99": float(np.percentile(lat[5:], 99)),
                     "success_rate": ok / F, "joint_step_rad_median": float(np.median(steps)) if steps else None,
                     "joint_step_rad_max": float(np.max(steps)) if steps else None}
    res["frames"] = F
    res["workload"] = ("Panda + 60 link spheres, 24 obstacle spheres moving every frame, target on a 0.12 m circle, "
                       "1 target x 1000 seeds per frame")
    return res


PAPER_CONTEXT = {
    "hardware": "NVIDIA GeForce RTX 4060 laptop GPU (sm_89), per the paper; other hardware, context only",
    "ms_per_solve_B1000": {"panda_open_world": 4.22, "panda_box_panda_collision_free": 5.04,
                           "dof_7": 4.25, "dof_12": 4.55, "dof_18": 4.62, "dof_24": 4.66},
    "note": "the paper reports wall time per solve (one target, B polished seeds); no throughput",
}


def latency_leg(ctx, args, dev):
    """One target, 1000 seeds, top-1, end to end through hjcd_solve with pinned
    host buffers (the paper's per-solve timing shape): the Panda in the open
    world, and the Panda with 60 link spheres in the main workload's scene."""
    import torch
    from paper_2510_07514_gb300 import inputs
    wl = inputs.cfg2(64, 1000)
    out = {}
    for name, rob, scene in (("panda_open_world", inputs.panda(), None),
                             ("panda_spheres_in_scene", wl.robot, wl.scene)):
        rid = ctx.add_robot(rob)
        sid = ctx.set_scene(scene) if scene is not None else -1
        tg, got, _ = collision_free_targets(ctx, rid, sid, rob, wl.theta_gen[:2000], 64, dev)
        tg_h = tg.cpu().pin_memory()
        h1 = (torch.empty((1, 1, 7)).pin_memory(), torch.empty((1, 1, 2)).pin_memory(),
              torch.empty((1,), dtype=torch.int32).pin_memory())
        lat, ok = [], 0
        for i in range(70):
            t0 = time.perf_counter()
            ctx.solve(rid, sid, tg_h[i % got:i % got + 1], 1000, 1, 500 + i, 7, out=h1)
            if i >= 10:
                lat.append(1e3 * (time.perf_counter() - t0))
                e = h1[1][0, 0].numpy()
                ok += int(h1[2][0] > 0 and e[0] <= 1e-3 and e[1] <= 1e-2)
        out[name] = {"ms_p50": float(np.median(lat)), "ms_p99": float(np.percentile(lat, 99)),
                     "success_rate": ok / len(lat)}
    out["paper"] = PAPER_CONTEXT
    return out


def _serve_run(ctx, reqs, trace, idx, rate_scale, server_kw):
    """Submit requests idx at the trace's arrival times (divided by rate_scale)
    to a server started with server_kw; per-request latency and throughput."""
    from paper_2510_07514_gb300 import hjcd
    hjcd.hjcd_server_start(ctx.h, **server_kw)
    ids, t_sub = [], []
    try:
        t0 = time.perf_counter()
        base = trace.t[idx[0]] / rate_scale
        for k in idx:
            due = t0 + trace.t[k] / rate_scale - base
            while True:
                now = time.perf_counter()
                if now >= due:
                    break
                if due - now > 2e-3:
                    time.sleep(due - now - 1e-3)
            t_sub.append(time.perf_counter())
            ids.append(hjcd.hjcd_submit(ctx.h, reqs[k][0]))
        infos = [hjcd.hjcd_wait(ctx.h, i, 600.0) for i in ids]
    finally:
        hjcd.hjcd_server_stop(ctx.h)
    lat = np.array([inf.total_ms for inf in infos])
    done = np.array(t_sub) + lat / 1e3
    span = float(done.max() - t_sub[0])
    T = int(sum(trace.n_targets[k] for k in idx))
    ok = all(inf.status == 0 for inf in infos)
    succ = []
    for k in idx:
        c, e = reqs[k][1][2].numpy(), reqs[k][1][1].numpy()
        succ.append((c > 0) & (e[:, 0, 0] <= 1e-3) & (e[:, 0, 1] <= 1e-2))
    return {"requests": len(idx), "offered_req_per_s": float(len(idx) / max(trace.t[idx[-1]] / rate_scale - base, 1e-9)),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "solves_per_s": T / span, "req_per_s": len(idx) / span,
            "mean_batch_requests": float(np.mean([inf.batch_requests for inf in infos])),
            "success_rate": float(np.mean(np.concatenate(succ))), "all_ok": ok}


def _crossing(points, target):
    """Offered rate (and throughput) where p99 reaches `target` on a sweep of
    (rate, p99, solves/s) points: log-linear interpolation between the fastest
    point at or below the target and the next faster one; None when no point
    meets the target."""
    pts = sorted(points)
    ok = [q for q in pts if q[1] <= target]
    if not ok:
        return None
    lo = max(ok)
    up = [q for q in pts if q[0] > lo[0] and q[1] > target]
    if not up:
        return {"rate": lo[0], "solves_per_s": lo[2], "bracketed": False}
    hi = min(up)
    f = (target - lo[1]) / (hi[1] - lo[1])
    rate = float(np.exp(np.log(lo[0]) + f * (np.log(hi[0]) - np.log(lo[0]))))
    sps = float(np.exp(np.log(lo[2]) + f * (np.log(hi[2]) - np.log(lo[2]))))
    return {"rate": rate, "solves_per_s": sps, "bracketed": True}


def serving_leg(ctx, args, dev):
    """Served (continuous batching) vs plain (one request per launch sequence)
    on the Poisson trace of 1-8 targets x 32-4096 seeds requests for four
    resident chains, each request with its own 0-500-sphere scene.

    The served path runs the whole trace at 2000 requests/s.  The plain path is
    swept: halved rates on short runs until its p99 is no worse than the served
    p99 (the bracket), then rates 1.25x apart across the bracket with at least
    2000 requests each, repeated on other stretches of the trace; in each repeat
    the rate (and throughput) at which the plain p99 equals the served p99 is
    interpolated, and served/plain solves/s at equal p99 is its ratio.  Both
    paths are also run at 2x and 4x the offered rate (their ceilings)."""
    import torch
    from paper_2510_07514_gb300 import api, inputs
    chains = inputs.cfg3_chains()
    rids = [ctx.add_robot(chains[i]) for i in inputs.CFG4_ROBOTS]
    tpls = inputs.cfg4_templates()
    banks = []
    for tp in tpls:
        sid = ctx.set_scene(tp.scene)
        rob = chains[inputs.CFG4_ROBOTS[tp.robot]]
        tg, got, _ = collision_free_targets(ctx, rids[tp.robot], sid, rob, tp.pool, 8, dev)
        banks.append(tg.cpu().numpy())
    rate = 2000.0
    trace = inputs.cfg4_trace(rate, args.serve_seconds, len(tpls))
    # templates whose scene leaves no collision-free sample are replaced by the next usable one
    usable = [i for i in range(len(tpls)) if len(banks[i]) > 0]
    reqs = []
    for k in range(len(trace.t)):
        j = int(trace.template[k])
        if len(banks[j]) == 0:
            j = usable[j % len(usable)]
        tp, bank = tpls[j], banks[j]
        T = int(min(trace.n_targets[k], len(bank)))
        trace.n_targets[k] = T
        rob = chains[inputs.CFG4_ROBOTS[tp.robot]]
        tg = torch.as_tensor(np.ascontiguousarray(bank[:T]), dtype=torch.float32)
        reqs.append(ctx.batch_item(rids[tp.robot], -1, tg, int(trace.seeds[k]), 1, int(trace.seed[k]), rob.n,
                                   spheres=tp.scene.sph_xyzr, boxes=None, device=torch.device("cpu")))
    idx = np.arange(len(trace.t))
    served_kw, plain_kw = dict(max_inflight=3), dict(max_inflight=1, max_batch_requests=1)
    served = _serve_run(ctx, reqs, trace, idx, 1.0, served_kw)
    target = served["p99_ms"]
    # bracket: halved rates, short runs
    bracket = []
    scale = 1.0
    for _ in range(8):
        n_req = int(min(len(idx), max(600, rate * scale * 1.5)))
        r = _serve_run(ctx, reqs, trace, idx[:n_req], scale, plain_kw)
        r["rate_scale"] = scale
        bracket.append(r)
        if r["p99_ms"] <= target:
            break
        scale /= 2.0
    # refine: 1.25x steps across [scale, 2 scale], >= 2000 requests per point, on other stretches
    repeats = []
    n_req = int(min(len(idx), max(2000, 2 * rate * scale)))
    for rep in range(max(1, args.serve_repeats)):
        start = (rep * n_req) % max(1, len(idx) - n_req)
        sub = idx[start:start + n_req]
        pts, runs = [], []
        for i in range(1, 5):  # the bracket's low point met the target on a short run
            sc = scale * 1.25 ** i
            r = _serve_run(ctx, reqs, trace, sub, sc, plain_kw)
            r["rate_scale"] = sc
            runs.append(r)
            pts.append((r["offered_req_per_s"], r["p99_ms"], r["solves_per_s"]))
        cross = _crossing(pts, target)
        repeats.append({"runs": runs, "crossing": cross,
                        "served_over_plain": served["solves_per_s"] / cross["solves_per_s"] if cross else None})
    ratios = [r["served_over_plain"] for r in repeats if r["served_over_plain"]]
    med = float(np.median(ratios)) if ratios else None
    # ceilings: both paths at 2x and 4x the offered rate
    ceilings = {}
    for mult in (2.0, 4.0):
        n_c = int(min(len(idx), 2 * rate * mult))
        ceilings[f"{mult:g}x"] = {
            "served": _serve_run(ctx, reqs, trace, idx[:n_c], mult, served_kw),
            "plain": _serve_run(ctx, reqs, trace, idx[:min(n_c, 3000)], mult, plain_kw)}
    return {"trace": f"Poisson {rate:.0f} req/s for {args.serve_seconds:g} s ({len(idx)} requests); 1-8 targets, "
                     "32-4096 seeds, 4 resident chains (7/12/16/20 DoF), own scene of 0-500 spheres per request",
            "templates_usable": f"{len(usable)} of {len(tpls)}",
            "served": served, "plain_bracket": bracket, "plain_repeats": repeats,
            "served_over_plain_at_equal_p99": med,
            "served_over_plain_spread": (float((max(ratios) - min(ratios)) / med) if ratios else None),
            "plain_reached_served_p99": bool(ratios), "ceilings": ceilings}


def hjcd_arm(args):
    world, rank, local = dist_env()
    import torch
    from paper_2510_07514_gb300 import api, build, hjcd, inputs
    if not os.path.exists(hjcd.lib_path()):
        build.build()
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    wl = inputs.cfg2(args.targets, args.seeds)
    rob = wl.robot
    n, T, S, K = rob.n, args.targets, args.seeds, args.top_k
    ctx = api.Context(local)
    rid, sid = ctx.add_robot(rob), ctx.set_scene(wl.scene)

    # targets: the library's own FK of joint samples its own collision check keeps
    pool = torch.as_tensor(np.ascontiguousarray(wl.theta_gen.T), dtype=torch.float32, device=dev)
    hit = ctx.collide(rid, sid, pool).bool()
    keep = pool[:, ~hit][:, :T].contiguous()
    assert keep.shape[1] == T, "not enough collision-free joint samples in the pool"
    tg = ctx.fk(rid, keep).contiguous()
    tg_host = tg.cpu().pin_memory()
    out = (torch.empty((T, K, n), device=dev), torch.empty((T, K, 2), device=dev),
           torch.empty((T,), dtype=torch.int32, device=dev))
    hout = (torch.empty((T, K, n)).pin_memory(), torch.empty((T, K, 2)).pin_memory(),
            torch.empty((T,), dtype=torch.int32).pin_memory())
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def step(targets, outs):
        ctx.solve(rid, sid, targets, S, K, wl.seed, n, wl.eps_pos, wl.eps_ori, stream=stream, out=outs)

    hjcd.hjcd_set_profiling(ctx.h, True)
    for _ in range(args.warmup):
        flush.zero_()
        step(tg, out)
    torch.cuda.synchronize(dev)

    hjcd.hjcd_counters(ctx.h, reset=True)
    l0 = hjcd.hjcd_launch_count(ctx.h)
    clocks = ClockSampler(local)
    clocks.start()
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    phases = []
    barrier(dist, local)
    torch.cuda.synchronize(dev)
    for i in range(args.steps):
        flush.zero_()
        e0[i].record(stream)
        step(tg, out)
        e1[i].record(stream)
        phases.append(hjcd.hjcd_phase_times(ctx.h))
    torch.cuda.synchronize(dev)
    barrier(dist, local)
    clk = clocks.stop()
    launches = hjcd.hjcd_launch_count(ctx.h) - l0
    ms = [a.elapsed_time(b) for a, b in zip(e0, e1)]
    cnt = hjcd.hjcd_counters(ctx.h, reset=True)
    total_s = max_over_ranks(dist, sum(ms) / 1e3, dev)
    value = world * T * args.steps / total_s

    cnt_h, err_h = out[2].cpu().numpy(), out[1].cpu().numpy()
    success = float(np.mean((cnt_h > 0) & (err_h[:, 0, 0] <= wl.eps_pos) & (err_h[:, 0, 1] <= wl.eps_ori)))

    # end to end through the C ABI with host buffers (copies inside the region)
    e2e_ms = []
    for i in range(max(2, args.steps // 2) + 1):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        step(tg_host, hout)
        t1 = time.perf_counter()
        if i > 0:
            e2e_ms.append(1e3 * (t1 - t0))
    e2e_total = max_over_ranks(dist, sum(e2e_ms) / 1e3, dev)
    e2e_value = world * T * len(e2e_ms) / e2e_total
    h2d = T * 7 * 4 + 2 * (T + 1) * 8
    d2h = T * K * (n + 2) * 4 + T * 4

    # roofline of the dominant kernel
    ph_raw = np.mean(np.asarray(phases), axis=0)  # ccd, dup, lm, collide, rank, whole
    names = ["po_ccd", "topk_dup", "pjik", "collide", "rank"]
    steps = args.steps
    n_sph = len(rob.sph_body)
    fl = {
        "po_ccd": cnt[0] / steps * flops_ccd_iter(n),
        "pjik": cnt[1] / steps * flops_lm_iter(n) + (cnt[2] - cnt[1]) / steps * flops_fk_trial(n)
                + cnt[7] / steps * FLOPS_COORD_TRIAL,
        "collide": (cnt[3] * FLOPS_SPHERE_TEST + cnt[6] * FLOPS_BOX_TEST) / steps
                   + cnt[4] / steps * flops_collide_cand(n, n_sph),
    }
    props = torch.cuda.get_device_properties(dev)
    sm_max = clk.get("sm_max_mhz") or 2070.0
    peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    # with the ranked collision filter (default) the collision work runs inside the rank phase
    ph = np.array(ph_raw, dtype=float)
    ph[names.index("collide")] += ph[names.index("rank")]
    ph[names.index("rank")] = 0.0
    dom = int(np.argmax(ph[:5]))
    dom_name = names[dom] if names[dom] in fl else max(fl, key=lambda k: fl[k] / max(ph[names.index(k)], 1e-9))
    dom_ms = ph[names.index(dom_name)]
    achieved = fl[dom_name] / (dom_ms * 1e-3) / 1e12
    roof = {"bound": "alu", "kernel": dom_name, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": recorded_traffic(dom_name),
            "peak_note": f"FP32 CUDA-core peak from unit counts: {props.multi_processor_count} SMs x 128 lanes x 2 "
                         f"x {sm_max:.0f} MHz (max SM clock); no FP32 peak in MEASURED_PEAKS.json",
            "per_kernel": {k: {"ms": float(ph[names.index(k)]), "gflop": fl[k] / 1e9,
                               "tflops": fl[k] / (ph[names.index(k)] * 1e-3) / 1e12} for k in fl}}
    ffma = hjcd.hjcd_ffma_probe(ctx.h, 2048, stream)
    # the same against the FP32 rate an FFMA loop measures on this GPU in this run (of measured)
    roof["frac_of_measured_ffma"] = achieved / ffma if ffma > 0 else None
    # and by the coarser pre-implementation estimate of a PO-CCD iteration, 210 n flops (FK 90 n and
    # 2n trials of about 60 flops), which leaves out part of what each trial computes
    if dom_name == "po_ccd":
        ach_s = cnt[0] / steps * 210 * n / (dom_ms * 1e-3) / 1e12
        roof["by_coarse_count"] = {"flop_per_iter": 210 * n, "achieved": ach_s, "frac": ach_s / peak}
        # and by the FP32 operations ncu counted per iteration on these kernel sources (Panda)
        meas = recorded_fp32_ops("po_ccd") if n == 7 else None
        if meas:
            ach_m = cnt[0] / steps * meas / (dom_ms * 1e-3) / 1e12
            roof["by_ncu_fp32_ops"] = {"flop_per_iter": meas, "achieved": ach_m, "frac": ach_m / peak}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(np.mean(ms)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": DATA,
        "config": step_config(args, world),
        "candidates_per_s": value * S, "success_rate": success,
        "phase_ms": {nm: float(v) for nm, v in zip(names + ["step"], ph_raw)},
        "phase_note": "with the ranked collision filter (default) the collision checks run in the rank phase",
        "work_per_step": {"ccd_iters": cnt[0] / steps, "lm_iters": cnt[1] / steps, "lm_fk_passes": cnt[2] / steps,
                          "lm_coord_trials": cnt[7] / steps,
                          "sphere_tests": cnt[3] / steps, "box_tests": cnt[6] / steps,
                          "collide_candidates": cnt[4] / steps},
        "roofline": roof, "ffma_probe_tflops": ffma,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": float(np.mean(e2e_ms))},
        "clocks": clk, "gpu_launches": int(launches),
    }
    if world == 1:
        # the same step with the collision filter over every polished candidate (mode 0) instead of
        # in rank order until top_k are found (mode 1, the default; identical results)
        hjcd.hjcd_set_collision_mode(ctx.h, 0)
        try:
            step(tg, out)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            a0.record(stream)
            for _ in range(3):
                step(tg, out)
            a1.record(stream)
            torch.cuda.synchronize(dev)
            ph_a = hjcd.hjcd_phase_times(ctx.h)
        finally:
            hjcd.hjcd_set_collision_mode(ctx.h, 1)
        line["collision_all_candidates"] = {
            "ms_per_step": a0.elapsed_time(a1) / 3, "solves_per_s": T / (a0.elapsed_time(a1) / 3 * 1e-3),
            "phase_ms_last_step": {nm: float(v) for nm, v in zip(names + ["step"], ph_a)}}
    if world == 1 and args.ccd_baseline:
        # the same step with the position-only CCD (Alg. 1) in place of PO-CCD (Alg. 3)
        pb = api.make_params(cd_variant=1)
        ctx.solve(rid, sid, tg, S, K, wl.seed, n, wl.eps_pos, wl.eps_ori, params=pb, stream=stream, out=out)
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        b0.record(stream)
        for _ in range(3):
            ctx.solve(rid, sid, tg, S, K, wl.seed, n, wl.eps_pos, wl.eps_ori, params=pb, stream=stream, out=out)
        b1.record(stream)
        torch.cuda.synchronize(dev)
        ph_b = hjcd.hjcd_phase_times(ctx.h)
        ms_b = b0.elapsed_time(b1) / 3
        cb, eb = out[2].cpu().numpy(), out[1].cpu().numpy()
        # and with the target-wide break (cd_variant 2, lock-step per target)
        p2 = api.make_params(cd_variant=2)
        ctx.solve(rid, sid, tg, S, K, wl.seed, n, wl.eps_pos, wl.eps_ori, params=p2, stream=stream, out=out)
        flush.zero_()
        b0.record(stream)
        for _ in range(3):
            ctx.solve(rid, sid, tg, S, K, wl.seed, n, wl.eps_pos, wl.eps_ori, params=p2, stream=stream, out=out)
        b1.record(stream)
        torch.cuda.synchronize(dev)
        ph_2 = hjcd.hjcd_phase_times(ctx.h)
        c2, e2 = out[2].cpu().numpy(), out[1].cpu().numpy()
        line["ccd_target_break"] = {
            "initialiser": "PO-CCD, all seeds of a target stop at the first convergence (lock-step per target)",
            "ms_per_step": b0.elapsed_time(b1) / 3, "solves_per_s": T / (b0.elapsed_time(b1) / 3 * 1e-3),
            "success_rate": float(np.mean((c2 > 0) & (e2[:, 0, 0] <= wl.eps_pos) & (e2[:, 0, 1] <= wl.eps_ori))),
            "phase_ms_last_step": {nm: float(v) for nm, v in zip(names + ["step"], ph_2)}}
        line["ccd_baseline"] = {
            "initialiser": "position-only CCD (Alg. 1), the rest of Alg. 2 unchanged",
            "ms_per_step": ms_b, "solves_per_s": T / (ms_b * 1e-3),
            "success_rate": float(np.mean((cb > 0) & (eb[:, 0, 0] <= wl.eps_pos) & (eb[:, 0, 1] <= wl.eps_ori))),
            "phase_ms_last_step": {nm: float(v) for nm, v in zip(names + ["step"], ph_b)}}
    if world == 1 and args.uneven_steps > 0:
        line["uneven_batch"] = uneven_leg(ctx, args, dev, stream)
    if world == 1 and args.large_steps > 0:
        line["large"] = large_leg(ctx, args, dev, stream)
    if world == 1 and args.dof_scaling:
        line["dof_scaling"] = dof_scaling_leg(ctx, args, dev, stream)
    if world == 1 and args.latency:
        line["single_target_latency"] = latency_leg(ctx, args, dev)
    if world == 1 and args.tracking_frames > 0:
        line["tracking"] = tracking_leg(ctx, args, dev)
    if world == 1 and args.serve_seconds > 0:
        line["serving"] = serving_leg(ctx, args, dev)
    ctx.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_sample, S)
    if rank == 0:
        print(json.dumps(line), flush=True)
    barrier(dist, local)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        hjcd_arm(args)


if __name__ == "__main__":
    main()
