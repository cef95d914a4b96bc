"""Throughput of one optimizer iteration of per-pixel stochastic gradient estimation.

Workload (the batched-estimator configuration): UV sphere of 8,192 triangles
(64 x 64 segments, 4,034 welded vertices), 512^2 RGB float32 texture, 512^2
render, 8 seeded views on a sphere of radius 3, 64 antithetic pairs per view
per iteration, all in one persistent launch; the whole iteration (estimate +
Adam step, lr = eps as in the paper's Section 5) is captured in a CUDA graph.
Synthetic data: seeded meshes/textures, targets rendered from a seeded target
scene.  A "step" is one such iteration: 8 x 64 x 512^2 = 134,217,728
antithetic pixel pairs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (test infrastructure, single thread) on a
bounded sample of the same workload.  With N > 1 (torchrun) every rank runs an
independent replica (the estimator does not need a collective), and rank 0
prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "antithetic render-pair pixels/s and param-gradients/s vs plain path; HBM GB/s fraction"
UNIT = "pixel-pairs/s"
WORKLOAD = "sphere8k_tex512_r512_8views_x_64pairs"
N_VIEWS, PAIRS, RENDER = 8, 64, 512
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Roofline of the dominant kernel (k_estimate_fast): nothing on the path is a dense contraction
# and it moves about a byte of DRAM per pixel pair, so its roofline is the SMs' lane rate
# (152 SMs x 128 FP32/INT32 lanes x clock).  The work is counted from the method, not from the
# kernel: method_ops() below.  The kernel's own executed instructions per pixel pair (ncu
# smsp__inst_executed x active lanes of the same build) give the issue efficiency beside it.
# Arithmetic of one covered side of a pixel pair (Section 4.3 R, Algorithm 2 G), in 32-bit
# operations: the visible triangle's coverage test (3 edge functions of 2 multiply-adds, 3
# compares), barycentrics (3 conversions, 3 multiplies) and depth (3 multiplies, 2 adds): 20;
# perspective-correct UV (3 + 6 multiplies, 2 + 4 adds, 2 divides): 17; the bilinear footprint
# (per axis a multiply, 2 subtracts, floor, conversion; wrap and clamp): 14; per read texture the
# 4 bilinear weights (6) and per texel channel the perturbed value and its weighted add (2).
OPS_VISIBLE, OPS_UV, OPS_FOOT, OPS_WEIGHTS, OPS_PER_TEXEL_CHANNEL = 20, 17, 14, 6, 2
OPS_SHADE = {0: 0, 1: 55, 2: 125}  # unlit; Lambert with a normal map; GGX + Lambert (per side)
OPS_LOSS_DIFF = 12  # per pixel pair: sum_c (I+ - I-)(I+ + I- - 2I)
OPS_CREDIT = 2      # per contribution: one add to the parameter's sum, one to its count
# One ncu --set full capture of this build's k_estimate_fast<unlit> on this workload (one launch =
# one estimate call, 134.2 M pixel pairs): smsp__inst_executed.sum 5.158 G x 22.74 active lanes =
# 874 thread instructions per pixel pair; dram__bytes_read.sum + dram__bytes_write.sum =
# 164.16 MB + 6.58 MB per launch.  Set to None when the kernel changes until it is captured again.
NCU_INSTR_PER_PIXEL_PAIR = 874.0
NCU_DRAM_BYTES_PER_LAUNCH = 170.74e6


def method_ops(shading: int, read_channels, covered_sides: float, covered_pairs: float, contributions: float):
    """32-bit operations the method performs in one estimate call, from quantities the run
    counts: covered_sides (pixel pairs x sides showing a triangle), covered_pairs (pixel pairs with
    a triangle on either side), contributions (sum over pixel pairs of |K(p)|, from the counts)."""
    per_side = OPS_VISIBLE + OPS_UV + OPS_FOOT + OPS_SHADE[shading] + \
        sum(OPS_WEIGHTS + 4 * c * OPS_PER_TEXEL_CHANNEL for c in read_channels)
    return covered_sides * per_side + covered_pairs * OPS_LOSS_DIFF + contributions * OPS_CREDIT


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def job_throughput(seconds: float, units_per_rank: float, device=None):
    """Whole-job rate of independent replicas: every rank processed units_per_rank in its own
    `seconds`; the job took the slowest rank's time (max over ranks, one all-reduce on the
    process group when there is one), and processed world x units_per_rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    if world > 1:
        t = torch.tensor([seconds], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        seconds = float(t.item())
    return world * units_per_rank / seconds, seconds


def make_scene():
    import synth
    return synth.config_batched(n_views=N_VIEWS, pairs=PAIRS, render=RENDER)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out, _ = self.p.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


_ORACLE = {}


def _oracle_worker_init():
    import oracle
    import synth
    sc = make_scene()
    tg = oracle.render_targets(sc, synth.target_scene(sc))
    _ORACLE["osc"] = oracle.OracleScene(sc, tg)


def _oracle_pairs(args):
    import oracle
    view, first, n = args
    t0 = time.perf_counter()
    # one estimate per pair index: the oracle draws every pair's signs from (seed, iter, view, pair)
    for p in range(first, first + n):
        oracle.estimate(_ORACLE["osc"], 1, p, [view], 1)
    return time.perf_counter() - t0


def cpu_baseline(budget_s: float = 12.0):
    """The oracle (as it stands) on a bounded sample of the workload, on every host core: one
    process per core, each running single-pair estimates of its own view; the sample grows
    until it takes about budget_s of wall time."""
    import multiprocessing as mp
    cores = max(1, os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_oracle_worker_init) as pool:
        pool.map(_oracle_pairs, [(k % N_VIEWS, 0, 1) for k in range(cores)])  # warm: scene + library
        n = 1
        while True:
            t0 = time.perf_counter()
            pool.map(_oracle_pairs, [(k % N_VIEWS, 1000 * k, n) for k in range(cores)])
            dt = time.perf_counter() - t0
            if dt >= budget_s / 3 or n >= 64:
                break
            n = min(64, max(n + 1, int(n * budget_s / 3 / max(dt, 1e-3))))
    px = cores * n * RENDER * RENDER
    return {"value": px / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes x {n} single-pair estimates of one view each at "
                      f"{RENDER}x{RENDER} ({px} pixel pairs), {dt:.1f} s wall"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import synth
    sc = make_scene()
    tg = oracle.render_targets(sc, synth.target_scene(sc))
    osc = oracle.OracleScene(sc, tg)
    for w in range(args.warmup):
        oracle.estimate(osc, 1, w, [w % N_VIEWS], 1)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        oracle.estimate(osc, 1, 100 + k, [k % N_VIEWS], 1)
        times.append(time.perf_counter() - t0)
    per_step = RENDER * RENDER  # one pair of one view per step (a bounded sample of the iteration)
    value = per_step * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "1 pair of 1 view per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} steps x 1 antithetic pair at {RENDER}^2"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    import synth
    from paper_2404_09758_gb300 import STEP_ADAM, IterState, Scene

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev) if "device_id" in dist.init_process_group.__code__.co_varnames \
            else dist.init_process_group("nccl")

    sc = make_scene()
    tgt_scene = Scene.from_arrays(synth.target_scene(sc))
    targets = tgt_scene.render_targets()
    torch.cuda.synchronize()
    del tgt_scene
    g = Scene.from_arrays(sc, targets=targets)
    grad, counts = g.new_grad_buffers()
    m = torch.zeros(g.n_params, device=dev)
    v = torch.zeros(g.n_params, device=dev)
    loss = torch.zeros(N_VIEWS, device=dev)
    views = list(range(N_VIEWS))
    lr_tex = [t[1] for t in g.textures]
    n_total = N_VIEWS * PAIRS
    st = torch.cuda.Stream(device=dev)

    def iteration(it, t):
        # `it` and `t` are host values (eager warm-up) or one IterState in device memory that the
        # captured graph reads and advances, so that every replay is the next iteration
        loss.zero_()
        g.estimate_grad(1, it, views, PAIRS, grad, counts, loss=loss, stream=st)
        # Adam with the paper's settings: beta1 0.9, beta2 0.999, learning rate = eps (Section 5)
        g.step(STEP_ADAM, grad, counts, n_total, sc.eps_pos, lr_tex, m=m, v=v, t=t, stream=st)
        if isinstance(it, IterState):
            it.advance(1, 1, stream=st)

    # contributions of one iteration (parameter gradients credited), counted exactly
    with torch.cuda.stream(st):
        g.estimate_grad(1, 0, views, PAIRS, grad, counts, stream=st)
    st.synchronize()
    contributions = int(counts.to(torch.int64).sum().item())
    touched = int((counts != 0).sum().item())
    grad.zero_()
    counts.zero_()
    assert g.status(st) == 0
    # pixels each view covers (unperturbed render): the method's work per pair and side
    covered_px = 0
    for vw in views:
        k, _, _ = g.render_idb(vw, side=0, stream=st)
        st.synchronize()  # the render runs on st; the count below on the current stream
        covered_px += int((k != -1).sum().item())
    ops_per_step = method_ops(sc.shading, [int(t.data.shape[2]) for t in sc.textures[:1]],
                              2.0 * PAIRS * covered_px, float(PAIRS * covered_px), float(contributions))

    # warm up eagerly, then capture one iteration in a CUDA graph; the iteration index and
    # Adam's step number live in device memory (continuing the warm-up's sequence) and the
    # graph's last node advances them
    for w in range(max(args.warmup, 1)):
        iteration(w, w + 1)
    st.synchronize()
    state = IterState(max(args.warmup, 1), max(args.warmup, 1) + 1, device=dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=st):
        iteration(state, state)
    st.synchronize()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()

    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB of L2
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(st):
                flush.fill_(k & 0xFF)
                ev[k][0].record(st)
                graph.replay()
                ev[k][1].record(st)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    px_per_step = N_VIEWS * PAIRS * RENDER * RENDER
    value, t_total = job_throughput(sum(ms) / 1000.0, px_per_step * args.steps, device=dev)
    assert g.status(st) == 0

    # dominant kernel: the library records CUDA events on `st` around each launch of the fast
    # estimator; the whole estimate call (binning prologue + vertex pass + estimator) is timed too
    ek = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    g.kernel_timing(True)
    with torch.cuda.stream(st):
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            ek[k][0].record(st)
            g.estimate_grad(1, 2000 + k, views, PAIRS, grad, counts, stream=st)
            ek[k][1].record(st)
    torch.cuda.synchronize()
    fast_total_ms, fast_launches = g.kernel_time()
    g.kernel_timing(False)
    fast_ms = fast_total_ms / fast_launches
    est_ms = statistics.mean(a.elapsed_time(b) for a, b in ek)
    grad.zero_()
    counts.zero_()

    # plain path: one estimate after another, separate R and G launches (baseline of the batched path)
    plain_steps = 1
    with torch.cuda.stream(st):
        g.estimate_grad_plain(1, 3000, views, PAIRS, grad, counts, stream=st)  # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for k in range(plain_steps):
            g.estimate_grad_plain(1, 3001 + k, views, PAIRS, grad, counts, stream=st)
        e1.record(st)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1) / plain_steps
    grad.zero_()
    counts.zero_()

    # end to end through the C ABI from pinned host memory (sge_iterate_host): parameters and
    # targets copied in, the estimate, the Adam step and the advance, the updated parameters and
    # the loss copied out, every step
    host_theta = torch.cat([p.detach().reshape(-1) for p in g.param_groups()]).cpu().pin_memory()
    host_targets = targets.reshape(-1).cpu().pin_memory()
    host_theta_out = torch.empty_like(host_theta).pin_memory()
    host_loss = torch.empty(N_VIEWS, pin_memory=True)
    h2d = host_theta.numel() * 4 + host_targets.numel() * 4
    d2h = host_theta_out.numel() * 4 + host_loss.numel() * 4
    e2e_steps = max(1, min(args.steps, 5))
    e2e_state = IterState(5000, 1, device=dev)
    ee = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(e2e_steps)]
    with torch.cuda.stream(st):
        for k in range(e2e_steps):
            flush.fill_(k & 0xFF)
            ee[k][0].record(st)
            g.iterate_host(1, e2e_state, views, PAIRS, grad, counts, m, v, sc.eps_pos, lr_tex, kind=STEP_ADAM,
                           loss_dev=loss, theta_in=host_theta, targets_in=host_targets, theta_out=host_theta_out,
                           loss_out=host_loss, stream=st)
            ee[k][1].record(st)
    torch.cuda.synchronize()
    assert g.status(st) == 0
    e2e_s = sum(a.elapsed_time(b) for a, b in ee) / 1000.0
    e2e_value = world * px_per_step * e2e_steps / e2e_s

    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    clocks = clk.summary()
    sm_clock_mhz = peaks.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    # peak: every SM issues one instruction per lane per cycle on its 128 FP32/INT32 lanes
    peak = n_sm * 128 * sm_clock_mhz * 1e6 / 1e12
    # the method's operations of args.steps iterations over the fast kernel's time (the one launch
    # per call runs every estimate of the call)
    achieved = ops_per_step * args.steps / (fast_total_ms / 1000.0) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T ops/s",
                "frac": achieved / peak,
                "traffic": NCU_DRAM_BYTES_PER_LAUNCH,
                "work": f"{ops_per_step / px_per_step:.1f} method operations per pixel pair (method_ops: "
                        f"{covered_px / (N_VIEWS * RENDER * RENDER):.3f} of the pixels covered, "
                        f"{contributions / px_per_step:.2f} contributions per pixel pair)",
                "kernel": f"k_estimate_fast<unlit>, {fast_ms:.3f} ms per launch (CUDA events around "
                          f"its {fast_launches} launches on the launching stream)",
                "peak_source": f"{n_sm} SMs x 128 lanes x {sm_clock_mhz:.0f} MHz (sm_max_mhz of MEASURED_PEAKS.json)"}
    if NCU_INSTR_PER_PIXEL_PAIR is not None:
        # executed thread instructions (ncu, this build) at the kernel's measured time: how busy the
        # lanes are, wasted work included
        roofline["issue_efficiency"] = NCU_INSTR_PER_PIXEL_PAIR * px_per_step / (fast_ms / 1000.0) / 1e12 / peak
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "views": N_VIEWS, "pairs_per_view": PAIRS,
                       "render": f"{RENDER}x{RENDER}", "triangles": int(sc.pos_idx.shape[0]),
                       "params": int(g.n_params), "l2": "flushed between timed steps (256 MB write)",
                       "graph": "estimate + Adam step + iteration advance captured in one CUDA graph; "
                                "every replay is the next iteration (device-resident iteration index "
                                "and Adam step)",
                       "parallelism": f"replicas x{world}"},
            "param_gradients_per_s": world * contributions * args.steps / t_total,
            "touched_params_per_s": world * touched * args.steps / t_total,
            "contributions_per_step": contributions,
            "estimate_ms": est_ms,
            "fast_kernel_ms": fast_ms,
            "plain_path": {"value": px_per_step / (plain_ms / 1000.0), "unit": UNIT, "ms_per_step": plain_ms,
                           "param_gradients_per_s": contributions / (plain_ms / 1000.0)},
            "batched_over_plain": plain_ms / (1000.0 * t_total / args.steps),
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "api": "sge_iterate_host with pinned host buffers (theta and targets in, theta and loss out)"},
            # per iteration: 3 binning kernels, the pruning pass, the vertex pass, the texel sign
            # planes, the fast and the heavy-bin estimator, the background-loss kernel, the step
            # kernel and the advance
            "gpu_launches": 11 * args.steps,
            "clocks": clocks}
    if rank == 0 and world == 1:
        line["cpu_baseline"] = cpu_baseline()
        if not args.no_sub:
            # the uneven-batch and scale configurations, a few graph replays each (their own
            # workloads give the full lines): ms per iteration and pixel pairs per second
            del graph, g, grad, counts, m, v, flush
            torch.cuda.empty_cache()
            sub = {}
            for name, fn, k in (("uneven32_r512_4views_x_8pairs", measure_uneven, 3),
                                ("gridsphere1m_4x2048_ggx_r2048_16views_x_16pairs", measure_scale, 2)):
                r = fn(k, 3)
                sub[name] = {"ms_per_iteration": r["ms_per_step"], "pixel_pairs_per_s": r["value"],
                             "param_gradients_per_s": r["param_gradients_per_s"], "steps": k,
                             "clocks": r["clocks"]}
                torch.cuda.empty_cache()
            line["sub_results"] = sub
            line["atomic_ceiling"] = {"unit": "fp32 red.global.add per s", **measure_atomics()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_uneven(args):
    print(json.dumps(measure_uneven(args.steps, args.warmup)), flush=True)


def measure_uneven(steps: int, warmup: int):
    """Uneven batch: 32 seeded assets (1K..200K triangles, 256^2..2048^2 RGB textures), each
    at 512^2 from 4 views with 8 antithetic pairs, all estimates in one persistent launch per
    estimator kernel (autotuned launch shape), then an Adam step per asset; the iteration is
    captured in a CUDA graph.  Not the default workload: a second configuration."""
    import torch

    import synth
    from paper_2404_09758_gb300 import STEP_ADAM, Batch, IterState, Scene

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    views_n, pairs, render = 4, 8, 512
    scs = synth.config_uneven(n_views=views_n, pairs=pairs, render=render)
    st = torch.cuda.Stream(device=dev)
    assets = []
    for sc in scs:
        ts = Scene.from_arrays(synth.target_scene(sc), max_pairs_per_call=pairs)
        tg = ts.render_targets()
        torch.cuda.synchronize()
        del ts
        g = Scene.from_arrays(sc, targets=tg, max_pairs_per_call=pairs)
        grad, counts = g.new_grad_buffers()
        assets.append(dict(sc=sc, g=g, grad=grad, counts=counts, loss=torch.zeros(views_n, device=dev),
                           m=torch.zeros(g.n_params, device=dev), v=torch.zeros(g.n_params, device=dev)))
    views = list(range(views_n))
    b = Batch([(a["g"], views, a["grad"], a["counts"], a["loss"]) for a in assets])
    tune_ms = b.autotune(pairs, repeats=2, stream=st)
    with torch.cuda.stream(st):
        b.estimate_grad(1, 0, pairs, stream=st)
    st.synchronize()
    contributions = [int(a["counts"].to(torch.int64).sum().item()) for a in assets]
    for a in assets:
        assert a["g"].status(st) == 0
        a["grad"].zero_()
        a["counts"].zero_()

    def iteration(it, t):
        for a in assets:
            a["loss"].zero_()
        b.estimate_grad(1, it, pairs, stream=st)
        for a in assets:
            a["g"].step(STEP_ADAM, a["grad"], a["counts"], views_n * pairs, a["sc"].eps_pos,
                        [tt[1] for tt in a["g"].textures], m=a["m"], v=a["v"], t=t, stream=st)
        if isinstance(it, IterState):
            it.advance(1, 1, stream=st)

    for w in range(warmup):
        iteration(w, w + 1)
    st.synchronize()
    state = IterState(warmup, warmup + 1, device=dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=st):
        iteration(state, state)
    st.synchronize()
    for _ in range(warmup):
        graph.replay()
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with ClockSampler(local) as clk:
        for k in range(steps):
            with torch.cuda.stream(st):
                flush.fill_(k & 0xFF)
                ev[k][0].record(st)
                graph.replay()
                ev[k][1].record(st)
        torch.cuda.synchronize()
    t_total = sum(a.elapsed_time(c) for a, c in ev) / 1000.0
    px_per_step = len(assets) * views_n * pairs * render * render
    value = px_per_step * steps / t_total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": warmup, "ms_per_step": 1000.0 * t_total / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "uneven32_r512_4views_x_8pairs", "assets": len(assets),
                       "triangles": [int(a["sc"].pos_idx.shape[0]) for a in assets],
                       "texture_sizes": [int(a["sc"].textures[0].data.shape[0]) for a in assets],
                       "l2": "flushed between timed steps (256 MB write)",
                       "graph": "batched estimate + per-asset Adam steps + iteration advance captured in one "
                                "CUDA graph (every replay is the next iteration)",
                       "tuning": {"pairs_per_item": b.tuning.pairs_per_item,
                                  "blocks_per_sm": b.tuning.blocks_per_sm, "light_bin": b.tuning.light_bin,
                                  "autotune_ms": tune_ms}},
            "param_gradients_per_s": sum(contributions) * steps / t_total,
            "contributions_per_asset": contributions,
            # per asset: 3 binning kernels, background loss, vertex pass, texel sign planes, Adam
            # step; per call: the batched pruning pass, the fast and the heavy-bin estimator, the
            # advance
            "gpu_launches": (7 * len(assets) + 4) * steps,
            "clocks": clk.summary()}
    return line


def run_scale(args):
    print(json.dumps(measure_scale(args.steps, args.warmup)), flush=True)


def measure_scale(steps: int, warmup: int):
    """Scale configuration: 1,048,576-triangle displaced grid sphere, four 2048^2 RGB maps,
    GGX with one light, 2048^2 render, 16 views x 16 antithetic pairs per iteration, the
    iteration (estimate + Adam step) captured in a CUDA graph.  A second configuration."""
    import torch

    import synth
    from paper_2404_09758_gb300 import STEP_ADAM, IterState, Scene

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sc = synth.config_scale()
    nv, pairs = sc.n_views, sc.pairs_per_view
    ts = Scene.from_arrays(synth.target_scene(sc))
    targets = ts.render_targets()
    torch.cuda.synchronize()
    del ts
    g = Scene.from_arrays(sc, targets=targets, max_pairs_per_call=pairs)
    grad, counts = g.new_grad_buffers()
    m = torch.zeros(g.n_params, device=dev)
    v = torch.zeros(g.n_params, device=dev)
    loss = torch.zeros(nv, device=dev)
    views = list(range(nv))
    lr_tex = [t[1] for t in g.textures]
    st = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(st):
        g.estimate_grad(1, 0, views, pairs, grad, counts, stream=st)
    st.synchronize()
    contributions = int(counts.to(torch.int64).sum().item())
    assert g.status(st) == 0
    grad.zero_()
    counts.zero_()

    def iteration(it, t):
        loss.zero_()
        g.estimate_grad(1, it, views, pairs, grad, counts, loss=loss, stream=st)
        g.step(STEP_ADAM, grad, counts, nv * pairs, sc.eps_pos, lr_tex, m=m, v=v, t=t, stream=st)
        if isinstance(it, IterState):
            it.advance(1, 1, stream=st)

    for w in range(warmup):
        iteration(w, w + 1)
    st.synchronize()
    state = IterState(warmup, warmup + 1, device=dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=st):
        iteration(state, state)
    st.synchronize()
    graph.replay()
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with ClockSampler(local) as clk:
        for k in range(steps):
            with torch.cuda.stream(st):
                flush.fill_(k & 0xFF)
                ev[k][0].record(st)
                graph.replay()
                ev[k][1].record(st)
        torch.cuda.synchronize()
    t_total = sum(a.elapsed_time(c) for a, c in ev) / 1000.0
    g.kernel_timing(True)
    with torch.cuda.stream(st):
        for k in range(2):
            g.estimate_grad(1, 2000 + k, views, pairs, grad, counts, stream=st)
    fast_ms, fast_n = g.kernel_time()
    g.kernel_timing(False)
    assert g.status(st) == 0
    px_per_step = nv * pairs * sc.width * sc.height
    line = {"metric": METRIC, "value": px_per_step * steps / t_total, "unit": UNIT, "n_gpus": 1,
            "steps": steps, "warmup": warmup, "ms_per_step": 1000.0 * t_total / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "gridsphere1m_4x2048_ggx_r2048_16views_x_16pairs", "views": nv,
                       "pairs_per_view": pairs, "render": f"{sc.width}x{sc.height}",
                       "triangles": int(sc.pos_idx.shape[0]), "params": int(g.n_params),
                       "l2": "inputs larger than L2; 256 MB flush between timed steps",
                       "graph": "estimate + Adam step + iteration advance captured in one CUDA graph "
                                "(every replay is the next iteration)"},
            "param_gradients_per_s": contributions * steps / t_total,
            "contributions_per_step": contributions,
            "fast_kernel_ms": fast_ms / max(fast_n, 1),
            # as the default workload's iteration: 11 kernels
            "gpu_launches": 11 * steps,
            "clocks": clk.summary()}
    return line


def measure_atomics(repeats: int = 5):
    """Ceiling of global float atomics on this GPU (the per-contribution AtomicAdd of Algorithm 2):
    sge_atomic_bench's fire-and-forget fp32 reductions, one address per thread and 1-of-K hot
    addresses, timed with CUDA events (best of `repeats`).  Reductions per second."""
    import torch
    from paper_2404_09758_gb300 import _abi
    L = _abi.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    n_threads, per = 152 * 2048 * 8, 32
    buf = torch.zeros(n_threads, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()
    out = {}
    for name, n_addr in (("distinct", n_threads), ("hot_1_of_32768", 32768), ("hot_1_of_1024", 1024),
                         ("hot_1_of_32", 32), ("hot_1", 1)):
        best = None
        for r in range(repeats + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            _abi.check(L.sge_atomic_bench(buf.data_ptr(), n_addr, n_threads, per, st.cuda_stream))
            e1.record(st)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            if r > 0:
                best = ms if best is None else min(best, ms)
        out[name] = n_threads * per / (best / 1000.0)
    return out


def run_atomics(args):
    import torch
    torch.cuda.set_device(dist_env()[2])
    rates = measure_atomics()
    line = {"metric": "global fp32 atomic reductions per second (ceiling of Algorithm 2's AtomicAdd)",
            "value": rates["distinct"], "unit": "reductions/s", "n_gpus": 1, "steps": 5, "warmup": 1,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": "red_global_add_f32_2.5M_threads_x32"}, "rates": rates}
    print(json.dumps(line), flush=True)


def run_full_image(args):
    """The full-image estimator (Eq. 4 with the whole-image error) on the batched configuration's
    workload (8 views x 64 pairs, 512^2): every estimate renders both sides (staged ID/UV
    buffers), sums f+ - f- over the image, and every parameter is credited dF s_i.  The paper
    shows it converging far slower than the per-pixel form (Section 6.1); it is timed here as
    the comparison estimator, eagerly, one estimate after another."""
    import torch

    import synth
    from paper_2404_09758_gb300 import Scene

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sc = make_scene()
    ts = Scene.from_arrays(synth.target_scene(sc))
    targets = ts.render_targets()
    torch.cuda.synchronize()
    del ts
    g = Scene.from_arrays(sc, targets=targets)
    grad, counts = g.new_grad_buffers()
    views = list(range(N_VIEWS))
    st = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(st):
        for w in range(args.warmup):
            g.estimate_grad_full_image(1, w, views, PAIRS, grad, counts, stream=st)
    st.synchronize()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        with torch.cuda.stream(st):
            for k in range(args.steps):
                flush.fill_(k & 0xFF)
                ev[k][0].record(st)
                g.estimate_grad_full_image(1, 100 + k, views, PAIRS, grad, counts, stream=st)
                ev[k][1].record(st)
        torch.cuda.synchronize()
    assert g.status(st) == 0
    px_per_step = N_VIEWS * PAIRS * RENDER * RENDER
    value, t_total = job_throughput(sum(a.elapsed_time(b) for a, b in ev) / 1000.0, px_per_step * args.steps)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD + "_full_image_estimator", "views": N_VIEWS, "pairs_per_view": PAIRS,
                       "l2": "flushed between timed steps (256 MB write)", "graph": "none (eager)"},
            "param_gradients_per_s": g.n_params * N_VIEWS * PAIRS * args.steps / t_total,
            # per estimate: raster of both sides, loss differences, image sum; per call: binning,
            # the per-parameter accumulation
            "gpu_launches": (3 * N_VIEWS * PAIRS + 4) * args.steps,
            "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_transparent(args):
    """Transparent geometry (Section 4.4): three overlapping semi-transparent 2,048-triangle
    spheres, one 512^2 RGBA albedo, 512^2 render, 8 views x 16 pairs per call.  Each estimate
    keeps both sides' deep ID buffers (four fragments a pixel), composites them front to back and
    credits every listed fragment; one launch runs every estimate of the call."""
    import torch

    import synth
    from paper_2404_09758_gb300 import Scene

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nv, pairs, render = 8, 16, 512
    sc = synth.config_transparent(n_views=nv, pairs=pairs, render=render, tex=512)
    ts = Scene.from_arrays(synth.target_scene(sc))
    targets = ts.render_targets()
    torch.cuda.synchronize()
    del ts
    g = Scene.from_arrays(sc, targets=targets)
    grad, counts = g.new_grad_buffers()
    views = list(range(nv))
    st = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(st):
        g.estimate_grad(1, 0, views, pairs, grad, counts, stream=st)
    st.synchronize()
    contributions = int(counts.to(torch.int64).sum().item())
    with torch.cuda.stream(st):
        for w in range(args.warmup):
            g.estimate_grad(1, w, views, pairs, grad, counts, stream=st)
    st.synchronize()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        with torch.cuda.stream(st):
            for k in range(args.steps):
                flush.fill_(k & 0xFF)
                ev[k][0].record(st)
                g.estimate_grad(1, 100 + k, views, pairs, grad, counts, stream=st)
                ev[k][1].record(st)
        torch.cuda.synchronize()
    assert g.status(st) == 0
    px_per_step = nv * pairs * render * render
    value, t_total = job_throughput(sum(a.elapsed_time(b) for a, b in ev) / 1000.0, px_per_step * args.steps)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": sc.name + f"_{nv}views_x_{pairs}pairs", "views": nv, "pairs_per_view": pairs,
                       "triangles": int(len(sc.pos_idx)), "params": int(g.n_params),
                       "l2": "flushed between timed steps (256 MB write)", "graph": "none (eager)"},
            "contributions_per_s": contributions * args.steps / t_total,
            # per call: the three binning kernels, the vertex pass, the texel sign planes, the
            # deep estimator and the count expansion
            "gpu_launches": 7 * args.steps,
            "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_soup(args):
    """Section 6.1's experiment: triangle soups of 1,024, 10,240 and 102,400 triangles (12
    parameters each: three vertices and an RGB colour; 12,288 to 1,228,800 parameters) fitted to a smooth 512^2
    image with Adam (lr = eps), 8 antithetic pairs per iteration, once with the per-pixel
    estimator (Eq. 8) and once with the full-image one (Eq. 4).  Reports the image error left
    after each number of iterations, and the time per iteration."""
    import torch

    import synth
    from paper_2404_09758_gb300 import STEP_ADAM, Scene

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    iters, pairs, render = 200, 8, 512
    marks = (0, 25, 50, 100, 200)
    out, ms = {}, {}
    for n in (1024, 10240, 102400):
        sc, tg = synth.triangle_soup(n, render, seed=0)
        # a 1,024-triangle soup's triangles span up to 5 x 5 tiles: more bin entries than the
        # default capacity (6 per triangle + 8 per tile) assumes
        cap = 32 * n + 16 * ((render + 15) // 16) ** 2
        for kind in ("per_pixel", "full_image"):
            g = Scene.from_arrays(sc, targets=tg, bin_capacity=cap)
            grad, counts = g.new_grad_buffers()
            m = torch.zeros(g.n_params, device=dev)
            v = torch.zeros(g.n_params, device=dev)
            curve, t_opt = {}, 0.0
            for it in range(iters + 1):
                if it in marks:
                    curve[it] = float(g.loss([0]).item())
                if it == iters:
                    break
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if kind == "per_pixel":
                    g.estimate_grad(1, it, [0], pairs, grad, counts)
                else:
                    g.estimate_grad_full_image(1, it, [0], pairs, grad, counts)
                g.step(STEP_ADAM, grad, counts, pairs, sc.eps_pos, [sc.textures[0].eps], m=m, v=v, t=it + 1)
                torch.cuda.synchronize()
                t_opt += time.perf_counter() - t0
            assert g.status() == 0
            out[f"{n}_{kind}"] = {str(k): round(c / curve[0], 4) for k, c in curve.items()}
            ms[f"{n}_{kind}"] = round(1000.0 * t_opt / iters, 3)
            del g, grad, counts, m, v
    line = {"metric": "image error left after Adam iterations, per-pixel (Eq. 8) vs full-image (Eq. 4) estimator",
            "value": out["102400_per_pixel"][str(iters)], "unit": "fraction of the initial image error",
            "n_gpus": 1, "steps": iters, "warmup": 0, "ms_per_step": ms["102400_per_pixel"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"triangle_soups_1k_10k_100k_r{render}_{pairs}pairs_adam", "iterations": iters,
                       "params_per_triangle": 12, "graph": "none (eager)"},
            "error_left": out, "ms_per_iteration": ms}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_converge(args):
    """Many-step optimisation of the autograd configuration (32,768-triangle displaced sphere,
    1024^2 RGBA albedo + normal map, Lambert, 1024^2, 16 views x 16 pairs per iteration, Adam with
    the paper's settings) for a fixed wall time: the image error of all views against time, like the
    paper's teaser snapshots (130 s / 720 s on its own scene and GPU, context only).  With
    --control catmull_clark the rendered surface is two Catmull-Clark levels of a 2,048-triangle
    control sphere (47,616 triangles, the teaser's construction) and the parameters optimised are
    the control vertices (refined every iteration; their sums through R^T) and the textures."""
    import torch

    import synth
    from paper_2404_09758_gb300 import STEP_ADAM, ControlMesh, IterState, Scene

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    control = args.control == "catmull_clark"
    if control:
        sc, ctl, R, _ = synth.config_control()
    else:
        sc = synth.config_autograd()
    views = list(range(sc.n_views))
    pairs = sc.pairs_per_view
    ts = Scene.from_arrays(synth.target_scene(sc), max_pairs_per_call=pairs)
    targets = ts.render_targets()
    torch.cuda.synchronize()
    del ts
    g = Scene.from_arrays(sc, targets=targets, max_pairs_per_call=pairs)
    grad, counts = g.new_grad_buffers()
    lr_tex = [t[1] for t in g.textures]
    st = torch.cuda.Stream(device=dev)
    if control:
        cm = ControlMesh(g, ctl, R)
        opt = cm.params  # the control vertices and the shared textures
        grad_c, counts_c = cm.new_grad_buffers()
    else:
        opt = g
    m = torch.zeros(opt.n_params, device=dev)
    v = torch.zeros(opt.n_params, device=dev)

    def image_error():
        with torch.cuda.stream(st):
            if control:
                cm.refine(stream=st)
            e = g.loss(views, stream=st)
        st.synchronize()
        return float(e.sum().item())

    # one iteration, captured once: the iteration index and Adam's step number live in device
    # memory (state), read by the estimate and the step and advanced by the graph's last node
    state = IterState(0, 1, device=dev)

    def iteration():
        if not control:
            g.estimate_grad(1, state, views, pairs, grad, counts, stream=st)
            g.step(STEP_ADAM, grad, counts, len(views) * pairs, sc.eps_pos, lr_tex, m=m, v=v, t=state, stream=st)
        else:
            cm.refine(stream=st)
            g.estimate_grad(1, state, views, pairs, grad, counts, stream=st)
            cm.control_sums(grad, grad_c, stream=st)
            grad.zero_()
            counts.zero_()
            opt.step(STEP_ADAM, grad_c, counts_c, len(views) * pairs, sc.eps_pos, lr_tex, m=m, v=v, t=state,
                     stream=st)
        state.advance(1, 1, stream=st)

    e0 = image_error()
    # capture on a scratch copy of the optimised state (m, v, parameters are restored after the
    # capture's warm-up launch), then replay: iteration k of the loop is replay k
    saved = [p.detach().clone() for p in opt.param_groups()]
    with torch.cuda.stream(st):
        iteration()
    st.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=st):
        iteration()
    st.synchronize()
    for p, q in zip(opt.param_groups(), saved):
        p.copy_(q)
    if control:
        cm.refine(stream=st)
    m.zero_()
    v.zero_()
    grad.zero_()
    counts.zero_()
    state.tensor.copy_(torch.tensor([0, 1], dtype=torch.int32))
    torch.cuda.synchronize()
    curve = [(0.0, e0)]
    t0 = time.perf_counter()
    n_iter = 0
    next_sample = 1.0
    while True:
        with torch.cuda.stream(st):  # the loss below runs on st too: one stream orders both
            graph.replay()
        st.synchronize()  # no backlog: the clock reads finished work
        n_iter += 1
        el = time.perf_counter() - t0
        if el >= next_sample or el >= args.seconds:
            m0 = time.perf_counter()
            curve.append((round(el, 3), image_error()))
            t0 += time.perf_counter() - m0  # the measurement is not optimisation time
            next_sample = el * 2.0 if el < 8.0 else el + 8.0
            if el >= args.seconds:
                break
    line = {"metric": "image error against optimisation time (autograd configuration)", "value": curve[-1][1],
            "unit": "sum of squared errors, all views", "n_gpus": 1, "steps": n_iter, "warmup": 0,
            "ms_per_step": 1000.0 * curve[-1][0] / n_iter, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": sc.name + "_16views_x_16pairs_adam" + ("_control_mesh" if control else ""),
                       "triangles": int(len(sc.pos_idx)), "params": int(opt.n_params),
                       "seconds": args.seconds,
                       "graph": "one iteration captured in a CUDA graph and replayed (device-resident iteration "
                                "index and Adam step); the error is measured between replays"},
            "initial_error": e0, "curve": curve, "reduction": curve[-1][1] / e0,
            # per iteration: 4 binning and pruning kernels, the vertex pass, the texel sign planes, the
            # two estimators, the background loss, the step, the advance (+ the two refine products
            # of the control mesh)
            "gpu_launches": (13 if control else 11) * n_iter}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-sub", action="store_true",
                    help="default workload only: skip the uneven-batch and scale sub-results")
    ap.add_argument("--seconds", type=float, default=60.0, help="wall time of --workload converge")
    ap.add_argument("--control", choices=["none", "catmull_clark"], default="none",
                    help="--workload converge: optimise a Catmull-Clark control mesh instead of the surface")
    ap.add_argument("--workload", choices=["batched", "uneven", "scale", "full_image", "converge", "transparent",
                                           "soup", "atomics"],
                    default="batched",
                    help="batched: the headline configuration; uneven: 32 assets in one batched call; "
                         "scale: 1M triangles, GGX, 2048^2; full_image: Eq. 4's whole-image estimator on "
                         "the batched configuration; converge: optimise the autograd configuration "
                         "for --seconds and report the image error against time; transparent: deep ID "
                         "buffers of three overlapping semi-transparent spheres; soup: Section 6.1's "
                         "per-pixel vs full-image comparison on triangle soups; atomics: the ceiling of "
                         "global fp32 atomic reductions")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "uneven":
        run_uneven(args)
    elif args.workload == "scale":
        run_scale(args)
    elif args.workload == "full_image":
        run_full_image(args)
    elif args.workload == "converge":
        run_converge(args)
    elif args.workload == "transparent":
        run_transparent(args)
    elif args.workload == "soup":
        run_soup(args)
    elif args.workload == "atomics":
        run_atomics(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
