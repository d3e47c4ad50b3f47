#!/usr/bin/env python
"""Throughput of the multi-swarm PSO iteration for the QAP on one GB300 per rank.

Workload (the paper-shaped n = 64 case): D = Manhattan distances on an 8 x 8 grid,
F symmetric with 30 % log-uniform flows in [1, 99]; 16 swarms x 640 particles
(10 240), ring migration of each swarm's best every 20 iterations, full swap local
search, SecondTarget depth 2, Norm velocities. A step is one iteration over every
particle. Inputs are synthetic (QAPLIB is not available).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). The reference arm times the plain CPU oracle on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-iterations/s and swap-Δ evals/s on 1 GB300, n=64, 10k particles"
UNIT = "particle-iterations/s"
N, SWARMS, SWARM_SIZE, RING_PERIOD = 64, 16, 640, 20
L2_BYTES = 129 * 1024 * 1024


def workload_config(storage="fp32"):
    return {"workload": "grid64: n=64 8x8-grid Manhattan D, 30% log-uniform F; 16 swarms x 640 "
                        "particles, ring migration every 20 iterations, full swap local search",
            "n": N, "swarms": SWARMS, "swarm_size": SWARM_SIZE, "particles": SWARMS * SWARM_SIZE,
            "v_storage": storage, "sx": "SecondTarget depth 2 (Algorithm 1)", "sv": "Norm",
            "c": [0.8, 0.5, 0.5],
            "l2": ("V (168 MB fp32) is larger than L2: timed iterations back to back"
                   if storage == "fp32" else "L2 flushed (256 MiB write) before every timed iteration"),
            "timing": "value: K iterations replayed from the captured CUDA graphs, CUDA events on the "
                      "state's stream; kernel_ms_per_step: min(K, 30) further iterations launched kernel "
                      "by kernel with events around each, L2 flushed before each"}


def params(Q, storage):
    return Q.default_params(swarms=SWARMS, swarm_size=SWARM_SIZE, mig_kind=Q.MIG_RING,
                            mig_period=RING_PERIOD, v_storage=storage, depth=2, sv_kind=Q.SV_NORM)


# ----------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = str(gpu_index)
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", self.gpu, "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------- our arm

# DRAM bytes (read + write) of one launch of each kernel on this workload, from one
# ncu capture of each (dram__bytes_read.sum + dram__bytes_write.sum); set to None
# when the kernel changes
PROFILED_TRAFFIC = {"cost_ls": 865280, "update": 277471232}
STEADY_FROM = 200      # the steady window starts after this many iterations
FULL_ITERS = 300       # iterations of the whole configuration
QUALITY_SEEDS = 8      # seeds of the fp32 / bf16 whole runs


def aggregate(units, span_s, dist, torch, device):
    """Whole-job figures of a multi-rank run: the units every rank processed (summed)
    and the slowest rank's time (max); one rank returns its own."""
    if not dist:
        return units, span_s
    t = torch.tensor([span_s], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], device=device, dtype=torch.float64)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return int(u.item()), float(t.item())


def algorithmic(n, dmoves, drounds, particles, swarms, storage_bytes):
    """Algorithmic work of one iteration: the update's bytes (V read and written once,
    X and P^L read, the S_x result written, P^G once per swarm), local-search integer
    ops (below; dmoves = accepted moves in the iteration) and the set-up product's
    tensor flops (2 n^3 per particle)."""
    npairs = n * (n - 1) // 2
    upd_bytes = particles * (2 * n * n * storage_bytes + 3 * n) + swarms * n
    # integer ops of the goal function and a swap local search with a Delta table
    # (symmetric form): n(n-1)/2 for the cost, 3 (n-2) per pair for the table, and per
    # accepted move 3 (n-2) per pair touching the swapped positions plus 7 per other pair
    touching = 2 * (n - 2) + 1
    ls_ops = (particles * (npairs + npairs * (n - 2) * 3)
              + dmoves * (touching * (n - 2) * 3 + (npairs - touching) * 7))
    ls_tc_flops = particles * 2 * n ** 3
    return upd_bytes, ls_ops, ls_tc_flops


def measure(Q, W, torch, storage, steps, warmup, rank, flush):
    inst = W.grid64()
    gi = Q.Instance(inst.F, inst.D)
    stream = torch.cuda.Stream()
    prm = params(Q, storage)
    sw = Q.Swarm(gi, prm, seed=64 + rank, stream=stream.cuda_stream)
    sw.step(warmup)
    torch.cuda.synchronize()
    s0 = sw.stats()
    return sw, s0, stream


def timed_steps(sw, torch, stream, steps, flush, flush_each):
    """Seconds of `steps` iterations replayed from the captured graphs, CUDA events on
    the state's stream (the L2 flushed before each iteration when V fits in L2)."""
    with torch.cuda.stream(stream):
        pairs = []
        if flush_each:
            for _ in range(steps):
                flush.fill_(1)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                sw.step(1)
                b.record()
                pairs.append((a, b))
        else:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            sw.step(steps)
            b.record()
            pairs = [(a, b)]
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in pairs) / 1e3


def whole_runs(Q, W, torch, storage, seeds, iters, flush):
    """The whole n = 64 configuration (init excluded, `iters` iterations) for each
    seed: particle-iterations/s over the run and the final best cost. With bf16 V
    (84 MB, smaller than L2) the L2 is flushed before every iteration."""
    inst = W.grid64()
    gi = Q.Instance(inst.F, inst.D)
    stream = torch.cuda.Stream()
    flush_each = SWARMS * SWARM_SIZE * N * N * (4 if storage == Q.V_FP32 else 2) <= L2_BYTES
    out = []
    for seed in seeds:
        sw = Q.Swarm(gi, params(Q, storage), seed=seed, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        span = timed_steps(sw, torch, stream, iters, flush, flush_each)
        best, _, it = sw.best()
        out.append({"seed": seed, "best": best, "best_iter": it,
                    "value": SWARMS * SWARM_SIZE * iters / span})
        sw.close()
    gi.close()
    return out


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1504_05158_gb300 import build as B
    B.build()
    from paper_1504_05158_gb300 import qap_pso as Q
    from paper_1504_05158_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist:
            dist.barrier()

    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device="cuda")
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak_tops = 152 * 128 * 2 * sm_max * 1e6 / 1e12  # int32 lanes x (mul + add) x clock

    results = {}
    wanted = [v.strip() for v in args.variants.split(",") if v.strip()]
    for storage_name, storage in (("fp32", Q.V_FP32), ("bf16", Q.V_BF16)):
        if storage_name not in wanted:
            continue
        sw, s0, stream = measure(Q, W, torch, storage, args.steps, args.warmup, rank, flush)
        v_bytes = SWARMS * SWARM_SIZE * N * N * (4 if storage == Q.V_FP32 else 2)
        flush_each = v_bytes <= L2_BYTES  # V larger than L2 needs no flush between iterations
        barrier()
        torch.cuda.synchronize()
        # timed region: K iterations replayed from the captured graphs (the path a
        # pso_step caller takes), CUDA events on the state's stream
        with ClockSampler(torch.cuda.current_device() if world == 1 else local_rank) as clk:
            span = timed_steps(sw, torch, stream, args.steps, flush, flush_each)
        barrier()
        s1 = sw.stats()
        pits, span = aggregate(SWARMS * SWARM_SIZE * args.steps, span, dist, torch, "cuda")
        dfull = s1["delta_full"] - s0["delta_full"]
        dincr = s1["delta_incr"] - s0["delta_incr"]
        # per-kernel breakdown: further iterations launched one kernel at a time with
        # events around each (L2 flushed before each iteration, outside the spans)
        kb = min(args.steps, 30)
        ms = sw.step_timed(kb, flush.data_ptr(), flush.numel())
        s2 = sw.stats()
        dmoves = s2["ls_moves"] - s1["ls_moves"]
        drounds = s2["ls_rounds"] - s1["ls_rounds"]
        upd_bytes, ls_ops, ls_flops = algorithmic(
            N, dmoves / kb, drounds / kb, SWARMS * SWARM_SIZE, SWARMS, 4 if storage == Q.V_FP32 else 2)
        upd_ms, ls_ms, bests_ms, _, _ = (m / kb for m in ms)
        best, _, best_it = sw.best()
        # the search kernels side by side on this iteration's S_x results (the same
        # permutations): tensor-core set-up, int32 SIMT set-up, int64 SIMT set-up, direct
        search_kernels = None
        if storage == Q.V_FP32 and not args.no_extras and world == 1:
            xs = sw.export_state()["X_sx"]
            gi2 = Q.Instance(W.grid64().F, W.grid64().D)
            search_kernels = {}
            for kname, kk in (("tensor", Q.SEARCH_TENSOR), ("simt", Q.SEARCH_SIMT), ("int64", Q.SEARCH_INT64),
                              ("direct", Q.SEARCH_DIRECT)):
                _, _, mv, _, kms = gi2.search_with(kk, xs, 0, timed=True)
                _, ops, _ = algorithmic(N, int(mv.sum()), 0, len(xs), SWARMS, 4)
                search_kernels[kname] = {"ms": kms, "moves": int(mv.sum()),
                                         "tops": ops / (kms / 1e3) / 1e12}
            gi2.close()
        # the steady window: the same population advanced (untimed) past STEADY_FROM
        # iterations, where the swarms have converged and S_x meets many equal maxima
        steady = None
        if not args.no_steady:
            done = args.warmup + args.steps + kb
            if done < STEADY_FROM:
                sw.step(STEADY_FROM - done)
            torch.cuda.synchronize()
            s3 = sw.stats()
            k_st = max(args.steps, 20)
            st_span = timed_steps(sw, torch, stream, k_st, flush, flush_each)
            s4 = sw.stats()
            ms_st = sw.step_timed(10, flush.data_ptr(), flush.numel())
            s5 = sw.stats()
            pit4 = s4["particle_iterations"] - s3["particle_iterations"]
            steady = {"from_iteration": s3["iteration"], "iterations": k_st,
                      "value": SWARMS * SWARM_SIZE * k_st / st_span, "ms_per_step": st_span * 1e3 / k_st,
                      "kernel_ms_per_step": {"update": ms_st[0] / 10, "cost_ls": ms_st[1] / 10,
                                             "bests_migration": ms_st[2] / 10},
                      "sx_ties_per_particle": (s4["sx_ties"] - s3["sx_ties"]) / pit4,
                      "moves_per_particle": (s5["ls_moves"] - s4["ls_moves"]) / (10 * SWARMS * SWARM_SIZE)}
        results[storage_name] = dict(
            value=pits / span, ms_per_step=span * 1e3 / args.steps,
            delta_evals_per_s=(dfull + dincr) * world / span,
            delta_full_per_s=dfull * world / span, delta_incr_per_s=dincr * world / span,
            kernel_ms={"update": upd_ms, "cost_ls": ls_ms, "bests_migration": bests_ms},
            upd_gbs=upd_bytes / (upd_ms / 1e3) / 1e9,
            ls_tops=ls_ops / (ls_ms / 1e3) / 1e12, ls_tc_tflops=ls_flops / (ls_ms / 1e3) / 1e12,
            upd_bytes=upd_bytes, ls_ops=ls_ops,
            moves_per_pit=dmoves / (SWARMS * SWARM_SIZE * kb), flush_each=flush_each,
            breakdown_iterations=kb,
            best_cost=best, best_iter=best_it, iterations=args.warmup + args.steps,
            clocks=clk.summary(), steady=steady, search_kernels=search_kernels)
        sw.close()

    # the whole configuration (300 iterations) over several seeds, fp32 and bf16: the
    # throughput averaged over entire runs and the final best costs (quality of bf16)
    full = None
    if not args.no_quality and world == 1:
        seeds = [1000 + i for i in range(QUALITY_SEEDS)]
        full = {"iterations": FULL_ITERS, "seeds": seeds}
        for name, storage in (("fp32", Q.V_FP32), ("bf16", Q.V_BF16)):
            runs = whole_runs(Q, W, torch, storage, seeds, FULL_ITERS, flush)
            bests = np.array([r["best"] for r in runs], np.float64)
            full[name] = {"value": float(np.mean([r["value"] for r in runs])),
                          "best": [int(b) for b in bests], "best_mean": float(bests.mean()),
                          "best_std": float(bests.std(ddof=1)), "best_min": int(bests.min())}
        full["bf16_vs_fp32_mean"] = full["bf16"]["best_mean"] / full["fp32"]["best_mean"] - 1.0
        full["target"] = "bf16 mean final best within 0.5 % of fp32"
        full["within_target"] = abs(full["bf16_vs_fp32_mean"]) <= 0.005

    extras = {}
    if not args.no_extras and world == 1:
        extras["batch64"] = run_batch(args, quick=True)
        extras["serve"] = run_serve(args, quick=True)
    int_peak = None
    try:
        mad, add = Q.int32_peak()
        int_peak = {"mad_tops": mad / 1e12, "add_tops": add / 1e12}
    except Exception as e:  # measurement helper only
        int_peak = {"error": str(e)}

    # end to end through the C-ABI with host buffers: instance upload, init, K iterations
    # each followed by a read-back of the best cost and permutation
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, Q, W, torch, dist, rank, world)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args)

    if rank == 0:
        if int_peak and "mad_tops" in int_peak:
            alu_peak_tops = max(int_peak["mad_tops"], int_peak["add_tops"])
            alu_src = "measured: qap_int32_peak, best of 32-bit multiply-add (2 ops) and add (1 op) lane rates"
        else:
            alu_src = "derived: 152 SMs x 128 int32 lanes x 2 ops x max SM clock"
        line = result_line(args, results, e2e, cpu, world, hbm_peak, alu_peak_tops, alu_src)
        line["full_run"] = full
        line["int32_peak"] = int_peak
        line.update(extras)
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def run_e2e(args, Q, W, torch, dist, rank, world):
    inst = W.grid64()
    F = torch.from_numpy(inst.F).pin_memory()
    D = torch.from_numpy(inst.D).pin_memory()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    gi = Q.Instance(F.numpy(), D.numpy())
    sw = Q.Swarm(gi, params(Q, Q.V_FP32), seed=640 + rank)
    for _ in range(args.steps):
        sw.step(1)
        sw.best()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    sw.close()
    gi.close()
    units, e2e_s = aggregate(SWARMS * SWARM_SIZE * args.steps, e2e_s, dist, torch, "cuda")
    return {"value": units / e2e_s, "unit": UNIT,
            "h2d_bytes_per_step": 2 * N * N * 4 / args.steps,
            "d2h_bytes_per_step": 8 + 4 + N,
            "what": "qap_create_instance + pso_init + K x (pso_step(1) + pso_best), host F and D"}


def result_line(args, results, e2e, cpu, world, hbm_peak, alu_peak_tops, alu_src):
    if True:
        # the fp32 population is the headline; a bf16-only run (--variants bf16) reports bf16
        head = "fp32" if "fp32" in results else "bf16"
        r = results[head]
        km = r["kernel_ms"]
        roofs = {
            "cost_ls": {"kernel": "k_ls_team (goal function + swap local search)", "bound": "alu",
                        "achieved": r["ls_tops"], "peak": alu_peak_tops, "unit": "Tops/s",
                        "frac": r["ls_tops"] / alu_peak_tops, "traffic": PROFILED_TRAFFIC["cost_ls"],
                        "peak_source": alu_src,
                        "op_count": "ops of a swap search with a table of swap values, every add, "
                                    "subtract and multiply one op: n(n-1)/2 for the cost, 3(n-2) per "
                                    "pair for the table, per accepted move 3(n-2) per pair touching "
                                    "the swapped positions and 7 per other pair"},
            "update": {"kernel": "k_update (Eq. 4 + S_v, Eq. 5 with SecondTarget, Algorithm 1)",
                       "bound": "hbm", "achieved": r["upd_gbs"], "peak": hbm_peak, "unit": "GB/s",
                       "frac": r["upd_gbs"] / hbm_peak,
                       "traffic": PROFILED_TRAFFIC["update"] if head == "fp32" else None,
                       "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
                       "bytes": "V read and written once (2 n^2 x %d B), X and P^L read, S_x result "
                                "written (3 n B) per particle, P^G once per swarm" % (4 if head == "fp32" else 2)},
        }
        roof = roofs[max(roofs, key=lambda k: km[k])]  # the kernel that takes longest
        line = {
            "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(head),
            "delta_evals_per_s": r["delta_evals_per_s"],
            "delta_full_per_s": r["delta_full_per_s"], "delta_incr_per_s": r["delta_incr_per_s"],
            "kernel_ms_per_step": r["kernel_ms"],
            "roofline": roof,
            "roofline_all": roofs,
            "ls_setup_tensor_tflops": r["ls_tc_tflops"],
            "search_kernels": ({k: dict(v, frac=v["tops"] / alu_peak_tops) for k, v in r["search_kernels"].items()}
                               if r.get("search_kernels") else None),
            "bf16": ({k: results["bf16"][k] for k in ("value", "ms_per_step", "delta_evals_per_s",
                                                       "kernel_ms", "upd_gbs", "best_cost", "steady")}
                     if head == "fp32" and "bf16" in results else None),
            "moves_per_particle_iteration": r["moves_per_pit"],
            "steady": r["steady"],
            # kernels per iteration: update, search, bests; bf16 populations run the update
            # and the search in two parts of whole swarms (two launches each)
            "e2e": e2e, "gpu_launches": (3 if head == "fp32" else 5) * args.steps, "clocks": r["clocks"],
            "cpu_baseline": cpu,
        }
        return line


# ----------------------------------------------------------------------- oracle

def oracle_sample(steps, warmup, budget_s=None):
    """The oracle as it stands on a bounded sample of the workload: 8 swarms x 64
    particles of the same instance and parameters, its per-particle iteration spread
    over every host core (oracle.step_parallel), `warmup` untimed then up to `steps`
    timed iterations (fewer if the time budget runs out)."""
    from oracle import oracle as O
    from paper_1504_05158_gb300 import workloads as W
    inst = W.grid64()
    m, ss = 8, 64
    cores = os.cpu_count() or 1
    q = O.make_params(swarms=m, swarm_size=ss, mig_kind=2, mig_period=RING_PERIOD, depth=2)
    s = O.init(q, inst.F, inst.D, 64)
    O.step_parallel(q, inst.F, inst.D, 64, s, warmup, threads=cores)
    c0 = s.counters.copy()
    t0 = time.perf_counter()
    done = 0
    for _ in range(steps):
        O.step_parallel(q, inst.F, inst.D, 64, s, 1, threads=cores)
        done += 1
        if budget_s and time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    c1 = s.counters
    pit = int(c1[O.C_PIT] - c0[O.C_PIT])
    dev = int(c1[O.C_DELTA_FULL] + c1[O.C_DELTA_INCR] - c0[O.C_DELTA_FULL] - c0[O.C_DELTA_INCR])
    return {"value": pit / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "delta_evals_per_s": dev / dt, "steps_done": done, "sample_ms_per_step": 1e3 * dt / done,
            "sample": f"{m} swarms x {ss} particles of the same n=64 instance, {done} timed "
                      f"iterations after {warmup} warm-up, the oracle's particle iteration on "
                      f"{cores} host threads"}


def cpu_baseline(args):
    return oracle_sample(steps=40, warmup=3, budget_s=15.0)


def run_reference(args, rank, world):
    if rank != 0:
        return
    r = oracle_sample(steps=args.steps, warmup=args.warmup, budget_s=120.0)
    cfg = workload_config("fp64 (oracle)")
    cfg["l2"] = "host cores (no GPU)"
    cfg["timing"] = ("wall clock of each step over a sample of the workload (8 swarms x 64 particles "
                     "of the same instance and parameters), scaled to particle-iterations/s")
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": r["sample_ms_per_step"],
            "ms_per_step_is": "the sample's time per iteration (512 particles), not the workload's",
            "workload_ms_per_step_est": 1e3 * SWARMS * SWARM_SIZE / r["value"],
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg, "impl": "reference",
            "cpu_baseline": {k: r[k] for k in ("kind", "cores", "sample", "value", "unit")},
            "delta_evals_per_s": r["delta_evals_per_s"],
            "e2e": {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# --------------------------------------------------------------- other workloads

def run_batch(args, quick=False):
    """64 instances with n uniform in [20, 128] (half dense uniform, half grid with
    sparse flows), 8 swarms x 256 particles each, bf16 velocity storage, all in one
    batch (one launch per phase, graph replay, autotuned shapes). quick: a summary
    dict for the main line (5 warm-up, 20 timed iterations) instead of a JSON line."""
    import torch

    from paper_1504_05158_gb300 import build as B
    B.build()
    from paper_1504_05158_gb300 import qap_pso as Q
    from paper_1504_05158_gb300 import workloads as W
    insts = W.uneven_batch(64)
    gis = [Q.Instance(i.F, i.D) for i in insts]
    prm = [Q.default_params(swarms=8, swarm_size=256, v_storage=Q.V_BF16) for _ in insts]
    bstream = torch.cuda.Stream()
    b = Q.Batch(gis, prm, [4096 + i for i in range(len(insts))], stream=bstream.cuda_stream, autotune=True)
    warm, steps = (5, 20) if quick else (args.warmup, args.steps)
    b.step(warm)
    torch.cuda.synchronize()
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device="cuda")
    # the whole-batch rate from graph replays (the path pso_batch_step takes), then a
    # per-phase breakdown launched kernel by kernel
    stream = bstream  # the batch's own stream: its launches and the events
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        a.record(stream)
        b.step(steps)
        z.record(stream)
        torch.cuda.synchronize()
    graph_ms = a.elapsed_time(z)
    ms = b.step_timed(min(steps, 10), flush.data_ptr(), flush.numel())
    kb = min(steps, 10)
    P = sum(p.swarms * p.swarm_size for p in prm)
    ns = [i.n for i in insts]
    out = {"metric": "particle-iterations/s, uneven batch", "value": P * steps / (graph_ms / 1e3),
           "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": warm,
           "ms_per_step": graph_ms / steps, "higher_is_better": True, "dtype": "f32 (bf16 V)",
           "data": "synthetic",
           "config": {"workload": "64 instances, n uniform in [20, 128], 8 x 256 particles each, bf16 V",
                      "n_min": min(ns), "n_max": max(ns), "particles": P,
                      "ls_kernels": {"team1 (n<=32)": sum(n <= 32 for n in ns),
                                     "team2 (n<=64)": sum(32 < n <= 64 for n in ns),
                                     "team8 (n<=128)": sum(64 < n <= 128 for n in ns),
                                     "simt (n>128)": sum(n > 128 for n in ns)}},
           "kernel_ms_per_step": {"update": ms[0] / kb, "cost_ls": ms[1] / kb, "bests_migration": ms[2] / kb},
           "timing": "value: graph replays of the whole batch, CUDA events; kernel_ms_per_step: "
                     "further iterations launched kernel by kernel, L2 flushed before each",
           "clocks": clk.summary(), "gpu_launches": None}
    b.close()
    for g in gis:
        g.close()
    if quick:
        return {k: out[k] for k in ("value", "ms_per_step", "steps", "warmup", "config", "kernel_ms_per_step",
                                    "timing")}
    print(json.dumps(out))


def run_serve(args, quick=False):
    """Poisson arrivals at args.rate requests/s for args.duration s; each request a
    fresh instance with n in {32, 64, 100, 150}, 4 096-16 384 particles in 8-32
    swarms, 150 iterations; admitted under a 120 GB device-memory budget. quick: the
    first args.serve_quick_s seconds of the same stream, as a summary dict for the
    main line."""
    import torch

    from paper_1504_05158_gb300 import build as B
    B.build()
    from paper_1504_05158_gb300 import serve as S
    from paper_1504_05158_gb300 import workloads as W
    duration = args.serve_quick_s if quick else args.duration
    reqs = W.serving_stream(rate_hz=args.rate, duration_s=duration, iterations=args.serve_iters)
    jobs = S.jobs_from_stream(reqs)
    torch.cuda.synchronize()
    srv = S.Server(budget_bytes=120 * 10**9, inflight_particles=args.inflight)
    with ClockSampler(torch.cuda.current_device()) as clk:
        rep = srv.run(jobs, realtime=True)
    summ = rep.summary()
    out = {"metric": "serving: latency p50/p99 and aggregate particle-iterations/s", "unit": UNIT,
           "value": summ["particle_iterations_per_s"], "p50_s": summ["p50_s"], "p99_s": summ["p99_s"],
           "requests": summ["requests"], "failed": summ["failed"], "makespan_s": summ["makespan_s"],
           "peak_bytes": summ["peak_bytes"], "peak_slots": summ["peak_slots"],
           "peak_inflight_particles": summ["peak_inflight_particles"],
           "config": {"workload": f"Poisson {args.rate}/s for {duration} s, n in {{32,64,100,150}}, "
                                  f"4096-16384 particles, {args.serve_iters} iterations, 120 GB budget",
                      "inflight_particles": args.inflight,
                      "latency": "arrival to read-back of the best solution"},
           "higher_is_better": True, "data": "synthetic", "clocks": clk.summary()}
    if quick:
        out["config"]["note"] = (f"the first {duration} s of arrivals of the 60 s stream: the whole stream asks "
                                 "for several times what one GPU delivers, so latency is mostly queueing")
        return {k: out[k] for k in ("value", "p50_s", "p99_s", "requests", "failed", "makespan_s", "config")}
    print(json.dumps(out))


def run_table1(args):
    """The configuration space of section 4.1, Table 1 (inertia c1 in {0.5, 0.8},
    c2 = c3 in {0.3, 0.5}, Raw or Norm velocity kernel, migration factor 0 or 33 %:
    Algorithm 2 with d = floor(0.33 m) every iteration) on synthetic instances shaped
    like the table's rows (QAPLIB is not available): dense uniform n = 26 and n = 60,
    and the n = 64 grid instance; 200 swarms x 50 particles, args.table1_iters
    iterations each. One JSON line: best cost, iteration found, median final cost and
    particle-iterations/s per setting."""
    import itertools

    import torch

    from paper_1504_05158_gb300 import build as B
    B.build()
    from paper_1504_05158_gb300 import qap_pso as Q
    from paper_1504_05158_gb300 import workloads as W
    insts = {"dense26": W.dense_uniform(26, 26), "dense60": W.dense_uniform(60, 60), "grid64": W.grid64()}
    m, ss, iters = 200, 50, args.table1_iters
    rows = []
    stream = torch.cuda.Stream()
    for name, inst in insts.items():
        gi = Q.Instance(inst.F, inst.D)
        for c1, c23, sv, mig in itertools.product((0.5, 0.8), (0.3, 0.5), (Q.SV_RAW, Q.SV_NORM), (0.0, 0.33)):
            prm = Q.default_params(swarms=m, swarm_size=ss, c1=c1, c2=c23, c3=c23, sv_kind=sv,
                                   mig_kind=Q.MIG_RANK if mig else Q.MIG_NONE, mig_depth=int(mig * m),
                                   mig_period=1)
            sw = Q.Swarm(gi, prm, seed=2015, stream=stream.cuda_stream)
            torch.cuda.synchronize()
            span = timed_steps(sw, torch, stream, iters, None, False)
            best, _, it = sw.best()
            st = sw.stats()
            rows.append({"instance": name, "n": inst.n, "c1": c1, "c2": c23, "c3": c23,
                         "velocity": "Raw" if sv == Q.SV_RAW else "Norm", "migration": mig,
                         "best": best, "iteration": it, "final_p50": st["p50"],
                         "value": m * ss * iters / span})
            sw.close()
        gi.close()
    print(json.dumps({"metric": "Table 1 configuration space on synthetic instances", "unit": UNIT,
                      "config": {"swarms": m, "swarm_size": ss, "iterations": iters, "seed": 2015,
                                 "sx": "SecondTarget depth 2 (Algorithm 1)", "v_max": 1.0,
                                 "local_search": "full swap search every iteration"},
                      "data": "synthetic", "rows": rows}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-steady", action="store_true", help="skip the steady window (iterations 200+)")
    ap.add_argument("--no-quality", action="store_true", help="skip the whole 300-iteration fp32/bf16 runs")
    ap.add_argument("--no-extras", action="store_true", help="skip the batch and serving summaries")
    ap.add_argument("--serve-quick-s", type=float, default=2.0,
                    help="seconds of arrivals of the serving summary on the main line")
    ap.add_argument("--variants", default="fp32,bf16",
                    help="velocity storage formats to time (fp32 is the headline)")
    ap.add_argument("--workload", choices=("grid64", "batch64", "serve", "table1"), default="grid64",
                    help="grid64: the headline n = 64 workload; batch64 / serve: the batch and "
                         "serving workloads; table1: the configuration sweep of section 4.1 "
                         "(separate JSON lines)")
    ap.add_argument("--table1-iters", type=int, default=100)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--duration", type=float, default=60.0)
    ap.add_argument("--serve-iters", type=int, default=150)
    ap.add_argument("--inflight", type=int, default=49152,
                    help="serving: particles with work in flight at once (oldest requests first)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batch64":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "table1":
        run_table1(args)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
