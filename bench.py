#!/usr/bin/env python
"""Benchmark of the transformer density-operator VMC hot path on GB300.

Workload (the headline configuration): dissipative transverse-field Ising chain N=16 (PBC, V=2, g=1,
gamma=1), transformer with token embedding, d=64, 8 heads, 4 layers, MLP 4d (P = 198,274 parameters,
N(0, 0.02) seed 0), 16384 Metropolis chains per GPU, one sample per chain per step.

One step = one VMC step through the C ABI: one Metropolis sweep (2N proposals per chain), then the SR
step on the chain states (connections, log rho of every connected configuration, L_loc and cost, cost
gradient, log-derivatives, SR conjugate-gradient solve, parameter update).  The headline times each step
as one launch of the whole-step CUDA graph (tdo_vmc_step with tdo_set_step_graph); the same trajectory
run call by call (tdo_sample + tdo_sr_step), with CUDA events around every kernel group, gives the
per-group breakdown and the rooflines.

The timed arm is the FP16 tensor-core context (tcgen05 GEMMs with FP16 operands, FP32 accumulation);
shorter comparison runs time the BF16 tensor-core and the FP32 CUDA-core contexts.  A BF16 backward's
rounding, amplified by the SR solve's 1 / diag_shift, makes the BF16 optimisation leave the FP32
trajectory after a few steps; the FP16 one follows it.

Prints one JSON line.  --impl reference times the FP64 CPU oracle on a bounded sample of the same step.
The cpu_baseline leg runs that oracle on a fixed subset of the run's final samples: its local estimator there
is also the reference of the "at set error" figures (L_loc and cost of the FP16, BF16 and FP32 contexts
at the run's final parameters against it).
"""
from __future__ import annotations

import argparse
import re
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2502_20723_gb300 import synth  # noqa: E402

N_SITES, D, HEADS, LAYERS, MLP = 16, 64, 8, 4, 4
N_SAMPLES = 16384
LR, SHIFT = 0.0061, 0.004   # eta_0 and lambda_0 of the paper's learning-rate and SR-shift schedules
METRIC = "VMC steps/s and log rho evals/s (N=16, d=64, 4 layers)"
WORKLOAD = "ising_n16_d64_l4_h8_mlp4_ns16384"


def flops_per_sequence(n=N_SITES, d=D, layers=LAYERS, r=MLP) -> float:
    """Algorithmic FLOPs of one sequence forward: per layer QKV 6Nd^2, W^O 2Nd^2, scores and A V 4N^2 d,
    MLP 4 r N d^2 (embedding lookup, pooling and head are negligible)."""
    return layers * (8.0 * n * d * d + 4.0 * n * n * d + 4.0 * r * n * d * d)


F_EVAL = 2.0 * flops_per_sequence()   # one log rho = both orders of the doubled configuration


def max_over_ranks(value: float, world: int, device: str = "cuda") -> float:
    """Largest per-rank value (every rank times its own replica); the run's only collective."""
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_rate(world: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job rate of `world` replicas that each finished `units_per_rank` within `seconds`."""
    return world * units_per_rank / seconds


def replica_seeds(rank: int) -> tuple[int, int]:
    """(initial-configuration seed, Metropolis seed) of a replica: every rank runs its own chains."""
    return 1000 + rank, 12345 + rank


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self) -> dict:
        rows = [r.split(",") for r in (self.out or "").strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows]
        smax = float(rows[0][2])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].strip()[:1].isdigit())
                if any(r[3].strip()[:1].isdigit() for r in rows) else None}


# ---------------------------------------------------------------------------------------------- ours
def run_ours(args) -> dict | None:
    import torch
    import torch.distributed as dist

    from paper_2502_20723_gb300 import tdo

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2502_20723_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()

    prob = synth.ising_chain(N_SITES, V=2.0, g=1.0, gamma=1.0)
    spec = synth.model_spec(D, HEADS, LAYERS, MLP)
    theta = synth.init_params(spec, seed=0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2

    def measure(precision: str, steps: int, warmup: int, e2e: bool):
        ctx = tdo.Context(prob, spec, theta, precision, stream=stream.cuda_stream)
        if precision != "fp32":
            ctx.set_sr_product(args.sr_product)
        cfg_seed, seed = replica_seeds(rank)
        s0, s1 = synth.random_configs(N_SITES, N_SAMPLES, seed=cfg_seed)
        sig = torch.as_tensor(s0.astype(np.int64)).to(torch.int32).cuda()
        sigp = torch.as_tensor(s1.astype(np.int64)).to(torch.int32).cuda()
        counter = [0]
        ctx.sample(sig, sigp, args.burn_in, seed, counter[0])     # burn-in (untimed)
        counter[0] += args.burn_in * 2 * N_SITES

        def step():
            ctx.sample(sig, sigp, 1, seed, counter[0])
            counter[0] += 2 * N_SITES
            return ctx.sr_step(sig, sigp, LR, SHIFT)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        # timed region: per-step CUDA events on the launching stream, L2 flushed between steps
        ctx.timing(True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        costs, sr_iters = [], []
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            for i in range(steps):
                flush.zero_()
                ev[i][0].record(stream)
                costs.append(step())
                ev[i][1].record(stream)
                sr_iters.append(ctx.sr_info()[0])
            torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t_ms = sum(a.elapsed_time(b) for a, b in ev)
        groups = {}
        for g in ("fwd", "sample", "bwd_vjp", "bwd_jac", "conn", "lloc", "sr", "update"):
            ms, n = ctx.timing_read(g)
            groups[g] = {"ms": ms / steps, "launches": n / steps}
        launches = int(sum(v["launches"] for v in groups.values()) * steps)
        ms, n = ctx.timing_read("sr_mv")   # the S' v kernel alone (inside "sr")
        sr_mv = {"ms": ms / steps, "launches": n / steps, "shape": ctx.sr_product_shape()}
        ctx.timing(False)
        lloc_rows = int(ctx.connections(sig, sigp)[0].sum().item())
        out = {"t_ms": max_over_ranks(t_ms, world), "groups": groups, "sr_mv": sr_mv, "launches": launches,
               "lloc_rows": lloc_rows, "costs": costs, "sr_iters": sr_iters, "clocks": clk.summary(), "P": ctx.P,
               "theta": ctx.get_params(),
               "subset": ((sig[:SET_ERROR_SAMPLES].cpu().numpy().astype(np.int64) & 0xFFFFFFFF).astype(np.uint32),
                          (sigp[:SET_ERROR_SAMPLES].cpu().numpy().astype(np.int64) & 0xFFFFFFFF).astype(np.uint32))}
        ctx.close()
        if e2e and not args.no_graph:
            # the same trajectory again (a fresh context from the same parameters and chains, the same
            # burn-in), each step one launch of the whole-step CUDA graph (tdo_set_step_graph + vmc_step):
            # first with the chains on the device (CUDA events per step on the launching stream: the
            # headline), then end to end with the chains in pinned host memory (copies inside the timed
            # region, wall clock)
            sched = tdo.Schedule(eta0=LR, lambda0=SHIFT)   # constant: the schedules switch at step 30000
            for host in (False, True):
                ctx = tdo.Context(prob, spec, theta, precision, stream=stream.cuda_stream)
                if precision != "fp32":
                    ctx.set_sr_product(args.sr_product)
                sig = torch.as_tensor(s0.astype(np.int64)).to(torch.int32).cuda()
                sigp = torch.as_tensor(s1.astype(np.int64)).to(torch.int32).cuda()
                ctx.sample(sig, sigp, args.burn_in, seed, 0)
                ctr = args.burn_in * 2 * N_SITES
                ctx.set_step_graph(True)
                for k in range(warmup):
                    _, ctr = ctx.vmc_step(sig, sigp, 1, seed, ctr, k, sched)
                a, b = sig, sigp
                if host:
                    hs = torch.empty(N_SAMPLES, dtype=torch.int32).pin_memory()
                    hp = torch.empty(N_SAMPLES, dtype=torch.int32).pin_memory()
                    hs.copy_(sig.cpu())
                    hp.copy_(sigp.cpu())
                    a, b = hs.numpy(), hp.numpy()
                torch.cuda.synchronize()
                gcosts, giters = [], []
                gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                       for _ in range(steps)]
                if world > 1:
                    dist.barrier()
                torch.cuda.synchronize()
                with ClockSampler(local) as gclk:
                    t0 = time.perf_counter()
                    for i in range(steps):
                        flush.zero_()
                        gev[i][0].record(stream)
                        c_i, ctr = ctx.vmc_step(a, b, 1, seed, ctr, warmup + i, sched)
                        gev[i][1].record(stream)
                        gcosts.append(c_i)
                        giters.append(ctx.sr_info()[0])
                    torch.cuda.synchronize()
                    wall = time.perf_counter() - t0
                if world > 1:
                    dist.barrier()
                # the same steps as the call-by-call run up to the order of float atomics in the gradient
                diff = float(np.max(np.abs(np.array(gcosts) - np.array(costs)) / np.abs(costs)))
                rec, nl = ctx.step_graph_stats()
                if host:
                    out["e2e_steps_per_s"] = replicas_rate(world, steps, max_over_ranks(wall, world))
                    out["e2e_cost_max_rel_diff"] = diff
                else:
                    out["graph"] = {"t_ms": max_over_ranks(sum(x.elapsed_time(y) for x, y in gev), world),
                                    "costs": gcosts, "sr_iters": giters, "cost_max_rel_diff": diff,
                                    "recordings": rec,
                                    "launches": nl, "clocks": gclk.summary()}
                ctx.close()
        return out

    peak_fp32 = tdo.measure_peak("fp32", stream.cuda_stream)
    peak_fp64 = tdo.measure_peak("fp64", stream.cuda_stream)
    main = measure(args.precision, args.steps, args.warmup, True)
    others = {}
    if not args.no_compare:
        for prec in ("fp16", "bf16", "fp8", "fp32"):
            if prec != args.precision:
                others[prec] = measure(prec, max(2, min(args.steps, 3)), 3, False)
    t_max, groups, launches, lloc_rows = main["t_ms"], main["groups"], main["launches"], main["lloc_rows"]
    fwd_evals = lloc_rows
    sample_evals = N_SAMPLES * (1 + 2 * N_SITES)
    clk_summary = main["clocks"]

    # at set error: L_loc and cost of both precisions on a fixed subset of the final samples, at the final
    # parameters of the timed run (compared below with the oracle's values from the cpu_baseline leg)
    sub_s, sub_p = main["subset"]
    set_err_gpu = {}
    for prec in ("fp16", "bf16", "fp8", "fp32"):
        c2 = tdo.Context(prob, spec, main["theta"], prec, stream=stream.cuda_stream)
        ll, cost, _ = c2.local_estimator(sub_s.astype(np.uint32), sub_p.astype(np.uint32))
        set_err_gpu[prec] = (np.asarray(ll[:, 0] + 1j * ll[:, 1]), cost)
        c2.close()

    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return None

    peaks = measured_peaks()
    P = main["P"]
    tensor = args.precision in ("bf16", "fp16", "fp8")
    if tensor:
        # FP16 and BF16 dense MMA share one nominal rate (2.25 PFLOP/s), so the measured BF16 figure serves both
        peak_t = float(peaks.get("bf16_tflops_sustained", 1700.0))
        t_src = ("MEASURED_PEAKS bf16_tflops_sustained (of measured; FP16 at the same nominal rate)"
                 if "bf16_tflops_sustained" in peaks else "fallback 1700 TFLOP/s sustained")
    else:
        peak_t, t_src = peak_fp32, "tdo_measure_peak FP32 FFMA, this run (of measured)"
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "MEASURED_PEAKS hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback 6800 GB/s"

    def compute_roof(group, units, per_unit, desc):
        ms, n = groups[group]["ms"], groups[group]["launches"]
        flops = units * per_unit
        ach = flops / (ms * 1e-3) / 1e12 if ms else 0.0
        return {"bound": "tensor" if tensor else "alu", "kernel": desc, "group": group, "achieved": ach,
                "peak": peak_t, "unit": "TFLOP/s", "frac": ach / peak_t, "traffic": None,
                "algorithmic_per_step": flops, "units_per_step": units, "per_unit": per_unit,
                "ms_per_step": ms, "launches_per_step": n, "peak_source": t_src}

    rooflines = {
        "fwd": compute_roof("fwd", fwd_evals, F_EVAL, "forward of every connected row (log rho evals)"),
        "bwd_vjp": compute_roof("bwd_vjp", lloc_rows, 2 * F_EVAL, "gradient backward (VJP of every connected row)"),
        "sample": compute_roof("sample", sample_evals, F_EVAL, "Metropolis sweep (one log rho per proposal)"),
    }
    mv = main["sr_mv"]
    ob = 8 if args.precision == "fp32" else 4   # tensor-core contexts store O - obar as BF16 pairs
    # algorithmic bytes of one product: the passes over O that the product makes, each streaming all of
    # O (two for the two-pass product, one for the one-pass products)
    used = mv["shape"][0] if args.precision != "fp32" else 0
    reads = 2 if used == 0 else 1
    byts = reads * N_SAMPLES * P * ob
    ach = byts * mv["launches"] / (mv["ms"] * 1e-3) / 1e9 if mv["ms"] else 0.0
    traffic, traffic_src = None, None
    if args.precision != "fp32":   # the captures are of the BF16-pair products
        per_row, traffic_src = sr_traffic_per_row(mode=used)
        traffic = per_row * N_SAMPLES if per_row else None
    kern = {0: "S' v product, two passes (k_sr_tpart + k_sr_wpart and reductions)",
            1: "S' v product, one pass on thread-block clusters (k_sr_fused and reductions)",
            2: "S' v product, one pass over the whole grid (k_sr_grid and reductions)"}[used]
    rooflines["sr_mv"] = {"bound": "hbm", "kernel": kern, "product": SR_PRODUCT_NAMES[used],
                          "group": "sr_mv", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                          "traffic": traffic, "traffic_source": traffic_src,
                          "algorithmic_per_launch": byts,
                          "algorithmic": f"{reads} read(s) of O (Ns x P elements) per product",
                          "o_element_bytes": ob, "o_reads_per_product": reads,
                          "products_per_step": mv["launches"], "ms_per_step": mv["ms"], "peak_source": hbm_src}
    # the headline roofline: the dominant kernel group of the timed steps
    dom_ms = {"fwd": groups["fwd"]["ms"], "bwd_vjp": groups["bwd_vjp"]["ms"], "sample": groups["sample"]["ms"],
              "sr_mv": mv["ms"]}
    dom = max(dom_ms, key=dom_ms.get)
    roof = dict(rooflines[dom])
    fwd_tflops = rooflines["fwd"]["achieved"]
    # --no-graph (profiling runs: no conditional graph nodes under the profiler): the call-by-call run
    # stands in for the graph leg and there is no end-to-end leg
    gr = main.get("graph") or {"t_ms": t_max, "costs": main["costs"], "sr_iters": main["sr_iters"],
                               "cost_max_rel_diff": 0.0, "recordings": 0, "launches": 0, "clocks": clk_summary}
    res = {
        "metric": METRIC,
        "value": replicas_rate(world, args.steps, gr["t_ms"] * 1e-3),
        "unit": "VMC steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": gr["t_ms"] / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp32": "f32", "bf16": "bf16", "fp16": "f16", "fp8": "e4m3 (evaluation) + f16"}[args.precision],
        "data": "synthetic (seeded random initial chains, Metropolis-sampled; random-init N(0,0.02) weights)",
        "config": {"workload": WORKLOAD, "n_sites": N_SITES, "d_model": D, "heads": HEADS, "layers": LAYERS,
                   "mlp_ratio": MLP, "samples_per_gpu": N_SAMPLES, "params": P, "precision": args.precision,
                   "sweeps_per_step": 1, "lr": LR, "diag_shift": SHIFT,
                   "sr_product": args.sr_product if args.precision != "fp32" else "two_pass",
                   "l2": "256 MB buffer written between timed steps",
                   "timing": "each step one launch of the whole-step CUDA graph (tdo_set_step_graph), CUDA events "
                             "per step; kernel groups, rooflines and gpu_launches from the call-by-call run of the "
                             "same trajectory (tdo_sample + tdo_sr_step, CUDA events per kernel group)",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "logrho_evals_per_s": (fwd_evals + sample_evals) * world * args.steps / (t_max * 1e-3),
        "logrho_evals_per_s_fwd_kernel": fwd_evals / (groups["fwd"]["ms"] * 1e-3) if groups["fwd"]["ms"] else None,
        "rows_per_step": {"lloc_rows": lloc_rows, "sample_evals": sample_evals},
        "breakdown_ms_per_step": {g: round(v["ms"], 3) for g, v in groups.items()},
        "costs": [round(c, 6) for c in gr["costs"]],
        "sr_cg_iterations": gr["sr_iters"],
        "call_by_call": {"value": replicas_rate(world, args.steps, t_max * 1e-3), "unit": "VMC steps/s",
                         "ms_per_step": t_max / args.steps, "costs": [round(c, 6) for c in main["costs"]],
                         "sr_cg_iterations": main["sr_iters"],
                         "clocks": clk_summary,
                         "graph_cost_max_rel_diff": gr["cost_max_rel_diff"]},
        "graph": {"recordings": gr["recordings"], "launches": gr["launches"]},
        "fwd_kernel_tflops": fwd_tflops,
        "roofline": roof,
        "rooflines": rooflines,
        "peaks_measured_here": {"fp32_fma_tflops": peak_fp32, "fp64_fma_tflops": peak_fp64},
        "clocks": gr["clocks"],
        # chains in (2 x 4 B per chain) and the step's 32-byte value block; chains out, the cost statistics
        # (16 B), the L_loc, timeout and update flags (3 x 4 B) and the CG scalars (14 x 8 B)
        "e2e": {"value": main.get("e2e_steps_per_s"), "unit": "VMC steps/s",
                "h2d_bytes_per_step": 2 * 4 * N_SAMPLES + 32, "d2h_bytes_per_step": 2 * 4 * N_SAMPLES + 16 + 12 + 112,
                "steps": args.steps, "call": "tdo_vmc_step in graph mode with the chains in pinned host memory",
                "trajectory": "the timed steps replayed from the same parameters and chains",
                "cost_max_rel_diff_vs_timed_steps": main.get("e2e_cost_max_rel_diff")},
        "gpu_launches": launches,
    }
    res["compare"] = {}
    for prec, other in others.items():
        og = other["groups"]
        res["compare"][prec] = {
            "value": world * len(other["costs"]) / (other["t_ms"] * 1e-3), "unit": "VMC steps/s",
            "steps": len(other["costs"]), "warmup": 3, "ms_per_step": other["t_ms"] / len(other["costs"]),
            "logrho_evals_per_s_fwd_kernel": fwd_evals / (og["fwd"]["ms"] * 1e-3) if og["fwd"]["ms"] else None,
            "breakdown_ms_per_step": {g: round(v["ms"], 3) for g, v in og.items()},
            "costs": [round(c, 6) for c in other["costs"]], "sr_cg_iterations": other["sr_iters"]}
    if not args.no_config5:
        res["config5"] = config5_leg(tdo, torch, stream, flush)
    if world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(args.cpu_budget, main["theta"], sub_s, sub_p)
        ref_l, ref_c = base.pop("lloc_ref"), base.pop("cost_ref")
        res["cpu_baseline"] = base
        res["at_set_error"] = set_error_report(set_err_gpu, ref_l, ref_c)
    return res


# ------------------------------------------------------------------ chains of uneven length (one launch)
CONFIG5_N = (8, 12, 16, 20, 24, 32)
CONFIG5_SAMPLES = 32768


def config5_leg(tdo, torch, stream, flush, reps: int = 5) -> dict:
    """The XYZ chains (Jx = 0.9, Jy = Jz = 1, gamma = 1) of N in {8, 12, 16, 20, 24, 32}, 32,768 samples
    in equal shares (two Metropolis sweeps from uniform configurations, FP16 context per N), and every
    configuration the Lindbladian connects to them, evaluated as one interleaved batch by
    tdo_log_rho_ragged: one persistent tensor-core launch across the lengths (autotuned on its first
    call), timed over `reps` calls with the L2 flushed between them."""
    spec = synth.model_spec(D, HEADS, LAYERS, MLP)
    theta = synth.init_params(spec, seed=0)
    per = CONFIG5_SAMPLES // len(CONFIG5_N)
    rn, rs, rp = [], [], []
    for i, n in enumerate(CONFIG5_N):
        k = per + (CONFIG5_SAMPLES - per * len(CONFIG5_N) if i == 0 else 0)
        ctx = tdo.Context(synth.xyz_chain(n, Jx=0.9, Jy=1.0, Jz=1.0), spec, theta, "fp16", stream=stream.cuda_stream)
        s0, s1 = synth.random_configs(n, k, seed=500 + n)
        sig = torch.as_tensor(s0.astype(np.int64)).to(torch.int32).cuda()
        sigp = torch.as_tensor(s1.astype(np.int64)).to(torch.int32).cuda()
        ctx.sample(sig, sigp, 2, 77 + n, 0)
        cnt, cs, cp, _ = ctx.connections(sig, sigp)
        mask = torch.arange(cs.shape[1], device="cuda")[None, :] < cnt[:, None]
        rs.append(cs[mask])
        rp.append(cp[mask])
        rn.append(torch.full((int(mask.sum().item()),), n, dtype=torch.int32, device="cuda"))
        ctx.close()
    n_all, s_all, p_all = torch.cat(rn), torch.cat(rs), torch.cat(rp)
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    order = torch.randperm(len(n_all), device="cuda", generator=g)   # interleaved lengths
    n_all, s_all, p_all = n_all[order].contiguous(), s_all[order].contiguous(), p_all[order].contiguous()
    counts = {int(n): int((n_all == n).sum().item()) for n in CONFIG5_N}
    flops = sum(c * 2.0 * flops_per_sequence(n=n) for n, c in counts.items())
    mix = sum(1 << (n - 1) for n in CONFIG5_N)
    peaks = measured_peaks()
    peak_t = float(peaks.get("bf16_tflops_sustained", 1700.0))
    out = {"workload": "xyz_uneven_n8-32_d64_l4_h8_mlp4_ns32768", "samples": CONFIG5_SAMPLES,
           "rows_per_n": counts, "rows": int(len(n_all)), "algorithmic_flop_per_call": flops, "reps": reps,
           "precisions": {}}
    for prec in ("fp16", "bf16", "fp8", "fp32"):
        ctx = tdo.Context(synth.xyz_chain(16), spec, theta, prec, stream=stream.cuda_stream)
        ctx.log_rho_ragged(n_all, s_all, p_all)   # first call: bucketing and (tensor core) autotuning
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.log_rho_ragged(n_all, s_all, p_all)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        t = statistics.median(ms)
        r = {"ms_per_call": t, "logrho_evals_per_s": len(n_all) / (t * 1e-3), "tflops": flops / (t * 1e-3) / 1e12}
        if prec == "fp8":   # E4M3 runs at twice the BF16 rate (nominal 4.5 against 2.25 PFLOP/s)
            r["tensor_frac_of_fp8_peak"] = r["tflops"] / (2.0 * peak_t)
            r["fp8_peak_source"] = "MEASURED_PEAKS bf16_tflops_sustained x 2 (nominal FP8 / BF16 ratio)"
        if prec != "fp32":
            r["tensor_frac_of_bf16_sustained"] = r["tflops"] / peak_t
            r["tuned_shape"] = dict(zip(("ctas_per_sm", "descending", "dynamic"), ctx.ragged_tuning(mix)))
        out["precisions"][prec] = r
        ctx.close()
    # matched error: per chain length, L_loc of 256 of the samples by each tensor-core context against the
    # FP32 context (itself within 1e-6 of the oracle in the parity tests): max |dL| / max |L|.  At the
    # N(0, 0.02) initial weights rho is nearly flat and L_loc hides the operand rounding, so the error is
    # taken at wider weights, with the spread (standard deviation) of Re log rho they give
    err = {}
    for std in (0.1, 0.15):
        th = synth.init_params(spec, seed=0, std=std)
        per_n = {}
        for n in CONFIG5_N:
            prob = synth.xyz_chain(n, Jx=0.9, Jy=1.0, Jz=1.0)
            s0, s1 = synth.random_configs(n, 256, seed=900 + n)
            sig = torch.as_tensor(s0.astype(np.int64)).to(torch.int32).cuda()
            sigp = torch.as_tensor(s1.astype(np.int64)).to(torch.int32).cuda()
            ll, spread = {}, 0.0
            for prec in ("fp32", "fp16", "bf16", "fp8"):
                ctx = tdo.Context(prob, spec, th, prec, stream=stream.cuda_stream)
                v, _, _ = ctx.local_estimator(sig, sigp)
                v = v.cpu().numpy()
                ll[prec] = v[:, 0] + 1j * v[:, 1]
                if prec == "fp32":
                    spread = float(np.std(ctx.log_rho(sig, sigp).cpu().numpy()[:, 0]))
                ctx.close()
            ref = ll["fp32"]
            per_n[n] = {"re_logrho_std": spread,
                        **{p: float(np.abs(ll[p] - ref).max() / np.abs(ref).max()) for p in ("fp16", "bf16", "fp8")}}
        err[f"weights N(0,{std})"] = per_n
    out["lloc_max_rel_vs_fp32"] = err
    out["vmc"] = config5_vmc(tdo, torch, stream, spec, theta)
    return out


# ---------------------------------------------------------------------------------- oracle on the CPU
SET_ERROR_SAMPLES = 256
TOL_COST_REL_BF16 = 1e-3


def config5_vmc(tdo, torch, stream, spec, theta, steps: dict = None) -> dict:
    """VMC steps of the N in {8, ..., 32} workload: each chain length is its own Lindbladian, so one step
    is, for every N, one Metropolis sweep and one SR step (connections, L_loc, cost, gradient,
    log-derivatives, CG solve, update) on that length's share of the 32,768 chains, in a context per N
    with the same initial parameters.  Timed with CUDA events around the whole multi-length step after
    warm-up steps, FP16 against FP32.  The FP16 contexts run each length's step as one launch of its
    whole-step CUDA graph (tdo_set_step_graph); the FP32 contexts, which have no graph mode, call by call."""
    steps = steps or {"fp16": (2, 3), "fp32": (1, 2)}   # (warm-up, timed)
    per = CONFIG5_SAMPLES // len(CONFIG5_N)
    out = {"definition": "one sweep + one SR step of every chain length N in {8,12,16,20,24,32}, "
                         f"{per}-{per + CONFIG5_SAMPLES - per * len(CONFIG5_N)} chains each (32,768 in all)",
           "lr": LR, "diag_shift": SHIFT}
    for prec, (warm, timed) in steps.items():
        ctxs, chains = [], []
        for i, n in enumerate(CONFIG5_N):
            k = per + (CONFIG5_SAMPLES - per * len(CONFIG5_N) if i == 0 else 0)
            ctx = tdo.Context(synth.xyz_chain(n, Jx=0.9, Jy=1.0, Jz=1.0), spec, theta, prec, stream=stream.cuda_stream)
            s0, s1 = synth.random_configs(n, k, seed=700 + n)
            sig = torch.as_tensor(s0.astype(np.int64)).to(torch.int32).cuda()
            sigp = torch.as_tensor(s1.astype(np.int64)).to(torch.int32).cuda()
            ctx.sample(sig, sigp, 2, 91 + n, 0)
            ctx.set_step_graph(prec != "fp32")
            ctxs.append(ctx)
            chains.append([sig, sigp, 2 * 2 * n])
        costs = []
        sched = tdo.Schedule(eta0=LR, lambda0=SHIFT)
        k_step = [0]

        def one_step():
            c = []
            for (ctx, ch), n in zip(zip(ctxs, chains), CONFIG5_N):
                if prec != "fp32":
                    cost, ch[2] = ctx.vmc_step(ch[0], ch[1], 1, 91 + n, ch[2], k_step[0], sched)
                    c.append(cost)
                else:
                    ctx.sample(ch[0], ch[1], 1, 91 + n, ch[2])
                    ch[2] += 2 * n
                    c.append(ctx.sr_step(ch[0], ch[1], LR, SHIFT))
            k_step[0] += 1
            return c

        for _ in range(warm):
            one_step()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(timed):
            costs.append(one_step())
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / timed
        out[prec] = {"steps_per_s": 1e3 / ms, "ms_per_step": ms, "warmup": warm, "steps": timed,
                     "graph": prec != "fp32",
                     "costs_last_step": dict(zip((str(n) for n in CONFIG5_N), (round(x, 5) for x in costs[-1])))}
        for ctx in ctxs:
            ctx.close()
    out["speedup_fp16_over_fp32"] = out["fp16"]["steps_per_s"] / out["fp32"]["steps_per_s"]
    return out


SR_PRODUCT_NAMES = {0: "two_pass", 1: "one_pass", 2: "grid"}
SR_TRAFFIC_PROFILES = {0: "k_sr_tpart_wpart_ising_n16_d64_l4.md", 2: "k_sr_grid_ising_n16_d64_l4.md"}


def sr_traffic_per_row(prof: str = None, src: str = None, mode: int = 0):
    """DRAM bytes per sample row of one S' v product from the committed ncu summary of that product
    (mode 0: the two passes, 2: the grid product), valid only while the SR source has the SHA-1 recorded
    with that capture: (bytes or None, source)."""
    here = os.path.dirname(os.path.abspath(__file__))
    if prof is None:
        if mode not in SR_TRAFFIC_PROFILES:
            return None, None
        prof = os.path.join(here, "profiles", SR_TRAFFIC_PROFILES[mode])
    src = src or os.path.join(here, "paper_2502_20723_gb300", "csrc", "k_sr.cu")
    try:
        m = re.search(r"bench-traffic sr_mv: k_sr\.cu sha1=([0-9a-f]{40}) bytes_per_sample_row=(\d+)", open(prof).read())
        sha = hashlib.sha1(open(src, "rb").read()).hexdigest()
    except OSError:
        return None, None
    if not m:
        return None, None
    if m.group(1) != sha:
        return None, "k_sr.cu changed since the ncu capture in profiles/: traffic not known"
    kern = "k_sr_tpart + k_sr_wpart" if "tpart" in os.path.basename(prof) else "k_sr_grid"
    return int(m.group(2)), (f"ncu dram__bytes_read.sum + dram__bytes_write.sum of {kern} on a reduced sample "
                             f"count, scaled by the samples (profiles/{os.path.basename(prof)})")


def set_error_report(gpu: dict, ref_l: np.ndarray, ref_c: float) -> dict:
    """L_loc and cost of each precision against the oracle on the same samples and parameters:
    lloc_max_rel = max_s |L_gpu - L_ref| / max_s |L_ref|, lloc_rms_rel = ||L_gpu - L_ref|| / ||L_ref||,
    cost_rel = |cost_gpu - cost_ref| / cost_ref."""
    out = {"samples": int(len(ref_l)), "parameters": "final parameters of the timed run", "cost_oracle": ref_c,
           "cost_tolerance_bf16": TOL_COST_REL_BF16}
    for prec, (l, c) in gpu.items():
        d = np.abs(l - ref_l)
        out[prec] = {"lloc_max_rel": float(d.max() / np.abs(ref_l).max()),
                     "lloc_rms_rel": float(np.linalg.norm(l - ref_l) / np.linalg.norm(ref_l)),
                     "cost": c, "cost_rel": float(abs(c - ref_c) / ref_c)}
    for prec in gpu:
        if prec != "fp32":
            out[prec]["within_tolerance"] = out[prec]["cost_rel"] <= TOL_COST_REL_BF16
    return out


def _timed(fn, count: int, target_s: float, grow: int = 8):
    """Run fn(count); if it took well under target_s, rerun once with a count scaled to the target.
    Returns (seconds per unit, count used, seconds of the counted run)."""
    t0 = time.perf_counter()
    fn(count)
    dt = time.perf_counter() - t0
    if dt < 0.5 * target_s:
        count = int(count * min(grow, max(1.0, target_s / max(dt, 1e-3))))
        t0 = time.perf_counter()
        fn(count)
        dt = time.perf_counter() - t0
    return dt / count, count, dt


def oracle_step_estimate(budget_s: float, theta=None) -> dict:
    """Time the FP64 oracle on a bounded sample of one VMC step of the workload and extrapolate.
    Parts: Metropolis proposals (one log rho each), the local estimator and gradient over each sample's
    connected configurations, the log-derivatives.  The SR solve is not included: the oracle's dense
    Cholesky needs P^2 = 3.9e10 doubles (315 GB) at this P, so its time is unavailable."""
    import torch

    from oracle import estimators as E, transformer as T

    prob = synth.ising_chain(N_SITES, V=2.0, g=1.0, gamma=1.0)
    spec = synth.model_spec(D, HEADS, LAYERS, MLP)
    th = synth.init_params(spec, seed=0) if theta is None else theta

    def ev(k):
        a, b = synth.random_configs(N_SITES, k, seed=1)
        T.log_rho_np(spec, th, a, b, N_SITES)

    def gr(k):
        a, b = synth.random_configs(N_SITES, k, seed=2)
        E.grad_estimator(prob, spec, th, a, b)

    def jc(k):
        a, b = synth.random_configs(N_SITES, k, seed=3)
        E.jacobian(spec, th, a, b, N_SITES)

    t_eval, nf, s1 = _timed(ev, 128, 0.35 * budget_s)
    t_grad, ng, s2 = _timed(gr, 4, 0.4 * budget_s)
    t_jac, nj, s3 = _timed(jc, 2, 0.25 * budget_s)
    step_s = N_SAMPLES * (2 * N_SITES * t_eval + t_grad + t_jac)
    timed = s1 + s2 + s3
    return {"step_s": step_s, "timed_s": timed, "extrapolation_factor": step_s / timed,
            "cores": torch.get_num_threads(), "host_cpus": os.cpu_count(),
            "sample": (f"{nf} log rho evals, gradient estimator on {ng} samples (with their connected "
                       f"configurations), log-derivatives of {nj} samples, timed {timed:.1f} s; extrapolated to "
                       f"16384 samples x (32 Metropolis proposals + estimator + gradient + log-derivatives) "
                       f"= x{step_s / timed:.0f}; SR solve excluded (oracle dense Cholesky infeasible at "
                       f"P=198,274)")}


def cpu_baseline(budget_s: float, theta=None, sub_s=None, sub_p=None) -> dict:
    """The oracle on the host cores: one VMC step extrapolated from a timed sample, plus its local
    estimator on the given subset of samples (the reference of the at-set-error figures)."""
    from oracle import estimators as E
    est = oracle_step_estimate(budget_s, theta)
    out = {"value": 1.0 / est["step_s"], "unit": "VMC steps/s", "cores": est["cores"], "kind": "oracle",
           "sample": est["sample"], "timed_s": est["timed_s"], "extrapolation_factor": est["extrapolation_factor"],
           "host_cpus": est["host_cpus"]}
    if sub_s is not None:
        prob = synth.ising_chain(N_SITES, V=2.0, g=1.0, gamma=1.0)
        spec = synth.model_spec(D, HEADS, LAYERS, MLP)
        t0 = time.perf_counter()
        ll = E.local_estimator(prob, spec, theta, sub_s, sub_p)
        out["lloc_ref"], out["cost_ref"] = ll, float(np.mean(np.abs(ll) ** 2))
        out["set_error_oracle_s"] = time.perf_counter() - t0
    return out


def _single_thread_estimate(budget_s: float) -> dict:
    """The same oracle sample with one thread (numpy/BLAS and torch), in a child process."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", str(budget_s)],
                       capture_output=True, text=True, env=env, timeout=600)
    for line in r.stdout.splitlines()[::-1]:
        if line.startswith("{"):
            return json.loads(line)
    return {"error": (r.stderr or "no output")[-300:]}


def run_reference(args) -> dict | None:
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    budget = max(2.0, 120.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_step_estimate(min(budget, 2.0))
    est_steps = [oracle_step_estimate(budget) for _ in range(args.steps)]
    step_s = statistics.mean(e["step_s"] for e in est_steps)
    timed_s = statistics.mean(e["timed_s"] for e in est_steps)
    v = 1.0 / step_s
    single = _single_thread_estimate(budget)
    return {"metric": METRIC, "value": v, "unit": "VMC steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_s * 1e3, "ms_per_step_kind": "extrapolated",
            "timed_s_per_step": timed_s, "extrapolation_factor": step_s / timed_s,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "n_sites": N_SITES, "d_model": D, "heads": HEADS, "layers": LAYERS,
                       "mlp_ratio": MLP, "samples_per_gpu": N_SAMPLES, "parallelism": "CPU oracle"},
            "cpu_baseline": {"value": v, "unit": "VMC steps/s", "cores": est_steps[0]["cores"], "kind": "oracle",
                             "host_cpus": est_steps[0]["host_cpus"], "sample": est_steps[0]["sample"],
                             "single_thread": {"value": 1.0 / single["step_s"] if "step_s" in single else None,
                                               "timed_s": single.get("timed_s"), "cores": 1,
                                               "note": single.get("error")}},
            "e2e": {"value": v, "unit": "VMC steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_kernel_case(args) -> None:
    """One call of one kind on the workload's model with a reduced sample count (for ncu captures):
    fwd (log rho of all connected rows), grad (gradient backward), jac (log-derivatives), sample (one
    sweep), sr (one SR step: gradient, log-derivatives in the step's own layout, CG solve, update).  Runs the call twice (first warms up)."""
    import torch

    from paper_2502_20723_gb300 import build, tdo
    build.build()
    prob = synth.ising_chain(N_SITES, V=2.0, g=1.0, gamma=1.0)
    spec = synth.model_spec(D, HEADS, LAYERS, MLP)
    ctx = tdo.Context(prob, spec, synth.init_params(spec, seed=0), args.precision)
    if args.precision != "fp32":
        ctx.set_sr_product(args.sr_product)
    s0, s1 = synth.random_configs(N_SITES, args.case_samples, seed=1)
    sig = torch.as_tensor(s0.astype(np.int64)).to(torch.int32).cuda()
    sigp = torch.as_tensor(s1.astype(np.int64)).to(torch.int32).cuda()
    ctx.sample(sig, sigp, 1, 1, 0)
    cnt, cs, cp, _ = ctx.connections(sig, sigp)
    rows_s = torch.cat([cs[i, :cnt[i]] for i in range(len(cnt))]).contiguous()
    rows_p = torch.cat([cp[i, :cnt[i]] for i in range(len(cnt))]).contiguous()
    for _ in range(2):
        if args.kernel_case == "fwd":
            ctx.log_rho(rows_s, rows_p)
        elif args.kernel_case == "grad":
            ctx.grad(sig, sigp)
        elif args.kernel_case == "jac":
            ctx.jacobian(sig, sigp)
        elif args.kernel_case == "sample":
            ctx.sample(sig, sigp, 1, 1, 0)
        elif args.kernel_case == "sr":
            ctx.sr_step(sig, sigp, LR, SHIFT)   # the step's own O layout (BF16 pairs in BF16 contexts)
    torch.cuda.synchronize()
    print(json.dumps({"kernel_case": args.kernel_case, "samples": args.case_samples, "rows": int(len(rows_s))}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp16", choices=["fp32", "bf16", "fp16", "fp8"])
    ap.add_argument("--no-compare", action="store_true", help="skip the other-precision comparison runs")
    ap.add_argument("--burn-in", type=int, default=4)
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-config5", action="store_true", help="skip the uneven-length (N = 8..32) leg")
    ap.add_argument("--no-graph", action="store_true",
                    help="time call by call only (no step-graph or end-to-end leg): for profiler runs")
    ap.add_argument("--kernel-case", default=None, choices=["fwd", "grad", "jac", "sample", "sr"],
                    help="run one call of one kind on a reduced sample count (profiling) and exit")
    ap.add_argument("--case-samples", type=int, default=1024)
    ap.add_argument("--sr-product", default="two_pass", choices=["two_pass", "one_pass", "grid"],
                    help="how the CG forms S' v in tensor-core contexts (tdo_set_sr_product)")
    ap.add_argument("--oracle-sample", type=float, default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_sample is not None:   # child process of the reference arm (single-thread timing)
        import torch
        torch.set_num_threads(1)
        print(json.dumps({k: v for k, v in oracle_step_estimate(args.oracle_sample).items() if k != "sample"}))
        return
    if args.kernel_case:
        run_kernel_case(args)
        return
    args.warmup = max(args.warmup, 3)
    res = run_reference(args) if args.impl == "reference" else run_ours(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
