"""Benchmark of the force-field minimization hot path on GB300.

Workload (N = 1): the paper-scale 30,000-atom globule (seed 3, the
10^4-variable scale of the paper is the smaller 3,334-atom case) with the
plain FP64 pair kernel.  One step = one capped L-BFGS run (m = 10, LS_PAR,
10 accepted steps = 1 + 10 x 4 evaluations of E or E + grad E) from the
jittered start: every row of the hot path (pair kernel, bonded terms,
reductions, line search, two-loop direction, history update, stopping test)
runs each step.  value = unique pair interactions per second over the
step's evaluations, E + grad E and energy-only alike (N(N-1)/2 per
evaluation; the E + grad E and E-only kernel rates are reported apart).  The
same step in MIXED precision, minimizations per second to |grad E|_inf < 0.1
(a 16-system subset of the batched workload in FP64, MIXED and MIXED with the
learned preconditioner, the 256-system batch, the 3,334-atom system), the
device roofline of the dominant kernel and the FP64 CPU oracle on one and on
all host cores are reported beside it.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank runs its own replica (independent systems, no
collective on the data path); value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "E+grad pair interactions/s and minimizations/s to ‖∇E‖∞<0.1, vs plain GPU"
N_ATOMS = 30000
SEED = 3
CAP_ITERS = 10
# Algorithmic work: 35 flops per unique pair for E + grad E, 23 for E only
# (FMA = 2, rsqrt = 1: d 3, r^2 5, rsqrt 1, r^-2 1, q_i q_j 1, E_c 1,
# sigma_ij 1, (s/r)^2 2, s^6 2, s^12 1, eps_ij 1, E_lj 2, E acc 2, f/r 6,
# grad acc 6), N(N-1)/2 unique pairs per evaluation: the roofline's
# `achieved`.  Hardware work of the row sweep, beside it: each unordered pair
# is evaluated twice (rows i and j), N(N-1) evaluations of 32 flops (21 E
# only) with the per-atom factors precombined (d 3, r^2 5, r^-1 1, r^-2 1,
# e_cul 2, r^-6 2, C6/C12 2, t1 2, E acc 3, t2 2, F 3, grad acc 6).
FLOPS_UNIQUE_EG = 35.0
FLOPS_UNIQUE_E = 23.0
FLOPS_PER_PAIR_EG = 32.0
FLOPS_PER_PAIR_E = 21.0
# hardware flops per unique pair of each kernel form: the FP64 symmetric
# tiles evaluate a pair once and add its force to both atoms (32 + 6); the
# FP32 E + grad row sweep evaluates it twice (2 x 32); the energy-only and
# difference-trial forms run on the symmetric tiles once (21; ~40 for the
# exact-difference identities)
HW_SYM_EG, HW_SYM_E, HW_ROW_EG, HW_DELTA = 38.0, 21.0, 64.0, 40.0
# ALU peaks derived from unit counts at the maximum SM clock: FP32 152 SMs x
# 128 lanes x 2 flops; FP64 152 SMs x 2 FMA per clock x 2 flops (the GB300
# nominal 1.25 TFLOP/s at 2,070 MHz)
FP32_LANES_X2 = 152 * 128 * 2
FP64_LANES_X2 = 152 * 2 * 2
# minimizations replay their rounds from the host (--host-loop): the same
# work, with every kernel visible to a kernel-level profiler
HOST_LOOP = 0
PROFILE_SUMMARY = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles",
                               "pair_kernels_30k.md")


def profiled_traffic(kernel):
    """DRAM bytes (read + write) of one launch of `kernel` from the committed
    ncu summary (a line 'traffic_bytes <kernel>: <bytes>'), else None."""
    try:
        with open(PROFILE_SUMMARY) as f:
            for ln in f:
                ln = ln.strip().strip("`")
                if ln.startswith(f"traffic_bytes {kernel}:"):
                    return int(ln.split(":")[1])
    except OSError:
        pass
    return None


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = []
        mx = None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[3 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def shard(seq, rank, ws):
    """The units (systems) of one rank: a strided share, no overlap."""
    return list(seq)[rank::ws]


def reduce_time_units(seconds, units, device=None):
    """(max over ranks of seconds, sum over ranks of units); identity at one
    rank.  The only collective of the benchmark, outside the timed region."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds), float(units)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p))
    except Exception:
        return {}


def flush_l2(buf):
    buf.zero_()


def step_config(system=None):
    """The workload of one benchmark step (both arms), with the SHA-256 of
    the generated inputs when the system is given."""
    out = {"workload": f"{N_ATOMS}-atom chain globule (seed {SEED}), plain FP64 path, "
                       f"L-BFGS m=10 capped at {CAP_ITERS} steps per step",
           "n_atoms": N_ATOMS, "l2": "flushed (256 MB write) between steps",
           "minimize_driver": ("host-replayed graph of 8 rounds" if HOST_LOOP else
                               "one graph launch (conditional WHILE node over the rounds)")}
    if system is not None:
        from paper_1810_03358_gb300 import synth
        out["input_sha256"] = synth.digest(system)
    return out


def bench_gpu(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_1810_03358_gb300 import build as gbuild
    gbuild.build()
    from paper_1810_03358_gb300 import ffmin, synth

    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    s = synth.make_system(N_ATOMS, SEED + 1000 * rank)
    pairs_per_eval = N_ATOMS * (N_ATOMS - 1) // 2
    x0 = torch.tensor(s.x.reshape(-1), dtype=torch.float64, device=dev)
    l2 = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def run_steps(S, steps, warmup, e2e=False):
        x = torch.empty_like(x0)
        xh = s.x.reshape(-1).copy()
        pin = torch.empty(x0.numel(), dtype=torch.float64, pin_memory=True)
        evals = []
        for _ in range(warmup):
            x.copy_(x0)
            S.minimize(x, method="LBFGS", lbfgs_m=10, max_iter=CAP_ITERS, host_loop=HOST_LOOP)
        torch.cuda.synchronize()
        times = []
        launches = 0
        for _ in range(steps):
            flush_l2(l2)
            x.copy_(x0)
            barrier()
            torch.cuda.synchronize()
            if e2e:
                t0 = time.perf_counter()
                pin.copy_(torch.from_numpy(xh))
                r = S.minimize_host(pin.numpy(), method="LBFGS", lbfgs_m=10, max_iter=CAP_ITERS, host_loop=HOST_LOOP)
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
            else:
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record()
                r = S.minimize(x, method="LBFGS", lbfgs_m=10, max_iter=CAP_ITERS, host_loop=HOST_LOOP)
                ev1.record()
                torch.cuda.synchronize()
                times.append(ev0.elapsed_time(ev1) / 1e3)
            barrier()
            evals.append(r[0]["energy_evals"] + r[0]["grad_evals"])
            launches += S.last_stats()["launches"]
        return times, evals, launches, r[0]

    out = {}
    sampler = ClockSampler(local if ws > 1 else 0)
    # ---- primary: plain FP64 ----
    S64 = ffmin.System([s], ffmin.FFMIN_FP64)
    density64 = S64.autotune(x0)
    sampler.start()
    t64, ev64, launches, r64_run = run_steps(S64, args.steps, args.warmup)
    clocks = sampler.stop()
    total_t, total_pairs = reduce_time_units(sum(t64), sum(ev64) * pairs_per_eval, dev)
    value = total_pairs / total_t
    # e2e through the host entry point (H2D of x and D2H of the result inside)
    te2e, ev_e2e, _, _ = run_steps(S64, max(1, min(args.steps, 3)), 1, e2e=True)
    e2e_value = sum(ev_e2e) * pairs_per_eval * ws / sum(te2e)
    # dominant kernel: FP64 pair kernel, E + grad mode, timed alone on its stream
    ms_pair = S64.time_pair_kernel(x0, with_grad=True, reps=5)
    ms_pair_e = S64.time_pair_kernel(x0, with_grad=False, reps=5)
    e64, g64 = S64.energy_grad(x0.clone())
    g64 = g64.cpu().numpy()
    S64.close()
    # ---- mixed precision, same step ----
    S32 = ffmin.System([s], ffmin.FFMIN_MIXED)
    density32 = S32.autotune(x0)
    t32, ev32, launches32, _ = run_steps(S32, args.steps, args.warmup)
    ms_pair32 = S32.time_pair_kernel(x0, with_grad=True, reps=20)
    ms_pair32_e = S32.time_pair_kernel(x0, with_grad=False, reps=20)
    ms_pair32_d = S32.time_pair_kernel(x0, with_grad=2, reps=20)
    # error of one MIXED E + grad at the start against the FP64 path (which
    # the parity tests hold to 2e-11 of sum|terms| of the FP64 oracle)
    e32, g32 = S32.energy_grad(x0.clone())
    g32 = g32.cpu().numpy()
    mixed_err = {"energy_rel": abs(e32[0] - e64[0]) / abs(e64[0]),
                 "grad_rel_to_max": float(np.abs(g32 - g64).max() / np.abs(g64).max())}
    S32.close()
    t32_tot, pairs32 = reduce_time_units(sum(t32), sum(ev32) * pairs_per_eval, dev)
    value32 = pairs32 / t32_tot

    minim = {} if args.no_minimize else minimizations(args, ffmin, synth, torch, dev, rank, ws)

    sm_max_mhz = float(load_peaks().get("sm_max_mhz", 2070.0))
    fp32_derived = FP32_LANES_X2 * sm_max_mhz * 1e6 / 1e12
    fp64_derived = FP64_LANES_X2 * sm_max_mhz * 1e6 / 1e12
    # the roofline divides by the peaks derived from unit counts and the
    # maximum clock; the FMA-chain probe of this GPU is reported beside them
    fp32_probe = ffmin.ffmin_alu_peak(ffmin.FFMIN_MIXED, reps=20)
    fp64_probe = ffmin.ffmin_alu_peak(ffmin.FFMIN_FP64, reps=20)

    unique = N_ATOMS * (N_ATOMS - 1) // 2

    def roof(ms, unique_flops, hw_flops, peak):
        """Algorithmic FLOP/s (unique pairs x the per-pair count) and the
        kernel's executed FLOP/s (its own per-pair formula), against peak."""
        achieved = unique_flops * unique / (ms / 1e3) / 1e12
        hw = hw_flops * unique / (ms / 1e3) / 1e12
        return {"achieved": achieved, "frac": achieved / peak, "hw_achieved": hw, "hw_frac": hw / peak,
                "ms_per_launch": ms, "unique_pairs_per_s": unique / (ms / 1e3)}

    r64 = roof(ms_pair, FLOPS_UNIQUE_EG, HW_SYM_EG, fp64_derived)
    r64e = roof(ms_pair_e, FLOPS_UNIQUE_E, HW_SYM_E, fp64_derived)
    r32 = roof(ms_pair32, FLOPS_UNIQUE_EG, HW_ROW_EG, fp32_derived)
    r32e = roof(ms_pair32_e, FLOPS_UNIQUE_E, HW_SYM_E, fp32_derived)
    r32d = roof(ms_pair32_d, FLOPS_UNIQUE_E, HW_DELTA, fp32_derived)
    n_eg, n_e = r64_run["grad_evals"], r64_run["energy_evals"]
    # the dominant kernel over the step: k_pair64_sym in both of its forms,
    # weighted by the step's own launch mix (n_eg E + grad, n_e energy only)
    step_ms = n_eg * ms_pair + n_e * ms_pair_e
    step_alg = (n_eg * FLOPS_UNIQUE_EG + n_e * FLOPS_UNIQUE_E) * unique / (step_ms / 1e3) / 1e12
    step_hw = (n_eg * HW_SYM_EG + n_e * HW_SYM_E) * unique / (step_ms / 1e3) / 1e12
    step32_ms = ms_pair32 + 3 * ms_pair32_d  # a MIXED L-BFGS step: one E + grad, three trials
    step32_alg = (FLOPS_UNIQUE_EG + 3 * FLOPS_UNIQUE_E) * unique / (step32_ms / 1e3) / 1e12
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "pair interactions/s (E and E+grad evaluations)",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * total_t / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": dict(step_config(s), evals_per_step={"e_grad": n_eg, "e_only": n_e},
                       autotuned_items_per_block=density64, parallelism=f"replicas x{ws}"),
        "rates": {"note": "value counts N(N-1)/2 unique pairs per evaluation over all evaluations of "
                          "the step; the kernel rates below are one launch each, timed alone",
                  "e_grad_unique_pairs_per_s": r64["unique_pairs_per_s"],
                  "e_only_unique_pairs_per_s": r64e["unique_pairs_per_s"]},
        "e2e": {"value": e2e_value, "unit": "pair interactions/s (E and E+grad evaluations)",
                "h2d_bytes_per_step": 8 * 3 * N_ATOMS, "d2h_bytes_per_step": 8 * 3 * N_ATOMS},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "roofline": {"bound": "alu", "achieved": step_alg, "peak": fp64_derived, "unit": "TFLOP/s",
                     "frac": step_alg / fp64_derived, "traffic": profiled_traffic("k_pair64_sym E+grad"),
                     "kernel": "k_pair64_sym (E+grad and E-only launches in the step's mix)",
                     "work": f"{FLOPS_UNIQUE_EG:.0f} (E+grad) / {FLOPS_UNIQUE_E:.0f} (E) flops x N(N-1)/2 "
                             f"unique pairs per launch (algorithmic); {n_eg} + {n_e} launches per step",
                     "ms_per_launch": step_ms / (n_eg + n_e),
                     "hw_achieved": step_hw, "hw_frac": step_hw / fp64_derived,
                     "hw_work": f"{HW_SYM_EG:.0f} / {HW_SYM_E:.0f} flops per unique pair as executed "
                                "(each pair once, force added to both atoms)",
                     "peak_source": f"derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x {sm_max_mhz:.0f} MHz",
                     "peak_probe": fp64_probe, "frac_of_probe": step_alg / fp64_probe,
                     "e_grad": {"ms_per_launch": ms_pair, "achieved": r64["achieved"], "frac": r64["frac"],
                                "hw_frac": r64["hw_frac"]},
                     "e_only": {"ms_per_launch": ms_pair_e, "achieved": r64e["achieved"], "frac": r64e["frac"],
                                "hw_frac": r64e["hw_frac"]}},
        "mixed": {"value": value32, "unit": "pair interactions/s (E and E+grad evaluations)",
                  "ms_per_step": 1e3 * sum(t32) / len(t32),
                  "autotuned_items_per_block": density32,
                  "vs_plain_gpu": value32 / value,
                  "error_vs_fp64_at_start": mixed_err,
                  "roofline": {"bound": "alu", "kernel": "k_pair<float,64,2> (a MIXED L-BFGS step's mix: "
                                                            "one E+grad row sweep, three difference trials)",
                               "achieved": step32_alg, "peak": fp32_derived, "unit": "TFLOP/s",
                               "frac": step32_alg / fp32_derived,
                               "e_grad": {"ms_per_launch": ms_pair32, "frac": r32["frac"],
                                          "hw_frac": r32["hw_frac"]},
                               "traffic": profiled_traffic("k_pair<float,64,2> E+grad"),
                               "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 flops x {sm_max_mhz:.0f} MHz",
                               "peak_probe": fp32_probe, "frac_of_probe": step32_alg / fp32_probe,
                               "e_only": {"ms_per_launch": ms_pair32_e, "frac": r32e["frac"],
                                          "hw_frac": r32e["hw_frac"]},
                               "difference_trial": {"ms_per_launch": ms_pair32_d, "frac": r32d["frac"],
                                                    "hw_frac": r32d["hw_frac"],
                                                    "vs_e_grad": ms_pair32_d / ms_pair32}}},
        "minimize": minim,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def minimizations(args, ffmin, synth, torch, dev, rank=0, ws=1):
    """Minimizations per second to |grad E|_inf < 0.1 (L-BFGS m = 10): the
    256-system batch (atom counts log-uniform in [200, 5000], seeds 1000 + b)
    in MIXED precision with and without the learned preconditioner (trained
    on other seeds); its first 16 systems in plain FP64, MIXED and MIXED +
    learned (like for like, on the batched path; the whole batch in FP64
    would take many minutes) with the final energies of the forms compared
    system by system; and the paper-scale 3,334-atom system.  Each run is
    timed once with CUDA events."""
    import numpy as np

    from paper_1810_03358_gb300 import learn
    w16 = learn.load_weights()

    def run(systems, prec, learned=False, tune=True):
        S = ffmin.System(systems, prec)
        if learned:
            ffmin.ffmin_set_precond(S.handle, w16)
        x = torch.tensor(np.concatenate([q.x.reshape(-1) for q in systems]), dtype=torch.float64, device=dev)
        if tune:
            S.autotune(x)
        tuning = S.get_tuning()
        S.minimize(x.clone(), method="LBFGS", max_iter=2, use_learned_precond=int(learned))  # warm-up
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        r = S.minimize(x, method="LBFGS", lbfgs_m=10, gtol_inf=0.1, max_iter=100000,
                       use_learned_precond=int(learned))
        ev1.record()
        torch.cuda.synchronize()
        st = S.last_stats()
        S.close()
        t = ev0.elapsed_time(ev1) / 1e3
        ok = sum(1 for q in r if q["status_name"] == "ok")
        if shard_all:  # every rank ran its share: max time, summed units
            t, ok = reduce_time_units(t, ok, dev)
        return {"n_sys": len(systems), "converged": ok, "seconds": t, "minimizations_per_s": ok / t,
                "final_energies": [q["energy"] if q["status_name"] == "ok" else None for q in r]
                if len(systems) <= 16 else None,
                "max_final_grad_inf": max(q["grad_inf"] for q in r),
                "iterations_max": max(q["iterations"] for q in r),
                "iterations_sum": sum(q["iterations"] for q in r),
                "fp64_phase_iterations_max": max(q["fp64_iterations"] for q in r),
                "not_converged": [b for b, q in enumerate(r) if q["status_name"] != "ok"],
                "tuning": {"items_per_block": tuning[0], "f32_atoms_per_thread": tuning[1]},
                "pair_interactions_per_s": st["pair_interactions"] / t, "gpu_launches": st["launches"]}

    def ratio(a, b):
        return out[a]["minimizations_per_s"] / max(out[b]["minimizations_per_s"], 1e-30)

    def energy_gap(a, b):
        """Final energies of the same systems in two forms: relative
        differences (median, max) over the systems both converged."""
        ea, eb = out[a]["final_energies"], out[b]["final_energies"]
        d = [abs(x - y) / abs(y) for x, y in zip(ea, eb) if x is not None and y is not None]
        return {"median": float(np.median(d)) if d else None, "max": max(d) if d else None, "n": len(d)}

    out = {"learned_weights": "paper_1810_03358_gb300/precond_w16.npy" if w16 is not None else None}
    batch = synth.make_batch(256)
    shard_all = ws > 1
    mine = shard(batch, rank, ws)  # systems are independent: each rank minimizes its share
    out["batch256_mixed"] = run(mine, ffmin.FFMIN_MIXED)
    if w16 is not None:
        out["batch256_mixed_learned"] = run(mine, ffmin.FFMIN_MIXED, learned=True)
        out["batch256_learned_vs_mixed"] = ratio("batch256_mixed_learned", "batch256_mixed")
    shard_all = False  # the comparisons below run on every rank's GPU alike
    # like for like: the first 16 systems of the batch (the n_sys >= 8
    # batched path), plain FP64, MIXED and MIXED + learned in the same run
    sub = batch[:16]
    out["subset16_fp64"] = run(sub, ffmin.FFMIN_FP64)
    out["subset16_mixed"] = run(sub, ffmin.FFMIN_MIXED)
    out["subset16_mixed_vs_plain_gpu"] = ratio("subset16_mixed", "subset16_fp64")
    out["subset16_mixed_energy_vs_fp64"] = energy_gap("subset16_mixed", "subset16_fp64")
    if w16 is not None:
        out["subset16_mixed_learned"] = run(sub, ffmin.FFMIN_MIXED, learned=True)
        out["subset16_mixed_learned_vs_plain_gpu"] = ratio("subset16_mixed_learned", "subset16_fp64")
        out["subset16_mixed_learned_vs_mixed"] = ratio("subset16_mixed_learned", "subset16_mixed")
        out["subset16_learned_energy_vs_fp64"] = energy_gap("subset16_mixed_learned", "subset16_fp64")
    s3 = synth.make_system(3334, 2)
    if not getattr(args, "no_methods", False) and ws == 1:  # per-method runs: single-GPU runs only
        out["methods_3334"] = methods_3334(ffmin, torch, dev, s3)
    out["n3334_fp64"] = run([s3], ffmin.FFMIN_FP64)
    out["n3334_mixed"] = run([s3], ffmin.FFMIN_MIXED)
    out["n3334_mixed_vs_plain_gpu"] = ratio("n3334_mixed", "n3334_fp64")
    out["n3334_mixed_energy_vs_fp64"] = energy_gap("n3334_mixed", "n3334_fp64")
    if w16 is not None:
        out["n3334_mixed_learned"] = run([s3], ffmin.FFMIN_MIXED, learned=True)
        out["n3334_mixed_learned_vs_plain_gpu"] = ratio("n3334_mixed_learned", "n3334_fp64")
    return out


def methods_3334(ffmin, torch, dev, s3, cap=3000, gradfree_sweeps=10):
    """Every minimizer of the paper from the same jittered start of the
    3,334-atom globule (10^4 variables), in FP64 and MIXED: to |grad E|_inf
    < 0.1 or `cap` iterations (the gradient-free search: `gradfree_sweeps`
    sweeps of N moves, one atom at a time and in parallel epochs over 64
    parts).  One timed run each (CUDA events)."""
    x0 = torch.tensor(s3.x.reshape(-1), dtype=torch.float64, device=dev)
    res = {}
    for prec, tag in ((ffmin.FFMIN_FP64, "fp64"), (ffmin.FFMIN_MIXED, "mixed")):
        S = ffmin.System([s3], prec)
        S.autotune(x0)
        if prec == ffmin.FFMIN_FP64:
            res["start_energy"] = S.energy_grad(x0.clone())[0][0]
        runs = [(m, m, {}) for m in ("GD", "FGM", "CG", "LBFGS", "OGM", "GRADFREE")]
        runs.insert(2, ("FGM_RESTART", "FGM", dict(fgm_restart=1)))
        runs.append(("GRADFREE_EPOCHS64", "GRADFREE", dict(gradfree_parts=64, gradfree_margin=1.0)))
        for name, method, extra in runs:
            cap_m = gradfree_sweeps * s3.n_atoms if method == "GRADFREE" else cap
            S.minimize(x0.clone(), method=method, max_iter=2, **extra)  # warm-up (graphs, buffers)
            x = x0.clone()
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            r = S.minimize(x, method=method, max_iter=cap_m, **extra)[0]
            ev1.record()
            torch.cuda.synchronize()
            res[f"{name}_{tag}"] = {"status": r["status_name"], "iterations": r["iterations"],
                                    "evals": r["energy_evals"] + r["grad_evals"],
                                    "seconds": ev0.elapsed_time(ev1) / 1e3, "energy": r["energy"],
                                    "grad_inf": r["grad_inf"]}
        S.close()
    return res


_CPU = {}


def _cpu_init(s):
    """Worker set-up of the all-cores oracle timing: the system, loaded once."""
    from oracle import oracle
    oracle.lib()
    _CPU["ff"], _CPU["x"] = oracle.FF(s), s.x


def _cpu_rows(i0, i1):
    from oracle import oracle
    d, st, g = oracle.energy_rows(_CPU["ff"], _CPU["x"], i0, i1, grad=True)
    return d["total"], g


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


class OracleCores:
    """The FP64 oracle as it stands on every host core: one E + grad E of a
    system split into row blocks of equal pair counts, one block per worker
    process (started with 'spawn'), energies and gradients summed in block
    order by the caller."""

    def __init__(self, s, workers=None):
        import concurrent.futures as cf
        import multiprocessing as mp
        self.n = s.n_atoms
        self.workers = workers or (os.cpu_count() or 1)
        self.pool = cf.ProcessPoolExecutor(self.workers, mp_context=mp.get_context("spawn"),
                                           initializer=_cpu_init, initargs=(s,))
        k = self.workers
        cuts = sorted({int(round(self.n * (1.0 - math.sqrt(1.0 - q / k)))) for q in range(k + 1)})
        self.blocks = list(zip(cuts[:-1], cuts[1:]))
        list(self.pool.map(_cpu_rows, [0], [1]))  # start every worker

    def energy_grad(self):
        import numpy as np
        parts = list(self.pool.map(_cpu_rows, *zip(*self.blocks)))
        e = sum(p[0] for p in parts)
        g = np.sum([p[1] for p in parts], axis=0)
        return e, g

    def close(self):
        self.pool.shutdown()


def cpu_baseline():
    """The FP64 oracle, as it stands, on the GPU host's cores: one E + grad E
    of the same 30,000-atom system on one core (a bounded sample of the step's
    evaluations), and the same evaluation split over every core."""
    from oracle import oracle
    from paper_1810_03358_gb300 import synth
    s = synth.make_system(N_ATOMS, SEED)
    pairs = N_ATOMS * (N_ATOMS - 1) // 2
    t0 = time.perf_counter()
    oracle.energy_grad(s, s.x)
    dt1 = time.perf_counter() - t0
    oc = OracleCores(s)
    oc.energy_grad()  # warm-up
    reps = 3
    t0 = time.perf_counter()
    for _ in range(reps):
        oc.energy_grad()
    dtn = (time.perf_counter() - t0) / reps
    oc.close()
    return {"value": pairs / dtn, "unit": "pair interactions/s", "cores": oc.workers, "kind": "oracle",
            "sample": f"one E+grad evaluation of the {N_ATOMS}-atom globule split into {len(oc.blocks)} row "
                      f"blocks over {oc.workers} worker processes, mean of {reps} ({dtn:.2f} s each)",
            "cpu_model": cpu_model(), "build": "gcc -O3 -ffp-contract=off, single-threaded oracle per process",
            "one_core": {"value": pairs / dt1, "cores": 1,
                         "sample": f"one E+grad evaluation of the {N_ATOMS}-atom globule ({dt1:.1f} s)"}}


def bench_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from paper_1810_03358_gb300 import synth
    s = synth.make_system(N_ATOMS, SEED)
    pairs = N_ATOMS * (N_ATOMS - 1) // 2
    oc = OracleCores(s)
    for _ in range(args.warmup):
        oc.energy_grad()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oc.energy_grad()
        times.append(time.perf_counter() - t0)
    oc.close()
    value = args.steps * pairs / sum(times)
    sample = (f"one full E+grad evaluation of the {N_ATOMS}-atom globule per step (a bounded sample of the "
              f"GPU step's evaluations), row blocks over {oc.workers} worker processes")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pair interactions/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": step_config(s),
        "cpu_baseline": {"value": value, "unit": "pair interactions/s", "cores": oc.workers, "kind": "oracle",
                         "sample": sample, "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": "pair interactions/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


def profile_run(args):
    """Small fixed workloads for ncu captures.  Default: E + grad E and E of
    the 30,000-atom globule in FP64, then E + grad E, E and one difference
    trial in MIXED.
    --profile-minimize K: a K-step MIXED L-BFGS run of the 3,334-atom globule
    (every kernel of the minimizer pipeline).  --profile-batch K: K steps of
    the 256-system batch.  --profile-vectors K: K FP64 L-BFGS steps of 1,024
    systems of 500 atoms (the update and direction kernels at full history)."""
    import numpy as np
    import torch
    from paper_1810_03358_gb300 import build as gbuild
    gbuild.build()
    from paper_1810_03358_gb300 import ffmin, synth
    if args.profile_batch:
        systems = synth.make_batch(256)
        S = ffmin.System(systems, ffmin.FFMIN_MIXED)
        x = torch.tensor([v for s in systems for v in s.x.reshape(-1)], dtype=torch.float64, device="cuda")
        S.minimize(x.clone(), method="LBFGS", max_iter=1, host_loop=HOST_LOOP)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        r = S.minimize(x.clone(), method="LBFGS", max_iter=args.profile_batch, host_loop=HOST_LOOP)
        ev1.record()
        torch.cuda.synchronize()
        st = S.last_stats()
        print("profile-batch", st, "ms", ev0.elapsed_time(ev1), "ms/tick", ev0.elapsed_time(ev1) / st["ticks"])
        S.close()
        return
    if args.profile_epochs:
        # one epoch of the parallel gradient-free search on the 30,000-atom
        # globule, MIXED, 128 parts (the k_epoch workload)
        s = synth.make_system(N_ATOMS, SEED)
        S = ffmin.System([s], ffmin.FFMIN_MIXED)
        x = torch.tensor(s.x.reshape(-1), dtype=torch.float64, device="cuda")
        r = S.minimize(x, method="GRADFREE", max_iter=args.profile_epochs, gradfree_parts=128,
                       gradfree_margin=1.0)
        torch.cuda.synchronize()
        print("profile-epochs", r[0]["iterations"], S.last_stats())
        S.close()
        return
    if args.profile_vectors:
        # 1,024 systems of 500 atoms (512,000 atoms, vectors of 12.3 MB; 64
        # chains, each under 16 coordinate jitters): FP64
        # L-BFGS m = 10 for profile_vectors iterations; all systems take the
        # same number of line-search trials, so after 10 iterations every
        # tick's update / direction launches cover every atom with a full
        # history (the vector-kernel workload)
        import dataclasses
        base = [synth.make_system(500, 50000 + b) for b in range(64)]
        systems = []
        for b in range(1024):  # 64 chains x 16 jitters of the reference coordinates
            s0 = base[b % 64]
            jr = np.random.default_rng(60000 + b)
            systems.append(dataclasses.replace(s0, x=np.ascontiguousarray(
                s0.x_ref + jr.normal(0.0, synth.JITTER_SIGMA, size=s0.x_ref.shape))))
        S = ffmin.System(systems, ffmin.FFMIN_FP64)
        x = torch.tensor(np.concatenate([s.x.reshape(-1) for s in systems]), dtype=torch.float64,
                         device="cuda")
        r = S.minimize(x.clone(), method="LBFGS", max_iter=args.profile_vectors, host_loop=HOST_LOOP)
        torch.cuda.synchronize()
        print("profile-vectors", S.last_stats(), sorted({q["iterations"] for q in r}))
        S.close()
        return
    if args.profile_minimize:
        s = synth.make_system(3334, 2)
        x = torch.tensor(s.x.reshape(-1), dtype=torch.float64, device="cuda")
        S = ffmin.System([s], ffmin.FFMIN_MIXED)
        S.minimize(x.clone(), method="LBFGS", max_iter=2, host_loop=HOST_LOOP)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        r = S.minimize(x.clone(), method="LBFGS", max_iter=args.profile_minimize, host_loop=HOST_LOOP)
        ev1.record()
        torch.cuda.synchronize()
        st = S.last_stats()
        print("profile-minimize", r[0]["iterations"], st, "ms", ev0.elapsed_time(ev1),
              "ms/tick", ev0.elapsed_time(ev1) / st["ticks"])
        S.close()
        return
    # FP64 first (k_pair64_sym: E + grad, then E only), then MIXED (k_pair:
    # E + grad, E only, then a difference trial, i.e. the E + grad of its base
    # and the trial itself); the MIXED object's FP64 kernel launches are empty
    s = synth.make_system(args.profile_atoms, SEED)
    x = torch.tensor(s.x.reshape(-1), dtype=torch.float64, device="cuda")
    r = -torch.ones_like(x) / math.sqrt(x.numel())
    for prec in (ffmin.FFMIN_FP64, ffmin.FFMIN_MIXED):
        S = ffmin.System([s], prec)
        e, g = S.energy_grad(x)
        e1 = S.energy(x)
        if prec == ffmin.FFMIN_MIXED:
            S.energy_delta(x, r, 0.01)
        torch.cuda.synchronize()
        print("profile", prec, e[0], e1[0])
        S.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ffmin")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-minimize", action="store_true", help="skip the minimizations/s runs")
    ap.add_argument("--no-methods", action="store_true", help="skip the per-method 3,334-atom runs")
    ap.add_argument("--profile", action="store_true", help="small fixed workload for ncu")
    ap.add_argument("--profile-atoms", type=int, default=N_ATOMS)
    ap.add_argument("--profile-minimize", type=int, default=0)
    ap.add_argument("--profile-batch", type=int, default=0)
    ap.add_argument("--profile-vectors", type=int, default=0)
    ap.add_argument("--profile-epochs", type=int, default=0)
    ap.add_argument("--host-loop", action="store_true",
                    help="minimizations replay their rounds from the host (for kernel-level profiling)")
    args = ap.parse_args()
    global HOST_LOOP
    HOST_LOOP = int(args.host_loop)
    if args.profile:
        profile_run(args)
    elif args.impl == "reference":
        bench_reference(args)
    else:
        bench_gpu(args)


if __name__ == "__main__":
    main()
