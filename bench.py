"""Benchmark of the evidence hot path (one step = one full evidence solve:
discover + refine + laplace) on the seeded synthetic d=1024, K=8 mixture.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sb|reference]
                    [--workload 4] [--prec bf16|tf32|fp64]

Prints one JSON line (rank 0). `--impl reference` times the FP64 CPU oracle on
the host cores (the benchmark's reference arm) on a bounded sample of the
same workload. Under torchrun each rank solves its own replica (no data-path
collective); value = evaluations of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# DRAM bytes per algorithmic byte of the L-BFGS step with bf16 pairs: ncu
# dram__bytes_read.sum + dram__bytes_write.sum of step launches 40-42 of a solve at
# d=1024, K=8, 8192 walkers (2.831 GB in all) against the step's own algorithmic-byte
# count for the same three launches (4.889 GB). The second pass of the two-loop
# recursion is served by the shared-memory ring (the newest groups) and L2.
LBFGS_DRAM_PER_ALGORITHMIC_BYTE = 0.579

METRIC = "logL+grad evals/sec and evidence solves/sec at d=1024 K=8 vs plain FP64 GPU; |ΔlogZ|"
PREC = {"fp64": 0, "tf32": 1, "bf16": 2}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sb", choices=["sb", "reference"])
    ap.add_argument("--workload", type=int, default=4,
                    help="0: d=8 Gaussian; 1: d=64 K=4 mixture; 2: d=256 correlated Gaussian; "
                         "3: 512 batched mixtures; 4: d=1024 K=8 mixture")
    ap.add_argument("--adjoint", action="store_true",
                    help="time the forward solve and the d log Z / d (mu, L) adjoint (one JSON line)")
    ap.add_argument("--chisao", action="store_true",
                    help="time discovery + the ChiSao oscillation (one JSON line): FP64 on the d=64 K=4 mixture, "
                         "or --chisao-workload 4 for the d=1024 K=8 mixture at --prec")
    ap.add_argument("--chisao-workload", type=int, default=1, choices=[1, 4])
    ap.add_argument("--next-rows", action="store_true",
                    help="time the preprocessing probe, the V2V/V2E/W2W segment pass and the black-box "
                         "derivatives (one JSON line)")
    ap.add_argument("--prec", default=None, choices=list(PREC),
                    help="likelihood precision; default the workload's own: fp64 for 0 and 1, tf32 for 3, "
                         "bf16 for 2 (which reports every precision) and 4")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-chisao", action="store_true",
                    help="headline step without ChiSao (sunburst-only discovery, refinement, Laplace)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU comparator")
    ap.add_argument("--fp64-scale", type=float, default=1.0 / 32,
                    help="ray and start counts of the FP64 comparator solve, as a fraction of the workload's")
    # profiling cases (small, for ncu captures; not bench lines)
    ap.add_argument("--kernel-only", action="store_true",
                    help="time only the tensor-core l+grad contraction on --n-points points")
    ap.add_argument("--n-points", type=int, default=16384)
    ap.add_argument("--scale", type=float, default=None, help="scale ray/start counts (profiling only)")
    args = ap.parse_args()
    if args.prec is None:
        args.prec = {0: "fp64", 1: "fp64", 2: "bf16", 3: "tf32", 4: "bf16"}[args.workload]
    return args


def workload_cfg(wid, prec, scale=None):
    from paper_2601_19957_gb300.instances import workload

    insts, cfg = workload(wid, scale=scale)
    cfg.prec = PREC[prec]
    if wid == 4:
        cfg.cand_cap = 64  # Hessians of 64 candidates at d=1024 = 512 MB of scratch
    return insts[0], cfg


def workload_name(wid, inst, cfg, chisao=None):
    name = (f"seeded synthetic Gaussian mixture d={inst.d} K={inst.K}, uniform prior [-10,10]^d, "
            f"{cfg.n_rays} sunburst rays x {cfg.n_steps} steps, {cfg.n_starts} L-BFGS starts, m={cfg.m}")
    if chisao is True:
        name += ", ChiSao 3 oscillations (anti-convergence step 0.1), Laplace stage over every final sample"
    elif chisao is False:
        name += ", sunburst-only discovery"
    return name


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.proc = None
        self.lines = []
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ----------------------------------------------------------------------------- cpu baseline
def cpu_baseline(inst, cfg, seconds):
    """The FP64 oracle as it stands, on the host cores: a whole oracle solve at
    d=1024 is far too slow for a bounded sample, so the sample is l+grad
    evaluations of oracle L-BFGS on batches of walkers started at seeded points
    spread over the prior box, each batch run to its end, until about
    `seconds` of wall time."""
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(7)
    # batches of `cores` walkers from seeded points spread over the prior box
    # (like ray samples), each run to its own end, until about `seconds` of
    # wall time is spent
    n_walk = max(cores, 1)
    evals, batches, t_total = 0, 0, 0.0
    while t_total < seconds and batches < 64:
        x0 = rng.uniform(inst.lo, inst.hi, (n_walk, inst.d))
        t0 = time.perf_counter()
        r = oracle.lbfgs(inst, cfg, x0, n_threads=cores)
        t_total += time.perf_counter() - t0
        evals += int(r.evals)
        batches += 1
    return {"value": evals / t_total, "unit": "evals/s", "cores": cores, "kind": "oracle",
            "sample": f"{evals} l+grad evaluations of FP64 oracle L-BFGS ({batches} batches of {n_walk} walkers "
                      f"from box-uniform starts, d={inst.d}, K={inst.K}) in {t_total:.1f} s"}


# ----------------------------------------------------------------------------- dist helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_over_ranks(t_seconds, evals, dist, device):
    """Replicas: whole-job time is the slowest rank's, work is the sum over ranks."""
    import torch

    tt = torch.tensor([float(t_seconds)], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ev = torch.tensor([float(evals)], device=device, dtype=torch.float64)
    dist.all_reduce(ev, op=dist.ReduceOp.SUM)
    return float(tt.item()), int(ev.item())


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    import torch

    import paper_2601_19957_gb300 as sb
    from paper_2601_19957_gb300 import build as sbbuild

    sbbuild.build()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload == 3:
        return run_batched(sb, args)
    if args.workload == 2:
        return run_precision(sb, args)
    if args.adjoint:
        return run_adjoint(sb, args)
    if args.chisao:
        return run_chisao(sb, args)
    if args.next_rows:
        return run_next_rows(sb, args)
    inst, cfg = workload_cfg(args.workload, args.prec, args.scale)
    prob = sb.Problem(inst)
    c = sb.make_config(cfg)
    if args.kernel_only:
        return kernel_only(sb, inst, prob, cfg, args)
    use_chisao = not args.no_chisao
    cc = sb.make_chisao_config()
    wsp = sb.chisao_workspace(prob, c) if use_chisao else sb.workspace(prob, c)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 512 MB > L2
    L = sb.lib()
    logV = float(np.log(inst.hi - inst.lo).sum())
    closed = float(np.log(np.exp(inst.log_w).sum())) - logV

    bufs = sb.EvidenceBuffers(inst.d, c.cand_cap)  # the same outputs every step: one cached graph

    def one_step():
        if use_chisao:
            return sb.evidence_chisao(prob, c, cc, ws=wsp, out=bufs, sync_check=False)
        return sb.evidence(prob, c, ws=wsp, sync_check=False, out=bufs)

    def counts():
        """(l-only evaluations, l+grad evaluations, modes kept) of the last step."""
        if use_chisao:
            ray, lb, anti, nm = sb.chisao_stats(prob, c, wsp)
            return ray, lb + anti, nm
        st = (sb.C.c_int64 * 4)()
        L.sb_evidence_stats(sb.C.byref(prob.s), sb.C.byref(c), wsp.ptr, sb.C.c_size_t(wsp.nbytes), st, sb._stream())
        return int(st[0]), int(st[1]), int(st[3])

    for _ in range(args.warmup):
        out = one_step()

    # timed region: CUDA events around the steps on the launching stream; profiling off, so
    # every step replays the library's cached CUDA graph (the refinement's loop a
    # device-decided WHILE node)
    clk = ClockSampler(local)
    clk.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times, n_l, n_lg = [], 0, 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = one_step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        a1, a2, _ = counts()
        n_l += a1
        n_lg += a2
    torch.cuda.synchronize()
    clocks = clk.stop()
    t_total = sum(times) / 1e3
    if dist:
        t_total, n_lg = reduce_over_ranks(t_total, n_lg, dist, "cuda")
    value = n_lg / t_total
    ms_per_step = 1e3 * t_total / args.steps
    l_per_step, lg_per_step, n_modes = counts()

    # the same steps run eagerly with CUDA events around every launch of the dominant
    # kernel class (the L-BFGS step): its per-launch time, algorithmic bytes and the
    # launch count per step (the timed graph replays launch the same kernels)
    L.sb_profile_read(None, None)
    L.sb_profile_bytes(3)
    L.sb_profile_classes(1 << 3)
    launches0 = L.sb_launch_count()
    eager_times = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one_step()
        e1.record(stream)
        e1.synchronize()
        eager_times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    launches = (L.sb_launch_count() - launches0) // args.steps * args.steps
    L.sb_profile_classes(0)
    lb_ms_c = (sb.C.c_double * 8)()
    lb_n_c = (sb.C.c_int64 * 8)()
    L.sb_profile_read(lb_ms_c, lb_n_c)
    lb_bytes = L.sb_profile_bytes(3)  # algorithmic bytes of the L-BFGS step launches in those steps

    # per-class device time from a separate pass (events around every launch), untimed
    L.sb_profile_enable(1)
    prof_steps = 2
    for _ in range(prof_steps):
        one_step()
    torch.cuda.synchronize()
    L.sb_profile_enable(0)
    prof_ms = (sb.C.c_double * 8)()
    prof_n = (sb.C.c_int64 * 8)()
    L.sb_profile_read(prof_ms, prof_n)
    L.sb_profile_bytes(3)

    dlogZ = abs(out.logZ - closed)
    modes = out.modes.cpu().numpy()
    found = sorted({int(np.argmin(np.abs(inst.mu - m).max(1))) for m in modes})
    closed_found = float(np.log(np.exp(inst.log_w[found]).sum())) - logV if found else -math.inf
    dlogZ_found = abs(out.logZ - closed_found) if found else None
    accuracy_met = len(found) == inst.K and dlogZ <= 1e-9

    d, K = inst.d, inst.K
    names = ["tc_z_walkers", "tc_z_rays", "tc_grad", "lbfgs_step", "f64_z", "f64_grad", "cholesky", "other"]
    share = {names[i]: {"ms_per_step": prof_ms[i] / prof_steps, "launches_per_step": int(prof_n[i]) // prof_steps}
             for i in range(8) if prof_n[i]}
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "of measured" if peaks else "of fallback"
    lb_ms, lb_n = lb_ms_c[3], max(int(lb_n_c[3]), 1)
    if cfg.prec == 0:
        roof = fp64_roofline(sb, prof_ms, prof_n, prof_steps, lg_per_step, d, K)
    else:
        per_launch = lb_bytes / lb_n
        achieved = lb_bytes / (lb_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": per_launch * LBFGS_DRAM_PER_ALGORITHMIC_BYTE if cfg.prec == 2 else None,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of k_lbfgs_cta launches, as a "
                                  "fraction of their algorithmic bytes, times this run's algorithmic bytes per launch",
                "kernel": "k_lbfgs_cta (FP32 L-BFGS step, bf16 pairs)", "peak_source": peak_src + " HBM copy",
                "algorithmic_bytes_per_launch": per_launch, "ms_per_launch": lb_ms / lb_n,
                "launches_timed": int(lb_n_c[3]),
                "timing": "CUDA events around every k_lbfgs_cta launch of an eager pass of the same steps "
                          "(profiling off in the timed steps)"}

    res = {
        "metric": METRIC,
        "value": value,
        "unit": "evals/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {0: "f64", 1: "tf32", 2: "bf16"}[cfg.prec],
        "data": "synthetic",
        "config": {"workload": workload_name(args.workload, inst, cfg, use_chisao),
                   "d": d, "K": K, "n_rays": cfg.n_rays, "n_steps": cfg.n_steps, "n_starts": cfg.n_starts,
                   "m": cfg.m, "prec": args.prec, "laplace": "fp64", "chisao": use_chisao,
                   "parallelism": f"replicas x{ws}",
                   "l2": "512 MB buffer zeroed between timed steps; per-step working set > L2",
                   "evals_counted": "value: l+grad evaluations (L-BFGS walkers and anti-convergence steps); "
                                    "l-only evaluations at ray samples are reported apart"},
        "solves_per_sec": ws * args.steps / t_total,
        "lgrad_evals_per_step": lg_per_step,
        "l_only_evals_per_step": l_per_step,
        "l_only_evals_per_sec": ws * args.steps * l_per_step / t_total,
        "n_modes": n_modes,
        "logZ": out.logZ,
        "logZ_closed_form": closed,
        "abs_dlogZ_vs_closed_form": dlogZ,
        "abs_dlogZ_given_found_modes": dlogZ_found,
        "components_found": f"{len(found)}/{inst.K}",
        "accuracy_met": accuracy_met,
        "accuracy_target": "every component found and |dlogZ| vs closed form <= 1e-9",
        "gpu_launches": int(launches),
        "gpu_launches_source": "library launch counter over an eager pass of the same steps (the timed steps replay "
                               "one CUDA graph that launches the same kernels)",
        "execution": "CUDA graph replay (device-decided refinement loop; no host reads inside a step)",
        "eager_ms_per_step": sum(eager_times) / len(eager_times),
        "clocks": clocks,
        "roofline": roof,
        "kernel_ms": share,
        "kernel_ms_source": f"separate profiled pass of {prof_steps} steps (CUDA events around every launch)",
        "step_ms": [round(t, 3) for t in times],
    }
    if rank == 0 and not args.no_e2e:
        res["e2e"] = e2e_measure(sb, inst, cfg, c, cc if use_chisao else None, args, lg_per_step, flush)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(inst, cfg, args.cpu_seconds)
    if rank == 0 and not args.no_fp64 and args.prec != "fp64":  # an FP64 line is its own comparator
        res["fp64_gpu"] = fp64_comparator(sb, args, use_chisao)
        res["fp64_peak"] = fp64_peak(sb)
    if rank == 0:
        print(json.dumps(res))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def fp64_roofline(sb, prof_ms, prof_n, prof_steps, lg_per_step, d, K):
    """FP64 path: its z and gradient contractions against the measured FP64 FMA peak."""
    peak = fp64_peak(sb)["tflops"] * 1e3
    ms = (prof_ms[4] + prof_ms[5]) / prof_steps
    gflops = lg_per_step * 2 * K * d * (d + 1) / (ms / 1e3) / 1e9
    return {"bound": "alu", "achieved": gflops, "peak": peak, "unit": "GFLOP/s", "frac": gflops / peak,
            "traffic": None, "kernel": "f64_z + f64_grad", "peak_source": "of measured FP64 FMA loop (fp64_peak)"}


def run_adjoint(sb, args):
    """Forward log Z (the headline solve: discovery, ChiSao, Laplace over every final
    sample; sunburst-only with --no-chisao) and the hand-written adjoint d log Z / d mu_k,
    d log Z / d L_k (FP64, H recomputed at each mode) on the d=1024, K=8 workload."""
    import torch

    inst, cfg = workload_cfg(args.workload, args.prec, args.scale)
    prob = sb.Problem(inst)
    c = sb.make_config(cfg)
    use_chisao = not args.no_chisao
    cc = sb.make_chisao_config()
    wsp = sb.chisao_workspace(prob, c) if use_chisao else sb.workspace(prob, c)
    forward = (lambda: sb.evidence_chisao(prob, c, cc, ws=wsp)) if use_chisao else (lambda: sb.evidence(prob, c, ws=wsp))
    out = forward()
    for _ in range(max(args.warmup, 1)):
        sb.evidence_backward(prob, out.modes, out.logZk, out.n_modes)
    torch.cuda.synchronize()
    reps = max(args.steps, 1)
    t0 = time.perf_counter()
    for _ in range(reps):
        dmu, dL = sb.evidence_backward(prob, out.modes, out.logZk, out.n_modes)
    torch.cuda.synchronize()
    dt_b = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        out = forward()
    torch.cuda.synchronize()
    dt_f = (time.perf_counter() - t0) / reps
    d, K, nm = inst.d, inst.K, out.n_modes
    # the blocked Cholesky runs where a mode is not one-hot: an overlapping pair of
    # components at the same d (means 2 apart, standard deviations 0.6-1, as in the
    # adjoint's GPU test), whose backward pass factors H at both modes (d^3 / 3 flop
    # each); CUDA events around the factorisation alone in one backward call
    import numpy as np
    from paper_2601_19957_gb300.instances import SolveConfig, make_instance

    ov = make_instance(d, 2, 41, s_range=(0.6, 1.0), mean_box=(-3, 3), sep=0.0, prior=(-12.0, 12.0))
    e = np.random.default_rng(3).normal(size=d)
    ov.mu[1] = ov.mu[0] + 2.0 * e / np.linalg.norm(e)
    ov = ov.contiguous()
    pov = sb.Problem(ov)
    cov = sb.make_config(SolveConfig(n_rays=256, n_steps=64, n_starts=256, m=20, seed=5, prec=PREC["bf16"],
                                     cand_cap=16))
    oo = sb.evidence(pov, cov)
    sb.evidence_backward(pov, oo.modes, oo.logZk, oo.n_modes)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        sb.evidence_backward(pov, oo.modes, oo.logZk, oo.n_modes)
    torch.cuda.synchronize()
    dt_ov = (time.perf_counter() - t0) / reps
    L = sb.lib()
    L.sb_profile_read(None, None)
    L.sb_profile_classes(1 << 6)
    sb.evidence_backward(pov, oo.modes, oo.logZk, oo.n_modes)
    torch.cuda.synchronize()
    L.sb_profile_classes(0)
    prof_ms = (sb.C.c_double * 8)()
    prof_n = (sb.C.c_int64 * 8)()
    L.sb_profile_read(prof_ms, prof_n)
    peak = fp64_peak(sb)
    chol = {"workload": f"d={d}, two overlapping components (means 2 apart), {oo.n_modes} modes not one-hot",
            "ms_backward": dt_ov * 1e3, "factorizations": int(prof_n[6]), "peak_source": peak["source"],
            "fp64_peak_TFLOPs": peak["tflops"]}
    if prof_n[6] > 0:
        chol_ms = prof_ms[6] / int(prof_n[6])
        rate = d ** 3 / 3.0 / (chol_ms / 1e3) / 1e12
        chol.update({"ms_per_factorization": chol_ms, "fp64_TFLOPs": rate, "frac": rate / peak["tflops"]})
    print(json.dumps({"case": "adjoint", "workload": f"d={d} K={K}, {cfg.n_starts} starts, m={cfg.m}",
                      "forward": "discovery + ChiSao + Laplace" if use_chisao else "sunburst-only discovery + Laplace",
                      "n_modes": nm, "ms_forward": dt_f * 1e3, "ms_backward": dt_b * 1e3, "overlapping_modes": chol,
                      "backward_fp64_flop_model": 2.0 * nm * d ** 3,
                      "max_abs_dmu": float(dmu.abs().max()), "max_abs_dL": float(dL.abs().max())}))
    return 0


def run_chisao(sb, args):
    """Discovery followed by the ChiSao oscillation (3 oscillations, one sample per discovered
    start): FP64 on the d=64, K=4 mixture, or the d=1024, K=8 mixture at the mixed precision
    given by --prec; one step = sb_discover + sb_chisao. Reports
    the time per step, the device time per kernel class, and the components found as peaks
    against those whose peak passes the stick test and against the plain evidence solve."""
    import torch

    wid = args.chisao_workload
    prec = "fp64" if wid == 1 else args.prec
    inst, cfg = workload_cfg(wid, prec, args.scale)
    prob = sb.Problem(inst)
    c = sb.make_config(cfg)
    cc = sb.make_chisao_config()
    wsc = sb.chisao_workspace(prob, c)
    L = sb.lib()

    def step():
        starts, _ = sb.discover(prob, c, ws=wsc)
        return sb.chisao(prob, c, cc, starts, ws=wsc)

    for _ in range(max(args.warmup, 1)):
        out = step()
    torch.cuda.synchronize()
    L.sb_profile_enable(1)
    launches0 = L.sb_launch_count()
    t0 = time.perf_counter()
    reps = max(args.steps, 1)
    for _ in range(reps):
        out = step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    launches = (L.sb_launch_count() - launches0) // reps
    L.sb_profile_enable(0)
    prof_ms = (sb.C.c_double * 8)()
    prof_n = (sb.C.c_int64 * 8)()
    L.sb_profile_read(prof_ms, prof_n)
    peaks = out.x[out.stuck].cpu().numpy()
    found = sorted({int(np.argmin(np.abs(inst.mu - m).max(1))) for m in peaks})
    heights = sb.loglik(prob, torch.as_tensor(inst.mu, device="cuda"), want_grad=False).cpu().numpy()
    expect = [int(k) for k in np.flatnonzero(heights >= heights.max() + math.log(0.1))]
    plain = sb.evidence(prob, c, ws=wsc)
    plain_found = sorted({int(np.argmin(np.abs(inst.mu - m).max(1))) for m in plain.modes.cpu().numpy()})
    # the stick rule keeps only peaks within log 10 of the highest; the Laplace stage run on
    # every final sample shows which components the oscillation reached
    lap = sb.laplace(prob, c, out.x, out.ell, ws=wsc)
    # the whole pipeline through its own entry point (discover, ChiSao, Laplace over every sample)
    sb.evidence_chisao(prob, c, cc, ws=wsc)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for _ in range(reps):
        full = sb.evidence_chisao(prob, c, cc, ws=wsc)
    torch.cuda.synchronize()
    dt_full = (time.perf_counter() - t1) / reps
    lap_found = sorted({int(np.argmin(np.abs(inst.mu - m).max(1))) for m in lap.modes.cpu().numpy()})
    logV = float(np.log(inst.hi - inst.lo).sum())
    closed = float(np.log(np.exp(inst.log_w).sum())) - logV
    names = ["tc_z_walkers", "tc_z_rays", "tc_grad", "lbfgs_step_f32", "f64_z", "f64_grad", "cholesky", "other"]
    print(json.dumps({"case": "chisao", "workload": workload_name(wid, inst, cfg) + f", {prec}, 3 oscillations",
                      "ms_per_step": dt * 1e3, "steps": reps, "launches_per_step": int(launches),
                      "n_peaks": out.n_peaks, "components_found": found, "components_passing_stick_test": expect,
                      "components_found_without_chisao": plain_found,
                      "components_found_by_laplace_on_all_final_samples": lap_found,
                      "logZ_laplace_on_all_final_samples": lap.logZ, "logZ_closed_form_all_components": closed,
                      "logZ_without_chisao": plain.logZ,
                      "ms_per_evidence_chisao": dt_full * 1e3, "evidence_chisao_n_modes": full.n_modes,
                      "evidence_chisao_logZ": full.logZ,
                      "device_ms_per_step": {nm: prof_ms[i] / reps for i, nm in enumerate(names) if prof_n[i]}}))
    return 0


def run_next_rows(sb, args):
    """Device time of the preprocessing probe, the segment pass and the experimental quadratic
    coarse pass (FP32 form, 16384 rays x 64 steps) on the d=1024, K=8 mixture and of the
    black-box derivatives (full Hessian) on the d=64, K=4 mixture, each with its
    algorithmic work: the probe reads the L_k twice (2 K d^2 x 8 B); the segment pass does one
    FP64 z GEMM over 2 n_rays end points (2 n_rays K d(d+1)/2 multiply-adds); the derivatives
    evaluate l at 2 d^2 + 2d + 3 points (K d(d+1) flop each)."""
    import torch

    reps = max(args.steps, 1)

    def timed(fn):
        for _ in range(max(args.warmup, 1)):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    big, _ = workload_cfg(4, "fp64")
    pb = sb.Problem(big)
    d, K = big.d, big.K
    ms_pre = timed(lambda: sb.precheck(pb))
    n_rays, n_steps, n_ref = 4096, 64, 64
    ms_seg = timed(lambda: sb.segments(pb, sb.RAY_W2W, 7, n_rays, n_steps, 10.0, n_ref))
    g = torch.Generator(device="cpu").manual_seed(11)
    U = torch.randn((16384, d), generator=g, dtype=torch.float64)
    U = (U / U.norm(dim=1, keepdim=True)).cuda()
    ms_rq = timed(lambda: sb.ray_loglik_quad(pb, U, 64, form=1))
    ms_rq2 = timed(lambda: sb.ray_loglik_quad(pb, U, 64, form=2))
    small, _ = workload_cfg(1, "fp64")
    ps = sb.Problem(small)
    x = torch.as_tensor(small.mu[0] + 0.1, device="cuda")
    ms_fd = timed(lambda: sb.fd_derivatives(ps, x, full=True))
    ds, Ks = small.d, small.K
    pts = 2 * ds * ds + 2 * ds + 3
    print(json.dumps({"case": "next-rows",
                      "precheck": {"workload": f"d={d} K={K}", "ms": ms_pre,
                                   "algorithmic_GBps": 2 * K * d * d * 8 / (ms_pre * 1e-3) / 1e9},
                      "segments": {"workload": f"d={d} K={K}, W2W, {n_rays} rays x {n_steps} + {n_ref} samples",
                                   "ms": ms_seg,
                                   "fp64_TFLOPs": 2 * n_rays * K * d * (d + 1) / (ms_seg * 1e-3) / 1e12},
                      "ray_loglik_quad_f32": {"workload": f"d={d} K={K}, 16384 rays x 64 steps", "ms": ms_rq,
                                              "fp32_TFLOPs": 16384 * K * d * (d + 1) / (ms_rq * 1e-3) / 1e12},
                      "ray_loglik_quad_bf16_split": {"workload": f"d={d} K={K}, 16384 rays x 64 steps", "ms": ms_rq2,
                                                     "tensor_TFLOPs_3_products":
                                                         3 * 16384 * K * d * (d + 1) / (ms_rq2 * 1e-3) / 1e12},
                      "fd_full_hessian": {"workload": f"d={ds} K={Ks}, {pts} points", "ms": ms_fd,
                                          "l_evals_per_s": pts / (ms_fd * 1e-3)}}))
    return 0


def run_precision(sb, args):
    """Precision table: |dlogZ| per likelihood dtype, with and without the FP64 Newton polish,
    on the d=256 correlated Gaussian (s log-uniform in [0.01, 1], condition number up to 1e4;
    log Z = -log V exactly). Also the evidence solves/sec of each form."""
    import torch
    from paper_2601_19957_gb300.instances import workload

    insts, cfg = workload(2, scale=args.scale)
    inst = insts[0]
    prob = sb.Problem(inst)
    closed = -float(np.log(inst.hi - inst.lo).sum())
    out = {"case": "precision", "workload": "d=256 correlated Gaussian, s in [0.01,1], 8192 starts, m=10",
           "closed_form_logZ": closed, "rows": []}
    for pname in ("fp64", "tf32", "bf16"):
        for ns in (0, 3):
            c = sb.make_config(cfg, prec=PREC[pname], newton_steps=ns)
            ws = sb.workspace(prob, c)
            sb.evidence(prob, c, ws=ws)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            reps = max(1, args.steps)
            for _ in range(reps):
                r = sb.evidence(prob, c, ws=ws)
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t0) / reps
            out["rows"].append({"prec": pname, "newton_steps": ns, "n_modes": r.n_modes, "logZ": r.logZ,
                                "abs_dlogZ": abs(r.logZ - closed), "rel_dlogZ": abs(r.logZ - closed) / abs(closed),
                                "ms_per_solve": dt * 1e3})
    print(json.dumps(out))
    return 0


def run_batched(sb, args):
    """Batched mixtures: 512 independent problems (d in {16..512}, K in 1..8, TF32 likelihood,
    FP64 Laplace) per step, one library call; in graph mode the whole batch is one cached
    CUDA graph (one launch per step)."""
    import torch
    from paper_2601_19957_gb300.instances import workload

    insts, cfg = workload(3, scale=args.scale)
    cfg.prec = PREC[args.prec]
    cfg.cand_cap = 32
    probs = [sb.Problem(i) for i in insts]
    c = sb.make_config(cfg)
    workers = 16
    use_chisao = not args.no_chisao
    cc = sb.make_chisao_config() if use_chisao else None
    ws = sb.batched_workspace(probs, c, workers, chisao=use_chisao)
    out = (torch.empty(len(probs), dtype=torch.float64, device="cuda"),
           torch.empty(len(probs), dtype=torch.int32, device="cuda"))
    t0 = time.perf_counter()
    sb.evidence_batched(probs, c, n_workers=workers, ws=ws, out=out, cc=cc)  # tunes the tiles, captures the graph
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0
    for _ in range(max(args.warmup - 1, 0)):
        sb.evidence_batched(probs, c, n_workers=workers, ws=ws, out=out, cc=cc)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        logZ, nm = sb.evidence_batched(probs, c, n_workers=workers, ws=ws, out=out, cc=cc)
    e1.record(stream)
    e1.synchronize()
    dt = e0.elapsed_time(e1) / 1e3 / args.steps
    lz = logZ.cpu().numpy()
    nmv = nm.cpu().numpy()
    logV = np.array([np.log(i.hi - i.lo).sum() for i in insts])
    closed = np.array([np.log(np.exp(i.log_w).sum()) for i in insts]) - logV
    allk = nmv == np.array([i.K for i in insts])
    print(json.dumps({"case": "batched", "workload": "512 problems, d in {16..512}, K in 1..8, 256 starts each, "
                                                     "m=10, TF32 likelihood, FP64 Laplace"
                                                     + (", ChiSao 3 oscillations" if use_chisao else ""),
                      "problems": len(insts), "ms_per_batch": dt * 1e3, "problems_per_sec": len(insts) / dt,
                      "prec": {1: "tf32", 2: "bf16", 0: "fp64"}[cfg.prec], "workers": workers,
                      "execution": "one cached CUDA graph per call (device-decided refinement loops)",
                      "first_call_s": first_s, "steps": args.steps,
                      "all_K_found": int(allk.sum()),
                      "max_abs_dlogZ_where_all_found": float(np.max(np.abs(lz - closed)[allk], initial=0.0))}))
    return 0


def kernel_only(sb, inst, prob, cfg, args):
    """The tensor-core l+grad contraction alone (profiling case)."""
    import torch

    rng = np.random.default_rng(3)
    n = args.n_points
    X = torch.as_tensor(inst.mu[rng.integers(0, inst.K, n)] + rng.normal(0, 0.3, (n, inst.d)), device="cuda")
    wsl = sb.Workspace(sb.lib().sb_loglik_workspace_bytes(sb.C.byref(prob.s), cfg.prec, n))
    for _ in range(args.warmup):
        sb.loglik(prob, X, prec=cfg.prec, ws=wsl)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        sb.loglik(prob, X, prec=cfg.prec, ws=wsl)
    e1.record()
    e1.synchronize()
    dt = e0.elapsed_time(e1) / 1e3 / max(args.steps, 1)
    flop = n * 2 * inst.K * inst.d * (inst.d + 1)
    print(json.dumps({"case": "kernel-only", "n": n, "d": inst.d, "K": inst.K, "prec": args.prec,
                      "ms": dt * 1e3, "evals_per_sec": n / dt, "algorithmic_tflops": flop / dt / 1e12}))
    return 0


def e2e_measure(sb, inst, cfg, c, cc, args, lg_per_step, flush):
    """The same metric through the host-buffer entry point (sb_evidence_chisao_host, or
    sb_evidence_host without ChiSao): page-locked host arrays in, log Z and the modes out,
    every copy inside the timed call; the L2 flush runs before each call, outside it."""
    import torch

    host = sb.PinnedHost(inst, c)
    if cc is not None:
        wsh = sb.evidence_chisao_host_workspace(inst, c)
        call = lambda: sb.evidence_chisao_host(inst, c, cc, wsh, host=host)
    else:
        wsh = sb.evidence_host_workspace(inst, c)
        call = lambda: sb.evidence_host(inst, c, wsh, host=host)
    call()  # warm
    times = []
    for _ in range(max(1, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        logZ, modes, zk, nm = call()  # synchronises: its outputs are on the host when it returns
        times.append(time.perf_counter() - t0)
    dt = sum(times) / len(times)
    h2d = 8 * (inst.K + inst.K * inst.d + inst.K * inst.d * inst.d + 2 * inst.d)
    d2h = 8 + 4 + 8 * min(nm, cfg.cand_cap) * (inst.d + 1)
    return {"value": lg_per_step / dt, "unit": "evals/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": dt * 1e3, "steps": len(times), "host_memory": "pinned",
            "entry_point": "sb_evidence_chisao_host" if cc is not None else "sb_evidence_host",
            "l2": "512 MB buffer zeroed before each call (outside the timed call)", "logZ": logZ}


def fp64_comparator(sb, args, use_chisao):
    """Plain FP64 GPU path (every stage FP64 on CUDA cores) on the same instance, with the
    ray and start counts scaled by --fp64-scale (an FP64 solve at full counts takes minutes),
    next to the mixed-precision path at the same counts."""
    import torch

    out = {"scale": args.fp64_scale}
    for name in ("fp64", args.prec):
        inst, cfg = workload_cfg(args.workload, name, args.fp64_scale)
        prob = sb.Problem(inst)
        c = sb.make_config(cfg)
        cc = sb.make_chisao_config()
        ws = sb.chisao_workspace(prob, c) if use_chisao else sb.workspace(prob, c)
        bufs = sb.EvidenceBuffers(inst.d, c.cand_cap)
        solve = ((lambda: sb.evidence_chisao(prob, c, cc, ws=ws, out=bufs)) if use_chisao
                 else (lambda: sb.evidence(prob, c, ws=ws, out=bufs)))
        if name != "fp64":
            solve()  # warm (the FP64 leg's warm-up is its own first launch set; one solve is long)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        r = solve()
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        if use_chisao:
            ray, lb, anti, _ = sb.chisao_stats(prob, c, ws)
            lg = lb + anti
        else:
            st = (sb.C.c_int64 * 4)()
            sb.lib().sb_evidence_stats(sb.C.byref(prob.s), sb.C.byref(c), ws.ptr, sb.C.c_size_t(ws.nbytes), st,
                                       sb._stream())
            ray, lg = int(st[0]), int(st[1])
        logV = float(np.log(inst.hi - inst.lo).sum())
        closed = float(np.log(np.exp(inst.log_w).sum())) - logV
        found = sorted({int(np.argmin(np.abs(inst.mu - m).max(1))) for m in r.modes.cpu().numpy()})
        out[name] = {"ms_per_solve": ms, "solves_per_sec": 1e3 / ms, "lgrad_evals_per_sec": lg / (ms / 1e3),
                     "lgrad_evals": lg, "l_only_evals": ray, "n_starts": cfg.n_starts,
                     "components_found": f"{len(found)}/{inst.K}", "abs_dlogZ_vs_closed_form": abs(r.logZ - closed)}
    out["speedup_" + args.prec + "_vs_fp64_solves"] = out["fp64"]["ms_per_solve"] / out[args.prec]["ms_per_solve"]
    return out


def fp64_peak(sb):
    """FP64 FMA throughput of this GPU, measured by the library's own FMA loop kernel."""
    if not hasattr(fp64_peak, "cache"):
        tf = float(sb.lib().sb_fp64_fma_peak(None))
        fp64_peak.cache = {"tflops": tf, "source": "sb_fp64_fma_peak: independent FMA chains on every SM, "
                                                   "CUDA-event timed, best of 5"}
    return fp64_peak.cache


def run_reference(args, ws, rank):
    """Reference arm: the FP64 oracle on the host cores, same metric and config."""
    if rank != 0:
        return 0
    inst, cfg = workload_cfg(args.workload, args.prec)
    per_step = max(1.0, 60.0 / max(args.steps + args.warmup, 1))
    for _ in range(args.warmup):
        cpu_baseline(inst, cfg, min(per_step, 3.0))
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(inst, cfg, per_step))
    dt = time.perf_counter() - t0
    v = float(np.mean([r["value"] for r in vals]))
    res = {"metric": METRIC, "value": v, "unit": "evals/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": workload_name(args.workload, inst, cfg, not args.no_chisao), "d": inst.d,
                      "K": inst.K},
           "cpu_baseline": {"value": v, "unit": "evals/s", "cores": vals[0]["cores"], "kind": "oracle",
                            "sample": vals[0]["sample"]},
           "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res))
    return 0


if __name__ == "__main__":
    sys.exit(main() or 0)
