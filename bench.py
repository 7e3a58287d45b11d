"""Benchmark of one full FMM velocity evaluation (Fig. 1 stages 1-10) on GB300.

Default workload: N = 2^20 uniform particles in [0, 1)^2, gamma ~ N(0, 1)/N, sigma = 0.5/sqrt(N), depth 7,
p = 17, precision form (FP32 near field, FP32/FP64 sweep), CUDA-graph replay. One step = one evaluation on
inputs resident in HBM; L2 is flushed (a 256 MiB write) before every timed step, outside the timed events.

Prints ONE JSON line (rank 0). Extra keys: roofline of the dominant kernel (near-field P2P), cpu_baseline
(the FP64 oracle on the host cores), e2e (the host-buffer entry point with copies inside the timed region),
exposed sweep time, FP64-form throughput, accuracy of the precision form, clocks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload uniform_1m|patches_16m]
"""
from __future__ import annotations

import argparse
import csv
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mparticles/s per FMM eval @ rel-err ≤1e-6 (FP32 form vs FP64); exposed sweep ms"
P2P_FLOPS_PER_PAIR = 22  # §3 of the paper
SMS, FP32_LANES, MAX_SM_GHZ = 152, 128, 2.07
FP32_PEAK_TFLOPS = SMS * FP32_LANES * 2 * MAX_SM_GHZ / 1000.0  # 80.5 TFLOP/s at the maximum SM clock


def workload(name: str):
    import fmm_inputs as fi

    if name == "uniform_1m":
        return fi.uniform_1m(), "N=2^20 uniform in [0,1)^2, gamma~N(0,1)/N, sigma=0.5/sqrt(N), depth 7, p=17"
    if name == "patches_16m":
        return fi.patches_16m(), ("N=2^24 from 8 Gaussian patches (std 0.05, circulations +-1), sigma=0.5/sqrt(N), "
                                  "uniform depth 9, p=20")
    if name == "patches_4m":  # a smaller case of the same recipe, for counter captures
        return (fi.patches(1 << 22, seed_index=2, depth=8, p=20, name="patches_4m"),
                "N=2^22 from 8 Gaussian patches, sigma=0.5/sqrt(N), uniform depth 8, p=20")
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for r in csv.reader(fh):
                if len(r) >= 9:
                    rows.append([c.strip() for c in r])
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def whole_job(total_ms: float, steps: int, n_per_rank: int, world: int, dist=None, device: str = "cpu"):
    """(ms per step, Mparticles/s) of the whole job: every rank evaluates its own replica on its own GPU, so the
    job takes as long as the slowest rank (max over ranks of its timed total) and processes world x n particles
    per step."""
    if dist is not None and world > 1:
        import torch

        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / steps
    return ms_per_step, world * n_per_rank / (ms_per_step / 1e3) / 1e6


def timed_steps(fn, steps: int, flush, stream, stage_times=None, stage_index: int = 1):
    """Per-step device time (ms) with CUDA events on the launching stream; L2 flushed before each step. With
    stage_times, also the handle's stage time number stage_index of every step (1: near field, 7: fork to join)."""
    import torch

    ms, stage = [], []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        if stage_times is not None:
            t = stage_times()
            if len(t) > stage_index:
                stage.append(t[stage_index])
    return ms, stage


def overlap(f, x, y, g, u, v, flush, stream, nrep: int = 20, ms_full=None, timing=False) -> dict:
    """The paper's overlap claim (Fig. 1: the near field hides the sweep), measured on one handle in graph replays
    (the handle's launch configuration), medians of nrep steps with L2 flushed before each:
      sweep alone  = the sweep stream's fork-to-join span inside far-only replays (the handle's stage events are
                     event nodes of the graph; stages 4-7, and L2P where it runs on that stream);
      exposed      = T(full evaluation) - T(near-field-only evaluation);
      hidden       = 1 - exposed / sweep alone.
    The full and near-only series run with the same stage events (`timing`, the mode ms_full was taken in), since
    every event node costs the graph a few microseconds. A warm-up call precedes each series, so graph captures
    stay outside the timed steps."""
    f.set_timing(timing)
    full = ms_full
    if not full or len(full) < nrep:
        f.velocity(x, y, g, u, v)
        full = timed_steps(lambda: f.velocity(x, y, g, u, v), nrep, flush, stream)[0]
    f.velocity_near(x, y, g, u, v)
    near = timed_steps(lambda: f.velocity_near(x, y, g, u, v), nrep, flush, stream)[0]
    f.set_timing(True)
    f.velocity_far(x, y, g, u, v)
    far, fork_join = timed_steps(lambda: f.velocity_far(x, y, g, u, v), nrep, flush, stream, f.stage_times, 7)
    f.set_timing(timing)
    f.velocity(x, y, g, u, v)  # leave the full evaluation's graph in place
    t_full, t_near, t_far = (statistics.median(a) for a in (full, near, far))
    sweep = statistics.median(fork_join) if fork_join else None
    exposed = max(t_full - t_near, 0.0)
    return {"exposed_sweep_ms": exposed, "sweep_alone_ms": sweep,
            "hidden_fraction": (max(0.0, 1.0 - exposed / sweep) if sweep else None),
            "full_ms": t_full, "near_only_ms": t_near, "far_only_ms": t_far, "replays": nrep,
            "timing": "graph replays, medians, L2 flushed; sweep alone = fork-to-join in far-only replays"}


def arm_config(args, desc: str, world: int) -> dict:
    """The workload both arms report (the reference arm times the oracle on the same workload and metric)."""
    return {"workload": f"{args.workload}: {desc}", "precision": args.precision,
            "l2": "flushed before every timed step (256 MiB write, outside the timed events)",
            "graph": True, "parallelism": f"{world} independent replicas" if world > 1 else "1 GPU"}


def run_ours(args, rank: int, world: int, local_rank: int) -> dict | None:
    import numpy as np
    import torch

    from paper_1008_2410_gb300 import api

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist_

        dist = dist_
    w, desc = workload(args.workload)
    n = w.n
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    x, y, g = dev(w.x), dev(w.y), dev(w.gamma)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    f = api.FMM(w.depth, w.p, w.sigma, precision=args.precision, domain=w.domain, graph=True)
    # the autotuner picks the near-field tile shape and the M2L engine for this workload (depth stays the
    # workload's); --tile pins them instead (for profiling one configuration)
    if args.tile:
        th, kt = (int(t) for t in args.tile.split(","))
        f.set_p2p_tile(th, kt)
        if args.m2l_engine:
            f.set_m2l_engine(args.m2l_engine)
        tuned = f.params()
    else:
        tuned = f.autotune(x, y, g, w.depth, w.depth)
    f.set_timing("near")  # the near field's two events (the roofline's kernel time) and no other event node
    u = torch.empty_like(x)
    v = torch.empty_like(x)
    step = lambda: f.velocity(x, y, g, u, v)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    launches0 = f.kernel_launches()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms, p2p_ms = timed_steps(step, args.steps, flush, stream, f.stage_times)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = f.kernel_launches() - launches0
    clk = clocks.stop()
    ms_per_step, value = whole_job(sum(ms), args.steps, n, world, dist, device="cuda")

    out = {"metric": METRIC, "value": value, "unit": "Mparticles/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64 (precision form)" if args.precision == "mixed" else "f64",
           "data": "synthetic (seeded; the paper uses no dataset)",
           "config": arm_config(args, desc, world),
           "gpu_launches": int(launches), "clocks": clk,
           "p2p_tile": [tuned["p2p_threads"], tuned["p2p_targets_per_thread"]], "m2l_engine": tuned["m2l_engine"]}
    if rank != 0 and world > 1:
        return None
    if args.quick:
        return out

    # exposed sweep: full evaluation minus the near-field-only evaluation; the sweep alone from its fork-to-join
    # span in far-only replays (same handle, same graph launch configuration)
    ov = overlap(f, x, y, g, u, v, flush, stream, max(20, args.steps), ms_full=ms, timing="near")
    f.set_graph(False)
    f.velocity(x, y, g, u, v)
    st = f.stage_times()  # [bin, near, up, m2l, l2l, combine, total, overlapped]
    f.set_graph(True)
    out["exposed_sweep_ms"] = ov["exposed_sweep_ms"]
    ov["stage_ms_eager"] = dict(zip(["binning", "near", "up", "m2l", "l2l", "l2p_sum", "total", "fork_to_join"], st))
    out["sweep"] = ov

    if args.precision == "mixed":
        out["m2l"] = m2l_leg(api, w, x, y, g, args.steps, flush, stream)
    out["advect"] = advect_leg(api, w, x, y, g, tuned, args.precision, flush, stream)
    out["batched"] = batched_leg(api, args.precision, flush, stream)
    out["adjoint"], adj_check = adjoint_leg(api, w, x, y, g, flush, stream)
    if args.workload == "patches_16m" or args.adaptive:
        f.velocity(x, y, g, u, v)
        out["adaptive"] = adaptive_leg(api, w, x, y, g, u, v, args.precision, flush, stream,
                                       leaf_capacity=args.adaptive or 48, max_depth=args.max_depth)
    elif args.workload == "uniform_1m" and not args.no_clustered:
        out["clustered_patches_16m"] = clustered_leg(api, args.precision, flush, stream, args.max_depth)

    # roofline of the dominant kernel: near-field P2P, 22 flops per ordered pair (§3)
    f.set_count_pairs(True)
    f.velocity(x, y, g, u, v)
    pairs = f.pair_count()
    f.set_count_pairs(False)
    p2p_avg = statistics.mean(p2p_ms) if p2p_ms else None
    achieved = P2P_FLOPS_PER_PAIR * pairs / (p2p_avg / 1e3) / 1e12 if p2p_avg else None
    traffic = None
    kname = "k_p2p32s" if tuned["p2p_threads"] == 128 else "k_p2p32"
    tr_path = os.path.join(ROOT, "profiles", f"{kname}_{args.workload}.txt")
    if args.precision == "mixed" and os.path.exists(tr_path):
        try:
            import hashlib

            rec = dict(line.split(": ", 1) for line in open(tr_path).read().splitlines() if ": " in line)
            src = open(os.path.join(ROOT, "paper_1008_2410_gb300", "csrc", "p2p.cu"), "rb").read()
            if rec.get("p2p_cu_sha1", "").strip() == hashlib.sha1(src).hexdigest():
                # per-tile capture if the summary has one for the tile the autotuner picked
                tile_key = f"dram_bytes_per_launch_{tuned['p2p_threads']}x{tuned['p2p_targets_per_thread']}"
                traffic = float(rec.get(tile_key, rec["dram_bytes_per_launch"]))
        except Exception:
            traffic = None
    out["roofline"] = {"bound": "alu", "kernel": (f"{kname} (near field, stage 9, tile {tuned['p2p_threads']}x"
                                                   f"{tuned['p2p_targets_per_thread']})") if args.precision == "mixed"
                       else "k_p2p64 (near field, stage 9)",
                       "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                       "frac": achieved / FP32_PEAK_TFLOPS if achieved else None, "traffic": traffic,
                       "pairs_per_launch": pairs, "avg_launch_ms": p2p_avg,
                       "peak_note": "FP32 FMA peak derived: 152 SMs x 128 lanes x 2 flop x 2.07 GHz"}

    # accuracy of the precision form against the plain FP64 form (same tree, same p) and FP64 throughput
    if args.precision == "mixed":
        f64 = api.FMM(w.depth, w.p, w.sigma, precision="fp64", domain=w.domain, graph=True)
        u64, v64 = f64.velocity(x, y, g)
        f64.velocity(x, y, g, u64, v64)
        ms64, _ = timed_steps(lambda: f64.velocity(x, y, g, u64, v64), max(2, min(5, args.steps)), flush, stream)
        f.velocity(x, y, g, u, v)
        torch.cuda.synchronize()
        num = torch.sqrt(((u - u64) ** 2).sum() + ((v - v64) ** 2).sum())
        den = torch.sqrt((u64**2).sum() + (v64**2).sum())
        out["rel_err_vs_fp64_form"] = float(num / den)
        fc = api.FMM(w.depth, w.p, w.sigma, precision="mixed", domain=w.domain, coarse_level=4)
        uc, vc = fc.velocity(x, y, g)
        torch.cuda.synchronize()
        numc = torch.sqrt(((uc - u64) ** 2).sum() + ((vc - v64) ** 2).sum())
        out["rel_err_vs_fp64_form_fp64_coarse_levels"] = float(numc / den)
        fc.close()
        out["fp64_form"] = {"value": n / (statistics.median(ms64) / 1e3) / 1e6, "unit": "Mparticles/s",
                            "ms_per_step": statistics.median(ms64)}
        f64.close()

    # end to end through the host-buffer entry point: H2D of x, y, gamma and D2H of u, v inside the timed region
    xh, yh, gh = (torch.from_numpy(a).pin_memory() for a in (w.x, w.y, w.gamma))
    uh = torch.empty(n, dtype=torch.float64).pin_memory()
    vh = torch.empty(n, dtype=torch.float64).pin_memory()
    f.velocity_host(xh, yh, gh, uh, vh)
    ke = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    each = []
    for _ in range(ke):
        t1 = time.perf_counter()
        f.velocity_host(xh, yh, gh, uh, vh)  # synchronous: returns once u, v are in host memory
        each.append(time.perf_counter() - t1)
    te = (time.perf_counter() - t0) / ke
    out["e2e"] = {"value": n / te / 1e6, "unit": "Mparticles/s", "h2d_bytes_per_step": 3 * 8 * n,
                  "d2h_bytes_per_step": 2 * 8 * n, "ms_per_step": te * 1e3, "calls": ke,
                  "ms_min_median_max": [1e3 * min(each), 1e3 * statistics.median(each), 1e3 * max(each)]}

    # the paper's overlap bound (§4) with P = resident warps of this GPU
    from paper_1008_2410_gb300 import model

    P = SMS * 64
    out["model"] = {"B_actual": n / 4**w.depth, "B_min_for_overlap": model.min_leaf_occupancy_for_overlap(w.p, n, P),
                    "P_warps": P, "B_opt": model.b_opt(w.p)}

    try:
        from paper_1008_2410_gb300 import _lib as L

        out["probed_peaks"] = L.probe_peaks()
        out["roofline"]["frac_of_probed_fp32"] = (achieved / out["probed_peaks"]["fp32_tflops"]
                                                  if achieved else None)
    except Exception as exc:  # the probe is a report, not part of the metric
        out["probed_peaks"] = {"error": str(exc)}

    # the smallest p that keeps the precision form within 1e-6 of the FP64 form at p = 32 (fmm_autotune_p)
    if args.precision == "mixed":
        fp = api.FMM(w.depth, w.p, w.sigma, precision="mixed", domain=w.domain, graph=True)
        fp.set_p2p_tile(tuned["p2p_threads"], tuned["p2p_targets_per_thread"])
        pt, est = fp.autotune_p(x, y, g, 1e-6, 4, 24)
        up, vp = torch.empty_like(x), torch.empty_like(x)
        for _ in range(3):
            fp.velocity(x, y, g, up, vp)
        msp, _ = timed_steps(lambda: fp.velocity(x, y, g, up, vp), 10, flush, stream)
        fp.close()
        out["tuned_p"] = {"target_rel_err": 1e-6, "p": pt, "estimated_rel_err": est,
                          "value": n / (statistics.median(msp) / 1e3) / 1e6, "unit": "Mparticles/s",
                          "note": "fmm_autotune_p against the FP64 form at p = 32; the headline keeps the workload's p"}

    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, u.cpu().numpy(), v.cpu().numpy(), adj_check)
    f.close()
    return out


def m2l_translations(w) -> int:
    """M2L translations over non-empty boxes (target and source both non-empty), levels 2..L (§3 stage 6)."""
    import numpy as np

    L = w.depth
    if L < 2:
        return 0
    x0, y0, side = w.domain
    ns = 1 << L
    ix = np.clip(np.floor((w.x - x0) * (ns / side)).astype(np.int64), 0, ns - 1)
    iy = np.clip(np.floor((w.y - y0) * (ns / side)).astype(np.int64), 0, ns - 1)
    occ = np.zeros((ns, ns), dtype=bool)
    occ[iy, ix] = True
    total = 0
    for l in range(L, 1, -1):
        n = 1 << l
        pad = np.pad(occ, 3)
        for cy in (0, 1):
            for cx in (0, 1):
                tgt = occ[cy::2, cx::2]
                for dy in range(-2 - cy, 4 - cy):
                    for dx in range(-2 - cx, 4 - cx):
                        if -1 <= dx <= 1 and -1 <= dy <= 1:
                            continue
                        src = pad[3 + cy + dy:3 + cy + dy + n:2, 3 + cx + dx:3 + cx + dx + n:2]
                        total += int((tgt & src).sum())
        occ = occ.reshape(n // 2, 2, n // 2, 2).any(axis=(1, 3))
    return total


def tf32_peak_tflops() -> tuple[float, str]:
    """Dense TF32 tensor peak: the measured bf16 burst figure x the nominal TF32 / bf16 ratio (1.1 / 2.25)."""
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(peaks["bf16_tflops"]) * 1.1 / 2.25, "of measured (bf16 burst x 1.1/2.25)"
    except Exception:
        return 1900.0 * 1.1 / 2.25, "of fallback (1.9 PFLOP/s bf16 x 1.1/2.25)"


def m2l_leg(api, w, x, y, g, steps, flush, stream) -> dict:
    """M2L (stage 6) timed alone inside far-field-only evaluations, on the tensor cores and on the CUDA cores.

    Algorithmic work: 8 p^2 real flops per translation (p^2 complex multiply-adds), over non-empty boxes. The
    tensor-core path (levels <= 7) runs a layout pass and k_m2l_tc; the latter executes, per tile of 256 target
    positions of one class, 27 offsets x KP / 8 K steps x 2 (window hi, lo) MMAs of 2 x 128 x 256 x 8 flops
    (KP = 2p rounded up to 8 within p's bucket 8, 12, 16, 20)."""
    import statistics as st_

    import torch

    res = {}
    for engine in ("tensor", "cuda_cores"):
        fe = api.FMM(w.depth, w.p, w.sigma, precision="mixed", domain=w.domain, m2l_engine=engine)
        fe.set_timing(True)
        u = torch.empty_like(x)
        v = torch.empty_like(x)
        fe.velocity_far(x, y, g, u, v)
        ts = []
        for _ in range(max(5, min(steps, 20))):
            flush.zero_()
            fe.velocity_far(x, y, g, u, v)
            ts.append(fe.stage_times()[3])
        res[engine] = st_.median(ts)
        fe.close()
    T = m2l_translations(w)
    p = w.p
    pb = 8 if p <= 8 else 12 if p <= 12 else 16 if p <= 16 else 20
    KP = (2 * pb + 7) // 8 * 8
    tiles = sum(4 * ((2 ** (l - 1) * (2 ** (l - 1) + 2) + 255) // 256) for l in range(2, min(w.depth, 7) + 1))
    tc_flops = tiles * 27 * (KP // 8) * 2 * (2 * 128 * 256 * 8)
    peak, peak_note = tf32_peak_tflops()
    t = res["tensor"] / 1e3
    return {"kernel": "k_m2l_tc_layout + k_m2l_tc (tcgen05.mma kind::tf32, TF32 hi + lo on both operands, N = 256)",
            "ms": res["tensor"],
            "cuda_cores_ms": res["cuda_cores"], "translations": T, "flops_per_translation": 8 * p * p,
            "paper_flops_per_translation": 2 + 17 * p * p,
            "achieved_algorithmic_tflops": 8 * p * p * T / t / 1e12,
            "cuda_cores_achieved_algorithmic_tflops": 8 * p * p * T / (res["cuda_cores"] / 1e3) / 1e12,
            "cuda_cores_frac_of_fp32_peak": 8 * p * p * T / (res["cuda_cores"] / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
            "tensor_flops_executed": tc_flops, "achieved_tensor_tflops": tc_flops / t / 1e12,
            "peak_tf32_tflops": peak, "frac_tensor": tc_flops / t / 1e12 / peak, "peak_note": peak_note,
            "timing": "stage events around the M2L launch in far-field-only evaluations, L2 flushed"}


def advect_leg(api, w, x, y, g, tuned, precision, flush, stream) -> dict:
    """Eq. 3 time stepping through fmm_advect: RK2 (midpoint) steps of the whole workload, two evaluations per
    step, graph replay, bounding-box root square (particles may leave the unit square); dt moves the fastest
    particle by 0.05 sigma per step."""
    import statistics as st_

    import torch

    fa = api.FMM(w.depth, w.p, w.sigma, precision=precision, graph=True)
    fa.set_p2p_tile(tuned["p2p_threads"], tuned["p2p_targets_per_thread"])
    if precision == "mixed":
        fa.set_m2l_engine(tuned["m2l_engine"])
    u, v = fa.velocity(x, y, g)
    dt = 0.05 * w.sigma / float(torch.sqrt(u * u + v * v).max())
    xs, ys = x.clone(), y.clone()
    fa.advect(xs, ys, g, dt, 2, 2)  # warm-up (captures the graph)
    steps, ts = 3, []
    for _ in range(5):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fa.advect(xs, ys, g, dt, steps, 2)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) / steps)
    fa.sync()
    fa.close()
    ms = st_.median(ts)
    return {"scheme": "RK2 midpoint (2 evaluations per step)", "ms_per_step": ms,
            "value": w.n / (ms / 1e3) / 1e6, "unit": "Mparticle-steps/s", "dt": dt}


def batched_leg(api, precision, flush, stream) -> dict:
    """64 independent uniform systems of uneven size (4096 .. 262144 particles, depth round(log4(N/64)), p = 14)
    in one evaluation (one launch per stage, graph replay): total particles per second."""
    import statistics as st_

    import numpy as np
    import torch

    import fmm_inputs as fi

    bt = fi.batched()
    xs = np.concatenate([s.x for s in bt.systems])
    ys = np.concatenate([s.y for s in bt.systems])
    gs = np.concatenate([s.gamma for s in bt.systems])
    off = np.concatenate([[0], np.cumsum([s.n for s in bt.systems])])
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    x, y, g = dev(xs), dev(ys), dev(gs)
    f = api.FMM(bt.systems[0].depth, bt.p, bt.systems[0].sigma, precision=precision, graph=True)
    kw = dict(depths=[s.depth for s in bt.systems], sigmas=[s.sigma for s in bt.systems],
              domains=[list(s.domain) for s in bt.systems])
    u, v = f.velocity_batched(off, x, y, g, **kw)
    ms, _ = timed_steps(lambda: f.velocity_batched(off, x, y, g, u=u, v=v, **kw), 10, flush, stream)
    # the batched autotuner: leaf occupancy (per-system depths) and near-field tile
    tuned = f.autotune_batched(off, x, y, g, sigmas=kw["sigmas"], domains=kw["domains"])
    kwt = dict(kw, depths=tuned["depths"])
    f.velocity_batched(off, x, y, g, u=u, v=v, **kwt)
    mst, _ = timed_steps(lambda: f.velocity_batched(off, x, y, g, u=u, v=v, **kwt), 10, flush, stream)
    f.close()
    t, tt = st_.median(ms), st_.median(mst)
    occ = [float(s.n) / 4 ** d for s, d in zip(bt.systems, tuned["depths"])]
    return {"systems": len(bt.systems), "particles": int(off[-1]), "ms_per_step": t,
            "value": int(off[-1]) / (t / 1e3) / 1e6, "unit": "Mparticles/s",
            "config": "depth_k = round(log4(N_k / 64)), default tile",
            "autotuned": {"ms_per_step": tt, "value": int(off[-1]) / (tt / 1e3) / 1e6,
                          "p2p_tile": [tuned["p2p_threads"], tuned["p2p_targets_per_thread"]],
                          "depths": tuned["depths"], "mean_leaf_occupancy": sum(occ) / len(occ)}}


def adjoint_leg(api, w, x, y, g, flush, stream) -> dict:
    """Exact adjoint (dL/dgamma, dL/dx, dL/dy) for the loss L = 1/2 |u - u*|^2, u* the FMM velocity of the perturbed
    circulations gamma* = gamma + 0.01 N(0, 1)/N (the adjoint workload), FP64 form, on the same particles. Returns
    the timing and, for the CPU leg's accuracy check, the seeds and the GPU gradients."""
    import statistics as st_

    import numpy as np
    import torch

    import fmm_inputs as fi

    f = api.FMM(w.depth, w.p, w.sigma, precision="fp64", domain=w.domain)
    gs = torch.from_numpy(fi.adjoint_target_gamma(w)).cuda()
    us, vs = f.velocity(x, y, gs)
    u, v = f.velocity(x, y, g)
    gu, gv = u - us, v - vs
    f.adjoint(x, y, g, gu, gv)
    ms, _ = timed_steps(lambda: f.adjoint(x, y, g, gu, gv), 3, flush, stream)
    dg, dx, dy = f.adjoint(x, y, g, gu, gv)
    # the near-field part in FP32 (fmm_set_adjoint_precision): time and distance from the FP64 adjoint
    f.set_adjoint_precision("mixed")
    f.adjoint(x, y, g, gu, gv)
    ms32, _ = timed_steps(lambda: f.adjoint(x, y, g, gu, gv), 5, flush, stream)
    dg32, dx32, dy32 = f.adjoint(x, y, g, gu, gv)
    f.sync()
    f.close()
    t = st_.median(ms)
    t32 = st_.median(ms32)
    rel = lambda a, b: float(torch.sqrt(sum(((p - q) ** 2).sum() for p, q in zip(a, b)) / sum((q**2).sum() for q in b)))
    loss = float(0.5 * (gu * gu + gv * gv).sum())
    out = {"form": "fp64", "loss": "1/2 |u - u*|^2, u* from gamma + 0.01 N(0,1)/N", "loss_value": loss,
           "ms_per_step": t, "value": w.n / (t / 1e3) / 1e6, "unit": "Mparticles/s",
           "fp32_near_field": {"ms_per_step": t32, "value": w.n / (t32 / 1e3) / 1e6, "unit": "Mparticles/s",
                               "rel_diff_dgamma_vs_fp64": rel((dg32,), (dg,)),
                               "rel_diff_dxdy_vs_fp64": rel((dx32, dy32), (dx, dy))}}
    # the same loss on a 2^16-particle case of the recipe (depth 5): the oracle's adjoint of all particles takes
    # about 40 s at 2^20 (that size is checked by the GPU tests), a few seconds here
    ws = fi.uniform(1 << 16, seed_index=1, depth=5, p=w.p)  # sigma = 0.5 / sqrt(N), as the recipe
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    xs, ys, gs_ = dev(ws.x), dev(ws.y), dev(ws.gamma)
    f = api.FMM(ws.depth, ws.p, ws.sigma, precision="fp64", domain=ws.domain)
    us, vs = f.velocity(xs, ys, dev(fi.adjoint_target_gamma(ws)))
    u, v = f.velocity(xs, ys, gs_)
    gu, gv = u - us, v - vs
    dg, dx, dy = f.adjoint(xs, ys, gs_, gu, gv)
    f.sync()
    f.close()
    check = {"workload": ws, **{k: a.cpu().numpy() for k, a in (("gu", gu), ("gv", gv), ("dg", dg), ("dx", dx),
                                                                 ("dy", dy))}}
    return out, check


FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 rate (no measured FP64 peak on this machine)


def adaptive_leg(api, w, x, y, g, u_uni, v_uni, precision, flush, stream, leaf_capacity: int = 48,
                 max_depth: int = 11) -> dict:
    """The adaptive quadtree (U, V, W, X lists) on this workload in the run's precision: graph-replay
    throughput (median of 20), its near-field kernel against the FP32 (or FP64) rate, near pairs, the
    difference from the uniform-tree result of the main run and, for the precision form, from the FP64 form
    of the adaptive tree."""
    import torch

    f = api.FMM(max_depth, w.p, w.sigma, precision=precision, domain=w.domain, graph=True,
                leaf_capacity=leaf_capacity)
    u, v = torch.empty_like(x), torch.empty_like(x)
    for _ in range(3):
        f.velocity(x, y, g, u, v)
    ms, _ = timed_steps(lambda: f.velocity(x, y, g, u, v), 20, flush, stream)
    u_s, v_s = torch.empty_like(x), torch.empty_like(x)
    ov = overlap(f, x, y, g, u_s, v_s, flush, stream, 20, ms_full=ms)
    f.set_graph(False)
    f.set_timing(True)
    f.set_count_pairs(True)
    f.velocity(x, y, g, u, v)
    st = f.stage_times()  # [binning, near, -, -, -, final, total, fork_to_join]
    pairs = f.pair_count()
    f.set_count_pairs(False)
    # the near-field kernel alone (no sweep beside it): median of 5 near-only evaluations
    near_alone = []
    u2, v2 = torch.empty_like(x), torch.empty_like(x)
    for _ in range(5):
        flush.zero_()
        f.velocity_near(x, y, g, u2, v2)
        sa = f.stage_times()
        if sa:
            near_alone.append(sa[1])
    f.close()
    t = statistics.median(ms)
    near_ms = statistics.median(near_alone) if near_alone else None
    achieved = P2P_FLOPS_PER_PAIR * pairs / (near_ms / 1e3) / 1e12 if near_ms else None
    peak = FP32_PEAK_TFLOPS if precision == "mixed" else FP64_PEAK_TFLOPS
    out = {"leaf_capacity": leaf_capacity, "max_depth": max_depth, "precision": precision,
           "value": w.n / (t / 1e3) / 1e6, "unit": "Mparticles/s", "ms_per_step": t, "near_pairs": pairs,
           "sweep": ov, "exposed_sweep_ms": ov["exposed_sweep_ms"], "hidden_fraction": ov["hidden_fraction"],
           "stage_ms_eager": dict(zip(["binning", "near", "up_lists_p2l_p2m_m2m", "down_l2l_m2l", "w_list_l2p",
                                       "final", "total", "fork_to_join"], st)),
           "roofline_near": {"bound": "alu", "kernel": "k_ad_near32" if precision == "mixed" else "k_ad_near",
                             "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak if achieved else None,
                             "avg_launch_ms": near_ms,
                             "note": ("near stage (split + near kernel) timed alone in near-only evaluations; "
                                      "22 flops per ordered pair; peak " +
                                      ("FP32 FMA derived" if precision == "mixed" else "nominal FP64"))}}
    torch.cuda.synchronize()
    den = torch.sqrt((u_uni**2).sum() + (v_uni**2).sum())
    out["rel_diff_vs_uniform_tree"] = float(torch.sqrt(((u - u_uni) ** 2).sum() + ((v - v_uni) ** 2).sum()) / den)
    if precision == "mixed":
        f64 = api.FMM(max_depth, w.p, w.sigma, precision="fp64", domain=w.domain, leaf_capacity=leaf_capacity)
        u64, v64 = f64.velocity(x, y, g)
        torch.cuda.synchronize()
        d64 = torch.sqrt((u64**2).sum() + (v64**2).sum())
        out["rel_err_vs_fp64_form"] = float(torch.sqrt(((u - u64) ** 2).sum() + ((v - v64) ** 2).sum()) / d64)
        f64.close()
    return out


def clustered_leg(api, precision, flush, stream, max_depth: int = 11, leaf_capacity: int = 48) -> dict:
    """The clustered workload (patches_16m, 2^24 particles from 8 Gaussian patches) on both trees in the run's
    precision: the uniform depth-9 tree (autotuned near-field tile and M2L engine) and the adaptive tree
    (leaf capacity 48, maximum depth 11), graph replays, medians of 10; their relative difference; the adaptive
    tree end to end from pinned host buffers."""
    import numpy as np
    import torch

    w, _ = workload("patches_16m")
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    x, y, g = dev(w.x), dev(w.y), dev(w.gamma)
    fu = api.FMM(w.depth, w.p, w.sigma, precision=precision, domain=w.domain, graph=True)
    tuned = fu.autotune(x, y, g, w.depth, w.depth)
    uu, vu = torch.empty_like(x), torch.empty_like(x)
    for _ in range(3):
        fu.velocity(x, y, g, uu, vu)
    msu, _ = timed_steps(lambda: fu.velocity(x, y, g, uu, vu), 10, flush, stream)
    u_s, v_s = torch.empty_like(x), torch.empty_like(x)
    ov_u = overlap(fu, x, y, g, u_s, v_s, flush, stream, 20)
    fu.close()
    fa = api.FMM(max_depth, w.p, w.sigma, precision=precision, domain=w.domain, graph=True,
                 leaf_capacity=leaf_capacity)
    ua, va = torch.empty_like(x), torch.empty_like(x)
    for _ in range(3):
        fa.velocity(x, y, g, ua, va)
    msa, _ = timed_steps(lambda: fa.velocity(x, y, g, ua, va), 10, flush, stream)
    ov_a = overlap(fa, x, y, g, u_s, v_s, flush, stream, 20)
    fa.set_timing(False)
    # the autotuner's leaf capacity (maximum depth 11 kept) on a second handle
    ft = api.FMM(max_depth, w.p, w.sigma, precision=precision, domain=w.domain, graph=True, leaf_capacity=leaf_capacity)
    tuned_a = ft.autotune(x, y, g, max_depth, max_depth)
    ut, vt = torch.empty_like(x), torch.empty_like(x)
    for _ in range(3):
        ft.velocity(x, y, g, ut, vt)
    mst, _ = timed_steps(lambda: ft.velocity(x, y, g, ut, vt), 10, flush, stream)
    ft.close()
    # end to end through the host-buffer entry point (pinned inputs copied in, velocities copied out)
    xh, yh, gh = (torch.from_numpy(a).pin_memory() for a in (w.x, w.y, w.gamma))
    uh, vh = torch.empty(w.n, dtype=torch.float64).pin_memory(), torch.empty(w.n, dtype=torch.float64).pin_memory()
    fa.velocity_host(xh, yh, gh, uh, vh)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    each = []
    for _ in range(3):
        t1 = time.perf_counter()
        fa.velocity_host(xh, yh, gh, uh, vh)
        each.append(time.perf_counter() - t1)
    te = (time.perf_counter() - t0) / 3
    fa.close()
    torch.cuda.synchronize()
    den = torch.sqrt((uu**2).sum() + (vu**2).sum())
    tu, ta = statistics.median(msu), statistics.median(msa)
    return {"n": w.n, "p": w.p, "precision": precision,
            "uniform_tree": {"depth": w.depth, "value": w.n / (tu / 1e3) / 1e6, "unit": "Mparticles/s",
                             "ms_per_step": tu, "p2p_tile": [tuned["p2p_threads"], tuned["p2p_targets_per_thread"]],
                             "m2l_engine": tuned["m2l_engine"], "sweep": ov_u,
                             "exposed_sweep_ms": ov_u["exposed_sweep_ms"],
                             "hidden_fraction": ov_u["hidden_fraction"]},
            "adaptive_tree": {"max_depth": max_depth, "leaf_capacity": leaf_capacity,
                              "value": w.n / (ta / 1e3) / 1e6, "unit": "Mparticles/s", "ms_per_step": ta,
                              "sweep": ov_a, "exposed_sweep_ms": ov_a["exposed_sweep_ms"],
                              "hidden_fraction": ov_a["hidden_fraction"],
                              "e2e": {"value": w.n / te / 1e6, "unit": "Mparticles/s", "ms_per_step": te * 1e3,
                                      "h2d_bytes_per_step": 3 * 8 * w.n, "d2h_bytes_per_step": 2 * 8 * w.n,
                                      "ms_min_median_max": [1e3 * min(each), 1e3 * statistics.median(each),
                                                            1e3 * max(each)]},
                              "autotuned": {"leaf_capacity": tuned_a["leaf_capacity"],
                                            "value": w.n / (statistics.median(mst) / 1e3) / 1e6,
                                            "ms_per_step": statistics.median(mst)}},
            "rel_diff_adaptive_vs_uniform": float(torch.sqrt(((ua - uu) ** 2).sum() + ((va - vu) ** 2).sum()) / den)}


def cpu_baseline(w, u_gpu, v_gpu, adj=None) -> dict:
    """The FP64 oracle as it stands, on all host cores: one full FMM evaluation of the same workload (or, above
    2^21 particles, its far field plus near field at 4096 sampled targets), plus accuracy figures of the GPU
    result against it and against the direct sum at 256 sampled targets, and (adj) of the GPU adjoint against the
    oracle's transposed stages for the same seeds."""
    import numpy as np

    import fmm_inputs as fi
    import oracle

    oracle.build()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    full = w.n <= (1 << 21)
    t = None if full else fi.sample_targets(w.n, 4096)
    t0 = time.perf_counter()
    uo, vo, _ = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, domain=w.domain, targets=t)
    dt = time.perf_counter() - t0
    count = w.n if full else 4096
    ug, vg = (u_gpu, v_gpu) if full else (u_gpu[t], v_gpu[t])
    err_fmm = float(np.sqrt(np.sum((ug - uo) ** 2 + (vg - vo) ** 2) / np.sum(uo**2 + vo**2)))
    ts = fi.sample_targets(w.n, 256, seed_index=8)
    ud, vd = oracle.direct(w.x, w.y, w.gamma, w.sigma, targets=ts)
    err_dir = float(np.sqrt(np.sum((u_gpu[ts] - ud) ** 2 + (v_gpu[ts] - vd) ** 2) / np.sum(ud**2 + vd**2)))
    res = {"value": count / dt / 1e6, "unit": "Mparticles/s", "cores": cores, "kind": "oracle",
           "sample": ("full evaluation, all targets" if full else
                      "far field of all particles + near field at 4096 sampled targets; rate = targets/s"),
           "seconds": dt, "gpu_rel_err_vs_oracle_fmm": err_fmm, "gpu_rel_err_vs_direct_sum_256": err_dir}
    if adj is not None:
        rel = lambda a, b: float(np.linalg.norm(np.concatenate([np.ravel(t) for t in a]) -
                                                np.concatenate([np.ravel(t) for t in b])) /
                                 np.linalg.norm(np.concatenate([np.ravel(t) for t in b])))
        wa = adj["workload"]
        t0 = time.perf_counter()
        og, ox, oy = oracle.fmm_adjoint(wa.x, wa.y, wa.gamma, wa.sigma, wa.depth, wa.p, adj["gu"], adj["gv"],
                                        domain=wa.domain)
        res["adjoint_check"] = {"gpu_rel_err_dgamma_vs_oracle": rel((adj["dg"],), (og,)),
                                "gpu_rel_err_dxdy_vs_oracle": rel((adj["dx"], adj["dy"]), (ox, oy)),
                                "oracle_seconds": time.perf_counter() - t0,
                                "case": f"N = {wa.n} uniform, depth {wa.depth}, p {wa.p}, loss 1/2 |u - u*|^2, "
                                        "all particles"}
    return res


def run_reference(args, rank: int, world: int) -> dict | None:
    """The oracle timed on the host cores on this arm's workload and metric; each step is one full oracle FMM
    evaluation (above 2^21 particles: the far field plus the near field at 4096 sampled targets)."""
    if rank != 0:
        return None
    import fmm_inputs as fi
    import oracle

    oracle.build()
    w, desc = workload(args.workload)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    full = w.n <= (1 << 21)
    t = None if full else fi.sample_targets(w.n, 4096)
    count = w.n if full else 4096
    steps = max(1, args.steps)
    warm = max(0, args.warmup)
    for _ in range(warm):
        oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, domain=w.domain, targets=t)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.depth, w.p, domain=w.domain, targets=t)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / steps
    value = count / (ms / 1e3) / 1e6
    sample = "full evaluation, all targets" if full else "far field + near field at 4096 sampled targets"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mparticles/s", "n_gpus": world,
            "steps": steps, "warmup": warm, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded; the paper uses no dataset)",
            "config": arm_config(args, desc, world),
            "cpu_baseline": {"value": value, "unit": "Mparticles/s", "cores": cores, "kind": "oracle",
                             "sample": sample, "precision": "fp64 (the CPU oracle)"},
            "e2e": {"value": value, "unit": "Mparticles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_profile_once(args) -> dict:
    """One eager evaluation on the workload (the uniform tree, or the adaptive tree with --adaptive B and
    --max-depth), for kernel launch lists and counter captures; no timing."""
    import numpy as np
    import torch

    from paper_1008_2410_gb300 import api

    w, desc = workload(args.workload)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    x, y, g = dev(w.x), dev(w.y), dev(w.gamma)
    depth = args.max_depth if args.adaptive else w.depth
    f = api.FMM(depth, w.p, w.sigma, precision=args.precision, domain=w.domain, leaf_capacity=args.adaptive)
    if args.tile:
        f.set_p2p_tile(*(int(t) for t in args.tile.split(",")))
    u, v = f.velocity(x, y, g)
    f.sync()
    return {"profile_once": args.workload, "precision": args.precision, "depth": depth,
            "leaf_capacity": args.adaptive, "max_abs_u": float(u.abs().max())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="uniform_1m", choices=["uniform_1m", "patches_16m", "patches_4m"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clustered", action="store_true",
                    help="skip the clustered-workload leg (both trees on patches_16m) of the default run")
    ap.add_argument("--adaptive", type=int, default=0,
                    help="also time the adaptive tree with this leaf capacity (always on for patches_16m, capacity 48)")
    ap.add_argument("--quick", action="store_true", help="main timing only")
    ap.add_argument("--max-depth", type=int, default=11, help="maximum depth of the adaptive tree")
    ap.add_argument("--profile-once", action="store_true",
                    help="one eager evaluation, no timing (for ncu launch lists and captures)")
    ap.add_argument("--tile", default=None, help="near-field tile 'threads,targets' instead of the autotuner's")
    ap.add_argument("--m2l-engine", default=None, choices=["tensor", "cuda_cores"],
                    help="M2L engine instead of the autotuner's (with --tile)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.profile_once:
        out = run_profile_once(args)
    elif args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist

            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        out = run_ours(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
    if out is not None and rank == 0:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
