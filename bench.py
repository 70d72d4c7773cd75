#!/usr/bin/env python
"""Benchmark of the staggered even-odd CG on the paper's lattice size.

Workload: 28^3 x 96 lattice (the MILC fine lattice of Sec. 2), asqtad-form
operator (fat links 0.6 U_a + 0.4 U_b, Naik links -(1/24) U_c, three
independent synthetic SU(3) fields U = exp(0.3 i H)), m = 0.0062, Gaussian
even-site source, tol 1e-10 on the true residual |b - A x| / |b|.

One step = one pass of the whole path: stag_create_ex (eta folding and
layout packing of both link fields from device-resident inputs),
stag_cg_solve (Fig. 1 to the tolerance, true FP64 residual, restarts) and
stag_destroy.  The link fields (2 x 1.2 GB in, 4.9 GB packed) are far larger
than the 126 MB L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the host cores on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time to |r|/|b|≤1e-10 at 28³×96 vs FP64 plain CG; Dslash GB/s vs HBM peak"
UNIT = "s"
DIMS = (28, 28, 28, 96)
MASS = 0.0062
SECOND_MASS = 0.031  # the workload's second mass (forms only)
TOL = 1e-10
MAX_ITER = 40000  # far above the expected count; bounds a run that fails to converge
FORM_WARMUP_ITERS = 64  # the warm-up solve before each timed solve of the forms table
FALLBACK_HBM_GBS = 6800.0
# Fig. 1 iterations of this system (28^3 x 96 asqtad-form, m = 0.0062, source
# seed 0, tol 1e-10), used only to scale the oracle's per-A-application time
# to a whole solve in the reference leg, which cannot afford to run it.
REFERENCE_ITERS = 1454
PAPER_CONTEXT = "35 GFLOP/s FP64 CG on one GPU of a GTX 295 (Sec. 3.4, CUDA 2.3, cc 1.3)"


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["single", "batched", "learned", "decomposed"], default="single")
    p.add_argument("--pairs", type=int, default=2000)
    p.add_argument("--test-sources", type=int, default=64)
    p.add_argument("--epochs", type=int, default=4)
    p.add_argument("--stride", type=int, default=2)
    p.add_argument("--min-rel", type=float, default=0.05)
    p.add_argument("--lr", type=float, default=1e-3)
    p.add_argument("--arith", choices=["ff", "f64"], default="ff")
    p.add_argument("--long-recon", type=int, choices=[0, 12], default=0,
                   help="12: float-float kernels keep two rows of each Naik link (-U/24) and rebuild the third")
    p.add_argument("--mass", type=float, default=MASS)
    p.add_argument("--dims", type=int, nargs=4, default=list(DIMS))
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-sequential", action="store_true",
                   help="batched workload: skip the one-at-a-time comparison solves")
    p.add_argument("--main-only", action="store_true",
                   help="batched workload: only the 16 right-hand sides on the 32^3 x 64 field")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-forms", "--no-f64", dest="no_forms", action="store_true")
    return p.parse_args()


# ------------------------------------------------------------------ helpers
def workload_config(dims, mass, world):
    """The `config` object of the default workload, identical in both arms."""
    return {
        "workload": f"staggered even-odd CG, asqtad-form (fat 0.6U_a+0.4U_b, Naik -U_c/24), "
                    f"{'x'.join(map(str, dims))}, m={mass}, tol={TOL}",
        "lattice": list(dims),
        "mass": mass,
        "tol": TOL,
        "step": "stag_create_ex + stag_cg_solve + stag_destroy (device-resident inputs)",
        "l2": "inputs (2.4 GB AoS links, 4.9 GB packed) larger than L2; no flush",
        "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
    }


def host_cpu():
    """(CPU model, logical cores) of this host, from lscpu or /proc/cpuinfo."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu model")):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return model or "unknown", os.cpu_count() or 1


def dist_env():
    from paper_1010_4782_gb300.replicas import dist_env as _env

    return _env()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


DSLASH_SOURCES = ("dslash.cu", "ff.cuh", "stag_internal.cuh")
MULTI_SOURCES = ("multi.cu", "multi.cuh", "stag_internal.cuh")


def dslash_source_hash(files=DSLASH_SOURCES):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1010_4782_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_key, files=DSLASH_SOURCES):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[kernel_key]
        if e.get("source_hash") != dslash_source_hash(files):
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        mhz, max_mhz, reasons = [], None, set()
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                max_mhz = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(self.NAMES, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not mhz:
            return None
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": max_mhz,
                "reasons": sorted(reasons), "samples": len(mhz)}


# ----------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch

    from paper_1010_4782_gb300 import accounting, binding, build, inputs

    world, rank, local = dist_env()
    dims = tuple(args.dims)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    from paper_1010_4782_gb300.replicas import Replicas

    reps = Replicas(world, rank, dev)
    barrier, max_over_ranks, sum_over_ranks = reps.barrier, reps.max, reps.sum

    build.build()
    binding.load()
    fat, lng = inputs.asqtad_form_fields(dims)
    b = inputs.gaussian_even_source(dims, reps.source_seed())  # independent replica per rank
    fat_d = torch.from_numpy(fat).to(dev)
    lng_d = torch.from_numpy(lng).to(dev)
    b_d = torch.from_numpy(b).to(dev)
    x_d = torch.zeros_like(b_d)
    vh = accounting.half_sites(dims)
    arith = binding.STAG_ARITH_FF if args.arith == "ff" else binding.STAG_ARITH_F64
    stream = torch.cuda.current_stream(dev)

    def options(ar, timing):
        o = binding.stag_default_options()
        o.arith = ar
        o.timing = 1 if timing else 0
        if ar == binding.STAG_ARITH_FF and args.long_recon == 12:
            o.long_recon, o.long_scale = 12, inputs.NAIK_COEFF
        return o

    rec = {"launches": 0, "k_ms": [0.0] * 4, "k_n": [0] * 4, "infos": []}

    def step(fat_in, lng_in, b_in, x_in, ar=arith, timing=True, record=True):
        h = binding.stag_create_ex(fat_in, lng_in, dims, args.mass, options(ar, timing))
        try:
            binding.stag_set_stream(h, stream)
            if hasattr(x_in, "zero_"):
                x_in.zero_()
            else:
                x_in[...] = 0
            code, info = binding.stag_cg_solve(h, b_in, x_in, TOL, MAX_ITER)
            if code != binding.STAG_OK:
                raise RuntimeError(f"solve failed: status {code}: {binding.stag_last_error(h)}")
            if record:
                rec["launches"] += binding.stag_launch_count(h)
                for k in range(4):
                    ms, n = binding.stag_kernel_stats(h, k)
                    rec["k_ms"][k] += ms
                    rec["k_n"][k] += n
                rec["infos"].append(info)
        finally:
            binding.stag_destroy(h)
        return info

    # ---- warm-up, then K timed steps (device-resident inputs) with the library's
    # defaults (CUDA graphs of check_interval iterations, no per-kernel events)
    for _ in range(args.warmup):
        step(fat_d, lng_d, b_d, x_d, timing=False, record=False)
    torch.cuda.synchronize(dev)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(fat_d, lng_d, b_d, x_d, timing=False)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    host_s = time.perf_counter() - t0
    barrier()
    clock_info = clocks.stop()
    elapsed_s = max_over_ranks(ev0.elapsed_time(ev1) / 1e3)
    total_solves = args.steps * world
    value = reps.time_per_solve(elapsed_s, args.steps)
    infos = rec["infos"]
    iters = infos[-1]["iters"]
    gpu_launches = int(sum_over_ranks(rec["launches"]))

    # ---- one more, instrumented solve (CUDA events around every CG kernel, no graphs),
    # outside the timed region: per-kernel durations for the roofline and the shares
    rec["k_ms"], rec["k_n"] = [0.0] * 4, [0] * 4
    inst = step(fat_d, lng_d, b_d, x_d, timing=True)

    # ---- dominant kernel: the half-Dslash D_oe (Naik), CUDA events on the library's stream
    naik = True
    two_row = args.arith == "ff" and args.long_recon == 12
    bytes_per_launch = accounting.compulsory_bytes_per_site(naik, long_entries=6 if two_row else 9) * vh
    flops_per_launch = accounting.flops_per_site(naik) * vh
    oe_ms = rec["k_ms"][0] / max(1, rec["k_n"][0])
    eo_ms = rec["k_ms"][1] / max(1, rec["k_n"][1])
    achieved = bytes_per_launch / (oe_ms / 1e3) / 1e9
    peak, peak_src = measured_peaks()
    kernel_key = f"dslash_oe_{args.arith}_naik{'12' if two_row else ''}_{'x'.join(map(str, dims))}"
    roofline = {
        "bound": "hbm",
        "achieved": round(achieved, 1),
        "peak": peak,
        "unit": "GB/s",
        "frac": round(achieved / peak, 4),
        "traffic": recorded_traffic(kernel_key),
        "kernel": f"half-Dslash D_oe, Naik{' (two-row links)' if two_row else ''}, {args.arith.upper()} "
                  f"arithmetic ({kernel_key})",
        "algorithmic_bytes_per_launch": bytes_per_launch,
        "avg_launch_ms": round(oe_ms, 4),
        "launch_times_from": "CUDA events on the library's stream around every launch of one instrumented "
                             "solve after the timed steps",
        "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback",
    }
    k_total = sum(rec["k_ms"])
    kernel_shares = {binding.KERNEL_NAMES[k]: {"launches": rec["k_n"][k], "ms": round(rec["k_ms"][k], 2),
                                               "share_of_cg_kernels": round(rec["k_ms"][k] / k_total, 4)}
                     for k in range(4)}
    kernel_shares["instrumented_solve_ms"] = round(inst["time_ms"], 2)
    solve_ms = statistics.median(i["time_ms"] for i in infos[:args.steps])

    # ---- the native-FP64 half-Dslash D_oe (Naik) on its roofline: min(HBM, FP64 FMA).
    # Per-launch time from a short instrumented FP64 CG run (events around every launch);
    # the DFMA ceiling is measured by the library's FMA probe on this GPU.
    roof64 = None
    if not args.no_forms:
        o64 = options(binding.STAG_ARITH_F64, True)
        h64 = binding.stag_create_ex(fat_d, lng_d, dims, args.mass, o64)
        try:
            binding.stag_set_stream(h64, stream)
            x64i = torch.zeros_like(b_d)
            binding.stag_cg_solve(h64, b_d, x64i, TOL, 96)
            ms64, n64 = binding.stag_kernel_stats(h64, binding.STAG_KERNEL_DSLASH_OE)
        finally:
            binding.stag_destroy(h64)
        del x64i
        dfma_rate = binding.stag_measure_fma_rate(64)
        ffma_rate = binding.stag_measure_fma_rate(32)
        t64 = ms64 / max(1, n64) / 1e3
        bytes64 = accounting.compulsory_bytes_per_site(naik) * vh
        dfma64 = accounting.fma_per_site(naik) * vh
        t_hbm, t_alu = bytes64 / (peak * 1e9), dfma64 / dfma_rate
        roof64 = {
            "bound": "hbm" if t_hbm >= t_alu else "alu",
            "kernel": "half-Dslash D_oe, Naik, native FP64 (dslash_kernel<ArithF64>)",
            "avg_launch_ms": round(t64 * 1e3, 4),
            "launches_timed": n64,
            "algorithmic_bytes_per_launch": bytes64,
            "achieved_gbs": round(bytes64 / t64 / 1e9, 1),
            "hbm_peak_gbs": peak,
            "hbm_frac": round(bytes64 / t64 / 1e9 / peak, 4),
            "traffic": recorded_traffic(f"dslash_oe_f64_naik_{'x'.join(map(str, dims))}"),
            "dfma_per_launch": dfma64,
            "achieved_dfma_per_s": round(dfma64 / t64, 1),
            "dfma_peak_per_s": round(dfma_rate, 1),
            "dfma_frac": round(dfma64 / t64 / dfma_rate, 4),
            "ffma_peak_per_s": round(ffma_rate, 1),
            "frac_of_binding_bound": round(max(t_hbm, t_alu) / t64, 4),
            "peak_sources": "hbm: MEASURED_PEAKS.json hbm_gbs; dfma/ffma: measured now by stag_measure_fma_rate",
        }
    # paper's convention: Dslash flops only, two half-Dslash per CG iteration
    gflops = 2 * flops_per_launch * iters / (solve_ms / 1e3) / 1e9

    # ---- end to end: host (pinned) inputs, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        fat_h = torch.from_numpy(fat).pin_memory()
        lng_h = torch.from_numpy(lng).pin_memory()
        b_h = torch.from_numpy(b).pin_memory()
        x_h = torch.zeros_like(b_h).pin_memory()
        step(fat_h, lng_h, b_h, x_h, timing=False, record=False)
        torch.cuda.synchronize(dev)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step(fat_h, lng_h, b_h, x_h, timing=False, record=False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        e2e_s = max_over_ranks(e0.elapsed_time(e1) / 1e3)
        vec_bytes = b_h.numel() * 16
        e2e = {"value": round(e2e_s / total_solves, 4), "unit": UNIT,
               "h2d_bytes_per_step": int(fat_h.numel() * 16 + lng_h.numel() * 16 + 2 * vec_bytes),
               "d2h_bytes_per_step": int(vec_bytes)}
        del fat_h, lng_h

    # ---- every form at this accuracy, against plain FP64 GPU CG (native FP64 kernels):
    # asqtad-form operator (this workload) and the one-hop operator on the same lattice
    forms = None
    if not args.no_forms:
        def solve_once(fat_in, lng_in, b_in, ar, inner, recon=0, long_recon=0):
            o = binding.stag_default_options()
            o.arith = ar
            o.inner = inner
            o.link_recon = recon
            if long_recon:
                o.long_recon, o.long_scale = 12, inputs.NAIK_COEFF
            h = binding.stag_create_ex(fat_in, lng_in, dims, args.mass, o)
            try:
                binding.stag_set_stream(h, stream)
                # warm-up: a short solve on the same handle (kernels loaded, graphs instantiated)
                x = torch.zeros_like(b_in)
                binding.stag_cg_solve(h, b_in, x, TOL, FORM_WARMUP_ITERS)
                x.zero_()
                code, info = binding.stag_cg_solve(h, b_in, x, TOL, MAX_ITER)
            finally:
                binding.stag_destroy(h)
            return code, info, x

        variants = [("fp64_plain", binding.STAG_ARITH_F64, binding.STAG_INNER_NONE),
                    ("ff_plain", binding.STAG_ARITH_FF, binding.STAG_INNER_NONE),
                    ("mixed_fp32", binding.STAG_ARITH_FF, binding.STAG_INNER_F32),
                    ("mixed_fp16", binding.STAG_ARITH_FF, binding.STAG_INNER_F16),
                    ("mixed_bf16", binding.STAG_ARITH_FF, binding.STAG_INNER_BF16),
                    ("mixed_fp32_fp16links", binding.STAG_ARITH_FF, binding.STAG_INNER_F32_L16),
                    # 12-parameter SU(3) links (Sec. 3.3): unitary one-hop links only
                    ("mixed_fp32_recon12", binding.STAG_ARITH_FF, binding.STAG_INNER_F32),
                    # the same form for the Naik links (-U/24 = scale x SU(3)) of the asqtad operator
                    ("mixed_fp32_longrecon12", binding.STAG_ARITH_FF, binding.STAG_INNER_F32)]
        forms = {}
        one_hop = torch.from_numpy(inputs.gauge_field(dims, 1)).to(dev)
        for op_name, f_in, l_in in (("asqtad", fat_d, lng_d), ("one_hop", one_hop, None)):
            res, x64 = {}, None
            for name, ar, inner in variants:
                recon = 12 if name.endswith("_recon12") else 0
                long_recon = 12 if name.endswith("longrecon12") else 0
                if (recon and l_in is not None) or (long_recon and l_in is None):
                    continue
                code, info, x = solve_once(f_in, l_in, b_d, ar, inner, recon, long_recon)
                if x64 is None:
                    x64 = x
                rec = {"time_s": round(info["time_ms"] / 1e3, 4), "status": code, "iters": info["iters"],
                       "reliable_updates": info["reliable_updates"], "fallbacks": info["fallbacks"],
                       "true_rel_residual": info["true_rel_residual"],
                       "rel_diff_vs_fp64_plain": float(torch.linalg.vector_norm(x - x64) /
                                                       torch.linalg.vector_norm(x64))}
                res[name] = rec
            base = res["fp64_plain"]["time_s"]
            for rec in res.values():
                rec["speedup_vs_fp64_plain"] = round(base / rec["time_s"], 3)
            forms[op_name] = res
        del one_hop
        # the asqtad operator at the workload's second mass, where 16-bit storage converges
        if args.mass == MASS:
            saved = args.mass
            args.mass = SECOND_MASS
            res, x64 = {}, None
            for name, ar, inner in variants:
                if name.endswith("_recon12"):
                    continue
                long_recon = 12 if name.endswith("longrecon12") else 0
                code, info, x = solve_once(fat_d, lng_d, b_d, ar, inner, 0, long_recon)
                if x64 is None:
                    x64 = x
                res[name] = {"time_s": round(info["time_ms"] / 1e3, 4), "status": code, "iters": info["iters"],
                             "reliable_updates": info["reliable_updates"], "fallbacks": info["fallbacks"],
                             "true_rel_residual": info["true_rel_residual"],
                             "rel_diff_vs_fp64_plain": float(torch.linalg.vector_norm(x - x64) /
                                                             torch.linalg.vector_norm(x64))}
            for rec in res.values():
                rec["speedup_vs_fp64_plain"] = round(res["fp64_plain"]["time_s"] / rec["time_s"], 3)
            forms[f"asqtad_m{SECOND_MASS}"] = res
            args.mass = saved

    # ---- CPU baseline: the FP64 oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(fat, lng, b, dims, args.mass, iters, infos[-1]["restarts"])

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": round(value, 4),
            "unit": UNIT,
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(elapsed_s / args.steps * 1e3, 2),
            "higher_is_better": False,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "ff64" if arith == binding.STAG_ARITH_FF else "f64",
            "data": "synthetic (seeded SU(3) fields exp(0.3 i H), Gaussian source)",
            "config": workload_config(dims, args.mass, world),
            "roofline": roofline,
            "roofline_f64": roof64,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": gpu_launches,
            "clocks": clock_info,
            "solve": {"iters": iters, "restarts": infos[-1]["restarts"],
                      "true_rel_residual": infos[-1]["true_rel_residual"],
                      "solve_ms_median": round(solve_ms, 2), "host_s_timed": round(host_s, 3)},
            "gflops_paper_convention": round(gflops, 1),
            "dslash_eo_cg_avg_ms": round(eo_ms, 4),
            "kernel_shares": kernel_shares,
            "forms": forms,
            "paper_context": PAPER_CONTEXT,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------- batched workload
BATCH_MAIN = (32, 32, 32, 64)
BATCH_NRHS = 16
BATCH_LATTICES = [(8, 8, 8, 8)] * 8 + [(16, 16, 16, 16)] * 8 + [(24, 24, 24, 48)] * 8


def run_batched(args):
    """16 Gaussian right-hand sides on one 32^3 x 64 asqtad-form field (m = 0.0062) plus
    24 independent lattices (8^4, 16^4, 24^3 x 48; one-hop fields, m from 0.01 to 0.05),
    all solved to 1e-10 by one batch; compared with solving them one at a time."""
    import numpy as np
    import torch

    from paper_1010_4782_gb300 import accounting, binding, build, inputs

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    binding.load()
    stream = torch.cuda.current_stream(dev)
    fat, lng = inputs.asqtad_form_fields(BATCH_MAIN, seeds=(21, 22, 23))
    fat_d, lng_d = torch.from_numpy(fat).to(dev), torch.from_numpy(lng).to(dev)
    del fat, lng
    fats, lngs, dims, masses, bs = [], [], [], [], []
    for k in range(BATCH_NRHS):
        fats.append(fat_d)
        lngs.append(lng_d)
        dims.append(BATCH_MAIN)
        masses.append(MASS)
        bs.append(torch.from_numpy(inputs.gaussian_even_source(BATCH_MAIN, 1000 * rank + k)).to(dev))
    ms_lat = np.linspace(0.01, 0.05, len(BATCH_LATTICES))
    for j, d in enumerate([] if args.main_only else BATCH_LATTICES):
        fats.append(torch.from_numpy(inputs.gauge_field(d, 500 + j)).to(dev))
        lngs.append(None)
        dims.append(d)
        masses.append(float(ms_lat[j]))
        bs.append(torch.from_numpy(inputs.gaussian_even_source(d, 600 + j)).to(dev))
    n = len(bs)

    def step():
        bt = binding.stag_batch_create(fats, lngs, dims, masses)
        try:
            binding.stag_batch_set_stream(bt, stream)
            xs = [torch.zeros_like(b) for b in bs]
            code, infos = binding.stag_batch_solve(bt, bs, xs, TOL, MAX_ITER)
            tuning = binding.stag_batch_tuning(bt, 0)
        finally:
            binding.stag_batch_destroy(bt)
        if code != binding.STAG_OK:
            raise RuntimeError(f"batch solve failed: {code}")
        return infos, tuning

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        infos, tuning = step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clock_info = clocks.stop()
    elapsed = e0.elapsed_time(e1) / 1e3
    value = elapsed / args.steps

    # the same systems one at a time: mixed FP32 (the batch's inner arithmetic) and plain FP64
    def sequential(ar, inner):
        t0 = time.perf_counter()
        its = 0
        for k in range(n):
            o = binding.stag_default_options()
            o.arith = ar
            o.inner = inner
            h = binding.stag_create_ex(fats[k], lngs[k], dims[k], masses[k], o)
            try:
                x = torch.zeros_like(bs[k])
                code, info = binding.stag_cg_solve(h, bs[k], x, TOL, MAX_ITER)
                its += info["iters"]
            finally:
                binding.stag_destroy(h)
            if code != binding.STAG_OK:
                raise RuntimeError("sequential solve failed")
        torch.cuda.synchronize(dev)
        return time.perf_counter() - t0, its

    if args.no_sequential:
        seq32 = it32 = seq64 = it64 = None
    else:
        seq32, it32 = sequential(binding.STAG_ARITH_FF, binding.STAG_INNER_F32)
        seq64, it64 = sequential(binding.STAG_ARITH_F64, binding.STAG_INNER_NONE)
    rb, bsz, ms, sweep = tuning
    vh = accounting.half_sites(BATCH_MAIN)
    bytes_launch = vh * accounting.multi_rhs_bytes_per_site(BATCH_NRHS)  # FP32 links once + each RHS in and out
    peak, peak_src = measured_peaks()
    achieved = bytes_launch / (ms / 1e3) / 1e9
    line = {
        "metric": METRIC + " [batched workload]",
        "value": round(value, 4),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(value * 1e3, 2),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 (FP64-class reliable updates)",
        "data": "synthetic (seeded SU(3) fields exp(0.3 i H), Gaussian sources)",
        "config": {"workload": f"batched: {BATCH_NRHS} RHS on 32x32x32x64 asqtad-form (m={MASS})"
                               + ("" if args.main_only else
                                  " + 24 one-hop lattices (8x 8^4, 8x 16^4, 8x 24^3x48; m 0.01..0.05)")
                               + ", tol 1e-10",
                   "step": "stag_batch_create + stag_batch_solve + stag_batch_destroy"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4),
                     "traffic": recorded_traffic(f"multi_dslash_oe_f32_{BATCH_NRHS}rhs_32x32x32x64_rb{rb}_bs{bsz}_"
                                                 f"{'sweep' if sweep else 'runs'}", MULTI_SOURCES),
                     "kernel": f"multi-RHS D_oe, 16 RHS, FP32, {rb} RHS/thread, {bsz} threads/block, "
                               f"{'resident sweep' if sweep else 'contiguous tile runs'} "
                               "(autotuner's CUDA-event time)",
                     "algorithmic_bytes_per_launch": bytes_launch, "avg_launch_ms": round(ms, 4)},
        "clocks": clock_info,
        "systems": n,
        "iters_main_group": [i["iters"] for i in infos[:BATCH_NRHS]],
        "max_true_rel_residual": max(i["true_rel_residual"] for i in infos),
        "sequential_mixed_fp32_s": seq32 and round(seq32, 3),
        "sequential_fp64_plain_s": seq64 and round(seq64, 3),
        "speedup_vs_sequential_mixed_fp32": seq32 and round(seq32 / value, 3),
        "speedup_vs_sequential_fp64_plain": seq64 and round(seq64 / value, 3),
        "iters_total": {"batched": sum(i["iters"] for i in infos), "sequential_fp32": it32,
                        "sequential_fp64": it64},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------ learned workload
LEARNED_DIMS = (32, 32, 32, 64)


def run_learned(args):
    """Flexible CG with the parallel-transport network on a 32^3 x 64 asqtad-form field,
    m = 0.0062: training pairs from plain-CG solves of Gaussian sources, training on the
    GPU, then fresh test sources solved to 1e-10 with and without the network."""
    import numpy as np
    import torch

    from paper_1010_4782_gb300 import binding, build, inputs

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    binding.load()
    dims = LEARNED_DIMS
    fat, lng = inputs.asqtad_form_fields(dims, seeds=(31, 32, 33))
    opt = binding.stag_default_options()
    opt.arith = binding.STAG_ARITH_FF
    h = binding.Handle(torch.from_numpy(fat).to(dev), dims, args.mass, naik_long=torch.from_numpy(lng).to(dev),
                       options=opt)
    del fat, lng
    net = binding.stag_ptnet_create(h.h, binding.STAG_ARITH_BF16, 5)
    t0 = time.perf_counter()
    npairs, k = 0, 0
    while npairs < args.pairs:
        src = [torch.from_numpy(inputs.gaussian_even_source(dims, 7000 + k)).to(dev)]
        npairs = binding.stag_ptnet_add_pairs(net, src, stride=args.stride, min_rel_residual=args.min_rel,
                                              max_pairs=args.pairs)
        k += 1
    t_pairs = time.perf_counter() - t0
    loss0 = binding.stag_ptnet_dataset_loss(net)
    t0 = time.perf_counter()
    t_fcg0 = None
    # the network before training (its polynomial start) on the first test source
    b0 = torch.from_numpy(inputs.gaussian_even_source(dims, 90000)).to(dev)
    x0 = torch.zeros_like(b0)
    _, info_init = binding.stag_fcg_solve(h.h, net, b0, x0, TOL, MAX_ITER)
    losses = binding.stag_ptnet_train(net, args.epochs, 16, args.lr, seed=1)
    t_train = time.perf_counter() - t0
    loss1 = binding.stag_ptnet_dataset_loss(net)
    # the same network untrained: the library's polynomial start with the same seed
    net0 = binding.stag_ptnet_create(h.h, binding.STAG_ARITH_BF16, 5)
    res = {"fcg": [], "fcg_untrained": [], "fcg_fp32": [], "fcg_layered": [], "cg": []}
    for j in range(args.test_sources):
        b = torch.from_numpy(inputs.gaussian_even_source(dims, 90000 + j)).to(dev)
        runs = [("fcg", net, binding.STAG_ARITH_BF16), ("fcg_untrained", net0, binding.STAG_ARITH_BF16)]
        if j < 16:
            runs.append(("fcg_fp32", net, binding.STAG_ARITH_F32))
        for key, nt, prec in runs:
            binding.stag_ptnet_set_inference_precision(nt, prec)
            x = torch.zeros_like(b)
            code, info = binding.stag_fcg_solve(h.h, nt, b, x, TOL, MAX_ITER)
            res[key].append((code, info))
        binding.stag_ptnet_set_inference_precision(net, binding.STAG_ARITH_BF16)
        if j < 4:
            # the same network evaluated layer by layer (BF16 activations, tensor-core layer)
            binding.stag_ptnet_set_inference_form(net, binding.STAG_PTNET_LAYERED)
            x = torch.zeros_like(b)
            res["fcg_layered"].append(binding.stag_fcg_solve(h.h, net, b, x, TOL, MAX_ITER))
            binding.stag_ptnet_set_inference_form(net, binding.STAG_PTNET_COLLAPSED)
        x2 = torch.zeros_like(b)
        code2, info2 = binding.stag_cg_solve(h.h, b, x2, TOL, MAX_ITER)
        res["cg"].append((code2, info2))
    binding.stag_ptnet_destroy(net0)
    binding.stag_ptnet_destroy(net)
    h.close()
    # plain CG with native FP64 Dirac kernels (the FP64 comparison) on the first 4 sources
    opt64 = binding.stag_default_options()
    opt64.arith = binding.STAG_ARITH_F64
    fat, lng = inputs.asqtad_form_fields(dims, seeds=(31, 32, 33))
    h64 = binding.Handle(torch.from_numpy(fat).to(dev), dims, args.mass, naik_long=torch.from_numpy(lng).to(dev),
                         options=opt64)
    del fat, lng
    res["cg64"] = []
    for j in range(min(4, args.test_sources)):
        b = torch.from_numpy(inputs.gaussian_even_source(dims, 90000 + j)).to(dev)
        x3 = torch.zeros_like(b)
        res["cg64"].append(binding.stag_cg_solve(h64.h, b, x3, TOL, MAX_ITER))
    h64.close()

    def summary(rs):
        its = [i["iters"] for _, i in rs]
        ts = [i["time_ms"] / 1e3 for _, i in rs]
        return {"solved": sum(1 for c, _ in rs if c == binding.STAG_OK), "iters_mean": float(np.mean(its)),
                "time_s_mean": round(float(np.mean(ts)), 4),
                "max_true_rel_residual": max(i["true_rel_residual"] for _, i in rs),
                "restarts": sum(i["restarts"] for _, i in rs),
                "fallbacks": sum(i.get("fallbacks", 0) for _, i in rs)}

    fcg, fcg32, cg = summary(res["fcg"]), summary(res["fcg_fp32"]), summary(res["cg"])
    fcg0 = summary(res["fcg_untrained"])
    cg64 = summary(res["cg64"])
    fcg4 = summary(res["fcg"][:len(res["cg64"])])
    line = {
        "metric": METRIC + " [learned-preconditioner workload]",
        "value": fcg["time_s_mean"],
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.test_sources,
        "warmup": 0,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "float-float CG; network: BF16-stored intermediate, FP32 arithmetic (two-hop form)",
        "data": "synthetic (seeded SU(3) fields exp(0.3 i H), Gaussian sources)",
        "config": {"workload": f"flexible CG + 3-layer PT network (1-8-8-1 complex channels), "
                               f"{'x'.join(map(str, dims))} asqtad-form, m={args.mass}, tol {TOL}",
                   "pairs": npairs, "sources_for_pairs": k, "epochs": args.epochs, "batch": 16,
                   "pair_stride": args.stride, "pairs_while_rel_residual_above": args.min_rel,
                   "test_sources": args.test_sources},
        "pair_generation_s": round(t_pairs, 2),
        "training_s": round(t_train, 2),
        "untrained_start_first_source": {"iters": info_init["iters"], "restarts": info_init["restarts"],
                                         "fallbacks": info_init["fallbacks"]},
        "learning_rate": args.lr,
        "loss_before": loss0,
        "loss_after": loss1,
        "epoch_losses": [float(v) for v in losses],
        "fcg": fcg,
        "fcg_untrained_polynomial_start": fcg0,
        "iteration_gain_of_training": round(fcg0["iters_mean"] / fcg["iters_mean"], 3),
        "fcg_fp32_inference_first_16_sources": fcg32,
        "fcg_layered_bf16_tensor_cores_first_4_sources": summary(res["fcg_layered"]),
        "plain_cg_ff": cg,
        "plain_cg_fp64_first_sources": cg64,
        "time_ratio_fcg_over_fp64_cg_same_sources": round(fcg4["time_s_mean"] / cg64["time_s_mean"], 3),
        "iteration_gain_fp32_inference": round(summary(res["cg"][:16])["iters_mean"] / fcg32["iters_mean"], 3),
        "time_ratio_fp32_inference_over_cg": round(fcg32["time_s_mean"] / summary(res["cg"][:16])["time_s_mean"],
                                                   3),
        "iteration_gain": round(cg["iters_mean"] / fcg["iters_mean"], 3),
        "time_ratio_fcg_over_cg": round(fcg["time_s_mean"] / cg["time_s_mean"], 3),
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------- decomposed workload
# Sec. 4, Table 2: per-node times of the multi-GPU CG on 28^3 x 96 (FP64, one-hop
# operator, GTX 295 per node, 20 Gb InfiniBand), in ms.
PAPER_TABLE2 = {4: {"dirac": 4.7, "collect": 0.9, "d2h": 2.9, "exchange": 2.3, "h2d": 3.4},
                8: {"dirac": 2.45, "collect": 0.5, "d2h": 2.1, "exchange": 1.8, "h2d": 1.7}}


def run_decomposed(args):
    """The paper's decomposition emulated on one GPU: 28^3 x 96, one-hop FP64 operator,
    4 and 8 slabs along t; per-rank time of each step of one A application with the
    faces staged through the host (the paper's path) or copied device to device."""
    import numpy as np
    import torch

    from paper_1010_4782_gb300 import binding, build, inputs

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    binding.load()
    dims = tuple(args.dims)
    opt = binding.stag_default_options()
    opt.arith = binding.STAG_ARITH_F64
    h = binding.Handle(torch.from_numpy(inputs.gauge_field(dims, 1)).to(dev), dims, args.mass, options=opt)
    v = torch.from_numpy(inputs.gaussian_even_source(dims, 3)).to(dev)
    out = torch.empty_like(v)
    reps = 10
    results = {}
    for P in (4, 8):
        dd = binding.stag_dd_create(h.h, P)
        try:
            for mode, name in ((binding.STAG_DD_HOST, "host_staged"), (binding.STAG_DD_DEVICE, "device_direct"),
                               (binding.STAG_DD_HOST_OVERLAP, "host_staged_overlapped"),
                               (binding.STAG_DD_DEVICE_OVERLAP, "device_direct_overlapped")):
                binding.stag_dd_apply_A(dd, h.h, v, out, mode)  # warm-up
                acc = dict.fromkeys(binding.DD_PHASES, 0.0)
                for _ in range(reps):
                    ph = binding.stag_dd_apply_A(dd, h.h, v, out, mode)
                    for k in acc:
                        acc[k] += ph[k]
                per_rank = {k: round(acc[k] / reps / P, 4) for k in acc}
                if mode in (binding.STAG_DD_HOST_OVERLAP, binding.STAG_DD_DEVICE_OVERLAP):
                    # "dirac" is each whole overlapped half-Dslash; the host copies ran inside it
                    per_rank = {"overlapped_half_dslashes": per_rank["dirac"],
                                "host_copies_hidden": per_rank["exchange"], "total": per_rank["dirac"]}
                else:
                    per_rank["total"] = round(sum(per_rank.values()), 4)
                results[f"{P}_ranks_{name}"] = per_rank
            for mode, name in ((binding.STAG_DD_HOST, "host_staged"),
                               (binding.STAG_DD_HOST_OVERLAP, "host_staged_overlapped")):
                x = torch.zeros_like(v)
                code, info, ph = binding.stag_dd_cg_solve(dd, h.h, v, x, TOL, MAX_ITER, mode)
                results[f"{P}_ranks_cg_{name}"] = {
                    "status": code, "iters": info["iters"], "true_rel_residual": info["true_rel_residual"],
                    "time_s": round(info["time_ms"] / 1e3, 3),
                    "per_iteration_per_rank_ms": {k: round(ph[k] / max(1, info["iters"]) / P, 4) for k in ph}}
        finally:
            binding.stag_dd_destroy(dd)
    ref = torch.empty_like(v)
    binding.stag_apply_A(h.h, v, ref)
    h.close()
    line = {
        "metric": METRIC + " [emulated decomposition, Table 2]",
        "value": results["4_ranks_host_staged"]["total"],
        "unit": "ms per A application per rank",
        "n_gpus": world,
        "higher_is_better": False,
        "dtype": "f64",
        "data": "synthetic (seeded SU(3) field exp(0.3 i H), Gaussian vector)",
        "config": {"workload": f"{'x'.join(map(str, dims))} one-hop FP64, slabs along t, m={args.mass}",
                   "note": "all ranks on one GPU: per-rank = total over ranks / ranks"},
        "results": results,
        "paper_table2_per_node_ms": PAPER_TABLE2,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------- the oracle on the host cores
def _slab_worker(rank, n_workers, shm_names, shapes, dims, mass, halo, reps, start, out_q):
    """One process of the all-core oracle timing: oracle.Operator.apply_A, unchanged, on
    this process's t-slab widened by `halo` t-slices on each side (periodic).  Reports
    "ready" once its slab is built, waits for `start`, applies A `reps` times, reports
    "done" with its own time and then the interior rows of the result."""
    import numpy as np
    from multiprocessing import shared_memory

    import oracle

    try:
        shms = [shared_memory.SharedMemory(name=n) for n in shm_names]
        try:
            arrs = [np.ndarray(shp, dtype=np.complex128, buffer=m.buf) for m, shp in zip(shms, shapes)]
            fat, chi = arrs[0], arrs[-1]
            lng = arrs[1] if len(arrs) == 3 else None
            lx, ly, lz, lt = dims
            ts = lt // n_workers
            idx = [(rank * ts - halo + k) % lt for k in range(ts + 2 * halo)]
            dims_s = (lx, ly, lz, ts + 2 * halo)
            op = oracle.Operator(fat[idx], None if lng is None else lng[idx], mass, dims_s)
            v = oracle.restrict(chi[idx], dims_s, 0)
            del fat, lng, chi, arrs
        finally:
            for m in shms:
                m.close()
    except BaseException as e:
        out_q.put(("error", rank, repr(e)))
        raise
    out_q.put(("ready", rank))
    start.wait()
    t0 = time.perf_counter()
    for _ in range(reps):
        y = op.apply_A(v)
    dt = time.perf_counter() - t0
    out_q.put(("done", rank, dt))
    v3h = lx * ly * lz // 2
    out_q.put(("rows", rank, y[halo * v3h:(halo + ts) * v3h]))


def _slab_workers(lt, cores, halo):
    """Most processes w <= cores (at most 16) that split lt into equal slabs of even
    length (so each slab's parity matches the lattice's), each narrower than the lattice
    once widened by the halo; 1 when no split helps."""
    for w in range(min(16, cores), 1, -1):
        if lt % w == 0 and (lt // w) % 2 == 0 and lt // w + 2 * halo < lt:
            return w
    return 1


def oracle_apply_A_all_cores(fat, lng, b, dims, mass, reps):
    """Time oracle.Operator.apply_A on the host cores: the lattice split into t-slabs, one
    spawned process per slab, each applying the oracle's A, unchanged, to its slab widened
    by the reach of A (2 t-slices one-hop, 6 with Naik) and keeping the interior rows.
    Returns (seconds per A application over the whole lattice, processes, A b)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory

    import numpy as np

    import oracle

    halo = 6 if lng is not None else 2
    w = _slab_workers(dims[3], os.cpu_count() or 1, halo)
    if w == 1:
        op = oracle.Operator(fat, lng, mass, dims)
        t0 = time.perf_counter()
        for _ in range(reps):
            y = op.apply_A(b)
        return (time.perf_counter() - t0) / reps, 1, y
    chi = oracle.embed(b, dims, 0)
    srcs = [fat] + ([lng] if lng is not None else []) + [chi]
    shms = []
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    try:
        for a in srcs:
            m = shared_memory.SharedMemory(create=True, size=a.nbytes)
            np.ndarray(a.shape, dtype=np.complex128, buffer=m.buf)[...] = a
            shms.append(m)
        for k in saved:  # one thread per process: the process count is the core count used
            os.environ[k] = "1"
        ctx = mp.get_context("spawn")
        start = ctx.Event()
        out_q = ctx.Queue()
        procs = [ctx.Process(target=_slab_worker,
                             args=(r, w, [m.name for m in shms], [a.shape for a in srcs], tuple(dims), mass,
                                   halo, reps, start, out_q)) for r in range(w)]
        for p in procs:
            p.start()

        inbox = {"ready": {}, "done": {}, "rows": {}}

        def collect(kind):
            """Wait until every process has sent a message of this kind (messages of
            later kinds that arrive meanwhile are kept for their own wait)."""
            while len(inbox[kind]) < w:
                try:
                    msg = out_q.get(timeout=5)
                except Exception:
                    if any(not p.is_alive() and p.exitcode for p in procs):
                        raise RuntimeError("an oracle process died")
                    continue
                if msg[0] == "error":
                    raise RuntimeError(f"oracle process {msg[1]} failed: {msg[2]}")
                inbox[msg[0]][msg[1]] = msg[2:]
            return inbox[kind]

        try:
            collect("ready")            # every slab built
            t0 = time.perf_counter()
            start.set()
            collect("done")             # every process applied A reps times
            dt = time.perf_counter() - t0
            parts = {r: v[0] for r, v in collect("rows").items()}
        finally:
            for p in procs:
                p.join(timeout=60)
                if p.is_alive():
                    p.terminate()
        y = np.concatenate([parts[r] for r in range(w)])
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
        for m in shms:
            m.close()
            m.unlink()
    return dt / reps, w, y


def cpu_baseline(fat, lng, b, dims, mass, iters, restarts):
    """The oracle on the host: Fig. 1 (cg_fig1, initial residual + one iteration = two A
    applications) on one core, and A applied on all cores (t-slab processes); the value
    scales the all-core time per A application to the GPU solve's A applications."""
    import numpy as np

    import oracle

    model, ncpu = host_cpu()
    op = oracle.Operator(fat, lng, mass, dims)
    t0 = time.perf_counter()
    oracle.cg_fig1(op.apply_A, b, np.zeros_like(b), TOL, 1)
    dt1 = time.perf_counter() - t0
    del op
    per_a1 = dt1 / 2
    per_aw, w, _ = oracle_apply_A_all_cores(fat, lng, b, dims, mass, reps=2)
    n_a = 1 + iters + (restarts + 1)
    return {"value": round(per_aw * n_a, 1), "unit": UNIT, "cores": w, "kind": "oracle",
            "sample": f"numpy FP64 oracle on {'x'.join(map(str, dims))}: oracle.Operator.apply_A on {w} "
                      f"processes (t-slabs widened by the reach of A, one thread each), 2 applications; "
                      f"value = time per A application x the {n_a} A applications of the GPU solve",
            "per_A_application_s": round(per_aw, 3),
            "single_core": {"per_A_application_s": round(per_a1, 3), "value": round(per_a1 * n_a, 1),
                            "sample": "cg_fig1 on the full system: initial residual + 1 iteration = "
                                      f"2 A applications in {dt1:.1f} s"},
            "host_cpu": model, "host_logical_cores": ncpu}


# ----------------------------------------------------------- reference arm
def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle  # noqa: F401  (the arm runs the oracle only)
    from paper_1010_4782_gb300 import inputs

    dims = tuple(args.dims)
    fat, lng = inputs.asqtad_form_fields(dims)
    b = inputs.gaussian_even_source(dims, 0)
    model, ncpu = host_cpu()
    # warm-up applications, then K timed ones, all on the host cores
    if args.warmup:
        oracle_apply_A_all_cores(fat, lng, b, dims, args.mass, reps=args.warmup)
    per_a, w, _ = oracle_apply_A_all_cores(fat, lng, b, dims, args.mass, reps=max(1, args.steps))
    if REFERENCE_ITERS is not None:
        n_a = REFERENCE_ITERS + 2
        value = per_a * n_a
        sample = (f"numpy FP64 oracle: oracle.Operator.apply_A on {w} processes (t-slabs of "
                  f"{'x'.join(map(str, dims))} widened by the reach of A, one thread each), {args.steps} timed "
                  f"applications; value = time per A application x {n_a} A applications of a solve "
                  f"({REFERENCE_ITERS} Fig. 1 iterations)")
    else:
        value = per_a
        sample = "time per A application (iteration count of the solve not recorded)"
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": round(value, 4),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(per_a * 1e3, 1),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded SU(3) fields exp(0.3 i H), Gaussian source)",
        "config": workload_config(dims, args.mass, world),
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": w, "kind": "oracle",
                         "sample": sample, "host_cpu": model, "host_logical_cores": ncpu},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "decomposed":
        run_decomposed(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
