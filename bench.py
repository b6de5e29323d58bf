#!/usr/bin/env python3
"""Benchmark of the batched block-Toeplitz solve on one GB300 per rank.

Workload (one step): solve Z x = v for the 32 x 32 array, b = 64 basis
functions per element (65,536 Toeplitz unknowns) and 512 edge unknowns, one
right-hand side of ones, mixed precision (FP32 FFT products inside GMRES(30),
FP64 refinement) to relative residual 1e-8.  The plan (the FFT'd generating
blocks, B and C) is built once and stays resident, as the method intends; its
build time is reported separately.

Printed (rank 0, one JSON line): solves/s of the mixed path (`value`), the
same through the host-buffer C-ABI call with the copies inside the timed
region (`e2e`), the plain FP64 path on the same inputs, the FFT-matvec GB/s,
p50/p99 solve latency, the roofline of the dominant kernel measured live with
CUDA events, SM clocks during the timed region, and the CPU oracle timed on a
bounded sample (`cpu_baseline`).

`--impl reference` times the CPU FP64 oracle instead (direct products of the
same system on the host cores; each step is a row sample of one product,
extrapolated to a full solve).

Multi-GPU (`torchrun --nproc-per-node N`): independent replicas, one system
per rank, no collective on the data path (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "c2_32x32_b64"
WORKLOAD_DESC = ("32x32 array, b=64 (65,536 Toeplitz + 512 edge unknowns), 1 RHS of ones, "
                 "mixed FP32/FP64 GMRES(30)-IR to rel. residual 1e-8")
METRIC = "solves/s & FFT-matvec HBM GB/s, mixed vs FP64 plain at 1e-8 residual; p50/p99"
# Products of one FP64 GMRES(30) solve of this system to 1e-8 (300 iterations
# + 11 true-residual products), used to extrapolate the CPU oracle's product
# time to a solve in the reference arm, which runs no GPU code.
PRODUCTS_PER_SOLVE_FP64 = 311


def env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def dist_setup():
    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    local = env_int("LOCAL_RANK", 0)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi sampler for the timed region."""

    def __init__(self, gpu_id: str):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", gpu_id, f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        # the sampler's start-up (NVML initialisation) stays out of the timed
        # region: wait for its first sample (at most 5 s)
        t0 = time.perf_counter()
        while self.p is not None and self.p.poll() is None and time.perf_counter() - t0 < 5.0:
            if os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.05)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def profiled_traffic(profile: str, kernel_pattern: str):
    """DRAM bytes per launch recorded by an ncu capture under profiles/, or None
    when the kernel's source text has changed since the capture."""
    import hashlib
    import re
    try:
        text = open(os.path.join(ROOT, "profiles", profile)).read()
        src = open(os.path.join(ROOT, "paper_2506_04710_gb300", "csrc", "matvec.cu")).read()
    except OSError:
        return None
    t = re.search(r"traffic_bytes_per_launch: (\d+)", text)
    h = re.search(r"kernel_source_sha256_16: (\w+)", text)
    m = re.search(kernel_pattern, src, re.S)
    if not (t and h and m) or hashlib.sha256(m.group(0).encode()).hexdigest()[:16] != h.group(1):
        return None
    return int(t.group(1))


def oracle_product_seconds(prob, fraction: float):
    """CPU oracle: direct FP64 product on a row sample; returns (sample s, full-product s)."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import numpy as np
    import oracle
    step = max(1, int(round(1.0 / fraction)))
    rows = np.arange(0, prob.n, step)
    t = time.perf_counter()
    oracle.matvec_rows(prob, prob.V, rows)
    dt = time.perf_counter() - t
    return dt, dt * prob.n / len(rows), len(rows)


def omp_threads():
    return env_int("OMP_NUM_THREADS", os.cpu_count() or 1)


def run_reference(args, world, rank):
    """CPU oracle arm: each step times the oracle's direct FP64 product on a
    1/16 row sample of the same system; a whole solve is out of reach on the
    host (311 full products), so `value` is extrapolated from the median step
    and labelled as such, while `ms_per_step` is the measured sample time."""
    if rank != 0:
        return
    from paper_2506_04710_gb300 import synth
    prob, tol = synth.config_problem(WORKLOAD)
    frac = 1.0 / 16
    for _ in range(max(0, args.warmup)):
        oracle_product_seconds(prob, frac / 4)
    samples, fulls = [], []
    for _ in range(max(5, args.steps)):
        dt, full, nrows = oracle_product_seconds(prob, frac)
        samples.append(dt)
        fulls.append(full)
    full_med = statistics.median(fulls)
    value = 1.0 / (full_med * PRODUCTS_PER_SOLVE_FP64)
    sample = (f"per step: direct FP64 product (oracle_matvec_rows) on {nrows} of {prob.n} rows (1/16); "
              f"value = 1 / (median over {len(samples)} steps of the sample time x 16 x "
              f"{PRODUCTS_PER_SOLVE_FP64} products of a GMRES(30) solve)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": len(samples), "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(samples),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": {"workload": WORKLOAD_DESC},
            "extrapolated": True,
            "extrapolation": ("ms_per_step is the measured 1/16-row sample; value extrapolates it to a whole "
                              f"solve ({PRODUCTS_PER_SOLVE_FP64} full products)"),
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": omp_threads(), "kind": "oracle",
                             "sample": sample, "sample_seconds": sum(samples),
                             "full_product_s_median": full_med},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    from paper_2506_04710_gb300 import build as libbuild
    libbuild.build()
    from paper_2506_04710_gb300 import synth, ztoep
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prob, tol = synth.config_problem(WORKLOAD)
    stream = torch.cuda.current_stream(dev)

    structured = prob.edge_per_cell > 0 and args.structured_edges
    t0 = time.perf_counter()
    plan = ztoep.Plan.from_problem(prob, device=dev, autotune=0 if args.no_autotune else prob.nrhs,
                                   structured=structured)
    torch.cuda.synchronize(dev)
    plan_ms = 1e3 * (time.perf_counter() - t0)
    tune = plan.tune.as_dict() if plan.tune is not None else None
    V = torch.from_numpy(prob.V.copy()).to(dev)
    X = torch.zeros_like(V)
    N, nrhs = prob.n, prob.nrhs

    def opts(prec):
        o = ztoep.ztoep_default_opts()
        o.prec, o.tol, o.restart = prec, tol, args.restart
        o.flags = ztoep.ZTOEP_FLAG_ZERO_GUESS | (ztoep.ZTOEP_FLAG_HOST_LOOP if args.host_loop else 0)
        return o

    o_mixed = opts(ztoep.ZTOEP_MIXED)
    info = ztoep.info_array(nrhs)

    def solve(o):
        st = ztoep.ztoep_solve(plan.handle, o, nrhs, V, X, info, stream)
        if st != 0:
            raise RuntimeError(f"solve failed: {ztoep.ztoep_status_string(st)}")

    for _ in range(max(3, args.warmup)):
        solve(o_mixed)
    torch.cuda.synchronize(dev)

    # ---- timed region: mixed solves (one CUDA-graph launch each)
    props = torch.cuda.get_device_properties(dev)
    gpu_id = str(getattr(props, "uuid", local))
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) > 8:
        gpu_id = "GPU-" + gpu_id
    clocks = Clocks(gpu_id)
    launches0 = ztoep.ztoep_launch_count()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier(world)
    torch.cuda.synchronize(dev)
    evs[0].record(stream)
    for k in range(args.steps):
        solve(o_mixed)
        evs[k + 1].record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    launches = ztoep.ztoep_launch_count() - launches0
    clk = clocks.stop()
    step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    total_ms = allmax(world, sum(step_ms))
    value = world * args.steps * nrhs / (total_ms / 1e3)
    iters = info[0].inner_iters
    outer = info[0].outer
    relres = info[0].rel_residual
    X_mixed = X.clone()
    resident_mb = ztoep.ztoep_plan_get_info(plan.handle).resident_bytes / 1e6

    # ---- FFT-matvec (FP32 product, as inside the inner iterations) with live
    # per-kernel CUDA-event timing on the launching streams
    E, NT = prob.n_edge, prob.n_toep
    b, F = prob.b, plan.info.lx * plan.info.ly
    Xm = torch.from_numpy(np.ones((nrhs, N), np.complex128)).to(dev)
    Ym = torch.empty_like(Xm)
    for _ in range(3):
        ztoep.ztoep_matvec(plan.handle, ztoep.ZTOEP_MIXED, nrhs, Xm, Ym, stream)
    nmv = 50
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(nmv):
        ztoep.ztoep_matvec(plan.handle, ztoep.ZTOEP_MIXED, nrhs, Xm, Ym, stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    mv_ms = e0.elapsed_time(e1) / nmv
    ztoep.ztoep_timing_reset()
    ztoep.ztoep_timing_enable(1 << ztoep.K_EDGE | 1 << ztoep.K_BLOCKPROD | 1 << ztoep.K_FFT)
    for _ in range(nmv):
        ztoep.ztoep_matvec(plan.handle, ztoep.ZTOEP_MIXED, nrhs, Xm, Ym, stream)
    torch.cuda.synchronize(dev)
    ztoep.ztoep_timing_enable(0)
    kt = {}
    for name, c in (("fft", ztoep.K_FFT), ("blockprod", ztoep.K_BLOCKPROD), ("edge", ztoep.K_EDGE)):
        n, ms = ztoep.ztoep_timing_read(c)
        kt[name] = {"launches": n, "avg_us": 1e3 * ms / max(1, n)}
    # the same kernels alone: the edge branch serialised after the FFT chain,
    # so each kernel's time is its own (the roofline's), not shared HBM time
    ztoep.ztoep_timing_reset()
    ztoep.ztoep_timing_enable(1 << ztoep.K_EDGE | 1 << ztoep.K_BLOCKPROD | 1 << ztoep.K_FFT | ztoep.ZTOEP_TIMING_SERIAL)
    for _ in range(nmv):
        ztoep.ztoep_matvec(plan.handle, ztoep.ZTOEP_MIXED, nrhs, Xm, Ym, stream)
    torch.cuda.synchronize(dev)
    ztoep.ztoep_timing_enable(0)
    kt_alone = {}
    for name, c in (("fft", ztoep.K_FFT), ("blockprod", ztoep.K_BLOCKPROD), ("edge", ztoep.K_EDGE)):
        n, ms = ztoep.ztoep_timing_read(c)
        kt_alone[name] = {"launches": n, "avg_us": 1e3 * ms / max(1, n)}
    That_bytes = plan.info.n_pairs * b * b * 8
    # edge coupling: dense B read once, or the 4k side-generator spectra read twice (B x_T, B^T x_E)
    edge_stream = (2 * 4 * prob.edge_per_cell * F * b * 8) if structured else E * NT * 8
    mv_bytes = That_bytes + 2 * NT * nrhs * 8 + 4 * F * b * nrhs * 8 + edge_stream + E * E * 8 + 4 * E * nrhs * 8
    mv_gbs = mv_bytes / (mv_ms / 1e3) / 1e9

    # roofline of the edge-coupling kernel (one pass over B, FP32), the largest
    # HBM stream of the product
    pk = peaks()
    hbm = pk.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    # [B | C] read once (B and C in one pass), x read, B^T x_E and y_E written
    edge_bytes = E * (NT + E) * 8 + (NT + E) * 8 * nrhs + (NT + E) * 8 * nrhs
    edge_us = kt_alone["edge"]["avg_us"]
    edge_gbs = edge_bytes / (edge_us / 1e6) / 1e9 if edge_us > 0 else None
    bp_bytes = plan.info.n_pairs * b * b * 8 + 2 * F * b * nrhs * 8
    bp_us = kt_alone["blockprod"]["avg_us"]
    bp_gbs = bp_bytes / (bp_us / 1e6) / 1e9 if bp_us > 0 else None
    if structured:  # B is gone: the largest HBM stream is the spectrum in the block product
        roofline = {"kernel": "k_blockprod_tma (FP32 per-frequency block product, half spectrum)", "bound": "hbm",
                    "achieved": bp_gbs, "peak": hbm, "unit": "GB/s",
                    "frac": (bp_gbs / hbm) if bp_gbs else None,
                    "traffic": profiled_traffic("k_blockprod_tma_c2_32x32_b64.md",
                                                r"template <typename R, int NST>\n__global__ void __launch_bounds__\(256\) k_blockprod_tma\(.*?\n}\n"),
                    "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, "
                                      "profiles/k_blockprod_tma_c2_32x32_b64.md",
                    "bytes_per_launch": bp_bytes, "avg_launch_us": bp_us,
                    "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                    "timed": f"CUDA events around each block-product launch over {nmv} FP32 products, "
                             "branches serialised (the kernel alone)",
                    "frac_concurrent": (bp_bytes / (kt["blockprod"]["avg_us"] / 1e6) / 1e9 / hbm)
                    if kt["blockprod"]["avg_us"] > 0 else None}
    else:
        roofline = {"kernel": "k_edge3 (FP32 B x_T + C x_E and B^T x_E, one pass over [B | C])", "bound": "hbm",
                    "achieved": edge_gbs, "peak": hbm, "unit": "GB/s",
                    "frac": (edge_gbs / hbm) if edge_gbs else None,
                    "traffic": profiled_traffic("k_edge3_c2_32x32_b64.md",
                                                r"template <int RC>\n__global__ void __launch_bounds__\(256\) k_edge3\(.*?\n}\n"),
                    "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, "
                                      "profiles/k_edge3_c2_32x32_b64.md",
                    "bytes_per_launch": edge_bytes, "avg_launch_us": edge_us,
                    "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                    "timed": f"CUDA events around each k_edge3 launch over {nmv} FP32 products, "
                             "branches serialised (the kernel alone)",
                    "frac_concurrent": (edge_bytes / (kt["edge"]["avg_us"] / 1e6) / 1e9 / hbm)
                    if kt["edge"]["avg_us"] > 0 else None}

    # ---- FP64 plain path on the same inputs
    o64 = opts(ztoep.ZTOEP_FP64)
    solve(o64)
    torch.cuda.synchronize(dev)
    k64 = max(2, args.steps // 3)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(k64):
        solve(o64)
    f1.record(stream)
    torch.cuda.synchronize(dev)
    fp64_ms = allmax(world, f0.elapsed_time(f1)) / k64
    fp64_value = world * nrhs / (fp64_ms / 1e3)
    fp64_iters, fp64_outer = info[0].inner_iters, info[0].outer

    # ---- end to end through the host-buffer C-ABI call (copies in the timed region)
    Vh = torch.from_numpy(prob.V.copy()).pin_memory()
    Xh = torch.zeros_like(Vh).pin_memory()
    for _ in range(2):
        ztoep.ztoep_solve_host(plan.handle, o_mixed, nrhs, Vh, Xh, info, stream)
    barrier(world)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st = ztoep.ztoep_solve_host(plan.handle, o_mixed, nrhs, Vh, Xh, info, stream)
        assert st == 0
    torch.cuda.synchronize(dev)
    e2e_s = allmax(world, time.perf_counter() - t0)
    barrier(world)
    e2e_value = world * args.steps * nrhs / e2e_s

    # FFT passes on their own (the metric's FFT-matvec GB/s for the passes,
    # separate from the whole product): x pass (Nx + Lx) Ny b r, y pass
    # (Ny + Ly) Lx b r complex64 read + written, two of each per product
    lx, ly = plan.info.lx, plan.info.ly
    fft_bytes = 2 * ((prob.nx + lx) * prob.ny + (prob.ny + ly) * lx) * b * nrhs * 8
    fft_pass_us = kt_alone["fft"]["avg_us"]
    fft_gbs = fft_bytes / (4 * fft_pass_us / 1e6) / 1e9 if fft_pass_us > 0 else None
    fft_passes = {"bytes_per_product": fft_bytes, "passes_per_product": 4, "avg_pass_us": fft_pass_us,
                  "GB/s": fft_gbs, "frac_of_hbm": fft_gbs / hbm if fft_gbs else None,
                  "note": "4 register-FFT passes per FP32 product, timed alone; at 1 RHS each pass moves "
                          "1.6-3.2 MB and is latency-bound; the >=60% target is met at 16+ RHS "
                          "(fp32_product_classes_us of the 64x64 b96 section and its ncu profile)"}

    cpu, oracle_check = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        oracle_check, full, times = c2_oracle_checks(prob, tol, plan, X_mixed, stream, dev, o_mixed)
        oracle_check["rel_residual_gpu"] = relres
        products = fp64_iters + fp64_outer
        cpu = {"value": 1.0 / (full * products), "unit": "solves/s", "cores": omp_threads(), "kind": "oracle",
               "extrapolated": True,
               "sample": (f"median of {len(times)} direct FP64 products of the full system "
                          f"(oracle_matvec_blocks, {min(times):.1f}-{max(times):.1f} s each), scaled by the "
                          f"{products} products of the FP64 GMRES(30) solve of this system")}

    sections = {}
    if rank == 0 and world == 1 and not args.headline_only:
        libs_cases = {"c2_32x32_b64_r1": (prob.nx, prob.ny, b, E, nrhs, lx, ly,
                                          {"fft_per_direction_us": 2 * fft_pass_us,
                                           "blockprod_us": kt_alone["blockprod"]["avg_us"],
                                           "edge_us": kt_alone["edge"]["avg_us"]})}
        plan.close()
        plan = None
        torch.cuda.empty_cache()
        sections["c2_structured_edges"] = section_c2_structured(args, dev, local)
        torch.cuda.empty_cache()
        sections["c3"] = section_c3(args, dev, local)
        torch.cuda.empty_cache()
        if not args.no_c4:
            sections["c4"] = section_c4(args, dev, local)
            cl = sections["c4"]["fp32_product_classes_us"]
            libs_cases["c4_64x64_b96_r32"] = (64, 64, 96, 1024, 32, sections["c4"]["lx"], sections["c4"]["ly"],
                                              {k: v["us_per_product"] for k, v in cl.items()})
            torch.cuda.empty_cache()
        if args.serve_requests > 0:
            gid = gpu_uuid(dev, local)
            serve_stream(args, "mixed", 4, dev)  # warm-up
            clocks = Clocks(gid)
            mixed = serve_stream(args, "mixed", args.serve_requests, dev)
            clk = clocks.stop()
            grouped = None
            if args.serve_group_max > 1:  # the same requests, grouped solves
                clocks = Clocks(gid)
                grouped = serve_stream(args, "mixed", args.serve_requests, dev, group_max=args.serve_group_max)
                grouped["clocks"] = clocks.stop()
            unique = None
            if args.serve_unique > 0:
                clocks = Clocks(gid)
                unique = serve_stream(args, "mixed", args.serve_unique, dev, designs=1 << 20)
                unique["clocks"] = clocks.stop()
            fp64s = None
            if args.serve_fp64 > 0:
                clocks = Clocks(gid)
                fp64s = serve_stream(args, "fp64", args.serve_fp64, dev)
                fp64s["clocks"] = clocks.stop()
            sections["serve"] = {"workload": SERVE_DESC, "mixed": mixed, "clocks": clk,
                                 "mixed_grouped": grouped, "mixed_unique_designs": unique,
                                 "fp64_plain_prefix": fp64s}
            torch.cuda.empty_cache()
        sections["libs"] = section_libs(dev, stream, libs_cases)

    if rank == 0:
        s_sorted = sorted(step_ms)
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64 products + f64 refinement",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "nx": prob.nx, "ny": prob.ny, "b": prob.b, "n_edge": E,
                       "edge_coupling": (f"perimeter side-Toeplitz, {prob.edge_per_cell} per cell side "
                                         "(side generator spectra)") if structured else "dense B",
                       "nrhs": nrhs, "tol": tol, "restart": args.restart, "lx": lx,
                       "ly": ly,
                       "l2": "inputs larger than L2: each timed step (one whole solve) streams the plan "
                             "(FP32 and FP64 spectra, edge data) and the Krylov basis, "
                             f"{resident_mb:.0f} MB resident "
                             "> 129 MB L2",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": int(nrhs * N * 16),
                    "d2h_bytes_per_step": int(nrhs * N * 16)},
            "gpu_launches": int(launches),
            "clocks": clk,
            "latency_ms": {"p50": s_sorted[len(s_sorted) // 2],
                           "p99": s_sorted[min(len(s_sorted) - 1, int(0.99 * len(s_sorted)))]},
            "solve": {"iterations": iters, "sweeps": outer, "rel_residual": relres},
            "fp64_plain": {"value": fp64_value, "ms_per_step": fp64_ms, "iterations": fp64_iters,
                           "sweeps": fp64_outer},
            "speedup_vs_fp64": value / fp64_value,
            "fft_matvec": {"GB/s": mv_gbs, "us": mv_ms * 1e3, "bytes": mv_bytes,
                           "frac_of_hbm": mv_gbs / hbm,
                           "scope": "the whole FP32 product (dense B is 268 of its 347 MB), public call"},
            "fft_passes": fft_passes,
            "oracle_check": oracle_check,
            "blockprod": {"GB/s": bp_gbs, "bytes_per_launch": bp_bytes},
            "product_kernels_us": kt,
            "product_kernels_alone_us": kt_alone,
            "plan_ms": plan_ms,
            "autotune": tune,
            "launches_per_step": launches / args.steps,
        }
        line.update(sections)
        print(json.dumps(line), flush=True)
    if plan is not None:
        plan.close()


def gpu_uuid(dev, local):
    import torch
    gid = str(getattr(torch.cuda.get_device_properties(dev), "uuid", local))
    if gid and not gid.startswith("GPU-") and len(gid) > 8:
        gid = "GPU-" + gid
    return gid


def oracle_module():
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle
    return oracle


def c2_oracle_checks(prob, tol, plan, X, stream, dev, o_mixed):
    """The headline solve checked against the oracle, and the oracle timed.
    Its direct FP64 product of the GPU's final solution gives the true
    residual; a manufactured x* (V* = Z x* by the oracle) solved on the GPU at
    the configuration's tolerance gives the forward error; three more direct
    products of the RHS complete five timings of a full product (median)."""
    import numpy as np
    import torch
    from paper_2506_04710_gb300 import synth, ztoep
    orc = oracle_module()
    times = []
    Xh = X.cpu().numpy()
    t = time.perf_counter()
    ZX = orc.matvec_blocks(prob, Xh)
    times.append(time.perf_counter() - t)
    res = float(np.max(np.linalg.norm(prob.V - ZX, axis=1) / np.linalg.norm(prob.V, axis=1)))
    xs = synth.manufactured_solution(prob, 1, seed=77)
    t = time.perf_counter()
    Vs = orc.matvec_blocks(prob, xs)
    times.append(time.perf_counter() - t)
    Vd = torch.from_numpy(Vs).to(dev)
    Xd = torch.zeros_like(Vd)
    info = ztoep.info_array(1)
    st = ztoep.ztoep_solve(plan.handle, o_mixed, 1, Vd, Xd, info, stream)
    torch.cuda.synchronize(dev)
    err = float(np.linalg.norm(Xd.cpu().numpy() - xs) / np.linalg.norm(xs))
    for _ in range(3):
        t = time.perf_counter()
        orc.matvec_blocks(prob, prob.V)
        times.append(time.perf_counter() - t)
    full = statistics.median(times)
    check = {"oracle_rel_residual": res, "rel_residual_gpu": None,
             "manufactured": {"status": int(st), "tol": tol, "rel_residual_gpu": info[0].rel_residual,
                              "forward_error": err,
                              "note": "x* seeded, V* = Z x* by the oracle's direct product, mixed solve at "
                                      "the configuration's tolerance; forward error <= cond(Z) x residual"}}
    return check, full, times


def section_c2_structured(args, dev, local):
    """The headline system with its perimeter edge layout declared: the plan keeps
    the 2-D spectra of the side generators instead of B (B x_T and B^T x_E in
    the frequency domain of the FFT product), mixed and FP64 plain."""
    import torch
    from paper_2506_04710_gb300 import synth, ztoep
    prob, tol = synth.config_problem(WORKLOAD)
    stream = torch.cuda.current_stream(dev)
    plan = ztoep.Plan.from_problem(prob, device=dev, autotune=prob.nrhs, structured=True)
    V = torch.from_numpy(prob.V.copy()).to(dev)
    X = torch.zeros_like(V)
    info = ztoep.info_array(1)

    def timed(prec, k):
        o = ztoep.ztoep_default_opts()
        o.prec, o.tol, o.restart = prec, tol, 30
        o.flags = ztoep.ZTOEP_FLAG_ZERO_GUESS
        assert ztoep.ztoep_solve(plan.handle, o, 1, V, X, info, stream) == 0
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record(stream)
        for _ in range(k):
            assert ztoep.ztoep_solve(plan.handle, o, 1, V, X, info, stream) == 0
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / k, info[0].inner_iters, info[0].rel_residual

    clocks = Clocks(gpu_uuid(dev, local))
    ms, it, res = timed(ztoep.ZTOEP_MIXED, 10)
    ms64, it64, res64 = timed(ztoep.ZTOEP_FP64, 2)
    clk = clocks.stop()
    cl = product_classes(plan, 1, dev, stream)
    plan.close()
    return {"workload": WORKLOAD_DESC + "; perimeter edge layout (4 per cell side) through the side "
                                        "generator spectra instead of dense B",
            "mixed": {"solves_per_s": 1e3 / ms, "ms_per_solve": ms, "iterations": it, "rel_residual": res},
            "fp64_plain": {"solves_per_s": 1e3 / ms64, "ms_per_solve": ms64, "iterations": it64,
                           "rel_residual": res64},
            "speedup_vs_fp64": ms64 / ms, "fp32_product_classes_us": cl, "clocks": clk}


def section_c3(args, dev, local):
    """Two coupled 9x9 arrays as a 19x9 grid with a one-cell gap (Sec. III-B
    scale): 162 delta-port RHS in one batched solve, mixed and FP64 plain, each
    solution against the oracle's LU (the LU timed as the CPU baseline)."""
    import numpy as np
    import torch
    from paper_2506_04710_gb300 import synth, ztoep
    orc = oracle_module()
    prob, tol = synth.config_problem("c3_19x9gap_b48")
    stream = torch.cuda.current_stream(dev)
    nrhs = prob.nrhs
    plan = ztoep.Plan.from_problem(prob, device=dev, autotune=nrhs)
    V = torch.from_numpy(prob.V.copy()).to(dev)
    X = torch.zeros_like(V)
    info = ztoep.info_array(nrhs)

    def opts(prec):
        o = ztoep.ztoep_default_opts()
        o.prec, o.tol, o.restart = prec, tol, 30
        o.flags = ztoep.ZTOEP_FLAG_ZERO_GUESS
        return o

    def solve(o):
        st = ztoep.ztoep_solve(plan.handle, o, nrhs, V, X, info, stream)
        if st != 0:
            raise RuntimeError(f"c3 solve failed: {ztoep.ztoep_status_string(st)}")

    om, o64 = opts(ztoep.ZTOEP_MIXED), opts(ztoep.ZTOEP_FP64)
    for _ in range(2):
        solve(om)
    clocks = Clocks(gpu_uuid(dev, local))
    k = 5
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(k + 1)]
    torch.cuda.synchronize(dev)
    evs[0].record(stream)
    for i in range(k):
        solve(om)
        evs[i + 1].record(stream)
    torch.cuda.synchronize(dev)
    ms = sorted(evs[i].elapsed_time(evs[i + 1]) for i in range(k))
    it_m = max(i.inner_iters for i in info)
    Xm = X.cpu().numpy()
    solve(o64)  # warm-up (graph build)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    f0.record(stream)
    solve(o64)
    f1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms64 = f0.elapsed_time(f1)
    it_64 = max(i.inner_iters for i in info)
    X64 = X.cpu().numpy()
    plan.close()
    Z = orc.assemble(prob)
    t = time.perf_counter()
    lu = orc.LU(Z)
    lu_s = time.perf_counter() - t
    t = time.perf_counter()
    xref = lu.solve(prob.V)
    sol_s = time.perf_counter() - t

    def ferr(Xg):
        e = np.linalg.norm(Xg - xref, axis=1) / np.linalg.norm(xref, axis=1)
        return {"max": float(e.max()), "median": float(np.median(e))}

    mask = orc.unknown_mask(prob)
    med = ms[len(ms) // 2]
    return {"workload": "19x9 grid (two 9x9 arrays, one-cell gap), b=48, 324 edge unknowns, 162 delta-port RHS "
                        "in one batched solve, GMRES(30)-IR to rel. residual 1e-8",
            "n": prob.n, "nrhs": nrhs, "lx": plan.info.lx, "ly": plan.info.ly,
            "mixed": {"rhs_solves_per_s": nrhs / (med / 1e3), "ms_per_solve": {"p50": med, "max": ms[-1]},
                      "iterations": it_m, "forward_error_vs_lu": ferr(Xm),
                      "oracle_rel_residual_max": float(orc.relres(Z, Xm, prob.V).max()),
                      "gap_column_exactly_zero": bool(np.all(Xm[:, mask == 0] == 0))},
            "fp64_plain": {"rhs_solves_per_s": nrhs / (ms64 / 1e3), "ms_per_solve": ms64, "iterations": it_64,
                           "forward_error_vs_lu": ferr(X64),
                           "oracle_rel_residual_max": float(orc.relres(Z, X64, prob.V).max())},
            "speedup_vs_fp64": ms64 / med,
            "cpu_baseline": {"value": nrhs / (lu_s + sol_s), "unit": "RHS solves/s", "kind": "oracle",
                             "cores": omp_threads(), "lu_s": lu_s, "solve_s": sol_s,
                             "sample": f"oracle LU with partial pivoting of the dense {prob.n}x{prob.n} Z "
                                       "and the 162-RHS triangular solves, one run (> 10 s)"},
            "clocks": clk}


def product_classes(plan, nrhs, dev, stream, reps=10):
    """Per-class kernel time of the FP32 product (public call, branches
    serialised so each kernel runs alone), us per product."""
    import torch
    from paper_2506_04710_gb300 import ztoep
    x = torch.ones((nrhs, plan.n), dtype=torch.complex128, device=dev)
    y = torch.empty_like(x)
    ztoep.ztoep_matvec(plan.handle, ztoep.ZTOEP_MIXED, nrhs, x, y, stream)
    names = ["fft", "blockprod", "edge", "arnoldi", "misc", "tensor_lockstep", "tensor_pipe"]
    ztoep.ztoep_timing_reset()
    ztoep.ztoep_timing_enable(((1 << len(names)) - 1) | ztoep.ZTOEP_TIMING_SERIAL)
    for _ in range(reps):
        ztoep.ztoep_matvec(plan.handle, ztoep.ZTOEP_MIXED, nrhs, x, y, stream)
    torch.cuda.synchronize(dev)
    ztoep.ztoep_timing_enable(0)
    out = {}
    for c, n in enumerate(names):
        k, t = ztoep.ztoep_timing_read(c)
        if k:
            out[n] = {"launches_per_product": k / reps, "us_per_product": 1e3 * t / reps}
    return out


def section_c4(args, dev, local):
    """64x64 array, b=96, 32 plane-wave RHS: one mixed solve (autotuned plan,
    CUDA-graph solve), the FP64 plain solve under a stated time cap, and the
    oracle's residual components on sampled rows of the mixed solution."""
    import numpy as np
    import torch
    from paper_2506_04710_gb300 import synth, ztoep
    orc = oracle_module()
    t = time.perf_counter()
    prob, tol = synth.config_problem("c4_64x64_b96")
    gen_s = time.perf_counter() - t
    stream = torch.cuda.current_stream(dev)
    nrhs = prob.nrhs
    t = time.perf_counter()
    plan = ztoep.Plan.from_problem(prob, device=dev, autotune=nrhs)
    torch.cuda.synchronize(dev)
    plan_s = time.perf_counter() - t
    V = torch.from_numpy(prob.V).to(dev)
    X = torch.zeros_like(V)
    info = ztoep.info_array(nrhs)

    def opts(prec, cap_s=0.0):
        o = ztoep.ztoep_default_opts()
        o.prec, o.tol, o.restart = prec, tol, 30
        o.flags = ztoep.ZTOEP_FLAG_ZERO_GUESS
        o.timeout_ns = int(cap_s * 1e9)
        return o

    om = opts(ztoep.ZTOEP_MIXED)
    assert ztoep.ztoep_solve(plan.handle, om, nrhs, V, X, info, stream) == 0
    clocks = Clocks(gpu_uuid(dev, local))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    st = ztoep.ztoep_solve(plan.handle, om, nrhs, V, X, info, stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    it_m = max(i.inner_iters for i in info)
    res_m = max(i.rel_residual for i in info)
    Xm = X.cpu().numpy()
    classes = product_classes(plan, nrhs, dev, stream)
    cap = args.c4_fp64_cap_s
    o64 = opts(ztoep.ZTOEP_FP64, cap)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    f0.record(stream)
    st64 = ztoep.ztoep_solve(plan.handle, o64, nrhs, V, X, info, stream)
    f1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms64 = f0.elapsed_time(f1)
    it_64 = max(i.inner_iters for i in info)
    res_64 = max(i.rel_residual for i in info)
    plan.close()
    rows = np.unique(np.concatenate([np.random.default_rng(5).choice(prob.n, 48, replace=False),
                                     np.arange(prob.n_toep, prob.n, 128), [0, prob.n - 1]]))
    r = prob.V[:, rows] - orc.matvec_rows(prob, Xm, rows)
    vn = np.linalg.norm(prob.V, axis=1)
    ratio = float(np.max(np.abs(r) / (tol * vn[:, None])))
    fp64 = {"status": ztoep.ztoep_status_string(st64), "ms": ms64, "iterations": it_64,
            "worst_rel_residual": res_64, "cap_s": cap,
            "ms_per_iteration": ms64 / max(1, it_64)}
    if st64 == 0:
        fp64["rhs_solves_per_s"] = nrhs / (ms64 / 1e3)
    # FFT passes of the FP32 product at this size (kernels alone, clocks above):
    # x pass (Nx + Lx) Ny b r, y pass (Ny + Ly) Lx b r complex64 read + written
    lx, ly = plan.info.lx, plan.info.ly
    fft_bytes = 2 * ((prob.nx + lx) * prob.ny + (prob.ny + ly) * lx) * prob.b * nrhs * 8
    fft_us = classes.get("fft", {}).get("us_per_product")
    hbm = peaks().get("hbm_gbs")
    fft_passes = {"bytes_per_product": fft_bytes, "us_per_product": fft_us,
                  "GB/s": fft_bytes / fft_us / 1e3 if fft_us else None,
                  "frac_of_hbm": fft_bytes / fft_us / 1e3 / hbm if (fft_us and hbm) else None,
                  "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    return {"workload": "64x64 array, b=96 (393,216 Toeplitz + 1,024 edge unknowns), 32 plane-wave RHS, "
                        "GMRES(30)-IR to rel. residual 1e-8",
            "fft_passes": fft_passes,
            "n": prob.n, "nrhs": nrhs, "lx": plan.info.lx, "ly": plan.info.ly,
            "host_generation_s": gen_s, "plan_and_autotune_s": plan_s,
            "mixed": {"status": ztoep.ztoep_status_string(st), "ms_per_solve": ms,
                      "rhs_solves_per_s": nrhs / (ms / 1e3), "iterations": it_m, "worst_rel_residual": res_m,
                      "ms_per_iteration": ms / max(1, it_m),
                      "oracle_sampled_residual": {"rows": int(len(rows)), "max_abs_r_over_tol_norm_v": ratio,
                                                  "note": "|r_k| <= tol ||v|| must hold for every row k "
                                                          "(ratio <= 1)"}},
            "fp64_plain": fp64,
            "iteration_speedup_vs_fp64": (ms64 / max(1, it_64)) / (ms / max(1, it_m)),
            "fp32_product_classes_us": classes,
            "clocks": clk}


def section_libs(dev, stream, cases):
    """Library yardsticks, timing only (never on the product path): cuFFT
    through torch.fft.fft2/ifft2 on the zero-padded planes, cuBLAS batched
    complex GEMM through torch.matmul for the per-frequency block product,
    and cuBLAS complex GEMM/GEMV for B x_T and B^T x_E; each beside the
    library's own kernels on the same shape (FP32 product, kernels alone)."""
    import torch

    def tm(fn, reps=20):
        for _ in range(3):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return 1e3 * a.elapsed_time(b) / reps

    out = {}
    for name, (nx, ny, b, E, r, lx, ly, ours) in cases.items():
        F, NT = lx * ly, nx * ny * b
        g = torch.Generator(device=dev).manual_seed(0)
        planes = torch.zeros((r * b, ly, lx), dtype=torch.complex64, device=dev)
        planes[:, :ny, :nx] = torch.randn((r * b, ny, nx), dtype=torch.complex64, device=dev, generator=g)
        us_f = tm(lambda: torch.fft.fft2(planes))
        spec = torch.fft.fft2(planes)
        us_i = tm(lambda: torch.fft.ifft2(spec))
        fbytes = 2 * r * b * F * 8
        A = torch.randn((F, b, b), dtype=torch.complex64, device=dev, generator=g)
        Xh = torch.randn((F, b, r), dtype=torch.complex64, device=dev, generator=g)
        us_bp = tm(lambda: torch.matmul(A, Xh))
        bp_bytes = F * b * b * 8 + 2 * F * b * r * 8
        del A, Xh, planes, spec
        res = {"cufft_fwd_us": us_f, "cufft_inv_us": us_i, "cufft_fwd_GBps": fbytes / us_f / 1e3,
               "cublas_blockprod_us": us_bp, "cublas_blockprod_GBps": bp_bytes / us_bp / 1e3,
               "blockprod_bytes": bp_bytes, "fft_bytes_per_direction": fbytes, "ours": ours}
        if E > 0:
            B = torch.randn((E, NT), dtype=torch.complex64, device=dev, generator=g)
            xt = torch.randn((NT, r), dtype=torch.complex64, device=dev, generator=g)
            xe = torch.randn((E, r), dtype=torch.complex64, device=dev, generator=g)
            us_e1 = tm(lambda: torch.matmul(B, xt))
            us_e2 = tm(lambda: torch.matmul(B.transpose(0, 1), xe))
            ebytes = E * NT * 8
            res.update({"cublas_Bx_us": us_e1, "cublas_BTx_us": us_e2, "cublas_edge_total_us": us_e1 + us_e2,
                        "cublas_edge_GBps_per_pass_over_B": ebytes / us_e1 / 1e3, "edge_B_bytes": ebytes})
            del B, xt, xe
        torch.cuda.empty_cache()
        out[name] = res
    return out


SERVE_DESC = ("Poisson stream, mean 50 requests/s: square arrays Nx=Ny ~ U{8..48}, b ~ {32,48,64,96}, "
              "E = 16 Nx, 1-64 plane-wave RHS, 4 element designs (seeds); solved to rel. residual 1e-8")


def serve_stream(args, prec_name, n_req, dev, designs=4, group_max=1):
    """Replays the first n_req requests of the stream at their arrival times
    through the scheduler.  Inputs are generated on the device by the client
    ahead of arrival (bounded by --serve-input-gb of unconsumed inputs) and
    freed once the scheduler has built the plan.  Latency = arrival -> the
    solution is in device memory (scheduler completion)."""
    import torch
    from paper_2506_04710_gb300 import synth, ztoep
    reqs = synth.serving_requests(n=n_req, rate=50.0, seed=0, designs=designs)
    prec = ztoep.ZTOEP_MIXED if prec_name == "mixed" else ztoep.ZTOEP_FP64
    sched = ztoep.Scheduler(hbm_budget=int(args.serve_budget_gb * 2**30), workers=args.serve_workers,
                            device=dev.index or 0, group_max=group_max)
    gen = torch.cuda.Stream(dev)
    cap = args.serve_input_gb * 2**30
    live = {}  # rid -> input bytes still held
    ids = []
    late = []

    def reap():
        for rid in list(live):
            if sched.drop_inputs(rid):
                del live[rid]

    launches0 = ztoep.ztoep_launch_count()
    t0 = time.perf_counter()
    for (t_arr, nx, b, nrhs, seed) in reqs:
        while live and sum(live.values()) > cap:
            reap()
            time.sleep(0.001)
        with torch.cuda.stream(gen):
            d = synth.make_problem_device(nx, nx, b, 16 * nx, seed, nrhs, device=dev)
            X = torch.empty_like(d["V"])
        gen.synchronize()
        o = ztoep.ztoep_default_opts()
        o.prec, o.tol = prec, 1e-8
        wait = t_arr - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        key = (nx << 40) | (b << 24) | (seed & 0xFFFFFF) | (1 << 62)
        t_sub = time.perf_counter() - t0
        k = 4  # E = 16 Nx on a square array: 4 per cell side (side-generator spectra, no dense B)
        rid = sched.submit((nx, nx, b, 16 * nx, None, 0, 0, k), d["T"], d["B"], d["C"], d["V"], X, opts=o,
                           plan_key=key, on_device=True)
        live[rid] = sum(t.numel() * 16 for t in (d["T"], d["B"], d["C"]))
        del d, X
        ids.append((rid, t_arr, nrhs, nx, b))
        late.append(max(0.0, t_sub - t_arr))
        reap()
    lat, svc, worst_res, fails, rhs_total = [], [], 0.0, 0, 0
    for (rid, t_arr, nrhs, nx, b), lt in zip(ids, late):
        rc, st, info = sched.wait(rid, 600000)
        if rc != 0 or st.status != 0:
            fails += 1
        lat.append(lt * 1e3 + st.latency_ms)
        svc.append(st.latency_ms - st.queue_ms)
        worst_res = max(worst_res, max(i["rel_residual"] for i in info))
        rhs_total += nrhs
        sched.release(rid)
    t_end = time.perf_counter() - t0
    stats = sched.stats()
    launches = ztoep.ztoep_launch_count() - launches0
    sched.close()
    lat.sort()
    svc.sort()
    span = t_end - reqs[0][0]
    return {"requests": n_req, "offered_rate_per_s": 50.0, "span_s": span,
            "requests_per_s": n_req / span, "rhs_solves_per_s": rhs_total / span, "rhs_total": rhs_total,
            "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                           "max": lat[-1]},
            "service_ms": {"p50": svc[len(svc) // 2], "p99": svc[min(len(svc) - 1, int(0.99 * len(svc)))],
                           "note": "admission -> result (latency_ms minus the time queued)"},
            "element_designs": designs,
            "plan_reuse_rate": int(stats.plans_reused) / max(1, n_req),
            "failed": fails, "worst_rel_residual": worst_res,
            "max_in_flight": int(stats.max_in_flight), "peak_bytes": int(stats.peak_bytes),
            "plans_built": int(stats.plans_built), "plans_reused": int(stats.plans_reused),
            "plans_evicted": int(stats.plans_evicted), "gpu_launches": int(launches),
            "workers": args.serve_workers, "budget_gb": args.serve_budget_gb,
            "group_max": group_max, "grouped_solves": int(stats.groups)}


def run_serve(args, world, rank, local):
    """Serving benchmark: the request stream through the scheduler, mixed
    precision, then the FP64 plain path on a shorter prefix of the same stream."""
    import torch
    from paper_2506_04710_gb300 import build as libbuild
    libbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank != 0:
        return
    props = torch.cuda.get_device_properties(dev)
    gpu_id = str(getattr(props, "uuid", local))
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) > 8:
        gpu_id = "GPU-" + gpu_id
    serve_stream(args, "mixed", 4, dev)  # warm-up: library, generator, allocator
    clocks = Clocks(gpu_id)
    mixed = serve_stream(args, "mixed", args.serve, dev)
    grouped = (serve_stream(args, "mixed", args.serve, dev, group_max=args.serve_group_max)
               if args.serve_group_max > 1 else None)
    fp64 = serve_stream(args, "fp64", args.serve_fp64, dev) if args.serve_fp64 > 0 else None
    clk = clocks.stop()
    line = {"metric": METRIC, "mode": "serving", "value": mixed["rhs_solves_per_s"], "unit": "RHS solves/s",
            "higher_is_better": True, "n_gpus": 1, "dtype": "c64 products + f64 refinement",
            "data": "synthetic", "config": {"workload": SERVE_DESC, "requests": args.serve},
            "mixed": mixed, "mixed_grouped": grouped, "fp64_plain": fp64, "clocks": clk}
    print(json.dumps(line), flush=True)


def run_many_port(args, local):
    """Many-port workload (Sec. IV-B, at the 32x32 b64 array's scale): one
    delta excitation per element (basis 0), all ports solved in mixed precision
    to 1e-8 in batches of --port-batch RHS (tensor-core products), then the
    admittance and power-wave scattering matrices of all ports (unit edge
    lengths, 50-ohm references).  Inputs and solutions stay on the device; the
    timed region is the batched solves plus the port matrices."""
    import numpy as np
    import torch
    from paper_2506_04710_gb300 import build as libbuild
    libbuild.build()
    from paper_2506_04710_gb300 import synth, ztoep
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nx = args.ports_nx
    prob = synth.make_problem(nx, nx, 64, 16 * nx, seed=0, rhs="ports")
    p, N = prob.V.shape
    ports = np.flatnonzero(prob.active.reshape(-1)) * prob.b
    plan = ztoep.Plan.from_problem(prob, device=dev, autotune=min(args.port_batch, p))
    V = torch.from_numpy(prob.V).to(dev)
    X = torch.zeros_like(V)
    o = ztoep.ztoep_default_opts()
    o.prec = ztoep.ZTOEP_MIXED
    o.tol = 1e-8
    o.flags = ztoep.ZTOEP_FLAG_ZERO_GUESS
    s = torch.cuda.current_stream(dev)
    nb = args.port_batch
    # warm-up: one batch (graph build, workspaces)
    info = ztoep.info_array(nb)
    st = ztoep.ztoep_solve(plan.handle, o, min(nb, p), V[:nb], X[:nb], info, s)
    assert st == 0, st
    lens, z0 = np.ones(p), np.full(p, 50.0)
    gpu_id = str(getattr(torch.cuda.get_device_properties(dev), "uuid", local))
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) > 8:
        gpu_id = "GPU-" + gpu_id
    clocks = Clocks(gpu_id)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    torch.cuda.synchronize(dev)
    e0.record(s)
    worst, iters = 0.0, []
    for b0 in range(0, p, nb):
        k = min(nb, p - b0)
        info = ztoep.info_array(k)
        st = ztoep.ztoep_solve(plan.handle, o, k, V[b0:b0 + k], X[b0:b0 + k], info, s)
        assert st == 0, st
        worst = max(worst, max(info[r].rel_residual for r in range(k)))
        iters.append(max(info[r].inner_iters for r in range(k)))
    e1.record(s)
    Y, S = ztoep.port_matrices(X, ports, lens, z0, s)
    e2.record(s)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    solve_ms, port_ms = e0.elapsed_time(e1), e1.elapsed_time(e2)
    Sh = S.cpu().numpy()
    recip = float(np.max(np.abs(Sh - Sh.T)) / np.max(np.abs(Sh)))
    line = {"metric": "port solves/s (delta excitations) and port-matrix time", "mode": "many_port",
            "value": p / ((solve_ms + port_ms) / 1e3), "unit": "port solves/s", "higher_is_better": True,
            "n_gpus": 1, "dtype": "c64 products + f64 refinement; f64 port matrices", "data": "synthetic",
            "config": {"workload": f"{nx}x{nx} array, b=64, E={16 * nx}: {p} element ports (basis 0), "
                                   f"delta excitations, mixed GMRES(30)-IR to rel. residual 1e-8 in batches "
                                   f"of {nb}, then Y = L I^ L and S (z0 = 50 ohm, unit edge lengths)",
                       "ports": p, "n": N, "batch": nb, "lx": plan.info.lx, "ly": plan.info.ly},
            "solve_ms": solve_ms, "port_matrices_ms": port_ms, "iterations_per_batch": iters,
            "worst_rel_residual": worst, "S_reciprocity_rel": recip, "clocks": clk}
    print(json.dumps(line), flush=True)
    plan.close()


def run_far_field(args, local):
    """Far field of the 32x32 b64 solution on the 64 x 64 array-factor grid
    (Eqs. farfieldBasis / tensorProd; synthetic per-basis tensor, 2
    polarisations): the plan's FP64 forward spectrum plus one b-term dot per
    (direction, polarisation), timed with CUDA events; the oracle's direct sum
    over the 1024 parts on a sample of directions beside it."""
    import numpy as np
    import torch
    from paper_2506_04710_gb300 import build as libbuild
    libbuild.build()
    from paper_2506_04710_gb300 import synth, ztoep
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prob, tol = synth.config_problem(WORKLOAD)
    plan = ztoep.Plan.from_problem(prob, device=dev)
    V = torch.from_numpy(prob.V.copy()).to(dev)
    o = ztoep.ztoep_default_opts()
    o.tol = tol
    X, _, st = plan.solve(V, opts=o)
    assert st == 0
    uv = synth.grid_directions(plan.info.lx, plan.info.ly)
    Fh = torch.from_numpy(synth.far_field_basis(prob, uv, 2)).to(dev)
    s = torch.cuda.current_stream(dev)
    for _ in range(3):
        F = plan.far_field(X, Fh, synth.K0, 376.73, s)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    torch.cuda.synchronize(dev)
    e0.record(s)
    for _ in range(reps):
        F = plan.far_field(X, Fh, synth.K0, 376.73, s)
    e1.record(s)
    torch.cuda.synchronize(dev)
    us = 1e3 * e0.elapsed_time(e1) / reps
    cpu = None
    if not args.no_cpu_baseline:
        sys.path.insert(0, os.path.join(ROOT, "oracle"))
        import oracle
        pick = np.arange(0, len(uv), 97)
        t = time.perf_counter()
        ref = oracle.far_field(prob, X.cpu().numpy()[:, :prob.n_toep], uv[pick], Fh.cpu().numpy()[pick],
                               synth.K0, 376.73)
        dt = time.perf_counter() - t
        Fg = F.cpu().numpy()[:, pick]
        cpu = {"directions": int(len(pick)), "seconds": dt, "us_per_direction": 1e6 * dt / len(pick),
               "max_rel_diff": float(np.max(np.abs(Fg - ref)) / np.max(np.abs(ref))), "kind": "oracle"}
    nb = prob.n_toep * 16 + plan.info.lx * plan.info.ly * (prob.b * 16 * 3 + 2 * 16 * 2)
    line = {"metric": "far-field grid time", "mode": "far_field", "value": us, "unit": "us",
            "higher_is_better": False, "n_gpus": 1, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"far field of the 32x32 b64 solution on the {plan.info.lx}x{plan.info.ly} "
                                   "array-factor grid, 2 polarisations, synthetic per-basis tensor",
                       "directions": int(len(uv)), "parts": prob.nx * prob.ny, "b": prob.b},
            "algorithmic_bytes": nb, "GB/s": nb / us / 1e3, "oracle_sample": cpu}
    print(json.dumps(line), flush=True)
    plan.close()


def run_product(args, local):
    """One configuration's FP32 product (the inner-iteration product) timed
    alone: per-class kernel times and the algorithmic GB/s and tensor flops.
    Used for kernel profiles of the larger systems."""
    import numpy as np
    import torch
    from paper_2506_04710_gb300 import build as libbuild
    libbuild.build()
    from paper_2506_04710_gb300 import synth, ztoep
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    key = args.workload
    if args.nrhs:
        cfg = dict(synth.CONFIGS[key])
        cfg.pop("tol")
        cfg.update(rhs="planewave", nrhs=args.nrhs)
        prob = synth.make_problem(seed=0, name=key, **cfg)
    else:
        prob, _ = synth.config_problem(key)
    structured = prob.edge_per_cell > 0 and args.structured_edges
    plan = ztoep.Plan.from_problem(prob, device=dev, autotune=0 if args.no_autotune else prob.nrhs,
                                   structured=structured)
    nr, N, NT, E, b = prob.nrhs, prob.n, prob.n_toep, prob.n_edge, prob.b
    F = plan.info.lx * plan.info.ly
    s = torch.cuda.current_stream(dev)
    x = torch.zeros((nr, N), dtype=torch.complex128, device=dev)
    y = torch.empty_like(x)
    for _ in range(max(3, args.warmup)):
        ztoep.ztoep_matvec(plan.handle, ztoep.ZTOEP_MIXED, nr, x, y, s)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(s)
    for _ in range(args.steps):
        ztoep.ztoep_matvec(plan.handle, ztoep.ZTOEP_MIXED, nr, x, y, s)
    e1.record(s)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    names = ["fft", "blockprod", "edge", "arnoldi", "misc", "tensor_lockstep", "tensor_pipe"]
    ztoep.ztoep_timing_reset()
    ztoep.ztoep_timing_enable((1 << len(names)) - 1)
    for _ in range(args.steps):
        ztoep.ztoep_matvec(plan.handle, ztoep.ZTOEP_MIXED, nr, x, y, s)
    torch.cuda.synchronize(dev)
    ztoep.ztoep_timing_enable(0)
    classes = {}
    for c, n in enumerate(names):
        k, t = ztoep.ztoep_timing_read(c)
        if k:
            classes[n] = {"launches_per_product": k / args.steps, "us_per_product": 1e3 * t / args.steps}
    tensor = nr >= 16
    spec = F * b * b * 8 if tensor else plan.info.n_pairs * b * b * 8
    k = prob.edge_per_cell
    bedge = (4 * k * F * b * 8 if structured else (2 if tensor else 1) * E * NT * 8) + E * E * 8
    byts = spec + bedge + 2 * NT * nr * 8 + 4 * F * b * nr * 8
    flops = 8.0 * F * b * b * nr + (16.0 * 4 * k * F * b * nr if structured else 16.0 * E * NT * nr)
    pk = peaks()
    line = {"mode": "product", "workload": key, "nrhs": nr, "n": N, "lx": plan.info.lx, "ly": plan.info.ly,
            "edge_coupling": "side generator spectra" if structured else "dense B",
            "product_ms": ms, "algorithmic_bytes": byts, "GB/s": byts / ms / 1e6,
            "frac_of_hbm": byts / ms / 1e6 / pk["hbm_gbs"] if pk.get("hbm_gbs") else None,
            "complex_flops": flops, "tf32_tflops_3x": 3 * flops / ms / 1e9 if tensor else None,
            "note": "product_ms includes the complex128 <-> complex64 conversions of the public call",
            "classes": classes}
    print(json.dumps(line), flush=True)
    plan.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="only the 32x32 b64 headline solve (no 19x9, 64x64, serving and library sections)")
    ap.add_argument("--no-c4", action="store_true", help="skip the 64x64 b96 section")
    ap.add_argument("--c4-fp64-cap-s", type=float, default=40.0,
                    help="time cap of the FP64 plain solve in the 64x64 b96 section")
    ap.add_argument("--serve-requests", type=int, default=60,
                    help="requests of the serving stream replayed in the default run (0: none)")
    ap.add_argument("--serve-unique", type=int, default=20,
                    help="requests replayed with a distinct element design each (no plan reuse)")
    ap.add_argument("--no-autotune", action="store_true", help="heuristic launch shapes, smallest embedding")
    ap.add_argument("--structured-edges", action="store_true",
                    help="use the side-generator spectra when the edge unknowns have the perimeter "
                         "side-Toeplitz layout (default: dense B; the serving mode always uses them)")
    ap.add_argument("--host-loop", action="store_true",
                    help="drive the solver loops from the host (for profilers; slower)")
    ap.add_argument("--serve", type=int, default=0,
                    help="serving mode: replay this many requests of the Poisson stream")
    ap.add_argument("--serve-fp64", type=int, default=6, help="requests replayed through the FP64 path")
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--serve-group-max", type=int, default=4,
                    help="also replay the requests with up to this many per grouped solve (1: skip)")
    ap.add_argument("--serve-budget-gb", type=float, default=96.0)
    ap.add_argument("--serve-input-gb", type=float, default=32.0)
    ap.add_argument("--product-only", action="store_true",
                    help="time the FP32 product of --workload (a configuration key) alone")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--nrhs", type=int, default=0, help="--product-only: plane-wave RHS count instead of the config's")
    ap.add_argument("--far-field", action="store_true",
                    help="far field of the 32x32 b64 solution on the array-factor grid")
    ap.add_argument("--many-port", action="store_true",
                    help="solve every element port of an --ports-nx square array (b=64) and form Y and S")
    ap.add_argument("--ports-nx", type=int, default=32)
    ap.add_argument("--port-batch", type=int, default=256)
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.product_only:
        if rank == 0:
            run_product(args, local)
    elif args.many_port:
        if rank == 0:
            run_many_port(args, local)
    elif args.far_field:
        if rank == 0:
            run_far_field(args, local)
    elif args.serve > 0:
        run_serve(args, world, rank, local)
    elif args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
