#!/usr/bin/env python3
"""Benchmark of the element volume term (Sec. 2, Eq. (2)) on GB300.

One step = one evaluation of the volume term over the whole timed workload:
order N = 7 (Nq = 8), 32^3 = 32768 elements (16,777,216 GLL points) on the
sine-warped 10 km box with the seeded perturbed hydrostatic state.  Metric:
GDOF/s = points per second / 1e9 (a DOF is a grid point, as in the paper's
Table 2), aggregated over all ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl numa|reference]

Under torchrun the ranks share one mesh of 32 x 32 x (32 ranks) elements by
contiguous element ranges (--shard elements, the default; each rank 32^3
elements) or each evaluates a replica of the workload (--shard replicas):
elements are independent in the volume term, so ranks need no data-path
collective (weak scaling).  Rank 0 prints one JSON line, with compact entries
for the batched and serving workloads and each mode's error against the
oracle.

--impl reference times the FP64 CPU oracle on the host cores instead (each step
a bounded sample of the same workload); only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "volume-RHS GDOF/s"
UNIT = "GDOF/s"
# Algorithmic HBM bytes per point: 5 state + 9 metric + Jinv + 2 reference arrays
# read, 5 rhs fields written; 8 bytes each in FP64 (176), 4 in FP32 (88).
BYTES_PER_NODE_FP64 = 176
BYTES_PER_NODE_MIXED = 88
# Algorithmic FP64 flops per point (an FMA counts 2, pow and divide count 1):
# EOS 5, three directions of u and fluxes 3 x 17, three D sweeps 30*Nq,
# Jinv scaling and gravity 8.
def flops_per_node_fp64(Nq: int) -> int:
    return 5 + 51 + 30 * Nq + 8


# FP64 CUDA-core peak of one GB300, used only when the FP64 pipe binds: the
# unit-count figure, and the rate a DFMA microbenchmark measured on the pool.
FP64_PEAK_TFLOPS = 1.25
FP64_DFMA_MEASURED_TFLOPS = 1.056
FALLBACK_HBM_GBS = 6800.0


def workload_full(n: int = 32):
    """The timed workload; a smaller n (elements per axis) is for ncu captures."""
    from paper_1604_08501_gb300 import workload as wl
    if n == wl.BENCH_FULL["n"]:
        return wl.bench_full(), wl.BENCH_FULL["name"]
    w = wl.make_workload(N=wl.BENCH_FULL["N"], n=n, seed=wl.BENCH_FULL["seed"])
    return w, f"N=7 (Nq=8), {n}^3={n ** 3} elements, warped 10 km box (profiling size)"


def shard_ranges(n: int, world: int):
    """Element layers of each rank when `world` ranks share one mesh of
    n x n x (n world) elements: rank r takes layers [n r, n (r + 1)), the
    contiguous elements [n^3 r, n^3 (r + 1)), an equal share Ne Nq^3 / world of
    the points."""
    return [(n * r, n * (r + 1)) for r in range(world)]


def workload_for_rank(n: int, rank: int, world: int, shard: str):
    """This rank's workload: under element sharding the rank's contiguous
    element range of one n x n x (n world)-element mesh (point for point the
    values of those elements in the whole mesh, so the ranks together evaluate
    the volume term of that mesh with no exchange: elements are independent);
    as replicas the whole n^3-element workload on every rank."""
    from paper_1604_08501_gb300 import workload as wl
    if world == 1 or shard == "replicas":
        return workload_full(n)
    z0, z1 = shard_ranges(n, world)[rank]
    w = wl.make_workload(N=wl.BENCH_FULL["N"], n=(n, n, n * world), seed=wl.BENCH_FULL["seed"],
                         z_range=(z0, z1))
    return w, (f"N=7 (Nq=8), one warped 10 km box of {n}x{n}x{n * world} elements shared by "
               f"{world} ranks by element layers ({n ** 3} elements, {w.M} points per rank)")


def workload_config(w, name):
    return {"workload": name, "N": w.N, "Nq": w.N + 1, "elements": w.Ne, "points": w.M,
            "seed": w.seed, "precision": "fp64",
            "l2": f"inputs larger than L2: {w.M * BYTES_PER_NODE_FP64 / 1e9:.2f} GB moved "
                  "per step against a 129 MB L2, no flush"}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback 6.8 TB/s (MEASURED_PEAKS.json absent)"


def sources_sha(paths) -> str:
    """sha256 (16 hex digits) over the code of the named C/CUDA source files, in
    order: comments removed and whitespace collapsed, so that an edit to a
    comment does not count as a change of the kernel."""
    import hashlib
    import re
    h = hashlib.sha256()
    for rel in paths:
        with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)   # block comments
        text = re.sub(r"//[^\n]*", " ", text)                # line comments
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def load_traffic(kernel: str):
    """DRAM bytes per full-size launch of ``kernel`` from the committed ncu
    summary, if none of the kernel's source files has changed since the
    counters were taken; None otherwise."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)[kernel]
        if sources_sha(d["sources"]) != d["sources_sha"]:
            return None
        return float(d["dram_bytes_per_launch"])
    except Exception:
        return None


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", self.gpu_id],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        time.sleep(0.3)

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = []
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append({"sm": float(f[1]), "max": float(f[2]), "power": float(f[3]),
                             "hw": f[5], "hw_thermal": f[6], "sw_thermal": f[7], "sw_power": f[8]})
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        # nvidia-smi prints no timestamps in this mode: samples are spaced ~50 ms
        # from start(); keep the busy ones (power well above idle) as "under load".
        pmax = max(r["power"] for r in rows)
        load = [r for r in rows if r["power"] >= 0.5 * pmax] or rows
        reasons = []
        for key, name in (("hw", "hw_slowdown"), ("hw_thermal", "hw_thermal_slowdown"),
                          ("sw_thermal", "sw_thermal_slowdown"), ("sw_power", "sw_power_cap")):
            if any(r[key].lower().startswith("active") for r in load):
                reasons.append(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load),
                "sm_max_mhz": max(r["max"] for r in load), "reasons": reasons,
                "samples_under_load": len(load), "power_w_max": pmax}


def gpu_id_for(device_index: int) -> str:
    import torch
    try:
        u = str(torch.cuda.get_device_properties(device_index).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            return vis.split(",")[device_index]
        return str(device_index)


# ---------------------------------------------------------------- distributed

def dist_setup(backend: str):
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend)
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, local, world


def reduce_max(x: float, device=None) -> float:
    """Max of x over ranks (identity without torch.distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def aggregate(units_per_rank: int, seconds_local: float, device=None):
    """Whole-job throughput: units all ranks processed / max time over ranks."""
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    tmax = reduce_max(seconds_local, device)
    return units_per_rank * world / tmax, tmax


# ---------------------------------------------------------------- CPU oracle

def cpu_model() -> str:
    """The host CPU's model string (x86 'model name', else the Arm implementer
    and part numbers), for the CPU baseline's record."""
    try:
        fields = {}
        for line in open("/proc/cpuinfo"):
            k, _, v = line.partition(":")
            fields.setdefault(k.strip(), v.strip())
        if "model name" in fields:
            return fields["model name"]
        if "CPU part" in fields:
            return f"{platform.machine()} implementer {fields.get('CPU implementer', '?')} " \
                   f"part {fields['CPU part']}"
    except OSError:
        pass
    return platform.machine()


def oracle_best_of(prob, q, repeats: int = 3, nthreads: int = 0):
    """Wall-clock seconds of `repeats` oracle O2 evaluations after one warm-up
    (page-in), each timed alone."""
    import oracle
    oracle.vol_rhs_o2(prob, q, nthreads)
    times = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        oracle.vol_rhs_o2(prob, q, nthreads)
        times.append(time.perf_counter() - t0)
    return times


def cpu_baseline(w, parity_w=None):
    """Oracle O2 on the host, wall clock, best of 3: one evaluation of the
    timed workload on all cores (the baseline value) and on one core, and the
    same for the small parity workload."""
    import oracle
    from paper_1604_08501_gb300 import workload as wl
    prob, q = w.problem(), w.q
    t_all = oracle_best_of(prob, q)
    t_one = oracle_best_of(prob, q, nthreads=1)
    pw = parity_w if parity_w is not None else wl.make_workload(4, 8, seed=0)
    pp = pw.problem()
    tp_all = oracle_best_of(pp, pw.q)
    tp_one = oracle_best_of(pp, pw.q, nthreads=1)
    rate = lambda m, ts: m / min(ts) / 1e9
    return {"value": rate(w.M, t_all), "unit": UNIT, "cores": oracle.max_threads(),
            "kind": "oracle",
            "sample": f"one evaluation of the whole timed workload ({w.Ne} elements, {w.M} "
                      f"points), oracle O2 (fluxes once per point, OpenMP over elements), best "
                      f"of 3 after a warm-up: " + ", ".join(f"{t:.3f}" for t in t_all) + " s",
            "single_core": {"value": rate(w.M, t_one), "unit": UNIT, "cores": 1,
                            "sample": "the same, one thread: "
                                      + ", ".join(f"{t:.3f}" for t in t_one) + " s"},
            "parity_workload": {"elements": pw.Ne, "points": pw.M,
                                "value": rate(pw.M, tp_all), "single_core": rate(pw.M, tp_one),
                                "unit": UNIT},
            "cpu_model": cpu_model()}


def run_reference(args):
    rank, local, world = dist_setup("gloo")
    if rank != 0:
        return 0
    import oracle
    w, name = workload_full(args.n)
    prob, q, m = w.problem(), w.q, w.M
    for _ in range(args.warmup):
        oracle.vol_rhs_o2(prob, q)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.vol_rhs_o2(prob, q)
    el = time.perf_counter() - t0
    value = args.steps * m / el / 1e9
    sample = (f"each step: oracle O2, one evaluation of the whole timed workload "
              f"({w.Ne} elements, {m} points) on all host cores")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w, name), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU

def time_variant(vt, q, q_host, dev, K, W, rank, e2e=True, min_region_s=0.0):
    """Device time of K launches (CUDA events on the launching stream, per
    launch and over the region), clocks sampled meanwhile, then K steps end to
    end through the host-buffer call.  With min_region_s > 0 the device-timed
    region runs more launches than K where K would take less than that long
    (the warm-up launches give the estimate); res["steps"] is the count."""
    import torch
    out = torch.empty_like(q)
    stream = torch.cuda.current_stream(dev)
    K_e2e = K
    w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0.record(stream)
    for _ in range(W):
        vt.rhs(q, out, stream)
    w1.record(stream)
    torch.cuda.synchronize(dev)
    if min_region_s > 0 and W > 0:
        est_ms = max(w0.elapsed_time(w1) / W, 1e-3)
        K = max(K, int(math.ceil(min_region_s * 1e3 / est_ms)))
        K = int(reduce_max(float(K), dev))   # every rank times the same count
    sampler = ClockSampler(gpu_id_for(dev.index)) if rank == 0 else None
    if sampler:
        sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(dev)
    torch.cuda.synchronize(dev)
    t_start.record(stream)
    for k in range(K):
        ev[k][0].record(stream)
        vt.rhs(q, out, stream)
        ev[k][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    barrier(dev)
    clocks = sampler.stop() if sampler else None
    per_launch = [a.elapsed_time(b) for a, b in ev]
    res = {"steps": K, "region_ms": t_start.elapsed_time(t_end),
           "kernel_ms": float(np.mean(per_launch)),
           "launch_ms": {"mean": float(np.mean(per_launch)),
                         "median": float(np.median(per_launch)), "best": float(np.min(per_launch))},
           "clocks": clocks, "e2e_s": None}
    if e2e:
        # H2D of q from pinned memory, the kernel, D2H of rhs, every step.
        out_host = torch.empty_like(q_host).pin_memory()
        for _ in range(3):
            vt.rhs_host(q_host, out_host)
        barrier(dev)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(K_e2e):
            vt.rhs_host(q_host, out_host)
        res["e2e_s"] = time.perf_counter() - t0
        barrier(dev)
    return res


def roofline_entries(kname, kernel_ms, w):
    peak, peak_src = measured_peaks()
    bpp = BYTES_PER_NODE_MIXED if "mixed" in kname else BYTES_PER_NODE_FP64
    hbm_gbs = bpp * w.M / (kernel_ms * 1e-3) / 1e9
    hbm = {"bound": "hbm", "achieved": hbm_gbs, "peak": peak, "unit": "GB/s",
           "frac": hbm_gbs / peak, "traffic": load_traffic(kname), "kernel": kname,
           "bytes_per_point": bpp, "peak_source": peak_src, "kernel_ms": kernel_ms}
    if "mixed" in kname:
        return hbm, None
    fp64_tfs = flops_per_node_fp64(w.N + 1) * w.M / (kernel_ms * 1e-3) / 1e12
    # FP64-equivalent flop rate against the FP64 pipe of one GB300 (152 SMs x
    # 2 DFMA/clk x 2 flop x 2.07 GHz = 1.26 TFLOP/s nominal).  It binds the
    # native kernel; the double-float kernel runs on the FP32 pipes.
    alu = {"bound": "alu", "achieved": fp64_tfs, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
           "frac": fp64_tfs / FP64_PEAK_TFLOPS, "traffic": load_traffic(kname), "kernel": kname,
           "flops_per_point": flops_per_node_fp64(w.N + 1),
           "peak_source": "FP64 pipe of one GB300 from its unit counts and clock: 152 SMs x 2 "
                          "DFMA/clk x 2 flop x 2.07 GHz = 1.26, quoted as the nominal 1.25 TFLOP/s",
           "peak_measured_dfma": FP64_DFMA_MEASURED_TFLOPS,
           "frac_of_measured_dfma": fp64_tfs / FP64_DFMA_MEASURED_TFLOPS,
           "peak_measured_source": "FMA-chain microbenchmark on this pool's GB300 (8 independent "
                                   "DFMA chains per thread): 528 G DFMA/s",
           "kernel_ms": kernel_ms}
    return (alu, hbm) if kname.startswith("vol_rhs_fp64") else (hbm, alu)


_ORACLE_RHS = {}


def oracle_rhs(w):
    """Oracle O2's volume term of workload w (computed once per process)."""
    import oracle
    key = (w.N, w.Ne, w.seed)
    if key not in _ORACLE_RHS:
        _ORACLE_RHS[key] = oracle.vol_rhs_o2(w.problem(), w.q)
    return _ORACLE_RHS[key]


def error_vs_oracle(x, ref):
    """Per-field normwise error of x against the FP64 oracle: max|x - ref| /
    max|ref| and ||x - ref||_2 / ||ref||_2."""
    names = ("rho", "rho_u", "rho_v", "rho_w", "rho_theta")
    out = {}
    for b in range(5):
        d = np.asarray(x[b], dtype=np.float64) - ref[b]
        out[names[b]] = {"max": float(np.max(np.abs(d)) / np.max(np.abs(ref[b]))),
                         "rms": float(np.linalg.norm(d) / np.linalg.norm(ref[b]))}
    return out


def run_gpu(args):
    import torch
    rank, local, world = dist_setup("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1604_08501_gb300 import build as lib_build
    if rank == 0 or world == 1:
        lib_build.build()
    barrier(dev)
    from paper_1604_08501_gb300.numa_vol import VolumeTerm

    w, name = workload_for_rank(args.n, rank, world, args.shard)
    K, W = args.steps, args.warmup

    results = {}
    for prec in args.precisions:
        # the mixed mode takes the FP32 perturbation state (input preparation,
        # outside the timed regions)
        # mixed-tc: the mixed mode with its D sums on the tensor cores
        mode = "mixed" if prec == "mixed-tc" else prec
        q_np = w.q_mixed() if mode == "mixed" else w.q
        q_host = torch.from_numpy(q_np).pin_memory()
        q = q_host.to(dev)
        step_bytes = q_np.nbytes
        vt = VolumeTerm.from_problem(w.problem(), precision=mode)
        if prec == "mixed-tc":
            vt.set_sweep("tensor_tf32")
        # The headline times exactly K launches; the other modes at least K
        # and at least 0.3 s of launches (the paper's timing loop, Sec. 4).
        r = time_variant(vt, q, q_host, dev, K, W, rank, e2e=not args.no_e2e,
                         min_region_s=0.0 if prec == args.precisions[0] else 0.3)
        r["kernel"] = vt.kernel_name
        if rank == 0 and not args.no_error:
            # one more evaluation (outside the timed regions) against the oracle
            out = vt.rhs(q)
            torch.cuda.synchronize(dev)
            r["error_vs_oracle"] = error_vs_oracle(out.cpu().numpy(), oracle_rhs(w))
            del out
        vt.close()
        Kv = r["steps"]
        value, tmax = aggregate(Kv * w.M, r["region_ms"] * 1e-3, dev)
        r["value"], r["ms_per_step"] = value / 1e9, tmax * 1e3 / Kv
        if r["e2e_s"] is not None:
            e2e_value, _ = aggregate(K * w.M, r["e2e_s"], dev)
            r["e2e"] = {"value": e2e_value / 1e9, "unit": UNIT,
                        "h2d_bytes_per_step": step_bytes, "d2h_bytes_per_step": step_bytes}
        else:
            r["e2e"] = None
        results[prec] = r

    if rank == 0:
        head_prec = args.precisions[0]
        head = results[head_prec]
        roof, other = roofline_entries(head["kernel"], head["kernel_ms"], w)
        dtypes = {"fp64": "f64", "df64": "df64 (FP32 hi+lo pairs, 48-bit)",
                  "mixed": "f32 (perturbation state)",
                  "mixed-tc": "f32 (perturbation state), D sums as TF32 split products"}
        cfg = workload_config(w, name)
        if world > 1:
            cfg["parallelism"] = (f"{world} ranks, " + ("contiguous element ranges of one mesh, "
                                  "no collective" if args.shard == "elements"
                                  else "a replica of the workload per rank, no collective"))
        line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world,
                "steps": K, "warmup": W, "ms_per_step": head["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": dtypes.get(head_prec, head_prec), "data": "synthetic",
                "config": cfg, "roofline": roof, "roofline_other": other,
                "e2e": head["e2e"], "gpu_launches": K, "clocks": head["clocks"],
                "precision": head_prec, "launch_ms": head["launch_ms"],
                "field_dof_rate": {"value": head["value"] * 5, "unit": "G field-DOF/s",
                                   "fields": 5}}
        variants = {}
        for prec in args.precisions[1:]:
            r = results[prec]
            vr, vo = roofline_entries(r["kernel"], r["kernel_ms"], w)
            variants[prec] = {"value": r["value"], "unit": UNIT, "ms_per_step": r["ms_per_step"],
                              "steps": r["steps"], "dtype": dtypes.get(prec, prec),
                              "roofline": vr, "roofline_other": vo, "e2e": r["e2e"],
                              "gpu_launches": r["steps"], "clocks": r["clocks"],
                              "launch_ms": r["launch_ms"]}
        if "error_vs_oracle" in head:
            line["error_vs_oracle"] = head["error_vs_oracle"]
        for prec in args.precisions[1:]:
            if "error_vs_oracle" in results[prec]:
                variants[prec]["error_vs_oracle"] = results[prec]["error_vs_oracle"]
        if world == 1 and not args.no_batched and args.n == 32:
            # the batched workload, compact: both precisions, 3 timed launches
            bres, bplan = batched_results(rank, dev, world, ["mixed", "fp64"], 64, 3, 3)
            variants["batched"] = {"metric": "batched volume-RHS GDOF/s (points x RK stages / s)",
                                   "workload": BATCHED_WORKLOAD.format(n=len(bplan)), **bres}
        if world == 1 and not args.no_serving and args.n == 32:
            # the serving workload at 200 req/s: 600 requests in the mixed
            # mode; FP64 (overloaded about 9x at this rate) the first 100 of
            # the same stream, so that the run stays short
            sres, splan = serving_results(rank, dev, world, ["mixed", "fp64"], 200.0, 600, 16,
                                          120, 4, "per_member", 3, {"fp64": 100})
            variants["serving"] = {
                "metric": "serving GDOF/s (points x RK stages / s) with p50/p99 request latency",
                "workload": f"Poisson arrivals at 200 req/s (mixed: 600 requests, fp64: the first "
                            f"100 of the same stream), each one of {len(splan)} instances "
                            f"(N in {{3,4,5,7}}, 512..32768 elements) advancing k in {{1,5,20}} "
                            f"LSRK(5,4) steps at dt = 0.01 s; budget 120 GB, <= 256 members, "
                            f"rounds of up to 4 steps, per-member round policy", **sres}
        if variants:
            line["variants"] = variants
        if world == 1 and not args.no_cpu_baseline and args.n == 32:
            line["cpu_baseline"] = cpu_baseline(w)
        print(json.dumps(line))
    return 0


def batched_results(rank, dev, world, precisions, instances, steps, warmup, orders=None):
    """The batched workload (run_batched's docstring) for each precision mode:
    rate, launch time and the autotuned configuration.  orders: keep only the
    plan's instances of these orders N."""
    import torch
    from paper_1604_08501_gb300 import workload as wl
    from paper_1604_08501_gb300.numa_vol import Batch, VolumeTerm
    plan = wl.batch_plan(count=instances)
    if orders:
        plan = [p for p in plan if p[0] in orders]
    works = [wl.integration_workload(N, n, seed) for N, n, seed in plan]
    nsteps, dt = 10, 0.01
    out = {}
    for name in precisions:
        # "mixed-tc": the mixed batch with its D sums on the tensor cores;
        # "mixed-auto": the autotuner picks the sweep per order
        # "mixed-tmem" / "mixed-smem": the CUDA-core tiles with the state in
        # tensor memory / shared memory, whatever the autotuner would choose
        prec, sweep = {"fp64": ("fp64", "cuda_cores"), "mixed": ("mixed", "cuda_cores"),
                       "mixed-tc": ("mixed", "tensor_tf32"),
                       "mixed-auto": ("mixed", "auto"), "mixed-tmem": ("mixed", "cuda_cores"),
                       "mixed-smem": ("mixed", "cuda_cores")}.get(name, (None, None))
        if prec is None:
            continue
        vts, states, points = [], [], 0
        for w in works:
            vts.append(VolumeTerm.from_problem(w.problem(), precision=prec))
            q0 = w.q_mixed() if prec == "mixed" else w.q
            states.append(torch.from_numpy(q0).to(dev))
            points += w.M
        b = Batch(prec, sweep=sweep)
        for vt, q in zip(vts, states):
            b.add(vt, q)
        b.autotune()
        if name in ("mixed-tmem", "mixed-smem"):
            b.set_config(state_in_tmem=name == "mixed-tmem")
        stream = torch.cuda.current_stream(dev)
        # Every launch integrates nsteps from the initial states: they are
        # restored before each launch, outside the timed events (the copy of
        # all states, larger than L2, also evicts it).
        saved = [q.clone() for q in states]

        def restore():
            for q, q0 in zip(states, saved):
                q.copy_(q0)

        for _ in range(warmup):
            restore()
            b.advance(nsteps, dt, stream)
        torch.cuda.synchronize(dev)
        sampler = ClockSampler(gpu_id_for(dev.index)) if rank == 0 else None
        if sampler:
            sampler.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        barrier(dev)
        for t0, t1 in ev:
            restore()
            t0.record(stream)
            b.advance(nsteps, dt, stream)
            t1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(dev)
        clocks = sampler.stop() if sampler else None
        ms = sum(t0.elapsed_time(t1) for t0, t1 in ev) / steps
        evals = points * 5 * nsteps
        value, tmax = aggregate(evals * steps, ms * 1e-3 * steps, dev)
        b.status()
        cfg = b.config()
        present = sorted({w.N + 1 for w in works})
        out[name] = {"value": value / 1e9, "unit": UNIT, "ms_per_launch": tmax * 1e3 / steps,
                     "steps": steps, "warmup": warmup, "gpu_launches": steps,
                     "points": points, "instances": len(plan), "sweep": sweep,
                     "dtype": {"fp64": "f64", "mixed": "f32 (perturbation state)"}[prec],
                     "autotuned": {"tile_elements_by_nq": {str(nq): cfg["tile"][nq] for nq in present},
                                   "sweep_by_nq": {str(nq): cfg["sweep"][nq] for nq in present},
                                   "ctas_per_sm": cfg["ctas_per_sm"] or "max",
                                   "costliest_first": cfg["costliest_first"],
                                   "state_in_tmem": cfg["state_in_tmem"],
                                   "tuned_ms_per_step": round(cfg["tuned_ms_per_step"], 4),
                                   "candidates_timed": cfg["tuned_candidates"]},
                     "clocks": clocks}
        b.close()
        for vt in vts:
            vt.close()
        del states, saved
        torch.cuda.empty_cache()
    return out, plan


BATCHED_WORKLOAD = ("{n} instances, N in {{3,4,5,7}}, 512..32768 elements (log-uniform, cubes), "
                    "smooth velocities (peak 10 m/s), 10 LSRK(5,4) steps at dt = 0.01 s per launch "
                    "from the initial states")


def run_batched(args):
    """The batched workload: 64 independent instances (N from {3,4,5,7},
    512..32768 elements) advanced by 10 low-storage RK steps at dt = 0.01 s in one
    graph-captured persistent launch.  Metric: volume-term evaluations per
    second, in GDOF/s (points x 5 stages x steps / time)."""
    import torch
    rank, local, world = dist_setup("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1604_08501_gb300 import build as lib_build
    lib_build.build()
    orders = [int(x) for x in args.orders.split(",") if x] if args.orders else None
    out, plan = batched_results(rank, dev, world, args.precisions, args.instances, args.steps,
                                args.warmup, orders)
    if rank == 0:
        head = args.precisions[0]
        line = {"metric": "batched volume-RHS GDOF/s (points x RK stages / s)",
                "value": out[head]["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": out[head]["ms_per_launch"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "df64": "df64 (FP32 hi+lo pairs, 48-bit)",
                          "mixed": "f32 (perturbation state)",
                          "mixed-tc": "f32 (perturbation state), TF32 split products",
                          "mixed-auto": "f32 (perturbation state)",
                          "mixed-tmem": "f32 (perturbation state)",
                          "mixed-smem": "f32 (perturbation state)"}[head],
                "data": "synthetic",
                "config": {"workload": BATCHED_WORKLOAD.format(n=len(plan))
                           + (f" (the plan's instances of orders N = {args.orders})" if orders else ""),
                           "points": out[head]["points"],
                           "l2": "states restored before each launch (a copy larger than L2)"},
                "gpu_launches": args.steps, "clocks": out[head]["clocks"], "precision": head,
                "autotuned": out[head]["autotuned"],
                "variants": {k: v for k, v in out.items() if k != head}}
        print(json.dumps(line))
    return 0


# The paper's Nq study: 3,538,944 points at Nq = 4, 8, 12 and 16 (Sec. 4, Table 2).
NQ_STUDY = {3: (48, 48, 24), 7: (24, 24, 12), 11: (16, 16, 8), 15: (12, 12, 6)}


def run_nq_sweep(args):
    """One evaluation per step of the 3,538,944-point mesh at each order of the
    paper's Nq study, NUMA_FP64, NUMA_DF64 (N <= 7) and NUMA_MIXED, with five fields and with three
    passive tracers (*_8fields: the paper's 8-field form, df64_8fields with
    df64 among the precisions; mixed_8fields is also its FP32 precision).  Inputs exceed L2 (0.68 GB FP64).  Metric: GDOF/s per
    order; `value` is Nq = 8."""
    import torch
    rank, local, world = dist_setup("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1604_08501_gb300 import build as lib_build
    from paper_1604_08501_gb300 import workload as wl
    from paper_1604_08501_gb300.numa_vol import VolumeTerm
    lib_build.build()
    stream = torch.cuda.current_stream(dev)
    per = {}
    launches = 0
    orders = [int(v) for v in args.orders.split(",")] if args.orders else list(NQ_STUDY)
    for N, shape in NQ_STUDY.items():
        if N not in orders:
            continue
        w = wl.make_workload(N, shape, seed=1, tracers=3)
        w5 = dataclasses.replace(w, q=w.q[:5])
        row = {"elements": w.Ne, "points": w.M}
        extra = ["fp64_8fields", "mixed_8fields"] + (
            ["df64_8fields"] if "df64" in args.precisions else [])
        for prec in list(args.precisions) + extra:
            if prec.startswith("df64") and N > 7:
                continue   # the double-float mode takes N <= 7
            # *_8fields: the paper's 8-field form (three passive tracers);
            # mixed_8fields is also the paper's precision (FP32)
            ww = w if prec.endswith("_8fields") else w5
            mode = prec.split("_")[0]
            vt = VolumeTerm.from_problem(ww.problem(), precision=mode)
            q = torch.from_numpy(np.ascontiguousarray(
                ww.q_mixed() if mode == "mixed" else ww.q)).to(dev)
            out = torch.empty_like(q)
            for _ in range(args.warmup):
                vt.rhs(q, out, stream=stream)
            torch.cuda.synchronize(dev)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            barrier(dev)
            for t0, t1 in ev:
                t0.record(stream)
                vt.rhs(q, out, stream=stream)
                t1.record(stream)
            torch.cuda.synchronize(dev)
            ms = statistics.median(t0.elapsed_time(t1) for t0, t1 in ev)
            value, tmax = aggregate(w.M * args.steps, ms * 1e-3 * args.steps, dev)
            row[prec] = {"gdofs": value / 1e9, "ms": tmax * 1e3 / args.steps,
                         "kernel": vt.kernel_name}
            launches += args.steps
            vt.close()
            del q, out
        per[str(N + 1)] = row
        torch.cuda.empty_cache()
    if rank == 0:
        head = args.precisions[0]
        ref_nq = "8" if "8" in per else sorted(per, key=int)[0]
        line = {"metric": "volume-RHS GDOF/s across orders, 3,538,944 points (Nq study)",
                "value": per[ref_nq][head]["gdofs"], "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": per[ref_nq][head]["ms"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "mixed": "f32 (perturbation state)",
                          "mixed-tc": "f32 (perturbation state), TF32 split products",
                          "mixed-auto": "f32 (perturbation state)"}[head],
                "data": "synthetic",
                "config": {"workload": "warped 10 km box, 3,538,944 points at Nq = 4, 8, 12, 16 "
                                       "(48x48x24, 24x24x12, 16x16x8, 12x12x6 elements), seed 1",
                           "l2": "inputs larger than L2 (0.68 GB FP64 per step), no flush"},
                "per_nq": per, "gpu_launches": launches, "precision": head}
        print(json.dumps(line))
    return 0


def serving_results(rank, dev, world, precisions, rate, requests, pool, budget_gb, round_steps,
                    round_policy, warmup, requests_by_prec=None):
    """The serving workload (run_serving's docstring) for each precision mode:
    delivered rate, offered load and request latencies."""
    import torch
    from paper_1604_08501_gb300 import workload as wl
    from paper_1604_08501_gb300.numa_vol import Engine, VolumeTerm
    local = dev.index
    plan = wl.batch_plan(count=pool)
    works = [wl.integration_workload(N, n, seed) for N, n, seed in plan]
    rng = np.random.Generator(np.random.PCG64(2024 + rank))
    total_max = max([requests] + list((requests_by_prec or {}).values()))
    gaps_all = rng.exponential(1.0 / rate, size=total_max)
    pick_all = rng.integers(0, len(works), size=total_max)
    ks_all = rng.choice(np.array([1, 5, 20]), size=total_max)
    dt = 0.01
    out = {}
    for prec in precisions:
        if prec not in ("fp64", "mixed"):
            continue
        # the first `total` requests of one seeded stream
        total = int((requests_by_prec or {}).get(prec, requests))
        gaps, pick, ks = gaps_all[:total], pick_all[:total], ks_all[:total]
        vts = [VolumeTerm.from_problem(w.problem(), precision=prec) for w in works]
        q0s = []
        for w in works:
            a = w.q_mixed() if prec == "mixed" else w.q
            t = torch.empty(a.shape, dtype=torch.float32 if prec == "mixed" else torch.float64,
                            pin_memory=True)
            t.numpy()[...] = a
            q0s.append(t)
        # Pinned output buffers, reused per mesh and allocated before the timed
        # region (a pinned allocation takes milliseconds and would stall the
        # serving loop): per mesh, as many as its requests arriving within any
        # 0.25 s; any further one is allocated on demand and counted.
        arrive_rel = np.cumsum(gaps)
        free = []
        for j in range(len(works)):
            t = arrive_rel[pick == j]
            need = int(np.max(np.searchsorted(t, t + 0.25) - np.arange(t.size))) if t.size else 0
            free.append([torch.empty(q0s[j].shape, dtype=q0s[j].dtype, pin_memory=True)
                         for _ in range(max(need, 1))])
        late = [0]

        def take(j):
            if free[j]:
                return free[j].pop()
            late[0] += 1
            return torch.empty(q0s[j].shape, dtype=q0s[j].dtype, pin_memory=True)

        with Engine(prec, budget_bytes=budget_gb << 30, max_members=256,
                    round_steps=round_steps, round_policy=round_policy) as eng:
            # warm-up: a few requests through the same path, not timed
            for j in range(min(warmup, len(works))):
                o = take(j)
                eng.submit(vts[j], q0s[j], o, 1, dt)
                eng.run_until_idle()
                free[j].append(o)
            base = eng.stats()
            late[0] = 0
            sampler = ClockSampler(gpu_id_for(local)) if rank == 0 else None
            if sampler:
                sampler.start()
            barrier(dev)
            t0 = time.monotonic()
            arrive = t0 + np.cumsum(gaps)
            ids, bufs, nxt, done = {}, {}, 0, 0
            while done < total:
                now = time.monotonic()
                while nxt < total and arrive[nxt] <= now:
                    j = int(pick[nxt])
                    o = take(j)
                    rid = eng.submit(vts[j], q0s[j], o, int(ks[nxt]), dt)
                    ids[rid], bufs[rid] = nxt, (j, o)
                    nxt += 1
                st = eng.stats()
                if st["queued"] == 0 and st["resident"] == 0:
                    if nxt >= total:
                        raise RuntimeError("engine idle with requests unaccounted for")
                    time.sleep(max(0.0, min(arrive[nxt] - time.monotonic(), 0.01)))
                    continue
                for rid in eng.progress():
                    j, o = bufs.pop(rid)
                    free[j].append(o)
                    done += 1
            lat, last = np.empty(total), 0.0
            for rid, i in ids.items():
                inf = eng.query(rid)
                lat[i] = inf["done_s"] - arrive[i]
                last = max(last, inf["done_s"])
            barrier(dev)
            clocks = sampler.stop() if sampler else None
            st = eng.stats()
            stages = st["point_stages"] - base["point_stages"]
            span = last - t0
            value, tmax = aggregate(int(stages), span, dev)
            offered = float(np.mean([works[int(j)].M for j in pick]) * 5 * np.mean(ks) * rate)
            out[prec] = {"value": value / 1e9, "span_s": tmax,
                         "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3),
                                        "p99": float(np.percentile(lat, 99) * 1e3),
                                        "max": float(lat.max() * 1e3)},
                         "offered_gdofs": offered / 1e9, "rounds": st["rounds"] - base["rounds"],
                         "requests": total, "rate_per_s": rate,
                         "late_pinned_allocations": late[0],
                         "clocks": clocks}
        for vt in vts:
            vt.close()
        del q0s, free
        torch.cuda.empty_cache()
    return out, plan


def run_serving(args):
    """The serving workload: a Poisson stream of ensemble-member requests (mean
    args.rate per second), each an instance drawn from a pool of meshes sized as
    in the batched workload (N in {3,4,5,7}, 512..32768 elements), advancing
    k in {1, 5, 20} LSRK steps at dt = 0.01 s on device-resident state.  The
    engine admits by a 120 GB HBM budget with up to 256 members resident and
    advances the resident members by up to --round-steps steps per round
    (continuous batching), under the chosen round policy.
    Latency of a request: from its scheduled arrival to the moment its final
    state is in host memory.  Throughput: point x stage evaluations of all
    requests over the span from the first arrival to the last completion."""
    import torch
    rank, local, world = dist_setup("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1604_08501_gb300 import build as lib_build
    lib_build.build()
    out, plan = serving_results(rank, dev, world, args.precisions, args.rate, args.requests,
                                args.pool, args.budget_gb, args.round_steps, args.round_policy,
                                args.warmup)
    total = args.requests
    if rank == 0:
        head = args.precisions[0]
        line = {"metric": "serving GDOF/s (points x RK stages / s) with p50/p99 request latency",
                "value": out[head]["value"], "unit": UNIT, "n_gpus": world, "steps": total,
                "warmup": args.warmup, "ms_per_step": out[head]["span_s"] * 1e3 / total,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "mixed": "f32 (perturbation state)",
                          "mixed-tc": "f32 (perturbation state), TF32 split products",
                          "mixed-auto": "f32 (perturbation state)"}[head],
                "data": "synthetic",
                "config": {"workload": f"Poisson arrivals at {args.rate:g} req/s, {total} requests, "
                                       f"each one of {len(plan)} instances (N in {{3,4,5,7}}, "
                                       f"512..32768 elements, smooth velocities) advancing "
                                       f"k in {{1,5,20}} LSRK(5,4) "
                                       f"steps at dt = 0.01 s; budget {args.budget_gb} GB, "
                                       f"<= 256 members resident, rounds of up to "
                                       f"{args.round_steps} step(s), {args.round_policy} "
                                       f"round policy"},
                "latency_ms": out[head]["latency_ms"], "offered_gdofs": out[head]["offered_gdofs"],
                "late_pinned_allocations": out[head]["late_pinned_allocations"],
                "gpu_launches": out[head]["rounds"], "clocks": out[head]["clocks"],
                "precision": head, "variants": {k: v for k, v in out.items() if k != head}}
        print(json.dumps(line))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 300 single, 5 batched, 50 nq-sweep)")
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["numa", "reference"], default="numa")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the timed oracle sample (for profiling runs)")
    ap.add_argument("--no-e2e", action="store_true",
                    help="skip the host-buffer end-to-end leg (for profiling runs)")
    ap.add_argument("--no-error", action="store_true",
                    help="skip the comparison with the oracle (for profiling runs)")
    ap.add_argument("--no-batched", action="store_true",
                    help="single workload: skip the compact batched entry (for profiling runs)")
    ap.add_argument("--no-serving", action="store_true",
                    help="single workload: skip the compact serving entry (for profiling runs)")
    ap.add_argument("--shard", choices=["elements", "replicas"], default="elements",
                    help="under torchrun: share one mesh by contiguous element ranges (each "
                         "rank n^3 elements of an n x n x (n ranks) mesh), or evaluate a "
                         "replica of the n^3-element workload per rank")
    ap.add_argument("--n", type=int, default=32,
                    help="elements per axis; 32 is the timed workload, smaller is for ncu")
    ap.add_argument("--precision", default=None,
                    help="comma-separated precision modes; the first is the headline value "
                         "(default fp64,df64,mixed; batched: fp64,mixed)")
    ap.add_argument("--workload", choices=["single", "batched", "serving", "nq-sweep"],
                    default="single",
                    help="single: one evaluation of the 32^3-element N=7 mesh per step (the "
                         "benchmark); batched: the 64-instance LSRK batch; serving: a Poisson "
                         "request stream through the continuous-batching engine; nq-sweep: "
                         "the paper's Nq study at 3,538,944 points")
    ap.add_argument("--instances", type=int, default=64, help="batched: number of instances")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: mean arrivals per second")
    ap.add_argument("--requests", type=int, default=600, help="serving: requests per precision")
    ap.add_argument("--pool", type=int, default=16, help="serving: distinct instances drawn from")
    ap.add_argument("--budget-gb", type=int, default=120, help="serving: HBM budget of the states")
    ap.add_argument("--round-steps", type=int, default=4,
                    help="serving: steps per engine round at most (never past a completion)")
    ap.add_argument("--round-policy", choices=["lockstep", "per_member"], default="per_member",
                    help="serving: every member the same steps per round, or each its own")
    ap.add_argument("--orders", default="",
                    help="nq-sweep: comma-separated orders N to run (default 3,7,11,15); "
                         "batched: keep only the plan's instances of these orders")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.steps is None:   # a few minutes at most for each workload
        args.steps = {"single": 300, "batched": 5, "nq-sweep": 50, "serving": 300}[args.workload]
    if args.precision is None:
        args.precision = {"single": "fp64,df64,mixed,mixed-tc",
                          "nq-sweep": "fp64,df64,mixed"}.get(args.workload, "fp64,mixed")
    args.precisions = [p for p in args.precision.split(",") if p]
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "nq-sweep":
        return run_nq_sweep(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
