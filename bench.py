#!/usr/bin/env python
"""FP64 stiffness assembly benchmark on GB300: split 2D x 1D vs standard 3D quadrature.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lam|reference]

Workload (synthetic, seeded by construction): in-plane cubic B-spline on 64x64
elements of the unit square under the curved map x = xi + 0.05 sin(2 pi xi)
sin(2 pi eta), y = eta + 0.05 sin(2 pi eta) cos(2 pi xi); 48 plies
[0/45/-45/90]_6s of 0.001 with one quadratic C0 element each (97 thickness
functions); orthotropic ply E1=140, E2=E3=10, G12=G13=5, G23=3.4, nu12=nu13=0.3,
nu23=0.49; 1,306,299 DOFs, 723,661,785 stored nonzeros.

One step = one call of lam_assemble_split (thickness integrals, in-plane Gram
blocks, fused combine into the CSR values) into a resident device buffer, in
FP64 arithmetic (the plan's default LAM_ARITH_FP64); the pattern is built once
before timing. Every timed step is preceded by a 256 MiB device write that
flushes the 129 MB L2 (outside the step's events). The line also reports the
opt-in double-float arithmetic (its time and its largest difference from the
FP64 matrix), the standard path (lam_assemble_standard) on the same plan, the
end-to-end figure through lam_assemble_split_host (ply angles in from pinned
host memory, all values out to pinned host memory) with its breakdown and the
host link measured alone, the roofline of the dominant kernel from the
library's own event timing, SM clocks sampled during the timed regions, and the
CPU oracle (standard assembly with the CSR scatter, on every host core) timed
on a bounded sample.

Under torchrun (N > 1) every rank assembles its own replica of the workload
(weak scaling, no collective on the data path); the step time is the maximum
over ranks and `value` counts the nonzeros of all ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FP64 K nnz/s on 1 GB300: split 2D×1D vs standard 3D quadrature; HBM roofline %"
UNIT = "nnz/s"
FALLBACK_HBM_GBS = 6800.0
FP64_PEAK_TFLOPS = 1.25          # nominal FP64 rate of the part (vector = tensor on GB300)
L2_FLUSH_BYTES = 256 << 20


def workload_desc(args) -> str:
    return (f"curved plate, cubic B-spline {args.n_el}x{args.n_el}, {8 * args.repeats} plies "
            f"[0/45/-45/90]_{args.repeats}s, quadratic C0 per ply")


# ----------------------------------------------------------------------------- distributed helpers
def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), int(
        os.environ.get("WORLD_SIZE", "1"))


def dist_init(backend: str):
    import torch.distributed as dist
    rank, local, world = dist_env()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29517")
        dist.init_process_group(backend, rank=rank, world_size=world)
    return rank, local, world


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over all ranks (x itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(units_per_rank: int, world: int, seconds_max: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return units_per_rank * world / seconds_max


# ----------------------------------------------------------------------------- peaks and profiles
NOMINAL_HBM_GBS = 8000.0  # GB300 HBM3e, nominal (~8 TB/s)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_sha(kernel: str) -> str:
    """sha256 of the definitions (from the __global__ / __device__ line to the
    closing brace at column 0) of the named functions in lam_kernels.cu;
    `kernel` is one name or several separated by '+'."""
    text = open(os.path.join(ROOT, "paper_1905_05417_gb300", "csrc", "lam_kernels.cu")).read().splitlines()
    h = hashlib.sha256()
    for name in kernel.split("+"):
        start = next(i for i, ln in enumerate(text)
                     if ("__global__" in ln or "__device__" in ln) and f" {name}(" in ln)
        end = next(i for i in range(start, len(text)) if text[i] == "}")
        h.update("\n".join(text[start:end + 1]).encode())
    return h.hexdigest()


def recorded_traffic(summary: str, kernel: str, key: str = "traffic_bytes_per_launch"):
    """DRAM bytes per launch recorded (under `key`) by an ncu capture of
    `kernel`, if that kernel's source has not changed since; else None."""
    path = os.path.join(ROOT, "profiles", summary)
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"(?m)^" + key + r":\s*([0-9.eE+]+)", text)
    s = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    if not m or not s or s.group(1) != kernel_source_sha(kernel):
        return None
    return float(m.group(1))


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 100):
        self.index = gpu_index
        self.period = period_ms
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            # the raw samples go to LAM_BENCH_OUT (default: the system temporary folder)
            out_dir = os.environ.get("LAM_BENCH_OUT") or tempfile.gettempdir()
            self.path = os.path.join(out_dir, f"clocks_rank{dist_env()[0]}.csv")
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader",
                                          "-i", str(self.index), "-lms", str(self.period)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1].split()[0]))
                smax.append(float(f[2].split()[0]))
                power.append(float(f[3].split()[0]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        # samples "under load": power above the midpoint of the observed range
        cut = min(power) + 0.5 * (max(power) - min(power))
        loaded = [c for c, p in zip(sm, power) if p >= cut] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "samples_under_load": len(loaded), "power_w_max": max(power)}


def bind_host_to_gpu(local_rank: int) -> dict:
    """Pin this process to the CPUs next to the GPU (its PCI device's
    local_cpulist), so that pinned host buffers allocated afterwards sit in the
    memory nearest to it. Best effort: returns what was done."""
    try:
        q = subprocess.run(["nvidia-smi", "--query-gpu=pci.bus_id", "--format=csv,noheader", "-i",
                            str(gpu_index(local_rank))], capture_output=True, text=True, timeout=20)
        bus = q.stdout.strip().lower()
        dom, rest = bus.split(":", 1)
        bus = f"{int(dom, 16) & 0xffff:04x}:{rest}"
        base = f"/sys/bus/pci/devices/{bus}"
        cpulist = open(f"{base}/local_cpulist").read().strip()
        node = open(f"{base}/numa_node").read().strip()
        cpus = set()
        for part in cpulist.split(","):
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
        os.sched_setaffinity(0, cpus)
        return {"pci": bus, "numa_node": node, "cpus": cpulist}
    except Exception as e:  # no sysfs entry, no nvidia-smi, ...
        return {"binding": f"none ({type(e).__name__})"}


def gpu_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v.strip() for v in vis.split(",") if v.strip()]
    if ids and all(v.isdigit() for v in ids) and local_rank < len(ids):
        return int(ids[local_rank])
    return local_rank


# ----------------------------------------------------------------------------- CPU oracle legs
def config_dict(args, n_dof: int, nnz: int) -> dict:
    """The workload, identical for both arms."""
    return {"workload": workload_desc(args), "n_dof": n_dof, "nnz": nnz,
            "l2": "256 MiB device write before every timed GPU step (L2 is 129 MB); outputs 5.8 GB per step"}


def oracle_threaded(lam, budget_s: float, nnz: int, prepared=None, threads: int | None = None):
    """CPU baseline: the oracle's standard assembly (element stiffness of
    Section 2.4, Eq. Km_0, plus the scatter into its own CSR) on the host's
    cores. Element colours (elements sharing no basis function) run one after
    another, each split over `threads` threads (the C calls release the GIL).
    A bounded sample of the workload -- whole colours, the last one cut short,
    about budget_s seconds -- is timed and scaled by the element count; the
    pattern is built once before timing. Plain C, not tuned for speed."""
    import numpy as np
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    threads = threads or os.cpu_count() or 1
    if prepared is None:
        prob = oracle.Problem(lam)
        row_ptr, col = oracle.pattern(lam)
        prepared = (prob, row_ptr, col, np.zeros(len(col)), oracle.element_colours(lam))
    prob, row_ptr, col, val, groups = prepared
    n_el = sum(len(g) for g in groups)
    t0 = time.perf_counter()
    oracle.assemble_elements(lam, row_ptr, col, groups[0][:1], val, prob)
    one = max(time.perf_counter() - t0, 1e-6)
    want = int(max(threads, min(n_el, budget_s * threads / one)))
    done = 0
    with ThreadPoolExecutor(threads) as ex:
        t0 = time.perf_counter()
        for g in groups:
            g = g[:want - done]
            if len(g) == 0:
                break
            list(ex.map(lambda c: oracle.assemble_elements(lam, row_ptr, col, c, val, prob),
                        [c for c in np.array_split(g, threads) if len(c)]))
            done += len(g)
        dt = time.perf_counter() - t0
    full = dt / done * n_el
    return {"value": nnz / full, "unit": UNIT, "cores": threads, "kind": "oracle",
            "nproc": os.cpu_count(),
            "sample": f"oracle standard assembly (element stiffness + CSR scatter) of {done} of {n_el} 3D elements "
                      f"(whole element colours in order), {dt:.1f} s on {threads} threads, scaled by the element count",
            "seconds_full_estimate": full}, prepared


def run_reference(args):
    rank, local, world = dist_env()
    if rank != 0:
        return 0
    import oracle
    lam = make_workload(args)
    n_dof, nnz = oracle.sizes(lam)
    budget = max(0.5, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    prepared = None
    for _ in range(args.warmup):
        _, prepared = oracle_threaded(lam, budget, nnz, prepared)
    vals = []
    for _ in range(args.steps):
        v, prepared = oracle_threaded(lam, budget, nnz, prepared)
        vals.append(v)
    secs = [nnz / v["value"] for v in vals]
    value = nnz / statistics.mean(secs)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config_dict(args, n_dof, nnz), "parallelism": f"host threads ({vals[0]['cores']})",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": vals[0]["cores"], "nproc": vals[0]["nproc"],
                             "kind": "oracle", "sample": vals[0]["sample"] + "; one such sample per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm
def standard_flops_per_step(info, lam):
    """FP64 flops of the standard kernel's algorithm: per 3D element piece, for
    every unordered pair of its (p+1)^2 (q+1) functions, (p+1)^2 (q+1) points x
    (9 FMA + 6 MUL) and the 81-FMA contraction with D."""
    nl = (lam.u.degree + 1) * (lam.v.degree + 1) * (lam.t.degree + 1)
    nq = (lam.u.degree + 1) * (lam.v.degree + 1) * (lam.t.degree + 1)
    pairs = nl * (nl + 1) // 2
    per_piece = pairs * (nq * (9 * 2 + 6) + 81 * 2)
    n_inplane = (len(set(lam.u.knots)) - 1) * (len(set(lam.v.knots)) - 1)
    return per_piece * info["n_pieces"] * n_inplane


def make_workload(args):
    import workloads as W
    return W.curved_plate(n_el=args.n_el, degree=3, repeats=args.repeats)


def run_adjoint(args, L, dev, flush, peak, peak_kind, world):
    """Gradient of L = sum(gbar * K) in the 21 constants and 24 ply angles of
    the 32 x 32 cubic [0/90]_12 plate (94.3 M stored entries), gbar ~ N(0, 1)
    on K's pattern from a seeded generator. Times lam_adjoint (Gram blocks,
    contraction, chain rule) and, beside it, the split assembly of the same plate."""
    import torch
    import workloads as W
    lam = W.adjoint_plate()
    plan = L.Plan.from_laminate(lam)
    nnz, nnz_s = plan.nnz, plan.info["nnz_inplane"]
    gen = torch.Generator(device=dev).manual_seed(1905)
    g = torch.randn(nnz, dtype=torch.float64, device=dev, generator=gen)
    vals = torch.empty(nnz, dtype=torch.float64, device=dev)

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        barrier()
        plan.profile_enable(True)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            evs[k][0].record()
            fn()
            evs[k][1].record()
        torch.cuda.synchronize()
        barrier()
        pr = plan.profile()
        plan.profile_enable(False)
        return max_over_ranks(sum(a.elapsed_time(b) for a, b in evs) / steps, dev), pr

    steps = args.adjoint_steps
    u = torch.randn(1, plan.n_dof, dtype=torch.float64, device=dev, generator=gen)
    ms_lr, _ = timed(lambda: plan.adjoint(u=u, v=u, want_dD=False), steps)
    ms, pr = timed(lambda: plan.adjoint(values=g, want_dD=False), steps)
    ms_fwd, _ = timed(lambda: plan.assemble_split(vals), steps)
    ms_df, prd = timed(lambda: plan.adjoint(values=g, want_dD=False, double_float=True), steps)
    k = pr["adjoint"]
    k_ms = k["ms"] / k["launches"]
    k_bytes = 8 * nnz + 8 * 9 * nnz_s
    # FP64 work of the contraction: 4 fused multiply-adds per cotangent entry (the
    # thickness sums of the four Q types, each entry counted once) and 81 per
    # (in-plane pair entry, ply) (S += z G)
    k_flops = 2 * (4 * nnz + 81 * nnz_s * len(lam.ply_angle))
    kd = prd["adjoint"]
    kd_ms = kd["ms"] / kd["launches"]
    out = {"workload": "adjoint plate: cubic B-spline 32x32 unit square, [0/90]_12 (24 plies x 0.0025), "
                       "CSR cotangent N(0,1) (torch seed 1905), outputs dL/dC (21) and dL/dtheta (24)",
           "metric": "cotangent entries contracted per second", "value": aggregate_throughput(nnz, world, ms / 1e3),
           "unit": UNIT, "ms_per_step": ms, "steps": steps, "nnz": nnz,
           "split_assembly_ms_same_plate": ms_fwd, "adjoint_over_assembly": ms / ms_fwd,
           "compliance_gradient_ms": ms_lr,
           "compliance_gradient": "L = u^T K u, u ~ N(0,1) per DOF (torch seed 1905): the low-rank cotangent u u^T",
           "arith": "FP64 (default)",
           "kernels_ms_per_step": {kk: pr[kk]["ms"] / steps for kk in L.KERNEL_KINDS if pr[kk]["launches"]},
           "gpu_launches": sum(pr[kk]["launches"] for kk in L.KERNEL_KINDS) // steps,
           "roofline": {"bound": "alu", "achieved": k_flops / (k_ms / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                        "unit": "TFLOP/s", "frac": k_flops / (k_ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
                        "traffic": None, "kernel": "adj_ply (FP64 CSR contraction)", "flops_per_launch": k_flops,
                        "ms_per_launch": k_ms, "hbm_frac": k_bytes / (k_ms / 1e3) / 1e9 / peak,
                        "peak_kind": "nominal FP64 rate (1.20 TFLOP/s measured by a DFMA probe)"},
           "double_float": {"ms_per_step": ms_df, "value": aggregate_throughput(nnz, world, ms_df / 1e3),
                            "arith": "double-float products on the FP32 pipes (LAM_ADJOINT_DOUBLE_FLOAT, opt-in)",
                            "roofline": {"bound": "hbm", "achieved": k_bytes / (kd_ms / 1e3) / 1e9, "peak": peak,
                                         "unit": "GB/s", "frac": k_bytes / (kd_ms / 1e3) / 1e9 / peak,
                                         "traffic": recorded_traffic("adj_ply_df_adjoint_plate_p3_32x32_24plies.md",
                                                                     "adj_ply_df"),
                                         "kernel": "adj_ply_df", "bytes_per_launch": k_bytes, "ms_per_launch": kd_ms,
                                         "peak_kind": f"{peak_kind} copy bandwidth"}}}
    plan.close()
    # the same plate as a general extrusion (lifted onto a bump, tilted a): FP64 contraction
    shell = L.Plan.from_laminate(W.laminate("adjoint_shell", W.BSPLINE, 3, 32, [math.degrees(x) for x in lam.ply_angle],
                                            0.0025, mapping=W.bump_map(0.05, inner=W.identity_map),
                                            extrusion=(0.05, -0.03, 1.0)))
    if shell.nnz == nnz:
        plan = shell
        ms_sh, _ = timed(lambda: shell.adjoint(values=g, want_dD=False), max(2, steps // 4))
        out["shell"] = {"workload": "the same plate lifted onto z = 0.05 sin(pi xi) sin(pi eta), extruded along "
                                    "a = (0.05, -0.03, 1) (general extrusion: FP64 contraction over 6x6 Gram blocks)",
                        "ms_per_step": ms_sh, "value": aggregate_throughput(nnz, world, ms_sh / 1e3), "unit": UNIT}
    shell.close()
    del g, vals
    torch.cuda.empty_cache()
    return out


def batch_combine_flops(plans) -> int:
    """FP64 flops of the batch combine (monoclinic FP64 rows): per in-plane pair,
    the slices' fused multiply-adds, 2 for each source term of an entry's kind
    (5 block-kind and 4 off-kind entries of the 3 x 3 block), and P of every
    configuration once per row (23 fused multiply-adds and 18 multiplies over the
    9 entries). Matches ncu's DFMA and DMUL counts of the kernel exactly."""
    total = 0
    for p in plans:
        i = p.info
        blk = i["combine_block_terms"]
        off = i["combine_source_terms"] - blk
        total += i["nnz_inplane"] * (2 * (5 * 2 * blk + 4 * 2 * off) + 64 * i["n_configs"])
    return total


def run_batch(args, L, dev, flush, peak, peak_kind, world):
    """The 256 seeded laminates (quadratic meshes 16..48 squared, 8..64 plies of
    uneven thickness, 1..4 materials; 1.9e10 stored entries, 155 GB of values)
    assembled by one lam_batch_assemble per step, and the same plans one by one
    with lam_assemble_split for comparison."""
    import torch
    import workloads as W
    lams = W.batch_laminates(count=args.batch_n)
    plans = [L.Plan.from_laminate(l) for l in lams]
    nnz = sum(p.nnz for p in plans)
    values = [torch.empty(p.nnz, dtype=torch.float64, device=dev) for p in plans]
    batch = L.Batch(plans)
    batch.assemble(values)  # tunes and captures the graph
    for _ in range(args.warmup):
        batch.assemble(values)
    torch.cuda.synchronize()
    barrier()
    steps = args.batch_steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        evs[k][0].record()
        batch.assemble(values)
        evs[k][1].record()
    torch.cuda.synchronize()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs) / steps, dev)
    # the same plans one by one (lam_assemble_split per plan), one timed pass
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.zero_()
    a.record()
    for p, v in zip(plans, values):
        p.assemble_split(v)
    b.record()
    torch.cuda.synchronize()
    seq_ms = a.elapsed_time(b)
    info = batch.info
    achieved = 8 * nnz / (ms / 1e3) / 1e9
    flops = batch_combine_flops(plans)
    out = {"workload": f"{args.batch_n} laminates from default_rng(517): quadratic B-spline meshes {{16,24,32,48}}^2 "
                       "on the unit square, 8..64 plies of thickness U[0.0005, 0.002], angles {0, +-45, 90}, "
                       "1..4 materials",
           "metric": "stored entries assembled per second", "value": aggregate_throughput(nnz, world, ms / 1e3),
           "unit": UNIT, "ms_per_step": ms, "steps": steps, "nnz_total": nnz, "n_plans": len(plans),
           "n_meshes": info["n_meshes"], "n_persistent": info["n_persistent"],
           "autotuner": {"axes": {"chunk_ctas": [4, 3, 2], "rows_per_item": [1, 2, 4], "ctas_per_sm": [1, 2, 3, 4]},
                         "chosen": {"chunk_ctas": info["chunk_ctas"], "rows_per_item": info["rows_per_item"],
                                    "ctas_per_sm": info["ctas_per_sm"]},
                         "ms": {f"h{h}/r{r}/c{c}": round(info["tuned_ms"][(hi * 3 + ri) * 4 + c - 1], 3)
                                for hi, h in enumerate((4, 3, 2)) for ri, r in enumerate((1, 2, 4))
                                for c in range(1, 5) if info["tuned_ms"][(hi * 3 + ri) * 4 + c - 1] > 0}},
           "cuda_graph": bool(info["graph"]),
           "one_plan_at_a_time_ms": seq_ms, "speedup_vs_one_at_a_time": seq_ms / ms,
           "roofline": {"bound": "alu", "achieved": flops / (ms / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                        "unit": "TFLOP/s", "frac": flops / (ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS, "traffic": None,
                        "kernel": "kc_batch (FP64 slices and P of every row; time of the whole batch call)",
                        "flops_per_step": flops,
                        "peak_kind": "nominal FP64 rate (1.20 TFLOP/s measured by a DFMA probe)",
                        "hbm_frac": achieved / peak, "hbm_achieved_gbs": achieved,
                        "hbm_peak_kind": f"{peak_kind} copy bandwidth"}}
    batch.close()
    for p in plans:
        p.close()
    del values
    torch.cuda.empty_cache()
    return out


def run_sweep(args):
    """The shape of the paper's experiment (Section 4, Figs. res1-res3): Pagano
    plate, one element of degree p through the thickness, p = 1..4, m = 1..64
    layers stacked 0/90/... and 0/45/-45/90/..., n x n in-plane elements.
    Prints one JSON line: split and standard assembly times per point and,
    per (p, stack), the ratio of the m = 64 and m = 8 times (the paper: split
    flat in m once m exceeds the number of configurations, standard linear)."""
    import torch
    import paper_1905_05417_gb300 as L
    import workloads as W
    torch.cuda.set_device(0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    layers = [1, 2, 4, 8, 16, 32, 64]
    points = []

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(sorted(ts)[len(ts) // 2])

    for p in (1, 2, 3, 4):
        for stack in ("cross", "quasi"):
            for m in layers:
                lam = W.pagano_sweep_plate(p, args.sweep_n, m, stack)
                plan = L.Plan.from_laminate(lam)
                v = torch.empty(plan.nnz, dtype=torch.float64, device="cuda")
                split_ms = timed(lambda: plan.assemble_split(v), 10)
                std_ms = timed(lambda: plan.assemble_standard(v), 3 if p < 4 else 1) if args.sweep_standard else None
                points.append({"p": p, "stack": stack, "layers": m, "nnz": plan.nnz,
                               "configs": plan.info["n_configs"], "split_ms": split_ms, "standard_ms": std_ms,
                               "speedup": None if std_ms is None else std_ms / split_ms})
                plan.close()
                del v
    shape = {}
    for p in (1, 2, 3, 4):
        for stack in ("cross", "quasi"):
            sel = {q["layers"]: q for q in points if q["p"] == p and q["stack"] == stack}
            shape[f"p{p}_{stack}"] = {"split_t64_over_t8": sel[64]["split_ms"] / sel[8]["split_ms"],
                                      "standard_t64_over_t8": (None if sel[8]["standard_ms"] is None else
                                                               sel[64]["standard_ms"] / sel[8]["standard_ms"]),
                                      "speedup_at_64": sel[64]["speedup"]}
    print(json.dumps({"sweep": "pagano_one_element_through_thickness", "n_el": args.sweep_n, "dtype": "f64",
                      "data": "synthetic", "points": points, "shape": shape}), flush=True)
    return 0


def run_large(args, L, dev, flush, peak, peak_kind, world):
    """The Lagrange Q2 96 x 96 plate with 64 plies [0/90]_32 (14.4 M DOFs,
    2.73e9 stored entries, 21.8 GB of values, int64 row pointers): split and
    standard assembly (--large-n-el sets the in-plane elements per direction)."""
    import torch
    import workloads as W
    n_el = args.large_n_el
    lam = W.lagrange_plate(n_el=n_el)
    plan = L.Plan.from_laminate(lam)
    nnz = plan.nnz
    values = torch.empty(nnz, dtype=torch.float64, device=dev)
    for _ in range(args.warmup):
        plan.assemble_split(values)
    torch.cuda.synchronize()
    barrier()
    steps = args.large_steps
    plan.profile_enable(True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        evs[k][0].record()
        plan.assemble_split(values)
        evs[k][1].record()
    torch.cuda.synchronize()
    pr = plan.profile()
    plan.profile_enable(False)
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs) / steps, dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.zero_()
    a.record()
    plan.assemble_standard(values)
    b.record()
    torch.cuda.synchronize()
    std_ms = a.elapsed_time(b)
    kc_ms = pr["combine"]["ms"] / steps
    kc_bytes = 8 * nnz + 72 * plan.info["nnz_inplane"]
    traffic = (recorded_traffic("kc_ws_lagrange_q2_96x96_64plies.md", "kcw_copy_pairs+kc_ws")
               if n_el == 96 else None)
    out = {"workload": f"Lagrange Q2 {n_el}x{n_el} unit square, [0/90]_32 (64 plies), Lagrange thickness",
           "value": aggregate_throughput(nnz, world, ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
           "nnz": nnz, "step_hbm_frac": 8 * nnz / (ms / 1e3) / 1e9 / peak,
           "kernels_ms_per_step": {k: pr[k]["ms"] / steps for k in L.KERNEL_KINDS if pr[k]["launches"]},
           "standard_ms": std_ms, "speedup_split_vs_standard": std_ms / ms,
           "roofline": {"bound": "hbm", "achieved": kc_bytes / (kc_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                        "frac": kc_bytes / (kc_ms / 1e3) / 1e9 / peak, "traffic": traffic, "kernel": "kc_ws",
                        "bytes_per_launch": kc_bytes, "peak_kind": f"{peak_kind} copy bandwidth"}}
    plan.close()
    del values
    torch.cuda.empty_cache()
    return out


def run_shell(args, L, dev, flush, peak, peak_kind, world):
    """A general extrusion (Eq. extrusion) of the benchmark's size: the curved
    plate's map lifted onto z = 0.05 sin(pi xi) sin(pi eta), extruded along
    a = (0.05, -0.03, 1), cubic 64 x 64, 48 plies. Split (6 x 6 Gram blocks, P
    per configuration, the combine) and one standard assembly."""
    import torch
    import workloads as W
    lam = W.shell_plate(n_el=args.shell_n_el)
    plan = L.Plan.from_laminate(lam)
    nnz = plan.nnz
    values = torch.empty(nnz, dtype=torch.float64, device=dev)
    for _ in range(args.warmup):
        plan.assemble_split(values)
    torch.cuda.synchronize()
    barrier()
    steps = args.shell_steps
    plan.profile_enable(True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        evs[k][0].record()
        plan.assemble_split(values)
        evs[k][1].record()
    torch.cuda.synchronize()
    pr = plan.profile()
    plan.profile_enable(False)
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs) / steps, dev)
    std_ms = None
    if args.standard_steps > 0:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        a.record()
        plan.assemble_standard(values)
        b.record()
        torch.cuda.synchronize()
        std_ms = a.elapsed_time(b)
    kc_ms = pr["combine"]["ms"] / steps
    # the combine writes K and reads P of every configuration (36 doubles per pair and configuration)
    kc_bytes = 8 * nnz + 8 * 36 * plan.info["nnz_inplane"] * plan.info["n_configs"]
    traffic = (recorded_traffic("kc_ws_curved_p3_64x64_48plies.md", "kcw_copy_pairs+kc_ws",
                                "shell_traffic_bytes_per_launch") if args.shell_n_el == 64 else None)
    out = {"workload": "curved shell: the curved plate's map on the surface z = 0.05 sin(pi xi) sin(pi eta), "
                       f"extruded along a = (0.05, -0.03, 1), cubic B-spline {args.shell_n_el}x{args.shell_n_el}, "
                       "48 plies [0/45/-45/90]_6s",
           "value": aggregate_throughput(nnz, world, ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
           "nnz": nnz, "step_hbm_frac": 8 * nnz / (ms / 1e3) / 1e9 / peak,
           "kernels_ms_per_step": {k: pr[k]["ms"] / steps for k in L.KERNEL_KINDS if pr[k]["launches"]},
           "standard_ms": std_ms, "speedup_split_vs_standard": None if std_ms is None else std_ms / ms,
           "roofline": {"bound": "hbm", "achieved": kc_bytes / (kc_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                        "frac": kc_bytes / (kc_ms / 1e3) / 1e9 / peak, "traffic": traffic, "kernel": "kc_ws",
                        "bytes_per_launch": kc_bytes, "peak_kind": f"{peak_kind} copy bandwidth"}}
    plan.close()
    del values
    torch.cuda.empty_cache()
    return out


def run_lam(args):
    import torch
    rank, local, world = dist_init("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1905_05417_gb300 as L
    lam = make_workload(args)
    plan = L.Plan.from_laminate(lam)  # FP64 arithmetic (LAM_ARITH_FP64, the default)
    assert plan.info["arith"] == L.ARITH_FP64
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, prepared = oracle_threaded(lam, args.cpu_budget, plan.nnz)
        del prepared
    info = plan.info
    nnz, nnz_s = info["nnz"], info["nnz_inplane"]
    row_ptr, col = plan.pattern()
    values = torch.empty(nnz, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        plan.assemble_split(values)
    torch.cuda.synchronize()
    peak, peak_kind = measured_peaks()

    with ClockSampler(gpu_index(local)) as clocks:
        # ---- split, timed
        barrier()
        torch.cuda.synchronize()
        plan.profile_enable(True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record()
            plan.assemble_split(values)
            ev[k][1].record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        barrier()
        prof = plan.profile()
        plan.profile_enable(False)
        step_ms = [a.elapsed_time(b) for a, b in ev]
        ms_local = sum(step_ms) / args.steps
        ms = max_over_ranks(ms_local, dev)
        launches = sum(prof[k]["launches"] for k in L.KERNEL_KINDS)

        # ---- the double-float variant (LAM_ARITH_DOUBLE_FLOAT, opt-in), against the FP64 result
        dfl = None
        if args.df_steps > 0:
            dplan = L.Plan.from_laminate(lam, arith=L.ARITH_DOUBLE_FLOAT)
            dvals = torch.empty(nnz, dtype=torch.float64, device=dev)
            for _ in range(args.warmup):
                dplan.assemble_split(dvals)
            torch.cuda.synchronize()
            barrier()
            dplan.profile_enable(True)
            dev_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(args.df_steps)]
            for k in range(args.df_steps):
                flush.zero_()
                dev_ev[k][0].record()
                dplan.assemble_split(dvals)
                dev_ev[k][1].record()
            torch.cuda.synchronize()
            dprof = dplan.profile()
            dms = max_over_ranks(sum(a.elapsed_time(b) for a, b in dev_ev) / args.df_steps, dev)
            rel = float((dvals - values).abs().max() / values.abs().max())
            dfl = {"value": aggregate_throughput(nnz, world, dms / 1e3), "unit": UNIT, "ms_per_step": dms,
                   "steps": args.df_steps, "arith": "double-float products and sums on the FP32 pipes (opt-in)",
                   "max_abs_diff_over_max_abs_vs_fp64": rel,
                   "kernels_ms_per_step": {k: dprof[k]["ms"] / args.df_steps for k in L.KERNEL_KINDS
                                           if dprof[k]["launches"]}}
            dplan.close()
            del dvals
            torch.cuda.empty_cache()

        # ---- standard, timed on the same plan
        std = None
        if args.standard_steps > 0:
            std_vals = values  # same buffer: the split result is not needed any more
            for _ in range(args.standard_warmup):
                plan.assemble_standard(std_vals)
            torch.cuda.synchronize()
            barrier()
            plan.profile_enable(True)
            sev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.standard_steps)]
            for k in range(args.standard_steps):
                flush.zero_()
                sev[k][0].record()
                plan.assemble_standard(std_vals)
                sev[k][1].record()
            torch.cuda.synchronize()
            barrier()
            sprof = plan.profile()
            plan.profile_enable(False)
            sms = max_over_ranks(sum(a.elapsed_time(b) for a, b in sev) / args.standard_steps, dev)
            flops = standard_flops_per_step(info, lam)
            k_ms = sprof["standard"]["ms"] / args.standard_steps
            std = {"value": aggregate_throughput(nnz, world, sms / 1e3), "unit": UNIT, "ms_per_step": sms,
                   "steps": args.standard_steps, "warmup": args.standard_warmup,
                   "roofline": {"bound": "alu", "achieved": flops / (k_ms / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                                "unit": "TFLOP/s", "frac": flops / (k_ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
                                "traffic": None, "flops_per_step": flops,
                                "peak_kind": "nominal FP64 rate (1.20 TFLOP/s measured by a DFMA probe)"},
                   "gpu_launches": sum(sprof[k]["launches"] for k in L.KERNEL_KINDS)}

    # ---- the large Lagrange plate
    large = run_large(args, L, dev, flush, peak, peak_kind, world) if args.large_steps > 0 else None
    shell = run_shell(args, L, dev, flush, peak, peak_kind, world) if args.shell_steps > 0 else None

    # ---- batch (lam_batch_*) of 256 seeded laminates
    batch = run_batch(args, L, dev, flush, peak, peak_kind, world) if args.batch_steps > 0 else None

    # ---- adjoint (lam_adjoint) on the 32 x 32 cubic 24-ply plate, CSR cotangent
    adj = run_adjoint(args, L, dev, flush, peak, peak_kind, world) if args.adjoint_steps > 0 else None

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if args.e2e_steps > 0:
        binding = bind_host_to_gpu(local)
        host = torch.empty(nnz, dtype=torch.float64, pin_memory=True)
        angles = torch.tensor(lam.ply_angle, dtype=torch.float64).pin_memory()
        plan.update(ply_angle=angles.numpy())
        plan.assemble_split_host(host)
        # the host link on its own: a plain copy of the same bytes into the same pinned buffer
        link = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            host.copy_(values, non_blocking=True)
            b.record()
            torch.cuda.synchronize()
            link.append(a.elapsed_time(b))
        link_gbs = 8 * nnz / (statistics.median(link) / 1e3) / 1e9
        torch.cuda.synchronize()
        barrier()
        plan.profile_enable(True)
        upd, asm = [], []
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            ta = time.perf_counter()
            plan.update(ply_angle=angles.numpy())
            tb = time.perf_counter()
            plan.assemble_split_host(host)
            tc = time.perf_counter()
            upd.append(tb - ta)
            asm.append(tc - tb)
        t_e2e = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, dev)
        eprof = plan.profile()
        plan.profile_enable(False)
        barrier()
        d2h = eprof["d2h_bytes"] // args.e2e_steps
        e2e = {"value": aggregate_throughput(nnz, world, t_e2e), "unit": UNIT,
               "h2d_bytes_per_step": eprof["h2d_bytes"] // args.e2e_steps + angles.numel() * 8,
               "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * t_e2e, "steps": args.e2e_steps,
               "call": "lam_plan_update (ply angles from pinned host memory) + lam_assemble_split_host "
                       "(values to pinned host memory)",
               "breakdown_ms_per_step": {
                   "plan_update_host": 1e3 * statistics.mean(upd),
                   "assemble_split_host": 1e3 * statistics.mean(asm),
                   "kernels": {k: eprof[k]["ms"] / args.e2e_steps for k in L.KERNEL_KINDS if eprof[k]["launches"]}},
               "d2h_gbs": d2h / statistics.mean(asm) / 1e9,
               "link_gbs": link_gbs, "link_bound_ms": 8 * nnz / link_gbs / 1e6,
               "over_link_bound": t_e2e / (8 * nnz / link_gbs / 1e9),
               "host_binding": binding}
        del host

    if rank != 0:
        return 0
    kc = prof["combine"]
    kc_ms = kc["ms"] / kc["launches"]  # kc_ws: one launch per step
    kc_bytes = 8 * nnz + 72 * nnz_s     # 8 B per stored value + the row's assembled Gram blocks (9 doubles per pair)
    achieved = kc_bytes / (kc_ms / 1e3) / 1e9
    traffic = (recorded_traffic("kc_ws_curved_p3_64x64_48plies.md", "kcw_copy_pairs+kc_ws")
               if (args.n_el, args.repeats) == (64, 6) else None)
    clk = clocks.summary()
    line = {
        "metric": METRIC,
        "value": aggregate_throughput(nnz, world, ms / 1e3),
        "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "arith": "FP64 (every product and sum an FP64 operation: LAM_ARITH_FP64)", "data": "synthetic",
        "config": config_dict(args, info["n_dof"], nnz),
        "parallelism": "replicas" if world > 1 else "single GPU",
        "plan": {"n_configs": info["n_configs"], "n_classes": info["n_classes"]},
        "step_ms_stats": {"median": statistics.median(step_ms), "min": min(step_ms), "max": max(step_ms),
                          "note": "this rank's timed steps; ms_per_step is their mean (max over ranks)"},
        "step_hbm_frac": 8 * nnz / (ms / 1e3) / 1e9 / peak,
        "step_hbm_frac_of_nominal": {"peak_gbs": NOMINAL_HBM_GBS, "frac": 8 * nnz / (ms / 1e3) / 1e9 / NOMINAL_HBM_GBS},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "kernel": "kc_ws", "bytes_per_launch": kc_bytes,
                     "ms_per_launch": kc_ms, "launches_per_call": kc["launches"] // args.steps,
                     "peak_kind": f"{peak_kind} copy bandwidth"},
        "kernels_ms_per_step": {k: prof[k]["ms"] / args.steps for k in L.KERNEL_KINDS if prof[k]["launches"]},
        "gpu_launches": launches,
        "wall_s_timed": wall,
        "clocks": clk,
    }
    if dfl is not None:
        line["double_float"] = dfl
    if std is not None:
        line["standard"] = std
        line["speedup_split_vs_standard"] = std["ms_per_step"] / ms
    if e2e is not None:
        line["e2e"] = e2e
    if adj is not None:
        line["adjoint"] = adj
    if batch is not None:
        line["batch"] = batch
    if large is not None:
        line["large"] = large
    if shell is not None:
        line["shell"] = shell
    if cpu is not None:
        line["cpu_baseline"] = {k: cpu[k] for k in ("value", "unit", "cores", "nproc", "kind", "sample")}
    print(json.dumps(line), flush=True)
    plan.close()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("lam", "reference"), default="lam")
    ap.add_argument("--standard-steps", type=int, default=2)
    ap.add_argument("--standard-warmup", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--df-steps", type=int, default=20, help="timed double-float assemblies (0 = skip)")
    ap.add_argument("--adjoint-steps", type=int, default=20, help="timed lam_adjoint calls (0 = skip)")
    ap.add_argument("--batch-steps", type=int, default=5, help="timed lam_batch_assemble calls (0 = skip)")
    ap.add_argument("--large-steps", type=int, default=5, help="timed split assemblies of the Lagrange plate (0 = skip)")
    ap.add_argument("--large-n-el", type=int, default=96, help="in-plane elements per direction of the Lagrange plate")
    ap.add_argument("--batch-n", type=int, default=256, help="laminates in the batch (the first n of the seeded 256)")
    ap.add_argument("--shell-n-el", type=int, default=64, help="in-plane elements per direction of the curved shell")
    ap.add_argument("--shell-steps", type=int, default=5, help="timed split assemblies of the curved shell (0 = skip)")
    ap.add_argument("--sweep", action="store_true", help="the paper's layer sweep (one element through the thickness)")
    ap.add_argument("--sweep-n", type=int, default=16, help="in-plane elements per direction in the sweep")
    ap.add_argument("--sweep-no-standard", dest="sweep_standard", action="store_false",
                    help="time only the split path in the sweep")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--n-el", type=int, default=64, help="in-plane elements per direction (64 = the benchmark)")
    ap.add_argument("--repeats", type=int, default=6, help="[0/45/-45/90]_{repeats}s stack (6 = 48 plies)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return run_sweep(args)
    return run_lam(args)


if __name__ == "__main__":
    sys.exit(main())
