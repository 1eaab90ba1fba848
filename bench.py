#!/usr/bin/env python3
"""Throughput of the G4 measurement step on one GB300 (or N independent replicas).

One step = one whole run of a workload through the public C ABI: reset the
FP64 accumulator, g4_compute_G for every measurement (G build + batch staging;
each full batch triggers the direct-term and exchange kernels), g4_finalize
(normalise by the sign sum, export transpose).  Inputs (M for every
measurement, G0, signs) are resident in HBM before the timed region; M totals
far more than the 129 MB L2, so no explicit flush is needed.

Printed JSON line: the metric of the G4 workload (element-updates/s = E*R/t),
the roofline of the dominant kernel (the exchange-type term: on tensor cores
bound by the HBM stream of its FP64 accumulator and operands, on CUDA cores by
the FP32 ALUs), the plain
FP64 per-measurement GPU path on the same problem dimensions for comparison,
an end-to-end number with host inputs, the same run fed from vertex
configurations (the transform to M before the path, with its own FP32 ALU
roofline), the oracle on the host cores, and the SM clocks sampled during the
timed region.

``--impl reference`` times the CPU oracle (the only reference this method
has) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
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

METRIC = "G4 element-updates/s, mixed vs FP64 plain on 1 GB300 at ≤2e-6 rel err; % roofline"
UNIT = "element-updates/s"
# FP32 ALU peak of one GB300: 152 SMs x 128 FP32 lanes x 2 flop/FMA x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_PEAK_TFLOPS = 1.25  # datasheet FP64 (non-tensor) rate of GB300, context only
TF32_PER_BF16 = 1.1 / 2.25  # nominal dense TF32 / BF16 tensor rate of GB300


def measured_peaks():
    """HBM GB/s and dense BF16 TFLOP/s measured on this machine (or the fallback)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0, "of fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c64_w64",
                    choices=["tiny_2x2", "c16_w64", "c36_w64", "group12", "c64_w64"])
    ap.add_argument("--m-pool", type=int, default=0,
                    help="distinct device M matrices cycled over the run (0 = the workload's "
                         "default: every measurement's own, one batch (128) for c64_w64)")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the error of the benched configuration against the oracle")
    ap.add_argument("--shards", type=int, default=0,
                    help="with N > 1 GPUs: transfer-frequency slabs per group (0 = the largest "
                         "divisor of N not above Nwex)")
    ap.add_argument("--sharded", action="store_true",
                    help="use the partitioned path even on one GPU (one slab, no collective)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-vertices", action="store_true",
                    help="skip the run fed from vertex configurations")
    ap.add_argument("--no-group", action="store_true",
                    help="skip the twelve-problem batching form in the default line")
    ap.add_argument("--measurements", type=int, default=0,
                    help="measurements per step (0 = the workload's own count)")
    ap.add_argument("--Nw", type=int, default=0,
                    help="positive frequencies of the grid (0 = the workload's own); for "
                         "small profiling cases of a workload's kernels")
    ap.add_argument("--Nwex", type=int, default=0,
                    help="bosonic transfers (0 = the workload's own); for profiling cases")
    ap.add_argument("--m-dtype", default="", choices=["", "c64", "c128"],
                    help="element type of M (default: the workload's own); for profiling cases")
    ap.add_argument("--transform-only", action="store_true",
                    help="with --stage vertices: time the transform to M alone (a handle of the "
                         "workload's cluster and grid with one transfer, under 1 GB)")
    ap.add_argument("--stage", default="m", choices=["m", "vertices"],
                    help="m: measurements enter as M (default); vertices: only the run fed "
                         "from vertex configurations, as the timed step")
    ap.add_argument("--channel", default="ph_magnetic",
                    choices=["ph_magnetic", "pp_updown", "ph_density", "ph_transverse"])
    ap.add_argument("--operands", default="fp16", choices=["fp16", "tf32"],
                    help="hi/lo operand pairs of the tensor-core GEMMs (mixed handle)")
    ap.add_argument("--accum", default="fp64", choices=["fp64", "f32pair"],
                    help="G4 accumulator: FP64, or compensated FP32 pairs")
    ap.add_argument("--staging", default="auto", choices=["auto", "deferred", "eager"],
                    help="deferred: the accumulation forms the operands from the staged M "
                         "(options.deferred); eager: g4_compute_G forms each G; auto: "
                         "deferred for complex64 M, eager for complex128 M (the faster on each)")
    return ap.parse_args()


CHANNEL_NAMES = {"ph_magnetic": "particle-hole magnetic", "pp_updown": "particle-particle up-down",
                 "ph_density": "particle-hole density", "ph_transverse": "particle-hole transverse"}


def workload_desc(p, name, channel="ph_magnetic"):
    return {
        "workload": "%s: Nc=%d (%dx%d), 2Nw=%d, Nwex=%d, Nkex=%d, beta=%g, R=%d, batch=%d"
                    % (name, p.Nc, p.Lx, p.Ly, p.Nw2, p.Nwex, p.Nkex, p.beta, p.R, p.batch),
        "channel": CHANNEL_NAMES[channel],
        "G4_entries": p.entries,
        "measurements": p.R,
        "batch": p.batch,
        "M_dtype": p.m_dtype,
    }


def bench_problem(args):
    """The workload, with its measurement count replaced by --measurements."""
    from paper_2105_00027_gb300 import inputs
    p = inputs.workload(args.workload)
    if args.measurements > 0:
        p = inputs.with_(p, R=args.measurements, batch=min(p.batch, args.measurements))
    if args.Nw > 0:
        p = inputs.with_(p, Nw=args.Nw)
    if args.Nwex > 0:
        p = inputs.with_(p, Nwex=args.Nwex)
    if args.m_dtype:
        p = inputs.with_(p, m_dtype=args.m_dtype)
    return p


# ---------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_id is not None:
            cmd += ["-i", str(gpu_id)]
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------- replicas
def replica_throughput(ms_local, units_local, world, device=None):
    """Whole-job figures of N independent replicas (one per GPU, each its own
    problem and seed, no data-path collective): the job's step time is the
    slowest rank's, its throughput every rank's units over that time.
    Returns (max step ms, total units, units/s); collective on N > 1."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    ms_max, units = float(t.item()), float(u.item())
    return ms_max, units, units / (ms_max / 1e3)


# ---------------------------------------------------------------- oracle
def oracle_sample(p, seed, n_meas=8, n_slabs=24, threads=0, channel="ph_magnetic"):
    """Time the CPU oracle on a bounded sample: n_meas measurements of the
    workload on n_slabs (q, m) slabs.  Returns (updates/s, sample text, cores)."""
    import numpy as np
    import oracle
    from paper_2105_00027_gb300 import inputs
    d = oracle.dims(p.Lx, p.Ly, p.Nw, p.Nwex, p.Nkex)
    qs, ms = oracle.all_slabs(d)
    pick = np.linspace(0, len(qs) - 1, n_slabs).astype(int)
    G0 = inputs.g0(p)
    s = inputs.signs(p, seed=seed)
    Ms = [inputs.measurement_M(p, r, seed=seed).numpy().astype(np.complex128) for r in range(n_meas)]
    oracle.load()
    t0 = time.perf_counter()
    oracle.run_stream(d, zip(Ms, s[:n_meas]), G0, qs[pick], ms[pick], nthreads=threads,
                      channel=channel)
    dt = time.perf_counter() - t0
    upd = n_meas * n_slabs * p.N * p.N
    cores = threads or os.cpu_count()
    return upd / dt, "%d measurements x %d (q,m) slabs of %d x %d (%.3g updates, %.1f s)" % (
        n_meas, n_slabs, p.N, p.N, upd, dt), cores


def cpu_model():
    """The host CPU's model name (lscpu or /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


# ---------------------------------------------------------------- accuracy
def accuracy_plan(p):
    """The prefix and slabs on which the benched configuration's error is
    measured: one full batch of the workload (its FP32 sums have the benched
    length) on the transfers (0, 0) and (Nkex-1, Nwex-1)."""
    R = min(p.R, p.batch)
    return R, [0, p.Nkex - 1], [0, p.Nwex - 1]


ACC_SEED = 1000


def _prefetched(fn, n, depth=3):
    """fn(0), ..., fn(n-1) in order, computed ahead by a small thread pool with
    at most `depth` results held (numpy's generators release the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(depth) as ex:
        futs = [ex.submit(fn, i) for i in range(min(depth, n))]
        for i in range(n):
            v = futs[i].result()
            futs[i] = None
            if i + depth < n:
                futs.append(ex.submit(fn, i + depth))
            yield v


def oracle_accuracy_ref(p, channel, threads):
    """The oracle's slabs for accuracy_plan(p) (run in a spawned process while
    the GPU legs run): (slabs, sign sum, seconds)."""
    import numpy as np
    import oracle
    from paper_2105_00027_gb300 import inputs
    R, qsel, msel = accuracy_plan(p)
    d = oracle.dims(p.Lx, p.Ly, p.Nw, p.Nwex, p.Nkex)
    s = inputs.signs(p, seed=ACC_SEED)[:R]
    oracle.load()
    t0 = time.perf_counter()
    gen = _prefetched(lambda r: inputs.measurement_M(p, r, seed=ACC_SEED).numpy().astype(np.complex128), R)
    ref, S = oracle.run_stream(d, zip(gen, s), inputs.g0(p), np.asarray(qsel, np.int32),
                               np.asarray(msel, np.int32), nthreads=threads, channel=channel)
    return ref, S, time.perf_counter() - t0


def start_oracle_accuracy(p, channel):
    """Spawn the oracle side of the accuracy check (before any CUDA call), on
    all host cores but two (one drives the GPU)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(1)
    threads = max(1, (os.cpu_count() or 4) - 2)
    return pool, pool.apply_async(oracle_accuracy_ref, (p, channel, threads))


def gpu_accuracy(p, dev, channel, out, pending, deferred=False):
    """The same prefix through a fresh handle of the benched configuration;
    the errors of Eqs. (2)-(3) against the oracle's slabs.  A deferred handle
    reads M when its batch accumulates: each batch's M stay on the device
    until then."""
    import numpy as np
    import torch
    import oracle
    from paper_2105_00027_gb300 import g4, inputs
    R, qsel, msel = accuracy_plan(p)
    pool, job = pending
    G0 = torch.from_numpy(inputs.g0(p)).to(dev)
    s = inputs.signs(p, seed=ACC_SEED)[:R]
    subs, times = {}, {}
    for accum in ("fp64", "f32pair"):
        # the benched configuration (FP64 accumulator) and the alternative of
        # compensated FP32 pairs, on the same measurements
        h = g4.G4.for_problem(p, precision="mixed", batch=p.batch, channel=channel, accum=accum,
                              deferred=deferred)
        h.profile(True)
        gen = _prefetched(lambda i: inputs.measurement_M(p, i, seed=ACC_SEED), R)
        held = []
        for r, M in enumerate(gen):
            Md = M.to(dev)
            h.compute_G(Md, G0, float(s[r]))
            if deferred:
                held.append(Md)
                if len(held) == p.batch:
                    h.accumulate()
                    held = []
        res, S = h.finalize(out)
        del held
        x_ms, x_n = h.profile_read("exchange")
        h.close()
        times[accum] = x_ms / max(1, math.ceil(R / p.batch))
        v = res.view(p.Nwex, p.Nw2, p.Nw2, p.Nkex, p.Nc, p.Nc)
        subs[accum] = np.stack([v[m, :, :, q].cpu().numpy() for q, m in zip(qsel, msel)])
        del v, res
    ref, Sref, secs = job.get(timeout=1800)
    pool.close()
    pool.join()
    err = oracle.errors(ref, subs["fp64"])
    alt = oracle.errors(ref, subs["f32pair"])
    return {"L2": err["L2"], "L1": err["L1"], "L2_re": err["L2_re"], "L2_im": err["L2_im"],
            "L1_re": err["L1_re"], "L1_im": err["L1_im"], "bound": 2e-6,
            "sign_sum_match": S == Sref,
            "sample": "%d measurements (one batch of %d), slabs (q,m) = %s, against the CPU "
                      "oracle (%.0f s)" % (R, p.batch, list(zip(qsel, msel)), secs),
            "accumulator": {"fp64": {"L2": err["L2"], "exchange_ms_per_batch": times["fp64"]},
                            "f32pair": {"L2": alt["L2"], "exchange_ms_per_batch": times["f32pair"]},
                            "chosen": "fp64"}}


# ---------------------------------------------------------------- roofline
# Source of each profiled kernel: the file, the markers around the kernel's
# code in it (its parameters, device helpers and the kernel), and the shared
# inline-PTX header.
KERNEL_SOURCES = {
    "exchange_tc": ("paper_2105_00027_gb300/csrc/g4_exchange_tc.cu",
                    "// ---------------------------------------------------------------- tensor-core kernel",
                    "// ---------------------------------------------------------------- host plan"),
}


def kernel_source_sha(kernel_key):
    """sha256 prefix of a kernel's source text (KERNEL_SOURCES), or None."""
    import hashlib
    ent = KERNEL_SOURCES.get(kernel_key)
    if ent is None:
        return None
    path, begin, end = ent
    try:
        text = open(os.path.join(ROOT, path)).read()
        ptx = open(os.path.join(ROOT, "paper_2105_00027_gb300/csrc/g4_ptx.cuh")).read()
    except OSError:
        return None
    a, b = text.find(begin), text.find(end)
    if a < 0 or b < a:
        return None
    return hashlib.sha256((text[a:b] + ptx).encode()).hexdigest()[:16]


def profiled_traffic(kernel_key):
    """DRAM bytes per G4 entry and batch measured by ncu for a kernel (a line
    'traffic <kernel_key> <bytes per entry per batch> <kernel_source_sha>' in a
    profiles/ summary), or None when no summary has it or the kernel's source
    has changed since the capture."""
    import glob
    sha = kernel_source_sha(kernel_key)
    if sha is None:
        return None
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            parts = line.strip().strip("`").split()
            if len(parts) == 4 and parts[0] == "traffic" and parts[1] == kernel_key:
                if parts[3] == sha:
                    return float(parts[2]), os.path.relpath(path, ROOT)
    return None


def roofline(p, prof, steps, nb_step, ms_step, operands="fp16"):
    """Roofline of the dominant kernel and of the whole step, on the
    algorithmic bytes of the accumulation: per batch of R_b measurements every
    G4 entry is read and written once in FP64 (32 B) and both spins' G are read
    once in complex64 (16 B per G entry pair), i.e. (32/R_b + 16/NQ) B per
    element-update.  Bytes the implementation adds (the hi/lo operand planes,
    the direct term's window and scratch) are reported beside it as overhead,
    not counted as work."""
    hbm_gbs, bf16_tf, peak_src = measured_peaks()
    E, Rb = p.entries, p.batch
    alg_batch = 32 * E + 16 * p.N * p.N * Rb
    per_step = {k: v[0] / steps for k, v in prof.items() if v[1]}
    dominant = max(per_step, key=per_step.get) if per_step else None
    x_ms, x_n = prof["exchange"]
    x_batch_ms = x_ms / (steps * nb_step)
    achieved = alg_batch / (x_batch_ms / 1e3) / 1e9
    path = alg_batch * nb_step / (ms_step / 1e3) / 1e9
    f16 = operands == "fp16"
    J = 2 * ((Rb + (63 if f16 else 31)) // (64 if f16 else 32) * (64 if f16 else 32))
    plane_b = 8 if f16 else 16      # hi + lo, both components, per G entry and K element
    tc_peak = bf16_tf if f16 else bf16_tf * TF32_PER_BF16
    flops = 16 * E * Rb
    tr = profiled_traffic("exchange_tc") if prof["pack_exchange"][1] else None
    return {
        "bound": "hbm", "kernel": "exchange (tensor cores)" if prof["pack_exchange"][1]
        else "exchange (CUDA cores)",
        "achieved": achieved, "peak": hbm_gbs, "unit": "GB/s", "frac": achieved / hbm_gbs,
        "traffic": tr[0] * E if tr else None,
        "traffic_source": tr[1] if tr else "no ncu capture of the current kernel source",
        "per": "batch of %d measurements (%d launches)" % (Rb, x_n // max(steps * nb_step, 1)),
        "algorithmic_bytes": alg_batch,
        "algorithmic_bytes_formula": "32 E + 16 N^2 R_b = (32/R_b + 16/NQ) B x E R_b",
        "ms": x_batch_ms,
        "peak_source": "hbm_gbs " + peak_src,
        "dominant_kernel_of_step": dominant,
        "path": {"achieved": path, "frac": path / hbm_gbs, "ms_per_step": ms_step,
                 "algorithmic_bytes_per_step": alg_batch * nb_step,
                 "note": "the same algorithmic bytes over the whole step (every kernel, "
                         "G build, finalize included)"},
        "overhead_bytes_per_batch": {
            "operand_planes_exchange": 2 * plane_b * J * p.N * p.N,
            "note": "%s hi/lo operand planes of the exchange, written by its pack and "
                    "read by the kernel (%d B per G entry and K element, twice); not "
                    "counted as algorithmic" % (operands.upper(), plane_b)},
        "tensor": {"achieved_tflops": flops / (x_batch_ms / 1e3) / 1e12, "peak_tflops": tc_peak,
                   "frac": flops / (x_batch_ms / 1e3) / 1e12 / tc_peak,
                   "useful_flops_per_batch": flops,
                   "executed_products": "3 per useful product (hi.hi + hi.lo + lo.hi)",
                   "peak_source": ("bf16_tflops %s (FP16 runs at the BF16 rate)" % peak_src.split()[1])
                   if f16 else "bf16_tflops %s x nominal TF32/BF16 %.3f" % (
                       peak_src.split()[1], TF32_PER_BF16)},
    }


# ---------------------------------------------------------------- ours
def default_pool(p, args):
    """Distinct device M matrices cycled over the run: every measurement's own,
    or for the largest grid one batch's worth (every slot of a batch reads a
    different M, so that no batch finds its inputs in L2)."""
    if args.m_pool:
        return args.m_pool
    return min(p.R, max(p.batch, 64)) if p.N >= 4096 else p.R


def staging_of(p, args):
    """The staging mode a run uses: --staging, with auto resolved by M's type."""
    if args.staging != "auto":
        return args.staging
    return "deferred" if p.m_dtype == "c64" else "eager"


def run_ours(args, rank, world, local_rank, pending_acc=None):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2105_00027_gb300 import build, g4, inputs

    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    p = bench_problem(args)
    N = p.N
    ctype = torch.complex128 if p.m_dtype == "c128" else torch.complex64
    pool = default_pool(p, args)
    stream = torch.cuda.current_stream()

    h = g4.G4.for_problem(p, precision="mixed", batch=p.batch, stream=stream, channel=args.channel,
                          operands=args.operands, accum=args.accum,
                          deferred=staging_of(p, args) == "deferred")
    G0 = torch.from_numpy(inputs.g0(p)).to(dev)
    signs = inputs.signs(p, seed=rank).tolist()
    M = None
    while M is None:
        try:
            M = torch.empty((pool, 2, N, N), dtype=ctype, device=dev)
        except torch.cuda.OutOfMemoryError:
            pool //= 2
            if pool < 1:
                raise
    inputs.fill_M_device(M, seed=rank)
    out = torch.empty(p.entries, dtype=torch.complex128, device=dev)
    nb = math.ceil(p.R / p.batch)

    def step():
        h.reset()
        for r in range(p.R):
            h.compute_G(M[r % pool], G0, signs[r])
        h.finalize(out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = None
    h.profile(True)
    for k in g4.KERNEL_KINDS:
        h.profile_read(k)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(gpu_id) if rank == 0 else None
    t_ev0 = torch.cuda.Event(enable_timing=True)
    t_ev1 = torch.cuda.Event(enable_timing=True)
    t_ev0.record(stream)
    for _ in range(args.steps):
        step()
    t_ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    ms = t_ev0.elapsed_time(t_ev1) / args.steps
    ms_max, _, value = replica_throughput(ms, p.updates, world, dev if world > 1 else None)

    prof = {k: h.profile_read(k) for k in g4.KERNEL_KINDS}
    h.profile(False)
    nb_step = math.ceil(p.R / p.batch)
    roof = roofline(p, prof, args.steps, nb_step, ms_max, args.operands)
    kernels = {k: {"ms_per_step": round(v[0] / args.steps, 3), "launches_per_step": v[1] / args.steps}
               for k, v in prof.items() if v[1]}
    launches = sum(v[1] for v in prof.values())
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "precision": "mixed: complex64 G; direct and exchange terms on tcgen05 tensor cores "
                     "as %s hi/lo operand pairs (hi.hi + hi.lo + lo.hi, FP32 MMA "
                     "accumulation; FP32 CUDA cores for Nwex > 16); one %s accumulator"
                     % (args.operands.upper(), "FP64" if args.accum == "fp64"
                        else "compensated FP32-pair"),
        "data": "synthetic (seeded N(0,1/N) M, P(s=+1)=0.9)",
        "config": dict(workload_desc(p, args.workload, args.channel), m_pool=pool,
                       l2="inputs larger than L2", staging=staging_of(p, args),
                       parallelism="replicas" if world > 1 else "single GPU"),
        "roofline": roof,
        "kernels": kernels,
        "gpu_launches": launches // args.steps * args.steps,
        "clocks": clk,
    }
    del M
    torch.cuda.empty_cache()

    def leg(key, fn):
        # the measurements beside the headline: each one on its own, with the
        # device's cached blocks returned first (they hold G4-sized buffers)
        torch.cuda.empty_cache()
        try:
            result[key] = fn()
        except Exception as exc:  # recorded, the headline stands
            result[key] = {"error": repr(exc)[:400]}
        torch.cuda.empty_cache()
        print("bench: %s done" % key, file=sys.stderr, flush=True)

    print("bench: timed region %.1f ms per step, %.4g %s" % (ms_max, value, UNIT), file=sys.stderr,
          flush=True)
    if not args.no_e2e:
        def e2e():
            r = run_e2e(p, h, G0, signs, dev, stream)
            r["h2d_gbs_measured"] = h2d_bandwidth(dev)
            return r
        leg("e2e", e2e)
    h.close()
    if pending_acc is not None:
        leg("accuracy", lambda: gpu_accuracy(p, dev, args.channel, out, pending_acc,
                                             deferred=staging_of(p, args) == "deferred"))
    del out
    if not args.no_fp64:
        leg("fp64_plain", lambda: run_fp64(p, dev, rank))
    if not args.no_vertices:
        leg("vertex_path", lambda: run_vertices(p, dev, rank, args.channel))
    if not args.no_group:
        def group():
            g = run_group(args, rank, 1, local_rank, steps=3, warmup=2, pool=16)
            r = {k: g[k] for k in ("value", "unit", "ms_per_step", "steps", "warmup", "config")}
            r["note"] = ("the batching form: twelve problems in grouped launches (one cached "
                         "CUDA graph per group shape)")
            return r
        leg("group12", group)
    return result


def run_e2e(p, h, G0, signs, dev, stream):
    """Same metric through the public API with host inputs: every step copies
    each measurement's M from pinned host memory into a ring of device buffers
    on a copy stream (deep enough to keep copying while a batch accumulates)
    and reads G4 back to pinned host memory.  A ring buffer is reused once the
    handle has read it: after its g4_compute_G (eager staging), or after its
    batch's g4_accumulate (deferred staging)."""
    import torch
    from paper_2105_00027_gb300 import inputs
    N = p.N
    ctype = torch.complex128 if p.m_dtype == "c128" else torch.complex64
    hp = min(16, p.R)
    host = torch.empty((hp, 2, N, N), dtype=ctype, pin_memory=True)
    for i in range(hp):
        host[i].copy_(inputs.measurement_M(p, i).to(ctype))
    G0h = G0.cpu().pin_memory()
    out_h = torch.empty(p.entries, dtype=torch.complex128, pin_memory=True)
    depth = min(p.R, p.batch + 32)
    ring = torch.empty((depth, 2, N, N), dtype=ctype, device=dev)
    g0d = torch.empty_like(G0)
    cs = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event() for _ in range(depth)]
    consumed = [torch.cuda.Event() for _ in range(depth)]
    for e in consumed:
        e.record(stream)

    deferred = bool(h.opt.deferred)

    def step():
        h.reset()
        g0d.copy_(G0h, non_blocking=True)
        pending = []
        for r in range(p.R):
            b = r % depth
            cs.wait_event(consumed[b])
            with torch.cuda.stream(cs):
                ring[b].copy_(host[r % hp], non_blocking=True)
                copied[b].record(cs)
            stream.wait_event(copied[b])
            h.compute_G(ring[b], g0d, signs[r])
            if not deferred:
                consumed[b].record(stream)
                continue
            pending.append(b)
            if len(pending) == p.batch or r == p.R - 1:
                h.accumulate()
                for bb in pending:
                    consumed[bb].record(stream)
                pending = []
        h.finalize(out_h)

    # the copy stream alone over the same pinned pool and ring (context for e2e:
    # the machine's host-to-device rate for this pattern)
    torch.cuda.synchronize()
    tc0 = time.perf_counter()
    with torch.cuda.stream(cs):
        for r in range(min(p.R, 4 * depth)):
            ring[r % depth].copy_(host[r % hp], non_blocking=True)
    torch.cuda.synchronize()
    copy_gbs = min(p.R, 4 * depth) * host[0].numel() * host.element_size() / (time.perf_counter() - tc0) / 1e9
    step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    step()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    h2d = p.R * 2 * N * N * host.element_size() + G0.numel() * G0.element_size()
    del ring
    return {"value": p.updates / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(p.entries * 16), "ms_per_step": dt * 1e3, "steps": 1,
            "host_pool": hp, "device_ring": depth, "h2d_copy_only_gbs": copy_gbs}


def h2d_bandwidth(dev):
    """Plain pinned-host -> device copy rate (GB/s) of this box, for context."""
    import torch
    a = torch.empty(1 << 30, dtype=torch.uint8, pin_memory=True)
    b = torch.empty(1 << 30, dtype=torch.uint8, device=dev)
    b.copy_(a, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(4):
        b.copy_(a, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    return 4 * (1 << 30) / (e0.elapsed_time(e1) / 1e3) / 1e9


def run_fp64(p, dev, rank):
    """The plain FP64 per-measurement GPU path on the same problem dimensions,
    on a 16-measurement prefix of the run (it is two orders slower)."""
    import torch
    from paper_2105_00027_gb300 import g4, inputs
    R = 16
    h = g4.G4.for_problem(p, precision="fp64", batch=8)
    G0 = torch.from_numpy(inputs.g0(p)).to(dev)
    ctype = torch.complex128 if p.m_dtype == "c128" else torch.complex64
    M = torch.empty((R, 2, p.N, p.N), dtype=ctype, device=dev)
    inputs.fill_M_device(M, seed=rank + 7)
    out = torch.empty(p.entries, dtype=torch.complex128, device=dev)
    s = inputs.signs(p, seed=rank)[:R].tolist()

    def step():
        h.reset()
        for r in range(R):
            h.compute_G(M[r], G0, s[r])
        h.finalize(out)

    step()
    torch.cuda.synchronize()
    h.profile(True)
    for k in g4.KERNEL_KINDS:
        h.profile_read(k)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    u_ms, u_n = h.profile_read("update_fp64")
    h.close()
    upd = p.entries * R
    return {"value": upd / (ms / 1e3), "unit": UNIT, "measurements": R, "ms": ms,
            "update_kernel_ms_avg": u_ms / max(u_n, 1),
            "fp64_tflops_of_update": p.entries * 24 / (u_ms / max(u_n, 1) / 1e3) / 1e12,
            "note": "same dimensions, %d-measurement prefix, per-measurement FP64 update" % R}


def transform_flops(p, n):
    """Algorithmic FP32/FP64 flops of the vertex transform of one spin with n
    vertices in its grouped form: left sums 2Nw n^2 complex x real products
    (4 flops), right sums N 2Nw n complex products (8 flops), and the two
    cluster transforms counted as Nc-point complex FFTs (5 Nc log2 Nc flops
    each) over the 2Nw n columns of the left product and the N 2Nw of the
    right."""
    fft = 5.0 * p.Nc * math.log2(p.Nc) if p.Nc > 1 else 0.0
    return 4.0 * n * n * p.Nw2 + 8.0 * p.N * p.Nw2 * n + fft * p.Nw2 * (n + p.N)


def run_vertices(p, dev, rank, channel, pool=16, steps=2, warmup=1, max_meas=1024):
    """The same run fed from vertex configurations (the step before the path:
    the non-uniform transform to M on the GPU, then the G build and the
    accumulation), configurations resident in HBM, a pool of distinct ones
    cycled over the measurements; on a prefix of at most max_meas measurements
    (whole batches) of the run."""
    import torch
    from paper_2105_00027_gb300 import g4, inputs
    if max_meas and p.R > max_meas:
        p = inputs.with_(p, R=max(p.batch, max_meas // p.batch * p.batch))
    h = g4.G4.for_problem(p, precision="mixed", batch=p.batch, channel=channel)
    G0 = torch.from_numpy(inputs.g0(p)).to(dev)
    cfgs = []
    for i in range(pool):
        n_up, n_dn, tau, site, Mt = inputs.vertex_config(p, i, seed=rank + 11)
        cfgs.append((n_up, n_dn, torch.from_numpy(tau).to(dev), torch.from_numpy(site).to(dev),
                     torch.from_numpy(Mt).to(dev)))
    h.reserve_vertices(max(max(c[0], c[1]) for c in cfgs))
    out = torch.empty(p.entries, dtype=torch.complex128, device=dev)
    s = inputs.signs(p, seed=rank).tolist()

    def step():
        h.reset()
        for r in range(p.R):
            c = cfgs[r % pool]
            h.compute_G_vertices(p.beta, c[0], c[1], c[2], c[3], c[4], G0, s[r])
        h.finalize(out)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    h.profile(True)
    for k in g4.KERNEL_KINDS:
        h.profile_read(k)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    prof = {k: h.profile_read(k) for k in g4.KERNEL_KINDS}
    t_ms, t_n = prof["nfft"]
    h.close()
    us = 1e3 * t_ms / max(t_n, 1)
    flops = sum(transform_flops(p, c[0]) + transform_flops(p, c[1]) for c in cfgs) / pool
    achieved = flops / (us / 1e6) / 1e12
    nbar = inputs.vertices_per_spin(p)
    return {"value": p.updates / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            # a transform record spans its four launches (sort, tables, left, right)
            "gpu_launches": (sum(v[1] for v in prof.values()) + 3 * t_n) // steps,
            "note": "whole step from vertex configurations: transform to M, G build, "
                    "accumulation; %d distinct configurations cycled; %d measurements"
                    % (pool, p.R),
            "vertices_per_spin": "%d +-10%% (beta U Nc / 2, U = 4)" % nbar,
            "transform_us_per_measurement": us,
            "transform_share_of_step": us * p.R / 1e3 / ms,
            "roofline": {"bound": "alu", "kernel": "vertex transform (site sort, sorted tables, "
                         "grouped products, cluster transforms)", "achieved": achieved,
                         "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP32_PEAK_TFLOPS,
                         "algorithmic_flops_per_measurement": flops,
                         "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz (derived)"}}


def run_transform_only(p, dev, rank, args, pool=16):
    """The transform alone (g4_vertex_M) at the workload's cluster and grid: a
    step is the workload's measurements transformed one by one; throughput in
    measurements/s, device time from the handle's launch records."""
    import torch
    from paper_2105_00027_gb300 import g4, inputs
    q = inputs.with_(p, Nwex=1, Nkex=1)
    h = g4.G4.for_problem(q, precision="mixed", batch=1)
    cfgs = []
    for i in range(pool):
        n_up, n_dn, tau, site, Mt = inputs.vertex_config(p, i, seed=rank + 11)
        cfgs.append((n_up, n_dn, torch.from_numpy(tau).to(dev), torch.from_numpy(site).to(dev),
                     torch.from_numpy(Mt).to(dev)))
    h.reserve_vertices(max(max(c[0], c[1]) for c in cfgs))
    M = torch.empty((2, p.N, p.N), dtype=torch.complex64, device=dev)

    def step():
        for r in range(p.R):
            c = cfgs[r % pool]
            h.vertex_M(p.beta, c[0], c[1], c[2], c[3], c[4], M)

    for _ in range(args.warmup):
        step()
    h.profile(True)
    h.profile_read("nfft")
    for _ in range(args.steps):
        step()
    t_ms, t_n = h.profile_read("nfft")
    h.close()
    us = 1e3 * t_ms / max(t_n, 1)
    flops = sum(transform_flops(p, c[0]) + transform_flops(p, c[1]) for c in cfgs) / pool
    achieved = flops / (us / 1e6) / 1e12
    return {
        "metric": "vertex configurations transformed to M per second", "value": 1e6 / us,
        "unit": "measurements/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": us * p.R / 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic vertex configurations (%d per spin +-10%%)" % inputs.vertices_per_spin(p),
        "config": {"workload": "transform of %s: Nc=%d (%dx%d), 2Nw=%d, beta=%g, %d measurements"
                               % (args.workload, p.Nc, p.Lx, p.Ly, p.Nw2, p.beta, p.R),
                   "l2": "inputs larger than L2 across the 16 configurations"},
        "roofline": {"bound": "alu", "kernel": "vertex transform", "achieved": achieved,
                     "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                     "traffic": None, "algorithmic_flops_per_measurement": flops,
                     "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz (derived)"},
        "gpu_launches": 4 * t_n // max(args.steps, 1),
        "transform_us_per_measurement": us,
    }


def run_vertex_stage(args, rank, world, local_rank):
    """The run fed from vertex configurations as the timed step (replicas on
    N > 1, like the default mode)."""
    import torch
    from paper_2105_00027_gb300 import build, inputs
    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    p = bench_problem(args)
    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = None
    clocks = Clocks(gpu_id) if rank == 0 else None
    if args.transform_only:
        res = run_transform_only(p, dev, rank, args)
        res["clocks"] = clocks.stop() if clocks else None
        return res
    v = run_vertices(p, dev, rank, args.channel, steps=args.steps, warmup=args.warmup)
    clk = clocks.stop() if clocks else None
    ms_max, _, value = replica_throughput(v["ms_per_step"], p.updates, world,
                                          dev if world > 1 else None)
    return {
        "metric": METRIC + " (from vertex configurations)", "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic vertex configurations (" + v["vertices_per_spin"] + ")",
        "config": dict(workload_desc(p, args.workload, args.channel), l2="inputs larger than L2",
                       parallelism="replicas" if world > 1 else "single GPU"),
        "roofline": v["roofline"], "gpu_launches": v["gpu_launches"],
        "transform_us_per_measurement": v["transform_us_per_measurement"],
        "transform_share_of_step": v["transform_share_of_step"], "clocks": clk,
    }


def run_group(args, rank, world, local_rank, steps=None, warmup=None, pool=None):
    """Twelve independent problems of uneven size; every round stages
    one batch per unfinished problem and accumulates them with one grouped
    (graph) launch."""
    import torch
    from paper_2105_00027_gb300 import build, g4, inputs
    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    probs = inputs.group_problems(seed=rank)
    stream = torch.cuda.current_stream()
    hs, Ms, G0s, sg = [], [], [], []
    pool = pool or args.m_pool or 16
    steps = steps or args.steps
    warmup = args.warmup if warmup is None else warmup
    for i, p in enumerate(probs):
        hs.append(g4.G4.for_problem(p, precision="mixed", batch=p.batch, stream=stream))
        M = torch.empty((min(pool, p.R), 2, p.N, p.N), dtype=torch.complex128, device=dev)
        inputs.fill_M_device(M, seed=rank * 100 + i)
        Ms.append(M)
        G0s.append(torch.from_numpy(inputs.g0(p)).to(dev))
        sg.append(inputs.signs(p, seed=rank, problem_index=i).tolist())
    outs = [torch.empty(p.entries, dtype=torch.complex128, device=dev) for p in probs]
    rounds = max(math.ceil(p.R / p.batch) for p in probs)

    def step():
        for h in hs:
            h.reset()
        for b in range(rounds):
            for i, p in enumerate(probs):
                for r in range(b * p.batch, min(p.R, (b + 1) * p.batch)):
                    hs[i].compute_G(Ms[i][r % Ms[i].shape[0]], G0s[i], sg[i][r])
            g4.accumulate_group(hs)
        for h, o in zip(hs, outs):
            h.finalize(o)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1) / steps
    upd = sum(p.updates for p in probs)
    ms_max, _, value = replica_throughput(ms, upd, world, dev if world > 1 else None)
    for h in hs:
        h.close()
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded N(0,1/N) M, P(s=+1)=0.9)",
        "config": {"workload": "group12: 12 problems, Nc in {4,8,16,36} x 2Nw in {16,32,64}, "
                               "Nwex=4, Nkex=Nc, grouped graph launch per round",
                   "problems": [[p.Nc, p.Nw2, p.R] for p in probs], "element_updates": upd,
                   "m_pool_per_problem": pool},
    }


# ---------------------------------------------------------------- partitioned G4
def run_sharded(args, rank, world, local_rank):
    """One problem on N GPUs with G4 partitioned over them (paper_2105_00027_gb300.shard):
    each rank holds a slab of the transfer frequencies; per batch round the
    ranks of a group all-gather their measurements' M over NCCL so that every
    rank stages the whole batch; groups (when N exceeds Nwex) split the
    measurements and sum their slabs at the end.  Strong scaling: the total
    work (E x R of the one problem) is fixed."""
    import torch
    import torch.distributed as dist
    from paper_2105_00027_gb300 import g4, inputs, shard
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    p = bench_problem(args)
    lay = shard.layout(rank, world, p.Nwex, args.shards)
    gpg, cpg = shard.ShardedRun.process_groups(dist, lay) if world > 1 else (None, None)
    stream = torch.cuda.current_stream()
    h = g4.G4.for_problem(p, precision="mixed", batch=p.batch, stream=stream, channel=args.channel,
                          wex_slab=(lay.m_first, lay.m_count))
    G0 = torch.from_numpy(inputs.g0(p)).to(dev)
    signs = inputs.signs(p, seed=0).tolist()
    ctype = torch.complex128 if p.m_dtype == "c128" else torch.complex64
    pool = min(default_pool(p, args), 64)
    M = torch.empty((pool, 2, p.N, p.N), dtype=ctype, device=dev)
    inputs.fill_M_device(M, seed=0)
    out = torch.empty(h.E, dtype=torch.complex128, device=dev)
    eng = shard.HandleEngine(h, G0, out)
    run = shard.ShardedRun(lay, dist, gpg, cpg)

    def step():
        h.reset()
        run.run(eng, p.R, p.batch, lambda r: M[r % pool], lambda r: signs[r])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    h.close()
    return {
        "metric": METRIC, "value": p.updates / (ms_max / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded N(0,1/N) M, P(s=+1)=0.9)",
        "config": dict(workload_desc(p, args.workload, args.channel), m_pool=pool,
                       l2="inputs larger than L2",
                       parallelism="G4 partitioned over %d transfer-frequency slabs x %d "
                                   "measurement groups, NCCL all-gather of M per batch"
                                   % (lay.shards, lay.groups)),
    }


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    from paper_2105_00027_gb300 import inputs
    if args.workload == "group12":
        p = inputs.group_problems()[-1]     # the largest problem of the group
        desc = {"workload": "group12 (oracle sampled on its largest problem, Nc=%d, 2Nw=%d)"
                            % (p.Nc, p.Nw2), "channel": CHANNEL_NAMES[args.channel]}
    else:
        p = bench_problem(args)
        # the same config as the GPU arm's line for this launch
        desc = dict(workload_desc(p, args.workload, args.channel), m_pool=default_pool(p, args),
                    l2="inputs larger than L2")
        if world > 1:
            from paper_2105_00027_gb300 import shard
            lay = shard.layout(0, world, p.Nwex, args.shards)
            desc["parallelism"] = ("G4 partitioned over %d transfer-frequency slabs x %d "
                                   "measurement groups, NCCL all-gather of M per batch"
                                   % (lay.shards, lay.groups))
        else:
            desc["staging"] = staging_of(p, args)
            desc["parallelism"] = "single GPU"
    # each step a sample of about 6e8 element-updates (1-2 s of the oracle on
    # the machine's host cores): 2 measurements on as many (q, m) slabs as that takes
    n_meas = 2
    n_slabs = int(min(p.NQ, max(1, math.ceil(6e8 / (n_meas * p.N * p.N)))))
    for _ in range(min(args.warmup, 1)):
        oracle_sample(p, 0, n_meas=1, n_slabs=1, channel=args.channel)
    vals, samples = [], None
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, samples, cores = oracle_sample(p, 0, n_meas=n_meas, n_slabs=n_slabs, channel=args.channel)
        vals.append(v)
    dt = (time.perf_counter() - t0) / args.steps
    v = statistics.median(vals)
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded N(0,1/N) M, P(s=+1)=0.9)",
            "config": desc,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": samples, "cpu_model": cpu_model()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    if args.workload == "group12":
        res = run_group(args, rank, world, local_rank)
        if rank == 0:
            print(json.dumps(res), flush=True)
        return
    if args.stage == "vertices":
        res = run_vertex_stage(args, rank, world, local_rank)
        if rank == 0:
            print(json.dumps(res), flush=True)
        return
    if world > 1 or args.sharded:
        from paper_2105_00027_gb300 import build
        if rank == 0:
            build.build()
        if world > 1:
            dist.barrier()
        res = run_sharded(args, rank, world, local_rank)
        if rank == 0:
            print(json.dumps(res), flush=True)
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    pending = None
    if rank == 0 and not args.no_accuracy and args.workload != "group12":
        pending = start_oracle_accuracy(bench_problem(args), args.channel)
    res = run_ours(args, rank, world, local_rank, pending)
    if rank == 0:
        if not args.no_cpu:
            from paper_2105_00027_gb300 import inputs
            p = bench_problem(args)
            v, sample, cores = oracle_sample(p, 0, channel=args.channel)
            v1, sample1, _ = oracle_sample(p, 0, n_meas=2, n_slabs=6, threads=1,
                                           channel=args.channel)
            res["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                   "sample": sample, "gpu_over_cpu": res["value"] / v,
                                   "cpu_model": cpu_model(),
                                   "single_core": {"value": v1, "sample": sample1}}
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
