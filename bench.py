#!/usr/bin/env python
"""Benchmark of the randomized approximate-Cholesky setup and PCG solve.

Metric: setup throughput in Mnnz(G)/s and time to solution (setup + PCG to a
true relative residual of 1e-8), for the FP64 method and beside it for the
mixed form (FP32-stored factor) and the batched form (many systems in one
parac_factor_many launch against one parac_factor call per system).
nnz(G) = nnz(F) + n (strict-lower factor entries plus the unit diagonal).

One step of the default run (inputs already resident in HBM, L2 flushed
before every phase, every phase timed with CUDA events):
  1. parac_factor of the 128^3 grid with the factor in FP64, then parac_pcg;
  2. the same with the factor stored and applied in FP32 (mixed form);
  3. parac_factor_many of the 200-system SDDM batch (FP32 factors), then
     parac_pcg_many on all of them;
  4. the same 200 systems factored one parac_factor call at a time.
value = nnz(G) of step 1 over its setup time; mixed_over_fp64_tts and
batched_over_loop are the ratios of steps 1/2 and 3/4.

  python bench.py [--steps K] [--warmup W] [--workload grid3d-128] [--prec 64|32]
                  [--ordering random|nnz] [--no-mixed] [--batch auto|on|off]
  python bench.py --workload sddm-batch-200   # the batch alone
  python bench.py --impl reference            # the CPU oracle on the same workload

Workloads: grid3d-128 (default), grid2d-64, rmat-N (R-MAT scale N), rmat-24
(32 right-hand sides, block PCG), sddm-batch-200, poisson-{uniform,aniso,contrast}-N.

Under torchrun (--gpus N > 1) every rank factors and solves its own replica
of the workload (the elimination does not shard; replicas only).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6800.0
WORKLOAD_DESC = {
    "grid3d-128": "3D 7-point grid Laplacian 128^3 (n=2,097,152), weights U[1,10), random ordering",
    "grid2d-64": "2D 5-point grid Laplacian 64x64 (n=4096), unit weights, random ordering",
    "rmat-22": "R-MAT scale 22, edge factor 16, lognormal(0,1) weights, largest component, random ordering",
    "rmat-24": "R-MAT scale 24, edge factor 16, lognormal(0,1) weights, largest component, random ordering, "
               "32 right-hand sides",
    "poisson-uniform-128": "3D 7-point Dirichlet Poisson 128^3, unit coefficients, random ordering",
    "poisson-aniso-128": "3D 7-point Dirichlet Poisson 128^3, weights 1, 1, 0.01 along x, y, z, random ordering",
    "poisson-contrast-128": "3D 7-point Dirichlet Poisson 128^3, coefficients 1 / 1e4 on 8^3 blocks "
                            "(harmonic means on edges), random ordering",
    "sddm-batch-200": "200 SDDM systems, n log-uniform in [1e3, 2e5] (2D grid / random geometric / Erdos-Renyi), "
                      "factorised in one parac_factor_many launch, one right-hand side each",
}


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


# source files each timed kernel is built from: recorded DRAM traffic stays valid
# while these are unchanged
KERNEL_SOURCES = {
    "k_trsv_fwd+k_trsv_bwd": ("solve.cu", "common.cuh", "kernels.h"),
    "k_trsv_fwd_h+k_trsv_bwd_h": ("solve.cu", "common.cuh", "kernels.h", "schedule.h", "schedule.cpp"),
    "elim_kernel": ("elim.cu", "common.cuh", "kernels.h"),
}
HYBRID_MAX_ROW = 2048     # the hybrid solves run on factors without longer rows or columns


def kernel_sha(kernel):
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        h.update(name.encode())
        with open(os.path.join(ROOT, "paper_2505_02977_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, alg_bytes):
    """DRAM bytes per launch from the last ncu capture of this kernel, scaled from the
    captured workload to this one by the ratio traffic / algorithmic bytes; None when
    the kernel's sources changed since the capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.txt")) as f:
            rec = json.load(f)
    except Exception:
        return None
    k = rec.get("kernels", {}).get(kernel)
    if not k or k.get("src_sha") != kernel_sha(kernel):
        return None
    return k["ratio"] * alg_bytes


def algorithmic_bytes_elim(st):
    """Bytes the elimination must move once (per launch): read the original
    strict-lower entries (12 B each), write and read back every fill entry
    (12 B twice), write every factor entry (12 B), one 4 B counter update per
    fill entry and per factor entry, and 24 B per vertex (pivot, queue push/pop,
    column bookkeeping)."""
    nnz_low, fill, nnzF, n = st["nnz_lower_input"], st["fill_entries"], st["nnz_F"], st["labels"]
    return 12 * nnz_low + 24 * fill + 12 * nnzF + 8 * (fill + nnzF) + 24 * n


def algorithmic_bytes_trsv_pair(st, prec):
    """Forward + backward triangular solve: each reads the factor once
    (value + index: 12 B in FP64, 8 B in FP32) and touches 20 B per row
    (pointer, schedule, right-hand side, result)."""
    sF = 12 if prec == 64 else 8
    return 2 * (sF * st["nnz_F"] + 20 * st["n"])


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0])); smax.append(float(parts[1]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[4:8]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def allreduce_max(pg, x):
    if pg is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def aggregate(values_per_rank_units, times_per_rank):
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return sum(values_per_rank_units) / max(times_per_rank)


# --------------------------------------------------------------------------- shared by both arms
METRIC = "setup Mnnz(G)/s; time-to-solution to rel-res 1e-8, mixed/batched vs FP64"
MIXED_DESC = "FP32-stored factor applied by FP32 triangular solves; FP64 elimination and PCG recurrences"
BATCH_SEED = 31


def use_batch(args):
    return args.batch == "on" or (args.batch == "auto" and args.workload == "grid3d-128")


def use_mixed(args):
    return not args.no_mixed and args.prec == 64 and not args.workload.startswith("sddm-batch")


def line_config(args, A, nrhs, world):
    """The workload description both arms print."""
    cfg = {"workload": WORKLOAD_DESC.get(args.workload, args.workload), "n": A.n, "nnz_L": A.nnz,
           "G_precision": args.prec, "tol": args.tol, "ordering": args.ordering,
           "samples_per_slot": args.samples, "nrhs": nrhs}
    if use_mixed(args):
        cfg["mixed"] = MIXED_DESC
    if use_batch(args):
        cfg["batch"] = WORKLOAD_DESC["sddm-batch-200"] + "; FP32-stored factors; vs one parac_factor call each"
    cfg["l2"] = "flushed before every timed phase (256 MB write)"
    cfg["parallelism"] = f"replicas x{world}"
    return cfg


def same_bits(Fa, Fb):
    """Bitwise equality of two exported factors (structure, values, pivots)."""
    return (Fa["n"] == Fb["n"] and np.array_equal(Fa["colptr"], Fb["colptr"])
            and np.array_equal(Fa["row"], Fb["row"])
            and np.array_equal(np.asarray(Fa["val"]).view(np.uint64), np.asarray(Fb["val"]).view(np.uint64))
            and np.array_equal(np.asarray(Fa["D"]).view(np.uint64), np.asarray(Fb["D"]).view(np.uint64)))


def oracle_solve(A, perm, seed, b, args, gpu_factor=None):
    """The oracle as it stands on one host core: one sequential factorisation
    and one PCG solve of the workload (FP64), timed separately; with the GPU's
    exported factor, a bitwise comparison of the two."""
    import oracle
    t0 = time.perf_counter()
    F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed, samples=args.samples)
    tf = time.perf_counter() - t0
    nnzG = len(F["row"]) + F["n"]
    bb = b if b.ndim == 1 else np.ascontiguousarray(b[:, 0])
    t0 = time.perf_counter()
    _, it, rr = oracle.pcg(A.colptr, A.rowind, A.val, F, perm, bb, args.tol, 2000)
    tp = time.perf_counter() - t0
    out = {"value": nnzG / tf / 1e6, "unit": "Mnnz(G)/s", "cores": 1, "kind": "oracle",
           "sample": f"one full sequential oracle factorisation ({tf:.1f} s) and one FP64 PCG solve "
                     f"({tp:.1f} s, first right-hand side) of {args.workload}",
           "fact_s": tf, "pcg_s": tp, "pcg_iters": int(it), "true_relres": float(rr), "tts_s": tf + tp,
           "nnz_G": nnzG}
    if gpu_factor is not None:
        out["bit_identical"] = bool(same_bits(gpu_factor, F))
    return out


# --------------------------------------------------------------------------- reference arm (CPU oracle)
def oracle_batch_sample(batch, seed, budget_s, gpu_factors=None):
    """The oracle on the batch's systems in order, system s keyed as in
    parac_factor_many (Philox counter word 2 = s), until budget_s seconds of
    host time are spent (at least one system); returns (nnz(G) of each system
    factored, seconds, all bitwise equal to gpu_factors[s] or None)."""
    import oracle
    nnz, t, same = [], 0.0, None if gpu_factors is None else True
    for s, (A, perm, b) in enumerate(batch):
        t0 = time.perf_counter()
        F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed, sys=s)
        t += time.perf_counter() - t0
        nnz.append(len(F["row"]) + F["n"])
        if gpu_factors is not None:
            same = same and same_bits(gpu_factors[s], F)
        if t >= budget_s:
            break
    return nnz, t, same


def run_reference_batch(args, world, rank):
    """Reference arm of sddm-batch-200: each step factors a bounded sample of
    the batch (its systems in order, ~cpu_budget seconds) with the oracle."""
    from paper_2505_02977_gb300 import workloads as W
    batch = W.sddm_batch(200)
    for _ in range(args.warmup):
        oracle_batch_sample(batch[:1], BATCH_SEED, 0.0)
    vals, steps_s, last = [], [], None
    for _ in range(args.steps):
        nnz, t, _ = oracle_batch_sample(batch, BATCH_SEED, args.cpu_budget)
        vals.append(sum(nnz) / t / 1e6); steps_s.append(t); last = nnz
    value = sum(vals) / len(vals)
    sample = (f"the first {len(last)} of 200 systems in order (nnz(G) {sum(last)}), about {args.cpu_budget:g} s "
              "of sequential oracle work per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mnnz(G)/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(steps_s) / len(steps_s), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": batch_config(args, batch, world),
        "cpu_baseline": {"value": value, "unit": "Mnnz(G)/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Mnnz(G)/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args, world, rank):
    """The oracle on our arm's workload: each step is one full sequential
    factorisation (the metric's setup); one FP64 PCG solve after the steps
    gives the oracle's time to solution."""
    if rank != 0:
        return 0
    if args.workload == "sddm-batch-200":
        return run_reference_batch(args, world, rank)
    import oracle
    from paper_2505_02977_gb300 import workloads as W
    A, perm, seed, b = W.config(args.workload)
    if args.ordering == "nnz":
        perm = W.nnz_sorted_ordering(A, seed)          # the ordering the library builds on the device
    small = W.config("grid2d-64")
    for _ in range(args.warmup):                     # untimed warm-up on a small case
        oracle.factor(small[0].colptr, small[0].rowind, small[0].val, small[1], seed=small[2])
    times, nnzG = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed, samples=args.samples)
        times.append(time.perf_counter() - t0)
        nnzG = len(F["row"]) + F["n"]
    value = nnzG * len(times) / sum(times) / 1e6
    bb = b if b.ndim == 1 else np.ascontiguousarray(b[:, 0])
    t0 = time.perf_counter()
    _, it, rr = oracle.pcg(A.colptr, A.rowind, A.val, F, perm, bb, args.tol, 2000)
    tp = time.perf_counter() - t0
    tf = sum(times) / len(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mnnz(G)/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tf, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": line_config(args, A, 1 if b.ndim == 1 else int(b.shape[1]), world),
        "nnz_G": nnzG, "tts_ms": 1e3 * (tf + tp), "setup_ms": 1e3 * tf, "pcg_ms": 1e3 * tp,
        "pcg_iters": int(it), "true_relres": float(rr),
        "cpu_baseline": {"value": value, "unit": "Mnnz(G)/s", "cores": 1, "kind": "oracle",
                         "sample": f"full sequential oracle factorisation of {args.workload} per step; "
                                   f"one FP64 PCG solve ({tp:.1f} s) after the steps",
                         "fact_s": tf, "pcg_s": tp, "pcg_iters": int(it), "tts_s": tf + tp},
        "e2e": {"value": value, "unit": "Mnnz(G)/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- our arm
class TimedStep:
    """NVTX range around one timed step ("timed_step"), so that a profiler can
    be restricted to the timed region (ncu --nvtx --nvtx-include timed_step/)."""

    def __enter__(self):
        import torch
        torch.cuda.nvtx.range_push("timed_step")
        return self

    def __exit__(self, *exc):
        import torch
        torch.cuda.nvtx.range_pop()
        return False


class Phases:
    """CUDA events around the named phases of every timed step (all on the
    stream the library runs on: the legacy default stream)."""

    def __init__(self, names, steps):
        import torch
        self.names = names
        self.ev = {nm: [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                        for _ in range(steps)] for nm in names}

    def start(self, nm, s):
        self.ev[nm][s][0].record()

    def stop(self, nm, s):
        self.ev[nm][s][1].record()

    def ms(self, nm):
        return [a.elapsed_time(b) for a, b in self.ev[nm]]


def run_ours(args, world, rank, local, pg):
    import torch
    from paper_2505_02977_gb300 import build as B
    B.build()
    from paper_2505_02977_gb300 import parac as P
    from paper_2505_02977_gb300 import workloads as W

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if args.workload.startswith("sddm-batch"):
        return run_batch(args, world, rank, local, pg)
    A, perm, seed, b = W.config(args.workload)
    order = P.ORDER_GIVEN
    if args.ordering == "nnz":                  # Sec. V NNZ-sorted ordering, built by the library on the device
        order = P.ORDER_NNZ
        perm = W.nnz_sorted_ordering(A, seed)   # its definition, for the oracle
    nrhs = 1 if b.ndim == 1 else int(b.shape[1])
    td = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    cp, ri, va, bd = td(A.colptr), td(A.rowind), td(A.val), td(b)
    od = td(perm) if order == P.ORDER_GIVEN else None
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)     # > L2 (129 MB)
    precs = [args.prec] + ([32] if use_mixed(args) else [])
    opts = {p: P.parac_opts_default(g_precision=p, timing=1, samples=args.samples, order=order) for p in precs}

    bsys = brhs = bopts = tune = None
    if use_batch(args):
        batch = W.sddm_batch(200)
        bsys = [(Ab.n, td(Ab.colptr), td(Ab.rowind), td(Ab.val), td(pb)) for (Ab, pb, _) in batch]
        brhs = [td(bb) for (_, _, bb) in batch]
        bopts, tune = P.parac_autotune(bsys[::10], BATCH_SEED, P.parac_opts_default(g_precision=32))

    phases = ["setup", "pcg"] + (["setup_mixed", "pcg_mixed"] if len(precs) > 1 else [])
    if bsys:
        phases += ["batch_setup", "batch_pcg", "loop_setup"]
    res = {"iters": {p: [] for p in precs}, "relres": {p: [] for p in precs}, "status": set(), "stats": {},
           "b_its": [], "b_rr": [], "b_nnz": 0, "loop_nnz": 0}

    def step(ph, s):
        for p in precs:
            flush.zero_()
            tag = "" if p == args.prec else "_mixed"
            if ph: ph.start("setup" + tag, s)
            G = P.parac_factor(A.n, cp, ri, va, od, seed, opts[p])
            if ph: ph.stop("setup" + tag, s); ph.start("pcg" + tag, s)
            _, it, rr, status = P.parac_pcg(G, A.n, None, None, None, bd, tol=args.tol, maxit=2000)
            if ph:
                ph.stop("pcg" + tag, s)
                res["iters"][p].append(int(max(it))); res["relres"][p].append(float(max(rr)))
                res["status"].add(status)
                if p not in res["stats"]:
                    res["stats"][p] = G.stats()
            G.free()
        if bsys:
            flush.zero_()
            if ph: ph.start("batch_setup", s)
            Gs = P.parac_factor_many(bsys, BATCH_SEED, bopts)
            if ph: ph.stop("batch_setup", s); ph.start("batch_pcg", s)
            _, its, rrs, bstat = P.parac_pcg_many(Gs, brhs, tol=args.tol, maxit=2000)
            if ph:
                ph.stop("batch_pcg", s)
                res["b_its"] += [int(v) for v in its]; res["b_rr"] += [float(v) for v in rrs]
                res["status"].add(bstat)
                if not res["b_nnz"]:
                    res["b_nnz"] = sum(G.stats()["nnz_G"] for G in Gs)
            for G in Gs:
                G.free()
            flush.zero_()
            if ph: ph.start("loop_setup", s)
            Gl = [P.parac_factor(*sy, BATCH_SEED + i, bopts) for i, sy in enumerate(bsys)]
            if ph:
                ph.stop("loop_setup", s)
                if not res["loop_nnz"]:
                    res["loop_nnz"] = sum(G.stats()["nnz_G"] for G in Gl)
            for G in Gl:
                G.free()

    for _ in range(args.warmup):
        step(None, 0)
    torch.cuda.synchronize()

    ph = Phases(phases, args.steps)
    clocks = ClockSampler(local)
    barrier(pg)
    torch.cuda.synchronize()
    launches0 = P.parac_kernel_launches()
    clocks.start()
    t_wall0 = time.perf_counter()
    for s in range(args.steps):
        with TimedStep():
            step(ph, s)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    launches = P.parac_kernel_launches() - launches0
    barrier(pg)
    ms = {nm: ph.ms(nm) for nm in phases}
    step_ms = [sum(ms[nm][s] for nm in phases) for s in range(args.steps)]
    med = {nm: statistics.median(v) for nm, v in ms.items()}
    st64 = res["stats"][args.prec]
    nnzG = st64["nnz_G"]

    # dominant kernel: the elimination (timed by the library with events around
    # its launch) or the triangular-solve pair of the preconditioner (timed here)
    G = P.parac_factor(A.n, cp, ri, va, od, seed, opts[args.prec])
    st_el = G.stats()
    r = td(np.random.default_rng(0).standard_normal(A.n))      # one right-hand side: the single-vector solves
    z = torch.empty_like(r)
    P.parac_precond_apply(G, r, z)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record()
    for _ in range(reps):
        P.parac_precond_apply(G, r, z)
    e1.record()
    torch.cuda.synchronize()
    trsv_ms = e0.elapsed_time(e1) / reps
    gpu_factor = G.export() if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None
    G.free()
    elim_ms = st_el["t_elim_ms"]
    peak, peak_kind = measured_peak_hbm()
    applies = statistics.median(res["iters"][args.prec]) + 1
    if elim_ms >= trsv_ms * applies:
        name, t_ms, alg = "elim_kernel", elim_ms, algorithmic_bytes_elim(st_el)
    else:
        hybrid = st_el.get("max_row_F", HYBRID_MAX_ROW + 1) <= HYBRID_MAX_ROW
        name = "k_trsv_fwd_h+k_trsv_bwd_h" if hybrid else "k_trsv_fwd+k_trsv_bwd"
        t_ms, alg = trsv_ms, algorithmic_bytes_trsv_pair(st_el, args.prec)
    achieved = alg / (t_ms * 1e-3) / 1e9

    # end to end through the public API: inputs from pinned host memory every
    # step, the solution read back to the host
    e2e = None
    if not args.no_e2e:
        hp = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hcp, hri, hva, hb = hp(A.colptr), hp(A.rowind), hp(A.val), hp(b)
        hod = hp(perm) if order == P.ORDER_GIVEN else None
        xh = torch.empty(hb.shape[::-1] if nrhs > 1 else hb.shape, dtype=torch.float64).pin_memory()
        if nrhs > 1:
            xh = xh.t()
        P.parac_factor(A.n, hcp, hri, hva, hod, seed, opts[args.prec]).free()
        e2e_setup, e2e_tts = [], []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            G = P.parac_factor(A.n, hcp, hri, hva, hod, seed, opts[args.prec])
            t1 = time.perf_counter()
            P.parac_pcg(G, A.n, None, None, None, hb, tol=args.tol, maxit=2000, X=xh)
            t2 = time.perf_counter()
            G.free()
            e2e_setup.append(t1 - t0); e2e_tts.append(t2 - t0)
        h2d = A.colptr.nbytes + A.rowind.nbytes + A.val.nbytes + b.nbytes + (perm.nbytes if hod is not None else 0)
        e2e = {"value": nnzG / statistics.median(e2e_setup) / 1e6, "unit": "Mnnz(G)/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(8 * A.n * nrhs + 4096),
               "tts_ms": 1e3 * statistics.median(e2e_tts)}

    total_setup_s = allreduce_max(pg, sum(ms["setup"]) * 1e-3)
    mean_step = allreduce_max(pg, statistics.mean(step_ms))
    value = world * nnzG * args.steps / total_setup_s / 1e6

    cpu = None
    if gpu_factor is not None:
        cpu = oracle_solve(A, perm, seed, b, args, gpu_factor)
        gpu_factor = None

    tts64 = med["setup"] + med["pcg"]
    line = {
        "metric": METRIC, "value": value, "unit": "Mnnz(G)/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.prec == 64 else "f64+f32G", "data": "synthetic",
        "config": line_config(args, A, nrhs, world),
        "nnz_G": nnzG, "tts_ms": tts64, "setup_ms": med["setup"], "pcg_ms": med["pcg"],
        "pcg_iters": statistics.median(res["iters"][args.prec]), "true_relres": max(res["relres"][args.prec]),
        "pcg_status": sorted(res["status"]),
        "vertices_per_s": A.n / (med["setup"] * 1e-3), "elim_ms": elim_ms, "depth": st_el.get("depth"),
    }
    if "setup_mixed" in med:
        tts32 = med["setup_mixed"] + med["pcg_mixed"]
        line["mixed"] = {"dtype": "f64+f32G", "tts_ms": tts32, "setup_ms": med["setup_mixed"], "pcg_ms": med["pcg_mixed"],
                         "pcg_iters": statistics.median(res["iters"][32]), "true_relres": max(res["relres"][32]),
                         "nnz_G": res["stats"][32]["nnz_G"]}
        line["mixed_over_fp64_tts"] = tts64 / tts32
        line["mixed_over_fp64_pcg"] = med["pcg"] / med["pcg_mixed"]
    if bsys:
        bval = res["b_nnz"] / (med["batch_setup"] * 1e-3) / 1e6
        lval = res["loop_nnz"] / (med["loop_setup"] * 1e-3) / 1e6
        line["batched"] = {"dtype": "f64+f32G", "systems": len(bsys), "n_total": int(sum(s[0] for s in bsys)),
                           "nnz_G": res["b_nnz"], "value": bval, "unit": "Mnnz(G)/s",
                           "setup_ms": med["batch_setup"], "pcg_ms": med["batch_pcg"],
                           "tts_ms": med["batch_setup"] + med["batch_pcg"],
                           "pcg_iters_mean": float(np.mean(res["b_its"])), "pcg_iters_max": int(max(res["b_its"])),
                           "true_relres_max": max(res["b_rr"]),
                           "one_at_a_time": {"value": lval, "setup_ms": med["loop_setup"], "nnz_G": res["loop_nnz"]},
                           "schedule": tune["best"]}
        line["batched_over_loop"] = bval / lval
    line.update({
        "roofline": {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_kind, "traffic": recorded_traffic(name, alg),
                     "algorithmic_bytes": alg, "kernel_ms": t_ms},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
        "phases_ms": med, "wall_s": t_wall,
    })
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def batch_config(args, batch, world):
    return {"workload": WORKLOAD_DESC["sddm-batch-200"], "systems": len(batch),
            "n_total": int(sum(A.n for A, _, _ in batch)), "G_precision": args.prec, "tol": args.tol,
            "l2": "flushed before every timed phase (256 MB write)", "parallelism": f"replicas x{world}"}


def run_batch(args, world, rank, local, pg):
    """sddm-batch-200: one step = parac_factor_many of the 200 systems (schedule
    from parac_autotune on every 10th system, tuned once before the timed region)
    and one PCG solve per system, all systems at once through parac_pcg_many.  value = sum nnz(G) / factor_many time; the
    same systems factored one parac_factor call at a time are timed beside it."""
    import torch
    from paper_2505_02977_gb300 import parac as P
    from paper_2505_02977_gb300 import workloads as W
    dev = torch.device("cuda", local)
    batch = W.sddm_batch(200)
    td = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    systems = [(A.n, td(A.colptr), td(A.rowind), td(A.val), td(perm)) for (A, perm, b) in batch]
    rhs = [td(b) for (A, perm, b) in batch]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    base = P.parac_opts_default(g_precision=args.prec)
    opts, tune_report = P.parac_autotune(systems[::10], BATCH_SEED, base)
    seed = BATCH_SEED

    def solve_all(Gs):
        xs, it, rr, st = P.parac_pcg_many(Gs, rhs, tol=args.tol, maxit=2000)
        return [int(v) for v in it], [float(v) for v in rr]

    for _ in range(args.warmup):
        Gs = P.parac_factor_many(systems, seed, opts)
        solve_all(Gs)
        for G in Gs: G.free()
    torch.cuda.synchronize()
    ph = Phases(["setup", "pcg"], args.steps)
    clocks = ClockSampler(local)
    barrier(pg)
    torch.cuda.synchronize()
    launches0 = P.parac_kernel_launches()
    clocks.start()
    its_all, rr_all, nnzG, gpu_factors = [], [], 0, None
    for s in range(args.steps):
        flush.zero_()
        with TimedStep():
            ph.start("setup", s)
            Gs = P.parac_factor_many(systems, seed, opts)
            ph.stop("setup", s); ph.start("pcg", s)
            its, rrs = solve_all(Gs)
            ph.stop("pcg", s)
        its_all += its; rr_all += rrs
        if s == 0:
            nnzG = sum(G.stats()["nnz_G"] for G in Gs)
            if rank == 0 and world == 1 and not args.no_cpu_baseline:
                gpu_factors = [G.export() for G in Gs[:40]]
        for G in Gs: G.free()
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = P.parac_kernel_launches() - launches0
    setup_ms, pcg_ms = ph.ms("setup"), ph.ms("pcg")
    # one system at a time (same schedule), for the batched-vs-loop ratio
    loop_ms = []
    for _ in range(3):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Gs = [P.parac_factor(*sy, seed + i, opts) for i, sy in enumerate(systems)]
        torch.cuda.synchronize()
        loop_ms.append(1e3 * (time.perf_counter() - t0))
        loop_nnz = sum(G.stats()["nnz_G"] for G in Gs)
        for G in Gs: G.free()
    total_setup_s = allreduce_max(pg, sum(setup_ms) * 1e-3)
    value = world * nnzG * args.steps / total_setup_s / 1e6
    loop_value = loop_nnz / (statistics.median(loop_ms) * 1e-3) / 1e6
    cpu = None
    if gpu_factors is not None:
        nnz, tc, same = oracle_batch_sample(batch, seed, args.cpu_budget, gpu_factors)
        cpu = {"value": sum(nnz) / tc / 1e6, "unit": "Mnnz(G)/s", "cores": 1, "kind": "oracle",
               "sample": f"the first {len(nnz)} of 200 systems in order, sequential oracle ({tc:.1f} s)",
               "bit_identical": bool(same)}
    line = {
        "metric": METRIC, "value": value, "unit": "Mnnz(G)/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": allreduce_max(pg, statistics.mean([a + b for a, b in zip(setup_ms, pcg_ms)])),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32G" if args.prec == 32 else "f64", "data": "synthetic",
        "config": dict(batch_config(args, batch, world), schedule=tune_report["best"]),
        "nnz_G": nnzG, "setup_ms": statistics.median(setup_ms), "pcg_ms": statistics.median(pcg_ms),
        "tts_ms": statistics.median([a + b for a, b in zip(setup_ms, pcg_ms)]),
        "pcg_iters_mean": float(np.mean(its_all)), "pcg_iters_max": int(max(its_all)),
        "true_relres_max": max(rr_all),
        "one_at_a_time": {"value": loop_value, "unit": "Mnnz(G)/s", "setup_ms": statistics.median(loop_ms),
                          "nnz_G": loop_nnz},
        "batched_over_loop": value / world / loop_value,
        "autotune": tune_report, "gpu_launches": int(launches), "clocks": clk,
        "roofline": None, "cpu_baseline": cpu, "e2e": None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_solve_reference(args):
    """A speed reference for the preconditioner apply, outside the hot path:
    the same exported factor applied by cuSPARSE's triangular solves (through
    torch.triangular_solve on CUDA sparse-CSR matrices, which runs cuSPARSE's
    analysis and solve on every call), against parac_precond_apply.  Both
    compute z = P^T (I+F)^{-T} D^+ (I+F)^{-1} P r in FP64; the line reports
    the median times and the relative difference of the two z."""
    import torch
    from paper_2505_02977_gb300 import build as B
    B.build()
    from paper_2505_02977_gb300 import parac as P
    from paper_2505_02977_gb300 import workloads as W
    import scipy.sparse as sp
    A, perm, seed, b = W.config(args.workload)
    G = P.parac_factor(A.n, A.colptr, A.rowind, A.val, perm, seed, P.parac_opts_default(g_precision=64))
    F = G.export()
    n = F["n"]
    nnzF = int(F["colptr"][-1])
    cp, row, val = F["colptr"], F["row"][:nnzF], F["val"][:nnzF]
    Fcsr = sp.csc_matrix((val, row, cp), shape=(n, n)).tocsr()
    Fcsr.sort_indices()
    dev = torch.device("cuda")
    lower = torch.sparse_csr_tensor(torch.from_numpy(Fcsr.indptr.astype(np.int64)),
                                    torch.from_numpy(Fcsr.indices.astype(np.int64)),
                                    torch.from_numpy(Fcsr.data), size=(n, n), device=dev)
    upper = torch.sparse_csr_tensor(torch.from_numpy(cp.astype(np.int64)), torch.from_numpy(row.astype(np.int64)),
                                    torch.from_numpy(val), size=(n, n), device=dev)     # CSR of F^T = CSC of F
    D = np.asarray(F["D"], np.float64)[:n]
    dplus = torch.from_numpy(np.where(D > 0, 1.0 / np.where(D > 0, D, 1.0), 0.0)).to(dev)
    order = torch.from_numpy(np.asarray(perm if perm is not None else np.arange(n), np.int64)).to(dev)
    r = torch.from_numpy(np.ascontiguousarray(W.gaussian_rhs(A.n, 1, 3)).reshape(-1).copy()).to(dev)

    def reference(rv):
        y = rv[order].unsqueeze(1)
        y = torch.triangular_solve(y, lower, upper=False, unitriangular=True).solution
        y = y * dplus.unsqueeze(1)
        y = torch.triangular_solve(y, upper, upper=True, unitriangular=True).solution
        z = torch.empty_like(rv)
        z[order] = y[:, 0]
        return z

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            out = fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts), out

    zo = torch.empty_like(r)
    for _ in range(3):
        P.parac_precond_apply(G, r, zo)
        reference(r)
    t_ours, zo = timed(lambda: P.parac_precond_apply(G, r, zo), 10)
    t_ref, zr = timed(lambda: reference(r), 5)
    diff = float(torch.linalg.norm(zo - zr) / torch.linalg.norm(zr))
    print(json.dumps({"solve_reference": {"workload": args.workload, "n": n, "nnz_F": nnzF,
                                          "parac_apply_ms": t_ours, "cusparse_apply_ms": t_ref,
                                          "cusparse": "torch.triangular_solve on sparse CSR (cuSPARSE analysis + solve per call), "
                                                      "forward and backward, D+ scale and permutations by torch",
                                          "rel_diff": diff}}), flush=True)
    G.free()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grid3d-128")
    ap.add_argument("--prec", type=int, default=None, choices=[64, 32],
                    help="precision G is stored and applied in (default: 32 for sddm-batch-200 and rmat-24, "
                         "whose configurations specify it, else 64)")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--solve-reference", action="store_true",
                    help="time cuSPARSE's triangular solves on the exported factor against parac_precond_apply, then exit")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ordering", default="random", choices=["random", "nnz"])
    ap.add_argument("--samples", type=int, default=1, help="samples per clique-tree slot (per-slot multi-sampling MS(k); 1: Alg. 2)")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the mixed-precision pass (FP32-stored factor) run beside the FP64 one")
    ap.add_argument("--batch", default="auto", choices=["auto", "on", "off"],
                    help="also run the 200-system SDDM batch (parac_factor_many vs one call per system) in every "
                         "step; auto: with the default workload only")
    ap.add_argument("--cpu-budget", type=float, default=10.0,
                    help="seconds of oracle work per step when the oracle runs on a sample of a batch")
    args = ap.parse_args()
    if args.prec is None:
        args.prec = 32 if args.workload in ("sddm-batch-200", "rmat-24") else 64
    if args.solve_reference:
        return run_solve_reference(args)
    world, rank, local, pg = dist_setup()
    try:
        if args.impl == "reference":
            return run_reference(args, world, rank)
        return run_ours(args, world, rank, local, pg)
    finally:
        if pg is not None:
            pg.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
