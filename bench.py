#!/usr/bin/env python
"""Benchmark of the randomized approximate-Cholesky setup and PCG solve.

One step = the whole hot path on one synthetic system already resident in
HBM: parac_factor (ingest, persistent elimination, compaction, solve-schedule
analysis) followed by parac_pcg to a true relative residual of 1e-8, then the
handle is released.  Headline value: setup throughput in Mnnz(G)/s, with
nnz(G) = nnz(F) + n (strict-lower factor entries plus the unit diagonal) and
the setup time measured with CUDA events around parac_factor.  Time-to-solution
(setup + PCG) is reported beside it.

  python bench.py [--steps K] [--warmup W] [--workload grid3d-128] [--prec 64|32]
                  [--ordering random|nnz]
  python bench.py --workload sddm-batch-200   # 200 SDDM systems: parac_factor_many vs a loop
  python bench.py --impl reference     # the CPU oracle on the same workload

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
    "elim_kernel": ("elim.cu", "common.cuh", "kernels.h"),
}


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


# --------------------------------------------------------------------------- reference arm (CPU oracle)
def oracle_batch_sample(batch, seed, budget_s):
    """The oracle on the batch's systems in order, system s keyed as in
    parac_factor_many (Philox counter word 2 = s), until budget_s seconds of
    host time are spent (at least one system); returns (nnz(G) of each system
    factored, seconds)."""
    import oracle
    nnz, t = [], 0.0
    for s, (A, perm, b) in enumerate(batch):
        t0 = time.perf_counter()
        F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed, sys=s)
        t += time.perf_counter() - t0
        nnz.append(len(F["row"]) + F["n"])
        if t >= budget_s:
            break
    return nnz, t


def run_reference_batch(args, world, rank):
    """Reference arm of sddm-batch-200: each step factors a bounded sample of
    the batch (its systems in order, ~cpu_budget seconds) with the oracle."""
    from paper_2505_02977_gb300 import workloads as W
    batch = W.sddm_batch(200)
    for _ in range(args.warmup):
        oracle_batch_sample(batch[:1], 31, 0.0)
    vals, steps_s, last = [], [], None
    for _ in range(args.steps):
        nnz, t = oracle_batch_sample(batch, 31, args.cpu_budget)
        vals.append(sum(nnz) / t / 1e6); steps_s.append(t); last = nnz
    value = sum(vals) / len(vals)
    sample = (f"the first {len(last)} of 200 systems in order (nnz(G) {sum(last)}), about {args.cpu_budget:g} s "
              "of sequential oracle work per step")
    line = {
        "impl": "reference", "metric": "setup Mnnz(G)/s", "value": value, "unit": "Mnnz(G)/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(steps_s) / len(steps_s), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC[args.workload], "systems": 200},
        "cpu_baseline": {"value": value, "unit": "Mnnz(G)/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Mnnz(G)/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    if args.workload == "sddm-batch-200":
        return run_reference_batch(args, world, rank)
    import oracle
    from paper_2505_02977_gb300 import workloads as W
    A, perm, seed, b = W.config(args.workload)
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
    line = {
        "impl": "reference", "metric": "setup Mnnz(G)/s", "value": value, "unit": "Mnnz(G)/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC.get(args.workload, args.workload), "nnz_G": nnzG},
        "cpu_baseline": {"value": value, "unit": "Mnnz(G)/s", "cores": 1, "kind": "oracle",
                         "sample": f"full sequential oracle factorisation of {args.workload} per step"},
        "e2e": {"value": value, "unit": "Mnnz(G)/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- our arm
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
    if args.ordering == "nnz":
        perm = W.nnz_sorted_ordering(A, seed + 1000)
    td = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    cp, ri, va, od, bd = td(A.colptr), td(A.rowind), td(A.val), td(perm), td(b)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)     # > L2 (129 MB)
    opts = P.parac_opts_default(g_precision=args.prec, timing=1, samples=args.samples)

    def step():
        G = P.parac_factor(A.n, cp, ri, va, od, seed, opts)
        x, it, rr, status = P.parac_pcg(G, A.n, None, None, None, bd, tol=args.tol, maxit=2000)
        return G, it[0], rr[0], status

    for _ in range(args.warmup):
        G, *_ = step()
        G.free()
    torch.cuda.synchronize()

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier(pg)
    torch.cuda.synchronize()
    launches0 = P.parac_kernel_launches()
    clocks.start()
    t_wall0 = time.perf_counter()
    iters, relres, stats, statuses = [], [], None, []
    for s in range(args.steps):
        flush.zero_()
        ev[s][0].record()
        G = P.parac_factor(A.n, cp, ri, va, od, seed, opts)
        ev[s][1].record()
        x, it, rr, status = P.parac_pcg(G, A.n, None, None, None, bd, tol=args.tol, maxit=2000)
        ev[s][2].record()
        iters.append(int(max(it))); relres.append(float(max(rr))); statuses.append(status)
        if stats is None:
            stats = G.stats()
        G.free()
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    launches = P.parac_kernel_launches() - launches0
    barrier(pg)
    setup_ms = [ev[s][0].elapsed_time(ev[s][1]) for s in range(args.steps)]
    pcg_ms = [ev[s][1].elapsed_time(ev[s][2]) for s in range(args.steps)]
    step_ms = [a + b for a, b in zip(setup_ms, pcg_ms)]
    nnzG = stats["nnz_G"]

    # dominant kernel: the elimination (timed by the library with events around
    # its launch) or the triangular-solve pair of the preconditioner (timed here)
    G = P.parac_factor(A.n, cp, ri, va, od, seed, opts)
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
    G.free()
    elim_ms = st_el["t_elim_ms"]
    peak, peak_kind = measured_peak_hbm()
    applies = statistics.median(iters) + 1
    if elim_ms >= trsv_ms * applies:
        name, t_ms, alg = "elim_kernel", elim_ms, algorithmic_bytes_elim(st_el)
    else:
        name, t_ms, alg = "k_trsv_fwd+k_trsv_bwd", trsv_ms, algorithmic_bytes_trsv_pair(st_el, args.prec)
    achieved = alg / (t_ms * 1e-3) / 1e9

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        b_host = np.ascontiguousarray(b)
        P.parac_factor(A.n, A.colptr, A.rowind, A.val, perm, seed, opts).free()
        e2e_setup, e2e_tts = [], []
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            G = P.parac_factor(A.n, A.colptr, A.rowind, A.val, perm, seed, opts)
            G.stats()
            t1 = time.perf_counter()
            xh, _, _, _ = P.parac_pcg(G, A.n, None, None, None, b_host, tol=args.tol, maxit=2000)
            t2 = time.perf_counter()
            G.free()
            e2e_setup.append(t1 - t0); e2e_tts.append(t2 - t0)
        h2d = A.colptr.nbytes + A.rowind.nbytes + A.val.nbytes + perm.nbytes
        e2e = {"value": nnzG / statistics.median(e2e_setup) / 1e6, "unit": "Mnnz(G)/s",
               "h2d_bytes_per_step": int(h2d + b_host.nbytes), "d2h_bytes_per_step": int(b_host.nbytes + 4096),
               "tts_ms": 1e3 * statistics.median(e2e_tts)}

    total_setup_s = allreduce_max(pg, sum(setup_ms) * 1e-3)
    mean_step = allreduce_max(pg, statistics.mean(step_ms))
    value = world * nnzG * args.steps / total_setup_s / 1e6

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        F = oracle.factor(A.colptr, A.rowind, A.val, perm, seed=seed, samples=args.samples)
        tc = time.perf_counter() - t0
        cpu = {"value": (len(F["row"]) + F["n"]) / tc / 1e6, "unit": "Mnnz(G)/s", "cores": 1, "kind": "oracle",
               "sample": f"one full sequential oracle factorisation of {args.workload} ({tc:.1f} s)",
               "bit_identical": bool(len(F["row"]) + F["n"] == nnzG)}

    line = {
        "metric": "setup Mnnz(G)/s; time-to-solution to rel-res 1e-8 in tts_ms",
        "value": value, "unit": "Mnnz(G)/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": mean_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC.get(args.workload, args.workload), "n": A.n, "nnz_L": A.nnz,
                   "nnz_G": nnzG, "G_precision": args.prec, "tol": args.tol, "ordering": args.ordering,
                   "samples_per_slot": args.samples,
                   "nrhs": 1 if b.ndim == 1 else int(b.shape[1]),
                   "l2": "flushed before every step (256 MB write)", "parallelism": f"replicas x{world}"},
        "tts_ms": statistics.median(step_ms), "setup_ms": statistics.median(setup_ms),
        "pcg_ms": statistics.median(pcg_ms), "pcg_iters": statistics.median(iters),
        "true_relres": max(relres), "pcg_status": sorted(set(statuses)),
        "vertices_per_s": A.n / (statistics.median(setup_ms) * 1e-3),
        "elim_ms": elim_ms, "depth": st_el.get("depth"),
        "roofline": {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_kind, "traffic": recorded_traffic(name, alg),
                     "algorithmic_bytes": alg, "kernel_ms": t_ms},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
        "wall_s": t_wall,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


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
    opts, tune_report = P.parac_autotune(systems[::10], 31, base)
    seed = 31

    def solve_all(Gs):
        xs, it, rr, st = P.parac_pcg_many(Gs, rhs, tol=args.tol, maxit=2000)
        return [int(v) for v in it], [float(v) for v in rr]

    for _ in range(args.warmup):
        Gs = P.parac_factor_many(systems, seed, opts)
        solve_all(Gs)
        for G in Gs: G.free()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    barrier(pg)
    torch.cuda.synchronize()
    launches0 = P.parac_kernel_launches()
    clocks.start()
    setup_ms, pcg_ms, its_all, rr_all, nnzG = [], [], [], [], 0
    for s in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Gs = P.parac_factor_many(systems, seed, opts)
        t1 = time.perf_counter()
        its, rrs = solve_all(Gs)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        setup_ms.append(1e3 * (t1 - t0)); pcg_ms.append(1e3 * (t2 - t1))
        its_all += its; rr_all += rrs
        nnz_sys = [G.stats()["nnz_G"] for G in Gs]
        nnzG = sum(nnz_sys)
        for G in Gs: G.free()
    clk = clocks.stop()
    launches = P.parac_kernel_launches() - launches0
    # one system at a time (same schedule), for the batched-vs-loop ratio
    loop_ms = []
    for _ in range(2):
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
    loop_value = loop_nnz / (min(loop_ms) * 1e-3) / 1e6
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nnz, tc = oracle_batch_sample(batch, seed, args.cpu_budget)
        cpu = {"value": sum(nnz) / tc / 1e6, "unit": "Mnnz(G)/s", "cores": 1, "kind": "oracle",
               "sample": f"the first {len(nnz)} of 200 systems in order, sequential oracle ({tc:.1f} s)",
               "bit_identical": nnz == nnz_sys[:len(nnz)]}
    line = {
        "metric": "setup Mnnz(G)/s (batched parac_factor_many); time-to-solution to rel-res 1e-8 in tts_ms",
        "value": value, "unit": "Mnnz(G)/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": allreduce_max(pg, statistics.mean([a + b for a, b in zip(setup_ms, pcg_ms)])),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC[args.workload], "systems": len(batch),
                   "n_total": sum(A.n for A, _, _ in batch), "nnz_G": nnzG, "G_precision": args.prec,
                   "tol": args.tol, "l2": "flushed before every step (256 MB write)",
                   "parallelism": f"replicas x{world}", "schedule": tune_report["best"]},
        "setup_ms": statistics.median(setup_ms), "pcg_ms": statistics.median(pcg_ms),
        "tts_ms": statistics.median([a + b for a, b in zip(setup_ms, pcg_ms)]),
        "pcg_iters_mean": float(np.mean(its_all)), "pcg_iters_max": int(max(its_all)),
        "true_relres_max": max(rr_all),
        "one_at_a_time": {"value": loop_value, "unit": "Mnnz(G)/s", "setup_ms": min(loop_ms), "nnz_G": loop_nnz,
                          "batched_over_loop": value / world / loop_value},
        "autotune": tune_report, "gpu_launches": int(launches), "clocks": clk,
        "roofline": None, "cpu_baseline": cpu, "e2e": None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


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
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ordering", default="random", choices=["random", "nnz"])
    ap.add_argument("--samples", type=int, default=1, help="samples per clique-tree slot (AC(k); 1: Alg. 2)")
    ap.add_argument("--cpu-budget", type=float, default=10.0,
                    help="seconds of oracle work per step when the oracle runs on a sample of a batch")
    args = ap.parse_args()
    if args.prec is None:
        args.prec = 32 if args.workload in ("sddm-batch-200", "rmat-24") else 64
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
