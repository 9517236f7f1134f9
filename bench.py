#!/usr/bin/env python
"""Benchmark of the MBE-FCI tuple-CASCI hot path on GB300.

One step = one pass of the whole hot path over the L=22 Hubbard-ring workload
(t=1, U=4, half filling, momentum-basis orbitals, empty reference space,
orders 1-6, tuples without an occupied or a virtual orbital skipped: 107,085
tuple CASCIs of 2-6 orbitals and up to 400 determinants): device tuple
enumeration, batched tuple CASCI, the increment recursion (Eq. 2) and the order
sums and total (Eq. 1), all through the C ABI.

Reported: tuple CASCI solves/s in mixed precision (the value) and in float64
(side by side), the largest |mixed - float64| tuple-energy difference, the
roofline of the dominant solver kernel, an end-to-end number through the
public API with host inputs, and the oracle timed on a bounded sample on the
host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "tuple CASCI solves/s at ≤1e-8 Eh, mixed vs FP64; sigma % of roofline"
UNIT = "tuple CASCI solves/s"
WORKLOAD = "hubbard22"
WORKLOAD_DESC = ("Hubbard ring L=22 t=1 U=4 half filling, momentum-basis orbitals, empty reference, "
                 "MBE orders 1-6 with the occupied/virtual skip rule (107,085 tuple CASCIs, "
                 "2-6 orbitals, <=400 determinants)")
L2_FLUSH_BYTES = 256 << 20

# ALU peaks: measured on the GPU at start-up by the library's FMA-chain kernel
# (mbe_fma_peak, best of 5 launches); the nominal figures below (unit counts at the
# 2070 MHz maximum SM clock, 152 SMs) are reported beside them for context.
NOMINAL_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
NOMINAL_FP64_TFLOPS = 1.25
PEAKS = {"fp64": NOMINAL_FP64_TFLOPS, "fp32": NOMINAL_FP32_TFLOPS, "source": "nominal"}


def measure_peaks(ctx):
    PEAKS["fp64"] = ctx.fma_peak("fp64", 5)
    PEAKS["fp32"] = ctx.fma_peak("fp32", 5)
    PEAKS["source"] = "measured on this GPU by mbe_fma_peak (FMA chains, 4 x 256 threads per SM, best of 5)"
    return dict(PEAKS)


def oracle_totals():
    """The oracle's totals of the full-size Hubbard workloads, written by
    tests/golden/make_oracle_totals.py (calls oracle/ only)."""
    try:
        return json.load(open(os.path.join(ROOT, "tests", "golden", "oracle_totals.json")))["workloads"]
    except (OSError, ValueError, KeyError):
        return {}


HARD_FAIL = (1, 2, 3)  # MAXITER, NONFINITE, BADINPUT; 4 (DEGENERATE) is a warning


def sigma_flops_per_det(n: int, k: int) -> int:
    """Algorithmic flops of one sigma element (direct string-driven form):
    same-spin 2 * Ns FMAs, opposite-spin R^2 FMAs, 2 flops per FMA."""
    ns = math.comb(n, k)
    r = k * (n - k + 1)
    return 2 * (2 * ns + r * r)


DAVIDSON_FLOPS_PER_DET = 72  # residual, preconditioner, 2-pass orthogonalisation, 3x3 projections, update


def solver_bucket(n: int, k: int, warp_max_ndet: int = 416):
    """(solver, dpl) the library uses for a class: the warp solver up to the tuned
    determinant limit (mbe_tuning.warp_max_ndet), else the block solver."""
    N = math.comb(n, k) ** 2
    if n <= 8 and N <= warp_max_ndet:
        for d in (1, 2, 4, 8, 13):
            if d * 32 >= N:
                return 0, d
    return 1, 0


# ----------------------------------------------------------------------------- utilities

class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(values, device=None):
    """Element-wise maximum of a list of floats over all ranks (identity for one
    rank).  The timed region of every rank is compared, so the slowest rank sets
    the whole-job time."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(values)
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.cpu().tolist()


def whole_job_rate(units_per_rank: int, world_size: int, ms_per_step_max: float) -> float:
    """Units all ranks processed per second: every rank runs its own replica."""
    return world_size * units_per_rank / (ms_per_step_max / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def source_hash() -> str:
    h = hashlib.sha256()
    for f in ("casci_dev.cuh", "casci_warp.cu", "casci_mixed.cu", "casci.cu", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1910_03527_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_key: str):
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu summary,
    if it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "counters.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    e = rec.get(kernel_key)
    if not e or e.get("source_hash") != source_hash():
        return None
    return e.get("dram_bytes_per_launch")


# ----------------------------------------------------------------------------- oracle leg

def oracle_sample(seconds: float, seed: int = 1910, shard: int = 0, nshards: int = 1):
    """Oracle tuple CASCIs on a seeded sample of the workload, stratified by order
    in proportion to the tuple counts, for about `seconds` of single-core work.
    With nshards > 1 this process takes every nshards-th tuple of the same
    stratified sequence, starting at `shard`."""
    import numpy as np
    from oracle import mbe as omb
    from workloads import workload

    w = workload(WORKLOAD)
    e_phi = omb.phi_energy(w.h1, w.eri, w.occ)
    lists = {n: omb.tuples(w.exp, w.ref, w.occ, n, w.skip) for n in w.orders}
    total = sum(len(v) for v in lists.values())
    rng = np.random.default_rng(seed)
    # interleave orders in proportion to their counts
    seq = []
    for n in w.orders:
        if lists[n]:
            idx = rng.permutation(len(lists[n]))
            seq += [(len(lists[n]) / total, i / len(lists[n]), n, lists[n][j]) for i, j in enumerate(idx)]
    seq.sort(key=lambda x: x[1])
    seq = seq[shard::nshards]
    t0 = time.perf_counter()
    done = 0
    per_order = {}
    for _, _, n, tup in seq:
        omb.tuple_energy(w.h1, w.eri, w.occ, w.ref, tup, e_phi, 0.0)
        done += 1
        per_order[n] = per_order.get(n, 0) + 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"tuples": done, "seconds": dt, "per_order": per_order}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_oracle_subprocess(seconds: float, nproc: int = 1):
    """The oracle sample in `nproc` single-threaded processes at once (one per
    host core), each on its own share of the stratified sequence; the rate is
    the tuples of all processes over the wall time of the slowest."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    procs = []
    t0 = time.perf_counter()
    for i in range(nproc):
        cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", str(seconds),
               "--oracle-shard", str(i), "--oracle-shards", str(nproc)]
        procs.append(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env,
                                      cwd=ROOT))
    res = []
    for p in procs:
        out, err = p.communicate(timeout=seconds * 4 + 180)
        if p.returncode != 0:
            raise RuntimeError("oracle sample failed: " + err[-2000:])
        res.append(json.loads(out.strip().splitlines()[-1]))
    wall = time.perf_counter() - t0
    per_order = {}
    for r in res:
        for k, v in r["per_order"].items():
            per_order[k] = per_order.get(k, 0) + v
    return {"tuples": sum(r["tuples"] for r in res), "seconds": max(r["seconds"] for r in res),
            "per_order": per_order, "processes": nproc, "wall": wall}


def cpu_baseline_entry(res, one=None):
    cores = res.get("processes", 1)
    out = {"value": res["tuples"] / res["seconds"], "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": (f"{res['tuples']} tuples of the same workload, seeded and stratified by order "
                      f"({res['per_order']}), {res['seconds']:.1f} s, {cores} single-threaded process(es), "
                      "one per host core")}
    if one is not None:
        out["one_core"] = {"value": one["tuples"] / one["seconds"], "unit": UNIT,
                           "sample": f"{one['tuples']} tuples, {one['seconds']:.1f} s, one process"}
    return out


# ----------------------------------------------------------------------------- our arm

def autotune_orders(ctx, eng, w, h1, eri, occ, opts_list):
    """mbe_autotune on every order of the workload, in each precision, before the
    timed steps: the library times the candidate launch choices on that order's
    whole tuple list (best of two runs after a warm-up) and keeps the fastest on
    the context.  Returns, per precision and order, the choice and the timed
    launch of the default choice next to the tuned one."""
    occ_host = w.occ.tolist()
    table = {}
    for opts in opts_list:
        prec = opts.precision
        rows = {}
        for order in w.orders:
            tup = ctx.mbe_tuples(w.norb, occ_host, w.exp, w.ref, order, w.skip)
            if tup.shape[0] == 0:
                continue
            default = ctx.get_tuning(prec, len(w.ref) + order)
            best, recs = ctx.autotune(h1, eri, occ, w.ref, 0.0, order, tup, opts)
            ms_default = next((ms for t, ms in recs if t == default), None)
            ms_best = min(ms for _, ms in recs)
            rows[str(order)] = {"tuples": int(tup.shape[0]), "choice": best, "default": default,
                                "ms_default": ms_default, "ms_tuned": ms_best,
                                "candidates": [[t["warp_max_ndet"], t["warp_warps"], t["block_basis"], ms]
                                               for t, ms in recs]}
        table[prec] = rows
    table["method"] = ("mbe_autotune per order: candidates warp_max_ndet {100, 225, 416}, warps per block "
                       "{2, 4}, block basis {12, 16, 20}, each field in turn with the others at their best "
                       "so far; one casci_batch over the order's tuples per candidate, best of 2 after a "
                       "warm-up, CUDA events")
    return table


def run_ours(args):
    import numpy as np
    import torch

    import paper_1910_03527_gb300 as eng
    from workloads import workload

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    eng.build()
    dev = torch.device("cuda", local)
    ctx = eng.Context(local)
    peaks = measure_peaks(ctx)
    w = workload(WORKLOAD)
    occ_host = w.occ.tolist()
    h1 = torch.tensor(w.h1, device=dev)
    eri = torch.tensor(w.eri, device=dev)
    occ = torch.tensor(w.occ, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    mixed, fp64 = eng.Opts(precision="mixed"), eng.Opts(precision="fp64")

    def step(opts):
        return eng.run_mbe(ctx, h1, eri, occ, w.ref, w.exp, w.orders, w.skip, opts, occ_host=occ_host)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step(mixed)
        step(fp64)
    torch.cuda.synchronize()
    tuning = None if args.no_autotune else autotune_orders(ctx, eng, w, h1, eri, occ, (mixed, fp64))
    if tuning is not None:
        for _ in range(2):  # the tuned launch shapes warmed up too
            step(mixed)
            step(fp64)
        torch.cuda.synchronize()

    def timed(opts):
        barrier()
        torch.cuda.synchronize()
        ctx.take_timings()
        ctx.set_timing(True)
        l0 = ctx.launches()
        evs, out = [], None
        for _ in range(args.steps):
            flush.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            out = step(opts)
            e.record()
            evs.append((s, e))
        torch.cuda.synchronize()
        barrier()
        launches = ctx.launches() - l0
        recs = ctx.take_timings()
        ctx.set_timing(False)
        ms = [s.elapsed_time(e) for s, e in evs]
        return ms, out, recs, launches

    sampler = ClockSampler(local)
    sampler.start()
    ms_mix, out_mix, recs_mix, launches = timed(mixed)
    ms_64, out_64, recs_64, _ = timed(fp64)
    clocks = sampler.stop()

    tot_mix, tot_64 = max_over_ranks([sum(ms_mix), sum(ms_64)], device=dev)
    n_tuples = sum(int(t.shape[0]) for t in out_mix["tuples"])
    ms_step_mix = tot_mix / args.steps
    ms_step_64 = tot_64 / args.steps
    value_mix = whole_job_rate(n_tuples, ws, ms_step_mix)
    value_64 = whole_job_rate(n_tuples, ws, ms_step_64)

    # accuracy of the mixed form against float64 on the same tuples
    diff = max([float((a - b).abs().max().item()) for a, b in zip(out_mix["eps"], out_64["eps"])
                if a.numel() > 0] + [0.0])
    bad = sum(int(((s >= 1) & (s <= 3)).sum().item()) for s in out_mix["status"] + out_64["status"])
    degenerate = sum(int((s == 4).sum().item()) for s in out_mix["status"] + out_64["status"])
    ref_tot = oracle_totals().get(WORKLOAD, {}).get("e_tot")

    def sigma_counts(out):
        it = torch.cat([x for x in out["iters"] if x.numel() > 0])
        n64 = ((it >> 16) & 0xffff).double().mean().item()
        n32 = (it & 0xffff).double().mean().item()
        return {"fp64_sigma_per_tuple": n64, "fp32_sigma_per_tuple": n32}

    solver_stats = {"mixed": sigma_counts(out_mix), "fp64": sigma_counts(out_64)}

    # ---- roofline of the dominant solver kernel (per launch, CUDA events inside the library)
    occ_np = np.asarray(w.occ)

    def roofline_of(recs, out, total_ms, prec):
        per_bucket = {}
        for (order, solver, dpl, ms) in recs:
            per_bucket.setdefault((order, solver, dpl), []).append(ms)
        key = max(per_bucket, key=lambda k: sum(per_bucket[k]))
        order, solver, dpl = key
        i = w.orders.index(order)
        tup = out["tuples"][i].cpu().numpy()
        iters = out["iters"][i].cpu().numpy()
        kk = occ_np[tup].sum(axis=1)
        n = len(w.ref) + order
        warp_max = ctx.get_tuning(prec, n)["warp_max_ndet"]
        f64 = f32 = 0.0
        for k in np.unique(kk):
            if solver_bucket(n, int(k), warp_max) != (solver, dpl):
                continue
            sel = kk == k
            # a sigma product computes the Ns(Ns+1)/2 determinants with Ia <= Ib (the rest
            # follow by the spin-flip symmetry); the Davidson algebra runs over all N
            ns = math.comb(n, int(k))
            per_it = sigma_flops_per_det(n, int(k)) * (ns * (ns + 1) // 2) + DAVIDSON_FLOPS_PER_DET * ns * ns
            f64 += float(((iters[sel] >> 16) & 0xffff).sum()) * per_it
            f32 += float((iters[sel] & 0xffff).sum()) * per_it
        launch_ms = statistics.mean(per_bucket[key])
        t_s = launch_ms / 1e3
        p64, p32 = PEAKS["fp64"], PEAKS["fp32"]
        achieved = (f64 + f32 * p64 / p32) / t_s / 1e12
        if solver == 0 and f32 > 0:
            kname = f"k_casci_warp_mixed<{dpl}>"
        else:
            kname = f"k_casci_warp<{dpl}, 0>" if solver == 0 else "k_casci_block"
        traffic = recorded_traffic(f"{kname}:order{order}")
        if solver == 0 and f32 > 0:
            kname += " (+ the float64 redo launch k_casci_warp<DPL, 2>, timed together)"
        return {"bound": "alu", "achieved": achieved, "peak": p64,
                "unit": "TFLOP/s (float64-equivalent: float32 flops weighted by the float64:float32 peak ratio; "
                        "frac = sum over the two pipes of flops / peak, over the launch time)",
                "peak_source": PEAKS["source"], "peak_fp32": p32,
                "peak_nominal": {"fp64": NOMINAL_FP64_TFLOPS, "fp32": NOMINAL_FP32_TFLOPS},
                "frac": achieved / p64,
                "traffic": traffic,
                "kernel": kname, "launch": f"order {order} solver launch",
                "ms_per_launch": launch_ms, "fp64_flop_per_launch": f64, "fp32_flop_per_launch": f32,
                "fp64_tflops": f64 / t_s / 1e12, "fp32_tflops": f32 / t_s / 1e12,
                "share_of_step": sum(per_bucket[key]) / total_ms}

    roofline = roofline_of(recs_mix, out_mix, sum(ms_mix), "mixed")
    roofline_64 = roofline_of(recs_64, out_64, sum(ms_64), "fp64")

    # ---- end to end through the public API with host inputs
    h1_h = torch.tensor(w.h1).pin_memory()
    eri_h = torch.tensor(w.eri).pin_memory()
    occ_h = torch.tensor(w.occ).pin_memory()
    e2e_times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h1_d = h1_h.to(dev, non_blocking=True)
        eri_d = eri_h.to(dev, non_blocking=True)
        occ_d = occ_h.to(dev, non_blocking=True)
        o = eng.run_mbe(ctx, h1_d, eri_d, occ_d, w.ref, w.exp, w.orders, w.skip, mixed, occ_host=occ_host)
        e_order = o["e_order"].cpu()
        e_total = o["e_total"].cpu()
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = max(statistics.mean(e2e_times), 1e-12)
    e2e = {"value": ws * n_tuples / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(h1_h.numel() * 8 + eri_h.numel() * 8 + occ_h.numel()),
           "d2h_bytes_per_step": int((e_order.numel() + e_total.numel()) * 8),
           "ms_per_step": e2e_s * 1e3, "clock": "host wall clock, synchronised"}

    result = {
        "metric": METRIC, "value": value_mix, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step_mix, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "tuples_per_step": n_tuples, "orders": "1-6",
                   "precision": "mixed (float32 Davidson to residual 1e-5, then anchored refinement: one float64 "
                                "sigma per anchor, float32 iterations on H - theta0 to residual 1e-7; energies to "
                                "float64 accuracy)",
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                   "parallelism": f"{ws} independent replica(s), no collective"},
        "fp64": {"value": value_64, "unit": UNIT, "ms_per_step": ms_step_64, "dtype": "f64",
                 "roofline": roofline_64},
        "accuracy": {"max_abs_eps_mixed_minus_fp64_Eh": diff, "non_ok_status": bad,
                     "degenerate_status": degenerate,
                     "e_total_mixed": float(out_mix["e_total"].item()),
                     "e_total_fp64": float(out_64["e_total"].item()),
                     "e_total_oracle": ref_tot,
                     "e_total_mixed_minus_oracle": (float(out_mix["e_total"].item()) - ref_tot) if ref_tot else None,
                     "e_total_fp64_minus_oracle": (float(out_64["e_total"].item()) - ref_tot) if ref_tot else None,
                     "oracle_source": "tests/golden/oracle_totals.json (tests/golden/make_oracle_totals.py)"},
        "solver": solver_stats,
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "alu_peaks_tflops": peaks,
        "autotune": tuning,
    }
    if rank == 0 and not args.no_cpu_baseline:
        one = run_oracle_subprocess(args.cpu_seconds / 2, 1)
        result["cpu_baseline"] = cpu_baseline_entry(run_oracle_subprocess(args.cpu_seconds, host_cores()), one)
    if rank == 0:
        print(json.dumps(result))
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    """The oracle as it stands, on the host cores: each step is a bounded sample
    of the same workload, timed on the wall clock."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    cores = host_cores()
    for _ in range(args.warmup):
        run_oracle_subprocess(args.ref_step_seconds / 4, cores)
    done = secs = 0.0
    per = []
    for _ in range(args.steps):
        r = run_oracle_subprocess(args.ref_step_seconds, cores)
        done += r["tuples"]
        secs += r["seconds"]
        per.append(r)
    value = done / secs
    res = {"tuples": int(done), "seconds": secs, "per_order": per[-1]["per_order"], "processes": cores}
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOAD_DESC, "orders": "1-6",
                      "sample": f"each step: about {args.ref_step_seconds:.0f} s of oracle tuple CASCIs "
                                f"from a seeded, order-stratified sample, in {cores} single-threaded "
                                "processes (one per host core)"},
           "cpu_baseline": cpu_baseline_entry(res),
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_ncu_case(args):
    """A small, fixed case for ncu captures: the order-`args.ncu_order` tuples of the
    workload through casci_batch, `args.steps` times, in the given precision."""
    import torch

    import paper_1910_03527_gb300 as eng
    from workloads import workload

    eng.build()
    w = workload(args.ncu_workload)
    dev = torch.device("cuda", 0)
    ctx = eng.Context(0)
    h1, eri, occ = (torch.tensor(x, device=dev) for x in (w.h1, w.eri, w.occ))
    tup = ctx.mbe_tuples(w.norb, w.occ.tolist(), w.exp, w.ref, args.ncu_order, w.skip)
    if args.ncu_tuples:
        tup = tup[: args.ncu_tuples].contiguous()
    opts = eng.Opts(precision=args.ncu_case)
    for _ in range(max(args.steps, 1)):
        eps, st, it = ctx.casci_batch(h1, eri, occ, w.ref, 0.0, args.ncu_order, tup, opts)
    torch.cuda.synchronize()
    print(json.dumps({"case": args.ncu_case, "order": args.ncu_order, "tuples": int(tup.shape[0]),
                      "non_ok": int(((st >= 1) & (st <= 3)).sum().item())}))
    ctx.close()


def run_large(args):
    """Single large CASCI on the synthetic 40-orbital molecule: one float64 and one
    float32 sigma at (12e,12o), (14e,14o), (16e,16o), timed with CUDA events inside
    the library, and Davidson solves (mixed and float64, residual 1e-8) of the
    --solve-sizes active spaces."""
    import numpy as np
    import torch

    import paper_1910_03527_gb300 as eng
    from workloads import synthetic_molecule

    eng.build()
    dev = torch.device("cuda", 0)
    ctx = eng.Context(0)
    measure_peaks(ctx)
    h1, eri, occ = synthetic_molecule(1910)
    th1, teri, tocc = (torch.tensor(x, device=dev) for x in (h1, eri, occ))
    actives = {12: list(range(2, 14)), 14: list(range(1, 15)), 16: list(range(0, 16))}
    out = {"metric": "single-CASCI sigma throughput (determinants/s) and fraction of ALU peak",
           "workload": "synthetic 40-orbital molecule (seed 1910), (12e,12o) {2..13}, (14e,14o) {1..14}, "
                       "(16e,16o) {0..15}", "sigma": {}}
    for n in args.large_sizes:
        A = actives[n]
        k = int(sum(int(occ[p]) for p in A))
        ns = math.comb(n, k)
        N = ns * ns
        r = k * (n - k + 1)
        conn = 1 + k * (n - k) + math.comb(k, 2) * math.comb(n - k, 2)
        flops = N * 2 * (2 * conn + r * r)
        c = torch.randn(N, dtype=torch.float64, device=dev)
        entry = {"determinants": N}
        for prec in ("fp64", "mixed"):
            ctx.casci_sigma_large(th1, teri, tocc, A, c, prec)  # warm-up (and set-up)
            torch.cuda.synchronize()
            ctx.take_timings()
            ctx.set_timing(True)
            for _ in range(args.steps):
                ctx.casci_sigma_large(th1, teri, tocc, A, c, prec)
            recs = ctx.take_timings()
            ctx.set_timing(False)
            ms = statistics.median([x[3] for x in recs if x[1] == 2])
            peak = PEAKS["fp64"] if prec == "fp64" else PEAKS["fp32"]
            entry[prec] = {"ms": ms, "dets_per_s": N / (ms / 1e3), "tflops": flops / (ms / 1e3) / 1e12,
                           "alu_frac": flops / (ms / 1e3) / 1e12 / peak,
                           "peak_tflops": peak, "flop_per_sigma": flops}
        out["sigma"][f"{n}o"] = entry
        del c
        torch.cuda.empty_cache()
    for n in ([] if args.no_solve else args.solve_sizes):
        solves = {}
        for prec in args.solve_precisions:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = ctx.casci_solve(th1, teri, tocc, actives[n], eng.Opts(precision=prec, tol=1e-8, max_iter=3000))
            torch.cuda.synchronize()
            solves[prec] = dict(res, seconds=time.perf_counter() - t0)
        if "mixed" in solves and "fp64" in solves:
            solves["abs_diff_lambda"] = abs(solves["mixed"]["lam"] - solves["fp64"]["lam"])
        solves["tol"] = 1e-8
        out[f"solve_{n}o"] = solves
    print(json.dumps(out))
    ctx.close()


def run_screened(args):
    """Screened expansion (Eq. 4 thresholds T_init = 1e-10, M_init = 3, a = 5, the
    paper's parameters; child spawning from each order's increments) on a Hubbard
    ring, through the C ABI: tuple counts per order and whole-pass solves/s."""
    import torch

    import paper_1910_03527_gb300 as eng
    from workloads import workload

    eng.build()
    w = workload(args.screened_workload)
    dev = torch.device("cuda", 0)
    ctx = eng.Context(0)
    th1, teri, tocc = (torch.tensor(x, device=dev) for x in (w.h1, w.eri, w.occ))
    occ_h = [int(v) for v in w.occ]
    opts = eng.Opts(precision="mixed")

    def one():
        return eng.run_mbe_screened(ctx, th1, teri, tocc, w.ref, w.exp, args.screened_max_order, w.skip,
                                    t_init=1e-10, m_init=3, a=5.0, opts=opts, occ_host=occ_h)

    one()
    torch.cuda.synchronize()
    times, out = [], None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        out = one()
        float(out["e_total"].item())
        times.append(time.perf_counter() - t0)
    counts = {int(n): int(out["tuples"][n - 1].shape[0]) for n in out["orders"]}
    m_occ = int(sum(occ_h[p] for p in w.exp))
    m_vir = len(w.exp) - m_occ
    full = {n: math.comb(len(w.exp), n) - ((math.comb(m_occ, n) + math.comb(m_vir, n)) if w.skip else 0)
            for n in out["orders"]}
    n_t = sum(counts.values())
    t = statistics.median(times)
    res = {"metric": "screened MBE-FCI pass: tuple CASCI solves/s (child spawning and Eq. 4 on the device)",
           "value": n_t / t, "unit": UNIT, "seconds_per_pass": t, "steps": args.steps,
           "workload": f"{w.description}, screened up to order {args.screened_max_order} "
                       "(T_init = 1e-10, M_init = 3, a = 5)",
           "tuples_per_order": counts, "unscreened_tuples_per_order": full,
           "e_total": float(out["e_total"].item()),
           "non_ok_status": int(sum(int(((s >= 1) & (s <= 3)).sum()) for s in out["status"])),
           "clock": "host wall clock around the whole pass (one stream synchronisation per order)"}
    print(json.dumps(res))
    ctx.close()


def run_expansion(args):
    """Type-1 or Type-2 expansion (Sec. 1, Fig. 1) of the Hubbard ring L=22 (t=1,
    U=4, momentum basis) through the C ABI: tuples whose active space exceeds 12
    orbitals (or --expansion-large-ndet determinants) are solved one at a time with
    the whole GPU (casci_batch_routed), the others in one batched call per order.
    Reports per-order tuple counts, active-space sizes and host wall-clock time."""
    import torch

    import paper_1910_03527_gb300 as eng
    from workloads import workload

    eng.build()
    w = workload("hubbard22")
    ref, exp = eng.expansion_spaces(w.occ, args.expansion)
    dev = torch.device("cuda", 0)
    ctx = eng.Context(0)
    th1, teri, tocc = (torch.tensor(x, device=dev) for x in (w.h1, w.eri, w.occ))
    occ_h = [int(v) for v in w.occ]
    opts = eng.Opts(precision=args.expansion_precision)
    orders = list(range(1, args.expansion_max_order + 1))
    large = args.expansion_large_ndet or None

    def one():
        return eng.run_mbe(ctx, th1, teri, tocc, ref, exp, orders, True, opts, occ_host=occ_h, large_ndet=large)

    one()
    torch.cuda.synchronize()
    times, out = [], None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        out = one()
        float(out["e_total"].item())
        times.append(time.perf_counter() - t0)
    per_order = {}
    for i, n in enumerate(orders):
        k = sum(occ_h[p] for p in ref) + (n if args.expansion == "type1" else 0)
        n_cas = len(ref) + n
        ndet = math.comb(n_cas, k) ** 2
        routed = n_cas > 12 or (large is not None and ndet > large)
        per_order[n] = {"tuples": int(out["tuples"][i].shape[0]), "cas_orbitals": n_cas, "determinants": ndet,
                        "routed": bool(routed)}
    t = statistics.median(times)
    n_t = sum(v["tuples"] for v in per_order.values())
    res = {"metric": f"{args.expansion} MBE-FCI pass: tuple CASCI solves/s",
           "value": n_t / t, "unit": UNIT, "seconds_per_pass": t, "steps": args.steps,
           "precision": args.expansion_precision,
           "workload": f"{w.description}; {args.expansion}: |R| = {len(ref)}, |exp| = {len(exp)}, "
                       f"orders 1-{args.expansion_max_order}",
           "per_order": per_order, "e_total": float(out["e_total"].item()),
           "e_ref_corr": float(out["e_ref_corr"]),
           "non_ok_status": int(sum(int(((st >= 1) & (st <= 3)).sum()) for st in out["status"])),
           "clock": "host wall clock around the whole pass"}
    print(json.dumps(res))
    ctx.close()


def run_molecule(args):
    """The synthetic 40-orbital molecule (seed 1910): (6e,6o) reference space
    {5..10}, expansion over the other 34 orbitals, orders 1..max_order, mixed
    precision, one pass after an order-1 warm-up; tuple CASCIs of 7-10 orbitals
    (up to 63,504 determinants, block solver)."""
    import torch

    import paper_1910_03527_gb300 as eng
    from workloads import workload

    import numpy as np

    eng.build()
    w = workload("molecule40")
    dev = torch.device("cuda", 0)
    ctx = eng.Context(0)
    measure_peaks(ctx)
    th1, teri, tocc = (torch.tensor(x, device=dev) for x in (w.h1, w.eri, w.occ))
    occ_h = [int(v) for v in w.occ]
    orders = list(range(1, args.molecule_max_order + 1))
    out = {"metric": "tuple CASCI solves/s, synthetic 40-orbital molecule", "unit": UNIT,
           "workload": "synthetic 40-orbital molecule (seed 1910), (6e,6o) reference {5..10}, "
                       f"34 expansion orbitals, orders 1-{orders[-1]}, no skip rule, max_iter 2000", "per_precision": {}}
    for prec in args.molecule_precisions:
        # this Hamiltonian converges slowly (ground states far below the diagonal):
        # a few order-3 tuples need more than the default 500 iterations per phase
        opts = eng.Opts(precision=prec, max_iter=2000)
        eng.run_mbe(ctx, th1, teri, tocc, w.ref, w.exp, [1], False, opts, occ_host=occ_h)
        torch.cuda.synchronize()
        ctx.take_timings()
        ctx.set_timing(True)
        t0 = time.perf_counter()
        res = eng.run_mbe(ctx, th1, teri, tocc, w.ref, w.exp, orders, False, opts, occ_host=occ_h)
        e_tot = float(res["e_total"].item())
        t = time.perf_counter() - t0
        recs = ctx.take_timings()
        ctx.set_timing(False)
        per_order = {}
        occ_np = np.asarray(w.occ)
        for i, n in enumerate(orders):
            ms = sum(r[3] for r in recs if r[0] == n)
            nt = int(res["tuples"][i].shape[0])
            it = res["iters"][i]
            # sigma flops of the order's solves (half space: Ns(Ns+1)/2 elements per
            # product), float64 and float32, over the summed solver-launch time; the
            # Davidson subspace algebra is not counted, so this is a lower bound
            roof = None
            if nt and ms > 0:
                tup = res["tuples"][i].cpu().numpy()
                its = it.cpu().numpy()
                kk = occ_np[tup].sum(axis=1) + int(occ_np[w.ref].sum())
                ncas = len(w.ref) + n
                f64 = f32 = 0.0
                for k in np.unique(kk):
                    sel = kk == k
                    ns = math.comb(ncas, int(k))
                    per = sigma_flops_per_det(ncas, int(k)) * (ns * (ns + 1) // 2)
                    f64 += float(((its[sel] >> 16) & 0xffff).sum()) * per
                    f32 += float((its[sel] & 0xffff).sum()) * per
                t_s = ms / 1e3
                ach = (f64 + f32 * PEAKS["fp64"] / PEAKS["fp32"]) / t_s / 1e12
                roof = {"bound": "alu", "kernel": "k_casci_block (+ warp-solver launches of the order)",
                        "fp64_tflops": f64 / t_s / 1e12, "fp32_tflops": f32 / t_s / 1e12,
                        "achieved_fp64_equivalent": ach, "frac_of_measured": ach / PEAKS["fp64"],
                        "counted": "sigma products only (lower bound)"}
            per_order[n] = {"tuples": nt, "solver_ms": ms, "solves_per_s": nt / (ms / 1e3) if ms > 0 else None,
                            "fp64_sigma_per_tuple": float(((it >> 16) & 0xffff).double().mean().item()) if nt else 0,
                            "fp32_sigma_per_tuple": float((it & 0xffff).double().mean().item()) if nt else 0,
                            "non_ok": int(((res["status"][i] >= 1) & (res["status"][i] <= 3)).sum().item()),
                            "roofline": roof}
        n_t = sum(v["tuples"] for v in per_order.values())
        out["per_precision"][prec] = {"value": n_t / t, "seconds": t, "e_total": e_tot, "per_order": per_order}
    print(json.dumps(out))
    ctx.close()


def run_adjoint(args):
    """The adjoint workload: Hubbard ring L=46, t=1, U=4, orders 1-4 with the skip
    rule (157,642 tuples). Forward pass (run_mbe) and backward pass (adjoint
    weights of Eq. 2 and the tuple density matrices, mbe_gradient) timed on the
    host clock, residual tolerance 1e-10; dE/dt and dE/dU from the gradient
    against central finite differences of the forward energy (step 1e-4)."""
    import torch

    import paper_1910_03527_gb300 as eng
    from workloads import hubbard_ring_momentum

    eng.build()
    L, t, U, orders = 46, 1.0, 4.0, [1, 2, 3, 4]
    dev = torch.device("cuda", 0)
    ctx = eng.Context(0)
    opts = eng.Opts(tol=1e-10)

    def tensors(tt, uu):
        h1, eri, occ, _ = hubbard_ring_momentum(L, tt, uu)
        return (torch.tensor(h1, device=dev), torch.tensor(eri, device=dev), torch.tensor(occ, device=dev),
                occ.tolist())

    def energy(tt, uu):
        h1, eri, occ, oh = tensors(tt, uu)
        out = eng.run_mbe(ctx, h1, eri, occ, [], list(range(L)), orders, True, opts, occ_host=oh)
        return float(out["e_total"].item())

    h1, eri, occ, oh = tensors(t, U)
    eng.run_mbe(ctx, h1, eri, occ, [], list(range(L)), [1, 2], True, opts, occ_host=oh)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fwd = eng.run_mbe(ctx, h1, eri, occ, [], list(range(L)), orders, True, opts, occ_host=oh)
    E = float(fwd["e_total"].item())
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    gh, ge, _ = eng.mbe_gradient(ctx, h1, eri, occ, [], list(range(L)), orders, True, opts, forward=fwd,
                                 occ_host=oh)
    torch.cuda.synchronize()
    t_bwd = time.perf_counter() - t0
    dEdt = float((gh * h1).sum()) / t
    dEdU = float((ge * eri).sum()) / U
    d = 1e-4
    fd_t = (energy(t + d, U) - energy(t - d, U)) / (2 * d)
    fd_U = (energy(t, U + d) - energy(t, U - d)) / (2 * d)
    n_t = sum(int(x.shape[0]) for x in fwd["tuples"])
    print(json.dumps({
        "metric": "MBE energy and gradient (adjoint) of the L=46 Hubbard ring",
        "workload": "Hubbard ring L=46 t=1 U=4 half filling, momentum basis, empty reference, orders 1-4, "
                    "skip rule, float64, residual tolerance 1e-10",
        "tuples": n_t, "forward_s": t_fwd, "backward_s": t_bwd,
        "forward_solves_per_s": n_t / t_fwd, "backward_tuples_per_s": n_t / t_bwd,
        "e_total": E, "dE_dt": dEdt, "dE_dU": dEdU, "fd_dE_dt": fd_t, "fd_dE_dU": fd_U,
        "homogeneity_residual": t * dEdt + U * dEdU - E, "trace_gamma_minus_N": float(torch.trace(gh)) - L,
        "clock": "host wall clock, synchronised"}))
    ctx.close()


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-step-seconds", type=float, default=8.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="time the default launch choices instead of tuning them per order in the warm-up")
    ap.add_argument("--oracle-sample", type=float, default=None, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-shard", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-shards", type=int, default=1, help=argparse.SUPPRESS)
    ap.add_argument("--ncu-case", choices=["fp64", "mixed"], default=None,
                    help="run only casci_batch on one order of the workload (for ncu captures)")
    ap.add_argument("--ncu-order", type=int, default=6)
    ap.add_argument("--ncu-workload", default=WORKLOAD, choices=["hubbard22", "molecule40"])
    ap.add_argument("--ncu-tuples", type=int, default=0, help="--ncu-case: only the first N tuples")
    ap.add_argument("--large", action="store_true",
                    help="single large CASCI: sigma throughput at 12/14/16 orbitals and a 12-orbital solve")
    ap.add_argument("--large-sizes", type=int, nargs="+", default=[12, 14, 16])
    ap.add_argument("--no-solve", action="store_true", help="--large: skip the Davidson solves")
    ap.add_argument("--solve-sizes", type=int, nargs="+", default=[12], choices=[12, 14, 16],
                    help="--large: active spaces solved in mixed and float64 precision (residual 1e-8)")
    ap.add_argument("--solve-precisions", nargs="+", default=["mixed", "fp64"], choices=["mixed", "fp64"])
    ap.add_argument("--screened", action="store_true",
                    help="screened expansion (Eq. 4) on a Hubbard ring: tuples per order and solves/s")
    ap.add_argument("--screened-workload", default="hubbard22",
                    choices=["hubbard22", "hubbard46", "hubbard22pm", "hubbard46pm"])
    ap.add_argument("--screened-max-order", type=int, default=8)
    ap.add_argument("--molecule", action="store_true",
                    help="the synthetic 40-orbital molecule: solves/s per order (block-solver sizes)")
    ap.add_argument("--molecule-max-order", type=int, default=3)
    ap.add_argument("--molecule-precisions", nargs="+", default=["mixed"], choices=["mixed", "fp64"])
    ap.add_argument("--adjoint", action="store_true",
                    help="L=46 Hubbard ring: forward and backward (gradient) times, finite-difference check")
    ap.add_argument("--expansion", choices=["type1", "type2"], default=None,
                    help="L=22 Hubbard ring as a Type-1 or Type-2 expansion (large tuple spaces routed)")
    ap.add_argument("--expansion-max-order", type=int, default=3)
    ap.add_argument("--expansion-large-ndet", type=int, default=0)
    ap.add_argument("--expansion-precision", choices=["mixed", "fp64"], default="mixed")
    args = ap.parse_args()
    if args.expansion:
        run_expansion(args)
        return
    if args.adjoint:
        run_adjoint(args)
        return
    if args.molecule:
        run_molecule(args)
        return
    if args.large:
        run_large(args)
        return
    if args.screened:
        run_screened(args)
        return
    if args.oracle_sample is not None:
        print(json.dumps(oracle_sample(args.oracle_sample, shard=args.oracle_shard, nshards=args.oracle_shards)))
        return
    if args.ncu_case is not None:
        run_ncu_case(args)
        return
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
