"""Benchmark: time-to-1e-8 solves of the delayed-assembly mixed-precision path.

One step = one complete solve of the workload (default: 3D, 243^3 cells,
64 seeded box inclusions of contrast 1e3, accuracies s = 1 -> 2 -> 4 -> 8
assembled on a side stream while FP32 V(2,2) cycles run under an FP64
flexible-CG outer loop, stopping at ||f - A u|| <= 1e-8 ||f|| with every
chunk at s = 8).  Problems are created before the timed region (their
grids, geometric stencils and vectors resident in HBM); the timed region
covers K mg_solve calls.  The working set of one solve (several GB) is far
larger than L2, so no flush is needed between steps.

Printed (one JSON line on rank 0): solves/s, p50/p99 time-to-solution, the
FP64 plain assemble-then-solve path on the same workload, the roofline of
the dominant kernel, the end-to-end figure through the C ABI with host
buffers, clocks sampled during the timed region and the CPU oracle baseline.

--impl reference times the CPU oracle (the reference arm of this build) on
a bounded sample per step, scaled to the same unit.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2005_03606_gb300 import inputs  # noqa: E402

METRIC = "solves/s & p50/p99 time-to-1e-8 residual, mixed vs FP64 plain; stencil GB/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload_desc(mg, name, path, n_cells=None):
    w = inputs.workload(name, n_cells)
    sched = w.s_schedule if path in (mg.PATH_FP64_DELAYED, mg.PATH_MIXED_DELAYED) else [w.s_final]
    return w, mg.problem_desc(w.dim, w.n_cells, w.eps, path=path, s_schedule=tuple(sched), rtol=1e-8,
                              max_cycles=3000)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"mg_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- algorithmic bytes
def sweep_traffic(workload):
    """DRAM bytes per launch of the finest-level sweep from the committed ncu
    summary, or None when that summary was taken on other source code or
    another workload."""
    import hashlib
    import re
    summ = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", "sweep_geo4_fixup_boxes3d_243.md")
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2005_03606_gb300", "csrc", "sweep.cu")
    if workload != "boxes3d" or not os.path.exists(summ):
        return None
    text = open(summ).read()
    mt = re.search(r"traffic_bytes_per_launch:\s*(\d+)", text)
    mh = re.search(r"source-sha256\(paper_2005_03606_gb300/csrc/sweep.cu\):\s*([0-9a-f]{64})", text)
    if not mt or not mh:
        return None
    if hashlib.sha256(open(src, "rb").read()).hexdigest() != mh.group(1):
        return None
    return int(mt.group(1))


def sweep_bytes(dim, n, cells_by_class, mixed, vec_bytes):
    """Algorithmic DRAM bytes of one finest-level sweep, counted per cell as
    the unit: the iterate read and written and the right-hand side read
    (3 x vec_bytes), plus the cell's stored operator read once.  Mixed paths:
    FP32 eps_c 4 + class byte 1 + the surplus payload of the cell's class
    (FP8: NP bytes + 4-byte scale, FP16: 2 NP + 4, FP32: 4 NP + 4, with NP = 28
    off-diagonals in 3D and 6 in 2D); FP64 paths: NP x 8 bytes.  Layout
    overheads (the (n+1)^d - n^d extra vertices, per-segment base offsets,
    record padding) are not algorithmic; `sweep_overhead_bytes` counts them."""
    ncell = n ** dim
    np_ = 28 if dim == 3 else 6
    b = ncell * 3 * vec_bytes
    if mixed:
        pay = (np_ + 4, 2 * np_ + 4, 4 * np_ + 4)
        b += ncell * (4 + 1)
        b += sum(int(cells_by_class[k + 1]) * pay[k] for k in range(3))
    else:
        b += ncell * np_ * 8
    return b


def sweep_overhead_bytes(dim, n, mixed, vec_bytes):
    """Bytes the layout adds to one sweep beyond `sweep_bytes`: the boundary
    ring of the vertex arrays and, on the compressed level, three u32 base
    offsets per 32-cell segment."""
    b = ((n + 1) ** dim - n ** dim) * 3 * vec_bytes
    if mixed:
        b += n ** (dim - 1) * ((n + 31) // 32) * 12
    return b


# ---------------------------------------------------------------- oracle baseline
def oracle_sample(name, cycles_full):
    """Oracle cost of the workload, estimated from a bounded sample:
    sampled-cell assembly at the final accuracy on the full grid, plus a
    complete oracle solve of the same field on a 27^3 grid (assembly at s_final
    and FCG cycles), scaled by cells and by the measured cycle count."""
    import oracle
    w = inputs.workload(name)
    f = oracle.Field(w.eps)
    n = w.n_cells
    rng = np.random.default_rng(1)
    ns = 4000
    cells = rng.choice(n ** w.dim, ns, replace=False)
    t0 = time.perf_counter()
    oracle.assemble_cells(f, n, w.s_final, cells)
    t_cell = (time.perf_counter() - t0) / ns
    nsmall = 27
    t0 = time.perf_counter()
    A = oracle.assemble(f, nsmall, w.s_final)
    t_asm_small = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, hist, k = oracle.solve(w.dim, nsmall, A, rtol=1e-8, max_cycles=400)
    t_solve = time.perf_counter() - t0
    t_cycle_vert = t_solve / max(k, 1) / (nsmall + 1) ** w.dim
    est = t_cell * n ** w.dim + t_cycle_vert * (n + 1) ** w.dim * cycles_full
    sample = (f"oracle FP64: {ns} sampled cells of {n}^{w.dim} at s={w.s_final} "
              f"({t_cell * 1e3:.3f} ms/cell) + full oracle solve at {nsmall}^{w.dim} "
              f"({k} FCG cycles, {t_solve:.1f} s; assembly {t_asm_small:.1f} s), scaled to {n}^{w.dim} cells "
              f"and {cycles_full} cycles")
    return 1.0 / est, sample, oracle.num_threads(), t_cell * ns + t_asm_small + t_solve


def oracle_full(name):
    """The oracle run in full on a workload: FP64 assembly at the final
    accuracy of every cell, then its FCG-preconditioned V(2,2) solve to 1e-8."""
    import oracle
    w = inputs.workload(name)
    f = oracle.Field(w.eps)
    t0 = time.perf_counter()
    A = oracle.assemble(f, w.n_cells, w.s_final)
    ta = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, hist, k = oracle.solve(w.dim, w.n_cells, A, rtol=1e-8, max_cycles=400)
    ts = time.perf_counter() - t0
    return {"workload": name, "n_cells": w.n_cells, "dim": w.dim, "s": w.s_final, "threads": oracle.num_threads(),
            "assembly_s": ta, "solve_s": ts, "cycles": int(k), "rel_residual": float(hist[-1]),
            "solves_per_s": 1.0 / (ta + ts)}


def oracle_probe(names, single_names):
    """Full oracle timings on the host cores: every workload in `names` with
    the OpenMP team of all cores, those in `single_names` also on one thread
    (a child process with OMP_NUM_THREADS=1)."""
    rows = [oracle_full(nm) for nm in names]
    for nm in single_names:
        env = dict(os.environ, OMP_NUM_THREADS="1")
        out = subprocess.run([sys.executable, "-c", f"import bench, json; print(json.dumps(bench.oracle_full({nm!r})))"],
                             cwd=ROOT, env=env, capture_output=True, text=True, check=True).stdout
        rows.append(json.loads(out.strip().splitlines()[-1]))
    return rows


# ---------------------------------------------------------------- arms
def run_reference(args, rank):
    if rank != 0:
        return
    cycles_full = args.ref_cycles
    vals, secs = [], []
    for i in range(args.warmup + args.steps):
        v, sample, cores, spent = oracle_sample(args.workload, cycles_full)
        if i >= args.warmup:
            vals.append(v)
            secs.append(spent)
    v = statistics.median(vals)
    line = {"metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "path": "oracle", "flush": "n/a (CPU)"},
            "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cores,
                             "kind": "oracle, extrapolated from 4000 sampled cells and a full 27^3 solve",
                             "sample": sample},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class Replicas:
    """Replica bookkeeping of a run on N ranks (one process per GPU): a
    barrier around the timed region and the max over ranks of its duration.
    The solves on different ranks are independent; there is no collective
    on the data path (gloo carries only the barrier and the max)."""

    def __init__(self, world: int):
        self.world = world
        self.dist = None
        if world > 1:
            import torch.distributed as dist
            if not dist.is_initialized():
                dist.init_process_group("gloo")
            self.dist = dist

    def barrier(self, device_sync=None):
        if device_sync is not None:
            device_sync()
        if self.dist:
            self.dist.barrier()

    def max(self, x: float) -> float:
        if not self.dist:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def aggregate(self, steps: int, region_ms: float) -> float:
        """Whole-job throughput: the steps of all ranks over the slowest rank's time."""
        return self.world * steps / (region_ms / 1e3)


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2005_03606_gb300 import mg
    torch.cuda.set_device(local_rank)
    rep = Replicas(world)
    lib = mg.load()

    def barrier():
        rep.barrier(torch.cuda.synchronize)

    max_over_ranks = rep.max

    w, desc = workload_desc(mg, args.workload, mg.PATH_MIXED_DELAYED)
    mixed_path = mg.PATH_MIXED_DELAYED
    # warm-up solves (also JIT of graphs, pool growth)
    for _ in range(args.warmup):
        with mg.Problem(desc) as P:
            P.solve()
    # device-resident timed region: K problems created beforehand
    probs = [mg.Problem(workload_desc(mg, args.workload, mixed_path)[1]) for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    barrier()
    l0 = lib.mg_launch_count()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    infos, walls = [], []
    for P in probs:
        t0 = time.perf_counter()
        infos.append(P.solve())
        walls.append((time.perf_counter() - t0) * 1e3)
    ev1.record()
    barrier()
    ck = clocks.stop()
    launches = lib.mg_launch_count() - l0
    region_ms = max_over_ranks(ev0.elapsed_time(ev1))
    value = rep.aggregate(args.steps, region_ms)
    info0 = infos[-1]
    # roofline: the finest-level V-cycle sweep (most launched kernel) and the FP64 matvec
    P = probs[-1]
    n, dim = w.n_cells, w.dim
    ms_sweep = P.profile(0, 20)
    ms_mv = P.profile(1, 10)
    ms_gal = P.profile(3, 3)
    cbc = list(info0.cells_by_class)
    b_sweep = sweep_bytes(dim, n, cbc, True, 4)
    b_mv = sweep_bytes(dim, n, cbc, True, 8)
    peak, peak_kind = peaks()
    kernels = {
        "sweep_jacobi_f32": {"ms": ms_sweep, "bytes": b_sweep, "gbs": b_sweep / ms_sweep / 1e6,
                             "overhead_bytes": sweep_overhead_bytes(dim, n, True, 4)},
        "matvec_f64": {"ms": ms_mv, "bytes": b_mv, "gbs": b_mv / ms_mv / 1e6,
                       "overhead_bytes": sweep_overhead_bytes(dim, n, True, 8)},
        "galerkin_f32": {"ms": ms_gal},
    }
    for P in probs:
        P.close()
    # FP64 plain assemble-then-solve on the same workload
    _, d64 = workload_desc(mg, args.workload, mg.PATH_FP64_PLAIN)
    fp64_ms, fp64_cycles = [], []
    for _ in range(args.fp64_steps):
        with mg.Problem(d64) as P:
            barrier()
            t0 = time.perf_counter()
            inf = P.solve()
            fp64_ms.append((time.perf_counter() - t0) * 1e3)
            fp64_cycles.append(inf.cycles)
    # mixed assemble-then-solve at the same precision: separates the effect of
    # delayed assembly from that of FP32 smoothing and lossy storage
    _, dmp = workload_desc(mg, args.workload, mg.PATH_MIXED_PLAIN)
    mp_ms, mp_cycles, mp_asm = [], [], []
    for _ in range(args.fp64_steps):
        with mg.Problem(dmp) as P:
            barrier()
            t0 = time.perf_counter()
            inf = P.solve()
            mp_ms.append((time.perf_counter() - t0) * 1e3)
            mp_cycles.append(inf.cycles)
            mp_asm.append(float(inf.assembly_ms))
    # end to end through the C ABI with host buffers: create from the host
    # descriptor, solve, read u back to the host, destroy
    e2e_ms = []
    nvert = (n + 1) ** dim
    # the result lands in pinned host memory (the copy runs at the host link's speed)
    u_host = torch.empty(nvert, dtype=torch.float64, pin_memory=True).numpy()
    # one untimed step first, as the device loop has its warm-up steps: the
    # first creation of a problem of this footprint grows the device memory
    # pool (about 30 ms once per process; 3 ms per creation afterwards)
    for step in range(1 + max(1, args.e2e_steps)):
        barrier()
        t0 = time.perf_counter()
        with mg.Problem(workload_desc(mg, args.workload, mixed_path)[1]) as P:
            P.solve()
            P.solution(out=u_host)
        barrier()
        if step > 0:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_val = rep.aggregate(len(e2e_ms), max_over_ranks(sum(e2e_ms)))
    # the mixed path's solution under the FP64 operator of the final accuracy:
    # how far the lossy FP32 surplus storage moves the answer
    with mg.Problem(mg.problem_desc(w.dim, n, w.eps, path=mg.PATH_FP64_PLAIN, s_schedule=(w.s_final,),
                                    u0=u_host)) as P:
        P.assemble(w.s_final)
        rel_fp64_op = P.vcycle(0)
    serving = (serving_leg(mg, args.serving_requests, load_factors=(0.5, 0.7, 0.9))
               if args.serving_requests > 0 else None)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, sample, cores, _ = oracle_sample(args.workload, int(info0.cycles))
        cpu = {"value": v, "unit": "solves/s", "cores": cores,
               "kind": "oracle, extrapolated from 4000 sampled cells and a full 27^3 solve", "sample": sample}
    if rank != 0:
        return
    walls_sorted = sorted(walls)
    p50 = float(np.percentile(walls_sorted, 50))
    p99 = float(np.percentile(walls_sorted, 99))
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": region_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (fp8/fp16/fp32 surplus storage)",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {dim}D {n}^{dim} cells, {w.eps.n_boxes or w.eps.n_modes} "
                               f"{'boxes' if w.eps.n_boxes else 'modes'}, s={w.s_schedule}",
                   "path": "mixed delayed (FP32 V(2,2) + FP64 FCG)", "parallelism": f"replicas x{world}",
                   "flush": "working set > L2 (no flush)"},
        "p50_ms": p50, "p99_ms": p99,
        "cycles": int(info0.cycles), "publishes": int(info0.publishes), "rel_residual": info0.rel_residual,
        "rel_residual_fp64_operator": rel_fp64_op,
        "cells_by_class": cbc, "stencil_bytes": int(info0.payload_bytes),
        "fp64_plain": {"solves_per_s": 1e3 / statistics.median(fp64_ms), "ms": fp64_ms, "cycles": fp64_cycles},
        "speedup_vs_fp64_plain": statistics.median(fp64_ms) / p50,
        "mixed_plain": {"solves_per_s": 1e3 / statistics.median(mp_ms), "ms": mp_ms, "cycles": mp_cycles,
                        "assembly_ms": mp_asm},
        "delayed_vs_mixed_plain": statistics.median(mp_ms) / p50,
        "cycles_per_solve": [int(i.cycles) for i in infos],
        "roofline": {"bound": "hbm", "kernel": "sweep_jacobi_f32 (finest level, V-cycle smoother)",
                     "achieved": kernels["sweep_jacobi_f32"]["gbs"], "peak": peak, "unit": "GB/s",
                     "frac": kernels["sweep_jacobi_f32"]["gbs"] / peak, "peak_kind": peak_kind,
                     "traffic": sweep_traffic(args.workload) if n == 243 else None},
        "kernels": kernels,
        "e2e": {"value": e2e_val, "unit": "solves/s", "h2d_bytes_per_step": int(ctypes_sizeof_desc()),
                "d2h_bytes_per_step": int(nvert * 8)},
        "gpu_launches": int(launches),
        "clocks": ck,
        "cpu_baseline": cpu,
        "serving": serving,
    }
    print(json.dumps(line), flush=True)


def serving_leg(mg, n_requests, seed=2004, load_factors=(0.7,), max_active=8):
    """The request loop (configuration 'serving'): seeded requests of mixed
    sizes, each with its own lognormal eps, mixed delayed path to 1e-8.
    Closed loop first (all submitted at once: throughput), then open loop
    with Poisson arrivals at each load factor x that throughput; time-to-solution
    of a request runs from its submission to its completion (server clock)."""
    reqs = inputs.serving_requests(n_requests, seed=seed, rate_per_s=1.0)

    def desc(r):
        return mg.problem_desc(r["dim"], r["n_cells"], r["eps"], path=mg.PATH_MIXED_DELAYED,
                               s_schedule=(1, 2, 4, 8), rtol=1e-8, max_cycles=3000)

    def wait_all(S, tickets, res):
        while tickets:
            for t in list(tickets):
                st, r = S.poll(t)
                if st != mg.MG_ERR_PENDING:
                    res.append((st, r))
                    tickets.remove(t)
            time.sleep(0.0005)

    S = mg.Server(max_active=max_active)
    try:
        res = []
        t0 = time.perf_counter()
        tickets = [S.submit(desc(r)) for r in reqs]
        wait_all(S, tickets, res)
        closed_s = time.perf_counter() - t0
        thr = len(reqs) / closed_s
        ok_closed = sum(1 for st, _ in res if st == mg.MG_OK)
        open_loops = []
        for lf in load_factors:
            rate = lf * thr
            res2, tickets = [], []
            t0 = time.perf_counter()
            for r in reqs:
                due = t0 + r["arrival_s"] / rate
                while time.perf_counter() < due:
                    for t in list(tickets):
                        st, rr = S.poll(t)
                        if st != mg.MG_ERR_PENDING:
                            res2.append((st, rr))
                            tickets.remove(t)
                    time.sleep(0.0002)
                tickets.append(S.submit(desc(r)))
            wait_all(S, tickets, res2)
            open_s = time.perf_counter() - t0
            tts = sorted(r.total_ms for st, r in res2 if st == mg.MG_OK)
            open_loops.append({"load_factor": lf, "arrival_rate_per_s": rate, "solves_per_s": len(res2) / open_s,
                               "ok": len(tts), "p50_ms": float(np.percentile(tts, 50)) if tts else None,
                               "p99_ms": float(np.percentile(tts, 99)) if tts else None})
    finally:
        S.close()
    out = {"requests": len(reqs), "sizes": "uniform over 27^3, 81^3, 243^3 (3D) and 243^2, 729^2 (2D)",
           "eps": "lognormal, sigma ~ U[0.5, 2], 16 Fourier modes", "path": "mixed delayed, s = 1 -> 8, rtol 1e-8",
           "max_active": max_active,
           "closed_loop": {"solves_per_s": thr, "ok": ok_closed, "seconds": closed_s},
           "open_loop": next((o for o in open_loops if o["load_factor"] == 0.7), open_loops[0])}
    if len(open_loops) > 1:
        out["open_loop_by_load"] = open_loops
    return out


def run_probe(args, local_rank):
    """Small-case kernel probe for profilers: one problem of the workload at
    --n cells, assembled to its final accuracy, then `--probe-reps` launches
    of one kernel through mg_profile_kernel."""
    import torch
    from paper_2005_03606_gb300 import mg
    torch.cuda.set_device(local_rank)
    if args.probe == "serving":   # --probe-reps requests, open loop at 0.5, 0.7 and 0.9 of the closed-loop rate
        print(json.dumps({"probe": "serving", **serving_leg(mg, args.probe_reps, load_factors=(0.5, 0.7, 0.9))}),
              flush=True)
        return
    if args.probe == "oracle":   # the CPU oracle in full on configurations 1 and 2
        print(json.dumps({"probe": "oracle", "nproc": os.cpu_count(),
                          "rows": oracle_probe(["disc2d", "fourier3d"],
                                              ["disc2d"] + (["fourier3d"] if args.oracle_single_3d else []))}),
              flush=True)
        return
    if args.probe == "peaks":   # arithmetic pipe rates of this GPU (FP32 / FP64 FMA, FP32 exp)
        print(json.dumps({"probe": "peaks", "fp32_fma_per_s": mg.measure_peak(0),
                          "fp64_fma_per_s": mg.measure_peak(1), "fp32_exp_per_s": mg.measure_peak(2)}), flush=True)
        return
    if args.probe == "assembly":   # the integration kernel alone: eps samples per second
        w = inputs.workload(args.workload, args.n)
        path = mg.PATH_FP64_PLAIN if args.probe_fp64 else mg.PATH_MIXED_PLAIN
        d = mg.problem_desc(w.dim, w.n_cells, w.eps, path=path, s_schedule=(w.s_final,), rtol=1e-8)
        with mg.Problem(d) as P:
            ms = P.profile(4, args.probe_reps)
        # the first chunk of the default chunking (9 slabs from 27 cells per axis);
        # piecewise-constant fields integrate only its interface cells (count not reported)
        pc = w.eps.kind in (inputs.KIND_BOXES, inputs.KIND_DISC, inputs.KIND_CONST)
        ncell = w.n_cells ** w.dim // (9 if w.n_cells >= 27 else 1)
        samples = ncell * w.s_final ** w.dim
        print(json.dumps({"probe": "assembly", "workload": args.workload, "n_cells": w.n_cells, "fp64": args.probe_fp64,
                          "s": w.s_final, "cells": None if pc else int(ncell), "ms_per_launch": ms,
                          "samples_per_s": None if pc else samples / (ms * 1e-3)}), flush=True)
        return
    if args.probe == "transfer":   # finest Jacobi sweep pair, residual + restriction, restriction alone
        w = inputs.workload(args.workload, args.n)
        rows = []
        for fused in (True, False):
            if fused:
                os.environ["MG_FUSED_RESTRICT"] = "1"
            else:
                os.environ.pop("MG_FUSED_RESTRICT", None)
            d = mg.problem_desc(w.dim, w.n_cells, w.eps, path=mg.PATH_MIXED_PLAIN, s_schedule=(w.s_final,), rtol=1e-8)
            with mg.Problem(d) as P:
                P.assemble(w.s_final)
                rows.append({"fused": fused, "jacobi_ms": P.profile(0, args.probe_reps),
                             "resid_restrict_ms": P.profile(5, args.probe_reps),
                             "restrict_ms": P.profile(6, args.probe_reps),
                             "vcycle_ms": P.profile(7, args.probe_reps),
                             "vcycle_coarse_ms": P.profile(8, args.probe_reps),
                             "vcycle_coarse2_ms": P.profile(9, args.probe_reps)})
        os.environ.pop("MG_FUSED_RESTRICT", None)
        print(json.dumps({"probe": "transfer", "workload": args.workload, "n_cells": w.n_cells, "rows": rows}),
              flush=True)
        return
    if args.probe == "precision":   # storage classes of the lossy surplus against the bound tau
        # On piecewise-constant fields the FP64 outer residual applies the exact
        # operator, so tau only sets how closely the FP32 V-cycle's operator
        # follows it: larger bounds move cells to the FP8 / FP16 classes while
        # the solution still meets 1e-8 under the exact operator.
        w = inputs.workload(args.workload, args.n)
        rows = []
        for tau in (1e-6, 1e-4, 1e-3, 1e-2):
            d = mg.problem_desc(w.dim, w.n_cells, w.eps, path=mg.PATH_MIXED_DELAYED, s_schedule=tuple(w.s_schedule),
                                rtol=1e-8, max_cycles=3000, tau=tau)
            ms, cyc = [], []
            for _ in range(args.probe_reps):
                with mg.Problem(d) as P:
                    info = P.solve()
                ms.append(info.time_ms)
                cyc.append(info.cycles)
            rows.append({"tau": tau, "ms": ms, "cycles": cyc, "rel_residual": info.rel_residual,
                         "cells_by_class": [int(c) for c in info.cells_by_class],
                         "payload_bytes": int(info.payload_bytes)})
        print(json.dumps({"probe": "precision", "workload": args.workload, "n_cells": w.n_cells, "rows": rows}),
              flush=True)
        return
    if args.probe == "iteration":   # inner iteration with and without the host round trip
        w, d = workload_desc(mg, args.workload, mg.PATH_MIXED_PLAIN, n_cells=args.n)
        with mg.Problem(d) as P:
            P.solve()
            rows = {"back_to_back_ms": P.profile(10, args.probe_reps), "with_host_read_ms": P.profile(11, args.probe_reps)}
        print(json.dumps({"probe": "iteration", "workload": args.workload, "n_cells": w.n_cells, **rows}), flush=True)
        return
    if args.probe == "solve":   # whole mixed delayed solves, for launch lists
        w, d = workload_desc(mg, args.workload, mg.PATH_MIXED_DELAYED, n_cells=args.n)
        ms = []
        for _ in range(args.probe_reps):
            with mg.Problem(d) as P:
                t0 = time.perf_counter()
                info = P.solve()
                ms.append((time.perf_counter() - t0) * 1e3)
        print(json.dumps({"probe": "solve", "workload": args.workload, "n_cells": w.n_cells, "ms": ms,
                          "cycles": int(info.cycles), "publishes": int(info.publishes)}), flush=True)
        return
    if args.probe == "adaptive":   # adaptive per-cell accuracy (C = 1%) against the whole schedule
        w = inputs.workload(args.workload, args.n)
        rows = []
        for path, name in ((mg.PATH_MIXED_DELAYED, "mixed delayed"), (mg.PATH_MIXED_PLAIN, "mixed plain")):
            for C in (0.0, 0.01):
                sched = tuple(w.s_schedule) if (C > 0 or path == mg.PATH_MIXED_DELAYED) else (w.s_final,)
                d = mg.problem_desc(w.dim, w.n_cells, w.eps, path=path, s_schedule=sched, rtol=1e-8,
                                    max_cycles=3000, adapt_C=C)
                ms = []
                for _ in range(args.probe_reps):
                    with mg.Problem(d) as P:
                        t0 = time.perf_counter()
                        info = P.solve()
                        ms.append((time.perf_counter() - t0) * 1e3)
                        acc = P.cell_accuracy()
                # samples integrated per cell: every schedule level up to the cell's own
                walked = [sum(t ** w.dim for t in sched if 1 < t <= a) for a in (int(v) for v in np.unique(acc))]
                cnt = {int(v): int((acc == v).sum()) for v in np.unique(acc)}
                samples = sum(wk * cnt[a] for wk, a in zip(walked, sorted(cnt))) / acc.size
                rows.append({"path": name, "adapt_C": C, "ms": ms, "cycles": int(info.cycles),
                             "rel_residual": float(info.rel_residual), "cells_by_s": cnt,
                             "samples_per_cell": samples})
        print(json.dumps({"probe": "adaptive", "workload": args.workload, "n_cells": w.n_cells, "rows": rows}),
              flush=True)
        return
    if args.probe == "paper_format":   # Table "memory-footprint": accuracy and compression per cycle
        # 2D theta setup at h = 1/27, adaptive accuracy C = 1%, one accuracy level per
        # cycle, the paper's truncated format at an absolute 1e-8 on the surplus
        n = args.n or 27
        out = {}
        for theta, keep in ((1.0, 0), (16.0, 0), (64.0, 0), (1.0, 1), (16.0, 1), (64.0, 1)):
            d = mg.problem_desc(2, n, inputs.theta_field(2, theta), path=mg.PATH_FP64_PLAIN,
                                s_schedule=tuple(range(1, 9)), adapt_C=0.01, adapt_keep=keep)
            rows = []
            with mg.Problem(d) as P:
                for s in range(1, 11):
                    if s > 1:
                        P.assemble(s)
                    acc = P.cell_accuracy()
                    p3, _, st = P.paper_format(1e-8)
                    rows.append({"cycle": s, "max_n": int(acc.max()), "avg_n": float(acc.mean()),
                                 "compression": st["compression"], "cells_by_p3": st["cells_by_p3"],
                                 "max_abs_error": st["max_abs_error"]})
            out[f"theta={theta:g} {'keep-old' if keep else 'keep-new'}"] = rows
        print(json.dumps({"probe": "paper_format", "n_cells": n, "delta": 1e-8, "C": 0.01, "theta": out}),
              flush=True)
        return
    if args.probe == "cycles":   # the multiplicative V-cycle against the additive cycles of Section adaFAC-x
        w = inputs.workload(args.workload, args.n)
        names = {mg.CYCLE_V: "V(2,2)", mg.CYCLE_ADDITIVE: "additive", mg.CYCLE_ADAFAC_PI: "adaFAC-PI",
                 mg.CYCLE_ADAFAC_JAC: "adaFAC-Jac"}
        for path, pname in ((mg.PATH_MIXED_DELAYED, "mixed delayed"), (mg.PATH_FP64_PLAIN, "fp64 plain")):
            sched = tuple(w.s_schedule) if path == mg.PATH_MIXED_DELAYED else (w.s_final,)
            for outer, oname in ((mg.OUTER_FCG, "fcg"), (mg.OUTER_RICHARDSON, "richardson")):
                for cyc, cname in names.items():
                    d = mg.problem_desc(w.dim, w.n_cells, w.eps, path=path, s_schedule=sched, rtol=1e-8,
                                        max_cycles=args.max_cycles, outer=outer, cycle=cyc)
                    with mg.Problem(d) as P:
                        t0 = time.perf_counter()
                        info = P.solve(check=False)
                        ms = (time.perf_counter() - t0) * 1e3
                    print(json.dumps({"probe": "cycles", "workload": args.workload, "n_cells": w.n_cells,
                                      "path": pname, "outer": oname, "cycle": cname, "status": int(info.status),
                                      "cycles": int(info.cycles), "ms": ms,
                                      "rel_residual": float(info.rel_residual)}), flush=True)
        return
    if args.probe == "coarse":   # compressed coarse-level operators against full FP32 ones
        w = inputs.workload(args.workload, args.n)
        rec = {2: (0, 16, 16, 32), 3: (0, 32, 64, 112)}[w.dim]
        np_ = 6 if w.dim == 2 else 28
        for tau in (0.0, 1e-6):
            d = mg.problem_desc(w.dim, w.n_cells, w.eps, path=mg.PATH_MIXED_DELAYED, s_schedule=tuple(w.s_schedule),
                                rtol=1e-8, max_cycles=3000, coarse_tau=tau)
            ms = []
            for _ in range(args.probe_reps):
                with mg.Problem(d) as P:
                    t0 = time.perf_counter()
                    info = P.solve()
                    ms.append((time.perf_counter() - t0) * 1e3)
                    levels = []
                    if tau > 0:
                        l, nl = 1, w.n_cells // 3
                        while nl >= 3:
                            cls = P.coarse_classes(l)
                            cnt = [int((cls == k).sum()) for k in range(4)]
                            levels.append({"level": l, "cells": int(cls.size), "cells_by_class": cnt,
                                           "bytes_full": int(cls.size) * np_ * 4,
                                           "bytes_stored": int(sum(c * (5 + rec[k]) for k, c in enumerate(cnt)))})
                            l, nl = l + 1, nl // 3
            print(json.dumps({"probe": "coarse", "workload": args.workload, "n_cells": w.n_cells, "coarse_tau": tau,
                              "ms": ms, "cycles": int(info.cycles), "rel_residual": float(info.rel_residual),
                              "levels": levels}), flush=True)
        return
    if args.probe == "paths":   # time-to-solution of the four paths on one workload
        names = {mg.PATH_MIXED_DELAYED: "mixed delayed", mg.PATH_MIXED_PLAIN: "mixed plain",
                 mg.PATH_FP64_DELAYED: "fp64 delayed", mg.PATH_FP64_PLAIN: "fp64 plain"}
        for path, name in names.items():
            w, d = workload_desc(mg, args.workload, path, n_cells=args.n)
            runs = []
            for _ in range(args.probe_reps):
                with mg.Problem(d) as P:
                    t0 = time.perf_counter()
                    info = P.solve()
                    runs.append({"ms": (time.perf_counter() - t0) * 1e3, "cycles": int(info.cycles),
                                 "publishes": int(info.publishes), "rel_residual": float(info.rel_residual),
                                 "assembly_ms": float(info.assembly_ms)})
            print(json.dumps({"probe": "paths", "workload": args.workload, "n_cells": w.n_cells, "path": name,
                              "runs": runs}), flush=True)
        return
    if args.probe == "starvation":   # per-iteration residual and pending assembly jobs
        # 2D 243^2 (59,049 unknowns), eps in {1e-5, 1}: disc of radius 0.3
        fld = inputs.disc_field(2, v_in=1e-5, v_out=1.0)
        n = args.n or 243
        out = {}
        for path, name in ((mg.PATH_FP64_PLAIN, "fp64 precomputed"), (mg.PATH_FP64_DELAYED, "fp64 delayed"),
                           (mg.PATH_MIXED_DELAYED, "mixed delayed")):
            sched = (8,) if path == mg.PATH_FP64_PLAIN else (1, 2, 4, 8)
            d = mg.problem_desc(2, n, fld, path=path, s_schedule=sched, rtol=1e-10, max_cycles=3000)
            with mg.Problem(d) as P:
                info = P.solve()
                tr = P.trace()
            out[name] = {"cycles": int(info.cycles), "publishes": int(info.publishes),
                         "rel_residual": float(info.rel_residual),
                         "trace": [[t["cycle"], round(t["rel_residual_est"], 14), t["pending_jobs"],
                                    round(t["time_ms"], 3)] for t in tr]}
        print(json.dumps({"probe": "starvation", "n_cells": n, "eps": "disc r=0.3, 1e-5 inside, 1 outside",
                          "trace_fields": ["cycle", "rel_residual_est", "pending_jobs", "ms"], "paths": out}),
              flush=True)
        return
    which = {"sweep": 0, "matvec": 1, "residual": 2, "galerkin": 3}[args.probe]
    path = mg.PATH_FP64_PLAIN if args.probe_fp64 else mg.PATH_MIXED_PLAIN
    w, d = workload_desc(mg, args.workload, path, n_cells=args.n)
    with mg.Problem(d) as P:
        P.assemble(w.s_final)
        ms = P.profile(which, args.probe_reps)
    print(json.dumps({"probe": args.probe, "workload": args.workload, "n_cells": w.n_cells, "fp64": args.probe_fp64,
                      "ms_per_launch": ms}), flush=True)


def ctypes_sizeof_desc():
    import ctypes
    from paper_2005_03606_gb300 import mg
    return ctypes.sizeof(mg.mg_problem_desc)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="boxes3d", choices=["boxes3d", "fourier3d", "jump3d", "disc2d"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--ref-cycles", type=int, default=140,
                    help="cycle count used to scale the oracle sample in --impl reference: the FP64 "
                         "assemble-then-solve iteration the oracle runs needs 140 cycles on boxes3d 243^3")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=512,
                    help="requests of the serving leg (0: skip)")
    ap.add_argument("--probe", choices=["oracle", "peaks", "assembly", "transfer", "iteration", "precision", "sweep", "matvec", "residual", "galerkin", "solve", "serving",
                                        "adaptive", "starvation", "paths", "paper_format", "cycles", "coarse"],
                    help="profile one kernel on a small case instead of benchmarking")
    ap.add_argument("--probe-fp64", action="store_true", help="probe the FP64 plain path's kernel")
    ap.add_argument("--probe-reps", type=int, default=3)
    ap.add_argument("--oracle-single-3d", action="store_true",
                    help="--probe oracle: also time the 81^3 workload on one thread (several minutes)")
    ap.add_argument("--max-cycles", type=int, default=600, help="cycle limit of --probe cycles")
    ap.add_argument("--n", type=int, default=None, help="cells per axis for --probe")
    args = ap.parse_args()
    if args.probe:
        run_probe(args, int(os.environ.get("LOCAL_RANK", "0")))
        return
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
