"""Benchmark of the RAFEM time step on one B300: time-steps/s at 2.1M DoF per system, FP64 and mixed.

Workload: the 127^3-cell cube (2,097,152 nodes, 12,290,298 P1 tetrahedra, 31,065,598 nonzeros per system),
interior jitter +-10% of the cell width, lognormal sigma0 (mean 0.333 S/m, 10% CV), dt = 1 s, relative
residual 1e-10, Jacobi preconditioning. A step is one backward-Euler step: assemble A_V(sigma(T)) and its
lifted rhs, solve V, assemble the thermal rhs (Joule + mass term), solve T, all in one CUDA graph.
Inputs are synthetic (seeded) and resident in HBM before the timed region; each step streams both
matrices (373 MB each in FP64) and the element data, far more than the 126 MB L2.

The headline `value` is the mixed-precision form (FP32 inner Krylov, FP64 refinement to the same 1e-10 FP64
residual); the FP64 path is reported beside it in `fp64`, with the mixed-vs-FP64 field error and PSNR.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl rafem|reference]
Prints one JSON line (rank 0).
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

METRIC = "time-steps/s at 2.1M DoF (FP64 vs mixed vs oracle); SpMV HBM GB/s vs peak"
UNIT = "time-steps/s"
WORKLOAD = ("RAFEM cube 127^3 cells, 2,097,152 nodes, 12,290,298 P1 tets, 31,065,598 nnz per system; jitter 10%, "
            "lognormal sigma0; dt=1 s; Jacobi-PCG to FP64 relative residual 1e-10; steps W+1..W+K of the 900-step "
            "run")
ORACLE_SAMPLE_N = 24          # oracle sample: the same workload family on a 24^3-cell cube (15,625 nodes)
ORACLE_SAMPLE_STEPS = 5


def reduce_over_ranks(values, op, dist):
    """All-reduce a few floats over the ranks ('max' or 'sum'), on the device the process group's backend uses
    (CUDA tensors for NCCL, host tensors for gloo). Without a process group the values come back unchanged."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return [float(v) for v in t.cpu()]


def aggregate_rate(units_per_rank, ms_per_rank_max):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time (ms)."""
    return units_per_rank / (ms_per_rank_max * 1e-3)


def partition_instances(costs, world):
    """Balanced split of independent instances over `world` ranks: longest processing time first (largest cost to
    the least loaded rank, ties to the lower rank), deterministic on every rank. Returns one index list per rank,
    each in increasing order."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def _measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


def _oracle_sample(n: int, steps: int) -> dict:
    """Time the FP64 oracle (dense/sparse direct LU, one thread) on steps of an n^3 instance."""
    from oracle import rafem_oracle as O
    from paper_2409_13036_b300 import meshgen as mg
    import numpy as np
    m = mg.cube_mesh(n, jitter=0.10, seed=mg.SEED_BASE + 2, sigma0="lognormal")
    model = O.Model(m)
    T = np.full(m.n_nodes, 37.0)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        T, V, _ = model.step(T)
        times.append(time.perf_counter() - t0)
    return {"n": n, "nodes": m.n_nodes, "times": times}


def _host_info() -> dict:
    """The host the CPU baseline ran on: logical CPUs and the CPU model (Linux /proc/cpuinfo)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "oracle_threads": 1}


def _oracle_stream(which: str, steps: int) -> None:
    """Time the FP64 oracle on one of the named workloads, printing one JSON line per phase as it completes (the
    parent may stop the child after any line): the set-up (mesh-constant geometry, mass and thermal matrices),
    then each time step (the first also factors the constant thermal matrix, kept for the later steps)."""
    from oracle import rafem_oracle as O
    from paper_2409_13036_b300 import meshgen as mg
    import numpy as np
    m = mg.workload_48() if which == "c2_48" else mg.workload_single_step_8()
    t0 = time.perf_counter()
    model = O.Model(m)
    print(json.dumps({"phase": "setup", "s": time.perf_counter() - t0, "nodes": m.n_nodes}), flush=True)
    T = np.full(m.n_nodes, 37.0)
    for k in range(steps):
        t0 = time.perf_counter()
        T, V, _ = model.step(T)
        print(json.dumps({"phase": "step", "k": k + 1, "s": time.perf_counter() - t0}), flush=True)


class OracleTimer:
    """The oracle timed in a child process (one thread, spawned by exec: no CUDA state is inherited) while the
    parent runs its GPU legs; lines are collected by a reader thread."""

    def __init__(self, which: str, steps: int):
        import threading
        env = dict(os.environ)
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[k] = "1"
        env["CUDA_VISIBLE_DEVICES"] = ""
        code = ("import sys; sys.path.insert(0, %r); import bench; bench._oracle_stream(%r, %d)"
                % (ROOT, which, steps))
        self.which, self.steps = which, steps
        self.t_start = time.perf_counter()
        self.proc = subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                                     stderr=subprocess.DEVNULL, text=True, env=env, cwd=ROOT)
        self.lines = []
        self.reader = threading.Thread(target=self._read, daemon=True)
        self.reader.start()

    def _read(self):
        for line in self.proc.stdout:
            try:
                self.lines.append(json.loads(line))
            except ValueError:
                pass

    def finish(self, min_steps: int, max_wait_s: float) -> dict:
        """Wait until min_steps steps are timed (or the child ends, or max_wait_s since the start), then stop it."""
        while True:
            done = sum(1 for x in self.lines if x.get("phase") == "step")
            if done >= min_steps or self.proc.poll() is not None:
                break
            if time.perf_counter() - self.t_start > max_wait_s:
                break
            time.sleep(0.5)
        if self.proc.poll() is None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=10)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.proc.wait()
        self.reader.join(timeout=5)
        setup = next((x for x in self.lines if x.get("phase") == "setup"), None)
        steps = [x["s"] for x in self.lines if x.get("phase") == "step"]
        return {"setup_s": setup["s"] if setup else None, "nodes": setup["nodes"] if setup else None,
                "step_s": steps}


def run_oracle_subprocess(n: int, steps: int) -> dict:
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench._oracle_sample(%d, %d)))" % (ROOT, n, steps))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = ""

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self) -> dict:
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k, v in enumerate(r[3]) if v.lower().startswith("active")})
        loaded = [r[0] for r in rows if r[2] > 200.0] or [r[0] for r in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


def _source_hash(path: str) -> str:
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def _ncu_traffic(kernel: str):
    """DRAM bytes per iteration of `kernel` from the committed ncu summary, if taken on the current source."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        e = json.load(f).get(kernel)
    if not e:
        return None
    # every source file the kernel is built from must be unchanged since the capture
    for name, sha in zip(e.get("sources", [e.get("source")]), e.get("sources_sha256", [e.get("source_sha256")])):
        if not name or _source_hash(os.path.join(ROOT, "paper_2409_13036_b300", "csrc", name)) != sha:
            return None
    return e


def alg_bytes_cg64(N: int, nnz: int, iters: float, col_bytes: int, given_r0: bool = True) -> float:
    """Algorithmic HBM bytes of one FP64 Chronopoulos-Gear Jacobi-PCG solve launch (stored format).
    Per iteration: SpMV w = A u streams (8 + col_bytes) B per nonzero (value + column index) and reads u once and
    writes w (16N); the vector phase reads u, w, p, s, x, r, dinv and writes p, s, x, r, u (96N). Start-up
    (r = b - Ax, u, w = Au) and the final true-residual SpMV add two more iterations' worth. given_r0: the
    projection predictor handed over the starting residual (every step with history), so the start-up reads it
    (8N, in place of the x gather) instead of streaming the matrix."""
    per_iter = (8 + col_bytes) * nnz + 16 * N + 96 * N
    return (iters + 2) * per_iter - (given_r0 * (8 + col_bytes) * nnz)


def alg_bytes_pipecg(N: int, nnz: int, iters: float, col_bytes: int) -> float:
    """Algorithmic HBM bytes of one FP64 pipelined Jacobi-PCG solve launch (stored format).
    Per iteration: SpMV n = A m streams (8 + col_bytes) B per nonzero and gathers m once (8N); the fused row
    epilogue reads m, w, u, z, q, s, p, x, r, dinv and writes z, q, s, p, x, r, u, w and the next m (152N).
    Start-up (r = b - Ax and u; w = Au and m) and the final true-residual SpMV add three iterations' worth."""
    per_iter = (8 + col_bytes) * nnz + 160 * N
    return (iters + 3) * per_iter


def alg_bytes_mixed(N: int, nnz: int, iters: float, refinements: float, col_bytes: int,
                    given_r0: bool = True) -> float:
    """Algorithmic HBM bytes of one mixed-precision solve launch (stored format).
    Inner FP32 iteration: SpMV (4 + col_bytes) B per nonzero + 8N (u read, w written); vector phase 12 x 4N.
    Each FP64 refinement: x64 += d32 (8N + 4N read, 8N written), the FP64 residual SpMV ((8 + col_bytes) B per
    nonzero + 8N x + 8N b) writing r32, u32, d32 (12N) and reading dinv32 (4N), and the FP32 start SpMV
    ((4 + col_bytes) B per nonzero + 8N). given_r0: the first residual was handed over by the projection
    predictor (every step with history) and is read (8N, in place of the x gather) instead of computed."""
    inner = (4 + col_bytes) * nnz + 8 * N + 48 * N
    outer = (20 * N) + ((8 + col_bytes) * nnz + 16 * N + 16 * N) + ((4 + col_bytes) * nnz + 8 * N)
    return iters * inner + (refinements + 1) * outer - (given_r0 * (8 + col_bytes) * nnz)


def alg_bytes_ilu(Np: int, nnz_p: int, iters: float, nf: int | None = None, cb: int = 4, mixed: bool = False,
                  refinements: float = 0.0) -> float:
    """Algorithmic HBM bytes of one ILU(0)-PCG solve launch on the ring layouts: P A P^T (nnz_p stored entries) and
    the strictly lower and upper factors (nf entries together; about nnz_p - Np when not given), each entry a value
    plus cb column bytes (0 with shared slice patterns).
    FP64: per iteration phase A streams A and reads z and p, q and writes p, q; phase B reads x, p, q, r and writes x,
    r (and z on level-0 rows); the level sweeps stream L and U once and read r, z, 1/u_ii and write z: ~16 vector
    accesses of 8 B per row. Start-up (gather, residual, first preconditioning) and the final true residual add about
    two iterations' worth.
    Mixed: the inner iteration the same in FP32 (values and vectors of 4 B: ~16 accesses of 4 B per row); each FP64
    refinement streams A in FP64 ((8 + cb) nnz_p), reads b and gathers x and writes r, d, z in FP32 (~28 B per row),
    then adds d to x (20 B per row)."""
    if nf is None:
        nf = max(nnz_p - Np, 0)
    if not mixed:
        per_iter = (8 + cb) * (nnz_p + nf) + 128 * Np
        return (iters + 2) * per_iter
    inner = (4 + cb) * (nnz_p + nf) + 64 * Np
    outer = (8 + cb) * nnz_p + 28 * Np + 20 * Np
    return iters * inner + (refinements + 1) * outer + (4 + cb) * nf + 32 * Np


def alg_bytes_bicgstab(N: int, nnz: int, iters: float, col_bytes: int) -> float:
    """Algorithmic HBM bytes of one Jacobi-BiCGSTAB solve launch (SELL-32 primary storage): two SpMVs per
    iteration ((8 + col_bytes) B per stored entry each, plus the gathered vector read and the product written, 16N)
    and the row-local phases (A: 5 reads + 2 writes, B: 1 read, C: 3 reads + 2 writes, D: 1 read, E: 7 reads +
    2 writes of 8N = 168N). Start-up and the final true residual add about one iteration's worth."""
    per_iter = 2 * ((8 + col_bytes) * nnz + 16 * N) + 168 * N
    return (iters + 1) * per_iter


def alg_bytes_gmres(N: int, nnz: int, steps: float, cycles: float, col_bytes: int, m: int = 30) -> float:
    """Algorithmic HBM bytes of one GMRES(m) solve launch (single-pass Gram-Schmidt, the second pass being taken
    only when the first cancels more than 99% of the vector's squared norm, which on these systems never happens): per Arnoldi step j an SpMV ((8 + col_bytes) B
    per stored entry, plus u and dinv gathered and v_j, w written: 32N), the dots pass (w and the j + 1 basis vectors
    read) and the update pass (the j + 1 basis vectors read, w read and written); the last step of a cycle skips the
    update. Per cycle the residual SpMV ((8 + col_bytes) nnz + 24N) and the update of x (k + 2 vectors). j averages
    about half the steps per cycle."""
    cycles = max(cycles, 1.0)
    steps_per_cycle = steps / cycles
    j_avg = (steps_per_cycle - 1) / 2.0
    per_step = (8 + col_bytes) * nnz + 32 * N + (j_avg + 2) * 8 * N + (j_avg + 3) * 8 * N
    per_cycle = (8 + col_bytes) * nnz + 24 * N + (steps_per_cycle + 2) * 8 * N - (steps_per_cycle * 8 * N + 16 * N)
    return steps * per_step + cycles * per_cycle


def alg_fma_gmres(N: int, nnz: int, steps: float, cycles: float) -> float:
    """FP64 operations of one GMRES(m) solve launch. The Gram-Schmidt dots and updates and the update of x run in
    double-word arithmetic on the FP32 pipes (the basis is stored as float pairs), so the FP64 pipe carries per
    Arnoldi step one FMA per stored entry (SpMV) and ~5 per row (scaling of w and of the new basis vector, (w, w),
    the double-word to FP64 rounding of w, the Jacobi scaling), and per cycle the residual SpMV and ~2 per row."""
    cycles = max(cycles, 1.0)
    return steps * (nnz + 5 * N) + cycles * (nnz + 2 * N)


def fp64_pipe_line(fma: float, solve_ms: float) -> dict:
    """FP64 FMA rate of a launch against the FP64 pipe: B300 retires 2 FP64 FMAs per clock per SM (148 SMs at
    2.032 GHz: 0.60 TFMA/s)."""
    peak_fma = 148 * 2 * 2.032e9
    return {"bound": "alu", "achieved": fma / (solve_ms * 1e-3) / 1e12, "peak": peak_fma / 1e12,
            "unit": "TFMA/s (FP64)", "frac": fma / (solve_ms * 1e-3) / peak_fma,
            "peak_kind": "2 FP64 FMA/clk/SM x 148 SMs x 2.032 GHz (unit count and clock)"}


def cpu_baseline_line(t: dict, c1: dict | None, small: dict | None) -> dict:
    """The cpu_baseline object: the oracle's steps/s on the 48^3 workload (117,649 nodes, jitter 10%, 60 steps at
    dt = 1 s to relative residual 1e-10 in its configuration) from the steps timed, with the 60-step run
    extrapolated, the 8^3 single-step workload beside it, and the GPU's steps/s on the same 48^3 workload."""
    steps = t["step_s"]
    if not steps:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "host": _host_info(),
                "sample": "the 48^3 oracle timing did not complete a step within the wait", "c1_8": c1}
    later = steps[1:] or steps
    value = len(later) / sum(later)
    run60 = (t["setup_s"] or 0.0) + steps[0] + 59 * (sum(later) / len(later))
    out = {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "host": _host_info(),
           "config": "48^3 cells, 117,649 nodes, 663,552 tets, jitter 10% (the 60-step FP64 workload)",
           "sample": (f"FP64 oracle (own assembly + SuperLU direct solves, 1 thread) on the 48^3 workload: set-up "
                      f"and the first {len(steps)} steps timed; value = steps/s over steps 2..{len(steps)} (step 1 "
                      f"also factors the constant thermal matrix); the 60-step run extrapolated as set-up + step 1 "
                      f"+ 59 x the mean later step"),
           "setup_s": t["setup_s"], "step_s": steps, "extrapolated_60_step_run_s": run60}
    if c1:
        out["c1_8"] = c1
    if small and "fp64_cg" in small:
        out["gpu_same_config_steps_per_s"] = {k: small[k]["steps_per_s"] for k in ("fp64_cg", "mixed")
                                              if k in small}
    return out


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = ORACLE_SAMPLE_N
    res = run_oracle_subprocess(n, args.warmup + args.steps)
    t = res["times"][args.warmup:]
    value = len(t) / sum(t)
    sample = (f"FP64 oracle (own assembly + SuperLU direct solve, 1 thread) on the same workload family at "
              f"{n}^3 cells ({res['nodes']} nodes): {len(t)} timed steps after {args.warmup} warm-up; "
              f"the direct LU does not finish at 127^3")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(t) / len(t),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "oracle_sample_cells": n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "host": _host_info()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def measure(rafem, torch, mesh, precision, args, local, dist, want_clocks, precond=0, solver=0, **extra):
    """Warm up, time K steps with CUDA events on the context's stream, then a few traced steps."""
    stream = torch.cuda.Stream()
    ctx = rafem.Context(mesh, stream=stream.cuda_stream, precision=precision, precond=precond, solver=solver,
                        **extra)
    N, nnz, n_colors = ctx.pattern_info()
    layout = ctx.layout_info()
    if precond == rafem.RAFEM_PRECOND_ILU0:
        info = ctx.precond_info()
        layout["ilu"] = {"levels": info["n_levels"], "padded_rows": info["padded_rows"],
                         "factor_stored": info["factor_stored"], "column_bytes": info["column_bytes"],
                         "nnz_stored": info["nnz_stored"]}
    s, st = ctx.run(args.warmup)
    if s < 0:
        raise RuntimeError(f"warm-up failed: {rafem.status_string(s)}")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local) if want_clocks else None
    if clk:
        clk.__enter__()
    ev0.record(stream)
    s, st = ctx.run(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    if clk:
        clk.__exit__()
    if dist:
        dist.barrier()
    ms = reduce_over_ranks([ev0.elapsed_time(ev1)], "max", dist)[0]
    fields = (ctx.get_field(rafem.RAFEM_SYS_T), ctx.get_field(rafem.RAFEM_SYS_V))
    graph = ctx.graph_info()
    # region split and iteration counts of the same K steps: replayed from the initial state with tracing on (the
    # traced launches are identical; tracing only adds an event and a synchronisation between regions)
    ctx.reset()
    ctx.run(args.warmup)
    ctx.set_tracing(True)
    ctx.run(args.steps)
    tr = ctx.get_trace()
    ctx.set_tracing(False)
    return {"ctx": ctx, "ms": ms, "status": rafem.status_string(s), "last": st.as_dict(), "trace": tr,
            "fields": fields, "N": N, "nnz": nnz, "n_colors": n_colors, "layout": layout, "graph": graph,
            "clocks": clk.summary() if clk else None}


def roofline(res, mixed, peaks, peak_kind):
    tr = res["trace"]
    N, nnz = res["N"], res["nnz"]
    steps = tr["steps"]
    solve_ms = tr["ms_solve_V"] / steps
    iters = tr["iters_V"] / steps
    code = res["layout"]["kernel_code"]
    # kernel code 3: the ring solvers (CG family, BiCGSTAB, GMRES) stream no per-entry columns (one column pattern
    # per slice)
    cb_cg = 0 if code == 3 else res["layout"]["column_bytes"]
    cb = res["layout"]["column_bytes"]
    if res.get("solver") == "gmres":
        ref = tr["refine_V"] / steps
        alg = alg_bytes_gmres(N, nnz, iters, ref, cb_cg)
        kern = "k_gmres"
    elif res.get("solver") == "pipecg":
        ref = 0.0
        alg = alg_bytes_pipecg(N, nnz, iters, cb_cg)
        kern = f"k_pcg64<{code}>"
    elif res.get("solver") == "bicgstab":
        ref = 0.0
        alg = alg_bytes_bicgstab(N, nnz, iters, cb_cg)
        kern = "k_bicgstab"
    elif "ilu" in res["layout"]:
        ref = 0.0
        il = res["layout"]["ilu"]
        ref = tr["refine_V"] / steps if mixed else 0.0
        alg = alg_bytes_ilu(il["padded_rows"], il["nnz_stored"], iters, il["factor_stored"], il["column_bytes"], mixed,
                            ref)
        kern = "k_ilu_ring<mixed>" if mixed else "k_ilu_ring<fp64>"
    elif mixed:
        ref = tr["refine_V"] / steps
        alg = alg_bytes_mixed(N, nnz, iters, ref, cb_cg)
        kern = f"k_cg_mixed<{code}>"
    else:
        ref = 0.0
        alg = alg_bytes_cg64(N, nnz, iters, cb_cg)
        kern = f"k_cg64<{code}>"
    achieved = alg / (solve_ms * 1e-3) / 1e9
    fp64_pipe = None
    if kern.startswith("k_cg64"):
        # the FP64 solver is co-limited by the FP64 pipe: per iteration one FMA per stored entry (SpMV) and ~10 per
        # row (vector phase)
        fp64_pipe = fp64_pipe_line((iters + 2) * (res["layout"]["nnz_stored"] + 10 * N), solve_ms)
    elif kern == "k_gmres":
        # GMRES's FP64 work: its SpMVs and a few operations per row (Gram-Schmidt runs on the FP32 pipes)
        fp64_pipe = fp64_pipe_line(alg_fma_gmres(N, res["layout"]["nnz_stored"], iters, ref), solve_ms)
    nc = _ncu_traffic(kern)
    traffic = None
    if nc:
        # DRAM bytes of one ncu capture (smaller case of the same workload), scaled by algorithmic bytes
        traffic = nc["dram_per_alg_byte"] * alg
    dram = traffic / (solve_ms * 1e-3) / 1e9 if traffic else None
    return {"bound": "hbm", "kernel": f"{kern} (potential-system persistent solver, one launch per step)",
            "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
            "peak_kind": ("measured copy bandwidth, MEASURED_PEAKS.json hbm_gbs (of measured)"
                          if peak_kind == "measured" else "fallback 6.4 TB/s (of fallback)"),
            "traffic": traffic,
            "dram_achieved": dram, "dram_frac": dram / peaks["hbm_gbs"] if dram else None,
            "traffic_note": ("ncu DRAM read+write of the 112^3 capture scaled by algorithmic bytes" if traffic else
                             "no ncu capture for the current source"),
            "launch_ms": solve_ms, "iters_per_launch": iters, "refinements_per_launch": ref,
            "alg_bytes_per_launch": alg, **({"fp64_pipe": fp64_pipe} if fp64_pipe else {})}


def measure_batch(rafem, torch, mg, args, dist=None):
    """Batching form: the 96-instance workload (sizes 12^3..64^3 cells, electrode 10-40 V at 10-30 mm, sigma0
    0.25-0.45 S/m, seeded) in one context per precision, schedule from the autotuner, against one context per
    instance run one after the other (FP64). Throughput in instance-steps per second. Under several ranks the
    instances are split by node count (partition_instances; no collective on the data path) and the rates are
    aggregated over the slowest rank."""
    from paper_2409_13036_b300.autotune import autotune_schedule
    draws = mg.batch_draws()
    world = dist.get_world_size() if dist else 1
    rank = dist.get_rank() if dist else 0
    mine = partition_instances([(d[0] + 1) ** 3 for d in draws], world)[rank]
    meshes = [mg.batch_mesh(draws[i]) for i in mine]
    nodes = sum(m.n_nodes for m in meshes)
    kb = args.batch_steps
    out = {"instances": len(draws), "instances_this_rank": len(meshes), "nodes_this_rank": nodes, "steps": kb,
           "warmup": 3, "partition": "by instance, node-count balanced (largest first)" if world > 1 else "single"}
    stream = torch.cuda.Stream()
    for name, prec in (("mixed", rafem.RAFEM_PRECISION_MIXED), ("fp64", rafem.RAFEM_PRECISION_FP64)):
        ctx = rafem.Context.batch(meshes, stream=stream.cuda_stream, precision=prec)
        T0, V0 = ctx.get_field(rafem.RAFEM_SYS_T), ctx.get_field(rafem.RAFEM_SYS_V)
        tune = autotune_schedule(ctx, steps=2)
        ctx.set_state(T=T0, V=V0, step=0)  # back to the initial state: same trajectory as the sequential runs
        ctx.run(3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s, st = ctx.run(kb)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = reduce_over_ranks([e0.elapsed_time(e1)], "max", dist)[0]
        per = ctx.batch_stats()
        out[name] = {"instance_steps_per_s": aggregate_rate(len(draws) * kb, ms), "ms_per_step": ms / kb,
                     "status": rafem.status_string(s), "rows_per_tile": tune["rows_per_tile"],
                     "tuned_from_cache": tune["cached"],
                     "iters_V_min_max": [min(q["iters_V"] for q in per), max(q["iters_V"] for q in per)]}
        ctx.close()
    # the same instances one context at a time, FP64
    total_ms = 0.0
    for m in meshes:
        ctx = rafem.Context(m, stream=stream.cuda_stream, precision=rafem.RAFEM_PRECISION_FP64)
        ctx.run(3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        ctx.run(kb)
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
        ctx.close()
    total_ms = reduce_over_ranks([total_ms], "max", dist)[0]
    out["sequential_fp64"] = {"instance_steps_per_s": aggregate_rate(len(draws) * kb, total_ms),
                              "ms_per_step_all_instances": total_ms / kb}
    out["speedup_mixed_batch_vs_sequential_fp64"] = (out["mixed"]["instance_steps_per_s"] /
                                                     out["sequential_fp64"]["instance_steps_per_s"])
    return out


def measure_adjoint(rafem, torch, mg, args):
    """Differentiation form on the 64^3-cell workload (274,625 nodes): loss = |T^N - T_target|^2 after N steps,
    with T_target from the same forward model run with the hidden two-region sigma0 (tumour sphere, 0.5 S/m
    inside 0.333 S/m liver). Parameters are FP32 tensors (uniform liver sigma0 and k); the gradient comes from
    the torch.autograd bridge (rafem_tape_begin + rafem_adjoint, checkpoint every 10 steps). Central differences
    (relative step 1e-6, FP64 parameters) on 32 seeded random elements check dL/dsigma0."""
    import numpy as np
    from paper_2409_13036_b300.adjoint import final_temperature
    n_steps, every, n_fd = args.adjoint_steps, 10, args.fd_elements
    mesh = mg.cube_mesh(64, jitter=0.10, seed=mg.SEED_BASE + 4)
    dev = torch.device("cuda")
    ctx = rafem.Context(mesh, tol=1e-13)
    # target field: the same forward model with the hidden tumour conductivity
    ctx.set_params(mg.tumour_sigma0(mesh), mesh.k)
    ctx.reset()
    ctx.run(n_steps)
    target = torch.empty(mesh.n_nodes, dtype=torch.float64, device=dev)
    ctx.get_field_device(rafem.RAFEM_SYS_T, target)
    s0 = torch.tensor(mesh.sigma0, dtype=torch.float32, device=dev, requires_grad=True)
    kk = torch.tensor(mesh.k, dtype=torch.float32, device=dev, requires_grad=True)
    # warm-up: one full forward + backward (graph capture, checkpoint and adjoint workspace, lazy module loads)
    ((final_temperature(ctx, s0, kk, n_steps, checkpoint_every=every) - target) ** 2).sum().backward()
    s0.grad = None
    kk.grad = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    T = final_temperature(ctx, s0, kk, n_steps, checkpoint_every=every)
    loss = ((T - target) ** 2).sum()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    adj = T.grad_fn.adjoint_stats if hasattr(T.grad_fn, "adjoint_stats") else {}
    g = s0.grad.double().cpu().numpy()
    # central differences on seeded random elements, FP64 parameters at the FP32-rounded values
    base_s = s0.detach().double().cpu().numpy()
    base_k = kk.detach().double().cpu().numpy()
    tgt = target.cpu().numpy()
    rng = np.random.default_rng(mg.SEED_BASE + 5)
    elems = rng.choice(mesh.n_tets, size=n_fd, replace=False)

    # central differences of the forward model solved as smoothly as possible in the parameters: tolerance 1e-13,
    # each solve started from the previous step's solution (no extrapolation) so that both perturbed runs follow
    # the same iteration paths, and FP64 element passes (the double-word passes round at 2^-48, which the
    # difference quotient divides by eps)
    ctx.close()
    ctx = rafem.Context(mesh, tol=1e-13, predictor=0, arith=rafem.RAFEM_ARITH_FP64)

    def fd_at(eps, ctx=ctx):
        # Two forms of the same quotient. "loss difference" subtracts the two losses (each ~1e5, so their
        # difference of ~1e-6 loses everything below the rounding of a 274,625-term FP64 sum, ~1e-10);
        # "field difference" forms L+ - L- = sum_i (T+_i - T-_i)(T+_i + T-_i - 2 T*_i) node by node, which is
        # the same number without that cancellation. The gap between the two is the loss-rounding noise floor.
        fd, fd_loss = np.empty(n_fd), np.empty(n_fd)
        for i, e in enumerate(elems):
            h = eps * base_s[e]
            fields = []
            for sgn in (1.0, -1.0):
                q = base_s.copy()
                q[e] += sgn * h
                ctx.set_params(q, base_k)
                ctx.reset()
                ctx.run(n_steps)
                fields.append(ctx.get_field(rafem.RAFEM_SYS_T))
            tp, tm = fields
            fd[i] = float(np.sum((tp - tm) * (tp + tm - 2.0 * tgt))) / (2 * h)
            fd_loss[i] = (float(np.sum((tp - tgt) ** 2)) - float(np.sum((tm - tgt) ** 2))) / (2 * h)
        err = np.abs(g[elems] - fd)
        err_loss = np.abs(g[elems] - fd_loss)
        return {"eps": eps, "max_abs_err_over_max_abs_grad": float(err.max() / np.abs(fd).max()),
                "median_rel_err": float(np.median(err / np.maximum(np.abs(fd), 1e-300))),
                "max_abs_grad": float(np.abs(fd).max()),
                "loss_difference_form": {
                    "max_abs_err_over_max_abs_grad": float(err_loss.max() / np.abs(fd).max()),
                    "median_rel_err": float(np.median(err_loss / np.maximum(np.abs(fd), 1e-300)))}}

    t3 = time.perf_counter()
    checks = [fd_at(1e-6), fd_at(1e-3)]
    # the noise floor at eps = 1e-6: the same differences with the forward solved 10x less tightly; an error that
    # grows with the solver tolerance is the solves' termination noise in T+ - T-, divided by 2h
    ctx12 = rafem.Context(mesh, tol=1e-12, predictor=0, arith=rafem.RAFEM_ARITH_FP64)
    noise = fd_at(1e-6, ctx12)
    noise["forward_tol"] = 1e-12
    ctx12.close()
    t4 = time.perf_counter()
    ctx.close()
    return {"workload": "64^3 cells (274,625 nodes, 1,572,864 tets), jitter +-10%, tumour-sigma0 target",
            "steps": n_steps, "checkpoint_every": every, "solver_tol": 1e-13, "params_dtype": "float32",
            "fd_forward": "tol 1e-13, predictor order 0, FP64 element passes",
            "fd_quotient": "(L+ - L-)/(2h) with L+ - L- summed node by node from the two temperature fields",
            "loss": float(loss.item()), "forward_ms": (t1 - t0) * 1e3, "backward_ms": (t2 - t1) * 1e3,
            "backward_over_forward": (t2 - t1) / (t1 - t0), "adjoint": adj,
            "fd_check": {"elements": n_fd, "relative_steps": checks, "forward_tol_1e-12_at_eps_1e-6": noise,
                         "seconds": t4 - t3}}


def measure_accuracy(rafem, torch, mesh, args):
    """Accuracy over the paper's run (Sec. IV: per-step error and PSNR, Eq. 1-2, against a reference run) on the
    headline workload, every 100 steps of the first `accuracy_steps` (default 900, 15 simulated minutes). The
    reference is the tightest run the library can make: FP64 Krylov, FP64 element and node passes, relative
    residual 1e-13. Against it: the mixed path at relative residuals 1e-6 ... 1e-12 (the tolerance sweep), the
    FP64 path (double-word element passes, the default) at 1e-10, the FP64 path with FP64 element passes at 1e-10,
    and the double-word FP64 path at 1e-13 (which isolates the element-pass arithmetic from the solver tolerance).
    Reported per arm: relative L2 differences of T and V, PSNR of T (peak over the reference run) and the arm's
    steps/s over the run (host-synchronised every 100 steps)."""
    import numpy as np
    n = args.accuracy_steps
    marks = list(range(100, n, 100)) + [n]
    stream = torch.cuda.Stream()

    def trajectory(ctx):
        Ts, Vs, done, t_run, worst = [], [], 0, 0.0, 0
        ctx.reset()
        for m in marks:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s, st = ctx.run(m - done)
            torch.cuda.synchronize()
            t_run += time.perf_counter() - t0
            worst = max(worst, s)
            done = m
            Ts.append(ctx.get_field(rafem.RAFEM_SYS_T))
            Vs.append(ctx.get_field(rafem.RAFEM_SYS_V))
        return Ts, Vs, n / t_run, rafem.status_string(worst)

    ref = rafem.Context(mesh, stream=stream.cuda_stream, precision=rafem.RAFEM_PRECISION_FP64, tol=1e-13,
                        arith=rafem.RAFEM_ARITH_FP64)
    Tr, Vr, ref_rate, ref_status = trajectory(ref)
    ref.close()
    peak = max(float(T.max()) for T in Tr)
    out = {"steps": n, "marks": marks,
           "reference": {"precision": "fp64", "element_arith": "fp64", "tol": 1e-13, "steps_per_s": ref_rate,
                         "status": ref_status}}

    def compare(Ta, Va):
        eT = [float(np.linalg.norm(a - b) / np.linalg.norm(b)) for a, b in zip(Ta, Tr)]
        eV = [float(np.linalg.norm(a - b) / np.linalg.norm(b)) for a, b in zip(Va, Vr)]
        psnr = [float(20 * np.log10(peak / np.sqrt(max(float(np.mean((a - b) ** 2)), 1e-300))))
                for a, b in zip(Ta, Tr)]
        return {"rel_err_T_max": max(eT), "rel_err_V_max": max(eV), "psnr_T_db_min": min(psnr), "rel_err_T": eT,
                "rel_err_V": eV}

    out["mixed"] = []
    ctx = rafem.Context(mesh, stream=stream.cuda_stream, precision=rafem.RAFEM_PRECISION_MIXED)
    for tol in (1e-6, 1e-8, 1e-10, 1e-12):
        ctx.set_tol(tol)
        Tm, Vm, rate, status = trajectory(ctx)
        out["mixed"].append({"tol": tol, "steps_per_s": rate, "status": status, **compare(Tm, Vm)})
    ctx.close()
    out["fp64"] = []
    for name, tol, arith in (("fp64 double-word elements", 1e-10, rafem.RAFEM_ARITH_DW),
                             ("fp64 FP64 elements", 1e-10, rafem.RAFEM_ARITH_FP64),
                             ("fp64 double-word elements", 1e-13, rafem.RAFEM_ARITH_DW)):
        ctx = rafem.Context(mesh, stream=stream.cuda_stream, precision=rafem.RAFEM_PRECISION_FP64, tol=tol,
                            arith=arith)
        Tf, Vf, rate, status = trajectory(ctx)
        ctx.close()
        out["fp64"].append({"arm": name, "tol": tol, "steps_per_s": rate, "status": status, **compare(Tf, Vf)})
    return out


def accuracy_headline(acc: dict) -> dict:
    """The accuracy figures the headline is quoted beside: mixed and FP64 at the configured 1e-10, and the
    double-word element passes against FP64 ones (both at 1e-13), each against the tight FP64 reference."""
    keys = ("rel_err_T_max", "rel_err_V_max", "psnr_T_db_min", "steps_per_s", "status")
    pick = lambda d: {k: d[k] for k in keys}
    mixed = next(d for d in acc["mixed"] if d["tol"] == 1e-10)
    fp64 = next(d for d in acc["fp64"] if d["tol"] == 1e-10 and d["arm"] == "fp64 double-word elements")
    fp64a = next(d for d in acc["fp64"] if d["tol"] == 1e-10 and d["arm"] == "fp64 FP64 elements")
    dw = next(d for d in acc["fp64"] if d["tol"] == 1e-13)
    return {"reference": acc["reference"], "steps": acc["steps"],
            "mixed_tol_1e-10": pick(mixed), "fp64_tol_1e-10": pick(fp64), "fp64_fp64_elements_tol_1e-10": pick(fp64a),
            "double_word_vs_fp64_elements_tol_1e-13": pick(dw)}


def measure_small(rafem, torch, mg, args):
    """The 48^3-cell workload (117,649 nodes, jitter 10%): its matrices and vectors fit in L2, so a solver
    iteration is bounded by its grid barriers and latency rather than HBM (no roofline fraction is claimed).
    FP64 CG, FP64 pipelined CG (one barrier per iteration instead of two) and the mixed path over the same
    W + K steps."""
    mesh = mg.workload_48()
    stream = torch.cuda.Stream()
    out = {"workload": "48^3 cells, 117,649 nodes, jitter 10%, dt = 1 s, tol 1e-10", "steps": args.small_steps}
    for name, kw in (("fp64_cg", {}), ("fp64_pipecg", {"solver": rafem.RAFEM_SOLVER_PIPECG}),
                     ("mixed", {"precision": rafem.RAFEM_PRECISION_MIXED})):
        ctx = rafem.Context(mesh, stream=stream.cuda_stream, **kw)
        ctx.run(args.warmup)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        s, st = ctx.run(args.small_steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        ctx.reset()
        ctx.run(args.warmup)
        ctx.set_tracing(True)
        ctx.run(args.small_steps)
        tr = ctx.get_trace()
        ctx.close()
        out[name] = {"steps_per_s": args.small_steps / (ms * 1e-3), "status": rafem.status_string(s),
                     "iters_V_per_step": tr["iters_V"] / tr["steps"], "iters_T_per_step": tr["iters_T"] / tr["steps"],
                     "solve_V_us_per_iter": 1e3 * tr["ms_solve_V"] / max(tr["iters_V"], 1)}
    return out


def measure_monolithic(rafem, torch, mesh, args):
    """The paper's 2N x 2N system shape: V and T of each step solved together by Newton's method (corrector_tol
    1e-6 degC on max |dT|, at most 20 iterations, inexact linear solves) on the 127^3 workload, with each Newton
    linear solver: flexible GMRES preconditioned by split-system solves (the default) and block-Jacobi BiCGSTAB.
    K steps after W warm-up, CUDA events on the context's stream, then (flexible GMRES) one untimed step as direct
    launches for per-kernel profilers. Reported beside the staggered (lagged) step; the two compute different time
    discretisations (implicit vs lagged coupling)."""
    out = {"steps": args.monolithic_steps}
    for name, solver in (("fgmres_split_precond", rafem.RAFEM_COUPLED_FGMRES),
                         ("bicgstab_block_jacobi", rafem.RAFEM_COUPLED_BICGSTAB)):
        stream = torch.cuda.Stream()
        ctx = rafem.Context(mesh, stream=stream.cuda_stream, coupling=rafem.RAFEM_COUPLING_MONOLITHIC,
                            n_corrector=20, corrector_tol=1e-6, coupled_solver=solver)
        ctx.run(args.warmup)
        ctx.set_tracing(False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s, st = ctx.run(args.monolithic_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        r = {"steps_per_s": args.monolithic_steps / (ms * 1e-3), "ms_per_step": ms / args.monolithic_steps,
             "newton_iterations_last_step": st.correctors, "status": rafem.status_string(s),
             "unknowns": 2 * ctx.N, "graph": ctx.graph_info()["corrector_graph"]}
        if solver == rafem.RAFEM_COUPLED_FGMRES:
            r.update({"outer_iterations_last_step": st.refine_V, "inner_potential_cg_iterations_last_step": st.iters_V,
                      "inner_thermal_cg_iterations_last_step": st.iters_T})
            # one more step as direct launches (untimed): per-kernel profilers list these one by one
            ctx.set_tracing(True)
            s2, st2 = ctx.run(1)
            ctx.set_tracing(False)
            r["traced_step"] = {"newton_iterations": st2.correctors, "outer_iterations": st2.refine_V,
                                "status": rafem.status_string(s2)}
        else:
            r["bicgstab_iterations_last_step"] = st.iters_V
        out[name] = r
        ctx.close()
    # the default solver's rate as the arm's headline
    out["steps_per_s"] = out["fgmres_split_precond"]["steps_per_s"]
    return out


def measure_numbering(rafem, torch, mg, mesh, args):
    """Sensitivity to the node numbering (mixed precision, 127^3): the lattice numbering, a seeded random
    renumbering (no locality: 32-bit columns, scattered gathers) and that random mesh renumbered by the library's
    reverse Cuthill-McKee order (rafem_reorder_rcm). Same K-step timing as the headline, fresh context each."""
    out = {"steps": args.numbering_steps}
    shuffled, _ = mg.shuffled_nodes(mesh, mg.SEED_BASE + 6)
    t0 = time.perf_counter()
    perm = rafem.reorder_rcm(shuffled)
    out["rcm_host_s"] = time.perf_counter() - t0
    for name, m in (("lattice", mesh), ("random", shuffled), ("rcm_of_random", mg.permute_nodes(shuffled, perm))):
        stream = torch.cuda.Stream()
        ctx = rafem.Context(m, stream=stream.cuda_stream, precision=rafem.RAFEM_PRECISION_MIXED)
        lay = ctx.layout_info()
        ctx.run(args.warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s, st = ctx.run(args.numbering_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = {"steps_per_s": args.numbering_steps / (ms * 1e-3), "kernel_code": lay["kernel_code"],
                     "column_bytes": lay["column_bytes"], "status": rafem.status_string(s)}
        ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="rafem", choices=["rafem", "reference"])
    ap.add_argument("--cells", type=int, default=127)
    ap.add_argument("--e2e-steps", type=int, default=0, help="end-to-end steps (0 = the timed K steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=3, help="oracle steps timed on the 48^3 workload")
    ap.add_argument("--cpu-wait", type=float, default=900.0,
                    help="seconds after its start at which the 48^3 oracle timing is stopped")
    ap.add_argument("--only", choices=["fp64", "mixed", "ilu0", "bicgstab", "gmres", "pipecg"], default=None,
                    help="run one solver configuration only")
    ap.add_argument("--batch-steps", type=int, default=10, help="timed steps of the batching form (0 = skip)")
    ap.add_argument("--adjoint-steps", type=int, default=120, help="steps of the differentiation form (0 = skip)")
    ap.add_argument("--ilu-steps", type=int, default=10, help="timed steps with the ILU(0) preconditioner (0 = skip)")
    ap.add_argument("--bicgstab-steps", type=int, default=5, help="timed steps with BiCGSTAB (0 = skip)")
    ap.add_argument("--gmres-steps", type=int, default=5, help="timed steps with GMRES(30) (0 = skip)")
    ap.add_argument("--numbering-steps", type=int, default=10, help="timed steps per node numbering (0 = skip)")
    ap.add_argument("--monolithic-steps", type=int, default=3, help="timed monolithic Newton steps (0 = skip)")
    ap.add_argument("--fd-elements", type=int, default=32, help="finite-difference checks of the gradient")
    ap.add_argument("--pipecg-steps", type=int, default=10, help="timed steps with pipelined CG (0 = skip)")
    ap.add_argument("--small-steps", type=int, default=60, help="timed steps of the 48^3 workload (0 = skip)")
    ap.add_argument("--accuracy-steps", type=int, default=900,
                    help="steps of the tolerance sweep / long-run parity against FP64 (0 = skip)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return reference_arm(args)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    # CPU baseline: the FP64 oracle on the host, one thread. The 8^3 single-step workload is timed whole, first,
    # in a child process (no CUDA context in this process yet); the 48^3 workload (configs' 60-step FP64 case)
    # is timed in a child that runs while the GPU legs after the headline run, and is collected at the end.
    cpu_c1 = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t = OracleTimer("c1_8", 1).finish(1, 120.0)
        if t["step_s"]:
            cpu_c1 = {"steps_per_s": 1.0 / t["step_s"][0], "setup_s": t["setup_s"], "step_s": t["step_s"],
                      "nodes": t["nodes"], "workload": "8^3 cells (729 nodes, 3,072 tets), no jitter, one step"}

    import numpy as np
    import torch
    from paper_2409_13036_b300 import build, meshgen as mg, rafem

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()

    mesh = mg.workload_127() if args.cells == 127 else mg.cube_mesh(args.cells, jitter=0.1,
                                                                     seed=mg.SEED_BASE + 2, sigma0="lognormal")
    peaks, peak_kind = _measured_peaks()
    runs = {}
    for name, prec in (("fp64", rafem.RAFEM_PRECISION_FP64), ("mixed", rafem.RAFEM_PRECISION_MIXED)):
        if args.only and args.only != name:
            continue
        r = measure(rafem, torch, mesh, prec, args, local, dist, want_clocks=(name == "mixed" or args.only == name))
        r["roofline"] = roofline(r, prec == rafem.RAFEM_PRECISION_MIXED, peaks, peak_kind)
        runs[name] = r
        if name == "fp64" and args.only is None:
            r["ctx"].close()
            r["ctx"] = None
    if args.ilu_steps > 0 and args.only in (None, "ilu0"):
        ilu_args = argparse.Namespace(**vars(args))
        ilu_args.steps = args.ilu_steps
        r = measure(rafem, torch, mesh, rafem.RAFEM_PRECISION_FP64, ilu_args, local, dist, want_clocks=False,
                    precond=rafem.RAFEM_PRECOND_ILU0)
        r["roofline"] = roofline(r, False, peaks, peak_kind)
        r["steps"] = args.ilu_steps
        if args.only != "ilu0":
            r["ctx"].close()
            r["ctx"] = None
        runs["fp64_ilu0"] = r
        # the same preconditioner in the precision form: FP32 factors, values and vectors in the inner iterations
        r = measure(rafem, torch, mesh, rafem.RAFEM_PRECISION_MIXED, ilu_args, local, dist, want_clocks=False,
                    precond=rafem.RAFEM_PRECOND_ILU0)
        r["roofline"] = roofline(r, True, peaks, peak_kind)
        r["steps"] = args.ilu_steps
        r["ctx"].close()
        r["ctx"] = None
        runs["mixed_ilu0"] = r
    if args.bicgstab_steps > 0 and args.only in (None, "bicgstab"):
        b_args = argparse.Namespace(**vars(args))
        b_args.steps = args.bicgstab_steps
        r = measure(rafem, torch, mesh, rafem.RAFEM_PRECISION_FP64, b_args, local, dist, want_clocks=False,
                    solver=rafem.RAFEM_SOLVER_BICGSTAB)
        r["solver"] = "bicgstab"
        r["roofline"] = roofline(r, False, peaks, peak_kind)
        r["steps"] = args.bicgstab_steps
        if args.only != "bicgstab":
            r["ctx"].close()
            r["ctx"] = None
        runs["fp64_bicgstab"] = r
    if args.gmres_steps > 0 and args.only in (None, "gmres"):
        g_args = argparse.Namespace(**vars(args))
        g_args.steps = args.gmres_steps
        r = measure(rafem, torch, mesh, rafem.RAFEM_PRECISION_FP64, g_args, local, dist, want_clocks=False,
                    solver=rafem.RAFEM_SOLVER_GMRES)
        r["solver"] = "gmres"
        r["roofline"] = roofline(r, False, peaks, peak_kind)
        r["steps"] = args.gmres_steps
        if args.only != "gmres":
            r["ctx"].close()
            r["ctx"] = None
        runs["fp64_gmres30"] = r
        # the adaptive cycle length (Sec. III-B): between 10 and 30 steps per cycle
        r = measure(rafem, torch, mesh, rafem.RAFEM_PRECISION_FP64, g_args, local, dist, want_clocks=False,
                    solver=rafem.RAFEM_SOLVER_GMRES, gmres_min_restart=10)
        r["solver"] = "gmres"
        r["roofline"] = roofline(r, False, peaks, peak_kind)
        r["steps"] = args.gmres_steps
        r["ctx"].close()
        r["ctx"] = None
        runs["fp64_gmres_adaptive"] = r
    if args.pipecg_steps > 0 and args.only in (None, "pipecg"):
        p_args = argparse.Namespace(**vars(args))
        p_args.steps = args.pipecg_steps
        r = measure(rafem, torch, mesh, rafem.RAFEM_PRECISION_FP64, p_args, local, dist, want_clocks=False,
                    solver=rafem.RAFEM_SOLVER_PIPECG)
        r["solver"] = "pipecg"
        r["roofline"] = roofline(r, False, peaks, peak_kind)
        r["steps"] = args.pipecg_steps
        if args.only != "pipecg":
            r["ctx"].close()
            r["ctx"] = None
        runs["fp64_pipecg"] = r
    head_name = next(n for n in ("mixed", "fp64", "fp64_ilu0", "fp64_bicgstab", "fp64_gmres30", "fp64_pipecg")
                     if n in runs)
    head = runs[head_name]
    ctx = head["ctx"]
    N, nnz, n_colors = head["N"], head["nnz"], head["n_colors"]

    # end to end through the C-ABI with host buffers, over the same steps as the device-timed region: back to the
    # initial state, the W warm-up steps, then per step one rafem_step_host call: H2D of the state (T, V) from
    # pinned buffers, the step, D2H of both fields into the same buffers (V's copies overlap the step)
    hT = torch.empty(N, dtype=torch.float64).pin_memory()
    hV = torch.empty(N, dtype=torch.float64).pin_memory()
    ctx.reset()
    ctx.run(args.warmup - 1)
    ctx.get_field_ptr(rafem.RAFEM_SYS_T, hT.data_ptr(), 0)
    ctx.get_field_ptr(rafem.RAFEM_SYS_V, hV.data_ptr(), 0)
    e2e_steps = args.steps if args.e2e_steps <= 0 else min(args.e2e_steps, args.steps)
    ptrs = (hT.data_ptr(), hV.data_ptr(), hT.data_ptr(), hV.data_ptr())
    ctx.step_host_ptr(*ptrs)  # the last warm-up step, through the call timed below (builds its graph)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        ctx.step_host_ptr(*ptrs)
    t_e2e = reduce_over_ranks([time.perf_counter() - t0], "max", dist)[0]
    ctx.close()
    # the 48^3 oracle timing runs on a host core from here on, beside the remaining GPU legs (the timed headline
    # and end-to-end regions above are over)
    c2_timer = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.cpu_steps > 0:
        c2_timer = OracleTimer("c2_48", args.cpu_steps)

    def summary(r):
        tr = r["trace"]
        k = r.get("steps", args.steps)
        return {"value": aggregate_rate(world * k, r["ms"]), "unit": UNIT, "ms_per_step": r["ms"] / k, "steps": k,
                "status": r["status"], "last_step": r["last"],
                "iters_V_per_step": tr["iters_V"] / tr["steps"], "iters_T_per_step": tr["iters_T"] / tr["steps"],
                "refine_V_per_step": tr["refine_V"] / tr["steps"],
                "regions_ms_per_step": {k: tr[k] / tr["steps"] for k in ("ms_assemble_V", "ms_predict_V",
                                                                          "ms_solve_V", "ms_assemble_T",
                                                                          "ms_predict_T", "ms_solve_T")},
                "roofline": r["roofline"]}

    # kernels of the timed region: the kernel nodes of the captured step graph per step, plus the step-counter
    # kernel rafem_run launches once
    per_step_launches = head["graph"]["step_kernels"]
    head_sum = summary(head)
    line = {"metric": METRIC, "value": head_sum["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head_sum["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if head_name == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nodes": N, "nnz_per_system": nnz, "colours": n_colors,
                       "precision": head_name, "layout": "SELL-32",
                       "element_arith": "double-word" if head["layout"]["arith"] == rafem.RAFEM_ARITH_DW else "fp64",
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (two 373 MB FP64 matrices + element data per step)"},
            "status": head_sum["status"], "last_step": head_sum["last_step"],
            "iters_V_per_step": head_sum["iters_V_per_step"], "iters_T_per_step": head_sum["iters_T_per_step"],
            "refine_V_per_step": head_sum["refine_V_per_step"],
            "regions_ms_per_step": head_sum["regions_ms_per_step"],
            "roofline": head["roofline"],
            "e2e": {"value": aggregate_rate(world * e2e_steps, 1e3 * t_e2e), "unit": UNIT, "h2d_bytes_per_step": 16 * N,
                    "d2h_bytes_per_step": 16 * N, "steps": e2e_steps,
                    "note": "same steps as the device-timed region, replayed from the initial state; one "
                            "rafem_step_host call per step (state in, step, fields out)"},
            "gpu_launches": per_step_launches * args.steps + 1,
            "clocks": head["clocks"]}
    if "fp64" in runs and head_name != "fp64":
        line["fp64"] = summary(runs["fp64"])
        # the mixed form's accuracy against the FP64 GPU path after the same W+K steps (Sec. IV PSNR, Eq. 1-2)
        Tf, Vf = runs["fp64"]["fields"]
        Tm, Vm = head["fields"]
        mse_T = float(np.mean((Tm - Tf) ** 2))
        line["mixed_vs_fp64"] = {
            "rel_err_T": float(np.linalg.norm(Tm - Tf) / np.linalg.norm(Tf)),
            "rel_err_V": float(np.linalg.norm(Vm - Vf) / np.linalg.norm(Vf)),
            "psnr_T_db": float("inf") if mse_T == 0 else float(20 * np.log10(Tf.max() / np.sqrt(mse_T))),
            "speedup": head_sum["value"] / line["fp64"]["value"]}
    if "fp64_bicgstab" in runs:
        line["fp64_bicgstab"] = summary(runs["fp64_bicgstab"])
    if "fp64_gmres30" in runs:
        line["fp64_gmres30"] = summary(runs["fp64_gmres30"])
    if "fp64_gmres_adaptive" in runs:
        line["fp64_gmres_adaptive"] = summary(runs["fp64_gmres_adaptive"])
        line["fp64_gmres_adaptive"]["restart"] = "adaptive, 10..30 steps per cycle"
    if "fp64_pipecg" in runs and head_name != "fp64_pipecg":
        line["fp64_pipecg"] = summary(runs["fp64_pipecg"])
    for name in ("fp64_ilu0", "mixed_ilu0"):
        if name in runs:
            line[name] = summary(runs[name])
            line[name]["levels"] = runs[name]["layout"]["ilu"]["levels"]
    if args.batch_steps > 0 and args.only is None and args.cells == 127:
        try:
            line["batch"] = measure_batch(rafem, torch, mg, args, dist)
        except Exception as exc:  # the headline line must still be printed
            line["batch"] = {"error": repr(exc)[:300]}
    if args.small_steps > 0 and args.only in (None, "pipecg"):
        try:
            line["small_48"] = measure_small(rafem, torch, mg, args)
        except Exception as exc:
            line["small_48"] = {"error": repr(exc)[:300]}
    if args.accuracy_steps > 0 and args.only is None:
        try:
            line["accuracy"] = measure_accuracy(rafem, torch, mesh, args)
            line["accuracy_headline"] = accuracy_headline(line["accuracy"])
        except Exception as exc:
            line["accuracy"] = {"error": repr(exc)[:300]}
    if args.monolithic_steps > 0 and args.only is None:
        try:
            line["monolithic"] = measure_monolithic(rafem, torch, mesh, args)
        except Exception as exc:
            line["monolithic"] = {"error": repr(exc)[:300]}
    if args.numbering_steps > 0 and args.only is None and args.cells == 127:
        try:
            line["numbering"] = measure_numbering(rafem, torch, mg, mesh, args)
        except Exception as exc:
            line["numbering"] = {"error": repr(exc)[:300]}
    if args.adjoint_steps > 0 and args.only is None and args.cells == 127:
        try:
            line["adjoint"] = measure_adjoint(rafem, torch, mg, args)
        except Exception as exc:
            line["adjoint"] = {"error": repr(exc)[:300]}
    if c2_timer is not None:
        t = c2_timer.finish(args.cpu_steps, args.cpu_wait)
        line["cpu_baseline"] = cpu_baseline_line(t, cpu_c1, line.get("small_48"))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
