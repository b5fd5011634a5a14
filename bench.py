"""Benchmark: pseudo-time iterations of the component-splitting LU-SGS scheme on one GB300.

Workload (one "step" = one full pseudo-time iteration: residual, split LU-SGS operator,
CS-1 correction and update): 2D Mach 15 flow over a cylinder, 384 x 256 cells over the windward half,
11-species two-temperature ionised air with 21 reactions, FP64.  Synthetic, seeded: the run
starts from the uniform freestream.

Metric: Mcell-iter/s (cells x iterations / second), higher is better.  ``value`` is the
device time of the timed iterations (CUDA events on the library's stream, L2 flushed before
every iteration); ``e2e`` is the same metric through the C ABI with host buffers (state
uploaded, iterated, downloaded every step).  ``--impl reference`` times the FP64 oracle on
the host cores instead.

Multi-GPU (torchrun): every rank runs an independent replica (the LU-SGS sweep of one case
does not shard exactly); value = total cells x iterations / max rank time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import inputs  # noqa: E402

NI, NJ = 384, 256
MECH = inputs.MECH_AIR11
MACH, T_INF, P_INF, T_WALL = 15.0, 300.0, 500.0, 500.0
# CFL 20 reached by a geometric ramp from 0.5 over 2000 iterations, with the source radius in the
# local time step (option dtau_source, Sec. 2.2): the setting in which C2 reaches a 1e-8 drop
CFL, CFL_START, RAMP = 20.0, 0.5, 2000
DTAU_SOURCE = 1
WORKLOAD = "half-cylinder-384x256-air11-2T-mach15-CS1-fp64"
# Floating-point operations per cell and iteration of each phase (2 x FMA + MUL + ADD thread
# instructions counted by ncu on this workload, one launch from the 5th iteration, divided by
# the cell count; the primitive phase varies with the Newton iteration count, i.e. with the
# state).  On GB300 every residual kernel keeps its FP64 pipe 74-86 % busy at <15 % of DRAM
# peak, so the roofline of this path is the FP64 ALU, not HBM; the sweeps are latency-bound
# (one dependent hyperplane step after another).
FP64_FLOPS_PER_CELL = {
    "primitive": 1078.0,       # k_primitive, mean over the 20 timed iterations
    "gradient": 400.0,
    # k_eta (55 per direction) + k_flux (1148 per direction) + k_chem (5011), which runs on a
    # second stream beside the gradient and fluxes; the flux phase ends when both are done
    "flux": 7417.0,
    "assemble": 130.0,
    "spectral": 361.0,
    "sweep_fwd": 1128.0,       # couplings (k_sweep_mat, 753) + both sweeps (k_split_p2p, 374)
    "sweep_bwd": 0.0,
    "correct": 109.0,
}
FLOPS_SOURCE = ("ncu FP64 thread instructions (2 DFMA + DMUL + DADD) per cell; k_primitive and "
                "k_chem (the latter counted in the flux phase, beside which it runs on a second "
                "stream): means over the launches of the timed iterations 6..25 "
                "(profiles/primitive_chem_fp64_counts_timed_window_384x256_air11.md); other phases: one "
                "launch of the 5th iteration (profiles/kernels_half_cylinder_384x256_air11.md; k_flux and k_eta: "
                "profiles/launches_half_cylinder_384x256_air11_fp64.md)")
# the mixed operator's sweep phase: couplings formed (k_sweep_mat, 753 flop) and swept
# (k_split_p2p, 374 flop) in FP32, the FP64 forms' counts
FP64_FLOPS_PER_CELL_SWEEP_MIXED = 0.0
FP32_FLOPS_PER_CELL_SWEEP = 1127.0
# DRAM bytes per launch measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum)
DRAM_BYTES_PER_LAUNCH = {
    "primitive": None,         # the split k_primitive / k_chem kernels: DRAM not captured
    "flux": 69.1e6 + 70.0e6, "sweep_fwd": None, "gradient": 17.4e6,
    "spectral": 54.1e6, "assemble": 33.9e6, "correct": 24.4e6,
}
DRAM_BYTES_SWEEP_FP32 = None              # FP32 records: not captured with ncu
# both coupled sweeps of the 384 x 256 grid: one read of the operator's inputs (the diagonal
# blocks' inverses, states, increments), the DRAM bytes ncu measured for the one-lane-per-row
# kernel k_ci_cluster, which re-reads nothing; the default kernels (k_ci_mat + k_ci_mat_sweep)
# also write and read the assembled neighbour blocks and were not captured
CI_SWEEP_ALGO_BYTES = 367.3e6
# FP64 peak: measured on the device at the start of every run (cs_measure_fp64_rate: DFMA
# chains on every SM); the nominal 1.25 TFLOP/s of the platform only if that fails.  FP32: 152
# SMs x 128 lanes x 2 flop x 2.07 GHz.
FP64_NOMINAL_GFLOPS = 1250.0
FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.07
# Algorithmic HBM bytes per cell and iteration of the four-pass split design (every array
# crosses HBM once per pass: words = 7 s + 3 g + 3 a + 4 n with s stored conserved values, g
# geometry values, a auxiliary values and n split unknowns per cell).  2D, 11 species, 2T:
# s 15, g 5, a 23, n 16 -> 253 words; 3D: s 16, g 10, a 26, n 17 -> 288 words.
ALGO_BYTES_PER_CELL = {"c2": 8 * (7 * 15 + 3 * 5 + 3 * 23 + 4 * 16),
                       "c3": 8 * (7 * 16 + 3 * 10 + 3 * 26 + 4 * 17)}


def job_time_ms(local_ms, dist=None, device="cpu"):
    """Time of the whole job: the slowest rank's timed-region time (max over ranks, then a
    barrier so that no rank starts the next phase early).  Replicas only: this is the one
    collective of a multi-GPU run, outside the timed region."""
    if dist is None:
        return local_ms
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_value(world, cells, steps, total_ms):
    """Whole-job throughput in Mcell-iter/s: every rank's cells x iterations over the job time."""
    return world * cells * steps / (total_ms / 1e3) / 1e6


def log(*a):
    print(*a, file=sys.stderr, flush=True)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, n in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


C3 = False      # --workload c3: the 3D sphere-cone instead of the half cylinder
C3_DIMS = (192, 128, 96)
C3_MACH = 20.0


def make_case(P):
    if C3:
        nodes = inputs.sphere_cone(*C3_DIMS)
        fs = inputs.freestream(MECH, T=T_INF, p=P_INF, mach=C3_MACH)
        return nodes, fs
    nodes = inputs.cylinder_half(NI, NJ, dr1=5e-5 / 8)
    fs = inputs.freestream(MECH, T=T_INF, p=P_INF, mach=MACH)
    return nodes, fs


def case_bc():
    return inputs.sphere_cone_bc() if C3 else inputs.cylinder_half_bc()


def case_cells():
    return C3_DIMS[0] * C3_DIMS[1] * C3_DIMS[2] if C3 else NI * NJ


PRECISION = 0   # 0: FP64 operator, 1: FP32 operator (mixed); set by --precision


SCHEME = (0, 1)   # (scheme, correction): CS-1 split by default; --scheme cs2 / ci


def step_kwargs(iters):
    return dict(scheme=SCHEME[0], correction=SCHEME[1], clip=1, cfl=CFL, cfl_start=CFL_START,
                ramp_iters=RAMP, iters=iters, precision=PRECISION)


ORACLE_BUILD = "gcc -O3 -ffp-contract=off, one thread"
ORACLE_BUILD_OMP = ("gcc -O3 -ffp-contract=off -fopenmp: per-cell and per-face loops (primitives, "
                    "chemistry, gradients, fluxes, radii) on all host cores, sweeps serial")


def oracle_rate_all_cores(iters, seconds_cap=30.0):
    """The oracle's OpenMP build on every host core, timed in a child process (the serial and
    the OpenMP oracle libraries cannot share one process): (Mcell-iter/s, iterations,
    seconds, threads) or None."""
    env = dict(os.environ)
    env.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-leg", "omp", "--cpu-leg-iters", str(iters),
           "--cpu-leg-seconds", str(seconds_cap)]
    if C3:
        cmd += ["--workload", "c3"]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env)
        d = json.loads(r.stdout.strip().splitlines()[-1])
        return d["value"], d["iters"], d["seconds"], int(env["OMP_NUM_THREADS"])
    except (OSError, subprocess.SubprocessError, ValueError, IndexError, KeyError):
        return None


def oracle_rate(iters, seconds_cap=30.0):
    """Time the FP64 oracle (host, one core) on the same workload: iterations from the
    freestream, bounded by iteration count and seconds."""
    import oracle
    oracle.build()
    nodes, fs = make_case(None)
    g = oracle.OracleGrid(nodes, case_bc(), MECH)
    g.set_boundary(fs, Tw=T_WALL)
    g.set_dtau_source(DTAU_SOURCE)
    g.set_state(g.freestream_state())
    done, t0 = 0, time.perf_counter()
    kw = step_kwargs(1)
    kw.pop("precision")
    while done < iters:
        g.step(**kw)
        done += 1
        if time.perf_counter() - t0 > seconds_cap:
            break
    dt = time.perf_counter() - t0
    return case_cells() * done / dt / 1e6, done, dt


def run_reference(args, rank):
    if rank != 0:
        return
    # warm-up (untimed), then timed iterations; each iteration is a bounded sample of the
    # same workload (one full pseudo-time iteration of the 384 x 256 grid)
    import oracle
    oracle.build()
    nodes, fs = make_case(None)
    g = oracle.OracleGrid(nodes, case_bc(), MECH)
    g.set_boundary(fs, Tw=T_WALL)
    g.set_dtau_source(DTAU_SOURCE)
    g.set_state(g.freestream_state())
    kw = step_kwargs(1)
    kw.pop("precision")
    for _ in range(args.warmup):
        g.step(**kw)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        g.step(**kw)
    dt = time.perf_counter() - t0
    v = case_cells() * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": "Mcell-iter/s", "value": v, "unit": "Mcell-iter/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": case_cells(),
                   "cfl": f"{CFL_START} ramped geometrically to {CFL} over {RAMP} iterations",
                   "dtau_source": DTAU_SOURCE},
        "cpu_baseline": {"value": v, "unit": "Mcell-iter/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} iterations of the full grid from the freestream"},
        "e2e": {"value": v, "unit": "Mcell-iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batch(args, rank, world, local):
    """Batched serving workload: independent half-cylinder cases of uneven size (64 x 48 to
    512 x 384, Mach 6-20, 5 or 11 species), tuned, then stepped together through one CUDA graph
    per iteration; value = sum of cells x iterations / device time."""
    import numpy as np
    import torch
    import paper_2403_03440_gb300 as P
    P.build()
    torch.cuda.set_device(local)
    cases = inputs.batch_cases(args.batch_cases, seed=0)
    grids = []
    for c in cases:
        nodes = inputs.cylinder_half(c["ni"], c["nj"], dr1=5e-5 * 48 / c["ni"])
        fs = inputs.freestream(c["mech"], T=T_INF, p=P_INF, mach=c["mach"])
        g = P.Grid(nodes, inputs.cylinder_half_bc(), c["mech"])
        g.set_boundary(fs, Tw=T_WALL)
        g.init_freestream()
        grids.append(g)
    cells = sum(g.ncell for g in grids)
    batch = P.Batch(grids)
    t0 = time.perf_counter()
    choice = batch.tune(precision=PRECISION, trials=2)
    tune_s = time.perf_counter() - t0
    # CS-1, each case's CFL reached by a geometric ramp from 0.5 over 500 iterations
    opts = [dict(scheme=0, correction=1, clip=1, cfl=c["cfl"], cfl_start=0.5, ramp_iters=500,
                 precision=PRECISION) for c in cases]
    K = args.iters_per_graph
    if args.steps % K or args.warmup % K:
        raise SystemExit("--steps and --warmup must be multiples of --iters-per-graph")
    batch.step(opts, iters=args.warmup, iters_per_graph=K)
    stream = torch.cuda.ExternalStream(batch.stream())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        stats = batch.step(opts, iters=args.steps, iters_per_graph=K)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    value = cells * args.steps / (ms / 1e3) / 1e6
    # end to end through the public API with host buffers: every case's state uploaded from
    # pinned memory, one batched iteration, every state downloaded
    hq = [torch.empty((g.nq, g.ncell), dtype=torch.float64, pin_memory=True).numpy() for g in grids]
    for g, q in zip(grids, hq):
        g.get_state(q)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        for g, q in zip(grids, hq):
            g.set_state(q)
        batch.step(opts, iters=K, iters_per_graph=K)
        for g, q in zip(grids, hq):
            g.get_state(q)
    e2e_s = time.perf_counter() - t0
    nbytes = int(sum(q.nbytes for q in hq))
    e2e = cells * K * args.e2e_steps / e2e_s / 1e6
    # kernels per case and iteration: cfl, primitive, gradient, 2 fluxes, assemble + norms,
    # spectral, sweep (records + wavefront kernel, or one cluster kernel), correction
    per_iter = sum(9 + (2 if kind in (2, 3) else 1) for kind, _ in choice)
    if rank == 0:
        line = {
            "metric": "Mcell-iter/s", "value": value, "unit": "Mcell-iter/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if PRECISION == 0 else "f64 residual/update, f32 operator",
            "data": "synthetic",
            "config": {"workload": f"batch-{len(cases)}-half-cylinders-64x48-to-512x384-mach6-20-"
                                   f"air5-or-air11-CS1-{'fp64' if PRECISION == 0 else 'mixed'}",
                       "cases": len(cases), "cells": cells, "iters_per_graph": K,
                       "cfl": "ramp from 0.5 over 500 iterations to each case's CFL (5-200)",
                       "l2": "inputs (all cases' state and work arrays) far larger than L2",
                       "tune_seconds": tune_s,
                       "tuned": {f"{kind}:{C}": sum(1 for x in choice if x == (kind, C))
                                 for kind, C in set(choice)},
                       "parallelism": f"replicas x{world}"},
            "clocks": clk.summary(),
            "e2e": {"value": e2e, "unit": "Mcell-iter/s", "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes},
            "gpu_launches": per_iter * args.steps,
            "cases_failed": sum(1 for st in stats if st["status_cell"] != -1),
        }
        print(json.dumps(line), flush=True)


def measured_hbm_peak():
    """(GB/s, description): the measured copy bandwidth of the GB300s, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured copy bandwidth (of measured)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s (of fallback)"


def run_species(args, rank, world, local):
    """Species-count scaling test (Sec. 3.1): one implicit step of the split (CS) and coupled
    (CI) operators for a uniform non-reacting flow of ns species in a 10 x 10 x 10 box, ns from
    16 to 4096 (CI up to 1024: its dense per-cell factors would need 134 GB at 4096).  Device
    time per step, L2 flushed (256 MiB write) before every timed step.  value = CS time per
    step at the largest ns; the table gives both operators, their growth against ns = 16 and
    the speed-up (t_CI - t_CS) / t_CI the paper reports."""
    import numpy as np
    import torch
    import paper_2403_03440_gb300 as P
    P.build()
    torch.cuda.set_device(local)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    cfl = 10.0
    table = []
    with ClockSampler(local) as clk:
        for ns in args.species:
            case = inputs.species_box(ns, seed=0)
            box = P.SpeciesBox(case)
            rhs = torch.from_numpy(inputs.species_box_rhs(ns, box.ncell, seed=1)).cuda()
            row = {"ns": ns}
            for scheme, key in ((0, "cs_ms"), (1, "ci_ms")):
                if scheme == 1 and ns > args.ci_max_species:
                    row[key] = None
                    continue
                reps = args.steps if (scheme == 0 or ns <= 256) else max(3, args.steps // 10)
                for _ in range(args.warmup if (scheme == 0 or ns <= 256) else 1):
                    box.step(scheme, cfl, rhs)
                row[key] = box.time(scheme, cfl, rhs, reps, flush=flush)
            table.append(row)
            del box
            torch.cuda.empty_cache()
    base = table[0]
    for row in table:
        row["cs_growth"] = row["cs_ms"] / base["cs_ms"]
        if row["ci_ms"] is not None and base["ci_ms"]:
            row["ci_growth"] = row["ci_ms"] / base["ci_ms"]
            row["speedup_pct"] = 100.0 * (row["ci_ms"] - row["cs_ms"]) / row["ci_ms"]
    last = table[-1]
    # algorithmic HBM bytes of the CS step per species-cell: rhs read, forward increment
    # written and read back, increment written (4 x 8 B); per cell the 5-unknown flow block
    N = 1000
    bytes_cs = N * (32 * last["ns"] + 5 * 8 * 8)
    achieved = bytes_cs / (last["cs_ms"] / 1e3) / 1e9
    peak = measured_hbm_peak()
    if rank == 0:
        line = {
            "metric": "implicit step time (CS)", "value": last["cs_ms"], "unit": "ms",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": last["cs_ms"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"species-box-10x10x10-nonreacting-ns{args.species[0]}-{args.species[-1]}",
                       "cfl": cfl, "l2": "flushed before every timed step (256 MiB write)",
                       "parallelism": "single GPU"},
            "table": table,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak[0], "unit": "GB/s",
                         "frac": achieved / peak[0], "traffic": None, "peak_kind": peak[1],
                         "note": "CS step at the largest ns; latency-bound (2 x 28 dependent "
                                 "hyperplanes), bytes are the algorithmic ones"},
            "clocks": clk.summary(),
            "gpu_launches": 3 * args.steps,
        }
        print(json.dumps(line), flush=True)


def measured_bf16_peak():
    """(TFLOP/s, description): the measured cuBLAS bf16 burst rate, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured cuBLAS bf16 burst (of measured)"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback 1.9 PFLOP/s (of fallback)"


def run_mlp(args, rank, world, local):
    """Surrogate network inference (the fused tcgen05 kernel) on as many rows as the 384 x 256
    grid has cells: inputs resident on the device, L2 flushed before every timed call."""
    import torch
    import paper_2403_03440_gb300 as P
    P.build()
    torch.cuda.set_device(local)
    rows = NI * NJ
    net = P.MLP(inputs.mlp_init(0), max_batch=rows)
    gen = torch.Generator(device="cpu").manual_seed(0)
    X = torch.randn((rows, 14), generator=gen, dtype=torch.float32).cuda()
    Y = torch.empty((rows, 22), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        net.forward(X, Y)
    torch.cuda.synchronize()
    total = 0.0
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(k & 0xff)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            net.forward(X, Y)
            e1.record()
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
    ms = total / args.steps
    flop = 2.0 * rows * (14 * 128 + 2 * 128 * 128 + 128 * 22)
    peak = measured_bf16_peak()
    tf = flop / (ms / 1e3) / 1e12
    if rank == 0:
        print(json.dumps({
            "metric": "surrogate inference rows/s", "value": rows / (ms / 1e3), "unit": "rows/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 x bf16 -> f32", "data": "synthetic",
            "config": {"workload": f"mlp-14-128-128-128-22-silu-{rows}-rows", "rows": rows,
                       "l2": "flushed before every timed call (256 MiB write)"},
            "roofline": {"bound": "tensor", "achieved": tf, "peak": peak[0], "unit": "TFLOP/s",
                         "frac": tf / peak[0], "traffic": None, "peak_kind": peak[1],
                         "note": "CUDA events around cs_mlp_forward (includes its error-flag memset and status read)"},
            "clocks": clk.summary(), "gpu_launches": args.steps}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "batch", "species", "mlp"])
    ap.add_argument("--species", type=lambda t: [int(x) for x in t.split(",")],
                    default=[16, 64, 256, 1024, 4096])
    ap.add_argument("--ci-max-species", type=int, default=1024)
    ap.add_argument("--dual-dt", type=float, default=0.0,
                    help="physical time step of dual time stepping (0: steady pseudo-time iteration)")
    ap.add_argument("--scheme", default="cs1", choices=["cs1", "cs2", "ci", "ci_eig"])
    ap.add_argument("--batch-cases", type=int, default=64)
    ap.add_argument("--iters-per-graph", type=int, default=1)
    ap.add_argument("--no-convergence", action="store_true",
                    help="skip the C1 time-to-1e-8 runs of the default line")
    ap.add_argument("--no-batch", action="store_true", help="skip the batch throughput of the default line")
    ap.add_argument("--cpu-leg", choices=["omp"], default=None, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-leg-iters", type=int, default=3, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-leg-seconds", type=float, default=30.0, help=argparse.SUPPRESS)
    args = ap.parse_args()
    global PRECISION, WORKLOAD, C3, SCHEME
    SCHEME = {"cs1": (0, 1), "cs2": (0, 2), "ci": (1, 1), "ci_eig": (1, 1)}[args.scheme]
    if args.workload == "c3":
        C3 = True
        WORKLOAD = "sphere-cone-192x128x96-air11-2T-mach20-CS1-fp64"
        args.no_cpu_baseline = True      # one oracle iteration of 2.4 M cells takes minutes
    if args.precision == "mixed":
        PRECISION = 1
        WORKLOAD = WORKLOAD.replace("fp64", "mixed-fp32-operator")
    if args.scheme != "cs1":
        WORKLOAD = WORKLOAD.replace("CS1", args.scheme.upper())
    if args.dual_dt > 0:
        WORKLOAD += f"-dual-dt{args.dual_dt:g}"
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.cpu_leg == "omp":
        # child process of oracle_rate_all_cores: the OpenMP oracle only, no GPU
        import oracle
        oracle.use_openmp()
        v, it, dt = oracle_rate(args.cpu_leg_iters, args.cpu_leg_seconds)
        print(json.dumps({"value": v, "iters": it, "seconds": dt}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.warmup < 3:
        raise SystemExit("warmup must be >= 3")
    if args.workload == "batch":
        run_batch(args, rank, world, local)
        return
    if args.workload == "species":
        run_species(args, rank, world, local)
        return
    if args.workload == "mlp":
        run_mlp(args, rank, world, local)
        return

    run_iteration(args, rank, world, local)


def make_grid(P):
    nodes, fs = make_case(P)
    g = P.Grid(nodes, case_bc(), MECH)
    g.set_boundary(fs, Tw=T_WALL)
    g.set_option("dtau_source", DTAU_SOURCE)
    return g, fs


def prepare_grid(P, args):
    """A grid of the workload run from the freestream through the warm-up iterations."""
    g, _ = make_grid(P)
    if args.scheme == "ci_eig":
        g.set_option("ci_splitting", 1)
    g.init_freestream()
    if args.dual_dt > 0:
        # dual time stepping: one physical step begun from the freestream, theta = 1/2 (the
        # pseudo-time iterations below are its inner iterations)
        g.set_dual(args.dual_dt, 0.5)
        g.dual_advance()
    for _ in range(args.warmup):
        g.step(**step_kwargs(1))
    return g


def c1_time_to_drop(tol=1e-8, with_network=True):
    """Time to a `tol` drop of both residual monitors on C1 (half cylinder 48 x 32, 5-species
    1T air, Mach 10, minmod, CFL 10 ramped from 1 over 100 iterations, from the freestream):
    CS-1 with the FP64 operator, CS-1 with the FP32 operator, CS-1 with the FP32 operator and
    the network's chemistry diagonal (trained first on states of the same case), and the
    coupled (CI) operator in FP64.  Every run checks the monitors after its first iteration
    and then every 100 iterations."""
    import paper_2403_03440_gb300.surrogate as S
    c = S.CASES["c1"]
    keys = ("status", "iterations", "seconds", "device_seconds", "q_stag", "drop", "fallback_chunks")
    out = {"case": "half-cylinder-48x32-air5-1T-mach10-minmod-cfl10", "cells": c["ni"] * c["nj"],
           "tol": tol, "runs": {}}
    legs = [("cs1_fp64", dict(precision=0, scheme=0)), ("cs1_fp32_operator", dict(precision=1, scheme=0)),
            ("ci_fp64", dict(precision=0, scheme=1))]
    for name, kw in legs:
        try:
            r = S.run_to(c, tol, 20000, 100, **kw)
            out["runs"][name] = {k: r[k] for k in keys}
        except Exception as e:          # report, do not lose the bench line
            out["runs"][name] = {"status": f"error: {e}"}
    if with_network:
        try:
            t0 = time.perf_counter()
            X, T = S.collect(c, 3000, 10, 0)
            norm = S.standardisation(X, T)
            net, record, val = S.train(X, T, norm, epochs=20, max_batch=c["ni"] * c["nj"])
            norm_used, _ = S.calibrate(net, norm, val, q=c["calib_q"])
            train_s = time.perf_counter() - t0
            r = S.run_to(c, tol, 20000, 100, net=net, norm=norm_used, precision=1)
            out["runs"]["cs1_fp32_operator_network"] = {k: r[k] for k in keys}
            out["network"] = {"samples": int(X.shape[0]), "epochs": 20, "collect_and_train_seconds": train_s,
                              "final_loss": record[-1]}
        except Exception as e:
            out["runs"]["cs1_fp32_operator_network"] = {"status": f"error: {e}"}
    base = out["runs"].get("cs1_fp64", {})
    for r in out["runs"].values():
        if "q_stag" in r and "q_stag" in base and base["q_stag"]:
            r["q_rel_diff_vs_cs1_fp64"] = abs(r["q_stag"] - base["q_stag"]) / abs(base["q_stag"])
            r["time_ratio_vs_cs1_fp64"] = r["seconds"] / base["seconds"]
    return out


def c2_time_to_drop(tol=1e-8):
    """Time to a `tol` drop of both residual monitors on C2 itself (the 384 x 256 grid of the
    throughput line; first order, update limit 0.2, CFL ramped from 0.5 to 20 over 2000
    iterations with the source radius in the local time step): CS-1 with the FP64 operator and
    with the FP32 operator, monitors checked every 500 iterations, device time between two
    synchronisations around each run."""
    from paper_2403_03440_gb300 import convergence as CV
    out = {"case": "half-cylinder-384x256-air11-2T-mach15-first-order-cfl20-dtau-source",
           "cells": 98304, "tol": tol, "runs": {}}
    for name, prec in (("cs1_fp64", 0), ("cs1_fp32_operator", 1)):
        try:
            r = CV.run("c2", "cs1", CFL, CFL_START, RAMP, tol, 40000, 500, 0, prec,
                       update_limit=0.2, dtau_source=1)
            out["runs"][name] = {k: r[k] for k in ("status", "iterations", "seconds", "ms_per_iter",
                                                   "q_stag_final", "min_drop")}
        except Exception as e:          # report, do not lose the bench line
            out["runs"][name] = {"status": f"error: {e}"}
    return out


def batch_throughput(P, precision=0, steps=6, warmup=3, ncases=64):
    """Mcell-iter/s of the 64-case batch (64 x 48 to 512 x 384 half cylinders, Mach 6-20, CFL
    5-200, 5 or 11 species; CS-1, tuned, one graph launch per iteration), device time."""
    import torch
    cases = inputs.batch_cases(ncases, seed=0)
    grids = []
    for c in cases:
        nodes = inputs.cylinder_half(c["ni"], c["nj"], dr1=5e-5 * 48 / c["ni"])
        fs = inputs.freestream(c["mech"], T=T_INF, p=P_INF, mach=c["mach"])
        g = P.Grid(nodes, inputs.cylinder_half_bc(), c["mech"])
        g.set_boundary(fs, Tw=T_WALL)
        g.init_freestream()
        grids.append(g)
    cells = sum(g.ncell for g in grids)
    batch = P.Batch(grids)
    t0 = time.perf_counter()
    choice = batch.tune(precision=precision, trials=2)
    tune_s = time.perf_counter() - t0
    opts = [dict(scheme=0, correction=1, clip=1, cfl=c["cfl"], cfl_start=0.5, ramp_iters=500,
                 precision=precision) for c in cases]
    batch.step(opts, iters=warmup, iters_per_graph=1)
    stream = torch.cuda.ExternalStream(batch.stream())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    stats = batch.step(opts, iters=steps, iters_per_graph=1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out = {"workload": f"batch-{len(cases)}-half-cylinders-64x48-to-512x384-mach6-20-air5-or-air11-CS1",
           "cases": len(cases), "cells": cells, "iterations": steps, "ms_per_iteration": ms / steps,
           "value": cells * steps / (ms / 1e3) / 1e6, "unit": "Mcell-iter/s", "tune_seconds": tune_s,
           "sweep_kernels_chosen": {str(kd): sum(1 for kk, _ in choice if kk == kd) for kd in sorted({kk for kk, _ in choice})},
           "cases_failed": sum(1 for st in stats if st["status_cell"] != -1),
           "launch": "one CUDA graph per iteration of all cases (each case's sweeps one cluster launch)"}
    del batch
    return out


def host_cpu():
    """(model name, logical cores) of the host."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
            for line in r.stdout.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return model or "unknown", os.cpu_count()


def run_iteration(args, rank, world, local):
    """The default workload: pseudo-time iterations of one grid (C2 unless --workload c3)."""
    import torch
    import paper_2403_03440_gb300 as P
    P.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    try:
        fp64_peak, fp64_kind = P.measure_fp64_rate(), "measured DFMA throughput (cs_measure_fp64_rate)"
    except P.CSError:
        fp64_peak, fp64_kind = FP64_NOMINAL_GFLOPS, "nominal FP64 (1.25 TFLOP/s; the measurement failed)"

    # Two grids run the same warm-up from the freestream: A times iterations W+1 .. W+K on the
    # device, B the same iterations end to end with host buffers.  The runs are deterministic,
    # so both legs time the same iterations from the same state (checked at the end).
    g = prepare_grid(P, args)
    ge = prepare_grid(P, args)
    N = g.ncell
    # L2 flush buffer (larger than the 126 MiB L2)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    g.profile(True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev0[k].record(stream)
            st = g.step(**step_kwargs(1))
            ev1[k].record(stream)
        torch.cuda.synchronize()
    prof = g.profile(False)
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    total_ms = job_time_ms(sum(step_ms), dist, "cuda")
    value = job_value(world, N, args.steps, total_ms)

    # ---- end to end through the C ABI with host buffers: every iteration uploads the state
    # from pinned host memory (cs_load_state: the run continues, warm starts and CFL ramp
    # kept), iterates and downloads the new state ----
    Qh = torch.empty((ge.nq, N), dtype=torch.float64, pin_memory=True).numpy()
    ge.get_state(Qh)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ge.load_state(Qh)
        ge.step(**step_kwargs(1))
        ge.get_state(Qh)
    e2e_s = time.perf_counter() - t0
    e2e = world * N * args.steps / e2e_s / 1e6
    nbytes = Qh.nbytes
    Qa = g.get_state()
    same = float(np.max(np.abs(Qa - Qh).max(axis=1) / np.maximum(np.abs(Qa).max(axis=1), 1e-300)))

    # ---- roofline of the dominant phase (live CUDA-event timing inside the timed region) ----
    dom = max(prof, key=lambda p: prof[p][0])
    dom_ms = prof[dom][0] / args.steps
    launches = sum(v[1] for v in prof.values())
    fp32_sweep = PRECISION == 1 and dom.startswith("sweep")
    flops = (FP32_FLOPS_PER_CELL_SWEEP if fp32_sweep else FP64_FLOPS_PER_CELL[dom]) * N
    peak = FP32_PEAK_GFLOPS if fp32_sweep else fp64_peak
    achieved = flops / (dom_ms / 1e3) / 1e9
    hbm, hbm_kind = measured_hbm_peak()
    wl = "c3" if C3 else "c2"
    algo_gbs = ALGO_BYTES_PER_CELL[wl] * N / (total_ms / args.steps / 1e3) / 1e9
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GFLOP/s",
            "frac": achieved / peak,
            "traffic": DRAM_BYTES_SWEEP_FP32 if fp32_sweep else DRAM_BYTES_PER_LAUNCH.get(dom),
            "kernel_phase": dom + (" (k_flux x 2 beside k_chem)" if dom == "flux" else ""),
            "peak_kind": ("FP32 from unit counts and clock (152 x 128 x 2 x 2.07 GHz)" if fp32_sweep
                          else fp64_kind),
            "flops_per_cell": flops / N,
            "flops_source": FLOPS_SOURCE,
            "note": ("the sweeps are bound by the latency of one dependent hyperplane step after "
                     "another, not by throughput" if dom.startswith("sweep")
                     else "FP64-ALU bound (ncu: FP64 pipe busy, DRAM far below its peak)"),
            "hbm": {"bytes_per_cell": ALGO_BYTES_PER_CELL[wl], "achieved": algo_gbs, "peak": hbm,
                    "unit": "GB/s", "frac": algo_gbs / hbm, "peak_kind": hbm_kind,
                    "scope": "whole iteration: algorithmic bytes of the four-pass design over the "
                             "device time per iteration"},
            "phases_ms_per_step": {p: prof[p][0] / args.steps for p in prof},
            "phases_fp64_frac": {p: (FP64_FLOPS_PER_CELL[p] * N / (prof[p][0] / args.steps / 1e3) / 1e9
                                     / fp64_peak) if prof[p][0] > 0 else None for p in prof}}
    if PRECISION == 1 and prof["sweep_fwd"][0] > 0:
        roof["phases_fp64_frac"]["sweep_fwd"] = (FP64_FLOPS_PER_CELL_SWEEP_MIXED * N / (prof["sweep_fwd"][0] / args.steps / 1e3)
                                                 / 1e9 / fp64_peak)
    if SCHEME[0] == 1:
        # coupled operator: the sweep and block phases run other kernels (k_ci_mat,
        # k_ci_mat_sweep, k_ci_block), whose FP64 counts were not taken; the sweep is reported
        # against HBM with its algorithmic bytes
        for p in ("spectral", "sweep_fwd", "sweep_bwd"):
            roof["phases_fp64_frac"][p] = None
        if dom == "sweep_fwd":
            gbs = CI_SWEEP_ALGO_BYTES / (dom_ms / 1e3) / 1e9
            roof.update({"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                         "traffic": None, "peak_kind": hbm_kind})

    extras = {}
    if rank == 0 and not C3 and args.scheme == "cs1" and args.dual_dt == 0 and not args.no_convergence:
        extras["time_to_1e8_c1"] = c1_time_to_drop()
        extras["time_to_1e8_c2"] = c2_time_to_drop()
    if rank == 0 and not C3 and args.scheme == "cs1" and args.dual_dt == 0 and not args.no_batch:
        try:
            extras["batch"] = batch_throughput(P, precision=PRECISION)
        except Exception as e:
            extras["batch"] = {"status": f"error: {e}"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, it, dt = oracle_rate(3, 30.0)
        model, ncpu = host_cpu()
        cpu = {"value": v, "unit": "Mcell-iter/s", "cores": 1, "kind": "oracle",
               "sample": f"{it} oracle iterations of the full 384x256 grid from the freestream ({dt:.1f} s)",
               "host_cpu": model, "host_logical_cores": ncpu, "build": ORACLE_BUILD}
        allc = oracle_rate_all_cores(3, 30.0)
        if allc is not None:
            cpu["all_cores"] = {"value": allc[0], "unit": "Mcell-iter/s", "cores": allc[3],
                                "sample": f"{allc[1]} oracle iterations of the same grid ({allc[2]:.1f} s)",
                                "build": ORACLE_BUILD_OMP}
    if rank == 0:
        line = {
            "metric": "Mcell-iter/s", "value": value, "unit": "Mcell-iter/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if PRECISION == 0 else "f64 residual/update, f32 operator",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": N, "species": 11, "temperatures": 2,
                       "scheme": {"cs1": "CS-1 split LU-SGS", "cs2": "CS-2 split LU-SGS",
                                  "ci": "coupled (CI) LU-SGS",
                                  "ci_eig": "coupled (CI) LU-SGS, eigenvalue splitting"}[args.scheme],
                       "cfl": f"{CFL_START} ramped geometrically to {CFL} over {RAMP} iterations",
                       "dtau_source": DTAU_SOURCE,
                       "timed_iterations": f"{args.warmup + 1}..{args.warmup + args.steps} from the freestream",
                       "l2": "flushed before every timed iteration (256 MiB write)",
                       "parallelism": f"replicas x{world}"},
            "clocks": clk.summary(),
            "e2e": {"value": e2e, "unit": "Mcell-iter/s", "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes, "same_iterations_as_value": same <= 1e-12,
                    "state_rel_diff_vs_value_leg": same},
            "gpu_launches": int(launches),
            "roofline": roof,
            "cpu_baseline": cpu,
            "last_stats": {k: (float(v) if isinstance(v, float) else v) for k, v in st.items()},
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
