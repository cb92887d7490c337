"""Benchmark: dense OMM-CG solves per second at 1e-8 relative energy accuracy.

One step = one whole solve of the 512-atom dense workload (8x8x8 jittered
grid, 8 orbitals per atom: m = 4096, n = 1024): the per-(H,S) setup
(Gershgorin shift, operand packing) plus conjugate-gradient minimisation from
the seeded W0 until the RelTol test and, for the mixed form, the
orthonormality test pass.  H, S and W0 are resident in HBM when the timed
region starts (value); the e2e figure repeats the same solves through the C
ABI from pinned host buffers, copies included.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl omm|reference]
                    [--precision mixed|fp64]

Multi-GPU runs (torchrun) are independent replicas: each rank solves its own
systems; only the timing is reduced (max over ranks).
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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = dict(dims=(8, 8, 8), seed=0)
METRIC = "OMM solves/s & time-to-converge @1e-8 rel energy; p50/p99 latency; %roofline"
UNIT = "solves/s"
TOL = {"fp64": dict(tol=1e-10, orth_tol=0.0), "mixed": dict(tol=1e-10, orth_tol=1e-6)}


def workload_name(sysm):
    nx, ny, nz = WORKLOAD["dims"]
    return (f"dense OMM-CG, {sysm.natoms} atoms ({nx}x{ny}x{nz} jittered grid), 8 orbitals/atom, "
            f"m={sysm.m}, n={sysm.n}, seed {WORKLOAD['seed']}")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def golden():
    p = os.path.join(ROOT, "tests", "golden", "oracle_reference.json")
    return json.load(open(p)) if os.path.exists(p) else {}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
            # the timed region starts once nvidia-smi has taken its first sample: its
            # start-up (NVML initialisation) competes with the host driving the GPU
            t_end = time.perf_counter() + 1.0
            while time.perf_counter() < t_end and self.proc.poll() is None and os.path.getsize(self.file.name) == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, sm_max_nominal=2070.0):
        if self.proc is None or self.file is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.file.flush()
        rows = []
        for line in open(self.file.name):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(parts)
            except Exception:
                pass
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else sm_max_nominal, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------- distributed
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def barrier_max(value: float, ws: int):
    """Max of a per-rank value over the job (NCCL on the GPUs, gloo on host tensors)."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- oracle (CPU) arm
def oracle_sample(sysm, H, S, W0, n_iter: int):
    """Time the oracle's setup and n_iter CG steps on the host cores."""
    from oracle import omm as O
    t0 = time.perf_counter()
    eta = O.gershgorin_eta(H, S)
    t1 = time.perf_counter()
    res = O.omm_cg(H, S, W0, tol=0.0, eta=eta, max_iter=n_iter)
    t2 = time.perf_counter()
    return t1 - t0, (t2 - t1) / max(1, res.iters)


def cpu_baseline(sysm, H, S, W0, full_iters: int, n_iter: int = 2):
    cores = len(os.sched_getaffinity(0))
    t_setup, t_iter = oracle_sample(sysm, H, S, W0, n_iter)
    t_solve = t_setup + full_iters * t_iter
    return {"value": 1.0 / t_solve, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"oracle Gershgorin setup + {n_iter} FP64 CG steps on this workload, "
                       f"{t_iter:.3f} s/step, scaled to the oracle's {full_iters} steps per solve"),
            "seconds_per_solve": t_solve}


def run_reference(args):
    """The oracle on this workload, timed on the host cores: one whole FP64 solve
    (Gershgorin shift and CG to the same RelTol as the GPU arm's FP64 form),
    measured, not scaled.  A solve takes about 40 s on 16 cores, so this arm
    times exactly one, whatever --steps and --warmup say (the line reports
    steps = 1, warmup = 0 and says so)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import omm as O
    sysm = synth.make_system(*WORKLOAD["dims"], seed=WORKLOAD["seed"])
    H, S = sysm.dense_H(), sysm.dense_S()
    W0 = np.asfortranarray(sysm.W0_dense())
    tol = TOL["fp64"]["tol"]
    t0 = time.perf_counter()
    res = O.omm_cg(H, S, W0, tol=tol)
    t = time.perf_counter() - t0
    e_exact = golden().get("c2", {}).get("exact_E")
    cores = len(os.sched_getaffinity(0))
    line = {
        "impl": "reference", "metric": METRIC, "value": 1.0 / t, "unit": UNIT, "n_gpus": args.gpus,
        "steps": 1, "warmup": 0, "ms_per_step": 1e3 * t, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(sysm), "tol": tol,
                   "steps_note": (f"one whole oracle solve is timed (requested --steps {args.steps} "
                                  f"--warmup {args.warmup}); a solve takes tens of seconds on the host")},
        "accuracy": {"E": res.E, "iters": res.iters, "status": res.status,
                     "rel_err": abs(res.E - e_exact) / abs(e_exact) if e_exact else None},
        "cpu_baseline": {"value": 1.0 / t, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"one whole oracle solve of this workload ({res.iters} CG steps), measured"},
        "e2e": {"value": 1.0 / t, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def fp64_gemm_peak(size=8192, reps=5):
    """FP64 throughput of cuBLAS DGEMM (torch.matmul in float64) on this GPU: the
    measured FP64 denominator of the FP64 rooflines, as the driver's BF16 peak
    is cuBLAS's.  Best of `reps` timed products after one warm-up, TFLOP/s."""
    import torch
    a = torch.randn(size, size, dtype=torch.float64, device="cuda")
    b = torch.randn(size, size, dtype=torch.float64, device="cuda")
    c = a @ b
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b, c
    return 2.0 * size ** 3 / (best * 1e-3) / 1e12


# ---------------------------------------------------------------- GPU arm
def run_omm(args):
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2209_05934_gb300 import omm

    omm.lib()
    prec = args.precision
    sysm = synth.make_system(*WORKLOAD["dims"], seed=WORKLOAD["seed"])
    H, S = sysm.dense_H(), sysm.dense_S()
    W0 = np.asfortranarray(sysm.W0_dense())
    m, n = sysm.m, sysm.n
    dev = lambda a: torch.from_numpy(np.asfortranarray(a)).to("cuda")
    Hd, Sd, W0d = dev(H), dev(S), dev(W0)
    Wout = torch.zeros((n, m), dtype=torch.float64, device="cuda").T
    # a stream of its own (not the legacy default stream), so the library can
    # replay its chunks of CG steps as CUDA graphs; the inputs above are complete
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    opts = dict(precision=omm.PREC_MIXED if prec == "mixed" else omm.PREC_FP64,
                orth_tol=TOL[prec]["orth_tol"], stream=stream.cuda_stream, cholesky=int(args.cholesky),
                split_digits=args.split_digits, gemm_pair=args.gemm_pair, gemm_persistent=args.gemm_persistent,
                dir_digits=args.dir_digits)
    solver = omm.Solver(m, n, 8, **opts)
    tol = TOL[prec]["tol"]

    def step():
        solver.set_HS(Hd, Sd)
        E, iters, st = solver.solve(W0d, tol=tol, W_out=Wout)
        return E, iters

    for _ in range(args.warmup):
        E, iters = step()
    torch.cuda.synchronize()
    # per-stage device times for the roofline come from one profiled step
    # outside the timed region (profiling records events around every stage
    # and turns off the graph replay of CG chunks)
    solver.set_profiling(True)
    solver.stage_times(reset=True)
    step()
    torch.cuda.synchronize()
    solver.set_profiling(False)
    ms_stage, n_stage = solver.stage_times(reset=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = omm.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat = []
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            E, iters = step()
            b.record(stream)
            lat.append((a, b))
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = omm.kernel_launches() - launches0
    t_ms = ev0.elapsed_time(ev1)
    lat_ms = sorted(a.elapsed_time(b) for a, b in lat)
    if ws > 1:
        torch.distributed.barrier()
    t_max = barrier_max(t_ms, ws)
    diag = solver.diag()
    # accuracy against the exact minimum (2 x sum of the n lowest eigenvalues)
    g = golden().get("c2", {})
    e_exact = g.get("exact_E")
    rel_err = abs(E - e_exact) / abs(e_exact) if e_exact else None

    # ---- the density matrix of the solution (Eq. 5), what an SCF step consumes
    rho_d = torch.zeros((m, m), dtype=torch.float64, device="cuda").T
    solver.get_density(omm.DENSITY_RHO, rho_d)          # first call allocates its workspace
    torch.cuda.synchronize()
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for _ in range(3):
        solver.get_density(omm.DENSITY_RHO, rho_d)
    r1.record(stream)
    torch.cuda.synchronize()
    density = {"rho_ms": r0.elapsed_time(r1) / 3, "trace_rho_S": float(torch.sum(rho_d * Sd).item()),
               "electrons": 2 * n}
    del rho_d

    # ---- the plain FP64 GPU form beside the chosen one: one whole FP64 solve
    fp64_beside = None
    if prec == "mixed" and not args.no_fp64_beside:
        warm = omm.Solver(m, n, 8, precision=omm.PREC_FP64, stream=stream.cuda_stream, max_iter=2,
                          cholesky=int(args.cholesky))
        warm.set_HS(Hd, Sd)
        warm.solve(W0d, tol=TOL["fp64"]["tol"], raise_on_error=False)
        warm.close()
        s64 = omm.Solver(m, n, 8, precision=omm.PREC_FP64, stream=stream.cuda_stream,
                         orth_tol=TOL["mixed"]["orth_tol"], cholesky=int(args.cholesky))
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        s64.set_HS(Hd, Sd)
        E64, it64, st64 = s64.solve(W0d, tol=TOL["fp64"]["tol"], raise_on_error=False)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1)
        d64 = s64.diag()
        fp64_beside = {"form": "plain FP64 on CUDA cores (DFMA GEMMs), same handle API", "ms_per_solve": ms64,
                       "solves_per_s": 1e3 / ms64, "E": E64, "status": int(st64), "iters": int(it64),
                       "orth": d64.orth, "tol": TOL["fp64"]["tol"],
                       "rel_err": abs(E64 - e_exact) / abs(e_exact) if e_exact else None,
                       "chosen_form_speedup": ms64 / (t_max / args.steps)}
        s64.close()

    # ---- kinetic-energy preconditioning (Eq. 6) on the kinetic workload H + T:
    # the same S and W0, a spectrum widened by the kinetic term; one warm solve
    # per form (P is formed, chunks captured), then one timed solve each
    kinetic = None
    if prec == "mixed" and not args.cholesky and not args.no_kinetic:
        Hk, Tk = dev(sysm.dense_H_kinetic()), dev(sysm.dense_T())
        kinetic = {"workload": workload_name(sysm) + ", H + T (kinetic onsite 0.5-400 eV)",
                   "tau_T_eV": omm.default_options().tau_T}
        for name, extra in (("plain", {}), ("precon", {"precon": -1})):
            sk = omm.Solver(m, n, 8, **opts, **extra)
            sk.set_HS(Hk, Sd)
            if extra:
                sk.set_T(Tk)
            sk.solve(W0d, tol=tol, raise_on_error=False)
            torch.cuda.synchronize()
            k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            k0.record(stream)
            Ek, itk, stk = sk.solve(W0d, tol=tol, raise_on_error=False)
            k1.record(stream)
            torch.cuda.synchronize()
            dk = sk.diag()
            kinetic[name] = {"ms_per_solve": k0.elapsed_time(k1), "iters": int(itk), "iters_mixed": dk.iters_mixed,
                             "iters_refine": dk.iters_refine, "E": Ek, "status": int(stk), "orth": dk.orth}
            sk.close()
        kinetic["E_rel_diff"] = abs(kinetic["precon"]["E"] - kinetic["plain"]["E"]) / abs(kinetic["plain"]["E"])
        del Hk, Tk

    # ---- e2e: the same solves through the C ABI from pinned host buffers
    Hh = torch.from_numpy(np.asfortranarray(H)).pin_memory()
    Sh = torch.from_numpy(np.asfortranarray(S)).pin_memory()
    W0h = torch.from_numpy(np.asfortranarray(W0)).pin_memory()
    Wh = torch.zeros((n, m), dtype=torch.float64).pin_memory().T
    solver_h = omm.Solver(m, n, 8, **opts)
    solver_h.set_HS(Hh, Sh)
    solver_h.solve(W0h, tol=tol, W_out=Wh)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(1, min(args.steps, 3))
    e0.record(stream)
    for _ in range(e2e_steps):
        solver_h.set_HS(Hh, Sh)
        Eh, _, _ = solver_h.solve(W0h, tol=tol, W_out=Wh)
    e1.record(stream)
    torch.cuda.synchronize()
    t_e2e = barrier_max(e0.elapsed_time(e1), ws)
    solver_h.close()

    # ---- roofline of the dominant stage
    pk, pk_kind = peaks()
    fp64_peak = fp64_gemm_peak(4096)
    pk = dict(pk, fp64_tflops=fp64_peak)
    # the dominant kernel is the split GEMM (tc_gemm); its products stage launches nothing
    # else, while the gradient and contraction stages also hold exact-digit GEMMs.  The
    # FP64 form reports its largest stage.
    dom = 0 if prec == "mixed" else (int(np.argmax(ms_stage[:6])) if sum(ms_stage[:6]) > 0 else 0)
    roof = roofline_entry(prec, dom, ms_stage, n_stage, m, n, pk, pk_kind)
    if roof is not None and prec == "mixed":
        # BF16 digit-pair products per FP64-equivalent product in the products stage:
        # both phases multiply the split_digits digits of [H'; S] by D, which carries
        # one digit (dir_digits = 1: 2 pairs with two digits, 3 with three) or
        # split_digits digits (3 or 6 pairs); bf16_issue_frac counts the BF16 flops
        # the tensor cores issue against the same measured BF16 peak
        if args.dir_digits == 1:
            pairs = args.split_digits
        else:
            pairs = 3 if args.split_digits == 2 else 6
        roof["bf16_pairs_per_product"] = pairs
        roof["bf16_issue_frac"] = roof["frac"] * pairs
    tkey = (roof or {}).get("kernel"), args.split_digits, args.dir_digits, bool(args.gemm_pair)
    if roof is not None and prec == "mixed" and tkey in TRAFFIC:
        roof["traffic"] = TRAFFIC[tkey]["bytes_per_launch"]
        roof["traffic_source"] = TRAFFIC[tkey]["source"]
        roof["tensor_pipe_active_ncu"] = TRAFFIC[tkey]["tensor_pipe_active"]

    if rank != 0:
        solver.close()
        return
    full_iters = int(g.get("oracle_iters", iters))
    cpu = cpu_baseline(sysm, H, S, W0, full_iters) if ws == 1 else None
    value = ws * args.steps / (t_max / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == "fp64" else "bf16-split+f64",
        "data": "synthetic",
        "config": {"workload": workload_name(sysm) + (" cholesky-reduced" if args.cholesky else ""),
                   "precision": prec, "tol": tol, "cholesky": bool(args.cholesky),
                   "split_digits": args.split_digits, "gemm_pair": bool(args.gemm_pair),
                   "gemm_persistent": bool(args.gemm_persistent), "dir_digits": args.dir_digits,
                   "refine": "exact-digit tensor cores" if prec == "mixed" else None,
                   "orth_tol": TOL[prec]["orth_tol"], "parallelism": f"replicas x{ws}",
                   "l2": "working set (H, S = 256 MiB, plus W/D/products) exceeds the 129 MB L2"},
        "time_to_converge_ms": {"p50": lat_ms[len(lat_ms) // 2],
                                "p99": lat_ms[min(len(lat_ms) - 1, int(math.ceil(0.99 * len(lat_ms))) - 1)]},
        "accuracy": {"E": E, "exact_E": e_exact, "rel_err": rel_err, "orth": diag.orth,
                     "iters": diag.iters, "iters_mixed": diag.iters_mixed,
                     "iters_refine": diag.iters_refine},
        "stages_ms_per_step": {name: ms_stage[i] for i, name in enumerate(STAGES)},   # one profiled step
        "roofline": roof,
        "cpu_baseline": cpu,
        "fp64_gpu_beside": fp64_beside,
        "density_matrix": density,
        "kinetic_preconditioning": kinetic,
        "fp64_peak": {"tflops": fp64_peak, "how": "cuBLAS DGEMM via torch.matmul, float64 4096^3, best of 5, "
                                                 "this run"},
        "e2e": {"value": ws * e2e_steps / (t_e2e / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": int(2 * m * m * 8 + m * n * 8),
                "d2h_bytes_per_step": int(m * n * 8 + 8)},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if args.extras:
        # short runs of the other workloads, so that the default line carries them too
        import copy
        solver.close()
        torch.cuda.synchronize()
        ex = {}
        a3 = copy.copy(args)
        a3.steps, a3.max_iter, a3.screen_eps = 1, 20, 0.0
        r3 = run_c3(a3, quiet=True)
        ex["c3_20_steps"] = {"workload": r3["config"]["workload"], "ms_per_iteration": r3["ms_per_iteration"],
                             "stages_ms": r3["stages_ms_20_steps"], "roofline_fp64": r3["roofline"],
                             "fp64_peak_tflops": r3["fp64_peak_tflops"], "nnzb": r3["config"]["nnzb"],
                             "note": "20 CG steps from W0 (the converged solve is bench.py --config c3)"}
        a4 = copy.copy(args)
        a4.steps, a4.warmup, a4.tile_mode = 2, 2, -1
        r4 = run_c4(a4, quiet=True)
        ex["c4"] = {k: r4[k] for k in ("value", "unit", "ms_per_step", "tuning", "streams", "one_by_one",
                                       "results_equal_alone", "all_ok", "iters")}
        ex["c4"]["workload"] = r4["config"]["workload"]
        a5 = copy.copy(args)
        a5.sequences, a5.rates, a5.fp64_sequences = 12, [50.0], 0
        r5 = run_c5(a5, quiet=True)
        ex["c5_short"] = {"workload": r5["config"]["workload"], "rate": r5["rates"][0],
                          "note": "12 sequences at one rate (the full sweep is bench.py --config c5)"}
        line["other_workloads"] = ex
        print(json.dumps(line), flush=True)
        return
    print(json.dumps(line), flush=True)
    solver.close()


STAGES = ["products", "contract", "linesearch", "update", "gradient", "direction", "setup", "start",
          "pack", "anchor", "precon"]


# DRAM bytes per launch of the dominant kernel, from one ncu capture of the current
# kernel on this workload, keyed by (stage, split_digits, dir_digits, CTA pairs);
# an entry is removed whenever its kernel changes, and added when it is captured again.
TRAFFIC = {("products", 2, 1, True): {
    "bytes_per_launch": 150.687488e6 + 36.777728e6,
    "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one first-phase products launch "
              "(tc_gemm_pair_kernel with the specialised FP32 epilogue, two digits of [H'; S], one digit "
              "of D), m=4096, n=1024",
    # the same capture's sm__pipe_tensor_cycles_active (of the SMs' active and of elapsed cycles)
    "tensor_pipe_active": {"of_active_cycles": 0.663, "of_elapsed_cycles": 0.542}}}


def roofline_entry(prec, dom, ms_stage, n_stage, m, n, pk, pk_kind):
    if n_stage[dom] == 0:
        return None
    avg_ms = ms_stage[dom] / n_stage[dom]
    # algorithmic flops per launch of each stage (dense)
    flops = {0: 4.0 * m * m * n, 1: 2.0 * (2 * n) * (2 * n) * m, 4: 2.0 * m * n * (2 * n)}
    if prec == "fp64":
        fp64_peak = pk["fp64_tflops"]
        f = flops.get(dom)
        if f is None:
            return None
        ach = f / (avg_ms * 1e-3) / 1e12
        return {"bound": "alu", "kernel": STAGES[dom], "achieved": ach, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": ach / fp64_peak, "traffic": None,
                "peak_source": "cuBLAS DGEMM (4096^3, best of 5) measured in this run"}
    f = flops.get(dom)
    if f is None:
        return None
    ach = f / (avg_ms * 1e-3) / 1e12
    peak = pk["bf16_tflops_sustained"]
    return {"bound": "tensor", "kernel": STAGES[dom], "achieved": ach, "peak": peak,
            "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
            "peak_source": f"bf16 sustained ({pk_kind}); achieved counts FP64-equivalent flops"}


C3 = dict(dims=(16, 16, 16), seed=0, radius=6.0)


def sparse_setup(omm, max_iter, precision=None):
    sysm = synth.make_system(*C3["dims"], seed=C3["seed"])
    rp, col, Hv, Sv = sysm.bsr()
    wrp, wcol = sysm.w_pattern(C3["radius"])
    import torch
    s = omm.SparseSolver(sysm.m, sysm.n, 8, 2, rp, col, wrp, wcol, max_iter=max_iter,
                         stream=torch.cuda.current_stream().cuda_stream,
                         precision=omm.PREC_FP64 if precision is None else precision)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
    return sysm, s, dev(Hv), dev(Sv), dev(sysm.W0_bsr_values(C3["radius"]))


def run_profile_c3(args):
    import torch
    from paper_2209_05934_gb300 import omm

    omm.lib()
    prec = omm.PREC_MIXED if args.c3_precision == "mixed" else omm.PREC_FP64
    sysm, s, Hd, Sd, W0d = sparse_setup(omm, args.max_iter if args.max_iter > 0 else 10, prec)
    s.set_profiling(True)
    s.set_HS(Hd, Sd)
    E, iters, st = s.solve(W0d, tol=0.0, raise_on_error=False)
    torch.cuda.synchronize()
    ms, cnt = s.stage_times()
    # rho on the pattern of S: first call builds its gather lists, the second is timed
    t0 = time.perf_counter()
    s.get_density(omm.DENSITY_RHO)
    t_first = time.perf_counter() - t0
    t0 = time.perf_counter()
    s.get_density(omm.DENSITY_RHO)
    t_rho = time.perf_counter() - t0
    print(json.dumps({"profile": True, "config": "c3", "E": E, "iters": iters, "status": st, "nnzb": s.nnzb,
                      "rho_ms": {"first_call_with_list_build": 1e3 * t_first,
                                 "call_including_host_copy": 1e3 * t_rho},
                      "stages_ms": {n: ms[i] for i, n in enumerate(STAGES)},
                      "stage_launches": {n: int(cnt[i]) for i, n in enumerate(STAGES)}}), flush=True)
    s.close()


def run_c3(args, quiet=False):
    """The linear-scaling workload solved to convergence: 4096 atoms (16^3),
    m = 32768, n = 8192, R_C = 6 A, FP64 block-sparse, RelTol 1e-10 (or
    --max-iter steps).  A 20-step handle warms up (gather lists uploaded,
    modules loaded) and gives the per-stage times of the sparse kernels'
    rooflines (FP64 flops and algorithmic bytes per launch); the timed solve
    runs from W0 with set_HS inside each step."""
    import torch
    from paper_2209_05934_gb300 import omm

    omm.lib()
    sysm = synth.make_system(*C3["dims"], seed=C3["seed"])
    rp, col, Hv, Sv = sysm.bsr()
    wrp, wcol = sysm.w_pattern(C3["radius"])
    stream = torch.cuda.Stream()
    max_iter = args.max_iter if args.max_iter > 0 else 20000
    prec = omm.PREC_MIXED if args.c3_precision == "mixed" else omm.PREC_FP64
    mk = lambda k: omm.SparseSolver(sysm.m, sysm.n, 8, 2, rp, col, wrp, wcol, max_iter=k,
                                    stream=stream.cuda_stream, screen_eps=args.screen_eps, precision=prec)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
    Hd, Sd, W0d = dev(Hv), dev(Sv), dev(sysm.W0_bsr_values(C3["radius"]))
    torch.cuda.synchronize()
    tol = 1e-10
    # warm-up and per-stage device times: 20 CG steps on their own handle
    p = mk(20)
    p.set_HS(Hd, Sd)
    p.solve(W0d, tol=tol, raise_on_error=False)
    torch.cuda.synchronize()
    p.set_profiling(True)
    p.stage_times(reset=True)
    p.set_HS(Hd, Sd)
    p.solve(W0d, tol=tol, raise_on_error=False)
    torch.cuda.synchronize()
    ms, cnt = p.stage_times(reset=True)
    p.close()
    s = mk(max_iter)

    def step():
        s.set_HS(Hd, Sd)
        return s.solve(W0d, tol=tol, raise_on_error=False)

    launches0 = omm.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            E, iters, st = step()
        e1.record(stream)
        torch.cuda.synchronize()
    t_ms = e0.elapsed_time(e1) / args.steps
    launches = omm.kernel_launches() - launches0
    fp64_peak = fp64_gemm_peak(4096)
    nnz = s.nnzb
    TRIPLES = sparse_triples(sysm, rp, col, wrp, wcol)
    d = s.diag()
    rows = {
        "products": {"flop": 2 * 2 * 8 * 8 * 2 * TRIPLES["HW"], "bytes": 8 * (2 * 64 * nnz["H"] + 16 * nnz["W"]
                                                                              + 2 * 16 * nnz["HW"])},
        # X, Y on all of P_N; D^T H'D, D^T S D (symmetric) on its upper triangle: ~3 of the 4
        "contract": {"flop": 3 * 2 * 2 * 2 * 8 * TRIPLES["N"], "bytes": 8 * (2 * 16 * nnz["W"] + 2 * 16 * nnz["HW"]
                                                                             + 4 * 4 * nnz["N"])},
        "gradient": {"flop": 2 * 2 * 8 * 2 * 2 * TRIPLES["G"], "bytes": 8 * (2 * 16 * nnz["HW"] + 2 * 4 * nnz["N"]
                                                                             + 16 * nnz["W"])},
    }
    roof = {}
    # the mixed form's first phase runs these products in FP32 (half the bytes); its
    # ceiling is the FP32 pipe: 152 SMs x 128 lanes x 2 flop x the clock
    fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    for i, name in enumerate(STAGES):
        if name in rows and cnt[i] > 0:
            per = ms[i] / cnt[i]
            tf = rows[name]["flop"] / (per * 1e-3) / 1e12
            if args.c3_precision == "mixed":
                roof[name] = {"ms_per_launch": per, "fp32_tflops": tf, "frac_fp32": tf / fp32_peak,
                              "hbm_gbs": 0.5 * rows[name]["bytes"] / (per * 1e-3) / 1e9,
                              "bound": "alu (FP32 pipe, 80.5 TFLOP/s at 2.07 GHz)"}
            else:
                roof[name] = {"ms_per_launch": per, "fp64_tflops": tf, "frac_fp64": tf / fp64_peak,
                              "hbm_gbs": rows[name]["bytes"] / (per * 1e-3) / 1e9,
                              "bound": "alu (FP64 pipe; peak: cuBLAS DGEMM measured in this run)"}
    line = {"metric": "OMM solves/s & time-to-converge, linear-scaling form", "value": 1e3 / t_ms,
            "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "warmup": 1, "ms_per_step": t_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": (f"linear-scaling OMM-CG, 4096 atoms (16x16x16 jittered grid), m={sysm.m}, "
                                    f"n={sysm.n}, R_C={C3['radius']} A, BSR 8x8 / 8x2, filter 1e-8"),
                       "tol": tol, "max_iter": max_iter, "screen_eps": args.screen_eps, "nnzb": nnz,
                       "precision": args.c3_precision},
            "iters_mixed": int(d.iters_mixed), "iters_refine": int(d.iters_refine),
            "time_to_converge_ms": t_ms, "iters": int(iters), "status": int(st), "E": E, "eta": d.eta,
            "ms_per_iteration": t_ms / max(1, int(iters)),
            "stages_ms_20_steps": {n_: ms[i] for i, n_ in enumerate(STAGES)},
            "roofline": roof, "fp64_peak_tflops": fp64_peak,
            "gpu_launches": int(launches), "clocks": clk.summary()}
    if not quiet:
        print(json.dumps(line), flush=True)
    s.close()
    return line


def sparse_triples(sysm, rp, col, wrp, wcol):
    """Block-product triples of the sparse step: H'W (H block (I,K) x W block (K,J)),
    the contractions W^T (H'W) (W block (I,J1) x H'W block (I,J2)) and the masked
    gradient (H'W block (I,K) x N block (K,J) kept on W's pattern)."""
    import scipy.sparse as sps
    N = sysm.natoms
    PH = sps.csr_matrix((np.ones(len(col)), col, rp), shape=(N, N))
    PW = sps.csr_matrix((np.ones(len(wcol)), wcol, wrp), shape=(N, N))
    PHW = (PH @ PW).tocsr()
    PHW.data[:] = 1.0
    PN = (PW.T @ PHW).tocsr()
    PN.data[:] = 1.0
    hw = float((PH @ PW).sum())
    n_ = float((PW.T @ PHW).sum())
    g = float((PHW @ PN).multiply(PW).sum())
    return {"HW": hw, "N": n_, "G": g}


def run_profile(args):
    """One solve, nothing else: the command that ncu captures of the solve's kernels run."""
    import torch
    from paper_2209_05934_gb300 import omm

    omm.lib()
    if args.config == "c3":
        run_profile_c3(args)
        return
    sysm = synth.make_system(*WORKLOAD["dims"], seed=WORKLOAD["seed"])
    dev = lambda a: torch.from_numpy(np.asfortranarray(a)).to("cuda")
    H, S, W0 = dev(sysm.dense_H()), dev(sysm.dense_S()), dev(sysm.W0_dense())
    prec = args.precision
    opts = dict(precision=omm.PREC_MIXED if prec == "mixed" else omm.PREC_FP64,
                orth_tol=TOL[prec]["orth_tol"], stream=torch.cuda.current_stream().cuda_stream,
                cholesky=int(args.cholesky), split_digits=args.split_digits, gemm_pair=args.gemm_pair,
                gemm_persistent=args.gemm_persistent, dir_digits=args.dir_digits)
    if args.max_iter > 0:
        opts["max_iter"] = args.max_iter
    solver = omm.Solver(sysm.m, sysm.n, 8, **opts)
    solver.set_profiling(True)
    solver.set_HS(H, S)
    E, iters, st = solver.solve(W0, tol=TOL[prec]["tol"], raise_on_error=False)
    torch.cuda.synchronize()
    ms, cnt = solver.stage_times()
    d = solver.diag()
    print(json.dumps({"profile": True, "precision": prec, "E": E, "iters": iters, "status": st,
                      "iters_mixed": d.iters_mixed, "iters_refine": d.iters_refine, "orth": d.orth,
                      "stages_ms": {n: ms[i] for i, n in enumerate(STAGES)},
                      "stage_launches": {n: int(cnt[i]) for i, n in enumerate(STAGES)},
                      "gpu_launches": omm.kernel_launches()}), flush=True)
    solver.close()


# ---------------------------------------------------------------- MD steps
def run_md(args):
    """Successive MD snapshots of a straight-line trajectory (section "C† matrix
    initialization and update"): each step's solve starts fresh from W0, from
    the previous step's W carried onto the new pattern, or from the linear
    extrapolation of the two previous steps (omm_md_guess).  Dense: the C2
    geometry, mixed precision, one handle per chain.  Sparse: a 6x6x6 system,
    R_C = 4.5 A, FP64, one handle per snapshot (the W pattern changes)."""
    import torch
    from paper_2209_05934_gb300 import omm

    omm.lib()
    nsteps, step = args.md_steps, args.md_step
    dev = lambda a: torch.from_numpy(np.asfortranarray(a)).to("cuda")
    stream = torch.cuda.Stream()
    launches0 = omm.kernel_launches()

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        r = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return r, a.elapsed_time(b)

    # ---- dense chains
    snaps = [synth.make_md_system(*WORKLOAD["dims"], seed=WORKLOAD["seed"], t=float(t), step=step)
             for t in range(nsteps)]
    m, n = snaps[0].m, snaps[0].n
    HS = [(dev(s.dense_H()), dev(s.dense_S())) for s in snaps]
    W0 = dev(snaps[0].W0_dense())
    opts = dict(precision=omm.PREC_MIXED, orth_tol=TOL["mixed"]["orth_tol"], stream=stream.cuda_stream)
    tol = TOL["mixed"]["tol"]
    warm = omm.Solver(m, n, 8, **opts)       # graphs captured, modules loaded
    warm.set_HS(*HS[0])
    warm.solve(W0, tol=tol)
    warm.close()
    chains = {"fresh": [omm.Solver(m, n, 8, **opts)], "carried": [omm.Solver(m, n, 8, **opts)],
              "extrapolated": [omm.Solver(m, n, 8, **opts), omm.Solver(m, n, 8, **opts)]}
    dense = {k: [] for k in chains}
    for t in range(nsteps):
        for mode, hs in chains.items():
            h = hs[t % len(hs)]
            h.set_HS(*HS[t])
            if mode == "fresh" or t == 0:
                (E, it, st), ms = timed(lambda: h.solve(W0, tol=tol, raise_on_error=False))
            else:
                if mode == "extrapolated" and t >= 2:
                    # h holds W_{t-2}, the other handle W_{t-1}: 2 W_{t-1} - W_{t-2} in place
                    h.md_guess(hs[(t - 1) % 2], h)
                elif mode == "extrapolated":
                    h.md_guess(hs[(t - 1) % 2])
                (E, it, st), ms = timed(lambda: h.solve(None, tol=tol, raise_on_error=False))
            dense[mode].append({"t": t, "iters": int(it), "ms": ms, "E": E, "status": int(st)})
    for hs in chains.values():
        for h in hs:
            h.close()
    del HS

    # ---- sparse chains: one handle per snapshot and chain
    R_C = 4.5
    ssnaps = [synth.make_md_system(6, 6, 6, seed=1, t=float(t), step=step) for t in range(nsteps)]
    sparse = {k: [] for k in ("fresh", "carried", "extrapolated")}
    guess_ms = []
    for mode in sparse:
        prev = []
        for t, sysm in enumerate(ssnaps):
            rp, col, Hv, Sv = sysm.bsr()
            wrp, wcol = sysm.w_pattern(R_C)
            h = omm.SparseSolver(sysm.m, sysm.n, 8, 2, rp, col, wrp, wcol, stream=stream.cuda_stream,
                                 max_iter=args.md_max_iter)
            h.set_HS(Hv, Sv)
            if mode == "fresh" or t == 0:
                (E, it, st), ms = timed(lambda: h.solve(sysm.W0_bsr_values(R_C), tol=1e-10, raise_on_error=False))
            else:
                g0 = time.perf_counter()
                h.md_guess(prev[-1], prev[-2] if mode == "extrapolated" and t >= 2 else None)
                guess_ms.append((time.perf_counter() - g0) * 1e3)
                (E, it, st), ms = timed(lambda: h.solve(None, tol=1e-10, raise_on_error=False))
            sparse[mode].append({"t": t, "iters": int(it), "ms": ms, "E": E, "status": int(st),
                                 "nnzb_W": int(len(wcol))})
            prev.append(h)
            if len(prev) > 2:
                prev.pop(0).close()
        for h in prev:
            h.close()
    print(json.dumps({"md": True, "step_A_per_unit_t": step, "steps": nsteps,
                      "dense": {"workload": workload_name(snaps[0]) + ", MD snapshots", "precision": "mixed",
                                "tol": tol, "chains": dense},
                      "sparse": {"workload": f"localised OMM-CG, 216 atoms (6x6x6), m={ssnaps[0].m}, "
                                             f"n={ssnaps[0].n}, R_C={R_C} A, MD snapshots",
                                 "precision": "fp64", "tol": 1e-10, "chains": sparse,
                                 "md_guess_ms_host_wall": guess_ms},
                      "gpu_launches": int(omm.kernel_launches() - launches0)}), flush=True)


# ---------------------------------------------------------------- C4: batched uneven solves
def run_c4(args, quiet=False):
    """64 uneven dense systems (k-point/spin-like), mixed precision, solved
    together: as one group (each CG step's split products as one persistent
    grouped launch over all systems, tile mode autotuned, chunks of steps as a
    CUDA graph) and, for comparison in the same run, one handle per stream driven
    together, and one by one."""
    import torch
    from paper_2209_05934_gb300 import omm

    omm.lib()
    count = args.batch
    sizes = synth.batch_sizes(count, seed=4, lo=32, hi=384)
    systems = [synth.make_batch_system(int(N), seed=4000 + i) for i, N in enumerate(sizes)]
    dev = lambda a: torch.from_numpy(np.asfortranarray(a)).to("cuda")
    data = [(dev(s.dense_H()), dev(s.dense_S()), dev(s.W0_dense())) for s in systems]
    solvers = [omm.Solver(s.m, s.n, 8, precision=omm.PREC_MIXED, orth_tol=1e-6, graphs=args.graphs,
                          gemm_pair=args.gemm_pair, dir_digits=args.dir_digits) for s in systems]

    def set_all():
        for sv, (H, S, _) in zip(solvers, data):
            sv.set_HS(H, S)

    def grouped_step():
        set_all()
        E, it, st, rc = omm.batch_solve_grouped(solvers, [d[2] for d in data], tol=1e-10, tile_mode=args.tile_mode)
        return E, it, st

    def streams_step():
        set_all()
        return omm.batch_solve(solvers, [d[2] for d in data], tol=1e-10)

    def timed(fn, steps):
        for _ in range(args.warmup):
            out = fn()
        torch.cuda.synchronize()
        l0 = omm.kernel_launches()
        t0 = time.perf_counter()
        with ClockSampler(0) as clk:
            for _ in range(steps):
                out = fn()
            torch.cuda.synchronize()
        return out, (time.perf_counter() - t0) / steps, omm.kernel_launches() - l0, clk.summary()

    # the two executions alternate (streams, grouped, streams, grouped) so that
    # neither gains from running second
    (Es, its, sts), t_s1, _, _ = timed(streams_step, max(1, args.steps // 2))
    (Eg, itg, stg), t_g1, launches, clocks = timed(grouped_step, args.steps)
    modes, tune_ms = omm.batch_last_tuning()
    (Es, its, sts), t_s2, _, _ = timed(streams_step, max(1, args.steps // 2))
    (Eg, itg, stg), t_g2, launches, clocks = timed(grouped_step, args.steps)
    t_group, t_streams = min(t_g1, t_g2), min(t_s1, t_s2)
    t0 = time.perf_counter()
    serial = []
    for sv, (H, S, W0) in zip(solvers, data):
        sv.set_HS(H, S)
        serial.append(sv.solve(W0, tol=1e-10, raise_on_error=False))
    torch.cuda.synchronize()
    t_serial = time.perf_counter() - t0
    same = all(serial[i][0] == Eg[i] and serial[i][1] == itg[i] for i in range(count))
    same_streams = bool(np.array_equal(Es, Eg) and np.array_equal(its, itg))
    names = ["single CTA", "CTA pair"]
    line = {"metric": "OMM solves/s, batched uneven systems", "value": count / t_group, "unit": "solves/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_group,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16-split+f64",
            "data": "synthetic",
            "config": {"workload": (f"{count} dense systems, atoms round(exp(U(ln 32, ln 384))) (seed 4): "
                                    f"m {int(min(s.m for s in systems))}..{int(max(s.m for s in systems))}, n = m/4"),
                       "precision": "mixed", "tol": 1e-10, "orth_tol": 1e-6,
                       "execution": ("one group: per CG step of the first phase, each split product of all "
                                     "systems as one persistent grouped tensor-core launch, line minimum/updates/"
                                     "direction per system on its own stream in between, chunks of 8 steps as "
                                     "one CUDA graph; the refinement per system"),
                       "tile_mode_requested": args.tile_mode},
            "tuning": {"products": names[int(modes[0])], "contractions": names[int(modes[1])],
                       "gradient": names[int(modes[2])],
                       "timed_ms_single_pair": tune_ms.tolist()},
            "streams": {"value": count / t_streams, "unit": "solves/s", "ms": 1e3 * t_streams,
                        "results_equal_grouped": same_streams,
                        "ms_runs": [1e3 * t_s1, 1e3 * t_s2]},
            "grouped_ms_runs": [1e3 * t_g1, 1e3 * t_g2],
            "one_by_one": {"value": count / t_serial, "unit": "solves/s", "ms": 1e3 * t_serial},
            "results_equal_alone": bool(same), "all_ok": bool((stg == omm.OK).all()),
            "iters": {"min": int(itg.min()), "max": int(itg.max())},
            "gpu_launches": int(launches), "clocks": clocks}
    if not quiet:
        print(json.dumps(line), flush=True)
    for sv in solvers:
        sv.close()
    return line


# ---------------------------------------------------------------- C5: serving
def run_c5(args, quiet=False):
    """Serving loop: Poisson arrivals of SCF-like sequences (one dense system,
    then perturbed Hamiltonians H <- H + sym(N(0, 1e-3 eV)) on its nonzeros,
    each solve warm-started from the resident W), dense m = 8 x round(exp(U(ln 64,
    ln 1024))) atoms (512 .. 8192), n = m/4.  The same sequence set is served at
    every arrival rate; each rate's run is timed from the first arrival to the
    last result, and every solve's time-to-converge runs from its submission
    (the sequence's arrival, or the previous solve's result) to its result."""
    import torch
    from paper_2209_05934_gb300 import omm, serving

    omm.lib()
    rng = np.random.Generator(np.random.PCG64(5))
    natoms = np.round(np.exp(rng.uniform(np.log(64), np.log(1024), args.sequences))).astype(int)
    t_gen = time.perf_counter()
    seqs = [synth.make_batch_system(int(N), seed=5000 + i) for i, N in enumerate(natoms)]
    dev = lambda a: torch.from_numpy(np.asfortranarray(a)).to("cuda")
    base = []
    for sq in seqs:
        H = sq.dense_H()
        base.append((dev(H), dev(sq.dense_S()), dev(sq.W0_dense()), torch.from_numpy(H != 0).to("cuda")))
    t_gen = time.perf_counter() - t_gen

    def make_inputs_factory(i):
        H0, S, _, mask = base[i]

        def make(k):
            if k == 0:
                return H0, S
            g = torch.Generator(device="cuda")
            g.manual_seed(10_000 * i + k)
            noise = torch.randn(H0.shape, generator=g, device="cuda", dtype=torch.float64) * 1e-3
            noise = 0.5 * (noise + noise.T) * mask
            Hk = (H0 + noise).T.contiguous().T
            # the handles run on their own non-blocking streams: H_k must be complete first
            torch.cuda.current_stream().synchronize()
            return Hk, S
        return make

    ms = [int(sq.m) for sq in seqs]
    out = {"metric": "OMM serving: solves/s and p50/p99 time-to-converge", "unit": "solves/s", "n_gpus": 1,
           "data": "synthetic", "higher_is_better": True, "dtype": "bf16-split+f64",
           "config": {"workload": (f"{args.sequences} sequences served at each rate, each 1 + {args.scf_steps - 1} "
                                   "SCF-like perturbations H <- H + sym(N(0, 1e-3 eV)) on the nonzeros, "
                                   "warm-started; dense m = 8 round(exp(U(ln 64, ln 1024))), n = m/4"),
                      "m_min": min(ms), "m_max": max(ms), "m_median": int(np.median(ms)),
                      "precision": "mixed", "tol": 1e-10, "orth_tol": 1e-6,
                      "hbm_budget_gb": args.hbm_budget_gb, "input_generation_s": t_gen}, "rates": []}
    # warm-up: modules loaded, one small and one large solve
    for i in (int(np.argmin(ms)), int(np.argmax(ms))):
        w = omm.Solver(seqs[i].m, seqs[i].n, 8, precision=omm.PREC_MIXED, orth_tol=1e-6)
        w.set_HS(base[i][0], base[i][1])
        w.solve(base[i][2], tol=1e-10, raise_on_error=False)
        w.close()
    torch.cuda.synchronize()
    launches0 = omm.kernel_launches()
    for ri, rate in enumerate(args.rates):
        arr_rng = np.random.Generator(np.random.PCG64(500 + ri))
        arrivals = np.cumsum(arr_rng.exponential(1.0 / rate, size=len(seqs)))
        arrivals -= arrivals[0]
        reqs = [serving.Request(rid=i, arrival=float(arrivals[i]), m=seqs[i].m, n=seqs[i].n, steps=args.scf_steps,
                                make_inputs=make_inputs_factory(i), W0=base[i][2], graphs=args.graphs)
                for i in range(len(seqs))]
        server = serving.Server(hbm_budget_bytes=int(args.hbm_budget_gb * (1 << 30)))
        with ClockSampler(0) as clk:
            t0 = time.perf_counter()
            recs = server.run(reqs)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        st = serving.latency_stats(recs)
        cold = serving.latency_stats([r for r in recs if r.step == 0])
        warm = serving.latency_stats([r for r in recs if r.step > 0])
        big = serving.latency_stats([r for r in recs if r.m >= 4096])
        out["rates"].append({"rate_seq_per_s": rate, "solves": st["solves"], "solves_per_s": st["solves"] / wall,
                             "wall_s": wall, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                             "cold": {"p50_ms": cold["p50_ms"], "p99_ms": cold["p99_ms"]},
                             "warm": {"p50_ms": warm["p50_ms"], "p99_ms": warm["p99_ms"]},
                             "m_ge_4096": {"p50_ms": big["p50_ms"], "p99_ms": big["p99_ms"], "solves": big["solves"]},
                             "max_inflight": server.max_inflight,
                             "all_ok": all(r.status == omm.OK for r in recs),
                             "statuses": sorted({int(r.status) for r in recs}),
                             "iters_cold_mean": float(np.mean([r.iters for r in recs if r.step == 0])),
                             "iters_warm_mean": float(np.mean([r.iters for r in recs if r.step > 0])),
                             "clocks": clk.summary()})
    out["value"] = max(r["solves_per_s"] for r in out["rates"])
    out["gpu_launches"] = int(omm.kernel_launches() - launches0)

    # the same request set served by the mixed form and by the plain FP64 GPU form
    if args.fp64_sequences > 0:
        pick = [i for i in np.argsort(ms) if ms[i] <= 2048][-args.fp64_sequences:]
        rate = 50.0
        arrivals = np.cumsum(np.random.Generator(np.random.PCG64(55)).exponential(1.0 / rate, size=len(pick)))
        arrivals -= arrivals[0]
        cmp = {"sequences": len(pick), "rate_seq_per_s": rate, "m": [ms[i] for i in pick]}
        for name, p in (("mixed", omm.PREC_MIXED), ("fp64", omm.PREC_FP64)):
            reqs = [serving.Request(rid=int(i), arrival=float(arrivals[j]), m=seqs[i].m, n=seqs[i].n,
                                    steps=args.scf_steps, make_inputs=make_inputs_factory(int(i)), W0=base[i][2],
                                    precision=p) for j, i in enumerate(pick)]
            server = serving.Server(hbm_budget_bytes=int(args.hbm_budget_gb * (1 << 30)))
            t0 = time.perf_counter()
            recs = server.run(reqs)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            st = serving.latency_stats(recs)
            cmp[name] = {"solves_per_s": st["solves"] / wall, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                         "all_ok": all(r.status == omm.OK for r in recs),
                         "E_last": {r.rid: float(r.E) for r in recs if r.step == args.scf_steps - 1}}
        cmp["max_rel_E_diff"] = max(abs(cmp["mixed"]["E_last"][i] - cmp["fp64"]["E_last"][i])
                                    / abs(cmp["fp64"]["E_last"][i]) for i in cmp["fp64"]["E_last"])
        for name in ("mixed", "fp64"):
            del cmp[name]["E_last"]
        out["mixed_vs_fp64"] = cmp
    if args.c5_sparse_steps > 0:
        out["sparse_sequence"] = run_c5_sparse(args)
    if not quiet:
        print(json.dumps(out), flush=True)
    return out


def run_c5_sparse(args):
    """One SCF-like sequence of the linear-scaling workload (C3 system, m = 32768,
    mixed form): a cold solve from W0, then c5_sparse_steps - 1 solves each after an
    onsite update of H (every diagonal block B <- B + sym(N(0, 1e-3 eV)), drawn per
    step), warm-started from the resident W.  Solves run back to back (one
    sequence, no queueing); each time-to-converge is the device time of
    omm_set_HS + omm_solve."""
    import torch
    from paper_2209_05934_gb300 import omm

    sysm = synth.make_system(*C3["dims"], seed=C3["seed"])
    rp, col, Hv, Sv = sysm.bsr()
    wrp, wcol = sysm.w_pattern(C3["radius"])
    stream = torch.cuda.Stream()
    s = omm.SparseSolver(sysm.m, sysm.n, 8, 2, rp, col, wrp, wcol, max_iter=40000, stream=stream.cuda_stream,
                         precision=omm.PREC_MIXED)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
    Sd, W0d = dev(Sv), dev(sysm.W0_bsr_values(C3["radius"]))
    diag_blocks = np.array([k for i in range(len(rp) - 1) for k in range(rp[i], rp[i + 1]) if col[k] == i])
    solves = []
    for k in range(args.c5_sparse_steps):
        Hk = Hv.copy()
        if k > 0:
            g = np.random.Generator(np.random.PCG64(7000 + k))
            nz = g.normal(0.0, 1e-3, size=(len(diag_blocks), 8, 8))
            Hk[diag_blocks] += 0.5 * (nz + nz.transpose(0, 2, 1))
        Hd = dev(Hk)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.set_HS(Hd, Sd)
        E, iters, st = s.solve(W0d if k == 0 else None, tol=1e-10, raise_on_error=False)
        e1.record(stream)
        torch.cuda.synchronize()
        d = s.diag()
        solves.append({"step": k, "ms": e0.elapsed_time(e1), "iters": int(iters), "iters_mixed": int(d.iters_mixed),
                       "iters_refine": int(d.iters_refine), "status": int(st), "E": E})
    s.close()
    warm = [r["ms"] for r in solves[1:]]
    return {"workload": (f"C3 system (4096 atoms, m={sysm.m}, n={sysm.n}, R_C={C3['radius']} A), mixed form, "
                         "1 cold + onsite-perturbed warm-started solves, tol 1e-10"),
            "cold_ms": solves[0]["ms"], "warm_ms_median": float(np.median(warm)) if warm else None,
            "all_ok": all(r["status"] == omm.OK for r in solves), "solves": solves}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="omm", choices=["omm", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--profile", action="store_true",
                    help="run one solve only (for ncu captures); prints stage times, no benchmark line")
    ap.add_argument("--max-iter", type=int, default=0, help="with --profile: cap on CG steps")
    ap.add_argument("--fp64-peak", action="store_true",
                    help="print the measured FP64 GEMM throughput (the FP64 roofline denominator) and exit")
    ap.add_argument("--no-fp64-beside", action="store_true",
                    help="c2: skip the plain FP64 GPU solve reported beside the mixed form")
    ap.add_argument("--fp64-sequences", type=int, default=3,
                    help="c5: sequences of the mixed-vs-FP64 serving comparison (0 skips it)")
    ap.add_argument("--split-digits", type=int, default=2, choices=[2, 3],
                    help="mixed form: BF16 digits per operand in the first phase (3 pairs or 6)")
    ap.add_argument("--gemm-pair", type=int, default=1, choices=[0, 1],
                    help="mixed form: split products on CTA pairs (cta_group::2) or one CTA per tile")
    ap.add_argument("--dir-digits", type=int, default=1, choices=[0, 1],
                    help="mixed form: BF16 digits kept of each search direction (1: the H'D, SD products "
                         "take two digit pairs; 0: two digits, three pairs)")
    ap.add_argument("--gemm-persistent", type=int, default=0, choices=[0, 1],
                    help="mixed form: split products as persistent tile-list launches")
    ap.add_argument("--graphs", type=int, default=1, choices=[0, 1],
                    help="c4/c5: replay chunks of CG steps as captured CUDA graphs")
    ap.add_argument("--extras", type=int, default=1, choices=[0, 1],
                    help="c2: also run short C3 (20 CG steps), C4 and C5 (12 sequences, one rate) "
                         "and add them to the line")
    ap.add_argument("--no-kinetic", action="store_true",
                    help="skip the kinetic-energy preconditioning comparison on H + T")
    ap.add_argument("--cholesky", action="store_true",
                    help="c2: Cholesky-reduced variant (S = L L^T factored inside each step's setup)")
    ap.add_argument("--config", default="c2", choices=["c2", "c3", "c4", "c5", "md"],
                    help="c2 dense workload (default); c3 linear-scaling to convergence; "
                         "c4 batched uneven solves; c5 serving loop")
    ap.add_argument("--batch", type=int, default=64, help="c4: number of systems")
    ap.add_argument("--tile-mode", type=int, default=-1, choices=[-1, 0, 1],
                    help="c4: grouped launch tile mode (-1 autotune, 0 single CTA, 1 CTA pair)")
    ap.add_argument("--c3-precision", default="fp64", choices=["fp64", "mixed"],
                    help="c3: FP64 throughout, or FP32 increments on FP64 state with an FP64 refinement")
    ap.add_argument("--screen-eps", type=float, default=0.0,
                    help="c3: norm-based screening threshold of the sparse block products (0: off)")
    ap.add_argument("--md-steps", type=int, default=5, help="md: snapshots per chain")
    ap.add_argument("--md-step", type=float, default=0.03, help="md: Angstrom per snapshot per unit velocity")
    ap.add_argument("--md-max-iter", type=int, default=20000, help="md: CG step cap of the sparse solves")
    ap.add_argument("--sequences", type=int, default=91,
                    help="c5: sequences served at each arrival rate (91 x 11 solves = 1001 per rate)")
    ap.add_argument("--scf-steps", type=int, default=11, help="c5: solves per sequence (1 + perturbations)")
    ap.add_argument("--c5-sparse-steps", type=int, default=0,
                    help="c5: also serve one linear-scaling sequence (m = 32768) of this many solves")
    ap.add_argument("--rates", type=float, nargs="+", default=[10.0, 20.0, 50.0, 100.0, 200.0, 500.0],
                    help="c5: sequence arrivals per second")
    ap.add_argument("--hbm-budget-gb", type=float, default=200.0, help="c5: admission budget")
    args = ap.parse_args()
    if args.fp64_peak:
        import torch  # noqa: F401
        print(json.dumps({"fp64_peak_tflops": {str(n): fp64_gemm_peak(n) for n in (2048, 4096, 8192)},
                          "how": "cuBLAS DGEMM via torch.matmul in float64, n^3, best of 5"}), flush=True)
        return
    if args.profile:
        run_profile(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.config == "c3":
        run_c3(args)
        return
    if args.config == "c4":
        run_c4(args)
        return
    if args.config == "c5":
        run_c5(args)
        return
    if args.config == "md":
        run_md(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_omm(args)


if __name__ == "__main__":
    main()
