"""Continuous-batching request loop for OMM solves (host-side scheduling only).

Requests arrive as SCF-like sequences: one system (dense H, S) followed by
perturbed Hamiltonians, each solve warm-started from the previous W that is
still resident in the sequence's handle.  The scheduler

* admits a sequence when its device footprint fits the HBM budget (else it
  waits in arrival order),
* keeps every admitted solve in flight on its own CUDA stream through the
  library's non-blocking driver (omm_solve_begin / omm_solve_progress /
  omm_solve_end), so solves that arrive while others run overlap with them,
* records for every solve its submit time (arrival of the sequence, or the end
  of the previous solve of the same sequence) and its completion time.

All arithmetic runs in the library's kernels; this module only decides what
runs when.  Results do not depend on the mix: each handle's kernels use fixed
reduction orders, independent of other streams.
"""
from __future__ import annotations

import dataclasses
import heapq
import time
from typing import Callable, List, Optional

import numpy as np

from . import omm


@dataclasses.dataclass
class Request:
    """One sequence: `steps` solves on an m x n problem.

    make_inputs(k) returns (H, S) device arrays (column-major) for solve k; W0 is
    the first solve's initial guess; later solves warm-start.
    """
    rid: int
    arrival: float                       # seconds after the start of the run
    m: int
    n: int
    steps: int
    make_inputs: Callable[[int], tuple]
    W0: object
    tol: float = 1e-10
    precision: int = omm.PREC_MIXED
    orth_tol: float = 1e-6
    fixed_S: bool = True                 # later solves change H only (omm_set_H keeps S)
    cholesky: int = 0
    graphs: int = 1                      # replay chunks of CG steps as CUDA graphs


@dataclasses.dataclass
class SolveRecord:
    rid: int
    step: int
    m: int
    submit: float
    start: float
    finish: float
    E: float
    iters: int
    status: int

    @property
    def latency(self) -> float:
        return self.finish - self.submit


def footprint_bytes(m: int, n: int, precision: int, exact_digits: int = 7) -> int:
    """Device memory of one dense handle (what omm_create allocates)."""
    f64 = 8 * (2 * m * m + 6 * m * n + 2 * n * n + 4 * n * n + 2 * m * n)
    if precision == omm.PREC_MIXED:
        ldm = (m + 7) // 8 * 8
        ld2n = (2 * n + 7) // 8 * 8
        f64 += 2 * 3 * (2 * m * ldm + 4 * n * ldm + m * ld2n + n * ld2n)          # split digits
        f64 += 4 * (2 * m * n + 4 * n * n + 4 * m * n)                             # FP32 increments
        f64 += 2 * exact_digits * (2 * m * ldm + 3 * n * ldm + m * ld2n + n * ld2n)  # exact digits
    return int(f64)


class _Active:
    def __init__(self, req: Request, solver: omm.Solver, t_submit: float):
        self.req = req
        self.solver = solver
        self.step = 0
        self.t_submit = t_submit
        self.t_start = t_submit


class Server:
    def __init__(self, hbm_budget_bytes: int, stream_factory=None):
        self.budget = hbm_budget_bytes
        self.used = 0
        self.records: List[SolveRecord] = []
        self.queue: List[tuple] = []          # (arrival, rid, Request) waiting for memory
        self.active: List[_Active] = []
        self.max_inflight = 0

    def _admit(self, req: Request, now: float) -> bool:
        need = footprint_bytes(req.m, req.n, req.precision)
        if self.active and self.used + need > self.budget:
            return False
        s = omm.Solver(req.m, req.n, 8, precision=req.precision, orth_tol=req.orth_tol, cholesky=req.cholesky,
                       graphs=req.graphs)
        self.used += need
        H, S = req.make_inputs(0)
        s.set_HS(H, S)
        a = _Active(req, s, t_submit=req.arrival)
        a.t_start = now
        s.begin(req.W0, tol=req.tol)
        self.active.append(a)
        return True

    def run(self, requests: List[Request], clock: Optional[Callable[[], float]] = None,
            poll_sleep: float = 0.0) -> List[SolveRecord]:
        """Serve all requests; arrival times are honoured against the wall clock."""
        clock = clock or time.perf_counter
        t0 = clock()
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        pi = 0
        while pi < len(pending) or self.queue or self.active:
            now = clock() - t0
            while pi < len(pending) and pending[pi].arrival <= now:
                heapq.heappush(self.queue, (pending[pi].arrival, pending[pi].rid, pending[pi]))
                pi += 1
            while self.queue:
                arr, rid, req = self.queue[0]
                if not self._admit(req, clock() - t0):
                    break
                heapq.heappop(self.queue)
            self.max_inflight = max(self.max_inflight, len(self.active))
            progressed = False
            for a in list(self.active):
                if not a.solver.progress(blocking=False):
                    continue
                progressed = True
                t_fin = clock() - t0
                E, iters, st = a.solver.end(raise_on_error=False)
                self.records.append(SolveRecord(a.req.rid, a.step, a.req.m, a.t_submit, a.t_start, t_fin, E,
                                                iters, st))
                a.step += 1
                if a.step < a.req.steps:
                    H, S = a.req.make_inputs(a.step)
                    if a.req.fixed_S:
                        a.solver.set_H(H)
                    else:
                        a.solver.set_HS(H, S)
                    a.t_submit = a.t_start = clock() - t0
                    a.solver.begin(None, tol=a.req.tol)        # warm start from the resident W
                else:
                    a.solver.close()
                    self.used -= footprint_bytes(a.req.m, a.req.n, a.req.precision)
                    self.active.remove(a)
            if not progressed and poll_sleep > 0:
                time.sleep(poll_sleep)
            if not progressed and not self.active and pi < len(pending):
                # idle until the next arrival
                wait = pending[pi].arrival - (clock() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.01))
        return self.records


def latency_stats(records: List[SolveRecord]) -> dict:
    lat = np.array([r.latency for r in records]) * 1e3
    if lat.size == 0:
        return {"p50_ms": None, "p99_ms": None, "solves": 0}
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "solves": int(lat.size)}
