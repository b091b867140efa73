"""Served solves with continuous batching.

Requests (2D Euler Q2 four-quadrant Riemann solves of different mesh sizes and end times) arrive
as a Poisson stream. The engine keeps every admitted solve's state resident on the GPU and advances
them with dg_batch_run in chunks of a few steps; at every chunk boundary it retires the solves that
reached their end time (each stops exactly at its own T) and admits waiting requests while the
device-memory budget allows. Latency = completion time - arrival time.

In the FP32 form a round is one dg_batch_run over the chosen solves; the plain FP64 path (no
batched kernel) advances each chosen solve on its own with dg_advance_to, at most a chunk of steps.

Which resident solves a round advances is the scheduling policy: "all" advances every one; "srpt"
(shortest remaining work first) advances the solves with the least estimated remaining work,
(T - t) * side^3 (steps grow with side / CFL, cells with side^2), adding them until they cover
`fill_cells` cells, enough to occupy the GPU, so short requests are not held behind long ones while
the device stays busy.
"""
from __future__ import annotations

import dataclasses
import math
import time

from . import _native as N
from . import inputs as I

SIDES = (128, 256, 512, 1024)


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float      # seconds after the start of the session
    side: int
    T: float
    seed: int


def poisson_requests(rate, n, seed, seeds, sides=SIDES, t_range=(0.05, 0.25)):
    """n requests with exponential inter-arrival times (mean 1/rate); side uniform in `sides`, end
    time uniform in t_range, Riemann data from the screened seed list `seeds`."""
    g = I.SplitMix64(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += -math.log(1.0 - g.uniform(0.0, 1.0)) / rate
        side = sides[min(int(g.uniform(0, len(sides))), len(sides) - 1)]
        T = g.uniform(*t_range)
        out.append(Request(i, t, side, T, seeds[i % len(seeds)]))
    return out


@dataclasses.dataclass
class Result:
    rid: int
    side: int
    T: float
    arrival: float
    admitted: float
    done: float
    steps: int
    dofs: int
    status: int
    state: object = None

    @property
    def latency(self):
        return self.done - self.arrival


class Engine:
    """Continuous-batching loop over resident solves.

    budget_bytes: device memory the admitted solves may hold together (dg_workspace_size each).
    chunk_steps: steps per dg_batch_run call (the admission / retirement granularity).
    positivity: the Zhang-Shu limiter after the filter (on by default: random four-quadrant data
        reach near-vacuum states that the unlimited scheme cannot hold).
    """

    def __init__(self, budget_bytes=120e9, chunk_steps=16, precision=N.PREC_FP32_MIXED, stream=None,
                 keep_states=False, max_active=512, positivity=1, policy="srpt", fill_cells=1 << 19):
        self.budget = budget_bytes
        self.chunk = chunk_steps
        self.precision = precision
        self.stream = stream
        self.keep = keep_states
        self.max_active = max_active
        self.positivity = positivity
        self.policy = policy
        self.fill_cells = fill_cells

    def _bytes(self, req):
        return N.Solver.workspace_size(dim=2, nx=req.side, ny=req.side, bc=(N.BC_OUTFLOW,) * 4, k=2,
                                       eq=N.EQ_EULER, precision=self.precision)

    def _start(self, req):
        s = N.Solver(dim=2, nx=req.side, ny=req.side, x0=0.0, x1=1.0, y0=0.0, y1=1.0,
                     bc=(N.BC_OUTFLOW,) * 4, k=2, eq=N.EQ_EULER, precision=self.precision,
                     stream=self.stream, positivity=self.positivity)
        s.set_initial(N.IC_QUADRANT2D, I.quadrant_params(req.seed))
        s.set_target(req.T)
        s.last_t = 0.0
        return s

    def run(self, requests, clock=time.perf_counter):
        pending = sorted(requests, key=lambda r: r.arrival)
        active = []          # (request, solver, admitted time, bytes)
        used = 0.0
        results = []
        peak_active = 0
        peak_bytes = 0.0
        t0 = clock()
        now = lambda: clock() - t0  # noqa: E731
        while pending or active:
            # admission: arrived requests, in arrival order, while memory and slots allow
            while pending and pending[0].arrival <= now() and len(active) < self.max_active:
                need = self._bytes(pending[0])
                if used + need > self.budget and active:
                    break
                req = pending.pop(0)
                active.append((req, self._start(req), now(), need))
                used += need
            peak_active = max(peak_active, len(active))
            peak_bytes = max(peak_bytes, used)
            if not active:
                time.sleep(max(0.0, min(0.01, pending[0].arrival - now())))
                continue
            if self.policy == "srpt":
                rem = [(req.T - s.last_t) * req.side ** 3 for req, s, adm, need in active]
                pick = pick_round(rem, [req.side * req.side for req, s, adm, need in active], self.fill_cells)
            else:
                pick = list(range(len(active)))
            if self.precision == N.PREC_FP64:
                # the plain FP64 path: batched stepping is FP32-form only, so each solve advances
                # on its own, up to chunk steps toward its end time (the solves stay resident)
                for i in pick:
                    active[i][1].advance_toward(active[i][0].T, self.chunk)
            else:
                N.batch_run([active[i][1] for i in pick], self.chunk)
            still = []
            for idx, (req, s, adm, need) in enumerate(active):
                if idx not in pick:
                    still.append((req, s, adm, need))
                    continue
                status, t, steps = s.sync()
                s.last_t = t
                if status != 0 or t >= req.T:
                    state = None
                    if self.keep and status == 0:
                        state = s.read_state()[0]
                    else:
                        s.mass()          # the solve's result summary reaches the host
                    results.append(Result(req.rid, req.side, req.T, req.arrival, adm, now(), steps,
                                          s.size, status, state))
                    s.close()
                    used -= need
                else:
                    still.append((req, s, adm, need))
            active = still
        return results, {"peak_active": peak_active, "peak_bytes": peak_bytes}


def pick_round(remaining, cells, fill_cells):
    """Indices of the solves one round advances under shortest-remaining-work-first: ascending
    estimated remaining work, until their cells reach fill_cells (all of them if they never do)."""
    order = sorted(range(len(remaining)), key=lambda i: (remaining[i], i))
    chosen, total = [], 0
    for i in order:
        chosen.append(i)
        total += cells[i]
        if total >= fill_cells:
            break
    return sorted(chosen)


def summarize(results, wall):
    lat = sorted(r.latency for r in results if r.status == 0)
    if not lat:
        return {"completed": 0}

    def pct(p):
        i = min(len(lat) - 1, max(0, int(math.ceil(p / 100.0 * len(lat))) - 1))
        return lat[i]

    dof_stage = sum(3.0 * r.dofs * r.steps for r in results if r.status == 0)
    return {"completed": len(lat), "failed": sum(r.status != 0 for r in results),
            "p50_s": pct(50), "p99_s": pct(99), "mean_s": sum(lat) / len(lat),
            "throughput_solves_per_s": len(lat) / wall, "dof_stage_per_s": dof_stage / wall, "wall_s": wall}
