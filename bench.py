"""Benchmark: DOF-stage updates/s of the fused RKDG jump-filter stage kernel.

Workload: 2D Euler, gamma = 1.4, 2048 x 2048 cells on [0,1]^2, Q2 tensor-product Legendre DG (36
DOFs per cell, 151 M DOFs), LLF flux, SSP-RK3, jump filter after every stage, outflow boundaries,
seeded four-quadrant Riemann data projected on the GPU. One benchmark step = one SSP-RK3 step over
the whole mesh = 3 stage launches = 3 x 151 M DOF-stage updates.

Headline `value`: the FP32 form (FP32 stage arithmetic, cell averages in double-float), inputs
resident in HBM. Beside it: the plain FP64 path, the end-to-end figure through the C ABI with host
buffers, the roofline of the stage kernel, GPU clocks during the timed region, and the FP64 CPU
oracle timed on this host's cores. `--impl reference` times that oracle alone (the reference arm).

Contract: python bench.py --gpus N --steps K --warmup W; for N > 1 launched by torch.distributed.run,
one rank per GPU (replicas: every rank solves its own copy, no data-path collective).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "euler2d_q2_2048x2048_quadrant_riemann"
METRIC = "2D Euler P2 DOF-stage updates/s (FP32 vs FP64) + served-solve p50/p99 latency"
UNIT = "DOF-stage/s"
QUADRANT_SEED_FILE = os.path.join(ROOT, "tests", "golden", "quadrant_seeds.txt")
FALLBACK_HBM_GBS = 6800.0


def first_accepted_seed():
    try:
        with open(QUADRANT_SEED_FILE) as f:
            for line in f:
                if line.startswith("#") or not line.strip():
                    continue
                s, ok, _ = line.split()
                if int(ok):
                    return int(s)
    except OSError:
        pass
    return 1


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


# Sources whose compiled form is the timed stage kernel: the DRAM traffic recorded in profiles/ is
# reported only while they are unchanged since the capture.
KERNEL_SOURCES = ["paper_2407_19169_gb300/csrc/stage2d.cuh", "paper_2407_19169_gb300/csrc/dg_device.cuh",
                  "paper_2407_19169_gb300/csrc/stage_common.cuh", "paper_2407_19169_gb300/csrc/stage2d_units.cu",
                  "paper_2407_19169_gb300/csrc/dg_tables.cuh"]
TRAFFIC_PROFILE = "profiles/stage2d_f32_q2_euler_2048_traffic.md"


def kernel_sources_hash():
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def recorded_traffic():
    """dram read + write bytes per stage launch from the committed ncu capture of the 2048^2
    benchmark, or None when the kernel sources changed since (or the record is missing)."""
    try:
        rec = {}
        with open(os.path.join(ROOT, TRAFFIC_PROFILE)) as f:
            for line in f:
                if ":" in line and not line.startswith(("|", "#", " ")):
                    k, v = line.split(":", 1)
                    rec[k.strip()] = v.strip()
        if rec.get("kernel_sources_sha256") != kernel_sources_hash():
            return None
        return float(rec["traffic_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.samples = []
        if self.proc is None:
            return
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def summary(self):
        if not getattr(self, "samples", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(p[1]) for p in self.samples if p[1].replace(".", "").isdigit()]
        mx = [float(p[2]) for p in self.samples if p[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in self.samples for i in range(4) if p[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(torch, dist, ms_local, work_local, world, device):
    """Whole-job throughput over replicas: the work of all ranks divided by the slowest rank's time
    (max over ranks of the timed region). Returns (value, ms_max)."""
    if world == 1:
        return work_local / (ms_local * 1e-3), ms_local
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([work_local], dtype=torch.float64, device=device)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    ms_max = float(t.item())
    return float(w.item()) / (ms_max * 1e-3), ms_max


def accepted(name):
    out = []
    try:
        with open(os.path.join(ROOT, "tests", "golden", name)) as f:
            for line in f:
                if line.startswith("#") or not line.strip():
                    continue
                sd, ok, _ = line.split()
                if int(ok):
                    out.append(int(sd))
    except OSError:
        pass
    return out or [1]


def make_instance(N, I, spec, stream, tiles):
    """One batched instance (FP32 form) from inputs.batched_specs."""
    kind, n, k = spec["kind"], spec["n"], spec["k"]
    H, W = tiles.get(k, (0, 0)) if spec["dim"] == 2 else (0, 0)
    if spec["dim"] == 1:
        bc = (N.BC_OUTFLOW,) * 4 if kind == "riemann1d" else (N.BC_PERIODIC,) * 4
        s = N.Solver(dim=1, nx=n, k=k, eq=N.EQ_EULER, bc=bc, precision=N.PREC_FP32_MIXED, stream=stream,
                     positivity=1)
        if kind == "riemann1d":
            s.set_initial(N.IC_RIEMANN1D, I.riemann1d_params(spec["seed"]))
        else:
            s.set_initial(N.IC_ENTROPY1D, [1.0, 0.2, 2 * math.pi, 1.0, 1.0])
    elif kind == "quadrant2d":
        s = N.Solver(dim=2, nx=n, ny=n, k=k, eq=N.EQ_EULER, bc=(N.BC_OUTFLOW,) * 4,
                     precision=N.PREC_FP32_MIXED, stream=stream, tile_rows=H, tile_warps=W, positivity=1)
        s.set_initial(N.IC_QUADRANT2D, I.quadrant_params(spec["seed"]))
    else:
        s = N.Solver(dim=2, nx=n, ny=n, x0=0.0, x1=10.0, y0=-5.0, y1=5.0, k=k, eq=N.EQ_EULER,
                     bc=(N.BC_PERIODIC,) * 4, precision=N.PREC_FP32_MIXED, stream=stream, tile_rows=H,
                     tile_warps=W, positivity=1)
        s.set_initial(N.IC_VORTEX2D, [5.0, 0.0, 5.0, 0.0])
    return s


def run_batched(torch, N, stream, steps, n_inst, tile_rows=0):
    """S2: n_inst uneven instances (inputs.batched_specs), each advanced `steps` steps by dg_batch_run
    (one graph-captured work-list launch per class and stage), then the same instances afresh by
    dg_batch_run_persistent (one persistent launch per class for all steps); autotuned 2D tiles per
    degree; the positivity-preserving limiter after the filter, as the paper does for hard Riemann
    data."""
    from paper_2407_19169_gb300 import inputs as I
    from paper_2407_19169_gb300 import tuning
    specs = I.batched_specs(n=n_inst, riemann_seeds=accepted("riemann1d_seeds.txt"),
                            quadrant_seeds=accepted("quadrant_seeds.txt"))
    # tiles per degree, tuned at the median side of that degree's 2D instances
    med = {}
    for k in (1, 2, 3):
        sides = sorted(sp["n"] for sp in specs if sp["dim"] == 2 and sp["k"] == k)
        med[k] = sides[len(sides) // 2] if sides else 256
    tiles = ({k: (tile_rows, 4) for k in (1, 2, 3)} if tile_rows else
             {k: tuning.tune_2d(med[k], med[k], k=k) for k in (1, 2, 3)})
    def one(persistent):
        t0 = time.perf_counter()
        inst = [make_instance(N, I, sp, stream.cuda_stream, tiles) for sp in specs]
        setup_s = time.perf_counter() - t0
        torch.cuda.synchronize()
        dofs = [x.size for x in inst]
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = inst[0].kernel_launches()
        e0.record(stream)
        st = N.batch_run(inst, steps, persistent=persistent)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        launches = inst[0].kernel_launches() - l0
        done = [x.sync() for x in inst]
        ok = [d[0] == 0 and d[2] == steps for d in done]
        work = sum(3.0 * d * steps for d, o in zip(dofs, ok) if o)
        for x in inst:
            x.close()
        rec = {"value": work / (ms * 1e-3), "unit": UNIT, "instances": n_inst, "steps_each": steps,
               "total_dofs": int(sum(dofs)), "ms": ms, "failed_instances": int(len(ok) - sum(ok)),
               "status": st, "setup_s": setup_s, "gpu_launches": launches, "dtype": "f32+df64",
               "positivity_limiter": True}
        return rec, [d[1] for d in done]

    graph, t_graph = one(False)
    graph["tiles_by_degree"] = {str(k): list(v) for k, v in tiles.items()}
    graph["tuned_at_side"] = {str(k): v for k, v in med.items()}
    # the same instances advanced by dg_batch_run_persistent: one cooperative launch per class runs all
    # steps, per-instance stage barriers on device counters
    pers, t_pers = one(True)
    pers["same_end_times_as_graph"] = bool(t_pers == t_graph)
    graph["persistent"] = pers
    return graph


def run_small_configs(torch, N, stream, barrier):
    """The two small workloads of the method: Burgers 0.5 + sin(pi x) on [0, 2], 200 cells, P2, FP64;
    1D Euler seeded Riemann data, 65,536 cells, P3, FP64 and FP32 form. At these sizes a stage is a
    few microseconds of work, so the figures show the graph-replayed launch rate."""
    from paper_2407_19169_gb300 import inputs as I
    out = {}
    cases = [("burgers1d_p2_200", dict(dim=1, nx=200, x0=0.0, x1=2.0, k=2, eq=N.EQ_BURGERS,
                                       bc=(N.BC_PERIODIC,) * 4), (N.IC_SINE, [0.5, 1.0, math.pi, 0.0]),
              (N.PREC_FP64,), 2000),
             ("euler1d_p3_65536", dict(dim=1, nx=65536, x0=0.0, x1=1.0, k=3, eq=N.EQ_EULER,
                                       bc=(N.BC_OUTFLOW,) * 4),
              (N.IC_RIEMANN1D, I.riemann1d_params(accepted("riemann1d_seeds.txt")[0])),
              (N.PREC_FP64, N.PREC_FP32_MIXED), 2000)]
    for name, kw, (ic, prm), precs, steps in cases:
        for prec in precs:
            s = N.Solver(precision=prec, stream=stream.cuda_stream, **kw)
            s.set_initial(ic, prm)
            s.advance_steps(10)
            torch.cuda.synchronize()
            ms, _ = time_steps(torch, s, steps, stream, barrier)
            nv, nm, nc = s.shape
            out["%s_%s" % (name, "f64" if prec == N.PREC_FP64 else "f32")] = {
                "value": 3.0 * nv * nm * nc * steps / (ms * 1e-3), "unit": UNIT, "steps": steps,
                "us_per_step": 1e3 * ms / steps}
            s.close()
    return out


def run_served(N, stream, rate, n_req, budget, policy="srpt", precision=None, sides=None):
    """S3: a Poisson stream of 2D Euler Q2 quadrant solves served with continuous batching (FP32
    form; precision=PREC_FP64 serves the plain FP64 path, each solve stepped on its own)."""
    from paper_2407_19169_gb300 import serve as S
    precision = N.PREC_FP32_MIXED if precision is None else precision
    reqs = S.poisson_requests(rate=rate, n=n_req, seed=5, seeds=accepted("quadrant_seeds.txt"),
                              sides=sides or S.SIDES)
    eng = S.Engine(budget_bytes=budget, chunk_steps=16, stream=stream.cuda_stream, positivity=1, policy=policy,
                   precision=precision)
    t0 = time.perf_counter()
    results, stats = eng.run(reqs)
    wall = time.perf_counter() - t0
    out = S.summarize(results, wall)
    out.update({"rate_per_s": rate, "requests": n_req, "budget_gb": budget / 1e9, **stats,
                "sides": sorted({r.side for r in reqs}),
                "precision": "FP64" if precision == N.PREC_FP64 else "FP32 form", "positivity_limiter": True,
                "policy": policy})
    return out


def _legendre_vander(k, pts):
    """[l, point] values of P_l, l = 0..k (Bonnet's recurrence)."""
    import numpy as np
    V = np.zeros((k + 1, len(pts)))
    V[0] = 1.0
    if k >= 1:
        V[1] = pts
    for l in range(1, k):
        V[l + 1] = ((2 * l + 1) * pts * V[l] - l * V[l - 1]) / (l + 1)
    return V


def _l1_vs_finer(uc, nc, uf, nf, k, var, area):
    """L1 over the domain of (coarse Q^k solution - finer one) for one variable, integrated on the
    finer mesh's cells at (k+3)^2 Gauss points (the coarse polynomial evaluated there)."""
    import numpy as np
    r = nf // nc
    xg, wg = np.polynomial.legendre.leggauss(k + 3)
    W = np.outer(wg, wg).ravel() * (area / (nf * nf) / 4.0)

    def vander(pts_x, pts_y):
        Vx, Vy = _legendre_vander(k, pts_x), _legendre_vander(k, pts_y)
        return np.stack([np.outer(Vy[q], Vx[p]).ravel() for q in range(k + 1) for p in range(k + 1)])

    Vf = vander(xg, xg)
    UF = uf[var].reshape(-1, nf, nf)
    UC = uc[var].reshape(-1, nc, nc)
    tot = 0.0
    for b in range(r):
        for a in range(r):
            Vc = vander((2 * a + 1 + xg) / r - 1.0, (2 * b + 1 + xg) / r - 1.0)
            tot += (W[:, None, None] * np.abs(np.einsum("mg,mji->gji", Vc, UC)
                                              - np.einsum("mg,mji->gji", Vf, UF[:, b::r, a::r]))).sum()
    return tot


def run_accuracy(N, stream):
    """The error statement of the FP32 form (the kernels of every timed result here), measured
    against the FP64 path, which matches the FP64 oracle within relative L1 1e-11 in the parity tests:
    smooth - the isentropic vortex, Q2, 128^2, 100 steps: relative L1 (max over variables at 5x5
    Gauss points per cell) of FP32 against FP64; shock - the benchmark's problem type (Q2 four-quadrant
    Riemann data, outflow) at 256^2 to T = 0.05: the L1 error of each path against a 2x finer FP64 run,
    and their ratio (bar: within 2%)."""
    import numpy as np
    from paper_2407_19169_gb300 import inputs as I
    out = {}
    # smooth
    res = {}
    for prec in (N.PREC_FP64, N.PREC_FP32_MIXED):
        s = N.Solver(dim=2, nx=128, ny=128, x0=0.0, x1=10.0, y0=-5.0, y1=5.0, bc=(N.BC_PERIODIC,) * 4, k=2,
                     eq=N.EQ_EULER, precision=prec, stream=stream.cuda_stream)
        s.set_initial(N.IC_VORTEX2D, [5.0, 0.0, 5.0, 0.0])
        s.advance_steps(100)
        st = s.sync()[0]
        res[prec] = s.read_state()[0] if st == 0 else None
        s.close()
    xg, _ = np.polynomial.legendre.leggauss(5)
    V1 = _legendre_vander(2, xg)
    V = np.stack([np.outer(V1[q], V1[p]).ravel() for q in range(3) for p in range(3)])
    a, b = res[N.PREC_FP32_MIXED], res[N.PREC_FP64]
    worst = max(np.abs(V.T @ (a[v] - b[v])).sum() / np.abs(V.T @ b[v]).sum() for v in range(4))
    out["smooth"] = {"problem": "isentropic vortex, Q2, 128^2 on [0,10]x[-5,5], 100 steps",
                     "fp32_vs_fp64_rel_l1": float(worst), "bar": 1e-5}
    # shock
    seed = first_accepted_seed()
    T = 0.05
    sol = {}
    for name, prec, n in (("ref", N.PREC_FP64, 512), ("fp64", N.PREC_FP64, 256), ("fp32", N.PREC_FP32_MIXED, 256)):
        s = N.Solver(dim=2, nx=n, ny=n, bc=(N.BC_OUTFLOW,) * 4, k=2, eq=N.EQ_EULER, precision=prec,
                     stream=stream.cuda_stream)
        s.set_initial(N.IC_QUADRANT2D, I.quadrant_params(seed))
        s.advance_to(T)
        sol[name] = s.read_state()[0]
        s.close()
    e64 = [_l1_vs_finer(sol["fp64"], 256, sol["ref"], 512, 2, v, 1.0) for v in range(4)]
    e32 = [_l1_vs_finer(sol["fp32"], 256, sol["ref"], 512, 2, v, 1.0) for v in range(4)]
    ratio = [x / y for x, y in zip(e32, e64)]
    out["shock"] = {"problem": "four-quadrant Riemann data (seed %d), Q2, 256^2 to T = %g, L1 per variable "
                               "against a 512^2 FP64 run" % (seed, T),
                    "l1_fp64": e64, "l1_fp32": e32, "ratio_fp32_over_fp64": ratio,
                    "max_rel_deviation": max(abs(r - 1.0) for r in ratio), "bar": 0.02}
    out["reference"] = "the FP64 path, equal to the FP64 oracle within relative L1 1e-11 (tests/test_gpu_parity.py)"
    return out


def run_served_rates(N, stream, args):
    """S3 at each requested arrival rate (FP32 form; with --served-fp64 also the plain FP64 path on
    the two smallest sides). Every rate above the measured service rate saturates one GPU, so the
    latency there is queueing time; `saturation_solves_per_s` is the throughput the GPU sustained."""
    rates = [float(x) for x in args.served_rates.split(",") if x.strip()]
    per_rate = []
    for r in rates:
        per_rate.append(run_served(N, stream, r, args.served_requests, args.served_budget_gb * 1e9,
                                   args.served_policy))
        if args.served_fp64:
            per_rate.append(run_served(N, stream, r, args.served_requests, args.served_budget_gb * 1e9,
                                       args.served_policy, precision=N.PREC_FP64, sides=(128, 256)))
    fp32 = [x for x in per_rate if x.get("precision") == "FP32 form" and x.get("completed")]
    return {"per_rate": per_rate,
            "saturation_solves_per_s": max((x["throughput_solves_per_s"] for x in fp32), default=None),
            "failed_total": sum(x.get("failed", 0) for x in per_rate)}


def make_solver(N, precision, nx, seed, stream, tile=(0, 0), hybrid=0):
    from paper_2407_19169_gb300 import inputs as I
    s = N.Solver(dim=2, nx=nx, ny=nx, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc=(N.BC_OUTFLOW,) * 4, k=2,
                 eq=N.EQ_EULER, filter=1, cfl=0.1, gamma=1.4, precision=precision, stream=stream,
                 tile_rows=tile[0], tile_warps=tile[1], hybrid=hybrid)
    s.set_initial(N.IC_QUADRANT2D, I.quadrant_params(seed))
    return s


def time_steps(torch, s, steps, stream, barrier):
    """K steps bracketed by a barrier and synchronize on both sides, CUDA events on the solver's
    stream. Returns (ms, kernel launches inside the timed region)."""
    barrier()
    torch.cuda.synchronize()
    l0 = s.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.advance_steps(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    st, t, n = s.sync()
    if st != 0:
        raise RuntimeError("solver reported status %d during the timed steps" % st)
    return e0.elapsed_time(e1), s.kernel_launches() - l0


def cpu_baseline(nx_sample, seconds, seed):
    """The FP64 oracle (as it stands) on this host's cores, on the same problem at a bounded size."""
    import oracle as O
    from paper_2407_19169_gb300 import inputs as I
    cores = os.cpu_count() or 1
    O.set_threads(cores)
    p = O.Problem(dim=2, nx=nx_sample, ny=nx_sample, x0=0, x1=1, y0=0, y1=1, k=2, eq=O.EQ_EULER,
                  bc=(O.BC_OUTFLOW,) * 4, cfl=0.1)
    u = O.project(p, O.IC_QUADRANT2D, I.quadrant_params(seed))
    steps = 0
    t0 = time.perf_counter()
    while True:
        u = O.step(p, u, O.dt(p, u))
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds and steps >= 2:
            break
    dofs = p.ncell * p.nvars * p.nmodes
    return {"value": 3.0 * dofs * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%dx%d Q2 Euler quadrant problem, %d SSP-RK3 steps (%.1f s), FP64, %d threads"
                      % (nx_sample, nx_sample, steps, el, cores)}


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, each step a bounded sample (one SSP-RK3
    step of the same problem on a 128 x 128 mesh)."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle as O
    from paper_2407_19169_gb300 import inputs as I
    cores = os.cpu_count() or 1
    O.set_threads(cores)
    nxs = 128
    p = O.Problem(dim=2, nx=nxs, ny=nxs, x0=0, x1=1, y0=0, y1=1, k=2, eq=O.EQ_EULER,
                  bc=(O.BC_OUTFLOW,) * 4, cfl=0.1)
    seed = first_accepted_seed()
    u = O.project(p, O.IC_QUADRANT2D, I.quadrant_params(seed))
    for _ in range(args.warmup):
        u = O.step(p, u, O.dt(p, u))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u = O.step(p, u, O.dt(p, u))
    el = time.perf_counter() - t0
    dofs = p.ncell * p.nvars * p.nmodes
    value = 3.0 * dofs * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "reference_step": "one SSP-RK3 step on a 128x128 mesh of "
                       "the same problem (bounded sample)", "seed": seed},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "128x128 Q2 Euler quadrant problem, %d steps, %d threads"
                                       % (args.steps, cores)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mesh", type=int, default=2048, help="cells per side (2048 = the benchmark workload)")
    ap.add_argument("--fp64-steps", type=int, default=20, help="timed steps of the (slow) FP64 leg")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--skip-tune", action="store_true")
    ap.add_argument("--tile-rows", type=int, default=0, help="force the 2D tile rows (skips tuning)")
    ap.add_argument("--tile-warps", type=int, default=0, help="force the warps per block")
    ap.add_argument("--skip-hybrid", action="store_true")
    ap.add_argument("--hybrid-steps", type=int, default=100)
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--batched-instances", type=int, default=512)
    ap.add_argument("--batched-steps", type=int, default=200)
    ap.add_argument("--batched-tile-rows", type=int, default=0, help="2D tile rows of the batch (0 = autotuned)")
    ap.add_argument("--skip-served", action="store_true")
    ap.add_argument("--skip-small", action="store_true")
    ap.add_argument("--skip-accuracy", action="store_true")
    ap.add_argument("--served-policy", default="srpt", choices=["srpt", "all"],
                    help="which resident solves each round advances (serve.Engine)")
    ap.add_argument("--served-rates", default="10,500",
                    help="comma-separated Poisson arrival rates (requests/s), one served run each")
    ap.add_argument("--served-requests", type=int, default=12)
    ap.add_argument("--served-fp64", action="store_true",
                    help="also serve the plain FP64 path (sides 128 and 256) at each rate")
    ap.add_argument("--served-only", action="store_true",
                    help="run the served sweep alone and print its JSON (no headline line)")
    ap.add_argument("--served-budget-gb", type=float, default=120.0)
    args = ap.parse_args()
    if args.warmup < 3 and args.mesh == 2048:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    from paper_2407_19169_gb300 import _native as N
    if not os.path.exists(N.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

        def barrier():
            dist.barrier()
    else:
        def barrier():
            pass
    # a stream of our own: the legacy default stream (handle 0) cannot hold a captured graph, and the
    # events below must sit on the stream the kernels run on
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sh = stream.cuda_stream
    assert sh != 0
    seed = first_accepted_seed()
    nx = args.mesh
    out = {}
    if args.served_only:
        if rank == 0:
            print(json.dumps({"served": run_served_rates(N, stream, args)}), flush=True)
        return

    # ---- headline: the FP32 form, inputs resident, autotuned tile shape ----
    tile = (args.tile_rows, args.tile_warps)
    if not args.skip_tune and not args.tile_rows:
        from paper_2407_19169_gb300 import tuning
        tile = tuning.tune_2d(nx, nx, k=2)
    s32 = make_solver(N, N.PREC_FP32_MIXED, nx, seed, sh, tile)
    nv, nm, nc = s32.shape
    ndof = nv * nm * nc
    s32.advance_steps(args.warmup)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms32, launches32 = time_steps(torch, s32, args.steps, stream, barrier)
    clocks = clk.summary()
    state_bytes32 = nv * nc * (8 + 4 * (nm - 1))

    # ---- the plain FP64 path ----
    fp64 = None
    if not args.skip_fp64:
        # the library's default schedule: the FP32 tile does not carry over (the FP64 kernel's row
        # slots are twice as large, so fewer of its blocks fit in shared memory)
        s64 = make_solver(N, N.PREC_FP64, nx, seed, sh)
        s64.advance_steps(args.warmup)
        torch.cuda.synchronize()
        k64 = args.fp64_steps
        ms64, launches64 = time_steps(torch, s64, k64, stream, barrier)
        fp64 = {"value": 3.0 * ndof * k64 / (ms64 * 1e-3), "unit": UNIT, "steps": k64,
                "ms_per_step": ms64 / k64, "stage_kernel_ms": ms64 / (3 * k64), "dtype": "f64",
                "tile": "library default",
                "hbm_frac": (8.0 / 3.0) * 8 * ndof / (ms64 / (3 * k64) * 1e-3) / 1e9 / peaks()[0]}
        s64.close()
        del s64

    # ---- the hybrid limiter of Algorithm 1 on the same problem (stage kernel + blend kernel) ----
    hybrid = None
    if not args.skip_hybrid:
        sh_ = make_solver(N, N.PREC_FP32_MIXED, nx, seed, sh, tile, hybrid=1)
        sh_.advance_steps(args.warmup)
        torch.cuda.synchronize()
        msh, launchesh = time_steps(torch, sh_, args.hybrid_steps, stream, barrier)
        hybrid = {"value": 3.0 * ndof * args.hybrid_steps / (msh * 1e-3), "unit": UNIT, "steps": args.hybrid_steps,
                  "ms_per_step": msh / args.hybrid_steps, "gpu_launches": launchesh, "dtype": "f32+df64",
                  "note": "Algorithm 1 after every stage: eta and filter factors from the stage kernel, "
                          "max eta, then the troubled cells blended by a second kernel"}
        sh_.close()
        del sh_

    # ---- end to end through the C ABI with pinned host buffers ----
    e2e = None
    if not args.skip_e2e:
        host = torch.empty(ndof, dtype=torch.float64, pin_memory=True)
        s32.read_state_host_ptr(host.data_ptr(), ndof)          # a valid initial state
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s32.write_state_host_ptr(host.data_ptr(), ndof, 0.0)
        s32.advance_steps(args.steps)
        s32.read_state_host_ptr(host.data_ptr(), ndof)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        barrier()
        e2e = {"value": 3.0 * ndof * args.steps / el, "unit": UNIT,
               "h2d_bytes_per_step": int(8 * ndof / args.steps), "d2h_bytes_per_step": int(8 * ndof / args.steps),
               "note": "one solve of K steps per timed region: the FP64 canonical state is copied in "
                       "from pinned host memory before the steps and read back after them"}
    s32.close()

    # ---- roofline of the stage kernel (the only kernel in the timed region) ----
    hbm, src = peaks()
    launch_ms = ms32 / (3 * args.steps)
    alg_bytes = (8.0 / 3.0) * state_bytes32          # 8 state moves per 3 stages
    achieved = alg_bytes / (launch_ms * 1e-3) / 1e9
    dist_mod = None
    if world > 1:
        import torch.distributed as dist_mod
    value, ms32 = aggregate(torch, dist_mod, ms32, 3.0 * ndof * args.steps, world, "cuda")

    batched = None if args.skip_batched else run_batched(torch, N, stream, args.batched_steps,
                                                         args.batched_instances, args.batched_tile_rows)
    served = None if args.skip_served else run_served_rates(N, stream, args)
    small = None if args.skip_small else run_small_configs(torch, N, stream, barrier)
    accuracy = None if args.skip_accuracy else run_accuracy(N, stream)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+df64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "mesh": [nx, nx], "degree": 2, "basis": "Q2", "dofs": ndof,
                   "seed": seed, "precision": "FP32 stage arithmetic, cell averages double-float",
                   "l2": "inputs larger than L2 (state %.0f MB per buffer)" % (state_bytes32 / 1e6),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "tile": {"rows": tile[0], "warps": tile[1], "source": "forced" if args.tile_rows else ("autotuned" if tile[0] else "default")}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": recorded_traffic() if nx == 2048 else None, "peak_source": src,
                     "kernel": "stage2d_kernel<2,EULER,Q,FP32 form>", "launch_ms": launch_ms,
                     "alg_bytes_per_launch": alg_bytes},
        "clocks": clocks,
        "gpu_launches": launches32,
        "fp64": fp64,
        "fp32_over_fp64": (value / fp64["value"]) if fp64 else None,
        "e2e": e2e,
        "hybrid": hybrid,
        "batched": batched,
        "served": served,
        "small_configs": small,
        "accuracy": accuracy,
    }
    if not args.skip_cpu:
        line["cpu_baseline"] = cpu_baseline(128 if nx >= 128 else nx, args.cpu_seconds, seed)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
