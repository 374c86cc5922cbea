#!/usr/bin/env python
"""Benchmark: frequency-domain FWI misfit + adjoint-state gradient throughput.

One step = f and g = E^T sum w^2 Re(conj(u) v) over a fixed set of (source,
frequency) pairs: 2 batched Helmholtz solves per pair (forward and adjoint),
complex64 FGMRES + ML-GMRES inner solves inside FP64 iterative refinement,
receiver restriction, adjoint sources and gradient accumulation, all in
libhelm.so's kernels.

Default workload (N=1): the multi-frequency differentiation model -- 192^3
physical grid, h = 25 m, 10-cell damping layers (213^3 computational nodes),
seeded layered velocity 1500-4500 m/s with 20 Gaussian inclusions as the true
model and its smoothed version as the evaluation model, 128 sources on an 8x16
surface grid, receivers at every surface node, 8 frequencies 2-8 Hz.  A step
evaluates one source (the one nearest the centre) at all 8 frequencies: 8 of
the workload's 1024 pairs, each solve on the full grid.  With N ranks
(torchrun) rank r takes the next source along, and the ranks sum f and g with
one all-reduce (the paper's sum over workers): weak scaling.

`--workload layered64` selects the smaller 64^3 layered model (4 Hz, 16
sources per step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "misfit+gradient (src·freq)/s and stencil Gpts/s, % HBM roofline, at ≤1e-8 rel err"
METRIC_GN = "Gauss-Newton Hessian-vector product J^T J dm (src\u00b7freq)/s (3 PDE solves per pair)"
METRIC_HESS = "full Hessian-vector product of the misfit (src\u00b7freq)/s (4 PDE solves per pair)"
UNIT = "(src·freq)/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--precond", default="mlgmres", choices=["mlgmres", "jacobi", "none"])
    p.add_argument("--levels", type=int, default=2)
    p.add_argument("--tol", type=float, default=None,
                   help="FP64 relative residual of every solve (default 2e-10 on the 192^3 model, 1e-9 on the 64^3 one)")
    p.add_argument("--tol-inner", type=float, default=0.1)
    p.add_argument("--k-inner", type=int, default=0, help="outer FGMRES cycle length (0: 8 on the 192^3 step, "
                   "10 elsewhere with ML-GMRES, else 30)")
    p.add_argument("--reorth", type=int, default=None,
                   help="outer Gram-Schmidt re-orthogonalisation (default 0 on the 192^3 step, 1 elsewhere)")
    p.add_argument("--max-batch", type=int, default=0, help="right-hand sides solved together (0 = all)")
    p.add_argument("--smoother", default=None, help="ML-GMRES (k_so, k_si, k_co, k_ci); default 3,6,8,6 on "
                   "multifreq192, 3,6,3,6 on layered64")
    p.add_argument("--workload", default="multifreq192", choices=["multifreq192", "layered64"])
    p.add_argument("--step-sources", type=int, default=1,
                   help="multifreq192: sources per step (each at all 8 frequencies)")
    p.add_argument("--n", type=int, default=64, help="layered64: grid size")
    p.add_argument("--e2e-steps", type=int, default=3, help="steps timed end to end from host buffers")
    p.add_argument("--fp64-calls", type=int, default=5, help="timed calls of the FP64 per-source baseline")
    p.add_argument("--no-accuracy", action="store_true")
    p.add_argument("--shape", type=int, default=None, help="apply mode: time only this stencil tile shape")
    p.add_argument("--no-fp64-baseline", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=None,
                   help="oracle sample per process (default 20 s on the 192^3 model, 15 s on the 64^3 one)")
    p.add_argument("--workers", type=int, default=4, help="batch mode: models in flight together")
    p.add_argument("--op", default="misfit_grad", choices=["misfit_grad", "gn", "hess"],
                   help="step mode: misfit + gradient, the Gauss-Newton product J^T J dm, or the full Hessian product")
    p.add_argument("--nk", type=int, default=16, help="2.5D mode: k_y quadrature nodes")
    p.add_argument("--lam", type=float, default=1e4, help="WRI mode: penalty weight lambda")
    p.add_argument("--mode", default="step", choices=["step", "apply", "batch", "25d", "wri", "full"],
                   help="step: the misfit+gradient benchmark; apply: the stencil alone (helm_apply on the "
                        "workload's 16 complex64 fields)")
    a = p.parse_args()
    big_step = a.workload == "multifreq192" and a.mode in ("step", "full")
    if a.reorth is None:
        a.reorth = 0 if big_step else 1
    if a.k_inner == 0 and big_step:
        a.k_inner = 8
    if a.tol is None:
        a.tol = 2e-10 if a.workload == "multifreq192" and a.mode in ("step", "full") else 1e-9
    if a.cpu_seconds is None:
        a.cpu_seconds = 20.0 if a.workload == "multifreq192" else 15.0
    if a.smoother is None:
        a.smoother = "3,6,8,6" if a.mode in ("step", "full") and a.workload == "multifreq192" else "3,6,3,6"
    return a


def run_apply(args):
    """Stencil microbenchmark: y = H x for the workload's step fields (192^3 model: 8 fields of 213^3;
    64^3 model: 16 fields of 85^3), complex64 with every tile shape and the tuned one, and complex128."""
    import torch
    from paper_1703_09268_gb300 import helm
    dev = torch.device("cuda", 0)
    wl, name = make_workload(args, 0, 1)
    nf = wl.nsrc * wl.nfreq
    plan = helm.Plan(helm.make_grid(3, wl.n, wl.h, wl.npml, wl.v_ref, levels=args.levels), helm.default_opts(),
                     device=dev)
    m0 = torch.as_tensor(wl.m0.ravel(), dtype=torch.float64, device=dev)
    hbm, kind = peaks()
    out = dict(mode="apply", workload=name, grid_comp=list(plan.N), fields=nf, peak=hbm, peak_kind=kind)

    def timed(x, y):
        for _ in range(args.warmup):
            helm.helm_apply(plan, m0, wl.freqs_hz[0], x, out=y)
        helm.profile_enable(True)
        for _ in range(args.steps):
            helm.helm_apply(plan, m0, wl.freqs_hz[0], x, out=y)
        prof = helm.profile_read()
        helm.profile_enable(False)
        return prof

    kinds = (("c64", torch.complex64, 16.0), ("c128", torch.complex128, 32.0))
    if args.shape is not None:
        kinds = kinds[:1]  # one forced complex64 shape (for a profiler capture)
    for name_, dt, bpp in kinds:
        x = torch.randn(nf, plan.n_comp, dtype=dt, device=dev)
        y = torch.empty_like(x)
        if args.shape is not None:
            shapes = [(args.shape, helm.stencil_variants()[args.shape])]
        else:
            shapes = ([(v, sh) for v, sh in enumerate(helm.stencil_variants())] if name_ == "c64" else []) + \
                [(-1, None)]
        for v, sh in shapes:
            helm.stencil_select(v)
            st = timed(x, y)["stencil_" + name_]
            t = st["ms"] / 1e3
            rec = dict(gpts=round(st["bytes"] / bpp / t / 1e9, 1), gbs=round(st["bytes"] / t / 1e9, 1),
                       frac=round(st["bytes"] / t / 1e9 / hbm, 3), us_per_launch=round(1e6 * t / st["launches"], 2))
            if v >= 0:
                out.setdefault("c64_shapes", []).append(dict(shape=sh, **rec))
            else:
                tuned = helm.stencil_tuned(plan, 0)
                out[name_] = dict(rec, tuned_shape=tuned[0] if tuned and name_ == "c64" else None)
        helm.stencil_select(-1)
    print(json.dumps(out), flush=True)


def run_batch(args):
    """Batching workload: 8 models of uneven size (48^3 ... 160^3, h = 25 m, smooth random
    velocity) x 32 sources x 3 frequencies (3, 4, 5 Hz) = 768 (source, frequency) pairs per
    step, evaluated by one helm_misfit_and_gradient_batch call (a work queue of models, each on
    its own stream).  Reports throughput with `--workers` models in flight and with one."""
    import torch
    from paper_1703_09268_gb300 import helm, synth
    dev = torch.device("cuda", 0)
    wls = sorted(synth.batch_models(), key=lambda w: -w.n_phys)  # large models first
    kso, ksi, kco, kci = (int(v) for v in args.smoother.split(","))
    reqs = []
    for wl in wls:
        grid = helm.make_grid(3, wl.n, wl.h, wl.npml, wl.v_ref, levels=2)
        opts = helm.default_opts(precision=helm.MIXED if args.precision == "mixed" else helm.FP64,
                                 tol=args.tol, tol_inner=args.tol_inner, k_so=kso, k_si=ksi, k_co=kco, k_ci=kci,
                                 max_batch=args.max_batch or 32)
        plan = helm.Plan(grid, opts, device=dev)
        T = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
        src, Q, rec = T(wl.src_idx, torch.int32), T(wl.Q, torch.complex128), T(wl.rec_idx, torch.int32)
        # observed data: forward modelling in the true model (input generation, untimed), complex64 inner
        # solves refined in FP64 to 1e-11
        p_obs = helm.Plan(grid, helm.default_opts(precision=helm.MIXED, tol=1e-11, k_so=kso, k_si=ksi, k_co=kco,
                                                  k_ci=kci, max_batch=32), device=dev)
        _, d, _ = helm.helm_forward(p_obs, T(wl.m_true.ravel(), torch.float64), wl.freqs_hz, src, Q, rec,
                                    want_fields=False)
        p_obs.close()
        del p_obs
        torch.cuda.empty_cache()
        reqs.append(dict(plan=plan, m_phys=T(wl.m0.ravel(), torch.float64), freqs_hz=wl.freqs_hz, src_idx=src, Q=Q,
                         rec_idx=rec, d_obs=d))
    units = sum(len(w.freqs_hz) * w.nsrc for w in wls)
    out = dict(mode="batch", models=[w.name for w in wls], pairs=units, precision=args.precision, tol=args.tol)
    # FP64 (the workload as stated) is ~10x slower: timed with the work queue only
    for nw in ((args.workers,) if args.precision == "fp64" else (args.workers, 1)):
        for _ in range(args.warmup):
            helm.misfit_and_gradient_batch(reqs, nworkers=nw)
        torch.cuda.synchronize()
        t0 = time.time()
        for _ in range(args.steps):
            res = helm.misfit_and_gradient_batch(reqs, nworkers=nw)
        torch.cuda.synchronize()
        dt = (time.time() - t0) / args.steps
        out[f"workers_{nw}"] = dict(value=round(units / dt, 3), unit=UNIT, s_per_step=round(dt, 3),
                                    max_rel_resid=max(r["rel_resid"] for _, _, rep in res for r in rep),
                                    statuses=sorted({r["status"] for _, _, rep in res for r in rep}))
    out["max_batch"] = args.max_batch or 32
    print(json.dumps(out), flush=True)


def peaks():
    try:
        with open(PEAKS_FILE) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


def workload(n, rank, world):
    """64^3 layered model: 16 sources per rank on a (4*world) x 4 surface grid; rank r takes every world-th."""
    from paper_1703_09268_gb300 import synth
    wl = synth.workload_3d_layered(n=n, h=25.0 * 64 / n)
    if world > 1:
        nx_s = 4 * world
        nodes = [(int((i + 0.5) * n / nx_s), int((j + 0.5) * n / 4), 2) for j in range(4) for i in range(nx_s)]
        nodes = nodes[rank::world]
        wl.src_idx, wl.Q = synth.point_sources(wl.n, nodes)
    return wl


def step_columns(wl, rank, k):
    """Source columns of rank r's step: k consecutive sources starting after the
    centre source's r*k predecessors (the centre source first on rank 0)."""
    from paper_1703_09268_gb300 import synth
    s0 = synth.centre_source(wl)
    return [(s0 + rank * k + i) % wl.nsrc for i in range(k)]


def workload_multifreq(rank, world, k):
    """192^3 x 128 sources x 8 frequencies; the step's sources of this rank, all frequencies."""
    from paper_1703_09268_gb300 import synth
    wl = synth.workload_3d_multifreq()
    cols = step_columns(wl, rank, k)
    wl.meta["columns"] = cols
    wl.meta["nsrc_total"] = wl.nsrc
    wl.src_idx, wl.Q = synth.source_subset(wl, cols)
    return wl


def make_workload(args, rank, world):
    if args.workload == "multifreq192":
        wl = workload_multifreq(rank, world, args.step_sources)
        name = (f"{wl.name}: step = {wl.nsrc} source(s) x {wl.nfreq} frequencies "
                f"({wl.nsrc * wl.nfreq} of {wl.meta['nsrc_total'] * wl.nfreq} pairs)")
        return wl, name
    wl = workload(args.n, rank, world)
    return wl, wl.name


# DRAM traffic of the single-precision stencil from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of k_stencil_plain<float, 0, 4,
# 128, 32, 8> on the 8 fields of 213^3 of one step, `bench.py --mode apply
# --shape 6`).  It scales with the points a launch processes.  Set to None when
# the kernel changes until it is captured again.
STENCIL_TRAFFIC = dict(kernel="k_stencil_plain<float, 0, 4, 128, 32, 8>", dram_bytes=739.457792e6 + 581.15968e6,
                       algorithmic_bytes=8 * 9663597 * 16 + 9663597 * 4)


def stencil_traffic(kernel_class, bytes_per_launch):
    if kernel_class != "stencil_c64" or STENCIL_TRAFFIC is None:
        return None
    t = STENCIL_TRAFFIC
    return round(t["dram_bytes"] * bytes_per_launch / t["algorithmic_bytes"], 1)


# ---------------------------------------------------------------------------
# CPU baseline: the oracle's restarted GMRES on the same operator
# ---------------------------------------------------------------------------

def _host_mem_gb():
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return float(line.split()[1]) / 1e6
    except OSError:
        pass
    return None


def _oracle_setup(spec):
    """Operator, right-hand side of one pair of the workload `spec` (oracle only)."""
    import numpy as _np
    from oracle import helmholtz as O
    from paper_1703_09268_gb300 import synth
    if spec["kind"] == "multifreq192":
        wl = synth.workload_3d_multifreq()
        src, Q = synth.source_subset(wl, [synth.centre_source(wl)])
        fr = wl.freqs_hz[spec["k"] % wl.nfreq]
    else:
        wl = synth.workload_3d_layered(n=spec["n"], h=25.0 * 64 / spec["n"])
        src, Q = wl.src_idx, wl.Q[:, spec["k"] % wl.nsrc:spec["k"] % wl.nsrc + 1]
        fr = wl.freqs_hz[0]
    g = O.make_grid(3, wl.n, wl.h, wl.npml, wl.v_ref, levels=2)
    H = O.helmholtz_matrix(g, O.extend(g, wl.m0), 2 * _np.pi * fr)
    q = O.source_fields(g, src, Q)[0]
    return O, H, q, list(g.N)


_ORACLE = {}


def _oracle_init(kind, n):
    """Pool initializer: build this process's operator and right-hand side once
    (process i takes frequency / source i of the workload)."""
    import multiprocessing as _mp
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    sys.path.insert(0, ROOT)
    ident = _mp.current_process()._identity
    k = (ident[0] - 1) if ident else 0
    t0 = time.time()
    O, H, q, N = _oracle_setup(dict(kind=kind, n=n, k=k))
    _ORACLE.update(O=O, H=H, q=q, N=N, setup=time.time() - t0)


def _oracle_time(args):
    """The oracle's GMRES(60) on the full-size operator: cycles of `cycle_iters`
    iterations until `seconds` are spent (at least one cycle)."""
    seconds, cycle_iters = args
    O, H, q = _ORACLE["O"], _ORACLE["H"], _ORACLE["q"]
    it_total, t_run, x = 0, 0.0, None
    while t_run < seconds or it_total == 0:
        t1 = time.time()
        x, it, _ = O.gmres(H, q, tol=1e-30, restart=60, maxiter=cycle_iters, x0=x)
        t_run += time.time() - t1
        it_total += it
    return dict(iters=it_total, seconds=t_run, setup=_ORACLE["setup"], grid=_ORACLE["N"])


class OraclePool:
    """Spawned single-thread processes holding the oracle's full-size operator
    (as many as the host cores and memory allow)."""

    def __init__(self, kind, n):
        import multiprocessing as mp
        per_proc_gb = 13.0 if kind == "multifreq192" else 1.5  # GMRES(60) basis + operator per process
        mem = _host_mem_gb()
        self.procs = max(1, min(os.cpu_count() or 1, 16, int(mem // per_proc_gb) if mem else 16))
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"  # one BLAS thread per spawned process (set before the children import numpy)
        try:
            self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_oracle_init, initargs=(kind, n))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def sample(self, seconds, cycle_iters):
        return self.pool.map(_oracle_time, [(seconds, cycle_iters)] * self.procs, chunksize=1)

    def close(self):
        self.pool.close()
        self.pool.join()


def _iteration_counts(kind, n):
    name = "gmres_iterations_3d_multifreq_32.json" if kind == "multifreq192" else f"gmres_iterations_3d_layered_{n}.json"
    path = os.path.join(ROOT, "oracle", "data", name)
    if not os.path.exists(path):
        return None, path
    with open(path) as fh:
        d = json.load(fh)
    if kind == "multifreq192":
        return float(d["iterations_per_pair"]), path
    return float(d["forward_iterations"] + d["adjoint_iterations"]), path


def cpu_baseline(kind, n, seconds, cycle_iters=60, pool=None):
    """(src.freq)/s of the oracle on the host cores: a bounded sample of GMRES(60)
    iterations on the full-size operator, one spawned single-thread process per
    core (as many as host memory allows), scaled by the oracle's own iteration
    count for a forward + adjoint solve."""
    per_pair_iters, path = _iteration_counts(kind, n)
    if per_pair_iters is None:
        return None
    own = pool is None
    if own:
        pool = OraclePool(kind, n)
    try:
        res = pool.sample(seconds, cycle_iters)
    finally:
        if own:
            pool.close()
    procs = pool.procs
    t_iter = float(np.mean([r["seconds"] / r["iters"] for r in res]))
    value = procs / (per_pair_iters * t_iter)
    grid = res[0]["grid"]
    if kind == "multifreq192":
        how = (f"the oracle's iteration count per pair ({per_pair_iters:.0f}, forward + adjoint to tol 1e-9, mean over "
               f"the 8 frequencies) measured on the 32^3 crop of the same recipe ({os.path.basename(path)}); the count "
               f"only grows with the grid, so this is an upper bound on the oracle's throughput")
    else:
        how = f"the oracle's {per_pair_iters:.0f} iterations for one forward + adjoint solve ({os.path.basename(path)})"
    cyc = ("full GMRES(60) cycles" if cycle_iters >= 60 else
           f"the first {cycle_iters} iterations of GMRES(60) cycles (the cheapest of a cycle, so the time per "
           f"iteration is a lower bound)")
    return dict(value=value, unit=UNIT, cores=procs, kind="oracle",
                sample=(f"{procs} spawned single-thread processes, each timing {cyc} on the full {grid} operator "
                        f"(~{max(seconds, 0):.0f} s, {int(np.mean([r['iters'] for r in res]))} iterations, "
                        f"{t_iter*1e3:.0f} ms each; assembly {np.mean([r['setup'] for r in res]):.0f} s excluded), "
                        f"scaled by {how}"))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = []
    big = args.workload == "multifreq192"
    if _iteration_counts(args.workload, args.n)[0] is None:
        print(json.dumps(dict(impl="reference", unavailable="the oracle's iteration counts are missing")))
        return
    pool = OraclePool(args.workload, args.n)
    walls = []
    try:
        for i in range(args.warmup + args.steps):
            # multifreq192: each step times the first 3 iterations of a GMRES(60) cycle per process (cheaper
            # than the cycle's mean, so the value is an upper bound)
            t0 = time.perf_counter()
            cb = cpu_baseline(args.workload, args.n, 0.0 if big else max(2.0, args.cpu_seconds / 3),
                              cycle_iters=3 if big else 60, pool=pool)
            if i >= args.warmup:
                steps.append(cb["value"])
                walls.append(time.perf_counter() - t0)
    finally:
        pool.close()
    v = float(np.median(steps))
    cb["value"] = v
    wl_name = ("3d-multifreq-192^3-h25-128src-8f (1 source x 8 frequencies)" if big
               else f"3d-layered-{args.n}^3-h25-pml10-4Hz-16src")
    units = 8 if big else 16
    # a step is the bounded sample the oracle processes ran (their wall time); the value extrapolates it
    # to the step's pairs as cpu_baseline.sample states
    line = dict(impl="reference", metric=METRIC, value=v, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=round(1e3 * float(np.median(walls)), 1), higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                extrapolated_ms_per_step=round(1e3 * units / v, 1),
                config=dict(workload=wl_name, pairs_per_step=units),
                cpu_baseline=cb, e2e=dict(value=v, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["unavailable"])
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return dict(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(smax) if smax else None,
                    reasons=sorted(reasons), samples=len(sm))


def run_25d(args):
    """2.5D misfit + gradient on a 401 x 201 layered x-z model: each (source,
    frequency) pair is nk shifted 2D solves and nk adjoint solves."""
    import torch
    from paper_1703_09268_gb300 import helm, synth

    dev = torch.device("cuda", 0)
    wl = synth.workload_25d()
    grid = helm.make_grid(2, wl.n, wl.h, wl.npml, wl.v_ref, levels=2)
    kso, ksi, kco, kci = (int(v) for v in args.smoother.split(","))
    mk = lambda prec, tol: helm.Plan(grid, helm.default_opts(  # noqa: E731
        precision=prec, precond=helm.PRECOND_MLGMRES, k_inner=args.k_inner or 10, tol=tol, max_cycles=400,
        tol_inner=args.tol_inner, k_so=kso, k_si=ksi, k_co=kco, k_ci=kci, max_batch=args.max_batch), device=dev)
    plan = mk(helm.MIXED if args.precision == "mixed" else helm.FP64, args.tol)
    # Gauss-Legendre k_y nodes on [0, 1.2 w / v_min] (Sec. 3, 2.5D), receivers in the sources' plane
    om = 2 * np.pi * wl.freqs_hz[0]
    t, w = np.polynomial.legendre.leggauss(args.nk)
    kmax = 1.2 * om / wl.meta["vmin"]
    ky = 0.5 * kmax * (t + 1)
    ck = 0.5 * kmax * w / np.pi
    T = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
    m0 = T(wl.m0.ravel(), torch.float64)
    src, Q, rec = T(wl.src_idx, torch.int32), T(wl.Q, torch.complex128), T(wl.rec_idx, torch.int32)
    rng = np.random.default_rng(9)
    d_obs = T(1e-4 * (rng.standard_normal((1, wl.nsrc, wl.nrec)) + 1j * rng.standard_normal((1, wl.nsrc, wl.nrec))),
              torch.complex128)
    step = lambda p: helm.misfit_and_gradient_25d(p, m0, wl.freqs_hz, ky, ck, src, Q, rec, d_obs)  # noqa: E731
    for _ in range(args.warmup):
        step(plan)
    torch.cuda.synchronize()
    launches0 = helm.kernel_launch_count()
    stream = torch.cuda.current_stream(dev)
    times = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f, g, rep = step(plan)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    launches = helm.kernel_launch_count() - launches0
    ms = float(np.mean(times))
    units = wl.nsrc * wl.nfreq
    helm.profile_enable(True)
    step(plan)
    torch.cuda.synchronize()
    prof = helm.profile_read()
    helm.profile_enable(False)
    hbm, hbm_kind = peaks()
    tot = sum(v["ms"] for v in prof.values())
    dom = max((k for k in prof if prof[k]["bytes"] > 0), key=lambda k: prof[k]["ms"])
    achieved = prof[dom]["bytes"] / (prof[dom]["ms"] / 1e3) / 1e9
    f64, g64, _ = step(mk(helm.FP64, 1e-13))
    out = dict(mode="25d", metric="2.5D misfit+gradient (src\u00b7freq)/s", value=round(units / (ms / 1e3), 3),
               unit=UNIT, ms_per_step=round(ms, 3), steps=args.steps, warmup=args.warmup, n_gpus=1,
               config=dict(workload=wl.name, grid_comp=list(plan.N), nk=args.nk, kmax=round(kmax, 6),
                           sources=wl.nsrc, receivers=wl.nrec, solves_per_step=2 * args.nk * units,
                           data="seeded random observed data (the work does not depend on it)"),
               roofline=dict(bound="hbm", kernel=dom, achieved=round(achieved, 1), peak=hbm, peak_kind=hbm_kind,
                             unit="GB/s", frac=round(achieved / hbm, 3),
                             share={k: round(v["ms"] / tot, 3) for k, v in prof.items() if v["launches"]}),
               gpu_launches=int(launches),
               solver=dict(outer_iters_per_solve_pair=float(np.mean([r["iters"] for r in rep]))),
               accuracy=dict(reference="FP64 GPU path to rel. residual 1e-13",
                             f_rel_err=float(abs(f.item() - f64.item()) / abs(f64.item())),
                             g_rel_err=float((g - g64).norm().item() / g64.norm().item())))
    print(json.dumps(out), flush=True)


def run_wri(args):
    """WRI (penalty) objective + gradient on the 401 x 201 x-z section of the
    2.5D workload (as a 2D problem): per pair one state solve plus two solves per
    receiver-space CG iteration."""
    import torch
    from paper_1703_09268_gb300 import helm, synth

    dev = torch.device("cuda", 0)
    wl = synth.workload_25d()
    grid = helm.make_grid(2, wl.n, wl.h, wl.npml, wl.v_ref, levels=2)
    kso, ksi, kco, kci = (int(v) for v in args.smoother.split(","))
    plan = helm.Plan(grid, helm.default_opts(
        precision=helm.MIXED if args.precision == "mixed" else helm.FP64, precond=helm.PRECOND_MLGMRES,
        k_inner=args.k_inner or 10, tol=args.tol, max_cycles=400, tol_inner=args.tol_inner, k_so=kso, k_si=ksi,
        k_co=kco, k_ci=kci, max_batch=args.max_batch), device=dev)
    T = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
    m0 = T(wl.m0.ravel(), torch.float64)
    src, Q, rec = T(wl.src_idx, torch.int32), T(wl.Q, torch.complex128), T(wl.rec_idx, torch.int32)
    # observed data: the 2D field of the true model at the receivers (input generation, untimed)
    p64 = helm.Plan(grid, helm.default_opts(precision=helm.FP64, precond=helm.PRECOND_MLGMRES, tol=1e-12,
                                            max_cycles=400), device=dev)
    _, d_obs, _ = helm.helm_forward(p64, T(wl.m_true.ravel(), torch.float64), wl.freqs_hz, src, Q, rec,
                                    want_fields=False)
    step = lambda: helm.wri_misfit_and_gradient(plan, m0, wl.freqs_hz, src, Q, rec, d_obs, args.lam,  # noqa: E731
                                                cg_tol=1e-9, cg_maxit=200)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    times = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f, g, rep = step()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = float(np.mean(times))
    units = wl.nsrc * wl.nfreq
    out = dict(mode="wri", metric="WRI misfit+gradient (src\u00b7freq)/s", value=round(units / (ms / 1e3), 3),
               unit=UNIT, ms_per_step=round(ms, 3), steps=args.steps, warmup=args.warmup, n_gpus=1,
               step_ms=dict(median=round(float(np.median(times)), 1), min=round(float(np.min(times)), 1),
                            max=round(float(np.max(times)), 1)),
               config=dict(workload=wl.name.replace("2.5d", "2d"), grid_comp=list(plan.N), lam=args.lam,
                           cg_tol=1e-9, sources=wl.nsrc, receivers=wl.nrec),
               solver=dict(solver_iters_per_pair=float(np.mean([r["iters"] for r in rep])),
                           statuses=sorted({r["status"] for r in rep})),
               f=float(f.item()))
    if not args.no_accuracy:
        # the same objective from FP64 solves to 1e-12 and receiver-space CG to 1e-12
        p64 = helm.Plan(grid, helm.default_opts(precision=helm.FP64, precond=helm.PRECOND_MLGMRES, k_inner=10,
                                                tol=1e-12, max_cycles=400, k_so=kso, k_si=ksi, k_co=kco, k_ci=kci,
                                                max_batch=args.max_batch), device=dev)
        f64, g64, _ = helm.wri_misfit_and_gradient(p64, m0, wl.freqs_hz, src, Q, rec, d_obs, args.lam, cg_tol=1e-12,
                                                   cg_maxit=400)
        out["accuracy"] = dict(reference="FP64 solves to 1e-12, CG to 1e-12",
                               f_rel_err=float(abs(f.item() - f64.item()) / abs(f64.item())),
                               g_rel_err=float((g - g64).norm().item() / g64.norm().item()))
    print(json.dumps(out), flush=True)


def run_full(args):
    """The whole 192^3 x 128-source x 8-frequency objective once, through the
    differentiable FWIObjective (policy "auto"), and its gradient checked by
    Richardson-extrapolated central differences of the misfit on 16 seeded
    smooth random directions over the step's pairs (one source, 8 frequencies).
    Prints one JSON line; no timing contract."""
    import torch
    from paper_1703_09268_gb300 import autograd, helm, synth
    dev = torch.device("cuda", 0)
    wl = synth.workload_3d_multifreq()
    grid = helm.make_grid(3, wl.n, wl.h, wl.npml, wl.v_ref, levels=2)
    kso, ksi, kco, kci = (int(v) for v in args.smoother.split(","))
    mk = lambda tol: helm.Plan(grid, helm.default_opts(  # noqa: E731
        precision=helm.MIXED, precond=helm.PRECOND_MLGMRES, k_inner=args.k_inner or 10, reorth=args.reorth, tol=tol,
        max_cycles=400, tol_inner=0.1, k_so=kso, k_si=ksi, k_co=kco, k_ci=kci, max_batch=args.max_batch or 32),
        device=dev)
    T = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
    src, Q, rec = T(wl.src_idx, torch.int32), T(wl.Q, torch.complex128), T(wl.rec_idx, torch.int32)
    out = dict(mode="full", workload=wl.name, grid_comp=None, pairs=wl.nsrc * wl.nfreq, smoother=args.smoother)
    # observed data of every pair: complex64 inner solves refined in FP64 to 1e-11 in the true model
    p_obs = mk(1e-11)
    out["grid_comp"] = list(p_obs.N)
    t0 = time.perf_counter()
    _, d_obs, rep = helm.helm_forward(p_obs, T(wl.m_true.ravel(), torch.float64), wl.freqs_hz, src, Q, rec,
                                      want_fields=False)
    torch.cuda.synchronize()
    out["observed_data"] = dict(seconds=round(time.perf_counter() - t0, 1),
                                max_rel_resid=max(r["rel_resid"] for r in rep))
    p_obs.close()
    del p_obs
    torch.cuda.empty_cache()
    # the full objective and gradient through torch autograd
    plan = mk(args.tol)
    prob = autograd.FWIProblem(plan=plan, freqs_hz=wl.freqs_hz, src_idx=src, Q=Q, rec_idx=rec, d_obs=d_obs,
                               policy="auto")
    policy = prob.resolve_policy()
    m = T(wl.m0.ravel(), torch.float64).requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f = autograd.fwi_objective(m, prob)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    (g,) = torch.autograd.grad(f, m)
    torch.cuda.synchronize()
    t_all = time.perf_counter() - t0
    out["objective"] = dict(policy=policy, f=float(f.item()), g_norm=float(g.norm().item()),
                            forward_seconds=round(t_fwd, 1), total_seconds=round(t_all, 1),
                            pairs_per_second=round(wl.nsrc * wl.nfreq / t_all, 4),
                            peak_memory_gb=round(torch.cuda.max_memory_allocated() / 1e9, 1))
    del g, f, prob
    plan.close()
    del plan
    torch.cuda.empty_cache()
    # central differences on 16 directions over the step's pairs, misfit-only solves to 1e-11
    cols = step_columns(wl, 0, 1)
    s_sub, q_sub = synth.source_subset(wl, cols)
    s_sub, q_sub = T(s_sub, torch.int32), T(q_sub, torch.complex128)
    d_sub = d_obs[:, cols].contiguous()
    pfd = mk(1e-11)
    m0 = wl.m0.ravel()
    _, g_sub, _ = helm.misfit_and_gradient(pfd, T(m0, torch.float64), wl.freqs_hz, s_sub, q_sub, rec, d_sub)
    g_sub = g_sub.cpu().numpy()
    rng = np.random.default_rng(16)

    def fval(mm):
        f_, _, _, _ = helm.helm_misfit(pfd, T(mm, torch.float64), wl.freqs_hz, s_sub, q_sub, rec, d_sub)
        return f_.item()

    # the largest relative model change is t_fd: the phase of an 8 Hz wave across the model moves by well
    # under a radian, so the Richardson remainder (fourth order in t_fd) stays far below the 1e-6 bar
    t_fd = 5e-4
    rows = []
    t0 = time.perf_counter()
    for k in range(16):
        dm = synth._gaussian_smooth(rng.standard_normal(wl.m0.shape), 8.0).ravel()
        dm = dm / np.abs(dm).max() * m0  # a relative perturbation of at most 1 per unit step

        def cd(h):
            return (fval(m0 + h * dm) - fval(m0 - h * dm)) / (2 * h)

        c1, c2 = cd(t_fd), cd(t_fd / 2)
        fd = (4 * c2 - c1) / 3
        an = float(g_sub @ dm)
        rows.append(dict(direction=k, adjoint=an, central_difference=fd, rel_diff=abs(fd - an) / abs(an),
                         plain_cd_half_step_rel_diff=abs(c2 - an) / abs(an)))
    out["finite_differences"] = dict(
        pairs=f"source column {cols[0]} x {wl.nfreq} frequencies", directions=16,
        recipe="smoothed (sigma 8 cells) seeded Gaussian noise scaled to max |.| = 1, times m0 (relative change)",
        step=t_fd, extrapolation="Richardson, (4 cd(t/2) - cd(t)) / 3", solve_tol=1e-11,
        max_rel_diff=max(r["rel_diff"] for r in rows), seconds=round(time.perf_counter() - t0, 1), table=rows)
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "apply":
        return run_apply(args)
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "25d":
        return run_25d(args)
    if args.mode == "wri":
        return run_wri(args)
    if args.mode == "full":
        return run_full(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    big = args.workload == "multifreq192"
    # the oracle's process pool is spawned before the first GPU call
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.op == "misfit_grad":
        cpu = cpu_baseline(args.workload, args.n, args.cpu_seconds, cycle_iters=10 if big else 60)

    import torch
    import torch.distributed as dist
    from paper_1703_09268_gb300 import helm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    wl, wl_name = make_workload(args, rank, world)
    levels = args.levels if args.precond == "mlgmres" else max(1, args.levels)
    grid = helm.make_grid(3, wl.n, wl.h, wl.npml, wl.v_ref, levels=levels)
    prec = {"mlgmres": helm.PRECOND_MLGMRES, "jacobi": helm.PRECOND_JACOBI, "none": helm.PRECOND_NONE}[args.precond]
    kin = args.k_inner or (10 if prec == helm.PRECOND_MLGMRES else 30)
    kso, ksi, kco, kci = (int(v) for v in args.smoother.split(","))
    opts = helm.default_opts(precision=helm.MIXED if args.precision == "mixed" else helm.FP64, precond=prec,
                             k_inner=kin, tol=args.tol, max_cycles=400, tol_inner=args.tol_inner, max_refine=60,
                             reorth=args.reorth, k_so=kso, k_si=ksi, k_co=kco, k_ci=kci, max_batch=args.max_batch)
    plan = helm.Plan(grid, opts, device=dev)
    T = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
    m0 = T(wl.m0.ravel(), torch.float64)
    src = T(wl.src_idx, torch.int32)
    Q = T(wl.Q, torch.complex128)
    rec = T(wl.rec_idx, torch.int32)
    # observed data: forward modelling in the true model (input generation, untimed): FP64 on the 64^3 model,
    # complex64 inner solves refined in FP64 to 1e-11 on the 192^3 one
    ref_opts = dict(precond=helm.PRECOND_MLGMRES, max_cycles=400, k_so=kso, k_si=ksi, k_co=kco, k_ci=kci)
    p_obs = helm.Plan(grid, helm.default_opts(precision=helm.MIXED if big else helm.FP64, tol=1e-11 if big else 1e-13,
                                              **ref_opts), device=dev)
    _, d_obs, _ = helm.helm_forward(p_obs, T(wl.m_true.ravel(), torch.float64), wl.freqs_hz, src, Q, rec,
                                    want_fields=False)
    p_obs.close()
    del p_obs
    torch.cuda.empty_cache()
    nsrc, nfreq = wl.nsrc, wl.nfreq
    units = nsrc * nfreq
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    gn, hess = args.op == "gn", args.op == "hess"
    # a seeded model perturbation for the Hessian products (input, resident)
    dmv = T(np.random.default_rng(7).standard_normal(wl.m0.size) * 1e-9, torch.float64) if gn or hess else None

    def step(p=plan, reduce=True, m=None, s_=None, q_=None, r_=None, d_=None, dm_=None, freqs=None):
        m, s_, q_, r_ = (m0 if m is None else m), (src if s_ is None else s_), (Q if q_ is None else q_), \
            (rec if r_ is None else r_)
        fr = wl.freqs_hz if freqs is None else freqs
        if gn or hess:
            dmx = dmv if dm_ is None else dm_
            if gn:
                h, rep = helm.helm_gn_hessvec(p, m, fr, s_, q_, r_, dmx)
            else:
                h, rep = helm.helm_hessvec(p, m, fr, s_, q_, r_, d_obs if d_ is None else d_, dmx)
            if world > 1 and reduce:
                dist.all_reduce(h)
            return None, h, rep
        f, g, rep = helm.misfit_and_gradient(p, m, fr, s_, q_, r_, d_obs if d_ is None else d_)
        if world > 1 and reduce:
            dist.all_reduce(f)
            dist.all_reduce(g)
        return f, g, rep

    for _ in range(args.warmup):
        f, g, rep = step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    launches0 = helm.kernel_launch_count()
    times = []
    for _ in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (256 MB > 129 MB L2), outside the events
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f, g, rep = step()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    launches = helm.kernel_launch_count() - launches0
    ms = float(np.mean(times))
    ms_t = torch.tensor([ms], device=dev)
    if world > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    value = units * world / (ms_max / 1e3)
    iters = [r["iters"] for r in rep]
    refs = [r["refinements"] for r in rep]

    # one profiled step: per-kernel-class device time and algorithmic bytes
    helm.profile_enable(True)
    flush.zero_()
    torch.cuda.synchronize()
    t_prof = time.perf_counter()
    step(reduce=False)
    torch.cuda.synchronize()
    wall_prof_ms = 1e3 * (time.perf_counter() - t_prof)
    prof = helm.profile_read()
    helm.profile_enable(False)
    hbm, hbm_kind = peaks()
    tot_ms = sum(v["ms"] for v in prof.values())
    dom = max((k for k in prof if prof[k]["bytes"] > 0), key=lambda k: prof[k]["ms"])
    dn = prof[dom]
    achieved = dn["bytes"] / (dn["ms"] / 1e3) / 1e9
    roofline = dict(bound="hbm", kernel=dom, achieved=round(achieved, 1), peak=hbm, unit="GB/s",
                    frac=round(achieved / hbm, 3), traffic=None, peak_kind=hbm_kind,
                    launches=dn["launches"], avg_launch_us=round(1e3 * dn["ms"] / max(dn["launches"], 1), 2),
                    bytes_per_launch=dn["bytes"] / max(dn["launches"], 1),
                    share={k: round(v["ms"] / tot_ms, 3) for k, v in prof.items() if v["launches"]},
                    class_frac={k: round(v["bytes"] / (v["ms"] / 1e3) / 1e9 / hbm, 3)
                                for k, v in prof.items() if v["launches"] and v["bytes"] > 0 and v["ms"] > 0},
                    gpu_busy=round(tot_ms / wall_prof_ms, 3))
    roofline["traffic"] = stencil_traffic(dom, roofline["bytes_per_launch"])
    st = prof["stencil_c64"] if prof["stencil_c64"]["launches"] else prof["stencil_c128"]
    sbytes_pt = 16.0 if prof["stencil_c64"]["launches"] else 32.0
    stencil = dict(gpts=round(st["bytes"] / sbytes_pt / (st["ms"] / 1e3) / 1e9, 1),
                   gbs=round(st["bytes"] / (st["ms"] / 1e3) / 1e9, 1),
                   frac=round(st["bytes"] / (st["ms"] / 1e3) / 1e9 / hbm, 3),
                   launches=st["launches"], avg_launch_us=round(1e3 * st["ms"] / max(st["launches"], 1), 2))

    cfg = dict(workload=wl_name if world == 1 else f"{wl_name}-x{world}ranks", grid_comp=list(plan.N),
               pairs_per_step_per_rank=units, sources_per_rank=nsrc, freqs_hz=[round(float(x), 4) for x in wl.freqs_hz],
               receivers=wl.nrec, precond=args.precond, levels=levels, k_inner=kin, smoother=args.smoother,
               tol=args.tol, tol_inner=args.tol_inner, reorth=args.reorth, l2="flushed between timed steps (256 MB)",
               parallelism=f"dp{world} over sources, f and g all-reduced" if world > 1 else "1 GPU",
               op="J^T J dm (3 solves per pair)" if gn else
               "full Hessian times dm (4 solves per pair)" if hess else "misfit + gradient (2 solves per pair)")
    if big:
        cfg["source_columns"] = wl.meta["columns"]
    out = dict(metric=METRIC_GN if gn else METRIC_HESS if hess else METRIC, value=round(value, 4), unit=UNIT,
               n_gpus=world, steps=args.steps,
               warmup=args.warmup, ms_per_step=round(ms_max, 3), higher_is_better=True, scaling="weak",
               vs_baseline=None, dtype="c64 inner / f64 refine" if args.precision == "mixed" else "f64",
               data=("synthetic (seeded layered model with inclusions; observed data modelled in the true model, "
                     "complex64 inner / FP64 refinement to 1e-11)" if big else
                     "synthetic (seeded layered model, observed data modelled in FP64)"),
               config=cfg, roofline=roofline, stencil=stencil, gpu_launches=int(launches),
               solver=dict(outer_iters_per_pair=float(np.mean(iters)), refinements_per_pair=float(np.mean(refs)),
                           max_rel_resid=float(max(r["rel_resid"] for r in rep)),
                           iters_per_pair=iters),
               step_ms=dict(median=round(float(np.median(times)), 3), min=round(float(np.min(times)), 3),
                            max=round(float(np.max(times)), 3)),
               clocks=clk)
    if rank == 0:
        # accuracy against the FP64 GPU path (itself checked against the oracle in tests)
        if args.precision == "mixed" and not args.no_accuracy:
            tol64 = 1e-11 if big else 1e-13
            p64 = helm.Plan(grid, helm.default_opts(precision=helm.FP64, tol=tol64, **ref_opts), device=dev)
            t0 = time.perf_counter()
            if gn or hess:
                _, h64, _ = step(p=p64, reduce=False)
                _, h1, _ = step(reduce=False)
                out["accuracy"] = dict(reference=f"FP64 GPU path, FGMRES+ML-GMRES to rel. residual {tol64:g}",
                                       hessvec_rel_err=float((h1 - h64).norm().item() / h64.norm().item()))
            else:
                f64, g64, _ = step(p=p64, reduce=False)
                f1, g1, _ = step(reduce=False)
                out["accuracy"] = dict(
                    reference=f"FP64 GPU path, FGMRES+ML-GMRES to rel. residual {tol64:g}, same pairs",
                    f_rel_err=float(abs(f1.item() - f64.item()) / abs(f64.item())),
                    g_rel_err=float((g1 - g64).norm().item() / g64.norm().item()))
            torch.cuda.synchronize()
            out["accuracy"]["reference_seconds"] = round(time.perf_counter() - t0, 1)
            p64.close()
            del p64
            torch.cuda.empty_cache()
        if not args.no_fp64_baseline and not (gn or hess):
            # plain FP64 solves, one right-hand side at a time, same preconditioner and tolerance; on the
            # 192^3 model over the middle frequency's pair of the step (its mixed cost is near the step's mean)
            pb = helm.Plan(grid, helm.default_opts(precision=helm.FP64, precond=prec, k_inner=kin, tol=args.tol,
                                                   max_cycles=400, max_batch=1, k_so=kso, k_si=ksi, k_co=kco,
                                                   k_ci=kci), device=dev)
            if big:
                kf = nfreq // 2
                bfr, bd, bs, bq = wl.freqs_hz[kf:kf + 1], d_obs[kf:kf + 1, :1].contiguous(), src[:1], Q[:1, :1]
                bunits = 1
            else:
                bfr, bd, bs, bq, bunits = wl.freqs_hz, d_obs, src, Q, units
            helm.misfit_and_gradient(pb, m0, bfr, bs, bq, rec, bd)
            t64 = []
            for _ in range(max(1, args.fp64_calls)):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                helm.misfit_and_gradient(pb, m0, bfr, bs, bq, rec, bd)
                e1.record(stream)
                torch.cuda.synchronize()
                t64.append(e0.elapsed_time(e1))
            tm = float(np.median(t64))
            rate = bunits / (tm / 1e3)
            out["fp64_per_source"] = dict(
                value=round(rate, 4), unit=UNIT, ms_per_call=round(tm, 1), calls=len(t64),
                ms_all=[round(t, 1) for t in t64], pairs_per_call=bunits,
                speedup_of_value=round(value / rate, 2),
                what=("FP64 FGMRES + the same preconditioner and tolerance, one right-hand side at a time; median "
                      "of the timed calls" + (f"; each call = the step's {wl.freqs_hz[kf]:.3f} Hz pair" if big else
                                               "; each call = all pairs of the step")))
            pb.close()
            del pb
            torch.cuda.empty_cache()
        # end to end through the public API with host buffers
        hm = torch.as_tensor(wl.m0.ravel(), dtype=torch.float64).pin_memory()
        hd = d_obs.cpu().pin_memory()
        hdm = dmv.cpu().pin_memory() if dmv is not None else None
        hs, hq, hr = src.cpu().pin_memory(), Q.cpu().pin_memory(), rec.cpu().pin_memory()
        e2e_t = []
        for i in range(max(1, args.e2e_steps) + 1):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dm, dd = hm.to(dev, non_blocking=True), hd.to(dev, non_blocking=True)
            ddm = hdm.to(dev, non_blocking=True) if hdm is not None else None
            ds, dq, dr = hs.to(dev, non_blocking=True), hq.to(dev, non_blocking=True), hr.to(dev, non_blocking=True)
            f, g, _ = step(reduce=False, m=dm, s_=ds, q_=dq, r_=dr, d_=dd, dm_=ddm)
            fh, gh = (f.cpu() if f is not None else torch.zeros(0)), g.cpu()
            e1.record(stream)
            torch.cuda.synchronize()
            if i > 0:
                e2e_t.append(e0.elapsed_time(e1))
        h2d = sum(t.numel() * t.element_size() for t in (hm, hd, hs, hq, hr)) + \
            (hdm.numel() * hdm.element_size() if hdm is not None else 0)
        d2h = fh.numel() * 8 + gh.numel() * 8
        out["e2e"] = dict(value=round(units / (np.mean(e2e_t) / 1e3), 4), unit=UNIT, h2d_bytes_per_step=int(h2d),
                          d2h_bytes_per_step=int(d2h), steps=len(e2e_t))
        if cpu is not None:
            out["cpu_baseline"] = cpu
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
