"""Count the oracle's restarted-GMRES iterations for forward and adjoint
solves of a workload, and store them beside the oracle.

The CPU baseline of the benchmark times a bounded number of oracle GMRES
iterations on the full-size operator and scales by these counts to the cost of
one (source, frequency) misfit+gradient evaluation.  Only oracle/ and the
input generators are used.

    python oracle/measure_gmres_iterations.py [n=64] [restart=60] [tol=1e-10]
        the 3D layered workload at n^3, its one frequency and first source
    python oracle/measure_gmres_iterations.py multifreq [n=32] [restart=60] [tol=1e-9]
        an n^3 crop of the multi-frequency workload (the 192^3 recipe at the
        same spacing, layers and frequencies), the source nearest the centre,
        every frequency (one spawned process per frequency)
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import helmholtz as O  # noqa: E402
from paper_1703_09268_gb300 import synth  # noqa: E402


def main(n=64, restart=60, tol=1e-10, levels=2):
    wl = synth.workload_3d_layered(n=n, h=25.0 * 64 / n)
    g = O.make_grid(3, wl.n, wl.h, wl.npml, wl.v_ref, levels=levels)
    om = 2 * np.pi * wl.freqs_hz[0]
    H = O.helmholtz_matrix(g, O.extend(g, wl.m0), om)
    q = O.source_fields(g, wl.src_idx, wl.Q)[0]
    t0 = time.time()
    u, it_f, rel_f = O.gmres(H, q, tol=tol, restart=restart)
    t1 = time.time()
    _, d = O.forward(g, wl.m_true, wl.freqs_hz, wl.src_idx[:1], wl.Q[:1, :1], wl.rec_idx, solver="gmres",
                     tol=tol, restart=restart)
    r = O.sample_receivers(g, u, wl.rec_idx) - d[0, 0]
    b = -O.spread_receivers(g, r, wl.rec_idx)
    t2 = time.time()
    _, it_a, rel_a = O.gmres(H.conj().T.tocsr(), b, tol=tol, restart=restart)
    t3 = time.time()
    out = dict(workload=wl.name, grid=list(g.N), restart=restart, tol=tol, levels_padding=levels,
               forward_iterations=it_f, adjoint_iterations=it_a, forward_rel=rel_f, adjoint_rel=rel_a,
               forward_seconds=t1 - t0, adjoint_seconds=t3 - t2, cores=os.cpu_count())
    path = os.path.join(ROOT, "oracle", "data", f"gmres_iterations_3d_layered_{n}.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out))


def multifreq_workload(n):
    return synth.workload_3d_multifreq(n=n)


def _one_frequency(args):
    n, k, restart, tol, levels = args
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    wl = multifreq_workload(n)
    s = synth.centre_source(wl)
    g = O.make_grid(3, wl.n, wl.h, wl.npml, wl.v_ref, levels=levels)
    om = 2 * np.pi * wl.freqs_hz[k]
    src, Q = synth.source_subset(wl, [s])
    q = O.source_fields(g, src, Q)[0]
    Ht = O.helmholtz_matrix(g, O.extend(g, wl.m_true), om)
    ut, _, _ = O.gmres(Ht, q, tol=tol, restart=restart)
    H = O.helmholtz_matrix(g, O.extend(g, wl.m0), om)
    t0 = time.time()
    u, it_f, rel_f = O.gmres(H, q, tol=tol, restart=restart)
    t1 = time.time()
    r = O.sample_receivers(g, u, wl.rec_idx) - O.sample_receivers(g, ut, wl.rec_idx)
    b = -O.spread_receivers(g, r, wl.rec_idx)
    t2 = time.time()
    _, it_a, rel_a = O.gmres(H.conj().T.tocsr(), b, tol=tol, restart=restart)
    t3 = time.time()
    return dict(freq_hz=float(wl.freqs_hz[k]), forward_iterations=it_f, adjoint_iterations=it_a,
                forward_rel=rel_f, adjoint_rel=rel_a, forward_seconds=t1 - t0, adjoint_seconds=t3 - t2)


def main_multifreq(n=32, restart=60, tol=1e-9, levels=2):
    wl = multifreq_workload(n)
    g = O.make_grid(3, wl.n, wl.h, wl.npml, wl.v_ref, levels=levels)
    nf = len(wl.freqs_hz)
    with mp.get_context("spawn").Pool(min(nf, os.cpu_count() or 1)) as pool:
        per = pool.map(_one_frequency, [(n, k, restart, tol, levels) for k in range(nf)])
    out = dict(workload=wl.name, grid=list(g.N), restart=restart, tol=tol, levels_padding=levels,
               source=synth.centre_source(wl), per_frequency=per,
               iterations_per_pair=float(np.mean([p["forward_iterations"] + p["adjoint_iterations"] for p in per])),
               cores=os.cpu_count())
    path = os.path.join(ROOT, "oracle", "data", f"gmres_iterations_3d_multifreq_{n}.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    a = sys.argv[1:]
    if a and a[0] == "multifreq":
        a = a[1:]
        main_multifreq(n=int(a[0]) if a else 32, restart=int(a[1]) if len(a) > 1 else 60,
                       tol=float(a[2]) if len(a) > 2 else 1e-9)
    else:
        main(n=int(a[0]) if a else 64, restart=int(a[1]) if len(a) > 1 else 60,
             tol=float(a[2]) if len(a) > 2 else 1e-10)
