"""Write tests/golden/layered64_fields.npz from the CPU oracle only.

The 64^3 layered workload (85^3 computational nodes with the 10-cell layers
and one padding cell, 4 Hz, receivers at every surface node) is solved for
two of its sixteen sources by the oracle's restarted GMRES (no
preconditioner, restart 60) down to a relative residual of 1e-14 in FP64.
The fixture keeps, per source: the receiver data P_r u, a seeded sample of
4096 field entries, the GMRES iteration count and the residual reached.

    python tests/golden/make_layered64.py     (two processes, ~30 minutes)
"""
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

SOURCES = (0, 9)
TOL = 1e-14
NSAMPLE = 4096


def sample_idx(size, k=NSAMPLE, seed=64):
    return np.sort(np.random.default_rng(seed).choice(size, size=k, replace=False))


def solve_one(s):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    sys.path.insert(0, ROOT)
    from oracle import helmholtz as O
    from paper_1703_09268_gb300 import synth
    wl = synth.workload_3d_layered()
    g = O.make_grid(3, wl.n, wl.h, wl.npml, wl.v_ref, levels=2)
    H = O.helmholtz_matrix(g, O.extend(g, wl.m0), 2 * np.pi * wl.freqs_hz[0])
    q = O.source_fields(g, wl.src_idx, wl.Q)[s]
    u, it, rel = O.gmres(H, q, tol=TOL, restart=60, maxiter=40000)
    true_rel = float(np.linalg.norm(q - H @ u) / np.linalg.norm(q))
    idx = sample_idx(g.size)
    return dict(s=s, it=it, rel=true_rel, D=O.sample_receivers(g, u, wl.rec_idx), idx=idx, U=u[idx])


def main():
    with mp.get_context("spawn").Pool(len(SOURCES)) as pool:
        res = pool.map(solve_one, SOURCES)
    np.savez_compressed(os.path.join(HERE, "layered64_fields.npz"), sources=np.array(SOURCES), tol=TOL,
                        iterations=np.array([r["it"] for r in res]), rel_resid=np.array([r["rel"] for r in res]),
                        D=np.stack([r["D"] for r in res]), idx=res[0]["idx"], U=np.stack([r["U"] for r in res]))
    for r in res:
        print("source", r["s"], "iterations", r["it"], "relative residual", r["rel"])


if __name__ == "__main__":
    main()
