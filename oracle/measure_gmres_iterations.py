"""Count the oracle's restarted-GMRES iterations for one forward and one adjoint
solve of a workload, and store them beside the oracle.

The CPU baseline of the benchmark times a bounded number of oracle GMRES
iterations on the full-size operator and scales by these counts to the cost of
one (source, frequency) misfit+gradient evaluation.  Only oracle/ and the
input generators are used.

    python oracle/measure_gmres_iterations.py  [n=64] [restart=60] [tol=1e-10]
"""
import json
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


if __name__ == "__main__":
    a = sys.argv[1:]
    main(n=int(a[0]) if a else 64, restart=int(a[1]) if len(a) > 1 else 60,
         tol=float(a[2]) if len(a) > 2 else 1e-10)
