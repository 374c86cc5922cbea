"""Write tests/golden/crop32_gradient.json from the CPU oracle only.

The differentiation workload (layered model with inclusions, surface sources
and receivers) cropped to a 32^3 physical grid with a 6-cell layer, 4 sources
on a 2x2 surface grid and 2 frequencies (2 and 4 Hz).  Observed data are the
oracle's forward modelling in the true model; f and g are the oracle's
adjoint-state misfit and gradient (sparse LU) at the smoothed model.  The
fixture keeps f, ||g||, 512 seeded samples of g and 8 seeded random
projections <g, r_k> (crop32_gradient.json) and the whole gradient
(crop32_gradient_full.npz, compared element by element).

    python tests/golden/make_crop32.py     (about 5 minutes on one core)
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import helmholtz as O  # noqa: E402
from paper_1703_09268_gb300 import synth  # noqa: E402

SPEC = dict(n=32, h=25.0, npml=6, nsx=2, nsy=2, nfreq=2, fmin=2.0, fmax=4.0, levels=2, seed=5)


def workload():
    s = SPEC
    return synth.workload_3d_multifreq(seed=s["seed"], n=s["n"], h=s["h"], npml=s["npml"], nsx=s["nsx"],
                                       nsy=s["nsy"], nfreq=s["nfreq"], fmin=s["fmin"], fmax=s["fmax"])


def projections(n, k=8, seed=123):
    return np.random.default_rng(seed).standard_normal((k, n))


def sample_idx(n, k=512, seed=7):
    return np.sort(np.random.default_rng(seed).choice(n, size=k, replace=False))


def main():
    wl = workload()
    g = O.make_grid(3, wl.n, wl.h, wl.npml, wl.v_ref, levels=SPEC["levels"])
    _, d = O.forward(g, wl.m_true, wl.freqs_hz, wl.src_idx, wl.Q, wl.rec_idx)
    f, gr = O.misfit_and_gradient(g, wl.m0, wl.freqs_hz, wl.src_idx, wl.Q, wl.rec_idx, d)
    gr = gr.ravel()
    idx = sample_idx(gr.size)
    out = dict(spec=SPEC, f=float(f), g_norm=float(np.linalg.norm(gr)), sample_idx=idx.tolist(),
               g_samples=gr[idx].tolist(), projections=(projections(gr.size) @ gr).tolist())
    with open(os.path.join(HERE, "crop32_gradient.json"), "w") as fh:
        json.dump(out, fh)
    # the oracle's observed data, the input both sides use
    np.savez_compressed(os.path.join(HERE, "crop32_dobs.npz"), d_obs=d)
    np.savez_compressed(os.path.join(HERE, "crop32_gradient_full.npz"), g=gr, f=float(f))
    print("f", f, "|g|", out["g_norm"])


if __name__ == "__main__":
    main()
