"""Full-size workloads on the GPU.

The oracle cannot solve these sizes in test time, so every right-hand side is
checked by an independent residual ||q - H u|| / ||q|| computed on the CPU
with the oracle's own sparse operator and sources, and the mixed-precision
fields are compared with the FP64 fields of the same GPU path.  On the 64^3
layered workload two sources also come with the oracle's own solution
(restarted GMRES to a relative residual below 1e-14, stored by
tests/golden/make_layered64.py): receiver data and 4096 seeded field entries
are compared element by element.
"""
import os

import numpy as np
import pytest
import torch

from oracle import helmholtz as O
from paper_1703_09268_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def helm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1703_09268_gb300 import helm as H
    return H


def T(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)


def oracle_residuals(wl, g, U, m):
    H = O.helmholtz_matrix(g, O.extend(g, m), 2 * np.pi * wl.freqs_hz[0])
    q = O.source_fields(g, wl.src_idx, wl.Q)
    return np.array([np.linalg.norm(q[s] - H @ U[0, s]) / np.linalg.norm(q[s]) for s in range(q.shape[0])])


def test_layered_64cubed_all_sources(helm):
    """64^3 layered model (85^3 with layers), 16 sources, 4 Hz: FP64 to 1e-10
    and mixed precision to 1e-10; independent oracle residuals; mixed vs FP64."""
    wl = synth.workload_3d_layered()
    g = O.make_grid(3, wl.n, wl.h, wl.npml, wl.v_ref, levels=2)
    grid = helm.make_grid(3, wl.n, wl.h, wl.npml, wl.v_ref, levels=2)
    args = (T(wl.m0.ravel(), torch.float64), wl.freqs_hz, T(wl.src_idx, torch.int32), T(wl.Q, torch.complex128),
            T(wl.rec_idx, torch.int32))
    p64 = helm.Plan(grid, helm.default_opts(precision=helm.FP64, tol=1e-10), device=DEV)
    U64, D64, rep64 = helm.helm_forward(p64, *args)
    pmx = helm.Plan(grid, helm.default_opts(precision=helm.MIXED, tol=1e-10), device=DEV)
    Umx, Dmx, repmx = helm.helm_forward(pmx, *args)
    U64, Umx = U64.cpu().numpy(), Umx.cpu().numpy()
    r64 = oracle_residuals(wl, g, U64, wl.m0)
    rmx = oracle_residuals(wl, g, Umx, wl.m0)
    assert np.all(r64 <= 1.05e-10), r64
    assert np.all(rmx <= 1.05e-10), rmx
    # the GPU's own FP64 residual report agrees with the oracle's
    assert np.allclose([r["rel_resid"] for r in rep64], r64, rtol=1e-3, atol=1e-14)
    for s in range(wl.nsrc):
        e = np.linalg.norm(Umx[0, s] - U64[0, s]) / np.linalg.norm(U64[0, s])
        assert e <= 1e-8, (s, e)
    d = np.linalg.norm(Dmx.cpu().numpy() - D64.cpu().numpy()) / np.linalg.norm(D64.cpu().numpy())
    assert d <= 1e-8


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("name,prec,tol,bar", [("fp64", 0, 1e-13, 1e-10), ("mixed", 1, 1e-11, 1e-8)])
def test_layered_64cubed_matches_oracle_fields(helm, name, prec, tol, bar):
    """The sampled sources' receiver data and field samples against the oracle's
    GMRES solution: relative L2 error <= 1e-10 (FP64 solves to 1e-13) and
    <= 1e-8 (complex64 inner solves refined in FP64 to 1e-11)."""
    gold = np.load(os.path.join(GOLDEN, "layered64_fields.npz"))
    assert np.all(gold["rel_resid"] < 1e-14)
    wl = synth.workload_3d_layered()
    srcs = [int(s) for s in gold["sources"]]
    grid = helm.make_grid(3, wl.n, wl.h, wl.npml, wl.v_ref, levels=2)
    plan = helm.Plan(grid, helm.default_opts(precision=prec, tol=tol), device=DEV)
    src, Q = synth.source_subset(wl, srcs)
    U, D, rep = helm.helm_forward(plan, T(wl.m0.ravel(), torch.float64), wl.freqs_hz, T(src, torch.int32),
                                  T(Q, torch.complex128), T(wl.rec_idx, torch.int32))
    U, D = U.cpu().numpy()[0], D.cpu().numpy()[0]
    idx = gold["idx"]
    for k, s in enumerate(srcs):
        eu = np.linalg.norm(U[k, idx] - gold["U"][k]) / np.linalg.norm(gold["U"][k])
        ed = np.linalg.norm(D[k] - gold["D"][k]) / np.linalg.norm(gold["D"][k])
        print(name, "source", s, "field-sample error", eu, "receiver-data error", ed, "residual", rep[k]["rel_resid"])
        assert eu <= bar and ed <= bar, (s, eu, ed)


def test_precision_workload_256cubed(helm):
    """256^3, h = 20 m, 12-cell layers (280^3 computational, 22 M nodes), layered
    model with 20 inclusions of +-400 m/s, 6 Hz, 32 sources: complex64 inner
    solves under FP64 refinement to relative residual 1e-8.  Every right-hand
    side reports its FP64 residual; two sampled sources are re-checked with the
    oracle's sparse operator on the CPU."""
    wl = synth.workload_3d_inclusions()
    grid = helm.make_grid(3, wl.n, wl.h, wl.npml, wl.v_ref, levels=2)
    plan = helm.Plan(grid, helm.default_opts(precision=helm.MIXED, tol=1e-8, max_batch=16), device=DEV)
    U, D, rep = helm.helm_forward(plan, T(wl.m0.ravel(), torch.float64), wl.freqs_hz, T(wl.src_idx, torch.int32),
                                  T(wl.Q, torch.complex128), T(wl.rec_idx, torch.int32))
    res = np.array([r["rel_resid"] for r in rep])
    print("per-RHS FP64 relative residuals:", res.tolist(), "outer iterations:", [r["iters"] for r in rep])
    assert np.all(res <= 1e-8), res
    g = O.make_grid(3, wl.n, wl.h, wl.npml, wl.v_ref, levels=2)
    H = O.helmholtz_matrix(g, O.extend(g, wl.m0), 2 * np.pi * wl.freqs_hz[0])
    q = O.source_fields(g, wl.src_idx[[0, 17]], wl.Q[np.ix_([0, 17], [0, 17])])
    for k, s in enumerate([0, 17]):
        u = U[0, s].cpu().numpy()
        r = np.linalg.norm(q[k] - H @ u) / np.linalg.norm(q[k])
        assert r <= 1.05e-8 and abs(r - res[s]) <= 1e-3 * res[s] + 1e-15, (s, r, res[s])
    # error per right-hand side against the FP64 GPU path (FP64 solves to 1e-11) for the two sampled
    # sources: reported for the refinement to 1e-8 above, and bounded by 1e-8 when the refinement
    # goes on to 1e-10
    sub = [0, 17]
    src2, Q2 = synth.source_subset(wl, sub)
    args2 = (T(wl.m0.ravel(), torch.float64), wl.freqs_hz, T(src2, torch.int32), T(Q2, torch.complex128),
             T(wl.rec_idx, torch.int32))
    p64 = helm.Plan(grid, helm.default_opts(precision=helm.FP64, tol=1e-11), device=DEV)
    U64, _, _ = helm.helm_forward(p64, *args2, want_data=False)
    del p64
    pm10 = helm.Plan(grid, helm.default_opts(precision=helm.MIXED, tol=1e-10), device=DEV)
    U10, _, rep10 = helm.helm_forward(pm10, *args2, want_data=False)
    for k, s in enumerate(sub):
        ref = U64[0, k]
        e8 = ((U[0, s] - ref).norm() / ref.norm()).item()
        e10 = ((U10[0, k] - ref).norm() / ref.norm()).item()
        print(f"source {s}: error vs FP64 {e8:.3e} (mixed, residual {res[s]:.2e}), "
              f"{e10:.3e} (mixed, residual {rep10[k]['rel_resid']:.2e})")
        assert e10 <= 1e-8, (s, e10)
        assert e8 <= 1e3 * res[s], (s, e8)  # the error stays within a modest multiple of the residual
