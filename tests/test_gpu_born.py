"""GPU parity of the linearised calls (Appendix A, Table derivstuff) with the
oracle: J dm (helm_born), J^T dD (helm_born_adjoint) and the Gauss-Newton
product J^T J dm (helm_gn_hessvec), on a 3D grid with several frequencies, a
wavelet, a mask and ragged batching, and on the 2D workload.

Tolerances (relative L2): FP64 solves to residual 5e-14 vs the oracle's direct
solves: 1e-10; complex64 inner solves refined in FP64 to 1e-11: 1e-8 (the
tolerances of the method's statement, as for the misfit gradient)."""
import numpy as np
import pytest
import torch

from oracle import helmholtz as O
from paper_1703_09268_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]

DEV = torch.device("cuda:0")
OPTS = {"fp64": dict(precision=0, precond=2, tol=5e-14), "mixed": dict(precision=1, precond=2, tol=1e-11)}


@pytest.fixture(scope="module")
def helm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1703_09268_gb300 import helm as H
    return H


def T(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)


def rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def p3d():
    rng = np.random.default_rng(41)
    n, h = (17, 14, 15), 50.0
    g = O.make_grid(3, n, h, (6, 6, 6), 4500.0, levels=2)
    v = synth.layered_velocity(rng, n, nlayers=5, smooth=1.5)
    m = synth.slowness2(synth._gaussian_smooth(v, 4.0))
    nodes = [(3, 3, 2), (12, 4, 2), (7, 10, 2), (13, 11, 2), (8, 7, 2)]
    src, Q = synth.point_sources(n, nodes)
    rec = synth.surface_receivers(n, 0)
    freqs = np.array([2.5, 3.5])
    wav = np.array([1.0 + 0.5j, 0.8 - 0.1j])
    mask = np.ones((2, 5), dtype=np.uint8)
    mask[0, 2] = 0
    mask[1, 4] = 0
    dm = rng.standard_normal(g.n_phys) * 1e-8
    dD = rng.standard_normal((2, 5, len(rec))) + 1j * rng.standard_normal((2, 5, len(rec)))
    J = O.born(g, m, freqs, src, Q, rec, dm, wav, mask)
    JT = O.born_adjoint(g, m, freqs, src, Q, rec, dD, wav, mask).ravel()
    GN = O.gauss_newton_hessvec(g, m, freqs, src, Q, rec, dm, wav, mask).ravel()
    return dict(g=g, n=n, h=h, m=m, src=src, Q=Q, rec=rec, freqs=freqs, wav=wav, mask=mask, dm=dm, dD=dD,
                J=J, JT=JT, GN=GN)


def _plan(helm, p, name, **extra):
    return helm.Plan(helm.make_grid(3, p["n"], p["h"], (6, 6, 6), 4500.0, levels=2),
                     helm.default_opts(**OPTS[name], **extra), device=DEV)


def _args(p):
    return (T(p["m"].ravel(), torch.float64), p["freqs"], T(p["src"], torch.int32), T(p["Q"], torch.complex128),
            T(p["rec"], torch.int32))


@pytest.mark.parametrize("name,extra", [("fp64", {}), ("mixed", {}), ("mixed", {"max_batch": 3})])
def test_born_3d(helm, p3d, name, extra):
    p = p3d
    plan = _plan(helm, p, name, **extra)
    tol = 1e-10 if name == "fp64" else 1e-8
    kw = dict(wavelet=T(p["wav"], torch.complex128), mask=T(p["mask"], torch.uint8))
    J, rep = helm.helm_born(plan, *_args(p), T(p["dm"], torch.float64), **kw)
    assert rel(J.cpu().numpy(), p["J"]) <= tol
    assert np.all(J.cpu().numpy()[0, 2] == 0) and np.all(J.cpu().numpy()[1, 4] == 0)
    assert rep[2]["iters"] == 0 and rep[0]["iters"] > 0
    JT, _ = helm.helm_born_adjoint(plan, *_args(p), T(p["dD"], torch.complex128), **kw)
    assert rel(JT.cpu().numpy(), p["JT"]) <= tol
    GN, _ = helm.helm_gn_hessvec(plan, *_args(p), T(p["dm"], torch.float64), **kw)
    assert rel(GN.cpu().numpy(), p["GN"]) <= tol
    # the adjoint identity from the GPU's own outputs
    lhs = float(np.real(np.vdot(J.cpu().numpy(), p["dD"] * p["mask"][..., None])))
    rhs = float(np.dot(p["dm"], JT.cpu().numpy()))
    assert abs(lhs - rhs) <= 10 * tol * abs(lhs)


def test_born_adjoint_of_residual_is_the_gradient(helm, p3d):
    p = p3d
    plan = _plan(helm, p, "fp64")
    rng = np.random.default_rng(42)
    _, D = O.forward(p["g"], p["m"], p["freqs"], p["src"], p["Q"], p["rec"], p["wav"], want_fields=False)
    d_obs = D + 0.05 * (rng.standard_normal(D.shape) + 1j * rng.standard_normal(D.shape))
    wav = T(p["wav"], torch.complex128)
    f, g, _ = helm.misfit_and_gradient(plan, *_args(p), T(d_obs, torch.complex128), wavelet=wav)
    JT, _ = helm.helm_born_adjoint(plan, *_args(p), T(D - d_obs, torch.complex128), wavelet=wav)
    assert rel(JT.cpu().numpy(), g.cpu().numpy()) <= 1e-10


def test_born_2d_workload(helm):
    wl = synth.workload_2d()
    g = O.make_grid(2, wl.n, wl.h, wl.npml, wl.v_ref, levels=2)
    rng = np.random.default_rng(43)
    dm = rng.standard_normal(g.n_phys) * 1e-9
    ref = O.gauss_newton_hessvec(g, wl.m0, wl.freqs_hz, wl.src_idx, wl.Q, wl.rec_idx, dm).ravel()
    J_ref = O.born(g, wl.m0, wl.freqs_hz, wl.src_idx, wl.Q, wl.rec_idx, dm)
    for name in ("fp64", "mixed"):
        plan = helm.Plan(helm.make_grid(2, wl.n, wl.h, wl.npml, wl.v_ref, levels=2), helm.default_opts(**OPTS[name]),
                         device=DEV)
        args = (T(wl.m0.ravel(), torch.float64), wl.freqs_hz, T(wl.src_idx, torch.int32),
                T(wl.Q, torch.complex128), T(wl.rec_idx, torch.int32))
        tol = 1e-10 if name == "fp64" else 1e-8
        J, _ = helm.helm_born(plan, *args, T(dm, torch.float64))
        assert rel(J.cpu().numpy(), J_ref) <= tol
        GN, rep = helm.helm_gn_hessvec(plan, *args, T(dm, torch.float64))
        assert rel(GN.cpu().numpy(), ref) <= tol
        assert all(r["status"] == 0 for r in rep)


@pytest.mark.parametrize("name,extra", [("fp64", {}), ("mixed", {"max_batch": 3})])
def test_full_hessvec_3d(helm, p3d, name, extra):
    p = p3d
    rng = np.random.default_rng(44)
    _, D = O.forward(p["g"], p["m"], p["freqs"], p["src"], p["Q"], p["rec"], p["wav"], want_fields=False)
    d_obs = D + 0.2 * (rng.standard_normal(D.shape) + 1j * rng.standard_normal(D.shape))
    ref = O.hessvec(p["g"], p["m"], p["freqs"], p["src"], p["Q"], p["rec"], d_obs, p["dm"], p["wav"],
                    p["mask"]).ravel()
    plan = _plan(helm, p, name, **extra)
    tol = 1e-10 if name == "fp64" else 1e-8
    Hdm, rep = helm.helm_hessvec(plan, *_args(p), T(d_obs, torch.complex128), T(p["dm"], torch.float64),
                                 wavelet=T(p["wav"], torch.complex128), mask=T(p["mask"], torch.uint8))
    assert rel(Hdm.cpu().numpy(), ref) <= tol
    assert rep[2]["iters"] == 0 and all(r["status"] == 0 for r in rep)
