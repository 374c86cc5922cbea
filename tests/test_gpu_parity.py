"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.

Tolerances (relative L2):
  * operator apply, FP64: 1e-13 (same formula, different rounding order);
  * operator apply, complex64: 2e-6 (single-precision coefficients and sums);
  * FP64 solves to residual 5e-14 vs the oracle's direct solve: 1e-10;
  * complex64 inner solves under FP64 refinement to residual 1e-11: 1e-8.
These are the tolerances of the method's statement (1e-10 FP64, 1e-8 mixed).
"""
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


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ---------------------------------------------------------------------------
# Operator
# ---------------------------------------------------------------------------

APPLY_CASES = [
    # dim, n, npml, levels (ragged against the 32x4 thread block and the 16-plane z run)
    (3, (19, 13, 23), (5, 4, 6), 1),
    (3, (40, 33, 35), (6, 6, 6), 2),
    (2, (37, 1, 29), (7, 0, 9), 1),
    (2, (101, 1, 101), (20, 0, 20), 2),
]


@pytest.mark.parametrize("dim,n,npml,levels", APPLY_CASES)
@pytest.mark.parametrize("adjoint", [False, True])
def test_apply_matches_oracle(helm, dim, n, npml, levels, adjoint):
    h, f, vref = 20.0, 6.0, 3000.0
    rng = np.random.default_rng(7)
    g = O.make_grid(dim, n, h, npml, vref, levels=levels)
    mp = 1 / rng.uniform(1500, 4500, size=g.phys_shape) ** 2
    H = O.helmholtz_matrix(g, O.extend(g, mp), 2 * np.pi * f)
    if adjoint:
        H = H.conj().T.tocsr()
    nrhs = 3
    x = rng.standard_normal((nrhs, g.size)) + 1j * rng.standard_normal((nrhs, g.size))
    ref = np.stack([H @ x[i] for i in range(nrhs)])
    plan = helm.Plan(helm.make_grid(dim, n, h, npml, vref, levels=levels),
                     helm.default_opts(precond=helm.PRECOND_MLGMRES if levels > 1 else helm.PRECOND_NONE),
                     device=DEV)
    assert plan.n_comp == g.size
    y64 = helm.helm_apply(plan, T(mp.ravel(), torch.float64), f, T(x, torch.complex128), adjoint=adjoint)
    y32 = helm.helm_apply(plan, T(mp.ravel(), torch.float64), f, T(x, torch.complex64), adjoint=adjoint)
    torch.cuda.synchronize()
    assert rel(y64.cpu().numpy(), ref) < 1e-13
    assert rel(y32.cpu().numpy(), ref) < 2e-6


def test_adjoint_identity_on_gpu(helm):
    """<H x, y> = <x, H^H y> with both sides from the GPU kernels (Sec. 5.1)."""
    n, npml, h = (30, 28, 26), (8, 8, 8), 25.0
    rng = np.random.default_rng(3)
    plan = helm.Plan(helm.make_grid(3, n, h, npml, 4000.0), helm.default_opts(precond=0), device=DEV)
    mp = 1 / rng.uniform(1500, 4500, size=plan.n_phys) ** 2
    x = rng.standard_normal((1, plan.n_comp)) + 1j * rng.standard_normal((1, plan.n_comp))
    y = rng.standard_normal((1, plan.n_comp)) + 1j * rng.standard_normal((1, plan.n_comp))
    m = T(mp, torch.float64)
    Hx = helm.helm_apply(plan, m, 5.0, T(x, torch.complex128)).cpu().numpy()
    HHy = helm.helm_apply(plan, m, 5.0, T(y, torch.complex128), adjoint=True).cpu().numpy()
    lhs, rhs = np.vdot(y, Hx), np.vdot(HHy, x)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


# ---------------------------------------------------------------------------
# Solves, misfit and gradient: 2D workload (101 x 101, 20-cell layer, 5 Hz)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def wl2d():
    wl = synth.workload_2d()
    g = O.make_grid(2, wl.n, wl.h, wl.npml, wl.v_ref, levels=2)
    _, d_obs = O.forward(g, wl.m_true, wl.freqs_hz, wl.src_idx, wl.Q, wl.rec_idx)
    f, gr, U, V = O.misfit_and_gradient(g, wl.m0, wl.freqs_hz, wl.src_idx, wl.Q, wl.rec_idx, d_obs,
                                        return_fields=True)
    return wl, g, d_obs, f, gr, U, V


OPTS = {
    # FP64 solves stop at 5e-14: the residual floor of the 2D problem is ~3e-14
    "fp64-mlgmres": dict(precision=0, precond=2, tol=5e-14),
    "fp64-none": dict(precision=0, precond=0, k_inner=30, tol=5e-14, max_cycles=2000),
    "fp64-jacobi": dict(precision=0, precond=1, k_inner=20, tol=5e-14, max_cycles=2000, jacobi_sweeps=2),
    "mixed-mlgmres": dict(precision=1, precond=2, tol=1e-11),
    "mixed-mlgmres-arnoldi-smoother": dict(precision=1, precond=2, tol=1e-11, sstep=0, reorth=0),
    "fp64-mlgmres-arnoldi-smoother": dict(precision=0, precond=2, tol=5e-14, sstep=0),
    "mixed-none": dict(precision=1, precond=0, k_inner=30, tol=1e-11, max_cycles=400),
}


@pytest.mark.parametrize("name", list(OPTS))
def test_2d_misfit_gradient_matches_oracle(helm, wl2d, name):
    wl, g, d_obs, f_ref, g_ref, U_ref, V_ref = wl2d
    o = helm.default_opts(**OPTS[name])
    plan = helm.Plan(helm.make_grid(2, wl.n, wl.h, wl.npml, wl.v_ref, levels=2), o, device=DEV)
    f, gr, rep = helm.misfit_and_gradient(plan, T(wl.m0.ravel(), torch.float64), wl.freqs_hz,
                                          T(wl.src_idx, torch.int32), T(wl.Q, torch.complex128),
                                          T(wl.rec_idx, torch.int32), T(d_obs, torch.complex128))
    tol = 1e-10 if OPTS[name]["precision"] == 0 else 1e-8
    assert all(r["status"] == 0 for r in rep), rep
    assert abs(f.item() - f_ref) <= tol * abs(f_ref)
    assert rel(gr.cpu().numpy(), g_ref) <= tol


@pytest.mark.parametrize("name", ["fp64-mlgmres", "mixed-mlgmres"])
def test_2d_forward_and_adjoint_fields(helm, wl2d, name):
    wl, g, d_obs, f_ref, g_ref, U_ref, V_ref = wl2d
    o = helm.default_opts(**OPTS[name])
    plan = helm.Plan(helm.make_grid(2, wl.n, wl.h, wl.npml, wl.v_ref, levels=2), o, device=DEV)
    m0 = T(wl.m0.ravel(), torch.float64)
    U, D, rep = helm.helm_forward(plan, m0, wl.freqs_hz, T(wl.src_idx, torch.int32), T(wl.Q, torch.complex128),
                                  T(wl.rec_idx, torch.int32))
    tol = 1e-10 if OPTS[name]["precision"] == 0 else 1e-8
    assert rel(U.cpu().numpy(), U_ref) <= tol
    D_ref = O.sample_receivers(g, U_ref, wl.rec_idx)
    assert rel(D.cpu().numpy(), D_ref) <= tol
    # adjoint solve of the data residual reproduces -V (helm_adjoint has no minus sign)
    R = D_ref - d_obs
    V, rep = helm.helm_adjoint(plan, m0, wl.freqs_hz, T(wl.rec_idx, torch.int32), T(R, torch.complex128))
    assert rel(-V.cpu().numpy(), V_ref) <= tol


# ---------------------------------------------------------------------------
# 3D: small grid with the oracle's direct solve; several frequencies, a mask,
# a wavelet, ragged batching
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def wl3d():
    rng = np.random.default_rng(21)
    n, h = (17, 14, 15), 50.0
    g = O.make_grid(3, n, h, (6, 6, 6), 4500.0, levels=2)
    v = synth.layered_velocity(rng, n, nlayers=5, smooth=1.5)
    mt = synth.slowness2(v)
    m0 = synth.slowness2(synth._gaussian_smooth(v, 4.0))
    nodes = [(3, 3, 2), (12, 4, 2), (7, 10, 2), (13, 11, 2), (8, 7, 2)]
    src, Q = synth.point_sources(n, nodes)
    Q[0, 1] = 0.3 - 0.2j  # source 1 also fires at location 0
    rec = synth.surface_receivers(n, 0)
    freqs = np.array([2.5, 3.5])
    wav = np.array([1.0 + 0.5j, 0.8 - 0.1j])
    _, d = O.forward(g, mt, freqs, src, Q, rec, wavelet=wav)
    mask = np.ones((2, 5), dtype=np.uint8)
    mask[0, 2] = 0
    mask[1, 4] = 0
    f, gr, U, V = O.misfit_and_gradient(g, m0, freqs, src, Q, rec, d, wavelet=wav, mask=mask,
                                        return_fields=True)
    return dict(g=g, n=n, h=h, m0=m0, src=src, Q=Q, rec=rec, freqs=freqs, wav=wav, d=d, mask=mask, f=f,
                gr=gr, U=U, V=V)


@pytest.mark.parametrize("name,extra", [("fp64-mlgmres", {}), ("mixed-mlgmres", {}),
                                        ("mixed-mlgmres", {"max_batch": 3}), ("fp64-none", {"max_batch": 4})])
def test_3d_misfit_gradient_matches_oracle(helm, wl3d, name, extra):
    w = wl3d
    o = helm.default_opts(**OPTS[name], **extra)
    plan = helm.Plan(helm.make_grid(3, w["n"], w["h"], (6, 6, 6), 4500.0, levels=2), o, device=DEV)
    f, gr, rep = helm.misfit_and_gradient(plan, T(w["m0"].ravel(), torch.float64), w["freqs"],
                                          T(w["src"], torch.int32), T(w["Q"], torch.complex128),
                                          T(w["rec"], torch.int32), T(w["d"], torch.complex128),
                                          wavelet=T(w["wav"], torch.complex128), mask=T(w["mask"], torch.uint8))
    tol = 1e-10 if OPTS[name]["precision"] == 0 else 1e-8
    assert abs(f.item() - w["f"]) <= tol * abs(w["f"])
    assert rel(gr.cpu().numpy(), w["gr"]) <= tol
    # masked-out pairs report nothing done
    assert rep[2]["iters"] == 0 and rep[2 + 5 * 0]["refinements"] == 0


def test_3d_forward_with_wavelet(helm, wl3d):
    w = wl3d
    o = helm.default_opts(**OPTS["mixed-mlgmres"], max_batch=4)
    plan = helm.Plan(helm.make_grid(3, w["n"], w["h"], (6, 6, 6), 4500.0, levels=2), o, device=DEV)
    g = w["g"]
    U_ref, D_ref = O.forward(g, w["m0"], w["freqs"], w["src"], w["Q"], w["rec"], wavelet=w["wav"])
    U, D, rep = helm.helm_forward(plan, T(w["m0"].ravel(), torch.float64), w["freqs"], T(w["src"], torch.int32),
                                  T(w["Q"], torch.complex128), T(w["rec"], torch.int32),
                                  wavelet=T(w["wav"], torch.complex128))
    assert rel(U.cpu().numpy(), U_ref) <= 1e-8
    assert rel(D.cpu().numpy(), D_ref) <= 1e-8
    assert all(r["rel_resid"] <= 1e-11 for r in rep)


def test_invalid_receiver_index_is_rejected(helm, wl3d):
    w = wl3d
    plan = helm.Plan(helm.make_grid(3, w["n"], w["h"], (6, 6, 6), 4500.0, levels=2), helm.default_opts(),
                     device=DEV)
    bad = w["rec"].copy()
    bad[5] = plan.n_phys  # one past the end
    with pytest.raises(helm.HelmError) as e:
        helm.helm_forward(plan, T(w["m0"].ravel(), torch.float64), w["freqs"], T(w["src"], torch.int32),
                          T(w["Q"], torch.complex128), T(bad, torch.int32))
    assert e.value.code == helm.HELM_E_INVAL


@pytest.mark.parametrize("name", ["fp64-mlgmres", "mixed-mlgmres"])
def test_3d_forward_warm_start(helm, wl3d, name):
    """Warm starts (helm_forward's U0): a guess that already solves the system
    to the tolerance takes no iteration and comes back unchanged; a guess
    whose residual is a small fraction of ||q|| converges to the oracle's
    fields in fewer iterations than a cold start; U0 may be the output array
    itself."""
    w = wl3d
    o = helm.default_opts(**OPTS[name], max_batch=4)
    plan = helm.Plan(helm.make_grid(3, w["n"], w["h"], (6, 6, 6), 4500.0, levels=2), o, device=DEV)
    args = (T(w["m0"].ravel(), torch.float64), w["freqs"], T(w["src"], torch.int32), T(w["Q"], torch.complex128),
            T(w["rec"], torch.int32))
    kw = dict(wavelet=T(w["wav"], torch.complex128))
    U_ref, _ = O.forward(w["g"], w["m0"], w["freqs"], w["src"], w["Q"], w["rec"], wavelet=w["wav"])
    tol = 1e-10 if OPTS[name]["precision"] == 0 else 1e-8
    U, D, rep = helm.helm_forward(plan, *args, **kw)
    cold = [r["iters"] for r in rep]
    # converged guess: zero iterations, the guess itself returned
    U2, D2, rep2 = helm.helm_forward(plan, *args, U0=U.clone(), **kw)
    assert all(r["iters"] == 0 for r in rep2), rep2
    assert torch.equal(U2, U) and torch.equal(D2, D)
    assert all(r["status"] == 0 and r["rel_resid"] <= o.tol for r in rep2)
    # a guess off by a relative 2e-4 (its residual is 2e-4 of ||q||): fewer iterations, the oracle's fields
    U0 = U * (1 + 2e-4)
    U3, _, rep3 = helm.helm_forward(plan, *args, U0=U0, **kw)
    assert rel(U3.cpu().numpy(), U_ref) <= tol
    assert sum(r["iters"] for r in rep3) < sum(cold), ([r["iters"] for r in rep3], cold)
    # in place: U0 is the output array
    U4 = U0.clone()
    code = helm.lib().helm_forward(plan._h, helm._ptr(args[0]), helm._freqs(w["freqs"]), len(w["freqs"]),
                                   helm._ptr(args[2]), args[2].numel(), helm._ptr(args[3]), args[3].shape[1],
                                   helm._ptr(kw["wavelet"]), helm._ptr(args[4]), args[4].numel(), helm._ptr(U4),
                                   helm._ptr(U4), None, *plan.workspace(plan.workspace_size(
                                       helm.CALL_FORWARD, len(w["freqs"]), args[3].shape[1], args[4].numel())),
                                   helm._reports(len(w["freqs"]) * args[3].shape[1]), helm._stream(DEV))
    assert code == helm.HELM_OK
    torch.cuda.synchronize()
    assert rel(U4.cpu().numpy(), U_ref) <= tol
