"""GPU parity of 2.5D modelling (Sec. 3, 2.5D) with the oracle: misfit and
gradient summed over k_y-shifted 2D solves, several frequencies, a wavelet,
and batching that splits the (frequency, source) groups across batches.
Tolerances: FP64 1e-10, mixed (complex64 inner, FP64 refinement) 1e-8."""
import numpy as np
import pytest
import torch

from oracle import helmholtz as O

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


@pytest.fixture(scope="module")
def p25():
    rng = np.random.default_rng(61)
    n, h, npml = (61, 1, 41), 20.0, (12, 0, 12)
    g = O.make_grid(2, n, h, npml, 3000.0, levels=2)
    X, Z = np.meshgrid(np.arange(n[0]), np.arange(n[2]), indexing="xy")
    v = 1800.0 + 30.0 * Z + 200.0 * np.exp(-((X - 30) ** 2 + (Z - 20) ** 2) / 50.0)
    m = (1.0 / v ** 2).ravel()
    src = np.array([2 * n[0] + 15, 2 * n[0] + 45, 2 * n[0] + 30], dtype=np.int32)
    Q = np.eye(3, dtype=np.complex128)
    rec = (np.arange(n[0]) + n[0]).astype(np.int32)
    freqs = np.array([5.0, 7.0])
    wav = np.array([1.0 - 0.2j, 0.6 + 0.4j])
    ky, ck = O.gauss_legendre_ky(1.2 * 2 * np.pi * 7.0 / 1800.0, 5, dy=15.0)
    D, _ = O.forward_25d(g, m, freqs, ky, ck, src, Q, rec, wav)
    d_obs = D * (1 + 0.1 * rng.standard_normal(D.shape))
    f, gr = O.misfit_and_gradient_25d(g, m, freqs, ky, ck, src, Q, rec, d_obs, wav)
    return dict(n=n, h=h, npml=npml, m=m, src=src, Q=Q, rec=rec, freqs=freqs, wav=wav, ky=ky, ck=ck, d=d_obs,
                f=f, g=gr.ravel())


@pytest.mark.parametrize("name,opts", [("fp64", dict(precision=0, precond=2, tol=5e-14)),
                                       ("mixed", dict(precision=1, precond=2, tol=1e-11)),
                                       ("mixed-batched", dict(precision=1, precond=2, tol=1e-11, max_batch=10))])
def test_25d_misfit_gradient(helm, p25, name, opts):
    p = p25
    plan = helm.Plan(helm.make_grid(2, p["n"], p["h"], p["npml"], 3000.0, levels=2), helm.default_opts(**opts),
                     device=DEV)
    f, g, rep = helm.misfit_and_gradient_25d(plan, T(p["m"], torch.float64), p["freqs"], p["ky"], p["ck"],
                                             T(p["src"], torch.int32), T(p["Q"], torch.complex128),
                                             T(p["rec"], torch.int32), T(p["d"], torch.complex128),
                                             wavelet=T(p["wav"], torch.complex128))
    tol = 1e-10 if name == "fp64" else 1e-8
    assert abs(f.item() - p["f"]) <= tol * abs(p["f"])
    gg = g.cpu().numpy()
    assert np.linalg.norm(gg - p["g"]) <= tol * np.linalg.norm(p["g"])
    assert len(rep) == 2 * 3 * 5 and all(r["status"] == 0 and r["iters"] > 0 for r in rep)


def test_25d_rejects_batches_smaller_than_the_quadrature(helm, p25):
    p = p25
    plan = helm.Plan(helm.make_grid(2, p["n"], p["h"], p["npml"], 3000.0, levels=2),
                     helm.default_opts(max_batch=3), device=DEV)
    with pytest.raises(helm.HelmError):
        helm.misfit_and_gradient_25d(plan, T(p["m"], torch.float64), p["freqs"], p["ky"], p["ck"],
                                     T(p["src"], torch.int32), T(p["Q"], torch.complex128),
                                     T(p["rec"], torch.int32), T(p["d"], torch.complex128))
