"""Every tile shape of the operator apply against the oracle, and the
launch-time tuner.

The complex64 apply has several tile shapes (columns per block, z-planes per
tile, register budget); every shape must give the oracle's H x and H^H x, and
all shapes must agree bit for bit (each node is computed with the same
arithmetic whatever the shape).  The residual form b - H x (reached through
damped-Jacobi sweeps of helm_precond_apply) is checked the same way.  With
tuning on, the first apply on a large grid records a shape for it."""
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
    yield H
    H.stencil_select(-1)


def T(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)


def rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# a grid above the tuning threshold (295 x 10^3 nodes, ragged in every axis) and a small 2D one
GRIDS = [(3, (61, 57, 53), (6, 5, 7), 2), (2, (45, 1, 39), (7, 0, 6), 2)]


@pytest.mark.parametrize("dim,n,npml,levels", GRIDS)
@pytest.mark.parametrize("adjoint", [False, True])
def test_every_shape_matches_oracle_and_each_other(helm, dim, n, npml, levels, adjoint):
    h, f, vref = 20.0, 6.0, 3000.0
    rng = np.random.default_rng(17)
    g = O.make_grid(dim, n, h, npml, vref, levels=levels)
    mp = 1 / rng.uniform(1500, 4500, size=g.phys_shape) ** 2
    H = O.helmholtz_matrix(g, O.extend(g, mp), 2 * np.pi * f)
    if adjoint:
        H = H.conj().T.tocsr()
    x = rng.standard_normal((3, g.size)) + 1j * rng.standard_normal((3, g.size))
    ref = np.stack([H @ xi for xi in x])
    plan = helm.Plan(helm.make_grid(dim, n, h, npml, vref, levels=levels), helm.default_opts(), device=DEV)
    m, xd = T(mp.ravel(), torch.float64), T(x, torch.complex64)
    outs = []
    try:
        for v in range(len(helm.stencil_variants())):
            helm.stencil_select(v)
            y = helm.helm_apply(plan, m, f, xd, adjoint=adjoint)
            torch.cuda.synchronize()
            outs.append(y.cpu().numpy())
            assert rel(outs[-1], ref) < 2e-6, (v, rel(outs[-1], ref))
    finally:
        helm.stencil_select(-1)
    for v, y in enumerate(outs[1:], 1):
        assert np.array_equal(y, outs[0]), v


def test_residual_form_in_jacobi_sweeps(helm):
    """Three damped-Jacobi sweeps z += w D^{-1}(b - H z) use the residual form of
    the apply: every shape gives the same z, equal to the oracle's sweeps."""
    dim, n, npml, levels = GRIDS[0]
    rng = np.random.default_rng(5)
    g = O.make_grid(dim, n, 20.0, npml, 3000.0, levels=1)
    mp = 1 / rng.uniform(1500, 4500, size=g.phys_shape) ** 2
    b = rng.standard_normal((2, g.size)) + 1j * rng.standard_normal((2, g.size))
    H = O.helmholtz_matrix(g, O.extend(g, mp), 2 * np.pi * 6.0)
    ref = np.stack([O.jacobi_precond(H, bi, 0.6, 3) for bi in b])
    plan = helm.Plan(helm.make_grid(dim, n, 20.0, npml, 3000.0, levels=1),
                     helm.default_opts(precision=helm.MIXED, precond=helm.PRECOND_JACOBI, jacobi_omega=0.6,
                                       jacobi_sweeps=3), device=DEV)
    m, bd = T(mp.ravel(), torch.float64), T(b, torch.complex64)
    outs = []
    try:
        for v in range(len(helm.stencil_variants())):
            helm.stencil_select(v)
            z = helm.helm_precond_apply(plan, m, 6.0, bd)
            torch.cuda.synchronize()
            outs.append(z.cpu().numpy())
    finally:
        helm.stencil_select(-1)
    assert rel(outs[0], ref) < 1e-5
    for v, z in enumerate(outs[1:], 1):
        assert np.array_equal(z, outs[0]), v


def test_tuner_records_a_shape_per_grid(helm):
    dim, n, npml, levels = GRIDS[0]
    plan = helm.Plan(helm.make_grid(dim, n, 20.0, npml, 3000.0, levels=levels), helm.default_opts(), device=DEV)
    helm.stencil_select(-1)
    m = torch.full((plan.n_phys,), 1 / 2500.0 ** 2, dtype=torch.float64, device=DEV)
    x = torch.randn(2, plan.n_comp, dtype=torch.complex64, device=DEV)
    y1 = helm.helm_apply(plan, m, 5.0, x)
    y2 = helm.helm_apply(plan, m, 5.0, x)
    torch.cuda.synchronize()
    tuned = helm.stencil_tuned(plan, 0)
    assert tuned is not None
    v, us = tuned
    assert 0 <= v < len(helm.stencil_variants()) and us > 0
    assert torch.equal(y1, y2)
    with pytest.raises(helm.HelmError):
        helm.stencil_select(len(helm.stencil_variants()))
