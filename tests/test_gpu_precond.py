"""GPU parity of the preconditioners (Sec. 4) through helm_precond_apply:
one ML-GMRES V-cycle, or damped Jacobi sweeps, against the oracle's
statement of the same cycle on the same seeded inputs.

Tolerances (relative L2):
  * FP64 with Arnoldi (GMRES) smoothers: 1e-10 -- the same Krylov steps,
    rounding order differs (classical vs modified Gram-Schmidt);
  * FP64 with s-step smoothers: the same minimal-residual polynomial over the
    same Krylov space, reached through the normal equations of a monomial
    basis; with s = 3 the scaled Gram matrix stays well conditioned and the
    cycle agrees to 1e-8;
  * Jacobi, FP64: 1e-13 (a few fused multiply-adds per point);
  * complex64 cycle (mixed-precision plans): 2e-4, single-precision rounding
    carried through ~40 operator applications and the small solves.
"""
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


def rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = {
    # name: dim, n, h, npml, levels, freq
    "2d": (2, (61, 1, 57), 20.0, (12, 0, 12), 2, 5.0),
    "2d-3lev": (2, (61, 1, 57), 20.0, (12, 0, 12), 3, 5.0),
    "3d": (3, (17, 14, 15), 50.0, (6, 6, 6), 2, 3.0),
}


def _setup(case, seed, nrhs):
    dim, n, h, npml, levels, f = CASES[case]
    rng = np.random.default_rng(seed)
    g = O.make_grid(dim, n, h, npml, 3000.0, levels=levels)
    v = 1800.0 + 1500.0 * rng.random(g.n_phys)
    mp = 1.0 / v ** 2
    b = rng.standard_normal((nrhs, g.size)) + 1j * rng.standard_normal((nrhs, g.size))
    return g, mp, b, f


def _gpu(helm, case, mp, b, f, adjoint, **opts):
    dim, n, h, npml, levels, _ = CASES[case]
    o = helm.default_opts(**opts)
    plan = helm.Plan(helm.make_grid(dim, n, h, npml, 3000.0, levels=levels), o, device=DEV)
    dt = torch.complex128 if o.precision == 0 else torch.complex64
    x = torch.as_tensor(b, dtype=dt, device=DEV)
    m = torch.as_tensor(mp.ravel(), dtype=torch.float64, device=DEV)
    z = helm.helm_precond_apply(plan, m, f, x, adjoint=adjoint)
    torch.cuda.synchronize()
    return z.cpu().numpy(), o


def _oracle_vcycle(case, g, mp, f, b, o, adjoint):
    M = O.MLGmres(g, O.extend(g, mp), 2 * np.pi * f, levels=CASES[case][4], k_so=o.k_so, k_si=o.k_si,
                  k_co=o.k_co, k_ci=o.k_ci, adjoint=adjoint)
    return np.stack([M(bi) for bi in b])


@pytest.mark.parametrize("case", ["2d", "2d-3lev", "3d"])
@pytest.mark.parametrize("adjoint", [False, True])
def test_vcycle_fp64_arnoldi_smoothers(helm, case, adjoint):
    g, mp, b, f = _setup(case, 11, 3)
    z, o = _gpu(helm, case, mp, b, f, adjoint, precision=0, precond=2, sstep=0)
    ref = _oracle_vcycle(case, g, mp, f, b, o, adjoint)
    for i in range(len(b)):
        assert rel(z[i], ref[i]) <= 1e-10, (i, rel(z[i], ref[i]))


@pytest.mark.parametrize("case", ["2d", "3d"])
def test_vcycle_fp64_sstep_smoothers(helm, case):
    g, mp, b, f = _setup(case, 12, 2)
    z, o = _gpu(helm, case, mp, b, f, False, precision=0, precond=2, sstep=1, k_si=3, k_ci=3)
    ref = _oracle_vcycle(case, g, mp, f, b, o, False)
    for i in range(len(b)):
        assert rel(z[i], ref[i]) <= 1e-8, (i, rel(z[i], ref[i]))


def test_vcycle_batches_and_ragged_tail(helm):
    """Five fields through max_batch = 2 (batches of 2, 2, 1)."""
    case = "2d"
    g, mp, b, f = _setup(case, 13, 5)
    z, o = _gpu(helm, "2d", mp, b, f, False, precision=0, precond=2, sstep=0, max_batch=2)
    ref = _oracle_vcycle(case, g, mp, f, b, o, False)
    for i in range(len(b)):
        assert rel(z[i], ref[i]) <= 1e-10, (i, rel(z[i], ref[i]))


@pytest.mark.parametrize("adjoint", [False, True])
def test_vcycle_complex64(helm, adjoint):
    case = "3d"
    g, mp, b, f = _setup(case, 14, 2)
    z, o = _gpu(helm, "3d", mp, b, f, adjoint, precision=1, precond=2)
    ref = _oracle_vcycle(case, g, mp, f, b, o, adjoint)
    for i in range(len(b)):
        assert rel(z[i], ref[i]) <= 2e-4, (i, rel(z[i], ref[i]))


@pytest.mark.parametrize("sweeps", [1, 3])
@pytest.mark.parametrize("adjoint", [False, True])
def test_jacobi_fp64(helm, sweeps, adjoint):
    g, mp, b, f = _setup("3d", 15, 2)
    z, o = _gpu(helm, "3d", mp, b, f, adjoint, precision=0, precond=1, jacobi_sweeps=sweeps, jacobi_omega=0.7)
    H = O.helmholtz_matrix(g, O.extend(g, mp), 2 * np.pi * f)
    if adjoint:
        H = H.conj().T.tocsr()
    for i in range(len(b)):
        ref = O.jacobi_precond(H, b[i], 0.7, sweeps)
        assert rel(z[i], ref) <= 1e-13


def test_no_preconditioner_is_a_copy(helm):
    g, mp, b, f = _setup("2d", 16, 2)
    z, o = _gpu(helm, "2d", mp, b, f, False, precision=0, precond=0)
    assert np.array_equal(z, b)
