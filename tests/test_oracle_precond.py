"""Pins of the oracle's preconditioners (Sec. 4) against facts that do not
come from the oracle itself: consistency of the rediscretised coarse operator
with the fine one (second order in h), exactness of the cycle when its GMRES
smoothers are exhaustive, the cycle's effect as a preconditioner, and the
closed-form limit of damped Jacobi sweeps."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import helmholtz as O


def _smooth_field(g):
    """A smooth field over the whole computational grid (layers included),
    vanishing on the Dirichlet walls one cell beyond the outermost nodes."""
    Nx, Ny, Nz = g.N
    X, Z = np.meshgrid(np.arange(Nx) + 1.0, np.arange(Nz) + 1.0, indexing="ij")
    sx, sz = np.pi * X / (Nx + 1), np.pi * Z / (Nz + 1)
    u = np.sin(sx) * np.sin(sz) * (1 + 0.3j * np.cos(sx))
    return u.T.ravel()  # (Nz, Nx) order, x fastest


def _coarse_consistency_error(n, npml, h):
    # fixed physical box (n-1)h and layer width npml h; only the spacing changes
    g = O.make_grid(2, (n, 1, n), h, (npml, 0, npml), 2000.0, levels=2)
    omega = 2 * np.pi * 3.0
    mc = np.full(g.size, 1 / 2000.0 ** 2)
    u = _smooth_field(g)
    H0 = O.level_matrix(g, mc, omega, 0)
    m1 = O.level_models(g, mc, 2)[1]
    H1 = O.level_matrix(g, m1, omega, 1)
    R = O.restriction(g.N, 2)
    lhs = H1 @ (R @ u)
    rhs = R @ (H0 @ u)
    return np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs)


def test_level0_is_the_helmholtz_matrix():
    g = O.make_grid(3, (7, 6, 5), 30.0, (3, 3, 3), 3000.0, levels=2)
    rng = np.random.default_rng(0)
    mc = rng.uniform(1e-7, 4e-7, g.size)
    d = O.level_matrix(g, mc, 9.0, 0) - O.helmholtz_matrix(g, mc, 9.0)
    assert abs(d).max() == 0.0


def test_coarse_operator_is_second_order_consistent():
    """H_1 R u - R H_0 u = O(h^2) for a smooth u: a wrong coarse spacing, node
    position or half-node offset leaves an O(1) or O(h) error instead."""
    e1 = _coarse_consistency_error(81, 16, 12.5)
    e2 = _coarse_consistency_error(161, 32, 6.25)
    assert e2 < 0.005
    assert e1 / e2 > 3.2  # tends to 4 for second order (3.6 at these sizes), 2 for first


def test_coarse_levels_and_sizes():
    g = O.make_grid(3, (20, 17, 9), 10.0, (5, 4, 6), 2000.0, levels=3)
    for l in range(3):
        N = O.level_N(g, l)
        H = O.level_matrix(g, np.ones(int(np.prod(N))) * 1e-7, 10.0, l)
        assert H.shape == (int(np.prod(N)),) * 2
    N0, N1, N2 = (O.level_N(g, l) for l in range(3))
    assert all(N0[d] == 2 * N1[d] + 1 and N1[d] == 2 * N2[d] + 1 for d in range(3))


def test_exhaustive_smoothing_makes_the_cycle_exact():
    """With GMRES smoothers run for as many steps as there are unknowns the
    pre-smoother solves H x = b exactly, so the cycle returns H^{-1} b."""
    g = O.make_grid(2, (5, 1, 5), 40.0, (2, 0, 2), 2000.0, levels=2)
    rng = np.random.default_rng(1)
    mc = O.extend(g, rng.uniform(1 / 3000.0 ** 2, 1 / 1500.0 ** 2, g.n_phys))
    omega = 2 * np.pi * 6.0
    M = O.MLGmres(g, mc, omega, levels=2, k_so=1, k_si=g.size, k_co=1, k_ci=4)
    b = rng.standard_normal(g.size) + 1j * rng.standard_normal(g.size)
    x = M(b)
    ref = spla.spsolve(sp.csc_matrix(O.helmholtz_matrix(g, mc, omega)), b)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-9


def _fgmres_iterations(A, b, M, tol, k=10, maxit=400):
    """Iterations of restarted FGMRES(k) (M None: GMRES) to ||b - A x|| <= tol ||b||."""
    x = np.zeros_like(b)
    bn = np.linalg.norm(b)
    its = 0
    while its < maxit:
        x = O.gmres_cycles(A, b, k, 1, x0=x, M=M)
        its += k
        if np.linalg.norm(b - A @ x) <= tol * bn:
            return its
    return its


@pytest.mark.parametrize("adjoint", [False, True])
def test_vcycle_is_an_effective_preconditioner(adjoint):
    """One V-cycle per Krylov step must cut the iteration count far below plain
    GMRES, and its coarse-grid correction must pay for itself: the cycle needs
    at most half the iterations of the same smoothing work without the
    correction (a wrong sign, scale or transfer fails this)."""
    g = O.make_grid(2, (61, 1, 61), 20.0, (12, 0, 12), 2500.0, levels=2)
    rng = np.random.default_rng(2)
    v = 2000.0 + 500.0 * rng.random(g.n_phys)
    mc = O.extend(g, 1.0 / v ** 2)
    omega = 2 * np.pi * 5.0
    H = O.helmholtz_matrix(g, mc, omega)
    A = sp.csr_matrix(H.conj().T) if adjoint else H
    M = O.MLGmres(g, mc, omega, levels=2, adjoint=adjoint)
    smooth_only = lambda r: O.gmres_cycles(A, r, M.k_si, 2 * M.k_so)  # noqa: E731
    b = np.zeros(g.size, dtype=np.complex128)
    b[g.size // 2] = 1.0
    plain = _fgmres_iterations(A, b, None, 1e-6, maxit=2000)
    prec = _fgmres_iterations(A, b, M, 1e-6)
    smo = _fgmres_iterations(A, b, smooth_only, 1e-6)
    assert prec * 10 <= plain, (prec, plain)
    assert prec * 2 <= smo, (prec, smo)


def test_three_level_cycle_matches_two_level_when_coarse_solve_is_exact():
    """With coarse solves run to (near) exactness the 3-level cycle and the
    2-level cycle return the same vector (both correct with H_1^{-1})."""
    g = O.make_grid(2, (9, 1, 9), 40.0, (3, 0, 3), 2500.0, levels=3)
    rng = np.random.default_rng(3)
    mc = O.extend(g, 1.0 / (2000.0 + 300 * rng.random(g.n_phys)) ** 2)
    omega = 2 * np.pi * 4.0
    n1 = int(np.prod(O.level_N(g, 1)))
    M2 = O.MLGmres(g, mc, omega, levels=2, k_co=1, k_ci=n1)
    M3 = O.MLGmres(g, mc, omega, levels=3, k_co=1, k_ci=n1)
    b = rng.standard_normal(g.size) + 1j * rng.standard_normal(g.size)
    z2, z3 = M2(b), M3(b)
    assert np.linalg.norm(z2 - z3) / np.linalg.norm(z2) < 1e-8


def test_jacobi_sweeps_converge_to_the_solution_on_a_dominant_diagonal():
    """z_{k+1} = z_k + w D^{-1}(b - H z_k) is a fixed-point iteration for
    H z = b; with a strongly dominant diagonal it converges to H^{-1} b."""
    g = O.make_grid(2, (15, 1, 13), 10.0, (4, 0, 4), 2000.0)
    mc = np.full(g.size, 5e-6)  # w^2 m >> 4/h^2
    omega = 2 * np.pi * 30.0
    H = O.helmholtz_matrix(g, mc, omega)
    rng = np.random.default_rng(4)
    b = rng.standard_normal(g.size) + 1j * rng.standard_normal(g.size)
    z = O.jacobi_precond(H, b, 0.8, 200)
    ref = spla.spsolve(sp.csc_matrix(H), b)
    assert np.linalg.norm(z - ref) / np.linalg.norm(ref) < 1e-10
    z1 = O.jacobi_precond(H, b, 0.8, 1)
    assert np.allclose(z1, 0.8 * b / H.diagonal(), rtol=0, atol=0)
