"""FP64 CPU oracle for the frequency-domain FWI misfit and adjoint-state gradient.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously-correct
statement of what the GPU library computes.  Only the test suite, the smoke
check and the benchmark's CPU-baseline leg may import it; the product path
never does, and it shares no code with the CUDA sources.

What it follows (Da Silva & Herrmann, "A Unified 2D/3D Large Scale Software
Environment for Nonlinear Inverse Problems"):
  * Sec. 2, eq. (helmholtz) and the extended-domain system: the Helmholtz
    operator (d~x^2 + d~y^2 + d~z^2 + w^2 m) with d~x = (1/eta(x)) dx inside the
    damping layer, zero Dirichlet on the outer boundary, m extended into the
    layer by copying in the normal direction;
  * Sec. 2, eq. (mainprob): f(m) = sum_{s,w} 1/2 || P_r H_w(m)^{-1} q_{s,w} - d_{s,w} ||^2;
  * Appendix A, eqs. (dU2), (dH), (dHadj): T dm = w^2 diag(u) dm with A = I,
    T* = w^2 diag(conj u), v = -H^{-H} P_r^T (P_r u - d), grad f = sum Re(T* v);
  * Table derivstuff / Listing pdefunc: the summation over sources and
    frequencies of Re(T(U)^H V), mapped back to the physical grid by the
    adjoint of the extension (to_phys); the linearised data J dm, its adjoint
    and the Gauss-Newton product J^T J dm;
  * Sec. 4 (Alg. vcycle text): linear-interpolation prolongation and its
    adjoint as restriction; the ML-GMRES V-cycle (GMRES smoothers, coarse
    FGMRES, rediscretised coarse operators) and damped Jacobi as
    preconditioners.

Readings taken where the paper is silent:
  * m = 1/v^2 and H = L_eta + w^2 diag(m);
  * eta_d(x) = 1 + i sigma_d(x)/w with sigma = sigma_max (dist/W)^2, W the
    layer width on that side, sigma_max = 3 v_ref ln(1000) / (2 npml h);
  * the stretched second derivative is discretised as
    a_i [ b_{i+1/2}(u_{i+1}-u_i) - b_{i-1/2}(u_i-u_{i-1}) ] / h^2 with
    a = 1/eta at nodes and b = 1/eta at half nodes (so A = I in eq. (dH));
  * sources and receivers sit on grid nodes: the windowed-sinc operators of
    Sec. 3 reduce to point sampling; a unit source is 1/h^dim at its node;
  * extra high-side layer cells ("pad") make (N+1) divisible by 2^(levels-1)
    for vertex-centred coarsening;
  * the V-cycle's "x~ <- x_f + P x_c" is x~ <- x~ + P x_c, the cycle starts
    from x = 0, the coarse m is the full-weighting restriction of the fine m and
    the coarse damping tables sample the same continuous sigma(x).

Every array here is complex128 / float64.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# ---------------------------------------------------------------------------
# Grid and damping layer (Sec. 2, extended domain Omega' of Omega)
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class Grid:
    """Computational grid: the physical box plus damping layers on every side.

    n    = (nx, ny, nz) physical nodes; 2D uses ny = 1 and npml[1] = 0.
    npml = layer cells per side; pad = extra cells on the high side."""
    dim: int
    n: tuple
    h: float
    npml: tuple
    pad: tuple
    v_ref: float
    sigma_max: tuple  # per axis

    @property
    def N(self):
        return tuple(self.n[d] + 2 * self.npml[d] + self.pad[d] for d in range(3))

    @property
    def shape(self):
        """Array shape (Nz, Ny, Nx) of a computational-grid field."""
        Nx, Ny, Nz = self.N
        return (Nz, Ny, Nx)

    @property
    def size(self):
        Nx, Ny, Nz = self.N
        return Nx * Ny * Nz

    @property
    def phys_shape(self):
        nx, ny, nz = self.n
        return (nz, ny, nx)

    @property
    def n_phys(self):
        return self.n[0] * self.n[1] * self.n[2]


def make_grid(dim: int, n: Sequence[int], h: float, npml: Sequence[int], v_ref: float,
              levels: int = 1, sigma_max: Optional[Sequence[float]] = None) -> Grid:
    """Build the extended grid.  With `levels` > 1 the high side receives extra
    layer cells so that N_d + 1 is divisible by 2^(levels-1) on every active axis."""
    n = tuple(int(v) for v in n)
    npml = tuple(int(v) for v in npml)
    if dim == 2:
        assert n[1] == 1 and npml[1] == 0
    q = 1 << max(levels - 1, 0)
    pad = []
    for d in range(3):
        if dim == 2 and d == 1:
            pad.append(0)
            continue
        base = n[d] + 2 * npml[d]
        pad.append((-(base + 1)) % q)
    if sigma_max is None:
        sigma_max = tuple((3.0 * v_ref * np.log(1000.0) / (2.0 * npml[d] * h)) if npml[d] > 0 else 0.0
                          for d in range(3))
    return Grid(dim=dim, n=n, h=float(h), npml=npml, pad=tuple(pad), v_ref=float(v_ref),
                sigma_max=tuple(float(s) for s in sigma_max))


def sigma_at(t: np.ndarray, d: int, g: Grid) -> np.ndarray:
    """Damping sigma_d at computational-grid coordinate t (in cells, may be
    half-integer) along axis d.  Zero inside the physical box; quadratic in the
    distance to the box across the layer of that side."""
    lo = g.npml[d]
    hi = g.npml[d] + g.n[d] - 1
    W_lo = g.npml[d] * g.h
    W_hi = (g.npml[d] + g.pad[d]) * g.h
    t = np.asarray(t, dtype=np.float64)
    s = np.zeros_like(t)
    if g.npml[d] == 0 and g.pad[d] == 0:
        return s
    below = t < lo
    above = t > hi
    if W_lo > 0:
        s[below] = g.sigma_max[d] * (((lo - t[below]) * g.h) / W_lo) ** 2
    if W_hi > 0:
        s[above] = g.sigma_max[d] * (((t[above] - hi) * g.h) / W_hi) ** 2
    return s


def axis_coefficients(g: Grid, d: int, omega: float):
    """1D stretched second-derivative coefficients along axis d.

    Returns (cm, cp, cd): for node i, (L_d u)_i = cm[i] u_{i-1} + cd[i] u_i + cp[i] u_{i+1}
    with cm = a_i b_{i-1/2} / h^2, cp = a_i b_{i+1/2} / h^2, cd = -(cm + cp),
    a = 1/eta at nodes, b = 1/eta at half nodes, eta = 1 + i sigma / omega."""
    N = g.N[d]
    i = np.arange(N, dtype=np.float64)
    a = 1.0 / (1.0 + 1j * sigma_at(i, d, g) / omega)
    b_minus = 1.0 / (1.0 + 1j * sigma_at(i - 0.5, d, g) / omega)
    b_plus = 1.0 / (1.0 + 1j * sigma_at(i + 0.5, d, g) / omega)
    h2 = g.h * g.h
    cm = a * b_minus / h2
    cp = a * b_plus / h2
    return cm, cp, -(cm + cp)


def second_difference_1d(cm, cp, cd) -> sp.csr_matrix:
    """Tridiagonal 1D matrix with zero Dirichlet values beyond both ends."""
    N = len(cd)
    return sp.diags([cm[1:], cd, cp[:-1]], offsets=[-1, 0, 1], shape=(N, N), format="csr",
                    dtype=np.complex128)


def helmholtz_matrix(g: Grid, m_comp: np.ndarray, omega: float) -> sp.csr_matrix:
    """H(m, omega) = sum_d L_d + omega^2 diag(m) on the computational grid.

    Linear index p = ix + Nx*(iy + Ny*iz), so the x operator acts on the
    fastest Kronecker factor."""
    Nx, Ny, Nz = g.N
    Ix, Iy, Iz = (sp.identity(k, dtype=np.complex128, format="csr") for k in (Nx, Ny, Nz))
    Lx = second_difference_1d(*axis_coefficients(g, 0, omega))
    Lz = second_difference_1d(*axis_coefficients(g, 2, omega))
    H = sp.kron(Iz, sp.kron(Iy, Lx)) + sp.kron(Lz, sp.kron(Iy, Ix))
    if g.dim == 3:
        Ly = second_difference_1d(*axis_coefficients(g, 1, omega))
        H = H + sp.kron(Iz, sp.kron(Ly, Ix))
    H = H + sp.diags(omega * omega * np.asarray(m_comp, dtype=np.float64).ravel())
    return sp.csr_matrix(H)


# ---------------------------------------------------------------------------
# Model extension E and its adjoint (Sec. 2; Listing pdefunc "to_phys")
# ---------------------------------------------------------------------------

def _phys_of_comp(g: Grid, d: int) -> np.ndarray:
    """For each computational node along axis d, the physical node it copies."""
    return np.clip(np.arange(g.N[d]) - g.npml[d], 0, g.n[d] - 1)


def extend(g: Grid, m_phys: np.ndarray) -> np.ndarray:
    """E m: copy the physical model into the layers along the normal direction."""
    m = np.asarray(m_phys, dtype=np.float64).reshape(g.phys_shape)
    ix, iy, iz = (_phys_of_comp(g, d) for d in range(3))
    return m[np.ix_(iz, iy, ix)]


def extend_adjoint(g: Grid, g_comp: np.ndarray) -> np.ndarray:
    """E^T g: sum each computational value onto the physical node it was copied from."""
    gc = np.asarray(g_comp, dtype=np.float64).reshape(g.shape)
    ix, iy, iz = (_phys_of_comp(g, d) for d in range(3))
    out = np.zeros(g.phys_shape)
    np.add.at(out, np.ix_(iz, iy, ix), gc)
    return out


# ---------------------------------------------------------------------------
# Sources, receivers (Sec. 2, P_r and the localised q; Listing pdefunc Ps, Pr)
# ---------------------------------------------------------------------------

def comp_index(g: Grid, phys_idx: np.ndarray) -> np.ndarray:
    """Computational linear index of a physical linear node index."""
    nx, ny, _ = g.n
    Nx, Ny, _ = g.N
    p = np.asarray(phys_idx, dtype=np.int64)
    ix = p % nx
    iy = (p // nx) % ny
    iz = p // (nx * ny)
    return (ix + g.npml[0]) + Nx * ((iy + g.npml[1]) + Ny * (iz + g.npml[2]))


def source_fields(g: Grid, src_idx, Q, weight: complex = 1.0) -> np.ndarray:
    """q_s = weight * sum_k Q[k, s] delta_h(x - x_k), delta_h = 1/h^dim at the node.
    Returns (nsrc, size)."""
    Q = np.asarray(Q, dtype=np.complex128)
    nsrc = Q.shape[1]
    q = np.zeros((nsrc, g.size), dtype=np.complex128)
    ci = comp_index(g, src_idx)
    for s in range(nsrc):
        np.add.at(q[s], ci, weight * Q[:, s] / g.h ** g.dim)
    return q


def sample_receivers(g: Grid, u: np.ndarray, rec_idx) -> np.ndarray:
    """P_r u for fields of shape (..., size)."""
    return np.asarray(u)[..., comp_index(g, rec_idx)]


def spread_receivers(g: Grid, r: np.ndarray, rec_idx) -> np.ndarray:
    """P_r^T r: place receiver values back on their nodes (zero elsewhere)."""
    r = np.asarray(r, dtype=np.complex128)
    out = np.zeros(r.shape[:-1] + (g.size,), dtype=np.complex128)
    ci = comp_index(g, rec_idx)
    flat = out.reshape(-1, g.size)
    rr = r.reshape(-1, r.shape[-1])
    for k in range(flat.shape[0]):
        np.add.at(flat[k], ci, rr[k])
    return out


# ---------------------------------------------------------------------------
# Linear solvers: sparse direct, and restarted GMRES (Saad & Schultz 1986)
# ---------------------------------------------------------------------------

class DirectSolver:
    """Sparse LU of H, factorised once and reused across right-hand sides
    (the 2D strategy of Sec. 3)."""

    def __init__(self, H: sp.spmatrix):
        self.H = sp.csc_matrix(H)
        self.lu = spla.splu(self.H)

    def solve(self, b: np.ndarray) -> np.ndarray:
        return self.lu.solve(np.asarray(b, dtype=np.complex128))

    def solve_adjoint(self, b: np.ndarray) -> np.ndarray:
        return self.lu.solve(np.asarray(b, dtype=np.complex128), trans="H")


def gmres(A, b: np.ndarray, tol: float = 1e-13, restart: int = 60, maxiter: int = 100000,
          x0: Optional[np.ndarray] = None):
    """Restarted GMRES without preconditioning.

    Arnoldi with modified Gram-Schmidt (one re-orthogonalisation pass), the
    Hessenberg least-squares problem reduced by Givens rotations, restart
    after `restart` steps.  Stops when the true residual ||b - A x|| <= tol ||b||.
    Returns (x, total_iterations, relative_residual)."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    it = 0
    r = b - A @ x
    beta = np.linalg.norm(r)
    while it < maxiter:
        if beta <= tol * bnorm:
            break
        V = np.zeros((restart + 1, b.size), dtype=np.complex128)
        Hh = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart, dtype=np.complex128)
        sn = np.zeros(restart, dtype=np.complex128)
        e = np.zeros(restart + 1, dtype=np.complex128)
        e[0] = beta
        V[0] = r / beta
        k_used = 0
        for j in range(restart):
            w = A @ V[j]
            for _pass in range(2):
                for i in range(j + 1):
                    hij = np.vdot(V[i], w)
                    Hh[i, j] += hij
                    w = w - hij * V[i]
            Hh[j + 1, j] = np.linalg.norm(w)
            if Hh[j + 1, j] != 0:
                V[j + 1] = w / Hh[j + 1, j]
            # apply previous rotations to the new column
            for i in range(j):
                t = cs[i] * Hh[i, j] + sn[i] * Hh[i + 1, j]
                Hh[i + 1, j] = -np.conj(sn[i]) * Hh[i, j] + np.conj(cs[i]) * Hh[i + 1, j]
                Hh[i, j] = t
            # new rotation zeroing Hh[j+1, j]
            a_, b_ = Hh[j, j], Hh[j + 1, j]
            rr = np.hypot(abs(a_), abs(b_))
            if rr == 0:
                cs[j], sn[j] = 1.0, 0.0
            else:
                cs[j] = a_ / rr
                sn[j] = b_ / rr
                # rotation G = [[conj(c), conj(s)], [-s, c]] maps (a, b) -> (rr, 0)
                cs[j] = np.conj(cs[j])
                sn[j] = np.conj(sn[j])
            Hh[j, j] = cs[j] * a_ + sn[j] * b_
            Hh[j + 1, j] = 0.0
            e[j + 1] = -np.conj(sn[j]) * e[j]
            e[j] = cs[j] * e[j]
            it += 1
            k_used = j + 1
            if abs(e[j + 1]) <= 0.5 * tol * bnorm or it >= maxiter:
                break
        y = np.linalg.solve(np.triu(Hh[:k_used, :k_used]), e[:k_used])
        x = x + V[:k_used].T @ y
        r = b - A @ x
        beta = np.linalg.norm(r)
    return x, it, beta / bnorm


class GmresSolver:
    """H^{-1} and H^{-H} by restarted GMRES on the explicit sparse matrix."""

    def __init__(self, H: sp.spmatrix, tol: float = 1e-13, restart: int = 60,
                 maxiter: int = 200000):
        self.H = sp.csr_matrix(H)
        self.HH = sp.csr_matrix(self.H.conj().T)
        self.tol, self.restart, self.maxiter = tol, restart, maxiter
        self.iterations = []

    def solve(self, b):
        x, it, _ = gmres(self.H, b, self.tol, self.restart, self.maxiter)
        self.iterations.append(it)
        return x

    def solve_adjoint(self, b):
        x, it, _ = gmres(self.HH, b, self.tol, self.restart, self.maxiter)
        self.iterations.append(it)
        return x


def make_solver(H, kind: str = "direct", **kw):
    if kind == "direct":
        return DirectSolver(H)
    if kind == "gmres":
        return GmresSolver(H, **kw)
    raise ValueError(kind)


# ---------------------------------------------------------------------------
# The three calls: forward modelling, adjoint solve, misfit + gradient
# ---------------------------------------------------------------------------

def _omega(f_hz: float) -> float:
    return 2.0 * np.pi * float(f_hz)


def forward(g: Grid, m_phys, freqs_hz, src_idx, Q, rec_idx, wavelet=None,
            solver: str = "direct", want_fields: bool = True, **solver_kw):
    """FORW_MODEL of Listing pdefunc: U = H^{-1} Q per frequency, D = P_r U.
    Returns (U [nfreq, nsrc, size] or None, D [nfreq, nsrc, nrec])."""
    mc = extend(g, m_phys)
    Qa = np.asarray(Q)
    nf, ns, nr = len(freqs_hz), Qa.shape[1], len(rec_idx)
    U = np.zeros((nf, ns, g.size), dtype=np.complex128) if want_fields else None
    D = np.zeros((nf, ns, nr), dtype=np.complex128)
    for k, fr in enumerate(freqs_hz):
        w = 1.0 if wavelet is None else wavelet[k]
        S = make_solver(helmholtz_matrix(g, mc, _omega(fr)), solver, **solver_kw)
        q = source_fields(g, src_idx, Qa, w)
        for s in range(ns):
            u = S.solve(q[s])
            if want_fields:
                U[k, s] = u
            D[k, s] = sample_receivers(g, u, rec_idx)
    return U, D


def adjoint(g: Grid, m_phys, freqs_hz, rec_idx, R_in, solver: str = "direct", **solver_kw):
    """V = H^{-H} P_r^T R per frequency and source.  Returns [nfreq, nsrc, size]."""
    mc = extend(g, m_phys)
    R_in = np.asarray(R_in, dtype=np.complex128)
    nf, ns = R_in.shape[0], R_in.shape[1]
    V = np.zeros((nf, ns, g.size), dtype=np.complex128)
    for k, fr in enumerate(freqs_hz):
        S = make_solver(helmholtz_matrix(g, mc, _omega(fr)), solver, **solver_kw)
        b = spread_receivers(g, R_in[k], rec_idx)
        for s in range(ns):
            V[k, s] = S.solve_adjoint(b[s])
    return V


def misfit_and_gradient(g: Grid, m_phys, freqs_hz, src_idx, Q, rec_idx, d_obs, wavelet=None,
                        mask=None, solver: str = "direct", return_fields: bool = False,
                        **solver_kw):
    """OBJ of Listing pdefunc with the least-squares misfit (Sec. 2):

        u   = H^{-1} q                     (state)
        r   = P_r u - d                    (grad of phi = 1/2 ||.||^2)
        f  += 1/2 ||r||^2
        v   = H^{-H} (-P_r^T r)            (adjoint state, Table derivstuff V(m))
        g  += Re( T(u)^* v ) = w^2 Re(conj(u) v)     (eq. (dHadj) with A = I)

    summed over frequencies and sources (optionally masked), then mapped to the
    physical grid by E^T.  Returns (f, g_phys[, U, V])."""
    mc = extend(g, m_phys)
    Qa = np.asarray(Q)
    d_obs = np.asarray(d_obs, dtype=np.complex128)
    nf, ns = len(freqs_hz), Qa.shape[1]
    f = 0.0
    gc = np.zeros(g.size)
    U = np.zeros((nf, ns, g.size), dtype=np.complex128) if return_fields else None
    V = np.zeros((nf, ns, g.size), dtype=np.complex128) if return_fields else None
    for k, fr in enumerate(freqs_hz):
        om = _omega(fr)
        w = 1.0 if wavelet is None else wavelet[k]
        S = make_solver(helmholtz_matrix(g, mc, om), solver, **solver_kw)
        q = source_fields(g, src_idx, Qa, w)
        for s in range(ns):
            if mask is not None and not mask[k][s]:
                continue
            u = S.solve(q[s])
            r = sample_receivers(g, u, rec_idx) - d_obs[k, s]
            f += 0.5 * float(np.vdot(r, r).real)
            v = S.solve_adjoint(-spread_receivers(g, r, rec_idx))
            gc += om * om * np.real(np.conj(u) * v)
            if return_fields:
                U[k, s], V[k, s] = u, v
    gp = extend_adjoint(g, gc)
    if return_fields:
        return f, gp, U, V
    return f, gp


def misfit(g: Grid, m_phys, freqs_hz, src_idx, Q, rec_idx, d_obs, wavelet=None, mask=None,
           solver: str = "direct", **solver_kw) -> float:
    """f(m) alone (one PDE solve per source and frequency, Table derivcosts)."""
    _, D = forward(g, m_phys, freqs_hz, src_idx, Q, rec_idx, wavelet, solver, want_fields=False,
                   **solver_kw)
    r = D - np.asarray(d_obs)
    if mask is not None:
        r = r * np.asarray(mask, dtype=np.float64)[..., None]
    return 0.5 * float(np.vdot(r, r).real)


# ---------------------------------------------------------------------------
# Linearised modelling (Appendix A; Table derivstuff): the Jacobian J of the
# data with respect to the physical m, its adjoint, and the Gauss-Newton
# Hessian-vector product J^T J
# ---------------------------------------------------------------------------

def born(g: Grid, m_phys, freqs_hz, src_idx, Q, rec_idx, dm_phys, wavelet=None, mask=None,
         solver: str = "direct", **solver_kw):
    """dD = J dm per frequency and source: with u = H^{-1} q the state,
    H du = -T dm with T dm = w^2 diag(u) E dm (eq. (dU2) with A = I), and
    dD = P_r du.  Pairs masked out return zeros.  Returns [nfreq, nsrc, nrec]."""
    mc = extend(g, m_phys)
    dmc = extend(g, dm_phys).ravel()
    Qa = np.asarray(Q)
    nf, ns = len(freqs_hz), Qa.shape[1]
    dD = np.zeros((nf, ns, len(rec_idx)), dtype=np.complex128)
    for k in range(nf):
        om = _omega(freqs_hz[k])
        w = 1.0 if wavelet is None else wavelet[k]
        S = make_solver(helmholtz_matrix(g, mc, om), solver, **solver_kw)
        q = source_fields(g, src_idx, Qa, w)
        for s in range(ns):
            if mask is not None and not mask[k][s]:
                continue
            u = S.solve(q[s])
            du = S.solve(-om * om * dmc * u)
            dD[k, s] = sample_receivers(g, du, rec_idx)
    return dD


def born_adjoint(g: Grid, m_phys, freqs_hz, src_idx, Q, rec_idx, dD, wavelet=None, mask=None,
                 solver: str = "direct", **solver_kw):
    """J^T dD for real m: sum over (s, w) of Re(T^* v) with v = -H^{-H} P_r^T dD
    (eq. (dHadj) with A = I: T^* v = w^2 conj(u) v), mapped by E^T.  Returns
    g_phys [n_phys] (the gradient formula with the data residual replaced by dD)."""
    mc = extend(g, m_phys)
    Qa = np.asarray(Q)
    dD = np.asarray(dD, dtype=np.complex128)
    nf, ns = len(freqs_hz), Qa.shape[1]
    gc = np.zeros(g.size)
    for k in range(nf):
        om = _omega(freqs_hz[k])
        w = 1.0 if wavelet is None else wavelet[k]
        S = make_solver(helmholtz_matrix(g, mc, om), solver, **solver_kw)
        q = source_fields(g, src_idx, Qa, w)
        for s in range(ns):
            if mask is not None and not mask[k][s]:
                continue
            u = S.solve(q[s])
            v = S.solve_adjoint(-spread_receivers(g, dD[k, s], rec_idx))
            gc += om * om * np.real(np.conj(u) * v)
    return extend_adjoint(g, gc)


def gauss_newton_hessvec(g: Grid, m_phys, freqs_hz, src_idx, Q, rec_idx, dm_phys, wavelet=None, mask=None,
                         solver: str = "direct", **solver_kw):
    """J^T J dm: three PDE solves per (s, w) (state, linearised state, adjoint),
    Table derivstuff's Gauss-Newton Hessian applied to dm."""
    dD = born(g, m_phys, freqs_hz, src_idx, Q, rec_idx, dm_phys, wavelet, mask, solver, **solver_kw)
    return born_adjoint(g, m_phys, freqs_hz, src_idx, Q, rec_idx, dD, wavelet, mask, solver, **solver_kw)


def hessvec(g: Grid, m_phys, freqs_hz, src_idx, Q, rec_idx, d_obs, dm_phys, wavelet=None, mask=None,
            solver: str = "direct", **solver_kw):
    """Full Hessian of the least-squares misfit applied to dm (Table derivstuff,
    last row; Appendix A with A = I and phi = 1/2 ||. - d||^2, so the Hessian of
    phi is the identity).  Four PDE solves per (s, w):

        u   = H^{-1} q,                 du  = -H^{-1} (w^2 (E dm) u)
        v   = -H^{-H} P_r^T (P_r u - d),
        dv  = H^{-H} ( -w^2 (E dm) v - P_r^T P_r du )      (DV(m)[dm] of the table)
        Hdm = E^T sum Re( w^2 conj(du) v + w^2 conj(u) dv ) (DT^*[dm, du] V + T^* DV)

    The sign of the DH^H v term follows from differentiating H^H v = -P_r^T r."""
    mc = extend(g, m_phys)
    dmc = extend(g, dm_phys).ravel()
    Qa = np.asarray(Q)
    d_obs = np.asarray(d_obs, dtype=np.complex128)
    nf, ns = len(freqs_hz), Qa.shape[1]
    gc = np.zeros(g.size)
    for k in range(nf):
        om = _omega(freqs_hz[k])
        w = 1.0 if wavelet is None else wavelet[k]
        S = make_solver(helmholtz_matrix(g, mc, om), solver, **solver_kw)
        q = source_fields(g, src_idx, Qa, w)
        for s in range(ns):
            if mask is not None and not mask[k][s]:
                continue
            u = S.solve(q[s])
            r = sample_receivers(g, u, rec_idx) - d_obs[k, s]
            v = S.solve_adjoint(-spread_receivers(g, r, rec_idx))
            du = S.solve(-om * om * dmc * u)
            dv = S.solve_adjoint(-om * om * dmc * v - spread_receivers(g, sample_receivers(g, du, rec_idx), rec_idx))
            gc += om * om * np.real(np.conj(du) * v + np.conj(u) * dv)
    return extend_adjoint(g, gc)


# ---------------------------------------------------------------------------
# Waveform Reconstruction Inversion (Sec. 3, penalty method; Appendix B):
# the field minimises ||P_r u - d||^2 + lambda^2 ||H u - q||^2 for fixed m
# ---------------------------------------------------------------------------

def wri_field(H: sp.spmatrix, P: sp.spmatrix, q: np.ndarray, d: np.ndarray, lam: float) -> np.ndarray:
    """u(m) of eq. (wrifieldeq) from its normal equations
    (P_r^T P_r + lambda^2 H^H H) u = P_r^T d + lambda^2 H^H q (sparse LU)."""
    H = sp.csc_matrix(H)
    Gm = sp.csc_matrix(P.T @ P + lam * lam * (H.conj().T @ H))
    rhs = P.T @ d + lam * lam * (H.conj().T @ q)
    return spla.spsolve(Gm, rhs)


def wri_field_dataspace(H: sp.spmatrix, P: sp.spmatrix, q: np.ndarray, d: np.ndarray, lam: float) -> np.ndarray:
    """The same field through solves with H and H^H only:
    u = u0 + lambda^-2 H^{-1} H^{-H} P^T z with u0 = H^{-1} q and
    (I + lambda^-2 P H^{-1} H^{-H} P^T) z = d - P u0 (the push-through identity
    applied to the normal equations; a dense nrec x nrec system here)."""
    S = DirectSolver(H)
    u0 = S.solve(q)
    nrec = P.shape[0]
    C = np.zeros((nrec, nrec), dtype=np.complex128)
    for k in range(nrec):
        e = np.zeros(nrec, dtype=np.complex128)
        e[k] = 1.0
        C[:, k] = P @ S.solve(S.solve_adjoint(P.T @ e))
    z = np.linalg.solve(np.eye(nrec) + C / (lam * lam), d - P @ u0)
    return u0 + S.solve(S.solve_adjoint(P.T @ z)) / (lam * lam)


def wri_misfit_and_gradient(g: Grid, m_phys, freqs_hz, src_idx, Q, rec_idx, d_obs, lam: float):
    """WRI objective f = sum 1/2 ||P_r u - d||^2 + lambda^2/2 ||H u - q||^2 at
    u = u(m) and its gradient lambda^2 E^T sum Re(T^* (H u - q)) =
    E^T sum lambda^2 w^2 Re(conj(u) (H u - q)) (Appendix B, variable projection)."""
    mc = extend(g, m_phys)
    Qa = np.asarray(Q)
    d_obs = np.asarray(d_obs, dtype=np.complex128)
    P = receiver_matrix(g, rec_idx)
    f = 0.0
    gc = np.zeros(g.size)
    for k, fr in enumerate(freqs_hz):
        om = _omega(fr)
        H = helmholtz_matrix(g, mc, om)
        q = source_fields(g, src_idx, Qa)
        for s in range(Qa.shape[1]):
            u = wri_field(H, P, q[s], d_obs[k, s], lam)
            ru = H @ u - q[s]
            rd = P @ u - d_obs[k, s]
            f += 0.5 * float(np.vdot(rd, rd).real) + 0.5 * lam * lam * float(np.vdot(ru, ru).real)
            gc += lam * lam * om * om * np.real(np.conj(u) * ru)
    return f, extend_adjoint(g, gc)


def receiver_matrix(g: Grid, rec_idx) -> sp.csr_matrix:
    """P_r as a sparse nrec x size matrix (point sampling)."""
    cols = comp_index(g, np.asarray(rec_idx))
    n = len(cols)
    return sp.csr_matrix((np.ones(n), (np.arange(n), cols)), shape=(n, g.size), dtype=np.complex128)


# ---------------------------------------------------------------------------
# 2.5D modelling (Sec. 3, "2.5D"): a y-invariant model, a Fourier transform in
# y, one 2D problem per wavenumber k_y with the shift -k_y^2, and a quadrature
# sum over k_y
# ---------------------------------------------------------------------------

def gauss_legendre_ky(k_max: float, nk: int, dy: float = 0.0):
    """Nodes k_i on [0, k_max] and weights c_i = w_i cos(k_i dy) / pi of the
    quadrature u(x, y_s + dy, z) = (1/pi) int_0^k_max u~_k(x, z) cos(k dy) dk
    (Gauss-Legendre, mapped from [-1, 1])."""
    t, w = np.polynomial.legendre.leggauss(nk)
    k = 0.5 * k_max * (t + 1.0)
    c = 0.5 * k_max * w * np.cos(k * dy) / np.pi
    return k, c


def helmholtz_matrix_25d(g: Grid, m_comp: np.ndarray, omega: float, ky: float) -> sp.csr_matrix:
    """H(k_y) = H(m, omega) - k_y^2 I on a 2D grid (the y derivative becomes -k_y^2)."""
    assert g.dim == 2
    H = helmholtz_matrix(g, m_comp, omega)
    return sp.csr_matrix(H - ky * ky * sp.identity(g.size, dtype=np.complex128, format="csr"))


def forward_25d(g: Grid, m_phys, freqs_hz, ky, ck, src_idx, Q, rec_idx, wavelet=None):
    """2.5D data D[k, s] = sum_i c_i P_r u~_{k_i}, H(k_i) u~ = q (2D point sources,
    1/h^2 at the node).  Returns (D [nfreq, nsrc, nrec], U [nfreq, nsrc, nk, size])."""
    mc = extend(g, m_phys)
    Qa = np.asarray(Q)
    nf, ns, nk = len(freqs_hz), Qa.shape[1], len(ky)
    D = np.zeros((nf, ns, len(rec_idx)), dtype=np.complex128)
    U = np.zeros((nf, ns, nk, g.size), dtype=np.complex128)
    for k, fr in enumerate(freqs_hz):
        w = 1.0 if wavelet is None else wavelet[k]
        q = source_fields(g, src_idx, Qa, w)
        for i in range(nk):
            S = DirectSolver(helmholtz_matrix_25d(g, mc, _omega(fr), ky[i]))
            for s in range(ns):
                U[k, s, i] = S.solve(q[s])
                D[k, s] += ck[i] * sample_receivers(g, U[k, s, i], rec_idx)
    return D, U


def misfit_and_gradient_25d(g: Grid, m_phys, freqs_hz, ky, ck, src_idx, Q, rec_idx, d_obs, wavelet=None):
    """f = sum_{k,s} 1/2 || sum_i c_i P_r u~_i - d ||^2 and its gradient: with the
    residual r shared by the k_y terms, v_i = -H(k_i)^{-H} P_r^T (c_i r) and
    g = E^T sum w^2 Re(conj(u~_i) v_i) (the sum structure the section notes for
    derivatives).  Returns (f, g_phys)."""
    mc = extend(g, m_phys)
    d_obs = np.asarray(d_obs, dtype=np.complex128)
    D, U = forward_25d(g, m_phys, freqs_hz, ky, ck, src_idx, Q, rec_idx, wavelet)
    f = 0.0
    gc = np.zeros(g.size)
    for k, fr in enumerate(freqs_hz):
        om = _omega(fr)
        for i in range(len(ky)):
            S = DirectSolver(helmholtz_matrix_25d(g, mc, om, ky[i]))
            for s in range(U.shape[1]):
                r = D[k, s] - d_obs[k, s]
                v = S.solve_adjoint(-ck[i] * spread_receivers(g, r, rec_idx))
                gc += om * om * np.real(np.conj(U[k, s, i]) * v)
    for k in range(len(freqs_hz)):
        for s in range(D.shape[1]):
            r = D[k, s] - d_obs[k, s]
            f += 0.5 * float(np.vdot(r, r).real)
    return f, extend_adjoint(g, gc)


# ---------------------------------------------------------------------------
# Inter-grid transfers of the V-cycle (Sec. 4): linear interpolation P and
# restriction R = 2^-dim P^T (full weighting)
# ---------------------------------------------------------------------------

def prolong_1d_matrix(Nc: int) -> sp.csr_matrix:
    """Linear interpolation from Nc coarse to 2*Nc+1 fine nodes, zero beyond the
    walls: fine 2j+1 = coarse j; fine 2j = (coarse j-1 + coarse j)/2."""
    Nf = 2 * Nc + 1
    rows, cols, vals = [], [], []
    for j in range(Nc):
        rows += [2 * j + 1, 2 * j, 2 * j + 2]
        cols += [j, j, j]
        vals += [1.0, 0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(Nf, Nc))


def prolongation(fine_N: Sequence[int], dim: int) -> sp.csr_matrix:
    """Tensor-product (bi/tri)linear interpolation for fine sizes (Nx, Ny, Nz)."""
    Nx, Ny, Nz = fine_N
    Px = prolong_1d_matrix((Nx - 1) // 2)
    Pz = prolong_1d_matrix((Nz - 1) // 2)
    Py = prolong_1d_matrix((Ny - 1) // 2) if dim == 3 else sp.identity(Ny, format="csr")
    return sp.csr_matrix(sp.kron(Pz, sp.kron(Py, Px)))


def restriction(fine_N: Sequence[int], dim: int) -> sp.csr_matrix:
    """R = 2^-dim P^T."""
    return sp.csr_matrix(prolongation(fine_N, dim).T) * (0.5 ** dim)


# ---------------------------------------------------------------------------
# The ML-GMRES preconditioner (Sec. 4): rediscretised coarse operators, fixed
# restarted GMRES / FGMRES cycles as smoothers and coarse solvers, the V-cycle;
# and the damped Jacobi alternative
# ---------------------------------------------------------------------------

def level_N(g: Grid, level: int) -> tuple:
    """Nodes per axis (x, y, z) at grid level `level` (vertex-centred coarsening,
    N_c = (N - 1) / 2 on every active axis)."""
    N = list(g.N)
    for _ in range(level):
        N = [N[d] if (g.dim == 2 and d == 1) else (N[d] - 1) // 2 for d in range(3)]
    return tuple(N)


def level_axis_coefficients(g: Grid, d: int, omega: float, level: int):
    """The stretched second derivative of axis_coefficients rediscretised at
    level `level`: spacing 2^level h; coarse node j sits on fine node
    (j + 1) 2^level - 1, its half nodes 2^(level-1) fine cells either side, and
    the damping profile is the same continuous sigma(x) of the finest grid."""
    q = 1 << level
    Nl = level_N(g, level)[d]
    t = (np.arange(Nl, dtype=np.float64) + 1.0) * q - 1.0
    a = 1.0 / (1.0 + 1j * sigma_at(t, d, g) / omega)
    b_minus = 1.0 / (1.0 + 1j * sigma_at(t - 0.5 * q, d, g) / omega)
    b_plus = 1.0 / (1.0 + 1j * sigma_at(t + 0.5 * q, d, g) / omega)
    hl = q * g.h
    cm = a * b_minus / (hl * hl)
    cp = a * b_plus / (hl * hl)
    return cm, cp, -(cm + cp)


def level_models(g: Grid, m_comp: np.ndarray, levels: int) -> list:
    """m on every level: the finest computational m, then full weighting
    (R = 2^-dim P^T) of the level above."""
    ms = [np.asarray(m_comp, dtype=np.float64).ravel()]
    for l in range(1, levels):
        R = restriction(level_N(g, l - 1), g.dim)
        ms.append(R @ ms[-1])
    return ms


def level_matrix(g: Grid, m_level: np.ndarray, omega: float, level: int) -> sp.csr_matrix:
    """H_level = sum_d L_d(level) + omega^2 diag(m_level) (same Kronecker
    layout as helmholtz_matrix, which is level 0)."""
    Nx, Ny, Nz = level_N(g, level)
    Ix, Iy, Iz = (sp.identity(k, dtype=np.complex128, format="csr") for k in (Nx, Ny, Nz))
    Lx = second_difference_1d(*level_axis_coefficients(g, 0, omega, level))
    Lz = second_difference_1d(*level_axis_coefficients(g, 2, omega, level))
    H = sp.kron(Iz, sp.kron(Iy, Lx)) + sp.kron(Lz, sp.kron(Iy, Ix))
    if g.dim == 3:
        Ly = second_difference_1d(*level_axis_coefficients(g, 1, omega, level))
        H = H + sp.kron(Iz, sp.kron(Ly, Ix))
    H = H + sp.diags(omega * omega * np.asarray(m_level, dtype=np.float64).ravel())
    return sp.csr_matrix(H)


def gmres_cycles(A, b: np.ndarray, k: int, cycles: int, x0: Optional[np.ndarray] = None,
                 M=None) -> np.ndarray:
    """`cycles` restarts of k steps of GMRES (M None) or flexible GMRES with the
    right preconditioner z = M(v) (Saad's FGMRES, used by Sec. 4 for the
    coarse solves), no stopping test: the fixed-work smoother / coarse solver.

    Arnoldi with modified Gram-Schmidt and one re-orthogonalisation pass; the
    least-squares problem min || beta e_1 - Hbar y || solved by a dense
    least-squares routine; x += V y (or Z y)."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    for _ in range(cycles):
        r = b - A @ x
        beta = np.linalg.norm(r)
        if beta == 0.0:
            break
        V = np.zeros((k + 1, b.size), dtype=np.complex128)
        Z = np.zeros((k, b.size), dtype=np.complex128) if M is not None else None
        Hh = np.zeros((k + 1, k), dtype=np.complex128)
        V[0] = r / beta
        used = 0
        for j in range(k):
            zj = V[j] if M is None else M(V[j])
            if Z is not None:
                Z[j] = zj
            w = A @ zj
            for _pass in range(2):
                for i in range(j + 1):
                    hij = np.vdot(V[i], w)
                    Hh[i, j] += hij
                    w = w - hij * V[i]
            Hh[j + 1, j] = np.linalg.norm(w)
            used = j + 1
            if Hh[j + 1, j] == 0.0:
                break
            V[j + 1] = w / Hh[j + 1, j]
        e1 = np.zeros(used + 1, dtype=np.complex128)
        e1[0] = beta
        y = np.linalg.lstsq(Hh[:used + 1, :used], e1, rcond=None)[0]
        x = x + (V[:used] if Z is None else Z[:used]).T @ y
    return x


class MLGmres:
    """The ML-GMRES V-cycle of Sec. 4 as a preconditioner z = M^{-1} b.

    Levels l = 0..L-1 with H_l rediscretised at spacing 2^l h (restricted m);
    transfers P (linear interpolation) and R = 2^-dim P^T.  One cycle at level
    l from a zero guess: pre-smooth with k_so cycles of GMRES(k_si), restrict
    the residual, solve the coarse problem with k_co cycles of FGMRES(k_ci)
    preconditioned by the level-(l+1) cycle (plain GMRES(k_ci) on the last
    level), add the prolonged coarse solution, post-smooth as before.
    adjoint=True builds the same cycle on the H_l^H."""

    def __init__(self, g: Grid, m_comp, omega: float, levels: int = 2, k_so: int = 3, k_si: int = 5,
                 k_co: int = 3, k_ci: int = 5, adjoint: bool = False):
        self.g, self.L = g, levels
        self.k_so, self.k_si, self.k_co, self.k_ci = k_so, k_si, k_co, k_ci
        ms = level_models(g, m_comp, levels)
        self.H = []
        for l in range(levels):
            H = level_matrix(g, ms[l], omega, l)
            self.H.append(sp.csr_matrix(H.conj().T) if adjoint else H)
        self.P = [prolongation(level_N(g, l), g.dim) for l in range(levels - 1)]
        self.R = [restriction(level_N(g, l), g.dim) for l in range(levels - 1)]

    def cycle(self, b: np.ndarray, level: int = 0) -> np.ndarray:
        H = self.H[level]
        x = gmres_cycles(H, b, self.k_si, self.k_so)
        bc = self.R[level] @ (b - H @ x)
        if level + 1 < self.L - 1:
            xc = gmres_cycles(self.H[level + 1], bc, self.k_ci, self.k_co,
                              M=lambda v: self.cycle(v, level + 1))
        else:
            xc = gmres_cycles(self.H[level + 1], bc, self.k_ci, self.k_co)
        x = x + self.P[level] @ xc
        return gmres_cycles(H, b, self.k_si, self.k_so, x0=x)

    def __call__(self, b):
        return self.cycle(np.asarray(b, dtype=np.complex128), 0)


def jacobi_precond(H: sp.spmatrix, b: np.ndarray, omega_j: float, sweeps: int) -> np.ndarray:
    """`sweeps` damped Jacobi sweeps z <- z + omega_j D^{-1} (b - H z) from z = 0,
    D = diag(H) (the simple preconditioner alternative of Sec. 4)."""
    b = np.asarray(b, dtype=np.complex128)
    D = H.diagonal()
    z = np.zeros_like(b)
    for _ in range(sweeps):
        z = z + omega_j * (b - H @ z) / D
    return z
