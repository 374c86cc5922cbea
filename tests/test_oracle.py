"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test targets a plausible mistake: a dropped term, a wrong sign, a wrong
scale, transposed axes, a wrong adjoint.  None of them compares the oracle
with itself or with the CUDA path.
"""
import numpy as np
import pytest
from scipy.special import hankel1

from oracle import helmholtz as O

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


def _const_grid(dim, n, h, npml, v0, levels=1):
    g = O.make_grid(dim, n, h, npml, v0, levels=levels)
    return g, np.full(g.phys_shape, 1.0 / v0 ** 2)


# ---------------------------------------------------------------------------
# Operator: closed-form spectrum of the Dirichlet Laplacian (no damping layer)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,n", [(3, (5, 6, 7)), (2, (9, 1, 6))])
def test_dirichlet_eigenpairs(dim, n):
    """Without a layer H = 7-pt (5-pt) Laplacian + w^2 m with zero Dirichlet
    walls one cell outside the grid.  Its eigenvectors are products of
    sin(pi k (i+1)/(N+1)) with eigenvalue sum_d -(4/h^2) sin^2(pi k_d / (2(N_d+1))) + w^2 m.
    Unequal N per axis pins the axis order; the constant pins w^2 m."""
    h, v0, f = 12.5, 1800.0, 3.0
    g, m = _const_grid(dim, n, h, (0, 0, 0), v0)
    om = 2 * np.pi * f
    H = O.helmholtz_matrix(g, O.extend(g, m), om)
    Nx, Ny, Nz = g.N
    iz, iy, ix = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    for k in [(1, 1, 1), (2, 1, 3), (Nx, Ny, 1), (3, Ny, Nz)]:
        kx, ky, kz = k
        ky = ky if dim == 3 else 1
        vec = np.sin(np.pi * kx * (ix + 1) / (Nx + 1)) * np.sin(np.pi * kz * (iz + 1) / (Nz + 1))
        lam = -(4 / h ** 2) * (np.sin(np.pi * kx / (2 * (Nx + 1))) ** 2
                               + np.sin(np.pi * kz / (2 * (Nz + 1))) ** 2)
        if dim == 3:
            vec = vec * np.sin(np.pi * ky * (iy + 1) / (Ny + 1))
            lam += -(4 / h ** 2) * np.sin(np.pi * ky / (2 * (Ny + 1))) ** 2
        lam += om ** 2 / v0 ** 2
        v = vec.ravel()
        Hv = H @ v
        assert np.linalg.norm(Hv - lam * v) <= 1e-12 * abs(lam) * np.linalg.norm(v)


def test_operator_pointwise_from_stretched_derivative():
    """Rebuild H entry by entry from the stretched second derivative
    (1/eta) d/dx (1/eta) d/dx evaluated with physical positions in metres
    (nodes and half nodes), on a tiny 3D grid with layers of different width
    on every axis, and compare with the oracle's Kronecker assembly."""
    n, h, npml, vref, f = (4, 3, 5), 10.0, (2, 1, 3), 2500.0, 7.0
    g = O.make_grid(3, n, h, npml, vref, levels=2)
    rng = np.random.default_rng(0)
    mp = rng.uniform(1 / 3000 ** 2, 1 / 1500 ** 2, size=g.phys_shape)
    om = 2 * np.pi * f
    H = O.helmholtz_matrix(g, O.extend(g, mp), om).toarray()

    def sigma_m(xm, d):
        # position xm in metres relative to the first physical node
        box_hi = (n[d] - 1) * h
        smax = 3 * vref * np.log(1000) / (2 * npml[d] * h)
        if xm < 0:
            return smax * (-xm / (npml[d] * h)) ** 2
        if xm > box_hi:
            return smax * ((xm - box_hi) / ((npml[d] + g.pad[d]) * h)) ** 2
        return 0.0

    def inv_eta(xm, d):
        return 1.0 / (1.0 + 1j * sigma_m(xm, d) / om)

    Nx, Ny, Nz = g.N
    Href = np.zeros_like(H)
    mc = O.extend(g, mp).ravel()
    for iz in range(Nz):
        for iy in range(Ny):
            for ix in range(Nx):
                p = ix + Nx * (iy + Ny * iz)
                idx = (ix, iy, iz)
                Href[p, p] += om ** 2 * mc[p]
                for d, stride in enumerate((1, Nx, Nx * Ny)):
                    x = (idx[d] - npml[d]) * h
                    a = inv_eta(x, d)
                    bp = inv_eta(x + h / 2, d)
                    bm = inv_eta(x - h / 2, d)
                    Href[p, p] += -a * (bp + bm) / h ** 2
                    if idx[d] + 1 < g.N[d]:
                        Href[p, p + stride] += a * bp / h ** 2
                    if idx[d] - 1 >= 0:
                        Href[p, p - stride] += a * bm / h ** 2
    assert np.max(np.abs(H - Href)) <= 1e-13 * np.max(np.abs(Href))


def test_damping_profile_properties():
    g = O.make_grid(3, (20, 20, 20), 25.0, (10, 10, 10), 4500.0, levels=3)
    om = 2 * np.pi * 4.0
    for d in range(3):
        cm, cp, cd = O.axis_coefficients(g, d, om)
        lo, hi = g.npml[d], g.npml[d] + g.n[d] - 1
        # undamped inside the physical box (half nodes included)
        assert np.allclose(cm[lo + 1:hi], 1 / g.h ** 2, rtol=0, atol=1e-18)
        assert np.allclose(cp[lo:hi], 1 / g.h ** 2, rtol=0, atol=1e-18)
        # damping reduces |coefficients| monotonically toward both walls
        mag = np.abs(cp)
        assert np.all(np.diff(mag[:lo + 1]) >= 0) and np.all(np.diff(mag[hi:]) <= 0)
        assert mag[0] < 0.2 * mag[lo]
        s = O.sigma_at(np.arange(g.N[d], dtype=float), d, g)
        assert np.all(s[lo:hi + 1] == 0) and s[0] > 0 and s[-1] > 0
        assert g.pad[d] >= 0 and (g.N[d] + 1) % 4 == 0


# ---------------------------------------------------------------------------
# Physics: free-space Green's functions (Sec. 5.1, analytic comparison)
# ---------------------------------------------------------------------------

def _green2d_error(h, Lx=1000.0, Lz=600.0, xs=300.0, zs=200.0, pml_m=200.0, f=10.0, v0=2000.0):
    nx, nz = int(round(Lx / h)) + 1, int(round(Lz / h)) + 1
    npml = int(round(pml_m / h))
    g = O.make_grid(2, (nx, 1, nz), h, (npml, 0, npml), v0)
    m = np.full(g.phys_shape, 1 / v0 ** 2)
    H = O.helmholtz_matrix(g, O.extend(g, m), 2 * np.pi * f)
    src = np.array([int(round(xs / h)) + nx * int(round(zs / h))])
    u = O.DirectSolver(H).solve(O.source_fields(g, src, np.ones((1, 1)))[0])
    u = u.reshape(g.shape)[npml:npml + nz, 0, npml:npml + nx]
    Z, X = np.meshgrid(np.arange(nz) * h, np.arange(nx) * h, indexing="ij")
    r = np.hypot(X - xs, Z - zs)
    sel = r > 150.0
    G = -0.25j * hankel1(0, 2 * np.pi * f / v0 * r[sel])
    return np.linalg.norm(u[sel] - G) / np.linalg.norm(G), u, G, sel


def test_green_2d_second_order():
    """(Lap + k^2) u = delta has the outgoing solution -(i/4) H0^(1)(k r).
    A non-square box with an off-centre source pins the axes; second-order
    convergence pins the stencil scale and the 1/h^2 source; a small error at
    all pins the outgoing sign of the damping layer."""
    e1, *_ = _green2d_error(20.0)
    e2, u, G, sel = _green2d_error(10.0)
    assert e2 < 0.05
    assert e1 / e2 > 3.3
    # phase: correlation with the analytic field is ~1 (a conjugated or
    # negated solution would give ~-1 or ~0)
    c = np.vdot(G, u[sel]) / (np.linalg.norm(G) * np.linalg.norm(u[sel]))
    assert c.real > 0.99


def _green3d_error(h, L=(400.0, 320.0, 480.0), xs=(160.0, 160.0, 200.0), pml_m=160.0, f=10.0,
                   v0=2000.0):
    n = tuple(int(round(l / h)) + 1 for l in L)
    npml = int(round(pml_m / h))
    g = O.make_grid(3, n, h, (npml,) * 3, v0)
    m = np.full(g.phys_shape, 1 / v0 ** 2)
    H = O.helmholtz_matrix(g, O.extend(g, m), 2 * np.pi * f)
    s = [int(round(c / h)) for c in xs]
    src = np.array([s[0] + n[0] * (s[1] + n[1] * s[2])])
    q = O.source_fields(g, src, np.ones((1, 1)))[0]
    if g.size < 12000:
        u = O.DirectSolver(H).solve(q)
    else:
        u, _, _ = O.gmres(H, q, tol=1e-8, restart=80)
    u = u.reshape(g.shape)[npml:npml + n[2], npml:npml + n[1], npml:npml + n[0]]
    Z, Y, X = np.meshgrid(*(np.arange(k) * h for k in (n[2], n[1], n[0])), indexing="ij")
    r = np.sqrt((X - s[0] * h) ** 2 + (Y - s[1] * h) ** 2 + (Z - s[2] * h) ** 2)
    sel = r > 80.0
    k = 2 * np.pi * f / v0
    G = -np.exp(1j * k * r[sel]) / (4 * np.pi * r[sel])
    err = np.linalg.norm(u[sel] - G) / np.linalg.norm(G)
    corr = (np.vdot(G, u[sel]) / (np.linalg.norm(G) * np.linalg.norm(u[sel]))).real
    return err, corr


def test_green_3d_second_order():
    """(Lap + k^2) u = delta in 3D has the outgoing solution -exp(ikr)/(4 pi r)
    (the paper prints it without the minus sign; the sign follows from its 2D
    formula and from the source term of eq. (helmholtz))."""
    e1, _ = _green3d_error(40.0)
    e2, c2 = _green3d_error(20.0)
    assert e2 < 0.10
    assert e1 / e2 > 3.5
    assert c2 > 0.99


# ---------------------------------------------------------------------------
# Solvers
# ---------------------------------------------------------------------------

def _small_3d_problem(seed=0, n=(7, 6, 8), npml=(3, 3, 3), h=20.0, f=6.0):
    rng = np.random.default_rng(seed)
    g = O.make_grid(3, n, h, npml, 3000.0)
    mp = 1 / rng.uniform(1500, 3000, size=g.phys_shape) ** 2
    H = O.helmholtz_matrix(g, O.extend(g, mp), 2 * np.pi * f)
    return g, mp, H, rng


def test_gmres_equals_direct_and_dense():
    g, mp, H, rng = _small_3d_problem()
    b = rng.standard_normal(g.size) + 1j * rng.standard_normal(g.size)
    xd = O.DirectSolver(H).solve(b)
    xg, it, rel = O.gmres(H, b, tol=1e-13, restart=30)
    xdense = np.linalg.solve(H.toarray(), b)
    assert rel <= 1e-13 and it > 0
    assert np.linalg.norm(xg - xdense) <= 1e-10 * np.linalg.norm(xdense)
    assert np.linalg.norm(xd - xdense) <= 1e-12 * np.linalg.norm(xdense)
    # adjoint solves against the explicit conjugate transpose
    HH = H.toarray().conj().T
    ya = O.DirectSolver(H).solve_adjoint(b)
    yg = O.GmresSolver(H, tol=1e-13, restart=30).solve_adjoint(b)
    assert np.linalg.norm(HH @ ya - b) <= 1e-12 * np.linalg.norm(b)
    assert np.linalg.norm(HH @ yg - b) <= 1e-12 * np.linalg.norm(b)


def test_adjoint_identity_of_solves():
    """<H^-1 x, y> = <x, H^-H y> (the adjoint test of Sec. 5.1 applied to the
    solution operator), vectors zero in the layer as in the paper."""
    g, mp, H, rng = _small_3d_problem(seed=3)
    inside = np.zeros(g.shape, dtype=bool)
    p = g.npml
    inside[p[2] + 1:p[2] + g.n[2] - 1, p[1] + 1:p[1] + g.n[1] - 1, p[0] + 1:p[0] + g.n[0] - 1] = True
    x = (rng.standard_normal(g.size) + 1j * rng.standard_normal(g.size)) * inside.ravel()
    y = (rng.standard_normal(g.size) + 1j * rng.standard_normal(g.size)) * inside.ravel()
    S = O.DirectSolver(H)
    lhs = np.vdot(y, S.solve(x))
    rhs = np.vdot(S.solve_adjoint(y), x)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


# ---------------------------------------------------------------------------
# Extension E and E^T
# ---------------------------------------------------------------------------

def test_extension_adjoint_pair():
    g = O.make_grid(3, (5, 4, 6), 10.0, (2, 3, 1), 2000.0, levels=2)
    rng = np.random.default_rng(1)
    m = rng.standard_normal(g.phys_shape)
    gc = rng.standard_normal(g.shape)
    assert abs(np.sum(O.extend(g, m) * gc) - np.sum(m * O.extend_adjoint(g, gc))) < 1e-12
    # E^T 1 counts how many computational nodes copy each physical node
    cnt = O.extend_adjoint(g, np.ones(g.shape))
    lo_x, hi_x = g.npml[0] + 1, g.npml[0] + g.pad[0] + 1
    lo_y, hi_y = g.npml[1] + 1, g.npml[1] + g.pad[1] + 1
    lo_z, hi_z = g.npml[2] + 1, g.npml[2] + g.pad[2] + 1
    assert cnt[2, 2, 2] == 1
    assert cnt[0, 0, 0] == lo_x * lo_y * lo_z
    assert cnt[-1, -1, -1] == hi_x * hi_y * hi_z
    assert cnt[0, 2, 2] == lo_z and cnt[2, 2, -1] == hi_x
    assert cnt.sum() == g.size
    # constants extend to constants
    assert np.all(O.extend(g, np.full(g.phys_shape, 3.5)) == 3.5)


# ---------------------------------------------------------------------------
# Misfit and gradient
# ---------------------------------------------------------------------------

def _toy_2d(seed=5, n=31, h=25.0, npml=8, freqs=(4.0, 6.0)):
    rng = np.random.default_rng(seed)
    g = O.make_grid(2, (n, 1, n), h, (npml, 0, npml), 2500.0)
    zz, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    v = 2000 + 400 * np.exp(-((xx - n / 2) ** 2 + (zz - n / 2) ** 2) / (2 * (n / 6) ** 2))
    m_true = (1 / v ** 2)[:, None, :]
    m0 = np.full(g.phys_shape, 1 / 2000 ** 2)
    src = np.array([3 + n * 2, n // 2 + n * 2, n - 4 + n * 2], dtype=np.int32)
    Q = np.eye(3, dtype=complex)
    Q[1, 0] = 0.5 - 0.25j  # one source combines two locations
    rec = (np.arange(n) + n * 2).astype(np.int32)
    wav = np.array([1.0 + 0.0j, 0.7 - 0.4j][:len(freqs)])
    _, d = O.forward(g, m_true, freqs, src, Q, rec, wavelet=wav)
    return g, m_true, m0, np.array(freqs), src, Q, rec, wav, d, rng


def _richardson_fd(f, m, dm, t):
    """Central differences at steps t and t/2 combined to cancel the t^2 term."""
    def cd(s):
        return (f(m + s * dm) - f(m - s * dm)) / (2 * s)
    return (4 * cd(t / 2) - cd(t)) / 3


def test_misfit_vanishes_at_true_model():
    g, m_true, m0, freqs, src, Q, rec, wav, d, _ = _toy_2d()
    f, gr = O.misfit_and_gradient(g, m_true, freqs, src, Q, rec, d, wavelet=wav)
    assert f == pytest.approx(0.0, abs=1e-28)
    assert np.all(gr == 0.0)
    f0 = O.misfit(g, m0, freqs, src, Q, rec, d, wavelet=wav)
    assert f0 > 0


def test_misfit_hand_computed():
    """f = 1/2 sum |P u - d|^2: perturb the observed data by known offsets."""
    g, m_true, m0, freqs, src, Q, rec, wav, d, _ = _toy_2d()
    d2 = d.copy()
    d2[0, 1, 4] += 3.0 - 4.0j      # |.|^2 = 25
    d2[1, 2, 7] += 1.0 + 1.0j      # |.|^2 = 2
    f = O.misfit(g, m_true, freqs, src, Q, rec, d2, wavelet=wav)
    assert f == pytest.approx(13.5, rel=1e-12)
    mask = np.array([[True, True, True], [True, True, False]])
    fm = O.misfit(g, m_true, freqs, src, Q, rec, d2, wavelet=wav, mask=mask)
    assert fm == pytest.approx(12.5, rel=1e-12)


def test_gradient_matches_central_differences_2d():
    """<grad f, dm> against central differences of f along random directions,
    including directions supported on the boundary nodes (which pins E^T)."""
    g, m_true, m0, freqs, src, Q, rec, wav, d, rng = _toy_2d()
    mask = np.array([[True, False, True], [True, True, True]])
    f0, gr = O.misfit_and_gradient(g, m0, freqs, src, Q, rec, d, wavelet=wav, mask=mask)
    for k in range(4):
        dm = rng.standard_normal(g.phys_shape) * m0
        if k == 3:
            dm = np.zeros(g.phys_shape)
            dm[0, 0, :] = m0[0, 0, :]
            dm[:, 0, -1] = m0[:, 0, -1]
        fd = _richardson_fd(lambda m: O.misfit(g, m, freqs, src, Q, rec, d, wavelet=wav, mask=mask),
                            m0, dm, 1e-3)
        an = np.sum(gr * dm)
        assert abs(fd - an) <= 1e-7 * abs(an)


def test_taylor_remainders():
    """f(m + t dm) - f(m) = O(t) and f(m + t dm) - f(m) - t <g, dm> = O(t^2) (Sec. 5.1)."""
    g, m_true, m0, freqs, src, Q, rec, wav, d, rng = _toy_2d(seed=9)
    f0, gr = O.misfit_and_gradient(g, m0, freqs, src, Q, rec, d, wavelet=wav)
    dm = rng.standard_normal(g.phys_shape) * m0
    ts = [2e-4 / 2 ** k for k in range(4)]
    e1, e2 = [], []
    for t in ts:
        ft = O.misfit(g, m0 + t * dm, freqs, src, Q, rec, d, wavelet=wav)
        e1.append(abs(ft - f0))
        e2.append(abs(ft - f0 - t * np.sum(gr * dm)))
    s1 = np.log2(np.array(e1[:-1]) / np.array(e1[1:]))
    s2 = np.log2(np.array(e2[:-1]) / np.array(e2[1:]))
    assert np.all(np.abs(s1 - 1) < 0.15)
    assert np.all(np.abs(s2 - 2) < 0.15)


def test_gradient_3d_central_differences_gmres():
    """3D, two frequencies, the oracle's iterative solver path."""
    rng = np.random.default_rng(11)
    n, h = (7, 6, 5), 25.0
    g = O.make_grid(3, n, h, (3, 3, 3), 3000.0)
    v = rng.uniform(1800, 2600, size=g.phys_shape)
    mt = 1 / v ** 2
    m0 = np.full(g.phys_shape, 1 / 2200 ** 2)
    src = np.array([1 + 7 * (2 + 6 * 1), 5 + 7 * (3 + 6 * 1)], dtype=np.int32)
    Q = np.eye(2, dtype=complex)
    rec = np.arange(7 * 6, dtype=np.int32)
    freqs = np.array([5.0, 8.0])
    kw = dict(solver="gmres", tol=1e-14, restart=40)
    _, d = O.forward(g, mt, freqs, src, Q, rec, **kw)
    f0, gr = O.misfit_and_gradient(g, m0, freqs, src, Q, rec, d, **kw)
    for _ in range(2):
        dm = rng.standard_normal(g.phys_shape) * m0
        fd = _richardson_fd(lambda m: O.misfit(g, m, freqs, src, Q, rec, d, **kw), m0, dm, 1e-3)
        an = np.sum(gr * dm)
        assert abs(fd - an) <= 1e-7 * abs(an)


# ---------------------------------------------------------------------------
# Inter-grid transfers (Sec. 4, linear interpolation and its adjoint)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,N", [(3, (9, 7, 11)), (2, (13, 1, 9))])
def test_prolongation_reproduces_linear_functions(dim, N):
    """P applied to coarse samples of a linear function returns its fine samples
    at every fine node whose interpolation stencil stays inside the walls."""
    P = O.prolongation(N, dim)
    Nx, Ny, Nz = N
    cx, cy, cz = (Nx - 1) // 2, (Ny - 1) // 2 if dim == 3 else Ny, (Nz - 1) // 2

    def lin(x, y, z):
        return 0.3 + 1.7 * x - 0.4 * y + 2.2 * z

    # coarse node j sits at fine coordinate 2j+1
    Zc, Yc, Xc = np.meshgrid(2 * np.arange(cz) + 1,
                             (2 * np.arange(cy) + 1) if dim == 3 else np.arange(Ny),
                             2 * np.arange(cx) + 1, indexing="ij")
    Zf, Yf, Xf = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    uf = (P @ lin(Xc, Yc, Zc).ravel()).reshape(Nz, Ny, Nx)
    inner = (Xf > 0) & (Xf < Nx - 1) & (Zf > 0) & (Zf < Nz - 1)
    if dim == 3:
        inner &= (Yf > 0) & (Yf < Ny - 1)
    assert np.allclose(uf[inner], lin(Xf, Yf, Zf)[inner], rtol=0, atol=1e-12)


def test_restriction_is_scaled_adjoint_and_averages():
    N, dim = (9, 7, 11), 3
    P, R = O.prolongation(N, dim), O.restriction(N, dim)
    rng = np.random.default_rng(2)
    xf = rng.standard_normal(P.shape[0])
    xc = rng.standard_normal(P.shape[1])
    assert abs(np.dot(R @ xf, xc) - 2.0 ** -dim * np.dot(xf, P @ xc)) < 1e-12
    # full weighting: weights of every coarse node sum to one
    assert np.allclose(R @ np.ones(P.shape[0]), 1.0)
