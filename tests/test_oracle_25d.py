"""Pins of the oracle's 2.5D modelling (Sec. 3, 2.5D): the quadrature sum of
shifted 2D solves reproduces the 3D Green's function of a homogeneous medium
in the source's plane (second-order convergence in h), and the 2.5D misfit
gradient matches central differences."""
import numpy as np
import pytest

from oracle import helmholtz as O

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


def split_quadrature(kap, p, n1, n2):
    """(1/pi) int_0^{p kap} F(k) dk with the k = kap square-root singularity
    removed: k = kap sin(theta) on [0, kap], k = kap cosh(t) beyond."""
    t, w = np.polynomial.legendre.leggauss(n1)
    th, wth = 0.25 * np.pi * (t + 1), 0.25 * np.pi * w
    t2, w2 = np.polynomial.legendre.leggauss(n2)
    T = np.arccosh(p)
    tt, wt = 0.5 * T * (t2 + 1), 0.5 * T * w2
    k = np.concatenate([kap * np.sin(th), kap * np.cosh(tt)])
    c = np.concatenate([wth * kap * np.cos(th), wt * kap * np.sinh(tt)]) / np.pi
    return k, c


def _green_error(h, f=10.0, v=2000.0):
    n = int(round(1000.0 / h)) + 1
    npml = int(round(200.0 / h))
    g = O.make_grid(2, (n, 1, n), h, (npml, 0, npml), v)
    m = np.full(g.n_phys, 1 / v ** 2)
    c = n // 2
    src = np.array([c * n + c], dtype=np.int32)
    X, Z = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    R = np.hypot((X - c) * h, (Z - c) * h)
    sel = (R > 150) & (R < 400)
    rec = (Z * n + X)[sel].astype(np.int32)
    kap = 2 * np.pi * f / v
    ky, ck = split_quadrature(kap, 2.0, 20, 10)
    D, _ = O.forward_25d(g, m, [f], ky, ck, src, np.eye(1, dtype=complex), rec)
    r = R[sel]
    G3 = -np.exp(1j * kap * r) / (4 * np.pi * r)  # 3D Green's function (reading 11's sign)
    return np.linalg.norm(D[0, 0] - G3) / np.linalg.norm(G3)


def test_25d_sum_reproduces_the_3d_greens_function():
    e20, e10 = _green_error(20.0), _green_error(10.0)
    assert e10 < 0.05
    assert e20 / e10 > 3.0  # second order in h (4 in the limit)


def test_gauss_legendre_ky_integrates_polynomials():
    k, c = O.gauss_legendre_ky(3.0, 5)
    # (1/pi) int_0^3 k^4 dk = 3^5 / (5 pi)
    assert abs(np.dot(c, k ** 4) - 3.0 ** 5 / (5 * np.pi)) < 1e-12
    k, c = O.gauss_legendre_ky(2.0, 6, dy=0.7)
    # (1/pi) int_0^2 cos(0.7 k) dk = sin(1.4) / (0.7 pi)
    assert abs(np.sum(c) - np.sin(1.4) / (0.7 * np.pi)) < 1e-10


def test_25d_gradient_matches_central_differences():
    rng = np.random.default_rng(51)
    n, h = (15, 1, 13), 25.0
    g = O.make_grid(2, n, h, (5, 0, 5), 2500.0)
    v = 2000.0 + 400.0 * rng.random(g.n_phys)
    m = 1 / v ** 2
    src = np.array([2 * 15 + 4, 2 * 15 + 10], dtype=np.int32)
    Q = np.eye(2, dtype=np.complex128)
    rec = np.arange(15, dtype=np.int32) + 15
    freqs = [6.0, 8.0]
    ky, ck = O.gauss_legendre_ky(1.3 * 2 * np.pi * 8.0 / 2000.0, 3, dy=10.0)
    D, _ = O.forward_25d(g, m, freqs, ky, ck, src, Q, rec)
    d_obs = D + 0.3 * (rng.standard_normal(D.shape) + 1j * rng.standard_normal(D.shape)) * np.abs(D).mean()
    f0, gr = O.misfit_and_gradient_25d(g, m, freqs, ky, ck, src, Q, rec, d_obs)
    dm = rng.standard_normal(g.n_phys) * 1e-8

    def f(t):
        return O.misfit_and_gradient_25d(g, m + t * dm, freqs, ky, ck, src, Q, rec, d_obs)[0]

    def cd(t):
        return (f(t) - f(-t)) / (2 * t)

    fd = (4 * cd(0.01) - cd(0.02)) / 3
    assert abs(fd - np.dot(gr.ravel(), dm)) <= 1e-6 * abs(fd)
    assert f0 > 0
