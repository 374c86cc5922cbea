"""Plant plausible mistakes in the oracle (on the CPU, by monkeypatching) and
check that the pins of test_oracle.py catch each of them."""
import numpy as np
import pytest

from oracle import helmholtz as O
import tests.test_oracle as T


def test_pin_catches_incoming_damping_sign(monkeypatch):
    """eta = 1 - i sigma/w (wrong sign for the exp(-iwt) convention) amplifies
    instead of absorbing: the Green's function comparison must fail."""
    real = O.sigma_at
    monkeypatch.setattr(O, "sigma_at", lambda t, d, g: -real(t, d, g))
    e2, *_ = T._green2d_error(10.0)
    assert e2 > 0.2


def test_pin_catches_dropped_mass_term(monkeypatch):
    real = O.helmholtz_matrix

    def no_mass(g, m_comp, omega):
        return real(g, np.zeros_like(m_comp), omega)

    monkeypatch.setattr(O, "helmholtz_matrix", no_mass)
    with pytest.raises(AssertionError):
        T.test_dirichlet_eigenpairs(3, (5, 6, 7))


def test_pin_catches_swapped_axes(monkeypatch):
    real = O.axis_coefficients

    def swapped(g, d, omega):
        return real(g, {0: 2, 2: 0}.get(d, d), omega)

    monkeypatch.setattr(O, "axis_coefficients", swapped)
    with pytest.raises(Exception):
        T.test_operator_pointwise_from_stretched_derivative()


def test_pin_catches_plain_restriction_instead_of_extension_adjoint(monkeypatch):
    """Mapping the gradient to the physical grid by cropping (instead of E^T)
    breaks the finite-difference check for boundary-supported directions."""
    def crop(g, g_comp):
        gc = np.asarray(g_comp).reshape(g.shape)
        p, n = g.npml, g.n
        return gc[p[2]:p[2] + n[2], p[1]:p[1] + n[1], p[0]:p[0] + n[0]].copy()

    monkeypatch.setattr(O, "extend_adjoint", crop)
    with pytest.raises(AssertionError):
        T.test_gradient_matches_central_differences_2d()


def test_pin_catches_conjugated_gradient(monkeypatch):
    """Using Re(u v) instead of Re(conj(u) v) must fail the FD check."""
    real_solver = O.DirectSolver

    class ConjAdjoint(real_solver):
        def solve_adjoint(self, b):
            return np.conj(super().solve_adjoint(b))

    monkeypatch.setattr(O, "DirectSolver", ConjAdjoint)
    with pytest.raises(AssertionError):
        T.test_gradient_matches_central_differences_2d()


# ---------------------------------------------------------------------------
# Preconditioner pins (tests/test_oracle_precond.py)
# ---------------------------------------------------------------------------

import tests.test_oracle_precond as TP  # noqa: E402


def test_pin_catches_coarse_spacing_not_doubled(monkeypatch):
    """Rediscretising the coarse level at spacing h instead of 2h."""
    real = O.level_axis_coefficients

    def fine_spacing(g, d, omega, level):
        cm, cp, cd = real(g, d, omega, level)
        f = float(1 << level) ** 2
        return cm * f, cp * f, cd * f

    monkeypatch.setattr(O, "level_axis_coefficients", fine_spacing)
    with pytest.raises(AssertionError):
        TP.test_coarse_operator_is_second_order_consistent()


def test_pin_catches_coarse_node_offset(monkeypatch):
    """Coarse node j placed on fine node 2j (instead of 2j+1) shifts the
    damping profile; the smooth-field consistency check must fail."""
    real_sigma = O.sigma_at

    def shifted_level(g, d, omega, level):
        q = 1 << level
        Nl = O.level_N(g, level)[d]
        t = np.arange(Nl, dtype=np.float64) * q
        a = 1.0 / (1.0 + 1j * real_sigma(t, d, g) / omega)
        bm = 1.0 / (1.0 + 1j * real_sigma(t - 0.5 * q, d, g) / omega)
        bp = 1.0 / (1.0 + 1j * real_sigma(t + 0.5 * q, d, g) / omega)
        hl = q * g.h
        cm, cp = a * bm / hl ** 2, a * bp / hl ** 2
        return cm, cp, -(cm + cp)

    monkeypatch.setattr(O, "level_axis_coefficients", shifted_level)
    with pytest.raises(AssertionError):
        TP.test_coarse_operator_is_second_order_consistent()


def test_pin_catches_subtracted_coarse_correction(monkeypatch):
    """x <- x - P x_c (wrong sign of the coarse-grid correction)."""
    real_prol = O.prolongation
    monkeypatch.setattr(O, "prolongation", lambda N, dim: -real_prol(N, dim))
    with pytest.raises(AssertionError):
        TP.test_vcycle_is_an_effective_preconditioner(False)


def test_pin_catches_unscaled_restriction(monkeypatch):
    """R = P^T without the 2^-dim factor over-weights the coarse correction."""
    real_prol = O.prolongation
    monkeypatch.setattr(O, "restriction", lambda N, dim: real_prol(N, dim).T.tocsr())
    with pytest.raises(AssertionError):
        TP.test_vcycle_is_an_effective_preconditioner(False)


def test_pin_catches_undamped_sign_flip_in_jacobi(monkeypatch):
    """z <- z - w D^{-1}(b - H z) diverges from the solution."""
    def wrong(H, b, omega_j, sweeps):
        D = H.diagonal()
        z = np.zeros_like(b)
        for _ in range(sweeps):
            z = z - omega_j * (b - H @ z) / D
        return z

    monkeypatch.setattr(O, "jacobi_precond", wrong)
    with pytest.raises(AssertionError):
        TP.test_jacobi_sweeps_converge_to_the_solution_on_a_dominant_diagonal()


# ---------------------------------------------------------------------------
# Linearised-modelling pins (tests/test_oracle_born.py)
# ---------------------------------------------------------------------------

import inspect  # noqa: E402

import tests.test_oracle_born as TB  # noqa: E402


def _born_problem():
    """The problem of test_oracle_born's fixture, built directly."""
    return inspect.unwrap(TB.prob)()


def test_pin_catches_born_source_sign(monkeypatch):
    """H du = +T dm (dropped minus sign of eq. (dU2))."""
    p = _born_problem()
    real_born = O.born
    monkeypatch.setattr(O, "born", lambda *a, **k: -real_born(*a, **k))
    with pytest.raises(AssertionError):
        TB.test_born_matches_central_differences(p)


def test_pin_catches_unconjugated_state_in_adjoint(monkeypatch):
    """T^* v computed as w^2 u v instead of w^2 conj(u) v."""
    p = _born_problem()

    def born_adjoint_noconj(g, m_phys, freqs_hz, src_idx, Q, rec_idx, dD, wavelet=None, mask=None, **kw):
        mc = O.extend(g, m_phys)
        gc = np.zeros(g.size)
        for k, fr in enumerate(freqs_hz):
            om = 2 * np.pi * fr
            w = 1.0 if wavelet is None else wavelet[k]
            S = O.DirectSolver(O.helmholtz_matrix(g, mc, om))
            q = O.source_fields(g, src_idx, np.asarray(Q), w)
            for s_ in range(np.asarray(Q).shape[1]):
                u = S.solve(q[s_])
                v = S.solve_adjoint(-O.spread_receivers(g, np.asarray(dD)[k, s_], rec_idx))
                gc += om * om * np.real(u * v)
        return O.extend_adjoint(g, gc)

    monkeypatch.setattr(O, "born_adjoint", born_adjoint_noconj)
    with pytest.raises(AssertionError):
        TB.test_adjoint_identity(p)


def test_pin_catches_zero_padded_perturbation(monkeypatch):
    """Extending dm by zeros in the layers (instead of E) changes J dm there."""
    p = _born_problem()
    real_extend = O.extend

    def zero_extend(g, x):
        out = np.zeros(g.shape)
        n, pm = g.n, g.npml
        out[pm[2]:pm[2] + n[2], pm[1]:pm[1] + n[1], pm[0]:pm[0] + n[0]] = np.asarray(x).reshape(g.phys_shape)
        return out

    real_born = O.born

    def born_zero_pad(g, m_phys, *a, **k):
        # m itself is extended by E; only the perturbation is zero-padded
        calls = {"n": 0}

        def ext(gg, x):
            calls["n"] += 1
            return real_extend(gg, x) if calls["n"] == 1 else zero_extend(gg, x)

        monkeypatch.setattr(O, "extend", ext)
        try:
            return real_born(g, m_phys, *a, **k)
        finally:
            monkeypatch.setattr(O, "extend", real_extend)

    monkeypatch.setattr(O, "born", born_zero_pad)
    with pytest.raises(AssertionError):
        TB.test_born_matches_central_differences(p)


def test_pin_catches_plus_sign_of_dh_adjoint_term(monkeypatch):
    """dv = H^{-H}(+w^2 dm v - P^T P du) (the other sign) fails the gradient
    central-difference check."""
    p = _born_problem()

    def hessvec_plus(g, m_phys, freqs_hz, src_idx, Q, rec_idx, d_obs, dm_phys, wavelet=None, mask=None, **kw):
        mc = O.extend(g, m_phys)
        dmc = O.extend(g, dm_phys).ravel()
        gc = np.zeros(g.size)
        Qa = np.asarray(Q)
        for k, fr in enumerate(freqs_hz):
            om = 2 * np.pi * fr
            w = 1.0 if wavelet is None else wavelet[k]
            S = O.DirectSolver(O.helmholtz_matrix(g, mc, om))
            q = O.source_fields(g, src_idx, Qa, w)
            for s_ in range(Qa.shape[1]):
                u = S.solve(q[s_])
                r = O.sample_receivers(g, u, rec_idx) - np.asarray(d_obs)[k, s_]
                v = S.solve_adjoint(-O.spread_receivers(g, r, rec_idx))
                du = S.solve(-om * om * dmc * u)
                dv = S.solve_adjoint(om * om * dmc * v
                                     - O.spread_receivers(g, O.sample_receivers(g, du, rec_idx), rec_idx))
                gc += om * om * np.real(np.conj(du) * v + np.conj(u) * dv)
        return O.extend_adjoint(g, gc)

    monkeypatch.setattr(O, "hessvec", hessvec_plus)
    with pytest.raises(AssertionError):
        TB.test_hessvec_matches_central_differences_of_the_gradient(p)


# ---------------------------------------------------------------------------
# 2.5D pins (tests/test_oracle_25d.py)
# ---------------------------------------------------------------------------

import tests.test_oracle_25d as T25  # noqa: E402


def test_pin_catches_wrong_sign_of_ky_shift(monkeypatch):
    """H(k_y) = H + k_y^2 I (the y derivative's sign flipped)."""
    real = O.helmholtz_matrix
    import scipy.sparse as sp_

    def plus(g, m_comp, omega, ky):
        return sp_.csr_matrix(real(g, m_comp, omega) + ky * ky * sp_.identity(g.size, dtype=np.complex128))

    monkeypatch.setattr(O, "helmholtz_matrix_25d", plus)
    with pytest.raises(AssertionError):
        T25.test_25d_sum_reproduces_the_3d_greens_function()


def test_pin_catches_unweighted_adjoint_source(monkeypatch):
    """The gradient evaluated without the quadrature weights c_i."""
    real = O.misfit_and_gradient_25d

    def unweighted(g, m_phys, freqs_hz, ky, ck, *a, **k):
        f, _ = real(g, m_phys, freqs_hz, ky, ck, *a, **k)
        _, gr = real(g, m_phys, freqs_hz, ky, np.ones_like(ck), *a, **k)
        return f, gr

    monkeypatch.setattr(O, "misfit_and_gradient_25d", unweighted)
    with pytest.raises(AssertionError):
        T25.test_25d_gradient_matches_central_differences()


# ---------------------------------------------------------------------------
# WRI pins (tests/test_oracle_wri.py)
# ---------------------------------------------------------------------------

import tests.test_oracle_wri as TW  # noqa: E402


def test_pin_catches_wri_gradient_without_penalty_weight(monkeypatch):
    """grad f = T^*(H u - q) without the lambda^2 factor."""
    real = O.wri_misfit_and_gradient

    def no_lam2(g, m_phys, freqs_hz, src_idx, Q, rec_idx, d_obs, lam):
        f, gr = real(g, m_phys, freqs_hz, src_idx, Q, rec_idx, d_obs, lam)
        return f, gr / (lam * lam)

    monkeypatch.setattr(O, "wri_misfit_and_gradient", no_lam2)
    with pytest.raises(AssertionError):
        TW.test_wri_gradient_matches_central_differences(inspect.unwrap(TW.wri)())
