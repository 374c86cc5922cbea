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
