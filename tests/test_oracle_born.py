"""Pins of the oracle's linearised modelling (Appendix A, Table derivstuff):
the adjoint identity of J, J dm against central differences of the forward
data, the misfit gradient as J^T applied to the data residual, and symmetry /
positivity of the Gauss-Newton product."""
import numpy as np
import pytest

from oracle import helmholtz as O

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


@pytest.fixture(scope="module")
def prob():
    rng = np.random.default_rng(31)
    n, h, npml = (23, 1, 19), 20.0, (6, 0, 6)
    g = O.make_grid(2, n, h, npml, 2500.0)
    v = 2000.0 + 400.0 * rng.random(g.n_phys)
    m = 1.0 / v ** 2
    src, Q = np.array([2 * 23 + 5, 2 * 23 + 17], dtype=np.int32), np.eye(2, dtype=np.complex128)
    rec = np.arange(23, dtype=np.int32) + 23  # row z = 1
    freqs = np.array([6.0, 9.0])
    wav = np.array([1.0 + 0.3j, 0.7 - 0.2j])
    dm = rng.standard_normal(g.n_phys) * 1e-8
    dD = rng.standard_normal((2, 2, len(rec))) + 1j * rng.standard_normal((2, 2, len(rec)))
    return dict(g=g, m=m, src=src, Q=Q, rec=rec, freqs=freqs, wav=wav, dm=dm, dD=dD, rng=rng)


def _J(p, dm, mask=None):
    return O.born(p["g"], p["m"], p["freqs"], p["src"], p["Q"], p["rec"], dm, p["wav"], mask)


def _JT(p, dD, mask=None):
    return O.born_adjoint(p["g"], p["m"], p["freqs"], p["src"], p["Q"], p["rec"], dD, p["wav"], mask).ravel()


def test_adjoint_identity(prob):
    """Re<J dm, dD> = <dm, J^T dD> (the paper's adjoint test for J, Sec. 5.1)."""
    lhs = float(np.real(np.vdot(_J(prob, prob["dm"]), prob["dD"])))
    rhs = float(np.dot(prob["dm"], _JT(prob, prob["dD"])))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_born_matches_central_differences(prob):
    """J dm = dD/dt of the forward data along dm (Richardson-extrapolated
    central differences)."""
    p = prob

    def data(t):
        _, D = O.forward(p["g"], p["m"] + t * p["dm"], p["freqs"], p["src"], p["Q"], p["rec"], p["wav"],
                         want_fields=False)
        return D

    def cd(t):
        return (data(t) - data(-t)) / (2 * t)

    t = 0.5
    fd = (4 * cd(t / 2) - cd(t)) / 3
    J = _J(p, p["dm"])
    assert np.linalg.norm(J - fd) / np.linalg.norm(J) < 1e-6


def test_misfit_gradient_is_adjoint_jacobian_of_the_residual(prob):
    """grad f = J^T (P_r u - d): two independent code paths of Appendix A."""
    p = prob
    _, D = O.forward(p["g"], p["m"], p["freqs"], p["src"], p["Q"], p["rec"], p["wav"], want_fields=False)
    d_obs = D + 0.1 * p["dD"]
    _, gr = O.misfit_and_gradient(p["g"], p["m"], p["freqs"], p["src"], p["Q"], p["rec"], d_obs, p["wav"])
    jt = _JT(p, D - d_obs)
    assert np.linalg.norm(gr.ravel() - jt) <= 1e-12 * np.linalg.norm(gr)


def test_gauss_newton_is_symmetric_positive(prob):
    p = prob
    a = p["dm"]
    b = p["rng"].standard_normal(p["g"].n_phys) * 1e-8
    Ha = O.gauss_newton_hessvec(p["g"], p["m"], p["freqs"], p["src"], p["Q"], p["rec"], a, p["wav"]).ravel()
    Hb = O.gauss_newton_hessvec(p["g"], p["m"], p["freqs"], p["src"], p["Q"], p["rec"], b, p["wav"]).ravel()
    assert abs(np.dot(a, Hb) - np.dot(Ha, b)) <= 1e-12 * abs(np.dot(a, Hb))
    Ja = _J(p, a)
    assert np.dot(a, Ha) > 0
    assert abs(np.dot(a, Ha) - np.vdot(Ja, Ja).real) <= 1e-12 * np.dot(a, Ha)


def test_mask_drops_pairs(prob):
    p = prob
    mask = np.array([[1, 0], [0, 1]], dtype=np.uint8)
    J = _J(p, p["dm"], mask)
    assert np.all(J[0, 1] == 0) and np.all(J[1, 0] == 0)
    full = _J(p, p["dm"])
    assert np.allclose(J[0, 0], full[0, 0]) and np.allclose(J[1, 1], full[1, 1])
    dD = p["dD"] * mask[..., None]
    assert np.allclose(_JT(p, p["dD"], mask), _JT(p, dD), rtol=1e-12, atol=0)


# ---------------------------------------------------------------------------
# Full Hessian-vector product (Table derivstuff, last row)
# ---------------------------------------------------------------------------

def _dobs(p, scale=0.2):
    _, D = O.forward(p["g"], p["m"], p["freqs"], p["src"], p["Q"], p["rec"], p["wav"], want_fields=False)
    return D + scale * p["dD"]


def _H(p, d_obs, dm):
    return O.hessvec(p["g"], p["m"], p["freqs"], p["src"], p["Q"], p["rec"], d_obs, dm, p["wav"]).ravel()


def test_hessvec_matches_central_differences_of_the_gradient(prob):
    p = prob
    d_obs = _dobs(p)

    def grad(t):
        _, g = O.misfit_and_gradient(p["g"], p["m"] + t * p["dm"], p["freqs"], p["src"], p["Q"], p["rec"], d_obs,
                                     p["wav"])
        return g.ravel()

    def cd(t):
        return (grad(t) - grad(-t)) / (2 * t)

    t = 0.5
    fd = (4 * cd(t / 2) - cd(t)) / 3
    Hdm = _H(p, d_obs, p["dm"])
    assert np.linalg.norm(Hdm - fd) / np.linalg.norm(Hdm) < 1e-6


def test_hessvec_is_symmetric(prob):
    """<dm1, H dm2> = <H dm1, dm2> (the paper's Hessian adjoint test, Sec. 5.1)."""
    p = prob
    d_obs = _dobs(p)
    a = p["dm"]
    b = p["rng"].standard_normal(p["g"].n_phys) * 1e-8
    Ha, Hb = _H(p, d_obs, a), _H(p, d_obs, b)
    assert abs(np.dot(a, Hb) - np.dot(Ha, b)) <= 1e-11 * abs(np.dot(a, Hb))


def test_hessvec_at_zero_residual_is_gauss_newton(prob):
    """With d = P_r u(m) the adjoint field vanishes and only J^T J dm remains."""
    p = prob
    H0 = _H(p, _dobs(p, 0.0), p["dm"])
    GN = O.gauss_newton_hessvec(p["g"], p["m"], p["freqs"], p["src"], p["Q"], p["rec"], p["dm"], p["wav"]).ravel()
    assert np.linalg.norm(H0 - GN) <= 1e-12 * np.linalg.norm(GN)
