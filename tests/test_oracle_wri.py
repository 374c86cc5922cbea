"""Pins of the oracle's Waveform Reconstruction Inversion (Sec. 3 penalty
method, Appendix B): the field from the normal equations equals the field
from H / H^H solves plus a receiver-space system (push-through identity); as
lambda grows the field tends to H^{-1} q and the objective to the FWI misfit,
both as lambda^-2; the variable-projection gradient matches central
differences of the objective."""
import numpy as np
import pytest

from oracle import helmholtz as O

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


@pytest.fixture(scope="module")
def wri():
    rng = np.random.default_rng(71)
    n, h = (21, 1, 17), 20.0
    g = O.make_grid(2, n, h, (5, 0, 5), 2500.0)
    m = 1 / (2000 + 400 * rng.random(g.n_phys)) ** 2
    src = np.array([2 * 21 + 5, 2 * 21 + 15], dtype=np.int32)
    Q = np.eye(2, dtype=complex)
    rec = (np.arange(21) + 21).astype(np.int32)
    freqs = [6.0, 8.0]
    _, D = O.forward(g, m, freqs, src, Q, rec, want_fields=False)
    d = D * (1 + 0.2 * rng.standard_normal(D.shape))
    return dict(g=g, m=m, src=src, Q=Q, rec=rec, freqs=freqs, d=d, rng=rng)


def _ops(p, k=0):
    g = p["g"]
    H = O.helmholtz_matrix(g, O.extend(g, p["m"]), 2 * np.pi * p["freqs"][k])
    return H, O.receiver_matrix(g, p["rec"]), O.source_fields(g, p["src"], p["Q"])


@pytest.mark.parametrize("lam", [1e-1, 1e2, 1e4])
def test_field_from_normal_equations_equals_dataspace_route(wri, lam):
    H, P, q = _ops(wri)
    u = O.wri_field(H, P, q[0], wri["d"][0, 0], lam)
    u2 = O.wri_field_dataspace(H, P, q[0], wri["d"][0, 0], lam)
    assert np.linalg.norm(u - u2) <= 1e-10 * np.linalg.norm(u)


def test_large_penalty_recovers_the_pde_solution_and_the_fwi_misfit(wri):
    p = wri
    H, P, q = _ops(p)
    u0 = O.DirectSolver(H).solve(q[0])
    e = [np.linalg.norm(O.wri_field(H, P, q[0], p["d"][0, 0], lam) - u0) / np.linalg.norm(u0) for lam in (1e5, 1e6)]
    assert e[1] < 1e-5 and e[0] / e[1] > 50  # lambda^-2
    f_fwi, _ = O.misfit_and_gradient(p["g"], p["m"], p["freqs"], p["src"], p["Q"], p["rec"], p["d"])
    f_wri, _ = O.wri_misfit_and_gradient(p["g"], p["m"], p["freqs"], p["src"], p["Q"], p["rec"], p["d"], 1e6)
    assert abs(f_wri - f_fwi) <= 1e-5 * f_fwi


def test_wri_gradient_matches_central_differences(wri):
    p = wri
    lam = 1e4
    dm = p["rng"].standard_normal(p["g"].n_phys) * 1e-8
    _, gr = O.wri_misfit_and_gradient(p["g"], p["m"], p["freqs"], p["src"], p["Q"], p["rec"], p["d"], lam)

    def f(t):
        return O.wri_misfit_and_gradient(p["g"], p["m"] + t * dm, p["freqs"], p["src"], p["Q"], p["rec"], p["d"],
                                         lam)[0]

    def cd(t):
        return (f(t) - f(-t)) / (2 * t)

    fd = (4 * cd(0.01) - cd(0.02)) / 3
    assert abs(fd - np.dot(gr.ravel(), dm)) <= 1e-6 * abs(fd)
