"""helm_misfit_and_gradient_batch: several models of different sizes in one
call.  Each model's f and g must equal the oracle's, and the number of host
workers (how many models are in flight together) must not change the result."""
import numpy as np
import pytest
import torch

from oracle import helmholtz as O
from paper_1703_09268_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]

DEV = torch.device("cuda:0")
SIZES = [(12, 11, 13), (16, 14, 15), (20, 18, 17)]


@pytest.fixture(scope="module")
def helm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1703_09268_gb300 import helm as H
    return H


def T(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)


@pytest.fixture(scope="module")
def models():
    rng = np.random.default_rng(17)
    out = []
    for n in SIZES:
        g = O.make_grid(3, n, 50.0, (4, 4, 4), 4500.0, levels=2)
        v = synth.smooth_random_velocity(rng, n, sigma=3.0)
        mt = synth.slowness2(v)
        m0 = synth.slowness2(synth._gaussian_smooth(v, 3.0))
        nodes = [(2, 2, 2), (n[0] - 3, 3, 2), (4, n[1] - 3, 2), (n[0] // 2, n[1] // 2, 2)]
        src, Q = synth.point_sources(n, nodes)
        rec = synth.surface_receivers(n, 0)
        freqs = np.array([2.0, 3.5])
        _, d = O.forward(g, mt, freqs, src, Q, rec)
        f, gr = O.misfit_and_gradient(g, m0, freqs, src, Q, rec, d)
        out.append(dict(n=n, m0=m0, src=src, Q=Q, rec=rec, freqs=freqs, d=d, f=f, g=gr))
    return out


def requests(helm, models):
    reqs = []
    for mdl in models:
        plan = helm.Plan(helm.make_grid(3, mdl["n"], 50.0, (4, 4, 4), 4500.0, levels=2),
                         helm.default_opts(tol=1e-11, max_batch=3), device=DEV)
        reqs.append(dict(plan=plan, m_phys=T(mdl["m0"].ravel(), torch.float64), freqs_hz=mdl["freqs"],
                         src_idx=T(mdl["src"], torch.int32), Q=T(mdl["Q"], torch.complex128),
                         rec_idx=T(mdl["rec"], torch.int32), d_obs=T(mdl["d"], torch.complex128)))
    return reqs


def test_batch_matches_oracle_for_every_model(helm, models):
    res = helm.misfit_and_gradient_batch(requests(helm, models), nworkers=3)
    for mdl, (f, g, rep) in zip(models, res):
        assert abs(f.item() - mdl["f"]) <= 1e-8 * abs(mdl["f"])
        gg = g.cpu().numpy()
        assert np.linalg.norm(gg - mdl["g"].ravel()) <= 1e-8 * np.linalg.norm(mdl["g"])
        assert all(r["status"] == 0 for r in rep)


def test_worker_count_does_not_change_results(helm, models):
    r1 = helm.misfit_and_gradient_batch(requests(helm, models), nworkers=1)
    r3 = helm.misfit_and_gradient_batch(requests(helm, models), nworkers=3)
    for (f1, g1, _), (f3, g3, _) in zip(r1, r3):
        assert f1.item() == f3.item()
        assert torch.equal(g1, g3)
