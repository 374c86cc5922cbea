"""Failure reporting of bounded device waits, without a GPU fault: a wait on
an mbarrier phase that nothing completes gives up after its limit, the call
returns HELM_E_TIMEOUT, and the context keeps working (an operator apply right
after matches the oracle)."""
import time

import numpy as np
import pytest
import torch

from oracle import helmholtz as O

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def helm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1703_09268_gb300 import helm as H
    return H


def test_unsatisfied_wait_reports_timeout_and_context_survives(helm):
    t0 = time.perf_counter()
    code = helm.check_bounded_wait(DEV)
    dt = time.perf_counter() - t0
    assert code == helm.HELM_E_TIMEOUT
    assert 0.05 < dt < 10.0
    # the context is still usable
    n, npml = (12, 11, 10), (4, 4, 4)
    g = O.make_grid(3, n, 30.0, npml, 3000.0)
    rng = np.random.default_rng(5)
    mp = 1 / rng.uniform(1500, 4500, g.n_phys) ** 2
    x = rng.standard_normal((2, g.size)) + 1j * rng.standard_normal((2, g.size))
    plan = helm.Plan(helm.make_grid(3, n, 30.0, npml, 3000.0), helm.default_opts(precond=0), device=DEV)
    y = helm.helm_apply(plan, torch.as_tensor(mp, device=DEV), 4.0, torch.as_tensor(x, device=DEV))
    H = O.helmholtz_matrix(g, O.extend(g, mp), 2 * np.pi * 4.0)
    ref = np.stack([H @ xi for xi in x])
    assert np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-13
