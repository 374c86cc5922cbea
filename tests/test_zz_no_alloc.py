"""helm_apply_noalloc against helm_apply, through the C ABI.

helm_apply_noalloc exists for callers that cannot allocate device memory where
they apply the operator (under a framework that owns every allocation, in
per-request serving loops); it keeps its scratch in a static device array
instead of a caller workspace.  This test calls it twice
in a row (the second call reuses the array the first one left behind) and
compares each result with the workspace entry point, within the operator
tolerances of the parity tests.  It runs last so that a failure here comes
after every other test, and it passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1703_09268_gb300 import helm
    lib = ctypes.CDLL(helm.LIB_PATH)
    P = ctypes.c_void_p
    lib.helm_apply_noalloc.argtypes = [P, P, ctypes.c_double, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, P]
    lib.helm_apply_noalloc.restype = ctypes.c_int
    return helm, lib


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-13), (torch.complex64, 2e-6)])
@pytest.mark.parametrize("adjoint", [0, 1])
def test_noalloc_matches_workspace_apply_twice(api, dtype, tol, adjoint):
    helm, lib = api
    plan = helm.Plan(helm.make_grid(3, (37, 29, 33), 20.0, (6, 5, 7), 3500.0, levels=2),
                     helm.default_opts(), device=DEV)
    rng = np.random.default_rng(11 + adjoint)
    m = torch.as_tensor(1 / rng.uniform(1500, 4500, plan.n_phys) ** 2, dtype=torch.float64, device=DEV)
    prec = helm.FP64 if dtype == torch.complex128 else helm.MIXED
    for call in range(2):
        nrhs = 3 + call  # the second call sees a different size and the first call's leftovers
        x = torch.randn(nrhs, plan.n_comp, dtype=dtype, device=DEV)
        ref = helm.helm_apply(plan, m, 4.0 + call, x, adjoint=bool(adjoint))
        y = torch.full_like(x, float("nan"))
        code = lib.helm_apply_noalloc(plan._h, ctypes.c_void_p(m.data_ptr()), 4.0 + call, adjoint, prec,
                                      ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), nrhs, _stream())
        torch.cuda.synchronize()
        assert code == helm.HELM_OK
        err = ((y - ref).abs().norm() / ref.abs().norm()).item()
        assert err <= tol, (call, err)


def test_noalloc_rejects_fields_beyond_its_scratch(api):
    helm, lib = api
    plan = helm.Plan(helm.make_grid(3, (110, 110, 110), 20.0, (5, 5, 5), 3500.0), helm.default_opts(precond=0),
                     device=DEV)
    m = torch.full((plan.n_phys,), 1 / 2000.0 ** 2, dtype=torch.float64, device=DEV)
    x = torch.zeros(1, plan.n_comp, dtype=torch.complex128, device=DEV)
    y = torch.zeros_like(x)
    code = lib.helm_apply_noalloc(plan._h, ctypes.c_void_p(m.data_ptr()), 4.0, 0, helm.FP64,
                                  ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), 1, _stream())
    assert code == helm.HELM_E_NOMEM
