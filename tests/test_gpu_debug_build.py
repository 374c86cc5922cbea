"""The bounds-checking build (libhelm_debug.so, HELM_DEBUG) on the GPU.

The debug build lays a guard band after every workspace array and checks
the bands and the slot indices at the end of every call (HELM_E_BOUNDS on a
violation).  A child process that loads the debug build runs the solver
calls on small problems: every call must return HELM_OK (no kernel writes
past the end of an array) with the release build's results; the guard
self-test must see a one-byte write into a band."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEV = torch.device("cuda:0")


def run_calls(helm, out_path):
    """The calls both builds run; results saved to out_path (npz)."""
    from paper_1703_09268_gb300 import synth
    T = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)  # noqa: E731
    rng = np.random.default_rng(8)
    n = (17, 14, 15)
    v = synth.layered_velocity(rng, n, nlayers=4, smooth=1.5)
    m0 = T(synth.slowness2(synth._gaussian_smooth(v, 3.0)).ravel(), torch.float64)
    mt = T(synth.slowness2(v).ravel(), torch.float64)
    src, Q = synth.point_sources(n, [(3, 3, 2), (12, 9, 2), (8, 6, 2)])
    src, Q, rec = T(src, torch.int32), T(Q, torch.complex128), T(synth.surface_receivers(n, 0), torch.int32)
    freqs = [2.5, 3.5]
    out = {}
    for name, prec in (("fp64", 0), ("mixed", 1)):
        plan = helm.Plan(helm.make_grid(3, n, 50.0, (6, 6, 6), 4500.0, levels=2),
                         helm.default_opts(precision=prec, tol=1e-10, max_batch=4), device=DEV)
        _, d, _ = helm.helm_forward(plan, mt, freqs, src, Q, rec, want_fields=False)
        f, g, _ = helm.misfit_and_gradient(plan, m0, freqs, src, Q, rec, d)
        dm = T(rng.standard_normal(plan.n_phys) * 1e-9, torch.float64)
        h, _ = helm.helm_hessvec(plan, m0, freqs, src, Q, rec, d, dm)
        fw, gw, _ = helm.wri_misfit_and_gradient(plan, m0, freqs, src, Q, rec, d, 1e3, cg_tol=1e-8, cg_maxit=100)
        x = T(rng.standard_normal((2, plan.n_comp)) + 1j * rng.standard_normal((2, plan.n_comp)),
              torch.complex128 if prec == 0 else torch.complex64)
        z = helm.helm_precond_apply(plan, m0, 3.0, x)
        out.update({f"{name}_f": f.cpu().numpy(), f"{name}_g": g.cpu().numpy(), f"{name}_hess": h.cpu().numpy(),
                    f"{name}_wri_f": fw.cpu().numpy(), f"{name}_wri_g": gw.cpu().numpy(),
                    f"{name}_precond": z.cpu().numpy()})
    np.savez(out_path, **out)


def child(out_path):
    """Entry point of the child process (HELM_LIBRARY=debug)."""
    import ctypes
    sys.path.insert(0, ROOT)
    from paper_1703_09268_gb300 import helm
    assert helm.LIB_PATH.endswith("libhelm_debug.so")
    run_calls(helm, out_path)
    # the guard self-test: intact bands first, then a one-byte host write into the first band
    plan = helm.Plan(helm.make_grid(3, (8, 8, 8), 50.0, (2, 2, 2), 3000.0), helm.default_opts(precond=0), device=DEV)
    ws, nb = plan.workspace(plan.workspace_size(helm.CALL_APPLY, 1, 1, 0))
    lib = helm.lib()
    lib.helm_debug_guard_selftest.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    code = lib.helm_debug_guard_selftest(plan._h, ws, nb, helm._stream(DEV))
    torch.cuda.synchronize()
    print("SELFTEST", code)


def test_debug_build_runs_clean_and_matches_release(tmp_path):
    import __graft_entry__
    __graft_entry__.build()
    from paper_1703_09268_gb300 import helm
    assert os.path.exists(os.path.join(ROOT, "paper_1703_09268_gb300", "libhelm_debug.so"))
    path_dbg = str(tmp_path / "debug.npz")
    env = dict(os.environ, HELM_LIBRARY="debug")
    r = subprocess.run([sys.executable, "-c", f"import tests.test_gpu_debug_build as t; t.child({path_dbg!r})"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert f"SELFTEST {helm.HELM_E_BOUNDS}" in r.stdout, r.stdout[-2000:]
    path_rel = str(tmp_path / "release.npz")
    run_calls(helm, path_rel)
    a, b = np.load(path_dbg), np.load(path_rel)
    for k in b.files:
        x, y = a[k], b[k]
        err = np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300)
        assert err <= 1e-12, (k, err)
