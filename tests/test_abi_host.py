"""Host-side checks of the C ABI: the library loads, exports every function
include/helm.h declares, and validates plans and sizes (no GPU calls)."""
import ctypes
import os
import re

import pytest

from oracle import helmholtz as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_1703_09268_gb300", "libhelm.so")


@pytest.fixture(scope="module")
def helm():
    if not os.path.exists(LIB):
        from paper_1703_09268_gb300 import build
        build.build()
    from paper_1703_09268_gb300 import helm as H
    return H


def declared_functions():
    src = open(os.path.join(ROOT, "include", "helm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"#ifdef HELM_DEBUG.*?#endif", "", src, flags=re.S)  # declared for the debug build only
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", src, flags=re.M))
                  - {"if", "defined"})


def test_every_declared_symbol_is_exported(helm):
    names = declared_functions()
    assert "misfit_and_gradient" in names and "helm_forward" in names and "helm_adjoint" in names
    lib = ctypes.CDLL(LIB)
    for name in names:
        assert hasattr(lib, name), name
    assert set(helm.EXPORTS) <= set(names)


def test_plan_dims_match_grid_rule(helm):
    for dim, n, npml, levels in [(3, (64, 64, 64), (10, 10, 10), 2), (3, (48, 50, 52), (10, 7, 12), 3),
                                 (2, (101, 1, 101), (20, 0, 20), 2), (3, (20, 21, 22), (3, 4, 5), 1)]:
        o = helm.default_opts(precond=helm.PRECOND_MLGMRES if levels > 1 else helm.PRECOND_NONE)
        p = helm.Plan(helm.make_grid(dim, n, 25.0, npml, 3000.0, levels=levels), o, device="cpu")
        g = O.make_grid(dim, n, 25.0, npml, 3000.0, levels=levels)
        assert p.N == g.N
        assert p.n_comp == g.size and p.n_phys == g.n_phys
        if levels > 1:
            for d in range(3):
                if g.N[d] > 1:
                    assert (p.N[d] + 1) % (1 << (levels - 1)) == 0
        p.close()


@pytest.mark.parametrize("bad", [
    dict(dim=4), dict(h=0.0), dict(h=-1.0), dict(levels=0), dict(levels=4), dict(npml=(-1, 2, 2)),
    dict(n=(1, 8, 8)), dict(v_ref=0.0),
])
def test_invalid_grid_rejected(helm, bad):
    args = dict(dim=3, n=(8, 8, 8), h=10.0, npml=(2, 2, 2), v_ref=2000.0, levels=1)
    args.update(bad)
    g = helm.make_grid(args["dim"], args["n"], args["h"], args["npml"], args["v_ref"], levels=args["levels"])
    o = helm.default_opts(precond=helm.PRECOND_NONE)
    h = ctypes.c_void_p()
    code = helm.lib().helm_plan_create(ctypes.byref(g), ctypes.byref(o), ctypes.byref(h))
    assert code == helm.HELM_E_INVAL and not h.value


@pytest.mark.parametrize("bad", [
    dict(precision=7), dict(precond=9), dict(k_inner=0), dict(k_inner=33), dict(tol=0.0), dict(tol=1.5),
    dict(max_cycles=0), dict(tol_inner=0.0), dict(max_refine=0), dict(k_si=0), dict(k_ci=40),
    dict(max_batch=-1),
])
def test_invalid_options_rejected(helm, bad):
    g = helm.make_grid(3, (8, 8, 8), 10.0, (2, 2, 2), 2000.0, levels=2)
    o = helm.default_opts(**bad)
    h = ctypes.c_void_p()
    assert helm.lib().helm_plan_create(ctypes.byref(g), ctypes.byref(o), ctypes.byref(h)) == helm.HELM_E_INVAL


def test_mlgmres_needs_levels_and_coarse_size(helm):
    o = helm.default_opts(precond=helm.PRECOND_MLGMRES)
    h = ctypes.c_void_p()
    g1 = helm.make_grid(3, (8, 8, 8), 10.0, (2, 2, 2), 2000.0, levels=1)
    assert helm.lib().helm_plan_create(ctypes.byref(g1), ctypes.byref(o), ctypes.byref(h)) == helm.HELM_E_INVAL
    g3 = helm.make_grid(3, (2, 2, 2), 10.0, (0, 0, 0), 2000.0, levels=3)
    assert helm.lib().helm_plan_create(ctypes.byref(g3), ctypes.byref(o), ctypes.byref(h)) == helm.HELM_E_INVAL


def test_workspace_sizes(helm):
    p = helm.Plan(helm.make_grid(3, (16, 16, 16), 25.0, (4, 4, 4), 3000.0, levels=2), helm.default_opts(),
                  device="cpu")
    a = p.workspace_size(helm.CALL_APPLY, 1, 4, 0)
    f1 = p.workspace_size(helm.CALL_FORWARD, 1, 4, 16)
    f2 = p.workspace_size(helm.CALL_FORWARD, 1, 8, 16)
    m = p.workspace_size(helm.CALL_MISFIT_GRAD, 1, 8, 16)
    assert 0 < a < f1 < f2 < m
    # batching bounds the workspace
    pb = helm.Plan(helm.make_grid(3, (16, 16, 16), 25.0, (4, 4, 4), 3000.0, levels=2),
                   helm.default_opts(max_batch=2), device="cpu")
    assert pb.workspace_size(helm.CALL_FORWARD, 1, 8, 16) < f2
    with pytest.raises(helm.HelmError):
        p.workspace_size(helm.CALL_FORWARD, 0, 4, 16)


def test_status_strings(helm):
    L = helm.lib()
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert L.helm_status_string(code)
    assert L.helm_status_string(123) == b"unknown status"


def test_workspace_sizes_of_the_other_calls(helm):
    p = helm.Plan(helm.make_grid(3, (16, 16, 16), 25.0, (4, 4, 4), 3000.0, levels=2), helm.default_opts(),
                  device="cpu")
    m = p.workspace_size(helm.CALL_MISFIT_GRAD, 1, 8, 16)
    pre = p.workspace_size(helm.CALL_PRECOND, 1, 8, 0)
    born = p.workspace_size(helm.CALL_BORN, 1, 8, 16)
    gn = p.workspace_size(helm.CALL_GN_HESSVEC, 1, 8, 16)
    hv = p.workspace_size(helm.CALL_HESSVEC, 1, 8, 16)
    # the preconditioner alone needs neither the outer basis nor the FP64 fields
    assert 0 < pre < m
    # the Gauss-Newton product keeps the linearised data, the full Hessian one more field
    assert pre < born < gn < hv
    p2 = helm.Plan(helm.make_grid(2, (31, 1, 21), 10.0, (5, 0, 5), 2000.0, levels=2), helm.default_opts(),
                   device="cpu")
    w1 = p2.workspace_size(helm.CALL_MISFIT_GRAD_25D, 4, 3, 11)
    w2 = p2.workspace_size(helm.CALL_MISFIT_GRAD_25D, 8, 3, 11)
    assert 0 < w1 < w2
    # WRI keeps the field accumulator and the receiver-space CG state besides the gradient's fields
    assert p.workspace_size(helm.CALL_WRI, 1, 8, 16) > m
    with pytest.raises(helm.HelmError):
        p.workspace_size(helm.CALL_WRI + 1, 1, 1, 1)


def test_new_calls_reject_bad_arguments_before_any_device_work(helm):
    """Null pointers, empty sizes, a 3D plan for 2.5D and non-finite wavenumbers
    are refused with HELM_E_INVAL on the host (no CUDA call is made)."""
    L = helm.lib()
    p3 = helm.Plan(helm.make_grid(3, (8, 8, 8), 25.0, (2, 2, 2), 3000.0), helm.default_opts(precond=0),
                   device="cpu")
    fr = (ctypes.c_double * 1)(5.0)
    fake = ctypes.c_void_p(256)  # never dereferenced: the checks fail before any use
    rep = (helm.HelmRhsReport * 4)()
    # helm_born without dm
    assert L.helm_born(p3._h, fake, fr, 1, fake, 1, fake, 1, None, fake, 1, None, None, fake, fake, 1 << 20,
                       rep, None) == helm.HELM_E_INVAL
    # helm_born_adjoint without dD
    assert L.helm_born_adjoint(p3._h, fake, fr, 1, fake, 1, fake, 1, None, fake, 1, None, None, fake, fake, 1 << 20,
                               rep, None) == helm.HELM_E_INVAL
    # helm_hessvec without d_obs
    assert L.helm_hessvec(p3._h, fake, fr, 1, fake, 1, fake, 1, None, fake, 1, None, fake, None, fake, fake,
                          1 << 20, rep, None) == helm.HELM_E_INVAL
    # helm_precond_apply with no fields
    assert L.helm_precond_apply(p3._h, fake, 5.0, 0, fake, fake, 0, fake, 1 << 20, None) == helm.HELM_E_INVAL
    # 2.5D needs a 2D plan, nk >= 1 and finite wavenumbers
    ky = (ctypes.c_double * 2)(0.01, 0.02)
    ck = (ctypes.c_double * 2)(0.5, 0.5)
    args = (fake, 1, fake, 1, None, fake, 1, fake, fake, fake, fake, 1 << 20, rep, None)
    assert L.helm_misfit_and_gradient_25d(p3._h, fake, fr, 1, ky, ck, 2, *args) == helm.HELM_E_INVAL
    p2 = helm.Plan(helm.make_grid(2, (11, 1, 9), 25.0, (3, 0, 3), 3000.0), helm.default_opts(precond=0),
                   device="cpu")
    assert L.helm_misfit_and_gradient_25d(p2._h, fake, fr, 1, ky, ck, 0, *args) == helm.HELM_E_INVAL
    bad = (ctypes.c_double * 2)(0.01, float("nan"))
    assert L.helm_misfit_and_gradient_25d(p2._h, fake, fr, 1, bad, ck, 2, *args) == helm.HELM_E_INVAL
    # WRI needs lambda > 0, cg_tol > 0 and at least one CG iteration
    wargs = (fake, 1, fake, 1, None, fake, 1, fake)
    tail = (fake, fake, fake, 1 << 20, rep, None)
    assert L.helm_wri_misfit_and_gradient(p3._h, fake, fr, 1, *wargs, 0.0, 1e-10, 10, *tail) == helm.HELM_E_INVAL
    assert L.helm_wri_misfit_and_gradient(p3._h, fake, fr, 1, *wargs, 1e3, 0.0, 10, *tail) == helm.HELM_E_INVAL
    assert L.helm_wri_misfit_and_gradient(p3._h, fake, fr, 1, *wargs, 1e3, 1e-10, 0, *tail) == helm.HELM_E_INVAL


def test_stored_field_type_is_checked_before_any_device_work(helm):
    """helm_misfit / helm_gradient accept complex128 or complex64 stored fields
    and refuse any other field type code with HELM_E_INVAL on the host."""
    L = helm.lib()
    p3 = helm.Plan(helm.make_grid(3, (8, 8, 8), 25.0, (2, 2, 2), 3000.0), helm.default_opts(precond=0),
                   device="cpu")
    fr = (ctypes.c_double * 1)(5.0)
    fake = ctypes.c_void_p(256)  # never dereferenced: the checks fail before any use
    rep = (helm.HelmRhsReport * 1)()
    assert helm.FIELD_C128 == 0 and helm.FIELD_C64 == 1
    for bad in (-1, 2):
        assert L.helm_misfit(p3._h, fake, fr, 1, fake, 1, fake, 1, None, fake, 1, fake, None, fake, None, fake, bad,
                             fake, 1 << 20, rep, None) == helm.HELM_E_INVAL
        assert L.helm_gradient(p3._h, fake, fr, 1, fake, 1, fake, 1, fake, bad, None, fake, fake, 1 << 20, rep,
                               None) == helm.HELM_E_INVAL


def test_debug_build_exports_the_same_calls_and_its_self_test(helm):
    """libhelm_debug.so (HELM_DEBUG) exports every call of the release library
    plus helm_debug_guard_selftest, and its workspaces are larger by the guard
    bands; the release library does not export the self-test."""
    from paper_1703_09268_gb300 import build
    if not os.path.exists(build.LIB_DEBUG):
        build.build(variants=("debug",))
    dbg = ctypes.CDLL(build.LIB_DEBUG)
    for name in declared_functions():
        assert hasattr(dbg, name), name
    assert hasattr(dbg, "helm_debug_guard_selftest")
    assert not hasattr(ctypes.CDLL(LIB), "helm_debug_guard_selftest")
    P, I, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    sizes = []
    for lib in (ctypes.CDLL(LIB), dbg):
        lib.helm_plan_create.argtypes = [ctypes.POINTER(helm.HelmGrid), ctypes.POINTER(helm.HelmSolveOpts),
                                         ctypes.POINTER(P)]
        lib.helm_workspace_size.argtypes = [P, I, I, I, I, ctypes.POINTER(S)]
        lib.helm_plan_destroy.argtypes = [P]
        lib.helm_plan_destroy.restype = None
        g = helm.make_grid(3, (16, 16, 16), 25.0, (4, 4, 4), 3000.0, levels=2)
        o = helm.default_opts()
        h = P()
        assert lib.helm_plan_create(ctypes.byref(g), ctypes.byref(o), ctypes.byref(h)) == 0
        b = S()
        assert lib.helm_workspace_size(h, helm.CALL_MISFIT_GRAD, 1, 4, 16, ctypes.byref(b)) == 0
        sizes.append(b.value)
        lib.helm_plan_destroy(h)
    assert sizes[1] > sizes[0]


def test_stencil_shape_calls_on_the_host(helm):
    """The tile-shape calls need no device: the shape list, the range check of
    a forced shape, going back to tuning, and 'not tuned yet' for a fresh grid."""
    shapes = helm.stencil_variants()
    assert len(shapes) >= 2
    assert shapes[0] == dict(threads=128, zplanes=16, min_blocks=6)
    for sh in shapes:
        assert sh["threads"] in (64, 128, 256) and sh["zplanes"] in (8, 16, 32) and sh["min_blocks"] >= 1
        assert sh["threads"] * sh["min_blocks"] <= 2048  # fits the SM's thread slots
    L = helm.lib()
    assert L.helm_stencil_select(len(shapes)) == helm.HELM_E_INVAL
    assert L.helm_stencil_select(-2) == helm.HELM_E_INVAL
    assert L.helm_stencil_variant_info(len(shapes), None, None, None) == helm.HELM_E_INVAL
    assert L.helm_stencil_select(1) == helm.HELM_OK
    assert L.helm_stencil_select(-1) == helm.HELM_OK
    p = helm.Plan(helm.make_grid(3, (9, 7, 5), 25.0, (2, 2, 2), 3000.0), helm.default_opts(precond=0), device="cpu")
    assert helm.stencil_tuned(p) is None
