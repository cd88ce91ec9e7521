"""The C-ABI library builds, loads and exports every entry point of include/recon.h.

These run without a GPU: only argument checks that return before any CUDA
call are exercised here; everything that computes is in the `gpu` tests.
"""

import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1203_4587_gb300 import build
    return build.build()


def _declared():
    hdr = open(os.path.join(ROOT, "include", "recon.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(recon_[a-z_]+)\s*\(", hdr)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("recon_plan_create", "recon_solve", "recon_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = C.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_export():
    from paper_1203_4587_gb300 import binding
    assert sorted(binding.EXPORTS) == _declared()


def test_invalid_arguments_rejected_before_any_cuda_call(libpath):
    from paper_1203_4587_gb300 import binding
    lib = binding.load(libpath)
    h = C.c_void_p()
    mask = (C.c_uint8 * 8)()
    sens = (C.c_float * 16)()
    o = binding.Opts()
    lib.recon_default_opts(C.byref(o))
    assert o.rho == pytest.approx(0.5) and o.max_iters == 50 and o.storage == 0 and o.objective == 1
    assert o.frame_levels == 2 and o.spatial_weight == pytest.approx(1.0) and o.cg_steps == 5
    cases = [
        (0, 4, 2, 1, 0.01, 0.1, 0),       # Nx = 0
        (4, 4, 2, 1, 0.01, 0.0, 0),       # mu = 0
        (4, 4, 2, 1, -1.0, 0.1, 0),       # lambda < 0
        (4, 4, 2, 1, 0.01, 0.1, 7),       # unknown prior
    ]
    for Nx, Ny, Nt, Nc, lam, mu, prior in cases:
        st = lib.recon_plan_create(C.byref(h), Nx, Ny, Nt, Nc, C.cast(mask, C.c_void_p), C.cast(sens, C.c_void_p),
                                   lam, mu, prior, None, None)
        assert st == 1, (Nx, mu, lam, prior)
        assert not h.value
        assert lib.recon_last_error()
    bad = binding.Opts()
    lib.recon_default_opts(C.byref(bad))
    bad.rho = -1.0
    st = lib.recon_plan_create(C.byref(h), 4, 4, 2, 1, C.cast(mask, C.c_void_p), C.cast(sens, C.c_void_p),
                               0.01, 0.1, 0, C.byref(bad), None)
    assert st == 1
    bad = binding.Opts()
    lib.recon_default_opts(C.byref(bad))
    assert bad.persistent == 0 and bad.overlap == 1
    for field in ("persistent", "overlap"):
        bad = binding.Opts()
        lib.recon_default_opts(C.byref(bad))
        setattr(bad, field, 2)
        st = lib.recon_plan_create(C.byref(h), 4, 4, 2, 1, C.cast(mask, C.c_void_p), C.cast(sens, C.c_void_p),
                                   0.01, 0.1, 0, C.byref(bad), None)
        assert st == 1, field
    assert lib.recon_plan_set_profile(None, 1) == 1
    for field, value in (("cg_steps", 0), ("cg_steps", 65), ("spatial_weight", -0.5)):   # spatio-temporal prior
        bad = binding.Opts()
        lib.recon_default_opts(C.byref(bad))
        setattr(bad, field, value)
        st = lib.recon_plan_create(C.byref(h), 4, 4, 2, 1, C.cast(mask, C.c_void_p), C.cast(sens, C.c_void_p),
                                   0.01, 0.1, 3, C.byref(bad), None)
        assert st == 1, field
    st = lib.recon_plan_create(C.byref(h), 4, 4096, 2, 1, C.cast(mask, C.c_void_p), C.cast(sens, C.c_void_p),
                               0.01, 0.1, 0, None, None)
    assert st == 7  # unsupported size
    st = lib.recon_plan_create_slab(C.byref(h), 8, 4, 2, 1, C.cast(mask, C.c_void_p), C.cast(sens, C.c_void_p),
                                    0.01, 0.1, 3, None, 0, 4, None)
    assert st == 7  # the spatio-temporal prior couples columns: no slab plans
    for mu in (0.0, float("inf"), float("nan")):    # the allocation-free inverse checks mu on the host
        st = lib.recon_gram_inverse_noalloc(8, 1, 1, C.cast(mask, C.c_void_p), C.cast(sens, C.c_void_p), mu,
                                            C.cast(sens, C.c_void_p), None)
        assert st == 1, mu
    for bad_limit in (0, 2000001):               # the wait self-test checks its limit before launching
        assert lib.recon_selftest_wait_timeout(bad_limit, None, None) == 1
    assert lib.recon_destroy(None) == 0
    assert lib.recon_solve(None, None, None, None, None) == 1
    assert lib.recon_status_string(2) == b"RECON_ERR_MASK_NOT_CARTESIAN"


@pytest.mark.parametrize("name,cls", [("recon_opts", "Opts"), ("recon_info", "Info"), ("recon_profile", "Profile")])
def test_struct_matches_header(name, cls):
    """The binding's ctypes structs list the header's fields in order and type."""
    import re
    from paper_1203_4587_gb300 import binding
    text = open(os.path.join(ROOT, "include", "recon.h")).read()
    body = re.search(r"typedef struct \{((?:(?!typedef struct).)*?)\} " + name + ";", text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(float|int|double)\s+(\w+)\s*;", body)
    ctype = {"float": C.c_float, "int": C.c_int, "double": C.c_double}
    assert [(n, ctype[t]) for t, n in fields] == list(getattr(binding, cls)._fields_)


def test_every_entry_point_rejects_null_and_empty_arguments(libpath):
    """recon.h: NULL handles and empty or out-of-range counts give
    RECON_ERR_INVALID_ARG (1) with a reason, before any device work; the
    destroy calls are NULL-safe (0)."""
    from paper_1203_4587_gb300 import binding
    lib = binding.load(libpath)
    out = C.c_void_p()
    one = (C.c_void_p * 1)(None)
    info = binding.Info()
    buf = (C.c_double * 4)()
    calls = {
        "recon_plan_set_mu": lambda: lib.recon_plan_set_mu(None, 0.1, None),
        "recon_solve_host": lambda: lib.recon_solve_host(None, None, None, None, None),
        "recon_solve_kspace": lambda: lib.recon_solve_kspace(None, None, None, None, None),
        "recon_get_trace": lambda: lib.recon_get_trace(None, buf, 4),
        "recon_get_profile": lambda: lib.recon_get_profile(None, None),
        "recon_apply_adjoint": lambda: lib.recon_apply_adjoint(None, None, None, None),
        "recon_apply_forward": lambda: lib.recon_apply_forward(None, None, None, None),
        "recon_apply_inverse": lambda: lib.recon_apply_inverse(None, None, None, None),
        "recon_export_inverse": lambda: lib.recon_export_inverse(None, 0, 0, None, None),
        "recon_autotune": lambda: lib.recon_autotune(None, None, None),
        "recon_batch_create (NULL plans)": lambda: lib.recon_batch_create(C.byref(out), None, 1),
        "recon_batch_create (n = 0)": lambda: lib.recon_batch_create(C.byref(out), one, 0),
        "recon_volume_create (nz = 0)": lambda: lib.recon_volume_create(C.byref(out), one, 0, 1.0),
        "recon_batch_solve": lambda: lib.recon_batch_solve(None, None, None, None),
        "recon_batch_info": lambda: lib.recon_batch_info(None, C.byref(info), None),
        "recon_batch_autotune": lambda: lib.recon_batch_autotune(None, None, None),
        "recon_grad_create (n = 0)": lambda: lib.recon_grad_create(C.byref(out), one, 0, 5),
        "recon_grad_forward": lambda: lib.recon_grad_forward(None, None, None, None),
        "recon_grad_backward": lambda: lib.recon_grad_backward(None, None, None, None, None, None),
    }
    for name, call in calls.items():
        assert call() == 1, name
        assert lib.recon_last_error(), name
    for destroy in (lib.recon_destroy, lib.recon_batch_destroy, lib.recon_grad_destroy):
        assert destroy(None) == 0
    for code in range(0, 9):
        assert lib.recon_status_string(code)
