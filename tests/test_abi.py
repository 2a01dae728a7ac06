"""The C ABI library builds, loads and exports every entry point include/tm.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1311_4462_gb300 import build
    from paper_1311_4462_gb300 import _lib

    build.build()
    return _lib.load()


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(tm_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["tm_dslash", "tm_dslash_dagger", "tm_precond_op", "tm_reconstruct_odd", "tm_prepare_rhs",
                     "tm_gauge_create", "tm_pack", "tm_unpack", "tm_mat"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol(lib):
    from paper_1311_4462_gb300 import _lib
    assert set(declared_functions()) <= set(_lib.exported_names())


def test_version_string(lib):
    assert b"sm_103a" in lib.tm_version()


def test_host_side_parameter_validation_without_gpu(lib):
    from paper_1311_4462_gb300 import _lib as L

    def create(Ls, kappa=0.16, mu=0.01, eps=0.0, flavor=1, recon=12):
        p = L.tm_params()
        p.L[:] = Ls
        p.kappa, p.mu, p.epsilon, p.flavor, p.t_antiperiodic, p.recon = kappa, mu, eps, flavor, 1, recon
        h = ctypes.c_void_p()
        st = lib.tm_gauge_create(ctypes.byref(p), ctypes.c_void_p(16), None, ctypes.byref(h))
        return st, L.last_error()

    assert create((3, 4, 4, 4))[0] == L.TM_ERR_ARG
    assert create((4, 4, 4, 0))[0] == L.TM_ERR_ARG
    st, msg = create((4, 4, 4, 4), eps=0.1, flavor=1)
    assert st == L.TM_ERR_ARG and "epsilon" in msg
    st, msg = create((4, 4, 4, 4), kappa=0.125, mu=0.0, eps=4.0, flavor=2)
    assert st == L.TM_ERR_ARG and "singular" in msg
    assert create((4, 4, 4, 4), recon=9)[0] == L.TM_ERR_ARG
    st, msg = create((128, 128, 128, 128))  # 24 * Vh beyond 32-bit chunk indexing: the maximum size
    assert st == L.TM_ERR_ARG and "too large" in msg
    assert create((4, 4, 4, 4), flavor=3)[0] == L.TM_ERR_ARG
    assert create((4, 4, 4, 4), kappa=-1.0)[0] == L.TM_ERR_ARG
    h = ctypes.c_void_p()
    assert lib.tm_gauge_create(None, None, None, ctypes.byref(h)) == L.TM_ERR_ARG
    assert lib.tm_gauge_destroy(None) == L.TM_OK
    d, n = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.tm_field_bytes(None, 4, 1, ctypes.byref(d), ctypes.byref(n)) == L.TM_ERR_ARG
    assert lib.tm_gauge_set_clover(None, 1.0, None) == L.TM_ERR_ARG
    assert lib.tm_local_op(None, None, None, 0, 0, 0, None) == L.TM_ERR_ARG
    assert lib.tm_field_upload(None, None, None, None, None) == L.TM_ERR_ARG
    assert lib.tm_field_download(None, None, None, None, None) == L.TM_ERR_ARG
