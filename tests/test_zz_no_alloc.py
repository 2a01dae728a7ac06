"""tm_norm2_noalloc: the reduction for callers that cannot allocate device memory.

It keeps its scratch in a static device array instead of a handle's allocation.  Checked here
through the C ABI against the handle-based tm_norm2 on two calls in a row (the second call
reuses the scratch the first left behind), for every storage precision.  This file is
collected last so that a failure here cannot hide the result of any other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1311_4462_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {8: 1e-14, 16: 1e-13, 4: 1e-6, 2: 1e-6}  # same bounds as the other reduction tests


def _noalloc(lib, field, Vh, nf):
    out = torch.full((max(field.nrhs, 1),), -1.0, dtype=torch.float64, device="cuda")
    st = lib.tm_norm2_noalloc(field.ref(), Vh, nf, ctypes.c_void_p(out.data_ptr()),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out


@pytest.mark.parametrize("prec", [8, 16, 4, 2])
def test_noalloc_norm_matches_handle_norm_twice(prec):
    import paper_1311_4462_gb300 as tmq
    from paper_1311_4462_gb300 import _lib as L
    lib = L.load()
    Lat = (6, 4, 2, 10)
    p = tmq.Params(Lat, 0.1612, 0.135, 0.15, flavor=tmq.TM_NDEG_DOUBLET, recon=12)
    g = tmq.Gauge(p, torch.from_numpy(inputs.gauge_field(Lat, 1400)))
    for call, seed in enumerate((2500, 2501)):
        f = tmq.pack(g, torch.from_numpy(inputs.spinor_field(Lat, 2, seed)), 0, prec)
        ref = tmq.norm2(g, f)
        st, out = _noalloc(lib, f, p.Vh, p.nf)
        assert st == L.TM_OK, L.last_error()
        torch.cuda.synchronize()
        got = out[0].item()
        assert abs(got - ref) / ref < TOL[prec], (call, got, ref)
    g.close()


@pytest.mark.parametrize("prec", [8, 16, 4, 2])
@pytest.mark.parametrize("nrhs", [3, 64])
def test_noalloc_norm_per_column_of_a_multi_rhs_field(prec, nrhs):
    """Every right-hand side's |x_r|^2 (its own column of the shared scratch) against the FP64 sum of
    the same stored values on the host, twice in a row, and column 0 against the handle's tm_norm2."""
    import paper_1311_4462_gb300 as tmq
    from paper_1311_4462_gb300 import _lib as L
    lib = L.load()
    Lat = (4, 4, 2, 6)
    p = tmq.Params(Lat, 0.1612, 0.004, 0.0, flavor=tmq.TM_TWIST_PLUS, recon=12)
    g = tmq.Gauge(p, torch.from_numpy(inputs.gauge_field(Lat, 1401)))
    for call, seed in enumerate((2510, 2511)):
        src = np.stack([inputs.spinor_field(Lat, 1, seed * 100 + r) * (1.0 + r) for r in range(nrhs)])
        f = tmq.pack(g, torch.from_numpy(src), 1, prec, nrhs=nrhs)
        stored = tmq.unpack(g, f, 1).cpu().numpy()  # the values as stored (rounded to the precision)
        host = (np.abs(stored.reshape(nrhs, -1)) ** 2).sum(axis=1)
        st, out = _noalloc(lib, f, p.Vh, p.nf)
        assert st == L.TM_OK, L.last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert got.shape == (nrhs,)
        assert np.all(np.abs(got - host) / host < TOL[prec]), (call, np.max(np.abs(got - host) / host))
        assert abs(got[0] - tmq.norm2(g, f)) / got[0] < TOL[prec]
    g.close()


def test_noalloc_rejects_too_many_rhs():
    import paper_1311_4462_gb300 as tmq
    from paper_1311_4462_gb300 import _lib as L
    lib = L.load()
    fake = L.tm_field(16, None, tmq.TM_PREC_F32, 65)
    out = torch.zeros(65, dtype=torch.float64, device="cuda")
    st = lib.tm_norm2_noalloc(ctypes.byref(fake), 128, 1, ctypes.c_void_p(out.data_ptr()), None)
    assert st == L.TM_ERR_ARG and "65" in L.last_error()
