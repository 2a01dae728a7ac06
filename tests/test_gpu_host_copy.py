"""tm_field_upload / tm_field_download: host copies of fields in the library's own layout.

A field downloaded to page-locked host memory and uploaded again must hold the same bytes
(data and, for FP16, the per-site norms), and the operator applied to the uploaded copy must give
the bits it gives on the original.
"""
import ctypes

import pytest

from paper_1311_4462_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [8, 4, 2, 16])
@pytest.mark.parametrize("nf", [1, 2])
def test_round_trip_and_operator_bits(prec, nf):
    import paper_1311_4462_gb300 as tmq
    Lat = (4, 4, 2, 6)
    p = tmq.Params(Lat, 0.1612, 0.135 if nf == 2 else 0.004, 0.15 if nf == 2 else 0.0,
                   flavor=tmq.TM_NDEG_DOUBLET if nf == 2 else tmq.TM_TWIST_PLUS, recon=12)
    g = tmq.Gauge(p, torch.from_numpy(inputs.gauge_field(Lat, 1500)))
    xe = tmq.pack(g, torch.from_numpy(inputs.spinor_field(Lat, nf, 2600)), 0, prec)
    hd, hn = tmq.host_buffers(g, prec)
    tmq.download(g, xe, hd, hn)
    ye = tmq.Field(g, prec).zero_()
    tmq.upload(g, ye, hd, hn)
    torch.cuda.synchronize()
    assert torch.equal(ye.data, xe.data)
    if prec == 2:
        assert torch.equal(ye.norm, xe.norm)
    a, b, t = tmq.Field(g, prec), tmq.Field(g, prec), tmq.Field(g, prec)
    tmq.precond_op(g, a, xe, t, tmq.TM_PC_ASYM, False)
    tmq.precond_op(g, b, ye, t, tmq.TM_PC_ASYM, False)
    # the result comes back to the host the same way
    ha, hna = tmq.host_buffers(g, prec)
    tmq.download(g, b, ha, hna)
    torch.cuda.synchronize()
    assert torch.equal(a.data.cpu(), ha)
    g.close()


def test_fp16_needs_its_norm_buffer():
    import paper_1311_4462_gb300 as tmq
    from paper_1311_4462_gb300 import _lib as L
    Lat = (4, 4, 2, 4)
    p = tmq.Params(Lat, 0.1612, 0.004, 0.0, flavor=tmq.TM_TWIST_PLUS, recon=12)
    g = tmq.Gauge(p, torch.from_numpy(inputs.gauge_field(Lat, 1501)))
    f = tmq.Field(g, tmq.TM_PREC_F16)
    hd, _ = tmq.host_buffers(g, tmq.TM_PREC_F16)
    st = L.load().tm_field_upload(g.h, f.ref(), ctypes.c_void_p(hd.data_ptr()), None, None)
    assert st == L.TM_ERR_ARG and "null" in L.last_error()
    g.close()
