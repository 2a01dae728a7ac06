"""The benchmark's roofline accounting, counted independently here: algorithmic bytes per even
site of M_asym (two launches: each reads 8 links and the input spinor and writes one spinor, the
second also reads x), the stated flop convention, and the launch-form names of the tune table."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _bench():
    saved = sys.argv
    sys.argv = ["bench.py"]
    try:
        import bench
    finally:
        sys.argv = saved
    return bench


def _spinor_bytes(prec):
    # 24 reals per site and flavour; FP16 adds its 4-byte per-site norm; DF64 stores two floats per real
    return {8: 24 * 8, 16: 24 * 8, 4: 24 * 4, 2: 24 * 2 + 4}[prec]


def _link_bytes(prec, recon):
    reals = 12 if (prec == 16 and recon == 8) else recon
    return reals * {8: 8, 16: 8, 4: 4, 2: 2}[prec]


@pytest.mark.parametrize("prec", [8, 16, 4, 2])
@pytest.mark.parametrize("nf", [1, 2])
@pytest.mark.parametrize("recon", [18, 12, 8])
def test_bytes_per_even_site(prec, nf, recon):
    b = _bench()
    links = 8 * _link_bytes(prec, recon)
    s = nf * _spinor_bytes(prec)
    a, bb = b.launch_bytes(prec, nf, recon)
    assert (a, bb) == (links + 2 * s, links + 3 * s)
    assert b.asym_bytes(prec, nf, recon) == a + bb


def test_headline_and_table_figures():
    b = _bench()
    assert b.asym_bytes(4, 2, 12) == 1728   # doublet FP32, 12-real links (the headline)
    assert b.asym_bytes(2, 2, 12) == 904    # doublet FP16 with norms
    assert b.asym_bytes(4, 1, 12) == 1248
    assert b.asym_bytes(2, 1, 12) == 644
    assert b.asym_bytes(8, 1, 12) == 2496
    assert b.asym_bytes(8, 2, 12) == 3456


def test_flop_convention():
    b = _bench()
    hop = 1320  # per hopping site and flavour
    # one flavour: two hopping terms, R on the even input, R^-1 on the odd intermediate, xpay
    assert b.FLOPS_PER_SITE[1] == 2 * hop + 48 + 72 + 48
    # doublet: both flavours hop, the flavour-mixing R (192) and R^-1 (240) per site, xpay per flavour
    assert b.FLOPS_PER_SITE[2] == 2 * 2 * hop + 192 + 240 + 2 * 48
    # the Wilson limit (R = 1): two hopping terms and the xpay, no twist
    assert b.FLOPS_WILSON == 2 * hop + 48


def test_launch_form_names():
    b = _bench()
    table = "f64:0:3:128 f32:0:8:128 f32:1:8:128 f16:0:9:128 f32:c:6 f16:c:3"
    assert "variant 8" in b.launch_form(table, "f32") and "paired" in b.launch_form(table, "f32")
    assert "3 buffers" in b.launch_form(table, "f16")
    assert "register cap" in b.launch_form(table, "f64")
    assert "staged" in b.launch_form(table, "f32", csw=1.6)
    assert b.launch_form(table, "f16", csw=1.6) == "clover, 3 blocks per SM"
    assert b.launch_form(table, "df64") == "?"
