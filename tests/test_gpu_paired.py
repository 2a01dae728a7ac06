"""The paired hop (launch forms 8 / 9: the doublet's flavours, or one flavour's two projected spin
rows, in register pairs with packed FMAs) performs per value the same binary32 operations in the
same order as the unpaired forms 6 / 7 (the link product is one FMA chain per colour in both), so
the results are bit-identical; checked for every operator, storage precision and link format."""
import pytest

from paper_1311_4462_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    ("nd_8x8x8x16", (8, 8, 8, 16), 2, 0.1612, 0.135, 0.15),
    ("plus_6x4x2x10", (6, 4, 2, 10), 1, 0.1612, 0.004, 0.0),
]

_cache = {}


def handle(case, recon):
    import paper_1311_4462_gb300 as tmq
    name, L, flavor, kappa, mu, eps = case
    key = (name, recon)
    if key not in _cache:
        p = tmq.Params(L, kappa, mu, eps, flavor=flavor, recon=recon)
        g = tmq.Gauge(p, torch.from_numpy(inputs.gauge_field(L, 1700 + len(name))))
        psi = torch.from_numpy(inputs.spinor_field(L, p.nf, 2700 + len(name)))
        _cache[key] = (tmq, g, psi)
    return _cache[key]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", [4, 2], ids=["f32", "f16"])
@pytest.mark.parametrize("recon", [18, 12, 8])
@pytest.mark.parametrize("forms", [(6, 8), (7, 9)], ids=["2buf", "3buf"])
def test_paired_forms_are_bit_identical(case, prec, recon, forms):
    tmq, g, psi = handle(case, recon)
    name = {4: "f32", 2: "f16"}[prec]
    xe = tmq.pack(g, psi, 0, prec)
    saved = tmq.tune_export(g)
    try:
        for pc in (0, 1):
            for dag in (False, True):
                outs = []
                for v in forms:
                    tmq.tune_import(g, f"{name}:0:{v}:128 {name}:1:{v}:128")
                    out, tmp = tmq.Field(g, prec).zero_(), tmq.Field(g, prec)
                    tmq.precond_op(g, out, xe, tmp, pc, dag)
                    outs.append((out.data.clone(), None if out.norm is None else out.norm.clone()))
                assert torch.equal(outs[0][0], outs[1][0]), (pc, dag)
                if outs[0][1] is not None:
                    assert torch.equal(outs[0][1], outs[1][1]), (pc, dag)
    finally:
        tmq.tune_import(g, saved)
