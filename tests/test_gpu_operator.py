"""Parity of the CUDA operator (through the C ABI) against the FP64 CPU oracle.

Element-by-element comparison of unpacked outputs with the oracle on the same seeded inputs.
Tolerances (relative L2 over the output parity): FP64 1e-13, FP32 1e-6, FP16 with per-site
norm 5e-3 per application.
"""
import numpy as np
import pytest

import oracle as orc
from paper_1311_4462_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {8: 1e-13, 16: 1e-13, 4: 1e-6, 2: 5e-3}  # 16: DF64 (double-float), held to the FP64 bound

# (name, L, flavor, kappa, mu, eps): covers L = 2 extents (x+mu == x-mu), ragged tails
# (Vh not a multiple of the 128-thread block), non-cubic shapes, both flavour signs.
CASES = [
    ("cfg1_4^4_doublet_deg", (4, 4, 4, 4), 2, 0.16, 0.01, 0.0),
    ("nd_6x4x2x10", (6, 4, 2, 10), 2, 0.1612, 0.135, 0.15),
    ("plus_2x4x6x8", (2, 4, 6, 8), 1, 0.1612, 0.004, 0.0),
    ("minus_8x6x4x10", (8, 6, 4, 10), -1, 0.1612, 0.004, 0.0),
    ("nd_2^4", (2, 2, 2, 2), 2, 0.16, 0.135, 0.15),
    # the Wilson limit mu = eps = 0 (the "Wilson" column of Table 1): R = 1, one flavour and a doublet
    ("wilson_4x2x6x4", (4, 2, 6, 4), 1, 0.1612, 0.0, 0.0),
    ("wilson_nd_6x4x4x2", (6, 4, 4, 2), 2, 0.16, 0.0, 0.0),
]
PRECS = [8, 16, 4, 2]
RECONS = [18, 12, 8]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


_cache = {}


def setup(case, recon):
    import paper_1311_4462_gb300 as tmq
    name, L, flavor, kappa, mu, eps = case
    key = (name, recon)
    if key not in _cache:
        p = tmq.Params(L, kappa, mu, eps, flavor=flavor, recon=recon)
        po = orc.Params(L, kappa, mu, eps, flavor=flavor)
        U = inputs.gauge_field(L, 1000 + len(name))
        g = tmq.Gauge(p, torch.from_numpy(U))
        psi = inputs.spinor_field(L, p.nf, 2000 + len(name))
        chi = inputs.spinor_field(L, p.nf, 2100 + len(name))
        _cache[key] = (tmq, p, po, U, g, psi, chi)
    return _cache[key]


def use_variant(tmq, g, variant, block=128):
    """Force the hopping-kernel launch choice (0 plain, 2 pipelined, 3/4/5 register-capped 128x4/64x8/256x2,
    6/7 shared-memory staged pipeline with 2/3 buffers, 8/9 the same with the flavour-paired doublet hop;
    prologue launches keep 0 for 2)."""
    pro_variant = variant if variant >= 3 else 0  # 2 has no prologue form
    tmq.tune_import(g, " ".join(f"{p}:0:{variant}:{block} {p}:1:{pro_variant}:{block}" for p in ("f64", "f32", "f16")))


def fields(tmq, g, prec, psi):
    c = torch.from_numpy(psi)
    return tmq.pack(g, c, 0, prec), tmq.pack(g, c, 1, prec)


def get(tmq, g, f, parity):
    return tmq.unpack(g, f, parity).cpu().numpy()


def mask(po, v, parity):
    return orc.project_parity(po, v, parity)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("recon", RECONS)
def test_pack_unpack_roundtrip(case, prec, recon):
    tmq, p, po, U, g, psi, chi = setup(case, recon)
    e, o = fields(tmq, g, prec, psi)
    back = get(tmq, g, e, 0) + get(tmq, g, o, 1)
    tol = {8: 0.0, 16: 1e-14, 4: 1e-7, 2: 6e-4}[prec]
    assert rel(back, psi) <= tol


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("recon", RECONS)
@pytest.mark.parametrize("pc", [0, 1], ids=["asym", "sym"])
@pytest.mark.parametrize("dagger", [False, True], ids=["", "dag"])
@pytest.mark.parametrize("variant", [0, 2, 3, 4, 5, 6, 7, 8, 9],
                         ids=["site", "pipe", "cap128x4", "cap64x8", "cap256x2", "async2", "async3", "pair2", "pair3"])
def test_precond_op(case, prec, recon, pc, dagger, variant):
    tmq, p, po, U, g, psi, chi = setup(case, recon)
    use_variant(tmq, g, variant, block=64 if variant == 2 else 128)
    xe, _ = fields(tmq, g, prec, psi)
    out, tmp = tmq.Field(g, prec), tmq.Field(g, prec)
    tmq.precond_op(g, out, xe, tmp, pc, dagger)
    got = get(tmq, g, out, 0)
    ref = orc.apply_M_pc(po, U, mask(po, psi, 0), sym=bool(pc), dagger=dagger)
    assert rel(got, ref) < TOL[prec]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("pc", [0, 1], ids=["asym", "sym"])
@pytest.mark.parametrize("dagger", [False, True], ids=["", "dag"])
@pytest.mark.parametrize("variant", [3, 8, 9], ids=["cap128x4", "pair2", "pair3"])
def test_normal_op(case, prec, pc, dagger, variant):
    """A^dag A with A = M_pc (or M_pc^dag): the symmetric case runs as M_asym^dag (R R^dag)^-1 M_asym."""
    tmq, p, po, U, g, psi, chi = setup(case, 12)
    use_variant(tmq, g, variant)
    xe, _ = fields(tmq, g, prec, psi)
    out, te, to = tmq.Field(g, prec), tmq.Field(g, prec), tmq.Field(g, prec)
    tmq.normal_op(g, out, xe, te, to, pc, dagger)
    a = orc.apply_M_pc(po, U, mask(po, psi, 0), sym=bool(pc), dagger=dagger)
    ref = orc.apply_M_pc(po, U, a, sym=bool(pc), dagger=not dagger)
    # two operator applications: the per-application FP16 bound twice
    assert rel(get(tmq, g, out, 0), ref) < (2 * TOL[prec] if prec == 2 else TOL[prec])


@pytest.mark.parametrize("case", CASES[:5], ids=[c[0] for c in CASES[:5]])
@pytest.mark.parametrize("recon", [12, 8])
@pytest.mark.parametrize("pc", [0, 1], ids=["asym", "sym"])
@pytest.mark.parametrize("dagger", [False, True], ids=["", "dag"])
def test_f64_full_links(case, recon, pc, dagger):
    """TM_GAUGE_F64_FULL_LINKS: the FP64 links keep all 18 reals, so the FP64 operator gives the
    bits of an 18-real handle (and meets the oracle at the FP64 bound), while FP32 and FP16 follow
    the handle's recon and give the bits of a handle without the flag."""
    import paper_1311_4462_gb300 as tmq
    _, p, po, U, g, psi, chi = setup(case, recon)
    g18 = setup(case, 18)[4]
    gf = tmq.Gauge(p, torch.from_numpy(U), f64_full_links=True)
    try:
        for h in (g, g18, gf):
            use_variant(tmq, h, 3)
        outs = {}
        for name, h in (("flag", gf), ("plain", g), ("r18", g18)):
            for prec in (8, 4, 2):
                xe, _ = fields(tmq, h, prec, psi)
                out, tmp = tmq.Field(h, prec), tmq.Field(h, prec)
                tmq.precond_op(h, out, xe, tmp, pc, dagger)
                outs[name, prec] = get(tmq, h, out, 0)
        assert np.array_equal(outs["flag", 8], outs["r18", 8])
        ref = orc.apply_M_pc(po, U, mask(po, psi, 0), sym=bool(pc), dagger=dagger)
        assert rel(outs["flag", 8], ref) < TOL[8]
        for prec in (4, 2):
            assert np.array_equal(outs["flag", prec], outs["plain", prec])
    finally:
        gf.close()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dagger", [False, True], ids=["", "dag"])
def test_full_operator(case, prec, dagger):
    tmq, p, po, U, g, psi, chi = setup(case, 12)
    use_variant(tmq, g, 2, block=256)
    xe, xo = fields(tmq, g, prec, psi)
    oe, oo = tmq.Field(g, prec), tmq.Field(g, prec)
    tmq.mat(g, oe, oo, xe, xo, dagger)
    got = get(tmq, g, oe, 0) + get(tmq, g, oo, 1)
    ref = orc.apply_M(po, U, psi, dagger=dagger)
    assert rel(got, ref) < TOL[prec]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dagger", [False, True], ids=["", "dag"])
@pytest.mark.parametrize("out_parity", [0, 1])
@pytest.mark.parametrize("variant", [0, 2, 3, 6, 7, 8, 9], ids=["site", "pipe", "cap4", "async2", "async3", "pair2", "pair3"])
def test_dslash_epilogues(case, prec, dagger, out_parity, variant):
    """Each fused epilogue of tm_dslash against the oracle's hopping term and twist."""
    tmq, p, po, U, g, psi, chi = setup(case, 12)
    use_variant(tmq, g, variant, block=96 if variant == 2 else 128)
    ip = 1 - out_parity
    fin = fields(tmq, g, prec, psi)[ip]
    fx = fields(tmq, g, prec, chi)[out_parity]
    t_in = mask(po, psi, ip)
    x = mask(po, chi, out_parity)
    D = mask(po, orc.hop(po, U, t_in, dagger=dagger), out_parity)
    k = p.kappa
    tw = lambda v, inv: orc.twist(po, v, inverse=inv, dagger=dagger)
    expect = {
        tmq.TM_EPI_NONE: D,
        tmq.TM_EPI_TWINV: tw(D, True),
        tmq.TM_EPI_TWXPAY_ASYM: tw(x, False) - k * k * D,
        tmq.TM_EPI_TWXPAY_SYM: x - k * k * tw(D, True),
        tmq.TM_EPI_XPAY: x + k * D,
        tmq.TM_EPI_TWINV_XPAY: tw(x + k * D, True),
    }
    fn = tmq.dslash_dagger if dagger else tmq.dslash
    for epi, ref in expect.items():
        out = tmq.Field(g, prec)
        fn(g, out, fin, out_parity, epi, fx)
        got = get(tmq, g, out, out_parity)
        assert rel(got, ref) < TOL[prec], epi


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("pc", [0, 1], ids=["asym", "sym"])
@pytest.mark.parametrize("dagger", [False, True], ids=["", "dag"])
def test_prepare_rhs_and_reconstruct(case, prec, pc, dagger):
    tmq, p, po, U, g, psi, chi = setup(case, 12)
    if prec == 16:
        be, bo = fields(tmq, g, prec, chi)
        with pytest.raises(tmq.TMError):  # the right-hand side is prepared in FP64, not DF64
            tmq.prepare_rhs(g, tmq.Field(g, prec), be, bo, pc, dagger)
        xe, _ = fields(tmq, g, prec, psi)
        xo = tmq.Field(g, prec)
        tmq.reconstruct_odd(g, xo, bo, xe, dagger)
        ref = orc.reconstruct_odd(po, U, mask(po, psi, 0), chi, dagger=dagger)
        assert rel(get(tmq, g, xo, 1), ref) < TOL[prec]
        return
    be, bo = fields(tmq, g, prec, chi)
    bp = tmq.Field(g, prec)
    tmq.prepare_rhs(g, bp, be, bo, pc, dagger)
    ref = orc.prepare_rhs(po, U, chi, sym=bool(pc), dagger=dagger)
    assert rel(get(tmq, g, bp, 0), ref) < TOL[prec]
    xe, _ = fields(tmq, g, prec, psi)
    xo = tmq.Field(g, prec)
    tmq.reconstruct_odd(g, xo, bo, xe, dagger)
    ref = orc.reconstruct_odd(po, U, mask(po, psi, 0), chi, dagger=dagger)
    assert rel(get(tmq, g, xo, 1), ref) < TOL[prec]


@pytest.mark.parametrize("case", CASES[:3], ids=[c[0] for c in CASES[:3]])
@pytest.mark.parametrize("prec", PRECS)
def test_twist(case, prec):
    tmq, p, po, U, g, psi, chi = setup(case, 12)
    xe, _ = fields(tmq, g, prec, psi)
    for inv in (False, True):
        for dag in (False, True):
            out = tmq.Field(g, prec)
            tmq.twist(g, out, xe, inv, dag)
            ref = orc.twist(po, mask(po, psi, 0), inverse=inv, dagger=dag)
            assert rel(get(tmq, g, out, 0), ref) < TOL[prec]


def test_fp16_matches_dequantized_inputs_closer():
    """FP16 kernel arithmetic on its own inputs: compare with the oracle fed the FP16-rounded spinor."""
    case = CASES[1]
    tmq, p, po, U, g, psi, chi = setup(case, 18)
    xe, _ = fields(tmq, g, 2, psi)
    deq = get(tmq, g, xe, 0)
    out, tmp = tmq.Field(g, 2), tmq.Field(g, 2)
    tmq.precond_op(g, out, xe, tmp, 0, False)
    ref_deq = orc.apply_M_pc(po, U, deq)
    ref_orig = orc.apply_M_pc(po, U, mask(po, psi, 0))
    got = get(tmq, g, out, 0)
    assert rel(got, ref_deq) < rel(got, ref_orig) + 1e-12
    assert rel(got, ref_deq) < 3e-3


def test_argument_errors_are_reported():
    import paper_1311_4462_gb300 as tmq
    tmq_, p, po, U, g, psi, chi = setup(CASES[0], 12)
    a, b = tmq.Field(g, 4), tmq.Field(g, 8)
    with pytest.raises(tmq.TMError) as e:
        tmq.dslash(g, a, b, 0)
    assert e.value.status == -1
    with pytest.raises(tmq.TMError):
        tmq.dslash(g, a, a, 0)  # aliasing
    with pytest.raises(tmq.TMError):
        tmq.precond_op(g, a, a, a, 0)
    bad = tmq.Params((3, 4, 4, 4), 0.16, 0.01, flavor=1)
    with pytest.raises(tmq.TMError):
        tmq.Gauge(bad, torch.zeros(bad.gauge_shape, dtype=torch.complex128))
    sing = tmq.Params((4, 4, 4, 4), 0.125, 0.0, eps=4.0, flavor=2)
    with pytest.raises(tmq.TMError):
        tmq.Gauge(sing, torch.zeros(sing.gauge_shape, dtype=torch.complex128))


def test_autotune_roundtrip_and_parity():
    import paper_1311_4462_gb300 as tmq
    case = CASES[1]
    tmq_, p, po, U, g, psi, chi = setup(case, 12)
    table = tmq.autotune(g)
    entries = table.split()
    single = [e for e in entries if e.split(":")[1] not in ("m", "c", "p")]
    multi = [e for e in entries if e.split(":")[1] == "m"]
    clov = [e for e in entries if e.split(":")[1] == "c"]
    fused = [e for e in entries if e.split(":")[1] == "p"]
    assert len(single) == 6 and all(len(e.split(":")) == 4 for e in single)
    assert len(multi) == 3 and all(e.split(":")[2] in ("2", "4", "8", "12", "14", "16", "32", "34", "36")
                                   or (e.startswith("f16") and e.split(":")[2] in ("13", "15", "33", "35"))
                                   for e in multi)
    assert len(clov) == 3 and all(e.split(":")[2] in ("1", "3", "4", "6") for e in clov)
    assert len(fused) == 2 and all(e.split(":")[2] in ("0", "1") for e in fused)
    tmq.tune_import(g, table)
    assert tmq.tune_export(g) == table
    for bad in ("f32:0:3:100",   # block not a multiple of 32
                "f32:m:3",       # right-hand sides per block not 2, 4 or 8 (or staged 12, 14)
                "f32:m:15",      # three-buffer staged multi-RHS forms: FP16 only
                "f16:c:2",       # clover occupancy not 1, 3 or 4
                "f16:p:1",       # no fused FP16 operator
                "f32:0:10:128",  # no such variant
                "f99:0:3:128"):  # no such precision
        with pytest.raises(tmq.TMError):
            tmq.tune_import(g, bad)
    assert tmq.tune_export(g) == table  # a rejected import leaves the table unchanged
    xe, _ = fields(tmq, g, 4, psi)
    out, tmp = tmq.Field(g, 4), tmq.Field(g, 4)
    tmq.precond_op(g, out, xe, tmp, 0, False)
    ref = orc.apply_M_pc(po, U, mask(po, psi, 0))
    assert rel(get(tmq, g, out, 0), ref) < TOL[4]


@pytest.mark.parametrize("prec", [8, 4, 2])
def test_pinned_host_canonical_buffers_are_used_in_place(prec):
    import ctypes
    import paper_1311_4462_gb300 as tmq
    from paper_1311_4462_gb300 import _lib as L
    tmq_, p, po, U, g, psi, chi = setup(CASES[1], 12)
    host = torch.from_numpy(psi).pin_memory()
    f_host = tmq.pack(g, host, 0, prec)
    f_dev = tmq.pack(g, host.to("cuda"), 0, prec)
    torch.cuda.synchronize()
    assert torch.equal(f_host.data, f_dev.data)
    out_host = torch.zeros(p.spinor_shape, dtype=torch.complex128).pin_memory()
    tmq.unpack(g, f_dev, 0, canon=out_host)
    torch.cuda.synchronize()
    assert torch.equal(out_host, tmq.unpack(g, f_dev, 0).cpu())
    # pageable host memory is refused (never dereferenced by a kernel)
    pageable = np.zeros(p.spinor_shape, dtype=np.complex128)
    st = L.load().tm_unpack(g.h, ctypes.c_void_p(pageable.ctypes.data), L.TM_C128, f_dev.ref(), 0, None)
    assert st == L.TM_ERR_ARG
    st = L.load().tm_pack(g.h, f_dev.ref(), ctypes.c_void_p(pageable.ctypes.data), L.TM_C128, 0, None)
    assert st == L.TM_ERR_ARG


@pytest.mark.parametrize("case", CASES[:3], ids=[c[0] for c in CASES[:3]])
@pytest.mark.parametrize("nrhs", [1, 3])
@pytest.mark.parametrize("where", ["device", "pinned"])
def test_chunk_copy_pack_matches_the_generic_path(case, nrhs, where):
    """FP32 fields from complex64 (16-byte aligned) take the shared-memory chunk path; an 8-byte
    aligned view of the same data takes the per-site path: both give the same bits, both ways."""
    tmq, p, po, U, g, psi, chi = setup(case, 12)
    src = np.stack([psi, chi, psi + 1j * chi][:nrhs]) if nrhs > 1 else psi
    src = torch.from_numpy(src.astype(np.complex64))
    dev = "cuda" if where == "device" else "cpu"

    def buffers():
        def one():
            big = torch.zeros(src.numel() + 1, dtype=torch.complex64, device=dev)
            return big.pin_memory() if where == "pinned" else big
        # separate allocations: a 16-byte aligned view and an 8-byte aligned one
        return one()[: src.numel()].view(src.shape), one()[1:].view(src.shape)

    a_in, m_in = buffers()
    a_in.copy_(src)
    m_in.copy_(src)
    for parity in (0, 1):
        fa = tmq.pack(g, a_in, parity, 4, nrhs=nrhs)
        fm = tmq.pack(g, m_in, parity, 4, nrhs=nrhs)
        torch.cuda.synchronize()
        assert torch.equal(fa.data, fm.data)
        a_out, m_out = buffers()
        tmq.unpack(g, fa, parity, canon=a_out)
        tmq.unpack(g, fa, parity, canon=m_out)
        torch.cuda.synchronize()
        assert torch.equal(a_out.cpu(), m_out.cpu())
        mask_ = torch.from_numpy(orc.parity_mask(po, parity))[..., None, None, None]
        assert torch.equal(a_out.cpu(), torch.where(mask_, src, torch.zeros_like(src)))
