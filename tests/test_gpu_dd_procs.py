"""The decomposed operator with one slab per process: two processes share the one GPU (each owns
half of the lattice in time) and exchange faces as gloo messages through host memory, their
reductions summed by all_reduce.  Checked against the undecomposed operator (same bits), the
oracle, and the full-system residual of the decomposed solve.  The processes only meet on the host
(blocking gloo messages between launches), so no kernel of one waits on the other."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import oracle as orc
from paper_1311_4462_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("case", [((4, 4, 2, 8), 2, 0.1612, 0.135, 0.15), ((6, 2, 4, 4), 1, 0.1612, 0.004, 0.0)],
                         ids=["nd_4x4x2x8", "plus_6x2x4x4"])
def test_two_processes_one_slab_each(tmp_path, case):
    import paper_1311_4462_gb300 as tmq
    L, flavor, kappa, mu, eps = case
    seed = 1750
    out = str(tmp_path / "dd")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_port()}", os.path.join(ROOT, "tests", "dd_worker.py"), out,
           ",".join(map(str, L)), str(flavor), str(kappa), str(mu), str(eps), str(seed)]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    ranks = [np.load(f"{out}.rank{k}.npz") for k in range(2)]
    p = tmq.Params(L, kappa, mu, eps, flavor=flavor, recon=12)
    po = orc.Params(L, kappa, mu, eps, flavor=flavor)
    U = inputs.gauge_field(L, seed)
    psi = inputs.spinor_field(L, p.nf, seed + 1000)
    g = tmq.Gauge(p, torch.from_numpy(U))
    for prec in (8, 4):
        xe = tmq.pack(g, torch.from_numpy(psi), 0, prec)
        o, t = tmq.Field(g, prec), tmq.Field(g, prec)
        for pc in (0, 1):
            for dag in (0, 1):
                tmq.precond_op(g, o, xe, t, pc, bool(dag))
                ref = tmq.unpack(g, o, 0).cpu().numpy()
                got = np.concatenate([rk[f"op_{prec}_{pc}_{dag}"] for rk in ranks])
                assert np.array_equal(got, ref), (prec, pc, dag)
    for rk in ranks:
        it, res, conv = rk["cg"]
        assert conv == 1.0 and res <= 1e-10
    x = np.concatenate([rk["x"] for rk in ranks])
    assert np.linalg.norm(orc.apply_M(po, U, x) - psi) / np.linalg.norm(psi) < 1e-7
    g.close()
