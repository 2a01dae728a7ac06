"""One rank of a two-process run of the decomposed operator (driven by tests/test_gpu_dd_procs.py
under torch.distributed.run): both ranks share the GPU, each holds one time slab, faces cross as
gloo messages through host memory.  Writes this rank's outputs to <out>.rank<r>.npz."""
import os
import sys

import numpy as np
import torch
import torch.distributed as dist

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import paper_1311_4462_gb300 as tmq  # noqa: E402
from paper_1311_4462_gb300 import dd, inputs  # noqa: E402


def main():
    out = sys.argv[1]
    L = tuple(int(v) for v in sys.argv[2].split(","))
    flavor, kappa, mu, eps, seed = int(sys.argv[3]), float(sys.argv[4]), float(sys.argv[5]), float(sys.argv[6]), int(sys.argv[7])
    torch.cuda.set_device(0)
    dist.init_process_group("gloo")
    rank, world = dist.get_rank(), dist.get_world_size()
    p = tmq.Params(L, kappa, mu, eps, flavor=flavor, recon=12)
    U = torch.from_numpy(inputs.gauge_field(L, seed)).to("cuda")
    psi = torch.from_numpy(inputs.spinor_field(L, p.nf, seed + 1000)).to("cuda")
    (slab,) = dd.make_slabs(p, U, world, ranks=[rank])
    tr = dd.TorchDistTransport()
    res = {}
    for prec in (8, 4):
        (xe,) = dd.pack_slabs([slab], dd.split_field([slab], psi), 0, prec)
        o, t = slab.field(prec), slab.field(prec)
        for pc in (0, 1):
            for dag in (0, 1):
                dd.precond_op([slab], [o], [xe], [t], tr, pc, bool(dag))
                res[f"op_{prec}_{pc}_{dag}"] = tmq.unpack(slab.g, o, 0).cpu().numpy()
    parts = dd.split_field([slab], psi)
    be, bo = dd.pack_slabs([slab], parts, 0), dd.pack_slabs([slab], parts, 1)
    bp, xe, xo = [slab.field()], [slab.field()], [slab.field()]
    dd.prepare_rhs([slab], bp, be, bo, tr)
    st = dd.cg([slab], xe, bp, tr, tol=1e-10)
    dd.reconstruct_odd([slab], xo, bo, xe, tr)
    x = tmq.unpack(slab.g, xe[0], 0)
    tmq.unpack(slab.g, xo[0], 1, canon=x)
    res["x"] = x.cpu().numpy()
    res["cg"] = np.array([st["iterations"], st["true_residual"], float(st["converged"])])
    res["t0"] = np.array([slab.t0, slab.lt])
    torch.cuda.synchronize()
    np.savez(f"{out}.rank{rank}.npz", **res)
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
