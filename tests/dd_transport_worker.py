"""One rank of a CPU-only gloo run of the decomposed lattice's transport (driven by
tests/test_dd_transport.py): every rank sends tagged face buffers to its neighbours and checks what
it receives, then sums a value with the transport's allreduce."""
import os
import sys

import torch
import torch.distributed as dist

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1311_4462_gb300 import dd  # noqa: E402


def main():
    dist.init_process_group("gloo")
    rank, world = dist.get_rank(), dist.get_world_size()
    tr = dd.TorchDistTransport()
    f = dd.Faces(24, device="cpu")
    for rep in range(3):
        f.send_next.fill_((rank * 16 + 1 + rep) % 256)
        f.send_prev.fill_((rank * 16 + 2 + rep) % 256)
        f.recv_prev.zero_()
        f.recv_next.zero_()
        tr.exchange_buffers(f)
        prv, nxt = (rank - 1) % world, (rank + 1) % world
        assert int(f.recv_prev[0]) == (prv * 16 + 1 + rep) % 256, (rank, rep, int(f.recv_prev[0]))
        assert int(f.recv_next[0]) == (nxt * 16 + 2 + rep) % 256, (rank, rep, int(f.recv_next[0]))
        assert bool((f.recv_prev == f.recv_prev[0]).all()) and bool((f.recv_next == f.recv_next[0]).all())
    total = tr.allreduce([0.5 * rank, 0.25])
    assert total == sum(0.5 * r + 0.25 for r in range(world)), total
    assert dd.slab_bounds(8 * world, world) == [(8 * r, 8) for r in range(world)]
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
