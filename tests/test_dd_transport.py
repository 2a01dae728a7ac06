"""Host logic of the decomposed lattice's transport on CPU (gloo, 1-3 ranks, no GPU): each rank's
face for the next slab arrives as that slab's face from the previous one and vice versa, also when
both neighbours are the same rank (two ranks) or the rank itself (one); reductions are summed over
the ranks; the slab bounds split the time extent evenly."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [1, 2, 3])
def test_face_exchange_and_allreduce_over_gloo(world):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={world}",
           "--master-addr=127.0.0.1", f"--master-port={_port()}", os.path.join(ROOT, "tests", "dd_transport_worker.py")]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-3000:]


def test_slab_bounds():
    from paper_1311_4462_gb300 import dd
    assert dd.slab_bounds(12, 3) == [(0, 4), (4, 4), (8, 4)]
    assert dd.slab_bounds(8, 4) == [(0, 2), (2, 2), (4, 2), (6, 2)]
    for Lt, n in ((8, 3), (12, 4), (6, 2)):
        with pytest.raises(ValueError):
            dd.slab_bounds(Lt, n)
