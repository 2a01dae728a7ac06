"""The fused operator's work list (host logic, no GPU): every second-pass group is claimed after
the first-pass groups that hold its sites' neighbours, so every bounded wait in the fused
launch is for work a running block has already claimed (no wait can depend on unclaimed work)."""
import ctypes

import numpy as np
import pytest

GROUP = 4 * 128  # sites per work item


@pytest.fixture(scope="module")
def lib():
    from paper_1311_4462_gb300 import build
    from paper_1311_4462_gb300 import _lib
    build.build()
    return _lib.load()


def work_list(lib, L, num_sms=152):
    Lc = (ctypes.c_int * 4)(*L)
    n = lib.tm_fused_work_list(Lc, num_sms, None, 0)
    assert n > 0
    buf = (ctypes.c_int * n)()
    assert lib.tm_fused_work_list(Lc, num_sms, buf, n) == n
    return np.frombuffer(buf, dtype=np.int32).copy()


def neighbour_cbs(L):
    """cb of the 8 neighbours of every even site, [Vh, 8] (periodic, lexicographic x fastest)."""
    Lx, Ly, Lz, Lt = L
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    even = ((x + y + z + t) % 2) == 0
    coords = [c[even] for c in (x, y, z, t)]
    lexe = coords[0] + Lx * (coords[1] + Ly * (coords[2] + Lz * coords[3]))
    order = np.argsort(lexe // 2)
    out = []
    for d in range(4):
        for s in (1, -1):
            c = [v.copy() for v in coords]
            c[d] = (c[d] + s) % L[d]
            lex = c[0] + Lx * (c[1] + Ly * (c[2] + Lz * c[3]))
            out.append((lex // 2)[order])
    return np.stack(out, axis=1)


@pytest.mark.parametrize("L", [(2, 2, 2, 2), (4, 4, 4, 6), (6, 4, 2, 10), (8, 8, 8, 16), (16, 16, 16, 32),
                               (24, 24, 24, 48), (32, 32, 32, 32), (8, 8, 8, 128), (64, 8, 8, 8), (32, 32, 32, 64)])
@pytest.mark.parametrize("num_sms", [1, 152])
def test_dependencies_come_first(lib, L, num_sms):
    items = work_list(lib, L, num_sms)
    Vh = int(np.prod(L)) // 2
    ngroups = (Vh + GROUP - 1) // GROUP
    assert len(items) == 2 * ngroups and len(set(items.tolist())) == 2 * ngroups
    pos = np.empty(2 * ngroups, dtype=np.int64)
    pos[items] = np.arange(len(items))  # pos[(group << 1) | pass]
    nb = neighbour_cbs(L)                # [Vh, 8] odd-field cb read by each even output site
    site_group = np.arange(Vh) // GROUP
    b_pos = pos[(site_group << 1) | 1]
    a_pos = pos[(nb // GROUP) << 1]
    assert (a_pos < b_pos[:, None]).all()


def test_invalid_extents(lib):
    assert lib.tm_fused_work_list((ctypes.c_int * 4)(3, 4, 4, 4), 152, None, 0) == -1
    Lc = (ctypes.c_int * 4)(4, 4, 4, 4)
    n = lib.tm_fused_work_list(Lc, 152, None, 0)
    assert lib.tm_fused_work_list(Lc, 152, (ctypes.c_int * 1)(), 1) == (-1 if n > 1 else n)
