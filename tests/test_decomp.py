"""Domain decomposition of one problem (host logic, CPU): the block partition,
the sub-problem fields over each block's interior and halo frame, and the
halo transport between gloo ranks (world sizes 2 and 4)."""
import os
import socket

import numpy as np
import pytest

from paper_1908_03876_gb300 import workloads as W
from paper_1908_03876_gb300.decomp import DIRS, OPP, Partition, block_workload


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("px,py", [(1, 1), (2, 1), (2, 2), (3, 2)])
def test_partition_tiles_the_grid(px, py):
    part = Partition(37, 29, px, py)
    cover = np.zeros((29, 37), int)
    for r in range(part.size):
        x0, y0, lx, ly = part.block(r)
        cover[y0:y0 + ly, x0:x0 + lx] += 1
        for d, (dx, dy) in DIRS.items():
            nb = part.neighbour(r, d)
            assert part.neighbour(nb, OPP[d]) == r  # the neighbour's opposite neighbour is this block
            bx, by = part.coords(r)
            assert part.coords(nb) == ((bx + dx) % px, (by + dy) % py)
    assert (cover == 1).all()


def test_block_fields_are_the_global_fields_with_periodic_frame():
    w = W.geometry(30, 26, 5, seed=2, precision=64, win=12, rmin=2, rmax=4)
    w.window = (5, 3, 14, 12)
    w.cmask = np.random.default_rng(0).integers(0, 2, (12, 14)).astype(np.uint8)
    part = Partition(w.nx, w.ny, 3, 2)
    seen = np.zeros((12, 14), int)
    for r in range(part.size):
        x0, y0, lx, ly = part.block(r)
        b = block_workload(w, part, r)
        assert (b.nx, b.ny, b.halo) == (lx + 2, ly + 2, 1)
        for name in ("theta", "u0", "v0", "u_tgt", "solid"):
            ref = np.roll(np.roll(getattr(w, name), 1 - y0, axis=0), 1 - x0, axis=1)[:ly + 2, :lx + 2]
            assert np.array_equal(getattr(b, name), ref), name
        sl = b.extra["ctrl_slice"]
        if sl is None:
            assert b.window == (0, 0, 1, 1)
            continue
        cx, cy, cnx, cny = sl
        bx0, by0, bnx, bny = b.window
        assert (bnx, bny) == (cnx, cny)
        # the local window maps onto the same global nodes as the slice of the global window
        assert (x0 + bx0 - 1, y0 + by0 - 1) == (w.window[0] + cx, w.window[1] + cy)
        assert 1 <= bx0 and bx0 + bnx <= lx + 1 and 1 <= by0 and by0 + bny <= ly + 1
        assert np.array_equal(b.cmask, w.cmask[cy:cy + cny, cx:cx + cnx])
        seen[cy:cy + cny, cx:cx + cnx] += 1
    assert (seen == 1).all()  # every controlled node belongs to exactly one block


@pytest.mark.parametrize("world,px,py", [(2, 2, 1), (2, 1, 2), (4, 2, 2)])
def test_halo_transport_between_gloo_ranks(tmp_path, world, px, py):
    """Every receive slot d holds what the block at e_d sent toward this block
    (its slot opp(d)), including messages to itself and several messages
    between the same pair of ranks (periodic wrap with two blocks per axis)."""
    import torch.multiprocessing as mp

    import _decomp_worker

    mp.start_processes(_decomp_worker.exchange_rank, args=(world, _free_port(), px, py, str(tmp_path)),
                       nprocs=world, start_method="spawn", join=True)
    part = Partition(12, 10, px, py)
    for r in range(world):
        got = np.load(os.path.join(tmp_path, f"recv{r}.npy"))
        _, _, lx, ly = part.block(r)
        sizes = [3 * (ly if d in (1, 3) else lx) if d <= 4 else 1 for d in range(1, 9)]
        offs = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
        for d in range(1, 9):
            src = part.neighbour(r, d)
            expect = np.arange(sizes[d - 1]) + 1000 * OPP[d] + 100000 * src
            assert np.array_equal(got[offs[d - 1]:offs[d]], expect), (r, d)
