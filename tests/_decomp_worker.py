"""Rank body of the multi-process domain-decomposition tests (spawned; not a test module)."""
import os

import numpy as np


def exchange_rank(rank, world, port, px, py, out_dir):
    """CPU gloo rank: fill each send slot with values naming (rank, direction,
    index), exchange, and save what arrived."""
    import torch
    import torch.distributed as dist

    from paper_1908_03876_gb300.decomp import Partition, exchange_slots

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        part = Partition(12, 10, px, py)
        _, _, lx, ly = part.block(rank)
        # slot d: 3 planes of a face (ly or lx cells) or 1 corner cell, int32 values
        sizes = [3 * (ly if d in (1, 3) else lx) if d <= 4 else 1 for d in range(1, 9)]
        offs = np.concatenate([[0], np.cumsum(sizes)]).astype(int) * 4
        total = int(offs[-1])
        send = torch.zeros(total, dtype=torch.uint8)
        vals = send.view(torch.int32)
        for d in range(1, 9):
            n = sizes[d - 1]
            vals[offs[d - 1] // 4:offs[d] // 4] = torch.arange(n, dtype=torch.int32) + 1000 * d + 100000 * rank
        # the receive slot d holds what the neighbour at e_d sent as its slot opp(d): same size here
        recv = torch.full((total,), 255, dtype=torch.uint8)
        exchange_slots(send, recv, list(offs[:-1]), list(offs[:-1]), total, part, rank)
        np.save(os.path.join(out_dir, f"recv{rank}.npy"), recv.view(torch.int32).numpy())
    finally:
        dist.destroy_process_group()


def solve_rank(rank, world, port, px, py, case, out_dir):
    """GPU rank (gloo transport, all ranks on cuda:0): the decomposed forward,
    gradient, vector-Jacobian product and two Armijo iterations of block
    `rank`; saves the block's results."""
    import torch
    import torch.distributed as dist

    from paper_1908_03876_gb300.decomp import DecomposedProblem, Partition
    from _decomp_cases import make_case

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        w, g, su, sv = make_case(case)
        part = Partition(w.nx, w.ny, px, py)
        dp = DecomposedProblem(w, part, rank)
        x0, y0, lx, ly = part.block(rank)
        gl = torch.as_tensor(dp.local_control(g), dtype=dp.dtype, device=dp.device).contiguous()
        J, E = dp.gradient(gl)
        u, v = dp.fields()
        dp.forward(gl)
        V = dp.vjp(gl, su[y0:y0 + ly, x0:x0 + lx], sv[y0:y0 + ly, x0:x0 + lx])
        gs = gl.clone()
        infos = [dp.step(gs) for _ in range(2)]
        np.savez(os.path.join(out_dir, f"block{rank}.npz"), J=J, E=E.cpu().numpy(), u=u.cpu().numpy(),
                 v=v.cpu().numpy(), V=V.cpu().numpy(), gs=gs.cpu().numpy(),
                 lam=[i["lam"] for i in infos], trials=[i["trials"] for i in infos], Js=[i["J"] for i in infos],
                 block=(x0, y0, lx, ly))
        dp.close()
    finally:
        dist.destroy_process_group()
