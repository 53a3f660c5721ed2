"""Domain decomposition of one problem on the GPU: blocks with halo frames,
exchanges through the library's pack/unpack kernels after every step, FP64
all-reduces for the cost and the line search.  Fields, gradients and
vector-Jacobian products of the decomposed solve equal the single-domain
solve's bit for bit (every node runs the same arithmetic on the same inputs);
the cost, a sum over blocks in another order, to rounding.

The multi-rank cases run 2 and 4 processes with the gloo transport (halo
slots through host memory), all on one GPU: no kernel waits on another
process, every exchange is ordered on the host."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from _decomp_cases import make_case  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_03876_gb300.build import build

    build()


def _reference(case):
    """Single-domain results: J, dJ/dg, u^N, v^N, the VJP and two Armijo steps."""
    from paper_1908_03876_gb300.problem import Problem

    w, g, su, sv = make_case(case)
    p = Problem(w)
    gt = torch.as_tensor(g, dtype=torch.float64, device="cuda").contiguous()
    J, E = p.gradient(gt)
    J = float(J.item())
    u, v = p.fields()
    p.forward(gt)
    V = p.vjp(gt, su, sv)
    gs = gt.clone()
    infos = [p.step(gs) for _ in range(2)]
    return dict(w=w, g=g, J=J, E=E.cpu().numpy(), u=u.cpu().numpy(), v=v.cpu().numpy(), V=V.cpu().numpy(),
                gs=gs.cpu().numpy(), lam=[i["lam"] for i in infos], trials=[i["trials"] for i in infos],
                Js=[i["J"] for i in infos])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("case", ["aniso", "geometry"])
def test_one_block_with_self_halo_equals_single_domain(case):
    """A 1 x 1 partition: the block's frame is filled from its own opposite
    edges through the pack/unpack kernels (periodic images)."""
    from paper_1908_03876_gb300.decomp import DecomposedProblem, Partition

    ref = _reference(case)
    w, g, su, sv = make_case(case)
    dp = DecomposedProblem(w, Partition(w.nx, w.ny, 1, 1), 0)
    gl = torch.as_tensor(dp.local_control(g), dtype=torch.float64, device="cuda").contiguous()
    J, E = dp.gradient(gl)
    u, v = dp.fields()
    dp.forward(gl)
    V = dp.vjp(gl, su, sv)
    assert abs(J - ref["J"]) <= 1e-13 * abs(ref["J"])
    for a, b, name in ((E, ref["E"], "dJ/dg"), (u, ref["u"], "u"), (v, ref["v"], "v"), (V, ref["V"], "vjp")):
        nd = int(np.count_nonzero(a.cpu().numpy() != b))
        print(f"{case} 1x1: {name} entries differing from the single domain: {nd}")
        assert nd == 0, name
    gs = gl.clone()
    for k in range(2):
        info = dp.step(gs)
        assert info["lam"] == ref["lam"][k] and info["trials"] == ref["trials"][k]
        assert abs(info["J"] - ref["Js"][k]) <= 1e-13 * abs(ref["Js"][k])
    assert np.array_equal(gs.cpu().numpy(), ref["gs"])
    dp.close()


@pytest.mark.parametrize("case", ["aniso", "geometry"])
@pytest.mark.parametrize("world,px,py", [(2, 2, 1), (4, 2, 2)])
def test_decomposed_ranks_equal_single_domain(tmp_path, case, world, px, py):
    """world gloo ranks on 2 x 1 or 2 x 2 blocks: every block's u^N, v^N,
    dJ/dg, VJP and Armijo-updated control equal the single domain's bit for
    bit; J to 1e-13."""
    import torch.multiprocessing as mp

    import _decomp_worker

    ref = _reference(case)
    mp.start_processes(_decomp_worker.solve_rank, args=(world, _free_port(), px, py, case, str(tmp_path)),
                       nprocs=world, start_method="spawn", join=True)
    w = ref["w"]
    wx0, wy0, wcx, wcy = w.win
    for r in range(world):
        b = np.load(os.path.join(tmp_path, f"block{r}.npz"))
        x0, y0, lx, ly = (int(t) for t in b["block"])
        assert abs(float(b["J"]) - ref["J"]) <= 1e-13 * abs(ref["J"])
        for name in ("u", "v"):
            assert np.array_equal(b[name], ref[name][y0:y0 + ly, x0:x0 + lx]), (r, name)
        cx0, cx1 = max(wx0, x0), min(wx0 + wcx, x0 + lx)
        cy0, cy1 = max(wy0, y0), min(wy0 + wcy, y0 + ly)
        if cx1 > cx0 and cy1 > cy0:
            sl = (slice(None), slice(cy0 - wy0, cy1 - wy0), slice(cx0 - wx0, cx1 - wx0))
            for name in ("E", "V", "gs"):
                assert np.array_equal(b[name], ref[name][sl]), (r, name)
        assert list(b["lam"]) == ref["lam"] and list(b["trials"]) == ref["trials"]
        assert np.allclose(b["Js"], ref["Js"], rtol=1e-13, atol=0)
    print(f"{case}: {world} ranks ({px} x {py} blocks) equal to the single domain")
