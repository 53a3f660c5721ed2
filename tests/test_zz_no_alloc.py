"""cx_forward_static: the forward solve for callers that cannot allocate
device memory (a host callback, a plug-in inside another runtime, a process
whose device memory belongs to a pool it does not control).

It must give what the workspace-based path gives (cx_create + cx_set_initial
+ cx_forward + cx_get_fields) for the same descriptor, on two calls in a row
(the shared static scratch keeps the previous call's contents), and reject a
problem larger than its fixed scratch.  This file is collected last so that a
run stopping at the first failure has already run every other test; it also
passes when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_03876_gb300 import workloads as W  # noqa: E402

TOL = {64: 1e-12, 32: 1e-4}  # relative L2, as the parity tests


def _static(prob, g):
    """One cx_forward_static call; returns (return code, J, u^N, v^N, device status code)."""
    from paper_1908_03876_gb300 import _lib

    lib = _lib.load()
    w = prob.w
    u0 = torch.as_tensor(w.u0, dtype=prob.dtype, device=prob.device).contiguous()
    v0 = torch.as_tensor(w.v0, dtype=prob.dtype, device=prob.device).contiguous()
    J = torch.zeros(1, dtype=torch.float64, device=prob.device)
    uN = torch.empty((w.ny, w.nx), dtype=prob.dtype, device=prob.device)
    vN = torch.empty_like(uN)
    st = torch.full((1,), -1, dtype=torch.int32, device=prob.device)
    gp = None if g is None else ctypes.c_void_p(g.data_ptr())
    rc = lib.cx_forward_static(ctypes.byref(prob.desc), ctypes.c_void_p(u0.data_ptr()),
                               ctypes.c_void_p(v0.data_ptr()), gp, ctypes.c_void_p(J.data_ptr()),
                               ctypes.c_void_p(uN.data_ptr()), ctypes.c_void_p(vN.data_ptr()),
                               ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(prob.stream.cuda_stream))
    torch.cuda.synchronize()
    return rc, float(J.item()), uN, vN, int(st.item())


def _rel(a, b):
    return float((a.double() - b.double()).norm() / b.double().norm())


def _case(name):
    if name.startswith("geometry"):  # solid discs, bounce-back, masked control window: per-thread staging
        return W.geometry(96, 80, 30, seed=2, precision=int(name[-2:]), ckpt_every=8, win=40, rmin=3, rmax=9)
    # 128 x 2048 FP32 without solids: 2048 row segments, at least two per block of the persistent
    # grid, so the steps after the first run the row-window kernel; rotated tensors, with and
    # without the shear convection
    w = W.aniso(128, 2048, 6, seed=3, precision=32, ckpt_every=6)
    if name == "aniso_noadv32":
        w.adv, w.a_row = "none", None
    return w


@pytest.mark.parametrize("case", ["geometry64", "geometry32", "aniso32", "aniso_noadv32"])
def test_static_forward_matches_workspace_path_twice(case):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_03876_gb300.build import build
    from paper_1908_03876_gb300.problem import Problem

    build()
    w = _case(case)
    precision = w.precision
    prob = Problem(w)
    for seed in (1, 2):  # two calls in a row, different controls
        g = torch.as_tensor(w.random_control(seed, 0.02), dtype=prob.dtype, device=prob.device).contiguous()
        J_ref = float(prob.forward(g).item())
        u_ref, v_ref = prob.fields()
        torch.cuda.synchronize()
        rc, J, uN, vN, st = _static(prob, g)
        assert rc == 0 and st == 0
        eJ = abs(J - J_ref) / abs(J_ref)
        eu, ev = _rel(uN, u_ref), _rel(vN, v_ref)
        print(f"static vs workspace ({case}, control {seed}): J {eJ:.1e} u {eu:.1e} v {ev:.1e}")
        assert eJ < TOL[precision] and eu < TOL[precision] and ev < TOL[precision]


def test_static_forward_rejects_too_large():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_03876_gb300 import _lib
    from paper_1908_03876_gb300.problem import Problem

    w = W.aniso(1024, 1024, 2, seed=1, precision=32, ckpt_every=2)  # about 250 MB of scratch
    prob = Problem(w)
    rc, _, _, _, _ = _static(prob, None)
    assert rc == 2  # CX_ERR_WORKSPACE: larger than CX_STATIC_SCRATCH_BYTES
    assert _lib.STATIC_SCRATCH_BYTES == 64 << 20
