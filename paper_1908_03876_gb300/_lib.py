"""ctypes view of the C ABI in include/cxlbm.h, include/cxarc.h and
include/cx3d.h (argument marshalling only).

Loading fails loudly if libcxlbm.so is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcxlbm.so")

CX_ANISO_CONST, CX_ANISO_ROTATED, CX_ANISO_FIELD = 0, 1, 2
CX_HALO_FWD, CX_HALO_ADJ, CX_HALO_SEED = 0, 1, 2
# the exchange callback type of cx_set_halo_exchange
HALO_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
CX_ADV_NONE, CX_ADV_ROW, CX_ADV_FIELD = 0, 1, 2

STATUS = {
    0: "CX_OK", 1: "CX_ERR_INVALID_ARG", 2: "CX_ERR_WORKSPACE", 3: "CX_ERR_CUDA", 4: "CX_ERR_STATE",
    5: "CX_ERR_UNSTABLE", 6: "CX_ERR_LINESEARCH", 7: "CX_ERR_TIMEOUT", 8: "CX_ERR_INTERNAL",
}

# every exported symbol of include/cxlbm.h
EXPORTS = [
    "cx_workspace_size", "cx_create", "cx_set_initial", "cx_forward", "cx_adjoint", "cx_adjoint_vjp",
    "cx_gradient", "cx_gradient_host", "cx_step",
    "cx_get_fields", "cx_get_psi0", "cx_get_norms", "cx_set_launch", "cx_set_timing", "cx_get_timing",
    "cx_destroy", "cx_status_string", "cx_forward_static", "cx_cg_step", "cx_cg_reset",
    "cx_tlm", "cx_lma_step", "cx_cadjoint", "cx_set_staging",
    "cx_batch_workspace_size", "cx_batch_create", "cx_batch_set_initial", "cx_batch_bind", "cx_batch_set_tiles",
    "cx_batch_forward", "cx_batch_gradient", "cx_batch_get_fields", "cx_batch_get_status", "cx_batch_destroy",
    "cx_batch_set_enabled", "cx_batch_step", "cx_batch_adjoint", "cx_batch_axpy", "cx_batch_prepare",
    "cx_batch_autotune", "cx_batch_set_staging",
    "cx_set_halo_exchange", "cx_halo_layout", "cx_halo_pack", "cx_halo_unpack", "cx_forward_trial",
    "cx_control_axpy",
    "cx_nn_conv_forward", "cx_nn_conv_backward_data", "cx_nn_conv_backward_weight_scratch",
    "cx_nn_conv_backward_weight", "cx_nn_relu_backward", "cx_nn_add", "cx_nn_pool2", "cx_nn_up2", "cx_nn_mse",
    "cx_nn_adam", "cx_nn_cast_bf16", "cx_nn_conv_forward_f32", "cx_nn_smooth", "cx_nn_packed_weights",
    "cx_nn_pack_weights", "cx_nn_conv_tc_tile", "cx_nn_conv_forward_tc", "cx_nn_conv_backward_weight_tc",
    # include/cxarc.h (three species)
    "cx3_workspace_size", "cx3_create", "cx3_set_initial", "cx3_forward", "cx3_adjoint", "cx3_gradient",
    "cx3_step", "cx3_get_fields", "cx3_get_norms", "cx3_set_staging", "cx3_set_timing", "cx3_get_timing",
    "cx3_destroy",
    # include/cx3d.h (D3Q19)
    "cx3d_workspace_size", "cx3d_create", "cx3d_set_initial", "cx3d_forward", "cx3d_adjoint", "cx3d_gradient",
    "cx3d_step", "cx3d_get_fields", "cx3d_get_norms", "cx3d_set_timing", "cx3d_get_timing", "cx3d_destroy",
]
STATIC_SCRATCH_BYTES = 64 << 20  # CX_STATIC_SCRATCH_BYTES of include/cxlbm.h


class CxError(RuntimeError):
    def __init__(self, code: int, call: str):
        self.code = code
        super().__init__(f"{call} failed: {STATUS.get(code, code)}")


class Desc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("n_steps", ctypes.c_int), ("lattice", ctypes.c_int),
        ("precision", ctypes.c_int), ("ckpt_every", ctypes.c_int), ("tau", ctypes.c_double),
        ("aniso", ctypes.c_int),
        ("D_u", ctypes.c_double * 3), ("D_v", ctypes.c_double * 3),
        ("lam_u", ctypes.c_double * 2), ("lam_v", ctypes.c_double * 2),
        ("theta", ctypes.c_void_p), ("D_u_field", ctypes.c_void_p), ("D_v_field", ctypes.c_void_p),
        ("d_u", ctypes.c_double), ("d_v", ctypes.c_double),
        ("chi", ctypes.c_double), ("r_vu", ctypes.c_double), ("r_vv", ctypes.c_double),
        ("adv", ctypes.c_int), ("a", ctypes.c_void_p),
        ("solid", ctypes.c_void_p),
        ("ctrl_x0", ctypes.c_int), ("ctrl_y0", ctypes.c_int), ("ctrl_nx", ctypes.c_int), ("ctrl_ny", ctypes.c_int),
        ("ctrl_mask", ctypes.c_void_p),
        ("u_target", ctypes.c_void_p), ("alpha", ctypes.c_double),
        ("s", ctypes.c_double * 7),
        ("source_order", ctypes.c_int),
        ("ctrl_windows", ctypes.c_int),
        ("halo", ctypes.c_int),
    ]


class Desc3(ctypes.Structure):
    """cx3_desc of include/cxarc.h."""
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("n_steps", ctypes.c_int), ("precision", ctypes.c_int),
        ("ckpt_every", ctypes.c_int), ("tau", ctypes.c_double), ("aniso", ctypes.c_int),
        ("D_u", ctypes.c_double * 3), ("D_v", ctypes.c_double * 3), ("D_w", ctypes.c_double * 3),
        ("lam_u", ctypes.c_double * 2), ("lam_v", ctypes.c_double * 2), ("lam_w", ctypes.c_double * 2),
        ("theta", ctypes.c_void_p), ("D_u_field", ctypes.c_void_p), ("D_v_field", ctypes.c_void_p),
        ("D_w_field", ctypes.c_void_p),
        ("d", ctypes.c_double), ("chi1", ctypes.c_double), ("chi2", ctypes.c_double),
        ("a1", ctypes.c_double), ("a2", ctypes.c_double),
        ("b1", ctypes.c_double), ("b2", ctypes.c_double), ("b3", ctypes.c_double),
        ("c1", ctypes.c_double), ("c2", ctypes.c_double),
        ("ctrl_species", ctypes.c_int), ("adv", ctypes.c_int), ("a", ctypes.c_void_p),
        ("u_target", ctypes.c_void_p), ("alpha", ctypes.c_double), ("s", ctypes.c_double * 7),
        ("source_order", ctypes.c_int),
    ]


class Desc3D(ctypes.Structure):
    """cx3d_desc of include/cx3d.h."""
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("n_steps", ctypes.c_int),
        ("precision", ctypes.c_int), ("ckpt_every", ctypes.c_int), ("tau", ctypes.c_double), ("aniso", ctypes.c_int),
        ("D_u", ctypes.c_double * 6), ("D_v", ctypes.c_double * 6),
        ("D_u_field", ctypes.c_void_p), ("D_v_field", ctypes.c_void_p),
        ("d_u", ctypes.c_double), ("d_v", ctypes.c_double),
        ("chi", ctypes.c_double), ("r_vu", ctypes.c_double), ("r_vv", ctypes.c_double),
        ("adv", ctypes.c_int), ("a", ctypes.c_void_p), ("u_target", ctypes.c_void_p), ("alpha", ctypes.c_double),
        ("s", ctypes.c_double * 7), ("source_order", ctypes.c_int),
    ]


class CGInfo(ctypes.Structure):
    _fields_ = [("J0", ctypes.c_double), ("J", ctypes.c_double), ("lam", ctypes.c_double),
                ("grad_sq", ctypes.c_double), ("beta", ctypes.c_double), ("trials", ctypes.c_int),
                ("restarted", ctypes.c_int)]


CG_VARIANTS = {"FR": 0, "PR": 1, "HS": 2, "DY": 3}


class StepInfo(ctypes.Structure):
    _fields_ = [("J0", ctypes.c_double), ("J", ctypes.c_double), ("lam", ctypes.c_double),
                ("grad_sq", ctypes.c_double), ("grad_inf", ctypes.c_double), ("trials", ctypes.c_int)]


_lib = None


def load():
    """Load libcxlbm.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"CUDA library {LIB_PATH} is missing; build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, cint, dp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
    D = ctypes.POINTER(Desc)
    D3 = ctypes.POINTER(Desc3)
    DD = ctypes.POINTER(Desc3D)
    sig = {
        "cx_workspace_size": [D, ctypes.POINTER(ctypes.c_size_t)],
        "cx_create": [D, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)],
        "cx_set_initial": [vp, vp, vp],
        "cx_forward": [vp, vp, vp],
        "cx_adjoint": [vp, vp, vp, vp, vp],
        "cx_adjoint_vjp": [vp, vp, vp, vp, vp],
        "cx_gradient": [vp, vp, vp, vp],
        "cx_gradient_host": [vp, vp, vp, vp, vp, vp],
        "cx_step": [vp, vp, vp, ctypes.POINTER(StepInfo)],
        "cx_get_fields": [vp, vp, vp],
        "cx_get_psi0": [vp, vp],
        "cx_get_norms": [vp, dp, dp, dp],
        "cx_set_launch": [vp, cint, cint],
        "cx_set_timing": [vp, cint],
        "cx_get_timing": [vp, dp, ctypes.POINTER(ctypes.c_longlong)],
        "cx_destroy": [vp],
        "cx_forward_static": [D, vp, vp, vp, vp, vp, vp, vp, vp],
        "cx_cg_step": [vp, vp, vp, cint, ctypes.POINTER(CGInfo)],
        "cx_cg_reset": [vp],
        "cx_tlm": [vp, vp, vp, vp, vp, dp],
        "cx_lma_step": [vp, vp, vp, ctypes.POINTER(StepInfo)],
        "cx_cadjoint": [vp, vp, vp],
        "cx_set_staging": [vp, cint],
        "cx_set_halo_exchange": [vp, vp, vp],
        "cx_halo_layout": [vp, cint, vp, vp, ctypes.POINTER(ctypes.c_size_t)],
        "cx_halo_pack": [vp, cint, vp, vp],
        "cx_halo_unpack": [vp, cint, vp, vp],
        "cx_forward_trial": [vp, vp, vp, ctypes.c_double, vp],
        "cx_control_axpy": [vp, vp, vp, ctypes.c_double],
        "cx_batch_workspace_size": [D, cint, ctypes.POINTER(ctypes.c_size_t)],
        "cx_batch_create": [D, cint, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)],
        "cx_batch_set_initial": [vp, vp, vp],
        "cx_batch_bind": [vp, vp, vp],
        "cx_batch_set_tiles": [vp, cint, cint, vp, vp],
        "cx_batch_forward": [vp, vp],
        "cx_batch_gradient": [vp, vp],
        "cx_batch_get_fields": [vp, cint, vp, vp],
        "cx_batch_get_status": [vp],
        "cx_batch_destroy": [vp],
        "cx_batch_set_enabled": [vp, vp],
        "cx_batch_step": [vp, ctypes.POINTER(StepInfo), vp],
        "cx_batch_adjoint": [vp, vp, cint, vp],
        "cx_batch_axpy": [vp, vp],
        "cx_batch_prepare": [vp],
        "cx_batch_set_staging": [vp, cint],
        "cx_batch_autotune": [vp, cint, ctypes.c_char_p, ctypes.POINTER(cint), vp, vp, dp],
        "cx_nn_conv_forward": [vp, vp, vp, vp, cint, cint, cint, cint, cint, cint, cint, vp],
        "cx_nn_conv_forward_f32": [vp, vp, vp, vp, cint, cint, cint, cint, cint, cint, vp],
        "cx_nn_smooth": [vp, vp, vp, cint, cint, cint, vp, cint, vp],
        "cx_nn_conv_backward_data": [vp, vp, vp, cint, cint, cint, cint, cint, cint, vp],
        "cx_nn_pack_weights": [vp, cint, cint, cint, vp, vp, vp],
        "cx_nn_conv_forward_tc": [vp, vp, vp, vp, cint, cint, cint, cint, cint, cint, cint, vp, vp],
        "cx_nn_conv_backward_weight": [vp, vp, vp, vp, vp, cint, cint, cint, cint, cint, cint, cint, vp],
        "cx_nn_conv_backward_weight_tc": [vp, vp, vp, vp, vp, cint, cint, cint, cint, cint, cint, cint, vp, vp],
        "cx_nn_relu_backward": [vp, vp, vp, ctypes.c_size_t, vp],
        "cx_nn_add": [vp, vp, vp, ctypes.c_size_t, vp],
        "cx_nn_pool2": [vp, vp, cint, cint, cint, cint, vp],
        "cx_nn_up2": [vp, vp, cint, cint, cint, cint, vp],
        "cx_nn_mse": [vp, vp, vp, vp, ctypes.c_size_t, vp],
        "cx_nn_adam": [vp, vp, vp, vp, vp, ctypes.c_size_t, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                       ctypes.c_float, cint, vp],
        "cx_nn_cast_bf16": [vp, vp, ctypes.c_size_t, vp],
        "cx3_workspace_size": [D3, ctypes.POINTER(ctypes.c_size_t)],
        "cx3_create": [D3, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)],
        "cx3_set_initial": [vp, vp, vp, vp],
        "cx3_forward": [vp, vp, vp],
        "cx3_adjoint": [vp, vp, vp, vp, vp, cint, vp],
        "cx3_gradient": [vp, vp, vp, vp],
        "cx3_step": [vp, vp, vp, ctypes.POINTER(StepInfo)],
        "cx3_get_fields": [vp, vp, vp, vp],
        "cx3_get_norms": [vp, dp, dp, dp],
        "cx3_set_staging": [vp, cint],
        "cx3_set_timing": [vp, cint],
        "cx3_get_timing": [vp, dp, ctypes.POINTER(ctypes.c_longlong)],
        "cx3_destroy": [vp],
        "cx3d_workspace_size": [DD, ctypes.POINTER(ctypes.c_size_t)],
        "cx3d_create": [DD, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)],
        "cx3d_set_initial": [vp, vp, vp],
        "cx3d_forward": [vp, vp, vp],
        "cx3d_adjoint": [vp, vp, vp, vp, cint, vp],
        "cx3d_gradient": [vp, vp, vp, vp],
        "cx3d_step": [vp, vp, vp, ctypes.POINTER(StepInfo)],
        "cx3d_get_fields": [vp, vp, vp],
        "cx3d_get_norms": [vp, dp, dp, dp],
        "cx3d_set_timing": [vp, cint],
        "cx3d_get_timing": [vp, dp, ctypes.POINTER(ctypes.c_longlong)],
        "cx3d_destroy": [vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = cint
    lib.cx_nn_conv_backward_weight_scratch.argtypes = [cint] * 7
    lib.cx_nn_conv_backward_weight_scratch.restype = ctypes.c_size_t
    lib.cx_nn_packed_weights.argtypes = [cint] * 4
    lib.cx_nn_conv_tc_tile.argtypes = [cint]
    lib.cx_nn_conv_tc_tile.restype = cint
    lib.cx_nn_packed_weights.restype = ctypes.c_size_t
    lib.cx_status_string.argtypes = [cint]
    lib.cx_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def check(code: int, call: str):
    if code != 0:
        raise CxError(code, call)
