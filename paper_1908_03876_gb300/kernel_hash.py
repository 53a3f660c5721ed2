"""Hash of the CUDA sources a kernel is compiled from, so that stored profiler
counters can be matched to the kernels they were taken from."""
import hashlib
import os

CSRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")

# sources of each profiled kernel (headers included)
KERNEL_SOURCES = {
    "k_forward": ("cx_device.cuh", "cx_fwd_body.cuh", "cx_internal.h", "cx_forward.cu"),
    "k_adjoint": ("cx_device.cuh", "cx_adj_body.cuh", "cx_internal.h", "cx_adjoint.cu"),
    "k_forward_rows": ("cx_device.cuh", "cx_fwd_body.cuh", "cx_internal.h", "cx_rows.cuh", "cx_forward.cu"),
    "k_adjoint_rows": ("cx_device.cuh", "cx_adj_body.cuh", "cx_internal.h", "cx_rows.cuh", "cx_adjoint.cu"),
    "k_batch": ("cx_device.cuh", "cx_fwd_body.cuh", "cx_adj_body.cuh", "cx_internal.h", "cx_state.h",
                "cx_batch.cu"),
    "k_batch_rows": ("cx_device.cuh", "cx_fwd_body.cuh", "cx_adj_body.cuh", "cx_internal.h", "cx_state.h",
                     "cx_batch.cu"),
    "k_tlm": ("cx_device.cuh", "cx_internal.h", "cx_tlm.cu"),
    "k_cadj": ("cx_device.cuh", "cx_internal.h", "cx_cadj.cu"),
    "k_tlm_rows": ("cx_device.cuh", "cx_internal.h", "cx_tlm.cu"),
    "k_cadj_rows": ("cx_device.cuh", "cx_internal.h", "cx_cadj.cu"),
    "k3_forward": ("cx_device.cuh", "cx_internal.h", "cx_rows.cuh", "cx_arc.cu"),
    "k3_forward_rows": ("cx_device.cuh", "cx_internal.h", "cx_rows.cuh", "cx_arc.cu"),
    "k3_adjoint": ("cx_device.cuh", "cx_internal.h", "cx_rows.cuh", "cx_arc.cu"),
    "k3d_forward": ("cx_device.cuh", "cx_internal.h", "cx_d3q19.cuh", "cx_d3q19_kernels.cuh", "cx_d3q19.cu"),
    "k3d_adjoint": ("cx_device.cuh", "cx_internal.h", "cx_d3q19.cuh", "cx_d3q19_kernels.cuh", "cx_d3q19.cu"),
    "nn": ("nn_kernels.cu",),
}


def kernel_source_hash(kernel=None) -> str:
    """Hash of the sources of `kernel` (a key of KERNEL_SOURCES), or of every
    CUDA source when kernel is None."""
    names = KERNEL_SOURCES[kernel] if kernel else sorted(
        n for n in os.listdir(CSRC) if n.endswith((".cu", ".cuh", ".h")))
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(CSRC, name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]
