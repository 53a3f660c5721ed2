"""Workloads of the domain-decomposition tests (helper module, not collected)."""
import numpy as np

from paper_1908_03876_gb300 import workloads as W


def make_case(case):
    """(workload, global control, seed_u, seed_v) of a named case, FP64."""
    if case == "aniso":  # rotated tensors, shear convection, chemotaxis, windowed control in time
        w = W.aniso(36, 28, 14, seed=3, precision=64, ckpt_every=5)
        w.windows = 7
        w.chi = -0.3
    elif case == "geometry":  # solid discs and frame, bounce-back, masked control window
        w = W.geometry(40, 36, 12, seed=4, precision=64, ckpt_every=4, win=20, rmin=2, rmax=5)
    else:
        raise ValueError(case)
    g = w.random_control(31, 0.05)
    rng = np.random.default_rng(32)
    su, sv = rng.standard_normal((w.ny, w.nx)), rng.standard_normal((w.ny, w.nx))
    if w.solid is not None:
        su *= 1 - w.solid
        sv *= 1 - w.solid
    return w, g, su, sv
