"""Seeded synthetic inputs for the chemotaxis optimal-control workloads.

This module only draws and shapes input data (initial states, targets,
diffusion-tensor fields, convection fields, solid masks, control windows and
random controls).  It holds none of the method's arithmetic, so both the CUDA
path and the CPU oracle may use it.

Named workloads (sizes and physics from the project's benchmark definitions;
the paper itself has no numerical experiments):
  * ``plain64``   -- 64x64 periodic D2Q5, FP64, 200 steps, isotropic D_u = 0.05 I,
    D_v = 0.2 I, chi = -0.05, Phi_v = 0.5 u - 0.1 v + g; u0 = 1 + 0.2 * four
    Gaussian bumps (sigma 4); u_target = one centred Gaussian (sigma 8, same mass).
  * ``aniso1024`` -- 1024x1024 periodic D2Q9, FP32, 2000 steps; D_u = D_v =
    R(theta(x)) diag(0.08, 0.02) R^T with a smoothly varying seeded angle;
    shear convection a = (0.05 sin(2 pi y / L), 0); chi = -0.1; checkpoint every 100.
  * ``geom4096``  -- 4096x4096 D2Q9 with a random-disc solid mask (radii 8..40,
    20% solid) and a solid frame, 5000 steps, control on a 256x256 window.
  * ``batch``     -- independent problems of sizes {64,128,256,512}^2 with random
    chi, anisotropy ratio and angle (see ``batch_workloads``).
Every generator takes explicit sizes so the tests can build small versions.

Chemotactic sensitivity.  With the source rates above, an attractive
sensitivity (chi > 0) of order 0.5-1 is deep in the Keller-Segel aggregation
regime: the PDE itself amplifies grid-scale modes by about e^{0.4} per step and
the solution collapses within a few tens of steps.  The workloads therefore use
the same magnitudes divided by ten with the repulsive sign (chi -> -chi/10),
which is stable for thousands of steps; chi is a signed parameter everywhere.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    N: int
    Q: int = 9
    precision: int = 64
    # diffusion tensors: "const" (D_u_const/D_v_const), "rotated" (lam_* along
    # the angle field theta), or "field" (D_u_field/D_v_field per node)
    aniso: str = "const"
    D_u_const: tuple = (0.05, 0.0, 0.05)
    D_v_const: tuple = (0.2, 0.0, 0.2)
    lam_u: tuple = (0.08, 0.02)
    lam_v: tuple = (0.08, 0.02)
    theta: np.ndarray | None = None
    D_u_field: np.ndarray | None = None
    D_v_field: np.ndarray | None = None
    d_u: float = 1.0
    d_v: float = 1.0
    chi: float = 0.5
    r_vu: float = 0.5
    r_vv: float = -0.1
    # convection: "none", "row" (a depends on y only, a_row [ny,2]) or "field"
    adv: str = "none"
    a_row: np.ndarray | None = None
    a_field: np.ndarray | None = None
    solid: np.ndarray | None = None
    window: tuple | None = None
    cmask: np.ndarray | None = None
    u0: np.ndarray = None
    v0: np.ndarray = None
    u_tgt: np.ndarray = None
    alpha: float = 1e-3
    s: tuple = (1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0)
    source_order: int = 2
    ckpt_every: int = 0
    windows: int = 0          # W > 0: control piecewise constant over W equal time windows
    halo: int = 0             # 1: a sub-domain whose outer one-node frame holds ghost copies of its neighbours
    extra: dict = field(default_factory=dict)

    # ---- views of the same inputs in per-node form (input shaping only)
    @property
    def win(self):
        return self.window or (0, 0, self.nx, self.ny)

    @property
    def ctrl_shape(self):
        w = self.win
        return (self.windows or self.N, w[3], w[2])

    def D_fields(self):
        """Per-node (Dxx, Dxy, Dyy) for both species, [ny, nx, 3] each."""
        if self.aniso == "field":
            return self.D_u_field, self.D_v_field
        if self.aniso == "const":
            Du = np.broadcast_to(np.asarray(self.D_u_const, float), (self.ny, self.nx, 3)).copy()
            Dv = np.broadcast_to(np.asarray(self.D_v_const, float), (self.ny, self.nx, 3)).copy()
            return Du, Dv
        return rotated_tensor(self.lam_u, self.theta), rotated_tensor(self.lam_v, self.theta)

    def a_fields(self):
        """Per-node convection velocity [ny, nx, 2] or None."""
        if self.adv == "none":
            return None
        if self.adv == "row":
            return np.broadcast_to(self.a_row[:, None, :], (self.ny, self.nx, 2)).copy()
        return self.a_field

    def random_control(self, seed: int, scale: float = 0.01):
        rng = np.random.default_rng(seed)
        g = scale * rng.standard_normal(self.ctrl_shape)
        if self.cmask is not None:
            g = g * self.cmask[None]
        if self.solid is not None:
            x0, y0, cx, cy = self.win
            g = g * (1 - self.solid[y0:y0 + cy, x0:x0 + cx])[None]
        return g


def rotated_tensor(lam, theta):
    """(Dxx, Dxy, Dyy) of R(theta) diag(lam1, lam2) R(theta)^T, per node."""
    c, s = np.cos(theta), np.sin(theta)
    l1, l2 = lam
    return np.stack([l1 * c * c + l2 * s * s, (l1 - l2) * s * c, l1 * s * s + l2 * c * c], axis=-1)


def _periodic_gauss(nx, ny, cx, cy, sigma):
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    dx = np.minimum(np.abs(x - cx), nx - np.abs(x - cx))
    dy = np.minimum(np.abs(y - cy), ny - np.abs(y - cy))
    return np.exp(-(dx * dx + dy * dy) / (2.0 * sigma * sigma))


def bumps(nx, ny, seed, sigma, n_bumps=4, amp=0.2, base=1.0):
    rng = np.random.default_rng(seed)
    cs = rng.uniform(0, 1, size=(n_bumps, 2))
    u = np.full((ny, nx), base)
    for cxf, cyf in cs:
        u += amp * _periodic_gauss(nx, ny, cxf * nx, cyf * ny, sigma)
    return u


def plain64(nx=64, ny=64, N=200, seed=0, sigma=4.0, Q=5, chi=-0.05):
    """Isotropic FP64 problem (D2Q5 by default)."""
    u0 = bumps(nx, ny, seed, sigma)
    u_tgt = 1.0 + 0.2 * _periodic_gauss(nx, ny, nx / 2, ny / 2, 2 * sigma)
    return Workload(name="plain64", nx=nx, ny=ny, N=N, Q=Q, precision=64, aniso="const",
                    D_u_const=(0.05, 0.0, 0.05), D_v_const=(0.2, 0.0, 0.2), chi=chi,
                    r_vu=0.5, r_vv=-0.1, u0=u0, v0=np.zeros((ny, nx)), u_tgt=u_tgt,
                    alpha=1e-3, ckpt_every=N)


def _angle_field(nx, ny, seed):
    rng = np.random.default_rng(seed)
    r0, p1, p2 = rng.uniform(0, 1), rng.uniform(0, 2 * np.pi), rng.uniform(0, 2 * np.pi)
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    return np.pi * (r0 + 0.25 * np.sin(2 * np.pi * x / nx + p1) * np.sin(2 * np.pi * y / ny + p2))


def aniso(nx=1024, ny=1024, N=2000, seed=1, precision=32, ckpt_every=100, chi=-0.1):
    """Anisotropic rotated-tensor problem with shear convection (D2Q9)."""
    L = nx
    theta = _angle_field(nx, ny, seed)
    y = np.arange(ny)
    a_row = np.stack([0.05 * np.sin(2 * np.pi * y / ny), np.zeros(ny)], axis=-1)
    sig = L / 16.0
    u0 = bumps(nx, ny, seed, sig)
    u_tgt = 1.0 + 0.2 * _periodic_gauss(nx, ny, nx / 2, ny / 2, 2 * sig)
    return Workload(name="aniso", nx=nx, ny=ny, N=N, Q=9, precision=precision, aniso="rotated",
                    lam_u=(0.08, 0.02), lam_v=(0.08, 0.02), theta=theta, chi=chi, r_vu=0.5,
                    r_vv=-0.1, adv="row", a_row=a_row, u0=u0, v0=np.zeros((ny, nx)), u_tgt=u_tgt,
                    alpha=1e-3, ckpt_every=ckpt_every)


def disc_mask(nx, ny, seed, rmin=8, rmax=40, fraction=0.2):
    """Random solid discs until the solid fraction is reached, a 1-cell solid
    frame, and fluid pockets cut off from the main fluid region filled."""
    rng = np.random.default_rng(seed)
    solid = np.zeros((ny, nx), dtype=np.uint8)
    y = np.arange(ny)[:, None]
    x = np.arange(nx)[None, :]
    while solid.mean() < fraction:
        r = rng.uniform(rmin, rmax)
        cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
        x0, x1 = int(max(0, cx - r - 1)), int(min(nx, cx + r + 2))
        y0, y1 = int(max(0, cy - r - 1)), int(min(ny, cy + r + 2))
        sub = (x[:, x0:x1] - cx) ** 2 + (y[y0:y1] - cy) ** 2 <= r * r
        solid[y0:y1, x0:x1] |= sub.astype(np.uint8)
    solid[0, :] = solid[-1, :] = 1
    solid[:, 0] = solid[:, -1] = 1
    try:
        from scipy import ndimage

        lab, n = ndimage.label(solid == 0)
        if n > 1:
            sizes = ndimage.sum(np.ones_like(lab), lab, index=np.arange(1, n + 1))
            keep = 1 + int(np.argmax(sizes))
            solid[(lab != keep) & (solid == 0)] = 1
    except ImportError:  # pragma: no cover - scipy is present on both machines
        pass
    return solid


def geometry(nx=4096, ny=4096, N=5000, seed=2, precision=32, ckpt_every=100, win=256,
             rmin=8, rmax=40):
    """Complex geometry: disc mask, bounce-back, control on a window strip.

    No convection: a velocity field that crosses the solid walls is not
    admissible there (the bounce-back walls carry no mass flux), and it makes
    the local grad-v estimate at wall nodes spurious."""
    w = aniso(nx, ny, N, seed=seed, precision=precision, ckpt_every=ckpt_every)
    w.adv, w.a_row = "none", None
    solid = disc_mask(nx, ny, seed, rmin, rmax)
    cy0 = max(1, ny // 2 - win // 2)
    window = (1, cy0, min(win, nx - 2), min(win, ny - 2))
    x0, y0, cnx, cny = window
    cmask = (1 - solid[y0:y0 + cny, x0:x0 + cnx]).astype(np.uint8)
    return replace(w, name="geom", solid=solid, window=window, cmask=cmask)


def batch_workloads(n_problems=256, N=1000, seed=3, sizes=(64, 128, 256, 512), ckpt_every=100, precision=32):
    """Independent problems for the batched launch."""
    out = []
    for i in range(n_problems):
        rng = np.random.default_rng(seed + i)
        nx, ny = int(rng.choice(sizes)), int(rng.choice(sizes))
        chi = -float(rng.uniform(0.2, 2.0)) / 20.0
        ratio = float(rng.uniform(1.0, 8.0))
        ang = float(rng.uniform(0, np.pi))
        sig = min(nx, ny) / 16.0
        u0 = bumps(nx, ny, seed + i, sig)
        u_tgt = 1.0 + 0.2 * _periodic_gauss(nx, ny, nx / 2, ny / 2, 2 * sig)
        lam = (0.08, 0.08 / ratio)
        out.append(Workload(name=f"batch{i}", nx=nx, ny=ny, N=N, Q=9, precision=precision, aniso="rotated",
                            lam_u=lam, lam_v=lam, theta=np.full((ny, nx), ang), chi=chi,
                            u0=u0, v0=np.zeros((ny, nx)), u_tgt=u_tgt, alpha=1e-3, ckpt_every=ckpt_every,
                            extra=dict(ratio=ratio, angle=ang)))
    return out


@dataclass
class Workload3:
    """Three-species (attraction-repulsion chemotaxis, logistic source) input
    set: the same tensor/convection vocabulary as ``Workload`` with a third
    species w, the kinetics coefficients and the controlled species."""
    name: str
    nx: int
    ny: int
    N: int
    precision: int = 64
    aniso: str = "rotated"
    D_u_const: tuple = (0.05, 0.0, 0.05)
    D_v_const: tuple = (0.2, 0.0, 0.2)
    D_w_const: tuple = (0.15, 0.0, 0.15)
    lam_u: tuple = (0.08, 0.02)
    lam_v: tuple = (0.2, 0.1)
    lam_w: tuple = (0.15, 0.05)
    theta: np.ndarray | None = None
    D_u_field: np.ndarray | None = None
    D_v_field: np.ndarray | None = None
    D_w_field: np.ndarray | None = None
    d: float = 1.0
    chi1: float = 0.1
    chi2: float = -0.08
    a1: float = 0.0
    a2: float = 0.0
    b1: float = 0.0
    b2: float = 0.0
    b3: float = 0.0
    c1: float = 0.0
    c2: float = 0.0
    ctrl_species: int = 2
    adv: str = "none"
    a_row: np.ndarray | None = None
    a_field: np.ndarray | None = None
    u0: np.ndarray = None
    v0: np.ndarray = None
    w0: np.ndarray = None
    u_tgt: np.ndarray = None
    alpha: float = 1e-3
    s: tuple = (1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0)
    source_order: int = 2
    ckpt_every: int = 0

    @property
    def ctrl_shape(self):
        return (self.N, self.ny, self.nx)

    def D_fields(self):
        """Per-node (Dxx, Dxy, Dyy) of u, v, w, [ny, nx, 3] each."""
        if self.aniso == "field":
            return self.D_u_field, self.D_v_field, self.D_w_field
        if self.aniso == "const":
            return tuple(np.broadcast_to(np.asarray(c, float), (self.ny, self.nx, 3)).copy()
                         for c in (self.D_u_const, self.D_v_const, self.D_w_const))
        return tuple(rotated_tensor(l, self.theta) for l in (self.lam_u, self.lam_v, self.lam_w))

    def a_fields(self):
        if self.adv == "none":
            return None
        if self.adv == "row":
            return np.broadcast_to(self.a_row[:, None, :], (self.ny, self.nx, 2)).copy()
        return self.a_field

    def random_control(self, seed: int, scale: float = 0.01):
        return scale * np.random.default_rng(seed).standard_normal(self.ctrl_shape)


def arc(nx=1024, ny=1024, N=2000, seed=5, precision=32, ckpt_every=100, ctrl_species=2):
    """Attraction-repulsion chemotaxis with a logistic source (D2Q9): rotated
    anisotropic tensors for the three species along one seeded angle field,
    shear convection a = (0.05 sin(2 pi y / L), 0), attraction toward v
    (chi1 = 0.1), repulsion from w (chi2 = -0.08), logistic growth of u,
    nonlinear consumption of v; u0 four seeded bumps on 1, v0 and w0 smooth
    seeded fields, u_target one centred bump.  Rates are per lattice step."""
    rng = np.random.default_rng(seed)
    theta = _angle_field(nx, ny, seed)
    y = np.arange(ny)
    a_row = np.stack([0.05 * np.sin(2 * np.pi * y / ny), np.zeros(ny)], axis=-1)
    sig = nx / 16.0
    u0 = bumps(nx, ny, seed, sig)
    x = np.arange(nx)[None, :]
    yy = np.arange(ny)[:, None]
    p = rng.uniform(0, 2 * np.pi, 3)
    v0 = 0.5 + 0.1 * np.sin(2 * np.pi * (x / nx + yy / ny) + p[0])
    w0 = 0.4 + 0.1 * np.cos(2 * np.pi * 2 * x / nx + p[1]) * np.cos(2 * np.pi * yy / ny + p[2])
    u_tgt = 1.0 + 0.2 * _periodic_gauss(nx, ny, nx / 2, ny / 2, 2 * sig)
    return Workload3(name="arc", nx=nx, ny=ny, N=N, precision=precision, aniso="rotated", theta=theta,
                     lam_u=(0.08, 0.02), lam_v=(0.2, 0.1), lam_w=(0.15, 0.05), chi1=0.1, chi2=-0.08,
                     a1=1e-3, a2=5e-4, b1=1e-3, b2=2e-3, b3=5e-4, c1=1e-3, c2=3e-3, ctrl_species=ctrl_species,
                     adv="row", a_row=a_row, u0=u0, v0=v0, w0=np.broadcast_to(w0, (ny, nx)).copy(), u_tgt=u_tgt,
                     alpha=1e-3, ckpt_every=ckpt_every)


def rotated_tensor3(lam, ax, ay):
    """(Dxx, Dxy, Dxz, Dyy, Dyz, Dzz) of R diag(lam) R^T, R a rotation by ay
    about y after ax about x (constant angles)."""
    cx, sx, cy, sy = np.cos(ax), np.sin(ax), np.cos(ay), np.sin(ay)
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    R = Ry @ Rx
    D = R @ np.diag(np.asarray(lam, float)) @ R.T
    return (D[0, 0], D[0, 1], D[0, 2], D[1, 1], D[1, 2], D[2, 2])


@dataclass
class Workload3D:
    """Two-species problem on a periodic nx x ny x nz D3Q19 lattice: constant
    ("const") or per-node ("field") tensors as (Dxx, Dxy, Dxz, Dyy, Dyz, Dzz),
    convection none / "row" (a function of y, [ny][3]) / "field"
    ([nz][ny][nx][3]); node fields [nz][ny][nx]; control [N][nz][ny][nx]."""
    name: str
    nx: int
    ny: int
    nz: int
    N: int
    precision: int = 64
    aniso: str = "const"
    D_u_const: tuple = (0.05, 0.0, 0.0, 0.05, 0.0, 0.05)
    D_v_const: tuple = (0.2, 0.0, 0.0, 0.2, 0.0, 0.2)
    D_u_field: np.ndarray | None = None
    D_v_field: np.ndarray | None = None
    d_u: float = 1.0
    d_v: float = 1.0
    chi: float = -0.1
    r_vu: float = 0.5
    r_vv: float = -0.1
    adv: str = "none"
    a_row: np.ndarray | None = None
    a_field: np.ndarray | None = None
    u0: np.ndarray = None
    v0: np.ndarray = None
    u_tgt: np.ndarray = None
    alpha: float = 1e-3
    s: tuple = (1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0)
    source_order: int = 2
    ckpt_every: int = 0

    @property
    def ctrl_shape(self):
        return (self.N, self.nz, self.ny, self.nx)

    def D_fields(self):
        """Per-node tensors of u and v, [nz, ny, nx, 6] each."""
        if self.aniso == "field":
            return self.D_u_field, self.D_v_field
        shape = (self.nz, self.ny, self.nx, 6)
        return (np.broadcast_to(np.asarray(self.D_u_const, float), shape).copy(),
                np.broadcast_to(np.asarray(self.D_v_const, float), shape).copy())

    def a_fields(self):
        if self.adv == "none":
            return None
        if self.adv == "row":
            return np.broadcast_to(self.a_row[None, :, None, :], (self.nz, self.ny, self.nx, 3)).copy()
        return self.a_field

    def random_control(self, seed: int, scale: float = 0.01):
        return scale * np.random.default_rng(seed).standard_normal(self.ctrl_shape)


def aniso3d(n=128, N=500, seed=6, precision=32, ckpt_every=50, nx=None, ny=None, nz=None):
    """Anisotropic three-dimensional problem (D3Q19): constant rotated tensors
    D_u = R diag(0.08, 0.04, 0.02) R^T, D_v = R' diag(0.12, 0.08, 0.04) R'^T
    (seeded angles), shear convection a = (0.05 sin(2 pi y / L), 0, 0),
    chi = -0.1, Phi_v = 0.5 u - 0.1 v + g; u0 = 1 + 0.2 * four seeded
    periodic Gaussian bumps (sigma L/16), v0 = 0, target one centred bump
    (sigma L/8)."""
    nx, ny, nz = nx or n, ny or n, nz or n
    rng = np.random.default_rng(seed)
    angs = rng.uniform(0, np.pi, 4)
    y = np.arange(ny)
    a_row = np.stack([0.05 * np.sin(2 * np.pi * y / ny), np.zeros(ny), np.zeros(ny)], axis=-1)
    sig = nx / 16.0

    def g3(c, s):
        X = np.arange(nx)[None, None, :]
        Y = np.arange(ny)[None, :, None]
        Z = np.arange(nz)[:, None, None]
        d = [np.minimum(np.abs(q - cq), L - np.abs(q - cq)) for q, cq, L in ((X, c[0], nx), (Y, c[1], ny), (Z, c[2], nz))]
        return np.exp(-(d[0] ** 2 + d[1] ** 2 + d[2] ** 2) / (2 * s * s))

    u0 = np.ones((nz, ny, nx))
    for c in rng.uniform(0, 1, size=(4, 3)):
        u0 = u0 + 0.2 * g3((c[0] * nx, c[1] * ny, c[2] * nz), sig)
    u_tgt = 1.0 + 0.2 * g3((nx / 2, ny / 2, nz / 2), 2 * sig)
    return Workload3D(name="aniso3d", nx=nx, ny=ny, nz=nz, N=N, precision=precision, aniso="const",
                      D_u_const=rotated_tensor3((0.08, 0.04, 0.02), angs[0], angs[1]),
                      D_v_const=rotated_tensor3((0.12, 0.08, 0.04), angs[2], angs[3]),
                      chi=-0.1, r_vu=0.5, r_vv=-0.1, adv="row", a_row=a_row, u0=u0, v0=np.zeros((nz, ny, nx)),
                      u_tgt=u_tgt, alpha=1e-3, ckpt_every=ckpt_every)
