"""FP64 CPU oracle for the MRT/AMRT chemotaxis optimal-control path.

TEST INFRASTRUCTURE.  This package is the plain, slow, obviously-correct
reference the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; the product path never does.  It shares no code with the CUDA library.

The arithmetic lives in ``mrt_oracle.c`` (plain C, FP64, one node at a time);
this module only builds it with gcc and marshals arrays through ctypes.  The
Armijo gradient-descent iteration below follows the paper's discrete-adjoint
algorithm (Sec. 3.2.1, the optimisation process after eq. JD-H-B) with the
heuristic first step min(1, 1/||E||_inf) (remark after the continuous gradient
algorithm, Sec. 2.3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "mrt_oracle.c")
_SRC3D = os.path.join(_HERE, "d3q19_oracle.c")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: x86_64 and aarch64; the
    per-node loops run on OpenMP threads, bitwise independent of their count)."""
    os.makedirs(_BUILD, exist_ok=True)
    deps = [_SRC, _SRC3D, os.path.join(_HERE, "mrt_oracle.h"), os.path.join(_HERE, "d3q19_oracle.h")]
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(os.path.getmtime(f) for f in deps):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fopenmp", "-o", tmp, _SRC, _SRC3D,
             "-lm"]
        )
        os.replace(tmp, _SO)
    return _SO


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("N", ctypes.c_int), ("Q", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("Du", ctypes.c_void_p), ("Dv", ctypes.c_void_p),
        ("d_u", ctypes.c_double), ("d_v", ctypes.c_double),
        ("chi", ctypes.c_double), ("r_vu", ctypes.c_double), ("r_vv", ctypes.c_double),
        ("a", ctypes.c_void_p), ("solid", ctypes.c_void_p),
        ("cx0", ctypes.c_int), ("cy0", ctypes.c_int), ("cnx", ctypes.c_int), ("cny", ctypes.c_int),
        ("cmask", ctypes.c_void_p),
        ("u_tgt", ctypes.c_void_p), ("alpha", ctypes.c_double),
        ("s", ctypes.c_double * 7),
        ("source_order", ctypes.c_int),
        ("u0", ctypes.c_void_p), ("v0", ctypes.c_void_p),
    ]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_Problem)
        vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
        lib.or_forward.argtypes = [P, vp, dp, vp, vp]
        lib.or_forward_trace.argtypes = [P, vp, vp, vp, vp]
        lib.or_tlm.argtypes = [P, vp, vp, vp, vp, vp, dp]
        lib.or_adjoint.argtypes = [P, vp, vp, vp, vp, vp, dp]
        lib.or_cadjoint.argtypes = [P, vp, vp, dp]
        lib.or_set_threads.argtypes = [ctypes.c_int]
        lib.or_set_threads.restype = ctypes.c_int
        lib.or_lattice.argtypes = [ctypes.c_int, vp, vp, vp, vp]
        lib.or_feq.argtypes = [ctypes.c_int, ctypes.c_double, vp, ctypes.c_double, vp]
        lib.or_collide_node.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp,
                                        ctypes.c_double, ctypes.c_double, vp, vp, dp]
        lib.or_adjoint_node.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_double,
                                        vp, vp, ctypes.c_int, ctypes.c_double, vp, vp, dp, dp]
        _lib = lib
    return _lib


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's per-node loops (n <= 0: leave as is); returns
    the count in use.  Results are bitwise the same for every count."""
    return int(_load().or_set_threads(int(n)))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _u8(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.uint8)


@dataclass
class Problem:
    """Problem data in the oracle's layout (see mrt_oracle.h).

    Du, Dv: [ny, nx, 3] (Dxx, Dxy, Dyy); a: [ny, nx, 2] or None; solid: [ny, nx]
    bool or None; window (cx0, cy0, cnx, cny) with optional cmask [cny, cnx].
    """

    nx: int
    ny: int
    N: int
    Q: int
    Du: np.ndarray
    Dv: np.ndarray
    u0: np.ndarray
    v0: np.ndarray
    u_tgt: np.ndarray
    d_u: float = 1.0
    d_v: float = 1.0
    chi: float = 0.0
    r_vu: float = 0.0
    r_vv: float = 0.0
    a: np.ndarray | None = None
    solid: np.ndarray | None = None
    window: tuple = None
    cmask: np.ndarray | None = None
    alpha: float = 0.0
    s: tuple = (1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0)
    source_order: int = 2
    tau: float = 1.0
    windows: int = 0
    _keep: list = field(default_factory=list, repr=False)

    @property
    def ctrl_shape(self):
        w = self.window or (0, 0, self.nx, self.ny)
        return (self.windows or self.N, w[3], w[2])

    # Time-windowed controls (windows = W > 0): the control is restricted to
    # the subspace g^n = G_{n // (N/W)} of the paper's space-time controls.
    # Every solve runs on the expanded per-step control P G; the gradient on
    # the subspace is the adjoint of P applied to the per-step gradient, i.e.
    # the sum of dJ/dg^n over the steps of each window.
    def expand(self, g):
        if g is None or not self.windows:
            return g
        g = np.asarray(g, dtype=np.float64)
        return np.repeat(g, self.N // self.windows, axis=0)

    def restrict_gradient(self, dJdg_steps):
        if not self.windows:
            return dJdg_steps
        L = self.N // self.windows
        return dJdg_steps.reshape((self.windows, L) + dJdg_steps.shape[1:]).sum(axis=1)

    def _struct(self):
        arrs = dict(
            Du=_f64(self.Du), Dv=_f64(self.Dv), a=_f64(self.a), solid=_u8(self.solid),
            cmask=_u8(self.cmask), u_tgt=_f64(self.u_tgt), u0=_f64(self.u0), v0=_f64(self.v0),
        )
        self._keep = list(arrs.values())
        w = self.window or (0, 0, self.nx, self.ny)
        st = _Problem()
        st.nx, st.ny, st.N, st.Q = self.nx, self.ny, self.N, self.Q
        st.tau = self.tau
        st.Du, st.Dv = _ptr(arrs["Du"]), _ptr(arrs["Dv"])
        st.d_u, st.d_v = self.d_u, self.d_v
        st.chi, st.r_vu, st.r_vv = self.chi, self.r_vu, self.r_vv
        st.a, st.solid = _ptr(arrs["a"]), _ptr(arrs["solid"])
        st.cx0, st.cy0, st.cnx, st.cny = w
        st.cmask = _ptr(arrs["cmask"])
        st.u_tgt = _ptr(arrs["u_tgt"])
        st.alpha = self.alpha
        st.s = (ctypes.c_double * 7)(*self.s)
        st.source_order = self.source_order
        st.u0, st.v0 = _ptr(arrs["u0"]), _ptr(arrs["v0"])
        return st


def _check(rc, name):
    if rc != 0:
        raise RuntimeError(f"oracle {name} failed with code {rc}")


def forward(p: Problem, g=None):
    """Forward MRT solve.  Returns (J, u^N, v^N)."""
    lib = _load()
    st = p._struct()
    g = _f64(p.expand(g))
    J = ctypes.c_double(0.0)
    uN = np.zeros((p.ny, p.nx))
    vN = np.zeros((p.ny, p.nx))
    _check(lib.or_forward(ctypes.byref(st), _ptr(g), ctypes.byref(J), _ptr(uN), _ptr(vN)), "forward")
    return J.value, uN, vN


def forward_trace(p: Problem, g=None):
    """Per-step sums over fluid nodes: (sum u^n, sum v^n, sum Phi^n), each [N]."""
    lib = _load()
    st = p._struct()
    mu, mv, sp = np.zeros(p.N), np.zeros(p.N), np.zeros(p.N)
    _check(lib.or_forward_trace(ctypes.byref(st), _ptr(_f64(p.expand(g))), _ptr(mu), _ptr(mv), _ptr(sp)), "trace")
    return mu, mv, sp


def tlm(p: Problem, g, dg, df0=None):
    """Tangent-linear model.  Returns (dJ, du^N, dv^N)."""
    lib = _load()
    st = p._struct()
    g, dg, df0 = _f64(p.expand(g)), _f64(p.expand(dg)), _f64(df0)
    dJ = ctypes.c_double(0.0)
    du = np.zeros((p.ny, p.nx))
    dv = np.zeros((p.ny, p.nx))
    _check(lib.or_tlm(ctypes.byref(st), _ptr(g), _ptr(dg), _ptr(df0), _ptr(du), _ptr(dv), ctypes.byref(dJ)), "tlm")
    return dJ.value, du, dv


def adjoint(p: Problem, g=None, seed_u=None, seed_v=None, want_psi0=False):
    """AMRT adjoint sweep.  Returns (J, dJ/dg [W or N, cny, cnx], psi0 [ny, nx, 2, Q] or None)."""
    lib = _load()
    st = p._struct()
    g, su, sv = _f64(p.expand(g)), _f64(seed_u), _f64(seed_v)
    w = p.window or (0, 0, p.nx, p.ny)
    dJdg = np.zeros((p.N, w[3], w[2]))
    psi0 = np.zeros((p.ny, p.nx, 2, p.Q)) if want_psi0 else None
    J = ctypes.c_double(0.0)
    _check(lib.or_adjoint(ctypes.byref(st), _ptr(g), _ptr(su), _ptr(sv), _ptr(dJdg), _ptr(psi0),
                          ctypes.byref(J)), "adjoint")
    return J.value, p.restrict_gradient(dJdg), psi0


def cadjoint(p: Problem, g=None):
    """Continuous-adjoint gradient (adjoint PDE solved by the MRT scheme with
    time reversed, see mrt_oracle.h).  Returns (J, dJ/dg [W or N, cny, cnx])."""
    lib = _load()
    st = p._struct()
    g = _f64(p.expand(g))
    w = p.window or (0, 0, p.nx, p.ny)
    dJdg = np.zeros((p.N, w[3], w[2]))
    J = ctypes.c_double(0.0)
    _check(lib.or_cadjoint(ctypes.byref(st), _ptr(g), _ptr(dJdg), ctypes.byref(J)), "cadjoint")
    return J.value, p.restrict_gradient(dJdg)


def lattice(Q: int):
    """(e [Q,2] int, w [Q], M [Q,Q], Minv [Q,Q]) as the oracle holds them."""
    lib = _load()
    e = np.zeros((Q, 2), dtype=np.int32)
    w, M, Mi = np.zeros(Q), np.zeros((Q, Q)), np.zeros((Q, Q))
    _check(lib.or_lattice(Q, _ptr(e), _ptr(w), _ptr(M), _ptr(Mi)), "lattice")
    return e, w, M, Mi


def feq(Q: int, Theta: float, a=(0.0, 0.0), d: float = 1.0):
    lib = _load()
    out = np.zeros(Q)
    av = np.asarray(a, dtype=np.float64)
    _check(lib.or_feq(Q, float(Theta), _ptr(av), float(d), _ptr(out)), "feq")
    return out


def collide_node(p: Problem, x, y, n, f_u, f_v, g=0.0, phi_prev=0.0):
    """Local forward collision at node (x, y), step n.  Returns (P_u, P_v, Phi)."""
    lib = _load()
    st = p._struct()
    fu, fv = _f64(f_u), _f64(f_v)
    Pu, Pv = np.zeros(p.Q), np.zeros(p.Q)
    phi = ctypes.c_double(0.0)
    _check(lib.or_collide_node(ctypes.byref(st), x, y, n, _ptr(fu), _ptr(fv), float(g), float(phi_prev),
                               _ptr(Pu), _ptr(Pv), ctypes.byref(phi)), "collide_node")
    return Pu, Pv, phi.value


def adjoint_node(p: Problem, x, y, n, f_u, f_v, rho_u, rho_v, g=0.0, sigma_next=None):
    """Local AMRT adjoint step at node (x, y), step n: the transpose of
    collide_node applied to the pulled adjoint populations (rho_u, rho_v) and,
    when sigma_next is given, to the adjoint c'_{n+1} sigma^{n+1} of Phi^n's
    use at step n + 1.  Returns (psi_u, psi_v, sigma^n, lambda_Phi)."""
    lib = _load()
    st = p._struct()
    fu, fv, ru, rv = _f64(f_u), _f64(f_v), _f64(rho_u), _f64(rho_v)
    psu, psv = np.zeros(p.Q), np.zeros(p.Q)
    sig, lam = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib.or_adjoint_node(ctypes.byref(st), x, y, n, _ptr(fu), _ptr(fv), float(g), _ptr(ru), _ptr(rv),
                               0 if sigma_next is None else 1, 0.0 if sigma_next is None else float(sigma_next),
                               _ptr(psu), _ptr(psv), ctypes.byref(sig), ctypes.byref(lam)), "adjoint_node")
    return psu, psv, sig.value, lam.value


def gd_step(p: Problem, g, lam_prev=None, c1=1e-4, max_trials=30):
    """One gradient-descent iteration with Armijo backtracking (FP64).

    Steps (discrete-adjoint algorithm, Sec. 3.2.1): forward -> adjoint ->
    gradient E -> trial g - lam E, halving lam until
    J(g - lam E) <= J(g) - c1 lam ||E||^2.  First trial: min(1, 1/||E||_inf)
    on the first iteration, 2 lam_prev afterwards.
    Returns (g_new, info dict).
    """
    J0, E, _ = adjoint(p, g)
    E2 = float(np.sum(E * E))
    Einf = float(np.max(np.abs(E))) if E.size else 0.0
    lam = min(1.0, 1.0 / Einf) if lam_prev is None else 2.0 * lam_prev
    for t in range(max_trials):
        gt = g - lam * E
        Jt, _, _ = forward(p, gt)
        if Jt <= J0 - c1 * lam * E2:
            return gt, dict(J0=J0, J=Jt, lam=lam, trials=t + 1, E2=E2, Einf=Einf)
        lam *= 0.5
    raise RuntimeError("Armijo line search failed")


def from_workload(w, N=None) -> Problem:
    """Oracle problem from a seeded workload (per-node tensor and velocity fields)."""
    Du, Dv = w.D_fields()
    return Problem(nx=w.nx, ny=w.ny, N=w.N if N is None else N, Q=w.Q, Du=Du, Dv=Dv, u0=w.u0, v0=w.v0,
                   u_tgt=w.u_tgt, d_u=w.d_u, d_v=w.d_v, chi=w.chi, r_vu=w.r_vu, r_vv=w.r_vv,
                   a=w.a_fields(), solid=w.solid, window=w.window, cmask=w.cmask, alpha=w.alpha,
                   s=tuple(w.s), source_order=w.source_order, windows=w.windows)


CG_VARIANTS = ("FR", "PR", "HS", "DY")


def cg_iteration(p: Problem, g, state=None, variant="PR", c1=1e-4, c2=0.1, max_trials=30):
    """One nonlinear conjugate-gradient iteration with a weak Wolfe-Powell
    line search (remark 2 after the gradient algorithm of Sec. 2.3).

    Direction D_k = -G_k at k = 0, else -G_k + r_{k-1} D_{k-1} with r from
    Fletcher-Reeves, Polak-Ribiere, Hestenes-Stiefel or Dai-Yuan; the update
    is z_{k+1} = z_k + zeta_k D_k (the printed "- zeta_k D_k" with D_0 = -G_0
    would ascend: read as the descent step).  Soft reset D = -G whenever the
    new direction is not a descent direction or successive gradients are far
    from orthogonal, |<G_{k+1}, G_k>| >= 0.2 ||G_{k+1}||^2 (Powell's restart
    test: the CG recurrence has stopped making progress).  Line search on
    phi(l) = J(g + l D): accept when phi(l) <= phi(0) + c1 l phi'(0) and
    phi'(l) >= c2 phi'(0); else bisect the bracket (doubling while it is
    open).  First trial min(1, 1/||G||_inf) at k = 0, else
    l_{k-1} phi'_{k-1}(0) / phi'_k(0).  If no trial meets both conditions
    (the CG direction makes no progress, e.g. at the rounding floor of an FP32
    lattice), the iteration falls back to a steepest-descent step with Armijo
    backtracking from min(1, 1/||G||_inf) (soft reset).

    state: None (k = 0) or the dict returned by the previous call.
    Returns (g_new, state, info)."""
    if state is None:
        J0, G, _ = adjoint(p, g)
        D = -G
        gd = float(np.sum(G * D))
        lam = min(1.0, 1.0 / float(np.max(np.abs(G)))) if G.size and np.max(np.abs(G)) > 0 else 1.0
        k = 0
    else:
        J0, G, D, gd = state["J"], state["G"], state["D"], state["gd"]
        lam = state["lam"] * state["gd_prev"] / gd
        k = state["k"]
    lo, hi = 0.0, np.inf
    for t in range(max_trials):
        gt = g + lam * D
        Jt, Gt, _ = adjoint(p, gt)
        if not np.isfinite(Jt) or Jt > J0 + c1 * lam * gd:
            hi = lam
        elif float(np.sum(Gt * D)) < c2 * gd:
            lo = lam
        else:
            break
        lam = 0.5 * (lo + hi) if np.isfinite(hi) else 2.0 * lam
    else:
        # soft reset: steepest descent with Armijo backtracking
        gg = float(np.sum(G * G))
        lam = min(1.0, 1.0 / float(np.max(np.abs(G)))) if np.max(np.abs(G)) > 0 else 1.0
        for t2 in range(max_trials):
            gt = g - lam * G
            Jt, Gt, _ = adjoint(p, gt)
            if np.isfinite(Jt) and Jt <= J0 - c1 * lam * gg:
                break
            lam *= 0.5
        else:
            raise RuntimeError("line search failed")
        gtgt = float(np.sum(Gt * Gt))
        info = dict(J0=J0, J=Jt, lam=lam, trials=max_trials + t2 + 1, r=0.0, restarted=True, grad_sq=gtgt)
        return gt, dict(J=Jt, G=Gt, D=-Gt, gd=-gtgt, gd_prev=-gg, lam=lam, k=k + 1), info
    gg = float(np.sum(G * G))
    y = Gt - G
    dy = float(np.sum(D * y))
    if variant == "FR":
        r = float(np.sum(Gt * Gt)) / gg
    elif variant == "PR":
        r = float(np.sum(Gt * y)) / gg
    elif variant == "HS":
        r = float(np.sum(Gt * y)) / dy
    elif variant == "DY":
        r = float(np.sum(Gt * Gt)) / dy
    else:
        raise ValueError(variant)
    Dn = -Gt + r * D
    gdn = float(np.sum(Gt * Dn))
    gtgt = float(np.sum(Gt * Gt))
    restarted = gdn >= 0.0 or abs(float(np.sum(Gt * G))) >= 0.2 * gtgt
    if restarted:
        Dn = -Gt
        gdn = float(np.sum(Gt * Gt)) * -1.0
    info = dict(J0=J0, J=Jt, lam=lam, trials=t + 1, r=r, restarted=restarted, grad_sq=float(np.sum(Gt * Gt)))
    return gt, dict(J=Jt, G=Gt, D=Dn, gd=gdn, gd_prev=gd, lam=lam, k=k + 1), info


def lma_step(p: Problem, g, c1=1e-4, max_trials=30):
    """One steepest-descent iteration with the step length of the quadratic
    model built from the sensitivity problem (eqs. LM / LMA, Sec. 2.3):
    u^N(g - lam E) ~ u^N(g) - lam du^N with du^N the tangent-linear response to
    E, so J(g - lam E) ~ J - lam ||E||^2 + lam^2 (||du^N||^2 + 2 alpha L ||E||^2)/2
    (L steps per control window), minimised by
    lam* = ||E||^2 / (||du^N||^2 + 2 alpha L ||E||^2).  Accepted under the
    Armijo test J(g - lam E) <= J - c1 lam ||E||^2, halving lam otherwise.
    Returns (g_new, info)."""
    J0, E, _ = adjoint(p, g)
    _, du, _ = tlm(p, g, E)
    e2 = float(np.sum(E * E))
    L = p.N // p.windows if p.windows else 1
    lam = e2 / (float(np.sum(du * du)) + 2.0 * p.alpha * L * e2)
    for t in range(max_trials):
        gt = g - lam * E
        Jt, _, _ = forward(p, gt)
        if Jt <= J0 - c1 * lam * e2:
            return gt, dict(J0=J0, J=Jt, lam=lam, trials=t + 1, E2=e2)
        lam *= 0.5
    raise RuntimeError("line search failed")


# ---------------------------------------------------------------- three species

class _Problem3(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("N", ctypes.c_int), ("tau", ctypes.c_double),
        ("Du", ctypes.c_void_p), ("Dv", ctypes.c_void_p), ("Dw", ctypes.c_void_p), ("d", ctypes.c_double),
        ("a", ctypes.c_void_p), ("chi1", ctypes.c_double), ("chi2", ctypes.c_double),
        ("a1", ctypes.c_double), ("a2", ctypes.c_double),
        ("b1", ctypes.c_double), ("b2", ctypes.c_double), ("b3", ctypes.c_double),
        ("c1", ctypes.c_double), ("c2", ctypes.c_double), ("ctrl_species", ctypes.c_int),
        ("u_tgt", ctypes.c_void_p), ("alpha", ctypes.c_double), ("s", ctypes.c_double * 7),
        ("source_order", ctypes.c_int), ("u0", ctypes.c_void_p), ("v0", ctypes.c_void_p), ("w0", ctypes.c_void_p),
    ]


@dataclass
class Problem3:
    """Three-species (attraction-repulsion chemotaxis, logistic source) problem
    in the oracle's layout (see mrt_oracle.h, or3_problem)."""

    nx: int
    ny: int
    N: int
    Du: np.ndarray
    Dv: np.ndarray
    Dw: np.ndarray
    u0: np.ndarray
    v0: np.ndarray
    w0: np.ndarray
    u_tgt: np.ndarray
    d: float = 1.0
    a: np.ndarray | None = None
    chi1: float = 0.0
    chi2: float = 0.0
    a1: float = 0.0
    a2: float = 0.0
    b1: float = 0.0
    b2: float = 0.0
    b3: float = 0.0
    c1: float = 0.0
    c2: float = 0.0
    ctrl_species: int = 2
    alpha: float = 0.0
    s: tuple = (1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0)
    source_order: int = 2
    tau: float = 1.0
    _keep: list = field(default_factory=list, repr=False)

    def _struct(self):
        arrs = dict(Du=_f64(self.Du), Dv=_f64(self.Dv), Dw=_f64(self.Dw), a=_f64(self.a), u_tgt=_f64(self.u_tgt),
                    u0=_f64(self.u0), v0=_f64(self.v0), w0=_f64(self.w0))
        self._keep = list(arrs.values())
        st = _Problem3()
        st.nx, st.ny, st.N, st.tau = self.nx, self.ny, self.N, self.tau
        for k in ("Du", "Dv", "Dw", "a", "u_tgt", "u0", "v0", "w0"):
            setattr(st, k, _ptr(arrs[k]))
        for k in ("d", "chi1", "chi2", "a1", "a2", "b1", "b2", "b3", "c1", "c2", "alpha"):
            setattr(st, k, float(getattr(self, k)))
        st.ctrl_species = self.ctrl_species
        st.s = (ctypes.c_double * 7)(*self.s)
        st.source_order = self.source_order
        return st


def _load3():
    lib = _load()
    if not hasattr(lib, "_or3_ready"):
        P = ctypes.POINTER(_Problem3)
        vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
        lib.or3_forward.argtypes = [P, vp, dp, vp]
        lib.or3_forward_trace.argtypes = [P, vp, vp]
        lib.or3_tlm.argtypes = [P, vp, vp, vp, vp, dp]
        lib.or3_adjoint.argtypes = [P, vp, vp, vp, vp, dp]
        lib.or3_collide_node.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_double, vp, vp,
                                         vp]
        lib.or3_adjoint_node.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_double, vp,
                                         ctypes.c_int, vp, vp, vp, vp]
        lib._or3_ready = True
    return lib


def forward3(p: Problem3, g=None):
    """Three-species forward solve.  Returns (J, uvw^N [3][ny][nx])."""
    lib = _load3()
    st = p._struct()
    J = ctypes.c_double(0.0)
    uvw = np.zeros((3, p.ny, p.nx))
    _check(lib.or3_forward(ctypes.byref(st), _ptr(_f64(g)), ctypes.byref(J), _ptr(uvw)), "forward3")
    return J.value, uvw


def forward3_trace(p: Problem3, g=None):
    """Per step: (masses of u, v, w before collision [N][3], sums of Phi_u, Phi_v, Phi_w [N][3])."""
    lib = _load3()
    st = p._struct()
    tr = np.zeros((p.N, 6))
    _check(lib.or3_forward_trace(ctypes.byref(st), _ptr(_f64(g)), _ptr(tr)), "forward3_trace")
    return tr[:, :3], tr[:, 3:]


def tlm3(p: Problem3, g, dg, df0=None):
    """Tangent-linear model.  Returns (dJ, duvw^N [3][ny][nx])."""
    lib = _load3()
    st = p._struct()
    dJ = ctypes.c_double(0.0)
    d = np.zeros((3, p.ny, p.nx))
    _check(lib.or3_tlm(ctypes.byref(st), _ptr(_f64(g)), _ptr(_f64(dg)), _ptr(_f64(df0)), _ptr(d), ctypes.byref(dJ)),
           "tlm3")
    return dJ.value, d


def adjoint3(p: Problem3, g=None, seeds=None, want_psi0=False):
    """Exact discrete adjoint.  Returns (J, dJ/dg [N][ny][nx], psi0 [ny][nx][3][9] or None)."""
    lib = _load3()
    st = p._struct()
    J = ctypes.c_double(0.0)
    E = np.zeros((p.N, p.ny, p.nx))
    psi0 = np.zeros((p.ny, p.nx, 3, 9)) if want_psi0 else None
    _check(lib.or3_adjoint(ctypes.byref(st), _ptr(_f64(g)), _ptr(_f64(seeds)), _ptr(E), _ptr(psi0),
                           ctypes.byref(J)), "adjoint3")
    return J.value, E, psi0


def collide3_node(p: Problem3, x, y, n, f, g=0.0, phi_prev=(0.0, 0.0, 0.0)):
    """One three-species collision at node (x, y), step n: f [3][9] ->
    (P [3][9], Phi^n [3])."""
    lib = _load3()
    st = p._struct()
    P, phi = np.zeros((3, 9)), np.zeros(3)
    _check(lib.or3_collide_node(ctypes.byref(st), x, y, n, _ptr(_f64(f)), float(g), _ptr(_f64(phi_prev)), _ptr(P),
                                _ptr(phi)), "collide3_node")
    return P, phi


def adjoint3_node(p: Problem3, x, y, n, f, rho, g=0.0, sigma_next=None):
    """Local three-species AMRT step at node (x, y), step n, the transpose of
    collide3_node applied to rho [3][9] and, when sigma_next [3] is given, to
    the adjoint c'_{n+1} sigma^{n+1} of each Phi^n's use at step n + 1.
    Returns (psi [3][9], sigma^n [3], lambda_Phi [3])."""
    lib = _load3()
    st = p._struct()
    psi, sig, lam = np.zeros((3, 9)), np.zeros(3), np.zeros(3)
    _check(lib.or3_adjoint_node(ctypes.byref(st), x, y, n, _ptr(_f64(f)), float(g), _ptr(_f64(rho)),
                                0 if sigma_next is None else 1, _ptr(_f64(sigma_next)), _ptr(psi), _ptr(sig),
                                _ptr(lam)), "adjoint3_node")
    return psi, sig, lam


def from_workload3(w, N=None) -> Problem3:
    """Three-species oracle problem from a seeded workload (per-node fields)."""
    Du, Dv, Dw = w.D_fields()
    return Problem3(nx=w.nx, ny=w.ny, N=w.N if N is None else N, Du=Du, Dv=Dv, Dw=Dw, u0=w.u0, v0=w.v0, w0=w.w0,
                    u_tgt=w.u_tgt, d=w.d, a=w.a_fields(), chi1=w.chi1, chi2=w.chi2, a1=w.a1, a2=w.a2, b1=w.b1,
                    b2=w.b2, b3=w.b3, c1=w.c1, c2=w.c2, ctrl_species=w.ctrl_species, alpha=w.alpha,
                    s=tuple(w.s), source_order=w.source_order)


# ------------------------------------------------------------------ D3Q19
class _Problem3D(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("N", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("Du", ctypes.c_void_p), ("Dv", ctypes.c_void_p), ("a", ctypes.c_void_p),
        ("u0", ctypes.c_void_p), ("v0", ctypes.c_void_p), ("u_tgt", ctypes.c_void_p),
        ("d_u", ctypes.c_double), ("d_v", ctypes.c_double), ("chi", ctypes.c_double),
        ("r_vu", ctypes.c_double), ("r_vv", ctypes.c_double), ("alpha", ctypes.c_double),
        ("s", ctypes.c_double * 7), ("source_order", ctypes.c_int),
    ]


@dataclass
class Problem3D:
    """Two-species problem on the D3Q19 lattice in the oracle's layout (see
    d3q19_oracle.h): node fields [nz][ny][nx], tensors [nz][ny][nx][6]
    (Dxx, Dxy, Dxz, Dyy, Dyz, Dzz), velocity [nz][ny][nx][3] or None."""

    nx: int
    ny: int
    nz: int
    N: int
    Du: np.ndarray
    Dv: np.ndarray
    u0: np.ndarray
    v0: np.ndarray
    u_tgt: np.ndarray
    a: np.ndarray | None = None
    d_u: float = 1.0
    d_v: float = 1.0
    chi: float = 0.0
    r_vu: float = 0.0
    r_vv: float = 0.0
    alpha: float = 0.0
    s: tuple = (1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0)
    source_order: int = 2
    tau: float = 1.0
    _keep: list = field(default_factory=list, repr=False)

    def _struct(self):
        arrs = dict(Du=_f64(self.Du), Dv=_f64(self.Dv), a=_f64(self.a), u0=_f64(self.u0), v0=_f64(self.v0),
                    u_tgt=_f64(self.u_tgt))
        self._keep = list(arrs.values())
        st = _Problem3D()
        st.nx, st.ny, st.nz, st.N, st.tau = self.nx, self.ny, self.nz, self.N, self.tau
        for k, v in arrs.items():
            setattr(st, k, _ptr(v))
        for k in ("d_u", "d_v", "chi", "r_vu", "r_vv", "alpha"):
            setattr(st, k, float(getattr(self, k)))
        st.s = (ctypes.c_double * 7)(*self.s)
        st.source_order = self.source_order
        return st


def _load3d():
    lib = _load()
    if not hasattr(lib, "_od3_ready"):
        P = ctypes.POINTER(_Problem3D)
        vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
        lib.od3_lattice.argtypes = [vp, vp, vp]
        lib.od3_forward.argtypes = [P, vp, dp, vp, vp]
        lib.od3_forward_trace.argtypes = [P, vp, vp, vp, vp]
        lib.od3_tlm.argtypes = [P, vp, vp, vp, vp, vp]
        lib.od3_adjoint.argtypes = [P, vp, vp, vp, vp, vp, dp]
        ci = ctypes.c_int
        lib.od3_collide_node.argtypes = [P, ci, ci, ci, ci, vp, ctypes.c_double, ctypes.c_double, vp, dp]
        lib.od3_adjoint_node.argtypes = [P, ci, ci, ci, ci, vp, ctypes.c_double, vp, ci, ctypes.c_double, vp, dp,
                                         dp]
        lib.od3_set_threads.argtypes = [ctypes.c_int]
        lib._od3_ready = True
    return lib


def lattice3d():
    """D3Q19 tables of the oracle: e [19][3], w [19], M [19][19]."""
    lib = _load3d()
    e = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19)
    M = np.zeros((19, 19))
    _check(lib.od3_lattice(_ptr(e), _ptr(w), _ptr(M)), "lattice3d")
    return e, w, M


def forward3d(p: Problem3D, g=None):
    """D3Q19 forward solve.  Returns (J, u^N, v^N), fields [nz][ny][nx]."""
    lib = _load3d()
    st = p._struct()
    J = ctypes.c_double(0.0)
    u = np.zeros((p.nz, p.ny, p.nx))
    v = np.zeros_like(u)
    _check(lib.od3_forward(ctypes.byref(st), _ptr(_f64(g)), ctypes.byref(J), _ptr(u), _ptr(v)), "forward3d")
    return J.value, u, v


def forward3d_trace(p: Problem3D, g=None):
    """Per step: mass of u, mass of v (before collision), sum of Phi_v."""
    lib = _load3d()
    st = p._struct()
    mu, mv, sp = np.zeros(p.N), np.zeros(p.N), np.zeros(p.N)
    _check(lib.od3_forward_trace(ctypes.byref(st), _ptr(_f64(g)), _ptr(mu), _ptr(mv), _ptr(sp)), "forward3d_trace")
    return mu, mv, sp


def tlm3d(p: Problem3D, g, dg, df0=None):
    """Tangent-linear model.  Returns (du^N, dv^N)."""
    lib = _load3d()
    st = p._struct()
    du = np.zeros((p.nz, p.ny, p.nx))
    dv = np.zeros_like(du)
    _check(lib.od3_tlm(ctypes.byref(st), _ptr(_f64(g)), _ptr(_f64(dg)), _ptr(_f64(df0)), _ptr(du), _ptr(dv)),
           "tlm3d")
    return du, dv


def adjoint3d(p: Problem3D, g=None, seed_u=None, seed_v=None, want_psi0=False):
    """Exact discrete adjoint.  Returns (J, dJ/dg [N][nz][ny][nx], psi0 [nz][ny][nx][2][19] or None)."""
    lib = _load3d()
    st = p._struct()
    J = ctypes.c_double(0.0)
    E = np.zeros((p.N, p.nz, p.ny, p.nx))
    psi0 = np.zeros((p.nz, p.ny, p.nx, 2, 19)) if want_psi0 else None
    _check(lib.od3_adjoint(ctypes.byref(st), _ptr(_f64(g)), _ptr(_f64(seed_u)), _ptr(_f64(seed_v)), _ptr(E),
                           _ptr(psi0), ctypes.byref(J)), "adjoint3d")
    return J.value, E, psi0


def collide3d_node(p: Problem3D, x, y, z, n, f, g=0.0, phi_prev=0.0):
    """One D3Q19 collision at node (x, y, z), step n: f [2][19] -> (P [2][19], Phi^n)."""
    lib = _load3d()
    st = p._struct()
    P, phi = np.zeros((2, 19)), ctypes.c_double(0.0)
    _check(lib.od3_collide_node(ctypes.byref(st), x, y, z, n, _ptr(_f64(f)), float(g), float(phi_prev), _ptr(P),
                                ctypes.byref(phi)), "collide3d_node")
    return P, phi.value


def adjoint3d_node(p: Problem3D, x, y, z, n, f, rho, g=0.0, sigma_next=None):
    """Local D3Q19 AMRT step at node (x, y, z), step n, the transpose of
    collide3d_node applied to rho [2][19] and, when sigma_next is given, to
    the adjoint c'_{n+1} sigma^{n+1} of Phi^n's use at step n + 1.
    Returns (psi [2][19], sigma^n, lambda_Phi)."""
    lib = _load3d()
    st = p._struct()
    psi, sig, lam = np.zeros((2, 19)), ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib.od3_adjoint_node(ctypes.byref(st), x, y, z, n, _ptr(_f64(f)), float(g), _ptr(_f64(rho)),
                                0 if sigma_next is None else 1, 0.0 if sigma_next is None else float(sigma_next),
                                _ptr(psi), ctypes.byref(sig), ctypes.byref(lam)), "adjoint3d_node")
    return psi, sig.value, lam.value


def from_workload3d(w, N=None) -> Problem3D:
    """D3Q19 oracle problem from a seeded workload (per-node fields)."""
    Du, Dv = w.D_fields()
    return Problem3D(nx=w.nx, ny=w.ny, nz=w.nz, N=w.N if N is None else N, Du=Du, Dv=Dv, u0=w.u0, v0=w.v0,
                     u_tgt=w.u_tgt, a=w.a_fields(), d_u=w.d_u, d_v=w.d_v, chi=w.chi, r_vu=w.r_vu, r_vv=w.r_vv,
                     alpha=w.alpha, s=tuple(w.s), source_order=w.source_order)
