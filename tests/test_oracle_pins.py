"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: the paper's
printed tables and moment listing, lattice isotropy identities, the BGK special
case, conservation laws, the closed-form anisotropic Gaussian, an independent
pseudo-spectral solution of the PDE, the tangent/adjoint dot-product identity
and brute-force finite differences.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1908_03876_gb300 import workloads as W
from paper_1908_03876_gb300.workloads import rotated_tensor

CS2 = 1.0 / 3.0


# ----------------------------------------------------------------- lattice

def test_d2q9_tables_match_paper(golden_dir):
    with open(os.path.join(golden_dir, "d2q9_lattice.json")) as fh:
        gold = json.load(fh)
    e, w, M, Minv = oracle.lattice(9)
    assert np.array_equal(e, np.array(gold["e"]))
    assert np.allclose(w * gold["w_den"], gold["w_num"], rtol=0, atol=1e-13)
    assert np.array_equal(M, np.array(gold["M0"], dtype=float))
    assert np.allclose(Minv @ M, np.eye(9), atol=1e-13)


@pytest.mark.parametrize("Q", [5, 9])
def test_lattice_isotropy(Q):
    """sum w = 1, sum w e = 0, sum w e e = Cs^2 I, sum w U = 0 (Sec. 3.1)."""
    e, w, M, Minv = oracle.lattice(Q)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose((w[:, None] * e).sum(0), 0.0, atol=1e-15)
    ee = np.einsum("i,ia,ib->ab", w, e, e)
    assert np.allclose(ee, CS2 * np.eye(2), atol=1e-15)
    U = np.einsum("ia,ib->iab", e, e) - CS2 * np.eye(2)[None]
    assert np.allclose(np.einsum("i,iab->ab", w, U), 0.0, atol=1e-15)
    # moment rows are mutually orthogonal (Gram-Schmidt basis)
    G = M @ M.T
    assert np.allclose(G - np.diag(np.diag(G)), 0.0)
    assert np.allclose(Minv @ M, np.eye(Q), atol=1e-13)


def test_equilibrium_moments_match_listing(golden_dir):
    """M phi^eq equals the paper's listed m^eq for random Theta, a, d."""
    with open(os.path.join(golden_dir, "meq_d2q9.json")) as fh:
        rows = np.array(json.load(fh)["rows"], dtype=float)
    e, w, M, _ = oracle.lattice(9)
    rng = np.random.default_rng(11)
    for _ in range(20):
        Th = rng.uniform(0.1, 3.0)
        a = rng.uniform(-0.2, 0.2, 2)
        d = rng.uniform(0.4, 1.5)
        B = (np.outer(a, a) + d * CS2 * np.eye(2)) * Th
        basis = np.array([Th, a[0] * Th, a[1] * Th, B[0, 0], B[1, 1], B[0, 1]])
        m = M @ oracle.feq(9, Th, a, d)
        assert np.allclose(m, rows @ basis, rtol=0, atol=1e-13)


@pytest.mark.parametrize("Q", [5, 9])
def test_equilibrium_constraints_TF0(Q):
    """sum phi^eq = Theta, sum e phi^eq = a Theta, sum e e phi^eq = (aa + d Cs^2 I) Theta
    (eq. TF0).  D2Q5 meets the stress condition only for d = 1, a = 0."""
    e, w, M, _ = oracle.lattice(Q)
    rng = np.random.default_rng(3)
    for _ in range(10):
        Th = rng.uniform(0.1, 3.0)
        a = rng.uniform(-0.2, 0.2, 2) if Q == 9 else np.zeros(2)
        d = rng.uniform(0.5, 1.5) if Q == 9 else 1.0
        f = oracle.feq(Q, Th, a, d)
        assert abs(f.sum() - Th) < 1e-13
        assert np.allclose(e.T @ f, a * Th, atol=1e-13)
        stress = np.einsum("ia,ib,i->ab", e, e, f)
        assert np.allclose(stress, (np.outer(a, a) + d * CS2 * np.eye(2)) * Th, atol=1e-13)


# ------------------------------------------------------ small problem helper

def _problem(n=12, N=10, Q=9, chi=-0.1, adv=True, solid=False, seed=0, source_order=2, alpha=1e-3):
    w = W.aniso(n, n, N, seed=seed, precision=64, chi=chi)
    if not adv:
        w.adv = "none"
    if Q == 5:
        w.Q = 5
        w.aniso, w.adv = "const", "none"
    if solid:
        w.solid = W.disc_mask(n, n, seed + 7, rmin=1.5, rmax=3.0, fraction=0.15)
        w.window = (2, 3, n - 5, n - 6)
        x0, y0, cx, cy = w.window
        w.cmask = (1 - w.solid[y0:y0 + cy, x0:x0 + cx]).astype(np.uint8)
    w.source_order = source_order
    w.alpha = alpha
    return w, oracle.from_workload(w)


# ------------------------------------------------- one node, one collision

@pytest.mark.parametrize("n", [0, 5])
def test_single_node_collision_moments(n):
    """The local collision at one node against the moment conditions the
    scheme is built on (Sec. 3.1: TF0, the K block acting on the fluxes, the
    source moments of eq. PhiS with V chosen after PC13), for arbitrary
    pre-collision populations and K from D by K = (D/(d Cs^2 tau) + I/2)^-1:
      Phi^n       = r_vu u + r_vv v + g                     (u, v the moments of f)
      sum P_u     = u                                       (no source for u; sum_i S_i = 0)
      sum P_v     = v + c_n Phi^n + c'_n Phi^{n-1}          (c_0 = tau, c'_0 = 0; else 3tau/2, -tau/2)
      sum e P_u   = j_u - K_u (j_u - a u)                   (chi = 0)
      sum e P_v   = j_v - K_v (j_v - a v) + V (c_n Phi^n + c'_n Phi^{n-1}),  V = (I - K_v/2) a
    and chi (the chemotactic cross-diffusion source of u) changes u's flux in
    proportion to chi and neither u's mass nor species v.  (The direction of
    that change, K_u G with G from v's non-equilibrium flux, is pinned by the
    pseudo-spectral PDE comparisons.)"""
    from dataclasses import replace

    w = W.aniso(12, 12, 8, seed=4, precision=64, chi=0.0)
    p0 = oracle.from_workload(w)
    e, _, _, _ = oracle.lattice(9)
    rng = np.random.default_rng(11 + n)
    tau = p0.tau
    c_now, c_prev = (tau, 0.0) if n == 0 else (1.5 * tau, -0.5 * tau)
    for _ in range(4):
        x, y = (int(v) for v in rng.integers(0, 12, 2))
        a = p0.a[y, x]
        fu = oracle.feq(9, rng.uniform(0.8, 1.2), a, p0.d_u) + rng.normal(0, 0.01, 9)
        fv = oracle.feq(9, rng.uniform(0.1, 0.5), a, p0.d_v) + rng.normal(0, 0.01, 9)
        g, phi_prev = rng.normal(0, 0.05), rng.normal(0, 0.05)
        u, v = fu.sum(), fv.sum()
        ju, jv = e.T @ fu, e.T @ fv
        Pu, Pv, Phi = oracle.collide_node(p0, x, y, n, fu, fv, g, phi_prev)

        def K_of(D, d):
            Dm = np.array([[D[0], D[1]], [D[1], D[2]]])
            return np.linalg.inv(Dm / (d * CS2 * tau) + 0.5 * np.eye(2))

        Ku, Kv = K_of(p0.Du[y, x], p0.d_u), K_of(p0.Dv[y, x], p0.d_v)
        src = c_now * Phi + c_prev * phi_prev
        assert abs(Phi - (p0.r_vu * u + p0.r_vv * v + g)) < 1e-14
        assert abs(Pu.sum() - u) < 1e-13
        assert abs(Pv.sum() - (v + src)) < 1e-13
        assert np.allclose(e.T @ Pu, ju - Ku @ (ju - a * u), rtol=0, atol=1e-13)
        V = (np.eye(2) - 0.5 * Kv) @ a
        assert np.allclose(e.T @ Pv, jv - Kv @ (jv - a * v) + V * src, rtol=0, atol=1e-13)

        per_chi = []
        for chi in (0.3, -0.7):
            Pu_c, Pv_c, _ = oracle.collide_node(replace(p0, chi=chi), x, y, n, fu, fv, g, phi_prev)
            assert abs(Pu_c.sum() - u) < 1e-13
            assert np.array_equal(Pv_c, Pv)  # chemotaxis acts on u only
            per_chi.append(e.T @ (Pu_c - Pu) / chi)
        assert np.allclose(per_chi[0], per_chi[1], rtol=1e-9, atol=1e-13)
        assert np.linalg.norm(per_chi[0]) > 1e-6


@pytest.mark.parametrize("n", [0, 5])
def test_local_adjoint_is_the_transposed_local_jacobian(n):
    """One node of the AMRT step against the dense Jacobian of one forward
    collision at that node, by central differences (the unit-level form of
    the adjoint checks; Sec. 3.2.1: transposed collision, scalar adjoint
    equilibrium, coupling terms CAE-L).  With L = rho_u.P_u + rho_v.P_v +
    lam Phi^n (lam = c'_{n+1} sigma^{n+1}, the adjoint of Phi^n's use at step
    n + 1): psi_u = dL/df_u, psi_v = dL/df_v, lambda_Phi = dL/dg and
    c'_n sigma^n = dL/dPhi^{n-1}, for every input of the 18 + 2."""
    w = W.aniso(12, 12, 8, seed=4, precision=64, chi=-0.4)
    w.r_vu, w.r_vv = 0.3, -0.2
    p = oracle.from_workload(w)
    e, _, _, _ = oracle.lattice(9)
    rng = np.random.default_rng(21 + n)
    tau = p.tau
    c_prev_n = 0.0 if n == 0 else -0.5 * tau
    c_prev_next = -0.5 * tau
    h = 1e-6
    for _ in range(3):
        x, y = (int(v) for v in rng.integers(0, 12, 2))
        a = p.a[y, x]
        fu = oracle.feq(9, rng.uniform(0.8, 1.2), a, p.d_u) + rng.normal(0, 0.01, 9)
        fv = oracle.feq(9, rng.uniform(0.1, 0.5), a, p.d_v) + rng.normal(0, 0.01, 9)
        g, phi_prev = rng.normal(0, 0.05), rng.normal(0, 0.05)
        ru, rv, sig_next = rng.normal(size=9), rng.normal(size=9), rng.normal()
        lam_next = c_prev_next * sig_next

        def L(fu_, fv_, g_, pp_):
            Pu, Pv, Phi = oracle.collide_node(p, x, y, n, fu_, fv_, g_, pp_)
            return ru @ Pu + rv @ Pv + lam_next * Phi

        dfu, dfv = np.zeros(9), np.zeros(9)
        for i in range(9):
            d = np.zeros(9)
            d[i] = h
            dfu[i] = (L(fu + d, fv, g, phi_prev) - L(fu - d, fv, g, phi_prev)) / (2 * h)
            dfv[i] = (L(fu, fv + d, g, phi_prev) - L(fu, fv - d, g, phi_prev)) / (2 * h)
        dg = (L(fu, fv, g + h, phi_prev) - L(fu, fv, g - h, phi_prev)) / (2 * h)
        dpp = (L(fu, fv, g, phi_prev + h) - L(fu, fv, g, phi_prev - h)) / (2 * h)

        psu, psv, sigma, lam_phi = oracle.adjoint_node(p, x, y, n, fu, fv, ru, rv, g=g, sigma_next=sig_next)
        scale = max(np.abs(dfu).max(), np.abs(dfv).max(), 1.0)
        assert np.allclose(psu, dfu, rtol=0, atol=1e-8 * scale)
        assert np.allclose(psv, dfv, rtol=0, atol=1e-8 * scale)
        assert abs(lam_phi - dg) < 1e-8 * scale
        assert abs(c_prev_n * sigma - dpp) < 1e-8 * scale


# ----------------------------------------------------------- special cases

def _bgk_numpy(p, s):
    """Independent BGK advection-diffusion loop: f <- f - s (f - f^eq), pull-stream."""
    e, w, _, _ = oracle.lattice(p.Q)
    n = p.nx
    a = p.a if p.a is not None else np.zeros((n, n, 2))
    def feq(Th, d):
        ea = np.einsum("ia,yxa->yxi", e, a)
        aa = np.einsum("yxa,yxb->yxab", a, a)
        U = np.einsum("ia,ib->iab", e, e) - CS2 * np.eye(2)[None]
        BU = np.einsum("yxab,iab->yxi", aa, U) + (d - 1) * CS2 * np.einsum("iaa->i", U)[None, None]
        return w[None, None] * Th[..., None] * (1 + ea / CS2 + BU / (2 * CS2 * CS2))
    fu, fv = feq(p.u0, p.d_u), feq(p.v0, p.d_v)
    for _ in range(p.N):
        for f, d in ((fu, p.d_u), (fv, p.d_v)):
            f -= s * (f - feq(f.sum(-1), d))
            for i in range(p.Q):
                f[..., i] = np.roll(np.roll(f[..., i], e[i, 0], axis=1), e[i, 1], axis=0)
    return fu.sum(-1), fv.sum(-1)


@pytest.mark.parametrize("Q", [5, 9])
def test_mrt_reduces_to_bgk(Q):
    """K = s I and s_1..s_6 = s: M^-1 Pi M = s I, the MRT is the BGK scheme."""
    s = 1.3
    w, p = _problem(n=10, N=15, Q=Q, chi=0.0)
    p.r_vu = p.r_vv = 0.0
    D = (1.0 / s - 0.5) * CS2          # K = s I  <=>  D = d Cs^2 tau (1/s - 1/2)
    p.Du = np.broadcast_to([D, 0.0, D], (10, 10, 3)).copy()
    p.Dv = p.Du.copy()
    p.s = (s,) * 7
    if Q == 9:
        p.a = np.random.default_rng(1).uniform(-0.05, 0.05, (10, 10, 2))
    _, u, v = oracle.forward(p)
    ub, vb = _bgk_numpy(p, s)
    assert np.abs(u - ub).max() < 1e-13
    assert np.abs(v - vb).max() < 1e-13


@pytest.mark.parametrize("solid", [False, True])
def test_mass_conservation(solid):
    """Periodic / bounce-back box, Phi = g = 0, chemotaxis on: sum u and sum v
    are invariant (sum_i S_i = 0, eq. TF0; collision conserves m0)."""
    w, p = _problem(n=16, N=40, chi=-0.1, solid=solid)
    p.r_vu = p.r_vv = 0.0
    p.v0 = 1.0 + 0.3 * np.sin(np.arange(16) / 3.0)[None, :] * np.ones((16, 1))
    mu, mv, _ = oracle.forward_trace(p)
    assert np.abs(mu / mu[0] - 1).max() < 1e-14
    assert np.abs(mv / mv[0] - 1).max() < 1e-14


@pytest.mark.parametrize("source_order", [1, 2])
def test_source_mass_balance(source_order):
    """sum v^{n+1} - sum v^n = tau sum [Phi^n + (1/2)(Phi^n - Phi^{n-1})], Phi^{-1} := Phi^0."""
    w, p = _problem(n=14, N=12, chi=-0.1, source_order=source_order)
    g = w.random_control(4, 0.05)
    mu, mv, sp = oracle.forward_trace(p, g)
    dv = np.diff(mv)
    prev = np.concatenate([[sp[0]], sp[:-1]])
    expect = sp + (0.5 * (sp - prev) if source_order == 2 else 0.0)
    assert np.allclose(dv, expect[:-1], rtol=0, atol=1e-12 * np.abs(mv).max())
    assert np.abs(mu / mu[0] - 1).max() < 1e-14


def _gauss_field(n, mu, Sig, mass):
    Si = np.linalg.inv(Sig)
    det = np.linalg.det(Sig)
    x = np.arange(n)[None, :]
    y = np.arange(n)[:, None]
    out = np.zeros((n, n))
    for ix in (-1, 0, 1):
        for iy in (-1, 0, 1):
            dx = x - mu[0] + ix * n
            dy = y - mu[1] + iy * n
            out += np.exp(-0.5 * (Si[0, 0] * dx * dx + 2 * Si[0, 1] * dx * dy + Si[1, 1] * dy * dy))
    return mass * out / (2 * np.pi * np.sqrt(det))


def _gauss_run(n, sig0, steps, lam, th, Q, a):
    D = rotated_tensor(lam, np.array(th))
    Dm = np.array([[D[0], D[1]], [D[1], D[2]]])
    mu = np.array([n / 2, n / 2])
    mass = 100.0 * (n / 32) ** 2
    u0 = 1.0 + _gauss_field(n, mu, sig0 ** 2 * np.eye(2), mass)
    Df = np.broadcast_to(D, (n, n, 3)).copy()
    af = np.broadcast_to(np.array(a, float), (n, n, 2)).copy()
    p = oracle.Problem(nx=n, ny=n, N=steps, Q=Q, Du=Df, Dv=Df, u0=u0, v0=np.zeros((n, n)),
                       u_tgt=np.zeros((n, n)), a=af)
    _, u, _ = oracle.forward(p)
    exact = 1.0 + _gauss_field(n, mu + np.array(a) * steps, sig0 ** 2 * np.eye(2) + 2 * Dm * steps, mass)
    return np.linalg.norm(u - exact) / np.linalg.norm(exact - 1.0), abs(u.sum() - u0.sum()) / u0.sum()


@pytest.mark.parametrize("Q,lam,th,adv", [(9, (0.08, 0.02), 0.6, 0.0), (9, (0.08, 0.02), 0.6, 0.04),
                                          (5, (0.1, 0.1), 0.0, 0.0)])
def test_anisotropic_gaussian_closed_form(Q, lam, th, adv):
    """chi = 0, no reaction, constant D = R diag(l1, l2) R^T: a Gaussian of
    covariance S0 evolves to S0 + 2 D t (centre moved by a t).  Pins the
    D -> K map D = d Cs^2 tau (K^-1 - I/2), M0, Pi and phi^eq: 2nd-order
    convergence under diffusive refinement (h/2, tau/4, a/2)."""
    errs = []
    for k, (n, s0, N) in enumerate([(32, 2.0, 25), (64, 4.0, 100), (128, 8.0, 400)]):
        a = (adv / 2 ** k, -adv / 2 ** (k + 1))
        e, dm = _gauss_run(n, s0, N, lam, th, Q, a)
        errs.append(e)
        assert dm < 1e-13
    assert errs[0] < 2.5e-2
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.6 and 3.5 < r2 < 4.6, errs


def _spectral_ref(L, T, Du, Dv, chi, rvu, rvv, u0, v0, dt=0.02):
    """Pseudo-spectral RK4 solution of u_t = div(D_u grad u - chi u grad v),
    v_t = div(D_v grad v) + r_vu u + r_vv v on a periodic square."""
    n = u0.shape[0]
    k = 2 * np.pi * np.fft.fftfreq(n, d=L / n)
    KX, KY = np.meshgrid(k, k)

    def d(f, K):
        return np.real(np.fft.ifft2(1j * K * np.fft.fft2(f)))

    def rhs(u, v):
        ux, uy, vx, vy = d(u, KX), d(u, KY), d(v, KX), d(v, KY)
        fxu = Du[0] * ux + Du[1] * uy - chi * u * vx
        fyu = Du[1] * ux + Du[2] * uy - chi * u * vy
        fxv = Dv[0] * vx + Dv[1] * vy
        fyv = Dv[1] * vx + Dv[2] * vy
        return d(fxu, KX) + d(fyu, KY), d(fxv, KX) + d(fyv, KY) + rvu * u + rvv * v

    u, v = u0.copy(), v0.copy()
    for _ in range(int(round(T / dt))):
        k1 = rhs(u, v)
        k2 = rhs(u + dt / 2 * k1[0], v + dt / 2 * k1[1])
        k3 = rhs(u + dt / 2 * k2[0], v + dt / 2 * k2[1])
        k4 = rhs(u + dt * k3[0], v + dt * k3[1])
        u = u + dt / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
        v = v + dt / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
    return u, v


@pytest.mark.slow
def test_chemotaxis_coupling_against_pde():
    """The coupled scheme (cross-diffusion S_u with A = K D_{u,1}/tau and the
    local grad v reading) converges at 2nd order to an independent
    pseudo-spectral solution of the PDE; the opposite chemotaxis sign does not."""
    L, T = 32, 20
    Du = rotated_tensor((0.08, 0.02), np.array(0.6))
    Dv = np.array([0.2, 0.0, 0.2])
    chi, rvu, rvv = -0.1, 0.02, -0.01

    def init(n):
        x = np.arange(n)[None, :] * L / n
        y = np.arange(n)[:, None] * L / n
        k = 2 * np.pi / L
        return 1 + 0.2 * np.cos(k * x) * np.sin(k * y) + 0.1 * np.sin(2 * k * x), \
            1 + 0.3 * np.sin(k * (x + y)) * np.ones_like(x)

    us, vs = _spectral_ref(L, T, Du, Dv, chi, rvu, rvv, *init(L))

    def lb(r, chi_):
        n = L * r
        u0, v0 = init(n)
        p = oracle.Problem(nx=n, ny=n, N=T * r * r, Q=9, Du=np.broadcast_to(Du, (n, n, 3)).copy(),
                           Dv=np.broadcast_to(Dv, (n, n, 3)).copy(), u0=u0, v0=v0, u_tgt=np.zeros((n, n)),
                           chi=chi_, r_vu=rvu / r ** 2, r_vv=rvv / r ** 2)
        _, u, v = oracle.forward(p)
        return u[::r, ::r], v[::r, ::r]

    errs = []
    for r in (1, 2, 4):
        u, v = lb(r, chi)
        errs.append((np.linalg.norm(u - us) / np.linalg.norm(us - us.mean()),
                     np.linalg.norm(v - vs) / np.linalg.norm(vs - vs.mean())))
    for c in range(2):
        r1, r2 = errs[0][c] / errs[1][c], errs[1][c] / errs[2][c]
        assert 3.5 < r1 < 4.6 and 3.5 < r2 < 4.6, errs
    u_flip, _ = lb(1, -chi)
    assert np.linalg.norm(u_flip - us) / np.linalg.norm(us - us.mean()) > 20 * errs[0][0]


# ------------------------------------------- convective source (V and grad v)
#
# The source weights w~_i = w_i (1 + V.e_i / Cs^2) with V = (I - K_v/2) a
# (eq. PhiS and the choice of V after PC13, kappa_x = 0) and the term
# (1/2) K_v a Phi_v of the local grad v (relation C146) only act where
# convection meets a source.  A mistake in either (V = a, a sign, swapped
# components, the term dropped) leaves an O(tau) error in the recovered PDE:
# under diffusive refinement that is O(h^2), the same order as the scheme's
# own truncation error, so a convergence-rate test against a closed form or an
# independent PDE solver cannot see it (the last two tests below pass with any
# of those mistakes planted).  The first two tests isolate each term with an
# observable that the PDE fixes exactly and that such a mistake moves at first
# order.

def _const_aniso(n, lam, th):
    return np.broadcast_to(rotated_tensor(lam, np.array(th)), (n, n, 3)).copy()


def _plume_centre_velocity_error(r, a=(0.08, 0.05), n=96, N=120, sig=3.0):
    """Relative error of the centre-of-mass velocity of a v plume that reacts
    linearly (Phi_v = r v), against the convection velocity a.

    For dv/dt = div(D grad v) - div(a v) + r v with constant D and a, the mass
    grows as e^{rt} and the centre of mass moves at exactly a, for every r.
    The plume stays far from the periodic edges, so sum x v / sum v is its
    centre.  Measured between N/2 and N steps (after the start-up transient)."""
    D = _const_aniso(n, (0.08, 0.02), 0.6)
    x = np.arange(n)[None, :]
    y = np.arange(n)[:, None]
    v0 = np.exp(-((x - 32.0) ** 2 + (y - 32.0) ** 2) / (2 * sig * sig))
    af = np.broadcast_to(np.array(a, float), (n, n, 2)).copy()
    centres = []
    for steps in (N // 2, N):
        p = oracle.Problem(nx=n, ny=n, N=steps, Q=9, Du=D, Dv=D, u0=np.zeros((n, n)), v0=v0,
                           u_tgt=np.zeros((n, n)), a=af, r_vv=r)
        _, _, v = oracle.forward(p)
        m = v.sum()
        centres.append(np.array([(v * x).sum() / m, (v * y).sum() / m]))
    w = (centres[1] - centres[0]) / (N - N // 2)
    return w / np.array(a) - 1.0


def test_reacting_plume_centre_moves_with_convection():
    """Pins V of the source weights (eq. PhiS, V after PC13).  The source
    deposits first moment V Phi per step; only V = (I - K_v/2) a makes the
    centre of a reacting plume move at a up to O(r^2) in the reaction rate per
    step r.  Planted V = a, V = (I + K_v/2) a or swapped components give a
    first-order error (r/2 and more; halving r only halves it), which this
    test rejects through the ratio of the errors at r and r/2 (measured 3.90
    and 2.1e-3 at r = 0.05 here, against ratios 1.45-1.97 and errors up to
    4.8e-2 with those mistakes)."""
    e0 = _plume_centre_velocity_error(0.0)
    e1 = _plume_centre_velocity_error(0.05)
    e2 = _plume_centre_velocity_error(0.025)
    print("centre-velocity errors", e0, e1, e2, e1 / e2)
    assert np.abs(e0).max() < 1e-10          # no source: exact transport speed
    assert np.abs(e1).max() < 4e-3
    assert np.all((e1 / e2 > 3.5) & (e1 / e2 < 4.5))


def _uniform_chemical_drift(N, chi=1.0, a=(0.06, -0.04), n=48, g0=0.01, sig=4.0):
    """u^N with and without chemotaxis when v is uniform and produced
    uniformly (Phi_v = g0 everywhere, r_vu = r_vv = 0): grad v = 0 exactly,
    so the PDE's chemotactic flux chi u grad v vanishes and u must not feel
    chi.  Returns ||u(chi) - u(0)|| / ||u(0) - 1||."""
    Du = _const_aniso(n, (0.08, 0.02), 0.6)
    Dv = _const_aniso(n, (0.2, 0.05), 1.0)
    x = np.arange(n)[None, :]
    y = np.arange(n)[:, None]
    u0 = 1.0 + 0.5 * np.exp(-((x - n / 2) ** 2 + (y - n / 2) ** 2) / (2 * sig * sig))
    af = np.broadcast_to(np.array(a, float), (n, n, 2)).copy()
    g = np.full((N, n, n), g0)
    us = []
    for c in (chi, 0.0):
        p = oracle.Problem(nx=n, ny=n, N=N, Q=9, Du=Du, Dv=Dv, u0=u0, v0=np.ones((n, n)),
                           u_tgt=np.zeros((n, n)), a=af, chi=c)
        _, u, v = oracle.forward(p, g)
        assert np.ptp(v) == 0.0   # the chemical stays uniform
        us.append(u)
    return np.linalg.norm(us[0] - us[1]) / np.linalg.norm(us[1] - 1.0)


def test_uniform_chemical_exerts_no_chemotactic_drift():
    """Pins the (1/2) K_v a Phi_v term of grad v (reading of C146) and,
    again, V.  With uniform v and uniform production Phi, the pre-collision
    flux settles at j_v - a v = K_v^-1 (V - a) Phi, so the local estimate is
    G = -[(V - a) + K_v a / 2] Phi / (d_v Cs^2): zero only with both terms as
    read.  From the equilibrium start G decays like (I - K_v)^n, giving u one
    bounded displacement; any mistake in either term leaves a constant G, a
    chemotactic drift of u that grows linearly in time.  Measured: 1.8e-4 at
    40 and 80 steps; 6e-3 to 4e-2, doubling from 40 to 80 steps, with the term
    dropped, its sign flipped, its factor 1/2 replaced by 1, or V = a."""
    d40, d80 = _uniform_chemical_drift(40), _uniform_chemical_drift(80)
    print("uniform-chemical drift", d40, d80)
    assert d80 < 1e-3
    assert d80 < 1.2 * d40


def test_advected_reacting_gaussian_closed_form():
    """Constant convection, anisotropic diffusion and a linear reaction on v
    (chi = 0): v(t) = e^{rt} G(x - a t; S0 + 2 D_v t) with G a Gaussian
    (periodic images summed).  Second-order convergence under diffusive
    refinement (h/2, tau/4, a/2, r/4).  Checks the reaction's time levels
    (c_n Phi^n + c'_n Phi^{n-1}) against e^{rt} together with convection and
    anisotropic diffusion; it does not see V (see above)."""
    D = rotated_tensor((0.08, 0.02), np.array(0.6))
    Dm = np.array([[D[0], D[1]], [D[1], D[2]]])
    errs = []
    for k in range(3):
        n, s0, N = 32 * 2 ** k, 2.0 * 2 ** k, 25 * 4 ** k
        a, r = np.array([0.08, -0.04]) / 2 ** k, 0.02 / 4 ** k
        mu, mass = np.array([n / 2, n / 2]), 100.0 * (n / 32) ** 2
        v0 = _gauss_field(n, mu, s0 ** 2 * np.eye(2), mass)
        Df = np.broadcast_to(D, (n, n, 3)).copy()
        p = oracle.Problem(nx=n, ny=n, N=N, Q=9, Du=Df, Dv=Df, u0=np.zeros((n, n)), v0=v0,
                           u_tgt=np.zeros((n, n)), a=np.broadcast_to(a, (n, n, 2)).copy(), r_vv=r)
        _, _, v = oracle.forward(p)
        exact = np.exp(r * N) * _gauss_field(n, mu + a * N, s0 ** 2 * np.eye(2) + 2 * Dm * N, mass)
        errs.append(np.linalg.norm(v - exact) / np.linalg.norm(exact))
    print("advected reacting Gaussian errors", errs)
    assert errs[0] < 4e-2
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.6 and 3.5 < r2 < 4.6, errs


def _spectral_shear_ref(L, T, Du, Dv, chi, rvu, rvv, a0, gsrc, u0, v0, dt=0.02):
    """Pseudo-spectral RK4 solution of
    u_t = div(D_u grad u - chi u grad v - a u),
    v_t = div(D_v grad v - a v) + r_vu u + r_vv v + g(x, t),
    a = (a0 sin(2 pi y / L), 0), on a periodic square."""
    n = u0.shape[0]
    k = 2 * np.pi * np.fft.fftfreq(n, d=L / n)
    KX, KY = np.meshgrid(k, k)
    x = np.arange(n)[None, :] * L / n
    y = np.arange(n)[:, None] * L / n
    ax = a0 * np.sin(2 * np.pi * y / L) * np.ones_like(x)

    def d(f, K):
        return np.real(np.fft.ifft2(1j * K * np.fft.fft2(f)))

    def rhs(u, v, t):
        ux, uy, vx, vy = d(u, KX), d(u, KY), d(v, KX), d(v, KY)
        fxu = Du[0] * ux + Du[1] * uy - chi * u * vx - ax * u
        fyu = Du[1] * ux + Du[2] * uy - chi * u * vy
        fxv = Dv[0] * vx + Dv[1] * vy - ax * v
        fyv = Dv[1] * vx + Dv[2] * vy
        return d(fxu, KX) + d(fyu, KY), d(fxv, KX) + d(fyv, KY) + rvu * u + rvv * v + gsrc(x, y, t)

    u, v, t = u0.copy(), v0.copy(), 0.0
    for _ in range(int(round(T / dt))):
        k1 = rhs(u, v, t)
        k2 = rhs(u + dt / 2 * k1[0], v + dt / 2 * k1[1], t + dt / 2)
        k3 = rhs(u + dt / 2 * k2[0], v + dt / 2 * k2[1], t + dt / 2)
        k4 = rhs(u + dt * k3[0], v + dt * k3[1], t + dt)
        u = u + dt / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
        v = v + dt / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
        t += dt
    return u, v


@pytest.mark.slow
def test_shear_convection_and_source_against_pde():
    """Chemotaxis with the shear convection of the benchmark workload and a
    smooth space-time control g: the scheme converges at second order to an
    independent pseudo-spectral solution (g^n = g(t_n) tau in lattice
    units).  A consistency check of the convective source path as a whole;
    by itself it cannot pin V or the (1/2) K_v a Phi_v term (see above)."""
    L, T = 32, 20
    Du = rotated_tensor((0.08, 0.02), np.array(0.6))
    Dv = rotated_tensor((0.2, 0.1), np.array(-0.3))
    chi, rvu, rvv, a0, gam = -0.1, 0.02, -0.01, 0.1, 0.01
    kk = 2 * np.pi / L

    def gsrc(x, y, t):
        return gam * (1 + np.sin(kk * x + 2 * np.pi * 0.3 * t / T) * np.cos(kk * y))

    def init(n):
        x = np.arange(n)[None, :] * L / n
        y = np.arange(n)[:, None] * L / n
        return 1 + 0.2 * np.cos(kk * x) * np.sin(kk * y) + 0.1 * np.sin(2 * kk * x), \
            1 + 0.3 * np.sin(kk * (x + y)) * np.ones_like(x)

    us, vs = _spectral_shear_ref(L, T, Du, Dv, chi, rvu, rvv, a0, gsrc, *init(L))
    errs = []
    for r in (1, 2, 4):
        n, N = L * r, T * r * r
        u0, v0 = init(n)
        x = np.arange(n)[None, :] / r
        y = np.arange(n)[:, None] / r
        ax = (a0 / r) * np.sin(kk * y) * np.ones_like(x)
        g = np.stack([gsrc(x, y, m / r ** 2) / r ** 2 for m in range(N)])
        p = oracle.Problem(nx=n, ny=n, N=N, Q=9, Du=np.broadcast_to(Du, (n, n, 3)).copy(),
                           Dv=np.broadcast_to(Dv, (n, n, 3)).copy(), u0=u0, v0=v0, u_tgt=np.zeros((n, n)),
                           chi=chi, r_vu=rvu / r ** 2, r_vv=rvv / r ** 2,
                           a=np.stack([ax, np.zeros_like(ax)], -1))
        _, u, v = oracle.forward(p, g)
        u, v = u[::r, ::r], v[::r, ::r]
        errs.append((np.linalg.norm(u - us) / np.linalg.norm(us - us.mean()),
                     np.linalg.norm(v - vs) / np.linalg.norm(vs - vs.mean())))
    print("shear + source vs pseudo-spectral", errs)
    for c in range(2):
        r1, r2 = errs[0][c] / errs[1][c], errs[1][c] / errs[2][c]
        assert 3.5 < r1 < 4.6 and 3.5 < r2 < 4.6, errs


# --------------------------------------------------------- adjoint / gradient

@pytest.mark.parametrize("case", [
    dict(Q=9, adv=True, solid=False, source_order=2),
    dict(Q=9, adv=True, solid=True, source_order=2),
    dict(Q=9, adv=False, solid=False, source_order=1),
    dict(Q=5, adv=False, solid=False, source_order=2),
])
def test_dot_product_identity(case):
    """<w, TLM(dg, df0)> = <ADJ(w), (dg, df0)>: the AMRT sweep is the exact
    transpose of the sensitivity LBE (LIBEG-V), to roundoff."""
    n = 12
    w, p = _problem(n=n, N=9, chi=-0.1, alpha=0.0, **case)
    rng = np.random.default_rng(5)
    g = w.random_control(1, 0.05)
    dg = rng.standard_normal(g.shape)
    if p.cmask is not None:
        dg *= p.cmask[None]
    df0 = rng.standard_normal((n, n, 2, p.Q))
    if p.solid is not None:
        df0 *= (1 - p.solid)[:, :, None, None]
    su, sv = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    if p.solid is not None:
        su *= 1 - p.solid
        sv *= 1 - p.solid
    _, du, dv = oracle.tlm(p, g, dg, df0)
    _, E, psi0 = oracle.adjoint(p, g, su, sv, want_psi0=True)
    lhs = np.sum(su * du) + np.sum(sv * dv)
    rhs = np.sum(E * dg) + np.sum(psi0 * df0)
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs)), (lhs, rhs)


def test_gradient_every_component_fd():
    """Every component of dJ/dg against central finite differences (8x8, 10 steps)."""
    w, p = _problem(n=8, N=10, chi=-0.1, alpha=1e-2)
    g = w.random_control(2, 0.05)
    J0, E, _ = oracle.adjoint(p, g)
    h = 1e-6
    fd = np.zeros_like(g)
    for idx in np.ndindex(g.shape):
        gp = g.copy()
        gp[idx] += h
        gm = g.copy()
        gm[idx] -= h
        fd[idx] = (oracle.forward(p, gp)[0] - oracle.forward(p, gm)[0]) / (2 * h)
    assert np.abs(fd - E).max() <= 1e-6 * np.abs(E).max()


@pytest.mark.parametrize("Q", [5, 9])
def test_gradient_fd_16x16(Q):
    """16x16, 50 steps, plain64 physics (sigma = 2): sampled components and a
    random direction against central finite differences."""
    w = W.plain64(16, 16, 50, sigma=2.0, Q=Q)
    w.chi = -0.05
    p = oracle.from_workload(w)
    g = w.random_control(9, 0.02)
    J0, E, _ = oracle.adjoint(p, g)
    h = 1e-6
    rng = np.random.default_rng(4)
    flat = rng.choice(g.size, 24, replace=False)
    for k in flat:
        idx = np.unravel_index(k, g.shape)
        gp = g.copy()
        gp[idx] += h
        gm = g.copy()
        gm[idx] -= h
        fd = (oracle.forward(p, gp)[0] - oracle.forward(p, gm)[0]) / (2 * h)
        assert abs(fd - E[idx]) <= 1e-6 * np.abs(E).max()
    d = rng.standard_normal(g.shape)
    fd = (oracle.forward(p, g + h * d)[0] - oracle.forward(p, g - h * d)[0]) / (2 * h)
    # central-difference roundoff is about eps * J / h
    assert abs(fd - np.sum(E * d)) <= 1e-7 * abs(fd) + 50 * np.finfo(float).eps * J0 / h


def test_gradient_fd_geometry():
    """Bounce-back, window control with a mask, advection: sampled FD components."""
    w, p = _problem(n=12, N=10, chi=-0.1, solid=True, alpha=1e-2)
    g = w.random_control(6, 0.05)
    J0, E, _ = oracle.adjoint(p, g)
    h = 1e-6
    rng = np.random.default_rng(8)
    for k in rng.choice(g.size, 30, replace=False):
        idx = np.unravel_index(k, g.shape)
        gp = g.copy()
        gp[idx] += h
        gm = g.copy()
        gm[idx] -= h
        fd = (oracle.forward(p, gp)[0] - oracle.forward(p, gm)[0]) / (2 * h)
        if p.cmask[idx[1], idx[2]] == 0:
            assert E[idx] == 0.0 and abs(fd) < 1e-12
        else:
            assert abs(fd - E[idx]) <= 1e-6 * np.abs(E).max()


def test_gd_step_decreases_cost():
    """One Armijo gradient-descent iteration lowers J (discrete-adjoint algorithm)."""
    w = W.plain64(16, 16, 30, sigma=2.0, Q=9)
    w.chi = -0.05
    p = oracle.from_workload(w)
    g = np.zeros(w.ctrl_shape)
    g1, info = oracle.gd_step(p, g)
    assert info["J"] < info["J0"]
    g2, info2 = oracle.gd_step(p, g1, lam_prev=info["lam"])
    assert info2["J"] < info["J"]


def test_windowed_gradient_fd():
    """Control piecewise constant over W time windows (the subspace g^n = G_w):
    every component of the window gradient against central finite differences
    of J(G), and W = N reproduces the per-step control exactly."""
    w = W.plain64(10, 10, 12, sigma=2.0, Q=9)
    w.chi = -0.05
    w.alpha = 1e-2
    w.windows = 3
    p = oracle.from_workload(w)
    assert w.ctrl_shape == (3, 10, 10)
    G = w.random_control(5, 0.05)
    J0, E, _ = oracle.adjoint(p, G)
    assert E.shape == G.shape
    h = 1e-6
    fd = np.zeros_like(G)
    for idx in np.ndindex(G.shape):
        gp = G.copy()
        gp[idx] += h
        gm = G.copy()
        gm[idx] -= h
        fd[idx] = (oracle.forward(p, gp)[0] - oracle.forward(p, gm)[0]) / (2 * h)
    assert np.abs(fd - E).max() <= 1e-6 * np.abs(E).max()
    # the same control written per step (windows = N) gives the same J and the
    # per-step gradient whose window sums are E
    w.windows = 0
    q = oracle.from_workload(w)
    g_steps = np.repeat(G, 4, axis=0)
    Jq, Eq, _ = oracle.adjoint(q, g_steps)
    assert Jq == J0
    assert np.abs(Eq.reshape(3, 4, 10, 10).sum(1) - E).max() <= 1e-14 * np.abs(E).max()


def _cg_problem():
    """A small chemotaxis problem (the control reaches u only through chi)."""
    w = W.plain64(8, 8, 8, sigma=1.5, Q=9, chi=-0.5)
    w.alpha = 1e-3
    w.windows = 2
    return w, oracle.from_workload(w)


def _reference_optimum(w, p):
    """The optimum by an independent optimiser (scipy's L-BFGS-B on the
    oracle's J and gradient), converged far below the tolerances used."""
    from scipy.optimize import minimize

    shape = w.ctrl_shape

    def fg(x):
        J, E, _ = oracle.adjoint(p, x.reshape(shape))
        return J, E.ravel()

    res = minimize(fg, np.zeros(int(np.prod(shape))), jac=True, method="L-BFGS-B",
                   options=dict(maxiter=2000, ftol=1e-15, gtol=1e-13, maxcor=30))
    return res.x.reshape(shape), float(res.fun)


@pytest.mark.parametrize("variant", ["FR", "PR", "HS", "DY"])
def test_cg_wolfe_steps_and_optimum(variant):
    """Nonlinear CG with the Wolfe-Powell search: every accepted step meets
    both Wolfe conditions (checked with fresh solves), the directions are
    descent directions, and the iterates reach the optimum found by an
    independent optimiser."""
    w, p = _cg_problem()
    gref, Jref = _reference_optimum(w, p)
    g = np.zeros(w.ctrl_shape)
    state = None
    for k in range(300):
        J_old, G_old, _ = oracle.adjoint(p, g)
        D = -G_old if state is None else state["D"]
        gd = float(np.sum(G_old * D))
        assert gd < 0
        g_new, state, info = oracle.cg_iteration(p, g, state, variant=variant)
        lam = info["lam"]
        J_new, G_new, _ = oracle.adjoint(p, g + lam * D)
        assert J_new <= J_old + 1e-4 * lam * gd + 1e-14 * abs(J_old)
        assert float(np.sum(G_new * D)) >= 0.1 * gd - 1e-14 * abs(gd)
        g = g_new
        if J_new - Jref <= 1e-11 * Jref:
            break
    assert J_new - Jref <= 1e-10 * Jref, (variant, k, J_new, Jref)
    assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref), np.linalg.norm(g - gref) / np.linalg.norm(gref)


def test_cg_beats_steepest_descent():
    """Polak-Ribiere CG needs fewer iterations than Armijo steepest descent to
    reach the reference optimum to 1e-9 (relative J)."""
    w, p = _cg_problem()
    _, Jref = _reference_optimum(w, p)

    def iterations(step):
        g = np.zeros(w.ctrl_shape)
        aux = None
        for k in range(1, 500):
            g, aux, info = step(g, aux)
            if info["J"] - Jref <= 1e-9 * Jref:
                return k
        return 500

    def sd(g, lam):
        g, info = oracle.gd_step(p, g, lam_prev=lam)
        return g, info["lam"], info

    def cg(g, st):
        return oracle.cg_iteration(p, g, st, variant="PR")

    n_sd, n_cg = iterations(sd), iterations(cg)
    print("iterations: steepest descent", n_sd, "CG", n_cg)
    assert n_cg < n_sd, (n_cg, n_sd)


def test_lma_step_minimises_the_quadratic_model():
    """The sensitivity-based step length (eq. LMA) is the minimiser of the
    quadratic model of J along -E: J at lam* matches the model to second
    order and the directional derivative there nearly vanishes (checked with
    fresh forward solves and central differences, not the adjoint)."""
    w, p = _cg_problem()
    g = w.random_control(3, 0.01)
    J0, E, _ = oracle.adjoint(p, g)
    g1, info = oracle.lma_step(p, g)
    lam = info["lam"]
    assert info["trials"] == 1 and info["J"] < J0
    e2 = float(np.sum(E * E))

    def phi(l):
        return oracle.forward(p, g - l * E)[0]

    h = 1e-4 * lam
    slope0 = (phi(h) - phi(-h)) / (2 * h)
    slope = (phi(lam + h) - phi(lam - h)) / (2 * h)
    assert abs(slope0 + e2) <= 1e-5 * e2          # phi'(0) = -||E||^2
    assert abs(slope) <= 0.02 * e2, (slope, e2)   # phi'(lam*) ~ 0 (the model is quadratic up to chemotaxis)
    # the exact 1-D minimiser lies within a few percent of lam*
    ls = lam * np.linspace(0.9, 1.1, 21)
    best = ls[int(np.argmin([phi(l) for l in ls]))]
    assert abs(best - lam) <= 0.05 * lam


def _cadjoint_gap(n, chi=-0.05):
    """Relative L2 gap between the continuous-adjoint gradient and the exact
    discrete gradient at g = 0, for the plain problem refined in the
    diffusive scaling (grid n, N = 40 (n/32)^2, bump width proportional to n)."""
    w = W.plain64(n, n, int(40 * (n / 32) ** 2), sigma=2.0 * n / 32, Q=9, chi=chi)
    w.alpha = 1e-3
    p = oracle.from_workload(w)
    g = np.zeros(w.ctrl_shape)
    _, E, _ = oracle.adjoint(p, g)
    _, Ec = oracle.cadjoint(p, g)
    return float(np.linalg.norm(Ec - E) / np.linalg.norm(E)), float(np.sum(E * Ec) / np.linalg.norm(E) / np.linalg.norm(Ec))


def test_continuous_adjoint_converges_to_discrete_gradient():
    """Alg. B (continuous adjoint solved by the MRT scheme with time reversed)
    is a consistent O(tau, h) approximation of the exact discrete gradient:
    the gap shrinks at first order under diffusive refinement (measured 12.4%,
    7.4%, 4.7% at 32, 48, 72 cells)."""
    gaps = [_cadjoint_gap(n) for n in (32, 48, 72)]
    print("continuous-adjoint gaps", gaps)
    assert gaps[0][0] > gaps[1][0] > gaps[2][0]
    assert gaps[2][0] < 0.06 and gaps[2][1] > 0.998
    # first order: the gap times the resolution stays about constant
    assert 0.5 < (gaps[2][0] * 72) / (gaps[0][0] * 32) < 1.5


def test_continuous_adjoint_without_chemotaxis():
    """chi = 0: the control cannot reach u, the adjoint v~ vanishes, and both
    gradients are exactly 2 alpha g."""
    w = W.plain64(16, 16, 12, sigma=2.0, Q=9, chi=0.0)
    w.alpha = 1e-2
    p = oracle.from_workload(w)
    g = w.random_control(4, 0.1)
    _, Ec = oracle.cadjoint(p, g)
    _, E, _ = oracle.adjoint(p, g)
    assert np.abs(Ec - 2 * w.alpha * g).max() == 0.0
    assert np.abs(E - 2 * w.alpha * g).max() <= 1e-15
