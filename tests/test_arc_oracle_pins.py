"""Pins of the three-species oracle (the attraction-repulsion chemotaxis model
with a logistic source, the ARC example of the paper's Sec. 2.2) against what
the mathematics fixes: the pinned two-species oracle as a special case, the
v <-> w symmetry, the closed-form logistic ODE, exact mass balances of the
nonlinear kinetics, an independent pseudo-spectral PDE solution, the
tangent/adjoint dot-product identity and central finite differences."""
import numpy as np
import pytest

import oracle
from paper_1908_03876_gb300.workloads import rotated_tensor

CS2 = 1.0 / 3.0


def _fields(n, seed):
    rng = np.random.default_rng(seed)
    x = np.arange(n)[None, :]
    y = np.arange(n)[:, None]
    k = 2 * np.pi / n
    u0 = 1.0 + 0.2 * np.cos(k * x + rng.uniform(0, 6)) * np.sin(k * y + rng.uniform(0, 6))
    v0 = 0.5 + 0.1 * np.sin(k * (x + y) + rng.uniform(0, 6)) * np.ones((n, n))
    w0 = 0.4 + 0.1 * np.cos(2 * k * x + rng.uniform(0, 6)) * np.ones((n, n))
    return u0, v0, w0


def _arc(n=10, N=8, seed=0, adv=True, **kw):
    u0, v0, w0 = _fields(n, seed)
    Du = np.broadcast_to(rotated_tensor((0.08, 0.02), np.array(0.6)), (n, n, 3)).copy()
    Dv = np.broadcast_to(rotated_tensor((0.2, 0.1), np.array(-0.3)), (n, n, 3)).copy()
    Dw = np.broadcast_to(rotated_tensor((0.15, 0.05), np.array(1.1)), (n, n, 3)).copy()
    a = None
    if adv:
        y = np.arange(n)[:, None] * np.ones((1, n))
        a = np.stack([0.04 * np.sin(2 * np.pi * y / n), np.zeros((n, n))], -1)
    par = dict(chi1=-0.1, chi2=0.08, a1=0.05, a2=0.03, b1=0.04, b2=0.02, b3=0.01, c1=0.03, c2=0.05,
               ctrl_species=2, alpha=1e-2)
    par.update(kw)
    return oracle.Problem3(nx=n, ny=n, N=N, Du=Du, Dv=Dv, Dw=Dw, u0=u0, v0=v0, w0=w0,
                           u_tgt=np.ones((n, n)), a=a, **par)


def test_reduces_to_the_two_species_model():
    """w = 0 throughout (w0 = 0, no w kinetics, chi2 = 0), no logistic term,
    linear v kinetics and the control on v: the three-species solve is the
    pinned two-species solve (fields, J and every gradient component)."""
    p3 = _arc(n=12, N=9, a1=0.0, a2=0.0, b3=0.0, c1=0.0, c2=0.0, chi2=0.0, ctrl_species=1)
    p3.w0 = np.zeros((12, 12))
    p2 = oracle.Problem(nx=12, ny=12, N=9, Q=9, Du=p3.Du, Dv=p3.Dv, u0=p3.u0, v0=p3.v0, u_tgt=p3.u_tgt,
                        chi=p3.chi1, r_vu=p3.b1, r_vv=-p3.b2, a=p3.a, alpha=p3.alpha)
    g = 0.05 * np.random.default_rng(1).standard_normal((9, 12, 12))
    J3, uvw = oracle.forward3(p3, g)
    J2, u2, v2 = oracle.forward(p2, g)
    assert np.abs(uvw[2]).max() == 0.0
    assert np.allclose(uvw[0], u2, rtol=1e-13, atol=0) and np.allclose(uvw[1], v2, rtol=1e-13, atol=0)
    assert abs(J3 - J2) <= 1e-13 * abs(J2)
    _, E3, _ = oracle.adjoint3(p3, g)
    _, E2, _ = oracle.adjoint(p2, g)
    assert np.abs(E3 - E2).max() <= 1e-12 * np.abs(E2).max()


def test_v_w_symmetry():
    """Exchanging the two chemicals (fields, tensors, kinetics, sensitivities
    and the controlled species) leaves u and J unchanged."""
    p = _arc(n=10, N=7, b3=0.0)
    q = _arc(n=10, N=7, b3=0.0)
    q.Dv, q.Dw, q.v0, q.w0 = p.Dw, p.Dv, p.w0, p.v0
    q.chi1, q.chi2 = p.chi2, p.chi1
    q.b1, q.b2, q.c1, q.c2 = p.c1, p.c2, p.b1, p.b2
    q.ctrl_species = 1
    g = 0.05 * np.random.default_rng(2).standard_normal((7, 10, 10))
    Jp, up = oracle.forward3(p, g)
    Jq, uq = oracle.forward3(q, g)
    assert np.allclose(up[0], uq[0], rtol=1e-13, atol=0)
    assert np.allclose(up[1], uq[2], rtol=1e-13, atol=0) and np.allclose(up[2], uq[1], rtol=1e-13, atol=0)
    assert abs(Jp - Jq) <= 1e-13 * abs(Jp)


def test_logistic_source_closed_form():
    """Uniform u and no chemicals: du/dt = r u (1 - u / K), solved exactly by
    u(t) = K u0 e^{rt} / (K + u0 (e^{rt} - 1)).  The source term with its
    (tau/2)(Phi^n - Phi^{n-1}) correction is a second-order time integrator:
    with the rate divided by 4 and the steps multiplied by 4 (same r t) the
    error falls 16x."""
    n, r, K, u00 = 4, 0.08, 2.0, 0.2
    errs = []
    for k in range(3):
        N = 40 * 4 ** k
        p = _arc(n=n, N=N, adv=False, chi1=0.0, chi2=0.0, a1=r / 4 ** k, a2=r / 4 ** k / K, b1=0.0, b2=0.0, b3=0.0,
                 c1=0.0, c2=0.0)
        p.u0 = np.full((n, n), u00)
        p.v0 = np.zeros((n, n))
        p.w0 = np.zeros((n, n))
        _, uvw = oracle.forward3(p)
        T = 40 * r  # r t is the same at every refinement
        exact = K * u00 * np.exp(T) / (K + u00 * (np.exp(T) - 1))
        assert np.ptp(uvw[0]) < 1e-14
        errs.append(abs(uvw[0, 0, 0] - exact) / exact)
    print("logistic errors", errs)
    assert errs[0] < 1e-3
    assert 14 < errs[0] / errs[1] < 18 and 14 < errs[1] / errs[2] < 18


def test_nonlinear_kinetics_mass_balance():
    """Streaming and collision conserve each species; the sources add exactly
    sum (c_n Phi^n + c'_n Phi^{n-1}) per step (Phi^{-1} := Phi^0), with the
    nonlinear kinetics of all three species and both chemotactic fluxes."""
    p = _arc(n=12, N=10)
    g = 0.03 * np.random.default_rng(3).standard_normal((10, 12, 12))
    mass, sphi = oracle.forward3_trace(p, g)
    prev = np.vstack([sphi[:1], sphi[:-1]])
    expect = sphi + 0.5 * (sphi - prev)
    dm = np.diff(mass, axis=0)
    assert np.allclose(dm, expect[:-1], rtol=0, atol=1e-12 * np.abs(mass).max())


def test_dot_product_identity_three_species():
    """<seeds, TLM(dg, df0)> = <ADJ(seeds), (dg, df0)>: the three-species
    adjoint is the exact transpose of the tangent-linear solve."""
    n, N = 10, 8
    p = _arc(n=n, N=N, alpha=0.0)
    rng = np.random.default_rng(4)
    g = 0.05 * rng.standard_normal((N, n, n))
    dg = rng.standard_normal((N, n, n))
    df0 = rng.standard_normal((n, n, 3, 9))
    seeds = rng.standard_normal((3, n, n))
    _, d = oracle.tlm3(p, g, dg, df0)
    _, E, psi0 = oracle.adjoint3(p, g, seeds, want_psi0=True)
    lhs = float(np.sum(seeds * d))
    rhs = float(np.sum(E * dg) + np.sum(psi0 * df0))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs)), (lhs, rhs)


@pytest.mark.parametrize("ctrl", [1, 2])
def test_gradient_fd_three_species(ctrl):
    """Sampled components of dJ/dg against central finite differences."""
    p = _arc(n=8, N=8, ctrl_species=ctrl)
    g = 0.05 * np.random.default_rng(5).standard_normal((8, 8, 8))
    _, E, _ = oracle.adjoint3(p, g)
    h = 1e-6
    rng = np.random.default_rng(6)
    for k in rng.choice(g.size, 20, replace=False):
        idx = np.unravel_index(k, g.shape)
        gp, gm = g.copy(), g.copy()
        gp[idx] += h
        gm[idx] -= h
        fd = (oracle.forward3(p, gp)[0] - oracle.forward3(p, gm)[0]) / (2 * h)
        assert abs(fd - E[idx]) <= 1e-6 * np.abs(E).max()


def _spectral_arc(L, T, D, par, a0, u0, v0, w0, dt=0.02):
    """Pseudo-spectral RK4 solution of the ARC system with shear convection
    a = (a0 sin(2 pi y / L), 0) on a periodic square."""
    n = u0.shape[0]
    k = 2 * np.pi * np.fft.fftfreq(n, d=L / n)
    KX, KY = np.meshgrid(k, k)
    y = np.arange(n)[:, None] * L / n
    ax = a0 * np.sin(2 * np.pi * y / L) * np.ones((1, n))

    def d(f, K):
        return np.real(np.fft.ifft2(1j * K * np.fft.fft2(f)))

    def div_flux(Dt, f, extra_x=0.0, extra_y=0.0):
        fx, fy = d(f, KX), d(f, KY)
        return d(Dt[0] * fx + Dt[1] * fy - ax * f + extra_x, KX) + d(Dt[1] * fx + Dt[2] * fy + extra_y, KY)

    def rhs(u, v, w):
        vx, vy, wx, wy = d(v, KX), d(v, KY), d(w, KX), d(w, KY)
        cx = -par["chi1"] * u * vx - par["chi2"] * u * wx
        cy = -par["chi1"] * u * vy - par["chi2"] * u * wy
        du = div_flux(D[0], u, cx, cy) + par["a1"] * u - par["a2"] * u * u
        dv = div_flux(D[1], v) + par["b1"] * u - par["b2"] * v - par["b3"] * u * v
        dw = div_flux(D[2], w) + par["c1"] * u - par["c2"] * w
        return du, dv, dw

    s = (u0.copy(), v0.copy(), w0.copy())
    for _ in range(int(round(T / dt))):
        k1 = rhs(*s)
        k2 = rhs(*(a + dt / 2 * b for a, b in zip(s, k1)))
        k3 = rhs(*(a + dt / 2 * b for a, b in zip(s, k2)))
        k4 = rhs(*(a + dt * b for a, b in zip(s, k3)))
        s = tuple(a + dt / 6 * (b1 + 2 * b2 + 2 * b3 + b4) for a, b1, b2, b3, b4 in zip(s, k1, k2, k3, k4))
    return s


@pytest.mark.slow
def test_arc_system_against_pde():
    """The three-species scheme converges at second order to an independent
    pseudo-spectral solution of the ARC PDE system (attraction toward v,
    repulsion from w, logistic growth, nonlinear v kinetics, shear
    convection) under diffusive refinement."""
    L, T, a0 = 32, 16, 0.08
    D = [rotated_tensor((0.08, 0.02), np.array(0.6)), rotated_tensor((0.2, 0.1), np.array(-0.3)),
         rotated_tensor((0.15, 0.05), np.array(1.1))]
    par = dict(chi1=-0.1, chi2=0.08, a1=0.02, a2=0.01, b1=0.03, b2=0.02, b3=0.01, c1=0.02, c2=0.03)

    def init(n):
        x = np.arange(n)[None, :] * L / n
        y = np.arange(n)[:, None] * L / n
        k = 2 * np.pi / L
        return (1 + 0.2 * np.cos(k * x) * np.sin(k * y), 0.5 + 0.1 * np.sin(k * (x + y)) * np.ones_like(x),
                0.4 + 0.1 * np.cos(2 * k * x) * np.ones_like(y))

    ref = _spectral_arc(L, T, D, par, a0, *init(L))
    errs = []
    for r in (1, 2, 4):
        n, N = L * r, T * r * r
        u0, v0, w0 = init(n)
        y = np.arange(n)[:, None] / r * np.ones((1, n))
        a = np.stack([(a0 / r) * np.sin(2 * np.pi * y / L), np.zeros((n, n))], -1)
        sc = {k: (v / r ** 2 if k not in ("chi1", "chi2") else v) for k, v in par.items()}
        p = oracle.Problem3(nx=n, ny=n, N=N, Du=np.broadcast_to(D[0], (n, n, 3)).copy(),
                            Dv=np.broadcast_to(D[1], (n, n, 3)).copy(), Dw=np.broadcast_to(D[2], (n, n, 3)).copy(),
                            u0=u0, v0=v0, w0=w0, u_tgt=np.zeros((n, n)), a=a, **sc)
        _, uvw = oracle.forward3(p)
        errs.append([np.linalg.norm(uvw[c][::r, ::r] - ref[c]) / np.linalg.norm(ref[c] - ref[c].mean())
                     for c in range(3)])
    print("ARC vs pseudo-spectral", errs)
    for c in range(3):
        r1, r2 = errs[0][c] / errs[1][c], errs[1][c] / errs[2][c]
        assert 3.5 < r1 < 4.6 and 3.5 < r2 < 4.6, errs


@pytest.mark.parametrize("n,ctrl", [(0, 1), (4, 2)])
def test_local_adjoint_is_the_transposed_local_jacobian(n, ctrl):
    """One node of the three-species AMRT step against the dense Jacobian of
    one collision at that node by central differences (27 populations, the
    control and the three Phi^{n-1}).  With L = rho.P + sum_s lam_s Phi_s^n
    (lam_s = c'_{n+1} sigma_s^{n+1}): psi = dL/df, lambda_Phi of the
    controlled species = dL/dg and c'_n sigma_s^n = dL/dPhi_s^{n-1}.  The maps
    are at most quadratic (chemotaxis u G, logistic u^2, consumption u v), so
    central differences are exact up to rounding."""
    p = _arc(n=8, N=6, seed=3, ctrl_species=ctrl)
    e, _, _, _ = oracle.lattice(9)
    rng = np.random.default_rng(40 + n)
    tau = p.tau
    c_prev_n = 0.0 if n == 0 else -0.5 * tau
    h = 1e-6
    for _ in range(2):
        x, y = (int(v) for v in rng.integers(0, 8, 2))
        a = p.a[y, x]
        f = np.stack([oracle.feq(9, rng.uniform(lo, hi), a, p.d) for lo, hi in ((0.8, 1.2), (0.3, 0.6), (0.2, 0.5))])
        f = f + rng.normal(0, 0.01, (3, 9))
        g, pp = rng.normal(0, 0.05), rng.normal(0, 0.05, 3)
        rho, sig_next = rng.normal(size=(3, 9)), rng.normal(size=3)
        lam_next = -0.5 * tau * sig_next

        def L(f_, g_, pp_):
            P, phi = oracle.collide3_node(p, x, y, n, f_, g_, pp_)
            return float(np.sum(rho * P) + lam_next @ phi)

        dfd = np.zeros((3, 9))
        for s in range(3):
            for i in range(9):
                d = np.zeros((3, 9))
                d[s, i] = h
                dfd[s, i] = (L(f + d, g, pp) - L(f - d, g, pp)) / (2 * h)
        dg = (L(f, g + h, pp) - L(f, g - h, pp)) / (2 * h)
        dpp = np.array([(L(f, g, pp + h * np.eye(3)[s]) - L(f, g, pp - h * np.eye(3)[s])) / (2 * h) for s in range(3)])

        psi, sigma, lam_phi = oracle.adjoint3_node(p, x, y, n, f, rho, g=g, sigma_next=sig_next)
        scale = max(np.abs(dfd).max(), 1.0)
        assert np.allclose(psi, dfd, rtol=0, atol=1e-8 * scale)
        assert abs(lam_phi[ctrl] - dg) < 1e-8 * scale
        assert np.allclose(c_prev_n * sigma, dpp, rtol=0, atol=1e-8 * scale)
