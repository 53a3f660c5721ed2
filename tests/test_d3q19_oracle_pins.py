"""Pins of the D3Q19 oracle (the two-species method on the three-dimensional
lattice of the Sec. 3.1 lattice remark) against what the paper and the
mathematics fix: the printed velocities and weights, lattice isotropy, an
orthogonal moment basis whose flux rows carry the K block, the BGK special
case against an independent BGK loop, the closed-form anisotropic Gaussian at
second order, the centre of a convected reacting plume, exact mass balance,
the dot-product identity with the tangent-linear model, central differences,
and an independent pseudo-spectral solution of the coupled PDE."""
import json
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
CS2 = 1.0 / 3.0


def _golden():
    with open(os.path.join(HERE, "golden", "d3q19_lattice.json")) as fh:
        g = json.load(fh)
    return np.array(g["e"]), np.array(g["w_times_36"]) / 36.0


def _iso(nx, ny, nz, D):
    return np.broadcast_to(np.asarray(D, float), (nz, ny, nx, 6)).copy()


def _rot_tensor(l1, l2, l3, ax=0.3, ay=0.5):
    """A rotated constant 3x3 diffusion tensor as (Dxx, Dxy, Dxz, Dyy, Dyz, Dzz)."""
    cx, sx, cy, sy = np.cos(ax), np.sin(ax), np.cos(ay), np.sin(ay)
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    R = Ry @ Rx
    D = R @ np.diag([l1, l2, l3]) @ R.T
    return D, (D[0, 0], D[0, 1], D[0, 2], D[1, 1], D[1, 2], D[2, 2])


def test_lattice_matches_the_paper_and_is_isotropic():
    e, w, M = oracle.lattice3d()
    eg, wg = _golden()
    assert np.array_equal(e, eg) and np.allclose(w, wg, rtol=0, atol=1e-16)
    I = np.eye(3)
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", w, e), 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, e, e), CS2 * I, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, e, e, e), 0, atol=1e-16)
    iso4 = CS2 ** 2 * (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I) + np.einsum("ad,bc->abcd", I, I))
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e), iso4, atol=1e-16)
    # an orthogonal basis whose first row is the mass and whose flux rows are j_x, j_y, j_z
    G = M @ M.T
    assert np.abs(G - np.diag(np.diag(G))).max() == 0.0 and np.linalg.matrix_rank(M) == 19
    assert np.array_equal(M[0], np.ones(19))
    for r, c in zip((3, 5, 7), range(3)):
        assert np.array_equal(M[r], e[:, c])


def _bgk_reference(e, w, f0u, f0v, a, s, d, steps):
    """Independent D3Q19 BGK advection-diffusion loop (numpy, periodic
    streaming by np.roll) for the MRT special case K = s I, all rates s."""
    def feq(T):
        ea = np.einsum("ic,zyxc->izyx", e, a)
        a2 = np.einsum("zyxc,zyxc->zyx", a, a)
        e2 = (e ** 2).sum(1)[:, None, None, None]
        al = 1 + 3 * ea + 4.5 * (ea ** 2 - a2 / 3) + 1.5 * (d - 1) * (e2 - 1)
        return w[:, None, None, None] * al * T[None]
    fu, fv = f0u.copy(), f0v.copy()
    for n in range(steps):
        Pu = fu - s * (fu - feq(fu.sum(0)))
        Pv = fv - s * (fv - feq(fv.sum(0)))
        for i in range(19):
            fu[i] = np.roll(Pu[i], shift=(e[i, 2], e[i, 1], e[i, 0]), axis=(0, 1, 2))
            fv[i] = np.roll(Pv[i], shift=(e[i, 2], e[i, 1], e[i, 0]), axis=(0, 1, 2))
    return fu.sum(0), fv.sum(0)


def test_mrt_equals_bgk_special_case():
    """K = sI and every free rate s: the MRT collision is the BGK one; the
    oracle equals an independent BGK loop (convection on, chi = 0, no source)."""
    nx, ny, nz, N, s = 8, 6, 5, 7, 1.3
    eg, wg = _golden()
    rng = np.random.default_rng(0)
    u0 = 1 + 0.1 * rng.standard_normal((nz, ny, nx))
    v0 = 0.5 + 0.1 * rng.standard_normal((nz, ny, nx))
    a = np.broadcast_to(np.array([0.03, -0.02, 0.05]), (nz, ny, nx, 3)).copy()
    for d in (1.0, 0.8):
        Dval = d * CS2 * (1 / s - 0.5)  # K = s I
        p = oracle.Problem3D(nx=nx, ny=ny, nz=nz, N=N, Du=_iso(nx, ny, nz, (Dval, 0, 0, Dval, 0, Dval)),
                             Dv=_iso(nx, ny, nz, (Dval, 0, 0, Dval, 0, Dval)), u0=u0, v0=v0,
                             u_tgt=np.zeros((nz, ny, nx)), a=a, d_u=d, d_v=d, s=(s,) * 7)
        _, u, v = oracle.forward3d(p)
        # the initial populations of the oracle are phi^eq(Theta_0) (the equilibrium of the loop)
        def feq0(T):
            ea = np.einsum("ic,zyxc->izyx", eg, a)
            a2 = np.einsum("zyxc,zyxc->zyx", a, a)
            e2 = (eg ** 2).sum(1)[:, None, None, None]
            return wg[:, None, None, None] * (1 + 3 * ea + 4.5 * (ea ** 2 - a2 / 3) + 1.5 * (d - 1) * (e2 - 1)) * T[None]
        ur, vr = _bgk_reference(eg, wg, feq0(u0), feq0(v0), a, s, d, N)
        assert np.abs(u - ur).max() < 1e-14 and np.abs(v - vr).max() < 1e-14


def _gauss_periodic(n, c, Sigma, images=2):
    """Periodic sum of a normalised 3-D Gaussian of covariance Sigma centred at c."""
    idx = np.arange(n)
    X, Y, Z = np.meshgrid(idx, idx, idx, indexing="xy")
    P = np.linalg.inv(Sigma)
    out = np.zeros((n, n, n))
    for ix in range(-images, images + 1):
        for iy in range(-images, images + 1):
            for iz in range(-images, images + 1):
                d = np.stack([X - c[0] + ix * n, Y - c[1] + iy * n, Z - c[2] + iz * n], -1)
                out += np.exp(-0.5 * np.einsum("...a,ab,...b->...", d, P, d))
    return np.transpose(out, (2, 0, 1)) / np.sqrt((2 * np.pi) ** 3 * np.linalg.det(Sigma))


@pytest.mark.slow
def test_anisotropic_gaussian_closed_form_second_order():
    """chi = 0, a = 0, no reaction, a constant rotated D: a Gaussian of
    covariance S0 stays Gaussian with S(t) = S0 + 2 D t (mass kept); relative
    L2 error falls about 4x per diffusive refinement (h/2, 4x steps)."""
    Dm, D6 = _rot_tensor(0.08, 0.04, 0.02)
    errs = []
    for r in (2, 4):
        n, N, sig = 12 * r, 12 * r * r, 1.6 * r
        S0 = sig ** 2 * np.eye(3)
        c = np.array([n / 2, n / 2, n / 2])
        v0 = _gauss_periodic(n, c, S0)
        p = oracle.Problem3D(nx=n, ny=n, nz=n, N=N, Du=_iso(n, n, n, D6), Dv=_iso(n, n, n, D6),
                             u0=np.zeros((n, n, n)), v0=v0, u_tgt=np.zeros((n, n, n)))
        _, _, v = oracle.forward3d(p)
        exact = _gauss_periodic(n, c, S0 + 2 * Dm * N)
        assert abs(v.sum() - v0.sum()) < 1e-12 * v0.sum()
        errs.append(np.linalg.norm(v - exact) / np.linalg.norm(exact))
    print("3-D Gaussian errors", errs)
    assert errs[0] < 2e-2 and 3.0 < errs[0] / errs[1] < 5.0


def _plume_velocity_error(r, n=48, N=40, a=(0.04, -0.03, 0.02)):
    """Relative error of the centre-of-mass velocity of a v plume that reacts
    linearly (Phi_v = r v) against the convection velocity a, between N/2 and
    N steps (after the start-up transient).  The plume stays far from the
    periodic edges (6 standard deviations), so sum x v / sum v is its centre."""
    _, D6 = _rot_tensor(0.12, 0.05, 0.08)
    v0 = _gauss_periodic(n, np.array([24.0, 23.0, 24.5]), 2.0 ** 2 * np.eye(3), images=0)
    idx = np.arange(n, dtype=float)
    coords = (idx[None, None, :], idx[None, :, None], idx[:, None, None])
    cs = []
    for steps in (N // 2, N):
        p = oracle.Problem3D(nx=n, ny=n, nz=n, N=steps, Du=_iso(n, n, n, D6), Dv=_iso(n, n, n, D6),
                             u0=np.zeros((n, n, n)), v0=v0, u_tgt=np.zeros((n, n, n)),
                             a=np.broadcast_to(np.array(a), (n, n, n, 3)).copy(), r_vv=r)
        _, _, v = oracle.forward3d(p)
        cs.append(np.array([(v * C).sum() / v.sum() for C in coords]))
    w = (cs[1] - cs[0]) / (N - N // 2)
    return w / np.array(a) - 1.0


def test_plume_centre_moves_with_a():
    """Phi_v = r v, constant a, anisotropic K: the PDE moves the centre of v
    at exactly a for every r.  Without source the scheme does so exactly;
    with V = (I - K_v/2) a the velocity error is O(r^2) (ratio near 4 when r
    halves); a wrong V leaves an O(r) error."""
    e0 = _plume_velocity_error(0.0)
    e1 = _plume_velocity_error(0.05)
    e2 = _plume_velocity_error(0.025)
    print("plume velocity errors", e0, e1, e2, e1 / e2)
    assert np.abs(e0).max() < 1e-7  # periodic tails at the 1e-8 level
    assert np.abs(e1).max() < 5e-3
    assert np.all((e1 / e2 > 3.5) & (e1 / e2 < 4.5))


def test_mass_balance_with_sources_and_chemotaxis():
    """Streaming and collision conserve each species; the v source adds
    exactly tau sum (c_n Phi^n + c'_n Phi^{n-1}) per step; S_u adds no mass."""
    nx, ny, nz, N = 7, 6, 5, 9
    rng = np.random.default_rng(1)
    _, D6 = _rot_tensor(0.1, 0.05, 0.03)
    p = oracle.Problem3D(nx=nx, ny=ny, nz=nz, N=N, Du=_iso(nx, ny, nz, D6), Dv=_iso(nx, ny, nz, D6),
                         u0=1 + 0.1 * rng.standard_normal((nz, ny, nx)),
                         v0=0.5 + 0.1 * rng.standard_normal((nz, ny, nx)), u_tgt=np.zeros((nz, ny, nx)),
                         a=0.03 * rng.standard_normal((nz, ny, nx, 3)), chi=-0.2, r_vu=0.05, r_vv=-0.03)
    g = 0.02 * rng.standard_normal((N, nz, ny, nx))
    mu, mv, sp = oracle.forward3d_trace(p, g)
    assert np.abs(np.diff(mu)).max() < 1e-12 * mu[0]
    prev = np.concatenate([sp[:1], sp[:-1]])
    expect = sp + 0.5 * (sp - prev)
    assert np.allclose(np.diff(mv), expect[:-1], rtol=0, atol=1e-12 * mv[0])


def _problem(n=(6, 5, 4), N=6, seed=2, alpha=0.0):
    nx, ny, nz = n
    rng = np.random.default_rng(seed)
    _, Du = _rot_tensor(0.1, 0.05, 0.03)
    _, Dv = _rot_tensor(0.2, 0.1, 0.06, ax=-0.4, ay=0.9)
    return oracle.Problem3D(nx=nx, ny=ny, nz=nz, N=N, Du=_iso(nx, ny, nz, Du), Dv=_iso(nx, ny, nz, Dv),
                            u0=1 + 0.1 * rng.standard_normal((nz, ny, nx)),
                            v0=0.5 + 0.1 * rng.standard_normal((nz, ny, nx)),
                            u_tgt=1 + 0.05 * rng.standard_normal((nz, ny, nx)),
                            a=0.03 * rng.standard_normal((nz, ny, nx, 3)), chi=-0.3, r_vu=0.05, r_vv=-0.04,
                            alpha=alpha, s=(1.0, 1.1, 0.9, 1.2, 1.05, 0.95, 1.15))


def test_dot_product_identity():
    """<(wu, wv), TLM(dg, df0)> = <ADJ(wu, wv), (dg, df0)>: the adjoint is the
    exact transpose of the tangent-linear solve."""
    p = _problem()
    rng = np.random.default_rng(3)
    g = 0.05 * rng.standard_normal((p.N, p.nz, p.ny, p.nx))
    dg = rng.standard_normal(g.shape)
    df0 = rng.standard_normal((p.nz, p.ny, p.nx, 2, 19))
    wu, wv = rng.standard_normal((2, p.nz, p.ny, p.nx))
    du, dv = oracle.tlm3d(p, g, dg, df0)
    _, E, psi0 = oracle.adjoint3d(p, g, wu, wv, want_psi0=True)
    lhs = float(np.sum(wu * du) + np.sum(wv * dv))
    rhs = float(np.sum(E * dg) + np.sum(psi0 * df0))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs)), (lhs, rhs)


def test_gradient_against_finite_differences():
    p = _problem(alpha=1e-2)
    rng = np.random.default_rng(4)
    g = 0.05 * rng.standard_normal((p.N, p.nz, p.ny, p.nx))
    _, E, _ = oracle.adjoint3d(p, g)
    h = 1e-6
    for k in rng.choice(g.size, 16, replace=False):
        idx = np.unravel_index(k, g.shape)
        gp, gm = g.copy(), g.copy()
        gp[idx] += h
        gm[idx] -= h
        fd = (oracle.forward3d(p, gp)[0] - oracle.forward3d(p, gm)[0]) / (2 * h)
        assert abs(fd - E[idx]) <= 1e-6 * np.abs(E).max()


def _spectral3d(L, T, Du, Dv, chi, r_vu, r_vv, u0, v0, dt=0.05):
    """Pseudo-spectral RK4 solution of du/dt = div(Du grad u - chi u grad v),
    dv/dt = div(Dv grad v) + r_vu u + r_vv v on a periodic cube."""
    n = u0.shape[0]
    k = 2 * np.pi * np.fft.fftfreq(n, d=L / n)
    KZ, KY, KX = np.meshgrid(k, k, k, indexing="ij")
    Ks = (KX, KY, KZ)

    def d(f, K):
        return np.real(np.fft.ifftn(1j * K * np.fft.fftn(f)))

    def rhs(u, v):
        gu = [d(u, K) for K in Ks]
        gv = [d(v, K) for K in Ks]
        fu = [sum(Du[a, b] * gu[b] for b in range(3)) - chi * u * gv[a] for a in range(3)]
        fv = [sum(Dv[a, b] * gv[b] for b in range(3)) for a in range(3)]
        return (sum(d(fu[a], Ks[a]) for a in range(3)),
                sum(d(fv[a], Ks[a]) for a in range(3)) + r_vu * u + r_vv * v)

    s = (u0.copy(), v0.copy())
    for _ in range(int(round(T / dt))):
        k1 = rhs(*s)
        k2 = rhs(*(a + dt / 2 * b for a, b in zip(s, k1)))
        k3 = rhs(*(a + dt / 2 * b for a, b in zip(s, k2)))
        k4 = rhs(*(a + dt * b for a, b in zip(s, k3)))
        s = tuple(a + dt / 6 * (b1 + 2 * b2 + 2 * b3 + b4) for a, b1, b2, b3, b4 in zip(s, k1, k2, k3, k4))
    return s


@pytest.mark.slow
def test_chemotaxis_coupling_against_pde():
    """The coupled D3Q19 scheme (anisotropic tensors, chemotaxis, linear
    reaction) converges at second order to an independent pseudo-spectral
    solution of the PDE under diffusive refinement."""
    L, T = 12, 6
    Dum, Du6 = _rot_tensor(0.1, 0.05, 0.03)
    Dvm, Dv6 = _rot_tensor(0.2, 0.1, 0.06, ax=-0.4, ay=0.9)
    chi, r_vu, r_vv = -0.2, 0.02, -0.03

    def init(n):
        x = np.arange(n) * L / n
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        k = 2 * np.pi / L
        return (1 + 0.2 * np.cos(k * X) * np.sin(k * Y + 0.3) * np.cos(k * Z),
                0.5 + 0.1 * np.sin(k * (X + Y + Z)))

    ref = _spectral3d(L, T, Dum, Dvm, chi, r_vu, r_vv, *init(L))
    errs = []
    for r in (1, 2):
        n, N = L * r, T * r * r
        u0, v0 = init(n)
        p = oracle.Problem3D(nx=n, ny=n, nz=n, N=N, Du=_iso(n, n, n, Du6), Dv=_iso(n, n, n, Dv6), u0=u0, v0=v0,
                             u_tgt=np.zeros((n, n, n)), chi=chi, r_vu=r_vu / r ** 2, r_vv=r_vv / r ** 2)
        _, u, v = oracle.forward3d(p)
        errs.append([np.linalg.norm(u[::r, ::r, ::r] - ref[0]) / np.linalg.norm(ref[0] - ref[0].mean()),
                     np.linalg.norm(v[::r, ::r, ::r] - ref[1]) / np.linalg.norm(ref[1] - ref[1].mean())])
    print("D3Q19 vs pseudo-spectral", errs)
    for c in range(2):
        assert 3.3 < errs[0][c] / errs[1][c] < 4.7, errs


@pytest.mark.parametrize("n", [0, 3])
def test_local_adjoint_is_the_transposed_local_jacobian(n):
    """One node of the D3Q19 AMRT step against the dense Jacobian of one
    collision at that node by central differences (38 populations, the
    control and Phi^{n-1}).  With L = rho.P + lam Phi^n (lam = c'_{n+1}
    sigma^{n+1}): psi = dL/df, lambda_Phi = dL/dg and c'_n sigma^n =
    dL/dPhi^{n-1}.  The map is at most quadratic (chemotaxis u G), so central
    differences are exact up to rounding."""
    p = _problem()
    _, wts, _ = oracle.lattice3d()
    rng = np.random.default_rng(50 + n)
    tau = 1.0
    c_prev_n = 0.0 if n == 0 else -0.5 * tau
    h = 1e-6
    for _ in range(2):
        x, y, z = int(rng.integers(0, 6)), int(rng.integers(0, 5)), int(rng.integers(0, 4))
        f = np.stack([wts * rng.uniform(0.8, 1.2), wts * rng.uniform(0.3, 0.6)]) + rng.normal(0, 0.005, (2, 19))
        g, pp = rng.normal(0, 0.05), rng.normal(0, 0.05)
        rho, sig_next = rng.normal(size=(2, 19)), rng.normal()
        lam_next = -0.5 * tau * sig_next

        def L(f_, g_, pp_):
            P, phi = oracle.collide3d_node(p, x, y, z, n, f_, g_, pp_)
            return float(np.sum(rho * P) + lam_next * phi)

        dfd = np.zeros((2, 19))
        for s in range(2):
            for i in range(19):
                d = np.zeros((2, 19))
                d[s, i] = h
                dfd[s, i] = (L(f + d, g, pp) - L(f - d, g, pp)) / (2 * h)
        dg = (L(f, g + h, pp) - L(f, g - h, pp)) / (2 * h)
        dpp = (L(f, g, pp + h) - L(f, g, pp - h)) / (2 * h)

        psi, sigma, lam_phi = oracle.adjoint3d_node(p, x, y, z, n, f, rho, g=g, sigma_next=sig_next)
        scale = max(np.abs(dfd).max(), 1.0)
        assert np.allclose(psi, dfd, rtol=0, atol=1e-8 * scale)
        assert abs(lam_phi - dg) < 1e-8 * scale
        assert abs(c_prev_n * sigma - dpp) < 1e-8 * scale
