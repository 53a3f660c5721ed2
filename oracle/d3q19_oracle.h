/*
 * d3q19_oracle.h -- FP64 CPU oracle of the coupled MRT lattice Boltzmann
 * forward solve, its tangent-linear model and its exact discrete (AMRT)
 * adjoint for the two-species chemotaxis system on the three-dimensional
 * D3Q19 lattice (Sec. 3.1: the velocities and weights of the D3Q19 remark;
 * the paper states that the D2Q9 construction carries over to D3Q19).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, plain reference that the
 * CUDA path is checked against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library.
 *
 * Readings (the paper gives no D3Q19 moment matrix):
 *   M     the orthogonal polynomial basis of the D3Q19 moments in the order
 *         (rho, e, eps, j_x, q_x, j_y, q_y, j_z, q_z, 3p_xx, 3pi_xx, p_ww,
 *         pi_ww, p_xy, p_yz, p_xz, m_x, m_y, m_z):
 *           1, 19|e|^2 - 30, (21|e|^4 - 53|e|^2 + 24)/2, e_x, (5|e|^2 - 9) e_x,
 *           e_y, (5|e|^2 - 9) e_y, e_z, (5|e|^2 - 9) e_z, 3e_x^2 - |e|^2,
 *           (3|e|^2 - 5)(3e_x^2 - |e|^2), e_y^2 - e_z^2, (3|e|^2 - 5)(e_y^2 - e_z^2),
 *           e_x e_y, e_y e_z, e_x e_z, (e_y^2 - e_z^2) e_x, (e_z^2 - e_x^2) e_y,
 *           (e_x^2 - e_y^2) e_z.
 *   Pi    the K block (3 x 3, from D = d Cs^2 tau (K^-1 - I/2)) on the flux
 *         moments (j_x, j_y, j_z) and free rates on the others:
 *         s[0] rho, s[1] e, s[2] eps, s[3] q, s[4] p (3p_xx, p_ww, p_xy, p_yz, p_xz),
 *         s[5] pi (3pi_xx, pi_ww), s[6] m.
 *   the rest as in two dimensions (mrt_oracle.h): equilibrium (phieq) with
 *   T = a Theta and C = (a a) Theta, S_u from D_{u,1} = chi u I, grad v from
 *   v's first non-equilibrium moment, w~_i = w_i (1 + V.e_i / Cs^2) with
 *   V = (I - K_v/2) a, the (tau/2)(Phi^n - Phi^{n-1}) term.
 *
 * Model: du/dt = div(D_u grad u - chi u grad v) - div(a u),
 *        dv/dt = div(D_v grad v) - div(a v) + r_vu u + r_vv v + g,
 *        J = 1/2 sum (u^N - u_target)^2 + alpha sum_n sum_x g^2.
 *
 * Layouts (row-major, double): node fields [nz][ny][nx]; tensors
 * [nz][ny][nx][6] = (Dxx, Dxy, Dxz, Dyy, Dyz, Dzz); velocity [nz][ny][nx][3];
 * control and gradient [N][nz][ny][nx]; populations [nz][ny][nx][2][19].
 */
#ifndef D3Q19_ORACLE_H
#define D3Q19_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny, nz, N;
    double tau;
    const double* Du;    /* [nz][ny][nx][6] */
    const double* Dv;
    const double* a;     /* [nz][ny][nx][3] or NULL */
    const double* u0;    /* [nz][ny][nx] */
    const double* v0;
    const double* u_tgt;
    double d_u, d_v, chi, r_vu, r_vv, alpha;
    double s[7];
    int source_order;    /* 2: keep the (tau/2)(Phi^n - Phi^{n-1}) term; 1: drop it */
} od3_problem;

/* lattice tables: e [19][3] (ints), w [19], M [19][19] (rows = moments) */
int od3_lattice(int* e, double* w, double* M);
/* J (may be NULL), u^N and v^N [nz][ny][nx] (may be NULL) */
int od3_forward(const od3_problem* p, const double* g, double* J, double* uN, double* vN);
/* per step n: mass of u, mass of v (before collision) and the sum of Phi_v^n */
int od3_forward_trace(const od3_problem* p, const double* g, double* mass_u, double* mass_v, double* sum_phi);
/* tangent-linear model along dg ([N][...], may be NULL) and df0 ([nz][ny][nx][2][19], may be NULL) */
int od3_tlm(const od3_problem* p, const double* g, const double* dg, const double* df0, double* duN, double* dvN);
/* exact discrete adjoint: seeds [nz][ny][nx] of u^N, v^N (seed_u NULL: u^N - u_tgt with the penalty;
 * otherwise the gradient of sum(seed . (u^N, v^N)) + alpha ||g||^2); dJdg [N][...]; psi0 (may be NULL) */
int od3_adjoint(const od3_problem* p, const double* g, const double* seed_u, const double* seed_v, double* dJdg,
                double* psi0, double* J);
/* One collision at node (x, y, z), step n (f [2][Q] -> P [2][Q], Phi^n), for
 * unit tests; Phi_prev is Phi^{n-1} (ignored at n = 0). */
int od3_collide_node(const od3_problem* p, int x, int y, int z, int n, const double* f, double g,
                     double Phi_prev, double* P, double* Phi_out);
/* One node of the AMRT step, the transpose of od3_collide_node: from the
 * pulled adjoint populations rho [2][Q] (and, when has_next, sigma^{n+1} for
 * Phi^n's use at step n + 1) it returns psi [2][Q], sigma^n and lam_Phi, the
 * adjoint of Phi^n (dJ/dg^n without the penalty term). */
int od3_adjoint_node(const od3_problem* p, int x, int y, int z, int n, const double* f, double g,
                     const double* rho, int has_next, double sigma_next, double* psi, double* sigma_out,
                     double* lam_Phi);
int od3_set_threads(int n);

#ifdef __cplusplus
}
#endif

#endif
