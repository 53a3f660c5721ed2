/*
 * mrt_oracle.h -- FP64 CPU oracle for the coupled MRT lattice Boltzmann
 * forward solve, its tangent-linear (sensitivity) model and its AMRT adjoint,
 * for the two-species chemotaxis system (u = cells, v = chemical, g = control
 * acting on v).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, plain reference that the
 * CUDA path is checked against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library.
 *
 * Every function follows the paper (Belmiloudi, "Optimal control for
 * chemotaxis systems and adjoint-based optimization with multiple-relaxation-
 * time lattice Boltzmann models"):
 *   - forward step:     eq. (LBE)/(LBEG) with (S), (PhiS), (phieq), M0, Pi (Sec. 3.1)
 *   - sensitivity step: eq. (LIBEG-V) (Sec. 3.2), the tangent of the forward step
 *   - adjoint step:     AMRT, eqs. (CAE), (AEDs), (AEDsM), (CAEL) (Sec. 3.2.1):
 *                       streaming along -e_i backward in time, collision with
 *                       the transposed operator, adjoint equilibrium as the
 *                       scalar broadcast T = sum_j w_j aleph_j m~_j, plus the
 *                       coupling terms dR/dphi and the gradient (gradientLattice).
 *
 * Array layouts (all row-major, all double unless noted):
 *   node fields          [ny][nx]
 *   tensor fields D      [ny][nx][3]  (Dxx, Dxy, Dyy)
 *   vector field a       [ny][nx][2]
 *   control g, dJ/dg     [N][cny][cnx]  (window x in [cx0,cx0+cnx), y in [cy0,cy0+cny))
 *   populations (psi0)   [ny][nx][2][Q]  (species 0 = u, 1 = v)
 */
#ifndef MRT_ORACLE_H
#define MRT_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny, N, Q;            /* grid, time steps, lattice (5 or 9) */
    double tau;                  /* lattice time step (h = tau = c = 1 in every test) */
    const double* Du;            /* [ny][nx][3] self-diffusion tensor of u */
    const double* Dv;            /* [ny][nx][3] self-diffusion tensor of v */
    double d_u, d_v;             /* d_Theta of the equilibrium (phieq) */
    double chi;                  /* chemotactic sensitivity: D_{u,1} = chi u I */
    double r_vu, r_vv;           /* Phi_v = r_vu u + r_vv v + g,  Phi_u = 0 */
    const double* a;             /* [ny][nx][2] convection velocity (T_Theta = a Theta) or NULL */
    const unsigned char* solid;  /* [ny][nx] 1 = solid node, or NULL (all fluid, periodic) */
    int cx0, cy0, cnx, cny;      /* control window */
    const unsigned char* cmask;  /* [cny][cnx] 1 = controlled node, or NULL (whole window) */
    const double* u_tgt;         /* [ny][nx] target u(T) */
    double alpha;                /* control penalty weight */
    double s[7];                 /* free relaxation rates s0..s6 of Pi */
    int source_order;            /* 2: keep (tau/2)(Phi^n - Phi^{n-1}); 1: drop it */
    const double* u0;            /* [ny][nx] initial u */
    const double* v0;            /* [ny][nx] initial v */
} or_problem;

/* Threads of the per-node loops (OpenMP builds; n <= 0 leaves the count as it
 * is).  Returns the count now in use (1 without OpenMP).  Results do not
 * depend on it. */
int or_set_threads(int n);

/* Lattice tables for unit tests: e [Q][2], w [Q], M [Q][Q], Minv [Q][Q]. */
int or_lattice(int Q, int* e, double* w, double* M, double* Minv);

/* Equilibrium populations (phieq) at one node: out[Q]. */
int or_feq(int Q, double Theta, const double a[2], double d, double* out);

/* One forward collision at one node (pre-collision f -> post-collision P),
 * exposing the local map for unit tests.  f_u, f_v, P_u, P_v are [Q]. */
int or_collide_node(const or_problem* p, int x, int y, int n,
                    const double* f_u, const double* f_v, double g, double Phi_prev,
                    double* P_u, double* P_v, double* Phi_out);

/* One node of the AMRT adjoint step at step n, exposing the local transposed
 * map for unit tests: given the node's pre-collision populations f_u, f_v and
 * control g at step n, and the pulled adjoint populations rho_u, rho_v, it
 * returns psi_u, psi_v (the node's adjoint populations psi^n), sigma^n =
 * sum_i rho_v,i w~_i and lam_Phi, the adjoint of Phi^n (dJ/dg^n without the
 * penalty term).  has_next: Phi^n is also used at step n + 1, whose
 * sigma^{n+1} is sigma_next.  All arrays are [Q]. */
int or_adjoint_node(const or_problem* p, int x, int y, int n, const double* f_u, const double* f_v, double g,
                    const double* rho_u, const double* rho_v, int has_next, double sigma_next, double* psi_u,
                    double* psi_v, double* sigma_out, double* lam_Phi);

/* Forward solve; uN, vN may be NULL.  Returns 0 on success. */
int or_forward(const or_problem* p, const double* g, double* J, double* uN, double* vN);

/* Forward solve that also returns, per step, the v-mass before collision and
 * Phi^n summed over fluid nodes ([N] each); used by the mass-balance pin. */
int or_forward_trace(const or_problem* p, const double* g, double* mass_u, double* mass_v,
                     double* sum_phi);

/* Tangent-linear model: perturbation dg of g and df0 ([ny][nx][2][Q], may be
 * NULL) of the initial populations.  Outputs duN, dvN ([ny][nx]) and the
 * directional derivative dJ of J. */
int or_tlm(const or_problem* p, const double* g, const double* dg, const double* df0,
           double* duN, double* dvN, double* dJ);

/* AMRT adjoint sweep and gradient.  seed_u / seed_v: adjoint of u^N / v^N
 * ([ny][nx]); seed_u == NULL means u^N - u_tgt (the cost's terminal term),
 * seed_v == NULL means 0.  With explicit seeds the gradient returned is that
 * of sum(seed_u*u^N + seed_v*v^N) + alpha*||g||^2.
 * Outputs dJdg [N][cny][cnx], psi0 [ny][nx][2][Q] (may be NULL), J (may be NULL). */
int or_adjoint(const or_problem* p, const double* g, const double* seed_u,
               const double* seed_v, double* dJdg, double* psi0, double* J);

/* Continuous-adjoint gradient (the algorithm of Sec. 3.2.1 that solves the
 * adjoint PDE system (FVM-PF-Adj) by the same MRT scheme with time reversed).
 * For Phi_u = 0, Phi_v = r_vu u + r_vv v + g, J = 1/2 |u(T) - u_tgt|^2 +
 * alpha int g^2, and s = T - t, the system reads
 *   du~/ds = div(D_u grad u~) + a.grad u~ + chi grad v . grad u~ + r_vu v~
 *   dv~/ds = div(D_v grad v~) + a.grad v~ + r_vv v~ - div(chi u grad u~)
 *   u~(s=0) = u^N - u_tgt,  v~(s=0) = 0,   dJ/dg = 2 alpha g + v~.
 * Output dJdg [N][cny][cnx] with dJ/dg^n = 2 alpha g^n + v~(t_{n+1}); J (may be
 * NULL). */
int or_cadjoint(const or_problem* p, const double* g, double* dJdg, double* J);

/* ---- three species: the attraction-repulsion chemotaxis model with a logistic
 * source (the ARC example of Sec. 2.2 of the paper, a case of its
 * three-equation system), D2Q9, periodic grid, control on the whole grid:
 *   du/dt = div(D_u grad u) - div(a u) - div(chi1 u grad v) - div(chi2 u grad w) + a1 u - a2 u^2
 *   dv/dt = div(D_v grad v) - div(a v) + b1 u - b2 v - b3 u v   (+ g if ctrl_species == 1)
 *   dw/dt = div(D_w grad w) - div(a w) + c1 u - c2 w            (+ g if ctrl_species == 2)
 *   J = 1/2 sum (u^N - u_tgt)^2 + alpha sum_{n<N} sum g^2.
 * Populations [ny][nx][3][Q]; fields [3][ny][nx] (u, v, w); controls [N][ny][nx]. */
typedef struct {
    int nx, ny, N;
    double tau;
    const double* Du;            /* [ny][nx][3] */
    const double* Dv;
    const double* Dw;
    double d;                    /* d_Theta of the equilibrium, all species */
    const double* a;             /* [ny][nx][2] or NULL */
    double chi1, chi2;           /* D_{u,1} = chi1 u I (toward v), D_{u,2} = chi2 u I (toward w) */
    double a1, a2;               /* logistic source of u */
    double b1, b2, b3;           /* kinetics of v */
    double c1, c2;               /* kinetics of w */
    int ctrl_species;            /* 1: g acts on v, 2: g acts on w */
    const double* u_tgt;
    double alpha;
    double s[7];
    int source_order;
    const double* u0;
    const double* v0;
    const double* w0;
} or3_problem;

int or3_forward(const or3_problem* p, const double* g, double* J, double* uvwN);
/* per step n: [n][6] = mass of u, v, w before collision, sum of Phi_u, Phi_v, Phi_w */
int or3_forward_trace(const or3_problem* p, const double* g, double* trace);
int or3_tlm(const or3_problem* p, const double* g, const double* dg, const double* df0, double* duvwN, double* dJ);
int or3_adjoint(const or3_problem* p, const double* g, const double* seeds, double* dJdg, double* psi0, double* J);
/* One collision of the three species at one node (pre-collision f [3][Q] ->
 * post-collision P [3][Q], Phi^n [3]), for unit tests; Phi_prev [3] is
 * Phi^{n-1} (ignored at n = 0). */
int or3_collide_node(const or3_problem* p, int x, int y, int n, const double* f, double g, const double* Phi_prev,
                     double* P, double* Phi_out);
/* One node of the three-species AMRT step, the transpose of or3_collide_node:
 * from the pulled adjoint populations rho [3][Q] (and, when has_next, the
 * species' sigma^{n+1} [3] for Phi^n's use at step n + 1) it returns psi
 * [3][Q], sigma^n [3] and lam_Phi [3], the adjoint of each species' Phi^n
 * (lam_Phi of the controlled species is dJ/dg^n without the penalty). */
int or3_adjoint_node(const or3_problem* p, int x, int y, int n, const double* f, double g, const double* rho,
                     int has_next, const double* sigma_next, double* psi, double* sigma_out, double* lam_Phi);

#ifdef __cplusplus
}
#endif
#endif
