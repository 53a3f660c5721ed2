/*
 * cx3d.h -- C ABI of the three-dimensional (D3Q19) solver of the two-species
 * chemotaxis control problem of cxlbm.h:
 *
 *     du/dt = div(D_u grad u - chi u grad v) - div(a u)
 *     dv/dt = div(D_v grad v) - div(a v) + r_vu u + r_vv v + g
 *     J     = 1/2 sum_x (u^N - u_target)^2 + alpha sum_{n<N} sum_x g^n(x)^2
 *
 * on a periodic nx x ny x nz lattice.  The scheme is the MRT / AMRT method of
 * Sec. 3.1 and 3.2.1 on the D3Q19 lattice of the Sec. 3.1 lattice remark
 * (velocities e_0..e_18 and weights 1/3, 1/18, 1/36 in the paper's order):
 * the paper gives no D3Q19 moment matrix, so the collision uses the
 * orthogonal polynomial basis (rho, e, eps, j, q, 3p_xx, 3pi_xx, p_ww, pi_ww,
 * p_xy, p_yz, p_xz, m) with the 3 x 3 block K (D = d Cs^2 tau (K^-1 - I/2))
 * on (j_x, j_y, j_z) and free rates s[0..6] = (rho, e, eps, q, p, pi, m) on
 * the others; equilibrium (phieq) with T = a Theta and C = (a a) Theta;
 * sources tau w~_i Phi_v + (tau/2) w~_i (Phi_v^n - Phi_v^{n-1}) with
 * w~_i = w_i (1 + V.e_i / Cs^2), V = (I - K_v/2) a; tau S_u,i =
 * (w_i / Cs^2) chi u e_i . K_u G, G = -(K_v (j_v - a v)/tau + K_v a Phi_v / 2)
 * / (d_v Cs^2).  The adjoint is the exact transpose of the discrete forward
 * step (streaming along -e_i backward in time, transposed collision,
 * adjoint-equilibrium broadcast, coupling terms) with dJ/dg assembled in the
 * same kernel.
 *
 * Conventions as in cxlbm.h: caller-owned device memory (one workspace), no
 * allocation by the library, calls ordered on the problem's stream.  T is
 * float (precision 32) or double (precision 64).  Node fields are
 * [nz][ny][nx]; control and gradient [n_steps][nz][ny][nx].
 */
#ifndef CX3D_H
#define CX3D_H

#include "cxlbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Tensors: CX_ANISO_CONST (D_u[6], D_v[6] = (Dxx, Dxy, Dxz, Dyy, Dyz, Dzz)) or
 * CX_ANISO_FIELD (device FP64 [nz][ny][nx][6] per species).  Convection:
 * CX_ADV_NONE, CX_ADV_ROW (a depends on y only: device FP64 [ny][3]) or
 * CX_ADV_FIELD (device FP64 [nz][ny][nx][3]). */
typedef struct {
    int nx, ny, nz;      /* periodic lattice, each >= 3                              */
    int n_steps;         /* N >= 1                                                   */
    int precision;       /* 32 or 64                                                 */
    int ckpt_every;      /* checkpoint interval k; 0 means N                         */
    double tau;          /* lattice time step (1)                                    */
    int aniso;           /* CX_ANISO_CONST or CX_ANISO_FIELD                         */
    double D_u[6], D_v[6];
    const double* D_u_field;
    const double* D_v_field;
    double d_u, d_v;     /* d of the equilibrium, > 0                                */
    double chi, r_vu, r_vv;
    int adv;             /* CX_ADV_*                                                 */
    const double* a;
    const double* u_target; /* device FP64 [nz][ny][nx]                              */
    double alpha;        /* >= 0                                                     */
    double s[7];         /* free rates in (0, 2)                                     */
    int source_order;    /* 2 or 1                                                   */
} cx3d_desc;

typedef struct cx3d_problem cx3d_problem;

/* Bytes of device workspace (host call).  Errors: CX_ERR_INVALID_ARG. */
cx_status cx3d_workspace_size(const cx3d_desc* desc, size_t* bytes);
/* Create a problem bound to a caller-owned workspace (256-byte aligned) and a
 * stream; converts the descriptor's fields into the workspace (K per node for
 * FIELD tensors, a, u_target) and synchronises once.  Every K must have its
 * eigenvalues in (0, 2).  Errors: CX_ERR_INVALID_ARG, CX_ERR_WORKSPACE,
 * CX_ERR_UNSTABLE, CX_ERR_CUDA. */
cx_status cx3d_create(const cx3d_desc* desc, void* workspace, size_t bytes, cudaStream_t stream,
                      cx3d_problem** out);
/* Initial populations phi^eq(u0), phi^eq(v0) (device FP64 [nz][ny][nx]). */
cx_status cx3d_set_initial(cx3d_problem* p, const double* u0, const double* v0);
/* Forward solve with control g (device T [N][nz][ny][nx] or NULL); checkpoints
 * every k steps and the last segment's tape (u, G per node and step); FP64
 * cost to J_dev (device double, may be NULL).  Errors: CX_ERR_STATE. */
cx_status cx3d_forward(cx3d_problem* p, const void* g, double* J_dev);
/* Exact discrete adjoint with fused gradient assembly at the control of the
 * preceding forward.  seed_u / seed_v (device T [nz][ny][nx]): both NULL uses
 * the cost's terminal term (u^N - u_target, 0); otherwise NULL is a zero seed.
 * penalty 0 leaves 2 alpha g out (the plain vector-Jacobian product).
 * Writes dJdg (device T [N][nz][ny][nx]).  Errors: CX_ERR_STATE, CX_ERR_INVALID_ARG. */
cx_status cx3d_adjoint(cx3d_problem* p, const void* g, const void* seed_u, const void* seed_v, int penalty,
                       void* dJdg);
/* cx3d_forward then cx3d_adjoint with NULL seeds. */
cx_status cx3d_gradient(cx3d_problem* p, const void* g, void* dJdg, double* J_dev);
/* One steepest-descent iteration with Armijo backtracking (as cx_step);
 * synchronises once per trial.  Errors: CX_ERR_LINESEARCH, CX_ERR_UNSTABLE. */
cx_status cx3d_step(cx3d_problem* p, void* g_inout, void* E_work, cx_step_info* info);
/* u^N and v^N of the last forward (device T [nz][ny][nx], either may be NULL). */
cx_status cx3d_get_fields(cx3d_problem* p, void* u_out, void* v_out);
/* J, ||dJ/dg||^2, max |dJ/dg| (host doubles, may be NULL); synchronises. */
cx_status cx3d_get_norms(cx3d_problem* p, double* J, double* grad_sq, double* grad_inf);
/* Per-phase device time (forward, recompute, adjoint) while timing is on. */
cx_status cx3d_set_timing(cx3d_problem* p, int enable);
cx_status cx3d_get_timing(cx3d_problem* p, double* ms, long long* launches);
cx_status cx3d_destroy(cx3d_problem* p);

#ifdef __cplusplus
}
#endif

#endif /* CX3D_H */
