/*
 * cxarc.h -- C ABI of the three-species solver: the attraction-repulsion
 * chemotaxis model with a logistic source (the ARC example of Sec. 2.2, a
 * case of the paper's three-equation system eq. ReacDiff):
 *
 *     du/dt = div(D_u grad u - chi1 u grad v - chi2 u grad w) - div(a u) + a1 u - a2 u^2
 *     dv/dt = div(D_v grad v) - div(a v) + b1 u - b2 v - b3 u v  [+ g]
 *     dw/dt = div(D_w grad w) - div(a w) + c1 u - c2 w           [+ g]
 *
 * with the distributed control g acting on v (ctrl_species = 1) or on w
 * (ctrl_species = 2).  The cell flux holds + chi1 u grad v + chi2 u grad w, so
 * chi1 > 0 attracts the cells toward v and chi2 < 0 repels them from w.
 *
 * Discrete problem (Sec. 3.1 and 3.2), the two-species scheme of cxlbm.h
 * widened to three species on D2Q9:
 *   forward   per species MRT collision with M0 and the block relaxation
 *             matrix Pi (K from D = d C_s^2 tau (K^-1 - I/2)); sources
 *             tau w~_i Phi + (tau/2) w~_i (Phi^n - Phi^{n-1}) for every species
 *             (eq. PhiS, w~_i = w_i (1 + V.e_i / C_s^2), V = (I - K/2) a); the
 *             cross-diffusion source of u (eq. S with D_{u,1} = chi1 u I and
 *             D_{u,2} = chi2 u I):
 *                 tau S_u,i = (w_i / C_s^2) e_i . K_u (chi1 u G_v + chi2 u G_w),
 *             G_Theta the local gradient of Theta from its first
 *             non-equilibrium moment (relation C146):
 *                 G = -(K (j - a Theta)/tau + K a Phi / 2) / (d C_s^2);
 *             periodic pull streaming.
 *   adjoint   the exact discrete adjoint (AMRT structure, Sec. 3.2.1):
 *             streaming along -e_i backward in time, transposed collisions,
 *             the adjoint-equilibrium broadcast and the coupling terms of the
 *             three sources; dJ/dg assembled in the same kernel.
 *   cost      J = 1/2 sum_x (u^N - u_target)^2 + alpha sum_{n<N} sum_x g^n(x)^2.
 *
 * Conventions: as in cxlbm.h.  Device pointers are caller-owned; the library
 * never allocates device memory (one caller workspace) and keeps no input
 * pointer past the call.  T is float (precision 32) or double (precision 64).
 * Node fields are [ny][nx]; control and gradient buffers [n_steps][ny][nx];
 * the populations of the three species [3][9][ny][nx] inside the workspace.
 * Calls are ordered on the problem's stream and asynchronous unless stated
 * otherwise; every call returns a cx_status (CX_OK = 0).
 */
#ifndef CXARC_H
#define CXARC_H

#include "cxlbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Problem description.  Tensors use the modes of cxlbm.h: CX_ANISO_CONST
 * (D_*[3] = (Dxx, Dxy, Dyy)), CX_ANISO_ROTATED (one angle field theta shared
 * by the three species, eigenvalues lam_*[2] per species), CX_ANISO_FIELD
 * (device FP64 [ny][nx][3] per species).  Convection: CX_ADV_NONE,
 * CX_ADV_ROW (device FP64 [ny][2]) or CX_ADV_FIELD (device FP64 [ny][nx][2]),
 * the same a(x) for all species. */
typedef struct {
    int nx, ny;          /* periodic lattice, 3 <= nx, ny                            */
    int n_steps;         /* N >= 1                                                   */
    int precision;       /* 32 or 64                                                 */
    int ckpt_every;      /* checkpoint interval k of the forward; 0 means N          */
    double tau;          /* lattice time step (1)                                    */
    int aniso;           /* CX_ANISO_*                                               */
    double D_u[3], D_v[3], D_w[3];             /* CONST                              */
    double lam_u[2], lam_v[2], lam_w[2];       /* ROTATED                            */
    const double* theta;                       /* ROTATED: device [ny][nx]           */
    const double* D_u_field;                   /* FIELD: device [ny][nx][3]          */
    const double* D_v_field;
    const double* D_w_field;
    double d;            /* d of the equilibrium (eq. phieq), all species, > 0       */
    double chi1, chi2;   /* chemotactic sensitivities toward v and w (signed)        */
    double a1, a2;       /* Phi_u = a1 u - a2 u^2                                    */
    double b1, b2, b3;   /* Phi_v = b1 u - b2 v - b3 u v                             */
    double c1, c2;       /* Phi_w = c1 u - c2 w                                      */
    int ctrl_species;    /* 1: g added to Phi_v; 2: g added to Phi_w                 */
    int adv;             /* CX_ADV_*                                                 */
    const double* a;     /* see above, or NULL                                       */
    const double* u_target; /* device FP64 [ny][nx]                                  */
    double alpha;        /* control penalty weight, >= 0                             */
    double s[7];         /* free relaxation rates in (0, 2)                          */
    int source_order;    /* 2: keep the (tau/2)(Phi^n - Phi^{n-1}) term; 1: drop it  */
} cx3_desc;

typedef struct cx3_problem cx3_problem; /* opaque, library-owned host object */

/* Bytes of device workspace (host call).  Errors: CX_ERR_INVALID_ARG. */
cx_status cx3_workspace_size(const cx3_desc* desc, size_t* bytes);

/* Create a problem bound to a caller-owned workspace (>= cx3_workspace_size
 * bytes, 256-byte aligned) and to `stream`.  Converts the descriptor's device
 * fields into the workspace (K per node or per problem, a, u_target) and
 * synchronises once; the descriptor's arrays may be freed afterwards.  Checks
 * that every K has eigenvalues in (0, 2).
 * Errors: CX_ERR_INVALID_ARG, CX_ERR_WORKSPACE, CX_ERR_UNSTABLE (K), CX_ERR_CUDA. */
cx_status cx3_create(const cx3_desc* desc, void* workspace, size_t bytes, cudaStream_t stream, cx3_problem** out);

/* Initial populations phi^eq(u0), phi^eq(v0), phi^eq(w0) from device FP64
 * [ny][nx] fields.  Errors: CX_ERR_INVALID_ARG. */
cx_status cx3_set_initial(cx3_problem* p, const double* u0, const double* v0, const double* w0);

/* Forward solve with control g (device T [N][ny][nx], or NULL for zero);
 * stores checkpoints every k steps and the last segment's adjoint tape
 * (u, v, G_v, G_w per node and step); writes the FP64 cost to J_dev (device
 * double, may be NULL).  Errors: CX_ERR_STATE (no initial state). */
cx_status cx3_forward(cx3_problem* p, const void* g, double* J_dev);

/* Exact discrete adjoint sweep with fused gradient assembly, segment by
 * segment backward in time with each segment's forward recomputed from its
 * checkpoint.  g must be the control of the preceding cx3_forward.  Seeds
 * (device T [ny][nx], the adjoints of u^N, v^N, w^N): all three NULL uses the
 * cost's own terminal term (u^N - u_target, 0, 0) and the gradient is dJ/dg;
 * otherwise NULL seeds are zero and the result is the gradient of
 * sum(seed . (u^N, v^N, w^N)) + penalty * alpha ||g||^2, penalty = 0 giving the
 * plain vector-Jacobian product.  Writes dJdg (device T [N][ny][nx]).
 * Errors: CX_ERR_STATE (no forward), CX_ERR_INVALID_ARG (dJdg NULL). */
cx_status cx3_adjoint(cx3_problem* p, const void* g, const void* seed_u, const void* seed_v, const void* seed_w,
                      int penalty, void* dJdg);

/* cx3_forward then cx3_adjoint with NULL seeds. */
cx_status cx3_gradient(cx3_problem* p, const void* g, void* dJdg, double* J_dev);

/* One steepest-descent iteration with Armijo backtracking (Sec. 3.2.1,
 * optimisation process): E_work (device T, control shape) receives
 * E = dJ/dg at g_inout; the first trial is min(1, 1/||E||_inf) on the first
 * call, then twice the previous accepted step; accept when
 * J(g - lam E) <= J(g) - 1e-4 lam ||E||^2 (FP64), halving lam up to 30 times,
 * then g_inout <- g - lam E.  Synchronises once per trial.  info (host) may
 * be NULL.  Errors: CX_ERR_LINESEARCH (g_inout unchanged), CX_ERR_UNSTABLE. */
cx_status cx3_step(cx3_problem* p, void* g_inout, void* E_work, cx_step_info* info);

/* u^N, v^N, w^N of the last forward (device T [ny][nx]; any may be NULL).
 * Errors: CX_ERR_STATE (no forward). */
cx_status cx3_get_fields(cx3_problem* p, void* u_out, void* v_out, void* w_out);

/* J, ||dJ/dg||^2 and max |dJ/dg| of the last forward / adjoint (host doubles,
 * any may be NULL); synchronises.  Errors: CX_ERR_UNSTABLE (a non-finite
 * cost or gradient was recorded), CX_ERR_CUDA. */
cx_status cx3_get_norms(cx3_problem* p, double* J, double* grad_sq, double* grad_inf);

/* Staging of the lattice kernels: 1 (default) runs the forward steps whose
 * inputs are all pulled (n >= 1) in the row-window kernel -- a producer warp
 * stages row segments by bulk asynchronous copies completed on mbarriers --
 * when rows are a whole number of 16-byte units, the planes 16-byte aligned
 * and the grid has at least two row segments per block; 0 uses the
 * per-thread kernels everywhere; 2 takes the row-window kernels for every
 * eligible forward and adjoint step (adjoint: below the terminal one)
 * whatever the grid size (tests; the adjoint's row-window form measured
 * slower).  Results agree to rounding.  A bounded wait of the pipeline that
 * runs out is reported as CX_ERR_TIMEOUT by cx3_step / cx3_get_norms.
 * Errors: CX_ERR_INVALID_ARG. */
cx_status cx3_set_staging(cx3_problem* p, int mode);

/* Per-phase device time (forward, recompute, adjoint: ms[3], launches[3])
 * accumulated while timing is enabled (events on the problem's stream).
 * cx3_get_timing synchronises. */
cx_status cx3_set_timing(cx3_problem* p, int enable);
cx_status cx3_get_timing(cx3_problem* p, double* ms, long long* launches);

cx_status cx3_destroy(cx3_problem* p);

#ifdef __cplusplus
}
#endif

#endif /* CXARC_H */
