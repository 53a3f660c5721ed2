/*
 * cxlbm.h -- C ABI of the GB300 (sm_103a) MRT / AMRT lattice Boltzmann
 * optimal-control library for the two-species chemotaxis system
 *
 *     du/dt = div(D_u grad u - chi u grad v) - div(a u)
 *     dv/dt = div(D_v grad v) - div(a v) + r_vu u + r_vv v + g
 *
 * (the paper's system (eq:ReacDiff) with Theta in {u, v}, D_{u,1} = chi u I,
 * convective flux T_Theta = a Theta, and the distributed control g acting on
 * the v equation; Sec. 2.1 states the control problem (EPS) and Sec. 3.2.1 the
 * discrete-adjoint optimisation process that the calls below follow).
 *
 * Discrete problem solved (Sec. 3.1 and 3.2):
 *   forward   eq. (LBE)/(LBEG): per species, MRT collision in moment space
 *             with M0 and the block relaxation matrix Pi (K block from
 *             D = d C_s^2 tau (K^-1 - I/2)), cross-diffusion source S_u (eq. S),
 *             reaction/control source (eq. PhiS) with the tau/2 time-derivative
 *             term, pull streaming with halfway bounce-back at solid nodes.
 *   adjoint   AMRT (eqs. CAE, AEDs, AEDsM, CAEL): reverse-time sweep streaming
 *             along -e_i, transposed collision, adjoint equilibrium broadcast,
 *             coupling terms; the gradient (gradientLattice / JD-H-B) is
 *             assembled inside the same kernel.
 *   cost      J = 1/2 sum_x (u^N - u_target)^2 + alpha sum_{n<N} sum_x g^n(x)^2.
 *
 * Conventions for every call:
 *   - Pointers documented as "device" are CUDA device pointers owned by the
 *     caller; the library never allocates device memory (the caller passes
 *     one workspace) and never frees caller memory.  It keeps no input pointer
 *     past the call that receives it.
 *   - "T" is float when precision == 32 and double when precision == 64.
 *   - Node fields are row-major [ny][nx]; control and gradient buffers are
 *     [n_steps][ctrl_ny][ctrl_nx]; population buffers are [2][Q][ny][nx]
 *     (species u then v).
 *   - All calls are ordered on the problem's stream and asynchronous unless
 *     stated otherwise; cx_step, cx_get_norms and cx_get_timing synchronise.
 *   - Every call returns a cx_status; CX_OK is 0.  A CUDA error (launch or a
 *     failed runtime call) returns CX_ERR_CUDA.  Errors a kernel detects (a
 *     non-finite cost or gradient, a bounded wait that ran out) are recorded
 *     in a device status word and reported by the next synchronising call.
 */
#ifndef CXLBM_H
#define CXLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* cudaStream_t; /* the CUDA runtime's stream handle */

typedef enum {
    CX_OK = 0,
    CX_ERR_INVALID_ARG = 1, /* bad descriptor or argument (checked on the host) */
    CX_ERR_WORKSPACE = 2,   /* workspace missing, too small or misaligned      */
    CX_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed     */
    CX_ERR_STATE = 4,       /* call out of order (e.g. adjoint before forward) */
    CX_ERR_UNSTABLE = 5,    /* non-finite cost or gradient                     */
    CX_ERR_LINESEARCH = 6,  /* Armijo backtracking found no acceptable step    */
    CX_ERR_TIMEOUT = 7,     /* a bounded device-side wait ran out              */
    CX_ERR_INTERNAL = 8
} cx_status;

enum { CX_ANISO_CONST = 0, CX_ANISO_ROTATED = 1, CX_ANISO_FIELD = 2 };
enum { CX_ADV_NONE = 0, CX_ADV_ROW = 1, CX_ADV_FIELD = 2 };

/* Problem descriptor.  Read once by cx_workspace_size / cx_create. */
typedef struct {
    int nx, ny;          /* lattice nodes (h = 1), 3 <= nx, ny                       */
    int n_steps;         /* N time steps (tau = T/N), >= 1                            */
    int lattice;         /* 9 (D2Q9, Sec. 3.1) or 5 (D2Q5)                            */
    int precision;       /* 32 or 64: type T of populations, controls and gradients  */
    int ckpt_every;      /* k: checkpoint interval of the forward; 0 means N          */
    double tau;          /* lattice time step, 1 in lattice units (c = h/tau = 1)     */
    /* self-diffusion tensors D_u, D_v (symmetric) */
    int aniso;           /* CX_ANISO_*                                                */
    double D_u[3], D_v[3];       /* CONST: (Dxx, Dxy, Dyy)                             */
    double lam_u[2], lam_v[2];   /* ROTATED: eigenvalues along (cos t, sin t) and its normal */
    const double* theta;         /* ROTATED: device [ny][nx] angle t(x)                */
    const double* D_u_field;     /* FIELD: device [ny][nx][3]                          */
    const double* D_v_field;     /* FIELD: device [ny][nx][3]                          */
    double d_u, d_v;     /* d_Theta of the equilibrium (eq. phieq), > 0               */
    double chi;          /* chemotactic sensitivity (signed)                         */
    double r_vu, r_vv;   /* Phi_v = r_vu u + r_vv v + g                               */
    int adv;             /* CX_ADV_*                                                  */
    const double* a;     /* ROW: device [ny][2]; FIELD: device [ny][nx][2]; else NULL */
    const uint8_t* solid;     /* device [ny][nx], 1 = solid (bounce-back), or NULL   */
    int ctrl_x0, ctrl_y0, ctrl_nx, ctrl_ny; /* control window; ctrl_nx = 0: whole grid */
    const uint8_t* ctrl_mask; /* device [ctrl_ny][ctrl_nx], 1 = controlled, or NULL   */
    const double* u_target;   /* device [ny][nx]                                     */
    double alpha;             /* control penalty weight, >= 0                        */
    double s[7];              /* free relaxation rates s0..s6 of Pi, in (0, 2)       */
    int source_order;         /* 2: keep (tau/2)(Phi^n - Phi^{n-1}); 1: drop it      */
    int ctrl_windows;         /* W: g piecewise constant in time over W equal windows
                                 (g^n = G_{n/(N/W)}, W divides N); 0: one value per
                                 step (W = N).  Controls and gradients are [W][ctrl]. */
    int halo;                 /* 1: this grid is one sub-domain of a larger problem and
                                 its outer one-node frame is a halo (see cx_set_halo_exchange):
                                 frame nodes are pulled from but never updated, costed or
                                 controlled.  0: the grid is the whole (periodic) problem. */
} cx_problem_desc;

typedef struct cx_problem cx_problem; /* opaque, library-owned host object */

typedef struct {
    double J0;      /* cost at the incoming control                  */
    double J;       /* cost at the accepted control                  */
    double lam;     /* accepted step length                          */
    double grad_sq; /* ||dJ/dg||^2 at the incoming control           */
    double grad_inf;/* max |dJ/dg| at the incoming control           */
    int trials;     /* forward solves spent in the line search       */
} cx_step_info;

/* Bytes of device workspace the problem needs (host call, no device work).
 * Errors: CX_ERR_INVALID_ARG for an inconsistent descriptor. */
cx_status cx_workspace_size(const cx_problem_desc* desc, size_t* bytes);

/* Create a problem bound to a caller-owned device workspace of at least
 * cx_workspace_size bytes (256-byte aligned) and to `stream`.  Copies and
 * converts every descriptor field (tensor, velocity, mask and target fields)
 * into the workspace, then synchronises the stream once.  The descriptor's
 * device arrays may be freed after the call.  Checks the relaxation blocks
 * K (eigenvalues in (0, 2), the stability remark after (UGS)).
 * Errors: CX_ERR_INVALID_ARG, CX_ERR_WORKSPACE, CX_ERR_CUDA. */
cx_status cx_create(const cx_problem_desc* desc, void* workspace, size_t bytes, cudaStream_t stream,
                    cx_problem** out);

/* Initial populations phi^eq(u0), phi^eq(v0) (device T [ny][nx] each),
 * the initial condition of the forward solve.  Errors: CX_ERR_INVALID_ARG. */
cx_status cx_set_initial(cx_problem* p, const void* u0, const void* v0);

/* Forward MRT solve over N steps with control g (device T [W][ctrl_ny][ctrl_nx],
 * W = ctrl_windows or N, or NULL for zero control) (step 2 of the discrete-adjoint algorithm, Sec. 3.2.1).  Stores every k-th
 * state as a checkpoint and the last segment's adjoint tape, then writes the
 * FP64 cost J to J_dev (device double, may be NULL).  Needs cx_set_initial.
 * Errors: CX_ERR_STATE (no initial state), CX_ERR_INVALID_ARG, CX_ERR_CUDA. */
cx_status cx_forward(cx_problem* p, const void* g, double* J_dev);

/* AMRT adjoint sweep with fused gradient assembly (steps 3-4 of the
 * algorithm, eqs. CAE/CAEL and gradientLattice): reverse-time, segment by
 * segment, recomputing each segment's forward from its checkpoint.
 * g must be the control of the preceding cx_forward.  seed_u / seed_v
 * (device T [ny][nx]) are the adjoint of u^N / v^N; seed_u == NULL uses
 * u^N - u_target (the cost's own terminal term), seed_v == NULL uses 0.
 * Writes dJdg (device T [W][ctrl_ny][ctrl_nx]): the gradient of
 * sum(seed_u u^N + seed_v v^N) + alpha ||g||^2 -- of J itself when both seeds
 * are NULL -- with zeros at uncontrolled nodes.  With time windows, the
 * gradient of window w is the sum of the per-step gradients over its steps
 * (the penalty alpha sum_n ||g^n||^2 counts each window N/W times).
 * Errors: CX_ERR_STATE (no forward since the last cx_create / cx_set_initial). */
cx_status cx_adjoint(cx_problem* p, const void* g, const void* seed_u, const void* seed_v, void* dJdg);

/* Vector-Jacobian product of the solve (u^N, v^N) = F(g): the same seeded
 * AMRT sweep as cx_adjoint (the adjoint system with the final condition
 * given by the seeds, Sec. 3.2.1) without the control-penalty term, i.e.
 *   vjp = (du^N/dg)^T seed_u + (dv^N/dg)^T seed_v,
 * device T [W][ctrl_ny][ctrl_nx], zero at uncontrolled nodes; with time
 * windows the per-step products summed over each window's steps (the chain
 * rule of g^n = G_w).  seed_u / seed_v: device T [ny][nx], NULL meaning a
 * zero seed.  g must be the control of the preceding cx_forward.  This is
 * the backward of a differentiable solve (an autograd function); J and the
 * penalty belong to cx_adjoint.  Errors: CX_ERR_INVALID_ARG (vjp NULL),
 * CX_ERR_STATE (no forward). */
cx_status cx_adjoint_vjp(cx_problem* p, const void* g, const void* seed_u, const void* seed_v, void* vjp);

/* cx_forward followed by cx_adjoint with NULL seeds: J (device double, may be
 * NULL) and dJ/dg. */
cx_status cx_gradient(cx_problem* p, const void* g, void* dJdg, double* J_dev);

/* cx_gradient with the control and the gradient in HOST memory: g_host (host
 * T [W][ctrl_ny][ctrl_nx], page-locked for the copies to overlap) is copied
 * into g_dev, the gradient computed into dJdg_dev (both device T of the same
 * size, caller-owned, not aliasing) and copied back into dJdg_host (host T,
 * same size); J goes to *J_host (host double, may be NULL).  The control
 * moves in chunks of windows on a copy stream of the problem's own, each
 * forward step waiting only for the chunk that holds its control; each
 * gradient chunk leaves on a second copy stream as soon as the reverse sweep
 * has finished it.  So the copies overlap the kernels except the first chunk
 * in and the last chunk out.  Synchronises before it returns (the host
 * buffers may be reused at once).  The two copy streams are created on the
 * first call and destroyed with the problem.  Errors: CX_ERR_INVALID_ARG (a
 * NULL buffer, or a sub-domain), CX_ERR_STATE (no initial state),
 * CX_ERR_CUDA, CX_ERR_UNSTABLE, CX_ERR_TIMEOUT. */
cx_status cx_gradient_host(cx_problem* p, const void* g_host, void* dJdg_host, double* J_host, void* g_dev,
                           void* dJdg_dev);

/* One steepest-descent iteration with Armijo backtracking (step 5 of the
 * algorithm; first trial min(1, 1/||E||_inf), the heuristic of the remark
 * after the continuous gradient algorithm, then twice the previous step).
 * g_inout (device T [W][ctrl_ny][ctrl_nx]) is updated in place to g - lam E
 * when J(g - lam E) <= J(g) - 1e-4 lam ||E||^2 (FP64 test); lam halves up to
 * 30 times.  E_work (device T, same shape, caller-owned) receives the
 * gradient E = dJ/dg at the incoming g.  Runs a forward first unless the
 * previous cx_forward / accepted cx_step left its state at g_inout (the
 * accepted trial's forward is reused, so each iteration costs one adjoint
 * plus its trial forwards).  Synchronises once per trial.  info (host) may be
 * NULL.  Errors: CX_ERR_LINESEARCH (g_inout unchanged), CX_ERR_UNSTABLE. */
cx_status cx_step(cx_problem* p, void* g_inout, void* E_work, cx_step_info* info);

/* Sensitivity (tangent-linear) problem along the control direction dg
 * (device T [W][ctrl], like g) about the trajectory of control g, which must
 * be the control of the preceding cx_forward (its checkpoints are reused;
 * the state stays valid for a following cx_adjoint or step).  The forward
 * step of cx_forward linearised about that trajectory, solved by the same
 * MRT scheme (the sensitivity system of the remark after the gradient
 * algorithm, Sec. 2.3), from du^0 = dv^0 = 0.  Writes du^N, dv^N (device T
 * [ny][nx], either may be NULL) and ||du^N||^2 (host double, may be NULL;
 * synchronising when given).  Errors: CX_ERR_STATE (no forward). */
cx_status cx_tlm(cx_problem* p, const void* g, const void* dg, void* du_out, void* dv_out, double* du_sq);

/* Continuous-adjoint gradient (the algorithm of Sec. 3.2.1 that solves the
 * adjoint PDE system (FVM-PF-Adj) by the MRT scheme with time reversed; an
 * O(tau, h) approximation of the exact discrete gradient of cx_adjoint).
 * For Phi_u = 0, Phi_v = r_vu u + r_vv v + g and the terminal cost, with
 * s = T - t:
 *   du~/ds = div(D_u grad u~) + a.grad u~ + chi grad v . grad u~ + r_vu v~
 *   dv~/ds = div(D_v grad v~) + a.grad v~ + r_vv v~ - div(chi u grad u~)
 *   u~(0) = u^N - u_target, v~(0) = 0;  dJ/dg^n = 2 alpha g^n + v~(t_{n+1})
 * (summed over a window's steps for windowed controls), solved with
 * convection -a, first-order sources, the chemotaxis-type source for the
 * cross term and u, grad v of the forward steps from the tape.  g must be
 * the control of the preceding cx_forward.  dJdg: device T [W][ctrl].
 * Errors: CX_ERR_STATE (no forward). */
cx_status cx_cadjoint(cx_problem* p, const void* g, void* dJdg);

/* One steepest-descent iteration whose step length minimises the quadratic
 * model of J along -E from the sensitivity problem (eqs. LM / LMA, Sec. 2.3):
 * lam* = ||E||^2 / (||du^N(E)||^2 + 2 alpha L ||E||^2), L = N/W steps per
 * control window; accepted under the Armijo test of cx_step (halved up to 30
 * times if it fails).  Costs one adjoint, one sensitivity pass and usually
 * one trial forward.  Arguments and errors as cx_step. */
cx_status cx_lma_step(cx_problem* p, void* g_inout, void* E_work, cx_step_info* info);

/* Nonlinear conjugate gradients (remark 2 after the gradient algorithm,
 * Sec. 2.3): direction D_k = -G_k (k = 0), else -G_k + r_{k-1} D_{k-1} with r
 * from Fletcher-Reeves, Polak-Ribiere, Hestenes-Stiefel or Dai-Yuan, reset to
 * -G_k when D_k is not a descent direction or |<G_k, G_{k-1}>| >= 0.2
 * ||G_k||^2; step g <- g + lam D_k with lam from a weak Wolfe-Powell line
 * search (J(g + lam D) <= J(g) + 1e-4 lam <G, D>, <G(g + lam D), D> >=
 * 0.1 <G, D>; bisection of the bracket, doubling while it is open, at most
 * 30 trials; first trial min(1, 1/||G||_inf), then lam_{k-1} <G,D>_{k-1} /
 * <G,D>_k).  Each trial costs a forward solve, and an AMRT sweep when the
 * decrease condition holds; the accepted trial's gradient is the next
 * iteration's.  If no trial meets both conditions (no progress along the CG
 * direction, e.g. at the rounding floor of FP32 lattices) the iteration
 * falls back to a steepest-descent step with Armijo backtracking from
 * min(1, 1/||G||_inf) (soft reset; trials then counts 30 + its trials).
 * work: device T [4][W][ctrl_ny][ctrl_nx], caller-owned and
 * kept between calls (gradients, direction, trial control).  The iteration
 * state refers to g_inout as the previous call left it: call cx_cg_reset
 * after changing g or the initial state (cx_set_initial resets it).
 * Synchronous.  Errors: CX_ERR_LINESEARCH (not even the fallback step
 * decreased J; the state is reset), CX_ERR_UNSTABLE, CX_ERR_STATE,
 * CX_ERR_INVALID_ARG. */
enum { CX_CG_FR = 0, CX_CG_PR = 1, CX_CG_HS = 2, CX_CG_DY = 3 };
typedef struct {
    double J0;      /* cost at the incoming control       */
    double J;       /* cost at the accepted control       */
    double lam;     /* accepted step length along D       */
    double grad_sq; /* ||G||^2 at the accepted control     */
    double beta;    /* r_k of the chosen formula           */
    int trials;     /* line-search trials (forward solves) */
    int restarted;  /* 1 if the new direction is -G       */
} cx_cg_info;
cx_status cx_cg_step(cx_problem* p, void* g_inout, void* work, int variant, cx_cg_info* info);
cx_status cx_cg_reset(cx_problem* p);

/* u^N and v^N of the last forward (device T [ny][nx] each, either may be NULL). */
cx_status cx_get_fields(cx_problem* p, void* u_out, void* v_out);

/* Adjoint populations psi^0 of the last cx_adjoint: the sensitivity of the
 * seeded functional to the initial populations (device T [2][Q][ny][nx]).
 * Solid nodes have no populations: their entries carry no meaning (on grids
 * with solid nodes they hold the bounce-back copies of the adjoint step). */
cx_status cx_get_psi0(cx_problem* p, void* out);

/* Synchronising: cost of the last forward, ||dJ/dg||^2 and max |dJ/dg| of the
 * last adjoint (host doubles, any may be NULL); returns any recorded device
 * error (CX_ERR_UNSTABLE for a non-finite value). */
cx_status cx_get_norms(cx_problem* p, double* J, double* grad_sq, double* grad_inf);

/* Launch shape of the persistent lattice kernels: `threads` per block (64,
 * 128 or 256) and `blocks` resident blocks (0: every SM at full occupancy).
 * Results do not depend on the shape.
 * Errors: CX_ERR_INVALID_ARG (also when blocks * threads / 32 > 32768). */
cx_status cx_set_launch(cx_problem* p, int threads, int blocks);
/* Staging of the lattice kernels' inputs.  row_windows = 1 (default): the
 * forward steps n >= 1 and the interior adjoint steps of grids without solid
 * nodes, whose rows are a whole number of 16-byte units, whose launch has
 * 128 or 256 threads and gives each block at least two row segments (the
 * sensitivity and continuous-adjoint passes too), stage each row segment of
 * the pulled populations and
 * the node-local planes in shared memory with bulk asynchronous copies
 * completed on an mbarrier (a wait that never completes ends the launch and
 * later calls return CX_ERR_TIMEOUT); other steps use per-thread
 * asynchronous copies.  row_windows = 0: per-thread copies everywhere.
 * Results are bitwise identical either way (same arithmetic per node).
 * row_windows = 2 is a test mode of the timeout path (the segment-count
 * condition is not applied): each stage expects 16
 * bytes more than it copies, so every wait runs out (0.2 s), the launch ends
 * early with the status bit set, later launches return at once, and the next
 * synchronising call returns CX_ERR_TIMEOUT; the problem stays in that state
 * (create a new one).  CX_ERR_INVALID_ARG for other values. */
cx_status cx_set_staging(cx_problem* p, int row_windows);

/* Per-phase timing with CUDA events on the problem's stream: enable != 0
 * starts accumulating.  cx_get_timing (synchronising) returns milliseconds
 * and kernel-launch counts for the phases [forward, recompute, adjoint,
 * other] (ms[4], launches[4]; either may be NULL) and resets them. */
cx_status cx_set_timing(cx_problem* p, int enable);
cx_status cx_get_timing(cx_problem* p, double* ms, long long* launches);

/* ------------------------------------------------------------------------
 * Batched problems: `count` independent problems (uneven sizes, tensors,
 * chemotaxis, masks, controls) that share n_steps, ckpt_every, lattice and
 * precision.  Every time step of every problem runs in one persistent launch
 * (tiles of all problems in one work list); the launch sequence of a forward
 * or gradient evaluation is captured once as a CUDA graph and replayed until
 * the bindings or tile shapes change.  Per node the arithmetic is that of
 * cx_forward / cx_adjoint (same formulas; results agree to rounding), and
 * replays of the captured graph are bitwise reproducible.
 *   descs            host array of `count` descriptors (as for cx_create)
 *   workspace        device, cx_batch_workspace_size bytes, 256-byte aligned
 *   stream           must not be the legacy default stream (graph capture)
 * Errors: CX_ERR_INVALID_ARG (mismatched n_steps/ckpt_every/lattice/precision,
 * count outside 1..4096), CX_ERR_WORKSPACE, CX_ERR_CUDA. */
typedef struct cx_batch cx_batch;
cx_status cx_batch_workspace_size(const cx_problem_desc* descs, int count, size_t* bytes);
cx_status cx_batch_create(const cx_problem_desc* descs, int count, void* workspace, size_t bytes,
                          cudaStream_t stream, cx_batch** out);
/* u0[i], v0[i]: device T [ny_i][nx_i] (host arrays of device pointers). */
cx_status cx_batch_set_initial(cx_batch* b, const void* const* u0, const void* const* v0);
/* Controls g[i] (device T [W][ctrl], NULL entries: zero control) and gradient
 * outputs dJdg[i] (device T, may be NULL for forward-only use); host arrays.
 * Synchronous (uploads the problem table). */
cx_status cx_batch_bind(cx_batch* b, const void* const* g, void* const* dJdg);
/* Tile shapes: `threads` per block (128 or 256), `blocks` persistent blocks
 * (0: every SM at full residency), tile_x[i] = tile width of problem i (a
 * power of two dividing threads, >= 32, threads / tile_x[i] <= 8; NULL:
 * threads), rows[i] = nodes each thread updates per tile, 1..32 (NULL: 2).
 * The tile height is (threads / tile_x[i]) rows[i].  Synchronous. */
cx_status cx_batch_set_tiles(cx_batch* b, int threads, int blocks, const int* tile_x, const int* rows);
/* Tile autotuner (the scheduling choice behind the one-launch-per-step batch;
 * no equation of the method changes with it).  Size class = problems with the
 * same nx.  Times a probe of min(probe_steps, N) forward steps, their segment
 * recompute and the AMRT adjoint sweep on the batch's own problems (the
 * kernels differ in their best tiles), with CUDA events on the batch stream:
 * for threads 128 and 256 the best of five uniform (tile_x, rows) shapes,
 * then coordinate descent per size class over rows {4, 8, 16, 32} and the
 * admissible widths {32, 64, 128, 256}, the others fixed.  The winner is
 * applied as by cx_batch_set_tiles (blocks = 0).
 * cache_path (may be NULL): a text file of one line per tuned batch,
 * "signature<TAB>threads<TAB>nx:tile_x:rows,...<TAB>ms", the signature
 * naming the device, lattice, precision and size-class histogram; a matching
 * line is applied without probing, a new result is added (the file is
 * rewritten through a temporary and renamed).
 * Needs cx_batch_set_initial and a binding with every dJdg set; the probe
 * overwrites checkpoints 1.. and the tapes, so the next evaluation starts
 * from the initial state.  Outputs (host, each may be NULL): threads_out,
 * tile_x_out[count] and rows_out[count] per problem, probe_ms_out (the
 * probe time of the winner, from the cache when it came from there).
 * Synchronous.  CX_ERR_INVALID_ARG for probe_steps < 1, CX_ERR_STATE
 * without the state above, CX_ERR_INTERNAL if the cache cannot be written. */
cx_status cx_batch_autotune(cx_batch* b, int probe_steps, const char* cache_path, int* threads_out,
                            int* tile_x_out, int* rows_out, double* probe_ms_out);
/* Staging of the batched kernel's inputs, as cx_set_staging for one problem:
 * row_windows = 1 stages each work item's rows of pulled
 * populations and node-local planes by bulk asynchronous copies completed on
 * an mbarrier, on every step but the first forward step and the terminal
 * adjoint step, when no problem has solid nodes, every nx is a whole number of
 * 16-byte units and the bound control and gradient arrays are 16-byte aligned
 * (otherwise, and with row_windows = 0, the default, per-thread copies).  A
 * wait that never completes ends the launch; later calls that read the status
 * return CX_ERR_TIMEOUT.  Results are bitwise identical either way.  The
 * default is per-thread staging because the batched kernel holds about 128
 * registers per thread (16 resident warps per SM), too few to hide the block
 * barrier each row-window item needs (measured 6.8 against 8.5 GLUPS for the
 * per-thread form on the 256-problem workload).  Drops the captured graphs.  CX_ERR_INVALID_ARG for
 * other values. */
cx_status cx_batch_set_staging(cx_batch* b, int row_windows);
/* Forward of every problem; J_dev (device double [count], may be NULL). */
cx_status cx_batch_forward(cx_batch* b, double* J_dev);
/* Forward + recompute + AMRT adjoint of every problem into the bound dJdg;
 * out_dev (device double [3 count], may be NULL): J, ||dJ/dg||^2, max |dJ/dg|. */
cx_status cx_batch_gradient(cx_batch* b, double* out_dev);
/* AMRT adjoint of every enabled problem seeded with seed_u[i] (device T
 * [ny_i][nx_i], the adjoint of u^N; NULL array or entry: u^N - u_target),
 * into the bound dJdg: the gradient of sum(seed_u u^N) + alpha ||g||^2 at the
 * bound controls.  add_to_cost_seed != 0: the seed is (u^N - u_target) +
 * seed_u[i] instead (the gradient of J + sum(seed_u u^N)).  Needs the preceding cx_batch_forward (or accepted
 * cx_batch_step) at those controls; out_dev (device double [3 count], may be
 * NULL) receives ||dJ/dg||^2 and max |dJ/dg| in its last 2 count entries.
 * Errors: CX_ERR_STATE (no forward state at the bound controls). */
cx_status cx_batch_adjoint(cx_batch* b, const void* const* seed_u, int add_to_cost_seed, double* out_dev);
/* g[i] <- g[i] - lam[i] dJdg[i] for every enabled problem (lam: host double
 * [count], 0 leaves a problem alone), rounded as a line-search trial;
 * forgets the step-length history.  Asynchronous. */
cx_status cx_batch_axpy(cx_batch* b, const double* lam);
/* Capture every launch sequence (forward, gradient, line-search trial,
 * adjoint) as CUDA graphs now rather than on first use, without running
 * them.  Needs the bindings; synchronous. */
cx_status cx_batch_prepare(cx_batch* b);
cx_status cx_batch_get_fields(cx_batch* b, int i, void* u_out, void* v_out);
/* Synchronising: CX_ERR_UNSTABLE if any problem's J or gradient was non-finite. */
cx_status cx_batch_get_status(cx_batch* b);
/* Switch problems on (enabled[i] != 0) or off for every later forward,
 * gradient and step (NULL: all on).  Switched-off problems cost no lattice
 * work; their outputs, fields and gradients are undefined until they are
 * switched on and evaluated again.  Synchronous. */
cx_status cx_batch_set_enabled(cx_batch* b, const int* enabled);
/* One steepest-descent iteration with Armijo backtracking for every enabled
 * problem, each with the rule of cx_step (its own step length and history):
 * the bound g[i] are updated in place, the bound dJdg[i] receive the
 * gradients at the incoming controls.  Each line-search trial is one batched
 * forward over the problems still searching.  The AMRT gradient reuses the
 * accepted trials' forward state when the previous step accepted every
 * problem.  info (host, count entries, may be NULL) as for cx_step (trials = 0
 * for switched-off or stationary problems); status (host int [count], may be
 * NULL): CX_OK, CX_ERR_LINESEARCH (no accepted trial: g[i] unchanged) or
 * CX_ERR_UNSTABLE per problem.  Every bound g[i] and dJdg[i] must be non-NULL.
 * Synchronous.  Errors: CX_ERR_STATE (no initial state or binding),
 * CX_ERR_INVALID_ARG, CX_ERR_CUDA. */
cx_status cx_batch_step(cx_batch* b, cx_step_info* info, int* status);
cx_status cx_batch_destroy(cx_batch* b);

/* ------------------------------------------------------------------------
 * Warm-start surrogate kernels.  (No counterpart in the paper: a small
 * convolutional network proposes the initial control that the paper's
 * gradient algorithm then refines.)  Tensors are NCHW; uint16_t* arguments are
 * BF16 device arrays, float* FP32 device arrays; every call is asynchronous
 * on `stream`.  Convolutions are 3x3 with zero padding 1 or 1x1 (ks), direct
 * convolutions on the tensor cores (BF16 products, FP32 accumulation) that
 * read weights in the packed layouts of cx_nn_pack_weights.
 * Errors: CX_ERR_INVALID_ARG for inconsistent shapes or NULL arguments,
 * CX_ERR_CUDA on a launch failure. */
/* Elements of the packed BF16 weights of a [Cout][Cin][ks][ks] layer:
 * which = 0 the forward pack, 1 the data-gradient pack. */
size_t cx_nn_packed_weights(int Cout, int Cin, int ks, int which);
/* Both packs of BF16 weights w[Cout][Cin][ks][ks]: w_fwd [ceil(Cin/16)][ks*ks][Cout][16]
 * and w_bwd [ceil(Cout/16)][ks*ks][Cin][16] (flipped taps, in/out swapped), zero-padded. */
cx_status cx_nn_pack_weights(const uint16_t* w, int Cout, int Cin, int ks, uint16_t* w_fwd, uint16_t* w_bwd,
                             cudaStream_t stream);
/* y[B][Cout][H][W] = act(bias + conv(x[B][Cin][H][W], w)); w_fwd the forward
 * pack of w; act = ReLU if relu.  bias may be NULL. */
cx_status cx_nn_conv_forward(const uint16_t* x, const uint16_t* w_fwd, const float* bias, uint16_t* y, int B,
                             int Cin, int Cout, int H, int W, int ks, int relu, cudaStream_t stream);
/* As cx_nn_conv_forward without activation, writing FP32 y (the network's output layer). */
cx_status cx_nn_conv_forward_f32(const uint16_t* x, const uint16_t* w_fwd, const float* bias, float* y, int B,
                                 int Cin, int Cout, int H, int W, int ks, cudaStream_t stream);
/* Tile of output channels of cx_nn_conv_forward_tc for Cout (the largest of
 * 256, 128, 64, 32 dividing it), 0 when Cout is not a multiple of 32. */
int cx_nn_conv_tc_tile(int Cout);
/* cx_nn_conv_forward on the 5th-generation tensor cores (tcgen05 MMA with the
 * accumulator in tensor memory; BF16 products, FP32 accumulation), for Cout a
 * multiple of 32.  status (device int, may be NULL): bit 0 set if a bounded
 * wait for the tensor cores timed out (the outputs of that tile are then not
 * written).  Errors: CX_ERR_INVALID_ARG (shape or Cout), CX_ERR_CUDA. */
cx_status cx_nn_conv_forward_tc(const uint16_t* x, const uint16_t* w_fwd, const float* bias, uint16_t* y, int B,
                                int Cin, int Cout, int H, int W, int ks, int relu, int* status, cudaStream_t stream);
/* Separable periodic low-pass of BC planes [H][W] (FP32): out = taps (*) along
 * x then y, taps[0..2 radius] a device FP32 array (radius <= 64); tmp is
 * scratch of the same size as in. */
cx_status cx_nn_smooth(const float* in, float* tmp, float* out, int BC, int H, int W, const float* taps, int radius,
                       cudaStream_t stream);
/* dx[B][Cin][H][W] = gradient w.r.t. x of sum(dy * conv(x, w)); w_bwd the data-gradient pack of w. */
cx_status cx_nn_conv_backward_data(const uint16_t* dy, const uint16_t* w_bwd, uint16_t* dx, int B, int Cin, int Cout,
                                   int H, int W, int ks, cudaStream_t stream);
/* FP32 scratch bytes for cx_nn_conv_backward_weight with `splits` pixel ranges. */
size_t cx_nn_conv_backward_weight_scratch(int B, int Cin, int Cout, int H, int W, int ks, int splits);
/* dw[Cout][Cin][ks][ks] (FP32) and db[Cout] (FP32, may be NULL): gradients of sum(dy * conv);
 * the pixel tiles are split over `splits` block ranges whose FP32 partials
 * (in scratch) are summed in a fixed order. */
cx_status cx_nn_conv_backward_weight(const uint16_t* x, const uint16_t* dy, float* dw, float* db, float* scratch,
                                     int splits, int B, int Cin, int Cout, int H, int W, int ks,
                                     cudaStream_t stream);
/* The same weight and bias gradients (3x3 only) on the tcgen05 tensor cores:
 * per block 128 output channels x 16 input channels x 9 taps accumulated in
 * tensor memory over 8 x 8 pixel tiles (K = pixels; the tap shifts of the
 * input are materialised in shared memory).  Same scratch size and partial
 * layout as cx_nn_conv_backward_weight, then the same fixed-order sum over
 * splits.  Needs H and W multiples of 8 and 16-byte aligned x, dy.  status
 * (device int, may be NULL) is set non-zero if a bounded wait ran out (dw, db
 * then hold no result).  Errors: CX_ERR_INVALID_ARG. */
cx_status cx_nn_conv_backward_weight_tc(const uint16_t* x, const uint16_t* dy, float* dw, float* db, float* scratch,
                                        int splits, int B, int Cin, int Cout, int H, int W, int ks, int* status,
                                        cudaStream_t stream);
/* dz = dy where y > 0, else 0 (y = ReLU output). */
cx_status cx_nn_relu_backward(const uint16_t* y, const uint16_t* dy, uint16_t* dz, size_t n, cudaStream_t stream);
cx_status cx_nn_add(const uint16_t* a, const uint16_t* b, uint16_t* out, size_t n, cudaStream_t stream);
/* 2x2 average pooling of [BC][H][W] (H, W even); backward: in = dY [BC][H/2][W/2], out = dX [BC][H][W]. */
cx_status cx_nn_pool2(const uint16_t* in, uint16_t* out, int BC, int H, int W, int backward, cudaStream_t stream);
/* nearest 2x upsampling of [BC][H][W]; backward: in = dY [BC][2H][2W], out = dX [BC][H][W]. */
cx_status cx_nn_up2(const uint16_t* in, uint16_t* out, int BC, int H, int W, int backward, cudaStream_t stream);
/* loss (device double, may be NULL) = mean((out - target)^2); dout (may be NULL) = its gradient. */
cx_status cx_nn_mse(const uint16_t* out, const float* target, uint16_t* dout, double* loss, size_t n,
                    cudaStream_t stream);
/* Adam step t >= 1 on FP32 master weights p (moments m, v), writing the BF16 copy p_bf16. */
cx_status cx_nn_adam(float* p, float* m, float* v, const float* g, uint16_t* p_bf16, size_t n, float lr, float b1,
                     float b2, float eps, int t, cudaStream_t stream);
cx_status cx_nn_cast_bf16(const float* in, uint16_t* out, size_t n, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Forward solve without any device allocation.  (No counterpart in the paper:
 * this is a deployment variant of cx_forward.)
 *
 * For callers that cannot call cudaMalloc or hand the library a workspace --
 * code running inside a host callback or a plug-in of another runtime, a
 * process whose device memory is reserved up front by a pool it does not
 * control, or code that must not touch the allocator while another library
 * holds it.  The call computes what cx_create + cx_set_initial + cx_forward +
 * cx_get_fields compute for the same descriptor (same kernels and launch
 * shapes), with every scratch buffer placed in one file-scope __device__
 * array of CX_STATIC_SCRATCH_BYTES that each GPU loading the library holds
 * until the process exits.  It calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *
 *   desc     as for cx_create; its device arrays, like u0, v0 and g, are read
 *            by work queued on `stream` and must stay valid until it completes
 *   u0, v0   device T [ny][nx] initial fields
 *   g        device T [W][ctrl_ny][ctrl_nx], W = ctrl_windows or N control, or NULL (zero control)
 *   J_dev    device double: the cost J (may be NULL)
 *   uN, vN   device T [ny][nx]: u^N, v^N (either may be NULL)
 *   status_dev device int (may be NULL): written when the queued work ends,
 *            with CX_OK, CX_ERR_TIMEOUT (a bounded wait of a row-window
 *            kernel ran out: the outputs are not valid) or CX_ERR_UNSTABLE
 *            (J is not finite).  The call's return value covers only what
 *            the host checks before queueing the work.
 *   stream   the stream every operation is ordered on; asynchronous
 *
 * Limits and sharing: the scratch is three population lattices (2Q planes
 * each), 5 to 13 node planes (Phi, u^N, v^N, the terminal seed and the
 * target, plus the angle, tensor or velocity fields the descriptor asks for),
 * two bytes per node of solid mask and bounce-back flags, one per control
 * node of control mask, and
 * 16 max(ceil(nx/32) ny, 32768) bytes of FP64 partial sums: about
 * (6Q + 6) sizeof(T) bytes per node for the rotated-tensor workloads, so up
 * to about 520 x 520 nodes in FP32 with D2Q9.  Problems that need more than
 * CX_STATIC_SCRATCH_BYTES are rejected with CX_ERR_WORKSPACE.  Every call
 * uses the same array and leaves its contents there; the call clears what it
 * accumulates into, but two calls that overlap on the GPU (different streams
 * or host threads) race on the array.  Each call looks up the array's device
 * address (cudaGetSymbolAddress, with the caller's device current), which
 * allocates nothing.
 * Errors: CX_ERR_INVALID_ARG, CX_ERR_WORKSPACE (too large), CX_ERR_CUDA. */
#define CX_STATIC_SCRATCH_BYTES (64u << 20)
cx_status cx_forward_static(const cx_problem_desc* desc, const void* u0, const void* v0, const void* g,
                            double* J_dev, void* uN, void* vN, int* status_dev, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Domain decomposition of one problem (2-D blocks over several devices or
 * processes).  Collision is local and streaming reaches only the nearest
 * neighbours (Sec. 3.1; the adjoint of Sec. 3.2.1 streams along -e_i), so a
 * block needs, before each step, the populations that cross its faces and
 * corners.  A block of lx x ly nodes is created as an (lx + 2) x (ly + 2)
 * problem with halo = 1 whose descriptor fields are the global fields over
 * the block and its one-node frame (periodic images at the edges of the
 * global grid); its frame nodes are ghosts, filled from the neighbouring
 * blocks.  The cost, gradient norms and control penalty of a block cover its
 * interior only; the sum over blocks is the problem's.
 *
 * Kinds of exchanged data: */
enum { CX_HALO_FWD = 0,  /* forward (and recompute) populations, [2][Q][plane] */
       CX_HALO_ADJ = 1,  /* adjoint populations, [2][Q][plane]                 */
       CX_HALO_SEED = 2  /* a node field [plane]: the terminal adjoint seed     */ };
/* Exchange callback: called on the calling host thread after every lattice
 * step of cx_forward / cx_forward_trial / cx_adjoint / cx_adjoint_vjp (kind
 * FWD or ADJ, `field` = the populations the step wrote) and after the
 * forward's terminal moments (kind SEED, `field` = the terminal seed
 * u^N - u_target).  Before returning it must queue on `stream` the work that
 * fills the ghost frame of `field` from the neighbouring blocks, usually
 * cx_halo_pack, a transfer of the slots, and cx_halo_unpack.  A non-zero
 * return ends the call with that status. */
typedef cx_status (*cx_halo_fn)(void* user, int kind, void* field, cudaStream_t stream);
/* Install (fn != NULL) or remove the callback of a problem created with
 * halo = 1.  On such a problem cx_step, cx_cg_step, cx_lma_step, cx_tlm and
 * cx_cadjoint return CX_ERR_INVALID_ARG: their line searches and dot
 * products need sums over all blocks (the caller's). */
cx_status cx_set_halo_exchange(cx_problem* p, cx_halo_fn fn, void* user);
/* Slots: direction d = 1..8 is the neighbour at offset e_d (E, N, W, S, NE,
 * NW, SW, SE).  Send slot d holds the interior cells along side d (a column
 * of ly, a row of lx, or one corner cell) for the planes the neighbour pulls
 * across that side: forward populations moving toward d (3 + 3 per face and
 * 1 + 1 per corner on D2Q9, 1 + 1 per face on D2Q5), adjoint populations
 * moving away from d, or the node field itself (SEED); each slot is
 * [planes][cells] of T.  The neighbour at e_d receives it as its receive slot
 * opp(d).  Byte offsets of the send slots (send_off[0..7], d = 1..8), of the
 * receive slots (recv_off[0..7]) and the bytes of either buffer (*bytes);
 * any pointer may be NULL.  Host call.  Errors: CX_ERR_INVALID_ARG (halo = 0
 * or an unknown kind). */
cx_status cx_halo_layout(const cx_problem* p, int kind, size_t* send_off, size_t* recv_off, size_t* bytes);
/* Gather the send slots of `field` (device, the kind's layout) into `send`
 * (device, cx_halo_layout bytes); scatter the receive slots of `recv` into
 * the ghost frame of `field`.  Asynchronous on the problem's stream. */
cx_status cx_halo_pack(cx_problem* p, int kind, const void* field, void* send);
cx_status cx_halo_unpack(cx_problem* p, int kind, const void* recv, void* field);
/* Forward solve at the trial control g - lam E (E device T [W][ctrl], each
 * value rounded as cx_control_axpy rounds it), as a line-search trial of
 * cx_step computes it; J_dev as for cx_forward.  The state is then that of
 * the trial control. */
cx_status cx_forward_trial(cx_problem* p, const void* g, const void* E, double lam, double* J_dev);
/* g <- g - lam E on the device (T [W][ctrl]), the accepted update of a line
 * search.  Asynchronous. */
cx_status cx_control_axpy(cx_problem* p, void* g, const void* E, double lam);

/* Release the host object (the workspace stays the caller's). */
cx_status cx_destroy(cx_problem* p);

/* Static text for a status code. */
const char* cx_status_string(cx_status s);

#ifdef __cplusplus
}
#endif
#endif /* CXLBM_H */
