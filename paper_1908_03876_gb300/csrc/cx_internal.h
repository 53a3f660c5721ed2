// cx_internal.h -- shared definitions of the library's host code and kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/cxlbm.h"

namespace cx {

// Per-problem constants, passed by value to every kernel.
struct CxConst {
    int nx, ny;
    long long plane;      // elements per node plane (nx*ny rounded up to 64)
    int Q, n_steps;
    int aniso, adv, has_solid;
    int ctrl_full;                    // control window = whole grid, no mask
    int halo;                         // outer one-node frame is a halo of ghost nodes (sub-domain)
    int bb_copy;                      // the adjoint's solid nodes carry bounce-back copies: every adjoint step
                                      // also writes each psi_i(x) whose next pull comes back to x (x - e_i
                                      // solid) into plane opp(i) at the solid node x - e_i, where the next
                                      // step's row windows hold it (solid grids without a halo)
    int cx0, cy0, cnx, cny;
    int source_order;
    double tau, d_u, d_v, chi, r_vu, r_vv, alpha;
    double s[7];
    double Ku[3], Kv[3];              // CONST tensors -> K (k11, k12, k22)
    double ku_bar, ku_d, kv_bar, kv_d; // ROTATED: K = kbar I + kd R(2t)-reflection
    const void* theta;                // T [plane]           (ROTATED)
    const void* Kfield;               // T [6][plane]        (FIELD)
    const void* a;                    // T [ny][2] or [2][plane]
    const uint8_t* solid;             // [plane] or null
    const uint8_t* bounce;            // [plane] with solid nodes: at a fluid node bit i-1 is set when x - e_i is
                                      // solid (the pull of direction i bounces back); 0 at solid nodes; or null
    const uint8_t* cmask;             // [cny*cnx] window & mask & fluid, or null
};

// The same constants in the kernels' own precision, precomputed on the host
// so that no FP64 arithmetic or conversion runs per node in FP32 mode.
template <typename T> struct KConst {
    T s[7];
    T sn[9];                 // rate of moment k times 1/|M row k|^2 (0 for the flux moments)
    T invn_jx, invn_jy;      // 1/|M row| of the two flux moments
    T chi, r_vu, r_vv, tau, inv_tau;
    T gsc;                   // -1 / (d_v Cs^2) = -3 / d_v
    T asc;                   //  1 / (d_v Cs^2) =  3 / d_v
    T d_u, d_v;
    T Ku[3], Kv[3];
    T ku_bar, ku_d, kv_bar, kv_d;
    T two_alpha;
    T c_first, c_now, c_prev; // source coefficients: step 0, steps >= 1 (Phi^n, Phi^{n-1})
};

// bits of a problem's device status word
enum { ST_UNSTABLE = 1, ST_TIMEOUT = 2 };

template <typename T> struct FwdArgs {
    const T* pin[18];    // plane j of [2][Q][plane] populations read (pull), or f^0 read locally at n = 0
    T* pout[18];         // plane j of the post-collision populations of step n
    T* phi;              // [plane] Phi^{n-1} in, Phi^n out (node-local, in place)
    T* phi_ckpt;         // [plane] copy of Phi^n when Pout is a checkpoint slot, else null
    const T* g;          // [cny*cnx] control g^n, or null (zero control)
    const T* E;          // [cny*cnx] gradient for trial controls g - lam E, or null
    T lam;
    T* tape;             // [3][plane] (u^n, G_x^n, G_y^n) or null
    double* gsq_part;    // per-warp partial of sum (g^n)^2 (accumulated over steps), or null
    int* status;         // status word (ST_TIMEOUT from the bulk-staged kernel), or null
    unsigned tx_pad;     // test mode of the bulk-staged kernel: bytes each stage expects beyond its copies
    int n;               // time step index
    __device__ __forceinline__ const T* in(int j) const { return pin[j]; }
    __device__ __forceinline__ T* out(int j) const { return pout[j]; }
};

template <typename T> struct TlmArgs {
    const T* pin[18];    // plane j of the tangent populations dP^{n-1} (pulled), or df^0 read locally at n = 0
    T* pout[18];         // plane j of dP^n
    T* dphi;             // [plane] dPhi^{n-1} in, dPhi^n out
    const T* tape;       // [3][plane] base (u^n, G_x^n, G_y^n)
    const T* dg;         // [cny*cnx] direction dg^n, or null
    int* status;         // status word (ST_TIMEOUT from the bulk-staged kernel), or null
    unsigned tx_pad;     // test mode of the bulk-staged kernel: bytes each stage expects beyond its copies
    int n;
    __device__ __forceinline__ const T* in(int j) const { return pin[j]; }
    __device__ __forceinline__ T* out(int j) const { return pout[j]; }
};

template <typename T> struct CadjArgs {
    const T* pin[18];    // plane j of the continuous-adjoint populations (pulled); unused at the first step
    T* pout[18];
    const T* w0;         // [plane] u~ at s = 0 (u^N - u_target), first step only
    const T* tape;       // [3][plane] forward (u^n, G_x^n, G_y^n)
    const T* g;          // [cny*cnx] g^n or null
    T* dJdg;             // [cny*cnx] gradient of control step n (window slot)
    double* e2_part;
    double* emax_part;
    int n;
    int first;           // n == N-1: populations phi^eq(w0, -a), 0
    int accum, norm;     // time windows, as the discrete adjoint
    int* status;         // status word (ST_TIMEOUT from the bulk-staged kernel), or null
    unsigned tx_pad;     // test mode of the bulk-staged kernel: bytes each stage expects beyond its copies
    __device__ __forceinline__ const T* in(int j) const { return pin[j]; }
    __device__ __forceinline__ T* out(int j) const { return pout[j]; }
};

template <typename T> struct AdjArgs {
    const T* rin[18];    // plane j of psi^{n+1} ([2][Q][plane]); unused at the terminal step
    const T* wu;         // terminal seeds psi^N_u,i = wu(x), psi^N_v,i = wv(x) (terminal step only)
    const T* wv;
    T* rout[18];         // plane j of psi^n
    const T* tape;       // [3][plane] (u^n, G_x^n, G_y^n)
    T* sigma;            // [plane] sigma^{n+1} in, sigma^n out
    const T* g;          // [cny*cnx] g^n or null
    T* dJdg;             // [cny*cnx] output dJ/dg^n
    double* e2_part;     // per-warp partial of sum E^2 (accumulated over steps)
    double* emax_part;   // per-warp partial of max |E| (accumulated over steps)
    int* status;         // status word (ST_TIMEOUT from the bulk-staged kernel), or null
    unsigned tx_pad;     // test mode of the bulk-staged kernel: bytes each stage expects beyond its copies
    int n;
    int terminal;        // n == N-1: psi^{n+1} is the broadcast seed
    int accum;           // time-windowed control: add to the window's gradient (not its last step)
    int norm;            // add this step's gradient values to the norm partials (window complete)
    __device__ __forceinline__ const T* in(int j) const { return rin[j]; }
    __device__ __forceinline__ T* out(int j) const { return rout[j]; }
};

struct Launch {
    dim3 grid, block;
    int row_windows = 1;   // steps that qualify use the row-window (bulk copy) kernels; 2: their
                           // test mode, every stage wait runs out (timeout path)
    unsigned rows_grid = 0; // blocks of the row-window kernels (0: grid.x)
};

// kernel launchers (cx_forward.cu / cx_adjoint.cu / cx_misc.cu), one per precision
template <typename T> KConst<T> make_kconst(const CxConst& C, int Q);
template <typename T>
cudaError_t launch_forward(const CxConst& C, const KConst<T>& K, const FwdArgs<T>& A, const Launch& L, cudaStream_t s);
template <typename T>
cudaError_t launch_adjoint(const CxConst& C, const KConst<T>& K, const AdjArgs<T>& A, const Launch& L, cudaStream_t s);
// resident blocks per SM of the row-window forward / adjoint kernels
template <typename T> int forward_rows_occupancy(int Q, int threads);
template <typename T> int adjoint_rows_occupancy(int Q, int threads);
template <typename T>
cudaError_t launch_init(const CxConst& C, const double* u0d, const double* v0d, const T* u0, const T* v0, T* P,
                        const Launch& L, cudaStream_t s);
template <typename T>
cudaError_t launch_final(const CxConst& C, const T* Pin, const T* u_tgt, T* uN, T* vN, T* wu, double* cost_part,
                         const Launch& L, cudaStream_t s);
cudaError_t launch_finalize(const double* part_a, int na, const double* part_b, int nb, double scale_b, double* out,
                            int* status, int status_bit, int mode, cudaStream_t s);
// resident blocks per SM of the per-thread forward kernel
template <typename T> int forward_occupancy(int Q, int threads);
template <typename T>
cudaError_t launch_cadj(const CxConst& C, const KConst<T>& K, const CadjArgs<T>& A, const Launch& L, cudaStream_t s);
template <typename T>
cudaError_t launch_tlm(const CxConst& C, const KConst<T>& K, const TlmArgs<T>& A, const Launch& L, cudaStream_t s);
// resident blocks per SM of the per-thread adjoint kernel (bb: the form that
// writes bounce-back copies)
template <typename T> int adjoint_occupancy(int Q, int threads, bool bb = false);
template <typename T>
cudaError_t launch_axpy(T* g, const T* E, T lam, size_t n, cudaStream_t s);
template <typename T>
cudaError_t launch_lincomb(T* out, const T* a, T alpha, const T* b, size_t n, cudaStream_t s);
template <typename T>
cudaError_t launch_dots(const T* const (&x)[4], const T* const (&y)[4], size_t n, double* part, double* out,
                        cudaStream_t s);
template <typename T>
cudaError_t launch_convert(const double* in, T* out, size_t n, cudaStream_t s);
template <typename T>
cudaError_t launch_setup_fields(const CxConst& C, const cx_problem_desc& d, T* theta, T* Kfield, T* a, T* u_tgt,
                                uint8_t* solid, uint8_t* cmask, uint8_t* bounce, cudaStream_t s);

} // namespace cx
