// cx_misc.cu -- initial equilibrium, final moments and cost, fixed-order
// FP64 reductions, control update and field set-up kernels.
#include <algorithm>
#include <cmath>

#include "cx_device.cuh"

namespace cx {

template <typename T> KConst<T> make_kconst(const CxConst& C, int Q);

// f^0 = phi^eq(Theta_0) for both species (eq. phieq; the initial condition of
// the forward solve).  Reads FP64 (u0d) or T (u0) initial fields.
template <typename T, int Q>
__global__ void k_init(const CxConst C, const KConst<T> KC, const double* u0d, const double* v0d, const T* u0,
                       const T* v0, T* P) {
    using L = Lat<Q>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= C.nx || y >= C.ny) return;
    const int k = y * C.nx + x;
    const size_t pl = (size_t)C.plane;
    const bool solid = C.has_solid && C.solid[k];
    NodeCoef<T> nc;
    node_coef<T>(C, KC, x, y, k, nc);
    const T Tu = solid ? T(0) : (u0d ? T(u0d[k]) : u0[k]);
    const T Tv = solid ? T(0) : (v0d ? T(v0d[k]) : v0[k]);
    const T a2 = nc.ax * nc.ax + nc.ay * nc.ay;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T ea = nc.ax * T(L::ex(i)) + nc.ay * T(L::ey(i));
        const T e2 = T(L::ex(i) * L::ex(i) + L::ey(i) * L::ey(i));
        const T base = T(1) + T(3) * ea + T(4.5) * (ea * ea - a2 * T(1.0 / 3.0));
        const T au = base + T(4.5) * (T(C.d_u) - T(1)) * (e2 - T(2.0 / 3.0)) * T(1.0 / 3.0);
        const T av = base + T(4.5) * (T(C.d_v) - T(1)) * (e2 - T(2.0 / 3.0)) * T(1.0 / 3.0);
        P[i * pl + k] = T(L::w(i)) * au * Tu;
        P[(Q + i) * pl + k] = T(L::w(i)) * av * Tv;
    }
}

template <typename T>
cudaError_t launch_init(const CxConst& C, const double* u0d, const double* v0d, const T* u0, const T* v0, T* P,
                        const Launch& L, cudaStream_t s) {
    const KConst<T> K = make_kconst<T>(C, C.Q);
    if (C.Q == 9)
        k_init<T, 9><<<L.grid, L.block, 0, s>>>(C, K, u0d, v0d, u0, v0, P);
    else
        k_init<T, 5><<<L.grid, L.block, 0, s>>>(C, K, u0d, v0d, u0, v0, P);
    return cudaGetLastError();
}

// u^N = sum_i f^N_u,i, v^N likewise (UGS), with f^N pulled from P^{N-1};
// wu = u^N - u_target seeds the adjoint (final condition of CAE); the block
// partial of 1/2 sum (u^N - u_target)^2 goes to cost_part in FP64.
template <typename T, int Q>
__global__ void __launch_bounds__(256) k_final(const CxConst C, const T* Pin, const T* u_tgt, T* uN, T* vN, T* wu,
                                                double* cost_part) {
    using L = Lat<Q>;
    __shared__ double red[32];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    double cst = 0.0;
    if (x < C.nx && y < C.ny) {
        const int k = y * C.nx + x;
        const size_t pl = (size_t)C.plane;
        T su = T(0), sv = T(0), w = T(0);
        const bool ghost = C.halo && (x == 0 || y == 0 || x == C.nx - 1 || y == C.ny - 1);
        if (!(C.has_solid && C.solid[k]) && !ghost) {
            const int xm = x == 0 ? C.nx - 1 : x - 1, xp = x == C.nx - 1 ? 0 : x + 1;
            const int ym = y == 0 ? C.ny - 1 : y - 1, yp = y == C.ny - 1 ? 0 : y + 1;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int xs = L::ex(i) > 0 ? xm : (L::ex(i) < 0 ? xp : x);
                const int ys = L::ey(i) > 0 ? ym : (L::ey(i) < 0 ? yp : y);
                const int ks = ys * C.nx + xs;
                if (C.has_solid && i != 0 && C.solid[ks]) {
                    su += Pin[L::opp(i) * pl + k];
                    sv += Pin[(Q + L::opp(i)) * pl + k];
                } else {
                    su += Pin[i * pl + ks];
                    sv += Pin[(Q + i) * pl + ks];
                }
            }
            w = su - u_tgt[k];
            cst = 0.5 * (double)w * (double)w;
        }
        uN[k] = su;
        vN[k] = sv;
        wu[k] = w;
    }
    const double b = block_sum(cst, red);
    if (threadIdx.x == 0 && threadIdx.y == 0) cost_part[blockIdx.x + gridDim.x * blockIdx.y] = b;
}

template <typename T>
cudaError_t launch_final(const CxConst& C, const T* Pin, const T* u_tgt, T* uN, T* vN, T* wu, double* cost_part,
                         const Launch& L, cudaStream_t s) {
    if (C.Q == 9)
        k_final<T, 9><<<L.grid, L.block, 0, s>>>(C, Pin, u_tgt, uN, vN, wu, cost_part);
    else
        k_final<T, 5><<<L.grid, L.block, 0, s>>>(C, Pin, u_tgt, uN, vN, wu, cost_part);
    return cudaGetLastError();
}

// One block, fixed order: thread t sums parts t, t+256, ... then a fixed tree.
// mode 0: out = sum(a) + scale_b * sum(b)          (cost J)
// mode 1: out[0] = sum(a), out[1] = max(b)         (gradient norms)
// A non-finite result sets status_bit in *status.
__global__ void __launch_bounds__(256) k_finalize(const double* a, int na, const double* b, int nb, double scale_b,
                                                   double* out, int* status, int status_bit, int mode) {
    __shared__ double sa[256], sb[256];
    const int t = threadIdx.x;
    double ra = 0.0, rb = 0.0;
    for (int i = t; i < na; i += 256) ra += a[i];
    if (b)
        for (int i = t; i < nb; i += 256) rb = (mode == 1) ? fmax(rb, b[i]) : rb + b[i];
    sa[t] = ra;
    sb[t] = rb;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (t < h) {
            sa[t] += sa[t + h];
            sb[t] = (mode == 1) ? fmax(sb[t], sb[t + h]) : sb[t] + sb[t + h];
        }
        __syncthreads();
    }
    if (t == 0) {
        if (mode == 0) {
            const double J = sa[0] + scale_b * sb[0];
            out[0] = J;
            if (!isfinite(J)) atomicOr(status, status_bit);
        } else {
            out[0] = sa[0];
            out[1] = sb[0];
            if (!isfinite(sa[0]) || !isfinite(sb[0])) atomicOr(status, status_bit);
        }
    }
}

cudaError_t launch_finalize(const double* a, int na, const double* b, int nb, double scale_b, double* out,
                            int* status, int status_bit, int mode, cudaStream_t s) {
    k_finalize<<<1, 256, 0, s>>>(a, na, b, nb, scale_b, out, status, status_bit, mode);
    return cudaGetLastError();
}

// out <- a + alpha b (fused; the CG trial control g - lam P and the direction
// update P <- G + r P)
template <typename T> __global__ void k_lincomb(T* out, const T* a, T alpha, const T* b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = fma(alpha, b[i], a[i]);
}

template <typename T> cudaError_t launch_lincomb(T* out, const T* a, T alpha, const T* b, size_t n, cudaStream_t s) {
    int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
    k_lincomb<T><<<std::max(blocks, 1), 256, 0, s>>>(out, a, alpha, b, n);
    return cudaGetLastError();
}

// Four dot products <x_j, y_j> (j < 4, FP64 products and sums): block
// partials part[j][block], then one block sums each j in a fixed order.
constexpr int DOT_BLOCKS = 512;
template <typename T>
__global__ void __launch_bounds__(256) k_dots(const T* x0, const T* y0, const T* x1, const T* y1, const T* x2,
                                               const T* y2, const T* x3, const T* y3, size_t n, double* part) {
    __shared__ double sh[4][256];
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        s[0] = fma((double)x0[i], (double)y0[i], s[0]);
        s[1] = fma((double)x1[i], (double)y1[i], s[1]);
        s[2] = fma((double)x2[i], (double)y2[i], s[2]);
        s[3] = fma((double)x3[i], (double)y3[i], s[3]);
    }
    for (int j = 0; j < 4; ++j) sh[j][threadIdx.x] = s[j];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int j = 0; j < 4; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int j = 0; j < 4; ++j) part[j * DOT_BLOCKS + blockIdx.x] = sh[j][0];
}

__global__ void __launch_bounds__(256) k_dots_final(const double* part, double* out) {
    __shared__ double sh[256];
    const int j = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < DOT_BLOCKS; i += 256) s += part[j * DOT_BLOCKS + i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = sh[0];
}

template <typename T>
cudaError_t launch_dots(const T* const (&x)[4], const T* const (&y)[4], size_t n, double* part, double* out,
                        cudaStream_t s) {
    k_dots<T><<<DOT_BLOCKS, 256, 0, s>>>(x[0], y[0], x[1], y[1], x[2], y[2], x[3], y[3], n, part);
    k_dots_final<<<4, 256, 0, s>>>(part, out);
    return cudaGetLastError();
}

// g <- g - lam E (accepted Armijo step)
template <typename T> __global__ void k_axpy(T* g, const T* E, T lam, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        g[i] = fma(-lam, E[i], g[i]); // bit-identical to the trial control of the forward
}

template <typename T> cudaError_t launch_axpy(T* g, const T* E, T lam, size_t n, cudaStream_t s) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_axpy<T><<<blocks, 256, 0, s>>>(g, E, lam, n);
    return cudaGetLastError();
}

template <typename T> __global__ void k_convert(const double* in, T* out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = T(in[i]);
}

template <typename T> cudaError_t launch_convert(const double* in, T* out, size_t n, cudaStream_t s) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_convert<T><<<blocks, 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

// Per-node set-up: angle / K fields, convection, target, solid copy, and the
// combined control mask (window & ctrl_mask & fluid).
// K from D = d Cs^2 tau (K^-1 - I/2): K = (D / (d Cs^2 tau) + I/2)^-1 (2x2 inverse).
template <typename T>
__global__ void k_setup(const CxConst C, const double* theta_in, const double* Du_in, const double* Dv_in,
                        const double* a_in, const double* ut_in, const uint8_t* solid_in, const uint8_t* cmask_in,
                        T* theta, T* Kfield, T* a, T* u_tgt, uint8_t* solid, uint8_t* cmask, uint8_t* bounce) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= C.nx || y >= C.ny) return;
    const int k = y * C.nx + x;
    const size_t pl = (size_t)C.plane;
    if (theta) theta[k] = T(theta_in[k]);
    if (Kfield) {
        const double* Ds[2] = {Du_in, Dv_in};
        const double dd[2] = {C.d_u, C.d_v};
        for (int sp = 0; sp < 2; ++sp) {
            const double sc = 1.0 / (dd[sp] * (1.0 / 3.0) * C.tau);
            const double A00 = Ds[sp][3 * k] * sc + 0.5, A01 = Ds[sp][3 * k + 1] * sc, A11 = Ds[sp][3 * k + 2] * sc + 0.5;
            const double det = A00 * A11 - A01 * A01;
            Kfield[(3 * sp + 0) * pl + k] = T(A11 / det);
            Kfield[(3 * sp + 1) * pl + k] = T(-A01 / det);
            Kfield[(3 * sp + 2) * pl + k] = T(A00 / det);
        }
    }
    if (a && C.adv == CX_ADV_FIELD) {
        a[k] = T(a_in[2 * k]);
        a[pl + k] = T(a_in[2 * k + 1]);
    }
    if (a && C.adv == CX_ADV_ROW && x == 0) {
        a[2 * y] = T(a_in[2 * y]);
        a[2 * y + 1] = T(a_in[2 * y + 1]);
    }
    u_tgt[k] = T(ut_in[k]);
    if (solid) solid[k] = solid_in[k] ? 1 : 0;
    if (bounce) { // which pulls of this fluid node bounce back (halfway bounce-back, periodic neighbours)
        unsigned bits = 0;
        if (!solid_in[k]) {
            const int xm = x == 0 ? C.nx - 1 : x - 1, xp = x == C.nx - 1 ? 0 : x + 1;
            const int ym = y == 0 ? C.ny - 1 : y - 1, yp = y == C.ny - 1 ? 0 : y + 1;
            for (int i = 1; i < C.Q; ++i) {
                const int ex = Lat<9>::ex(i), ey = Lat<9>::ey(i); // D2Q5 uses the first five D2Q9 velocities
                const int xs = ex > 0 ? xm : (ex < 0 ? xp : x), ys = ey > 0 ? ym : (ey < 0 ? yp : y);
                if (solid_in[ys * C.nx + xs]) bits |= 1u << (i - 1);
            }
        }
        bounce[k] = (uint8_t)bits;
    }
    if (cmask) {
        const int cx = x - C.cx0, cy = y - C.cy0;
        if (cx >= 0 && cy >= 0 && cx < C.cnx && cy < C.cny) {
            const int c = cy * C.cnx + cx;
            uint8_t m = 1;
            if (cmask_in && !cmask_in[c]) m = 0;
            if (solid_in && solid_in[k]) m = 0;
            cmask[c] = m;
        }
    }
}

template <typename T>
cudaError_t launch_setup_fields(const CxConst& C, const cx_problem_desc& d, T* theta, T* Kfield, T* a, T* u_tgt,
                                uint8_t* solid, uint8_t* cmask, uint8_t* bounce, cudaStream_t s) {
    dim3 block(32, 8), grid((C.nx + 31) / 32, (C.ny + 7) / 8);
    k_setup<T><<<grid, block, 0, s>>>(C, d.theta, d.D_u_field, d.D_v_field, d.a, d.u_target, d.solid, d.ctrl_mask,
                                      theta, Kfield, a, u_tgt, solid, cmask, bounce);
    return cudaGetLastError();
}

template <int Q> static void fold_rates(const CxConst& C, double* sn, double* jx, double* jy) {
    for (int k = 0; k < Q; ++k) {
        const int r = rate_index<Q>(k);
        sn[k] = r >= 0 ? C.s[r] * Lat<Q>::inv_n(k) : 0.0;
    }
    *jx = Lat<Q>::inv_n(Lat<Q>::JX);
    *jy = Lat<Q>::inv_n(Lat<Q>::JY);
}

template <typename T> KConst<T> make_kconst(const CxConst& C, int Q) {
    KConst<T> K{};
    for (int i = 0; i < 7; ++i) K.s[i] = T(C.s[i]);
    double sn[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, jx = 0.0, jy = 0.0;
    if (Q == 9)
        fold_rates<9>(C, sn, &jx, &jy);
    else
        fold_rates<5>(C, sn, &jx, &jy);
    for (int k = 0; k < 9; ++k) K.sn[k] = T(sn[k]);
    K.invn_jx = T(jx);
    K.invn_jy = T(jy);
    K.chi = T(C.chi);
    K.r_vu = T(C.r_vu);
    K.r_vv = T(C.r_vv);
    K.tau = T(C.tau);
    K.inv_tau = T(1.0 / C.tau);
    K.gsc = T(-3.0 / C.d_v);
    K.asc = T(3.0 / C.d_v);
    K.d_u = T(C.d_u);
    K.d_v = T(C.d_v);
    for (int i = 0; i < 3; ++i) {
        K.Ku[i] = T(C.Ku[i]);
        K.Kv[i] = T(C.Kv[i]);
    }
    K.ku_bar = T(C.ku_bar);
    K.ku_d = T(C.ku_d);
    K.kv_bar = T(C.kv_bar);
    K.kv_d = T(C.kv_d);
    K.two_alpha = T(2.0 * C.alpha);
    // tau Phi^n + (tau/2)(Phi^n - Phi^{n-1}); Phi^{-1} := Phi^0 at step 0
    K.c_first = T(C.tau);
    K.c_now = C.source_order == 1 ? T(C.tau) : T(1.5 * C.tau);
    K.c_prev = C.source_order == 1 ? T(0) : T(-0.5 * C.tau);
    return K;
}

#define CX_INST(T)                                                                                                   \
    template KConst<T> make_kconst<T>(const CxConst&, int);                                                               \
    template cudaError_t launch_init<T>(const CxConst&, const double*, const double*, const T*, const T*, T*,        \
                                        const Launch&, cudaStream_t);                                                 \
    template cudaError_t launch_final<T>(const CxConst&, const T*, const T*, T*, T*, T*, double*, const Launch&,      \
                                         cudaStream_t);                                                               \
    template cudaError_t launch_axpy<T>(T*, const T*, T, size_t, cudaStream_t);                                 \
    template cudaError_t launch_lincomb<T>(T*, const T*, T, const T*, size_t, cudaStream_t);                         \
    template cudaError_t launch_dots<T>(const T* const (&)[4], const T* const (&)[4], size_t, double*, double*,      \
                                        cudaStream_t);                                                               \
    template cudaError_t launch_convert<T>(const double*, T*, size_t, cudaStream_t);                                 \
    template cudaError_t launch_setup_fields<T>(const CxConst&, const cx_problem_desc&, T*, T*, T*, T*, uint8_t*,    \
                                                uint8_t*, uint8_t*, cudaStream_t);
CX_INST(float)
CX_INST(double)

} // namespace cx
