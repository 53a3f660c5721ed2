// cx_device.cuh -- device-side building blocks of the MRT / AMRT kernels.
//
// Lattices (Sec. 3.1): D2Q9 velocities e_0..e_8 and weights (4/9, 1/9 x4,
// 1/36 x4), the Gram-Schmidt moment matrix M0 (E0 = I for c = 1) with moment
// order (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy); D2Q5 uses the first five
// D2Q9 velocities, weights (1/3, 1/6 x4) and moments (rho, j_x, j_y, e, p_xx).
// M0 has orthogonal rows, so M^-1 = M^T diag(1/|row_k|^2).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "cx_internal.h"

namespace cx {

template <int Q> struct Lat;

template <> struct Lat<9> {
    static constexpr int Q = 9;
    __host__ __device__ static constexpr int ex(int i) {
        return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
    }
    __host__ __device__ static constexpr int ey(int i) {
        return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
    }
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : (i <= 4 ? ((i - 1 + 2) % 4) + 1 : ((i - 5 + 2) % 4) + 5);
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    // M0 (Sec. 3.1): row k, column i
    __host__ __device__ static constexpr int M(int k, int i) {
        constexpr int t[9][9] = {{1, 1, 1, 1, 1, 1, 1, 1, 1},
                                 {-4, -1, -1, -1, -1, 2, 2, 2, 2},
                                 {4, -2, -2, -2, -2, 1, 1, 1, 1},
                                 {0, 1, 0, -1, 0, 1, -1, -1, 1},
                                 {0, -2, 0, 2, 0, 1, -1, -1, 1},
                                 {0, 0, 1, 0, -1, 1, 1, -1, -1},
                                 {0, 0, -2, 0, 2, 1, 1, -1, -1},
                                 {0, 1, -1, 1, -1, 0, 0, 0, 0},
                                 {0, 0, 0, 0, 0, 1, -1, 1, -1}};
        return t[k][i];
    }
    // 1 / |row_k|^2
    __host__ __device__ static constexpr double inv_n(int k) {
        constexpr double t[9] = {1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 6, 1.0 / 12, 1.0 / 6, 1.0 / 12, 1.0 / 4, 1.0 / 4};
        return t[k];
    }
    // indices of the two flux moments j_x, j_y inside the moment vector
    static constexpr int JX = 3, JY = 5;
    // moment images of the source shapes (M0 applied to w_i, w_i e_x,i and w_i e_y,i):
    // a source s_i = w_i (a + b.e_i) has moments a src_A(k) + b_x src_Bx(k) + b_y src_By(k)
    __host__ __device__ static constexpr double src_A(int k) {
        constexpr double t[9] = {1, -2, 1, 0, 0, 0, 0, 0, 0};
        return t[k];
    }
    __host__ __device__ static constexpr double src_Bx(int k) {
        constexpr double t[9] = {0, 0, 0, 1.0 / 3, -1.0 / 3, 0, 0, 0, 0};
        return t[k];
    }
    __host__ __device__ static constexpr double src_By(int k) {
        constexpr double t[9] = {0, 0, 0, 0, 0, 1.0 / 3, -1.0 / 3, 0, 0};
        return t[k];
    }
};

template <> struct Lat<5> {
    static constexpr int Q = 5;
    __host__ __device__ static constexpr int ex(int i) { return i == 1 ? 1 : (i == 3 ? -1 : 0); }
    __host__ __device__ static constexpr int ey(int i) { return i == 2 ? 1 : (i == 4 ? -1 : 0); }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : ((i - 1 + 2) % 4) + 1; }
    __host__ __device__ static constexpr double w(int i) { return i == 0 ? 1.0 / 3.0 : 1.0 / 6.0; }
    __host__ __device__ static constexpr int M(int k, int i) {
        constexpr int t[5][5] = {{1, 1, 1, 1, 1}, {0, 1, 0, -1, 0}, {0, 0, 1, 0, -1}, {-4, 1, 1, 1, 1}, {0, 1, -1, 1, -1}};
        return t[k][i];
    }
    __host__ __device__ static constexpr double inv_n(int k) {
        constexpr double t[5] = {1.0 / 5, 1.0 / 2, 1.0 / 2, 1.0 / 20, 1.0 / 4};
        return t[k];
    }
    static constexpr int JX = 1, JY = 2;
    __host__ __device__ static constexpr double src_A(int k) {
        constexpr double t[5] = {1, 0, 0, -2.0 / 3, 0};
        return t[k];
    }
    __host__ __device__ static constexpr double src_Bx(int k) {
        constexpr double t[5] = {0, 1.0 / 3, 0, 0, 0};
        return t[k];
    }
    __host__ __device__ static constexpr double src_By(int k) {
        constexpr double t[5] = {0, 0, 1.0 / 3, 0, 0};
        return t[k];
    }
};

// Moment transforms.  m = M f and its transpose out = M^T r, written for D2Q9
// with the pair sums/differences of opposite directions (f1 +- f3, f2 +- f4,
// f5 +- f7, f6 +- f8), which M0's rows are built from; the generic table loop
// serves D2Q5.
template <typename T, int Q> struct Transform {
    __host__ __device__ static inline void moments(const T (&f)[Q], T (&m)[Q]) {
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            T s = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if (Lat<Q>::M(k, i) != 0) s += T(Lat<Q>::M(k, i)) * f[i];
            m[k] = s;
        }
    }
    __host__ __device__ static inline void transpose(const T (&r)[Q], T (&o)[Q]) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            T s = T(0);
#pragma unroll
            for (int k = 0; k < Q; ++k)
                if (Lat<Q>::M(k, i) != 0) s += T(Lat<Q>::M(k, i)) * r[k];
            o[i] = s;
        }
    }
    // transpose of (0, r_1, ..., r_{Q-1}): r[0] is not read
    __host__ __device__ static inline void transpose0(const T (&r)[Q], T (&o)[Q]) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            T s = T(0);
#pragma unroll
            for (int k = 1; k < Q; ++k)
                if (Lat<Q>::M(k, i) != 0) s += T(Lat<Q>::M(k, i)) * r[k];
            o[i] = s;
        }
    }
};
template <typename T> struct Transform<T, 9> {
    __host__ __device__ static inline void moments(const T (&f)[9], T (&m)[9]) {
        const T a = f[1] + f[3], b = f[2] + f[4], c = f[5] + f[7], d = f[6] + f[8];
        const T ax = f[1] - f[3], by = f[2] - f[4], cd = f[5] - f[7], dd = f[6] - f[8];
        const T ab = a + b, cs = c + d;
        m[0] = f[0] + ab + cs;
        m[1] = T(-4) * f[0] - ab + T(2) * cs;
        m[2] = T(4) * f[0] - T(2) * ab + cs;
        const T p = cd - dd, q = cd + dd;
        m[3] = ax + p;
        m[4] = T(-2) * ax + p;
        m[5] = by + q;
        m[6] = T(-2) * by + q;
        m[7] = a - b;
        m[8] = c - d;
    }
    __host__ __device__ static inline void transpose(const T (&r)[9], T (&o)[9]) {
        const T base1 = r[0] - r[1] - T(2) * r[2];
        const T base2 = r[0] + T(2) * r[1] + r[2];
        const T A = base1 + r[7], C = base1 - r[7];
        const T B = r[3] - T(2) * r[4], D = r[5] - T(2) * r[6];
        const T E = base2 + r[8], G = base2 - r[8];
        const T F = r[3] + r[4] + r[5] + r[6], H = r[5] + r[6] - r[3] - r[4];
        o[0] = r[0] - T(4) * r[1] + T(4) * r[2];
        o[1] = A + B;
        o[3] = A - B;
        o[2] = C + D;
        o[4] = C - D;
        o[5] = E + F;
        o[7] = E - F;
        o[6] = G + H;
        o[8] = G - H;
    }
    // transpose of (0, r_1, ..., r_8): r[0] is not read
    __host__ __device__ static inline void transpose0(const T (&r)[9], T (&o)[9]) {
        const T base1 = -r[1] - T(2) * r[2];
        const T base2 = T(2) * r[1] + r[2];
        const T A = base1 + r[7], C = base1 - r[7];
        const T B = r[3] - T(2) * r[4], D = r[5] - T(2) * r[6];
        const T E = base2 + r[8], G = base2 - r[8];
        const T F = r[3] + r[4] + r[5] + r[6], H = r[5] + r[6] - r[3] - r[4];
        o[0] = T(4) * (r[2] - r[1]);
        o[1] = A + B;
        o[3] = A - B;
        o[2] = C + D;
        o[4] = C - D;
        o[5] = E + F;
        o[7] = E - F;
        o[6] = G + H;
        o[8] = G - H;
    }
};

// relaxation rate of non-flux moment k (Pi = diag(s0,s1,s2) + K-block + diag(s4,s5,s6);
// the q_x rate is s3).  D2Q5: (rho, -, -, e, p_xx) -> (s0, s1, s5).
template <int Q> __host__ __device__ inline int rate_index(int k);
template <> __host__ __device__ inline int rate_index<9>(int k) {
    return k == 0 ? 0 : k == 1 ? 1 : k == 2 ? 2 : k == 4 ? 3 : k == 6 ? 4 : k == 7 ? 5 : k == 8 ? 6 : -1;
}
template <> __host__ __device__ inline int rate_index<5>(int k) { return k == 0 ? 0 : k == 3 ? 1 : k == 4 ? 5 : -1; }

// ------------------------------------------------------------ per-node data

template <typename T> struct NodeCoef {
    T Ku0, Ku1, Ku2; // K_u = [[Ku0, Ku1], [Ku1, Ku2]]
    T Kv0, Kv1, Kv2;
    T ax, ay;        // convection velocity a(x)
};

template <typename T> __device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// sin and cos of 2t: libm in FP64; in FP32 a reduction to [-pi, pi] then the
// hardware approximations (absolute error about 1e-6, far below the FP32
// tolerance of the fields).
__device__ __forceinline__ void sincos2(double t, double* s, double* c) { sincos(2.0 * t, s, c); }
__device__ __forceinline__ void sincos2(float t, float* s, float* c) {
    float x = 2.0f * t;
    x = fmaf(-6.28318530717958647692f, rintf(x * 0.15915494309189533577f), x);
    __sincosf(x, s, c);
}

// Node coefficients given the node's angle th (used only for ROTATED tensors).
template <typename T>
__device__ __forceinline__ void node_coef_th(const CxConst& C, const KConst<T>& KC, T th, int y, int k,
                                             NodeCoef<T>& c) {
    if (C.aniso == CX_ANISO_ROTATED) {
        // K = R diag(k1, k2) R^T = kbar I + kd [[cos 2t, sin 2t], [sin 2t, -cos 2t]]
        T s2, c2;
        sincos2(th, &s2, &c2);
        c.Ku0 = KC.ku_bar + KC.ku_d * c2;
        c.Ku1 = KC.ku_d * s2;
        c.Ku2 = KC.ku_bar - KC.ku_d * c2;
        c.Kv0 = KC.kv_bar + KC.kv_d * c2;
        c.Kv1 = KC.kv_d * s2;
        c.Kv2 = KC.kv_bar - KC.kv_d * c2;
    } else if (C.aniso == CX_ANISO_FIELD) {
        const T* K = reinterpret_cast<const T*>(C.Kfield);
        const size_t pl = C.plane;
        c.Ku0 = ldg(K + k);
        c.Ku1 = ldg(K + pl + k);
        c.Ku2 = ldg(K + 2 * pl + k);
        c.Kv0 = ldg(K + 3 * pl + k);
        c.Kv1 = ldg(K + 4 * pl + k);
        c.Kv2 = ldg(K + 5 * pl + k);
    } else {
        c.Ku0 = KC.Ku[0];
        c.Ku1 = KC.Ku[1];
        c.Ku2 = KC.Ku[2];
        c.Kv0 = KC.Kv[0];
        c.Kv1 = KC.Kv[1];
        c.Kv2 = KC.Kv[2];
    }
    if (C.adv == CX_ADV_ROW) {
        const T* a = reinterpret_cast<const T*>(C.a);
        c.ax = ldg(a + 2 * y);
        c.ay = ldg(a + 2 * y + 1);
    } else if (C.adv == CX_ADV_FIELD) {
        const T* a = reinterpret_cast<const T*>(C.a);
        c.ax = ldg(a + k);
        c.ay = ldg(a + C.plane + k);
    } else {
        c.ax = T(0);
        c.ay = T(0);
    }
}

template <typename T>
__device__ __forceinline__ void node_coef(const CxConst& C, const KConst<T>& KC, int x, int y, int k, NodeCoef<T>& c) {
    const T th = (C.aniso == CX_ANISO_ROTATED) ? ldg(reinterpret_cast<const T*>(C.theta) + k) : T(0);
    node_coef_th<T>(C, KC, th, y, k, c);
}


// Moments at unit density of the equilibrium phi^eq = w_i aleph_i Theta
// (eq. phieq with T = a Theta, C = (a a) Theta):
//   aleph_i = 1 + a.e_i / Cs^2 + ((a a) + (d - 1) Cs^2 I) : (e_i e_i - Cs^2 I) / (2 Cs^4).
// D2Q9 uses the paper's closed-form moment listing (m^eq after M0, with
// B = (a a + d Cs^2 I) Theta); D2Q5 sums M w aleph directly.
template <typename T, int Q>
__device__ __forceinline__ void meq_unit(T ax, T ay, T d, T (&mh)[Q]) {
    using L = Lat<Q>;
    if constexpr (Q == 9) {
        const T trB = ax * ax + ay * ay + T(2.0 / 3.0) * d;
        mh[0] = T(1);
        mh[1] = T(-4) + T(3) * trB;
        mh[2] = T(3) - T(3) * trB;
        mh[3] = ax;
        mh[4] = -ax;
        mh[5] = ay;
        mh[6] = -ay;
        mh[7] = ax * ax - ay * ay;
        mh[8] = ax * ay;
    } else {
        T al[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T ea = ax * T(L::ex(i)) + ay * T(L::ey(i));
            const T e2 = T(L::ex(i) * L::ex(i) + L::ey(i) * L::ey(i));
            al[i] = T(1) + T(3) * ea +
                    T(4.5) * (ea * ea - (ax * ax + ay * ay) * T(1.0 / 3.0) + (d - T(1)) * (e2 - T(2.0 / 3.0)) * T(1.0 / 3.0));
        }
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            T s = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if (L::M(k, i) != 0) s += T(L::M(k, i)) * T(L::w(i)) * al[i];
            mh[k] = s;
        }
    }
}

// Pi (m - m^eq) for one species: diagonal rates on non-flux moments, the
// 2x2 block K on (j_x, j_y).
template <typename T, int Q>
__device__ __forceinline__ void relax(const KConst<T>& KC, T K0, T K1, T K2, const T (&dm)[Q], T (&out)[Q]) {
    using L = Lat<Q>;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const int r = rate_index<Q>(k);
        if (r >= 0) out[k] = KC.s[r] * dm[k];
    }
    out[L::JX] = K0 * dm[L::JX] + K1 * dm[L::JY];
    out[L::JY] = K1 * dm[L::JX] + K2 * dm[L::JY];
}

// N^-1 Pi (m - m^eq) with the 1/|row|^2 factors folded into the rates
// (sn[k] = s_k / |row_k|^2).  Pi^T N^-1 has the same entries because K is
// symmetric and both flux rows have the same norm, so the adjoint uses it too.
template <typename T, int Q>
__device__ __forceinline__ void relax_n(const KConst<T>& KC, T K0, T K1, T K2, const T (&dm)[Q], T (&out)[Q]) {
    using L = Lat<Q>;
#pragma unroll
    for (int k = 0; k < Q; ++k)
        if (k != L::JX && k != L::JY) out[k] = KC.sn[k] * dm[k];
    out[L::JX] = (K0 * dm[L::JX] + K1 * dm[L::JY]) * KC.invn_jx;
    out[L::JY] = (K1 * dm[L::JX] + K2 * dm[L::JY]) * KC.invn_jy;
}

// Pi^T lambda (K symmetric, so the block is unchanged; diagonal rates too).
template <typename T, int Q>
__device__ __forceinline__ void relax_T(const KConst<T>& KC, T K0, T K1, T K2, const T (&lam)[Q], T (&out)[Q]) {
    relax<T, Q>(KC, K0, K1, K2, lam, out);
}

// ---------------------------------------------------- deterministic reductions
// (FP64 variants for the FP64 kernels; the FP32 kernels use the compensated
// FP32 helpers below.)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Compensated FP32 arithmetic (an unevaluated pair hi + lo): error-free
// two-sum (Knuth) and fma two-product give sums of squares with FP64-level
// accuracy while the FP32 kernels issue no FP64 instruction per node.
struct CF {
    float hi, lo;
};
__device__ __forceinline__ CF cf_add(CF a, CF b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb) + a.lo + b.lo;
    const float h = s + e;
    return CF{h, e - (h - s)};
}
__device__ __forceinline__ CF cf_sq(float x) {
    const float p = x * x;
    return CF{p, fmaf(x, x, -p)};
}

// Sum of x^2 over the block in a fixed order, as a double in thread 0.
__device__ __forceinline__ double block_sumsq(float x, double* sh) {
    CF v = cf_sq(x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        CF w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = cf_add(v, w);
    }
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nthr = blockDim.x * blockDim.y;
    if ((tid & 31) == 0) sh[tid >> 5] = (double)v.hi + (double)v.lo;
    __syncthreads();
    double r = 0.0;
    if (tid == 0)
        for (int w = 0; w < (nthr + 31) / 32; ++w) r += sh[w];
    __syncthreads();
    return r;
}
__device__ __forceinline__ double block_sumsq(double x, double* sh);
__device__ __forceinline__ float block_maxf(float x, float* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nthr = blockDim.x * blockDim.y;
    if ((tid & 31) == 0) sh[tid >> 5] = x;
    __syncthreads();
    float r = 0.0f;
    if (tid == 0)
        for (int w = 0; w < (nthr + 31) / 32; ++w) r = fmaxf(r, sh[w]);
    __syncthreads();
    return r;
}

// Block sum in a fixed order; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nthr = blockDim.x * blockDim.y;
    v = warp_sum(v);
    if ((tid & 31) == 0) sh[tid >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (tid == 0)
        for (int w = 0; w < (nthr + 31) / 32; ++w) r += sh[w];
    __syncthreads();
    return r;
}
__device__ __forceinline__ double block_max(double v, double* sh) {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nthr = blockDim.x * blockDim.y;
    v = warp_max(v);
    if ((tid & 31) == 0) sh[tid >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (tid == 0)
        for (int w = 0; w < (nthr + 31) / 32; ++w) r = fmax(r, sh[w]);
    __syncthreads();
    return r;
}

// index of node (x, y) inside the control window, or -1
__device__ __forceinline__ int ctrl_window(const CxConst& C, int x, int y) {
    const int cx = x - C.cx0, cy = y - C.cy0;
    if (cx < 0 || cy < 0 || cx >= C.cnx || cy >= C.cny) return -1;
    return cy * C.cnx + cx;
}
// window entry c is a controlled node (mask set, fluid)
__device__ __forceinline__ bool ctrl_active(const CxConst& C, int c) { return c >= 0 && (!C.cmask || C.cmask[c]); }

__device__ __forceinline__ double block_sumsq(double x, double* sh) { return block_sum(x * x, sh); }

// Sum of x^2 and max |x| over the block in one pass (thread 0 holds both).
__device__ __forceinline__ void block_sumsq_max(float x, double* sh, double* sum, double* mx) {
    CF v = cf_sq(x);
    float m = fabsf(x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        CF w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = cf_add(v, w);
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nthr = blockDim.x * blockDim.y;
    if ((tid & 31) == 0) {
        sh[tid >> 5] = (double)v.hi + (double)v.lo;
        sh[16 + (tid >> 5)] = (double)m;
    }
    __syncthreads();
    if (tid == 0) {
        double r = 0.0, q = 0.0;
        for (int w = 0; w < (nthr + 31) / 32; ++w) {
            r += sh[w];
            q = fmax(q, sh[16 + w]);
        }
        *sum = r;
        *mx = q;
    }
}
__device__ __forceinline__ void block_sumsq_max(double x, double* sh, double* sum, double* mx) {
    double v = warp_sum(x * x), m = warp_max(fabs(x));
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nthr = blockDim.x * blockDim.y;
    if ((tid & 31) == 0) {
        sh[tid >> 5] = v;
        sh[16 + (tid >> 5)] = m;
    }
    __syncthreads();
    if (tid == 0) {
        double r = 0.0, q = 0.0;
        for (int w = 0; w < (nthr + 31) / 32; ++w) {
            r += sh[w];
            q = fmax(q, sh[16 + w]);
        }
        *sum = r;
        *mx = q;
    }
}
__device__ __forceinline__ double block_maxd(double x, double* sh) { return block_max(fabs(x), sh); }
__device__ __forceinline__ double block_maxd(float x, double* sh) {
    return (double)block_maxf(fabsf(x), reinterpret_cast<float*>(sh));
}

// ------------------------------------------- programmatic dependent launch
// The lattice kernels are launched with programmatic stream serialisation: a
// step's grid may be scheduled while the previous step is finishing; it runs
// its index set-up, then waits here until the previous grid has completed and
// its writes are visible.  Launched without the attribute, the wait is a no-op.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void allow_next_grid() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// ------------------------------------------------ asynchronous staging copies
// 4- or 8-byte cp.async from global to the issuing thread's own shared slots;
// every thread reads back only what it staged itself, so a wait_group is the
// only synchronisation the pipelined kernels need.
template <typename T> __device__ __forceinline__ void cp_async(T* smem, const T* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Where a node's staged values sit in shared memory.  The bodies read
// population plane j (0..2Q-1) as pop(j, sx), sx = the x offset of the pulled
// neighbour (-e_x,i forward, +e_x,i adjoint), and node-local value v >= 2Q as
// val(v).
//
// ThreadSlots: per-thread staging; value v of the thread's own node at
// s[v NT] (s already offset by threadIdx.x); the staging copy resolved sx.
// fwd_bounce(i) / adj_bounce(i): whether the pull of direction i bounces back
// and must be read from the node's own opposite population instead (forward:
// x - e_i solid; adjoint: x + e_i solid).  The per-thread staging resolves
// bounce-back while copying, so it never reports one.  bb_bits(C, k): the
// node's bounce-back flags (bit i-1: x - e_i solid), which the adjoint body
// needs to write the bounce-back copies of a grid with C.bb_copy set; copies:
// whether the kernel writes them at all (BB: the single-problem adjoint,
// whose output row-window kernels may read).
template <typename T, int NT, bool BB = false> struct ThreadSlots {
    const T* s;
    __device__ __forceinline__ T pop(int j, int) const { return s[j * NT]; }
    __device__ __forceinline__ T val(int v) const { return s[v * NT]; }
    static constexpr bool fwd_bounce(int) { return false; }
    static constexpr bool adj_bounce(int) { return false; }
    static constexpr bool copies = BB;
    __device__ __forceinline__ unsigned bb_bits(const CxConst& C, int k) const { return __ldg(C.bounce + k); }
};
// RowWindow: per-block staging of a row segment [x0, x0 + NT): plane j as a
// window of the source row starting at x0 - H (H = 16 bytes of values),
// NT + 2H wide, so the thread of node x0 + t pulls from H + t + sx; then the
// node-local planes, NT each.  s is offset by threadIdx.x.
template <typename T, int Q, int NT> struct RowWindow {
    static constexpr int H = 16 / (int)sizeof(T);
    static constexpr int W = NT + 2 * H;
    const T* s;
    __device__ __forceinline__ T pop(int j, int sx) const { return s[j * W + H + sx]; }
    __device__ __forceinline__ T val(int v) const { return s[2 * Q * W + (v - 2 * Q) * NT]; }
    static constexpr bool fwd_bounce(int) { return false; }
    static constexpr bool adj_bounce(int) { return false; }
    static constexpr bool copies = false;
    static constexpr unsigned bb_bits(const CxConst&, int) { return 0u; }
};
// RowWindowSolid: a RowWindow on a grid with solid nodes, with the node's
// bounce-back flags (bit i-1: x - e_i is solid), staged as one byte per node.
// COPIES (the adjoint on a grid with C.bb_copy): the solid source of a
// bounced pull holds the node's own opposite population, written there by the
// previous step, so the window entry is the value to use.  Otherwise a window
// entry whose source is solid holds no population the node may use, and the
// node reads its own opposite population from global memory instead (the
// forward, and sub-domains, whose halo frame the exchange overwrites).
template <typename T, int Q, int NT, bool COPIES = false> struct RowWindowSolid : RowWindow<T, Q, NT> {
    unsigned bits;
    __device__ __forceinline__ bool fwd_bounce(int i) const {
        return !COPIES && i != 0 && ((bits >> (i - 1)) & 1u);
    }
    __device__ __forceinline__ bool adj_bounce(int i) const {
        return !COPIES && i != 0 && ((bits >> (Lat<Q>::opp(i) - 1)) & 1u);
    }
    static constexpr bool copies = COPIES;
    __device__ __forceinline__ unsigned bb_bits(const CxConst&, int) const { return bits; }
};

// Index of the periodic neighbour x + (dx, dy) (|dx|, |dy| <= 1) of node (x, y).
__device__ __forceinline__ int nbr_index(const CxConst& C, int x, int y, int dx, int dy) {
    int xn = x + dx, yn = y + dy;
    xn = xn < 0 ? C.nx - 1 : (xn == C.nx ? 0 : xn);
    yn = yn < 0 ? C.ny - 1 : (yn == C.ny ? 0 : yn);
    return yn * C.nx + xn;
}

// Row windows pay when each block of the persistent grid walks several row
// segments, so that one segment's copies run while the previous one is
// computed; with a segment or less per block (small, L2-resident grids) there
// is nothing to overlap and the per-thread staging is faster.  The test mode
// of the staging switch (2) takes the row-window kernels regardless.
inline bool rows_pipelined(const CxConst& C, const Launch& L, unsigned blocks) {
    if (L.row_windows == 2) return true;
    const long long segs = (long long)((C.nx + (int)L.block.x - 1) / (int)L.block.x) * C.ny;
    return segs >= 2LL * blocks;
}

// --------------------------------- bulk copies completed on an mbarrier
// Every wait is bounded in time (MBAR_WAIT_NS of the global timer): a wait
// that gives up returns false, the kernel reports ST_TIMEOUT through the
// problem's status word, and later launches that see the bit return at once.
constexpr unsigned long long MBAR_WAIT_NS = 200000000ull; // 0.2 s

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// makes the initialised barriers visible to the asynchronous proxy
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0 && global_ns() - t0 > MBAR_WAIT_NS) return false;
    }
}
// true in every thread of the block when an earlier launch recorded a
// timeout (read by thread 0, broadcast by the barrier, which also publishes
// the block's mbarrier initialisation)
__device__ __forceinline__ bool block_sees_timeout(const int* status) {
    return __syncthreads_or(threadIdx.x == 0 && status && (*(volatile const int*)status & ST_TIMEOUT)) != 0;
}
// global -> shared bulk copy: both addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Row window of one plane for RowWindow staging: source row `row` (nx
// values, nx a multiple of H), destination `dst` = the plane's window of
// NT + 2H values for nodes [x0, x0 + nv); the periodic neighbours of the row
// ends come from the other end of the row.  Always nv + 2H values in total.
template <typename T, int NT>
__device__ __forceinline__ void bulk_row_window(T* dst, const T* row, int x0, int nv, int nx, uint64_t* bar) {
    constexpr int H = 16 / (int)sizeof(T);
    const int xa = x0 - H < 0 ? 0 : x0 - H;
    const int xb = x0 + nv + H > nx ? nx : x0 + nv + H;
    bulk_g2s(dst + (xa - (x0 - H)), row + xa, (uint32_t)((xb - xa) * sizeof(T)), bar);
    if (x0 == 0) bulk_g2s(dst, row + nx - H, H * sizeof(T), bar);
    if (x0 + nv == nx) bulk_g2s(dst + H + nv, row, H * sizeof(T), bar);
}

// Compensated accumulation of x^2 across the nodes a thread owns, then one
// warp reduction; lane 0 adds the warp's share to its FP64 slot.
struct SqAcc {
    CF s{0.0f, 0.0f};
    float m = 0.0f;
    __device__ __forceinline__ void add(float x) {
        s = cf_add(s, cf_sq(x));
        m = fmaxf(m, fabsf(x));
    }
    __device__ __forceinline__ void flush(double* sum_slot, double* max_slot) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            CF w{__shfl_xor_sync(0xffffffffu, s.hi, o), __shfl_xor_sync(0xffffffffu, s.lo, o)};
            s = cf_add(s, w);
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        }
        if ((threadIdx.x & 31) == 0) {
            if (sum_slot) *sum_slot += (double)s.hi + (double)s.lo;
            if (max_slot) *max_slot = fmax(*max_slot, (double)m);
        }
    }
};
struct SqAccD {
    double s = 0.0, m = 0.0;
    __device__ __forceinline__ void add(double x) {
        s += x * x;
        m = fmax(m, fabs(x));
    }
    __device__ __forceinline__ void flush(double* sum_slot, double* max_slot) {
        s = warp_sum(s);
        m = warp_max(m);
        if ((threadIdx.x & 31) == 0) {
            if (sum_slot) *sum_slot += s;
            if (max_slot) *max_slot = fmax(*max_slot, m);
        }
    }
};
template <typename T> struct SqAccT;
template <> struct SqAccT<float> { using type = SqAcc; };
template <> struct SqAccT<double> { using type = SqAccD; };

// Work decomposition of the persistent lattice kernels: a chunk is one row
// segment of NT consecutive nodes; block b takes chunks b, b + G, b + 2G, ...
// The (row, segment) pair advances incrementally, so no per-node division.
struct NodeIdx {
    int x, y, k, c; // column, row, node index, control index (-1: none)
    bool fluid;     // inside the grid and not solid
    bool ctrl;      // controlled node (window & mask & fluid)
};

template <int NT> struct ChunkIter {
    int nseg, nch, ch, y, seg, dy, dseg;
    __device__ __forceinline__ ChunkIter(const CxConst& C) {
        nseg = (C.nx + NT - 1) / NT;
        nch = nseg * C.ny;
        ch = blockIdx.x;
        y = ch / nseg;
        seg = ch - y * nseg;
        dy = gridDim.x / nseg;
        dseg = gridDim.x - dy * nseg;
    }
    __device__ __forceinline__ bool valid() const { return ch < nch; }
    __device__ __forceinline__ void next() {
        ch += gridDim.x;
        seg += dseg;
        y += dy;
        if (seg >= nseg) {
            seg -= nseg;
            ++y;
        }
    }
    // control-vector index of node (x, y), or -1
    __device__ __forceinline__ int ctrl_index(const CxConst& C, int x, int k) const {
        if (C.ctrl_full) return k;
        const int cx = x - C.cx0, cy = y - C.cy0;
        return (cx >= 0 && cy >= 0 && cx < C.cnx && cy < C.cny) ? cy * C.cnx + cx : -1;
    }
    // the global bytes the node description needs: bit 0 solid, bit 1 control mask set
    __device__ __forceinline__ unsigned flags(const CxConst& C) const {
        const int x = seg * NT + (int)threadIdx.x;
        if (x >= C.nx) return 0u;
        const int k = y * C.nx + x;
        unsigned f = (C.has_solid && C.solid[k]) ? 1u : 0u;
        const int c = ctrl_index(C, x, k);
        if (C.cmask && c >= 0 && C.cmask[c]) f |= 2u;
        return f;
    }
    // the node description from its flags (no memory access)
    __device__ __forceinline__ NodeIdx node_from(const CxConst& C, unsigned f) const {
        NodeIdx r;
        r.x = seg * NT + (int)threadIdx.x;
        r.y = y;
        r.k = r.y * C.nx + r.x;
        r.fluid = r.x < C.nx && !(f & 1u) && !(C.halo && (r.x == 0 || r.y == 0 || r.x == C.nx - 1 || r.y == C.ny - 1));
        r.c = r.x < C.nx ? ctrl_index(C, r.x, r.k) : -1;
        r.ctrl = r.fluid && r.c >= 0 && (!C.cmask || (f & 2u));
        return r;
    }
    __device__ __forceinline__ NodeIdx node(const CxConst& C) const { return node_from(C, flags(C)); }
};
__device__ __forceinline__ NodeIdx no_node() {
    NodeIdx r;
    r.x = r.y = r.k = 0;
    r.c = -1;
    r.fluid = r.ctrl = false;
    return r;
}

} // namespace cx
