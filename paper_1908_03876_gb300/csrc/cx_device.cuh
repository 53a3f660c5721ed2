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

template <typename T>
__device__ __forceinline__ void node_coef(const CxConst& C, int x, int y, int k, NodeCoef<T>& c) {
    if (C.aniso == CX_ANISO_ROTATED) {
        // K = R diag(k1, k2) R^T = kbar I + kd [[cos 2t, sin 2t], [sin 2t, -cos 2t]]
        T th = ldg(reinterpret_cast<const T*>(C.theta) + k);
        T s2, c2;
        if constexpr (sizeof(T) == 4) sincosf(2.0f * th, &s2, &c2);
        else sincos(2.0 * th, &s2, &c2);
        c.Ku0 = T(C.ku_bar) + T(C.ku_d) * c2;
        c.Ku1 = T(C.ku_d) * s2;
        c.Ku2 = T(C.ku_bar) - T(C.ku_d) * c2;
        c.Kv0 = T(C.kv_bar) + T(C.kv_d) * c2;
        c.Kv1 = T(C.kv_d) * s2;
        c.Kv2 = T(C.kv_bar) - T(C.kv_d) * c2;
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
        c.Ku0 = T(C.Ku[0]);
        c.Ku1 = T(C.Ku[1]);
        c.Ku2 = T(C.Ku[2]);
        c.Kv0 = T(C.Kv[0]);
        c.Kv1 = T(C.Kv[1]);
        c.Kv2 = T(C.Kv[2]);
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
__device__ __forceinline__ void relax(const CxConst& C, T K0, T K1, T K2, const T (&dm)[Q], T (&out)[Q]) {
    using L = Lat<Q>;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const int r = rate_index<Q>(k);
        if (r >= 0) out[k] = T(C.s[r]) * dm[k];
    }
    out[L::JX] = K0 * dm[L::JX] + K1 * dm[L::JY];
    out[L::JY] = K1 * dm[L::JX] + K2 * dm[L::JY];
}

// Pi^T lambda (K symmetric, so the block is unchanged; diagonal rates too).
template <typename T, int Q>
__device__ __forceinline__ void relax_T(const CxConst& C, T K0, T K1, T K2, const T (&lam)[Q], T (&out)[Q]) {
    relax<T, Q>(C, K0, K1, K2, lam, out);
}

// ---------------------------------------------------- deterministic reductions

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

} // namespace cx
