// cx_d3q19.cuh -- the D3Q19 lattice of the Sec. 3.1 lattice remark: velocities
// e_0..e_18 in the paper's order (e_{2k} = -e_{2k-1}), weights 1/3, 1/18 (x6),
// 1/36 (x12), and the orthogonal polynomial moment basis used for the MRT
// collision in three dimensions, in the order
//   (rho, e, eps, j_x, q_x, j_y, q_y, j_z, q_z, 3p_xx, 3pi_xx, p_ww, pi_ww,
//    p_xy, p_yz, p_xz, m_x, m_y, m_z)
// with rows 1, 19|e|^2 - 30, (21|e|^4 - 53|e|^2 + 24)/2, e_x, (5|e|^2 - 9) e_x,
// ..., 3e_x^2 - |e|^2, (3|e|^2 - 5)(3e_x^2 - |e|^2), e_y^2 - e_z^2,
// (3|e|^2 - 5)(e_y^2 - e_z^2), e_x e_y, e_y e_z, e_x e_z, (e_y^2 - e_z^2) e_x,
// (e_z^2 - e_x^2) e_y, (e_x^2 - e_y^2) e_z.
//
// The transforms use the opposite pairs: with s_k = f_{2k-1} + f_{2k} and
// d_k = f_{2k-1} - f_{2k} (k = 1..9; pair k has e_{2k-1} = (1,0,0), (0,1,0),
// (0,0,1), (1,1,0), (1,-1,0), (1,0,1), (-1,0,1), (0,1,1), (0,1,-1)), the even
// moments depend on f_0 and the s_k only, the odd ones (j, q, m) on the d_k
// only; the transposed transform builds the pair's even and odd parts A_k and
// B_k and writes f_{2k-1} = A_k + B_k, f_{2k} = A_k - B_k.
#pragma once

namespace cx {
namespace d3 {

constexpr int Q = 19;
__host__ __device__ constexpr int ex(int i) {
    constexpr int t[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1, 0, 0, 0, 0};
    return t[i];
}
__host__ __device__ constexpr int ey(int i) {
    constexpr int t[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[i];
}
__host__ __device__ constexpr int ez(int i) {
    constexpr int t[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1};
    return t[i];
}
__host__ __device__ constexpr double w(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

// moment indices
enum { RHO = 0, EN = 1, EPS = 2, JX = 3, QX = 4, JY = 5, QY = 6, JZ = 7, QZ = 8, PXX = 9, PIXX = 10, PWW = 11,
       PIWW = 12, PXY = 13, PYZ = 14, PXZ = 15, MX = 16, MY = 17, MZ = 18 };

// 1 / |row_k|^2
__host__ __device__ constexpr double inv_n(int k) {
    constexpr double t[Q] = {1.0 / 19, 1.0 / 2394, 1.0 / 252, 1.0 / 10, 1.0 / 40, 1.0 / 10, 1.0 / 40,
                             1.0 / 10, 1.0 / 40,  1.0 / 36, 1.0 / 72, 1.0 / 12, 1.0 / 24, 1.0 / 4,
                             1.0 / 4,  1.0 / 4,   1.0 / 8,  1.0 / 8,  1.0 / 8};
    return t[k];
}
// free relaxation rate of moment k: s[0] rho, s[1] e, s[2] eps, s[3] q, s[4] p, s[5] pi, s[6] m; -1 at the fluxes
__host__ __device__ constexpr int rate_index(int k) {
    constexpr int t[Q] = {0, 1, 2, -1, 3, -1, 3, -1, 3, 4, 5, 4, 5, 4, 4, 4, 6, 6, 6};
    return t[k];
}
// moments of the source shapes w_i, w_i e_x, w_i e_y, w_i e_z (M applied to them)
__host__ __device__ constexpr double src_A(int k) { return k == RHO ? 1.0 : (k == EN ? -11.0 : (k == EPS ? 3.0 : 0.0)); }
__host__ __device__ constexpr double src_B(int c, int k) {
    return k == (c == 0 ? JX : (c == 1 ? JY : JZ)) ? 1.0 / 3.0 : (k == (c == 0 ? QX : (c == 1 ? QY : QZ)) ? -2.0 / 9.0 : 0.0);
}

template <typename T> struct Tr {
    __host__ __device__ static inline void moments(const T (&f)[Q], T (&m)[Q]) {
        T s[10], d[10];
#pragma unroll
        for (int k = 1; k <= 9; ++k) {
            s[k] = f[2 * k - 1] + f[2 * k];
            d[k] = f[2 * k - 1] - f[2 * k];
        }
        const T S1 = s[1] + s[2] + s[3];
        const T S2 = (s[4] + s[5]) + (s[6] + s[7]) + (s[8] + s[9]);
        m[RHO] = f[0] + S1 + S2;
        m[EN] = T(-30) * f[0] - T(11) * S1 + T(8) * S2;
        m[EPS] = T(12) * f[0] - T(4) * S1 + S2;
        const T e45 = s[4] + s[5], e67 = s[6] + s[7], e89 = s[8] + s[9];
        const T px = T(2) * s[1] - s[2] - s[3];               // the |e| = 1 part of 3p_xx
        const T pe = e45 + e67 - T(2) * e89;                  // the |e|^2 = 2 part
        m[PXX] = px + pe;
        m[PIXX] = T(-2) * px + pe;
        const T ww = s[2] - s[3], we = e45 - e67;
        m[PWW] = ww + we;
        m[PIWW] = T(-2) * ww + we;
        m[PXY] = s[4] - s[5];
        m[PYZ] = s[8] - s[9];
        m[PXZ] = s[6] - s[7];
        const T jxe = d[4] + d[5] + d[6] - d[7], jye = d[4] - d[5] + d[8] + d[9], jze = d[6] + d[7] + d[8] - d[9];
        m[JX] = d[1] + jxe;
        m[QX] = T(-4) * d[1] + jxe;
        m[JY] = d[2] + jye;
        m[QY] = T(-4) * d[2] + jye;
        m[JZ] = d[3] + jze;
        m[QZ] = T(-4) * d[3] + jze;
        m[MX] = d[4] + d[5] - d[6] + d[7];
        m[MY] = -d[4] + d[5] + d[8] + d[9];
        m[MZ] = d[6] + d[7] - d[8] + d[9];
    }
    // o = M^T r
    __host__ __device__ static inline void transpose(const T (&r)[Q], T (&o)[Q]) {
        const T c1 = r[RHO] - T(11) * r[EN] - T(4) * r[EPS]; // even part common to the axis pairs
        const T c2 = r[RHO] + T(8) * r[EN] + r[EPS];         // ... and to the edge pairs
        const T pp = r[PXX] + r[PIXX], pw = r[PWW] + r[PIWW];
        const T px1 = r[PXX] - T(2) * r[PIXX], pw1 = r[PWW] - T(2) * r[PIWW];
        T A[10], B[10];
        A[1] = c1 + T(2) * px1;
        A[2] = c1 - px1 + pw1;
        A[3] = c1 - px1 - pw1;
        A[4] = c2 + pp + pw + r[PXY];
        A[5] = c2 + pp + pw - r[PXY];
        A[6] = c2 + pp - pw + r[PXZ];
        A[7] = c2 + pp - pw - r[PXZ];
        A[8] = c2 - T(2) * pp + r[PYZ];
        A[9] = c2 - T(2) * pp - r[PYZ];
        const T jx = r[JX] + r[QX], jy = r[JY] + r[QY], jz = r[JZ] + r[QZ];
        B[1] = r[JX] - T(4) * r[QX];
        B[2] = r[JY] - T(4) * r[QY];
        B[3] = r[JZ] - T(4) * r[QZ];
        B[4] = jx + jy + r[MX] - r[MY];
        B[5] = jx - jy + r[MX] + r[MY];
        B[6] = jx + jz - r[MX] + r[MZ];
        B[7] = -jx + jz + r[MX] + r[MZ];
        B[8] = jy + jz + r[MY] - r[MZ];
        B[9] = jy - jz + r[MY] + r[MZ];
        o[0] = r[RHO] - T(30) * r[EN] + T(12) * r[EPS];
#pragma unroll
        for (int k = 1; k <= 9; ++k) {
            o[2 * k - 1] = A[k] + B[k];
            o[2 * k] = A[k] - B[k];
        }
    }
};

// moments at unit density of the equilibrium w_i aleph_i (eq. phieq with
// T = a Theta, C = (a a) Theta, in three dimensions):
//   (1, 19(|a|^2 + d) - 30, (17 - 11|a|^2 - 11d)/2, a_x, -2a_x/3, a_y, -2a_y/3,
//    a_z, -2a_z/3, 3a_x^2 - |a|^2, -(3a_x^2 - |a|^2)/2, a_y^2 - a_z^2,
//    -(a_y^2 - a_z^2)/2, a_x a_y, a_y a_z, a_x a_z, 0, 0, 0)
template <typename T> __host__ __device__ inline void meq_unit(T ax, T ay, T az, T d, T (&mh)[Q]) {
    const T a2 = ax * ax + ay * ay + az * az;
    const T pxx = T(3) * ax * ax - a2, pww = ay * ay - az * az;
    mh[RHO] = T(1);
    mh[EN] = T(19) * (a2 + d) - T(30);
    mh[EPS] = T(0.5) * (T(17) - T(11) * a2 - T(11) * d);
    mh[JX] = ax;
    mh[QX] = T(-2.0 / 3.0) * ax;
    mh[JY] = ay;
    mh[QY] = T(-2.0 / 3.0) * ay;
    mh[JZ] = az;
    mh[QZ] = T(-2.0 / 3.0) * az;
    mh[PXX] = pxx;
    mh[PIXX] = T(-0.5) * pxx;
    mh[PWW] = pww;
    mh[PIWW] = T(-0.5) * pww;
    mh[PXY] = ax * ay;
    mh[PYZ] = ay * az;
    mh[PXZ] = ax * az;
    mh[MX] = T(0);
    mh[MY] = T(0);
    mh[MZ] = T(0);
}

} // namespace d3
} // namespace cx
