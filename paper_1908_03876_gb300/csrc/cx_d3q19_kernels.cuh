// cx_d3q19_kernels.cuh -- node bodies and kernels of the D3Q19 solver
// (include/cx3d.h): the two-species forward MRT step and its exact discrete
// adjoint with the fused gradient, on a periodic nx x ny x nz lattice.
//
// Per node x and step n (tau in lattice units, Cs^2 = 1/3):
//   f_Theta,i(x) = P^{n-1}_Theta,i(x - e_i)    (f^0 = phi^eq(Theta_0) read locally)
//   Theta = sum_i f_i,  j_v = sum_i e_i f_v,i
//   Phi_v = r_vu u + r_vv v + g^n(x)           (Phi_u = 0)
//   G     = -(K_v (j_v - a v)/tau + K_v a Phi_v / 2) / (d_v Cs^2)
//   P_Theta = f - M^-1 Pi_Theta (M f - m^eq(Theta))
//   P_u,i += 3 w_i e_i . (chi u K_u G)          (tau S_u)
//   P_v,i += w~_i [c_n Phi^n + c'_n Phi^{n-1}], w~_i = w_i (1 + 3 V.e_i), V = (I - K_v/2) a
// Sources have the shape w_i (A + B.e_i): in FP32 they join the collision in
// moment space, in FP64 (parity mode) they are added per direction.
// Adjoint (exact transpose): rho_i(x) = psi^{n+1}_i(x + e_i); psi = rho -
// M^T Pi^T N^-1 M rho + Tcal (Tcal = sum_k z_k m^eq_k, z = N^-1 Pi M rho) plus
// the coupling terms of S_u (through u, j_v, v and Phi_v) and of the source;
// dJ/dg^n = c_n sigma^n + c'_{n+1} sigma^{n+1} - (a . K_v aG)/(2 d_v Cs^2) + 2 alpha g^n.
#pragma once

#include "cx_d3q19.cuh"
#include "cx_device.cuh"

namespace cx {
namespace d3 {

// per-problem constants (kernel parameter)
struct C3 {
    int nx, ny, nz;
    long long plane;
    int N, aniso, adv;
    const void* Kfield; // T [12][plane]: K_u (xx, xy, xz, yy, yz, zz), then K_v (FIELD)
    const void* a;      // T [ny][3] (ROW) or [3][plane] (FIELD)
};

template <typename T> struct K3 {
    T sn[Q];       // rate of moment k / |row k|^2 (0 at the fluxes)
    T invn_j;      // 1 / |row| of the flux moments (1/10)
    T Ku[6], Kv[6]; // CONST tensors -> K
    T tau, inv_tau, gsc, asc, d_u, d_v, chi, r_vu, r_vv, two_alpha, c_first, c_now, c_prev;
};

template <typename T> struct Coef {
    T Ku[6], Kv[6];
    T a[3];
};

template <typename T> __device__ __forceinline__ T ldt(const T* p) { return __ldg(p); }

template <typename T>
__device__ __forceinline__ void coef(const C3& C, const K3<T>& KC, int y, size_t k, Coef<T>& c) {
    if (C.aniso == CX_ANISO_FIELD) {
        const T* K = reinterpret_cast<const T*>(C.Kfield);
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            c.Ku[j] = ldt(K + (size_t)j * C.plane + k);
            c.Kv[j] = ldt(K + (size_t)(6 + j) * C.plane + k);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            c.Ku[j] = KC.Ku[j];
            c.Kv[j] = KC.Kv[j];
        }
    }
    if (C.adv == CX_ADV_ROW) {
        const T* a = reinterpret_cast<const T*>(C.a);
#pragma unroll
        for (int q = 0; q < 3; ++q) c.a[q] = ldt(a + 3 * y + q);
    } else if (C.adv == CX_ADV_FIELD) {
        const T* a = reinterpret_cast<const T*>(C.a);
#pragma unroll
        for (int q = 0; q < 3; ++q) c.a[q] = ldt(a + (size_t)q * C.plane + k);
    } else {
        c.a[0] = c.a[1] = c.a[2] = T(0);
    }
}

// y = K x for a symmetric K stored as (xx, xy, xz, yy, yz, zz)
template <typename T> __device__ __forceinline__ void kmul(const T (&K)[6], const T (&x)[3], T (&y)[3]) {
    y[0] = K[0] * x[0] + K[1] * x[1] + K[2] * x[2];
    y[1] = K[1] * x[0] + K[3] * x[1] + K[4] * x[2];
    y[2] = K[2] * x[0] + K[4] * x[1] + K[5] * x[2];
}

// N^-1 Pi dm (free rates on the non-flux moments, K on the fluxes)
template <typename T>
__device__ __forceinline__ void relax(const K3<T>& KC, const T (&K)[6], const T (&dm)[Q], T (&out)[Q]) {
#pragma unroll
    for (int k = 0; k < Q; ++k)
        if (k != JX && k != JY && k != JZ) out[k] = KC.sn[k] * dm[k];
    const T j[3] = {dm[JX], dm[JY], dm[JZ]};
    T kj[3];
    kmul(K, j, kj);
    out[JX] = kj[0] * KC.invn_j;
    out[JY] = kj[1] * KC.invn_j;
    out[JZ] = kj[2] * KC.invn_j;
}

// post-collision populations of one species with the source w_i (A + B.e_i)
template <typename T>
__device__ __forceinline__ void collide_write(const K3<T>& KC, const T (&f)[Q], const T (&m)[Q], const T (&mh)[Q],
                                              const T (&K)[6], T A, const T (&B)[3], T* out, size_t pl, size_t k) {
    constexpr bool fold = sizeof(T) == 4;
    T dm[Q], rl[Q], bt[Q];
    const T Th = m[RHO];
#pragma unroll
    for (int q = 0; q < Q; ++q) dm[q] = m[q] - Th * mh[q];
    relax<T>(KC, K, dm, rl);
    if constexpr (fold) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (src_A(q) != 0.0) rl[q] -= T(inv_n(q) * src_A(q)) * A;
#pragma unroll
            for (int c = 0; c < 3; ++c)
                if (src_B(c, q) != 0.0) rl[q] -= T(inv_n(q) * src_B(c, q)) * B[c];
        }
    }
    Tr<T>::transpose(rl, bt);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if constexpr (fold)
            out[i * pl + k] = f[i] - bt[i];
        else
            out[i * pl + k] = f[i] - bt[i] + T(w(i)) * (A + T(ex(i)) * B[0] + T(ey(i)) * B[1] + T(ez(i)) * B[2]);
    }
}

template <typename T> struct FArgs {
    const T* in;      // [2][Q][plane] pulled (P^{n-1}), or f^0 read locally at n = 0
    T* out;
    T* phi;           // [plane] Phi_v^{n-1} in, Phi_v^n out
    T* phi_ckpt;      // [plane] or null
    const T* g;       // [nodes] g^n or null
    const T* E;       // [nodes] trial direction or null
    T lam;
    T* tape;          // [4][plane] (u, G_x, G_y, G_z) or null
    double* gsq_part; // per-warp partials of sum (g^n)^2, or null
    int n;
};

template <typename T> struct AArgs {
    const T* in;      // [2][Q][plane] psi^{n+1} (unused at the terminal step)
    const T* seed_u;  // terminal seeds (null: 0), terminal step only
    const T* seed_v;
    T* out;
    const T* tape;    // [4][plane]
    T* sigma;         // [plane] sigma^{n+1} in, sigma^n out
    const T* g;       // [nodes] g^n or null
    T* dJdg;          // [nodes]
    double* e2_part;
    double* emax_part;
    int n, terminal;
};

// the three row/plane offsets of a node's neighbourhood: index of x + s e for
// s = -1, 0, +1 along each axis (periodic)
struct Nbr {
    long long zo[3], yo[3];
    int xv[3];
    __device__ __forceinline__ Nbr(const C3& C, int x, int y, int z) {
        const long long nxy = (long long)C.nx * C.ny;
        zo[0] = (long long)(z == 0 ? C.nz - 1 : z - 1) * nxy;
        zo[1] = (long long)z * nxy;
        zo[2] = (long long)(z == C.nz - 1 ? 0 : z + 1) * nxy;
        yo[0] = (long long)(y == 0 ? C.ny - 1 : y - 1) * C.nx;
        yo[1] = (long long)y * C.nx;
        yo[2] = (long long)(y == C.ny - 1 ? 0 : y + 1) * C.nx;
        xv[0] = x == 0 ? C.nx - 1 : x - 1;
        xv[1] = x;
        xv[2] = x == C.nx - 1 ? 0 : x + 1;
    }
    // x + s e_i (s = -1: the forward pull, s = +1: the adjoint pull)
    __device__ __forceinline__ size_t at(int i, int s) const {
        return (size_t)(zo[1 + s * ez(i)] + yo[1 + s * ey(i)] + xv[1 + s * ex(i)]);
    }
};

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k3d_forward(const C3 C, const K3<T> KC, const FArgs<T> A) {
    constexpr bool fold = sizeof(T) == 4;
    (void)fold;
    const size_t pl = (size_t)C.plane;
    const long long total = (long long)C.nx * C.ny * C.nz;
    const long long nxy = (long long)C.nx * C.ny;
    typename SqAccT<T>::type acc;
    for (long long kk = blockIdx.x * (long long)blockDim.x + threadIdx.x; kk < total;
         kk += (long long)gridDim.x * blockDim.x) {
        const size_t k = (size_t)kk;
        const int z = (int)(kk / nxy);
        const int rem = (int)(kk - (long long)z * nxy);
        const int y = rem / C.nx, x = rem - y * C.nx;
        T fu[Q], fv[Q];
        if (A.n == 0) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                fu[i] = ldt(A.in + i * pl + k);
                fv[i] = ldt(A.in + (Q + i) * pl + k);
            }
        } else {
            const Nbr nb(C, x, y, z);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const size_t ks = nb.at(i, -1);
                fu[i] = ldt(A.in + i * pl + ks);
                fv[i] = ldt(A.in + (Q + i) * pl + ks);
            }
        }
        const T prev = A.n > 0 ? A.phi[k] : T(0);
        T g = T(0);
        if (A.g) g = ldt(A.g + k);
        if (A.E) g = fma(-A.lam, ldt(A.E + k), g);
        if (A.gsq_part) acc.add(g);
        Coef<T> nc;
        coef<T>(C, KC, y, k, nc);

        T mu[Q], mv[Q];
        Tr<T>::moments(fu, mu);
        Tr<T>::moments(fv, mv);
        const T Tu = mu[RHO], Tv = mv[RHO];
        const T Phi = KC.r_vu * Tu + KC.r_vv * Tv + g;
        const T src = A.n == 0 ? KC.c_first * Phi : KC.c_now * Phi + KC.c_prev * prev;
        // G = -(K_v (j_v - a v)/tau + K_v a Phi / 2) / (d_v Cs^2)
        const T rr[3] = {(mv[JX] - nc.a[0] * Tv) * KC.inv_tau + T(0.5) * nc.a[0] * Phi,
                         (mv[JY] - nc.a[1] * Tv) * KC.inv_tau + T(0.5) * nc.a[1] * Phi,
                         (mv[JZ] - nc.a[2] * Tv) * KC.inv_tau + T(0.5) * nc.a[2] * Phi};
        T G[3];
        kmul(nc.Kv, rr, G);
#pragma unroll
        for (int q = 0; q < 3; ++q) G[q] *= KC.gsc;
        // species u: chemotactic source 3 w_i e_i . (chi u K_u G)
        {
            T mh[Q];
            meq_unit<T>(nc.a[0], nc.a[1], nc.a[2], KC.d_u, mh);
            const T F[3] = {KC.chi * Tu * G[0], KC.chi * Tu * G[1], KC.chi * Tu * G[2]};
            T KF[3];
            kmul(nc.Ku, F, KF);
            const T B[3] = {T(3) * KF[0], T(3) * KF[1], T(3) * KF[2]};
            collide_write<T>(KC, fu, mu, mh, nc.Ku, T(0), B, A.out, pl, k);
        }
        // species v: reaction/control source with w~ = w (1 + 3 V.e), V = (I - K_v/2) a
        {
            T mh[Q];
            meq_unit<T>(nc.a[0], nc.a[1], nc.a[2], KC.d_v, mh);
            T Ka[3];
            kmul(nc.Kv, nc.a, Ka);
            const T B[3] = {T(3) * src * (nc.a[0] - T(0.5) * Ka[0]), T(3) * src * (nc.a[1] - T(0.5) * Ka[1]),
                            T(3) * src * (nc.a[2] - T(0.5) * Ka[2])};
            collide_write<T>(KC, fv, mv, mh, nc.Kv, src, B, A.out + (size_t)Q * pl, pl, k);
        }
        A.phi[k] = Phi;
        if (A.phi_ckpt) A.phi_ckpt[k] = Phi;
        if (A.tape) {
            A.tape[k] = Tu;
            A.tape[pl + k] = G[0];
            A.tape[2 * pl + k] = G[1];
            A.tape[3 * pl + k] = G[2];
        }
    }
    if (A.gsq_part) acc.flush(A.gsq_part + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5), nullptr);
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k3d_adjoint(const C3 C, const K3<T> KC, const AArgs<T> A) {
    constexpr bool fold = sizeof(T) == 4;
    const size_t pl = (size_t)C.plane;
    const long long total = (long long)C.nx * C.ny * C.nz;
    const long long nxy = (long long)C.nx * C.ny;
    typename SqAccT<T>::type acc;
    for (long long kk = blockIdx.x * (long long)blockDim.x + threadIdx.x; kk < total;
         kk += (long long)gridDim.x * blockDim.x) {
        const size_t k = (size_t)kk;
        const int z = (int)(kk / nxy);
        const int rem = (int)(kk - (long long)z * nxy);
        const int y = rem / C.nx, x = rem - y * C.nx;
        const Nbr nb(C, x, y, z);
        T ru[Q], rv[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const size_t kd = nb.at(i, +1);
            if (A.terminal) {
                ru[i] = A.seed_u ? ldt(A.seed_u + kd) : T(0);
                rv[i] = A.seed_v ? ldt(A.seed_v + kd) : T(0);
            } else {
                ru[i] = ldt(A.in + i * pl + kd);
                rv[i] = ldt(A.in + (Q + i) * pl + kd);
            }
        }
        const T Tu = ldt(A.tape + k);
        const T G[3] = {ldt(A.tape + pl + k), ldt(A.tape + 2 * pl + k), ldt(A.tape + 3 * pl + k)};
        const T gv = A.g ? ldt(A.g + k) : T(0);
        const T sig_next = A.terminal ? T(0) : A.sigma[k]; // read before this node's stores
        Coef<T> nc;
        coef<T>(C, KC, y, k, nc);

        // species u: transposed collision; Y_c = sum_i 3 w_i e_c,i rho_u,i
        T psu[Q], Y[3] = {T(0), T(0), T(0)};
        {
            T mh[Q], mom[Q], zz[Q], mt[Q];
            meq_unit<T>(nc.a[0], nc.a[1], nc.a[2], KC.d_u, mh);
            Tr<T>::moments(ru, mom);
            if constexpr (fold) {
#pragma unroll
                for (int q = 0; q < Q; ++q)
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        if (src_B(c, q) != 0.0) Y[c] += T(3.0 * inv_n(q) * src_B(c, q)) * mom[q];
            } else {
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    Y[0] += T(3.0 * w(i) * ex(i)) * ru[i];
                    Y[1] += T(3.0 * w(i) * ey(i)) * ru[i];
                    Y[2] += T(3.0 * w(i) * ez(i)) * ru[i];
                }
            }
            relax<T>(KC, nc.Ku, mom, zz);
            T Tc = T(0);
#pragma unroll
            for (int q = 0; q < Q; ++q) Tc += zz[q] * mh[q];
            Tr<T>::transpose(zz, mt);
#pragma unroll
            for (int i = 0; i < Q; ++i) psu[i] = ru[i] - mt[i] + Tc;
        }
        // species v: transposed collision; sigma = sum_i w~_i rho_v,i
        T psv[Q], sigma = T(0);
        T Ka[3];
        kmul(nc.Kv, nc.a, Ka);
        const T V[3] = {nc.a[0] - T(0.5) * Ka[0], nc.a[1] - T(0.5) * Ka[1], nc.a[2] - T(0.5) * Ka[2]};
        {
            T mh[Q], mom[Q], zz[Q], mt[Q];
            meq_unit<T>(nc.a[0], nc.a[1], nc.a[2], KC.d_v, mh);
            Tr<T>::moments(rv, mom);
            if constexpr (fold) {
                T sA = T(0), sB[3] = {T(0), T(0), T(0)};
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    if (src_A(q) != 0.0) sA += T(inv_n(q) * src_A(q)) * mom[q];
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        if (src_B(c, q) != 0.0) sB[c] += T(3.0 * inv_n(q) * src_B(c, q)) * mom[q];
                }
                sigma = sA + V[0] * sB[0] + V[1] * sB[1] + V[2] * sB[2];
            } else {
#pragma unroll
                for (int i = 0; i < Q; ++i)
                    sigma += T(w(i)) * (T(1) + T(3) * (V[0] * T(ex(i)) + V[1] * T(ey(i)) + V[2] * T(ez(i)))) * rv[i];
            }
            relax<T>(KC, nc.Kv, mom, zz);
            T Tc = T(0);
#pragma unroll
            for (int q = 0; q < Q; ++q) Tc += zz[q] * mh[q];
            Tr<T>::transpose(zz, mt);
#pragma unroll
            for (int i = 0; i < Q; ++i) psv[i] = rv[i] - mt[i] + Tc;
        }
        // coupling through tau S_u = 3 w_i e_i . K_u (chi u G)
        T aF[3];
        kmul(nc.Ku, Y, aF); // K_u symmetric
        T aTu = KC.chi * (G[0] * aF[0] + G[1] * aF[1] + G[2] * aF[2]);
        const T aG[3] = {KC.chi * Tu * aF[0], KC.chi * Tu * aF[1], KC.chi * Tu * aF[2]};
        T KG[3];
        kmul(nc.Kv, aG, KG);
        const T aj[3] = {-KG[0] * KC.asc * KC.inv_tau, -KG[1] * KC.asc * KC.inv_tau, -KG[2] * KC.asc * KC.inv_tau};
        const T aKG = nc.a[0] * KG[0] + nc.a[1] * KG[1] + nc.a[2] * KG[2];
        T aTv = aKG * KC.asc * KC.inv_tau;
        T aPhi = T(-0.5) * aKG * KC.asc;
        aPhi += (A.n == 0 ? KC.c_first : KC.c_now) * sigma;
        if (!A.terminal) aPhi += KC.c_prev * sig_next;
        A.sigma[k] = sigma;
        aTu += KC.r_vu * aPhi;
        aTv += KC.r_vv * aPhi;
        const T E = aPhi + KC.two_alpha * gv;
        A.dJdg[k] = E;
        if (A.e2_part) acc.add(E);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            A.out[i * pl + k] = psu[i] + aTu;
            A.out[(Q + i) * pl + k] = psv[i] + aTv + T(ex(i)) * aj[0] + T(ey(i)) * aj[1] + T(ez(i)) * aj[2];
        }
    }
    if (A.e2_part) {
        const int wi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        acc.flush(A.e2_part + wi, A.emax_part + wi);
    }
}

// f^0 = phi^eq(Theta_0): w_i aleph_i Theta_0, aleph_i = 1 + 3 a.e + 4.5 ((a.e)^2 - |a|^2/3)
// + 1.5 (d - 1)(|e|^2 - 1)
template <typename T>
__global__ void k3d_init(const C3 C, const K3<T> KC, const double* u0, const double* v0, T* P) {
    const long long total = (long long)C.nx * C.ny * C.nz;
    const size_t pl = (size_t)C.plane;
    for (long long kk = blockIdx.x * (long long)blockDim.x + threadIdx.x; kk < total;
         kk += (long long)gridDim.x * blockDim.x) {
        const size_t k = (size_t)kk;
        const int y = (int)((kk % ((long long)C.nx * C.ny)) / C.nx);
        Coef<T> nc;
        coef<T>(C, KC, y, k, nc);
        const T Tu = T(u0[k]), Tv = T(v0[k]);
        const T a2 = nc.a[0] * nc.a[0] + nc.a[1] * nc.a[1] + nc.a[2] * nc.a[2];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T ea = nc.a[0] * T(ex(i)) + nc.a[1] * T(ey(i)) + nc.a[2] * T(ez(i));
            const T e2 = T(ex(i) * ex(i) + ey(i) * ey(i) + ez(i) * ez(i));
            const T base = T(1) + T(3) * ea + T(4.5) * (ea * ea - a2 * T(1.0 / 3.0));
            P[i * pl + k] = T(w(i)) * (base + T(1.5) * (KC.d_u - T(1)) * (e2 - T(1))) * Tu;
            P[(Q + i) * pl + k] = T(w(i)) * (base + T(1.5) * (KC.d_v - T(1)) * (e2 - T(1))) * Tv;
        }
    }
}

// u^N, v^N from the pulled P^{N-1}; the terminal seed u^N - u_target; block
// partials of 1/2 sum (u^N - u_target)^2 (FP64)
template <typename T>
__global__ void __launch_bounds__(256) k3d_final(const C3 C, const T* Pin, const T* ut, T* uN, T* vN, T* wu,
                                                  double* cost_part) {
    __shared__ double red[32];
    const long long total = (long long)C.nx * C.ny * C.nz;
    const long long nxy = (long long)C.nx * C.ny;
    const size_t pl = (size_t)C.plane;
    const long long kk = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double cst = 0.0;
    if (kk < total) {
        const size_t k = (size_t)kk;
        const int z = (int)(kk / nxy);
        const int rem = (int)(kk - (long long)z * nxy);
        const int y = rem / C.nx, x = rem - y * C.nx;
        const Nbr nb(C, x, y, z);
        T su = T(0), sv = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const size_t ks = nb.at(i, -1);
            su += Pin[i * pl + ks];
            sv += Pin[(Q + i) * pl + ks];
        }
        uN[k] = su;
        vN[k] = sv;
        const T wv = su - ut[k];
        wu[k] = wv;
        cst = 0.5 * (double)wv * (double)wv;
    }
    const double b = block_sum(cst, red);
    if (threadIdx.x == 0) cost_part[blockIdx.x] = b;
}

// descriptor fields in the kernels' precision: K per node (FIELD, eigenvalues
// checked in (0, 2)), a, u_target
template <typename T>
__global__ void k3d_setup(const C3 C, const cx3d_desc d, T* Kf, T* a, T* ut, int* status) {
    const long long total = (long long)C.nx * C.ny * C.nz;
    const size_t pl = (size_t)C.plane;
    for (long long kk = blockIdx.x * (long long)blockDim.x + threadIdx.x; kk < total;
         kk += (long long)gridDim.x * blockDim.x) {
        const size_t k = (size_t)kk;
        if (Kf) {
            const double* Ds[2] = {d.D_u_field, d.D_v_field};
            const double dd[2] = {d.d_u, d.d_v};
            for (int s = 0; s < 2; ++s) {
                const double sc = 1.0 / (dd[s] * (1.0 / 3.0) * d.tau);
                const double* D = Ds[s] + 6 * k;
                // A = D sc + I/2; K = A^-1 (symmetric)
                const double a00 = D[0] * sc + 0.5, a01 = D[1] * sc, a02 = D[2] * sc, a11 = D[3] * sc + 0.5,
                             a12 = D[4] * sc, a22 = D[5] * sc + 0.5;
                const double c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11;
                const double det = a00 * c00 + a01 * c01 + a02 * c02;
                const double K[6] = {c00 / det, c01 / det, c02 / det, (a00 * a22 - a02 * a02) / det,
                                     (a01 * a02 - a00 * a12) / det, (a00 * a11 - a01 * a01) / det};
                // A symmetric positive definite with eigenvalues > 1/2 <=> K eigenvalues in (0, 2):
                // check the leading minors of A and of A - I/2
                const double b00 = a00 - 0.5, b11 = a11 - 0.5, b22 = a22 - 0.5;
                const double m2 = b00 * b11 - a01 * a01;
                const double m3 = b00 * (b11 * b22 - a12 * a12) - a01 * (a01 * b22 - a12 * a02) +
                                  a02 * (a01 * a12 - b11 * a02);
                if (!(det > 0.0) || !(b00 > 0.0) || !(m2 > 0.0) || !(m3 > 0.0)) atomicOr(status, ST_UNSTABLE);
                for (int j = 0; j < 6; ++j) Kf[(size_t)(6 * s + j) * pl + k] = T(K[j]);
            }
        }
        if (a && C.adv == CX_ADV_FIELD)
            for (int q = 0; q < 3; ++q) a[(size_t)q * pl + k] = T(d.a[3 * k + q]);
        if (a && C.adv == CX_ADV_ROW && kk < C.ny)
            for (int q = 0; q < 3; ++q) a[3 * kk + q] = T(d.a[3 * kk + q]);
        ut[k] = T(d.u_target[k]);
    }
}

} // namespace d3
} // namespace cx
