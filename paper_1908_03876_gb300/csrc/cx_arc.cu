// cx_arc.cu -- the three-species solver of include/cxarc.h: the attraction-
// repulsion chemotaxis model with a logistic source (ARC example, Sec. 2.2)
// on D2Q9, forward MRT step, exact discrete adjoint step with fused gradient,
// and the host schedule (checkpoints, segment recompute with a tape, FP64
// reductions, Armijo search).
//
// Per node x and step n (tau in lattice units, Cs^2 = 1/3), species
// Theta in {u, v, w}:
//   f_Theta,i(x) = P^{n-1}_Theta,i(x - e_i)  (periodic pull; f^0 = phi^eq(Theta_0) read locally)
//   Theta = sum_i f_i,  j_Theta = sum_i e_i f_i
//   Phi_u = a1 u - a2 u^2,  Phi_v = b1 u - b2 v - b3 u v,  Phi_w = c1 u - c2 w  (+ g on v or w)
//   G_Theta = -(K_Theta (j_Theta - a Theta)/tau + K_Theta a Phi_Theta / 2) / (d Cs^2),  Theta = v, w
//             (local gradient from the first non-equilibrium moment, relation C146)
//   P_Theta = f - M^-1 Pi_Theta (M f - m^eq(Theta)) + w~_Theta,i [c_n Phi^n + c'_n Phi^{n-1}]
//             (eqs. MF, MC, PhiS; w~_i = w_i (1 + 3 V.e_i), V = (I - K_Theta/2) a;
//             c_n = 3 tau/2, c'_n = -tau/2, c_0 = tau, c'_0 = 0)
//   P_u,i  += 3 w_i e_i . K_u (chi1 u G_v + chi2 u G_w)         (tau S_u, eq. S)
// Every source has the shape w_i (A + B.e_i); in FP32 it joins the collision
// in moment space (s^ = M0 s, few nonzero moments), in FP64 (parity mode) it
// is added per direction.
//
// The adjoint of that step (exact transpose, run backward in time):
//   rho_Theta,i(x) = psi^{n+1}_Theta,i(x + e_i)     (streaming along -e_i)
//   psi_Theta     = rho - M^T Pi^T N^-1 M rho + Tcal_Theta   (transposed collision and the
//                   adjoint-equilibrium broadcast Tcal = sum_j w_j aleph_j (Lambda^T rho)_j)
//                   + the coupling terms of the three sources (the chain rule through
//                   Theta, j_Theta and Phi_Theta), and
//   dJ/dg^n       = lambda_Phi(ctrl species) + 2 alpha g^n,
//   lambda_Phi    = c_n sigma^n + c'_{n+1} sigma^{n+1} - (a . K aG)/(2 d Cs^2),
//   sigma^n       = sum_i w~_i rho_i.
// The tape of the recompute holds (u, v, G_v, G_w) per node and step.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/cxarc.h"
#include "cx_device.cuh"
#include "cx_rows.cuh"

namespace cx {
namespace arc {

using L9 = Lat<9>;

// per-problem constants (kernel parameter)
struct AC {
    int nx, ny;
    long long plane;
    int N, aniso, adv, ctrl;
    const void* theta;  // T [plane] (ROTATED)
    const void* Kfield; // T [9][plane]: species-major (k11, k12, k22) (FIELD)
    const void* a;      // T [ny][2] (ROW) or [2][plane] (FIELD)
};

// the same in the kernels' precision
template <typename T> struct AK {
    T sn[9];             // rate of moment k / |row k|^2 (0 at the flux moments)
    T invn_j;            // 1 / |row| of the flux moments (both 1/6)
    T K[3][3];           // CONST tensors -> K per species
    T kbar[3], kd[3];    // ROTATED: K = kbar I + kd [[cos 2t, sin 2t], [sin 2t, -cos 2t]]
    T tau, inv_tau, gsc, asc, d;
    T chi1, chi2, a1, a2, b1, b2, b3, c1, c2;
    T two_alpha, c_first, c_now, c_prev;
};

template <typename T> struct Coef3 {
    T K[3][3];
    T ax, ay;
};

template <typename T> __device__ __forceinline__ T ld(const T* p) { return __ldg(p); }

template <typename T>
__device__ __forceinline__ void coef3_th(const AC& C, const AK<T>& KC, int y, int k, T th, Coef3<T>& c) {
    if (C.aniso == CX_ANISO_ROTATED) {
        T s2, c2;
        sincos2(th, &s2, &c2);
#pragma unroll
        for (int sp = 0; sp < 3; ++sp) {
            c.K[sp][0] = KC.kbar[sp] + KC.kd[sp] * c2;
            c.K[sp][1] = KC.kd[sp] * s2;
            c.K[sp][2] = KC.kbar[sp] - KC.kd[sp] * c2;
        }
    } else if (C.aniso == CX_ANISO_FIELD) {
        const T* K = reinterpret_cast<const T*>(C.Kfield);
#pragma unroll
        for (int j = 0; j < 9; ++j) c.K[j / 3][j % 3] = ld(K + (size_t)j * C.plane + k);
    } else {
#pragma unroll
        for (int sp = 0; sp < 3; ++sp)
#pragma unroll
            for (int j = 0; j < 3; ++j) c.K[sp][j] = KC.K[sp][j];
    }
    if (C.adv == CX_ADV_ROW) {
        const T* a = reinterpret_cast<const T*>(C.a);
        c.ax = ld(a + 2 * y);
        c.ay = ld(a + 2 * y + 1);
    } else if (C.adv == CX_ADV_FIELD) {
        const T* a = reinterpret_cast<const T*>(C.a);
        c.ax = ld(a + k);
        c.ay = ld(a + C.plane + k);
    } else {
        c.ax = T(0);
        c.ay = T(0);
    }
}

template <typename T>
__device__ __forceinline__ void coef3(const AC& C, const AK<T>& KC, int y, int k, Coef3<T>& c) {
    coef3_th<T>(C, KC, y, k, C.aniso == CX_ANISO_ROTATED ? ld(reinterpret_cast<const T*>(C.theta) + k) : T(0), c);
}

// N^-1 Pi dm (Pi^T N^-1 has the same entries: K symmetric, equal flux-row norms)
template <typename T>
__device__ __forceinline__ void relax3(const AK<T>& KC, const T (&K)[3], const T (&dm)[9], T (&out)[9]) {
#pragma unroll
    for (int k = 0; k < 9; ++k)
        if (k != L9::JX && k != L9::JY) out[k] = KC.sn[k] * dm[k];
    out[L9::JX] = (K[0] * dm[L9::JX] + K[1] * dm[L9::JY]) * KC.invn_j;
    out[L9::JY] = (K[1] * dm[L9::JX] + K[2] * dm[L9::JY]) * KC.invn_j;
}

// Post-collision populations of one species with the source w_i (A + B.e_i),
// written to out[i * pl + k].
template <typename T>
__device__ __forceinline__ void collide_write(const AK<T>& KC, const T (&f)[9], const T (&m)[9], const T (&mh)[9],
                                              const T (&K)[3], T A, T Bx, T By, T* out, size_t pl, int k) {
    constexpr bool fold = sizeof(T) == 4;
    T dm[9], rl[9], bt[9];
    const T Th = m[0];
#pragma unroll
    for (int q = 0; q < 9; ++q) dm[q] = m[q] - Th * mh[q];
    relax3<T>(KC, K, dm, rl);
    if constexpr (fold) {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            if (L9::src_A(q) != 0.0) rl[q] -= T(L9::inv_n(q) * L9::src_A(q)) * A;
            if (L9::src_Bx(q) != 0.0) rl[q] -= T(L9::inv_n(q) * L9::src_Bx(q)) * Bx;
            if (L9::src_By(q) != 0.0) rl[q] -= T(L9::inv_n(q) * L9::src_By(q)) * By;
        }
    }
    Transform<T, 9>::transpose(rl, bt);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        if constexpr (fold)
            out[i * pl + k] = f[i] - bt[i];
        else
            out[i * pl + k] = f[i] - bt[i] + T(L9::w(i)) * (A + T(L9::ex(i)) * Bx + T(L9::ey(i)) * By);
    }
}

template <typename T> struct F3Args {
    const T* in;      // [27][plane] post-collision P^{n-1} (pulled), or f^0 (read locally) at n = 0
    T* out;           // [27][plane]
    T* phi;           // [3][plane] Phi^{n-1} in, Phi^n out (node-local, in place)
    T* phi_ckpt;      // [3][plane] copy of Phi^n (checkpoint slot) or null
    const T* g;       // [ny*nx] g^n or null
    const T* E;       // [ny*nx] gradient of a trial control g - lam E, or null
    T lam;
    T* tape;          // [6][plane] (u, v, G_v, G_w) or null
    double* gsq_part; // per-warp partials of sum (g^n)^2, or null
    int* status;      // status word (ST_TIMEOUT from the row-window kernels)
    int n;
};

// ------------------------------------------------------------ node bodies
// The forward and adjoint node bodies read their inputs through a source
// object: global memory (per-thread kernels) or a staged row window.

template <typename T, typename Src>
__device__ __forceinline__ void fwd3_body(const AC& C, const AK<T>& KC, const F3Args<T>& A, int y, int k,
                                          const Src& S, typename SqAccT<T>::type& acc) {
    const size_t pl = (size_t)C.plane;
    T f[3][9];
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
        for (int i = 0; i < 9; ++i) f[s][i] = S.pop(s, i);
    T prev[3];
    if (A.n > 0) {
#pragma unroll
        for (int s = 0; s < 3; ++s) prev[s] = S.phi(s);
    }
    T g = T(0);
    if (A.g) g = S.g();
    if (A.E) g = fma(-A.lam, S.E(), g); // same rounding as the accepted update
    if (A.gsq_part) acc.add(g);
    Coef3<T> nc;
    coef3_th<T>(C, KC, y, k, C.aniso == CX_ANISO_ROTATED ? S.theta() : T(0), nc);

    T m[3][9];
#pragma unroll
    for (int s = 0; s < 3; ++s) Transform<T, 9>::moments(f[s], m[s]);
    const T Tu = m[0][0], Tv = m[1][0], Tw = m[2][0];
    T Phi[3];
    Phi[0] = KC.a1 * Tu - KC.a2 * Tu * Tu;
    Phi[1] = KC.b1 * Tu - KC.b2 * Tv - KC.b3 * Tu * Tv + (C.ctrl == 1 ? g : T(0));
    Phi[2] = KC.c1 * Tu - KC.c2 * Tw + (C.ctrl == 2 ? g : T(0));
    T src[3];
#pragma unroll
    for (int s = 0; s < 3; ++s)
        src[s] = A.n == 0 ? KC.c_first * Phi[s] : KC.c_now * Phi[s] + KC.c_prev * prev[s];
    // local gradients of v and w
    T G[2][2];
#pragma unroll
    for (int s = 1; s < 3; ++s) {
        const T* K = nc.K[s];
        const T Th = m[s][0];
        const T rx = (m[s][L9::JX] - nc.ax * Th) * KC.inv_tau, ry = (m[s][L9::JY] - nc.ay * Th) * KC.inv_tau;
        const T Kax = K[0] * nc.ax + K[1] * nc.ay, Kay = K[1] * nc.ax + K[2] * nc.ay;
        G[s - 1][0] = KC.gsc * (K[0] * rx + K[1] * ry + T(0.5) * Kax * Phi[s]);
        G[s - 1][1] = KC.gsc * (K[1] * rx + K[2] * ry + T(0.5) * Kay * Phi[s]);
    }
    T mh[9];
    meq_unit<T, 9>(nc.ax, nc.ay, KC.d, mh);
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const T(&K)[3] = nc.K[s];
        const T Vx = nc.ax - T(0.5) * (K[0] * nc.ax + K[1] * nc.ay);
        const T Vy = nc.ay - T(0.5) * (K[1] * nc.ax + K[2] * nc.ay);
        T Bx = T(3) * src[s] * Vx, By = T(3) * src[s] * Vy;
        if (s == 0) { // tau S_u = 3 w_i e_i . K_u F,  F = u (chi1 G_v + chi2 G_w)
            const T Fx = Tu * (KC.chi1 * G[0][0] + KC.chi2 * G[1][0]);
            const T Fy = Tu * (KC.chi1 * G[0][1] + KC.chi2 * G[1][1]);
            Bx += T(3) * (K[0] * Fx + K[1] * Fy);
            By += T(3) * (K[1] * Fx + K[2] * Fy);
        }
        collide_write<T>(KC, f[s], m[s], mh, K, src[s], Bx, By, A.out + (size_t)s * 9 * pl, pl, k);
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        A.phi[s * pl + k] = Phi[s];
        if (A.phi_ckpt) A.phi_ckpt[s * pl + k] = Phi[s];
    }
    if (A.tape) {
        A.tape[k] = Tu;
        A.tape[pl + k] = Tv;
        A.tape[2 * pl + k] = G[0][0];
        A.tape[3 * pl + k] = G[0][1];
        A.tape[4 * pl + k] = G[1][0];
        A.tape[5 * pl + k] = G[1][1];
    }
}

template <typename T> struct A3Args {
    const T* in;       // [27][plane] psi^{n+1} (unused at the terminal step)
    const T* seed[3];  // terminal seeds psi^N_Theta,i = seed_Theta(x) (null: 0), terminal step only
    T* out;            // [27][plane] psi^n
    const T* tape;     // [6][plane]
    T* sigma;          // [3][plane] sigma^{n+1} in, sigma^n out
    const T* g;        // [ny*nx] g^n or null
    T* dJdg;           // [ny*nx] gradient of step n
    double* e2_part;   // per-warp partials of sum E^2 and max |E| (accumulated over steps)
    double* emax_part;
    int* status;       // status word (ST_TIMEOUT from the row-window kernels)
    int n, terminal;
};

template <typename T, typename Src>
__device__ __forceinline__ void adj3_body(const AC& C, const AK<T>& KC, const A3Args<T>& A, int y, int k,
                                          const Src& S, typename SqAccT<T>::type& acc) {
    constexpr bool fold = sizeof(T) == 4;
    const size_t pl = (size_t)C.plane;
    T r[3][9];
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
        for (int i = 0; i < 9; ++i) r[s][i] = S.pop(s, i);
    const T Tu = S.tape(0), Tv = S.tape(1);
    const T Gv[2] = {S.tape(2), S.tape(3)};
    const T Gw[2] = {S.tape(4), S.tape(5)};
    const T gv = A.g ? S.g() : T(0);
    // sigma^{n+1}: read with the other inputs, before this node's stores
    // (which the compiler cannot prove disjoint from it)
    T sig_next[3] = {T(0), T(0), T(0)};
    if (!A.terminal) {
#pragma unroll
        for (int s = 0; s < 3; ++s) sig_next[s] = S.sig(s);
    }
    Coef3<T> nc;
    coef3_th<T>(C, KC, y, k, C.aniso == CX_ANISO_ROTATED ? S.theta() : T(0), nc);
    T mh[9];
    meq_unit<T, 9>(nc.ax, nc.ay, KC.d, mh);

    // transposed collisions, sigma per species, Y = sum_i 3 w_i e_i rho_u,i
    T ps[3][9], sigma[3], Yx = T(0), Yy = T(0);
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const T(&K)[3] = nc.K[s];
        const T Vx = nc.ax - T(0.5) * (K[0] * nc.ax + K[1] * nc.ay);
        const T Vy = nc.ay - T(0.5) * (K[1] * nc.ax + K[2] * nc.ay);
        T mom[9], z[9], mt[9];
        Transform<T, 9>::moments(r[s], mom);
        if constexpr (fold) {
            T sA = T(0), sBx = T(0), sBy = T(0);
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                if (L9::src_A(q) != 0.0) sA += T(L9::inv_n(q) * L9::src_A(q)) * mom[q];
                if (L9::src_Bx(q) != 0.0) sBx += T(3.0 * L9::inv_n(q) * L9::src_Bx(q)) * mom[q];
                if (L9::src_By(q) != 0.0) sBy += T(3.0 * L9::inv_n(q) * L9::src_By(q)) * mom[q];
            }
            sigma[s] = sA + Vx * sBx + Vy * sBy;
            if (s == 0) {
                Yx = sBx;
                Yy = sBy;
            }
        } else {
            T sg = T(0);
#pragma unroll
            for (int i = 0; i < 9; ++i)
                sg += T(L9::w(i)) * (T(1) + T(3) * (Vx * T(L9::ex(i)) + Vy * T(L9::ey(i)))) * r[s][i];
            sigma[s] = sg;
            if (s == 0) {
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    Yx += T(3.0 * L9::w(i) * L9::ex(i)) * r[0][i];
                    Yy += T(3.0 * L9::w(i) * L9::ey(i)) * r[0][i];
                }
            }
        }
        relax3<T>(KC, K, mom, z);
        T Tc = T(0);
#pragma unroll
        for (int q = 0; q < 9; ++q) Tc += z[q] * mh[q];
        Transform<T, 9>::transpose(z, mt);
#pragma unroll
        for (int i = 0; i < 9; ++i) ps[s][i] = r[s][i] - mt[i] + Tc;
    }

    // chemotactic source of u: F = u (chi1 G_v + chi2 G_w), tau S_u = 3 w_i e_i . K_u F
    const T(&Ku)[3] = nc.K[0];
    const T aFx = Ku[0] * Yx + Ku[1] * Yy, aFy = Ku[1] * Yx + Ku[2] * Yy;
    T aT[3], aPhi[3], aj[3][2];
    aT[0] = (KC.chi1 * Gv[0] + KC.chi2 * Gw[0]) * aFx + (KC.chi1 * Gv[1] + KC.chi2 * Gw[1]) * aFy;
    aT[1] = T(0);
    aT[2] = T(0);
    aj[0][0] = aj[0][1] = T(0);
    const T chis[2] = {KC.chi1, KC.chi2};
#pragma unroll
    for (int s = 1; s < 3; ++s) {
        // G = -(K (j - a Theta)/tau + K a Phi/2) / (d Cs^2)
        const T(&K)[3] = nc.K[s];
        const T aGx = chis[s - 1] * Tu * aFx, aGy = chis[s - 1] * Tu * aFy;
        const T KGx = K[0] * aGx + K[1] * aGy, KGy = K[1] * aGx + K[2] * aGy;
        aj[s][0] = -KGx * KC.asc * KC.inv_tau;
        aj[s][1] = -KGy * KC.asc * KC.inv_tau;
        const T aKG = nc.ax * KGx + nc.ay * KGy;
        aT[s] = aKG * KC.asc * KC.inv_tau;
        aPhi[s] = T(-0.5) * aKG * KC.asc;
    }
    aPhi[0] = T(0);
    // sources: Phi^n at step n (c_n) and at step n + 1 (c'_{n+1})
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        aPhi[s] += (A.n == 0 ? KC.c_first : KC.c_now) * sigma[s];
        if (!A.terminal) aPhi[s] += KC.c_prev * sig_next[s];
        A.sigma[s * pl + k] = sigma[s];
    }
    // kinetics
    aT[0] += (KC.a1 - T(2) * KC.a2 * Tu) * aPhi[0] + (KC.b1 - KC.b3 * Tv) * aPhi[1] + KC.c1 * aPhi[2];
    aT[1] += -(KC.b2 + KC.b3 * Tu) * aPhi[1];
    aT[2] += -KC.c2 * aPhi[2];
    const T E = aPhi[C.ctrl] + KC.two_alpha * gv;
    A.dJdg[k] = E;
    if (A.e2_part) acc.add(E);
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
        for (int i = 0; i < 9; ++i)
            A.out[(s * 9 + i) * pl + k] = ps[s][i] + aT[s] + T(L9::ex(i)) * aj[s][0] + T(L9::ey(i)) * aj[s][1];
}

// ------------------------------------------------------ per-thread kernels
// One node per thread and iteration of a grid-stride loop; inputs straight
// from global memory.

template <typename T> struct GFwd {
    const AC& C;
    const F3Args<T>& A;
    size_t pl;
    int k, ks[9];
    __device__ __forceinline__ T pop(int s, int i) const { return ld(A.in + (s * 9 + i) * pl + ks[i]); }
    __device__ __forceinline__ T phi(int s) const { return A.phi[s * pl + k]; }
    __device__ __forceinline__ T g() const { return ld(A.g + k); }
    __device__ __forceinline__ T E() const { return ld(A.E + k); }
    __device__ __forceinline__ T theta() const { return ld(reinterpret_cast<const T*>(C.theta) + k); }
};

// FP32: 256 threads, at least 3 blocks per SM (<= 85 registers), measured faster
// than 2 blocks with more registers and than 4 blocks with heavier spilling.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) k3_forward(const AC C, const AK<T> KC, const F3Args<T> A) {
    const int total = C.nx * C.ny;
    typename SqAccT<T>::type acc;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        const int y = k / C.nx, x = k - y * C.nx;
        GFwd<T> S{C, A, (size_t)C.plane, k, {}};
        if (A.n == 0) {
#pragma unroll
            for (int i = 0; i < 9; ++i) S.ks[i] = k;
        } else {
            const int xm = x == 0 ? C.nx - 1 : x - 1, xp = x == C.nx - 1 ? 0 : x + 1;
            const int rm = (y == 0 ? C.ny - 1 : y - 1) * C.nx, r0 = y * C.nx;
            const int rp = (y == C.ny - 1 ? 0 : y + 1) * C.nx;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int xs = L9::ex(i) > 0 ? xm : (L9::ex(i) < 0 ? xp : x);
                S.ks[i] = (L9::ey(i) > 0 ? rm : (L9::ey(i) < 0 ? rp : r0)) + xs;
            }
        }
        fwd3_body<T>(C, KC, A, y, k, S, acc);
    }
    if (A.gsq_part) acc.flush(A.gsq_part + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5), nullptr);
}

template <typename T> struct GAdj {
    const AC& C;
    const A3Args<T>& A;
    size_t pl;
    int k, kd[9];
    __device__ __forceinline__ T pop(int s, int i) const {
        if (A.terminal) return A.seed[s] ? ld(A.seed[s] + kd[i]) : T(0);
        return ld(A.in + (s * 9 + i) * pl + kd[i]);
    }
    __device__ __forceinline__ T tape(int c) const { return ld(A.tape + c * pl + k); }
    __device__ __forceinline__ T sig(int s) const { return A.sigma[s * pl + k]; }
    __device__ __forceinline__ T g() const { return ld(A.g + k); }
    __device__ __forceinline__ T theta() const { return ld(reinterpret_cast<const T*>(C.theta) + k); }
};

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) k3_adjoint(const AC C, const AK<T> KC, const A3Args<T> A) {
    const int total = C.nx * C.ny;
    typename SqAccT<T>::type acc;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        const int y = k / C.nx, x = k - y * C.nx;
        const int xm = x == 0 ? C.nx - 1 : x - 1, xp = x == C.nx - 1 ? 0 : x + 1;
        const int rm = (y == 0 ? C.ny - 1 : y - 1) * C.nx, r0 = y * C.nx;
        const int rp = (y == C.ny - 1 ? 0 : y + 1) * C.nx;
        GAdj<T> S{C, A, (size_t)C.plane, k, {}};
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int xd = L9::ex(i) > 0 ? xp : (L9::ex(i) < 0 ? xm : x);
            S.kd[i] = (L9::ey(i) > 0 ? rp : (L9::ey(i) < 0 ? rm : r0)) + xd;
        }
        adj3_body<T>(C, KC, A, y, k, S, acc);
    }
    if (A.e2_part) {
        const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        acc.flush(A.e2_part + w, A.emax_part + w);
    }
}

// ------------------------------------------------------ row-window kernels
// Steps whose inputs are all pulled (forward n >= 1, adjoint below the
// terminal step) on grids whose rows are a whole number of 16-byte units:
// the warp-specialised pipeline of cx_rows.cuh.  A producer warp issues, per
// row segment (FNT or ANT nodes), one bulk copy per population plane of the source
// row window (the segment widened by 16 bytes on each side; periodic ends from
// the other end of the row) and of the node-local planes, completing on the
// stage's mbarrier; the compute warps read everything from shared memory.

// Row segments of FNT nodes (forward) and ANT nodes (adjoint): the forward's
// FP32 stages of 256 nodes leave two blocks per SM, which measured faster
// than four blocks of 128; FP64 (the parity mode) and the adjoint keep 128.
template <typename T> constexpr int FNT = sizeof(T) == 4 ? 256 : 128;
constexpr int ANT = 128;
template <typename T, int NT> struct RW3 {
    static constexpr int H = 16 / (int)sizeof(T);
    static constexpr int W = NT + 2 * H;
};
// stage layout: 27 population windows, then per-node planes of NT values
template <typename T> constexpr int fwd3_stage_values() { return 27 * RW3<T, FNT<T>>::W + 6 * FNT<T>; } // theta, g, E, Phi x3
template <typename T> constexpr int adj3_stage_values() {
    return 27 * RW3<T, ANT>::W + 11 * ANT; // tape x6, sigma x3, g, theta
}

template <typename T> struct SFwd {
    const T* s; // stage + threadIdx.x
    __device__ __forceinline__ T pop(int sp, int i) const { return s[(sp * 9 + i) * RW3<T, FNT<T>>::W + RW3<T, FNT<T>>::H - L9::ex(i)]; }
    __device__ __forceinline__ T theta() const { return s[27 * RW3<T, FNT<T>>::W]; }
    __device__ __forceinline__ T g() const { return s[27 * RW3<T, FNT<T>>::W + FNT<T>]; }
    __device__ __forceinline__ T E() const { return s[27 * RW3<T, FNT<T>>::W + 2 * FNT<T>]; }
    __device__ __forceinline__ T phi(int sp) const { return s[27 * RW3<T, FNT<T>>::W + (3 + sp) * FNT<T>]; }
};
template <typename T> struct SAdj {
    const T* s;
    __device__ __forceinline__ T pop(int sp, int i) const { return s[(sp * 9 + i) * RW3<T, ANT>::W + RW3<T, ANT>::H + L9::ex(i)]; }
    __device__ __forceinline__ T tape(int c) const { return s[27 * RW3<T, ANT>::W + c * ANT]; }
    __device__ __forceinline__ T sig(int sp) const { return s[27 * RW3<T, ANT>::W + (6 + sp) * ANT]; }
    __device__ __forceinline__ T g() const { return s[27 * RW3<T, ANT>::W + 9 * ANT]; }
    __device__ __forceinline__ T theta() const { return s[27 * RW3<T, ANT>::W + 10 * ANT]; }
};

template <typename T>
__device__ __forceinline__ void fwd3_issue(const AC& C, const F3Args<T>& A, int y, int x0, T* st, uint64_t* bar) {
    constexpr int H = RW3<T, FNT<T>>::H, W = RW3<T, FNT<T>>::W;
    const int nx = C.nx, nv = min(FNT<T>, nx - x0);
    const int rm = y == 0 ? C.ny - 1 : y - 1, rp = y == C.ny - 1 ? 0 : y + 1;
    const bool rot = C.aniso == CX_ANISO_ROTATED;
    const uint32_t nb = (uint32_t)nv * sizeof(T);
    const size_t pl = (size_t)C.plane, k0 = (size_t)y * nx + x0;
    mbar_expect_tx(bar, (uint32_t)(27 * (nv + 2 * H)) * sizeof(T) + nb * (3u + rot + (A.g ? 1u : 0u) + (A.E ? 1u : 0u)));
#pragma unroll
    for (int j = 0; j < 27; ++j) {
        const int i = j % 9;
        const int ys = L9::ey(i) > 0 ? rm : (L9::ey(i) < 0 ? rp : y); // pull from x - e_i
        bulk_row_window<T, FNT<T>>(st + j * W, A.in + j * pl + (size_t)ys * nx, x0, nv, nx, bar);
    }
    T* const loc = st + 27 * W;
    if (rot) bulk_g2s(loc, reinterpret_cast<const T*>(C.theta) + k0, nb, bar);
    if (A.g) bulk_g2s(loc + FNT<T>, A.g + k0, nb, bar);
    if (A.E) bulk_g2s(loc + 2 * FNT<T>, A.E + k0, nb, bar);
#pragma unroll
    for (int s = 0; s < 3; ++s) bulk_g2s(loc + (3 + s) * FNT<T>, A.phi + s * pl + k0, nb, bar);
}

template <typename T>
__device__ __forceinline__ void adj3_issue(const AC& C, const A3Args<T>& A, int y, int x0, T* st, uint64_t* bar) {
    constexpr int H = RW3<T, ANT>::H, W = RW3<T, ANT>::W;
    const int nx = C.nx, nv = min(ANT, nx - x0);
    const int rm = y == 0 ? C.ny - 1 : y - 1, rp = y == C.ny - 1 ? 0 : y + 1;
    const bool rot = C.aniso == CX_ANISO_ROTATED;
    const uint32_t nb = (uint32_t)nv * sizeof(T);
    const size_t pl = (size_t)C.plane, k0 = (size_t)y * nx + x0;
    mbar_expect_tx(bar, (uint32_t)(27 * (nv + 2 * H)) * sizeof(T) + nb * (9u + rot + (A.g ? 1u : 0u)));
#pragma unroll
    for (int j = 0; j < 27; ++j) {
        const int i = j % 9;
        const int ys = L9::ey(i) > 0 ? rp : (L9::ey(i) < 0 ? rm : y); // pull from x + e_i
        bulk_row_window<T, ANT>(st + j * W, A.in + j * pl + (size_t)ys * nx, x0, nv, nx, bar);
    }
    T* const loc = st + 27 * W;
#pragma unroll
    for (int c = 0; c < 6; ++c) bulk_g2s(loc + c * ANT, A.tape + c * pl + k0, nb, bar);
#pragma unroll
    for (int s = 0; s < 3; ++s) bulk_g2s(loc + (6 + s) * ANT, A.sigma + s * pl + k0, nb, bar);
    if (A.g) bulk_g2s(loc + 9 * ANT, A.g + k0, nb, bar);
    if (rot) bulk_g2s(loc + 10 * ANT, reinterpret_cast<const T*>(C.theta) + k0, nb, bar);
}

// Block: FNT (ANT) compute threads and one producer warp.  CC describes the grid to
// the pipeline's segment walk (no solid nodes, whole-grid control).
template <typename T>
// (register cap: two blocks of FNT + 32 threads per SM, which is what shared
// memory allows, without spills in FP32)
__global__ void __maxnreg__(sizeof(T) == 4 ? 104 : 224)
    k3_forward_rows(const CxConst CC, const AC C, const AK<T> KC, const F3Args<T> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RowsPipe<T, FNT<T>> pipe(smem_raw, fwd3_stage_values<T>());
    pipe.init();
    allow_next_grid();
    wait_prior_grid(); // the previous step's populations and node state are complete
    if (block_sees_timeout(A.status)) return;
    if (threadIdx.x >= FNT<T>) {
        pipe.produce(CC, A.status, [&](int y, int x0, T* st, uint64_t* bar) { fwd3_issue<T>(C, A, y, x0, st, bar); });
        return;
    }
    typename SqAccT<T>::type acc;
    pipe.consume(
        CC, A.status, [&](const NodeIdx&, T*) {},
        [&](const NodeIdx& nd, T* st) {
            if (nd.fluid) fwd3_body<T>(C, KC, A, nd.y, nd.k, SFwd<T>{st + threadIdx.x}, acc);
        });
    if (A.gsq_part) acc.flush(A.gsq_part + blockIdx.x * (FNT<T> >> 5) + (threadIdx.x >> 5), nullptr);
}

template <typename T>
__global__ void __launch_bounds__(ANT + 32, sizeof(T) == 4 ? 3 : 2)
    k3_adjoint_rows(const CxConst CC, const AC C, const AK<T> KC, const A3Args<T> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RowsPipe<T, ANT> pipe(smem_raw, adj3_stage_values<T>());
    pipe.init();
    allow_next_grid();
    wait_prior_grid();
    if (block_sees_timeout(A.status)) return;
    if (threadIdx.x >= ANT) {
        pipe.produce(CC, A.status, [&](int y, int x0, T* st, uint64_t* bar) { adj3_issue<T>(C, A, y, x0, st, bar); });
        return;
    }
    typename SqAccT<T>::type acc;
    pipe.consume(
        CC, A.status, [&](const NodeIdx&, T*) {},
        [&](const NodeIdx& nd, T* st) {
            if (nd.fluid) adj3_body<T>(C, KC, A, nd.y, nd.k, SAdj<T>{st + threadIdx.x}, acc);
        });
    if (A.e2_part) {
        const int w = blockIdx.x * (ANT >> 5) + (threadIdx.x >> 5);
        acc.flush(A.e2_part + w, A.emax_part + w);
    }
}

// f^0 = phi^eq(Theta_0) for the three species: w_i aleph_i Theta_0 with
// aleph_i = 1 + 3 a.e + 4.5 ((a.e)^2 - |a|^2/3) + 1.5 (d - 1)(|e|^2 - 2/3).
template <typename T>
__global__ void k3_init(const AC C, const AK<T> KC, const double* u0, const double* v0, const double* w0, T* P) {
    const int total = C.nx * C.ny;
    const size_t pl = (size_t)C.plane;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        const int y = k / C.nx;
        Coef3<T> nc;
        coef3<T>(C, KC, y, k, nc);
        const T Th[3] = {T(u0[k]), T(v0[k]), T(w0[k])};
        const T a2 = nc.ax * nc.ax + nc.ay * nc.ay;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const T ea = nc.ax * T(L9::ex(i)) + nc.ay * T(L9::ey(i));
            const T e2 = T(L9::ex(i) * L9::ex(i) + L9::ey(i) * L9::ey(i));
            const T al = T(1) + T(3) * ea + T(4.5) * (ea * ea - a2 * T(1.0 / 3.0)) +
                         T(1.5) * (KC.d - T(1)) * (e2 - T(2.0 / 3.0));
#pragma unroll
            for (int s = 0; s < 3; ++s) P[(s * 9 + i) * pl + k] = T(L9::w(i)) * al * Th[s];
        }
    }
}

// Theta^N = sum_i P^{N-1}_Theta,i(x - e_i) (eq. UGS), the terminal seed
// u^N - u_target and the block partial of 1/2 sum (u^N - u_target)^2 (FP64).
template <typename T>
__global__ void __launch_bounds__(256) k3_final(const AC C, const T* Pin, const T* ut, T* uvw, T* wu,
                                                 double* cost_part) {
    __shared__ double red[32];
    const int total = C.nx * C.ny;
    const size_t pl = (size_t)C.plane;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double cst = 0.0;
    if (k < total) {
        const int y = k / C.nx, x = k - y * C.nx;
        const int xm = x == 0 ? C.nx - 1 : x - 1, xp = x == C.nx - 1 ? 0 : x + 1;
        const int ym = y == 0 ? C.ny - 1 : y - 1, yp = y == C.ny - 1 ? 0 : y + 1;
        T s3[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int xs = L9::ex(i) > 0 ? xm : (L9::ex(i) < 0 ? xp : x);
            const int ys = L9::ey(i) > 0 ? ym : (L9::ey(i) < 0 ? yp : y);
#pragma unroll
            for (int s = 0; s < 3; ++s) s3[s] += Pin[(s * 9 + i) * pl + ys * C.nx + xs];
        }
#pragma unroll
        for (int s = 0; s < 3; ++s) uvw[s * pl + k] = s3[s];
        const T w = s3[0] - ut[k];
        wu[k] = w;
        cst = 0.5 * (double)w * (double)w;
    }
    const double b = block_sum(cst, red);
    if (threadIdx.x == 0) cost_part[blockIdx.x] = b;
}

// Descriptor fields in the kernels' precision: theta, K per node (FIELD; the
// map K = (D / (d Cs^2 tau) + I/2)^-1 with its eigenvalues checked in (0, 2)),
// a, u_target.
template <typename T>
__global__ void k3_setup(const AC C, const cx3_desc d, T* theta, T* Kf, T* a, T* ut, int* status) {
    const int total = C.nx * C.ny;
    const size_t pl = (size_t)C.plane;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        if (theta) theta[k] = T(d.theta[k]);
        if (Kf) {
            const double* D[3] = {d.D_u_field, d.D_v_field, d.D_w_field};
            const double sc = 1.0 / (d.d * (1.0 / 3.0) * d.tau);
            for (int s = 0; s < 3; ++s) {
                const double p = D[s][3 * k] * sc + 0.5, q = D[s][3 * k + 1] * sc, r = D[s][3 * k + 2] * sc + 0.5;
                const double det = p * r - q * q;
                const double k0 = r / det, k1 = -q / det, k2 = p / det;
                const double tr = k0 + k2, dt = k0 * k2 - k1 * k1;
                const double disc = sqrt(fmax(0.0, 0.25 * tr * tr - dt));
                if (!(det > 0.0) || !(0.5 * tr - disc > 0.0) || !(0.5 * tr + disc < 2.0)) atomicOr(status, ST_UNSTABLE);
                Kf[(3 * s) * pl + k] = T(k0);
                Kf[(3 * s + 1) * pl + k] = T(k1);
                Kf[(3 * s + 2) * pl + k] = T(k2);
            }
        }
        if (a && C.adv == CX_ADV_FIELD) {
            a[k] = T(d.a[2 * k]);
            a[pl + k] = T(d.a[2 * k + 1]);
        }
        if (a && C.adv == CX_ADV_ROW && k < C.ny) {
            a[2 * k] = T(d.a[2 * k]);
            a[2 * k + 1] = T(d.a[2 * k + 1]);
        }
        ut[k] = T(d.u_target[k]);
    }
}

} // namespace arc
} // namespace cx

using namespace cx;
using namespace cx::arc;

// ================================================================ host side

namespace {

struct Lay3 {
    size_t plane, esz;
    int N, k, S, nparts;
    size_t off_popA, off_popB, off_adjA, off_adjB, off_ckpt, off_phi, off_sigma, off_tape, off_uvw, off_wu,
        off_theta, off_K, off_a, off_ut, off_part, off_scal, off_status, total;
};

constexpr size_t AL = 256;
inline size_t upa(size_t v, size_t a) { return (v + a - 1) / a * a; }
constexpr int MAXW = 32768; // warps of a persistent launch

Lay3 layout3(const cx3_desc* d) {
    Lay3 L{};
    L.esz = d->precision == 64 ? 8 : 4;
    L.N = d->n_steps;
    L.k = d->ckpt_every > 0 ? std::min(d->ckpt_every, d->n_steps) : d->n_steps;
    L.S = (L.N + L.k - 1) / L.k;
    L.plane = upa((size_t)d->nx * d->ny, 64);
    L.nparts = std::max((int)((d->nx * (long long)d->ny + 255) / 256), MAXW);
    const size_t fld = L.plane * L.esz, pop = 27 * fld;
    size_t o = 0;
    auto take = [&](size_t b) {
        const size_t r = o;
        o = upa(o + b, AL);
        return r;
    };
    L.off_popA = take(pop);
    L.off_popB = take(pop);
    L.off_adjA = take(pop);
    L.off_adjB = take(pop);
    L.off_ckpt = take((pop + 3 * fld) * L.S); // per slot: 27 population planes, then Phi (3 planes)
    L.off_phi = take(3 * fld);
    L.off_sigma = take(3 * fld);
    L.off_tape = take(6 * fld * L.k);
    L.off_uvw = take(3 * fld);
    L.off_wu = take(fld);
    L.off_theta = take(d->aniso == CX_ANISO_ROTATED ? fld : 0);
    L.off_K = take(d->aniso == CX_ANISO_FIELD ? 9 * fld : 0);
    L.off_a = take(d->adv == CX_ADV_FIELD ? 2 * fld : (d->adv == CX_ADV_ROW ? 2 * (size_t)d->ny * L.esz : 0));
    L.off_ut = take(fld);
    L.off_part = take(sizeof(double) * 4 * (size_t)L.nparts);
    L.off_scal = take(sizeof(double) * 16);
    L.off_status = take(sizeof(int) * 4);
    L.total = o;
    return L;
}

cx_status validate3(const cx3_desc* d) {
    if (!d) return CX_ERR_INVALID_ARG;
    if (d->nx < 3 || d->ny < 3 || d->n_steps < 1) return CX_ERR_INVALID_ARG;
    if ((long long)d->nx * d->ny > (1LL << 30)) return CX_ERR_INVALID_ARG;
    if (d->precision != 32 && d->precision != 64) return CX_ERR_INVALID_ARG;
    if (d->ckpt_every < 0) return CX_ERR_INVALID_ARG;
    if (!(d->tau > 0.0) || !(d->d > 0.0) || !(d->alpha >= 0.0)) return CX_ERR_INVALID_ARG;
    const double pars[9] = {d->chi1, d->chi2, d->a1, d->a2, d->b1, d->b2, d->b3, d->c1, d->c2};
    for (double v : pars)
        if (!std::isfinite(v)) return CX_ERR_INVALID_ARG;
    for (int i = 0; i < 7; ++i)
        if (!(d->s[i] > 0.0 && d->s[i] < 2.0)) return CX_ERR_INVALID_ARG;
    if (d->source_order != 1 && d->source_order != 2) return CX_ERR_INVALID_ARG;
    if (d->ctrl_species != 1 && d->ctrl_species != 2) return CX_ERR_INVALID_ARG;
    if (d->aniso < 0 || d->aniso > 2 || d->adv < 0 || d->adv > 2) return CX_ERR_INVALID_ARG;
    if (d->aniso == CX_ANISO_ROTATED && !d->theta) return CX_ERR_INVALID_ARG;
    if (d->aniso == CX_ANISO_FIELD && (!d->D_u_field || !d->D_v_field || !d->D_w_field)) return CX_ERR_INVALID_ARG;
    if (d->adv != CX_ADV_NONE && !d->a) return CX_ERR_INVALID_ARG;
    if (!d->u_target) return CX_ERR_INVALID_ARG;
    return CX_OK;
}

// K = (D / (d Cs^2 tau) + I/2)^-1 with eigenvalues in (0, 2)
bool K_of(const double D[3], double dd, double tau, double K[3]) {
    const double sc = 1.0 / (dd * (1.0 / 3.0) * tau);
    const double a = D[0] * sc + 0.5, b = D[1] * sc, c = D[2] * sc + 0.5;
    const double det = a * c - b * b;
    if (!(det > 0.0)) return false;
    K[0] = c / det;
    K[1] = -b / det;
    K[2] = a / det;
    const double tr = K[0] + K[2], dt = K[0] * K[2] - K[1] * K[1];
    const double disc = std::sqrt(std::max(0.0, tr * tr / 4 - dt));
    return tr / 2 - disc > 0.0 && tr / 2 + disc < 2.0;
}

template <typename T> AK<T> make_ak(const cx3_desc& d, bool* ok) {
    AK<T> K{};
    *ok = true;
    for (int k = 0; k < 9; ++k) {
        const int r = rate_index<9>(k);
        K.sn[k] = r >= 0 ? T(d.s[r] * Lat<9>::inv_n(k)) : T(0);
    }
    K.invn_j = T(Lat<9>::inv_n(Lat<9>::JX));
    const double* Dc[3] = {d.D_u, d.D_v, d.D_w};
    const double* lam[3] = {d.lam_u, d.lam_v, d.lam_w};
    for (int s = 0; s < 3; ++s) {
        if (d.aniso == CX_ANISO_CONST) {
            double Kd[3];
            if (!K_of(Dc[s], d.d, d.tau, Kd)) *ok = false;
            for (int j = 0; j < 3; ++j) K.K[s][j] = T(Kd[j]);
        } else if (d.aniso == CX_ANISO_ROTATED) {
            double k1 = 1.0 / (lam[s][0] / (d.d * (1.0 / 3.0) * d.tau) + 0.5);
            double k2 = 1.0 / (lam[s][1] / (d.d * (1.0 / 3.0) * d.tau) + 0.5);
            if (!(k1 > 0.0 && k1 < 2.0 && k2 > 0.0 && k2 < 2.0 && lam[s][0] >= 0.0 && lam[s][1] >= 0.0)) *ok = false;
            K.kbar[s] = T(0.5 * (k1 + k2));
            K.kd[s] = T(0.5 * (k1 - k2));
        }
    }
    K.tau = T(d.tau);
    K.inv_tau = T(1.0 / d.tau);
    K.gsc = T(-3.0 / d.d);
    K.asc = T(3.0 / d.d);
    K.d = T(d.d);
    K.chi1 = T(d.chi1);
    K.chi2 = T(d.chi2);
    K.a1 = T(d.a1);
    K.a2 = T(d.a2);
    K.b1 = T(d.b1);
    K.b2 = T(d.b2);
    K.b3 = T(d.b3);
    K.c1 = T(d.c1);
    K.c2 = T(d.c2);
    K.two_alpha = T(2.0 * d.alpha);
    K.c_first = T(d.tau);
    K.c_now = T(d.source_order == 1 ? d.tau : 1.5 * d.tau);
    K.c_prev = T(d.source_order == 1 ? 0.0 : -0.5 * d.tau);
    return K;
}

struct Range3 {
    int phase;
    long long launches;
    cudaEvent_t a, b;
};

} // namespace

struct cx3_problem {
    cx3_desc d;
    AC C;
    Lay3 lay;
    cudaStream_t stream;
    char* ws;
    AK<float> Kf;
    AK<double> Kd;
    const AK<float>& kc(float*) const { return Kf; }
    const AK<double>& kc(double*) const { return Kd; }
    int grid_f = 1, grid_a = 1, nblk = 1; // persistent grids (forward, adjoint), blocks of k3_final
    int grid_fr = 1, grid_ar = 1;          // persistent grids of the row-window kernels
    int rows_mode = 1;                     // cx3_set_staging
    CxConst CC{};                          // the grid as the row-window pipeline walks it
    bool has_init = false, fwd_valid = false, adj_valid = false, tape_last_valid = false;
    bool have_lam = false;
    double lam_prev = 0.0;
    bool timing = false;
    std::vector<Range3> ranges;
    size_t n_ranges = 0;

    template <typename P> P* at(size_t off) const { return reinterpret_cast<P*>(ws + off); }
    size_t fld() const { return lay.plane * lay.esz; }
    char* slot(int s) const { return ws + lay.off_ckpt + (size_t)s * 30 * fld(); }
    char* slot_phi(int s) const { return slot(s) + 27 * fld(); }
    char* tape(int j) const { return ws + lay.off_tape + (size_t)j * 6 * fld(); }
};

#define CX3_CUDA(x)                                                                                                  \
    do {                                                                                                             \
        if ((x) != cudaSuccess) return CX_ERR_CUDA;                                                                  \
    } while (0)

namespace {

enum { R_FWD = 0, R_REC = 1, R_ADJ = 2 };

void rbegin(cx3_problem* p, int phase, Range3** r) {
    *r = nullptr;
    if (!p->timing) return;
    if (p->n_ranges == p->ranges.size()) {
        Range3 x{};
        cudaEventCreate(&x.a);
        cudaEventCreate(&x.b);
        p->ranges.push_back(x);
    }
    Range3* q = &p->ranges[p->n_ranges++];
    q->phase = phase;
    q->launches = 0;
    cudaEventRecord(q->a, p->stream);
    *r = q;
}
void rend(cx3_problem* p, Range3* r, long long launches) {
    if (!r) return;
    cudaEventRecord(r->b, p->stream);
    r->launches = launches;
}

// Row-window kernels for a step whose inputs are all pulled, on rows of whole
// 16-byte units with 16-byte aligned planes; mode 1 also asks for at least
// two row segments per block (else nothing overlaps the copies).
bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; }

template <typename T> bool rows_ok(const cx3_problem* p, const T* in, const T* g, const T* extra) {
    if (p->rows_mode == 0 || p->C.nx % (16 / (int)sizeof(T)) != 0) return false;
    if (!aligned16(in) || !aligned16(p->ws) || (g && !aligned16(g)) || (extra && !aligned16(extra))) return false;
    const long long segf = (long long)((p->C.nx + FNT<T> - 1) / FNT<T>) * p->C.ny;
    const long long sega = (long long)((p->C.nx + ANT - 1) / ANT) * p->C.ny;
    return p->rows_mode == 2 || (segf >= 2LL * p->grid_fr && sega >= 2LL * p->grid_ar);
}

template <typename T> cudaError_t launch_rows(const void* kern, int grid, int threads, size_t smem, cudaStream_t s,
                                               void** args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, kern, args);
}

template <typename T> cudaError_t launch_fwd3(cx3_problem* p, const F3Args<T>& A) {
    const AK<T>& K = p->kc((T*)nullptr);
    if (A.n > 0 && rows_ok<T>(p, A.in, A.g, A.E)) {
        void* args[] = {(void*)&p->CC, (void*)&p->C, (void*)&K, (void*)&A};
        return launch_rows<T>((const void*)k3_forward_rows<T>, p->grid_fr, FNT<T> + 32, rows_pipe_smem<T>(fwd3_stage_values<T>()),
                              p->stream, args);
    }
    k3_forward<T><<<p->grid_f, 256, 0, p->stream>>>(p->C, K, A);
    return cudaGetLastError();
}

// The adjoint takes the row-window kernel only when asked to (mode 2): at
// 1024^2 it measured slower than the per-thread kernel (57.7 against 53.8 us
// per step; 127 registers and 61 KB of stages leave 12 compute warps per SM
// to a body that issues on 60% of the cycles, against 24 warps).
template <typename T> cudaError_t launch_adj3(cx3_problem* p, const AK<T>& K, const A3Args<T>& A) {
    if (!A.terminal && p->rows_mode == 2 && rows_ok<T>(p, A.in, A.g, nullptr)) {
        void* args[] = {(void*)&p->CC, (void*)&p->C, (void*)&K, (void*)&A};
        return launch_rows<T>((const void*)k3_adjoint_rows<T>, p->grid_ar, ANT + 32, rows_pipe_smem<T>(adj3_stage_values<T>()),
                              p->stream, args);
    }
    k3_adjoint<T><<<p->grid_a, 256, 0, p->stream>>>(p->C, K, A);
    return cudaGetLastError();
}

template <typename T>
cx_status run3_forward(cx3_problem* p, const T* g, const T* E, double lam, double* J_dev, bool flag_unstable) {
    const Lay3& Ly = p->lay;
    const size_t nn = (size_t)p->d.nx * p->d.ny; // control and gradient planes are unpadded [N][ny][nx]
    double* part = p->at<double>(Ly.off_part);
    double* gsq = part + Ly.nparts;
    const int fw = std::max(p->grid_f * 8, p->grid_fr * (FNT<T> / 32));
    CX3_CUDA(cudaMemsetAsync(gsq, 0, sizeof(double) * fw, p->stream));
    Range3* r;
    rbegin(p, R_FWD, &r);
    const T* in = reinterpret_cast<const T*>(p->slot(0));
    T* phi = p->at<T>(Ly.off_phi);
    for (int n = 0; n < Ly.N; ++n) {
        const int seg = n / Ly.k;
        F3Args<T> A{};
        T* out;
        if (n + 1 < Ly.N && (n + 1) % Ly.k == 0) {
            out = reinterpret_cast<T*>(p->slot((n + 1) / Ly.k));
            A.phi_ckpt = reinterpret_cast<T*>(p->slot_phi((n + 1) / Ly.k));
        } else {
            out = p->at<T>((n % 2) ? Ly.off_popB : Ly.off_popA);
        }
        A.in = in;
        A.out = out;
        A.phi = phi;
        A.g = g ? g + (size_t)n * nn : nullptr;
        A.E = E ? E + (size_t)n * nn : nullptr;
        A.lam = T(lam);
        A.tape = (seg == Ly.S - 1) ? reinterpret_cast<T*>(p->tape(n - seg * Ly.k)) : nullptr;
        A.gsq_part = gsq;
        A.status = p->at<int>(Ly.off_status);
        A.n = n;
        CX3_CUDA(launch_fwd3<T>(p, A));
        in = out;
    }
    rend(p, r, Ly.N);
    double* cost = part;
    k3_final<T><<<p->nblk, 256, 0, p->stream>>>(p->C, in, p->at<T>(Ly.off_ut), p->at<T>(Ly.off_uvw),
                                                 p->at<T>(Ly.off_wu), cost);
    CX3_CUDA(cudaGetLastError());
    double* scal = p->at<double>(Ly.off_scal);
    CX3_CUDA(launch_finalize(cost, p->nblk, gsq, fw, p->d.alpha, scal, p->at<int>(Ly.off_status),
                             flag_unstable ? ST_UNSTABLE : 0, 0, p->stream));
    if (J_dev) CX3_CUDA(cudaMemcpyAsync(J_dev, scal, sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
    p->fwd_valid = true;
    p->adj_valid = false;
    p->tape_last_valid = true;
    return CX_OK;
}

template <typename T>
cx_status run3_adjoint(cx3_problem* p, const T* g, const T* const (&seeds)[3], bool penalty, T* dJdg) {
    const Lay3& Ly = p->lay;
    const size_t nn = (size_t)p->d.nx * p->d.ny; // control and gradient planes are unpadded [N][ny][nx]
    AK<T> KA = p->kc((T*)nullptr);
    if (!penalty) KA.two_alpha = T(0);
    double* part = p->at<double>(Ly.off_part);
    double* e2 = part + 2 * (size_t)Ly.nparts;
    double* emax = part + 3 * (size_t)Ly.nparts;
    CX3_CUDA(cudaMemsetAsync(e2, 0, sizeof(double) * 2 * Ly.nparts, p->stream));
    const int aw = std::max(p->grid_a * 8, p->grid_ar * (ANT / 32));
    T* sigma = p->at<T>(Ly.off_sigma);
    T* phi = p->at<T>(Ly.off_phi);
    const bool cost_seed = !seeds[0] && !seeds[1] && !seeds[2];
    const T* sd[3] = {cost_seed ? p->at<T>(Ly.off_wu) : seeds[0], seeds[1], seeds[2]};
    const T* psi_in = nullptr;
    for (int s = Ly.S - 1; s >= 0; --s) {
        const int n0 = s * Ly.k, n1 = std::min(Ly.N, n0 + Ly.k);
        if (s < Ly.S - 1 || !p->tape_last_valid) {
            Range3* r;
            rbegin(p, R_REC, &r);
            if (s >= 1)
                CX3_CUDA(cudaMemcpyAsync(phi, p->slot_phi(s), 3 * p->fld(), cudaMemcpyDeviceToDevice, p->stream));
            const T* in = reinterpret_cast<const T*>(p->slot(s));
            for (int n = n0; n < n1; ++n) {
                F3Args<T> A{};
                T* out = p->at<T>((n % 2) ? Ly.off_popB : Ly.off_popA);
                A.in = in;
                A.out = out;
                A.phi = phi;
                A.g = g ? g + (size_t)n * nn : nullptr;
                A.tape = reinterpret_cast<T*>(p->tape(n - n0));
                A.status = p->at<int>(Ly.off_status);
                A.n = n;
                CX3_CUDA(launch_fwd3<T>(p, A));
                in = out;
            }
            rend(p, r, n1 - n0);
        }
        Range3* r;
        rbegin(p, R_ADJ, &r);
        for (int n = n1 - 1; n >= n0; --n) {
            A3Args<T> A{};
            A.terminal = n == Ly.N - 1;
            T* out = p->at<T>((n % 2) ? Ly.off_adjB : Ly.off_adjA);
            A.in = psi_in;
            for (int q = 0; q < 3; ++q) A.seed[q] = sd[q];
            A.out = out;
            A.tape = reinterpret_cast<const T*>(p->tape(n - n0));
            A.sigma = sigma;
            A.g = g ? g + (size_t)n * nn : nullptr;
            A.dJdg = dJdg + (size_t)n * nn;
            A.e2_part = e2;
            A.emax_part = emax;
            A.status = p->at<int>(Ly.off_status);
            A.n = n;
            CX3_CUDA(launch_adj3<T>(p, KA, A));
            psi_in = out;
        }
        rend(p, r, n1 - n0);
    }
    double* scal = p->at<double>(Ly.off_scal);
    CX3_CUDA(launch_finalize(e2, aw, emax, aw, 0.0, scal + 2, p->at<int>(Ly.off_status), ST_UNSTABLE, 1, p->stream));
    p->adj_valid = true;
    if (Ly.S > 1) p->tape_last_valid = false;
    return CX_OK;
}

cx_status read3(cx3_problem* p, double* out4, int* status) {
    double h[4];
    int st = 0;
    CX3_CUDA(cudaMemcpyAsync(h, p->at<double>(p->lay.off_scal), sizeof(h), cudaMemcpyDeviceToHost, p->stream));
    CX3_CUDA(cudaMemcpyAsync(&st, p->at<int>(p->lay.off_status), sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    CX3_CUDA(cudaStreamSynchronize(p->stream));
    if (out4) std::memcpy(out4, h, sizeof(h));
    if (status) *status = st;
    return CX_OK;
}

template <typename T> cx_status run3_step(cx3_problem* p, T* g, T* E, cx_step_info* info) {
    cx_status rc;
    if (!p->fwd_valid) {
        rc = run3_forward<T>(p, g, nullptr, 0.0, nullptr, true);
        if (rc) return rc;
    }
    const T* none[3] = {nullptr, nullptr, nullptr};
    rc = run3_adjoint<T>(p, g, none, true, E);
    if (rc) return rc;
    double s4[4];
    int st = 0;
    rc = read3(p, s4, &st);
    if (rc) return rc;
    if (st & ST_TIMEOUT) return CX_ERR_TIMEOUT;
    if (st & ST_UNSTABLE) return CX_ERR_UNSTABLE;
    const double J0 = s4[0], e2 = s4[2], einf = s4[3];
    double lam = p->have_lam ? 2.0 * p->lam_prev : std::min(1.0, einf > 0.0 ? 1.0 / einf : 1.0);
    const size_t n = (size_t)p->lay.N * p->d.nx * p->d.ny;
    for (int t = 0; t < 30; ++t) {
        rc = run3_forward<T>(p, g, E, lam, nullptr, false);
        if (rc) return rc;
        double j4[4];
        rc = read3(p, j4, nullptr);
        if (rc) return rc;
        const double Jt = j4[0];
        if (std::isfinite(Jt) && Jt <= J0 - 1e-4 * lam * e2) {
            CX3_CUDA(launch_axpy<T>(g, E, T(lam), n, p->stream));
            p->fwd_valid = true; // the accepted trial's forward state is the new control's
            p->adj_valid = false;
            p->lam_prev = lam;
            p->have_lam = true;
            if (info) {
                info->J0 = J0;
                info->J = Jt;
                info->lam = lam;
                info->grad_sq = e2;
                info->grad_inf = einf;
                info->trials = t + 1;
            }
            return CX_OK;
        }
        lam *= 0.5;
    }
    p->fwd_valid = false;
    return CX_ERR_LINESEARCH;
}

int persistent_grid(const void* kern, int nsm, long long total) {
    int per = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, 0) != cudaSuccess || per < 1) per = 1;
    const long long need = (total + 255) / 256;
    long long gsz = std::min<long long>((long long)per * nsm, need);
    gsz = std::min<long long>(gsz, MAXW / 8);
    return (int)std::max<long long>(1, gsz);
}

} // namespace

extern "C" {

cx_status cx3_workspace_size(const cx3_desc* desc, size_t* bytes) {
    const cx_status v = validate3(desc);
    if (v) return v;
    if (!bytes) return CX_ERR_INVALID_ARG;
    *bytes = layout3(desc).total;
    return CX_OK;
}

cx_status cx3_create(const cx3_desc* desc, void* workspace, size_t bytes, cudaStream_t stream, cx3_problem** out) {
    const cx_status v = validate3(desc);
    if (v) return v;
    if (!out || !workspace) return CX_ERR_INVALID_ARG;
    const Lay3 L = layout3(desc);
    if (bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) % AL) != 0) return CX_ERR_WORKSPACE;
    bool okf = true, okd = true;
    const AK<float> Kf = make_ak<float>(*desc, &okf);
    const AK<double> Kd = make_ak<double>(*desc, &okd);
    if (!okf || !okd) return CX_ERR_UNSTABLE;
    cx3_problem* p = new (std::nothrow) cx3_problem();
    if (!p) return CX_ERR_INTERNAL;
    p->d = *desc;
    p->lay = L;
    p->stream = stream;
    p->ws = static_cast<char*>(workspace);
    p->Kf = Kf;
    p->Kd = Kd;
    AC& C = p->C;
    C.nx = desc->nx;
    C.ny = desc->ny;
    C.plane = (long long)L.plane;
    C.N = desc->n_steps;
    C.aniso = desc->aniso;
    C.adv = desc->adv;
    C.ctrl = desc->ctrl_species;
    C.theta = desc->aniso == CX_ANISO_ROTATED ? p->ws + L.off_theta : nullptr;
    C.Kfield = desc->aniso == CX_ANISO_FIELD ? p->ws + L.off_K : nullptr;
    C.a = desc->adv != CX_ADV_NONE ? p->ws + L.off_a : nullptr;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long total = (long long)desc->nx * desc->ny;
    p->nblk = (int)((total + 255) / 256);
    const bool f64 = desc->precision == 64;
    p->grid_f = persistent_grid(f64 ? (const void*)k3_forward<double> : (const void*)k3_forward<float>, nsm, total);
    p->grid_a = persistent_grid(f64 ? (const void*)k3_adjoint<double> : (const void*)k3_adjoint<float>, nsm, total);
    {
        const void* kf = f64 ? (const void*)k3_forward_rows<double> : (const void*)k3_forward_rows<float>;
        const void* ka = f64 ? (const void*)k3_adjoint_rows<double> : (const void*)k3_adjoint_rows<float>;
        const size_t sf = f64 ? rows_pipe_smem<double>(fwd3_stage_values<double>())
                              : rows_pipe_smem<float>(fwd3_stage_values<float>());
        const size_t sa = f64 ? rows_pipe_smem<double>(adj3_stage_values<double>())
                              : rows_pipe_smem<float>(adj3_stage_values<float>());
        int of = 1, oa = 1;
        if (cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf) != cudaSuccess ||
            cudaFuncSetAttribute(ka, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&of, kf, f64 ? FNT<double> + 32 : FNT<float> + 32, sf) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oa, ka, ANT + 32, sa) != cudaSuccess) {
            delete p;
            return CX_ERR_CUDA;
        }
        const int fnt = f64 ? FNT<double> : FNT<float>;
        const long long segf = (long long)((desc->nx + fnt - 1) / fnt) * desc->ny;
        const long long sega = (long long)((desc->nx + ANT - 1) / ANT) * desc->ny;
        p->grid_fr = (int)std::max(1LL, std::min<long long>((long long)std::max(of, 1) * nsm, segf));
        p->grid_ar = (int)std::max(1LL, std::min<long long>((long long)std::max(oa, 1) * nsm, sega));
        p->grid_fr = std::min(p->grid_fr, MAXW / (fnt / 32));
        p->grid_ar = std::min(p->grid_ar, MAXW / (ANT / 32));
    }
    CxConst& CC = p->CC;
    CC.nx = desc->nx;
    CC.ny = desc->ny;
    CC.plane = (long long)L.plane;
    CC.Q = 9;
    CC.n_steps = desc->n_steps;
    CC.ctrl_full = 1;
    CC.cnx = desc->nx;
    CC.cny = desc->ny;
    cudaError_t e = cudaMemsetAsync(p->at<int>(L.off_status), 0, sizeof(int) * 4, stream);
    const int sb = std::min(p->nblk, nsm * 8);
    if (e == cudaSuccess) {
        if (f64)
            k3_setup<double><<<sb, 256, 0, stream>>>(C, *desc, C.theta ? p->at<double>(L.off_theta) : nullptr,
                                                     C.Kfield ? p->at<double>(L.off_K) : nullptr,
                                                     C.a ? p->at<double>(L.off_a) : nullptr, p->at<double>(L.off_ut),
                                                     p->at<int>(L.off_status));
        else
            k3_setup<float><<<sb, 256, 0, stream>>>(C, *desc, C.theta ? p->at<float>(L.off_theta) : nullptr,
                                                    C.Kfield ? p->at<float>(L.off_K) : nullptr,
                                                    C.a ? p->at<float>(L.off_a) : nullptr, p->at<float>(L.off_ut),
                                                    p->at<int>(L.off_status));
        e = cudaGetLastError();
    }
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, p->at<int>(L.off_status), sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        delete p;
        return CX_ERR_CUDA;
    }
    if (st & ST_UNSTABLE) {
        delete p;
        return CX_ERR_UNSTABLE;
    }
    // the status word reports later errors only
    p->d.theta = p->d.D_u_field = p->d.D_v_field = p->d.D_w_field = p->d.a = p->d.u_target = nullptr;
    *out = p;
    return CX_OK;
}

cx_status cx3_set_initial(cx3_problem* p, const double* u0, const double* v0, const double* w0) {
    if (!p || !u0 || !v0 || !w0) return CX_ERR_INVALID_ARG;
    const int sb = std::max(1, std::min(p->nblk, 152 * 8));
    if (p->lay.esz == 8)
        k3_init<double><<<sb, 256, 0, p->stream>>>(p->C, p->Kd, u0, v0, w0, reinterpret_cast<double*>(p->slot(0)));
    else
        k3_init<float><<<sb, 256, 0, p->stream>>>(p->C, p->Kf, u0, v0, w0, reinterpret_cast<float*>(p->slot(0)));
    CX3_CUDA(cudaGetLastError());
    p->has_init = true;
    p->fwd_valid = p->adj_valid = p->tape_last_valid = false;
    p->have_lam = false;
    return CX_OK;
}

cx_status cx3_forward(cx3_problem* p, const void* g, double* J_dev) {
    if (!p) return CX_ERR_INVALID_ARG;
    if (!p->has_init) return CX_ERR_STATE;
    if (p->lay.esz == 8) return run3_forward<double>(p, (const double*)g, nullptr, 0.0, J_dev, true);
    return run3_forward<float>(p, (const float*)g, nullptr, 0.0, J_dev, true);
}

cx_status cx3_adjoint(cx3_problem* p, const void* g, const void* seed_u, const void* seed_v, const void* seed_w,
                      int penalty, void* dJdg) {
    if (!p || !dJdg) return CX_ERR_INVALID_ARG;
    if (!p->fwd_valid) return CX_ERR_STATE;
    if (p->lay.esz == 8) {
        const double* s[3] = {(const double*)seed_u, (const double*)seed_v, (const double*)seed_w};
        return run3_adjoint<double>(p, (const double*)g, s, penalty != 0, (double*)dJdg);
    }
    const float* s[3] = {(const float*)seed_u, (const float*)seed_v, (const float*)seed_w};
    return run3_adjoint<float>(p, (const float*)g, s, penalty != 0, (float*)dJdg);
}

cx_status cx3_gradient(cx3_problem* p, const void* g, void* dJdg, double* J_dev) {
    cx_status rc = cx3_forward(p, g, J_dev);
    if (rc) return rc;
    return cx3_adjoint(p, g, nullptr, nullptr, nullptr, 1, dJdg);
}

cx_status cx3_step(cx3_problem* p, void* g_inout, void* E_work, cx_step_info* info) {
    if (!p || !g_inout || !E_work) return CX_ERR_INVALID_ARG;
    if (!p->has_init) return CX_ERR_STATE;
    if (p->lay.esz == 8) return run3_step<double>(p, (double*)g_inout, (double*)E_work, info);
    return run3_step<float>(p, (float*)g_inout, (float*)E_work, info);
}

cx_status cx3_get_fields(cx3_problem* p, void* u_out, void* v_out, void* w_out) {
    if (!p) return CX_ERR_INVALID_ARG;
    if (!p->fwd_valid) return CX_ERR_STATE;
    void* o[3] = {u_out, v_out, w_out};
    const size_t n = (size_t)p->d.nx * p->d.ny * p->lay.esz;
    for (int s = 0; s < 3; ++s)
        if (o[s])
            CX3_CUDA(cudaMemcpyAsync(o[s], p->ws + p->lay.off_uvw + (size_t)s * p->fld(), n, cudaMemcpyDeviceToDevice,
                                     p->stream));
    return CX_OK;
}

cx_status cx3_get_norms(cx3_problem* p, double* J, double* grad_sq, double* grad_inf) {
    if (!p) return CX_ERR_INVALID_ARG;
    double s4[4];
    int st = 0;
    const cx_status rc = read3(p, s4, &st);
    if (rc) return rc;
    if (J) *J = s4[0];
    if (grad_sq) *grad_sq = s4[2];
    if (grad_inf) *grad_inf = s4[3];
    if (st & ST_TIMEOUT) return CX_ERR_TIMEOUT;
    return (st & ST_UNSTABLE) ? CX_ERR_UNSTABLE : CX_OK;
}

cx_status cx3_set_staging(cx3_problem* p, int mode) {
    if (!p || mode < 0 || mode > 2) return CX_ERR_INVALID_ARG;
    p->rows_mode = mode;
    return CX_OK;
}

cx_status cx3_set_timing(cx3_problem* p, int enable) {
    if (!p) return CX_ERR_INVALID_ARG;
    p->timing = enable != 0;
    p->n_ranges = 0;
    return CX_OK;
}

cx_status cx3_get_timing(cx3_problem* p, double* ms, long long* launches) {
    if (!p || !ms || !launches) return CX_ERR_INVALID_ARG;
    CX3_CUDA(cudaStreamSynchronize(p->stream));
    for (int i = 0; i < 3; ++i) {
        ms[i] = 0.0;
        launches[i] = 0;
    }
    for (size_t i = 0; i < p->n_ranges; ++i) {
        float t = 0.f;
        CX3_CUDA(cudaEventElapsedTime(&t, p->ranges[i].a, p->ranges[i].b));
        ms[p->ranges[i].phase] += t;
        launches[p->ranges[i].phase] += p->ranges[i].launches;
    }
    return CX_OK;
}

cx_status cx3_destroy(cx3_problem* p) {
    if (!p) return CX_ERR_INVALID_ARG;
    for (auto& r : p->ranges) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    delete p;
    return CX_OK;
}

} // extern "C"
