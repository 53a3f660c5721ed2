// cx_adj_body.cuh -- per-node body of the adjoint step: AMRT adjoint step with fused gradient assembly, one time
// step per launch, run backward in time (Sec. 3.2.1).
//
// The adjoint of the discrete forward step (exact transpose, so that the
// gradient is the gradient of the discrete cost):
//   rho_i(x)  = psi^{n+1}_i(x + e_i), or psi^{n+1}_{opp(i)}(x) if x + e_i is solid
//               (streaming along -e_i backward in time; bounce-back transposed)
//   m~        = Lambda^T rho = M^T Pi^T M^-T rho              (collision, eq. CAE)
//   Tcal      = sum_j w_j aleph_j m~_j                         (adjoint equilibrium,
//               the scalar broadcast m~^eq_i = Tcal of AEDsM and the ALEPH formula)
//   psi_i     = rho_i - m~_i + Tcal                            (Lambda^* (psi - psi^eq))
//   coupling  sum_k rho_k dR_k/dphi_i  for R_u = tau S_u(u, G(j_v, v, Phi)) and
//             R_v = w~ (c_n Phi^n + c'_n Phi^{n-1})             (eq. CAE-L)
//   dJ/dg^n   = lambda_Phi^n + 2 alpha g^n                     (gradientLattice),
//               lambda_Phi^n = c_n sigma^n + c'_{n+1} sigma^{n+1} + (G path),
//               sigma^n = sum_i rho_v,i w~_i.
// The tape (u^n, G^n) comes from the forward recompute of the segment.
// On grids whose solid nodes carry bounce-back copies (C.bb_copy), psi_i(x)
// with x - e_i solid is also written into plane opp(i) at x - e_i, where the
// next adjoint step's pull of direction opp(i) at x looks.
// In FP32, sums sum_i c_i rho_i with c_i = w_i (a + b.e_i) (sigma, and the
// weights of the chemotactic coupling) are taken from the moments m = M0 rho
// the collision needs anyway: sum_i c_i rho_i = sum_k (M0 c)_k m_k / |row_k|^2;
// FP64 (the parity mode) sums them per direction as written.
//
// Execution: the persistent, two-stage cp.async pipeline of the forward
// kernel (see cx_forward.cu), staging the pulled adjoint populations, the tape,
// sigma^{n+1}, g^n and the angle of the next node while the current one runs.
#pragma once

#include "cx_device.cuh"

namespace cx {

template <int Q> constexpr int adj_stage_values() { return 2 * Q + 6; } // pops, u, Gx, Gy, sigma, g, theta

template <typename T, int Q, int NT, typename Args>
__device__ __forceinline__ void adj_stage(const CxConst& C, const Args& A, const NodeIdx& nd, T* s) {
    using L = Lat<Q>;
    if (!nd.fluid) return;
    const int x = nd.x, y = nd.y, k = nd.k;
    const size_t pl = (size_t)C.plane;
    const int xm = x == 0 ? C.nx - 1 : x - 1, xp = x == C.nx - 1 ? 0 : x + 1;
    const int rm = (y == 0 ? C.ny - 1 : y - 1) * C.nx, r0 = y * C.nx, rp = (y == C.ny - 1 ? 0 : y + 1) * C.nx;
    const unsigned bb = C.has_solid ? C.bounce[k] : 0u; // forward pulls that bounce back
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int xd = L::ex(i) > 0 ? xp : (L::ex(i) < 0 ? xm : x);
        const int kd = (L::ey(i) > 0 ? rp : (L::ey(i) < 0 ? rm : r0)) + xd;
        // x + e_i is solid exactly when the forward pull of direction opp(i) bounces back
        const bool bounce = i != 0 && ((bb >> (L::opp(i) - 1)) & 1u);
        if (A.terminal) {
            // psi^N_i(x) is the seed w(x) in every direction
            cp_async(s + i * NT, A.wu + (bounce ? k : kd));
            if (A.wv) cp_async(s + (Q + i) * NT, A.wv + (bounce ? k : kd));
        } else if (bounce) {
            cp_async(s + i * NT, A.in(L::opp(i)) + k);
            cp_async(s + (Q + i) * NT, A.in(Q + L::opp(i)) + k);
        } else {
            cp_async(s + i * NT, A.in(i) + kd);
            cp_async(s + (Q + i) * NT, A.in(Q + i) + kd);
        }
    }
    cp_async(s + (2 * Q) * NT, A.tape + k);
    cp_async(s + (2 * Q + 1) * NT, A.tape + pl + k);
    cp_async(s + (2 * Q + 2) * NT, A.tape + 2 * pl + k);
    if (!A.terminal) cp_async(s + (2 * Q + 3) * NT, A.sigma + k);
    if (nd.ctrl && A.g) cp_async(s + (2 * Q + 4) * NT, A.g + nd.c);
    if (C.aniso == CX_ANISO_ROTATED) cp_async(s + (2 * Q + 5) * NT, reinterpret_cast<const T*>(C.theta) + k);
}

// Bounce-back copies of one species (planes base .. base + Q - 1): psi_i(x)
// to plane opp(i) at x - e_i for every i whose x - e_i is solid (flag bit
// i - 1).  Each solid slot has one writer: the fluid node x = s + e_i.
template <typename T, int Q, typename Args>
__device__ __forceinline__ void adj_bb_copies(const CxConst& C, const Args& A, int base, int k, unsigned bits,
                                              const T (&psi)[Q]) {
    using L = Lat<Q>;
    const int y = k / C.nx, x = k - y * C.nx; // rare (nodes next to a wall): recomputed, not kept in registers
#pragma unroll
    for (int i = 1; i < Q; ++i)
        if ((bits >> (i - 1)) & 1u) A.out(base + L::opp(i))[nbr_index(C, x, y, -L::ex(i), -L::ey(i))] = psi[i];
}

template <typename T, int Q, int NT, typename Args, typename Stage>
__device__ __forceinline__ void adj_compute(const CxConst& C, const KConst<T>& KC, const Args& A, const NodeIdx& nd,
                                            const Stage& S, typename SqAccT<T>::type& acc) {
    using L = Lat<Q>;
    if (!nd.fluid) {
        if (nd.c >= 0) A.dJdg[nd.c] = T(0); // solid window nodes are not controlled
        return;
    }
    const int y = nd.y, k = nd.k;
    T ru[Q], rv[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (S.adj_bounce(i)) { // bounce-back transposed: the node's own opposite adjoint population
            ru[i] = ldg(A.in(L::opp(i)) + k);
            rv[i] = ldg(A.in(Q + L::opp(i)) + k);
        } else {
            ru[i] = S.pop(i, L::ex(i));
            rv[i] = (A.terminal && !A.wv) ? T(0) : S.pop(Q + i, L::ex(i));
        }
    }
    const T Tu = S.val(2 * Q);
    const T Gx = S.val(2 * Q + 1);
    const T Gy = S.val(2 * Q + 2);
    const T sig_next = A.terminal ? T(0) : S.val(2 * Q + 3);
    const T gv = (nd.ctrl && A.g) ? S.val(2 * Q + 4) : T(0);
    NodeCoef<T> nc;
    node_coef_th<T>(C, KC, (C.aniso == CX_ANISO_ROTATED) ? S.val(2 * Q + 5) : T(0), y, k, nc);

    // --- transposed collisions: mt = M^T Pi^T (N^-1 M rho), Tcal = sum_k z_k mh_k
    T mh[Q], mom[Q], z[Q], mt[Q];
    T psu[Q], psv[Q];
    meq_unit<T, Q>(nc.ax, nc.ay, KC.d_u, mh);
    Transform<T, Q>::moments(ru, mom);
    // Y = sum_i 3 w_i e_i rho_u,i (the weights of tau S_u)
    constexpr bool fold = sizeof(T) == 4; // from the moments (FP32)
    T Yx = T(0), Yy = T(0);
    if constexpr (fold) {
#pragma unroll
        for (int kk = 0; kk < Q; ++kk) {
            if (L::src_Bx(kk) != 0.0) Yx += T(3.0 * L::inv_n(kk) * L::src_Bx(kk)) * mom[kk];
            if (L::src_By(kk) != 0.0) Yy += T(3.0 * L::inv_n(kk) * L::src_By(kk)) * mom[kk];
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            Yx += T(3.0 * L::w(i) * L::ex(i)) * ru[i];
            Yy += T(3.0 * L::w(i) * L::ey(i)) * ru[i];
        }
    }
    relax_n<T, Q>(KC, nc.Ku0, nc.Ku1, nc.Ku2, mom, z);
    // (FP32: the mass moment's term, z_0 in both mt and Tcal, cancels exactly
    // in psi = rho - mt + Tcal, so it is left out)
    T Tcu = T(0);
#pragma unroll
    for (int kk = fold ? 1 : 0; kk < Q; ++kk) Tcu += z[kk] * mh[kk];
    if constexpr (fold)
        Transform<T, Q>::transpose0(z, mt);
    else
        Transform<T, Q>::transpose(z, mt);
    // FP32 adds the node's scalar terms (Tcal, the coupling) once per
    // direction at the end; FP64 adds them in the order written above
#pragma unroll
    for (int i = 0; i < Q; ++i) psu[i] = fold ? ru[i] - mt[i] : ru[i] - mt[i] + Tcu;

    // sigma = sum_i w~_i rho_v,i with w~_i = w_i (1 + 3 V.e_i), V = (I - K_v/2) a
    const T Kax = nc.Kv0 * nc.ax + nc.Kv1 * nc.ay, Kay = nc.Kv1 * nc.ax + nc.Kv2 * nc.ay;
    const T Vx = nc.ax - T(0.5) * Kax, Vy = nc.ay - T(0.5) * Kay;
    meq_unit<T, Q>(nc.ax, nc.ay, KC.d_v, mh);
    Transform<T, Q>::moments(rv, mom);
    T sigma = T(0);
    if constexpr (fold) {
        T sA = T(0), sBx = T(0), sBy = T(0);
#pragma unroll
        for (int kk = 0; kk < Q; ++kk) {
            if (L::src_A(kk) != 0.0) sA += T(L::inv_n(kk) * L::src_A(kk)) * mom[kk];
            if (L::src_Bx(kk) != 0.0) sBx += T(3.0 * L::inv_n(kk) * L::src_Bx(kk)) * mom[kk];
            if (L::src_By(kk) != 0.0) sBy += T(3.0 * L::inv_n(kk) * L::src_By(kk)) * mom[kk];
        }
        sigma = sA + Vx * sBx + Vy * sBy;
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i)
            sigma += T(L::w(i)) * (T(1) + T(3) * (Vx * T(L::ex(i)) + Vy * T(L::ey(i)))) * rv[i];
    }
    relax_n<T, Q>(KC, nc.Kv0, nc.Kv1, nc.Kv2, mom, z);
    T Tcv = T(0);
#pragma unroll
    for (int kk = fold ? 1 : 0; kk < Q; ++kk) Tcv += z[kk] * mh[kk];
    if constexpr (fold)
        Transform<T, Q>::transpose0(z, mt);
    else
        Transform<T, Q>::transpose(z, mt);
#pragma unroll
    for (int i = 0; i < Q; ++i) psv[i] = fold ? rv[i] - mt[i] : rv[i] - mt[i] + Tcv;

    // --- coupling through tau S_u,i = 3 w_i chi u e_i . (K_u G)
    const T chi = KC.chi;
    T adj_Tu = chi * (Yx * (nc.Ku0 * Gx + nc.Ku1 * Gy) + Yy * (nc.Ku1 * Gx + nc.Ku2 * Gy));
    const T aGx = chi * Tu * (nc.Ku0 * Yx + nc.Ku1 * Yy);
    const T aGy = chi * Tu * (nc.Ku1 * Yx + nc.Ku2 * Yy);
    // G = -(K_v (j_v - a v)/tau + K_v a Phi/2) / (d_v Cs^2)
    const T KGx = nc.Kv0 * aGx + nc.Kv1 * aGy, KGy = nc.Kv1 * aGx + nc.Kv2 * aGy;
    const T sc = KC.asc; // 1 / (d_v Cs^2)
    const T ajx = -KGx * sc * KC.inv_tau, ajy = -KGy * sc * KC.inv_tau;
    const T aKG = nc.ax * KGx + nc.ay * KGy;
    T adj_Tv = aKG * sc * KC.inv_tau;
    T adj_Phi = T(-0.5) * aKG * sc;

    // --- reaction/control source: sigma^n and the use of Phi^n at step n+1
    adj_Phi += ((A.n == 0) ? KC.c_first : KC.c_now) * sigma;
    if (!A.terminal) adj_Phi += KC.c_prev * sig_next; // Phi^n feeds step n+1 with c'_{n+1}
    A.sigma[k] = sigma;
    adj_Tu += KC.r_vu * adj_Phi;
    adj_Tv += KC.r_vv * adj_Phi;

    if (nd.ctrl) {
        T E = adj_Phi + KC.two_alpha * gv;
        if (A.accum) E += A.dJdg[nd.c]; // chain rule of g^n = G_w: sum over the window's steps
        A.dJdg[nd.c] = E;
        if (A.norm) acc.add(E);
    } else if (nd.c >= 0) {
        A.dJdg[nd.c] = T(0);
    }
    const unsigned bbc = (Stage::copies && C.bb_copy) ? S.bb_bits(C, k) : 0u;
    if constexpr (fold) {
        // psi_i = (rho_i - mt_i) + c(e_i), c(e) = Tcal + adj_T + e.aj: three
        // x-classes, then +-aj_y
        const T cu = Tcu + adj_Tu, cv = Tcv + adj_Tv;
        const T cvx[3] = {cv - ajx, cv, cv + ajx};
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T cxi = cvx[L::ex(i) + 1];
            psu[i] = psu[i] + cu;
            psv[i] = psv[i] + (L::ey(i) == 0 ? cxi : (L::ey(i) > 0 ? cxi + ajy : cxi - ajy));
            A.out(i)[k] = psu[i];
            A.out(Q + i)[k] = psv[i];
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            psu[i] = psu[i] + adj_Tu;
            psv[i] = psv[i] + adj_Tv + T(L::ex(i)) * ajx + T(L::ey(i)) * ajy;
            A.out(i)[k] = psu[i];
            A.out(Q + i)[k] = psv[i];
        }
    }
    if (Stage::copies && bbc) {
        adj_bb_copies<T, Q>(C, A, 0, k, bbc, psu);
        adj_bb_copies<T, Q>(C, A, Q, k, bbc, psv);
    }
}

} // namespace cx
