// cx_fwd_body.cuh -- per-node body of the forward step: fused pull-stream + MRT collision for both species, one
// time step per launch (eq. LBE / LBEG, Sec. 3.1 and 3.2).
//
// Per fluid node x at step n (tau in lattice units, Cs^2 = 1/3):
//   f_i(x)   = P^{n-1}_i(x - e_i), or P^{n-1}_{opp(i)}(x) if x - e_i is solid
//              (halfway bounce-back); at n = 0 f = phi^eq(Theta_0) read locally.
//   Theta    = sum_i f_i,  j_v = sum_i e_i f_v,i
//   Phi_v    = r_vu u + r_vv v + g^n(x)                         (Phi_u = 0)
//   G        = -(K_v (j_v - a v)/tau + K_v a Phi_v / 2) / (d_v Cs^2)
//              (grad v from v's first non-equilibrium moment, relation C146)
//   P_Theta  = f - M^-1 Pi_Theta (M f - m^eq(Theta))               (eqs. MF, MC)
//   P_u,i   += (w_i / Cs^2) chi u e_i . (K_u G)                    (tau S_u, eq. S
//              with A_{u,1} = K_u D_{u,1} / tau, D_{u,1} = chi u I)
//   P_v,i   += w~_i [c_n Phi^n + c'_n Phi^{n-1}]                    (eq. PhiS with
//              V = (I - K_v/2) a, kappa_x = 0; c_n = 3 tau/2, c'_n = -tau/2;
//              c_0 = tau, c'_0 = 0 because Phi^{-1} := Phi^0)
// Both sources have the shape w_i (a + b.e_i).  In FP32 they join the
// collision in moment space: with s^ = M0 s (a few nonzero moments) and
// M0^-1 = M0^T N^-1, P = f - M0^T N^-1 (Pi (m - m^eq) - s^), one transform per
// species and fewer instructions.  FP64 (the parity mode) adds them per
// direction, in the order of operations of the equations as written.
// The node also writes Phi^n (node-local state for the next step), optionally
// the adjoint tape (u, G_x, G_y), and accumulates (g^n)^2 for the penalty.
//
// Execution: a persistent grid; each block walks row segments of blockDim.x
// nodes.  While a thread computes its current node it has already issued the
// cp.async copies of its next node's populations and per-node scalars into its
// own shared-memory slots (two stages), so DRAM latency overlaps the
// arithmetic without holding registers for loads in flight.
#pragma once

#include "cx_device.cuh"

namespace cx {

template <int Q> constexpr int fwd_stage_values() { return 2 * Q + 4; } // pops, theta, g, E, Phi^{n-1}

template <typename T, int Q, int NT, typename Args>
__device__ __forceinline__ void fwd_stage(const CxConst& C, const Args& A, const NodeIdx& nd, T* s) {
    using L = Lat<Q>;
    if (!nd.fluid) return;
    const int x = nd.x, y = nd.y, k = nd.k;
    if (A.n == 0) {
#pragma unroll
        for (int i = 0; i < 2 * Q; ++i) cp_async(s + i * NT, A.in(i) + k);
    } else {
        const int xm = x == 0 ? C.nx - 1 : x - 1, xp = x == C.nx - 1 ? 0 : x + 1;
        const int rm = (y == 0 ? C.ny - 1 : y - 1) * C.nx, r0 = y * C.nx, rp = (y == C.ny - 1 ? 0 : y + 1) * C.nx;
        const unsigned bb = C.has_solid ? C.bounce[k] : 0u; // pulls that bounce back
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int xs = L::ex(i) > 0 ? xm : (L::ex(i) < 0 ? xp : x);
            const int ks = (L::ey(i) > 0 ? rm : (L::ey(i) < 0 ? rp : r0)) + xs;
            if (i != 0 && ((bb >> (i - 1)) & 1u)) {
                cp_async(s + i * NT, A.in(L::opp(i)) + k);
                cp_async(s + (Q + i) * NT, A.in(Q + L::opp(i)) + k);
            } else {
                cp_async(s + i * NT, A.in(i) + ks);
                cp_async(s + (Q + i) * NT, A.in(Q + i) + ks);
            }
        }
        cp_async(s + (2 * Q + 3) * NT, A.phi + k);
    }
    if (C.aniso == CX_ANISO_ROTATED) cp_async(s + 2 * Q * NT, reinterpret_cast<const T*>(C.theta) + k);
    if (nd.ctrl) {
        if (A.g) cp_async(s + (2 * Q + 1) * NT, A.g + nd.c);
        if (A.E) cp_async(s + (2 * Q + 2) * NT, A.E + nd.c);
    }
}

template <typename T, int Q, int NT, typename Args, typename Stage>
__device__ __forceinline__ void fwd_compute(const CxConst& C, const KConst<T>& KC, const Args& A, const NodeIdx& nd,
                                            const Stage& S, typename SqAccT<T>::type& acc) {
    using L = Lat<Q>;
    if (!nd.fluid) return;
    const int y = nd.y, k = nd.k;
    T fu[Q], fv[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (S.fwd_bounce(i)) { // halfway bounce-back: the node's own opposite population
            fu[i] = ldg(A.in(L::opp(i)) + k);
            fv[i] = ldg(A.in(Q + L::opp(i)) + k);
        } else {
            fu[i] = S.pop(i, -L::ex(i));
            fv[i] = S.pop(Q + i, -L::ex(i));
        }
    }
    T g = T(0);
    if (nd.ctrl) {
        if (A.g) g = S.val(2 * Q + 1);
        if (A.E) g = fma(-A.lam, S.val(2 * Q + 2), g); // same rounding as the accepted update
        acc.add(g);
    }
    NodeCoef<T> nc;
    node_coef_th<T>(C, KC, (C.aniso == CX_ANISO_ROTATED) ? S.val(2 * Q) : T(0), y, k, nc);

    // moments m = M f of both species
    T mu[Q], mv[Q];
    Transform<T, Q>::moments(fu, mu);
    Transform<T, Q>::moments(fv, mv);
    const T Tu = mu[0], Tv = mv[0];
    const T jvx = mv[L::JX], jvy = mv[L::JY];

    // reaction and control source
    const T Phi = KC.r_vu * Tu + KC.r_vv * Tv + g;
    const T Phi_prev = (A.n == 0) ? Phi : S.val(2 * Q + 3);

    // grad v (reading of C146)
    const T rx = (jvx - nc.ax * Tv) * KC.inv_tau, ry = (jvy - nc.ay * Tv) * KC.inv_tau;
    const T Kax = nc.Kv0 * nc.ax + nc.Kv1 * nc.ay, Kay = nc.Kv1 * nc.ax + nc.Kv2 * nc.ay;
    const T Gx = KC.gsc * (nc.Kv0 * rx + nc.Kv1 * ry + T(0.5) * Kax * Phi);
    const T Gy = KC.gsc * (nc.Kv1 * rx + nc.Kv2 * ry + T(0.5) * Kay * Phi);

    // --- species u: MRT collision + chemotactic cross-diffusion source
    T mh[Q], dm[Q], rl[Q], bt[Q];
    meq_unit<T, Q>(nc.ax, nc.ay, KC.d_u, mh);
#pragma unroll
    for (int kk = 0; kk < Q; ++kk) dm[kk] = mu[kk] - Tu * mh[kk];
    relax_n<T, Q>(KC, nc.Ku0, nc.Ku1, nc.Ku2, dm, rl);
    // (w_i/Cs^2) chi u e_i.(K_u G) = 3 w_i e_i . F: moments 3 (F_x src_Bx + F_y src_By)
    const T Fx = KC.chi * Tu * (nc.Ku0 * Gx + nc.Ku1 * Gy);
    const T Fy = KC.chi * Tu * (nc.Ku1 * Gx + nc.Ku2 * Gy);
    constexpr bool fold = sizeof(T) == 4; // sources in moment space (FP32)
    if constexpr (fold) {
#pragma unroll
        for (int kk = 0; kk < Q; ++kk) {
            if (L::src_Bx(kk) != 0.0) rl[kk] -= T(3.0 * L::inv_n(kk) * L::src_Bx(kk)) * Fx;
            if (L::src_By(kk) != 0.0) rl[kk] -= T(3.0 * L::inv_n(kk) * L::src_By(kk)) * Fy;
        }
    }
    // M^-1 (Pi (m - m^eq) - s^) = M^T N^-1 (...); FP32: the mass moment of u's
    // non-equilibrium part is exactly zero (m_0 - Theta m^eq_0 = Theta - Theta)
    // and u has no mass source, so its row is left out
    if constexpr (fold)
        Transform<T, Q>::transpose0(rl, bt);
    else
        Transform<T, Q>::transpose(rl, bt);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if constexpr (fold) {
            A.out(i)[k] = fu[i] - bt[i];
        } else {
            const T src = T(3.0 * L::w(i)) * (T(L::ex(i)) * Fx + T(L::ey(i)) * Fy);
            A.out(i)[k] = fu[i] - bt[i] + src;
        }
    }

    // --- species v: MRT collision + reaction/control source with the tau/2
    //     time-derivative term
    meq_unit<T, Q>(nc.ax, nc.ay, KC.d_v, mh);
#pragma unroll
    for (int kk = 0; kk < Q; ++kk) dm[kk] = mv[kk] - Tv * mh[kk];
    relax_n<T, Q>(KC, nc.Kv0, nc.Kv1, nc.Kv2, dm, rl);
    const T Vx = nc.ax - T(0.5) * Kax, Vy = nc.ay - T(0.5) * Kay; // V = (I - K_v/2) a
    const T srcv = (A.n == 0) ? KC.c_first * Phi : KC.c_now * Phi + KC.c_prev * Phi_prev;
    // w~_i srcv = w_i (srcv + 3 srcv V.e_i): moments srcv src_A + 3 srcv (V_x src_Bx + V_y src_By)
    if constexpr (fold) {
        const T sVx = srcv * Vx, sVy = srcv * Vy;
#pragma unroll
        for (int kk = 0; kk < Q; ++kk) {
            if (L::src_A(kk) != 0.0) rl[kk] -= T(L::inv_n(kk) * L::src_A(kk)) * srcv;
            if (L::src_Bx(kk) != 0.0) rl[kk] -= T(3.0 * L::inv_n(kk) * L::src_Bx(kk)) * sVx;
            if (L::src_By(kk) != 0.0) rl[kk] -= T(3.0 * L::inv_n(kk) * L::src_By(kk)) * sVy;
        }
    }
    Transform<T, Q>::transpose(rl, bt);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if constexpr (fold) {
            A.out(Q + i)[k] = fv[i] - bt[i];
        } else {
            const T wt = T(L::w(i)) * (T(1) + T(3) * (Vx * T(L::ex(i)) + Vy * T(L::ey(i))));
            A.out(Q + i)[k] = fv[i] - bt[i] + wt * srcv;
        }
    }
    A.phi[k] = Phi;
    if (A.phi_ckpt) A.phi_ckpt[k] = Phi;
    if (A.tape) {
        const size_t pl = (size_t)C.plane;
        A.tape[k] = Tu;
        A.tape[pl + k] = Gx;
        A.tape[2 * pl + k] = Gy;
    }
}

} // namespace cx
