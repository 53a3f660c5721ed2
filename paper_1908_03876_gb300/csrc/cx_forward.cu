// cx_forward.cu -- fused pull-stream + MRT collision for both species, one
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
// The node also writes Phi^n (node-local state for the next step), optionally
// the adjoint tape (u, G_x, G_y), and adds sum (g^n)^2 to its block's FP64
// partial of the control penalty.
#include "cx_device.cuh"

namespace cx {

template <typename T, int Q>
__global__ void __launch_bounds__(256) k_forward(const CxConst C, const FwdArgs<T> A) {
    using L = Lat<Q>;
    __shared__ double red[32];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    double gsq = 0.0;
    const bool inside = (x < C.nx) && (y < C.ny);
    const int k = y * C.nx + x;
    const bool fluid = inside && !(C.has_solid && C.solid[k]);
    if (fluid) {
        const size_t pl = (size_t)C.plane;
        T fu[Q], fv[Q];
        if (A.n == 0) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                fu[i] = ldg(A.Pin + i * pl + k);
                fv[i] = ldg(A.Pin + (Q + i) * pl + k);
            }
        } else {
            const int xm = x == 0 ? C.nx - 1 : x - 1, xp = x == C.nx - 1 ? 0 : x + 1;
            const int ym = y == 0 ? C.ny - 1 : y - 1, yp = y == C.ny - 1 ? 0 : y + 1;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int xs = L::ex(i) > 0 ? xm : (L::ex(i) < 0 ? xp : x);
                const int ys = L::ey(i) > 0 ? ym : (L::ey(i) < 0 ? yp : y);
                const int ks = ys * C.nx + xs;
                if (C.has_solid && i != 0 && C.solid[ks]) {
                    fu[i] = ldg(A.Pin + L::opp(i) * pl + k);
                    fv[i] = ldg(A.Pin + (Q + L::opp(i)) * pl + k);
                } else {
                    fu[i] = ldg(A.Pin + i * pl + ks);
                    fv[i] = ldg(A.Pin + (Q + i) * pl + ks);
                }
            }
        }
        NodeCoef<T> nc;
        node_coef<T>(C, x, y, k, nc);

        // moments m = M f of both species
        T mu[Q], mv[Q];
#pragma unroll
        for (int kk = 0; kk < Q; ++kk) {
            T su = T(0), sv = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (L::M(kk, i) == 1) {
                    su += fu[i];
                    sv += fv[i];
                } else if (L::M(kk, i) == -1) {
                    su -= fu[i];
                    sv -= fv[i];
                } else if (L::M(kk, i) != 0) {
                    su += T(L::M(kk, i)) * fu[i];
                    sv += T(L::M(kk, i)) * fv[i];
                }
            }
            mu[kk] = su;
            mv[kk] = sv;
        }
        const T Tu = mu[0], Tv = mv[0];
        const T jvx = mv[L::JX], jvy = mv[L::JY];

        // control and reaction source
        T g = T(0);
        const int c = ctrl_window(C, x, y);
        if (ctrl_active(C, c)) {
            if (A.g) g = ldg(A.g + c);
            if (A.E) g = fma(-T(A.lam), ldg(A.E + c), g); // same rounding as the accepted update
            gsq = (double)g * (double)g;
        }
        const T Phi = T(C.r_vu) * Tu + T(C.r_vv) * Tv + g;
        const T Phi_prev = (A.n == 0) ? Phi : A.phi[k];

        // grad v (reading of C146)
        const T tau = T(C.tau);
        const T rx = (jvx - nc.ax * Tv) / tau, ry = (jvy - nc.ay * Tv) / tau;
        const T Kax = nc.Kv0 * nc.ax + nc.Kv1 * nc.ay, Kay = nc.Kv1 * nc.ax + nc.Kv2 * nc.ay;
        const T sc = T(-3.0) / T(C.d_v); // -1 / (d_v Cs^2)
        const T Gx = sc * (nc.Kv0 * rx + nc.Kv1 * ry + T(0.5) * Kax * Phi);
        const T Gy = sc * (nc.Kv1 * rx + nc.Kv2 * ry + T(0.5) * Kay * Phi);

        // --- species u: MRT collision + chemotactic cross-diffusion source
        T mh[Q], dm[Q], rl[Q];
        meq_unit<T, Q>(nc.ax, nc.ay, T(C.d_u), mh);
#pragma unroll
        for (int kk = 0; kk < Q; ++kk) dm[kk] = mu[kk] - Tu * mh[kk];
        relax<T, Q>(C, nc.Ku0, nc.Ku1, nc.Ku2, dm, rl);
#pragma unroll
        for (int kk = 0; kk < Q; ++kk) rl[kk] *= T(L::inv_n(kk));
        // (w_i/Cs^2) chi u e_i.(K_u G) = 3 w_i e_i . F
        const T Fx = T(C.chi) * Tu * (nc.Ku0 * Gx + nc.Ku1 * Gy);
        const T Fy = T(C.chi) * Tu * (nc.Ku1 * Gx + nc.Ku2 * Gy);
        T* Pu = A.Pout;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            T s = T(0);
#pragma unroll
            for (int kk = 0; kk < Q; ++kk)
                if (L::M(kk, i) != 0) s += T(L::M(kk, i)) * rl[kk];
            const T src = T(3.0 * L::w(i)) * (T(L::ex(i)) * Fx + T(L::ey(i)) * Fy);
            Pu[i * pl + k] = fu[i] - s + src;
        }

        // --- species v: MRT collision + reaction/control source with the
        //     tau/2 time-derivative term
        meq_unit<T, Q>(nc.ax, nc.ay, T(C.d_v), mh);
#pragma unroll
        for (int kk = 0; kk < Q; ++kk) dm[kk] = mv[kk] - Tv * mh[kk];
        relax<T, Q>(C, nc.Kv0, nc.Kv1, nc.Kv2, dm, rl);
#pragma unroll
        for (int kk = 0; kk < Q; ++kk) rl[kk] *= T(L::inv_n(kk));
        const T Vx = nc.ax - T(0.5) * Kax, Vy = nc.ay - T(0.5) * Kay; // V = (I - K_v/2) a
        T cn, cp;
        if (C.source_order == 1 || A.n == 0) {
            cn = tau;
            cp = T(0);
        } else {
            cn = T(1.5) * tau;
            cp = T(-0.5) * tau;
        }
        const T srcv = cn * Phi + cp * Phi_prev;
        T* Pv = A.Pout + (size_t)Q * pl;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            T s = T(0);
#pragma unroll
            for (int kk = 0; kk < Q; ++kk)
                if (L::M(kk, i) != 0) s += T(L::M(kk, i)) * rl[kk];
            const T wt = T(L::w(i)) * (T(1) + T(3) * (Vx * T(L::ex(i)) + Vy * T(L::ey(i))));
            Pv[i * pl + k] = fv[i] - s + wt * srcv;
        }
        A.phi[k] = Phi;
        if (A.phi_ckpt) A.phi_ckpt[k] = Phi;
        if (A.tape) {
            A.tape[k] = Tu;
            A.tape[pl + k] = Gx;
            A.tape[2 * pl + k] = Gy;
        }
    }
    if (A.gsq_part) {
        const double b = block_sum(gsq, red);
        if (threadIdx.x == 0 && threadIdx.y == 0) A.gsq_part[blockIdx.x + gridDim.x * blockIdx.y] += b;
    }
}

template <typename T>
cudaError_t launch_forward(const CxConst& C, const FwdArgs<T>& A, const Launch& L, cudaStream_t s) {
    if (C.Q == 9)
        k_forward<T, 9><<<L.grid, L.block, 0, s>>>(C, A);
    else
        k_forward<T, 5><<<L.grid, L.block, 0, s>>>(C, A);
    return cudaGetLastError();
}

template cudaError_t launch_forward<float>(const CxConst&, const FwdArgs<float>&, const Launch&, cudaStream_t);
template cudaError_t launch_forward<double>(const CxConst&, const FwdArgs<double>&, const Launch&, cudaStream_t);

} // namespace cx
