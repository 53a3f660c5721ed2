// cx_adjoint.cu -- AMRT adjoint step with fused gradient assembly, one time
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
#include "cx_device.cuh"

namespace cx {

template <typename T, int Q>
__global__ void __launch_bounds__(256) k_adjoint(const CxConst C, const AdjArgs<T> A) {
    using L = Lat<Q>;
    __shared__ double red[32];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    double e2 = 0.0, emax = 0.0;
    const bool inside = (x < C.nx) && (y < C.ny);
    const int k = y * C.nx + x;
    const bool fluid = inside && !(C.has_solid && C.solid[k]);
    if (fluid) {
        const size_t pl = (size_t)C.plane;
        T ru[Q], rv[Q];
        const int xm = x == 0 ? C.nx - 1 : x - 1, xp = x == C.nx - 1 ? 0 : x + 1;
        const int ym = y == 0 ? C.ny - 1 : y - 1, yp = y == C.ny - 1 ? 0 : y + 1;
        if (A.terminal) {
            const T wu0 = ldg(A.wu + k);
            const T wv0 = A.wv ? ldg(A.wv + k) : T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int xd = L::ex(i) > 0 ? xp : (L::ex(i) < 0 ? xm : x);
                const int yd = L::ey(i) > 0 ? yp : (L::ey(i) < 0 ? ym : y);
                const int kd = yd * C.nx + xd;
                if (i != 0 && C.has_solid && C.solid[kd]) {
                    ru[i] = wu0;
                    rv[i] = wv0;
                } else {
                    ru[i] = ldg(A.wu + kd);
                    rv[i] = A.wv ? ldg(A.wv + kd) : T(0);
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int xd = L::ex(i) > 0 ? xp : (L::ex(i) < 0 ? xm : x);
                const int yd = L::ey(i) > 0 ? yp : (L::ey(i) < 0 ? ym : y);
                const int kd = yd * C.nx + xd;
                if (i != 0 && C.has_solid && C.solid[kd]) {
                    ru[i] = ldg(A.Rin + L::opp(i) * pl + k);
                    rv[i] = ldg(A.Rin + (Q + L::opp(i)) * pl + k);
                } else {
                    ru[i] = ldg(A.Rin + i * pl + kd);
                    rv[i] = ldg(A.Rin + (Q + i) * pl + kd);
                }
            }
        }
        NodeCoef<T> nc;
        node_coef<T>(C, x, y, k, nc);
        const T Tu = ldg(A.tape + k);
        const T Gx = ldg(A.tape + pl + k);
        const T Gy = ldg(A.tape + 2 * pl + k);
        const T tau = T(C.tau);

        // --- transposed collisions: mt = M^T Pi^T (N^-1 M rho), Tcal = sum_k z_k mh_k
        T mh[Q], lam[Q], z[Q];
        T psu[Q], psv[Q];
        {
            meq_unit<T, Q>(nc.ax, nc.ay, T(C.d_u), mh);
#pragma unroll
            for (int kk = 0; kk < Q; ++kk) {
                T s = T(0);
#pragma unroll
                for (int i = 0; i < Q; ++i)
                    if (L::M(kk, i) != 0) s += T(L::M(kk, i)) * ru[i];
                lam[kk] = s * T(L::inv_n(kk));
            }
            relax_T<T, Q>(C, nc.Ku0, nc.Ku1, nc.Ku2, lam, z);
            T Tc = T(0);
#pragma unroll
            for (int kk = 0; kk < Q; ++kk) Tc += z[kk] * mh[kk];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                T s = T(0);
#pragma unroll
                for (int kk = 0; kk < Q; ++kk)
                    if (L::M(kk, i) != 0) s += T(L::M(kk, i)) * z[kk];
                psu[i] = ru[i] - s + Tc;
            }
        }
        {
            meq_unit<T, Q>(nc.ax, nc.ay, T(C.d_v), mh);
#pragma unroll
            for (int kk = 0; kk < Q; ++kk) {
                T s = T(0);
#pragma unroll
                for (int i = 0; i < Q; ++i)
                    if (L::M(kk, i) != 0) s += T(L::M(kk, i)) * rv[i];
                lam[kk] = s * T(L::inv_n(kk));
            }
            relax_T<T, Q>(C, nc.Kv0, nc.Kv1, nc.Kv2, lam, z);
            T Tc = T(0);
#pragma unroll
            for (int kk = 0; kk < Q; ++kk) Tc += z[kk] * mh[kk];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                T s = T(0);
#pragma unroll
                for (int kk = 0; kk < Q; ++kk)
                    if (L::M(kk, i) != 0) s += T(L::M(kk, i)) * z[kk];
                psv[i] = rv[i] - s + Tc;
            }
        }

        // --- coupling through tau S_u,i = 3 w_i chi u e_i . (K_u G)
        T Yx = T(0), Yy = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            Yx += T(3.0 * L::w(i) * L::ex(i)) * ru[i];
            Yy += T(3.0 * L::w(i) * L::ey(i)) * ru[i];
        }
        const T chi = T(C.chi);
        T adj_Tu = chi * (Yx * (nc.Ku0 * Gx + nc.Ku1 * Gy) + Yy * (nc.Ku1 * Gx + nc.Ku2 * Gy));
        const T aGx = chi * Tu * (nc.Ku0 * Yx + nc.Ku1 * Yy);
        const T aGy = chi * Tu * (nc.Ku1 * Yx + nc.Ku2 * Yy);
        // G = -(K_v (j_v - a v)/tau + K_v a Phi/2) / (d_v Cs^2)
        const T KGx = nc.Kv0 * aGx + nc.Kv1 * aGy, KGy = nc.Kv1 * aGx + nc.Kv2 * aGy;
        const T sc = T(3.0) / T(C.d_v);
        const T ajx = -KGx * sc / tau, ajy = -KGy * sc / tau;
        const T aKG = nc.ax * KGx + nc.ay * KGy;
        T adj_Tv = aKG * sc / tau;
        T adj_Phi = T(-0.5) * aKG * sc;

        // --- reaction/control source: sigma^n and the use of Phi^n at step n+1
        const T Kax = nc.Kv0 * nc.ax + nc.Kv1 * nc.ay, Kay = nc.Kv1 * nc.ax + nc.Kv2 * nc.ay;
        const T Vx = nc.ax - T(0.5) * Kax, Vy = nc.ay - T(0.5) * Kay;
        T sigma = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i)
            sigma += T(L::w(i)) * (T(1) + T(3) * (Vx * T(L::ex(i)) + Vy * T(L::ey(i)))) * rv[i];
        const T cn = (C.source_order == 1 || A.n == 0) ? tau : T(1.5) * tau;
        adj_Phi += cn * sigma;
        if (!A.terminal && C.source_order != 1) adj_Phi += T(-0.5) * tau * A.sigma[k];
        A.sigma[k] = sigma;
        adj_Tu += T(C.r_vu) * adj_Phi;
        adj_Tv += T(C.r_vv) * adj_Phi;

        const int c = ctrl_window(C, x, y);
        if (ctrl_active(C, c)) {
            const T gv = A.g ? ldg(A.g + c) : T(0);
            const T E = adj_Phi + T(2.0 * C.alpha) * gv;
            A.dJdg[c] = E;
            e2 = (double)E * (double)E;
            emax = fabs((double)E);
        } else if (c >= 0) {
            A.dJdg[c] = T(0);
        }
        T* Ou = A.Rout;
        T* Ov = A.Rout + (size_t)Q * pl;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            Ou[i * pl + k] = psu[i] + adj_Tu;
            Ov[i * pl + k] = psv[i] + adj_Tv + T(L::ex(i)) * ajx + T(L::ey(i)) * ajy;
        }
    } else if (inside) {
        // solid window nodes are not controlled: zero gradient
        const int c = ctrl_window(C, x, y);
        if (c >= 0) A.dJdg[c] = T(0);
    }
    const double b2 = block_sum(e2, red);
    const double bm = block_max(emax, red);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const int b = blockIdx.x + gridDim.x * blockIdx.y;
        A.e2_part[b] += b2;
        A.emax_part[b] = fmax(A.emax_part[b], bm);
    }
}

template <typename T>
cudaError_t launch_adjoint(const CxConst& C, const AdjArgs<T>& A, const Launch& L, cudaStream_t s) {
    if (C.Q == 9)
        k_adjoint<T, 9><<<L.grid, L.block, 0, s>>>(C, A);
    else
        k_adjoint<T, 5><<<L.grid, L.block, 0, s>>>(C, A);
    return cudaGetLastError();
}

template cudaError_t launch_adjoint<float>(const CxConst&, const AdjArgs<float>&, const Launch&, cudaStream_t);
template cudaError_t launch_adjoint<double>(const CxConst&, const AdjArgs<double>&, const Launch&, cudaStream_t);

} // namespace cx
