// cx_tlm.cu -- tangent-linear (sensitivity) step of the coupled MRT scheme: the
// forward step of cx_fwd_body.cuh differentiated about a base trajectory, for
// the linearised line search of Sec. 2.3 (the sensitivity problem solved by
// the same lattice Boltzmann method).
//
// Per fluid node, with the base state's (u, G) at step n read from the tape
// and the tangent populations df pulled as in the forward:
//   dTheta   = sum_i df_i,  dj_v = sum_i e_i df_v,i
//   dPhi     = r_vu du + r_vv dv + dg^n
//   dG       = -(K_v (dj_v - a dv)/tau + K_v a dPhi / 2) / (d_v Cs^2)
//   dP_Theta = df - M^-1 Pi_Theta (M df - m^eq(dTheta))         (linear map)
//   dP_u,i  += (w_i / Cs^2) chi e_i . K_u (du G + u dG)           (product rule)
//   dP_v,i  += w~_i [c_n dPhi^n + c'_n dPhi^{n-1}]
// Execution and staging as in the forward kernel: persistent grid, per-thread
// two-stage cp.async staging of the next node (k_tlm), or, on the steps and
// grids k_forward_rows takes, row windows staged by bulk copies completed on
// an mbarrier per stage (k_tlm_rows).
#include <algorithm>

#include "cx_device.cuh"

namespace cx {

template <int Q> constexpr int tlm_stage_values() { return 2 * Q + 6; } // pops, theta, dg, dPhi, u, Gx, Gy

template <typename T, int Q, int NT>
__device__ __forceinline__ void tlm_stage(const CxConst& C, const TlmArgs<T>& A, const NodeIdx& nd, T* s) {
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
        cp_async(s + (2 * Q + 2) * NT, A.dphi + k);
    }
    if (C.aniso == CX_ANISO_ROTATED) cp_async(s + 2 * Q * NT, reinterpret_cast<const T*>(C.theta) + k);
    if (nd.ctrl && A.dg) cp_async(s + (2 * Q + 1) * NT, A.dg + nd.c);
    const size_t pl = (size_t)C.plane;
    cp_async(s + (2 * Q + 3) * NT, A.tape + k);
    cp_async(s + (2 * Q + 4) * NT, A.tape + pl + k);
    cp_async(s + (2 * Q + 5) * NT, A.tape + 2 * pl + k);
}

template <typename T, int Q, int NT, typename Stage>
__device__ __forceinline__ void tlm_compute(const CxConst& C, const KConst<T>& KC, const TlmArgs<T>& A,
                                            const NodeIdx& nd, const Stage& S) {
    using L = Lat<Q>;
    if (!nd.fluid) return;
    const int y = nd.y, k = nd.k;
    T fu[Q], fv[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        fu[i] = S.pop(i, -L::ex(i));
        fv[i] = S.pop(Q + i, -L::ex(i));
    }
    const T dg = (nd.ctrl && A.dg) ? S.val(2 * Q + 1) : T(0);
    NodeCoef<T> nc;
    node_coef_th<T>(C, KC, (C.aniso == CX_ANISO_ROTATED) ? S.val(2 * Q) : T(0), y, k, nc);
    T mu[Q], mv[Q];
    Transform<T, Q>::moments(fu, mu);
    Transform<T, Q>::moments(fv, mv);
    const T dTu = mu[0], dTv = mv[0];
    const T Phi = KC.r_vu * dTu + KC.r_vv * dTv + dg;
    const T Phi_prev = (A.n == 0) ? Phi : S.val(2 * Q + 2);
    const T rx = (mv[L::JX] - nc.ax * dTv) * KC.inv_tau, ry = (mv[L::JY] - nc.ay * dTv) * KC.inv_tau;
    const T Kax = nc.Kv0 * nc.ax + nc.Kv1 * nc.ay, Kay = nc.Kv1 * nc.ax + nc.Kv2 * nc.ay;
    const T dGx = KC.gsc * (nc.Kv0 * rx + nc.Kv1 * ry + T(0.5) * Kax * Phi);
    const T dGy = KC.gsc * (nc.Kv1 * rx + nc.Kv2 * ry + T(0.5) * Kay * Phi);
    const T u = S.val(2 * Q + 3), Gx = S.val(2 * Q + 4), Gy = S.val(2 * Q + 5);

    T mh[Q], dm[Q], rl[Q], bt[Q];
    meq_unit<T, Q>(nc.ax, nc.ay, KC.d_u, mh);
#pragma unroll
    for (int kk = 0; kk < Q; ++kk) dm[kk] = mu[kk] - dTu * mh[kk];
    relax_n<T, Q>(KC, nc.Ku0, nc.Ku1, nc.Ku2, dm, rl);
    const T Sx = dTu * Gx + u * dGx, Sy = dTu * Gy + u * dGy; // d(u G)
    const T Fx = KC.chi * (nc.Ku0 * Sx + nc.Ku1 * Sy);
    const T Fy = KC.chi * (nc.Ku1 * Sx + nc.Ku2 * Sy);
    Transform<T, Q>::transpose(rl, bt);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T src = T(3.0 * L::w(i)) * (T(L::ex(i)) * Fx + T(L::ey(i)) * Fy);
        A.out(i)[k] = fu[i] - bt[i] + src;
    }
    meq_unit<T, Q>(nc.ax, nc.ay, KC.d_v, mh);
#pragma unroll
    for (int kk = 0; kk < Q; ++kk) dm[kk] = mv[kk] - dTv * mh[kk];
    relax_n<T, Q>(KC, nc.Kv0, nc.Kv1, nc.Kv2, dm, rl);
    const T Vx = nc.ax - T(0.5) * Kax, Vy = nc.ay - T(0.5) * Kay;
    const T srcv = (A.n == 0) ? KC.c_first * Phi : KC.c_now * Phi + KC.c_prev * Phi_prev;
    Transform<T, Q>::transpose(rl, bt);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T wt = T(L::w(i)) * (T(1) + T(3) * (Vx * T(L::ex(i)) + Vy * T(L::ey(i))));
        A.out(Q + i)[k] = fv[i] - bt[i] + wt * srcv;
    }
    A.dphi[k] = Phi;
}

template <typename T, int Q, int NT>
__global__ void __launch_bounds__(NT) k_tlm(const CxConst C, const KConst<T> KC, const TlmArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NV = tlm_stage_values<Q>();
    T* const s0 = reinterpret_cast<T*>(smem_raw) + threadIdx.x;
    T* const s1 = s0 + NV * NT;
    ChunkIter<NT> it(C);
    NodeIdx cur = it.valid() ? it.node(C) : no_node();
    allow_next_grid();
    wait_prior_grid();
    if (it.valid()) tlm_stage<T, Q, NT>(C, A, cur, s0);
    cp_async_commit();
    bool odd = false;
    while (it.valid()) {
        it.next();
        const NodeIdx nxt = it.valid() ? it.node(C) : no_node();
        if (it.valid()) tlm_stage<T, Q, NT>(C, A, nxt, odd ? s0 : s1);
        cp_async_commit();
        cp_async_wait<1>();
        tlm_compute<T, Q, NT>(C, KC, A, cur, ThreadSlots<T, NT>{odd ? s1 : s0});
        cur = nxt;
        odd = !odd;
    }
    cp_async_wait<0>();
}

template <typename T, int Q, int NT>
static cudaError_t launch_qn(const CxConst& C, const KConst<T>& K, const TlmArgs<T>& A, const Launch& L,
                             cudaStream_t s) {
    const size_t smem = (size_t)2 * tlm_stage_values<Q>() * NT * sizeof(T);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_tlm<T, Q, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = L.grid;
    cfg.blockDim = L.block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_tlm<T, Q, NT>, C, K, A);
}

template <typename T, int Q>
static cudaError_t launch_q(const CxConst& C, const KConst<T>& K, const TlmArgs<T>& A, const Launch& L,
                            cudaStream_t s) {
    switch (L.block.x) {
    case 64: return launch_qn<T, Q, 64>(C, K, A, L, s);
    case 128: return launch_qn<T, Q, 128>(C, K, A, L, s);
    case 256: return launch_qn<T, Q, 256>(C, K, A, L, s);
    default: return cudaErrorInvalidConfiguration;
    }
}

// ---- row-window form (steps n >= 1, no solid nodes, rows of whole 16-byte units)

// Bulk copies of one row segment's stage (issued by one thread): the 2Q
// tangent population windows, the angle (rotated tensors), dg (whole-grid
// control), dPhi^{n-1} and the base tape (u, G_x, G_y).
template <typename T, int Q, int NT>
__device__ __forceinline__ void tlm_issue_rows(const CxConst& C, const TlmArgs<T>& A, int y, int x0, T* st,
                                               uint64_t* bar) {
    using L = Lat<Q>;
    using RW = RowWindow<T, Q, NT>;
    const int nx = C.nx, nv = min(NT, nx - x0);
    const int rm = y == 0 ? C.ny - 1 : y - 1, rp = y == C.ny - 1 ? 0 : y + 1;
    const bool rot = C.aniso == CX_ANISO_ROTATED, gb = A.dg && C.ctrl_full;
    const uint32_t nb = (uint32_t)nv * sizeof(T);
    mbar_expect_tx(bar, (uint32_t)(2 * Q * (nv + 2 * RW::H)) * sizeof(T) + nb * (4u + rot + gb) + A.tx_pad);
#pragma unroll
    for (int j = 0; j < 2 * Q; ++j) {
        const int i = j < Q ? j : j - Q;
        const int ys = L::ey(i) > 0 ? rm : (L::ey(i) < 0 ? rp : y); // pull from x - e_i
        bulk_row_window<T, NT>(st + j * RW::W, A.in(j) + (size_t)ys * nx, x0, nv, nx, bar);
    }
    T* const loc = st + 2 * Q * RW::W;
    const size_t k0 = (size_t)y * nx + x0, pl = (size_t)C.plane;
    if (rot) bulk_g2s(loc, reinterpret_cast<const T*>(C.theta) + k0, nb, bar);
    if (gb) bulk_g2s(loc + NT, A.dg + k0, nb, bar);
    bulk_g2s(loc + 2 * NT, A.dphi + k0, nb, bar);
    bulk_g2s(loc + 3 * NT, A.tape + k0, nb, bar);
    bulk_g2s(loc + 4 * NT, A.tape + pl + k0, nb, bar);
    bulk_g2s(loc + 5 * NT, A.tape + 2 * pl + k0, nb, bar);
}

// dg of a controlled node when the control window is not the whole grid
template <typename T, int Q, int NT>
__device__ __forceinline__ void tlm_stage_ctrl(const CxConst& C, const TlmArgs<T>& A, const NodeIdx& nd, T* st) {
    using RW = RowWindow<T, Q, NT>;
    if (C.ctrl_full || !nd.ctrl || !A.dg) return;
    cp_async(st + 2 * Q * RW::W + NT + threadIdx.x, A.dg + nd.c);
}

template <typename T, int Q, int NT> constexpr int tlm_rows_stage_values() {
    return 2 * Q * RowWindow<T, Q, NT>::W + 6 * NT;
}
template <typename T, int Q, int NT> constexpr size_t tlm_rows_smem() {
    return (size_t)2 * tlm_rows_stage_values<T, Q, NT>() * sizeof(T) + 2 * sizeof(uint64_t);
}

template <typename T, int Q, int NT>
__global__ void __launch_bounds__(NT) k_tlm_rows(const CxConst C, const KConst<T> KC, const TlmArgs<T> A) {
    using RW = RowWindow<T, Q, NT>;
    constexpr int SV = tlm_rows_stage_values<T, Q, NT>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* const st0 = reinterpret_cast<T*>(smem_raw);
    T* const st1 = st0 + SV;
    uint64_t* const bar = reinterpret_cast<uint64_t*>(st1 + SV);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    ChunkIter<NT> it(C);
    NodeIdx cur = it.valid() ? it.node(C) : no_node();
    allow_next_grid();
    wait_prior_grid(); // the previous step's tangent populations and dPhi are complete
    if (block_sees_timeout(A.status)) return;
    if (it.valid()) {
        if (threadIdx.x == 0) tlm_issue_rows<T, Q, NT>(C, A, it.y, it.seg * NT, st0, &bar[0]);
        tlm_stage_ctrl<T, Q, NT>(C, A, cur, st0);
    }
    cp_async_commit();
    unsigned phase = 0; // bit b: parity of stage b's next completion
    int b = 0;          // stage of the current segment
    bool ok = true;
    while (it.valid()) {
        it.next();
        const NodeIdx nxt = it.valid() ? it.node(C) : no_node();
        T* const sn = b ? st0 : st1;
        if (it.valid()) { // stage b^1 is free: every thread passed the barrier that ended its last use
            if (threadIdx.x == 0) tlm_issue_rows<T, Q, NT>(C, A, it.y, it.seg * NT, sn, &bar[b ^ 1]);
            tlm_stage_ctrl<T, Q, NT>(C, A, nxt, sn);
        }
        cp_async_commit();
        cp_async_wait<1>();
        ok = mbar_wait(&bar[b], (phase >> b) & 1u);
        phase ^= 1u << b;
        if (ok) tlm_compute<T, Q, NT>(C, KC, A, cur, RW{(b ? st1 : st0) + threadIdx.x});
        if (__syncthreads_or(!ok)) { // all threads leave together when a stage never completed
            ok = false;
            break;
        }
        cur = nxt;
        b ^= 1;
    }
    if (!ok) {
        // bounded waits for the copies still in flight, then report
        if (it.valid()) mbar_wait(&bar[b ^ 1], (phase >> (b ^ 1)) & 1u);
        mbar_wait(&bar[b], ((phase >> b) & 1u) ^ 1u);
        if (threadIdx.x == 0 && A.status) atomicOr(A.status, ST_TIMEOUT);
    }
    cp_async_wait<0>();
}

template <typename T> static bool tlm_rows_eligible(const CxConst& C, const TlmArgs<T>& A, const Launch& L) {
    constexpr int H = 16 / (int)sizeof(T);
    auto al = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
    if (!L.row_windows || A.n == 0 || C.has_solid || C.nx % H != 0) return false;
    if (!rows_pipelined(C, L, L.grid.x)) return false;
    if (L.block.x != 128 && L.block.x != 256) return false;
    for (int j = 0; j < 2 * C.Q; ++j)
        if (!al(A.pin[j])) return false;
    if (!al(A.dphi) || !al(A.tape) || (C.plane * (long long)sizeof(T)) % 16 != 0) return false;
    if (C.aniso == CX_ANISO_ROTATED && !al(C.theta)) return false;
    if (C.ctrl_full && A.dg && !al(A.dg)) return false;
    return true;
}

template <typename T, int Q, int NT>
static cudaError_t launch_rows_qn(const CxConst& C, const KConst<T>& K, const TlmArgs<T>& A, const Launch& L,
                                  cudaStream_t s) {
    constexpr size_t smem = tlm_rows_smem<T, Q, NT>();
    static int blocks_cap = 0; // resident blocks on this device (the kernel keeps no per-block partials)
    if (blocks_cap == 0) {
        cudaError_t e =
            cudaFuncSetAttribute(k_tlm_rows<T, Q, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int dev = 0, nsm = 0, occ = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
            (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tlm_rows<T, Q, NT>, NT, smem)) != cudaSuccess)
            return e;
        blocks_cap = std::max(1, nsm * occ);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(std::min<unsigned>(L.grid.x, (unsigned)blocks_cap));
    cfg.blockDim = L.block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    TlmArgs<T> A2 = A;
    A2.tx_pad = L.row_windows == 2 ? 16u : 0u; // test mode: no stage ever completes
    return cudaLaunchKernelEx(&cfg, k_tlm_rows<T, Q, NT>, C, K, A2);
}

template <typename T, int Q>
static cudaError_t launch_rows_q(const CxConst& C, const KConst<T>& K, const TlmArgs<T>& A, const Launch& L,
                                 cudaStream_t s) {
    return L.block.x == 128 ? launch_rows_qn<T, Q, 128>(C, K, A, L, s) : launch_rows_qn<T, Q, 256>(C, K, A, L, s);
}

template <typename T>
cudaError_t launch_tlm(const CxConst& C, const KConst<T>& K, const TlmArgs<T>& A, const Launch& L, cudaStream_t s) {
    if (tlm_rows_eligible<T>(C, A, L))
        return C.Q == 9 ? launch_rows_q<T, 9>(C, K, A, L, s) : launch_rows_q<T, 5>(C, K, A, L, s);
    return C.Q == 9 ? launch_q<T, 9>(C, K, A, L, s) : launch_q<T, 5>(C, K, A, L, s);
}

template cudaError_t launch_tlm<float>(const CxConst&, const KConst<float>&, const TlmArgs<float>&, const Launch&,
                                       cudaStream_t);
template cudaError_t launch_tlm<double>(const CxConst&, const KConst<double>&, const TlmArgs<double>&, const Launch&,
                                        cudaStream_t);

} // namespace cx
