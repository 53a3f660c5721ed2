// cx_cadj.cu -- continuous-adjoint step (the algorithm of Sec. 3.2.1 that
// solves the adjoint PDE system (FVM-PF-Adj) with the MRT scheme by reversing
// time).  Specialised to Phi_u = 0, Phi_v = r_vu u + r_vv v + g and the
// terminal cost 1/2 |u(T) - u_tgt|^2, with s = T - t:
//   du~/ds = div(D_u grad u~) + a.grad u~ + chi grad v . grad u~ + r_vu v~
//   dv~/ds = div(D_v grad v~) + a.grad v~ + r_vv v~ - div(chi u grad u~)
//   u~(0) = u^N - u_tgt, v~(0) = 0,   dJ/dg^n = 2 alpha g^n + v~(t_{n+1}).
// Per fluid node the step is the forward MRT step of cx_fwd_body.cuh with
// convection velocity -a, first-order sources tau w~_i Phi (Phi_u~ =
// chi G.grad u~ + r_vu v~, Phi_v~ = r_vv v~), the chemotaxis-type source
// (w_i/Cs^2) chi u e_i.(K_v grad u~) for -div(chi u grad u~), and
// grad u~ = -K_u (j~_u + a u~) / (tau d_u Cs^2); u and G = grad v of forward
// step n come from the tape.  The first step (n = N-1) starts from
// phi^eq(u~(0), -a) and 0 read locally.
// Execution as the forward kernel: per-thread staging (k_cadj), or on the
// steps and grids the row-window forward takes, row windows staged by bulk
// copies completed on an mbarrier per stage (k_cadj_rows).
#include <algorithm>

#include "cx_device.cuh"

namespace cx {

template <int Q> constexpr int cadj_stage_values() { return 2 * Q + 5; } // pops, theta, g, u, Gx, Gy

template <typename T, int Q, int NT>
__device__ __forceinline__ void cadj_stage(const CxConst& C, const CadjArgs<T>& A, const NodeIdx& nd, T* s) {
    using L = Lat<Q>;
    if (!nd.fluid) return;
    const int x = nd.x, y = nd.y, k = nd.k;
    if (A.first) {
        cp_async(s, A.w0 + k);
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
    }
    if (C.aniso == CX_ANISO_ROTATED) cp_async(s + 2 * Q * NT, reinterpret_cast<const T*>(C.theta) + k);
    if (nd.ctrl && A.g) cp_async(s + (2 * Q + 1) * NT, A.g + nd.c);
    const size_t pl = (size_t)C.plane;
    cp_async(s + (2 * Q + 2) * NT, A.tape + k);
    cp_async(s + (2 * Q + 3) * NT, A.tape + pl + k);
    cp_async(s + (2 * Q + 4) * NT, A.tape + 2 * pl + k);
}

template <typename T, int Q, int NT, typename Stage>
__device__ __forceinline__ void cadj_compute(const CxConst& C, const KConst<T>& KC, const CadjArgs<T>& A,
                                             const NodeIdx& nd, const Stage& S, typename SqAccT<T>::type& acc) {
    using L = Lat<Q>;
    if (!nd.fluid) {
        if (nd.c >= 0 && !A.accum) A.dJdg[nd.c] = T(0);
        return;
    }
    const int y = nd.y, k = nd.k;
    NodeCoef<T> nc;
    node_coef_th<T>(C, KC, (C.aniso == CX_ANISO_ROTATED) ? S.val(2 * Q) : T(0), y, k, nc);
    const T ax = -nc.ax, ay = -nc.ay; // adjoint convection velocity
    T fu[Q], fv[Q];
    if (A.first) {
        const T w0 = S.pop(0, 0); // per-thread staging only (first step)
        const T a2 = ax * ax + ay * ay;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T ea = ax * T(L::ex(i)) + ay * T(L::ey(i));
            const T e2 = T(L::ex(i) * L::ex(i) + L::ey(i) * L::ey(i));
            const T base = T(1) + T(3) * ea + T(4.5) * (ea * ea - a2 * T(1.0 / 3.0));
            fu[i] = T(L::w(i)) * (base + T(4.5) * (KC.d_u - T(1)) * (e2 - T(2.0 / 3.0)) * T(1.0 / 3.0)) * w0;
            fv[i] = T(0);
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            fu[i] = S.pop(i, -L::ex(i));
            fv[i] = S.pop(Q + i, -L::ex(i));
        }
    }
    T mu[Q], mv[Q];
    Transform<T, Q>::moments(fu, mu);
    Transform<T, Q>::moments(fv, mv);
    const T ut = mu[0], vt = mv[0];
    const T rx = (mu[L::JX] - ax * ut) * KC.inv_tau, ry = (mu[L::JY] - ay * ut) * KC.inv_tau;
    const T gsu = T(-3) / KC.d_u; // -1 / (d_u Cs^2)
    const T gux = gsu * (nc.Ku0 * rx + nc.Ku1 * ry), guy = gsu * (nc.Ku1 * rx + nc.Ku2 * ry);
    const T u = S.val(2 * Q + 2), Gx = S.val(2 * Q + 3), Gy = S.val(2 * Q + 4);
    if (nd.ctrl) {
        const T gv = A.g ? S.val(2 * Q + 1) : T(0);
        T E = KC.two_alpha * gv + vt;
        if (A.accum) E += A.dJdg[nd.c];
        A.dJdg[nd.c] = E;
        if (A.norm) acc.add(E);
    } else if (nd.c >= 0 && !A.accum) {
        A.dJdg[nd.c] = T(0);
    }
    const T Phu = KC.chi * (Gx * gux + Gy * guy) + KC.r_vu * vt;
    const T Phv = KC.r_vv * vt;

    T mh[Q], dm[Q], rl[Q], bt[Q];
    meq_unit<T, Q>(ax, ay, KC.d_u, mh);
#pragma unroll
    for (int kk = 0; kk < Q; ++kk) dm[kk] = mu[kk] - ut * mh[kk];
    relax_n<T, Q>(KC, nc.Ku0, nc.Ku1, nc.Ku2, dm, rl);
    Transform<T, Q>::transpose(rl, bt);
    {
        const T Vx = ax - T(0.5) * (nc.Ku0 * ax + nc.Ku1 * ay), Vy = ay - T(0.5) * (nc.Ku1 * ax + nc.Ku2 * ay);
        const T su = KC.tau * Phu;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T wt = T(L::w(i)) * (T(1) + T(3) * (Vx * T(L::ex(i)) + Vy * T(L::ey(i))));
            A.out(i)[k] = fu[i] - bt[i] + wt * su;
        }
    }
    meq_unit<T, Q>(ax, ay, KC.d_v, mh);
#pragma unroll
    for (int kk = 0; kk < Q; ++kk) dm[kk] = mv[kk] - vt * mh[kk];
    relax_n<T, Q>(KC, nc.Kv0, nc.Kv1, nc.Kv2, dm, rl);
    Transform<T, Q>::transpose(rl, bt);
    {
        const T Vx = ax - T(0.5) * (nc.Kv0 * ax + nc.Kv1 * ay), Vy = ay - T(0.5) * (nc.Kv1 * ax + nc.Kv2 * ay);
        const T sv = KC.tau * Phv;
        const T Fx = KC.chi * u * (nc.Kv0 * gux + nc.Kv1 * guy), Fy = KC.chi * u * (nc.Kv1 * gux + nc.Kv2 * guy);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T wt = T(L::w(i)) * (T(1) + T(3) * (Vx * T(L::ex(i)) + Vy * T(L::ey(i))));
            const T src = T(3.0 * L::w(i)) * (T(L::ex(i)) * Fx + T(L::ey(i)) * Fy);
            A.out(Q + i)[k] = fv[i] - bt[i] + wt * sv + src;
        }
    }
}

template <typename T, int Q, int NT>
__global__ void __launch_bounds__(NT) k_cadj(const CxConst C, const KConst<T> KC, const CadjArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NV = cadj_stage_values<Q>();
    T* const s0 = reinterpret_cast<T*>(smem_raw) + threadIdx.x;
    T* const s1 = s0 + NV * NT;
    typename SqAccT<T>::type acc;
    ChunkIter<NT> it(C);
    NodeIdx cur = it.valid() ? it.node(C) : no_node();
    allow_next_grid();
    wait_prior_grid();
    if (it.valid()) cadj_stage<T, Q, NT>(C, A, cur, s0);
    cp_async_commit();
    bool odd = false;
    while (it.valid()) {
        it.next();
        const NodeIdx nxt = it.valid() ? it.node(C) : no_node();
        if (it.valid()) cadj_stage<T, Q, NT>(C, A, nxt, odd ? s0 : s1);
        cp_async_commit();
        cp_async_wait<1>();
        cadj_compute<T, Q, NT>(C, KC, A, cur, ThreadSlots<T, NT>{odd ? s1 : s0}, acc);
        cur = nxt;
        odd = !odd;
    }
    cp_async_wait<0>();
    const int slot = blockIdx.x * (NT >> 5) + (threadIdx.x >> 5);
    acc.flush(A.e2_part + slot, A.emax_part + slot);
}

template <typename T, int Q, int NT>
static cudaError_t launch_qn(const CxConst& C, const KConst<T>& K, const CadjArgs<T>& A, const Launch& L,
                             cudaStream_t s) {
    const size_t smem = (size_t)2 * cadj_stage_values<Q>() * NT * sizeof(T);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(k_cadj<T, Q, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024);
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
    return cudaLaunchKernelEx(&cfg, k_cadj<T, Q, NT>, C, K, A);
}

template <typename T, int Q>
static cudaError_t launch_q(const CxConst& C, const KConst<T>& K, const CadjArgs<T>& A, const Launch& L,
                            cudaStream_t s) {
    switch (L.block.x) {
    case 64: return launch_qn<T, Q, 64>(C, K, A, L, s);
    case 128: return launch_qn<T, Q, 128>(C, K, A, L, s);
    case 256: return launch_qn<T, Q, 256>(C, K, A, L, s);
    default: return cudaErrorInvalidConfiguration;
    }
}

// ---- row-window form (not the first step, no solid nodes, rows of whole 16-byte units)

// Bulk copies of one row segment's stage (issued by one thread): the 2Q
// population windows (pulled from x - e_i, as the forward scheme), the angle
// (rotated tensors), g (whole-grid control) and the forward tape (u, G_x, G_y).
template <typename T, int Q, int NT>
__device__ __forceinline__ void cadj_issue_rows(const CxConst& C, const CadjArgs<T>& A, int y, int x0, T* st,
                                                uint64_t* bar) {
    using L = Lat<Q>;
    using RW = RowWindow<T, Q, NT>;
    const int nx = C.nx, nv = min(NT, nx - x0);
    const int rm = y == 0 ? C.ny - 1 : y - 1, rp = y == C.ny - 1 ? 0 : y + 1;
    const bool rot = C.aniso == CX_ANISO_ROTATED, gb = A.g && C.ctrl_full;
    const uint32_t nb = (uint32_t)nv * sizeof(T);
    mbar_expect_tx(bar, (uint32_t)(2 * Q * (nv + 2 * RW::H)) * sizeof(T) + nb * (3u + rot + gb) + A.tx_pad);
#pragma unroll
    for (int j = 0; j < 2 * Q; ++j) {
        const int i = j < Q ? j : j - Q;
        const int ys = L::ey(i) > 0 ? rm : (L::ey(i) < 0 ? rp : y);
        bulk_row_window<T, NT>(st + j * RW::W, A.in(j) + (size_t)ys * nx, x0, nv, nx, bar);
    }
    T* const loc = st + 2 * Q * RW::W;
    const size_t k0 = (size_t)y * nx + x0, pl = (size_t)C.plane;
    if (rot) bulk_g2s(loc, reinterpret_cast<const T*>(C.theta) + k0, nb, bar);
    if (gb) bulk_g2s(loc + NT, A.g + k0, nb, bar);
    bulk_g2s(loc + 2 * NT, A.tape + k0, nb, bar);
    bulk_g2s(loc + 3 * NT, A.tape + pl + k0, nb, bar);
    bulk_g2s(loc + 4 * NT, A.tape + 2 * pl + k0, nb, bar);
}

// g of a controlled node when the control window is not the whole grid
template <typename T, int Q, int NT>
__device__ __forceinline__ void cadj_stage_ctrl(const CxConst& C, const CadjArgs<T>& A, const NodeIdx& nd, T* st) {
    using RW = RowWindow<T, Q, NT>;
    if (C.ctrl_full || !nd.ctrl || !A.g) return;
    cp_async(st + 2 * Q * RW::W + NT + threadIdx.x, A.g + nd.c);
}

template <typename T, int Q, int NT> constexpr int cadj_rows_stage_values() {
    return 2 * Q * RowWindow<T, Q, NT>::W + 5 * NT;
}
template <typename T, int Q, int NT> constexpr size_t cadj_rows_smem() {
    return (size_t)2 * cadj_rows_stage_values<T, Q, NT>() * sizeof(T) + 2 * sizeof(uint64_t);
}

template <typename T, int Q, int NT>
__global__ void __launch_bounds__(NT) k_cadj_rows(const CxConst C, const KConst<T> KC, const CadjArgs<T> A) {
    using RW = RowWindow<T, Q, NT>;
    constexpr int SV = cadj_rows_stage_values<T, Q, NT>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* const st0 = reinterpret_cast<T*>(smem_raw);
    T* const st1 = st0 + SV;
    uint64_t* const bar = reinterpret_cast<uint64_t*>(st1 + SV);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    typename SqAccT<T>::type acc;
    ChunkIter<NT> it(C);
    NodeIdx cur = it.valid() ? it.node(C) : no_node();
    allow_next_grid();
    wait_prior_grid();
    if (block_sees_timeout(A.status)) return;
    if (it.valid()) {
        if (threadIdx.x == 0) cadj_issue_rows<T, Q, NT>(C, A, it.y, it.seg * NT, st0, &bar[0]);
        cadj_stage_ctrl<T, Q, NT>(C, A, cur, st0);
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
            if (threadIdx.x == 0) cadj_issue_rows<T, Q, NT>(C, A, it.y, it.seg * NT, sn, &bar[b ^ 1]);
            cadj_stage_ctrl<T, Q, NT>(C, A, nxt, sn);
        }
        cp_async_commit();
        cp_async_wait<1>();
        ok = mbar_wait(&bar[b], (phase >> b) & 1u);
        phase ^= 1u << b;
        if (ok) cadj_compute<T, Q, NT>(C, KC, A, cur, RW{(b ? st1 : st0) + threadIdx.x}, acc);
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
    const int slot = blockIdx.x * (NT >> 5) + (threadIdx.x >> 5);
    acc.flush(A.e2_part + slot, A.emax_part + slot);
}

template <typename T> static bool cadj_rows_eligible(const CxConst& C, const CadjArgs<T>& A, const Launch& L) {
    constexpr int H = 16 / (int)sizeof(T);
    auto al = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
    if (!L.row_windows || A.first || C.has_solid || C.nx % H != 0) return false;
    if (!rows_pipelined(C, L, L.grid.x)) return false;
    if (L.block.x != 128 && L.block.x != 256) return false;
    for (int j = 0; j < 2 * C.Q; ++j)
        if (!al(A.pin[j])) return false;
    if (!al(A.tape) || (C.plane * (long long)sizeof(T)) % 16 != 0) return false;
    if (C.aniso == CX_ANISO_ROTATED && !al(C.theta)) return false;
    if (C.ctrl_full && A.g && !al(A.g)) return false;
    return true;
}

template <typename T, int Q, int NT>
static cudaError_t launch_rows_qn(const CxConst& C, const KConst<T>& K, const CadjArgs<T>& A, const Launch& L,
                                  cudaStream_t s) {
    constexpr size_t smem = cadj_rows_smem<T, Q, NT>();
    static int blocks_cap = 0; // resident blocks on this device (never above the grid the partials are sized for)
    if (blocks_cap == 0) {
        cudaError_t e =
            cudaFuncSetAttribute(k_cadj_rows<T, Q, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int dev = 0, nsm = 0, occ = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
            (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cadj_rows<T, Q, NT>, NT, smem)) != cudaSuccess)
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
    CadjArgs<T> A2 = A;
    A2.tx_pad = L.row_windows == 2 ? 16u : 0u; // test mode: no stage ever completes
    return cudaLaunchKernelEx(&cfg, k_cadj_rows<T, Q, NT>, C, K, A2);
}

template <typename T, int Q>
static cudaError_t launch_rows_q(const CxConst& C, const KConst<T>& K, const CadjArgs<T>& A, const Launch& L,
                                 cudaStream_t s) {
    return L.block.x == 128 ? launch_rows_qn<T, Q, 128>(C, K, A, L, s) : launch_rows_qn<T, Q, 256>(C, K, A, L, s);
}

template <typename T>
cudaError_t launch_cadj(const CxConst& C, const KConst<T>& K, const CadjArgs<T>& A, const Launch& L, cudaStream_t s) {
    if (cadj_rows_eligible<T>(C, A, L))
        return C.Q == 9 ? launch_rows_q<T, 9>(C, K, A, L, s) : launch_rows_q<T, 5>(C, K, A, L, s);
    return C.Q == 9 ? launch_q<T, 9>(C, K, A, L, s) : launch_q<T, 5>(C, K, A, L, s);
}

template cudaError_t launch_cadj<float>(const CxConst&, const KConst<float>&, const CadjArgs<float>&, const Launch&,
                                        cudaStream_t);
template cudaError_t launch_cadj<double>(const CxConst&, const KConst<double>&, const CadjArgs<double>&,
                                         const Launch&, cudaStream_t);

} // namespace cx
