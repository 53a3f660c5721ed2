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
// the adjoint tape (u, G_x, G_y), and accumulates (g^n)^2 for the penalty.
//
// Execution: a persistent grid; each block walks row segments of blockDim.x
// nodes.  While a thread computes its current node it has already issued the
// cp.async copies of its next node's populations and per-node scalars into its
// own shared-memory slots (two stages), so DRAM latency overlaps the
// arithmetic without holding registers for loads in flight.
//
// Row-window variant (k_forward_rows; steps n >= 1 of grids without solid
// nodes whose rows are a whole number of 16-byte units): the block stages a
// row segment at a time.  One thread issues, per population plane, bulk
// asynchronous copies of the source row window (the segment widened by 16
// bytes on each side, periodic ends taken from the other end of the row) and
// of the node-local planes, all completing on the stage's mbarrier; every
// thread then pulls its populations from the shared windows.  Two stages:
// the copies of segment s+1 run while segment s is computed.  This replaces
// the per-node address arithmetic and 4-byte copies of the per-thread
// pipeline with a few dozen instructions per segment.
#include <algorithm>

#include "cx_fwd_body.cuh"
#include "cx_rows.cuh"

namespace cx {

template <typename T, int Q, int NT>
__global__ void __launch_bounds__(NT) k_forward(const CxConst C, const KConst<T> KC, const FwdArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NV = fwd_stage_values<Q>();
    T* const s0 = reinterpret_cast<T*>(smem_raw) + threadIdx.x;
    T* const s1 = s0 + NV * NT;
    typename SqAccT<T>::type acc;
    ChunkIter<NT> it(C);
    NodeIdx cur = it.valid() ? it.node(C) : no_node();
    allow_next_grid();
    wait_prior_grid(); // the previous step's populations and node state are complete
    if (it.valid()) fwd_stage<T, Q, NT, FwdArgs<T>>(C, A, cur, s0);
    cp_async_commit();
    bool odd = false;
    while (it.valid()) {
        it.next();
        const NodeIdx nxt = it.valid() ? it.node(C) : no_node();
        if (it.valid()) fwd_stage<T, Q, NT, FwdArgs<T>>(C, A, nxt, odd ? s0 : s1);
        cp_async_commit();
        cp_async_wait<1>(); // this thread's copies for the current node have landed
        fwd_compute<T, Q, NT, FwdArgs<T>>(C, KC, A, cur, ThreadSlots<T, NT>{odd ? s1 : s0}, acc);
        cur = nxt;
        odd = !odd;
    }
    cp_async_wait<0>();
    if (A.gsq_part) acc.flush(A.gsq_part + blockIdx.x * (NT >> 5) + (threadIdx.x >> 5), nullptr);
}

template <typename T, int Q, int NT>
static cudaError_t launch_qn(const CxConst& C, const KConst<T>& K, const FwdArgs<T>& A, const Launch& L,
                             cudaStream_t s) {
    const size_t smem = (size_t)2 * fwd_stage_values<Q>() * NT * sizeof(T);
    static bool attr_set = false; // the attribute belongs to the function, once per process
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(k_forward<T, Q, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
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
    return cudaLaunchKernelEx(&cfg, k_forward<T, Q, NT>, C, K, A);
}

template <typename T, int Q>
static cudaError_t launch_q(const CxConst& C, const KConst<T>& K, const FwdArgs<T>& A, const Launch& L,
                            cudaStream_t s) {
    switch (L.block.x) {
    case 64: return launch_qn<T, Q, 64>(C, K, A, L, s);
    case 128: return launch_qn<T, Q, 128>(C, K, A, L, s);
    case 256: return launch_qn<T, Q, 256>(C, K, A, L, s);
    default: return cudaErrorInvalidConfiguration;
    }
}

// Bulk copies of one row segment's stage (issued by one thread): the 2Q
// population windows, the angle (rotated tensors), g and E (whole-grid
// control), Phi^{n-1} and, on grids with solid nodes, the bounce-back flags
// (one byte per node).
template <typename T, int Q, int NT>
__device__ __forceinline__ void fwd_issue_rows(const CxConst& C, const FwdArgs<T>& A, int y, int x0, T* st,
                                               uint64_t* bar) {
    using L = Lat<Q>;
    using RW = RowWindow<T, Q, NT>;
    const int nx = C.nx, nv = min(NT, nx - x0);
    const int rm = y == 0 ? C.ny - 1 : y - 1, rp = y == C.ny - 1 ? 0 : y + 1;
    const bool rot = C.aniso == CX_ANISO_ROTATED, gb = A.g && C.ctrl_full, eb = A.E && C.ctrl_full;
    const uint32_t nb = (uint32_t)nv * sizeof(T);
    mbar_expect_tx(bar, (uint32_t)(2 * Q * (nv + 2 * RW::H)) * sizeof(T) + nb * (1u + rot + gb + eb) +
                            (C.has_solid ? (uint32_t)nv : 0u) + A.tx_pad);
#pragma unroll
    for (int j = 0; j < 2 * Q; ++j) {
        const int i = j < Q ? j : j - Q;
        const int ys = L::ey(i) > 0 ? rm : (L::ey(i) < 0 ? rp : y); // pull from x - e_i
        bulk_row_window<T, NT>(st + j * RW::W, A.in(j) + (size_t)ys * nx, x0, nv, nx, bar);
    }
    T* const loc = st + 2 * Q * RW::W;
    const size_t k0 = (size_t)y * nx + x0;
    if (rot) bulk_g2s(loc, reinterpret_cast<const T*>(C.theta) + k0, nb, bar);
    if (gb) bulk_g2s(loc + NT, A.g + k0, nb, bar);
    if (eb) bulk_g2s(loc + 2 * NT, A.E + k0, nb, bar);
    bulk_g2s(loc + 3 * NT, A.phi + k0, nb, bar);
    if (C.has_solid) bulk_g2s(loc + 4 * NT, C.bounce + k0, (uint32_t)nv, bar);
}

// g and E of a controlled node when the control window is not the whole grid:
// per-thread copies into the node's own slots.
template <typename T, int Q, int NT>
__device__ __forceinline__ void fwd_stage_ctrl(const CxConst& C, const FwdArgs<T>& A, const NodeIdx& nd, T* st) {
    using RW = RowWindow<T, Q, NT>;
    if (C.ctrl_full || !nd.ctrl) return;
    T* const loc = st + 2 * Q * RW::W + threadIdx.x;
    if (A.g) cp_async(loc + NT, A.g + nd.c);
    if (A.E) cp_async(loc + 2 * NT, A.E + nd.c);
}

template <typename T, int Q, int NT> constexpr int fwd_rows_stage_values() {
    return 2 * Q * RowWindow<T, Q, NT>::W + 4 * NT + NT / (int)sizeof(T); // + one flag byte per node
}
template <typename T, int Q, int NT> constexpr size_t fwd_rows_smem() {
    return rows_pipe_smem<T>(fwd_rows_stage_values<T, Q, NT>());
}

// SB: the grid has solid nodes (bounce-back flags staged with each segment).
// Block: NT compute threads and one producer warp (see cx_rows.cuh).
template <typename T, int Q, int NT, bool SB>
__global__ void __launch_bounds__(NT + 32, sizeof(T) == 4 ? (NT == 256 ? 3 : 5) : 1)
    k_forward_rows(const CxConst C, const KConst<T> KC, const FwdArgs<T> A) {
    using RW = RowWindow<T, Q, NT>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RowsPipe<T, NT> pipe(smem_raw, fwd_rows_stage_values<T, Q, NT>());
    pipe.init();
    allow_next_grid();
    wait_prior_grid(); // the previous step's populations and node state are complete
    if (block_sees_timeout(A.status)) return;
    if (threadIdx.x >= NT) {
        pipe.produce(C, A.status,
                     [&](int y, int x0, T* st, uint64_t* bar) { fwd_issue_rows<T, Q, NT>(C, A, y, x0, st, bar); });
        return;
    }
    typename SqAccT<T>::type acc;
    pipe.consume(
        C, A.status, [&](const NodeIdx& nd, T* st) { fwd_stage_ctrl<T, Q, NT>(C, A, nd, st); },
        [&](const NodeIdx& nd, T* st) {
            if constexpr (SB) {
                const unsigned bits = reinterpret_cast<const uint8_t*>(st + 2 * Q * RW::W + 4 * NT)[threadIdx.x];
                fwd_compute<T, Q, NT, FwdArgs<T>>(C, KC, A, nd, RowWindowSolid<T, Q, NT>{{st + threadIdx.x}, bits},
                                                  acc);
            } else {
                fwd_compute<T, Q, NT, FwdArgs<T>>(C, KC, A, nd, RW{st + threadIdx.x}, acc);
            }
        });
    if (A.gsq_part) acc.flush(A.gsq_part + blockIdx.x * (NT >> 5) + (threadIdx.x >> 5), nullptr);
}

// a step the row-window kernel can take: pulled populations (n >= 1), rows a
// whole number of 16-byte units (of flag bytes too when there are solid
// nodes), 16-byte aligned planes
template <typename T> static bool rows_eligible(const CxConst& C, const FwdArgs<T>& A, const Launch& L) {
    constexpr int H = 16 / (int)sizeof(T);
    auto al = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
    if (!L.row_windows || A.n == 0 || C.nx % H != 0 || !al(A.phi)) return false;
    if (C.has_solid && (!C.bounce || C.nx % 16 != 0 || !al(C.bounce))) return false;
    if (!rows_pipelined(C, L, L.rows_grid ? std::min(L.rows_grid, L.grid.x) : L.grid.x)) return false;
    if (L.block.x != 128 && L.block.x != 256) return false;
    for (int j = 0; j < 2 * C.Q; ++j)
        if (!al(A.pin[j])) return false;
    if (C.aniso == CX_ANISO_ROTATED && !al(C.theta)) return false;
    if (C.ctrl_full && ((A.g && !al(A.g)) || (A.E && !al(A.E)))) return false;
    return true;
}

template <typename T, int Q, int NT, bool SB>
static cudaError_t launch_rows_qn(const CxConst& C, const KConst<T>& K, const FwdArgs<T>& A, const Launch& L,
                                  cudaStream_t s) {
    constexpr size_t smem = fwd_rows_smem<T, Q, NT>();
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(k_forward_rows<T, Q, NT, SB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(L.rows_grid ? std::min(L.rows_grid, L.grid.x) : L.grid.x);
    cfg.blockDim = dim3(L.block.x + 32); // compute threads + the producer warp
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    FwdArgs<T> A2 = A;
    A2.tx_pad = L.row_windows == 2 ? 16u : 0u; // test mode: no stage ever completes
    return cudaLaunchKernelEx(&cfg, k_forward_rows<T, Q, NT, SB>, C, K, A2);
}

template <typename T, int Q>
static cudaError_t launch_rows_q(const CxConst& C, const KConst<T>& K, const FwdArgs<T>& A, const Launch& L,
                                 cudaStream_t s) {
    if (C.has_solid)
        return L.block.x == 128 ? launch_rows_qn<T, Q, 128, true>(C, K, A, L, s)
                                : launch_rows_qn<T, Q, 256, true>(C, K, A, L, s);
    return L.block.x == 128 ? launch_rows_qn<T, Q, 128, false>(C, K, A, L, s)
                            : launch_rows_qn<T, Q, 256, false>(C, K, A, L, s);
}

template <typename T>
cudaError_t launch_forward(const CxConst& C, const KConst<T>& K, const FwdArgs<T>& A, const Launch& L,
                           cudaStream_t s) {
    if (rows_eligible<T>(C, A, L))
        return C.Q == 9 ? launch_rows_q<T, 9>(C, K, A, L, s) : launch_rows_q<T, 5>(C, K, A, L, s);
    return C.Q == 9 ? launch_q<T, 9>(C, K, A, L, s) : launch_q<T, 5>(C, K, A, L, s);
}

template cudaError_t launch_forward<float>(const CxConst&, const KConst<float>&, const FwdArgs<float>&, const Launch&,
                                           cudaStream_t);
template cudaError_t launch_forward<double>(const CxConst&, const KConst<double>&, const FwdArgs<double>&,
                                            const Launch&, cudaStream_t);

template <typename T, int Q, int NT> static int occ_qn() {
    cudaFuncSetAttribute(k_forward<T, Q, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    int nb = 0;
    const size_t smem = (size_t)2 * fwd_stage_values<Q>() * NT * sizeof(T);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_forward<T, Q, NT>, NT, smem) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}
template <typename T, int Q> static int occ_q(int threads) {
    return threads == 64 ? occ_qn<T, Q, 64>() : (threads == 128 ? occ_qn<T, Q, 128>() : occ_qn<T, Q, 256>());
}

// resident blocks per SM of the persistent kernel for a block size
template <typename T> int forward_occupancy(int Q, int threads) {
    return Q == 9 ? occ_q<T, 9>(threads) : occ_q<T, 5>(threads);
}
template int forward_occupancy<float>(int, int);
template int forward_occupancy<double>(int, int);


template <typename T, int Q, int NT, bool SB> static int rows_occ_qnb() {
    constexpr size_t smem = fwd_rows_smem<T, Q, NT>();
    cudaFuncSetAttribute(k_forward_rows<T, Q, NT, SB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_forward_rows<T, Q, NT, SB>, NT + 32, smem) !=
        cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}
// the smaller residency of the two forms (the persistent grid serves both)
template <typename T, int Q, int NT> static int rows_occ_qn() {
    return std::min(rows_occ_qnb<T, Q, NT, false>(), rows_occ_qnb<T, Q, NT, true>());
}
template <typename T, int Q> static int rows_occ_q(int threads) {
    return threads == 128 ? rows_occ_qn<T, Q, 128>() : rows_occ_qn<T, Q, 256>();
}
// resident blocks per SM of the row-window kernel (128 or 256 threads)
template <typename T> int forward_rows_occupancy(int Q, int threads) {
    return Q == 9 ? rows_occ_q<T, 9>(threads) : rows_occ_q<T, 5>(threads);
}
template int forward_rows_occupancy<float>(int, int);
template int forward_rows_occupancy<double>(int, int);

} // namespace cx
