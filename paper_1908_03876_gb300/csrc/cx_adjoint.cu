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
//
// Execution: the persistent, two-stage cp.async pipeline of the forward
// kernel (see cx_forward.cu), staging the pulled adjoint populations, the tape,
// sigma^{n+1}, g^n and the angle of the next node while the current one runs.
// Interior steps (not the terminal one) of grids without solid nodes use the
// row-window kernel k_adjoint_rows instead: bulk copies of the pulled
// population windows (rows y + e_y,i, widened by 16 bytes per side) and of the
// node-local planes per row segment, completed on an mbarrier per stage, as in
// k_forward_rows.
#include <algorithm>

#include "cx_adj_body.cuh"
#include "cx_rows.cuh"

namespace cx {

// BB: the grid's solid nodes carry bounce-back copies (C.bb_copy), which the
// kernel writes; a separate instantiation keeps the other grids' code as it is.
template <typename T, int Q, int NT, bool BB>
__global__ void __launch_bounds__(NT) k_adjoint(const CxConst C, const KConst<T> KC, const AdjArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NV = adj_stage_values<Q>();
    T* const s0 = reinterpret_cast<T*>(smem_raw) + threadIdx.x;
    T* const s1 = s0 + NV * NT;
    typename SqAccT<T>::type acc;
    ChunkIter<NT> it(C);
    NodeIdx cur = it.valid() ? it.node(C) : no_node();
    allow_next_grid();
    wait_prior_grid(); // the previous step's populations and node state are complete
    if (it.valid()) adj_stage<T, Q, NT, AdjArgs<T>>(C, A, cur, s0);
    cp_async_commit();
    bool odd = false;
    while (it.valid()) {
        it.next();
        const NodeIdx nxt = it.valid() ? it.node(C) : no_node();
        if (it.valid()) adj_stage<T, Q, NT, AdjArgs<T>>(C, A, nxt, odd ? s0 : s1);
        cp_async_commit();
        cp_async_wait<1>();
        adj_compute<T, Q, NT, AdjArgs<T>>(C, KC, A, cur, ThreadSlots<T, NT, BB>{odd ? s1 : s0}, acc);
        cur = nxt;
        odd = !odd;
    }
    cp_async_wait<0>();
    const int w = blockIdx.x * (NT >> 5) + (threadIdx.x >> 5);
    acc.flush(A.e2_part + w, A.emax_part + w);
}

template <typename T, int Q, int NT, bool BB>
static cudaError_t launch_qnb(const CxConst& C, const KConst<T>& K, const AdjArgs<T>& A, const Launch& L,
                              cudaStream_t s) {
    const size_t smem = (size_t)2 * adj_stage_values<Q>() * NT * sizeof(T);
    static bool attr_set = false; // the attribute belongs to the function, once per process
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(k_adjoint<T, Q, NT, BB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024);
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
    return cudaLaunchKernelEx(&cfg, k_adjoint<T, Q, NT, BB>, C, K, A);
}
template <typename T, int Q, int NT>
static cudaError_t launch_qn(const CxConst& C, const KConst<T>& K, const AdjArgs<T>& A, const Launch& L,
                             cudaStream_t s) {
    return C.bb_copy ? launch_qnb<T, Q, NT, true>(C, K, A, L, s) : launch_qnb<T, Q, NT, false>(C, K, A, L, s);
}

template <typename T, int Q>
static cudaError_t launch_q(const CxConst& C, const KConst<T>& K, const AdjArgs<T>& A, const Launch& L,
                            cudaStream_t s) {
    switch (L.block.x) {
    case 64: return launch_qn<T, Q, 64>(C, K, A, L, s);
    case 128: return launch_qn<T, Q, 128>(C, K, A, L, s);
    case 256: return launch_qn<T, Q, 256>(C, K, A, L, s);
    default: return cudaErrorInvalidConfiguration;
    }
}

// Bulk copies of one row segment's stage (issued by one thread): the 2Q
// windows of psi^{n+1}, the tape (u, G_x, G_y), sigma^{n+1}, g (whole-grid
// control), the angle (rotated tensors) and, on grids with solid nodes, the
// bounce-back flags (one byte per node).
template <typename T, int Q, int NT>
__device__ __forceinline__ void adj_issue_rows(const CxConst& C, const AdjArgs<T>& A, int y, int x0, T* st,
                                               uint64_t* bar) {
    using L = Lat<Q>;
    using RW = RowWindow<T, Q, NT>;
    const int nx = C.nx, nv = min(NT, nx - x0);
    const int rm = y == 0 ? C.ny - 1 : y - 1, rp = y == C.ny - 1 ? 0 : y + 1;
    const bool rot = C.aniso == CX_ANISO_ROTATED, gb = A.g && C.ctrl_full;
    const uint32_t nb = (uint32_t)nv * sizeof(T);
    mbar_expect_tx(bar, (uint32_t)(2 * Q * (nv + 2 * RW::H)) * sizeof(T) + nb * (4u + gb + rot) +
                            (C.has_solid ? (uint32_t)nv : 0u) + A.tx_pad);
#pragma unroll
    for (int j = 0; j < 2 * Q; ++j) {
        const int i = j < Q ? j : j - Q;
        const int ys = L::ey(i) > 0 ? rp : (L::ey(i) < 0 ? rm : y); // pull from x + e_i
        bulk_row_window<T, NT>(st + j * RW::W, A.in(j) + (size_t)ys * nx, x0, nv, nx, bar);
    }
    T* const loc = st + 2 * Q * RW::W;
    const size_t k0 = (size_t)y * nx + x0, pl = (size_t)C.plane;
    bulk_g2s(loc, A.tape + k0, nb, bar);
    bulk_g2s(loc + NT, A.tape + pl + k0, nb, bar);
    bulk_g2s(loc + 2 * NT, A.tape + 2 * pl + k0, nb, bar);
    bulk_g2s(loc + 3 * NT, A.sigma + k0, nb, bar);
    if (gb) bulk_g2s(loc + 4 * NT, A.g + k0, nb, bar);
    if (rot) bulk_g2s(loc + 5 * NT, reinterpret_cast<const T*>(C.theta) + k0, nb, bar);
    if (C.has_solid) bulk_g2s(loc + 6 * NT, C.bounce + k0, (uint32_t)nv, bar);
}

// g of a controlled node when the control window is not the whole grid
template <typename T, int Q, int NT>
__device__ __forceinline__ void adj_stage_ctrl(const CxConst& C, const AdjArgs<T>& A, const NodeIdx& nd, T* st) {
    using RW = RowWindow<T, Q, NT>;
    if (C.ctrl_full || !nd.ctrl || !A.g) return;
    cp_async(st + 2 * Q * RW::W + 4 * NT + threadIdx.x, A.g + nd.c);
}

template <typename T, int Q, int NT> constexpr int adj_rows_stage_values() {
    return 2 * Q * RowWindow<T, Q, NT>::W + 6 * NT + NT / (int)sizeof(T); // + one flag byte per node
}
template <typename T, int Q, int NT> constexpr size_t adj_rows_smem() {
    return rows_pipe_smem<T>(adj_rows_stage_values<T, Q, NT>());
}

// SB: 0 no solid nodes; 1 solid nodes, bounced pulls read from global memory;
// 2 solid nodes carrying bounce-back copies (C.bb_copy), so every pull reads
// the windows.  With solid nodes the bounce-back flags are staged with each
// segment.
// Block: NT compute threads and one producer warp (see cx_rows.cuh).
template <typename T, int Q, int NT, int SB>
__global__ void __launch_bounds__(NT + 32, sizeof(T) == 4 ? (NT == 256 ? 3 : 5) : 1)
    k_adjoint_rows(const CxConst C, const KConst<T> KC, const AdjArgs<T> A) {
    using RW = RowWindow<T, Q, NT>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RowsPipe<T, NT> pipe(smem_raw, adj_rows_stage_values<T, Q, NT>());
    pipe.init();
    allow_next_grid();
    wait_prior_grid(); // the previous step's populations and node state are complete
    if (block_sees_timeout(A.status)) return;
    if (threadIdx.x >= NT) {
        pipe.produce(C, A.status,
                     [&](int y, int x0, T* st, uint64_t* bar) { adj_issue_rows<T, Q, NT>(C, A, y, x0, st, bar); });
        return;
    }
    typename SqAccT<T>::type acc;
    pipe.consume(
        C, A.status, [&](const NodeIdx& nd, T* st) { adj_stage_ctrl<T, Q, NT>(C, A, nd, st); },
        [&](const NodeIdx& nd, T* st) {
            if constexpr (SB > 0) {
                const unsigned bits = reinterpret_cast<const uint8_t*>(st + 2 * Q * RW::W + 6 * NT)[threadIdx.x];
                adj_compute<T, Q, NT, AdjArgs<T>>(C, KC, A, nd, RowWindowSolid<T, Q, NT, SB == 2>{{st + threadIdx.x}, bits},
                                                  acc);
            } else {
                adj_compute<T, Q, NT, AdjArgs<T>>(C, KC, A, nd, RW{st + threadIdx.x}, acc);
            }
        });
    const int w = blockIdx.x * (NT >> 5) + (threadIdx.x >> 5);
    acc.flush(A.e2_part + w, A.emax_part + w);
}

// an interior step the row-window kernel can take (see k_forward_rows)
template <typename T> static bool rows_eligible(const CxConst& C, const AdjArgs<T>& A, const Launch& L) {
    constexpr int H = 16 / (int)sizeof(T);
    auto al = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
    if (!L.row_windows || A.terminal || C.nx % H != 0) return false;
    if (C.has_solid && (!C.bounce || C.nx % 16 != 0 || !al(C.bounce))) return false;
    if (!rows_pipelined(C, L, L.rows_grid ? std::min(L.rows_grid, L.grid.x) : L.grid.x)) return false;
    if (L.block.x != 128 && L.block.x != 256) return false;
    for (int j = 0; j < 2 * C.Q; ++j)
        if (!al(A.rin[j])) return false;
    if (!al(A.tape) || !al(A.sigma) || (C.plane * (long long)sizeof(T)) % 16 != 0) return false;
    if (C.aniso == CX_ANISO_ROTATED && !al(C.theta)) return false;
    if (C.ctrl_full && A.g && !al(A.g)) return false;
    return true;
}

template <typename T, int Q, int NT, int SB>
static cudaError_t launch_rows_qn(const CxConst& C, const KConst<T>& K, const AdjArgs<T>& A, const Launch& L,
                                  cudaStream_t s) {
    constexpr size_t smem = adj_rows_smem<T, Q, NT>();
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(k_adjoint_rows<T, Q, NT, SB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
    AdjArgs<T> A2 = A;
    A2.tx_pad = L.row_windows == 2 ? 16u : 0u; // test mode: no stage ever completes
    return cudaLaunchKernelEx(&cfg, k_adjoint_rows<T, Q, NT, SB>, C, K, A2);
}

template <typename T, int Q>
static cudaError_t launch_rows_q(const CxConst& C, const KConst<T>& K, const AdjArgs<T>& A, const Launch& L,
                                 cudaStream_t s) {
    if (C.has_solid && C.bb_copy)
        return L.block.x == 128 ? launch_rows_qn<T, Q, 128, 2>(C, K, A, L, s)
                                : launch_rows_qn<T, Q, 256, 2>(C, K, A, L, s);
    if (C.has_solid)
        return L.block.x == 128 ? launch_rows_qn<T, Q, 128, 1>(C, K, A, L, s)
                                : launch_rows_qn<T, Q, 256, 1>(C, K, A, L, s);
    return L.block.x == 128 ? launch_rows_qn<T, Q, 128, 0>(C, K, A, L, s)
                            : launch_rows_qn<T, Q, 256, 0>(C, K, A, L, s);
}

template <typename T>
cudaError_t launch_adjoint(const CxConst& C, const KConst<T>& K, const AdjArgs<T>& A, const Launch& L,
                           cudaStream_t s) {
    if (rows_eligible<T>(C, A, L))
        return C.Q == 9 ? launch_rows_q<T, 9>(C, K, A, L, s) : launch_rows_q<T, 5>(C, K, A, L, s);
    return C.Q == 9 ? launch_q<T, 9>(C, K, A, L, s) : launch_q<T, 5>(C, K, A, L, s);
}

template cudaError_t launch_adjoint<float>(const CxConst&, const KConst<float>&, const AdjArgs<float>&,
                                           const Launch&, cudaStream_t);
template cudaError_t launch_adjoint<double>(const CxConst&, const KConst<double>&, const AdjArgs<double>&,
                                            const Launch&, cudaStream_t);

template <typename T, int Q, int NT, bool BB> static int occ_qnb() {
    cudaFuncSetAttribute(k_adjoint<T, Q, NT, BB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024);
    int nb = 0;
    const size_t smem = (size_t)2 * adj_stage_values<Q>() * NT * sizeof(T);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adjoint<T, Q, NT, BB>, NT, smem) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}
template <typename T, int Q, int NT> static int occ_qn(bool bb) {
    return bb ? occ_qnb<T, Q, NT, true>() : occ_qnb<T, Q, NT, false>();
}
template <typename T, int Q> static int occ_q(int threads, bool bb) {
    return threads == 64 ? occ_qn<T, Q, 64>(bb) : (threads == 128 ? occ_qn<T, Q, 128>(bb) : occ_qn<T, Q, 256>(bb));
}

template <typename T> int adjoint_occupancy(int Q, int threads, bool bb) {
    return Q == 9 ? occ_q<T, 9>(threads, bb) : occ_q<T, 5>(threads, bb);
}
template int adjoint_occupancy<float>(int, int, bool);
template int adjoint_occupancy<double>(int, int, bool);

template <typename T, int Q, int NT, int SB> static int rows_occ_qnb() {
    constexpr size_t smem = adj_rows_smem<T, Q, NT>();
    cudaFuncSetAttribute(k_adjoint_rows<T, Q, NT, SB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adjoint_rows<T, Q, NT, SB>, NT + 32, smem) !=
        cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}
// the smallest residency of the three forms (the persistent grid serves all)
template <typename T, int Q, int NT> static int rows_occ_qn() {
    return std::min(rows_occ_qnb<T, Q, NT, 0>(), std::min(rows_occ_qnb<T, Q, NT, 1>(), rows_occ_qnb<T, Q, NT, 2>()));
}
template <typename T, int Q> static int rows_occ_q(int threads) {
    return threads == 128 ? rows_occ_qn<T, Q, 128>() : rows_occ_qn<T, Q, 256>();
}
// resident blocks per SM of the row-window kernel (128 or 256 threads)
template <typename T> int adjoint_rows_occupancy(int Q, int threads) {
    return Q == 9 ? rows_occ_q<T, 9>(threads) : rows_occ_q<T, 5>(threads);
}
template int adjoint_rows_occupancy<float>(int, int);
template int adjoint_rows_occupancy<double>(int, int);

} // namespace cx
