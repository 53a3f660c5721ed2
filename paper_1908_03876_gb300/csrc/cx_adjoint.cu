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
#include "cx_adj_body.cuh"

namespace cx {

template <typename T, int Q, int NT>
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
        adj_compute<T, Q, NT, AdjArgs<T>>(C, KC, A, cur, odd ? s1 : s0, acc);
        cur = nxt;
        odd = !odd;
    }
    cp_async_wait<0>();
    const int w = blockIdx.x * (NT >> 5) + (threadIdx.x >> 5);
    acc.flush(A.e2_part + w, A.emax_part + w);
}

template <typename T, int Q, int NT>
static cudaError_t launch_qn(const CxConst& C, const KConst<T>& K, const AdjArgs<T>& A, const Launch& L,
                             cudaStream_t s) {
    const size_t smem = (size_t)2 * adj_stage_values<Q>() * NT * sizeof(T);
    static bool attr_set = false; // the attribute belongs to the function, once per process
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(k_adjoint<T, Q, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024);
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
    return cudaLaunchKernelEx(&cfg, k_adjoint<T, Q, NT>, C, K, A);
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

template <typename T>
cudaError_t launch_adjoint(const CxConst& C, const KConst<T>& K, const AdjArgs<T>& A, const Launch& L,
                           cudaStream_t s) {
    return C.Q == 9 ? launch_q<T, 9>(C, K, A, L, s) : launch_q<T, 5>(C, K, A, L, s);
}

template cudaError_t launch_adjoint<float>(const CxConst&, const KConst<float>&, const AdjArgs<float>&,
                                           const Launch&, cudaStream_t);
template cudaError_t launch_adjoint<double>(const CxConst&, const KConst<double>&, const AdjArgs<double>&,
                                            const Launch&, cudaStream_t);

template <typename T, int Q, int NT> static int occ_qn() {
    cudaFuncSetAttribute(k_adjoint<T, Q, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024);
    int nb = 0;
    const size_t smem = (size_t)2 * adj_stage_values<Q>() * NT * sizeof(T);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adjoint<T, Q, NT>, NT, smem) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}
template <typename T, int Q> static int occ_q(int threads) {
    return threads == 64 ? occ_qn<T, Q, 64>() : (threads == 128 ? occ_qn<T, Q, 128>() : occ_qn<T, Q, 256>());
}

template <typename T> int adjoint_occupancy(int Q, int threads) {
    return Q == 9 ? occ_q<T, 9>(threads) : occ_q<T, 5>(threads);
}
template int adjoint_occupancy<float>(int, int);
template int adjoint_occupancy<double>(int, int);

} // namespace cx
