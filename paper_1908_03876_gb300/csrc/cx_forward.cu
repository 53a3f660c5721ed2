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
#include "cx_fwd_body.cuh"

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
        fwd_compute<T, Q, NT, FwdArgs<T>>(C, KC, A, cur, odd ? s1 : s0, acc);
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

template <typename T>
cudaError_t launch_forward(const CxConst& C, const KConst<T>& K, const FwdArgs<T>& A, const Launch& L,
                           cudaStream_t s) {
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

} // namespace cx
