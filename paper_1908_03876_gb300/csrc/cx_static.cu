// cx_static.cu -- cx_forward_static: the forward solve and cost of
// cx_forward without any device allocation, for callers that cannot call
// cudaMalloc (or own no allocator at all): code running inside a host
// callback or a plug-in of another runtime, processes whose device memory is
// reserved up front by a pool they do not control, or code that must not
// touch the allocator while another library holds it.
//
// All scratch memory of the call lives in one file-scope __device__ array of
// CX_STATIC_SCRATCH_BYTES (declared in include/cxlbm.h), which every GPU that
// loads the library holds until the process exits.  Host code cannot use the
// array's name as a device address, so every call looks the address up with
// cudaGetSymbolAddress (with the caller's device current; the lookup
// allocates nothing) and passes it to the kernels.  Nothing is cached, so a
// cudaDeviceReset between calls (which reloads the module) is harmless.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "cx_internal.h"

using namespace cx;

static __device__ __align__(256) unsigned char cx_static_scratch[CX_STATIC_SCRATCH_BYTES];

namespace {

inline size_t up256(size_t v) { return (v + 255) / 256 * 256; }

struct StaticLayout {
    size_t plane, nctrl, esz, total;
    int nparts;
    size_t off_P0, off_PA, off_PB, off_phi, off_uN, off_vN, off_wu, off_theta, off_K, off_a, off_ut, off_solid,
        off_bounce, off_cmask, off_part, off_scal, off_status;
};

StaticLayout static_layout(const cx_problem_desc* d) {
    StaticLayout L{};
    L.esz = d->precision == 64 ? 8 : 4;
    L.plane = (size_t)d->nx * d->ny;
    L.plane = (L.plane + 63) / 64 * 64;
    const int cnx = d->ctrl_nx > 0 ? d->ctrl_nx : d->nx, cny = d->ctrl_nx > 0 ? d->ctrl_ny : d->ny;
    L.nctrl = (size_t)cnx * cny;
    L.nparts = std::max(((d->nx + 31) / 32) * d->ny, 32768);
    const size_t pop = (size_t)2 * d->lattice * L.plane * L.esz, fld = L.plane * L.esz;
    size_t o = 0;
    auto take = [&](size_t b) {
        size_t r = o;
        o = up256(o + b);
        return r;
    };
    L.off_P0 = take(pop);
    L.off_PA = take(pop);
    L.off_PB = take(pop);
    L.off_phi = take(fld);
    L.off_uN = take(fld);
    L.off_vN = take(fld);
    L.off_wu = take(fld);
    L.off_theta = take(d->aniso == CX_ANISO_ROTATED ? fld : 0);
    L.off_K = take(d->aniso == CX_ANISO_FIELD ? 6 * fld : 0);
    L.off_a = take(d->adv == CX_ADV_FIELD ? 2 * fld : (d->adv == CX_ADV_ROW ? 2 * (size_t)d->ny * L.esz : 0));
    L.off_ut = take(fld);
    L.off_solid = take(d->solid ? L.plane : 0);
    L.off_bounce = take(d->solid ? L.plane : 0);
    L.off_cmask = take((d->solid || d->ctrl_mask) ? L.nctrl : 0);
    L.off_part = take(sizeof(double) * 2 * (size_t)L.nparts);
    L.off_scal = take(sizeof(double) * 16);
    L.off_status = take(sizeof(int) * 4);
    L.total = o;
    return L;
}

bool K_of(const double D[3], double dd, double tau, double K[3]) {
    const double sc = 1.0 / (dd * (1.0 / 3.0) * tau);
    const double a = D[0] * sc + 0.5, b = D[1] * sc, c = D[2] * sc + 0.5;
    const double det = a * c - b * b;
    if (!(det > 0.0)) return false;
    K[0] = c / det;
    K[1] = -b / det;
    K[2] = a / det;
    const double tr = K[0] + K[2], dt = K[0] * K[2] - K[1] * K[1];
    const double disc = std::sqrt(std::max(0.0, tr * tr / 4 - dt));
    return tr / 2 - disc > 0.0 && tr / 2 + disc < 2.0;
}

bool k_of(double lam, double dd, double tau, double* k) {
    *k = 1.0 / (lam / (dd * (1.0 / 3.0) * tau) + 0.5);
    return lam >= 0.0 && *k > 0.0 && *k < 2.0;
}

// The call's outcome as a cx_status code, from the status word the kernels set:
// a bounded wait of a row-window kernel that ran out, or a non-finite cost.
__global__ void k_status_code(const int* bits, int* out) {
    const int b = *bits;
    *out = (b & ST_TIMEOUT) ? (int)CX_ERR_TIMEOUT : ((b & ST_UNSTABLE) ? (int)CX_ERR_UNSTABLE : (int)CX_OK);
}

template <typename T>
cx_status run_static(const cx_problem_desc* d, const CxConst& C, const StaticLayout& Ly, char* ws, const T* u0,
                     const T* v0, const T* g, double* J_dev, T* uN, T* vN, int* status_dev, cudaStream_t s) {
    int nsm = 1, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CX_ERR_CUDA;
    // launch shapes as cx_create chooses them
    Launch L2;
    const int bx = d->nx >= 128 ? 128 : (d->nx >= 64 ? 64 : 32);
    L2.block = dim3(bx, 256 / bx);
    L2.grid = dim3((d->nx + bx - 1) / bx, (d->ny + 256 / bx - 1) / (256 / bx));
    const int nb2 = (int)(L2.grid.x * L2.grid.y);
    Launch Lf;
    const int nseg = (d->nx + 255) / 256;
    long long nb = (long long)nsm * forward_occupancy<T>(d->lattice, 256);
    nb = std::max(1LL, std::min(nb, (long long)nseg * d->ny));
    Lf.block = dim3(256);
    Lf.grid = dim3((unsigned)nb);
    Lf.rows_grid = (unsigned)std::min<long long>(nb, (long long)nsm * forward_rows_occupancy<T>(d->lattice, 256));
    const int fw = (int)(nb * 8);
    const KConst<T> K = make_kconst<T>(C, C.Q);

    T* P0 = reinterpret_cast<T*>(ws + Ly.off_P0);
    double* cost = reinterpret_cast<double*>(ws + Ly.off_part);
    double* gsq = cost + Ly.nparts;
    double* scal = reinterpret_cast<double*>(ws + Ly.off_scal);
    int* status = reinterpret_cast<int*>(ws + Ly.off_status);
    // the array keeps the previous call's contents: clear what accumulates
    if (cudaMemsetAsync(gsq, 0, sizeof(double) * fw, s) != cudaSuccess) return CX_ERR_CUDA;
    if (cudaMemsetAsync(status, 0, sizeof(int) * 4, s) != cudaSuccess) return CX_ERR_CUDA;
    if (launch_setup_fields<T>(C, *d, (T*)C.theta, (T*)C.Kfield, (T*)C.a, reinterpret_cast<T*>(ws + Ly.off_ut),
                               (uint8_t*)C.solid, (uint8_t*)C.cmask, (uint8_t*)C.bounce, s) != cudaSuccess)
        return CX_ERR_CUDA;
    if (launch_init<T>(C, nullptr, nullptr, u0, v0, P0, L2, s) != cudaSuccess) return CX_ERR_CUDA;
    const T* in = P0;
    const int win_len = d->ctrl_windows > 0 ? d->n_steps / d->ctrl_windows : 1;
    for (int n = 0; n < d->n_steps; ++n) {
        FwdArgs<T> A{};
        A.status = status;
        T* out = reinterpret_cast<T*>(ws + ((n % 2) ? Ly.off_PB : Ly.off_PA));
        for (int j = 0; j < 18; ++j) {
            A.pin[j] = j < 2 * C.Q ? in + (size_t)j * Ly.plane : nullptr;
            A.pout[j] = j < 2 * C.Q ? out + (size_t)j * Ly.plane : nullptr;
        }
        A.phi = reinterpret_cast<T*>(ws + Ly.off_phi);
        A.phi_ckpt = nullptr;
        A.g = g ? g + (size_t)(n / win_len) * Ly.nctrl : nullptr;
        A.E = nullptr;
        A.lam = T(0);
        A.tape = nullptr;
        A.gsq_part = gsq;
        A.n = n;
        if (launch_forward<T>(C, K, A, Lf, s) != cudaSuccess) return CX_ERR_CUDA;
        in = out;
    }
    T* uN_ws = reinterpret_cast<T*>(ws + Ly.off_uN);
    T* vN_ws = reinterpret_cast<T*>(ws + Ly.off_vN);
    if (launch_final<T>(C, in, reinterpret_cast<T*>(ws + Ly.off_ut), uN_ws, vN_ws,
                        reinterpret_cast<T*>(ws + Ly.off_wu), cost, L2, s) != cudaSuccess)
        return CX_ERR_CUDA;
    if (launch_finalize(cost, nb2, gsq, fw, C.alpha, scal, status, ST_UNSTABLE, 0, s) != cudaSuccess)
        return CX_ERR_CUDA;
    if (status_dev) {
        k_status_code<<<1, 1, 0, s>>>(status, status_dev);
        if (cudaGetLastError() != cudaSuccess) return CX_ERR_CUDA;
    }
    const size_t bytes = (size_t)d->nx * d->ny * sizeof(T);
    if (J_dev && cudaMemcpyAsync(J_dev, scal, sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return CX_ERR_CUDA;
    if (uN && cudaMemcpyAsync(uN, uN_ws, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return CX_ERR_CUDA;
    if (vN && cudaMemcpyAsync(vN, vN_ws, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return CX_ERR_CUDA;
    return CX_OK;
}

} // namespace

extern "C" cx_status cx_forward_static(const cx_problem_desc* desc, const void* u0, const void* v0, const void* g,
                                       double* J_dev, void* uN, void* vN, int* status_dev, cudaStream_t stream) {
    size_t check = 0;
    cx_status rc = cx_workspace_size(desc, &check); // same descriptor validation as cx_create
    if (rc) return rc;
    if (!u0 || !v0 || desc->halo) return CX_ERR_INVALID_ARG;
    const StaticLayout Ly = static_layout(desc);
    if (Ly.total > (size_t)CX_STATIC_SCRATCH_BYTES) return CX_ERR_WORKSPACE; // problem too large for the array
    // the array's device address on the current device (looked up on every call)
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, cx_static_scratch) != cudaSuccess || !ptr) return CX_ERR_CUDA;
    char* ws = static_cast<char*>(ptr);

    CxConst C{};
    C.nx = desc->nx;
    C.ny = desc->ny;
    C.plane = (long long)Ly.plane;
    C.Q = desc->lattice;
    C.n_steps = desc->n_steps;
    C.aniso = desc->aniso;
    C.adv = desc->adv;
    C.has_solid = desc->solid ? 1 : 0;
    C.ctrl_full = (desc->ctrl_nx == 0 || (desc->ctrl_x0 == 0 && desc->ctrl_y0 == 0 && desc->ctrl_nx == desc->nx &&
                                          desc->ctrl_ny == desc->ny)) &&
                  !desc->ctrl_mask && !desc->solid;
    if (desc->ctrl_nx > 0) {
        C.cx0 = desc->ctrl_x0;
        C.cy0 = desc->ctrl_y0;
        C.cnx = desc->ctrl_nx;
        C.cny = desc->ctrl_ny;
    } else {
        C.cnx = desc->nx;
        C.cny = desc->ny;
    }
    C.source_order = desc->source_order;
    C.tau = desc->tau;
    C.d_u = desc->d_u;
    C.d_v = desc->d_v;
    C.chi = desc->chi;
    C.r_vu = desc->r_vu;
    C.r_vv = desc->r_vv;
    C.alpha = desc->alpha;
    for (int i = 0; i < 7; ++i) C.s[i] = desc->s[i];
    if (desc->aniso == CX_ANISO_CONST) {
        if (!K_of(desc->D_u, desc->d_u, desc->tau, C.Ku) || !K_of(desc->D_v, desc->d_v, desc->tau, C.Kv))
            return CX_ERR_INVALID_ARG;
    } else if (desc->aniso == CX_ANISO_ROTATED) {
        double k1, k2;
        if (!k_of(desc->lam_u[0], desc->d_u, desc->tau, &k1) || !k_of(desc->lam_u[1], desc->d_u, desc->tau, &k2))
            return CX_ERR_INVALID_ARG;
        C.ku_bar = 0.5 * (k1 + k2);
        C.ku_d = 0.5 * (k1 - k2);
        if (!k_of(desc->lam_v[0], desc->d_v, desc->tau, &k1) || !k_of(desc->lam_v[1], desc->d_v, desc->tau, &k2))
            return CX_ERR_INVALID_ARG;
        C.kv_bar = 0.5 * (k1 + k2);
        C.kv_d = 0.5 * (k1 - k2);
    }
    C.theta = desc->aniso == CX_ANISO_ROTATED ? ws + Ly.off_theta : nullptr;
    C.Kfield = desc->aniso == CX_ANISO_FIELD ? ws + Ly.off_K : nullptr;
    C.a = desc->adv != CX_ADV_NONE ? ws + Ly.off_a : nullptr;
    C.solid = desc->solid ? reinterpret_cast<uint8_t*>(ws + Ly.off_solid) : nullptr;
    C.bounce = desc->solid ? reinterpret_cast<uint8_t*>(ws + Ly.off_bounce) : nullptr;
    C.cmask = (desc->solid || desc->ctrl_mask) ? reinterpret_cast<uint8_t*>(ws + Ly.off_cmask) : nullptr;
    if (desc->precision == 64)
        return run_static<double>(desc, C, Ly, ws, (const double*)u0, (const double*)v0, (const double*)g, J_dev,
                                  (double*)uN, (double*)vN, status_dev, stream);
    return run_static<float>(desc, C, Ly, ws, (const float*)u0, (const float*)v0, (const float*)g, J_dev,
                             (float*)uN, (float*)vN, status_dev, stream);
}
