// cx_d3q19.cu -- host side of the D3Q19 solver (include/cx3d.h): descriptor
// validation, workspace layout, the checkpoint / segment-recompute schedule of
// a gradient evaluation, FP64 reductions and the Armijo search.  The
// arithmetic is in cx_d3q19_kernels.cuh.
//
// Schedule (the discrete-adjoint algorithm of Sec. 3.2.1, as in two
// dimensions): forward n = 0..N-1 with the output of step s*k - 1 written
// straight into checkpoint slot s and the last segment writing the tape
// (u, G); adjoint segments s = S-1..0: recompute steps s*k .. s*k+k-1 from slot
// s with the tape (skipped for the last segment), then the adjoint steps of
// the segment backward in time.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/cx3d.h"
#include "cx_d3q19_kernels.cuh"

using namespace cx;
using namespace cx::d3;

namespace {

constexpr size_t AL3 = 256;
inline size_t up3(size_t v, size_t a) { return (v + a - 1) / a * a; }
constexpr int MAXW3 = 32768;

struct L3d {
    size_t plane, esz, nodes;
    int N, k, S, nparts;
    size_t off_popA, off_popB, off_adjA, off_adjB, off_ckpt, off_phi, off_sigma, off_tape, off_uN, off_vN, off_wu,
        off_K, off_a, off_ut, off_part, off_scal, off_status, total;
};

L3d layout(const cx3d_desc* d) {
    L3d L{};
    L.esz = d->precision == 64 ? 8 : 4;
    L.N = d->n_steps;
    L.k = d->ckpt_every > 0 ? std::min(d->ckpt_every, d->n_steps) : d->n_steps;
    L.S = (L.N + L.k - 1) / L.k;
    L.nodes = (size_t)d->nx * d->ny * d->nz;
    L.plane = up3(L.nodes, 64);
    L.nparts = (int)std::max<size_t>((L.nodes + 255) / 256, (size_t)MAXW3);
    const size_t fld = L.plane * L.esz, pop = 2 * Q * fld;
    size_t o = 0;
    auto take = [&](size_t b) {
        const size_t r = o;
        o = up3(o + b, AL3);
        return r;
    };
    L.off_popA = take(pop);
    L.off_popB = take(pop);
    L.off_adjA = take(pop);
    L.off_adjB = take(pop);
    L.off_ckpt = take((pop + fld) * L.S); // per slot: 38 population planes, then Phi_v
    L.off_phi = take(fld);
    L.off_sigma = take(fld);
    L.off_tape = take(4 * fld * L.k);
    L.off_uN = take(fld);
    L.off_vN = take(fld);
    L.off_wu = take(fld);
    L.off_K = take(d->aniso == CX_ANISO_FIELD ? 12 * fld : 0);
    L.off_a = take(d->adv == CX_ADV_FIELD ? 3 * fld : (d->adv == CX_ADV_ROW ? 3 * (size_t)d->ny * L.esz : 0));
    L.off_ut = take(fld);
    L.off_part = take(sizeof(double) * 4 * (size_t)L.nparts);
    L.off_scal = take(sizeof(double) * 16);
    L.off_status = take(sizeof(int) * 4);
    L.total = o;
    return L;
}

// D positive definite (leading minors): K = (D / (d Cs^2 tau) + I/2)^-1 then has its eigenvalues in (0, 2)
bool pos_def(const double D[6]) {
    const double m1 = D[0], m2 = D[0] * D[3] - D[1] * D[1];
    const double m3 = D[0] * (D[3] * D[5] - D[4] * D[4]) - D[1] * (D[1] * D[5] - D[4] * D[2]) +
                      D[2] * (D[1] * D[4] - D[3] * D[2]);
    return m1 > 0.0 && m2 > 0.0 && m3 > 0.0;
}

void K_of(const double D[6], double dd, double tau, double K[6]) {
    const double sc = 1.0 / (dd * (1.0 / 3.0) * tau);
    const double a00 = D[0] * sc + 0.5, a01 = D[1] * sc, a02 = D[2] * sc, a11 = D[3] * sc + 0.5, a12 = D[4] * sc,
                 a22 = D[5] * sc + 0.5;
    const double c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11;
    const double det = a00 * c00 + a01 * c01 + a02 * c02;
    K[0] = c00 / det;
    K[1] = c01 / det;
    K[2] = c02 / det;
    K[3] = (a00 * a22 - a02 * a02) / det;
    K[4] = (a01 * a02 - a00 * a12) / det;
    K[5] = (a00 * a11 - a01 * a01) / det;
}

cx_status validate(const cx3d_desc* d) {
    if (!d) return CX_ERR_INVALID_ARG;
    if (d->nx < 3 || d->ny < 3 || d->nz < 3 || d->n_steps < 1) return CX_ERR_INVALID_ARG;
    if ((long long)d->nx * d->ny * d->nz > (1LL << 31) - 1) return CX_ERR_INVALID_ARG;
    if (d->precision != 32 && d->precision != 64) return CX_ERR_INVALID_ARG;
    if (d->ckpt_every < 0) return CX_ERR_INVALID_ARG;
    if (!(d->tau > 0.0) || !(d->d_u > 0.0) || !(d->d_v > 0.0) || !(d->alpha >= 0.0)) return CX_ERR_INVALID_ARG;
    if (!std::isfinite(d->chi) || !std::isfinite(d->r_vu) || !std::isfinite(d->r_vv)) return CX_ERR_INVALID_ARG;
    for (int i = 0; i < 7; ++i)
        if (!(d->s[i] > 0.0 && d->s[i] < 2.0)) return CX_ERR_INVALID_ARG;
    if (d->source_order != 1 && d->source_order != 2) return CX_ERR_INVALID_ARG;
    if (d->aniso != CX_ANISO_CONST && d->aniso != CX_ANISO_FIELD) return CX_ERR_INVALID_ARG;
    if (d->aniso == CX_ANISO_FIELD && (!d->D_u_field || !d->D_v_field)) return CX_ERR_INVALID_ARG;
    if (d->adv < 0 || d->adv > 2 || (d->adv != CX_ADV_NONE && !d->a)) return CX_ERR_INVALID_ARG;
    if (!d->u_target) return CX_ERR_INVALID_ARG;
    return CX_OK;
}

template <typename T> K3<T> make_k(const cx3d_desc& d) {
    K3<T> K{};
    for (int k = 0; k < Q; ++k) {
        const int r = rate_index(k);
        K.sn[k] = r >= 0 ? T(d.s[r] * inv_n(k)) : T(0);
    }
    K.invn_j = T(inv_n(JX));
    if (d.aniso == CX_ANISO_CONST) {
        double Ku[6], Kv[6];
        K_of(d.D_u, d.d_u, d.tau, Ku);
        K_of(d.D_v, d.d_v, d.tau, Kv);
        for (int j = 0; j < 6; ++j) {
            K.Ku[j] = T(Ku[j]);
            K.Kv[j] = T(Kv[j]);
        }
    }
    K.tau = T(d.tau);
    K.inv_tau = T(1.0 / d.tau);
    K.gsc = T(-3.0 / d.d_v);
    K.asc = T(3.0 / d.d_v);
    K.d_u = T(d.d_u);
    K.d_v = T(d.d_v);
    K.chi = T(d.chi);
    K.r_vu = T(d.r_vu);
    K.r_vv = T(d.r_vv);
    K.two_alpha = T(2.0 * d.alpha);
    K.c_first = T(d.tau);
    K.c_now = T(d.source_order == 1 ? d.tau : 1.5 * d.tau);
    K.c_prev = T(d.source_order == 1 ? 0.0 : -0.5 * d.tau);
    return K;
}

struct Rng {
    int phase;
    long long launches;
    cudaEvent_t a, b;
};

} // namespace

struct cx3d_problem {
    cx3d_desc d;
    C3 C;
    L3d lay;
    cudaStream_t stream;
    char* ws;
    K3<float> Kf;
    K3<double> Kd;
    const K3<float>& kc(float*) const { return Kf; }
    const K3<double>& kc(double*) const { return Kd; }
    int grid_f = 1, grid_a = 1, nblk = 1;
    bool has_init = false, fwd_valid = false, tape_last_valid = false, have_lam = false;
    double lam_prev = 0.0;
    bool timing = false;
    std::vector<Rng> ranges;
    size_t n_ranges = 0;

    template <typename P> P* at(size_t off) const { return reinterpret_cast<P*>(ws + off); }
    size_t fld() const { return lay.plane * lay.esz; }
    char* slot(int s) const { return ws + lay.off_ckpt + (size_t)s * (2 * Q + 1) * fld(); }
    char* slot_phi(int s) const { return slot(s) + 2 * Q * fld(); }
    char* tape(int j) const { return ws + lay.off_tape + (size_t)j * 4 * fld(); }
};

#define CX3D_CUDA(x)                                                                                                 \
    do {                                                                                                             \
        if ((x) != cudaSuccess) return CX_ERR_CUDA;                                                                  \
    } while (0)

namespace {

void rbegin(cx3d_problem* p, int phase, Rng** r) {
    *r = nullptr;
    if (!p->timing) return;
    if (p->n_ranges == p->ranges.size()) {
        Rng x{};
        cudaEventCreate(&x.a);
        cudaEventCreate(&x.b);
        p->ranges.push_back(x);
    }
    Rng* q = &p->ranges[p->n_ranges++];
    q->phase = phase;
    q->launches = 0;
    cudaEventRecord(q->a, p->stream);
    *r = q;
}
void rend(cx3d_problem* p, Rng* r, long long launches) {
    if (!r) return;
    cudaEventRecord(r->b, p->stream);
    r->launches = launches;
}

template <typename T>
cx_status run_fwd(cx3d_problem* p, const T* g, const T* E, double lam, double* J_dev, bool flag_unstable) {
    const L3d& Ly = p->lay;
    const size_t nn = Ly.nodes;
    double* part = p->at<double>(Ly.off_part);
    double* gsq = part + Ly.nparts;
    const int fw = p->grid_f * 8;
    CX3D_CUDA(cudaMemsetAsync(gsq, 0, sizeof(double) * fw, p->stream));
    Rng* r;
    rbegin(p, 0, &r);
    const T* in = reinterpret_cast<const T*>(p->slot(0));
    T* phi = p->at<T>(Ly.off_phi);
    for (int n = 0; n < Ly.N; ++n) {
        const int seg = n / Ly.k;
        FArgs<T> A{};
        T* out;
        if (n + 1 < Ly.N && (n + 1) % Ly.k == 0) {
            out = reinterpret_cast<T*>(p->slot((n + 1) / Ly.k));
            A.phi_ckpt = reinterpret_cast<T*>(p->slot_phi((n + 1) / Ly.k));
        } else {
            out = p->at<T>((n % 2) ? Ly.off_popB : Ly.off_popA);
        }
        A.in = in;
        A.out = out;
        A.phi = phi;
        A.g = g ? g + (size_t)n * nn : nullptr;
        A.E = E ? E + (size_t)n * nn : nullptr;
        A.lam = T(lam);
        A.tape = (seg == Ly.S - 1) ? reinterpret_cast<T*>(p->tape(n - seg * Ly.k)) : nullptr;
        A.gsq_part = gsq;
        A.n = n;
        k3d_forward<T><<<p->grid_f, 256, 0, p->stream>>>(p->C, p->kc((T*)nullptr), A);
        CX3D_CUDA(cudaGetLastError());
        in = out;
    }
    rend(p, r, Ly.N);
    k3d_final<T><<<p->nblk, 256, 0, p->stream>>>(p->C, in, p->at<T>(Ly.off_ut), p->at<T>(Ly.off_uN),
                                                  p->at<T>(Ly.off_vN), p->at<T>(Ly.off_wu), part);
    CX3D_CUDA(cudaGetLastError());
    double* scal = p->at<double>(Ly.off_scal);
    CX3D_CUDA(launch_finalize(part, p->nblk, gsq, fw, p->d.alpha, scal, p->at<int>(Ly.off_status),
                              flag_unstable ? ST_UNSTABLE : 0, 0, p->stream));
    if (J_dev) CX3D_CUDA(cudaMemcpyAsync(J_dev, scal, sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
    p->fwd_valid = true;
    p->tape_last_valid = true;
    return CX_OK;
}

template <typename T>
cx_status run_adj(cx3d_problem* p, const T* g, const T* seed_u, const T* seed_v, bool penalty, T* dJdg) {
    const L3d& Ly = p->lay;
    const size_t nn = Ly.nodes;
    K3<T> KA = p->kc((T*)nullptr);
    if (!penalty) KA.two_alpha = T(0);
    double* part = p->at<double>(Ly.off_part);
    double* e2 = part + 2 * (size_t)Ly.nparts;
    double* emax = part + 3 * (size_t)Ly.nparts;
    CX3D_CUDA(cudaMemsetAsync(e2, 0, sizeof(double) * 2 * Ly.nparts, p->stream));
    const int aw = p->grid_a * 8;
    T* sigma = p->at<T>(Ly.off_sigma);
    T* phi = p->at<T>(Ly.off_phi);
    const bool cost_seed = !seed_u && !seed_v;
    const T* su = cost_seed ? p->at<T>(Ly.off_wu) : seed_u;
    const T* psi_in = nullptr;
    for (int s = Ly.S - 1; s >= 0; --s) {
        const int n0 = s * Ly.k, n1 = std::min(Ly.N, n0 + Ly.k);
        if (s < Ly.S - 1 || !p->tape_last_valid) {
            Rng* r;
            rbegin(p, 1, &r);
            if (s >= 1) CX3D_CUDA(cudaMemcpyAsync(phi, p->slot_phi(s), p->fld(), cudaMemcpyDeviceToDevice, p->stream));
            const T* in = reinterpret_cast<const T*>(p->slot(s));
            for (int n = n0; n < n1; ++n) {
                FArgs<T> A{};
                T* out = p->at<T>((n % 2) ? Ly.off_popB : Ly.off_popA);
                A.in = in;
                A.out = out;
                A.phi = phi;
                A.g = g ? g + (size_t)n * nn : nullptr;
                A.tape = reinterpret_cast<T*>(p->tape(n - n0));
                A.n = n;
                k3d_forward<T><<<p->grid_f, 256, 0, p->stream>>>(p->C, p->kc((T*)nullptr), A);
                CX3D_CUDA(cudaGetLastError());
                in = out;
            }
            rend(p, r, n1 - n0);
        }
        Rng* r;
        rbegin(p, 2, &r);
        for (int n = n1 - 1; n >= n0; --n) {
            AArgs<T> A{};
            A.terminal = n == Ly.N - 1;
            T* out = p->at<T>((n % 2) ? Ly.off_adjB : Ly.off_adjA);
            A.in = psi_in;
            A.seed_u = su;
            A.seed_v = seed_v;
            A.out = out;
            A.tape = reinterpret_cast<const T*>(p->tape(n - n0));
            A.sigma = sigma;
            A.g = g ? g + (size_t)n * nn : nullptr;
            A.dJdg = dJdg + (size_t)n * nn;
            A.e2_part = e2;
            A.emax_part = emax;
            A.n = n;
            k3d_adjoint<T><<<p->grid_a, 256, 0, p->stream>>>(p->C, KA, A);
            CX3D_CUDA(cudaGetLastError());
            psi_in = out;
        }
        rend(p, r, n1 - n0);
    }
    double* scal = p->at<double>(Ly.off_scal);
    CX3D_CUDA(launch_finalize(e2, aw, emax, aw, 0.0, scal + 2, p->at<int>(Ly.off_status), ST_UNSTABLE, 1, p->stream));
    if (Ly.S > 1) p->tape_last_valid = false;
    return CX_OK;
}

cx_status read4(cx3d_problem* p, double* out4, int* status) {
    double h[4];
    int st = 0;
    CX3D_CUDA(cudaMemcpyAsync(h, p->at<double>(p->lay.off_scal), sizeof(h), cudaMemcpyDeviceToHost, p->stream));
    CX3D_CUDA(cudaMemcpyAsync(&st, p->at<int>(p->lay.off_status), sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    CX3D_CUDA(cudaStreamSynchronize(p->stream));
    if (out4) std::memcpy(out4, h, sizeof(h));
    if (status) *status = st;
    return CX_OK;
}

template <typename T> cx_status run_step(cx3d_problem* p, T* g, T* E, cx_step_info* info) {
    cx_status rc;
    if (!p->fwd_valid) {
        rc = run_fwd<T>(p, g, nullptr, 0.0, nullptr, true);
        if (rc) return rc;
    }
    rc = run_adj<T>(p, g, nullptr, nullptr, true, E);
    if (rc) return rc;
    double s4[4];
    int st = 0;
    rc = read4(p, s4, &st);
    if (rc) return rc;
    if (st & ST_UNSTABLE) return CX_ERR_UNSTABLE;
    const double J0 = s4[0], e2 = s4[2], einf = s4[3];
    double lam = p->have_lam ? 2.0 * p->lam_prev : std::min(1.0, einf > 0.0 ? 1.0 / einf : 1.0);
    const size_t n = (size_t)p->lay.N * p->lay.nodes;
    for (int t = 0; t < 30; ++t) {
        rc = run_fwd<T>(p, g, E, lam, nullptr, false);
        if (rc) return rc;
        double j4[4];
        rc = read4(p, j4, nullptr);
        if (rc) return rc;
        const double Jt = j4[0];
        if (std::isfinite(Jt) && Jt <= J0 - 1e-4 * lam * e2) {
            CX3D_CUDA(launch_axpy<T>(g, E, T(lam), n, p->stream));
            p->fwd_valid = true;
            p->lam_prev = lam;
            p->have_lam = true;
            if (info) {
                info->J0 = J0;
                info->J = Jt;
                info->lam = lam;
                info->grad_sq = e2;
                info->grad_inf = einf;
                info->trials = t + 1;
            }
            return CX_OK;
        }
        lam *= 0.5;
    }
    p->fwd_valid = false;
    return CX_ERR_LINESEARCH;
}

int pgrid(const void* kern, int nsm, long long total) {
    int per = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, 0) != cudaSuccess || per < 1) per = 1;
    const long long need = (total + 255) / 256;
    long long gsz = std::min<long long>((long long)per * nsm, need);
    gsz = std::min<long long>(gsz, MAXW3 / 8);
    return (int)std::max<long long>(1, gsz);
}

} // namespace

extern "C" {

cx_status cx3d_workspace_size(const cx3d_desc* desc, size_t* bytes) {
    const cx_status v = validate(desc);
    if (v) return v;
    if (!bytes) return CX_ERR_INVALID_ARG;
    *bytes = layout(desc).total;
    return CX_OK;
}

cx_status cx3d_create(const cx3d_desc* desc, void* workspace, size_t bytes, cudaStream_t stream,
                      cx3d_problem** out) {
    const cx_status v = validate(desc);
    if (v) return v;
    if (!out || !workspace) return CX_ERR_INVALID_ARG;
    const L3d L = layout(desc);
    if (bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) % AL3) != 0) return CX_ERR_WORKSPACE;
    if (desc->aniso == CX_ANISO_CONST && (!pos_def(desc->D_u) || !pos_def(desc->D_v))) return CX_ERR_UNSTABLE;
    cx3d_problem* p = new (std::nothrow) cx3d_problem();
    if (!p) return CX_ERR_INTERNAL;
    p->d = *desc;
    p->lay = L;
    p->stream = stream;
    p->ws = static_cast<char*>(workspace);
    p->Kf = make_k<float>(*desc);
    p->Kd = make_k<double>(*desc);
    C3& C = p->C;
    C.nx = desc->nx;
    C.ny = desc->ny;
    C.nz = desc->nz;
    C.plane = (long long)L.plane;
    C.N = desc->n_steps;
    C.aniso = desc->aniso;
    C.adv = desc->adv;
    C.Kfield = desc->aniso == CX_ANISO_FIELD ? p->ws + L.off_K : nullptr;
    C.a = desc->adv != CX_ADV_NONE ? p->ws + L.off_a : nullptr;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long total = (long long)L.nodes;
    p->nblk = (int)((total + 255) / 256);
    const bool f64 = desc->precision == 64;
    p->grid_f = pgrid(f64 ? (const void*)k3d_forward<double> : (const void*)k3d_forward<float>, nsm, total);
    p->grid_a = pgrid(f64 ? (const void*)k3d_adjoint<double> : (const void*)k3d_adjoint<float>, nsm, total);
    cudaError_t e = cudaMemsetAsync(p->at<int>(L.off_status), 0, sizeof(int) * 4, stream);
    const int sb = std::min(p->nblk, nsm * 8);
    if (e == cudaSuccess) {
        if (f64)
            k3d_setup<double><<<sb, 256, 0, stream>>>(C, *desc, C.Kfield ? p->at<double>(L.off_K) : nullptr,
                                                      C.a ? p->at<double>(L.off_a) : nullptr, p->at<double>(L.off_ut),
                                                      p->at<int>(L.off_status));
        else
            k3d_setup<float><<<sb, 256, 0, stream>>>(C, *desc, C.Kfield ? p->at<float>(L.off_K) : nullptr,
                                                     C.a ? p->at<float>(L.off_a) : nullptr, p->at<float>(L.off_ut),
                                                     p->at<int>(L.off_status));
        e = cudaGetLastError();
    }
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, p->at<int>(L.off_status), sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        delete p;
        return CX_ERR_CUDA;
    }
    if (st & ST_UNSTABLE) {
        delete p;
        return CX_ERR_UNSTABLE;
    }
    p->d.D_u_field = p->d.D_v_field = p->d.a = p->d.u_target = nullptr;
    *out = p;
    return CX_OK;
}

cx_status cx3d_set_initial(cx3d_problem* p, const double* u0, const double* v0) {
    if (!p || !u0 || !v0) return CX_ERR_INVALID_ARG;
    const int sb = std::max(1, std::min(p->nblk, 152 * 8));
    if (p->lay.esz == 8)
        k3d_init<double><<<sb, 256, 0, p->stream>>>(p->C, p->Kd, u0, v0, reinterpret_cast<double*>(p->slot(0)));
    else
        k3d_init<float><<<sb, 256, 0, p->stream>>>(p->C, p->Kf, u0, v0, reinterpret_cast<float*>(p->slot(0)));
    CX3D_CUDA(cudaGetLastError());
    p->has_init = true;
    p->fwd_valid = p->tape_last_valid = p->have_lam = false;
    return CX_OK;
}

cx_status cx3d_forward(cx3d_problem* p, const void* g, double* J_dev) {
    if (!p) return CX_ERR_INVALID_ARG;
    if (!p->has_init) return CX_ERR_STATE;
    if (p->lay.esz == 8) return run_fwd<double>(p, (const double*)g, nullptr, 0.0, J_dev, true);
    return run_fwd<float>(p, (const float*)g, nullptr, 0.0, J_dev, true);
}

cx_status cx3d_adjoint(cx3d_problem* p, const void* g, const void* seed_u, const void* seed_v, int penalty,
                       void* dJdg) {
    if (!p || !dJdg) return CX_ERR_INVALID_ARG;
    if (!p->fwd_valid) return CX_ERR_STATE;
    if (p->lay.esz == 8)
        return run_adj<double>(p, (const double*)g, (const double*)seed_u, (const double*)seed_v, penalty != 0,
                               (double*)dJdg);
    return run_adj<float>(p, (const float*)g, (const float*)seed_u, (const float*)seed_v, penalty != 0, (float*)dJdg);
}

cx_status cx3d_gradient(cx3d_problem* p, const void* g, void* dJdg, double* J_dev) {
    cx_status rc = cx3d_forward(p, g, J_dev);
    if (rc) return rc;
    return cx3d_adjoint(p, g, nullptr, nullptr, 1, dJdg);
}

cx_status cx3d_step(cx3d_problem* p, void* g_inout, void* E_work, cx_step_info* info) {
    if (!p || !g_inout || !E_work) return CX_ERR_INVALID_ARG;
    if (!p->has_init) return CX_ERR_STATE;
    if (p->lay.esz == 8) return run_step<double>(p, (double*)g_inout, (double*)E_work, info);
    return run_step<float>(p, (float*)g_inout, (float*)E_work, info);
}

cx_status cx3d_get_fields(cx3d_problem* p, void* u_out, void* v_out) {
    if (!p) return CX_ERR_INVALID_ARG;
    if (!p->fwd_valid) return CX_ERR_STATE;
    const size_t n = p->lay.nodes * p->lay.esz;
    if (u_out) CX3D_CUDA(cudaMemcpyAsync(u_out, p->ws + p->lay.off_uN, n, cudaMemcpyDeviceToDevice, p->stream));
    if (v_out) CX3D_CUDA(cudaMemcpyAsync(v_out, p->ws + p->lay.off_vN, n, cudaMemcpyDeviceToDevice, p->stream));
    return CX_OK;
}

cx_status cx3d_get_norms(cx3d_problem* p, double* J, double* grad_sq, double* grad_inf) {
    if (!p) return CX_ERR_INVALID_ARG;
    double s4[4];
    int st = 0;
    const cx_status rc = read4(p, s4, &st);
    if (rc) return rc;
    if (J) *J = s4[0];
    if (grad_sq) *grad_sq = s4[2];
    if (grad_inf) *grad_inf = s4[3];
    return (st & ST_UNSTABLE) ? CX_ERR_UNSTABLE : CX_OK;
}

cx_status cx3d_set_timing(cx3d_problem* p, int enable) {
    if (!p) return CX_ERR_INVALID_ARG;
    p->timing = enable != 0;
    p->n_ranges = 0;
    return CX_OK;
}

cx_status cx3d_get_timing(cx3d_problem* p, double* ms, long long* launches) {
    if (!p || !ms || !launches) return CX_ERR_INVALID_ARG;
    CX3D_CUDA(cudaStreamSynchronize(p->stream));
    for (int i = 0; i < 3; ++i) {
        ms[i] = 0.0;
        launches[i] = 0;
    }
    for (size_t i = 0; i < p->n_ranges; ++i) {
        float t = 0.f;
        CX3D_CUDA(cudaEventElapsedTime(&t, p->ranges[i].a, p->ranges[i].b));
        ms[p->ranges[i].phase] += t;
        launches[p->ranges[i].phase] += p->ranges[i].launches;
    }
    return CX_OK;
}

cx_status cx3d_destroy(cx3d_problem* p) {
    if (!p) return CX_ERR_INVALID_ARG;
    for (auto& r : p->ranges) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    delete p;
    return CX_OK;
}

} // extern "C"
