// cx_api.cu -- host side of the C ABI declared in include/cxlbm.h.
//
// The host code only validates descriptors, lays out the caller's workspace,
// orders kernel launches on the problem's stream and reads back FP64 scalars
// where a call is documented to synchronise.  All arithmetic of the method runs
// in the kernels of cx_forward.cu, cx_adjoint.cu and cx_misc.cu.
//
// Time schedule of a gradient evaluation (discrete-adjoint algorithm, Sec. 3.2.1):
//   forward  n = 0..N-1: the output of step s*k - 1 goes straight into
//            checkpoint slot s (no extra copy), Phi^{s*k-1} into its slot; the
//            last segment writes the adjoint tape (u, G) as it goes;
//   adjoint  segments s = S-1..0: recompute steps s*k..s*k+k-1 from slot s
//            writing the tape (skipped for the last segment), then run the
//            AMRT steps of the segment backward in time.
// Storage is O(N/k) lattices plus k tape planes of 3 scalars.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "cx_state.h"

using namespace cx;

// ------------------------------------------------------------ validation

static cx_status validate(const cx_problem_desc* d) {
    if (!d) return CX_ERR_INVALID_ARG;
    if (d->nx < 3 || d->ny < 3 || d->n_steps < 1) return CX_ERR_INVALID_ARG;
    if ((long long)d->nx * d->ny > (1LL << 31) - 1) return CX_ERR_INVALID_ARG;
    if (d->lattice != 9 && d->lattice != 5) return CX_ERR_INVALID_ARG;
    if (d->precision != 32 && d->precision != 64) return CX_ERR_INVALID_ARG;
    if (d->ckpt_every < 0) return CX_ERR_INVALID_ARG;
    if (!(d->tau > 0.0) || !(d->d_u > 0.0) || !(d->d_v > 0.0) || !(d->alpha >= 0.0)) return CX_ERR_INVALID_ARG;
    if (!std::isfinite(d->chi) || !std::isfinite(d->r_vu) || !std::isfinite(d->r_vv)) return CX_ERR_INVALID_ARG;
    for (int i = 0; i < 7; ++i)
        if (!(d->s[i] > 0.0 && d->s[i] < 2.0)) return CX_ERR_INVALID_ARG;
    if (d->source_order != 1 && d->source_order != 2) return CX_ERR_INVALID_ARG;
    if (d->halo != 0 && d->halo != 1) return CX_ERR_INVALID_ARG;
    if (d->ctrl_windows < 0 || d->ctrl_windows > d->n_steps ||
        (d->ctrl_windows > 0 && d->n_steps % d->ctrl_windows != 0))
        return CX_ERR_INVALID_ARG;
    if (d->aniso == CX_ANISO_ROTATED && !d->theta) return CX_ERR_INVALID_ARG;
    if (d->aniso == CX_ANISO_FIELD && (!d->D_u_field || !d->D_v_field)) return CX_ERR_INVALID_ARG;
    if (d->aniso < 0 || d->aniso > 2 || d->adv < 0 || d->adv > 2) return CX_ERR_INVALID_ARG;
    if (d->adv != CX_ADV_NONE && !d->a) return CX_ERR_INVALID_ARG;
    if (d->lattice == 5 && d->adv != CX_ADV_NONE) return CX_ERR_INVALID_ARG; // D2Q5 lacks the a-a moments
    if (!d->u_target) return CX_ERR_INVALID_ARG;
    if (d->ctrl_nx < 0 || d->ctrl_ny < 0) return CX_ERR_INVALID_ARG;
    if (d->ctrl_nx > 0) {
        if (d->ctrl_ny <= 0 || d->ctrl_x0 < 0 || d->ctrl_y0 < 0 || d->ctrl_x0 + d->ctrl_nx > d->nx ||
            d->ctrl_y0 + d->ctrl_ny > d->ny)
            return CX_ERR_INVALID_ARG;
    }
    return CX_OK;
}

Layout cx::make_layout(const cx_problem_desc* d) {
    Layout L{};
    L.esz = d->precision == 64 ? 8 : 4;
    L.Q = d->lattice;
    L.N = d->n_steps;
    L.k = d->ckpt_every > 0 ? std::min(d->ckpt_every, d->n_steps) : d->n_steps;
    L.S = (L.N + L.k - 1) / L.k;
    L.nwin = d->ctrl_windows > 0 ? d->ctrl_windows : d->n_steps;
    L.win_len = L.N / L.nwin;
    L.plane = up((size_t)d->nx * d->ny, 64);
    const int cnx = d->ctrl_nx > 0 ? d->ctrl_nx : d->nx, cny = d->ctrl_nx > 0 ? d->ctrl_ny : d->ny;
    L.nctrl = (size_t)cnx * cny;
    // partial buffers: per-block sums of the 2D kernels (blocks of 256 threads,
    // at most (nx/32 + 1) * ny of them) or per-warp sums of the persistent ones
    L.nparts = std::max(((d->nx + 31) / 32) * d->ny, MAX_WARPS);
    const size_t pop = (size_t)2 * L.Q * L.plane * L.esz, fld = L.plane * L.esz;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o = up(o + bytes, ALIGN);
        return r;
    };
    L.off_popA = take(pop);
    L.off_popB = take(pop);
    L.off_adjA = take(pop);
    L.off_adjB = take(pop);
    L.off_ckpt = take(pop * L.S);
    L.off_ckpt_phi = take(fld * L.S);
    L.off_phi = take(fld);
    L.off_sigma = take(fld);
    L.off_tape = take(fld * 3 * L.k);
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
    L.off_part = take(sizeof(double) * 4 * (size_t)L.nparts);
    L.off_scal = take(sizeof(double) * 16);
    L.off_status = take(sizeof(int) * 4);
    L.off_tlm = take(4 * fld);
    L.total = o;
    return L;
}

// K = (D / (d Cs^2 tau) + I/2)^-1 for a constant tensor; eigenvalues checked in (0, 2).
static bool K_const(const double D[3], double dd, double tau, double K[3]) {
    const double sc = 1.0 / (dd * (1.0 / 3.0) * tau);
    const double a = D[0] * sc + 0.5, b = D[1] * sc, c = D[2] * sc + 0.5;
    const double det = a * c - b * b;
    if (!(det > 0.0)) return false;
    K[0] = c / det;
    K[1] = -b / det;
    K[2] = a / det;
    const double tr = K[0] + K[2], dt = K[0] * K[2] - K[1] * K[1];
    const double disc = std::sqrt(std::max(0.0, tr * tr / 4 - dt));
    const double e1 = tr / 2 + disc, e2 = tr / 2 - disc;
    return e2 > 0.0 && e1 < 2.0;
}

static bool k_rot(double lam, double dd, double tau, double* k) {
    *k = 1.0 / (lam / (dd * (1.0 / 3.0) * tau) + 0.5);
    return *k > 0.0 && *k < 2.0 && lam >= 0.0;
}

#define CX_CUDA(x)                                                                                                   \
    do {                                                                                                             \
        if ((x) != cudaSuccess) return CX_ERR_CUDA;                                                                  \
    } while (0)

// --------------------------------------------------------------- timing

static void range_begin(cx_problem* p, int phase, TimedRange** r) {
    *r = nullptr;
    if (!p->timing) return;
    if (p->n_ranges == p->ranges.size()) {
        TimedRange t{};
        if (cudaEventCreate(&t.a) != cudaSuccess || cudaEventCreate(&t.b) != cudaSuccess) return;
        p->ranges.push_back(t);
    }
    TimedRange* t = &p->ranges[p->n_ranges++];
    t->phase = phase;
    t->launches = 0;
    cudaEventRecord(t->a, p->stream);
    *r = t;
}
static void range_end(cx_problem* p, TimedRange* r, long long launches) {
    if (!r) return;
    r->launches = launches;
    cudaEventRecord(r->b, p->stream);
}

// ----------------------------------------------------------- templated core

// plane j of a [2][Q][plane] population buffer
template <typename T, typename P> static void set_planes(const cx_problem* p, P (&dst)[18], T* buf) {
    for (int j = 0; j < 18; ++j) dst[j] = j < 2 * p->lay.Q ? buf + (size_t)j * p->lay.plane : nullptr;
}

template <typename T> static cx_status run_forward(cx_problem* p, const T* g, const T* E, double lam, double* J_dev,
                                                  bool flag_unstable) {
    const Layout& Ly = p->lay;
    const CxConst& C = p->C;
    double* part = p->at<double>(Ly.off_part);
    double* gsq = part + Ly.nparts;
    const int fw = (int)(p->Lf.grid.x * (p->Lf.block.x / 32));
    CX_CUDA(cudaMemsetAsync(gsq, 0, sizeof(double) * fw, p->stream));
    TimedRange* r;
    range_begin(p, PH_FWD, &r);
    const T* in = reinterpret_cast<const T*>(p->ckpt_slot(0));
    T* phi = p->at<T>(Ly.off_phi);
    for (int n = 0; n < Ly.N; ++n) {
        const int seg = n / Ly.k;
        FwdArgs<T> A{};
        A.status = p->at<int>(p->lay.off_status);
        T* out;
        if (n + 1 < Ly.N && (n + 1) % Ly.k == 0) {
            out = reinterpret_cast<T*>(p->ckpt_slot((n + 1) / Ly.k));
            A.phi_ckpt = reinterpret_cast<T*>(p->ckpt_phi_slot((n + 1) / Ly.k));
        } else {
            out = p->at<T>((n % 2) ? Ly.off_popB : Ly.off_popA);
            A.phi_ckpt = nullptr;
        }
        set_planes(p, A.pin, in);
        set_planes(p, A.pout, out);
        A.phi = phi;
        A.g = g ? g + (size_t)(n / Ly.win_len) * Ly.nctrl : nullptr;
        A.E = E ? E + (size_t)(n / Ly.win_len) * Ly.nctrl : nullptr;
        A.lam = T(lam);
        A.tape = (seg == Ly.S - 1) ? reinterpret_cast<T*>(p->tape_slot(n - seg * Ly.k)) : nullptr;
        A.gsq_part = gsq;
        A.n = n;
        if (p->io_cw > 0 && n % Ly.win_len == 0 && (n / Ly.win_len) % p->io_cw == 0) // a control chunk's first step
            CX_CUDA(cudaStreamWaitEvent(p->stream, p->io_ev[(n / Ly.win_len) / p->io_cw], 0));
        CX_CUDA(launch_forward<T>(C, p->kc((T*)nullptr), A, p->Lf, p->stream));
        if (p->halo_fn) {
            const cx_status hs = p->halo_fn(p->halo_user, CX_HALO_FWD, out, p->stream);
            if (hs) return hs;
        }
        in = out;
    }
    range_end(p, r, Ly.N);
    range_begin(p, PH_OTHER, &r); // u^N, v^N, the terminal seed and the FP64 cost
    double* cost = part;
    CX_CUDA(launch_final<T>(C, in, p->at<T>(Ly.off_ut), p->at<T>(Ly.off_uN), p->at<T>(Ly.off_vN), p->at<T>(Ly.off_wu),
                            cost, p->L, p->stream));
    double* scal = p->at<double>(Ly.off_scal);
    CX_CUDA(launch_finalize(cost, p->nblocks, gsq, fw, C.alpha, scal, p->at<int>(Ly.off_status),
                            flag_unstable ? ST_UNSTABLE : 0, 0, p->stream));
    range_end(p, r, 2);
    if (p->halo_fn) { // the terminal adjoint step pulls the seed from the frame too
        const cx_status hs = p->halo_fn(p->halo_user, CX_HALO_SEED, p->at<T>(Ly.off_wu), p->stream);
        if (hs) return hs;
    }
    if (J_dev) CX_CUDA(cudaMemcpyAsync(J_dev, scal, sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
    p->fwd_valid = true;
    p->adj_valid = false;
    p->tape_last_valid = true;
    return CX_OK;
}

// penalty = false: the control-penalty term 2 alpha g^n is left out of the
// gradient, which is then the plain vector-Jacobian product of the solve.
template <typename T>
static cx_status run_adjoint(cx_problem* p, const T* g, const T* seed_u, const T* seed_v, T* dJdg,
                             bool penalty = true) {
    const Layout& Ly = p->lay;
    const CxConst& C = p->C;
    KConst<T> KA = p->kc((T*)nullptr);
    if (!penalty) KA.two_alpha = T(0);
    double* part = p->at<double>(Ly.off_part);
    double* e2 = part + 2 * (size_t)Ly.nparts;
    double* emax = part + 3 * (size_t)Ly.nparts;
    CX_CUDA(cudaMemsetAsync(e2, 0, sizeof(double) * 2 * Ly.nparts, p->stream));
    const int aw = (int)(p->La.grid.x * (p->La.block.x / 32));
    T* sigma = p->at<T>(Ly.off_sigma);
    CX_CUDA(cudaMemsetAsync(sigma, 0, Ly.plane * sizeof(T), p->stream));
    T* phi = p->at<T>(Ly.off_phi);
    const T* psi_in = nullptr;
    for (int s = Ly.S - 1; s >= 0; --s) {
        const int n0 = s * Ly.k, n1 = std::min(Ly.N, n0 + Ly.k);
        if (s < Ly.S - 1 || !p->tape_last_valid) {
            TimedRange* r;
            range_begin(p, PH_REC, &r);
            if (s >= 1)
                CX_CUDA(cudaMemcpyAsync(phi, p->ckpt_phi_slot(s), Ly.plane * sizeof(T), cudaMemcpyDeviceToDevice,
                                        p->stream));
            const T* in = reinterpret_cast<const T*>(p->ckpt_slot(s));
            for (int n = n0; n < n1; ++n) {
                FwdArgs<T> A{};
                A.status = p->at<int>(p->lay.off_status);
                T* out = p->at<T>((n % 2) ? Ly.off_popB : Ly.off_popA);
                set_planes(p, A.pin, in);
                set_planes(p, A.pout, out);
                A.phi = phi;
                A.phi_ckpt = nullptr;
                A.g = g ? g + (size_t)(n / Ly.win_len) * Ly.nctrl : nullptr;
                A.tape = reinterpret_cast<T*>(p->tape_slot(n - n0));
                A.gsq_part = nullptr;
                A.n = n;
                CX_CUDA(launch_forward<T>(C, p->kc((T*)nullptr), A, p->Lf, p->stream));
                if (p->halo_fn) {
                    const cx_status hs = p->halo_fn(p->halo_user, CX_HALO_FWD, out, p->stream);
                    if (hs) return hs;
                }
                in = out;
            }
            range_end(p, r, n1 - n0);
        }
        TimedRange* r;
        range_begin(p, PH_ADJ, &r);
        for (int n = n1 - 1; n >= n0; --n) {
            AdjArgs<T> A{};
            A.status = p->at<int>(p->lay.off_status);
            A.terminal = (n == Ly.N - 1);
            T* out = p->at<T>((n % 2) ? Ly.off_adjB : Ly.off_adjA);
            if (psi_in) set_planes(p, A.rin, psi_in);
            set_planes(p, A.rout, out);
            A.wu = seed_u ? seed_u : p->at<T>(Ly.off_wu);
            A.wv = seed_v;
            A.tape = reinterpret_cast<const T*>(p->tape_slot(n - n0));
            A.sigma = sigma;
            A.g = g ? g + (size_t)(n / Ly.win_len) * Ly.nctrl : nullptr;
            A.dJdg = dJdg + (size_t)(n / Ly.win_len) * Ly.nctrl;
            A.accum = (n % Ly.win_len) != Ly.win_len - 1; // the reverse sweep meets a window's last step first
            A.norm = (n % Ly.win_len) == 0;
            A.e2_part = e2;
            A.emax_part = emax;
            A.n = n;
            CX_CUDA(launch_adjoint<T>(C, KA, A, p->La, p->stream));
            if (p->io_cw > 0 && p->io_E_host && n % Ly.win_len == 0 && (n / Ly.win_len) % p->io_cw == 0) {
                // the chunk's lowest window is final: read the chunk back while the adjoint goes on
                const size_t w0 = (size_t)(n / Ly.win_len), w1 = std::min(w0 + (size_t)p->io_cw, (size_t)Ly.nwin);
                const size_t off = w0 * Ly.nctrl * sizeof(T), bytes = (w1 - w0) * Ly.nctrl * sizeof(T);
                cudaEvent_t ev = p->io_ev[(size_t)p->io_nch + w0 / (size_t)p->io_cw];
                CX_CUDA(cudaEventRecord(ev, p->stream));
                CX_CUDA(cudaStreamWaitEvent(p->io_d2h, ev, 0));
                CX_CUDA(cudaMemcpyAsync(static_cast<char*>(p->io_E_host) + off, reinterpret_cast<const char*>(dJdg) + off,
                                        bytes, cudaMemcpyDeviceToHost, p->io_d2h));
            }
            if (p->halo_fn && n > 0) {
                const cx_status hs = p->halo_fn(p->halo_user, CX_HALO_ADJ, out, p->stream);
                if (hs) return hs;
            }
            psi_in = out;
        }
        range_end(p, r, n1 - n0);
    }
    double* scal = p->at<double>(Ly.off_scal);
    CX_CUDA(launch_finalize(e2, aw, emax, aw, 0.0, scal + 2, p->at<int>(Ly.off_status), ST_UNSTABLE, 1,
                            p->stream));
    p->psi0 = const_cast<T*>(psi_in);
    p->adj_valid = true;
    if (Ly.S > 1) p->tape_last_valid = false; // recomputed segments overwrote the tape
    return CX_OK;
}

static cx_status read_scalars(cx_problem* p, double* out4, int* status) {
    double h[4];
    int st = 0;
    CX_CUDA(cudaMemcpyAsync(h, p->at<double>(p->lay.off_scal), sizeof(h), cudaMemcpyDeviceToHost, p->stream));
    CX_CUDA(cudaMemcpyAsync(&st, p->at<int>(p->lay.off_status), sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    CX_CUDA(cudaStreamSynchronize(p->stream));
    if (out4) std::memcpy(out4, h, sizeof(h));
    if (status) *status = st;
    return CX_OK;
}

template <typename T> static cx_status run_step(cx_problem* p, T* g, T* E, cx_step_info* info) {
    cx_status rc;
    if (!p->fwd_valid) {
        rc = run_forward<T>(p, g, nullptr, 0.0, nullptr, true);
        if (rc) return rc;
    }
    rc = run_adjoint<T>(p, g, nullptr, nullptr, E);
    if (rc) return rc;
    double s4[4];
    int st = 0;
    rc = read_scalars(p, s4, &st);
    if (rc) return rc;
    if (st & ST_TIMEOUT) return CX_ERR_TIMEOUT;
    if (st & ST_UNSTABLE) return CX_ERR_UNSTABLE;
    const double J0 = s4[0], e2 = s4[2], einf = s4[3];
    double lam = p->have_lam ? 2.0 * p->lam_prev : std::min(1.0, einf > 0.0 ? 1.0 / einf : 1.0);
    for (int t = 0; t < 30; ++t) {
        rc = run_forward<T>(p, g, E, lam, nullptr, false);
        if (rc) return rc;
        double j4[4];
        rc = read_scalars(p, j4, nullptr);
        if (rc) return rc;
        const double Jt = j4[0];
        if (std::isfinite(Jt) && Jt <= J0 - 1e-4 * lam * e2) {
            CX_CUDA(launch_axpy<T>(g, E, T(lam), (size_t)p->lay.nwin * p->lay.nctrl, p->stream));
            p->fwd_valid = true; // the accepted trial's forward state is the new control's
            p->adj_valid = false;
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

// Continuous-adjoint gradient (the adjoint PDE solved by the MRT scheme with
// time reversed): segment by segment in reverse, recompute the forward
// segment with its tape, then run the continuous-adjoint steps n = n1-1 ... n0
// on the adjoint's ping-pong lattices.  Needs the forward state of g (wu holds
// u^N - u_target).
template <typename T> static cx_status run_cadj(cx_problem* p, const T* g, T* dJdg) {
    const Layout& Ly = p->lay;
    const CxConst& C = p->C;
    double* part = p->at<double>(Ly.off_part);
    double* e2 = part + 2 * (size_t)Ly.nparts;
    double* emax = part + 3 * (size_t)Ly.nparts;
    CX_CUDA(cudaMemsetAsync(e2, 0, sizeof(double) * 2 * Ly.nparts, p->stream));
    const int aw = (int)(p->La.grid.x * (p->La.block.x / 32));
    T* phi = p->at<T>(Ly.off_phi);
    const T* in = nullptr;
    for (int s = Ly.S - 1; s >= 0; --s) {
        const int n0 = s * Ly.k, n1 = std::min(Ly.N, n0 + Ly.k);
        if (s < Ly.S - 1 || !p->tape_last_valid) {
            if (s >= 1)
                CX_CUDA(cudaMemcpyAsync(phi, p->ckpt_phi_slot(s), Ly.plane * sizeof(T), cudaMemcpyDeviceToDevice,
                                        p->stream));
            const T* fin = reinterpret_cast<const T*>(p->ckpt_slot(s));
            for (int n = n0; n < n1; ++n) {
                FwdArgs<T> A{};
                A.status = p->at<int>(p->lay.off_status);
                T* out = p->at<T>((n % 2) ? Ly.off_popB : Ly.off_popA);
                set_planes(p, A.pin, fin);
                set_planes(p, A.pout, out);
                A.phi = phi;
                A.g = g ? g + (size_t)(n / Ly.win_len) * Ly.nctrl : nullptr;
                A.tape = reinterpret_cast<T*>(p->tape_slot(n - n0));
                A.n = n;
                CX_CUDA(launch_forward<T>(C, p->kc((T*)nullptr), A, p->Lf, p->stream));
                fin = out;
            }
        }
        for (int n = n1 - 1; n >= n0; --n) {
            CadjArgs<T> A{};
            A.status = p->at<int>(p->lay.off_status);
            A.first = (n == Ly.N - 1);
            T* out = p->at<T>((n % 2) ? Ly.off_adjB : Ly.off_adjA);
            if (in) set_planes(p, A.pin, in);
            set_planes(p, A.pout, out);
            A.w0 = p->at<T>(Ly.off_wu);
            A.tape = reinterpret_cast<const T*>(p->tape_slot(n - n0));
            A.g = g ? g + (size_t)(n / Ly.win_len) * Ly.nctrl : nullptr;
            A.dJdg = dJdg + (size_t)(n / Ly.win_len) * Ly.nctrl;
            A.accum = (n % Ly.win_len) != Ly.win_len - 1;
            A.norm = (n % Ly.win_len) == 0;
            A.e2_part = e2;
            A.emax_part = emax;
            A.n = n;
            CX_CUDA(launch_cadj<T>(C, p->kc((T*)nullptr), A, p->La, p->stream));
            in = out;
        }
    }
    double* scal = p->at<double>(Ly.off_scal);
    CX_CUDA(launch_finalize(e2, aw, emax, aw, 0.0, scal + 2, p->at<int>(Ly.off_status), ST_UNSTABLE, 1,
                            p->stream));
    p->adj_valid = false; // psi^0 of the discrete adjoint is not available
    if (Ly.S > 1) p->tape_last_valid = false;
    return CX_OK;
}

// Tangent-linear (sensitivity) pass along the control direction dg about the
// base trajectory of control g (the state of the preceding forward): each
// checkpointed segment is recomputed with its tape, then the tangent steps of
// the segment run on the adjoint's ping-pong lattices (free here).  The
// tangent starts from df^0 = 0.  du_out / dv_out (may be null) receive du^N,
// dv^N; *du_sq (host, may be null) receives ||du^N||^2.
template <typename T>
static cx_status run_tlm(cx_problem* p, const T* g, const T* dg, T* du_out, T* dv_out, double* du_sq) {
    const Layout& Ly = p->lay;
    const CxConst& C = p->C;
    T* zero = p->at<T>(Ly.off_tlm);
    T* du = du_out ? du_out : zero + Ly.plane;
    T* dv = dv_out ? dv_out : zero + 2 * Ly.plane;
    T* scratch = zero + 3 * Ly.plane;
    T* dphi = p->at<T>(Ly.off_sigma);
    T* phi = p->at<T>(Ly.off_phi);
    T* dA = p->at<T>(Ly.off_adjA);
    T* dB = p->at<T>(Ly.off_adjB);
    CX_CUDA(cudaMemsetAsync(zero, 0, Ly.plane * sizeof(T), p->stream));
    CX_CUDA(cudaMemsetAsync(dA, 0, (size_t)2 * Ly.Q * Ly.plane * sizeof(T), p->stream)); // df^0 = 0
    const T* din = dA;
    for (int s = 0; s < Ly.S; ++s) {
        const int n0 = s * Ly.k, n1 = std::min(Ly.N, n0 + Ly.k);
        if (s >= 1)
            CX_CUDA(cudaMemcpyAsync(phi, p->ckpt_phi_slot(s), Ly.plane * sizeof(T), cudaMemcpyDeviceToDevice,
                                    p->stream));
        const T* in = reinterpret_cast<const T*>(p->ckpt_slot(s));
        for (int n = n0; n < n1; ++n) { // base recompute with tape
            FwdArgs<T> A{};
            A.status = p->at<int>(p->lay.off_status);
            T* out = p->at<T>((n % 2) ? Ly.off_popB : Ly.off_popA);
            set_planes(p, A.pin, in);
            set_planes(p, A.pout, out);
            A.phi = phi;
            A.g = g ? g + (size_t)(n / Ly.win_len) * Ly.nctrl : nullptr;
            A.tape = reinterpret_cast<T*>(p->tape_slot(n - n0));
            A.n = n;
            CX_CUDA(launch_forward<T>(C, p->kc((T*)nullptr), A, p->Lf, p->stream));
            in = out;
        }
        for (int n = n0; n < n1; ++n) { // tangent steps of the segment
            TlmArgs<T> A{};
            A.status = p->at<int>(p->lay.off_status);
            T* out = (din == dA) ? dB : dA;
            set_planes(p, A.pin, din);
            set_planes(p, A.pout, out);
            A.dphi = dphi;
            A.tape = reinterpret_cast<const T*>(p->tape_slot(n - n0));
            A.dg = dg ? dg + (size_t)(n / Ly.win_len) * Ly.nctrl : nullptr;
            A.n = n;
            CX_CUDA(launch_tlm<T>(C, p->kc((T*)nullptr), A, p->Lf, p->stream));
            din = out;
        }
    }
    double* part = p->at<double>(Ly.off_part);
    CX_CUDA(launch_final<T>(C, din, zero, du, dv, scratch, part, p->L, p->stream));
    double* out = p->at<double>(Ly.off_scal) + 12;
    CX_CUDA(launch_finalize(part, p->nblocks, nullptr, 0, 0.0, out, p->at<int>(Ly.off_status), ST_UNSTABLE, 0,
                            p->stream));
    p->tape_last_valid = true; // the last segment was recomputed last
    p->adj_valid = false;
    if (du_sq) {
        double h = 0.0;
        CX_CUDA(cudaMemcpyAsync(&h, out, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
        CX_CUDA(cudaStreamSynchronize(p->stream));
        *du_sq = 2.0 * h;
    }
    return CX_OK;
}

// One steepest-descent iteration with the step length of the quadratic model
// of J along -E built from the sensitivity problem (eqs. LM / LMA, Sec. 2.3):
// J(g - lam E) ~ J - lam ||E||^2 + lam^2 (||S E||^2 + 2 alpha L ||E||^2) / 2,
// minimised by lam* = ||E||^2 / (||S E||^2 + 2 alpha L ||E||^2), S E = du^N the
// tangent response to E and L the steps per control window.  The step is
// accepted under the Armijo test of cx_step (halved if it fails).
template <typename T> static cx_status run_lma_step(cx_problem* p, T* g, T* E, cx_step_info* info) {
    cx_status rc;
    if (!p->fwd_valid) {
        if ((rc = run_forward<T>(p, g, nullptr, 0.0, nullptr, true))) return rc;
    }
    if ((rc = run_adjoint<T>(p, g, nullptr, nullptr, E))) return rc;
    double s4[4];
    int st = 0;
    if ((rc = read_scalars(p, s4, &st))) return rc;
    if (st & ST_TIMEOUT) return CX_ERR_TIMEOUT;
    if (st & ST_UNSTABLE) return CX_ERR_UNSTABLE;
    const double J0 = s4[0], e2 = s4[2], einf = s4[3];
    double sesq = 0.0;
    if ((rc = run_tlm<T>(p, g, E, nullptr, nullptr, &sesq))) return rc;
    const double curv = sesq + 2.0 * p->C.alpha * p->lay.win_len * e2;
    double lam = curv > 0.0 ? e2 / curv : std::min(1.0, einf > 0.0 ? 1.0 / einf : 1.0);
    for (int t = 0; t < 30; ++t) {
        if ((rc = run_forward<T>(p, g, E, lam, nullptr, false))) return rc;
        double j4[4];
        if ((rc = read_scalars(p, j4, nullptr))) return rc;
        if (std::isfinite(j4[0]) && j4[0] <= J0 - 1e-4 * lam * e2) {
            CX_CUDA(launch_axpy<T>(g, E, T(lam), (size_t)p->lay.nwin * p->lay.nctrl, p->stream));
            p->fwd_valid = true;
            p->adj_valid = false;
            if (info) {
                info->J0 = J0;
                info->J = j4[0];
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

// Nonlinear conjugate gradients with a weak Wolfe-Powell line search (remark
// 2 after the gradient algorithm, Sec. 2.3).  The search direction is held
// negated, P = -D, so that trial controls are g - lam P as in the Armijo
// search.  work: [4][W][ctrl] = two gradient slots (current / trial), P, and
// the trial control.
template <typename T> static cx_status run_cg_step(cx_problem* p, T* g, T* work, int variant, cx_cg_info* info) {
    const size_t n = (size_t)p->lay.nwin * p->lay.nctrl;
    T* slot[2] = {work, work + n};
    T* P = work + 2 * n;
    T* gt = work + 3 * n;
    double* part = p->at<double>(p->lay.off_part);
    double* dots = p->at<double>(p->lay.off_scal) + 8;
    auto read_dots = [&](const T* x0, const T* y0, const T* x1, const T* y1, const T* x2, const T* y2, const T* x3,
                         const T* y3, double* out) -> cx_status {
        const T* const xs[4] = {x0, x1, x2, x3};
        const T* const ys[4] = {y0, y1, y2, y3};
        CX_CUDA(launch_dots<T>(xs, ys, n, part, dots, p->stream));
        CX_CUDA(cudaMemcpyAsync(out, dots, 4 * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
        CX_CUDA(cudaStreamSynchronize(p->stream));
        return CX_OK;
    };
    cx_status rc;
    double J0, gd, lam;
    if (p->cg_k < 0) {
        T* G = slot[0];
        rc = run_forward<T>(p, g, nullptr, 0.0, nullptr, true);
        if (rc) return rc;
        rc = run_adjoint<T>(p, g, nullptr, nullptr, G);
        if (rc) return rc;
        double s4[4];
        int st = 0;
        if ((rc = read_scalars(p, s4, &st))) return rc;
        if (st & ST_TIMEOUT) return CX_ERR_TIMEOUT;
        if (st & ST_UNSTABLE) return CX_ERR_UNSTABLE;
        CX_CUDA(cudaMemcpyAsync(P, G, n * sizeof(T), cudaMemcpyDeviceToDevice, p->stream));
        J0 = s4[0];
        p->cg_gg = s4[2];
        gd = -s4[2];
        lam = std::min(1.0, s4[3] > 0.0 ? 1.0 / s4[3] : 1.0);
        p->cg_ginf = s4[3];
        p->cg_slot = 0;
        p->cg_k = 0;
    } else {
        J0 = p->cg_J;
        gd = p->cg_gd;
        lam = p->cg_lam * p->cg_gd_prev / gd;
    }
    T* G = slot[p->cg_slot];
    T* Gt = slot[1 - p->cg_slot];
    const double c1 = 1e-4, c2 = 0.1;
    double lo = 0.0, hi = INFINITY, Jt = 0.0;
    int t = 0;
    bool ok = false;
    for (; t < 30; ++t) {
        CX_CUDA(launch_lincomb<T>(gt, g, T(-lam), P, n, p->stream));
        if ((rc = run_forward<T>(p, gt, nullptr, 0.0, nullptr, false))) return rc;
        double s4[4];
        if ((rc = read_scalars(p, s4, nullptr))) return rc;
        Jt = s4[0];
        if (!std::isfinite(Jt) || Jt > J0 + c1 * lam * gd) {
            hi = lam;
        } else {
            if ((rc = run_adjoint<T>(p, gt, nullptr, nullptr, Gt))) return rc;
            double d4[4];
            if ((rc = read_dots(Gt, P, Gt, P, Gt, P, Gt, P, d4))) return rc;
            const double dphi = -d4[0]; // <G(lam), D>
            if (dphi < c2 * gd) {
                lo = lam;
            } else {
                ok = true;
                break;
            }
        }
        lam = std::isfinite(hi) ? 0.5 * (lo + hi) : 2.0 * lam;
    }
    if (!ok) {
        // soft reset: steepest descent with Armijo backtracking
        double gnorm[4];
        if ((rc = read_dots(G, G, G, G, G, G, G, G, gnorm))) return rc;
        const double gg0 = gnorm[0];
        double lam2 = p->cg_ginf > 0.0 ? std::min(1.0, 1.0 / p->cg_ginf) : 1.0;
        int t2 = 0;
        bool ok2 = false;
        for (; t2 < 30; ++t2) {
            CX_CUDA(launch_lincomb<T>(gt, g, T(-lam2), G, n, p->stream));
            if ((rc = run_forward<T>(p, gt, nullptr, 0.0, nullptr, false))) return rc;
            double s4[4];
            if ((rc = read_scalars(p, s4, nullptr))) return rc;
            if (std::isfinite(s4[0]) && s4[0] <= J0 - c1 * lam2 * gg0) {
                Jt = s4[0];
                ok2 = true;
                break;
            }
            lam2 *= 0.5;
        }
        if (!ok2) {
            p->cg_k = -1;
            p->fwd_valid = false;
            return CX_ERR_LINESEARCH;
        }
        if ((rc = run_adjoint<T>(p, gt, nullptr, nullptr, Gt))) return rc;
        double s4[4];
        if ((rc = read_scalars(p, s4, nullptr))) return rc;
        CX_CUDA(cudaMemcpyAsync(P, Gt, n * sizeof(T), cudaMemcpyDeviceToDevice, p->stream));
        CX_CUDA(cudaMemcpyAsync(g, gt, n * sizeof(T), cudaMemcpyDeviceToDevice, p->stream));
        if (info) {
            info->J0 = J0;
            info->J = Jt;
            info->lam = lam2;
            info->grad_sq = s4[2];
            info->beta = 0.0;
            info->trials = 30 + t2 + 1;
            info->restarted = 1;
        }
        p->cg_J = Jt;
        p->cg_gg = s4[2];
        p->cg_ginf = s4[3];
        p->cg_gd_prev = -gg0;
        p->cg_gd = -s4[2];
        p->cg_lam = lam2;
        p->cg_slot = 1 - p->cg_slot;
        p->cg_k += 1;
        CX_CUDA(cudaStreamSynchronize(p->stream));
        return CX_OK;
    }
    {
        double s4[4];
        if ((rc = read_scalars(p, s4, nullptr))) return rc; // max |Gt| of the accepted trial's sweep
        p->cg_ginf = s4[3];
    }
    // a = <Gt,Gt>, b = <Gt,G>, c = <P,Gt>, d = <P,G>
    double q[4];
    if ((rc = read_dots(Gt, Gt, Gt, G, P, Gt, P, G, q))) return rc;
    const double a = q[0], b = q[1], c = q[2], d = q[3];
    const double dy = -(c - d); // <D, Gt - G>
    double r;
    switch (variant) {
    case CX_CG_FR: r = a / p->cg_gg; break;
    case CX_CG_PR: r = (a - b) / p->cg_gg; break;
    case CX_CG_HS: r = (a - b) / dy; break;
    default: r = a / dy; break;
    }
    double gd_new = -(a + r * c);
    const bool restart = !(gd_new < 0.0) || std::fabs(b) >= 0.2 * a;
    if (restart) {
        CX_CUDA(cudaMemcpyAsync(P, Gt, n * sizeof(T), cudaMemcpyDeviceToDevice, p->stream));
        gd_new = -a;
    } else {
        CX_CUDA(launch_lincomb<T>(P, Gt, T(r), P, n, p->stream)); // P <- Gt + r P
    }
    CX_CUDA(cudaMemcpyAsync(g, gt, n * sizeof(T), cudaMemcpyDeviceToDevice, p->stream));
    if (info) {
        info->J0 = J0;
        info->J = Jt;
        info->lam = lam;
        info->grad_sq = a;
        info->beta = r;
        info->trials = t + 1;
        info->restarted = restart ? 1 : 0;
    }
    p->cg_J = Jt;
    p->cg_gg = a;
    p->cg_gd_prev = gd;
    p->cg_gd = gd_new;
    p->cg_lam = lam;
    p->cg_slot = 1 - p->cg_slot;
    p->cg_k += 1;
    CX_CUDA(cudaStreamSynchronize(p->stream));
    return CX_OK;
}

// ------------------------------------------------------------------- C ABI

extern "C" {

cx_status cx_workspace_size(const cx_problem_desc* desc, size_t* bytes) {
    cx_status rc = validate(desc);
    if (rc) return rc;
    if (!bytes) return CX_ERR_INVALID_ARG;
    *bytes = make_layout(desc).total;
    return CX_OK;
}

static void set_2d(cx_problem* p) {
    const int bx = p->d.nx >= 128 ? 128 : (p->d.nx >= 64 ? 64 : 32);
    p->L.block = dim3(bx, 256 / bx);
    p->L.grid = dim3((p->d.nx + bx - 1) / bx, (p->d.ny + 256 / bx - 1) / (256 / bx));
    p->nblocks = (int)(p->L.grid.x * p->L.grid.y);
}

// Persistent grid: `blocks` blocks of `threads` threads (0 blocks: all SMs at
// full residency), never more blocks than row segments of work.
static cx_status set_persistent(cx_problem* p, Launch& L, int threads, int blocks, int per_sm) {
    const int nseg = (p->d.nx + threads - 1) / threads;
    const long long work = (long long)nseg * p->d.ny;
    long long nb = blocks > 0 ? blocks : (long long)p->nsm * per_sm;
    nb = std::min(nb, work);
    if (nb < 1) nb = 1;
    if (nb * (threads / 32) > MAX_WARPS) return CX_ERR_INVALID_ARG;
    L.block = dim3(threads);
    L.grid = dim3((unsigned)nb);
    return CX_OK;
}

cx_status cx_set_launch(cx_problem* p, int threads, int blocks) {
    if (!p || (threads != 64 && threads != 128 && threads != 256) || blocks < 0) return CX_ERR_INVALID_ARG;
    const bool dbl = p->lay.esz == 8;
    const bool bb = p->C.bb_copy != 0;
    const int of = dbl ? forward_occupancy<double>(p->lay.Q, threads) : forward_occupancy<float>(p->lay.Q, threads);
    const int oa = dbl ? adjoint_occupancy<double>(p->lay.Q, threads, bb) : adjoint_occupancy<float>(p->lay.Q, threads, bb);
    Launch f, a;
    cx_status rc = set_persistent(p, f, threads, blocks, of);
    if (rc) return rc;
    rc = set_persistent(p, a, threads, blocks, oa);
    if (rc) return rc;
    f.row_windows = a.row_windows = p->Lf.row_windows;
    if (blocks == 0 && threads != 64) { // the row-window kernels at their own residency
        const int rf = dbl ? forward_rows_occupancy<double>(p->lay.Q, threads)
                           : forward_rows_occupancy<float>(p->lay.Q, threads);
        const int ra = dbl ? adjoint_rows_occupancy<double>(p->lay.Q, threads)
                           : adjoint_rows_occupancy<float>(p->lay.Q, threads);
        f.rows_grid = std::min<unsigned>(f.grid.x, (unsigned)(p->nsm * rf));
        a.rows_grid = std::min<unsigned>(a.grid.x, (unsigned)(p->nsm * ra));
    }
    p->Lf = f;
    p->La = a;
    return CX_OK;
}

cx_status cx_set_staging(cx_problem* p, int row_windows) {
    if (!p || row_windows < 0 || row_windows > 2) return CX_ERR_INVALID_ARG;
    p->Lf.row_windows = p->La.row_windows = row_windows;
    return CX_OK;
}

cx_status cx_create(const cx_problem_desc* desc, void* workspace, size_t bytes, cudaStream_t stream,
                    cx_problem** out) {
    if (!out) return CX_ERR_INVALID_ARG;
    *out = nullptr;
    cx_status rc = validate(desc);
    if (rc) return rc;
    Layout Ly = make_layout(desc);
    if (!workspace || bytes < Ly.total || (reinterpret_cast<uintptr_t>(workspace) % ALIGN) != 0)
        return CX_ERR_WORKSPACE;
    CxConst C{};
    C.nx = desc->nx;
    C.ny = desc->ny;
    C.plane = (long long)Ly.plane;
    C.Q = desc->lattice;
    C.n_steps = desc->n_steps;
    C.aniso = desc->aniso;
    C.adv = desc->adv;
    C.has_solid = desc->solid ? 1 : 0;
    C.halo = desc->halo;
    C.bb_copy = (desc->solid && !desc->halo) ? 1 : 0;
    C.ctrl_full = (desc->ctrl_nx == 0 || (desc->ctrl_x0 == 0 && desc->ctrl_y0 == 0 && desc->ctrl_nx == desc->nx &&
                                          desc->ctrl_ny == desc->ny)) &&
                  !desc->ctrl_mask && !desc->solid;
    if (desc->ctrl_nx > 0) {
        C.cx0 = desc->ctrl_x0;
        C.cy0 = desc->ctrl_y0;
        C.cnx = desc->ctrl_nx;
        C.cny = desc->ctrl_ny;
    } else {
        C.cx0 = C.cy0 = 0;
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
        if (!K_const(desc->D_u, desc->d_u, desc->tau, C.Ku) || !K_const(desc->D_v, desc->d_v, desc->tau, C.Kv))
            return CX_ERR_INVALID_ARG;
    } else if (desc->aniso == CX_ANISO_ROTATED) {
        double k1, k2;
        if (!k_rot(desc->lam_u[0], desc->d_u, desc->tau, &k1) || !k_rot(desc->lam_u[1], desc->d_u, desc->tau, &k2))
            return CX_ERR_INVALID_ARG;
        C.ku_bar = 0.5 * (k1 + k2);
        C.ku_d = 0.5 * (k1 - k2);
        if (!k_rot(desc->lam_v[0], desc->d_v, desc->tau, &k1) || !k_rot(desc->lam_v[1], desc->d_v, desc->tau, &k2))
            return CX_ERR_INVALID_ARG;
        C.kv_bar = 0.5 * (k1 + k2);
        C.kv_d = 0.5 * (k1 - k2);
    }
    cx_problem* p = new (std::nothrow) cx_problem();
    if (!p) return CX_ERR_INTERNAL;
    p->d = *desc;
    p->lay = Ly;
    p->stream = stream;
    p->ws = reinterpret_cast<char*>(workspace);
    char* ws = p->ws;
    C.theta = desc->aniso == CX_ANISO_ROTATED ? ws + Ly.off_theta : nullptr;
    C.Kfield = desc->aniso == CX_ANISO_FIELD ? ws + Ly.off_K : nullptr;
    C.a = desc->adv != CX_ADV_NONE ? ws + Ly.off_a : nullptr;
    C.solid = desc->solid ? reinterpret_cast<uint8_t*>(ws + Ly.off_solid) : nullptr;
    C.bounce = desc->solid ? reinterpret_cast<uint8_t*>(ws + Ly.off_bounce) : nullptr;
    C.cmask = (desc->solid || desc->ctrl_mask) ? reinterpret_cast<uint8_t*>(ws + Ly.off_cmask) : nullptr;
    p->C = C;
    p->Kf = make_kconst<float>(C, C.Q);
    p->Kd = make_kconst<double>(C, C.Q);
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            delete p;
            return CX_ERR_CUDA;
        }
    }
    set_2d(p);
    if (cx_set_launch(p, 256, 0) != CX_OK) {
        delete p;
        return CX_ERR_INTERNAL;
    }
    cudaError_t e;
    if (desc->precision == 64)
        e = launch_setup_fields<double>(C, *desc, (double*)C.theta, (double*)C.Kfield, (double*)C.a,
                                        reinterpret_cast<double*>(ws + Ly.off_ut), (uint8_t*)C.solid,
                                        (uint8_t*)C.cmask, (uint8_t*)C.bounce, stream);
    else
        e = launch_setup_fields<float>(C, *desc, (float*)C.theta, (float*)C.Kfield, (float*)C.a,
                                       reinterpret_cast<float*>(ws + Ly.off_ut), (uint8_t*)C.solid,
                                       (uint8_t*)C.cmask, (uint8_t*)C.bounce, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws + Ly.off_status, 0, sizeof(int) * 4, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        delete p;
        return CX_ERR_CUDA;
    }
    // the descriptor's device pointers are not kept
    p->d.theta = p->d.D_u_field = p->d.D_v_field = p->d.a = p->d.u_target = nullptr;
    p->d.solid = p->d.ctrl_mask = nullptr;
    *out = p;
    return CX_OK;
}

cx_status cx_set_initial(cx_problem* p, const void* u0, const void* v0) {
    if (!p || !u0 || !v0) return CX_ERR_INVALID_ARG;
    cudaError_t e;
    if (p->lay.esz == 8)
        e = launch_init<double>(p->C, nullptr, nullptr, (const double*)u0, (const double*)v0,
                                reinterpret_cast<double*>(p->ckpt_slot(0)), p->L, p->stream);
    else
        e = launch_init<float>(p->C, nullptr, nullptr, (const float*)u0, (const float*)v0,
                               reinterpret_cast<float*>(p->ckpt_slot(0)), p->L, p->stream);
    if (e != cudaSuccess) return CX_ERR_CUDA;
    p->has_init = true;
    p->cg_k = -1;
    p->fwd_valid = p->adj_valid = false;
    p->have_lam = false;
    return CX_OK;
}

cx_status cx_forward(cx_problem* p, const void* g, double* J_dev) {
    if (!p) return CX_ERR_INVALID_ARG;
    if (!p->has_init) return CX_ERR_STATE;
    if (p->lay.esz == 8) return run_forward<double>(p, (const double*)g, nullptr, 0.0, J_dev, true);
    return run_forward<float>(p, (const float*)g, nullptr, 0.0, J_dev, true);
}

cx_status cx_adjoint(cx_problem* p, const void* g, const void* seed_u, const void* seed_v, void* dJdg) {
    if (!p || !dJdg) return CX_ERR_INVALID_ARG;
    if (!p->fwd_valid) return CX_ERR_STATE;
    if (p->lay.esz == 8)
        return run_adjoint<double>(p, (const double*)g, (const double*)seed_u, (const double*)seed_v, (double*)dJdg);
    return run_adjoint<float>(p, (const float*)g, (const float*)seed_u, (const float*)seed_v, (float*)dJdg);
}

cx_status cx_adjoint_vjp(cx_problem* p, const void* g, const void* seed_u, const void* seed_v, void* vjp) {
    if (!p || !vjp) return CX_ERR_INVALID_ARG;
    if (!p->fwd_valid) return CX_ERR_STATE;
    if (!seed_u) { // a zero seed for u^N: the first plane of the tangent-linear scratch, cleared here
        seed_u = p->ws + p->lay.off_tlm;
        CX_CUDA(cudaMemsetAsync(p->ws + p->lay.off_tlm, 0, p->lay.plane * p->lay.esz, p->stream));
    }
    if (p->lay.esz == 8)
        return run_adjoint<double>(p, (const double*)g, (const double*)seed_u, (const double*)seed_v, (double*)vjp,
                                   false);
    return run_adjoint<float>(p, (const float*)g, (const float*)seed_u, (const float*)seed_v, (float*)vjp, false);
}

cx_status cx_set_halo_exchange(cx_problem* p, cx_halo_fn fn, void* user) {
    if (!p || !p->d.halo) return CX_ERR_INVALID_ARG;
    p->halo_fn = fn;
    p->halo_user = fn ? user : nullptr;
    return CX_OK;
}

cx_status cx_forward_trial(cx_problem* p, const void* g, const void* E, double lam, double* J_dev) {
    if (!p || !E || !std::isfinite(lam)) return CX_ERR_INVALID_ARG;
    if (!p->has_init) return CX_ERR_STATE;
    if (p->lay.esz == 8) return run_forward<double>(p, (const double*)g, (const double*)E, lam, J_dev, true);
    return run_forward<float>(p, (const float*)g, (const float*)E, lam, J_dev, true);
}

cx_status cx_control_axpy(cx_problem* p, void* g, const void* E, double lam) {
    if (!p || !g || !E || !std::isfinite(lam)) return CX_ERR_INVALID_ARG;
    const size_t n = (size_t)p->lay.nwin * p->lay.nctrl;
    if (p->lay.esz == 8) CX_CUDA(launch_axpy<double>((double*)g, (const double*)E, lam, n, p->stream));
    else CX_CUDA(launch_axpy<float>((float*)g, (const float*)E, (float)lam, n, p->stream));
    return CX_OK;
}

cx_status cx_gradient(cx_problem* p, const void* g, void* dJdg, double* J_dev) {
    cx_status rc = cx_forward(p, g, J_dev);
    if (rc) return rc;
    return cx_adjoint(p, g, nullptr, nullptr, dJdg);
}

// One gradient evaluation from and to host memory.  The control arrives in
// chunks of io_cw windows on the upload stream, and the forward waits for a
// chunk only at the chunk's first step; the gradient leaves chunk by chunk on
// the read-back stream as soon as the reverse sweep has finished the chunk's
// lowest window.  So both copies overlap the kernels except the first chunk
// in and the last chunk out.
constexpr int HOST_CHUNKS = 32; // chunks per direction (the first in and the last out are not overlapped)

cx_status cx_gradient_host(cx_problem* p, const void* g_host, void* dJdg_host, double* J_host, void* g_dev,
                           void* dJdg_dev) {
    if (!p || !g_host || !dJdg_host || !g_dev || !dJdg_dev || p->d.halo) return CX_ERR_INVALID_ARG;
    if (!p->has_init) return CX_ERR_STATE;
    const Layout& Ly = p->lay;
    const int cw = std::max(1, Ly.nwin / HOST_CHUNKS);
    const int nch = (Ly.nwin + cw - 1) / cw;
    if (!p->io_h2d) {
        CX_CUDA(cudaStreamCreateWithFlags(&p->io_h2d, cudaStreamNonBlocking));
        CX_CUDA(cudaStreamCreateWithFlags(&p->io_d2h, cudaStreamNonBlocking));
    }
    while ((int)p->io_ev.size() < 2 * nch + 1) {
        cudaEvent_t e;
        CX_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        p->io_ev.push_back(e);
    }
    // the copies must not overtake work already queued on the problem's stream
    // (a previous call's kernels may still read g_dev or write dJdg_dev)
    cudaEvent_t start = p->io_ev[2 * nch];
    CX_CUDA(cudaEventRecord(start, p->stream));
    CX_CUDA(cudaStreamWaitEvent(p->io_h2d, start, 0));
    const size_t wbytes = Ly.nctrl * Ly.esz;
    for (int c = 0; c < nch; ++c) {
        const size_t w0 = (size_t)c * cw, w1 = std::min(w0 + (size_t)cw, (size_t)Ly.nwin);
        CX_CUDA(cudaMemcpyAsync(static_cast<char*>(g_dev) + w0 * wbytes, static_cast<const char*>(g_host) + w0 * wbytes,
                                (w1 - w0) * wbytes, cudaMemcpyHostToDevice, p->io_h2d));
        CX_CUDA(cudaEventRecord(p->io_ev[c], p->io_h2d));
    }
    // the read-back stream waits, per chunk, for the adjoint (queued inside)
    p->io_cw = cw;
    p->io_nch = nch;
    p->io_E_host = dJdg_host;
    cx_status rc = cx_gradient(p, g_dev, dJdg_dev, nullptr);
    p->io_cw = 0;
    p->io_E_host = nullptr;
    if (rc) {
        cudaStreamSynchronize(p->io_h2d);
        cudaStreamSynchronize(p->io_d2h);
        return rc;
    }
    double s4[4];
    int st = 0;
    rc = read_scalars(p, s4, &st);
    CX_CUDA(cudaStreamSynchronize(p->io_h2d));
    CX_CUDA(cudaStreamSynchronize(p->io_d2h));
    if (rc) return rc;
    if (J_host) *J_host = s4[0];
    if (st & ST_TIMEOUT) return CX_ERR_TIMEOUT;
    if (st & ST_UNSTABLE) return CX_ERR_UNSTABLE;
    return CX_OK;
}

cx_status cx_cg_step(cx_problem* p, void* g_inout, void* work, int variant, cx_cg_info* info) {
    if (!p || !g_inout || !work || variant < CX_CG_FR || variant > CX_CG_DY || p->d.halo) return CX_ERR_INVALID_ARG;
    if (!p->has_init) return CX_ERR_STATE;
    if (p->lay.esz == 8) return run_cg_step<double>(p, (double*)g_inout, (double*)work, variant, info);
    return run_cg_step<float>(p, (float*)g_inout, (float*)work, variant, info);
}

cx_status cx_tlm(cx_problem* p, const void* g, const void* dg, void* du_out, void* dv_out, double* du_sq) {
    if (!p || !dg || p->d.halo) return CX_ERR_INVALID_ARG;
    if (!p->fwd_valid) return CX_ERR_STATE;
    if (p->lay.esz == 8)
        return run_tlm<double>(p, (const double*)g, (const double*)dg, (double*)du_out, (double*)dv_out, du_sq);
    return run_tlm<float>(p, (const float*)g, (const float*)dg, (float*)du_out, (float*)dv_out, du_sq);
}

cx_status cx_cadjoint(cx_problem* p, const void* g, void* dJdg) {
    if (!p || !dJdg || p->d.halo) return CX_ERR_INVALID_ARG;
    if (!p->fwd_valid) return CX_ERR_STATE;
    if (p->lay.esz == 8) return run_cadj<double>(p, (const double*)g, (double*)dJdg);
    return run_cadj<float>(p, (const float*)g, (float*)dJdg);
}

cx_status cx_lma_step(cx_problem* p, void* g_inout, void* E_work, cx_step_info* info) {
    if (!p || !g_inout || !E_work || p->d.halo) return CX_ERR_INVALID_ARG;
    if (!p->has_init) return CX_ERR_STATE;
    if (p->lay.esz == 8) return run_lma_step<double>(p, (double*)g_inout, (double*)E_work, info);
    return run_lma_step<float>(p, (float*)g_inout, (float*)E_work, info);
}

cx_status cx_cg_reset(cx_problem* p) {
    if (!p) return CX_ERR_INVALID_ARG;
    p->cg_k = -1;
    return CX_OK;
}

cx_status cx_step(cx_problem* p, void* g_inout, void* E_work, cx_step_info* info) {
    if (!p || !g_inout || !E_work || p->d.halo) return CX_ERR_INVALID_ARG;
    if (!p->has_init) return CX_ERR_STATE;
    if (p->lay.esz == 8) return run_step<double>(p, (double*)g_inout, (double*)E_work, info);
    return run_step<float>(p, (float*)g_inout, (float*)E_work, info);
}

cx_status cx_get_fields(cx_problem* p, void* u_out, void* v_out) {
    if (!p) return CX_ERR_INVALID_ARG;
    if (!p->fwd_valid) return CX_ERR_STATE;
    const size_t b = (size_t)p->d.nx * p->d.ny * p->lay.esz;
    if (u_out) CX_CUDA(cudaMemcpyAsync(u_out, p->ws + p->lay.off_uN, b, cudaMemcpyDeviceToDevice, p->stream));
    if (v_out) CX_CUDA(cudaMemcpyAsync(v_out, p->ws + p->lay.off_vN, b, cudaMemcpyDeviceToDevice, p->stream));
    return CX_OK;
}

cx_status cx_get_psi0(cx_problem* p, void* out) {
    if (!p || !out) return CX_ERR_INVALID_ARG;
    if (!p->adj_valid || !p->psi0) return CX_ERR_STATE;
    const size_t nn = (size_t)p->d.nx * p->d.ny;
    // [2][Q][plane] -> [2][Q][ny][nx]
    for (int j = 0; j < 2 * p->lay.Q; ++j)
        CX_CUDA(cudaMemcpyAsync(static_cast<char*>(out) + j * nn * p->lay.esz,
                                static_cast<char*>(p->psi0) + j * p->lay.plane * p->lay.esz, nn * p->lay.esz,
                                cudaMemcpyDeviceToDevice, p->stream));
    return CX_OK;
}

cx_status cx_get_norms(cx_problem* p, double* J, double* grad_sq, double* grad_inf) {
    if (!p) return CX_ERR_INVALID_ARG;
    double s4[4];
    int st = 0;
    cx_status rc = read_scalars(p, s4, &st);
    if (rc) return rc;
    if (J) *J = s4[0];
    if (grad_sq) *grad_sq = s4[2];
    if (grad_inf) *grad_inf = s4[3];
    if (st & ST_TIMEOUT) return CX_ERR_TIMEOUT;
    if (st & ST_UNSTABLE) return CX_ERR_UNSTABLE;
    return CX_OK;
}

cx_status cx_set_timing(cx_problem* p, int enable) {
    if (!p) return CX_ERR_INVALID_ARG;
    p->timing = enable != 0;
    return CX_OK;
}

cx_status cx_get_timing(cx_problem* p, double* ms, long long* launches) {
    if (!p) return CX_ERR_INVALID_ARG;
    CX_CUDA(cudaStreamSynchronize(p->stream));
    double acc[4] = {0, 0, 0, 0};
    long long cnt[4] = {0, 0, 0, 0};
    for (size_t i = 0; i < p->n_ranges; ++i) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, p->ranges[i].a, p->ranges[i].b) != cudaSuccess) return CX_ERR_CUDA;
        acc[p->ranges[i].phase] += t;
        cnt[p->ranges[i].phase] += p->ranges[i].launches;
    }
    p->n_ranges = 0;
    if (ms) std::memcpy(ms, acc, sizeof(acc));
    if (launches) std::memcpy(launches, cnt, sizeof(cnt));
    return CX_OK;
}

cx_status cx_destroy(cx_problem* p) {
    if (!p) return CX_ERR_INVALID_ARG;
    for (auto& r : p->ranges) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : p->io_ev) cudaEventDestroy(e);
    if (p->io_h2d) cudaStreamDestroy(p->io_h2d);
    if (p->io_d2h) cudaStreamDestroy(p->io_d2h);
    delete p;
    return CX_OK;
}

const char* cx_status_string(cx_status s) {
    switch (s) {
    case CX_OK: return "ok";
    case CX_ERR_INVALID_ARG: return "invalid argument";
    case CX_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case CX_ERR_CUDA: return "CUDA runtime error";
    case CX_ERR_STATE: return "call out of order";
    case CX_ERR_UNSTABLE: return "non-finite cost or gradient";
    case CX_ERR_LINESEARCH: return "line search failed";
    case CX_ERR_TIMEOUT: return "device wait timed out";
    case CX_ERR_INTERNAL: return "internal error";
    }
    return "unknown status";
}

} // extern "C"
