// cx_state.h -- host-side state of one problem (layout of its workspace,
// launch shapes, schedule flags); shared by the single-problem and batched
// host code.
#pragma once

#include <cstddef>
#include <vector>

#include "cx_internal.h"

namespace cx {

constexpr size_t ALIGN = 256;
constexpr int MAX_WARPS = 32768; // warps of a persistent launch (partial-sum slots)
inline size_t up(size_t v, size_t a) { return (v + a - 1) / a * a; }

enum { PH_FWD = 0, PH_REC = 1, PH_ADJ = 2, PH_OTHER = 3 };

struct Layout {
    size_t plane, nctrl, esz;
    int Q, N, k, S, nparts;
    int nwin, win_len;   // control windows W and steps per window N / W
    size_t off_popA, off_popB, off_adjA, off_adjB, off_ckpt, off_ckpt_phi, off_phi, off_sigma, off_tape;
    size_t off_uN, off_vN, off_wu, off_theta, off_K, off_a, off_ut, off_solid, off_bounce, off_cmask, off_part,
        off_scal, off_status, off_tlm, total; // off_tlm: 4 planes for the tangent-linear pass (zero, du, dv, scratch)
};

struct TimedRange {
    int phase;
    long long launches;
    cudaEvent_t a, b;
};

Layout make_layout(const cx_problem_desc* d);

} // namespace cx

struct cx_problem {
    cx_problem_desc d;
    cx::CxConst C;
    cx::Layout lay;
    cudaStream_t stream;
    char* ws;
    cx::KConst<float> Kf;
    cx::KConst<double> Kd;
    const cx::KConst<float>& kc(float*) const { return Kf; }
    const cx::KConst<double>& kc(double*) const { return Kd; }
    cx::Launch L;      // 2D launch of the set-up, initial and final kernels
    cx::Launch Lf, La; // persistent launches of the forward and adjoint kernels
    int nblocks;       // blocks of L
    int nsm = 1;
    bool has_init = false, fwd_valid = false, adj_valid = false;
    bool tape_last_valid = false; // tape holds the last segment (written by the forward)
    bool have_lam = false;
    double lam_prev = 0.0;
    // nonlinear CG state (cx_cg_step): iteration, cost, <G,G>, <G,D>, the
    // previous <G,D> and step, and which work slot holds the current gradient
    int cg_k = -1;
    double cg_J = 0.0, cg_gg = 0.0, cg_gd = 0.0, cg_gd_prev = 0.0, cg_lam = 0.0, cg_ginf = 0.0;
    int cg_slot = 0;
    void* psi0 = nullptr;
    bool timing = false;
    std::vector<cx::TimedRange> ranges;
    // cx_gradient_host: copy streams (created on first use) and per-chunk
    // events ([0, n) control chunk landed, [n, 2n) gradient chunk final, 2n
    // the call's start; n = io_nch chunks of io_cw windows); while
    // io_cw > 0 the forward waits for each chunk's event before the chunk's
    // first step, and the adjoint queues each gradient chunk's read-back to
    // io_E_host once the chunk is final
    cudaStream_t io_h2d = nullptr, io_d2h = nullptr;
    std::vector<cudaEvent_t> io_ev;
    int io_cw = 0, io_nch = 0;
    void* io_E_host = nullptr;
    cx_halo_fn halo_fn = nullptr; // sub-domain: fills the halo frame after every lattice step
    void* halo_user = nullptr;
    size_t n_ranges = 0;

    template <typename P> P* at(size_t off) const { return reinterpret_cast<P*>(ws + off); }
    size_t pop_bytes() const { return (size_t)2 * lay.Q * lay.plane * lay.esz; }
    char* ckpt_slot(int s) const { return ws + lay.off_ckpt + (size_t)s * pop_bytes(); }
    char* ckpt_phi_slot(int s) const { return ws + lay.off_ckpt_phi + (size_t)s * lay.plane * lay.esz; }
    char* tape_slot(int j) const { return ws + lay.off_tape + (size_t)j * 3 * lay.plane * lay.esz; }
};
