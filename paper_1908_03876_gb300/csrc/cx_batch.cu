// cx_batch.cu -- many independent problems advanced together: one persistent
// launch per time step covers every problem's tiles, and the whole sequence
// of a gradient evaluation (forward, recompute, AMRT adjoint, reductions) is
// captured once as a CUDA graph and replayed.
//
// Problems share N, the checkpoint interval k, the lattice and the precision;
// sizes, tensors, chemotaxis, masks and controls differ.  Each problem keeps
// its own cx_problem workspace inside the batch workspace (same layout and
// set-up as a single problem); the batch adds a device table of per-problem
// records, the tile prefix array and per-tile FP64 reduction slots.
//
// Work decomposition: problem p is cut into tiles of TX_p x (NT / TX_p) nodes
// (TX_p per problem, chosen by the autotuner); tiles of all problems form one
// list; block b of the persistent grid takes tiles b, b + G, ...; the tile's
// problem is found by binary search in the prefix array held in shared
// memory.  Per node the arithmetic is the single-problem kernels' (the same
// stage/compute bodies); the current problem's descriptor and constants sit
// in a per-warp shared-memory slot, its argument block in registers, both
// refreshed only when the problem changes.  Reductions go to one slot per
// (tile, warp), summed per problem in a fixed order, so replays are bitwise
// reproducible.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "cx_adj_body.cuh"
#include "cx_fwd_body.cuh"
#include "cx_state.h"

namespace cx {

enum { ROLE_POPA = 0, ROLE_POPB = 1, ROLE_CKPT = 2, ROLE_ADJA = 3, ROLE_ADJB = 4 };

template <typename T> struct BRec {
    CxConst C;
    KConst<T> K;
    T* pop[5];       // base of popA, popB, checkpoint 0, adjA, adjB ([2][Q][plane] each)
    T* ckpt_phi;     // [S][plane]
    T* phi;
    T* sigma;
    T* tape;         // [k][3][plane]
    T* wu;
    const T* g;      // [N][nctrl] or null
    T* dJdg;         // [N][nctrl] or null
    long long plane, nctrl, pop_elems;
    int win_len;     // steps per control window (1: one control per step)
    int nwin;        // control windows
    int tile0;       // first global tile of this problem
    int tx, ty;      // threads of a block as tx x ty (tx * ty = NT)
    int tx_shift;    // log2 tx
    int rr;          // rows per thread: a tile is tx x (ty rr) nodes
    int tiles_x;
    int slot0;       // first reduction slot
};

struct BStep {
    int n;
    int in_role, in_slot;
    int out_role, out_slot;
    int phi_ckpt_slot; // -1: none
    int tape_slot;     // -1: none
    int want_sum;      // accumulate the sum of squares (g for the forward, E for the adjoint)
    int terminal;
    int trial;         // forward at the line-search trial g - lam_p dJ/dg (per-problem lam_p)
};

template <typename T> __device__ __forceinline__ T* role_ptr(const BRec<T>& R, int role, int slot) {
    return role == ROLE_CKPT ? R.pop[2] + (size_t)slot * R.pop_elems : R.pop[role];
}

template <typename T> struct BFwdArgs {
    const T* inb;
    T* outb;
    long long pl;
    T* phi;
    T* phi_ckpt;
    const T* g;
    const T* E;
    T lam;
    T* tape;
    int n;
    __device__ __forceinline__ const T* in(int j) const { return inb + (size_t)j * pl; }
    __device__ __forceinline__ T* out(int j) const { return outb + (size_t)j * pl; }
};

template <typename T> struct BAdjArgs {
    const T* rinb;
    T* routb;
    long long pl;
    const T* wu;
    const T* wv;
    const T* tape;
    T* sigma;
    const T* g;
    T* dJdg;
    int n;
    int terminal;
    int accum;
    int norm;
    __device__ __forceinline__ const T* in(int j) const { return rinb + (size_t)j * pl; }
    __device__ __forceinline__ T* out(int j) const { return routb + (size_t)j * pl; }
};

template <typename T>
__device__ __forceinline__ BFwdArgs<T> fwd_args(const BRec<T>& R, const BStep& st, const T* lam, int p) {
    BFwdArgs<T> A;
    A.inb = role_ptr(R, st.in_role, st.in_slot);
    A.outb = role_ptr(R, st.out_role, st.out_slot);
    A.pl = R.plane;
    A.phi = R.phi;
    A.phi_ckpt = st.phi_ckpt_slot >= 0 ? R.ckpt_phi + (size_t)st.phi_ckpt_slot * R.plane : nullptr;
    const size_t w = (size_t)(st.n / R.win_len) * R.nctrl;
    A.g = R.g ? R.g + w : nullptr;
    A.E = st.trial ? R.dJdg + w : nullptr;
    A.lam = st.trial ? lam[p] : T(0);
    A.tape = st.tape_slot >= 0 ? R.tape + (size_t)st.tape_slot * 3 * R.plane : nullptr;
    A.n = st.n;
    return A;
}

template <typename T> __device__ __forceinline__ BAdjArgs<T> adj_args(const BRec<T>& R, const BStep& st) {
    BAdjArgs<T> A;
    A.rinb = role_ptr(R, st.in_role, st.in_slot);
    A.routb = role_ptr(R, st.out_role, st.out_slot);
    A.pl = R.plane;
    A.wu = R.wu;
    A.wv = nullptr;
    A.tape = R.tape + (size_t)st.tape_slot * 3 * R.plane;
    A.sigma = R.sigma;
    const size_t w = (size_t)(st.n / R.win_len) * R.nctrl;
    A.g = R.g ? R.g + w : nullptr;
    A.dJdg = R.dJdg + w;
    A.n = st.n;
    A.terminal = st.terminal;
    A.accum = (st.n % R.win_len) != R.win_len - 1;
    A.norm = (st.n % R.win_len) == 0;
    return A;
}

// problem owning global tile t (tile0 ascending, sh[count] = total)
__device__ __forceinline__ int find_problem(const int* sh, int count, int t) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sh[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// this thread's first node (row step 0) of tile `local` of problem R
template <typename T> __device__ __forceinline__ void tile_origin(const BRec<T>& R, int local, int& x, int& y) {
    const int tyi = local / R.tiles_x, txi = local - tyi * R.tiles_x;
    x = txi * R.tx + ((int)threadIdx.x & (R.tx - 1));
    y = tyi * R.ty * R.rr + ((int)threadIdx.x >> R.tx_shift);
}

template <typename T> __device__ __forceinline__ NodeIdx node_at(const BRec<T>& R, int x, int y);
__device__ __forceinline__ NodeIdx node_at_c(const CxConst& C, int x, int y);
template <typename T> __device__ __forceinline__ NodeIdx node_at(const BRec<T>& R, int x, int y) {
    return node_at_c(R.C, x, y);
}
__device__ __forceinline__ NodeIdx node_at_c(const CxConst& C, int x, int y) {
    NodeIdx r;
    r.x = x;
    r.y = y;
    const bool in = r.x < C.nx && r.y < C.ny;
    r.k = in ? r.y * C.nx + r.x : 0;
    r.fluid = in && !(C.has_solid && C.solid[r.k]);
    if (!in) {
        r.c = -1;
    } else if (C.ctrl_full) {
        r.c = r.k;
    } else {
        const int cx = r.x - C.cx0, cy = r.y - C.cy0;
        r.c = (cx >= 0 && cy >= 0 && cx < C.cnx && cy < C.cny) ? cy * C.cnx + cx : -1;
    }
    r.ctrl = r.fluid && r.c >= 0 && (!C.cmask || C.cmask[r.c]);
    return r;
}

template <typename T, int Q, int NT, bool ADJ>
__global__ void __launch_bounds__(NT) k_batch(const BRec<T>* __restrict__ recs, const int* __restrict__ tile0, int count,
                                              int total, BStep st, double* sum_slots, double* max_slots,
                                              const int* __restrict__ active, const T* __restrict__ lam) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NV = ADJ ? 2 * Q + 6 : 2 * Q + 4;
    int* sh_tile0 = reinterpret_cast<int*>(smem_raw + (size_t)2 * NV * NT * sizeof(T));
    for (int i = threadIdx.x; i <= count; i += NT) sh_tile0[i] = tile0[i];
    __syncthreads();
    T* const s0 = reinterpret_cast<T*>(smem_raw) + threadIdx.x;
    T* const s1 = s0 + NV * NT;
    allow_next_grid();
    wait_prior_grid();

    // this block's tiles are blockIdx.x, blockIdx.x + G, ...; tiles of
    // problems switched off in `active` are skipped (a whole problem at once)
    const int G = gridDim.x;
    auto next_live = [&](int tt, int& q) -> int {
        while (tt < total) {
            q = find_problem(sh_tile0, count, tt);
            if (__ldg(active + q)) return tt;
            tt += ((sh_tile0[q + 1] - tt + G - 1) / G) * G;
        }
        return total;
    };
    // Work items are (tile, row step j < rr): the thread updates node
    // (x, y + j ty) of the tile; the next item is staged while the current
    // one is computed.  Cost / gradient partials accumulate over a run of
    // consecutive items of one problem and are flushed into the slot of the
    // run's first tile (the runs are the same at every launch, so the sums
    // are reproducible).
    // the argument block depends only on the problem (the step is the launch's):
    // built once per change of problem and carried from staging to compute
    using Args = std::conditional_t<ADJ, BAdjArgs<T>, BFwdArgs<T>>;
    auto make_args = [&](int q) -> Args {
        if constexpr (ADJ)
            return adj_args(recs[q], st);
        else
            return fwd_args(recs[q], st, lam, q);
    };
    // The current problem's descriptor and constants in a per-warp
    // shared-memory slot (two slots: the next problem's are loaded while the
    // current one's are in use), read at shared-memory latency by the node
    // indexing, the staging and the per-node arithmetic.
    struct ProbConst {
        CxConst C;
        KConst<T> K;
    };
    __shared__ ProbConst pc_sh[NT / 32][2];
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    auto load_kc = [&](int q, int slot) {
        static_assert(sizeof(CxConst) % 4 == 0 && sizeof(KConst<T>) % 4 == 0, "copied as 32-bit words");
        const uint32_t* srcC = reinterpret_cast<const uint32_t*>(&recs[q].C);
        const uint32_t* srcK = reinterpret_cast<const uint32_t*>(&recs[q].K);
        uint32_t* dstC = reinterpret_cast<uint32_t*>(&pc_sh[warp][slot].C);
        uint32_t* dstK = reinterpret_cast<uint32_t*>(&pc_sh[warp][slot].K);
        __syncwarp();
        for (int i = lane; i < (int)(sizeof(CxConst) / 4); i += 32) dstC[i] = __ldg(srcC + i);
        for (int i = lane; i < (int)(sizeof(KConst<T>) / 4); i += 32) dstK[i] = __ldg(srcK + i);
        __syncwarp();
    };
    int p = 0;
    int t = next_live(blockIdx.x, p);
    int j = 0, x = 0, y = 0;
    NodeIdx cur = no_node();
    Args Ac{};
    int sc = 0; // slot of the current problem's constants
    if (t < total) {
        load_kc(p, 0);
        tile_origin(recs[p], t - sh_tile0[p], x, y);
        cur = node_at_c(pc_sh[warp][0].C, x, y);
        Ac = make_args(p);
        if constexpr (ADJ)
            adj_stage<T, Q, NT>(pc_sh[warp][0].C, Ac, cur, s0);
        else
            fwd_stage<T, Q, NT>(pc_sh[warp][0].C, Ac, cur, s0);
    }
    cp_async_commit();
    int run_tile = t;
    typename SqAccT<T>::type acc;
    bool odd = false;
    while (t < total) {
        const BRec<T>& R = recs[p];
        int tn = t, pn = p, jn = j + 1, xn = x, yn = y + R.ty;
        if (jn == R.rr) {
            jn = 0;
            tn = next_live(t + G, pn);
            if (tn < total) tile_origin(recs[pn], tn - sh_tile0[pn], xn, yn);
        }
        NodeIdx nxt = no_node();
        Args An = Ac;
        if (tn < total) {
            const int sn = pn != p ? sc ^ 1 : sc;
            if (pn != p) {
                An = make_args(pn);
                load_kc(pn, sn);
            }
            const CxConst& Cn = pc_sh[warp][sn].C;
            nxt = node_at_c(Cn, xn, yn);
            if constexpr (ADJ)
                adj_stage<T, Q, NT>(Cn, An, nxt, odd ? s0 : s1);
            else
                fwd_stage<T, Q, NT>(Cn, An, nxt, odd ? s0 : s1);
        }
        cp_async_commit();
        cp_async_wait<1>();
        if constexpr (ADJ)
            adj_compute<T, Q, NT>(pc_sh[warp][sc].C, pc_sh[warp][sc].K, Ac, cur, ThreadSlots<T, NT>{odd ? s1 : s0},
                                  acc);
        else
            fwd_compute<T, Q, NT>(pc_sh[warp][sc].C, pc_sh[warp][sc].K, Ac, cur, ThreadSlots<T, NT>{odd ? s1 : s0},
                                  acc);
        if (pn != p || tn >= total) {
            if (st.want_sum) {
                const int slot = R.slot0 + (run_tile - sh_tile0[p]) * (NT >> 5) + ((int)threadIdx.x >> 5);
                acc.flush(sum_slots + slot, max_slots ? max_slots + slot : nullptr);
            }
            acc = typename SqAccT<T>::type{};
            run_tile = tn;
        }
        if (pn != p) sc ^= 1;
        t = tn;
        p = pn;
        j = jn;
        x = xn;
        y = yn;
        cur = nxt;
        Ac = An;
        odd = !odd;
    }
    cp_async_wait<0>();
}

// ---- row-window form of the batched kernel (no solid nodes in any problem,
// rows a whole number of 16-byte units; not the first forward step nor the
// terminal adjoint step).  An item's ty rows x tx columns are staged per
// population plane as ty row windows (the item's columns widened by 16 bytes
// per side, periodic ends from the other end of the row) plus the node-local
// planes, by bulk asynchronous copies that the lanes of warp 0 issue and an
// mbarrier per stage completes; otherwise the item order, the pipeline depth
// and the reduction runs are those of k_batch.

// Staged values of one item: thread (tyi, txi) of a tx-wide tile reads plane j
// at pop + j pw + H + sx (pop offset by tyi (tx + 2H) + txi, pw = ty (tx + 2H))
// and node-local value v at loc + (v - 2Q) NT (loc offset by threadIdx.x).
template <typename T, int Q> struct TileWindow {
    static constexpr int H = 16 / (int)sizeof(T);
    const T* pops;
    const T* loc;
    int pw, nt;
    __device__ __forceinline__ T pop(int j, int sx) const { return pops[j * pw + H + sx]; }
    __device__ __forceinline__ T val(int v) const { return loc[(v - 2 * Q) * nt]; }
    static constexpr bool fwd_bounce(int) { return false; } // grids with solid nodes use per-thread staging
    static constexpr bool adj_bounce(int) { return false; }
    static constexpr bool copies = false;
    static constexpr unsigned bb_bits(const CxConst&, int) { return 0u; }
};

// population part of a stage: 2Q planes of at most NT / 32 windows (tx >= 32)
template <typename T, int Q, int NT> constexpr int bwin_pop_values() {
    return 2 * Q * (NT + 2 * (16 / (int)sizeof(T)) * (NT / 32));
}
template <typename T, int Q, int NT, bool ADJ> constexpr int bwin_stage_values() {
    return bwin_pop_values<T, Q, NT>() + (ADJ ? 6 : 4) * NT;
}
template <typename T, int Q, int NT, bool ADJ> constexpr size_t bwin_smem_fixed() {
    return (size_t)2 * bwin_stage_values<T, Q, NT, ADJ>() * sizeof(T) + 2 * sizeof(uint64_t);
}

// Issue the copies of item (problem R, tile columns [xt, xt + tx), rows
// [yb, yb + ty)) into stage st; called by every lane of warp 0.
template <typename T, int Q, int NT, bool ADJ, typename Args>
__device__ __forceinline__ void bwin_issue(const BRec<T>& R, const Args& A, int xt, int yb, T* st, uint64_t* bar) {
    using L = Lat<Q>;
    constexpr int H = 16 / (int)sizeof(T);
    constexpr int NL = ADJ ? 6 : 4;
    const int lane = (int)threadIdx.x & 31;
    const int nx = R.C.nx, ny = R.C.ny, tx = R.tx, ty = R.ty;
    const int nv = min(tx, nx - xt), nr = max(0, min(ty, ny - yb)); // nr = 0: rows past the grid, nothing to copy
    const int wr = tx + 2 * H, pw = ty * wr;
    const bool rot = R.C.aniso == CX_ANISO_ROTATED, full = R.C.ctrl_full != 0;
    const T* locsrc[NL];
    if constexpr (ADJ) {
        locsrc[0] = A.tape;
        locsrc[1] = A.tape + R.plane;
        locsrc[2] = A.tape + 2 * R.plane;
        locsrc[3] = A.sigma;
        locsrc[4] = (A.g && full) ? A.g : nullptr;
        locsrc[5] = rot ? reinterpret_cast<const T*>(R.C.theta) : nullptr;
    } else {
        locsrc[0] = rot ? reinterpret_cast<const T*>(R.C.theta) : nullptr;
        locsrc[1] = (A.g && full) ? A.g : nullptr;
        locsrc[2] = (A.E && full) ? A.E : nullptr;
        locsrc[3] = A.phi;
    }
    if (lane == 0) {
        int nl = 0;
#pragma unroll
        for (int v = 0; v < NL; ++v) nl += locsrc[v] != nullptr;
        mbar_expect_tx(bar, (uint32_t)((2 * Q * nr * (nv + 2 * H) + nl * nr * nv) * (int)sizeof(T)));
    }
    __syncwarp();
    for (int idx = lane; idx < 2 * Q * nr; idx += 32) {
        const int j = idx / nr, r = idx - j * nr;
        const int i = j < Q ? j : j - Q;
        const int y = yb + r;
        const int dy = ADJ ? L::ey(i) : -L::ey(i); // pull from x + e_i (adjoint) or x - e_i (forward)
        const int ys = y + dy < 0 ? ny - 1 : (y + dy >= ny ? 0 : y + dy);
        bulk_row_window<T, NT>(st + j * pw + r * wr, A.in(j) + (size_t)ys * nx, xt, nv, nx, bar);
    }
    T* const loc = st + bwin_pop_values<T, Q, NT>();
#pragma unroll
    for (int v = 0; v < NL; ++v)
        if (locsrc[v] && lane < nr)
            bulk_g2s(loc + v * NT + lane * tx, locsrc[v] + (size_t)(yb + lane) * nx + xt, nv * sizeof(T), bar);
}

// g (and E) of a controlled node when the control window is not the whole
// grid: per-thread copies into the node's own local slots.
template <typename T, int Q, int NT, bool ADJ, typename Args>
__device__ __forceinline__ void bwin_stage_ctrl(const BRec<T>& R, const Args& A, const NodeIdx& nd, T* st) {
    if (R.C.ctrl_full || !nd.ctrl) return;
    T* const loc = st + bwin_pop_values<T, Q, NT>() + threadIdx.x;
    if constexpr (ADJ) {
        if (A.g) cp_async(loc + 4 * NT, A.g + nd.c);
    } else {
        if (A.g) cp_async(loc + NT, A.g + nd.c);
        if (A.E) cp_async(loc + 2 * NT, A.E + nd.c);
    }
}

template <typename T, int Q, int NT, bool ADJ>
__global__ void __launch_bounds__(NT) k_batch_rows(const BRec<T>* __restrict__ recs, const int* __restrict__ tile0,
                                                   int count, int total, BStep st, double* sum_slots,
                                                   double* max_slots, const int* __restrict__ active,
                                                   const T* __restrict__ lam, int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int SV = bwin_stage_values<T, Q, NT, ADJ>();
    T* const st0 = reinterpret_cast<T*>(smem_raw);
    T* const st1 = st0 + SV;
    uint64_t* const bar = reinterpret_cast<uint64_t*>(st1 + SV);
    int* sh_tile0 = reinterpret_cast<int*>(bar + 2);
    for (int i = threadIdx.x; i <= count; i += NT) sh_tile0[i] = tile0[i];
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    allow_next_grid();
    wait_prior_grid();
    if (block_sees_timeout(status)) return; // the barrier also publishes sh_tile0 and the mbarriers

    const int G = gridDim.x;
    auto next_live = [&](int tt, int& q) -> int {
        while (tt < total) {
            q = find_problem(sh_tile0, count, tt);
            if (__ldg(active + q)) return tt;
            tt += ((sh_tile0[q + 1] - tt + G - 1) / G) * G;
        }
        return total;
    };
    // copies of item (tile tt of problem q, rows step jj) into stage stg, by warp 0
    auto issue = [&](int q, int tt, int jj, T* stg, uint64_t* bb) {
        if (threadIdx.x >= 32) return;
        const BRec<T>& R = recs[q];
        const int local = tt - sh_tile0[q];
        const int tyi = local / R.tiles_x, txi = local - tyi * R.tiles_x;
        const int xt = txi * R.tx, yb = tyi * R.ty * R.rr + jj * R.ty;
        if constexpr (ADJ)
            bwin_issue<T, Q, NT, true>(R, adj_args(R, st), xt, yb, stg, bb);
        else
            bwin_issue<T, Q, NT, false>(R, fwd_args(R, st, lam, q), xt, yb, stg, bb);
    };
    auto stage_ctrl = [&](int q, const NodeIdx& nd, T* stg) {
        const BRec<T>& R = recs[q];
        if constexpr (ADJ)
            bwin_stage_ctrl<T, Q, NT, true>(R, adj_args(R, st), nd, stg);
        else
            bwin_stage_ctrl<T, Q, NT, false>(R, fwd_args(R, st, lam, q), nd, stg);
    };

    int p = 0;
    int t = next_live(blockIdx.x, p);
    int j = 0, x = 0, y = 0;
    NodeIdx cur = no_node();
    if (t < total) {
        tile_origin(recs[p], t - sh_tile0[p], x, y);
        cur = node_at(recs[p], x, y);
        issue(p, t, 0, st0, &bar[0]);
        stage_ctrl(p, cur, st0);
    }
    cp_async_commit();
    int run_tile = t;
    typename SqAccT<T>::type acc;
    unsigned phase = 0; // bit b: parity of stage b's next completion
    int b = 0;          // stage of the current item
    bool ok = true, next_issued = false;
    while (t < total) {
        const BRec<T>& R = recs[p];
        int tn = t, pn = p, jn = j + 1, xn = x, yn = y + R.ty;
        if (jn == R.rr) {
            jn = 0;
            tn = next_live(t + G, pn);
            if (tn < total) tile_origin(recs[pn], tn - sh_tile0[pn], xn, yn);
        }
        NodeIdx nxt = no_node();
        T* const sn = b ? st0 : st1;
        if (tn < total) { // stage b^1 is free: every thread passed the barrier that ended its last use
            nxt = node_at(recs[pn], xn, yn);
            issue(pn, tn, jn, sn, &bar[b ^ 1]);
            stage_ctrl(pn, nxt, sn);
        }
        next_issued = tn < total;
        cp_async_commit();
        cp_async_wait<1>();
        ok = mbar_wait(&bar[b], (phase >> b) & 1u);
        phase ^= 1u << b;
        if (ok) {
            constexpr int H = 16 / (int)sizeof(T);
            const T* sc = b ? st1 : st0;
            const int tyi = (int)threadIdx.x >> R.tx_shift, txi = (int)threadIdx.x & (R.tx - 1);
            const TileWindow<T, Q> S{sc + tyi * (R.tx + 2 * H) + txi, sc + bwin_pop_values<T, Q, NT>() + threadIdx.x,
                                     R.ty * (R.tx + 2 * H), NT};
            if constexpr (ADJ)
                adj_compute<T, Q, NT>(R.C, R.K, adj_args(R, st), cur, S, acc);
            else
                fwd_compute<T, Q, NT>(R.C, R.K, fwd_args(R, st, lam, p), cur, S, acc);
        }
        if (__syncthreads_or(!ok)) { // all threads leave together when a stage never completed
            ok = false;
            break;
        }
        if (pn != p || tn >= total) {
            if (st.want_sum) {
                const int slot = R.slot0 + (run_tile - sh_tile0[p]) * (NT >> 5) + ((int)threadIdx.x >> 5);
                acc.flush(sum_slots + slot, max_slots ? max_slots + slot : nullptr);
            }
            acc = typename SqAccT<T>::type{};
            run_tile = tn;
        }
        t = tn;
        p = pn;
        j = jn;
        x = xn;
        y = yn;
        cur = nxt;
        b ^= 1;
    }
    if (!ok) {
        // bounded waits for the copies still in flight, then report
        if (next_issued) mbar_wait(&bar[b ^ 1], (phase >> (b ^ 1)) & 1u);
        mbar_wait(&bar[b], ((phase >> b) & 1u) ^ 1u);
        if (threadIdx.x == 0 && status) atomicOr(status, ST_TIMEOUT);
    }
    cp_async_wait<0>();
}

// Per-problem fixed-order sums: J_p = cost_p + alpha_p * sum(gsq slots) (mode 0)
// or (sum E^2, max |E|) (mode 1).  One block per problem.
struct BFin {
    const double* cost; // per-problem cost partial array (block partials of k_final)
    int ncost;
    int slot0, nslots;
    double alpha;
};
__global__ void __launch_bounds__(256) k_bfinalize(const BFin* fin, const double* sums, const double* maxs, int mode,
                                                    double* out_a, double* out_b, int* status, const int* active) {
    __shared__ double sa[256], sb[256];
    if (!active[blockIdx.x]) return; // switched off: outputs left as they were
    const BFin F = fin[blockIdx.x];
    const int t = threadIdx.x;
    double ra = 0.0, rb = 0.0;
    if (mode == 0)
        for (int i = t; i < F.ncost; i += 256) ra += F.cost[i];
    for (int i = t; i < F.nslots; i += 256) {
        if (mode == 0) rb += sums[F.slot0 + i];
        else {
            ra += sums[F.slot0 + i];
            rb = fmax(rb, maxs[F.slot0 + i]);
        }
    }
    sa[t] = ra;
    sb[t] = rb;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (t < h) {
            sa[t] += sa[t + h];
            sb[t] = (mode == 1) ? fmax(sb[t], sb[t + h]) : sb[t] + sb[t + h];
        }
        __syncthreads();
    }
    if (t == 0) {
        if (mode == 0) {
            const double J = sa[0] + F.alpha * sb[0];
            out_a[blockIdx.x] = J;
            if (!isfinite(J)) atomicOr(status, ST_UNSTABLE);
        } else {
            out_a[blockIdx.x] = sa[0];
            if (out_b) out_b[blockIdx.x] = sb[0];
            if (!isfinite(sa[0])) atomicOr(status, ST_UNSTABLE);
        }
    }
}

// Accepted line-search steps: g_p <- g_p - lam_p dJ/dg_p for every problem
// with lam_p != 0, rounded as the trial control of the forward.
template <typename T> __global__ void k_baxpy(const BRec<T>* __restrict__ recs, int count, const T* __restrict__ lam) {
    const int p = blockIdx.y;
    if (p >= count || lam[p] == T(0)) return;
    const BRec<T>& R = recs[p];
    T* g = const_cast<T*>(R.g);
    const T* E = R.dJdg;
    const T l = lam[p];
    const size_t n = (size_t)R.nwin * R.nctrl;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        g[i] = fma(-l, E[i], g[i]);
}

// terminal adjoint seed plus a caller's addition: wu += add (n nodes)
template <typename T> __global__ void k_add_seed(T* wu, const T* add, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        wu[i] += add[i];
}

// Node-plane operations over all problems: zero sigma (op 0), restore Phi
// from checkpoint slot `slot` (op 1).
template <typename T>
__global__ void k_bplanes(const BRec<T>* __restrict__ recs, int count, int op, int slot) {
    const int p = blockIdx.y;
    if (p >= count) return;
    const BRec<T>& R = recs[p];
    const size_t n = (size_t)R.C.nx * R.C.ny;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        if (op == 0) R.sigma[i] = T(0);
        else R.phi[i] = R.ckpt_phi[(size_t)slot * R.plane + i];
    }
}

} // namespace cx

using namespace cx;

namespace {

struct BatchHost {
    int count = 0, threads = 256, blocks = 0, total_tiles = 0, nslots = 0;
    size_t slot_cap = 0;
    int Q = 9, N = 1, k = 1, S = 1;
    size_t esz = 4;
    std::vector<cx_problem*> probs;
    std::vector<int> tx; // tile width per problem
    std::vector<int> rr; // rows per thread per tile, per problem
    char* ws = nullptr;
    size_t off_rec = 0, off_tile0 = 0, off_fin = 0, off_sums = 0, off_maxs = 0, off_out = 0, off_status = 0;
    size_t off_active = 0, off_lam = 0;
    size_t rec_bytes = 0;
    std::vector<const void*> g;
    std::vector<void*> dJdg;
    cudaStream_t stream = nullptr;
    // captured launch sequences: forward, forward + adjoint, line-search trial forward, adjoint only
    cudaGraphExec_t graphs[4] = {nullptr, nullptr, nullptr, nullptr};
    bool has_init = false, bound = false;
    std::vector<int> enabled;      // problems the caller keeps switched on
    std::vector<double> lam_prev;  // last accepted step length per problem (0: none yet)
    std::vector<double> J_at_g;    // cost at the current control, valid while fwd_at_g
    bool J_on_device = false;      // ... or in out[0..count) (after cx_batch_forward / _gradient)
    bool fwd_at_g = false;         // every enabled problem's forward state (checkpoints, last
                                   // tape, final populations) belongs to its current control
    int row_windows = 0;           // 1: steps that qualify use k_batch_rows (slower here, see cx_batch_set_staging)
    bool rows_ok = false;          // every problem qualifies (no solids, aligned rows and controls)
    int rows_blocks[2] = {0, 0};   // persistent blocks of k_batch_rows (forward, adjoint)
};

enum { G_FWD = 0, G_GRAD = 1, G_TRIAL = 2, G_ADJ = 3 };

} // namespace

struct cx_batch {
    BatchHost h;
};

namespace {

constexpr int MAX_BATCH = 4096;

size_t rec_size(size_t esz) { return esz == 8 ? sizeof(BRec<double>) : sizeof(BRec<float>); }

// Reduction slots any admissible tiling of a problem can need: (threads/32)
// slots per tile, tiles = ceil(nx/tx) ceil(ny/ty) <= nx ny/128 + nx/32 + ny + 1
// for 128 <= threads = tx ty <= 256, tx >= 32, ty >= 1.
size_t slot_capacity(const cx_problem_desc& d) {
    const size_t nx = d.nx, ny = d.ny;
    return 8 * (nx * ny / 128 + nx / 32 + ny + 2);
}

// tiles and reduction slots for the current tile shapes
void plan_tiles(BatchHost& h, std::vector<int>& tile0, std::vector<int>& slot0) {
    tile0.assign(h.count + 1, 0);
    slot0.assign(h.count + 1, 0);
    for (int i = 0; i < h.count; ++i) {
        const int tx = h.tx[i], th = (h.threads / tx) * h.rr[i];
        const int nt = ((h.probs[i]->d.nx + tx - 1) / tx) * ((h.probs[i]->d.ny + th - 1) / th);
        tile0[i + 1] = tile0[i] + nt;
        slot0[i + 1] = slot0[i] + nt * (h.threads / 32);
    }
    h.total_tiles = tile0[h.count];
    h.nslots = slot0[h.count];
}

template <typename T> cx_status upload_table(BatchHost& h) {
    std::vector<int> tile0, slot0;
    plan_tiles(h, tile0, slot0);
    if ((size_t)h.nslots > h.slot_cap) return CX_ERR_INTERNAL; // cannot happen for admissible tilings
    std::vector<BRec<T>> recs(h.count);
    std::vector<BFin> fin(h.count);
    for (int i = 0; i < h.count; ++i) {
        cx_problem* p = h.probs[i];
        BRec<T>& R = recs[i];
        std::memset(&R, 0, sizeof(R));
        R.C = p->C;
        R.C.bb_copy = 0; // the batched kernels resolve bounce-back while staging
        R.K = p->kc((T*)nullptr);
        R.pop[ROLE_POPA] = p->at<T>(p->lay.off_popA);
        R.pop[ROLE_POPB] = p->at<T>(p->lay.off_popB);
        R.pop[ROLE_CKPT] = reinterpret_cast<T*>(p->ckpt_slot(0));
        R.pop[ROLE_ADJA] = p->at<T>(p->lay.off_adjA);
        R.pop[ROLE_ADJB] = p->at<T>(p->lay.off_adjB);
        R.ckpt_phi = reinterpret_cast<T*>(p->ckpt_phi_slot(0));
        R.phi = p->at<T>(p->lay.off_phi);
        R.sigma = p->at<T>(p->lay.off_sigma);
        R.tape = reinterpret_cast<T*>(p->tape_slot(0));
        R.wu = p->at<T>(p->lay.off_wu);
        R.g = h.g.empty() ? nullptr : static_cast<const T*>(h.g[i]);
        R.dJdg = h.dJdg.empty() ? nullptr : static_cast<T*>(h.dJdg[i]);
        R.plane = (long long)p->lay.plane;
        R.nctrl = (long long)p->lay.nctrl;
        R.win_len = p->lay.win_len;
        R.nwin = p->lay.nwin;
        R.pop_elems = (long long)(2 * p->lay.Q * p->lay.plane);
        R.tile0 = tile0[i];
        R.tx = h.tx[i];
        R.ty = h.threads / h.tx[i];
        R.tx_shift = 0;
        while ((1 << R.tx_shift) < R.tx) ++R.tx_shift;
        R.rr = h.rr[i];
        R.tiles_x = (p->d.nx + R.tx - 1) / R.tx;
        R.slot0 = slot0[i];
        fin[i].cost = p->at<double>(p->lay.off_part);
        fin[i].ncost = p->nblocks;
        fin[i].slot0 = slot0[i];
        fin[i].nslots = slot0[i + 1] - slot0[i];
        fin[i].alpha = p->C.alpha;
    }
    // row-window staging: no solid nodes, rows of whole 16-byte units, 16-byte aligned control arrays
    h.rows_ok = true;
    for (int i = 0; i < h.count; ++i) {
        const cx_problem* p = h.probs[i];
        auto al = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
        const bool gi = h.g.empty() || !h.g[i] || al(h.g[i]);
        const bool ei = h.dJdg.empty() || !h.dJdg[i] || al(h.dJdg[i]);
        if (p->C.has_solid || p->d.nx % (int)(16 / sizeof(T)) != 0 || !gi || !ei ||
            ((size_t)p->lay.plane * sizeof(T)) % 16 != 0)
            h.rows_ok = false;
    }
    if (cudaMemcpy(h.ws + h.off_rec, recs.data(), sizeof(BRec<T>) * h.count, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h.ws + h.off_tile0, tile0.data(), sizeof(int) * (h.count + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h.ws + h.off_fin, fin.data(), sizeof(BFin) * h.count, cudaMemcpyHostToDevice) != cudaSuccess)
        return CX_ERR_CUDA;
    return CX_OK;
}

void drop_graphs(BatchHost& h) {
    for (cudaGraphExec_t& g : h.graphs) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

template <typename T, int Q, int NT, bool ADJ>
cudaError_t launch_bq(const BatchHost& h, const BStep& st, int blocks) {
    constexpr int NV = ADJ ? 2 * Q + 6 : 2 * Q + 4;
    const size_t smem = (size_t)2 * NV * NT * sizeof(T) + sizeof(int) * (h.count + 1);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_batch<T, Q, NT, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             128 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = h.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    double* sums = reinterpret_cast<double*>(h.ws + h.off_sums);
    double* maxs = ADJ ? reinterpret_cast<double*>(h.ws + h.off_maxs) : nullptr;
    return cudaLaunchKernelEx(&cfg, k_batch<T, Q, NT, ADJ>, reinterpret_cast<const BRec<T>*>(h.ws + h.off_rec),
                              reinterpret_cast<const int*>(h.ws + h.off_tile0), h.count, h.total_tiles, st, sums,
                              maxs, reinterpret_cast<const int*>(h.ws + h.off_active),
                              reinterpret_cast<const T*>(h.ws + h.off_lam));
}

template <typename T, int Q, int NT, bool ADJ> size_t bwin_smem(int count) {
    return bwin_smem_fixed<T, Q, NT, ADJ>() + sizeof(int) * (count + 1);
}

template <typename T, int Q, int NT, bool ADJ>
cudaError_t launch_bq_rows(const BatchHost& h, const BStep& st, int blocks) {
    const size_t smem = bwin_smem<T, Q, NT, ADJ>(h.count);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_batch_rows<T, Q, NT, ADJ>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = h.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    double* sums = reinterpret_cast<double*>(h.ws + h.off_sums);
    double* maxs = ADJ ? reinterpret_cast<double*>(h.ws + h.off_maxs) : nullptr;
    return cudaLaunchKernelEx(&cfg, k_batch_rows<T, Q, NT, ADJ>, reinterpret_cast<const BRec<T>*>(h.ws + h.off_rec),
                              reinterpret_cast<const int*>(h.ws + h.off_tile0), h.count, h.total_tiles, st, sums,
                              maxs, reinterpret_cast<const int*>(h.ws + h.off_active),
                              reinterpret_cast<const T*>(h.ws + h.off_lam),
                              reinterpret_cast<int*>(h.ws + h.off_status));
}

// resident blocks per SM of k_batch_rows for this batch's table size
template <typename T, int Q, int NT, bool ADJ> int bwin_occupancy(int count) {
    const size_t smem = bwin_smem<T, Q, NT, ADJ>(count);
    if (smem > 200 * 1024) return 0;
    cudaFuncSetAttribute(k_batch_rows<T, Q, NT, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_rows<T, Q, NT, ADJ>, NT, smem) != cudaSuccess)
        return 0;
    return nb;
}
template <typename T, bool ADJ> int bwin_occ(int Q, int threads, int count) {
    if (Q == 9)
        return threads == 128 ? bwin_occupancy<T, 9, 128, ADJ>(count) : bwin_occupancy<T, 9, 256, ADJ>(count);
    return threads == 128 ? bwin_occupancy<T, 5, 128, ADJ>(count) : bwin_occupancy<T, 5, 256, ADJ>(count);
}

// persistent blocks of the row-window kernels (0: they do not fit; blocks > 0: the caller's count)
void set_rows_blocks(BatchHost& h, int threads, int blocks) {
    for (int a = 0; a < 2; ++a) {
        const int ro = h.esz == 8 ? (a ? bwin_occ<double, true>(h.Q, threads, h.count)
                                       : bwin_occ<double, false>(h.Q, threads, h.count))
                                  : (a ? bwin_occ<float, true>(h.Q, threads, h.count)
                                       : bwin_occ<float, false>(h.Q, threads, h.count));
        h.rows_blocks[a] = ro <= 0 ? 0 : (blocks > 0 ? blocks : h.probs[0]->nsm * ro);
    }
}

template <typename T, bool ADJ> cudaError_t launch_b(const BatchHost& h, const BStep& st) {
    const bool rows = h.row_windows && h.rows_ok && h.rows_blocks[ADJ ? 1 : 0] > 0 && (ADJ ? !st.terminal : st.n > 0);
    if (rows) {
        const int rb = std::max(1, std::min(h.rows_blocks[ADJ ? 1 : 0], h.total_tiles));
        if (h.Q == 9)
            return h.threads == 128 ? launch_bq_rows<T, 9, 128, ADJ>(h, st, rb) : launch_bq_rows<T, 9, 256, ADJ>(h, st, rb);
        return h.threads == 128 ? launch_bq_rows<T, 5, 128, ADJ>(h, st, rb) : launch_bq_rows<T, 5, 256, ADJ>(h, st, rb);
    }
    const int blocks = std::max(1, std::min(h.blocks, h.total_tiles));
    if (h.Q == 9) {
        if (h.threads == 128) return launch_bq<T, 9, 128, ADJ>(h, st, blocks);
        return launch_bq<T, 9, 256, ADJ>(h, st, blocks);
    }
    if (h.threads == 128) return launch_bq<T, 5, 128, ADJ>(h, st, blocks);
    return launch_bq<T, 5, 256, ADJ>(h, st, blocks);
}

template <typename T> cudaError_t launch_planes(const BatchHost& h, int op, int slot) {
    dim3 grid(64, h.count), block(256);
    k_bplanes<T><<<grid, block, 0, h.stream>>>(reinterpret_cast<const BRec<T>*>(h.ws + h.off_rec), h.count, op,
                                                 slot);
    return cudaGetLastError();
}

#define B_CUDA(x)                                                                                                    \
    do {                                                                                                             \
        if ((x) != cudaSuccess) return CX_ERR_CUDA;                                                                  \
    } while (0)

// Forward of every problem (at g_p, or at the trial g_p - lam_p dJ/dg_p); J_p into out[0..count).
template <typename T> cx_status enqueue_forward(BatchHost& h, bool trial) {
    double* sums = reinterpret_cast<double*>(h.ws + h.off_sums);
    B_CUDA(cudaMemsetAsync(sums, 0, sizeof(double) * h.nslots, h.stream));
    const int N = h.N, k = h.k, S = h.S;
    int in_role = ROLE_CKPT, in_slot = 0;
    for (int n = 0; n < N; ++n) {
        const int seg = n / k;
        BStep st{};
        st.n = n;
        st.in_role = in_role;
        st.in_slot = in_slot;
        if (n + 1 < N && (n + 1) % k == 0) {
            st.out_role = ROLE_CKPT;
            st.out_slot = (n + 1) / k;
            st.phi_ckpt_slot = (n + 1) / k;
        } else {
            st.out_role = (n % 2) ? ROLE_POPB : ROLE_POPA;
            st.out_slot = 0;
            st.phi_ckpt_slot = -1;
        }
        st.tape_slot = (seg == S - 1) ? n - seg * k : -1;
        st.want_sum = 1;
        st.trial = trial ? 1 : 0;
        B_CUDA((launch_b<T, false>(h, st)));
        in_role = st.out_role;
        in_slot = st.out_slot;
    }
    for (int i = 0; i < h.count; ++i) {
        cx_problem* p = h.probs[i];
        const T* in = in_role == ROLE_CKPT ? reinterpret_cast<const T*>(p->ckpt_slot(in_slot))
                                           : p->at<T>(in_role == ROLE_POPA ? p->lay.off_popA : p->lay.off_popB);
        B_CUDA(launch_final<T>(p->C, in, p->at<T>(p->lay.off_ut), p->at<T>(p->lay.off_uN), p->at<T>(p->lay.off_vN),
                               p->at<T>(p->lay.off_wu), p->at<double>(p->lay.off_part), p->L, h.stream));
    }
    k_bfinalize<<<h.count, 256, 0, h.stream>>>(reinterpret_cast<const BFin*>(h.ws + h.off_fin), sums, nullptr, 0,
                                                reinterpret_cast<double*>(h.ws + h.off_out), nullptr,
                                                reinterpret_cast<int*>(h.ws + h.off_status),
                                                reinterpret_cast<const int*>(h.ws + h.off_active));
    B_CUDA(cudaGetLastError());
    return CX_OK;
}

// Recompute + AMRT adjoint of every problem; ||E_p||^2, max|E_p| into out[count..3 count).
template <typename T> cx_status enqueue_adjoint(BatchHost& h) {
    double* sums = reinterpret_cast<double*>(h.ws + h.off_sums);
    double* maxs = reinterpret_cast<double*>(h.ws + h.off_maxs);
    B_CUDA(cudaMemsetAsync(sums, 0, sizeof(double) * h.nslots, h.stream));
    B_CUDA(cudaMemsetAsync(maxs, 0, sizeof(double) * h.nslots, h.stream));
    B_CUDA(launch_planes<T>(h, 0, 0));
    const int N = h.N, k = h.k, S = h.S;
    int in_role = -1, in_slot = 0;
    for (int s = S - 1; s >= 0; --s) {
        const int n0 = s * k, n1 = std::min(N, n0 + k);
        if (s < S - 1) { // the last segment's tape comes from the forward
            if (s >= 1) B_CUDA(launch_planes<T>(h, 1, s));
            int ri = ROLE_CKPT, rs = s;
            for (int n = n0; n < n1; ++n) {
                BStep st{};
                st.n = n;
                st.in_role = ri;
                st.in_slot = rs;
                st.out_role = (n % 2) ? ROLE_POPB : ROLE_POPA;
                st.out_slot = 0;
                st.phi_ckpt_slot = -1;
                st.tape_slot = n - n0;
                st.want_sum = 0;
                B_CUDA((launch_b<T, false>(h, st)));
                ri = st.out_role;
                rs = 0;
            }
        }
        for (int n = n1 - 1; n >= n0; --n) {
            BStep st{};
            st.n = n;
            st.terminal = (n == N - 1);
            st.in_role = st.terminal ? ROLE_ADJA : in_role;
            st.in_slot = in_slot;
            st.out_role = (n % 2) ? ROLE_ADJB : ROLE_ADJA;
            st.out_slot = 0;
            st.phi_ckpt_slot = -1;
            st.tape_slot = n - n0;
            st.want_sum = 1;
            B_CUDA((launch_b<T, true>(h, st)));
            in_role = st.out_role;
            in_slot = 0;
        }
    }
    double* out = reinterpret_cast<double*>(h.ws + h.off_out);
    k_bfinalize<<<h.count, 256, 0, h.stream>>>(reinterpret_cast<const BFin*>(h.ws + h.off_fin), sums, maxs, 1,
                                                out + h.count, out + 2 * h.count,
                                                reinterpret_cast<int*>(h.ws + h.off_status),
                                                reinterpret_cast<const int*>(h.ws + h.off_active));
    B_CUDA(cudaGetLastError());
    return CX_OK;
}

template <typename T> cx_status capture(BatchHost& h, int mode, cudaGraphExec_t* exec) {
    cudaGraph_t graph = nullptr;
    B_CUDA(cudaStreamBeginCapture(h.stream, cudaStreamCaptureModeThreadLocal));
    cx_status rc = CX_OK;
    if (mode != G_ADJ) rc = enqueue_forward<T>(h, mode == G_TRIAL);
    if (rc == CX_OK && (mode == G_GRAD || mode == G_ADJ)) rc = enqueue_adjoint<T>(h);
    const cudaError_t e = cudaStreamEndCapture(h.stream, &graph);
    if (rc != CX_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return rc != CX_OK ? rc : CX_ERR_CUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    return ei == cudaSuccess ? CX_OK : CX_ERR_CUDA;
}

template <typename T> cx_status run_graph(BatchHost& h, int mode) {
    cudaGraphExec_t* ex = &h.graphs[mode];
    if (!*ex) {
        cx_status rc = capture<T>(h, mode, ex);
        if (rc) return rc;
    }
    B_CUDA(cudaGraphLaunch(*ex, h.stream));
    const bool adj = mode == G_GRAD || mode == G_ADJ;
    for (cx_problem* p : h.probs) {
        p->fwd_valid = true;
        p->adj_valid = false;
        p->tape_last_valid = !adj || h.S == 1;
    }
    return CX_OK;
}

template <typename T> cx_status run(BatchHost& h, bool with_adjoint, double* out_dev) {
    cx_status rc = run_graph<T>(h, with_adjoint ? G_GRAD : G_FWD);
    if (rc) return rc;
    h.fwd_at_g = !with_adjoint || h.S == 1;
    h.J_on_device = true;
    if (out_dev)
        B_CUDA(cudaMemcpyAsync(out_dev, h.ws + h.off_out, sizeof(double) * (with_adjoint ? 3 : 1) * h.count,
                               cudaMemcpyDeviceToDevice, h.stream));
    return CX_OK;
}

cx_status upload_ints(BatchHost& h, size_t off, const std::vector<int>& v) {
    B_CUDA(cudaMemcpyAsync(h.ws + off, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice, h.stream));
    return CX_OK;
}

// per-problem step lengths in the precision T of the controls
cx_status upload_lam(BatchHost& h, const std::vector<double>& lam) {
    if (h.esz == 8) {
        B_CUDA(cudaMemcpyAsync(h.ws + h.off_lam, lam.data(), sizeof(double) * lam.size(), cudaMemcpyHostToDevice,
                               h.stream));
    } else {
        std::vector<float> f(lam.begin(), lam.end());
        B_CUDA(cudaMemcpyAsync(h.ws + h.off_lam, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice,
                               h.stream));
        B_CUDA(cudaStreamSynchronize(h.stream)); // f is a local
    }
    return CX_OK;
}

cx_status read_out(BatchHost& h, std::vector<double>& out, int& status) {
    out.resize(3 * (size_t)h.count);
    B_CUDA(cudaMemcpyAsync(out.data(), h.ws + h.off_out, sizeof(double) * out.size(), cudaMemcpyDeviceToHost,
                           h.stream));
    B_CUDA(cudaMemcpyAsync(&status, h.ws + h.off_status, sizeof(int), cudaMemcpyDeviceToHost, h.stream));
    B_CUDA(cudaStreamSynchronize(h.stream));
    return (status & ST_TIMEOUT) ? CX_ERR_TIMEOUT : CX_OK;
}

// One Armijo gradient step of every enabled problem (the single-problem rule
// of cx_step: c1 = 1e-4, first trial 2 lam_prev or min(1, 1/max|E|), halving,
// at most 30 trials).  Trials run as one batched forward over the problems
// still searching; the others are switched off in the device mask.
template <typename T> cx_status batch_step(BatchHost& h, cx_step_info* info, int* pstatus) {
    const int n = h.count;
    std::vector<int> act(h.enabled);
    cx_status rc = upload_ints(h, h.off_active, act);
    if (rc) return rc;
    std::vector<double> out;
    int dstat = 0;
    std::vector<double> J0(n), e2(n), einf(n);
    if (!h.fwd_at_g) {
        rc = run_graph<T>(h, G_GRAD);
        if (rc) return rc;
        rc = read_out(h, out, dstat);
        if (rc) return rc;
        for (int i = 0; i < n; ++i) J0[i] = out[i];
    } else {
        rc = run_graph<T>(h, G_ADJ);
        if (rc) return rc;
        rc = read_out(h, out, dstat);
        if (rc) return rc;
        if (h.J_on_device)
            for (int i = 0; i < n; ++i) J0[i] = out[i];
        else
            J0 = h.J_at_g;
    }
    std::vector<int> st(n, CX_OK), trials(n, 0);
    std::vector<double> lam(n, 0.0), Jt(n, 0.0), acc_lam(n, 0.0);
    std::vector<int> search(n, 0);
    int nsearch = 0;
    for (int i = 0; i < n; ++i) {
        e2[i] = out[n + i];
        einf[i] = out[2 * n + i];
        Jt[i] = J0[i];
        if (!h.enabled[i]) continue;
        if (!std::isfinite(J0[i]) || !std::isfinite(e2[i])) {
            st[i] = CX_ERR_UNSTABLE;
            continue;
        }
        if (e2[i] == 0.0) continue; // stationary: nothing to do
        lam[i] = h.lam_prev[i] > 0.0 ? 2.0 * h.lam_prev[i] : std::min(1.0, einf[i] > 0.0 ? 1.0 / einf[i] : 1.0);
        search[i] = 1;
        ++nsearch;
    }
    for (int t = 0; t < 30 && nsearch > 0; ++t) {
        if ((rc = upload_ints(h, h.off_active, search)) || (rc = upload_lam(h, lam))) return rc;
        rc = run_graph<T>(h, G_TRIAL);
        if (rc) return rc;
        rc = read_out(h, out, dstat);
        if (rc) return rc;
        for (int i = 0; i < n; ++i) {
            if (!search[i]) continue;
            ++trials[i];
            if (std::isfinite(out[i]) && out[i] <= J0[i] - 1e-4 * lam[i] * e2[i]) {
                Jt[i] = out[i];
                acc_lam[i] = lam[i];
                h.lam_prev[i] = lam[i];
                search[i] = 0;
                --nsearch;
            } else {
                lam[i] *= 0.5;
            }
        }
    }
    bool all_ok = true;
    for (int i = 0; i < n; ++i)
        if (search[i]) {
            st[i] = CX_ERR_LINESEARCH;
            all_ok = false;
        } else if (st[i] != CX_OK) {
            all_ok = false;
        }
    if ((rc = upload_lam(h, acc_lam))) return rc;
    k_baxpy<T><<<dim3(64, n), 256, 0, h.stream>>>(reinterpret_cast<const BRec<T>*>(h.ws + h.off_rec), n,
                                                   reinterpret_cast<const T*>(h.ws + h.off_lam));
    B_CUDA(cudaGetLastError());
    if ((rc = upload_ints(h, h.off_active, h.enabled))) return rc;
    // accepted trials left each problem's forward state at its new control
    h.J_at_g = Jt;
    h.J_on_device = false;
    h.fwd_at_g = all_ok;
    for (int i = 0; i < n; ++i) {
        if (pstatus) pstatus[i] = st[i];
        if (info) {
            info[i].J0 = J0[i];
            info[i].J = Jt[i];
            info[i].lam = acc_lam[i];
            info[i].grad_sq = e2[i];
            info[i].grad_inf = einf[i];
            info[i].trials = trials[i];
        }
    }
    B_CUDA(cudaStreamSynchronize(h.stream));
    return CX_OK;
}

cx_status batch_layout(const cx_problem_desc* d, int count, std::vector<size_t>* offs, size_t* table_off,
                       size_t* total) {
    if (!d || count < 1 || count > MAX_BATCH) return CX_ERR_INVALID_ARG;
    size_t o = 0;
    for (int i = 0; i < count; ++i) {
        if (d[i].halo) return CX_ERR_INVALID_ARG; // sub-domains of one problem are not independent problems
        if (d[i].n_steps != d[0].n_steps || d[i].lattice != d[0].lattice || d[i].precision != d[0].precision ||
            (d[i].ckpt_every ? d[i].ckpt_every : d[i].n_steps) != (d[0].ckpt_every ? d[0].ckpt_every : d[0].n_steps))
            return CX_ERR_INVALID_ARG;
        size_t b = 0;
        cx_status rc = cx_workspace_size(&d[i], &b);
        if (rc) return rc;
        if (offs) offs->push_back(o);
        o = up(o + b, ALIGN);
    }
    *table_off = o;
    // records, tile prefix, finalize records, slots (sized for the densest tiling), outputs, status
    size_t slots = 0;
    for (int i = 0; i < count; ++i) slots += slot_capacity(d[i]);
    const size_t esz = d[0].precision == 64 ? 8 : 4;
    o = up(o + rec_size(esz) * count, ALIGN);
    o = up(o + sizeof(int) * (count + 1), ALIGN);
    o = up(o + sizeof(BFin) * count, ALIGN);
    o = up(o + sizeof(double) * slots, ALIGN);
    o = up(o + sizeof(double) * slots, ALIGN);
    o = up(o + sizeof(double) * 3 * count, ALIGN);
    o = up(o + sizeof(int) * 4, ALIGN);
    o = up(o + sizeof(int) * count, ALIGN);    // enabled / searching mask
    o = up(o + sizeof(double) * count, ALIGN); // step lengths
    *total = o;
    return CX_OK;
}

// ---- autotuner: probe timing, search, cache ----

constexpr int TUNE_WIDTHS[4] = {32, 64, 128, 256};
constexpr int TUNE_ROWS[4] = {4, 8, 16, 32};
constexpr int TUNE_UNIFORM[5][2] = {{32, 8}, {64, 8}, {64, 16}, {128, 16}, {32, 16}};

bool tune_admissible(int threads, int nx, int t) {
    return t <= threads && threads % t == 0 && threads / t <= 8 && t <= std::max(32, 2 * nx);
}

int tune_widest(int threads, int nx) {
    int w = 0;
    for (int t : TUNE_WIDTHS)
        if (tune_admissible(threads, nx, t)) w = t;
    return w;
}

// The probe shortens the schedule to N' = min(N, probe) steps with interval
// k' = min(k, N') (S = 1) or min(k, ceil(N'/2)) (S >= 2), so that it has
// S' <= S segments (k' = k gives ceil(N'/k) <= S, otherwise S' <= 2 <= S) and
// a recompute: every checkpoint slot, tape plane and step index it touches
// exists for the full schedule too.  The guard puts N, k, S back on every
// return path.
struct ScheduleGuard {
    BatchHost& h;
    int N, k, S;
    ScheduleGuard(BatchHost& hh, int probe) : h(hh), N(hh.N), k(hh.k), S(hh.S) {
        const int n1 = std::min(N, probe);
        int k1 = std::min(k, n1);
        if (S >= 2 && n1 > 1) k1 = std::min(k, (n1 + 1) / 2);
        h.N = n1;
        h.k = k1;
        h.S = (n1 + k1 - 1) / k1;
    }
    ~ScheduleGuard() {
        h.N = N;
        h.k = k;
        h.S = S;
    }
};

// Mean time of one probe (forward, recompute, adjoint; direct launches) with
// the given tiles, after one untimed probe.
template <typename T>
cx_status time_probe(BatchHost& h, int threads, const std::vector<int>& tx, const std::vector<int>& rr,
                     cudaEvent_t e0, cudaEvent_t e1, double* ms) {
    B_CUDA(cudaStreamSynchronize(h.stream)); // nothing in flight reads the table while it is replaced
    h.threads = threads;
    h.tx = tx;
    h.rr = rr;
    const int occ = forward_occupancy<T>(h.Q, threads);
    h.blocks = h.probs[0]->nsm * occ;
    set_rows_blocks(h, threads, 0);
    cx_status rc = upload_table<T>(h);
    if (rc) return rc;
    constexpr int REPS = 2;
    for (int r = 0; r <= REPS; ++r) {
        if (r == 1) B_CUDA(cudaEventRecord(e0, h.stream));
        rc = enqueue_forward<T>(h, false);
        if (rc == CX_OK) rc = enqueue_adjoint<T>(h);
        if (rc) return rc;
    }
    B_CUDA(cudaEventRecord(e1, h.stream));
    B_CUDA(cudaEventSynchronize(e1));
    float t = 0.f;
    B_CUDA(cudaEventElapsedTime(&t, e0, e1));
    *ms = (double)t / REPS;
    return CX_OK;
}

struct TuneChoice {
    int threads = 0;
    std::map<int, int> tx, rr; // per size class (nx)
    double ms = 0.0;
};

template <typename T> cx_status tune_search(BatchHost& h, TuneChoice* best) {
    std::vector<int> classes;
    for (cx_problem* p : h.probs) classes.push_back(p->d.nx);
    std::sort(classes.begin(), classes.end());
    classes.erase(std::unique(classes.begin(), classes.end()), classes.end());
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return CX_ERR_CUDA;
    }
    cx_status rc = CX_OK;
    best->threads = 0;
    for (int threads : {128, 256}) {
        auto timed = [&](const std::map<int, int>& tx, const std::map<int, int>& rr, double* ms) {
            std::vector<int> vt(h.count), vr(h.count);
            for (int i = 0; i < h.count; ++i) {
                vt[i] = tx.at(h.probs[i]->d.nx);
                vr[i] = rr.at(h.probs[i]->d.nx);
            }
            return time_probe<T>(h, threads, vt, vr, e0, e1, ms);
        };
        TuneChoice cur;
        cur.threads = threads;
        bool have = false;
        for (const auto& u : TUNE_UNIFORM) {
            std::map<int, int> tx, rr;
            bool ok = true;
            for (int nx : classes) {
                const int t = std::min(u[0], tune_widest(threads, nx));
                ok = ok && t > 0 && tune_admissible(threads, nx, t);
                tx[nx] = t;
                rr[nx] = u[1];
            }
            if (!ok) continue;
            double ms = 0.0;
            if ((rc = timed(tx, rr, &ms))) break;
            if (!have || ms < cur.ms) {
                cur.tx = tx;
                cur.rr = rr;
                cur.ms = ms;
                have = true;
            }
        }
        if (rc) break;
        if (!have) continue;
        for (int nx : classes) {
            for (int r : TUNE_ROWS) {
                if (r == cur.rr[nx]) continue;
                std::map<int, int> rr = cur.rr;
                rr[nx] = r;
                double ms = 0.0;
                if ((rc = timed(cur.tx, rr, &ms))) break;
                if (ms < cur.ms) {
                    cur.rr = rr;
                    cur.ms = ms;
                }
            }
            if (rc) break;
            for (int t : TUNE_WIDTHS) {
                if (!tune_admissible(threads, nx, t) || t == cur.tx[nx]) continue;
                std::map<int, int> tx = cur.tx;
                tx[nx] = t;
                double ms = 0.0;
                if ((rc = timed(tx, cur.rr, &ms))) break;
                if (ms < cur.ms) {
                    cur.tx = tx;
                    cur.ms = ms;
                }
            }
            if (rc) break;
        }
        if (rc) break;
        if (best->threads == 0 || cur.ms < best->ms) *best = cur;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == CX_OK && best->threads == 0) rc = CX_ERR_INTERNAL;
    return rc;
}

std::string tune_signature(const BatchHost& h) {
    int dev = 0;
    cudaDeviceProp prop;
    std::string name = "device";
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    for (char& c : name)
        if (c == '\t' || c == '\n') c = ' ';
    std::map<int, int> hist;
    for (cx_problem* p : h.probs) ++hist[p->d.nx];
    std::string s = name + "|Q" + std::to_string(h.Q) + "|fp" + std::to_string(h.esz * 8) + "|";
    for (const auto& kv : hist) s += std::to_string(kv.first) + ":" + std::to_string(kv.second) + ",";
    return s;
}

std::vector<std::string> split_tabs(const std::string& line) {
    std::vector<std::string> f;
    size_t a = 0;
    for (;;) {
        const size_t b = line.find('\t', a);
        f.push_back(line.substr(a, b == std::string::npos ? std::string::npos : b - a));
        if (b == std::string::npos) break;
        a = b + 1;
    }
    return f;
}

// The cached choice for this signature, if the file has one that is
// admissible for every size class of the batch.
bool cache_lookup(const char* path, const std::string& sig, const BatchHost& h, TuneChoice* c) {
    std::ifstream in(path);
    std::string line;
    while (in && std::getline(in, line)) {
        const std::vector<std::string> f = split_tabs(line);
        if (f.size() != 4 || f[0] != sig) continue;
        TuneChoice t;
        t.threads = std::atoi(f[1].c_str());
        t.ms = std::atof(f[3].c_str());
        size_t a = 0;
        while (a < f[2].size()) {
            size_t b = f[2].find(',', a);
            if (b == std::string::npos) b = f[2].size();
            int nx = 0, tx = 0, r = 0;
            if (std::sscanf(f[2].substr(a, b - a).c_str(), "%d:%d:%d", &nx, &tx, &r) == 3) {
                t.tx[nx] = tx;
                t.rr[nx] = r;
            }
            a = b + 1;
        }
        if (t.threads != 128 && t.threads != 256) continue;
        bool ok = true;
        for (cx_problem* p : h.probs) {
            const int nx = p->d.nx;
            ok = ok && t.tx.count(nx) && t.rr.count(nx) && tune_admissible(t.threads, nx, t.tx[nx]) &&
                 (t.tx[nx] & (t.tx[nx] - 1)) == 0 && t.tx[nx] >= 32 && t.rr[nx] >= 1 && t.rr[nx] <= 32;
        }
        if (!ok) continue;
        *c = t;
        return true;
    }
    return false;
}

bool cache_store(const char* path, const std::string& sig, const TuneChoice& c) {
    std::vector<std::string> keep;
    {
        std::ifstream in(path);
        std::string line;
        while (in && std::getline(in, line))
            if (!line.empty() && split_tabs(line)[0] != sig) keep.push_back(line);
    }
    std::string entry = sig + "\t" + std::to_string(c.threads) + "\t";
    bool first = true;
    for (const auto& kv : c.tx) {
        if (!first) entry += ",";
        first = false;
        entry += std::to_string(kv.first) + ":" + std::to_string(kv.second) + ":" + std::to_string(c.rr.at(kv.first));
    }
    char ms[64];
    std::snprintf(ms, sizeof ms, "%.6f", c.ms);
    entry += "\t";
    entry += ms;
    keep.push_back(entry);
    const std::string tmp = std::string(path) + ".tmp";
    {
        std::ofstream out(tmp, std::ios::trunc);
        for (const std::string& l : keep) out << l << "\n";
        out.flush();
        if (!out) return false;
    }
    return std::rename(tmp.c_str(), path) == 0;
}

} // namespace

extern "C" {

cx_status cx_batch_workspace_size(const cx_problem_desc* descs, int count, size_t* bytes) {
    if (!bytes) return CX_ERR_INVALID_ARG;
    size_t toff = 0;
    return batch_layout(descs, count, nullptr, &toff, bytes);
}

cx_status cx_batch_set_tiles(cx_batch* b, int threads, int blocks, const int* tile_x, const int* rows) {
    if (!b || (threads != 128 && threads != 256) || blocks < 0) return CX_ERR_INVALID_ARG;
    BatchHost& h = b->h;
    std::vector<int> tx(h.count), rr(h.count);
    for (int i = 0; i < h.count; ++i) {
        const int t = tile_x ? tile_x[i] : std::min(threads, 256);
        if (t < 32 || t > threads || threads % t != 0 || threads / t > 8 || (t & (t - 1))) return CX_ERR_INVALID_ARG;
        const int r = rows ? rows[i] : 2;
        if (r < 1 || r > 32) return CX_ERR_INVALID_ARG;
        tx[i] = t;
        rr[i] = r;
    }
    h.threads = threads;
    h.tx = tx;
    h.rr = rr;
    const int occ = h.esz == 8 ? forward_occupancy<double>(h.Q, threads) : forward_occupancy<float>(h.Q, threads);
    h.blocks = blocks > 0 ? blocks : h.probs[0]->nsm * occ;
    set_rows_blocks(h, threads, blocks);
    drop_graphs(h);
    return h.esz == 8 ? upload_table<double>(h) : upload_table<float>(h);
}

cx_status cx_batch_create(const cx_problem_desc* descs, int count, void* workspace, size_t bytes, cudaStream_t stream,
                          cx_batch** out) {
    if (!out) return CX_ERR_INVALID_ARG;
    *out = nullptr;
    std::vector<size_t> offs;
    size_t toff = 0, total = 0;
    cx_status rc = batch_layout(descs, count, &offs, &toff, &total);
    if (rc) return rc;
    if (!workspace || bytes < total || reinterpret_cast<uintptr_t>(workspace) % ALIGN) return CX_ERR_WORKSPACE;
    cx_batch* b = new (std::nothrow) cx_batch();
    if (!b) return CX_ERR_INTERNAL;
    BatchHost& h = b->h;
    h.count = count;
    h.ws = static_cast<char*>(workspace);
    h.stream = stream;
    h.Q = descs[0].lattice;
    h.N = descs[0].n_steps;
    h.k = descs[0].ckpt_every > 0 ? std::min(descs[0].ckpt_every, h.N) : h.N;
    h.S = (h.N + h.k - 1) / h.k;
    h.esz = descs[0].precision == 64 ? 8 : 4;
    for (int i = 0; i < count; ++i) {
        cx_problem* p = nullptr;
        size_t pb = 0;
        rc = cx_workspace_size(&descs[i], &pb);
        if (rc == CX_OK) rc = cx_create(&descs[i], h.ws + offs[i], pb, stream, &p);
        if (rc) {
            for (cx_problem* q : h.probs) cx_destroy(q);
            delete b;
            return rc;
        }
        h.probs.push_back(p);
    }
    size_t o = toff;
    h.off_rec = o;
    o = up(o + rec_size(h.esz) * count, ALIGN);
    h.off_tile0 = o;
    o = up(o + sizeof(int) * (count + 1), ALIGN);
    h.off_fin = o;
    o = up(o + sizeof(BFin) * count, ALIGN);
    size_t slots = 0;
    for (int i = 0; i < count; ++i) slots += slot_capacity(descs[i]);
    h.slot_cap = slots;
    h.off_sums = o;
    o = up(o + sizeof(double) * slots, ALIGN);
    h.off_maxs = o;
    o = up(o + sizeof(double) * slots, ALIGN);
    h.off_out = o;
    o = up(o + sizeof(double) * 3 * count, ALIGN);
    h.off_status = o;
    o = up(o + sizeof(int) * 4, ALIGN);
    h.off_active = o;
    o = up(o + sizeof(int) * count, ALIGN);
    h.off_lam = o;
    h.enabled.assign(count, 1);
    h.lam_prev.assign(count, 0.0);
    h.J_at_g.assign(count, 0.0);
    if (cudaMemset(h.ws + h.off_status, 0, sizeof(int) * 4) != cudaSuccess ||
        cudaMemset(h.ws + h.off_lam, 0, sizeof(double) * count) != cudaSuccess ||
        cudaMemcpy(h.ws + h.off_active, h.enabled.data(), sizeof(int) * count, cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        cx_batch_destroy(b);
        return CX_ERR_CUDA;
    }
    rc = cx_batch_set_tiles(b, 256, 0, nullptr, nullptr);
    if (rc) {
        cx_batch_destroy(b);
        return rc;
    }
    *out = b;
    return CX_OK;
}

cx_status cx_batch_set_initial(cx_batch* b, const void* const* u0, const void* const* v0) {
    if (!b || !u0 || !v0) return CX_ERR_INVALID_ARG;
    for (int i = 0; i < b->h.count; ++i) {
        cx_status rc = cx_set_initial(b->h.probs[i], u0[i], v0[i]);
        if (rc) return rc;
    }
    b->h.has_init = true;
    b->h.fwd_at_g = false;
    b->h.lam_prev.assign(b->h.count, 0.0);
    return CX_OK;
}

cx_status cx_batch_bind(cx_batch* b, const void* const* g, void* const* dJdg) {
    if (!b) return CX_ERR_INVALID_ARG;
    BatchHost& h = b->h;
    h.g.assign(h.count, nullptr);
    h.dJdg.assign(h.count, nullptr);
    for (int i = 0; i < h.count; ++i) {
        if (g) h.g[i] = g[i];
        if (dJdg) h.dJdg[i] = dJdg[i];
    }
    h.bound = true;
    h.fwd_at_g = false;
    h.lam_prev.assign(h.count, 0.0);
    drop_graphs(h);
    return h.esz == 8 ? upload_table<double>(h) : upload_table<float>(h);
}

cx_status cx_batch_forward(cx_batch* b, double* J_dev) {
    if (!b) return CX_ERR_INVALID_ARG;
    if (!b->h.has_init || !b->h.bound) return CX_ERR_STATE;
    return b->h.esz == 8 ? run<double>(b->h, false, J_dev) : run<float>(b->h, false, J_dev);
}

cx_status cx_batch_gradient(cx_batch* b, double* out_dev) {
    if (!b) return CX_ERR_INVALID_ARG;
    if (!b->h.has_init || !b->h.bound) return CX_ERR_STATE;
    for (void* p : b->h.dJdg)
        if (!p) return CX_ERR_INVALID_ARG;
    return b->h.esz == 8 ? run<double>(b->h, true, out_dev) : run<float>(b->h, true, out_dev);
}

cx_status cx_batch_set_enabled(cx_batch* b, const int* enabled) {
    if (!b) return CX_ERR_INVALID_ARG;
    BatchHost& h = b->h;
    std::vector<int> e(h.count, 1);
    if (enabled)
        for (int i = 0; i < h.count; ++i) {
            if (!h.enabled[i] && enabled[i]) h.fwd_at_g = false; // its state may be stale
            e[i] = enabled[i] ? 1 : 0;
        }
    h.enabled = e;
    cx_status rc = upload_ints(h, h.off_active, h.enabled);
    if (rc) return rc;
    B_CUDA(cudaStreamSynchronize(h.stream));
    return CX_OK;
}

cx_status cx_batch_adjoint(cx_batch* b, const void* const* seed_u, int add_to_cost_seed, double* out_dev) {
    if (!b) return CX_ERR_INVALID_ARG;
    BatchHost& h = b->h;
    if (!h.has_init || !h.bound) return CX_ERR_STATE;
    if (!h.fwd_at_g) return CX_ERR_STATE; // needs the forward state of the bound controls
    for (void* p : h.dJdg)
        if (!p) return CX_ERR_INVALID_ARG;
    if (seed_u)
        for (int i = 0; i < h.count; ++i) {
            if (!seed_u[i] || !h.enabled[i]) continue;
            cx_problem* p = h.probs[i];
            const size_t n = (size_t)p->d.nx * p->d.ny;
            if (!add_to_cost_seed) {
                B_CUDA(cudaMemcpyAsync(p->ws + p->lay.off_wu, seed_u[i], n * h.esz, cudaMemcpyDeviceToDevice,
                                       h.stream));
            } else {
                const int blocks = (int)std::min<size_t>((n + 255) / 256, 1024);
                if (h.esz == 8)
                    k_add_seed<double><<<blocks, 256, 0, h.stream>>>(p->at<double>(p->lay.off_wu),
                                                                     static_cast<const double*>(seed_u[i]), n);
                else
                    k_add_seed<float><<<blocks, 256, 0, h.stream>>>(p->at<float>(p->lay.off_wu),
                                                                    static_cast<const float*>(seed_u[i]), n);
                B_CUDA(cudaGetLastError());
            }
        }
    cx_status rc = h.esz == 8 ? run_graph<double>(h, G_ADJ) : run_graph<float>(h, G_ADJ);
    if (rc) return rc;
    // the terminal seeds now hold seed_u and the recompute overwrote the tape:
    // the next step or gradient starts with a full forward
    h.fwd_at_g = false;
    if (out_dev)
        B_CUDA(cudaMemcpyAsync(out_dev + h.count, h.ws + h.off_out + sizeof(double) * h.count,
                               sizeof(double) * 2 * h.count, cudaMemcpyDeviceToDevice, h.stream));
    return CX_OK;
}

cx_status cx_batch_prepare(cx_batch* b) {
    if (!b) return CX_ERR_INVALID_ARG;
    BatchHost& h = b->h;
    if (!h.bound) return CX_ERR_STATE;
    for (int mode = 0; mode < 4; ++mode) {
        if (h.graphs[mode]) continue;
        bool have_E = !h.dJdg.empty();
        for (void* e : h.dJdg) have_E = have_E && e;
        if (mode != G_FWD && !have_E) continue; // gradient, trial and adjoint graphs read dJdg
        cx_status rc = h.esz == 8 ? capture<double>(h, mode, &h.graphs[mode]) : capture<float>(h, mode, &h.graphs[mode]);
        if (rc) return rc;
    }
    return CX_OK;
}

cx_status cx_batch_axpy(cx_batch* b, const double* lam) {
    if (!b || !lam) return CX_ERR_INVALID_ARG;
    BatchHost& h = b->h;
    if (!h.bound) return CX_ERR_STATE;
    std::vector<double> l(h.count, 0.0);
    for (int i = 0; i < h.count; ++i) {
        if (!std::isfinite(lam[i])) return CX_ERR_INVALID_ARG;
        if (!h.enabled[i] || lam[i] == 0.0) continue;
        if (!h.g[i] || !h.dJdg[i]) return CX_ERR_INVALID_ARG;
        l[i] = lam[i];
    }
    cx_status rc = upload_lam(h, l);
    if (rc) return rc;
    if (h.esz == 8)
        k_baxpy<double><<<dim3(64, h.count), 256, 0, h.stream>>>(
            reinterpret_cast<const BRec<double>*>(h.ws + h.off_rec), h.count,
            reinterpret_cast<const double*>(h.ws + h.off_lam));
    else
        k_baxpy<float><<<dim3(64, h.count), 256, 0, h.stream>>>(
            reinterpret_cast<const BRec<float>*>(h.ws + h.off_rec), h.count,
            reinterpret_cast<const float*>(h.ws + h.off_lam));
    B_CUDA(cudaGetLastError());
    h.fwd_at_g = false;
    h.lam_prev.assign(h.count, 0.0);
    return CX_OK;
}

cx_status cx_batch_step(cx_batch* b, cx_step_info* info, int* status) {
    if (!b) return CX_ERR_INVALID_ARG;
    BatchHost& h = b->h;
    if (!h.has_init || !h.bound) return CX_ERR_STATE;
    for (int i = 0; i < h.count; ++i)
        if (!h.g[i] || !h.dJdg[i]) return CX_ERR_INVALID_ARG;
    return h.esz == 8 ? batch_step<double>(h, info, status) : batch_step<float>(h, info, status);
}

cx_status cx_batch_get_fields(cx_batch* b, int i, void* u_out, void* v_out) {
    if (!b || i < 0 || i >= b->h.count) return CX_ERR_INVALID_ARG;
    return cx_get_fields(b->h.probs[i], u_out, v_out);
}

cx_status cx_batch_get_status(cx_batch* b) {
    if (!b) return CX_ERR_INVALID_ARG;
    int st = 0;
    if (cudaMemcpyAsync(&st, b->h.ws + b->h.off_status, sizeof(int), cudaMemcpyDeviceToHost, b->h.stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->h.stream) != cudaSuccess)
        return CX_ERR_CUDA;
    if (st & ST_TIMEOUT) return CX_ERR_TIMEOUT;
    return (st & ST_UNSTABLE) ? CX_ERR_UNSTABLE : CX_OK;
}

cx_status cx_batch_autotune(cx_batch* b, int probe_steps, const char* cache_path, int* threads_out,
                            int* tile_x_out, int* rows_out, double* probe_ms_out) {
    if (!b || probe_steps < 1) return CX_ERR_INVALID_ARG;
    BatchHost& h = b->h;
    if (!h.has_init || !h.bound) return CX_ERR_STATE;
    for (void* p : h.dJdg)
        if (!p) return CX_ERR_STATE;
    const std::string sig = tune_signature(h);
    TuneChoice c;
    const bool cached = cache_path && cache_lookup(cache_path, sig, h, &c);
    cx_status rc = CX_OK;
    if (!cached) {
        drop_graphs(h);
        {
            ScheduleGuard guard(h, probe_steps);
            rc = h.esz == 8 ? tune_search<double>(h, &c) : tune_search<float>(h, &c);
        }
        // the probe overwrote checkpoints past the first, the tapes and the populations
        h.fwd_at_g = false;
        h.J_on_device = false;
        for (cx_problem* p : h.probs) {
            p->fwd_valid = false;
            p->adj_valid = false;
            p->tape_last_valid = false;
        }
        if (rc) return rc;
    }
    B_CUDA(cudaStreamSynchronize(h.stream));
    std::vector<int> tx(h.count), rr(h.count);
    for (int i = 0; i < h.count; ++i) {
        tx[i] = c.tx.at(h.probs[i]->d.nx);
        rr[i] = c.rr.at(h.probs[i]->d.nx);
    }
    rc = cx_batch_set_tiles(b, c.threads, 0, tx.data(), rr.data());
    if (rc) return rc;
    if (threads_out) *threads_out = c.threads;
    if (tile_x_out) std::copy(tx.begin(), tx.end(), tile_x_out);
    if (rows_out) std::copy(rr.begin(), rr.end(), rows_out);
    if (probe_ms_out) *probe_ms_out = c.ms;
    if (!cached && cache_path && !cache_store(cache_path, sig, c)) return CX_ERR_INTERNAL;
    return CX_OK;
}

cx_status cx_batch_set_staging(cx_batch* b, int row_windows) {
    if (!b || (row_windows != 0 && row_windows != 1)) return CX_ERR_INVALID_ARG;
    if (b->h.row_windows != row_windows) drop_graphs(b->h);
    b->h.row_windows = row_windows;
    return CX_OK;
}

cx_status cx_batch_destroy(cx_batch* b) {
    if (!b) return CX_ERR_INVALID_ARG;
    drop_graphs(b->h);
    for (cx_problem* p : b->h.probs) cx_destroy(p);
    delete b;
    return CX_OK;
}

} // extern "C"
