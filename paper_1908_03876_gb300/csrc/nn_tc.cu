// nn_tc.cu -- 3x3 / 1x1 convolution forward on the 5th-generation tensor cores
// (tcgen05.mma, FP32 accumulators in tensor memory), for the warm-start
// surrogate's layers with 32..256 output channels.
//
// A CTA owns a 16 x 8 pixel tile of one image (M = 128 rows of the MMA) and N
// output channels (N = 32, 64, 128 or 256), and loops over the input channels
// in chunks of 16 (K = 16 per MMA).  Per chunk all threads stage
//   A: the (16+2) x (8+2) input patch, channel-interleaved as
//      [ci/8][patch position][8 ci] -- every 8 consecutive pixels of a patch
//      row form one 8 x 16-byte core matrix, so the operand of tap (dy, dx) is
//      the same buffer at byte offset (dy * 10 + dx) * 16 with core-matrix
//      strides 16 * 10 (next image row, M direction) and 16 * 180 (next 8
//      channels, K direction);
//   B: the chunk's weights of every tap as [tap][ci/8][oc][8 ci], core-matrix
//      strides 128 (next 8 channels out, N direction) and 16 * N (K direction)
//      -- the layout of the weight pack, so when the tile covers every output
//      channel the chunk arrives in one bulk asynchronous copy completed on
//      the buffer's load mbarrier;
// then one thread issues the 9 (or 1) MMAs of the chunk and commits them to
// the chunk buffer's MMA mbarrier.  Two buffers: staging chunk c+1 overlaps the
// MMAs of chunk c.  The epilogue reads the accumulator lanes of each warp
// (pixels 32 w .. 32 w + 31) with tcgen05.ld and applies bias and ReLU.
// Every mbarrier wait is bounded; on timeout the kernel sets *status, skips
// its stores, waits (bounded) for its own MMAs and frees its tensor memory.
#include <algorithm>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/cxlbm.h"

namespace nntc {

typedef __nv_bfloat16 bf16;

constexpr int NTHR = 128;
constexpr int TM = 128;        // MMA M: pixels per tile
constexpr int TH = 16, TW = 8; // tile rows x columns
constexpr unsigned WAIT_LIMIT = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared memory matrix descriptor, no swizzle, K-major core matrices of 8 rows x 16 bytes
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor: kind::f16, BF16 x BF16 -> FP32, both operands K-major, M = 128
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for the phase of the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    for (unsigned it = 0; it < WAIT_LIMIT; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// one bulk global -> shared copy (16-byte aligned, size a multiple of 16), completion on bar
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

template <int KS> struct TcGeom {
    static constexpr int PH = TH + KS - 1, PW = TW + KS - 1, PP = PH * PW, TAPS = KS * KS;
    static constexpr int A_BYTES = 2 * PP * 16;
    __host__ __device__ static constexpr int b_bytes(int n) { return TAPS * 2 * n * 16; }
    __host__ __device__ static constexpr int buf_bytes(int n) { return ((A_BYTES + b_bytes(n)) + 127) / 128 * 128; }
    __host__ __device__ static constexpr int smem_bytes(int n) { return 2 * buf_bytes(n) + 128; } // + 4 barriers
};

// Wp: the forward pack [ceil(IC/16)][taps][OC][16] (cx_nn_pack_weights)
template <int KS>
__global__ void __launch_bounds__(NTHR) k_conv_tc(const bf16* __restrict__ X, const bf16* __restrict__ Wp,
                                                  const float* __restrict__ bias, bf16* __restrict__ Y, int B,
                                                  int IC, int OC, int H, int W, int N, int relu, int* status) {
    using Gm = TcGeom<KS>;
    constexpr int PW = Gm::PW, PP = Gm::PP, TAPS = Gm::TAPS, OFF = KS / 2;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int bufb = Gm::buf_bytes(N);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * bufb); // MMAs of a buffer done
    uint64_t* lbar = mbar + 2;                                        // bulk weight copy of a buffer landed
    uint32_t* taddr_sh = reinterpret_cast<uint32_t*>(mbar + 4);
    int* abort_sh = reinterpret_cast<int*>(mbar + 5);
    const bool bulk = (N == OC); // the chunk's weight block is contiguous in the pack
    const uint32_t b_bytes = (uint32_t)Gm::b_bytes(N);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = (W + TW - 1) / TW, tiles_y = (H + TH - 1) / TH;
    int bt = blockIdx.x;
    const int b = bt / (tiles_x * tiles_y);
    bt -= b * tiles_x * tiles_y;
    const int y0 = (bt / tiles_x) * TH, x0 = (bt % tiles_x) * TW;
    const int oc0 = blockIdx.y * N;
    const size_t hw = (size_t)H * W;
    const bf16 zero = __float2bfloat16(0.0f);

    if (warp == 0) tmem_alloc(taddr_sh, (uint32_t)N);
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_init(&lbar[0], 1);
        mbar_init(&lbar[1], 1);
        *abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); // visible to the async proxy
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *taddr_sh;
    const uint32_t idesc = idesc_bf16(N);
    const int nchunks = (IC + 15) / 16;
    bool ok = true;
    int n_copy[2] = {0, 0}, n_commit[2] = {0, 0}; // thread 0: operations issued per buffer
    for (int c = 0; c < nchunks && ok; ++c) {
        const int buf = c & 1;
        unsigned char* A = smem + buf * bufb;
        unsigned char* Bm = A + Gm::A_BYTES;
        if (c >= 2) {
            ok = mbar_wait(&mbar[buf], (unsigned)(((c - 2) >> 1) & 1)); // MMAs of chunk c-2 done
            ok = __syncthreads_and(ok && !*abort_sh) != 0;                 // the same decision in every thread
            if (!ok) break;
        }
        if (bulk && tid == 0) {
            mbar_expect_tx(&lbar[buf], b_bytes);
            bulk_copy(Bm, Wp + (size_t)c * TAPS * 2 * OC * 8, b_bytes, &lbar[buf]);
            ++n_copy[buf];
        }
        // A: [ci/8][pos][8].  One thread per (8-channel group, patch position): eight
        // loads from the channel planes (coalesced along x across the warp), one
        // 16-byte store of the position's core-matrix row (no bank conflicts)
        for (int e = tid; e < 2 * PP; e += NTHR) {
            const int gq = e / PP, r = e - gq * PP;
            const int py = r / PW, px = r - py * PW;
            const int y = y0 - OFF + py, x = x0 - OFF + px;
            const bool inb = y >= 0 && y < H && x >= 0 && x < W;
            const int ic0 = c * 16 + gq * 8;
            const bf16* src = X + ((size_t)b * IC + ic0) * hw + (size_t)(inb ? y : 0) * W + (inb ? x : 0);
            uint32_t wv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bf16 lo = (inb && ic0 + 2 * q < IC) ? src[(size_t)(2 * q) * hw] : zero;
                const bf16 hi = (inb && ic0 + 2 * q + 1 < IC) ? src[(size_t)(2 * q + 1) * hw] : zero;
                wv[q] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
            }
            reinterpret_cast<uint4*>(A)[gq * PP + r] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
        // B: [tap][ci/8][oc][8] (thread copies when the tile is a part of the output channels)
        if (!bulk)
            for (int e = tid; e < TAPS * N * 2; e += NTHR) {
                const int th = e / N, o = e - th * N; // th = tap * 2 + h
                uint4 v = make_uint4(0, 0, 0, 0);
                if (oc0 + o < OC)
                    v = *reinterpret_cast<const uint4*>(Wp + (((size_t)c * TAPS * 2 + th) * OC + oc0 + o) * 8);
                *reinterpret_cast<uint4*>(Bm + ((size_t)th * N + o) * 16) = v;
            }
        proxy_fence(); // generic-proxy writes visible to the tensor cores
        __syncthreads();
        if (tid == 0 && bulk && !mbar_wait(&lbar[buf], (unsigned)((c >> 1) & 1))) *abort_sh = 1;
        if (tid == 0 && !*abort_sh) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(A), b0 = smem_u32(Bm);
#pragma unroll
            for (int t = 0; t < TAPS; ++t) {
                const int dy = t / KS, dx = t - dy * KS;
                const uint64_t ad = sdesc(a0 + (uint32_t)((dy * PW + dx) * 16), PP * 16, PW * 16);
                const uint64_t bd = sdesc(b0 + (uint32_t)(t * 2 * N * 16), N * 16, 128);
                mma_bf16(taddr, ad, bd, idesc, (c > 0 || t > 0) ? 1u : 0u);
            }
            mma_commit(&mbar[buf]);
            ++n_commit[buf];
        }
    }
    // the last commit covers every MMA issued before it
    const int last = nchunks - 1;
    __syncthreads();
    if (ok && !*abort_sh) ok = mbar_wait(&mbar[last & 1], (unsigned)((last >> 1) & 1));
    ok = __syncthreads_and(ok && !*abort_sh) != 0;
    tc_fence_after();
    if (!ok) {
        if (tid == 0) {
            if (status) atomicOr(status, 1);
            // bounded waits for copies and MMAs still in flight before the memory is freed
            for (int q = 0; q < 2; ++q) {
                if (n_copy[q] > 0) mbar_wait(&lbar[q], (unsigned)((n_copy[q] - 1) & 1));
                if (n_commit[q] > 0) mbar_wait(&mbar[q], (unsigned)((n_commit[q] - 1) & 1));
            }
        }
        __syncthreads();
    } else {
        const int m = warp * 32 + lane;
        const int y = y0 + m / TW, x = x0 + m % TW;
        const bool in = y < H && x < W;
        for (int col = 0; col < N; col += 32) {
            float v[32];
            tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)col, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int o = oc0 + col + j;
                if (!in || o >= OC) continue;
                float r = v[j] + (bias ? bias[o] : 0.0f);
                if (relu) r = fmaxf(r, 0.0f);
                Y[((size_t)b * OC + o) * hw + (size_t)y * W + x] = __float2bfloat16(r);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, (uint32_t)N);
}

// ------------------------------------------------------------ weight gradient
// dW[oc][ic][tap] = sum over pixels of dY[oc][p] X[ic][p + tap] as a GEMM on
// the tensor cores: D[M = 128 output channels][N = 144 = 16 input channels x
// 9 taps], K = pixels, 64 per chunk (one 8 x 8 pixel tile).  Both operands
// K-major (8 consecutive pixels of one tile row per 16-byte core-matrix row):
//   A (dY): core matrix (output-channel group g, tile row r) at (g * 8 + r) * 128 bytes;
//   B (X shifted by the tap): row n = ic_local * 9 + tap, core matrix
//       (n / 8, r) at (n / 8 * 8 + r) * 128.
// Pipeline per chunk j (two buffers): the dY rows and the raw input patch
// (10 patch rows x 16 channels x 24 pixels: the tile row with 8 pixels on each
// side, three aligned 16-byte pieces) of chunk j+1 are copied by cp.async while
// chunk j is built and multiplied; building materialises the tap shifts (the
// x-shifted rows by a 16-bit funnel shift) from the raw patch in shared
// memory; one thread issues the four MMAs (K = 16) and commits them to the
// buffer's mbarrier, which the copies into that buffer two chunks later wait
// on.  Rows of output channels >= OC are zeroed once and never copied.
// Accumulator: 144 of 256 allocated tensor-memory columns, lane = output
// channel.  Output: the split's partial sums partial[z][OC][IC * 9] (columns
// of chunk c contiguous), summed over splits afterwards; the blocks of the
// first input chunk also sum dY per output channel (bias gradient) from the
// staged rows.
constexpr int WG_N = 144;
constexpr int WG_A_BYTES = 16 * 8 * 128; // 128 output channels x 64 pixels
constexpr int WG_B_BYTES = 18 * 8 * 128; // 144 rows x 64 pixels
constexpr int WG_P_BYTES = 16 * 10 * 48; // raw patch: 10 rows x 16 channels x 24 pixels
constexpr int WG_BUF = WG_A_BYTES + WG_B_BYTES + WG_P_BYTES;
constexpr int WG_SMEM = 2 * WG_BUF + 64;

__device__ __forceinline__ void cp16(void* dst, const void* src, bool valid) {
    // 16-byte cp.async; src_size 0 fills the destination with zeros
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int NPEND> __device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(NPEND) : "memory");
}

__global__ void __launch_bounds__(NTHR) k_wgrad_tc(const bf16* __restrict__ X, const bf16* __restrict__ dY,
                                                   float* __restrict__ partial, float* __restrict__ bpart, int B,
                                                   int IC, int OC, int H, int W, int tps, int* status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * WG_BUF); // MMAs of a buffer done
    uint32_t* taddr_sh = reinterpret_cast<uint32_t*>(mbar + 2);
    int* abort_sh = reinterpret_cast<int*>(mbar + 3);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int c = blockIdx.x, oc0 = blockIdx.y * 128;
    const int tx = W >> 3, ty = H >> 3, ntiles = B * tx * ty;
    const int t_beg = blockIdx.z * tps, t_end = min(ntiles, t_beg + tps);
    const int nch = t_end > t_beg ? t_end - t_beg : 0;
    const size_t hw = (size_t)H * W;
    const size_t NC = (size_t)IC * 9;
    const bool bias = (c == 0) && bpart;
    const int noc = min(128, OC - oc0); // real output channels of this tile

    if (warp == 0) tmem_alloc(taddr_sh, 256u);
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        *abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    // A rows of output channels beyond OC: zero in both buffers, once
    for (int e = tid; e < 2 * (128 - noc) * 8; e += NTHR) {
        const int bufz = e / ((128 - noc) * 8), q = e - bufz * (128 - noc) * 8;
        const int o = noc + (q >> 3), r = q & 7;
        *reinterpret_cast<uint4*>(smem + bufz * WG_BUF + ((o >> 3) * 8 + r) * 128 + (o & 7) * 16) =
            make_uint4(0, 0, 0, 0);
    }
    // copies of chunk j into buffer j & 1: dY rows of the real output
    // channels, and the raw patch (zero outside the image / beyond IC)
    auto issue = [&](int j) {
        unsigned char* A = smem + (j & 1) * WG_BUF;
        unsigned char* P = A + WG_A_BYTES + WG_B_BYTES;
        const int tile = t_beg + j;
        const int b = tile / (tx * ty), bt = tile - b * tx * ty;
        const int y0 = (bt / tx) * 8, x0 = (bt % tx) * 8;
        for (int e = tid; e < noc * 8; e += NTHR) { // channel fastest: 16-byte rows of a core matrix, no bank conflict
            const int r = e / noc, o = e - r * noc;
            cp16(A + ((o >> 3) * 8 + r) * 128 + (o & 7) * 16,
                 dY + ((size_t)b * OC + oc0 + o) * hw + (size_t)(y0 + r) * W + x0, true);
        }
        for (int e = tid; e < 16 * 10 * 3; e += NTHR) {
            const int row = e / 3, piece = e - row * 3; // row = py * 16 + icl
            const int py = row >> 4, icl = row & 15;
            const int ic = c * 16 + icl, yy = y0 - 1 + py, xs = x0 - 8 + piece * 8;
            const bool ok = ic < IC && yy >= 0 && yy < H && xs >= 0 && xs < W;
            const bf16* src = ok ? X + ((size_t)b * IC + ic) * hw + (size_t)yy * W + xs : X;
            cp16(P + row * 48 + piece * 16, src, ok);
        }
        cp_commit();
    };
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *taddr_sh;
    const uint32_t idesc = idesc_bf16(WG_N);
    float bs = 0.0f; // bias: thread t < 128 sums output channel oc0 + t
    bool ok = true;
    int n_commit[2] = {0, 0};
    if (nch > 0) issue(0);
    for (int j = 0; j < nch && ok; ++j) {
        const int buf = j & 1;
        unsigned char* A = smem + buf * WG_BUF;
        unsigned char* Bm = A + WG_A_BYTES;
        const unsigned char* P = Bm + WG_B_BYTES;
        if (j + 1 < nch) {
            if (j >= 1) { // buffer (j+1)&1 held chunk j-1: its MMAs must be done
                ok = mbar_wait(&mbar[(j + 1) & 1], (unsigned)(((j - 1) >> 1) & 1));
                ok = __syncthreads_and(ok && !*abort_sh) != 0;
                if (!ok) break;
            }
            issue(j + 1);
            cp_wait<1>(); // this thread's copies of chunk j have landed
        } else {
            cp_wait<0>();
        }
        __syncthreads(); // every thread's copies of chunk j are visible
        if (bias && tid < noc) { // dY of output channel oc0 + tid over the tile
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const uint4 v = *reinterpret_cast<const uint4*>(A + ((tid >> 3) * 8 + r) * 128 + (tid & 7) * 16);
                const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) bs += __uint_as_float(w4[h] << 16) + __uint_as_float(w4[h] & 0xFFFF0000u);
            }
        }
        // B: the tap-shifted rows from the raw patch
        // (input channel fastest across the warp: the eight 16-byte rows of a
        // core matrix land in distinct banks)
        for (int e = tid; e < 16 * 10; e += NTHR) {
            const int py = e >> 4, icl = e & 15;
            const uint4* pr = reinterpret_cast<const uint4*>(P + e * 48);
            const uint4 v0 = pr[0], v1 = pr[1], v2 = pr[2];
            // pixels x0 - 1 + dx + q, q = 0..7: dx = 1 is v1; dx = 0 and 2 shift by one bf16 (16 bits)
            const uint4 s0 = make_uint4(__byte_perm(v0.w, v1.x, 0x5432), __byte_perm(v1.x, v1.y, 0x5432),
                                        __byte_perm(v1.y, v1.z, 0x5432), __byte_perm(v1.z, v1.w, 0x5432));
            const uint4 s2 = make_uint4(__byte_perm(v1.x, v1.y, 0x5432), __byte_perm(v1.y, v1.z, 0x5432),
                                        __byte_perm(v1.z, v1.w, 0x5432), __byte_perm(v1.w, v2.x, 0x5432));
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) {
                const int r = py - dy;
                if (r < 0 || r > 7) continue;
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const int n = icl * 9 + dy * 3 + dx;
                    *reinterpret_cast<uint4*>(Bm + ((n >> 3) * 8 + r) * 128 + (n & 7) * 16) =
                        dx == 0 ? s0 : (dx == 1 ? v1 : s2);
                }
            }
        }
        proxy_fence(); // generic-proxy writes (and the landed copies) visible to the tensor cores
        __syncthreads();
        if (tid == 0 && !*abort_sh) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(A), b0 = smem_u32(Bm);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint64_t ad = sdesc(a0 + (uint32_t)(2 * kk * 128), 128, 1024);
                const uint64_t bd = sdesc(b0 + (uint32_t)(2 * kk * 128), 128, 1024);
                mma_bf16(taddr, ad, bd, idesc, (j > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(&mbar[buf]);
            ++n_commit[buf];
        }
    }
    cp_wait<0>(); // no copy in flight when the block leaves (also after an abort)
    __syncthreads();
    if (ok && nch > 0 && !*abort_sh) {
        const int last = nch - 1;
        ok = mbar_wait(&mbar[last & 1], (unsigned)((last >> 1) & 1));
    }
    ok = __syncthreads_and(ok && !*abort_sh) != 0;
    tc_fence_after();
    if (!ok) {
        if (tid == 0) {
            if (status) atomicOr(status, 1);
            for (int q = 0; q < 2; ++q)
                if (n_commit[q] > 0) mbar_wait(&mbar[q], (unsigned)((n_commit[q] - 1) & 1));
        }
        __syncthreads();
    } else {
        const int oc = oc0 + warp * 32 + lane;
        float* dst = partial + ((size_t)blockIdx.z * OC + oc) * NC + (size_t)c * WG_N;
        const int ncols = min(WG_N, (IC - c * 16) * 9); // columns of real input channels
        for (int col = 0; col < WG_N; col += 32) {
            float v[32];
            tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)col, v);
            if (oc >= OC) continue;
#pragma unroll
            for (int q = 0; q < 32; ++q)
                if (col + q < ncols) dst[col + q] = nch > 0 ? v[q] : 0.0f;
        }
        if (bias && tid < noc) bpart[(size_t)blockIdx.z * OC + oc0 + tid] = bs;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, 256u);
}

// out[i] = sum over z of part[z][i], in z order
__global__ void k_sum_splits(const float* __restrict__ part, float* __restrict__ out, int splits, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int z = 0; z < splits; ++z) s += part[(size_t)z * n + i];
        out[i] = s;
    }
}

} // namespace nntc

using namespace nntc;

extern "C" {

int cx_nn_conv_tc_tile(int Cout) {
    for (int n = 256; n >= 32; n >>= 1)
        if (Cout % n == 0) return n;
    return 0;
}

cx_status cx_nn_conv_forward_tc(const uint16_t* x, const uint16_t* w_fwd, const float* bias, uint16_t* y, int B,
                                int Cin, int Cout, int H, int W, int ks, int relu, int* status, cudaStream_t stream) {
    if (!x || !w_fwd || !y || B < 1 || Cin < 1 || H < 1 || W < 1 || (ks != 1 && ks != 3)) return CX_ERR_INVALID_ARG;
    const int N = cx_nn_conv_tc_tile(Cout);
    if (N == 0) return CX_ERR_INVALID_ARG;
    const long long tiles = (long long)B * ((H + TH - 1) / TH) * ((W + TW - 1) / TW);
    if (tiles > 0x7fffffffLL) return CX_ERR_INVALID_ARG;
    dim3 grid((unsigned)tiles, Cout / N);
    const bf16* X = reinterpret_cast<const bf16*>(x);
    const bf16* Wp = reinterpret_cast<const bf16*>(w_fwd);
    bf16* Y = reinterpret_cast<bf16*>(y);
    if (ks == 3) {
        const int smem = TcGeom<3>::smem_bytes(N);
        if (cudaFuncSetAttribute(k_conv_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess)
            return CX_ERR_CUDA;
        k_conv_tc<3><<<grid, NTHR, smem, stream>>>(X, Wp, bias, Y, B, Cin, Cout, H, W, N, relu, status);
    } else {
        const int smem = TcGeom<1>::smem_bytes(N);
        if (cudaFuncSetAttribute(k_conv_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess)
            return CX_ERR_CUDA;
        k_conv_tc<1><<<grid, NTHR, smem, stream>>>(X, Wp, bias, Y, B, Cin, Cout, H, W, N, relu, status);
    }
    return cudaGetLastError() == cudaSuccess ? CX_OK : CX_ERR_CUDA;
}


cx_status cx_nn_conv_backward_weight_tc(const uint16_t* x, const uint16_t* dy, float* dw, float* db, float* scratch,
                                        int splits, int B, int Cin, int Cout, int H, int W, int ks, int* status,
                                        cudaStream_t stream) {
    if (!x || !dy || !dw || !scratch || ks != 3 || B < 1 || Cin < 1 || Cout < 1 || H < 8 || W < 8 || H % 8 ||
        W % 8 || splits < 1 || splits > 65535)
        return CX_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(x) & 15u) || (reinterpret_cast<uintptr_t>(dy) & 15u)) return CX_ERR_INVALID_ARG;
    const long long ntiles = (long long)B * (H / 8) * (W / 8);
    if (ntiles > 0x7fffffffLL) return CX_ERR_INVALID_ARG;
    const int tps = (int)((ntiles + splits - 1) / splits);
    dim3 grid((Cin + 15) / 16, (Cout + 127) / 128, splits);
    if (cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, WG_SMEM) != cudaSuccess)
        return CX_ERR_CUDA;
    const size_t mn = (size_t)Cout * Cin * 9;
    float* bpart = scratch + (size_t)splits * mn;
    k_wgrad_tc<<<grid, NTHR, WG_SMEM, stream>>>(reinterpret_cast<const bf16*>(x), reinterpret_cast<const bf16*>(dy),
                                                 scratch, db ? bpart : nullptr, B, Cin, Cout, H, W, tps, status);
    if (cudaGetLastError() != cudaSuccess) return CX_ERR_CUDA;
    auto blocks = [](size_t n) { return (unsigned)std::min<size_t>((n + 255) / 256, 152 * 8); };
    k_sum_splits<<<blocks(mn), 256, 0, stream>>>(scratch, dw, splits, mn);
    if (db) k_sum_splits<<<blocks((size_t)Cout), 256, 0, stream>>>(bpart, db, splits, (size_t)Cout);
    return cudaGetLastError() == cudaSuccess ? CX_OK : CX_ERR_CUDA;
}

} // extern "C"
