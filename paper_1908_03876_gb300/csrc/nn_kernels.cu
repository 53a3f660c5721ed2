// nn_kernels.cu -- kernels of the warm-start surrogate (a small convolutional
// U-Net that proposes the initial control).  BF16 weights and activations,
// FP32 accumulation, on the tensor cores through mma.sync m16n8k16.
//
// Convolutions (3x3 with zero padding 1, or 1x1) are direct: a block owns 64
// output channels x one 8x8 pixel tile of one image and loops over the input
// channels in chunks of 16.  Per chunk it stages the input patch (8+2)^2 x 16
// channel-last in shared memory once and reuses it for all 9 taps, with the
// chunk's weights pre-packed as [chunk][tap][out][16]:
//   forward        Y[b,o,p] = bias[o] + sum_{c,t} W[o,c,t] X[b,c,p+t]
//   data gradient  the same kernel on dY with the flipped, transposed pack
//   weight grad.   dW[o,c,t] = sum_{b,p} dY[b,o,p] X[b,c,p+t]: a block owns
//                  64 outputs x 16 inputs x 9 taps and loops over pixel tiles
//                  (split over blocks into FP32 partials reduced in a fixed
//                  order); the patch is staged twice (aligned and shifted by
//                  one column) so every fragment load is a 32-bit pair.
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/cxlbm.h"

namespace nn {

typedef __nv_bfloat16 bf16;

constexpr int NTHR = 128;
constexpr int CT = 64;  // output channels per block
constexpr int KC = 16;  // input channels per chunk
constexpr int KCP = 24; // padded channel stride of a staged pixel (halfs): conflict-free fragment loads

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// Weight packs, [c][t][h][o][8] with input channel 16c + 8h + jj:
// forward Wf = W[o][in][t] (out = Cout, in = Cin); data gradient
// Wb = W[in][o][taps-1-t] (out = Cin, in = Cout).  One chunk c is a
// contiguous [taps][2][out][8] block: the tensor-core kernel copies it to
// shared memory in one bulk copy.
__global__ void k_pack(const bf16* __restrict__ W, bf16* __restrict__ Wf, bf16* __restrict__ Wb, int Cout, int Cin,
                       int taps) {
    const size_t nf = (size_t)((Cin + KC - 1) / KC) * taps * Cout * KC;
    const size_t nb = (size_t)((Cout + KC - 1) / KC) * taps * Cin * KC;
    const bf16 zero = __float2bfloat16(0.0f);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nf + nb; i += (size_t)gridDim.x * blockDim.x) {
        const bool fwd = i < nf;
        const size_t e = fwd ? i : i - nf;
        const int OC = fwd ? Cout : Cin, IC = fwd ? Cin : Cout;
        const int jj = (int)(e % 8);
        const size_t r = e / 8;
        const int o = (int)(r % OC);
        const size_t r2 = r / OC;
        const int h = (int)(r2 % 2);
        const size_t r3 = r2 / 2;
        const int t = (int)(r3 % taps), c = (int)(r3 / taps);
        const int in = c * KC + h * 8 + jj;
        bf16 v = zero;
        if (in < IC) v = fwd ? W[((size_t)o * Cin + in) * taps + t] : W[((size_t)in * Cin + o) * taps + (taps - 1 - t)];
        (fwd ? Wf : Wb)[e] = v;
    }
}

// Direct convolution, one 8x8 pixel tile x 64 outputs per block (4 warps:
// 2 output halves x 2 pixel-row halves, each 2 x 4 mma tiles).
// OUT 0: BF16 output with bias and optional ReLU; 1: FP32 output with bias.
template <int KS, int OUT>
__global__ void __launch_bounds__(NTHR) k_conv(const bf16* __restrict__ X, const bf16* __restrict__ Wp,
                                               const float* __restrict__ bias, void* __restrict__ Yv, int B, int IC,
                                               int OC, int H, int W, int relu) {
    constexpr int PW = 8 + KS - 1, PP = PW * PW, TAPS = KS * KS, OFF = KS / 2;
    __shared__ __align__(16) bf16 Ps[PP][KCP];
    __shared__ __align__(16) bf16 Ws[TAPS][CT][KCP];
    const int tiles_x = (W + 7) >> 3, tiles_y = (H + 7) >> 3;
    int bt = blockIdx.x;
    const int b = bt / (tiles_x * tiles_y);
    bt -= b * tiles_x * tiles_y;
    const int y0 = (bt / tiles_x) * 8, x0 = (bt % tiles_x) * 8;
    const int oc0 = blockIdx.y * CT;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1, g = lane >> 2, tg = lane & 3;
    const size_t hw = (size_t)H * W;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;
    const int nchunks = (IC + KC - 1) / KC;
    const bf16 zero = __float2bfloat16(0.0f);
    for (int c = 0; c < nchunks; ++c) {
        // one thread per (8-channel group, patch position): eight loads, one 16-byte store
        for (int e = tid; e < (KC / 8) * PP; e += NTHR) {
            const int gq = e / PP, r = e - gq * PP;
            const int py = r / PW, px = r - py * PW;
            const int y = y0 - OFF + py, x = x0 - OFF + px;
            const bool inb = y >= 0 && y < H && x >= 0 && x < W;
            const int ic0 = c * KC + gq * 8;
            const bf16* src = X + ((size_t)b * IC + ic0) * hw + (size_t)(inb ? y : 0) * W + (inb ? x : 0);
            uint32_t wv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bf16 lo = (inb && ic0 + 2 * q < IC) ? src[(size_t)(2 * q) * hw] : zero;
                const bf16 hi = (inb && ic0 + 2 * q + 1 < IC) ? src[(size_t)(2 * q + 1) * hw] : zero;
                wv[q] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
            }
            *reinterpret_cast<uint4*>(&Ps[r][gq * 8]) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
        for (int e = tid; e < TAPS * CT * 2; e += NTHR) {
            const int t = e / (CT * 2), rem = e - t * CT * 2, o = rem >> 1, h = rem & 1;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (oc0 + o < OC)
                v = *reinterpret_cast<const uint4*>(Wp + ((((size_t)c * TAPS + t) * 2 + h) * OC + oc0 + o) * 8);
            *reinterpret_cast<uint4*>(&Ws[t][o][h * 8]) = v;
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < TAPS; ++t) {
            const int dy = t / KS, dx = t - dy * KS;
            uint32_t a[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int r0 = wm * 32 + mt * 16 + g;
                a[mt][0] = ld32(&Ws[t][r0][2 * tg]);
                a[mt][1] = ld32(&Ws[t][r0 + 8][2 * tg]);
                a[mt][2] = ld32(&Ws[t][r0][2 * tg + 8]);
                a[mt][3] = ld32(&Ws[t][r0 + 8][2 * tg + 8]);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int pos = (wn * 4 + nt + dy) * PW + g + dx;
                uint32_t bb[2] = {ld32(&Ps[pos][2 * tg]), ld32(&Ps[pos][2 * tg + 8])};
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) mma16816(acc[mt][nt], a[mt], bb);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int o = oc0 + wm * 32 + mt * 16 + g + (r >= 2 ? 8 : 0);
                const int y = y0 + wn * 4 + nt, x = x0 + 2 * tg + (r & 1);
                if (o >= OC || y >= H || x >= W) continue;
                float v = acc[mt][nt][r] + (bias ? bias[o] : 0.0f);
                const size_t idx = ((size_t)b * OC + o) * hw + (size_t)y * W + x;
                if (OUT == 0) {
                    if (relu) v = fmaxf(v, 0.0f);
                    reinterpret_cast<bf16*>(Yv)[idx] = __float2bfloat16(v);
                } else {
                    reinterpret_cast<float*>(Yv)[idx] = v;
                }
            }
}

// Weight gradient: a block owns outputs oc0..oc0+63 x inputs 16c..16c+15 x
// all taps (N = 16 taps columns, n = j*taps + t) and sums over pixel tiles
// [z*tps, (z+1)*tps) into partial[z][OC][IC*taps]; the blocks of the first
// input chunk also sum dY per output channel (the bias gradient) into
// bpart[z][OC].
template <int KS>
__global__ void __launch_bounds__(NTHR) k_wgrad(const bf16* __restrict__ X, const bf16* __restrict__ dY,
                                                float* __restrict__ partial, float* __restrict__ bpart, int B,
                                                int IC, int OC, int H, int W, int tps) {
    constexpr int PW = 8 + KS - 1, RS = PW + (PW & 1), TAPS = KS * KS, OFF = KS / 2;
    constexpr int NT8 = KC * TAPS / 8, NTW = (NT8 + 1) / 2;
    __shared__ __align__(16) bf16 As[CT][64 + 8];
    __shared__ __align__(16) bf16 P0[KC][PW][RS];
    __shared__ __align__(16) bf16 P1[KC][PW][RS];
    const int c = blockIdx.x, oc0 = blockIdx.y * CT;
    const int tiles_x = (W + 7) >> 3, tiles_y = (H + 7) >> 3, ntiles = B * tiles_x * tiles_y;
    const int t_beg = blockIdx.z * tps, t_end = min(ntiles, t_beg + tps);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1, g = lane >> 2, tg = lane & 3;
    const size_t hw = (size_t)H * W;
    const bf16 zero = __float2bfloat16(0.0f);
    float acc[2][NTW][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < NTW; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;
    float bsum = 0.0f; // thread o < 64 of the first input chunk: sum of dY over this block's pixels
    for (int tile = t_beg; tile < t_end; ++tile) {
        const int b = tile / (tiles_x * tiles_y), bt = tile - b * tiles_x * tiles_y;
        const int y0 = (bt / tiles_x) * 8, x0 = (bt % tiles_x) * 8;
        // dY tile: one 16-byte row of 8 pixels per (channel, tile row) when the row is whole and
        // aligned (widths that are multiples of 8), else element by element
        const bool rows16 = (W & 7) == 0 && x0 + 8 <= W && (reinterpret_cast<uintptr_t>(dY) & 15u) == 0;
        for (int e = tid; e < CT * 8; e += NTHR) {
            const int o = e >> 3, ry = e & 7, y = y0 + ry;
            const bool ok = oc0 + o < OC && y < H;
            const bf16* src = dY + ((size_t)b * OC + oc0 + o) * hw + (size_t)y * W + x0;
            if (rows16) {
                *reinterpret_cast<uint4*>(&As[o][ry * 8]) =
                    ok ? *reinterpret_cast<const uint4*>(src) : make_uint4(0, 0, 0, 0);
            } else {
#pragma unroll
                for (int px = 0; px < 8; ++px) As[o][ry * 8 + px] = (ok && x0 + px < W) ? src[px] : zero;
            }
        }
        for (int e = tid; e < KC * PW * PW; e += NTHR) {
            const int j = e / (PW * PW), r = e - j * PW * PW, py = r / PW, px = r - py * PW;
            const int ic = c * KC + j, y = y0 - OFF + py, x = x0 - OFF + px;
            bf16 v = zero;
            if (ic < IC && y >= 0 && y < H && x >= 0 && x < W) v = X[((size_t)b * IC + ic) * hw + (size_t)y * W + x];
            P0[j][py][px] = v;
            if (px > 0) P1[j][py][px - 1] = v;
            if (px == PW - 1) P1[j][py][px] = zero;
        }
        __syncthreads();
        if (c == 0 && tid < CT)
            for (int p = 0; p < 64; ++p) bsum += __bfloat162float(As[tid][(p + tid) & 63]);
#pragma unroll
        for (int s = 0; s < 4; ++s) { // k16 slab: pixel rows 2s, 2s+1 of the tile
            uint32_t a[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int r0 = wm * 32 + mt * 16 + g;
                a[mt][0] = ld32(&As[r0][16 * s + 2 * tg]);
                a[mt][1] = ld32(&As[r0 + 8][16 * s + 2 * tg]);
                a[mt][2] = ld32(&As[r0][16 * s + 8 + 2 * tg]);
                a[mt][3] = ld32(&As[r0 + 8][16 * s + 8 + 2 * tg]);
            }
#pragma unroll
            for (int q = 0; q < NTW; ++q) {
                const int nt = wn * NTW + q;
                if (nt >= NT8) break;
                const int n = nt * 8 + g, j = n / TAPS, t = n - j * TAPS, dyy = t / KS, dxx = t - dyy * KS;
                const int col = 2 * tg + dxx;
                uint32_t bb[2];
                if (dxx & 1) {
                    bb[0] = ld32(&P1[j][2 * s + dyy][col - 1]);
                    bb[1] = ld32(&P1[j][2 * s + 1 + dyy][col - 1]);
                } else {
                    bb[0] = ld32(&P0[j][2 * s + dyy][col]);
                    bb[1] = ld32(&P0[j][2 * s + 1 + dyy][col]);
                }
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) mma16816(acc[mt][q], a[mt], bb);
            }
        }
        __syncthreads();
    }
    const size_t NC = (size_t)IC * TAPS;
    if (c == 0 && tid < CT && oc0 + tid < OC) bpart[(size_t)blockIdx.z * OC + oc0 + tid] = bsum;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int q = 0; q < NTW; ++q) {
            const int nt = wn * NTW + q;
            if (nt >= NT8) break;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int o = oc0 + wm * 32 + mt * 16 + g + (r >= 2 ? 8 : 0);
                const int n = nt * 8 + 2 * tg + (r & 1);
                const int ic = c * KC + n / TAPS;
                if (o >= OC || ic >= IC) continue;
                partial[((size_t)blockIdx.z * OC + o) * NC + (size_t)c * KC * TAPS + n] = acc[mt][q][r];
            }
        }
}

// fixed-order sum of split-K partials; bias gradient as the sum of dY over pixels
__global__ void k_reduce_splits(const float* partial, float* dW, int splits, size_t mn) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < mn; i += (size_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int z = 0; z < splits; ++z) s += partial[(size_t)z * mn + i];
        dW[i] = s;
    }
}
__global__ void k_relu_bwd(const bf16* y, const bf16* dy, bf16* dz, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dz[i] = __bfloat162float(y[i]) > 0.0f ? dy[i] : __float2bfloat16(0.0f);
}
__global__ void k_add(const bf16* a, const bf16* b, bf16* o, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        o[i] = __float2bfloat16(__bfloat162float(a[i]) + __bfloat162float(b[i]));
}
// 2x2 average pooling (H, W even) and its adjoint
__global__ void k_pool2(const bf16* x, bf16* y, int BC, int H, int W, int backward) {
    const int Ho = H / 2, Wo = W / 2;
    const size_t n = (size_t)BC * Ho * Wo;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t bc = i / ((size_t)Ho * Wo);
        const int r = (int)(i - bc * Ho * Wo), yo = r / Wo, xo = r - yo * Wo;
        const size_t base = bc * H * W + (size_t)(2 * yo) * W + 2 * xo;
        if (!backward) {
            const float s = __bfloat162float(x[base]) + __bfloat162float(x[base + 1]) +
                            __bfloat162float(x[base + W]) + __bfloat162float(x[base + W + 1]);
            y[i] = __float2bfloat16(0.25f * s);
        } else { // x = dY (Ho x Wo), y = dX (H x W)
            const bf16 v = __float2bfloat16(0.25f * __bfloat162float(x[i]));
            y[base] = v;
            y[base + 1] = v;
            y[base + W] = v;
            y[base + W + 1] = v;
        }
    }
}
// nearest 2x upsampling (H, W = input size) and its adjoint
__global__ void k_up2(const bf16* x, bf16* y, int BC, int H, int W, int backward) {
    const size_t n = (size_t)BC * H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t bc = i / ((size_t)H * W);
        const int r = (int)(i - bc * H * W), yy = r / W, xx = r - yy * W;
        const size_t base = bc * 4 * H * W + (size_t)(2 * yy) * (2 * W) + 2 * xx;
        if (!backward) {
            y[base] = x[i];
            y[base + 1] = x[i];
            y[base + 2 * W] = x[i];
            y[base + 2 * W + 1] = x[i];
        } else { // x = dY (2H x 2W), y = dX (H x W)
            const float s = __bfloat162float(x[base]) + __bfloat162float(x[base + 1]) +
                            __bfloat162float(x[base + 2 * W]) + __bfloat162float(x[base + 2 * W + 1]);
            y[i] = __float2bfloat16(s);
        }
    }
}
// mean squared error in FP32 and its gradient (BF16)
__global__ void k_mse(const bf16* out, const float* tgt, bf16* dout, double* loss, size_t n) {
    __shared__ double sh[256];
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float d = __bfloat162float(out[i]) - tgt[i];
        s += (double)d * d;
        if (dout) dout[i] = __float2bfloat16(2.0f * d / (float)n);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) atomicAdd(loss, sh[0] / (double)n);
}
__global__ void k_adam(float* p, float* m, float* v, const float* g, bf16* pb, size_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        pb[i] = __float2bfloat16(pi);
    }
}
// separable periodic Gaussian low-pass of [BC][H][W] FP32 planes, one axis
// per launch (axis 0: along x, 1: along y); taps w[-r..r] in `taps`
__global__ void k_smooth(const float* in, float* out, int BC, int H, int W, int axis, const float* taps, int r) {
    const size_t n = (size_t)BC * H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t bc = i / ((size_t)H * W);
        const int rem = (int)(i - bc * H * W), y = rem / W, x = rem - y * W;
        const float* plane = in + bc * H * W;
        float acc = 0.0f;
        for (int d = -r; d <= r; ++d) {
            const int xx = axis == 0 ? ((x + d) % W + W) % W : x;
            const int yy = axis == 1 ? ((y + d) % H + H) % H : y;
            acc = fmaf(taps[d + r], plane[(size_t)yy * W + xx], acc);
        }
        out[i] = acc;
    }
}

__global__ void k_cast(const float* in, bf16* out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16(in[i]);
}

inline int grid_for(size_t n) {
    size_t b = (n + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    return b < 1 ? 1 : (int)b;
}

} // namespace nn

using namespace nn;

#define NN_CHECK()                                                                                                   \
    do {                                                                                                             \
        if (cudaGetLastError() != cudaSuccess) return CX_ERR_CUDA;                                                   \
    } while (0)

static bool shape_ok(int B, int Cin, int Cout, int H, int W, int ks) {
    return B > 0 && Cin > 0 && Cout > 0 && H > 0 && W > 0 && (ks == 1 || ks == 3) &&
           (long long)B * Cin * H * W < (1LL << 31) && (long long)B * Cout * H * W < (1LL << 31);
}

extern "C" {

size_t cx_nn_packed_weights(int Cout, int Cin, int ks, int which) {
    const int taps = ks * ks;
    if (which == 0) return (size_t)((Cin + KC - 1) / KC) * taps * Cout * KC;
    return (size_t)((Cout + KC - 1) / KC) * taps * Cin * KC;
}

cx_status cx_nn_pack_weights(const uint16_t* w, int Cout, int Cin, int ks, uint16_t* w_fwd, uint16_t* w_bwd,
                             cudaStream_t stream) {
    if (!w || !w_fwd || !w_bwd || Cout < 1 || Cin < 1 || (ks != 1 && ks != 3)) return CX_ERR_INVALID_ARG;
    const size_t n = cx_nn_packed_weights(Cout, Cin, ks, 0) + cx_nn_packed_weights(Cout, Cin, ks, 1);
    k_pack<<<grid_for(n), 256, 0, stream>>>(reinterpret_cast<const bf16*>(w), reinterpret_cast<bf16*>(w_fwd),
                                            reinterpret_cast<bf16*>(w_bwd), Cout, Cin, ks * ks);
    NN_CHECK();
    return CX_OK;
}

static cx_status launch_conv(const void* x, const uint16_t* wp, const float* bias, void* y, int B, int IC, int OC,
                             int H, int W, int ks, int relu, int out_f32, cudaStream_t stream) {
    // BF16 outputs with 32, 64 or 128 channels run on the tcgen05 tensor cores
    // (measured 1.1-1.4x faster there; with 256 channels per tile the grid of
    // the deep, small levels is too coarse and the mma.sync kernel wins)
    if (!out_f32 && OC <= 128 && cx_nn_conv_tc_tile(OC) == OC)
        return cx_nn_conv_forward_tc(reinterpret_cast<const uint16_t*>(x), wp, bias, reinterpret_cast<uint16_t*>(y),
                                     B, IC, OC, H, W, ks, relu, nullptr, stream);
    const long long tiles = (long long)B * ((H + 7) / 8) * ((W + 7) / 8);
    if (tiles > 0x7fffffffLL) return CX_ERR_INVALID_ARG;
    dim3 grid((unsigned)tiles, (OC + CT - 1) / CT);
    const bf16* X = reinterpret_cast<const bf16*>(x);
    const bf16* Wp = reinterpret_cast<const bf16*>(wp);
    if (ks == 3) {
        if (out_f32) k_conv<3, 1><<<grid, NTHR, 0, stream>>>(X, Wp, bias, y, B, IC, OC, H, W, 0);
        else k_conv<3, 0><<<grid, NTHR, 0, stream>>>(X, Wp, bias, y, B, IC, OC, H, W, relu);
    } else {
        if (out_f32) k_conv<1, 1><<<grid, NTHR, 0, stream>>>(X, Wp, bias, y, B, IC, OC, H, W, 0);
        else k_conv<1, 0><<<grid, NTHR, 0, stream>>>(X, Wp, bias, y, B, IC, OC, H, W, relu);
    }
    NN_CHECK();
    return CX_OK;
}

cx_status cx_nn_conv_forward(const uint16_t* x, const uint16_t* w_fwd, const float* bias, uint16_t* y, int B,
                             int Cin, int Cout, int H, int W, int ks, int relu, cudaStream_t stream) {
    if (!x || !w_fwd || !y || !shape_ok(B, Cin, Cout, H, W, ks)) return CX_ERR_INVALID_ARG;
    return launch_conv(x, w_fwd, bias, y, B, Cin, Cout, H, W, ks, relu, 0, stream);
}

cx_status cx_nn_conv_forward_f32(const uint16_t* x, const uint16_t* w_fwd, const float* bias, float* y, int B,
                                 int Cin, int Cout, int H, int W, int ks, cudaStream_t stream) {
    if (!x || !w_fwd || !y || !shape_ok(B, Cin, Cout, H, W, ks)) return CX_ERR_INVALID_ARG;
    return launch_conv(x, w_fwd, bias, y, B, Cin, Cout, H, W, ks, 0, 1, stream);
}

cx_status cx_nn_smooth(const float* in, float* tmp, float* out, int BC, int H, int W, const float* taps, int radius,
                       cudaStream_t stream) {
    if (!in || !tmp || !out || !taps || BC < 1 || H < 1 || W < 1 || radius < 0 || radius > 64)
        return CX_ERR_INVALID_ARG;
    const size_t n = (size_t)BC * H * W;
    k_smooth<<<grid_for(n), 256, 0, stream>>>(in, tmp, BC, H, W, 0, taps, radius);
    NN_CHECK();
    k_smooth<<<grid_for(n), 256, 0, stream>>>(tmp, out, BC, H, W, 1, taps, radius);
    NN_CHECK();
    return CX_OK;
}

cx_status cx_nn_conv_backward_data(const uint16_t* dy, const uint16_t* w_bwd, uint16_t* dx, int B, int Cin, int Cout,
                                   int H, int W, int ks, cudaStream_t stream) {
    if (!dy || !w_bwd || !dx || !shape_ok(B, Cin, Cout, H, W, ks)) return CX_ERR_INVALID_ARG;
    // dY has Cout channels, dX has Cin
    return launch_conv(dy, w_bwd, nullptr, dx, B, Cout, Cin, H, W, ks, 0, 0, stream);
}

size_t cx_nn_conv_backward_weight_scratch(int B, int Cin, int Cout, int H, int W, int ks, int splits) {
    return (size_t)splits * Cout * ((size_t)Cin * ks * ks + 1) * sizeof(float);
}

cx_status cx_nn_conv_backward_weight(const uint16_t* x, const uint16_t* dy, float* dw, float* db, float* scratch,
                                     int splits, int B, int Cin, int Cout, int H, int W, int ks,
                                     cudaStream_t stream) {
    if (!x || !dy || !dw || !scratch || splits < 1 || splits > 65535 || !shape_ok(B, Cin, Cout, H, W, ks))
        return CX_ERR_INVALID_ARG;
    const int ntiles = B * ((H + 7) / 8) * ((W + 7) / 8);
    const int tps = (ntiles + splits - 1) / splits;
    dim3 grid((Cin + KC - 1) / KC, (Cout + CT - 1) / CT, splits);
    const bf16* X = reinterpret_cast<const bf16*>(x);
    const bf16* dY = reinterpret_cast<const bf16*>(dy);
    const size_t mn = (size_t)Cout * Cin * ks * ks;
    float* bpart = scratch + (size_t)splits * mn;
    if (ks == 3) k_wgrad<3><<<grid, NTHR, 0, stream>>>(X, dY, scratch, bpart, B, Cin, Cout, H, W, tps);
    else k_wgrad<1><<<grid, NTHR, 0, stream>>>(X, dY, scratch, bpart, B, Cin, Cout, H, W, tps);
    NN_CHECK();
    k_reduce_splits<<<grid_for(mn), 256, 0, stream>>>(scratch, dw, splits, mn);
    NN_CHECK();
    if (db) {
        k_reduce_splits<<<grid_for(Cout), 256, 0, stream>>>(bpart, db, splits, Cout);
        NN_CHECK();
    }
    return CX_OK;
}

cx_status cx_nn_relu_backward(const uint16_t* y, const uint16_t* dy, uint16_t* dz, size_t n, cudaStream_t stream) {
    if (!y || !dy || !dz) return CX_ERR_INVALID_ARG;
    k_relu_bwd<<<grid_for(n), 256, 0, stream>>>(reinterpret_cast<const bf16*>(y), reinterpret_cast<const bf16*>(dy),
                                                reinterpret_cast<bf16*>(dz), n);
    NN_CHECK();
    return CX_OK;
}

cx_status cx_nn_add(const uint16_t* a, const uint16_t* b, uint16_t* out, size_t n, cudaStream_t stream) {
    if (!a || !b || !out) return CX_ERR_INVALID_ARG;
    k_add<<<grid_for(n), 256, 0, stream>>>(reinterpret_cast<const bf16*>(a), reinterpret_cast<const bf16*>(b),
                                           reinterpret_cast<bf16*>(out), n);
    NN_CHECK();
    return CX_OK;
}

cx_status cx_nn_pool2(const uint16_t* in, uint16_t* out, int BC, int H, int W, int backward, cudaStream_t stream) {
    if (!in || !out || H % 2 || W % 2) return CX_ERR_INVALID_ARG;
    k_pool2<<<grid_for((size_t)BC * H * W / 4), 256, 0, stream>>>(reinterpret_cast<const bf16*>(in),
                                                                   reinterpret_cast<bf16*>(out), BC, H, W, backward);
    NN_CHECK();
    return CX_OK;
}

cx_status cx_nn_up2(const uint16_t* in, uint16_t* out, int BC, int H, int W, int backward, cudaStream_t stream) {
    if (!in || !out) return CX_ERR_INVALID_ARG;
    k_up2<<<grid_for((size_t)BC * H * W), 256, 0, stream>>>(reinterpret_cast<const bf16*>(in),
                                                            reinterpret_cast<bf16*>(out), BC, H, W, backward);
    NN_CHECK();
    return CX_OK;
}

cx_status cx_nn_mse(const uint16_t* out, const float* target, uint16_t* dout, double* loss, size_t n,
                    cudaStream_t stream) {
    if (!out || !target) return CX_ERR_INVALID_ARG;
    if (loss && cudaMemsetAsync(loss, 0, sizeof(double), stream) != cudaSuccess) return CX_ERR_CUDA;
    k_mse<<<grid_for(n), 256, 0, stream>>>(reinterpret_cast<const bf16*>(out), target, reinterpret_cast<bf16*>(dout),
                                           loss, n);
    NN_CHECK();
    return CX_OK;
}

cx_status cx_nn_adam(float* p, float* m, float* v, const float* g, uint16_t* p_bf16, size_t n, float lr, float b1,
                     float b2, float eps, int t, cudaStream_t stream) {
    if (!p || !m || !v || !g || !p_bf16 || t < 1) return CX_ERR_INVALID_ARG;
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    k_adam<<<grid_for(n), 256, 0, stream>>>(p, m, v, g, reinterpret_cast<bf16*>(p_bf16), n, lr, b1, b2, eps, c1, c2);
    NN_CHECK();
    return CX_OK;
}

cx_status cx_nn_cast_bf16(const float* in, uint16_t* out, size_t n, cudaStream_t stream) {
    if (!in || !out) return CX_ERR_INVALID_ARG;
    k_cast<<<grid_for(n), 256, 0, stream>>>(in, reinterpret_cast<bf16*>(out), n);
    NN_CHECK();
    return CX_OK;
}

} // extern "C"
