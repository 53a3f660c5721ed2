// nn_kernels.cu -- kernels of the warm-start surrogate (a small convolutional
// U-Net that maps a problem's initial state and parameters to a proposed
// control).  BF16 weights and activations, FP32 accumulation.
//
// Convolutions (3x3, padding 1, or 1x1) are implicit GEMMs on the tensor
// cores with mma.sync m16n8k16 (BF16 inputs, FP32 accumulators):
//   forward        Y[b,co,p] = bias[co] + sum_{ci,t} W[co,ci,t] X[b,ci,p+t]
//                  (M = Cout, N = B*H*W pixels, K = Cin*ks*ks)
//   data gradient  the forward kernel applied to dY with W' [ci,co,flip(t)]
//   weight grad.   dW[co,ci,t] = sum_{b,p} dY[b,co,p] X[b,ci,p+t]
//                  (M = Cout, N = Cin*ks*ks, K = B*H*W, split over blocks into
//                  FP32 partials reduced in a fixed order)
// Tiles: 64 x 64 x 32 per block of 4 warps, each warp a 32 x 32 sub-tile of
// 2 x 4 mma tiles; operands staged in padded shared memory.
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/cxlbm.h"

namespace nn {

typedef __nv_bfloat16 bf16;

constexpr int BM = 64, BN = 64, BK = 32, PADK = BK + 8, NTHR = 128;

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

struct ConvShape {
    int B, Cin, Cout, H, W, ks;
};

// element (k, n) of the implicit im2col matrix of X: k = ci*ks*ks + t, n = b*H*W + y*W + x
__device__ __forceinline__ float im2col(const bf16* X, const ConvShape& s, int k, int n) {
    const int kk = s.ks * s.ks;
    const int ci = k / kk, t = k - ci * kk;
    const int hw = s.H * s.W;
    const int b = n / hw, r = n - b * hw;
    const int y = r / s.W, x = r - y * s.W;
    const int pad = s.ks / 2;
    const int yy = y + t / s.ks - pad, xx = x + t % s.ks - pad;
    if (yy < 0 || yy >= s.H || xx < 0 || xx >= s.W) return 0.0f;
    return __bfloat162float(X[((size_t)b * s.Cin + ci) * hw + (size_t)yy * s.W + xx]);
}

// mode 0: forward (A = W [Cout][K], B = im2col(X)), BF16 output; mode 2: the
// same with FP32 output; mode 1: weight gradient (A = dY as [Cout][pixels],
// B[k=pixel][n=(ci,t)] = im2col(X)[n][k]).
template <int MODE>
__global__ void __launch_bounds__(NTHR) k_conv_gemm(const bf16* __restrict__ A_src, const bf16* __restrict__ X,
                                                    const float* __restrict__ bias, bf16* __restrict__ Y,
                                                    float* __restrict__ partial, ConvShape s, int relu, int k_chunk) {
    __shared__ __align__(16) bf16 As[BM][PADK];
    __shared__ __align__(16) bf16 Bs[BN][PADK];
    const int kk = s.ks * s.ks;
    const int hw = s.H * s.W;
    const int M = s.Cout;
    constexpr bool FWD = MODE != 1;
    const int N = FWD ? s.B * hw : s.Cin * kk;
    const int Ktot = FWD ? s.Cin * kk : s.B * hw;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kbeg = FWD ? 0 : blockIdx.z * k_chunk;
    const int kend = FWD ? Ktot : min(Ktot, kbeg + k_chunk);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int g = lane >> 2, tg = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;

    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        // stage A [BM][BK] and B as [BN][BK]
        for (int e = tid; e < BM * BK; e += NTHR) {
            const int r = e / BK, c = e - r * BK;
            const int m = m0 + r, k = k0 + c;
            float v = 0.0f;
            if (m < M && k < kend) {
                if (FWD) v = __bfloat162float(A_src[(size_t)m * Ktot + k]);
                else {
                    const int b = k / hw, p = k - b * hw;
                    v = __bfloat162float(A_src[((size_t)b * s.Cout + m) * hw + p]);
                }
            }
            As[r][c] = __float2bfloat16(v);
        }
        for (int e = tid; e < BN * BK; e += NTHR) {
            const int r = e / BK, c = e - r * BK;
            const int n = n0 + r, k = k0 + c;
            float v = 0.0f;
            if (n < N && k < kend) v = FWD ? im2col(X, s, k, n) : im2col(X, s, n, k);
            Bs[r][c] = __float2bfloat16(v);
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int r0 = wm * 32 + mt * 16 + g;
                af[mt][0] = *reinterpret_cast<const uint32_t*>(&As[r0][ks + 2 * tg]);
                af[mt][1] = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][ks + 2 * tg]);
                af[mt][2] = *reinterpret_cast<const uint32_t*>(&As[r0][ks + 2 * tg + 8]);
                af[mt][3] = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][ks + 2 * tg + 8]);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int c = wn * 32 + nt * 8 + g;
                bfr[nt][0] = *reinterpret_cast<const uint32_t*>(&Bs[c][ks + 2 * tg]);
                bfr[nt][1] = *reinterpret_cast<const uint32_t*>(&Bs[c][ks + 2 * tg + 8]);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma16816(acc[mt][nt], af[mt], bfr[nt]);
        }
        __syncthreads();
    }
    // epilogue
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int m = m0 + wm * 32 + mt * 16 + g + (r >= 2 ? 8 : 0);
                const int n = n0 + wn * 32 + nt * 8 + 2 * tg + (r & 1);
                if (m >= M || n >= N) continue;
                float v = acc[mt][nt][r];
                if (FWD) {
                    if (bias) v += bias[m];
                    if (relu) v = fmaxf(v, 0.0f);
                    const int b = n / hw, p = n - b * hw;
                    if (MODE == 0) Y[((size_t)b * s.Cout + m) * hw + p] = __float2bfloat16(v);
                    else reinterpret_cast<float*>(Y)[((size_t)b * s.Cout + m) * hw + p] = v;
                } else {
                    partial[((size_t)blockIdx.z * M + m) * N + n] = v;
                }
            }
}

// W'[ci][co][t'] = W[co][ci][ks*ks-1-t]: the data gradient as a forward conv
__global__ void k_flip(const bf16* W, bf16* Wt, int Cout, int Cin, int kk) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Cout * Cin * kk) return;
    const int co = i / (Cin * kk), r = i - co * Cin * kk, ci = r / kk, t = r - ci * kk;
    Wt[((size_t)ci * Cout + co) * kk + (kk - 1 - t)] = W[i];
}

// fixed-order sum of split-K partials; bias gradient as the sum of dY over pixels
__global__ void k_reduce_splits(const float* partial, float* dW, int splits, size_t mn) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < mn; i += (size_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int z = 0; z < splits; ++z) s += partial[(size_t)z * mn + i];
        dW[i] = s;
    }
}
__global__ void k_bias_grad(const bf16* dY, float* db, int B, int C, int hw) {
    __shared__ float sh[256];
    const int c = blockIdx.x;
    float s = 0.0f;
    for (int i = threadIdx.x; i < B * hw; i += 256) {
        const int b = i / hw, p = i - b * hw;
        s += __bfloat162float(dY[((size_t)b * C + c) * hw + p]);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[c] = sh[0];
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

cx_status cx_nn_conv_forward(const uint16_t* x, const uint16_t* w, const float* bias, uint16_t* y, int B, int Cin,
                             int Cout, int H, int W, int ks, int relu, cudaStream_t stream) {
    if (!x || !w || !y || !shape_ok(B, Cin, Cout, H, W, ks)) return CX_ERR_INVALID_ARG;
    ConvShape s{B, Cin, Cout, H, W, ks};
    dim3 grid((B * H * W + BN - 1) / BN, (Cout + BM - 1) / BM);
    k_conv_gemm<0><<<grid, NTHR, 0, stream>>>(reinterpret_cast<const bf16*>(w), reinterpret_cast<const bf16*>(x),
                                              bias, reinterpret_cast<bf16*>(y), nullptr, s, relu, 0);
    NN_CHECK();
    return CX_OK;
}

cx_status cx_nn_conv_forward_f32(const uint16_t* x, const uint16_t* w, const float* bias, float* y, int B, int Cin,
                                 int Cout, int H, int W, int ks, cudaStream_t stream) {
    if (!x || !w || !y || !shape_ok(B, Cin, Cout, H, W, ks)) return CX_ERR_INVALID_ARG;
    ConvShape s{B, Cin, Cout, H, W, ks};
    dim3 grid((B * H * W + BN - 1) / BN, (Cout + BM - 1) / BM);
    k_conv_gemm<2><<<grid, NTHR, 0, stream>>>(reinterpret_cast<const bf16*>(w), reinterpret_cast<const bf16*>(x),
                                              bias, reinterpret_cast<bf16*>(y), nullptr, s, 0, 0);
    NN_CHECK();
    return CX_OK;
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

cx_status cx_nn_conv_backward_data(const uint16_t* dy, const uint16_t* w, uint16_t* dx, uint16_t* w_flip, int B,
                                   int Cin, int Cout, int H, int W, int ks, cudaStream_t stream) {
    if (!dy || !w || !dx || !w_flip || !shape_ok(B, Cin, Cout, H, W, ks)) return CX_ERR_INVALID_ARG;
    const int kk = ks * ks, nw = Cout * Cin * kk;
    k_flip<<<(nw + 255) / 256, 256, 0, stream>>>(reinterpret_cast<const bf16*>(w), reinterpret_cast<bf16*>(w_flip),
                                                 Cout, Cin, kk);
    NN_CHECK();
    ConvShape s{B, Cout, Cin, H, W, ks}; // dY has Cout channels, dX has Cin
    dim3 grid((B * H * W + BN - 1) / BN, (Cin + BM - 1) / BM);
    k_conv_gemm<0><<<grid, NTHR, 0, stream>>>(reinterpret_cast<const bf16*>(w_flip),
                                              reinterpret_cast<const bf16*>(dy), nullptr,
                                              reinterpret_cast<bf16*>(dx), nullptr, s, 0, 0);
    NN_CHECK();
    return CX_OK;
}

size_t cx_nn_conv_backward_weight_scratch(int B, int Cin, int Cout, int H, int W, int ks, int splits) {
    return (size_t)splits * Cout * Cin * ks * ks * sizeof(float);
}

cx_status cx_nn_conv_backward_weight(const uint16_t* x, const uint16_t* dy, float* dw, float* db, float* scratch,
                                     int splits, int B, int Cin, int Cout, int H, int W, int ks,
                                     cudaStream_t stream) {
    if (!x || !dy || !dw || !scratch || splits < 1 || !shape_ok(B, Cin, Cout, H, W, ks)) return CX_ERR_INVALID_ARG;
    ConvShape s{B, Cin, Cout, H, W, ks};
    const int Ktot = B * H * W;
    int chunk = (Ktot + splits - 1) / splits;
    chunk = (chunk + BK - 1) / BK * BK;
    const int used = (Ktot + chunk - 1) / chunk;
    const int N = Cin * ks * ks;
    dim3 grid((N + BN - 1) / BN, (Cout + BM - 1) / BM, used);
    k_conv_gemm<1><<<grid, NTHR, 0, stream>>>(reinterpret_cast<const bf16*>(dy), reinterpret_cast<const bf16*>(x),
                                              nullptr, nullptr, scratch, s, 0, chunk);
    NN_CHECK();
    const size_t mn = (size_t)Cout * N;
    k_reduce_splits<<<grid_for(mn), 256, 0, stream>>>(scratch, dw, used, mn);
    NN_CHECK();
    if (db) {
        k_bias_grad<<<Cout, 256, 0, stream>>>(reinterpret_cast<const bf16*>(dy), db, B, Cout, H * W);
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
