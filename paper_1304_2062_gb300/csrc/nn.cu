// Kernels of the learned surrogate: a 4-level U-Net (32-64-128-256
// channels), BF16 weights and activations, FP32 accumulation, trained on
// (corrupted image, method output) pairs that the inpainting method itself
// generates.
//
// Activations are NHWC bf16 with the channel count a multiple of 8; a 3x3
// convolution (padding 1) is the implicit GEMM of nn_gemm.cuh with
// k = tap * C + channel, tap = (dy+1)*3 + (dx+1). Layer list and parameter
// layout are in unet.cu.
#include <cuda_bf16.h>

#include "conv_loaders.cuh"
#include "conv_tc.cuh"
#include "nn.h"
#include "nn_gemm.cuh"

using namespace se2n::nn;

// Set by a tensor-core convolution whose bounded wait ran out (never expected;
// it would mean the device stopped making progress). Read by tc_fault().
__device__ int g_tc_fault;

namespace {

// B operand of backward data: B(k = tap*Cout + co, n = ci) = W[co][tap*Cin + ci],
// N-major (8 consecutive ci of one (tap, co)).
struct WeightNLoader {
    const __nv_bfloat16 *w;
    int Cout, Cin, K;  // K = 9 * Cout
    __device__ __forceinline__ const void *chunk(int k, int n) const {
        if (k >= K || n >= Cin) return nullptr;
        const int tap = k / Cout, co = k - tap * Cout;
        return w + (long long)co * 9 * Cin + tap * Cin + n;
    }
};

// A operand of backward weight: dOut[pix][co], M(=co)-major.
struct GradOutMLoader {
    const __nv_bfloat16 *g;
    int Cout, P;  // P = number of pixels (the GEMM's K)
    __device__ __forceinline__ const void *chunk(int k, int m) const {
        return (k < P && m < Cout) ? (const void *)(g + (long long)k * Cout + m) : nullptr;
    }
};

// B operand of backward weight: B(k = pixel, n = tap*Cin + ci) = In[shift(pixel, tap)][ci].
struct InNLoader {
    ConvInLoader in;  // flip = 0; chunk(m = pixel, k = n) gives the gathered input
    int P;
    __device__ __forceinline__ const void *chunk(int k, int n) const {
        if (k >= P) return nullptr;
        return in.chunk(k, n);
    }
};

template <int BM, int BN, bool AK, bool BK_, class LA, class LB>
__device__ __forceinline__ void run_tile(const LA &la, const LB &lb, int m0, int n0, int kt0, int kt1,
                                         float (&acc)[BM / 32][BN / 16][4]) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    gemm_mainloop<BM, BN, AK, BK_>(la, lb, m0, n0, kt0, kt1, (__nv_bfloat16 *)smem_raw, acc);
}

// Forward conv: out = relu(A W^T + bias) (relu optional), bf16 NHWC.
template <int BM, int BN>
__global__ void __launch_bounds__(128) k_conv_fwd(ConvInLoader la, WeightKLoader lb, const float *bias,
                                                  __nv_bfloat16 *out, int relu) {
    float acc[BM / 32][BN / 16][4];
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    run_tile<BM, BN, true, true>(la, lb, m0, n0, 0, (la.K + kBK - 1) / kBK, acc);
#pragma unroll
    for (int i = 0; i < BM / 32; ++i)
#pragma unroll
        for (int j = 0; j < BN / 16; ++j)
#pragma unroll
            for (int q = 0; q < 4; q += 2) {
                int m, n;
                acc_pos<BM, BN>(i, j, q, m, n);
                m += m0;
                n += n0;
                if (m < la.M && n < lb.N) {
                    float v0 = acc[i][j][q] + bias[n], v1 = acc[i][j][q + 1] + bias[n + 1];
                    if (relu) {
                        v0 = fmaxf(v0, 0.0f);
                        v1 = fmaxf(v1, 0.0f);
                    }
                    *(__nv_bfloat162 *)(out + (long long)m * lb.N + n) = __floats2bfloat162_rn(v0, v1);
                }
            }
}

// Backward data: dIn = dZ * W (flipped taps); multiplied by (act > 0) when
// the input was a ReLU output; channels >= split go to a second buffer.
template <int BM, int BN>
__global__ void __launch_bounds__(128) k_conv_dgrad(ConvInLoader la, WeightNLoader lb, const __nv_bfloat16 *act,
                                                    __nv_bfloat16 *din, __nv_bfloat16 *din2, int split) {
    float acc[BM / 32][BN / 16][4];
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    run_tile<BM, BN, true, false>(la, lb, m0, n0, 0, (la.K + kBK - 1) / kBK, acc);
    const int Cin = lb.Cin;
#pragma unroll
    for (int i = 0; i < BM / 32; ++i)
#pragma unroll
        for (int j = 0; j < BN / 16; ++j)
#pragma unroll
            for (int q = 0; q < 4; q += 2) {
                int m, n;
                acc_pos<BM, BN>(i, j, q, m, n);
                m += m0;
                n += n0;
                if (m >= la.M || n >= Cin) continue;
                float v0 = acc[i][j][q], v1 = acc[i][j][q + 1];
                if (n < split) {
                    if (act) {
                        const __nv_bfloat162 a = *(const __nv_bfloat162 *)(act + (long long)m * split + n);
                        if (!(__bfloat162float(a.x) > 0.0f)) v0 = 0.0f;
                        if (!(__bfloat162float(a.y) > 0.0f)) v1 = 0.0f;
                    }
                    *(__nv_bfloat162 *)(din + (long long)m * split + n) = __floats2bfloat162_rn(v0, v1);
                } else {
                    const int c2 = Cin - split;
                    *(__nv_bfloat162 *)(din2 + (long long)m * c2 + (n - split)) = __floats2bfloat162_rn(v0, v1);
                }
            }
}

// Backward weight (split K over pixels): dW[co][tap*Cin+ci] += sum dZ * In.
template <int BM, int BN>
__global__ void __launch_bounds__(128) k_conv_wgrad(GradOutMLoader la, InNLoader lb, float *dw, int N, int ktiles_per) {
    float acc[BM / 32][BN / 16][4];
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int kt_total = (lb.P + kBK - 1) / kBK;
    const int kt0 = blockIdx.z * ktiles_per;
    const int kt1 = min(kt_total, kt0 + ktiles_per);
    run_tile<BM, BN, false, false>(la, lb, m0, n0, kt0, kt1, acc);
    if (kt1 <= kt0) return;
#pragma unroll
    for (int i = 0; i < BM / 32; ++i)
#pragma unroll
        for (int j = 0; j < BN / 16; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int m, n;
                acc_pos<BM, BN>(i, j, q, m, n);
                m += m0;
                n += n0;
                if (m < la.Cout && n < N) atomicAdd(dw + (long long)m * N + n, acc[i][j][q]);
            }
}

// ---------------------------------------------------------------------------
// tcgen05 convolutions (conv_tc.cuh): forward and backward data
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *(const uint32_t *)&h;
}

// out[m][n..n+15] = relu?(v + bias), bf16; out has N channels per pixel.
struct FwdEpi {
    const float *bias;
    __nv_bfloat16 *out;
    int N, relu;
    __device__ __forceinline__ void operator()(int m, int n, const float (&v)[16]) const {
        uint32_t p[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            float a = v[2 * q] + bias[n + 2 * q], b = v[2 * q + 1] + bias[n + 2 * q + 1];
            if (relu) {
                a = fmaxf(a, 0.0f);
                b = fmaxf(b, 0.0f);
            }
            p[q] = pack_bf16(a, b);
        }
        uint4 *dst = (uint4 *)(out + (long long)m * N + n);
        dst[0] = make_uint4(p[0], p[1], p[2], p[3]);
        dst[1] = make_uint4(p[4], p[5], p[6], p[7]);
    }
};

// Backward data: columns < split go to din (times (act > 0) when act is
// given), the others to din2; N = total columns. split % 16 == 0.
struct DgradEpi {
    const __nv_bfloat16 *act;
    __nv_bfloat16 *din, *din2;
    int split, N;
    __device__ __forceinline__ void operator()(int m, int n, const float (&v)[16]) const {
        float w[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) w[q] = v[q];
        __nv_bfloat16 *dst;
        if (n < split) {
            if (act) {
                const uint4 *a4 = (const uint4 *)(act + (long long)m * split + n);
                const uint4 a0 = a4[0], a1 = a4[1];
                const uint32_t aw[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const __nv_bfloat162 h = *(const __nv_bfloat162 *)&aw[q];
                    if (!(__bfloat162float(h.x) > 0.0f)) w[2 * q] = 0.0f;
                    if (!(__bfloat162float(h.y) > 0.0f)) w[2 * q + 1] = 0.0f;
                }
            }
            dst = din + (long long)m * split + n;
        } else {
            dst = din2 + (long long)m * (N - split) + (n - split);
        }
        uint32_t p[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) p[q] = pack_bf16(w[2 * q], w[2 * q + 1]);
        uint4 *d4 = (uint4 *)dst;
        d4[0] = make_uint4(p[0], p[1], p[2], p[3]);
        d4[1] = make_uint4(p[4], p[5], p[6], p[7]);
    }
};

template <int BN, int STAGES, int LAG>
__global__ void __launch_bounds__(128) k_conv_fwd_tc(ConvInLoader la, WeightKLoader lb, FwdEpi epi) {
    tc::conv_tile<BN, STAGES, LAG>(la, lb, epi, &g_tc_fault);
}

template <int BN, int STAGES, int LAG>
__global__ void __launch_bounds__(128) k_conv_dgrad_tc(ConvInLoader la, WeightKLoader lb, DgradEpi epi) {
    tc::conv_tile<BN, STAGES, LAG>(la, lb, epi, &g_tc_fault);
}

// Weights rearranged for the data gradient, K-major in the output channel:
// wt[ci][tap * Cout + co] = w[co][tap * Cin + ci].
__global__ void k_transpose_dgrad(const __nv_bfloat16 *w, __nv_bfloat16 *wt, int Cout, int Cin) {
    const long long total = (long long)Cout * 9 * Cin;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int co = (int)(i % Cout);
        const long long t = i / Cout;
        const int tap = (int)(t % 9), ci = (int)(t / 9);
        wt[i] = w[((long long)co * 9 + tap) * Cin + ci];
    }
}

// Column sums of a [P][C] bf16 matrix into db[C] (bias gradients): each
// thread sums 8 channels (one 16-byte load) of every (256 / (C/8))-th row,
// the block combines its partial sums in shared memory, one atomic per
// channel per block.
__global__ void __launch_bounds__(256) k_colsum(const __nv_bfloat16 *g, long long P, int C, float *db) {
    __shared__ float part[256][8];
    const int groups = C / 8;                 // 4..32
    const int rows = blockDim.x / groups;     // rows per block step
    const int cg = threadIdx.x % groups, rr = threadIdx.x / groups;
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (rr < rows) {
        for (long long p = (long long)blockIdx.x * rows + rr; p < P; p += (long long)gridDim.x * rows) {
            const uint4 v = *(const uint4 *)(g + p * C + cg * 8);
            const __nv_bfloat16 *h = (const __nv_bfloat16 *)&v;
#pragma unroll
            for (int k = 0; k < 8; ++k) s[k] += __bfloat162float(h[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) part[threadIdx.x][k] = s[k];
    __syncthreads();
    if (threadIdx.x < C) {
        const int c8 = threadIdx.x / 8, k = threadIdx.x % 8;
        float t = 0.0f;
        for (int r = 0; r < rows; ++r) t += part[r * groups + c8][k];
        atomicAdd(db + threadIdx.x, t);
    }
}

// Input packing: x[b][y][x][0] = f*(mask!=0), [1] = mask, [2..7] = 0.
__global__ void k_pack_input(const float *f, const uint8_t *mask, __nv_bfloat16 *x, long long P) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const float m = mask[p] ? 1.0f : 0.0f;
        __nv_bfloat16 v[8];
        v[0] = __float2bfloat16_rn(f[p] * m);
        v[1] = __float2bfloat16_rn(m);
#pragma unroll
        for (int c = 2; c < 8; ++c) v[c] = __float2bfloat16_rn(0.0f);
        *(uint4 *)(x + p * 8) = *(uint4 *)v;
    }
}

// 2x2 average pooling, NHWC (input row stride ldi), 8 channels (16 bytes) per thread.
__global__ void k_pool(const __nv_bfloat16 *in, int ldi, __nv_bfloat16 *out, int B, int H, int W, int C) {
    const int Ho = H / 2, Wo = W / 2, C8 = C / 8;
    const long long total = (long long)B * Ho * Wo * C8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C8) * 8;
        long long t = i / C8;
        const int x = (int)(t % Wo);
        t /= Wo;
        const int y = (int)(t % Ho);
        const int b = (int)(t / Ho);
        const long long base = (((long long)b * H + 2 * y) * W + 2 * x) * ldi + c;
        const uint4 q0 = *(const uint4 *)(in + base), q1 = *(const uint4 *)(in + base + ldi);
        const uint4 q2 = *(const uint4 *)(in + base + (long long)W * ldi);
        const uint4 q3 = *(const uint4 *)(in + base + (long long)W * ldi + ldi);
        const __nv_bfloat16 *a = (const __nv_bfloat16 *)&q0, *b1 = (const __nv_bfloat16 *)&q1;
        const __nv_bfloat16 *c2 = (const __nv_bfloat16 *)&q2, *d3 = (const __nv_bfloat16 *)&q3;
        __align__(16) __nv_bfloat16 o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float s = __bfloat162float(a[k]) + __bfloat162float(b1[k]) + __bfloat162float(c2[k]) +
                            __bfloat162float(d3[k]);
            o[k] = __float2bfloat16_rn(0.25f * s);
        }
        *(uint4 *)(out + (((long long)b * Ho + y) * Wo + x) * C + c) = *(const uint4 *)o;
    }
}

// Nearest upsampling into the first C1 channels of a wider tensor: one
// block per output row (b, y), 16 bytes per thread.
__global__ void k_upsample_into(const __nv_bfloat16 *lo, int C1, __nv_bfloat16 *out, int ldo, int H, int W) {
    const int y = blockIdx.x % H;
    const long long b = blockIdx.x / H;
    const int C8 = C1 / 8, Wl = W / 2;
    const __nv_bfloat16 *src = lo + ((b * (H / 2) + y / 2) * Wl) * C1;
    __nv_bfloat16 *dst = out + ((b * H + y) * W) * (long long)ldo;
    for (int i = threadIdx.x; i < W * C8; i += blockDim.x) {
        const int x = i / C8, c = (i - x * C8) * 8;
        *(uint4 *)(dst + (long long)x * ldo + c) = *(const uint4 *)(src + (x / 2) * C1 + c);
    }
}

// First convolution straight from the image: the input channels are
// bf16(f m) and m (the other six are zero), so each of the 32 outputs is a
// sum over 9 taps x 2 channels, done in FP32 on the CUDA cores. A block
// takes 32 x 8 pixel tiles; the tile and its 1-pixel halo of (bf16(f m), m)
// are staged in shared memory with coalesced loads, and the weights sit
// there as [tap][channel][4 outputs] float4 (one 16-byte load per 4 FMAs).
constexpr int C0_TW = 32, C0_TH = 8;
__global__ void __launch_bounds__(256) k_conv0(const float *f, const uint8_t *mask, const __nv_bfloat16 *w,
                                               const float *bias, __nv_bfloat16 *out, int B, int H, int W) {
    __shared__ float4 sw[9][2][8];
    __shared__ float sb[32];
    __shared__ float2 tile[C0_TH + 2][C0_TW + 2];
    for (int i = threadIdx.x; i < 9 * 2 * 8; i += blockDim.x) {
        const int tap = i / 16, ci = (i / 8) % 2, q = i % 8;
        const __nv_bfloat16 *wq = w + tap * 8 + ci;  // w[co][tap][ci], 72 per output channel
        sw[tap][ci][q] = make_float4(__bfloat162float(wq[(4 * q + 0) * 72]), __bfloat162float(wq[(4 * q + 1) * 72]),
                                     __bfloat162float(wq[(4 * q + 2) * 72]), __bfloat162float(wq[(4 * q + 3) * 72]));
    }
    if (threadIdx.x < 32) sb[threadIdx.x] = bias[threadIdx.x];
    const int tx = threadIdx.x % C0_TW, ty = threadIdx.x / C0_TW;
    const int ntx = (W + C0_TW - 1) / C0_TW, nty = (H + C0_TH - 1) / C0_TH;
    const long long ntiles = (long long)B * ntx * nty;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int bx = (int)(t % ntx);
        const long long r = t / ntx;
        const int by = (int)(r % nty);
        const long long b = r / nty;
        const int x0 = bx * C0_TW, y0 = by * C0_TH;
        __syncthreads();  // the previous tile is consumed (and the tables are ready)
        for (int i = threadIdx.x; i < (C0_TH + 2) * (C0_TW + 2); i += blockDim.x) {
            const int ly = i / (C0_TW + 2), lx = i % (C0_TW + 2);
            const int yy = y0 + ly - 1, xx = x0 + lx - 1;
            float2 v = make_float2(0.0f, 0.0f);
            if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
                const long long q = (b * H + yy) * W + xx;
                const float m = mask[q] ? 1.0f : 0.0f;
                v = make_float2(__bfloat162float(__float2bfloat16_rn(f[q] * m)), m);
            }
            tile[ly][lx] = v;
        }
        __syncthreads();
        const int x = x0 + tx, y = y0 + ty;
        if (x >= W || y >= H) continue;
        float acc[32];
#pragma unroll
        for (int co = 0; co < 32; ++co) acc[co] = 0.0f;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const float2 v = tile[ty + tap / 3][tx + tap % 3];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4 a = sw[tap][0][q], c = sw[tap][1][q];
                acc[4 * q + 0] = fmaf(c.x, v.y, fmaf(a.x, v.x, acc[4 * q + 0]));
                acc[4 * q + 1] = fmaf(c.y, v.y, fmaf(a.y, v.x, acc[4 * q + 1]));
                acc[4 * q + 2] = fmaf(c.z, v.y, fmaf(a.z, v.x, acc[4 * q + 2]));
                acc[4 * q + 3] = fmaf(c.w, v.y, fmaf(a.w, v.x, acc[4 * q + 3]));
            }
        }
        __align__(16) __nv_bfloat16 o[32];
#pragma unroll
        for (int co = 0; co < 32; ++co) o[co] = __float2bfloat16_rn(fmaxf(acc[co] + sb[co], 0.0f));
        uint4 *dst = (uint4 *)(out + ((b * H + y) * W + x) * 32);
#pragma unroll
        for (int k = 0; k < 4; ++k) dst[k] = ((const uint4 *)o)[k];
    }
}

// Gradient into an encoder output e: g_e = (pool_backward(g_pooled) + g_skip) * (e > 0),
// 8 channels (16 bytes) per thread; e has lde channels per pixel.
__global__ void k_pool_bwd_add_mask(const __nv_bfloat16 *gp, const __nv_bfloat16 *gskip, const __nv_bfloat16 *e,
                                    int lde, __nv_bfloat16 *ge, int B, int H, int W, int C) {
    const int C8 = C / 8, Ho = H / 2, Wo = W / 2;
    const long long total = (long long)B * H * W * C8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C8) * 8;
        const long long pix = i / C8;
        const int x = (int)(pix % W);
        const long long t = pix / W;
        const int y = (int)(t % H);
        const long long b = t / H;
        const uint4 vp = *(const uint4 *)(gp + ((b * Ho + y / 2) * Wo + x / 2) * C + c);
        const uint4 ve = *(const uint4 *)(e + pix * lde + c);
        uint4 vs = make_uint4(0, 0, 0, 0);
        if (gskip) vs = *(const uint4 *)(gskip + pix * C + c);
        const __nv_bfloat16 *hp = (const __nv_bfloat16 *)&vp, *he = (const __nv_bfloat16 *)&ve,
                            *hs = (const __nv_bfloat16 *)&vs;
        __align__(16) __nv_bfloat16 o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float v = 0.25f * __bfloat162float(hp[k]);
            if (gskip) v += __bfloat162float(hs[k]);
            if (!(__bfloat162float(he[k]) > 0.0f)) v = 0.0f;
            o[k] = __float2bfloat16_rn(v);
        }
        *(uint4 *)(ge + pix * C + c) = *(const uint4 *)o;
    }
}

// Gradient into a half-resolution tensor d that was upsampled (nearest):
// g_d = (sum over the 2x2 block of g_up) * (d > 0), 8 channels per thread.
__global__ void k_up_bwd_mask(const __nv_bfloat16 *gup, const __nv_bfloat16 *d, __nv_bfloat16 *gd, int B, int Hl,
                              int Wl, int C) {
    const int C8 = C / 8, H = 2 * Hl, W = 2 * Wl;
    const long long total = (long long)B * Hl * Wl * C8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C8) * 8;
        const long long pix = i / C8;
        const int x = (int)(pix % Wl);
        const long long t = pix / Wl;
        const int y = (int)(t % Hl);
        const long long b = t / Hl;
        const long long base = ((b * H + 2 * y) * W + 2 * x) * C + c;
        const uint4 q0 = *(const uint4 *)(gup + base), q1 = *(const uint4 *)(gup + base + C);
        const uint4 q2 = *(const uint4 *)(gup + base + (long long)W * C);
        const uint4 q3 = *(const uint4 *)(gup + base + (long long)W * C + C);
        const uint4 vd = *(const uint4 *)(d + pix * C + c);
        const __nv_bfloat16 *a = (const __nv_bfloat16 *)&q0, *b1 = (const __nv_bfloat16 *)&q1,
                            *c2 = (const __nv_bfloat16 *)&q2, *d3 = (const __nv_bfloat16 *)&q3,
                            *hd = (const __nv_bfloat16 *)&vd;
        __align__(16) __nv_bfloat16 o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float v = __bfloat162float(a[k]) + __bfloat162float(b1[k]) + __bfloat162float(c2[k]) +
                      __bfloat162float(d3[k]);
            if (!(__bfloat162float(hd[k]) > 0.0f)) v = 0.0f;
            o[k] = __float2bfloat16_rn(v);
        }
        *(uint4 *)(gd + pix * C + c) = *(const uint4 *)o;
    }
}

// Head: out[p] = sum_c w[c] d[p][c] + b (1x1 conv to one channel, FP32 out).
__global__ void k_head(const __nv_bfloat16 *d, const float *w, const float *b, const float *f, const uint8_t *mask,
                       float *out, long long P, int C) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        float s = b[0];
        for (int c = 0; c < C; ++c) s = fmaf(w[c], __bfloat162float(d[p * C + c]), s);
        out[p] = (mask[p] ? f[p] : 0.0f) + s;
    }
}

// Loss L = mean over pixels of (out - target)^2 and its gradient at the
// head, back into d: g_d[p][c] = g_out[p] w[c] (d > 0); also the head's
// parameter gradients. One pixel's 32 channels per thread (four 16-byte
// loads and stores); the partial sums are reduced across the warp with
// shuffles, then across the block in shared memory, one atomic each.
__global__ void __launch_bounds__(256) k_loss_head_bwd(const float *out, const float *target,
                                                       const __nv_bfloat16 *d, const float *w, __nv_bfloat16 *gd,
                                                       float *gw, float *gb, float *loss, long long P, int C,
                                                       float inv_n) {
    __shared__ float sgw[8][33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float lg = 0.0f, lb = 0.0f;
    float lw[32], wc[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        lw[c] = 0.0f;
        wc[c] = w[c];
    }
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const float r = out[p] - target[p];
        lg += r * r;
        const float go = 2.0f * r * inv_n;
        lb += go;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 v = *(const uint4 *)(d + p * C + 8 * q);
            const __nv_bfloat16 *h = (const __nv_bfloat16 *)&v;
            __align__(16) __nv_bfloat16 o[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float dv = __bfloat162float(h[k]);
                lw[8 * q + k] = fmaf(go, dv, lw[8 * q + k]);
                o[k] = __float2bfloat16_rn(dv > 0.0f ? go * wc[8 * q + k] : 0.0f);
            }
            *(uint4 *)(gd + p * C + 8 * q) = *(const uint4 *)o;
        }
    }
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        float v = lw[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sgw[wid][c] = v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        lg += __shfl_xor_sync(0xffffffffu, lg, o);
        lb += __shfl_xor_sync(0xffffffffu, lb, o);
    }
    if (lane == 0) {
        sgw[wid][32] = lb;
        atomicAdd(loss, lg * inv_n);
    }
    __syncthreads();
    if (threadIdx.x < 33) {
        float t = 0.0f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sgw[k][threadIdx.x];
        if (threadIdx.x < 32) atomicAdd(gw + threadIdx.x, t);
        else atomicAdd(gb, t);
    }
}

// Adam on the FP32 master parameters; refreshes the bf16 copy of the conv
// weights (bf16 index map: for i < n_bf16_span the bf16 copy mirrors p).
__global__ void k_adam(float *p, const float *g, float *m, float *v, __nv_bfloat16 *pb, long long n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float upd = lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        const float pi = p[i] - upd;
        p[i] = pi;
        pb[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void k_to_bf16(const float *p, __nv_bfloat16 *pb, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        pb[i] = __float2bfloat16_rn(p[i]);
}

// Per-image residual on the known pixels: r[b] = sqrt(mean over known
// pixels of (out - f)^2) (the fallback criterion of the surrogate).
__global__ void k_known_residual(const float *out, const float *f, const uint8_t *mask, int HW, float *r) {
    const int b = blockIdx.x;
    float s = 0.0f, n = 0.0f;
    for (int i = threadIdx.x; i < HW; i += blockDim.x) {
        const long long p = (long long)b * HW + i;
        if (mask[p]) {
            const float d = out[p] - f[p];
            s += d * d;
            n += 1.0f;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        n += __shfl_xor_sync(0xffffffffu, n, o);
    }
    __shared__ float ss[32], sn[32];
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = s;
        sn[threadIdx.x >> 5] = n;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float ts = 0.0f, tn = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            ts += ss[w];
            tn += sn[w];
        }
        r[b] = tn > 0.0f ? sqrtf(ts / tn) : 0.0f;
    }
}

int grid_for(long long n) {
    long long g = (n + 255) / 256;
    if (g > 65536) g = 65536;
    return (int)(g < 1 ? 1 : g);
}

template <int BM, int BN>
cudaError_t launch_fwd(const ConvInLoader &la, const WeightKLoader &lb, const float *bias, __nv_bfloat16 *out,
                       int relu, cudaStream_t s) {
    using S = Smem<BM, BN, true, true>;
    auto *fn = &k_conv_fwd<BM, BN>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, S::BYTES);
    dim3 grid((la.M + BM - 1) / BM, (lb.N + BN - 1) / BN);
    fn<<<grid, 128, S::BYTES, s>>>(la, lb, bias, out, relu);
    return cudaGetLastError();
}

template <int BM, int BN>
cudaError_t launch_dgrad(const ConvInLoader &la, const WeightNLoader &lb, const __nv_bfloat16 *act,
                         __nv_bfloat16 *din, __nv_bfloat16 *din2, int split, cudaStream_t s) {
    using S = Smem<BM, BN, true, false>;
    auto *fn = &k_conv_dgrad<BM, BN>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, S::BYTES);
    dim3 grid((la.M + BM - 1) / BM, (lb.Cin + BN - 1) / BN);
    fn<<<grid, 128, S::BYTES, s>>>(la, lb, act, din, din2, split);
    return cudaGetLastError();
}

template <int BM, int BN>
cudaError_t launch_wgrad(const GradOutMLoader &la, const InNLoader &lb, float *dw, int N, int splits, cudaStream_t s) {
    using S = Smem<BM, BN, false, false>;
    auto *fn = &k_conv_wgrad<BM, BN>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, S::BYTES);
    const int kt_total = (lb.P + kBK - 1) / kBK;
    const int per = (kt_total + splits - 1) / splits;
    dim3 grid((la.Cout + BM - 1) / BM, (N + BN - 1) / BN, (kt_total + per - 1) / per);
    fn<<<grid, 128, S::BYTES, s>>>(la, lb, dw, N, per);
    return cudaGetLastError();
}

template <int BN, int STAGES, int LAG>
cudaError_t launch_fwd_tc(const ConvInLoader &la, const WeightKLoader &lb, const FwdEpi &epi, cudaStream_t s) {
    constexpr int bytes = tc::smem_bytes<BN, STAGES>();
    auto *fn = &k_conv_fwd_tc<BN, STAGES, LAG>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    dim3 grid((la.M + tc::BM - 1) / tc::BM, lb.N / BN);
    fn<<<grid, 128, bytes, s>>>(la, lb, epi);
    return cudaGetLastError();
}

template <int BN, int STAGES, int LAG>
cudaError_t launch_dgrad_tc(const ConvInLoader &la, const WeightKLoader &lb, const DgradEpi &epi, cudaStream_t s) {
    constexpr int bytes = tc::smem_bytes<BN, STAGES>();
    auto *fn = &k_conv_dgrad_tc<BN, STAGES, LAG>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    dim3 grid((la.M + tc::BM - 1) / tc::BM, lb.N / BN);
    fn<<<grid, 128, bytes, s>>>(la, lb, epi);
    return cudaGetLastError();
}

}  // namespace

namespace se2n {
namespace nn {

cudaError_t tc_fault(int *host_flag, bool reset) {
    cudaError_t e = cudaMemcpyFromSymbol(host_flag, g_tc_fault, sizeof(int));
    if (e == cudaSuccess && reset && *host_flag) {
        const int zero = 0;
        e = cudaMemcpyToSymbol(g_tc_fault, &zero, sizeof(int));
    }
    int t = 0;
    if (e == cudaSuccess) e = tma_fault(&t, reset);
    if (e == cudaSuccess) *host_flag |= t;
    return e;
}

cudaError_t conv_forward(const __nv_bfloat16 *in, const __nv_bfloat16 *lo, int C1, int B, int H, int W, int Cin,
                         const __nv_bfloat16 *w, const float *bias, int Cout, int relu, __nv_bfloat16 *out, int ldo,
                         cudaStream_t s) {
    if (!lo) {
        const cudaError_t e = conv_forward_tma(in, B, H, W, Cin, w, bias, Cout, relu, out, ldo, nullptr, s);
        if (e != cudaErrorNotSupported) return e;
    }
    ConvInLoader la{{B, H, W}, in, lo, Cin, C1, B * H * W, 9 * Cin, 0};
    WeightKLoader lb{w, Cout, 9 * Cin};
    const FwdEpi epi{bias, out, ldo, relu};
    switch (Cout) {
        case 32: return launch_fwd_tc<32, 4, 2>(la, lb, epi, s);
        case 64: return launch_fwd_tc<64, 4, 2>(la, lb, epi, s);
        case 128: return launch_fwd_tc<128, 4, 2>(la, lb, epi, s);
        case 256: return launch_fwd_tc<256, 4, 2>(la, lb, epi, s);
        default: break;
    }
    if (ldo != Cout) return cudaErrorNotSupported;
    if (Cout <= 32) return launch_fwd<128, 32>(la, lb, bias, out, relu, s);
    if (Cout <= 64) return launch_fwd<128, 64>(la, lb, bias, out, relu, s);
    return launch_fwd<128, 128>(la, lb, bias, out, relu, s);
}

cudaError_t conv_backward_data(const __nv_bfloat16 *gz, int B, int H, int W, int Cout, const __nv_bfloat16 *w, int Cin,
                               const __nv_bfloat16 *act, __nv_bfloat16 *din, __nv_bfloat16 *din2, int split,
                               __nv_bfloat16 *wt_scratch, cudaStream_t s) {
    ConvInLoader la{{B, H, W}, gz, nullptr, Cout, 0, B * H * W, 9 * Cout, 1};
    if (wt_scratch && Cin % 32 == 0 && split % 16 == 0) {
        const long long nw = (long long)Cout * 9 * Cin;
        k_transpose_dgrad<<<grid_for(nw), 256, 0, s>>>(w, wt_scratch, Cout, Cin);
        const cudaError_t e = conv_dgrad_tma(gz, B, H, W, Cout, wt_scratch, Cin, act, din, din2, split, s);
        if (e != cudaErrorNotSupported) return e;
        const WeightKLoader lt{wt_scratch, Cin, 9 * Cout};
        const DgradEpi epi{act, din, din2, split, Cin};
        switch (Cin) {
            case 32: return launch_dgrad_tc<32, 4, 2>(la, lt, epi, s);
            case 64: return launch_dgrad_tc<64, 4, 2>(la, lt, epi, s);
            case 96: return launch_dgrad_tc<96, 4, 2>(la, lt, epi, s);
            case 128: return launch_dgrad_tc<128, 4, 2>(la, lt, epi, s);
            case 192: return launch_dgrad_tc<192, 4, 2>(la, lt, epi, s);
            case 256: return launch_dgrad_tc<256, 4, 2>(la, lt, epi, s);
            case 384: return launch_dgrad_tc<192, 4, 2>(la, lt, epi, s);
            default: break;
        }
    }
    WeightNLoader lb{w, Cout, Cin, 9 * Cout};
    if (Cin <= 32) return launch_dgrad<128, 32>(la, lb, act, din, din2, split, s);
    if (Cin <= 64) return launch_dgrad<128, 64>(la, lb, act, din, din2, split, s);
    return launch_dgrad<128, 128>(la, lb, act, din, din2, split, s);
}

cudaError_t conv_backward_weight(const __nv_bfloat16 *gz, int B, int H, int W, int Cout, const __nv_bfloat16 *in,
                                 const __nv_bfloat16 *lo, int C1, int Cin, float *dw, cudaStream_t s) {
    if (!lo) {
        const cudaError_t e = conv_wgrad_tma(in, B, H, W, Cin, gz, Cout, dw, s);
        if (e != cudaErrorNotSupported) return e;
    }
    const int P = B * H * W;
    GradOutMLoader la{gz, Cout, P};
    InNLoader lb{{{B, H, W}, in, lo, Cin, C1, P, 9 * Cin, 0}, P};
    const int N = 9 * Cin;
    const int kt_total = (P + kBK - 1) / kBK;
    // enough CTAs to fill the GPU, each reducing a slab of pixels
    const int tiles = ((Cout + 63) / 64) * ((N + 63) / 64);
    int splits = (4 * 152 + tiles - 1) / tiles;
    if (splits > kt_total) splits = kt_total;
    if (splits < 1) splits = 1;
    if (Cout <= 32) return launch_wgrad<32, 64>(la, lb, dw, N, splits, s);
    if (Cout <= 64) return launch_wgrad<64, 64>(la, lb, dw, N, splits, s);
    return launch_wgrad<128, 64>(la, lb, dw, N, splits, s);
}

cudaError_t colsum(const __nv_bfloat16 *g, long long P, int C, float *db, cudaStream_t s) {
    k_colsum<<<1024, 256, 0, s>>>(g, P, C, db);
    return cudaGetLastError();
}

cudaError_t pack_input(const float *f, const uint8_t *mask, __nv_bfloat16 *x, long long P, cudaStream_t s) {
    k_pack_input<<<grid_for(P), 256, 0, s>>>(f, mask, x, P);
    return cudaGetLastError();
}

cudaError_t pool(const __nv_bfloat16 *in, int ldi, __nv_bfloat16 *out, int B, int H, int W, int C, cudaStream_t s) {
    k_pool<<<grid_for((long long)B * H * W * C / 32), 256, 0, s>>>(in, ldi, out, B, H, W, C);
    return cudaGetLastError();
}

cudaError_t upsample_into(const __nv_bfloat16 *lo, int C1, __nv_bfloat16 *out, int ldo, int B, int H, int W,
                          cudaStream_t s) {
    k_upsample_into<<<B * H, 256, 0, s>>>(lo, C1, out, ldo, H, W);
    return cudaGetLastError();
}

cudaError_t conv0_direct(const float *f, const uint8_t *mask, const __nv_bfloat16 *w, const float *bias,
                         __nv_bfloat16 *out, int B, int H, int W, cudaStream_t s) {
    // a few blocks per SM, each over many pixels: the weight table is built once per block
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int g = grid_for((long long)B * H * W);
    if (nsm > 0 && g > 8 * nsm) g = 8 * nsm;
    k_conv0<<<g, 256, 0, s>>>(f, mask, w, bias, out, B, H, W);
    return cudaGetLastError();
}

cudaError_t pool_backward_add_mask(const __nv_bfloat16 *gp, const __nv_bfloat16 *gskip, const __nv_bfloat16 *e, int lde,
                                   __nv_bfloat16 *ge, int B, int H, int W, int C, cudaStream_t s) {
    k_pool_bwd_add_mask<<<grid_for((long long)B * H * W * C / 8), 256, 0, s>>>(gp, gskip, e, lde, ge, B, H, W, C);
    return cudaGetLastError();
}

cudaError_t up_backward_mask(const __nv_bfloat16 *gup, const __nv_bfloat16 *d, __nv_bfloat16 *gd, int B, int Hl,
                             int Wl, int C, cudaStream_t s) {
    k_up_bwd_mask<<<grid_for((long long)B * Hl * Wl * C / 8), 256, 0, s>>>(gup, d, gd, B, Hl, Wl, C);
    return cudaGetLastError();
}

cudaError_t head(const __nv_bfloat16 *d, const float *w, const float *b, const float *f, const uint8_t *mask,
                 float *out, long long P, int C, cudaStream_t s) {
    k_head<<<grid_for(P), 256, 0, s>>>(d, w, b, f, mask, out, P, C);
    return cudaGetLastError();
}

cudaError_t loss_head_backward(const float *out, const float *target, const __nv_bfloat16 *d, const float *w,
                               __nv_bfloat16 *gd, float *gw, float *gb, float *loss, long long P, int C,
                               cudaStream_t s) {
    int g = grid_for(P);
    if (g > 2048) g = 2048;
    k_loss_head_bwd<<<g, 256, 0, s>>>(out, target, d, w, gd, gw, gb, loss, P, C, 1.0f / (float)P);
    return cudaGetLastError();
}

cudaError_t adam(float *p, const float *g, float *m, float *v, __nv_bfloat16 *pb, long long n, float lr, float b1,
                 float b2, float eps, int t, cudaStream_t s) {
    const float c1 = 1.0f / (1.0f - powf(b1, (float)t));
    const float c2 = 1.0f / (1.0f - powf(b2, (float)t));
    k_adam<<<grid_for(n), 256, 0, s>>>(p, g, m, v, pb, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t to_bf16(const float *p, __nv_bfloat16 *pb, long long n, cudaStream_t s) {
    k_to_bf16<<<grid_for(n), 256, 0, s>>>(p, pb, n);
    return cudaGetLastError();
}

cudaError_t known_residual(const float *out, const float *f, const uint8_t *mask, int B, int HW, float *r,
                           cudaStream_t s) {
    k_known_residual<<<B, 256, 0, s>>>(out, f, mask, HW, r);
    return cudaGetLastError();
}

}  // namespace nn
}  // namespace se2n
