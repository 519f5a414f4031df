// Operand loaders of the implicit-GEMM convolutions: each returns the address
// of the 16-byte chunk holding 8 consecutive elements along the operand's
// contiguous dimension, or null for a chunk of zeros.
#pragma once

#include <cuda_bf16.h>

namespace se2n {
namespace nn {

struct Geo {
    int B, H, W;
    __device__ __forceinline__ void pix(int m, int &b, int &y, int &x) const {
        x = m % W;
        const int t = m / W;
        y = t % H;
        b = t / H;
    }
};

// A operand of a forward conv: the input activation, gathered per tap. The
// input may be the concatenation [nearest-upsample(lo), skip] along
// channels: channels < C1 come from `lo` at half resolution, the rest from
// `skip` at full resolution.
struct ConvInLoader {
    Geo g;
    const __nv_bfloat16 *src;   // full-resolution source (or the skip part)
    const __nv_bfloat16 *lo;    // half-resolution upsampled part, or null
    int C, C1, M, K;            // C = total input channels; C1 = channels from `lo`
    int flip;                   // 1: taps mirrored (backward data)
    // Address of channels c..c+7 of input pixel (b, yy, xx), inside the image.
    __device__ __forceinline__ const void *at(int b, int yy, int xx, int c) const {
        if (lo && c < C1) {
            const int Wl = g.W >> 1, Hl = g.H >> 1;
            return lo + (((long long)b * Hl + (yy >> 1)) * Wl + (xx >> 1)) * C1 + c;
        }
        const int Cs = lo ? C - C1 : C;
        const int cs = lo ? c - C1 : c;
        return src + (((long long)b * g.H + yy) * g.W + xx) * Cs + cs;
    }
    __device__ __forceinline__ const void *chunk(int m, int k) const {
        if (m >= M || k >= K) return nullptr;
        const int tap = k / C, c = k - tap * C;
        int dy = tap / 3 - 1, dx = tap % 3 - 1;
        if (flip) {
            dy = -dy;
            dx = -dx;
        }
        int b, y, x;
        g.pix(m, b, y, x);
        const int yy = y + dy, xx = x + dx;
        if (yy < 0 || yy >= g.H || xx < 0 || xx >= g.W) return nullptr;
        return at(b, yy, xx, c);
    }
};

// B operand of a forward conv: weights W[co][k], K-major.
struct WeightKLoader {
    const __nv_bfloat16 *w;
    int N, K;
    __device__ __forceinline__ const void *chunk(int n, int k) const {
        return (n < N && k < K) ? (const void *)(w + (long long)n * K + k) : nullptr;
    }
};

}  // namespace nn
}  // namespace se2n
