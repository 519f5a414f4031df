// Pixel-wise stages of the path: orientation (smoothing and gradient in the
// DFT domain), lift, static restoration and projection. All HBM-bound:
// consecutive threads own consecutive pixel pairs, so every access of a
// plane is a coalesced 16-byte (two complex) or 8-byte (two float) access.
// H and W are even, so a pixel pair never straddles a plane and every plane
// starts 16-byte aligned.
#include "restore.cuh"
#include "se2n_internal.h"

namespace {

constexpr int kBlock = 256;

inline int grid_for(long long n, int per_block = kBlock) {
    long long g = (n + per_block - 1) / per_block;
    if (g > 1048576) g = 1048576;  // grid-stride beyond this
    return (int)(g < 1 ? 1 : g);
}

// spec = f * (mask != 0) as complex, two pixels per thread.
__global__ void k_orient_prep(const float2 *__restrict__ f, const uchar2 *__restrict__ mask,
                              float4 *__restrict__ spec, long long npairs) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npairs;
         i += (long long)gridDim.x * blockDim.x) {
        const float2 v = f[i];
        const uchar2 m = mask[i];
        spec[i] = make_float4(m.x ? v.x : 0.0f, 0.0f, m.y ? v.y : 0.0f, 0.0f);
    }
}

// From the image spectrum F, write the spectra of the smoothed x and y
// derivatives: F * g * (i 2 pi l~/W) and F * g * (i 2 pi k~/H), with
// g = exp(-2 pi^2 sigma^2 ((k~/H)^2 + (l~/W)^2)), k~, l~ the signed
// frequencies and the Nyquist derivative term set to zero.
__global__ void k_grad_spec(const float2 *__restrict__ F, float2 *__restrict__ gx, float2 *__restrict__ gy,
                            int H, int W, float sigma) {
    const long long HW = (long long)H * W;
    const float two_pi = 6.28318530717958647692f;
    const float c = -2.0f * 9.86960440108935861883f * sigma * sigma;  // -2 pi^2 sigma^2
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HW;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i / W), l = (int)(i - (long long)k * W);
        const int ks = (2 * k >= H) ? k - H : k;
        const int ls = (2 * l >= W) ? l - W : l;
        const float fy = (float)ks / (float)H, fx = (float)ls / (float)W;
        const float g = expf(c * (fx * fx + fy * fy));
        const float dx = (2 * ls == -W) ? 0.0f : two_pi * fx * g;
        const float dy = (2 * ks == -H) ? 0.0f : two_pi * fy * g;
        const float2 v = F[i];
        gx[i] = make_float2(-v.y * dx, v.x * dx);  // i * dx * F
        gy[i] = make_float2(-v.y * dy, v.x * dy);
    }
}

// max over pixels of |grad|^2 (real parts of the inverse transforms); the
// scale of the unnormalised inverse cancels in every later use.
__global__ void k_grad_max(const float2 *__restrict__ gx, const float2 *__restrict__ gy, long long HW,
                           unsigned int *__restrict__ gmax) {
    float m = 0.0f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HW;
         i += (long long)gridDim.x * blockDim.x) {
        const float x = gx[i].x, y = gy[i].x;
        m = fmaxf(m, fmaf(x, x, y * y));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wm[kBlock / 32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = (threadIdx.x < blockDim.x / 32) ? wm[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        // non-negative floats order like their bit patterns
        if (threadIdx.x == 0) atomicMax(gmax, __float_as_uint(m));
    }
}

// bin = floor(phi / dth + 1/2) mod N with phi = atan2(gy, gx) + pi/2 in
// [0, pi); flat pixels (|grad|^2 <= flat_tol^2 max|grad|^2) get SE2N_BIN_FLAT.
__global__ void k_bins(const float2 *__restrict__ gx, const float2 *__restrict__ gy, long long HW,
                       const unsigned int *__restrict__ gmax, float flat_tol2, int N, float inv_dth,
                       uint8_t *__restrict__ bins) {
    const float pi = 3.14159265358979323846f;
    const float thresh = flat_tol2 * __uint_as_float(*gmax);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HW;
         i += (long long)gridDim.x * blockDim.x) {
        const float x = gx[i].x, y = gy[i].x;
        const float m2 = fmaf(x, x, y * y);
        uint8_t b = SE2N_BIN_FLAT;
        if (!(m2 <= thresh)) {
            float phi = atan2f(y, x) + 0.5f * pi;
            if (phi >= pi) phi -= pi;
            if (phi < 0.0f) phi += pi;
            const float u = fmaf(phi, inv_dth, 0.5f);
            int r = (int)floorf(u);
            r %= N;
            if (r < 0) r += N;
            b = (uint8_t)r;
        }
        bins[i] = b;
    }
}

// vol[r][y][x] = f0 on the pixel's bin (all bins if flat), 0 elsewhere.
__global__ void k_lift(const float2 *__restrict__ f, const uchar2 *__restrict__ mask,
                       const uchar2 *__restrict__ bins, float4 *__restrict__ vol, long long npairs, int N) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npairs;
         i += (long long)gridDim.x * blockDim.x) {
        const float2 v = f[i];
        const uchar2 m = mask[i];
        const uchar2 b = bins[i];
        const float a0 = m.x ? v.x : 0.0f, a1 = m.y ? v.y : 0.0f;
        for (int r = 0; r < N; ++r) {
            const bool on0 = (b.x == r) || (b.x == SE2N_BIN_FLAT);
            const bool on1 = (b.y == r) || (b.y == SE2N_BIN_FLAT);
            vol[(long long)r * npairs + i] = make_float4(on0 ? a0 : 0.0f, 0.0f, on1 ? a1 : 0.0f, 0.0f);
        }
    }
}

using se2n::sr_value;

// ht_given (if not null): h(t) of every pixel, the maximum over all angles,
// of which vol may hold only some planes (an angle shard; bins then name
// no plane of vol for the pixels lifted elsewhere).
__global__ void k_mix(float4 *__restrict__ vol, const float2 *__restrict__ f, const uchar2 *__restrict__ mask,
                      const uchar2 *__restrict__ bins, long long npairs, int N, float scale, float eps,
                      float guard, const float2 *__restrict__ ht_given) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npairs;
         i += (long long)gridDim.x * blockDim.x) {
        float ht0 = -INFINITY, ht1 = -INFINITY;
        if (ht_given) {
            const float2 h = ht_given[i];
            ht0 = h.x;
            ht1 = h.y;
        } else {
            for (int r = 0; r < N; ++r) {
                const float4 v = vol[(long long)r * npairs + i];
                ht0 = fmaxf(ht0, v.x * scale);
                ht1 = fmaxf(ht1, v.z * scale);
            }
        }
        const float2 fv = f[i];
        const uchar2 m = mask[i];
        const uchar2 b = bins[i];
        const float a0 = m.x ? fv.x : 0.0f, a1 = m.y ? fv.y : 0.0f;
        // max over angles of the lift: the value itself if it sits on every
        // angle or is not negative (N >= 2 leaves zeros on the other angles)
        const float h00 = (b.x == SE2N_BIN_FLAT) ? a0 : fmaxf(a0, 0.0f);
        const float h01 = (b.y == SE2N_BIN_FLAT) ? a1 : fmaxf(a1, 0.0f);
        for (int r = 0; r < N; ++r) {
            const long long o = (long long)r * npairs + i;
            const float4 v = vol[o];
            const float l0 = ((b.x == r) || (b.x == SE2N_BIN_FLAT)) ? a0 : 0.0f;
            const float l1 = ((b.y == r) || (b.y == SE2N_BIN_FLAT)) ? a1 : 0.0f;
            vol[o] = make_float4(sr_value(v.x * scale, h00, ht0, l0, m.x != 0, eps, guard), 0.0f,
                                 sr_value(v.z * scale, h01, ht1, l1, m.y != 0, eps, guard), 0.0f);
        }
    }
}

__global__ void k_project(const float4 *__restrict__ vol, long long npairs, int N, float scale, int proj,
                          const float2 *__restrict__ f, const uchar2 *__restrict__ mask, float2 *__restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npairs;
         i += (long long)gridDim.x * blockDim.x) {
        float a0, a1;
        if (proj == SE2N_PROJ_MAX) {
            a0 = -INFINITY;
            a1 = -INFINITY;
            for (int r = 0; r < N; ++r) {
                const float4 v = vol[(long long)r * npairs + i];
                a0 = fmaxf(a0, v.x * scale);
                a1 = fmaxf(a1, v.z * scale);
            }
        } else {
            a0 = 0.0f;
            a1 = 0.0f;
            for (int r = 0; r < N; ++r) {
                const float4 v = vol[(long long)r * npairs + i];
                a0 += v.x * scale;
                a1 += v.z * scale;
            }
            a0 /= (float)N;
            a1 /= (float)N;
        }
        if (mask) {
            const uchar2 m = mask[i];
            const float2 fv = f[i];
            if (m.x) a0 = fv.x;
            if (m.y) a1 = fv.y;
        }
        out[i] = make_float2(a0, a1);
    }
}

// ---------------------------------------------------------------------------
// The same stages on the real volume of the Hermitian-half path: planes of
// H rows of Wp = W + 2 floats (the in-place R2C layout), pixel (y, x) of
// plane r at r * H * Wp + y * Wp + x. Two pixels per thread (W even).
// ---------------------------------------------------------------------------

__device__ __forceinline__ long long real_off(long long i, int W, int Wp) {
    const long long p = 2 * i;
    const long long y = p / W;
    return y * Wp + (p - y * W);
}

__global__ void k_lift_r(const float2 *__restrict__ f, const uchar2 *__restrict__ mask,
                         const uchar2 *__restrict__ bins, float *__restrict__ vol, long long npairs, int W, int Wp,
                         long long plane, int N) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npairs;
         i += (long long)gridDim.x * blockDim.x) {
        const float2 v = f[i];
        const uchar2 m = mask[i];
        const uchar2 b = bins[i];
        const float a0 = m.x ? v.x : 0.0f, a1 = m.y ? v.y : 0.0f;
        float2 *out = (float2 *)(vol + real_off(i, W, Wp));
        for (int r = 0; r < N; ++r) {
            const bool on0 = (b.x == r) || (b.x == SE2N_BIN_FLAT);
            const bool on1 = (b.y == r) || (b.y == SE2N_BIN_FLAT);
            out[(long long)r * (plane / 2)] = make_float2(on0 ? a0 : 0.0f, on1 ? a1 : 0.0f);
        }
    }
}

__global__ void k_mix_r(float *__restrict__ vol, const float2 *__restrict__ f, const uchar2 *__restrict__ mask,
                        const uchar2 *__restrict__ bins, long long npairs, int W, int Wp, long long plane, int N,
                        float scale, float eps, float guard) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npairs;
         i += (long long)gridDim.x * blockDim.x) {
        float2 *col = (float2 *)(vol + real_off(i, W, Wp));
        const long long ps = plane / 2;
        float ht0 = -INFINITY, ht1 = -INFINITY;
        for (int r = 0; r < N; ++r) {
            const float2 v = col[(long long)r * ps];
            ht0 = fmaxf(ht0, v.x * scale);
            ht1 = fmaxf(ht1, v.y * scale);
        }
        const float2 fv = f[i];
        const uchar2 m = mask[i];
        const uchar2 b = bins[i];
        const float a0 = m.x ? fv.x : 0.0f, a1 = m.y ? fv.y : 0.0f;
        const float h00 = (b.x == SE2N_BIN_FLAT) ? a0 : fmaxf(a0, 0.0f);
        const float h01 = (b.y == SE2N_BIN_FLAT) ? a1 : fmaxf(a1, 0.0f);
        for (int r = 0; r < N; ++r) {
            const float2 v = col[(long long)r * ps];
            const float l0 = ((b.x == r) || (b.x == SE2N_BIN_FLAT)) ? a0 : 0.0f;
            const float l1 = ((b.y == r) || (b.y == SE2N_BIN_FLAT)) ? a1 : 0.0f;
            col[(long long)r * ps] = make_float2(sr_value(v.x * scale, h00, ht0, l0, m.x != 0, eps, guard),
                                                 sr_value(v.y * scale, h01, ht1, l1, m.y != 0, eps, guard));
        }
    }
}

__global__ void k_project_r(const float *__restrict__ vol, long long npairs, int W, int Wp, long long plane, int N,
                            float scale, int proj, const float2 *__restrict__ f, const uchar2 *__restrict__ mask,
                            float2 *__restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npairs;
         i += (long long)gridDim.x * blockDim.x) {
        const float2 *col = (const float2 *)(vol + real_off(i, W, Wp));
        const long long ps = plane / 2;
        float a0, a1;
        if (proj == SE2N_PROJ_MAX) {
            a0 = -INFINITY;
            a1 = -INFINITY;
            for (int r = 0; r < N; ++r) {
                const float2 v = col[(long long)r * ps];
                a0 = fmaxf(a0, v.x * scale);
                a1 = fmaxf(a1, v.y * scale);
            }
        } else {
            a0 = 0.0f;
            a1 = 0.0f;
            for (int r = 0; r < N; ++r) {
                const float2 v = col[(long long)r * ps];
                a0 += v.x * scale;
                a1 += v.y * scale;
            }
            a0 /= (float)N;
            a1 /= (float)N;
        }
        if (mask) {
            const uchar2 m = mask[i];
            const float2 fv = f[i];
            if (m.x) a0 = fv.x;
            if (m.y) a1 = fv.y;
        }
        out[i] = make_float2(a0, a1);
    }
}

// ---------------------------------------------------------------------------
// Dynamic restoration (Section 5.3): the good set grows before a restoration.
// ---------------------------------------------------------------------------

// Image value h = max over angles of scale * Re psi and the angle of its
// first maximum, one pixel a thread; vol is the complex volume [N][HW].
__global__ void k_dr_max(const float2 *__restrict__ vol, long long HW, int N, float scale, float *__restrict__ h,
                         uint8_t *__restrict__ amax) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HW;
         i += (long long)gridDim.x * blockDim.x) {
        float best = -INFINITY;
        int arg = 0;
        for (int r = 0; r < N; ++r) {
            const float v = vol[(long long)r * HW + i].x * scale;
            if (v > best) {
                best = v;
                arg = r;
            }
        }
        h[i] = best;
        amax[i] = (uint8_t)arg;
    }
}

// The same on the real volume of the Hermitian-half path (planes of H rows
// of Wp = W + 2 floats).
__global__ void k_dr_max_r(const float *__restrict__ vol, long long HW, int W, int Wp, long long plane, int N,
                           float scale, float *__restrict__ h, uint8_t *__restrict__ amax) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HW;
         i += (long long)gridDim.x * blockDim.x) {
        const long long y = i / W;
        const float *col = vol + y * Wp + (i - y * W);
        float best = -INFINITY;
        int arg = 0;
        for (int r = 0; r < N; ++r) {
            const float v = col[(long long)r * plane] * scale;
            if (v > best) {
                best = v;
                arg = r;
            }
        }
        h[i] = best;
        amax[i] = (uint8_t)arg;
    }
}

// One growth step of the good set. A bad pixel with a good 8-neighbour joins
// when h exceeds the mean of h over the bad pixels of its 3x3 block inside
// the image: summed in FP32 row by row, top to bottom and left to right,
// then one IEEE division. Every decision reads mask_in only (the sets before
// the step); a joining pixel takes fref = h and bins = amax, which no other
// thread reads here. mask_out holds 1 for good, 0 for bad.
__global__ void k_dr_grow(const float *__restrict__ h, const uint8_t *__restrict__ amax,
                          const uint8_t *__restrict__ mask_in, uint8_t *__restrict__ mask_out, float *__restrict__ fref,
                          uint8_t *__restrict__ bins, int H, int W) {
    const long long HW = (long long)H * W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HW;
         i += (long long)gridDim.x * blockDim.x) {
        if (mask_in[i]) {
            mask_out[i] = 1;
            continue;
        }
        const int y = (int)(i / W);
        const int x = (int)(i - (long long)y * W);
        float sum = 0.0f;
        int cnt = 0;
        bool touches = false;
        for (int dy = -1; dy <= 1; ++dy) {
            const int yy = y + dy;
            if (yy < 0 || yy >= H) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                const int xx = x + dx;
                if (xx < 0 || xx >= W) continue;
                const long long q = (long long)yy * W + xx;
                if (mask_in[q]) {
                    touches = true;
                } else {
                    sum += h[q];
                    ++cnt;
                }
            }
        }
        const float hv = h[i];
        const bool join = touches && hv > sum / (float)cnt;  // cnt >= 1: the pixel itself
        mask_out[i] = join ? 1 : 0;
        if (join) {
            fref[i] = hv;
            bins[i] = amax[i];
        }
    }
}

__global__ void k_scale(float4 *__restrict__ v, long long n4, float s) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
         i += (long long)gridDim.x * blockDim.x) {
        float4 a = v[i];
        a.x *= s; a.y *= s; a.z *= s; a.w *= s;
        v[i] = a;
    }
}

}  // namespace

cudaError_t se2n_launch_orient_prep(const float *f, const uint8_t *mask, float2 *spec, long long HW,
                                    cudaStream_t s) {
    const long long n = HW / 2;
    k_orient_prep<<<grid_for(n), kBlock, 0, s>>>((const float2 *)f, (const uchar2 *)mask, (float4 *)spec, n);
    return cudaGetLastError();
}

cudaError_t se2n_launch_grad_spec(float2 *spec, int H, int W, float sigma, cudaStream_t s) {
    const long long HW = (long long)H * W;
    k_grad_spec<<<grid_for(HW), kBlock, 0, s>>>(spec, spec + HW, spec + 2 * HW, H, W, sigma);
    return cudaGetLastError();
}

cudaError_t se2n_launch_grad_max(const float2 *gx, const float2 *gy, long long HW, unsigned int *gmax,
                                 cudaStream_t s) {
    int g = grid_for(HW);
    if (g > 4096) g = 4096;
    k_grad_max<<<g, kBlock, 0, s>>>(gx, gy, HW, gmax);
    return cudaGetLastError();
}

cudaError_t se2n_launch_bins(const float2 *gx, const float2 *gy, long long HW, const unsigned int *gmax,
                             float flat_tol2, int N, int angle_conv, uint8_t *bins, cudaStream_t s) {
    const float dth = (angle_conv ? 2.0f : 1.0f) * 3.14159265358979323846f / (float)N;
    k_bins<<<grid_for(HW), kBlock, 0, s>>>(gx, gy, HW, gmax, flat_tol2, N, 1.0f / dth, bins);
    return cudaGetLastError();
}

cudaError_t se2n_launch_lift(const float *f, const uint8_t *mask, const uint8_t *bins, float2 *vol,
                             long long HW, int N, cudaStream_t s) {
    const long long n = HW / 2;
    k_lift<<<grid_for(n), kBlock, 0, s>>>((const float2 *)f, (const uchar2 *)mask, (const uchar2 *)bins,
                                          (float4 *)vol, n, N);
    return cudaGetLastError();
}

cudaError_t se2n_launch_mix(float2 *vol, const float *f, const uint8_t *mask, const uint8_t *bins,
                            long long HW, int N, float scale, float eps, float guard, cudaStream_t s) {
    const long long n = HW / 2;
    k_mix<<<grid_for(n), kBlock, 0, s>>>((float4 *)vol, (const float2 *)f, (const uchar2 *)mask,
                                         (const uchar2 *)bins, n, N, scale, eps, guard, nullptr);
    return cudaGetLastError();
}

cudaError_t se2n_launch_mix_given(float2 *vol, const float *f, const uint8_t *mask, const uint8_t *bins,
                                  const float *h_t, long long HW, int N, float eps, float guard, cudaStream_t s) {
    const long long n = HW / 2;
    k_mix<<<grid_for(n), kBlock, 0, s>>>((float4 *)vol, (const float2 *)f, (const uchar2 *)mask,
                                         (const uchar2 *)bins, n, N, 1.0f, eps, guard, (const float2 *)h_t);
    return cudaGetLastError();
}

cudaError_t se2n_launch_project(const float2 *vol, long long HW, int N, float scale, int proj, const float *f,
                                const uint8_t *mask, float *out, cudaStream_t s) {
    const long long n = HW / 2;
    k_project<<<grid_for(n), kBlock, 0, s>>>((const float4 *)vol, n, N, scale, proj, (const float2 *)f,
                                             (const uchar2 *)mask, (float2 *)out);
    return cudaGetLastError();
}

cudaError_t se2n_launch_lift_r(const float *f, const uint8_t *mask, const uint8_t *bins, float *vol, int H, int W,
                               int N, cudaStream_t s) {
    const long long n = (long long)H * W / 2;
    const int Wp = W + 2;
    k_lift_r<<<grid_for(n), kBlock, 0, s>>>((const float2 *)f, (const uchar2 *)mask, (const uchar2 *)bins, vol, n, W,
                                            Wp, (long long)H * Wp, N);
    return cudaGetLastError();
}

cudaError_t se2n_launch_mix_r(float *vol, const float *f, const uint8_t *mask, const uint8_t *bins, int H, int W,
                              int N, float scale, float eps, float guard, cudaStream_t s) {
    const long long n = (long long)H * W / 2;
    const int Wp = W + 2;
    k_mix_r<<<grid_for(n), kBlock, 0, s>>>(vol, (const float2 *)f, (const uchar2 *)mask, (const uchar2 *)bins, n, W, Wp,
                                           (long long)H * Wp, N, scale, eps, guard);
    return cudaGetLastError();
}

cudaError_t se2n_launch_project_r(const float *vol, int H, int W, int N, float scale, int proj, const float *f,
                                  const uint8_t *mask, float *out, cudaStream_t s) {
    const long long n = (long long)H * W / 2;
    const int Wp = W + 2;
    k_project_r<<<grid_for(n), kBlock, 0, s>>>(vol, n, W, Wp, (long long)H * Wp, N, scale, proj, (const float2 *)f,
                                               (const uchar2 *)mask, (float2 *)out);
    return cudaGetLastError();
}

cudaError_t se2n_launch_dr_max(const float2 *vol, long long HW, int N, float scale, float *h, uint8_t *amax,
                               cudaStream_t s) {
    k_dr_max<<<grid_for(HW), kBlock, 0, s>>>(vol, HW, N, scale, h, amax);
    return cudaGetLastError();
}

cudaError_t se2n_launch_dr_max_r(const float *vol, int H, int W, int N, float scale, float *h, uint8_t *amax,
                                 cudaStream_t s) {
    const long long HW = (long long)H * W;
    const int Wp = W + 2;
    k_dr_max_r<<<grid_for(HW), kBlock, 0, s>>>(vol, HW, W, Wp, (long long)H * Wp, N, scale, h, amax);
    return cudaGetLastError();
}

cudaError_t se2n_launch_dr_grow(const float *h, const uint8_t *amax, const uint8_t *mask_in, uint8_t *mask_out,
                                float *fref, uint8_t *bins, int H, int W, cudaStream_t s) {
    k_dr_grow<<<grid_for((long long)H * W), kBlock, 0, s>>>(h, amax, mask_in, mask_out, fref, bins, H, W);
    return cudaGetLastError();
}

cudaError_t se2n_launch_scale(float2 *vol, long long count, float scale, cudaStream_t s) {
    const long long n4 = count / 2;
    k_scale<<<grid_for(n4), kBlock, 0, s>>>((float4 *)vol, n4, scale);
    return cudaGetLastError();
}
