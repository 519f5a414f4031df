// The S-step propagator of the Crank-Nicolson integration of eq. (deceq).
//
// Every interval of se2n_inpaint integrates T/rounds in S steps with the same
// beta, so for one frequency the S steps are one fixed linear map: the
// step matrix M = B-^{-1} B+ raised to the power S. The paper notes that the
// integration can be replaced by such a precomputed propagator (Section 4,
// after Theorem 2). Here it is computed once per class of frequencies with
// bitwise equal coefficients and applied as one N x N matrix-vector product
// per frequency and interval.
//
// Classes. The coefficients depend on the frequency only through
// wx = sin(2 pi l / W) and wy = sin(2 pi k / H), which are equal for rows
// k and (H/2 - k) mod H and for columns l and (W/2 - l) mod W (pair_row):
// up to four frequencies {k, kb} x {l, lb} share one propagator.
//
// Increment form. M is I plus a small matrix (of order beta dt), and its
// powers are near I for the slow modes; stored as such in FP32 they would
// lose the small part. Every matrix here is D_m = M^m - I instead:
//   D_1 = 2 A'^{-1} L            (one step, as the packed kernel takes it)
//   D_2m = 2 D_m + D_m D_m       (squaring)
//   D_a+b = D_a + D_b + D_a D_b  (combination)
// and the propagator is applied as x <- x + D_S x, so rounding is relative to
// the change of x, as in the step-by-step integration.
//
// One step in scaled form: A' = (1/c) I - L, c = beta dt / 2, L the operator
// divided by beta (diagonal -2 - a_r^2/beta, off-diagonals and corners 1);
// x_{n+1} = x_n + 2 A'^{-1} L x_n. D_1 is built column by column: column i
// is 2 A'^{-1} (Lap e_i) - 2 (a_i^2/beta) A'^{-1} e_i, with Lap the cyclic
// second difference, so the -2 and the a_i^2/beta never meet in one FP32
// number. A' is cyclic tridiagonal: Thomas elimination of its torn part plus
// one Sherman-Morrison correction.
#include "diffuse_x2.cuh"

namespace se2n {

// Rows k and (H/2 - k) mod H have bitwise the same coefficients:
// sin_2pi_frac folds 2 pi k / H with integer arithmetic to the same argument
// of sinpif for both (up to the sign of a zero, which the square removes).
// The pairs are enumerated once each: k in [0, H/4] (partner H/2 - k) and
// k in [H/2 + 1, 3H/4] (partner 3H/2 - k); k = H/4 and 3H/4 are their own
// partners. H is even. The same holds for columns over W.
__host__ __device__ __forceinline__ int pair_rows(int H) { return H / 4 + 1 + (3 * H) / 4 - H / 2; }
__device__ __forceinline__ void pair_row(int s, int H, int &k, int &kb) {
    const int lo = H / 4 + 1;
    k = (s < lo) ? s : H / 2 + 1 + (s - lo);
    kb = (k <= H / 2) ? H / 2 - k : 3 * H / 2 - k;
}

namespace {

constexpr int kPropWarps = 4;   // warps a block in the build kernel
constexpr int kApplyWarps = 8;  // warps a block in the apply kernel

template <int N>
struct PropCfg {
    static constexpr int LPC = N < 32 ? N : 32;  // lanes a class
    static constexpr int CPW = 32 / LPC;         // classes a warp
    static constexpr int CPL = N / LPC;          // columns (or rows) a lane
    static constexpr int LD = N + 4;             // column stride in shared memory, floats
    static constexpr int MAT = N * LD;           // floats a matrix
    static constexpr int CLASS_FLOATS = 3 * MAT + 2 * N + 4;
    static constexpr int SMEM = kPropWarps * CPW * CLASS_FLOATS * 4;
    static_assert(N % 4 == 0 && LD % 4 == 0, "16-byte shared-memory vectors");
};

__device__ __forceinline__ void class_members(const PropArgs &a, long long u, int &k, int &kb, int &l, int &lb) {
    const int srow = (int)(u / a.col_slots);
    const int scol = (int)(u - (long long)srow * a.col_slots);
    pair_row(srow, a.H, k, kb);
    if (a.half) {
        l = scol;
        lb = a.W / 2 - scol;
    } else {
        pair_row(scol, a.W, l, lb);
    }
}

// out[:, c] = acc0[:, c] + A B[:, c] for this lane's columns, all in shared
// memory (column-major, stride LD); acc0 = two * X[:, c] + Y[:, c] (Y may be
// null). out differs from every input.
template <int N>
__device__ __forceinline__ void prop_gemm(const float *A, const float *B, const float *X, float two, const float *Y,
                                          float *out, int t) {
    using C = PropCfg<N>;
#pragma unroll 1
    for (int cc = 0; cc < C::CPL; ++cc) {
        const int c = t + cc * C::LPC;
        f32x2 acc[N / 2];
#pragma unroll
        for (int i = 0; i < N; i += 4) {
            const float4 xv = *reinterpret_cast<const float4 *>(X + c * C::LD + i);
            float4 yv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (Y) yv = *reinterpret_cast<const float4 *>(Y + c * C::LD + i);
            acc[i / 2] = pk2(fmaf(two, xv.x, yv.x), fmaf(two, xv.y, yv.y));
            acc[i / 2 + 1] = pk2(fmaf(two, xv.z, yv.z), fmaf(two, xv.w, yv.w));
        }
        // B[kk, c] four at a time (this lane's own column, no bank conflict with
        // the padded stride); A[:, kk] is the same address in every lane
#pragma unroll 1
        for (int k4 = 0; k4 < N; k4 += 4) {
            const float4 bv = *reinterpret_cast<const float4 *>(B + c * C::LD + k4);
            const float bk[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int kq = 0; kq < 4; ++kq) {
                const f32x2 s = dup2(bk[kq]);
                const float *col = A + (k4 + kq) * C::LD;
#pragma unroll
                for (int i = 0; i < N; i += 4) {
                    const float4 av = *reinterpret_cast<const float4 *>(col + i);
                    acc[i / 2] = fma2(pk2(av.x, av.y), s, acc[i / 2]);
                    acc[i / 2 + 1] = fma2(pk2(av.z, av.w), s, acc[i / 2 + 1]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < N; i += 4)
            *reinterpret_cast<float4 *>(out + c * C::LD + i) =
                make_float4(lo2(acc[i / 2]), hi2(acc[i / 2]), lo2(acc[i / 2 + 1]), hi2(acc[i / 2 + 1]));
    }
}

// x = A'^{-1} r in place (r: N values), with the torn factor's reciprocal
// pivots G and the Sherman-Morrison vector q = T^{-1} u in shared memory.
template <int N>
__device__ __forceinline__ void prop_solve(float (&x)[N], const float *G, const float *q, float inv_d0,
                                           float inv_den) {
#pragma unroll
    for (int j = 1; j < N; ++j) x[j] = fmaf(G[j - 1], x[j - 1], x[j]);
    x[N - 1] *= G[N - 1];
#pragma unroll
    for (int j = N - 2; j >= 0; --j) x[j] = (x[j] + x[j + 1]) * G[j];
    const float w = fmaf(x[N - 1], inv_d0, x[0]) * inv_den;
#pragma unroll
    for (int j = 0; j < N; ++j) x[j] = fmaf(-w, q[j], x[j]);
}

template <int N>
__global__ void __launch_bounds__(kPropWarps * 32) k_prop_build(const __grid_constant__ PropArgs a) {
    using C = PropCfg<N>;
    extern __shared__ __align__(16) float psm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / C::LPC, t = lane - g * C::LPC;
    float *base = psm + (warp * C::CPW + g) * C::CLASS_FLOATS;
    float *G = base + 3 * C::MAT;
    float *q = G + N;
    float *scal = q + N;  // 1/d0, 1/(1 + v.q)
    const long long stride = (long long)gridDim.x * kPropWarps * C::CPW;
    // classes are taken warp-uniformly so that every lane reaches each __syncwarp
    for (long long u0 = ((long long)blockIdx.x * kPropWarps + warp) * C::CPW; u0 < a.classes; u0 += stride) {
        const long long u = u0 + g;
        const bool live = u < a.classes;
        int k, kb, l, lb;
        class_members(a, live ? u : a.classes - 1, k, kb, l, lb);
        const float wx = sin_2pi_frac(l, a.W), wy = sin_2pi_frac(k, a.H);
        // torn factor of A' (lane 0 of the class), diagonal d_j = 1/c + 2 + a_j^2/beta
        if (t == 0) {
            float d0 = 0.f;
            float piv = 0.f;
#pragma unroll 1
            for (int j = 0; j < N; ++j) {
                const float ar = fmaf(wx, a.cs[j], wy * a.sn[j]);
                const float d = (a.inv_c + 2.0f) + ar * ar * a.inv_beta;
                float tj = d;
                if (j == 0) {
                    d0 = d;
                    tj = 2.0f * d;
                }
                if (j == N - 1) tj = d + 1.0f / d0;
                piv = (j == 0) ? tj : tj - G[j - 1];
                G[j] = 1.0f / piv;
            }
            // q = T^{-1} u, u = (-d0, 0, ..., 0, -1)
            float qq[N];
#pragma unroll
            for (int j = 0; j < N; ++j) qq[j] = 0.f;
            qq[0] = -d0;
            qq[N - 1] = -1.0f;
#pragma unroll
            for (int j = 1; j < N; ++j) qq[j] = fmaf(G[j - 1], qq[j - 1], qq[j]);
            qq[N - 1] *= G[N - 1];
#pragma unroll
            for (int j = N - 2; j >= 0; --j) qq[j] = (qq[j] + qq[j + 1]) * G[j];
#pragma unroll
            for (int j = 0; j < N; ++j) q[j] = qq[j];
            const float inv_d0 = 1.0f / d0;
            scal[0] = inv_d0;
            scal[1] = 1.0f / (1.0f + fmaf(qq[N - 1], inv_d0, qq[0]));
        }
        __syncwarp();
        const float inv_d0 = scal[0], inv_den = scal[1];
        // D_1, column by column: 2 A'^{-1} Lap e_c - 2 (a_c^2/beta) A'^{-1} e_c
        float *D1 = base;
#pragma unroll 1
        for (int cc = 0; cc < C::CPL; ++cc) {
            const int c = t + cc * C::LPC;
            const float ar = fmaf(wx, a.cs[c], wy * a.sn[c]);
            const float e2 = ar * ar * a.inv_beta;
            float x[N];
#pragma unroll
            for (int j = 0; j < N; ++j) x[j] = (j == c) ? 1.0f : 0.0f;
            prop_solve<N>(x, G, q, inv_d0, inv_den);
            float *dc = D1 + c * C::LD;  // this lane's column: first -2 (a_c^2/beta) A'^{-1} e_c
#pragma unroll
            for (int j = 0; j < N; j += 4)
                *reinterpret_cast<float4 *>(dc + j) = make_float4(-2.0f * e2 * x[j], -2.0f * e2 * x[j + 1],
                                                                  -2.0f * e2 * x[j + 2], -2.0f * e2 * x[j + 3]);
            const int cm = (c == 0) ? N - 1 : c - 1, cp = (c == N - 1) ? 0 : c + 1;
#pragma unroll
            for (int j = 0; j < N; ++j) x[j] = (j == c) ? -2.0f : ((j == cm || j == cp) ? 1.0f : 0.0f);
            prop_solve<N>(x, G, q, inv_d0, inv_den);
#pragma unroll
            for (int j = 0; j < N; j += 4) {
                const float4 v = *reinterpret_cast<const float4 *>(dc + j);
                *reinterpret_cast<float4 *>(dc + j) = make_float4(fmaf(2.0f, x[j], v.x), fmaf(2.0f, x[j + 1], v.y),
                                                                  fmaf(2.0f, x[j + 2], v.z), fmaf(2.0f, x[j + 3], v.w));
            }
        }
        __syncwarp();
        // binary powering: P runs through D_1, D_2, D_4, ...; R collects the set
        // bits of S; Tm is the free third buffer every product is written to
        float *P = base, *R = nullptr, *Tm = base + C::MAT, *spare = base + 2 * C::MAT;
        int s = a.steps;
#pragma unroll 1
        while (true) {
            if (s & 1) {
                if (!R) {
                    // R = P: copy this lane's columns into the spare buffer
                    R = spare;
#pragma unroll 1
                    for (int cc = 0; cc < C::CPL; ++cc) {
                        const int c = t + cc * C::LPC;
#pragma unroll
                        for (int j = 0; j < N; j += 4)
                            *reinterpret_cast<float4 *>(R + c * C::LD + j) =
                                *reinterpret_cast<const float4 *>(P + c * C::LD + j);
                    }
                } else {
                    prop_gemm<N>(R, P, R, 1.0f, P, Tm, t);  // R + P + R P
                    float *tmp = R;
                    R = Tm;
                    Tm = tmp;
                }
                __syncwarp();
            }
            s >>= 1;
            if (!s) break;
            prop_gemm<N>(P, P, P, 2.0f, nullptr, Tm, t);  // 2 P + P P
            float *tmp = P;
            P = Tm;
            Tm = tmp;
            __syncwarp();
        }
        // D_S, row-major: this lane writes rows t, t + LPC, ...
        if (live) {
            float *out = a.D + u * (long long)N * N;
#pragma unroll 1
            for (int cc = 0; cc < C::CPL; ++cc) {
                const int r = t + cc * C::LPC;
#pragma unroll
                for (int j = 0; j < N; j += 4)
                    *reinterpret_cast<float4 *>(out + (long long)r * N + j) =
                        make_float4(R[j * C::LD + r], R[(j + 1) * C::LD + r], R[(j + 2) * C::LD + r],
                                    R[(j + 3) * C::LD + r]);
            }
        }
        __syncwarp();
    }
}

// x <- x + D_S x for the (up to four) frequencies of every class.
template <int N>
__global__ void __launch_bounds__(kApplyWarps * 32) k_prop_apply(const __grid_constant__ PropArgs a) {
    using C = PropCfg<N>;
    __shared__ __align__(16) float2 xs[kApplyWarps][C::CPW][4][N];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / C::LPC, t = lane - g * C::LPC;
    const long long stride = (long long)gridDim.x * kApplyWarps * C::CPW;
    for (long long u0 = ((long long)blockIdx.x * kApplyWarps + warp) * C::CPW; u0 < a.classes; u0 += stride) {
        const long long u = u0 + g;
        const bool live = u < a.classes;
        int k, kb, l, lb;
        class_members(a, live ? u : a.classes - 1, k, kb, l, lb);
        const long long f[4] = {(long long)k * a.Wc + l, (long long)k * a.Wc + lb, (long long)kb * a.Wc + l,
                                (long long)kb * a.Wc + lb};
        const bool on[4] = {live, live && lb != l, live && kb != k, live && kb != k && lb != l};
        float2 mine[4][C::CPL];
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int cc = 0; cc < C::CPL; ++cc) {
                const int j = t + cc * C::LPC;
                mine[m][cc] = on[m] ? a.vol[(long long)j * a.HW + f[m]] : make_float2(0.f, 0.f);
                xs[warp][g][m][j] = mine[m][cc];
            }
        __syncwarp();
        const float *Dc = a.D + (live ? u : 0) * (long long)N * N;
#pragma unroll
        for (int cc = 0; cc < C::CPL; ++cc) {
            const int r = t + cc * C::LPC;
            const float *row = Dc + (long long)r * N;
            f32x2 acc[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) acc[m] = pk2(0.f, 0.f);
#pragma unroll 4
            for (int j = 0; j < N; j += 4) {
                const float4 dv = *reinterpret_cast<const float4 *>(row + j);
                const float dd[4] = {dv.x, dv.y, dv.z, dv.w};
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const f32x2 s = dup2(dd[jj]);
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const float2 xv = xs[warp][g][m][j + jj];
                        acc[m] = fma2(s, pk2(xv.x, xv.y), acc[m]);
                    }
                }
            }
#pragma unroll
            for (int m = 0; m < 4; ++m)
                if (on[m])
                    a.vol[(long long)r * a.HW + f[m]] =
                        make_float2(mine[m][cc].x + lo2(acc[m]), mine[m][cc].y + hi2(acc[m]));
        }
        __syncwarp();
    }
}

template <int N>
cudaError_t launch_build(const PropArgs &a, int num_sms, cudaStream_t s) {
    using C = PropCfg<N>;
    cudaError_t e = cudaFuncSetAttribute(k_prop_build<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_prop_build<N>, kPropWarps * 32, C::SMEM);
    if (e != cudaSuccess) return e;
    const long long per_block = (long long)kPropWarps * C::CPW;
    long long blocks = (a.classes + per_block - 1) / per_block;
    const long long cap = (long long)num_sms * (per_sm > 0 ? per_sm : 1);
    if (blocks > cap) blocks = cap;
    k_prop_build<N><<<(unsigned)blocks, kPropWarps * 32, C::SMEM, s>>>(a);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_apply(const PropArgs &a, int num_sms, cudaStream_t s) {
    using C = PropCfg<N>;
    const long long per_block = (long long)kApplyWarps * C::CPW;
    long long blocks = (a.classes + per_block - 1) / per_block;
    const long long cap = (long long)num_sms * 64;
    if (blocks > cap) blocks = cap;
    k_prop_apply<N><<<(unsigned)blocks, kApplyWarps * 32, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

}  // namespace se2n

bool se2n_prop_supported(int N) { return N == 16 || N == 32 || N == 64; }

int se2n_prop_col_slots(int W, bool half) { return half ? W / 4 + 1 : se2n::pair_rows(W); }

long long se2n_prop_classes(int H, int W, bool half) {
    return (long long)se2n::pair_rows(H) * se2n_prop_col_slots(W, half);
}

cudaError_t se2n_launch_prop_build(int N, const PropArgs &a, int num_sms, cudaStream_t s) {
    switch (N) {
        case 16: return se2n::launch_build<16>(a, num_sms, s);
        case 32: return se2n::launch_build<32>(a, num_sms, s);
        case 64: return se2n::launch_build<64>(a, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t se2n_launch_prop_apply(int N, const PropArgs &a, int num_sms, cudaStream_t s) {
    switch (N) {
        case 16: return se2n::launch_apply<16>(a, num_sms, s);
        case 32: return se2n::launch_apply<32>(a, num_sms, s);
        case 64: return se2n::launch_apply<64>(a, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}
