// The column pass of one restoration interval on the Hermitian half of the
// spectrum, fused. The volume between intervals is row-transformed: the DFT
// along x (l) of every row, stored as complex [Wc][N][H] so that column l's
// N x H block is contiguous (cuFFT writes and reads that layout). One block
// a column l:
//   1. takes the DFT along y (k) of every angle plane (unnormalised), which
//      completes the two-dimensional DFT of the lifted volume;
//   2. applies x <- x + D_S x to the N-vector of every frequency (k, l),
//      D_S the S-step propagator of its class, stored by 16-byte chunks of
//      its rows, chunk-major (eq. (deceq), Theorem 2,
//      integrated by S Crank-Nicolson steps; see propagator.cu), with the
//      angles reversed for rows H/2 + s and H - s;
//   3. takes the inverse DFT along k,
// all in shared memory, so the spectrum of the interval never goes through
// device memory.
//
// DFTs along k: mixed-radix Stockham (self-sorting) passes, radix 8 and then
// one pass of radix 2 or 4 where H is not a power of 8, with the twiddles
// exp(-/+ 2 pi i m / H) from a table. The first forward pass reads device
// memory and the last inverse pass writes it; the others run in place in
// shared memory (every read of a pass before its first write). The block
// [N][H] is kept with planes H + 1 complex apart (so that the lanes of the
// apply, one angle each, fall on different banks) and, inside a plane, each
// run of 16 complex permuted by an XOR of its low bits with a function of the
// run index: with it the three access patterns of the passes (consecutive,
// stride 8, and runs of 8 that are 64 apart) take no bank conflicts.
#include "diffuse_x2.cuh"
#include "prop_classes.cuh"
#include "se2n_internal.h"

namespace se2n {

namespace {

constexpr int kColThreads = 512;

// shared-memory index of element e = n L + i of the block
template <int L>
__device__ __forceinline__ int xsm(int e) {
    const int n = e / L, i = e & (L - 1), m = i >> 4;
    return n * (L + 1) + (i ^ ((m & 7) | ((m << 1) & 8)));
}

// a * w (forward) or a * conj(w) (inverse)
template <int DIR>
__device__ __forceinline__ float2 twiddle(float2 a, float2 w) {
    const float wy = DIR < 0 ? w.y : -w.y;
    return make_float2(fmaf(a.x, w.x, -a.y * wy), fmaf(a.x, wy, a.y * w.x));
}

// z times exp(DIR i pi / 2): -i z forward, i z inverse
template <int DIR>
__device__ __forceinline__ float2 quarter(float2 z) {
    return DIR < 0 ? make_float2(z.y, -z.x) : make_float2(-z.y, z.x);
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// V_k = sum_n v_n exp(DIR 2 pi i n k / R), in place, for R = 2, 4, 8.
template <int R, int DIR>
__device__ __forceinline__ void dft_small(float2 (&v)[R]) {
    if constexpr (R == 2) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        const float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        const float2 t2 = cadd(v[1], v[3]), t3 = quarter<DIR>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    } else {
        // even and odd halves, then V_k = E_k + w^k O_k, V_{k+4} = E_k - w^k O_k
        float2 e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
        dft_small<4, DIR>(e);
        dft_small<4, DIR>(o);
        constexpr float h = 0.70710678118654752f;  // cos(pi / 4)
        // w = exp(DIR i pi / 4) = (1 + DIR i) / sqrt(2)
        const float2 o1 = DIR < 0 ? make_float2(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x))
                                  : make_float2(h * (o[1].x - o[1].y), h * (o[1].y + o[1].x));
        const float2 o2 = quarter<DIR>(o[2]);
        const float2 o3 = quarter<DIR>(DIR < 0 ? make_float2(h * (o[3].x + o[3].y), h * (o[3].y - o[3].x))
                                               : make_float2(h * (o[3].x - o[3].y), h * (o[3].y + o[3].x)));
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);
        v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);
        v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);
        v[7] = csub(e[3], o3);
    }
}

// One Stockham pass of radix R over the N transforms of length L, whose
// sub-transforms of length NS are done: butterfly j of a transform reads
// elements j + r L / R, twiddles them by exp(DIR 2 pi i r (j mod NS) / (NS R)),
// and writes its outputs to (j / NS) NS R + (j mod NS) + r NS.
// SRC / DST: device memory (block of column l) instead of shared memory.
template <int N, int L, int R, int NS, int DIR, bool SRC, bool DST>
__device__ __forceinline__ void col_pass(const float2 *gin, float2 *gout, float2 *X, const float2 *tw, int tid) {
    constexpr int M = L / R;  // butterflies a transform
    constexpr int NB = N * M;
    constexpr int BPT = (NB + kColThreads - 1) / kColThreads;
    static_assert(kColThreads % M == 0, "j depends on the thread only");
    // butterfly b = tid + q kColThreads: transform b / M, index j = tid mod M
    // for every q, so the twiddles are read once
    const int j = tid % M, k = j & (NS - 1);
    float2 v[BPT][R];
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
        const int b = tid + q * kColThreads;
        if (NB % kColThreads == 0 || b < NB) {
            const int n = b / M;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int e = n * L + j + r * M;
                v[q][r] = SRC ? gin[e] : X[xsm<L>(e)];
            }
        }
    }
    float2 w[R];
    if constexpr (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) w[r] = tw[r * k * (L / (NS * R))];
    }
    if constexpr (!SRC && !DST) __syncthreads();  // in place
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
        const int b = tid + q * kColThreads;
        if (NB % kColThreads == 0 || b < NB) {
            const int n = b / M;
            if constexpr (NS > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) v[q][r] = twiddle<DIR>(v[q][r], w[r]);
            }
            dft_small<R, DIR>(v[q]);
            const int base = n * L + (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int e = base + r * NS;
                if constexpr (DST)
                    gout[e] = v[q][r];
                else
                    X[xsm<L>(e)] = v[q][r];
            }
        }
    }
}

// The DFT along k of the N planes of the block (L = 64, 128, 256 or 512:
// radix 8 x 8, 8 x 8 x 2, 8 x 8 x 4, 8 x 8 x 8). Ends with the block in
// shared memory (LAST = false) or in device memory.
template <int N, int L, int DIR, bool FIRST, bool LAST>
__device__ __forceinline__ void col_dft(const float2 *gin, float2 *gout, float2 *X, const float2 *tw, int tid) {
    static_assert(L == 64 || L == 128 || L == 256 || L == 512, "column length");
    col_pass<N, L, 8, 1, DIR, FIRST, false>(gin, nullptr, X, tw, tid);
    __syncthreads();
    if constexpr (L == 64) {
        col_pass<N, L, 8, 8, DIR, false, LAST>(nullptr, gout, X, tw, tid);
    } else {
        col_pass<N, L, 8, 8, DIR, false, false>(nullptr, nullptr, X, tw, tid);
        __syncthreads();
        constexpr int R = L == 128 ? 2 : (L == 256 ? 4 : 8);
        col_pass<N, L, R, 64, DIR, false, LAST>(nullptr, gout, X, tw, tid);
    }
}

// x <- x + D_S x for every frequency (k, l) of the column: one class (row
// slot s, this column's slot) per N/2 lanes, two rows of D_S a lane, held in
// registers; x_j of the slot's four rows is a shared-memory broadcast for
// the lanes of the class. Rows 2 and 3 of the slot are read and written with
// the angles reversed (angle -j in place of j).
template <int N, int L>
__device__ __forceinline__ void col_apply(float2 *X, const float *D, int scol, int col_slots, int tid) {
    constexpr int RPL = 2, LPC = N / RPL, CPW = 32 / LPC, WARPS = kColThreads / 32;
    constexpr int SLOTS = L / 4 + 1;
    const int warp = tid >> 5, lane = tid & 31;
    const int g = lane / LPC, t = lane - g * LPC;
    // slots are taken warp-uniformly so that every lane reaches each __syncwarp
    for (int s0 = warp * CPW; s0 < SLOTS; s0 += WARPS * CPW) {
        const int s = s0 + g;
        const bool live = s < SLOTS;
        const int sc = live ? s : SLOTS - 1;
        int k[4];
        bool kon[4];
        slot_rows(sc, L, k, kon);
        // D_S of the class, chunk-major: D[r][4c .. 4c + 3] is float4 c N + r
        const float4 *Dc = reinterpret_cast<const float4 *>(D + ((long long)sc * col_slots + scol) * (N * N));
        float drow[RPL][N];
#pragma unroll
        for (int i = 0; i < RPL; ++i) {
            const int r = t + i * LPC;
#pragma unroll
            for (int j = 0; j < N / 4; ++j) {
                const float4 d = __ldg(Dc + j * N + r);
                drow[i][4 * j] = d.x;
                drow[i][4 * j + 1] = d.y;
                drow[i][4 * j + 2] = d.z;
                drow[i][4 * j + 3] = d.w;
            }
        }
        f32x2 acc[RPL][4];
#pragma unroll
        for (int i = 0; i < RPL; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][q] = pk2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const int jr = (N - j) & (N - 1);
            f32x2 xv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 x = X[xsm<L>((q < 2 ? j : jr) * L + k[q])];
                xv[q] = pk2(x.x, x.y);
            }
#pragma unroll
            for (int i = 0; i < RPL; ++i) {
                const f32x2 sd = dup2(drow[i][j]);
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[i][q] = fma2(sd, xv[q], acc[i][q]);
            }
        }
        __syncwarp();
        if (live) {
#pragma unroll
            for (int i = 0; i < RPL; ++i) {
                const int r = t + i * LPC, rr = (N - r) & (N - 1);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (kon[q]) {
                        // slot r of a reversed row is angle -r
                        float2 &x = X[xsm<L>((q < 2 ? r : rr) * L + k[q])];
                        x = make_float2(x.x + lo2(acc[i][q]), x.y + hi2(acc[i][q]));
                    }
            }
        }
        __syncwarp();
    }
}

template <int N, int L>
struct ColCfg {
    static constexpr int XF = N * (L + 1);  // block with padded planes, complex
    static constexpr int SMEM = (XF + L) * 8;
};

// Block b takes column b / 2 (b even) or W/2 - b / 2 (b odd), so the two
// columns of a class run side by side and share its propagators in L2.
template <int N, int L>
__global__ void __launch_bounds__(kColThreads, 1) k_col_prop(const __grid_constant__ ColArgs a) {
    extern __shared__ __align__(16) float2 csm[];
    float2 *X = csm;
    float2 *tws = csm + ColCfg<N, L>::XF;
    const int tid = threadIdx.x;
    const int b = blockIdx.x, h = b >> 1;
    const int l = (b & 1) ? a.W / 2 - h : h;
    float2 *g = a.col + (long long)l * (N * L);
    for (int m = tid; m < L; m += kColThreads) tws[m] = a.tw[m];
    __syncthreads();
    col_dft<N, L, -1, true, false>(g, nullptr, X, tws, tid);
    __syncthreads();
    col_apply<N, L>(X, a.D, half_col_slot(l, a.W), a.col_slots, tid);
    __syncthreads();
    col_dft<N, L, 1, false, true>(nullptr, g, X, tws, tid);
}

template <int N, int L>
cudaError_t col_attr() {
    return cudaFuncSetAttribute(k_col_prop<N, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, ColCfg<N, L>::SMEM);
}

template <int N, int L>
cudaError_t col_launch(const ColArgs &a, cudaStream_t s) {
    cudaError_t e = col_attr<N, L>();
    if (e != cudaSuccess) return e;
    k_col_prop<N, L><<<a.Wc, kColThreads, ColCfg<N, L>::SMEM, s>>>(a);
    return cudaGetLastError();
}

template <int N>
cudaError_t col_dispatch(int H, const ColArgs *a, cudaStream_t s) {
    switch (H) {
        case 64: return a ? col_launch<N, 64>(*a, s) : col_attr<N, 64>();
        case 128: return a ? col_launch<N, 128>(*a, s) : col_attr<N, 128>();
        case 256: return a ? col_launch<N, 256>(*a, s) : col_attr<N, 256>();
        case 512: return a ? col_launch<N, 512>(*a, s) : col_attr<N, 512>();
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

}  // namespace se2n

bool se2n_col_supported(int N, int H) { return (N == 16 || N == 32) && (H == 64 || H == 128 || H == 256 || H == 512); }

cudaError_t se2n_col_prepare(int N, int H) {
    if (!se2n_col_supported(N, H)) return cudaErrorInvalidValue;
    return N == 16 ? se2n::col_dispatch<16>(H, nullptr, nullptr) : se2n::col_dispatch<32>(H, nullptr, nullptr);
}

cudaError_t se2n_launch_col_prop(int N, const ColArgs &a, cudaStream_t s) {
    if (!se2n_col_supported(N, a.H)) return cudaErrorInvalidValue;
    return N == 16 ? se2n::col_dispatch<16>(a.H, &a, s) : se2n::col_dispatch<32>(a.H, &a, s);
}
