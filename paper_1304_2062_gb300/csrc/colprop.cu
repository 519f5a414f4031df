// The column pass of one restoration interval on the Hermitian half of the
// spectrum, fused. Between intervals the volume is row-transformed: the DFT
// along x (index l) of every row of every angle plane, stored as complex
// [Wc][H][N] (rowfft.cu writes and reads it), so column l's H x N block is
// contiguous and a frequency's N angles are adjacent. One block a column l:
//   1. takes the DFT along y (index k) of every angle plane (unnormalised),
//      which completes the two-dimensional DFT of the lifted volume;
//   2. applies x <- x + D_S x to the N-vector of every frequency (k, l),
//      D_S the S-step propagator of its class, stored by 16-byte chunks of
//      its rows, chunk-major (eq. (deceq), Theorem 2, integrated by S
//      Crank-Nicolson steps; see propagator.cu), with the angles reversed
//      for rows H/2 + s and H - s;
//   3. takes the inverse DFT along k,
// in shared memory (smem_fft.cuh), so the spectrum of the interval never
// goes through device memory.
#include "diffuse_x2.cuh"
#include "prop_classes.cuh"
#include "se2n_internal.h"
#include "smem_fft.cuh"

namespace se2n {

namespace {

constexpr int kColThreads = 512;

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
        // the class this lane takes next, into L1 while this one is applied
        // (N^2 / 32 lines of 128 bytes a class, N / 16 a lane)
        if (s + WARPS * CPW < SLOTS) {
            const char *Dn = reinterpret_cast<const char *>(
                D + ((long long)(s + WARPS * CPW) * col_slots + scol) * (N * N));
#pragma unroll
            for (int c = 0; c < N / 16; ++c)
                asm volatile("prefetch.global.L1 [%0];" ::"l"(Dn + (t + c * LPC) * 128));
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
    static constexpr int XF = SmemBlock<N, L>::COMPLEX;
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
    // the column block [k][n] into transforms [n][k], two angles a 16-byte
    // load, every load of a thread issued before the first store
    constexpr int NV = N * L / 2 / kColThreads;
    static_assert(NV * 2 * kColThreads == N * L, "whole block");
    {
        float4 in[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) in[q] = reinterpret_cast<const float4 *>(g)[tid + q * kColThreads];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const int e = 2 * (tid + q * kColThreads), k = e / N, n = e % N;
            const int o = xoff<L>(k);
            X[n * (L + 1) + o] = make_float2(in[q].x, in[q].y);
            X[(n + 1) * (L + 1) + o] = make_float2(in[q].z, in[q].w);
        }
    }
    __syncthreads();
    fft_smem<kColThreads, N, L, -1, 1>(X, tws, tid);
    __syncthreads();
    col_apply<N, L>(X, a.D, half_col_slot(l, a.W), a.col_slots, tid);
    __syncthreads();
    fft_smem<kColThreads, N, L, 1, 1>(X, tws, tid);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const int e = 2 * (tid + q * kColThreads), k = e / N, n = e % N;
        const int o = xoff<L>(k);
        const float2 a = X[n * (L + 1) + o], c = X[(n + 1) * (L + 1) + o];
        reinterpret_cast<float4 *>(g)[tid + q * kColThreads] = make_float4(a.x, a.y, c.x, c.y);
    }
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
