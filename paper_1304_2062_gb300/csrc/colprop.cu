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
//
// The four rows s, H/2 - s, H/2 + s, H - s of a class have the parity of s,
// so a first radix-2 step (decimation in frequency) splits each column into
// its even and odd frequencies, u_k = x_k + x_{k+H/2} and
// v_k = (x_k - x_{k+H/2}) w^k (w = exp(-2 pi i / H)), whose H/2-point DFTs
// are X_{2k} and X_{2k+1}: each half holds whole classes. A block takes the
// halves one after the other (forward DFT, apply, inverse DFT), keeping v
// and then the even half's result y_e in the rows of its own column block,
// and ends with x_k = y_e,k + w^-k y_o,k, x_{k+H/2} = y_e,k - w^-k y_o,k.
// Half a column in shared memory (66 KB at H = 512, N = 32) lets two
// blocks share an SM, so the 257 columns of a 512 x 512 plane run in one
// wave and one block's loads overlap the other's arithmetic.
#include "diffuse_x2.cuh"
#include "prop_classes.cuh"
#include "se2n_internal.h"
#include "smem_fft.cuh"

namespace se2n {

namespace {

// threads a block: 256, and 512 for half columns of 384 and 512 (H = 768,
// 1024), whose transform passes would otherwise hold too many values a thread
template <int H>
__host__ __device__ constexpr int col_threads() { return H >= 768 ? 512 : 256; }

// x <- x + D_S x for every frequency (k, l) of one half of the column (its
// classes s = parity, parity + 2, ...; frequency k at index k / 2 of the
// half): one class per N/2 lanes, two rows of D_S a lane, held in registers;
// x_j of the class's four rows is a shared-memory broadcast for the lanes of
// the class. Rows 2 and 3 of the class are read and written with the angles
// reversed (angle -j in place of j).
template <int N, int H>
__device__ __forceinline__ void col_apply(float2 *X, const float *D, int scol, int col_slots, int parity, int tid) {
    constexpr int L = H / 2, RPL = 2, LPC = N / RPL, CPW = 32 / LPC, WARPS = col_threads<H>() / 32;
    const int count = parity ? H / 8 : H / 8 + 1;
    const int warp = tid >> 5, lane = tid & 31;
    const int g = lane / LPC, t = lane - g * LPC;
    // classes are taken warp-uniformly so that every lane reaches each __syncwarp
    for (int i0 = warp * CPW; i0 < count; i0 += WARPS * CPW) {
        const int i = i0 + g;
        const bool live = i < count;
        const int s = parity + 2 * (live ? i : count - 1);
        int k[4];
        bool kon[4];
        slot_rows(s, H, k, kon);
        // D_S of the class, chunk-major: D[r][4c .. 4c + 3] is float4 c N + r
        const float4 *Dc = reinterpret_cast<const float4 *>(D + ((long long)s * col_slots + scol) * (N * N));
        float drow[RPL][N];
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int r = t + q * LPC;
#pragma unroll
            for (int j = 0; j < N / 4; ++j) {
                const float4 d = __ldg(Dc + j * N + r);
                drow[q][4 * j] = d.x;
                drow[q][4 * j + 1] = d.y;
                drow[q][4 * j + 2] = d.z;
                drow[q][4 * j + 3] = d.w;
            }
        }
        // the class this lane takes next, into L1 while this one is applied
        // (N^2 / 32 lines of 128 bytes a class, N / 16 a lane)
        if (i + WARPS * CPW < count) {
            const char *Dn = reinterpret_cast<const char *>(
                D + ((long long)(s + 2 * WARPS * CPW) * col_slots + scol) * (N * N));
#pragma unroll
            for (int c = 0; c < N / 16; ++c)
                asm volatile("prefetch.global.L1 [%0];" ::"l"(Dn + (t + c * LPC) * 128));
        }
        f32x2 acc[RPL][4];
#pragma unroll
        for (int q = 0; q < RPL; ++q)
#pragma unroll
            for (int m = 0; m < 4; ++m) acc[q][m] = pk2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const int jr = (N - j) & (N - 1);
            f32x2 xv[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const float2 x = X[xsm<L>((m < 2 ? j : jr) * L + (k[m] >> 1))];
                xv[m] = pk2(x.x, x.y);
            }
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                const f32x2 sd = dup2(drow[q][j]);
#pragma unroll
                for (int m = 0; m < 4; ++m) acc[q][m] = fma2(sd, xv[m], acc[q][m]);
            }
        }
        __syncwarp();
        if (live) {
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                const int r = t + q * LPC, rr = (N - r) & (N - 1);
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    if (kon[m]) {
                        // slot r of a reversed row is angle -r
                        float2 &x = X[xsm<L>((m < 2 ? r : rr) * L + (k[m] >> 1))];
                        x = make_float2(x.x + lo2(acc[q][m]), x.y + hi2(acc[q][m]));
                    }
            }
        }
        __syncwarp();
    }
}

template <int N, int H>
struct ColCfg {
    static constexpr int L = H / 2;                      // half a column
    static constexpr int XF = SmemBlock<N, L>::COMPLEX;  // one half, complex
    static constexpr int SMEM = (XF + H + FftTw<L>::SIZE) * 8;  // and the twiddles
    // two angles (one float4) of one row of the upper half of the block a step
    static constexpr int T = col_threads<H>();
    static constexpr int NP = N * L / 2 / T;
    static_assert(NP * 2 * T == N * L, "whole half blocks");
};

// a float4 of two angles n, n + 1 of frequency (half row) k, from / into the
// half-column transforms [n][k]
template <int N, int L>
__device__ __forceinline__ void put2(float2 *X, int k, int n, float2 a, float2 b) {
    const int o = xoff<L>(k);
    X[n * (L + 1) + o] = a;
    X[(n + 1) * (L + 1) + o] = b;
}

// Block b takes column b / 2 (b even) or W/2 - b / 2 (b odd), so the two
// columns of a class run side by side and share its propagators in L2.
template <int N, int H>
__global__ void __launch_bounds__(col_threads<H>(), H >= 768 ? 1 : 2) k_col_prop(const __grid_constant__ ColArgs a) {
    using C = ColCfg<N, H>;
    constexpr int L = C::L, T = C::T, HALF4 = N * L / 2;  // float4s in half a block
    extern __shared__ __align__(16) float2 csm[];
    float2 *X = csm;
    float2 *tws = csm + C::XF;  // exp(-2 pi i m / H), m < H
    float2 *twp = tws + H;      // the transforms' pass tables
    const int tid = threadIdx.x;
    const int b = blockIdx.x, h = b >> 1;
    const int l = (b & 1) ? a.W / 2 - h : h;
    const int scol = half_col_slot(l, a.W);
    float4 *g = reinterpret_cast<float4 *>(a.col + (long long)l * (N * H));
    for (int m = tid; m < H; m += T) tws[m] = a.tw[m];
    fft_twiddles<T, L, 2>(twp, a.tw, tid);  // from the table in device memory
    __syncthreads();
    // 1. u = x_k + x_{k+L} into shared memory, v = (x_k - x_{k+L}) w^k into
    //    the upper rows of the block (each thread later reads back only what
    //    it wrote itself)
#pragma unroll 4
    for (int q = 0; q < C::NP; ++q) {
        const int f = tid + q * T, k = 2 * f / N, n = 2 * f % N;
        const float4 x0 = g[f], x1 = g[HALF4 + f];
        const float2 w = tws[k];
        put2<N, L>(X, k, n, make_float2(x0.x + x1.x, x0.y + x1.y), make_float2(x0.z + x1.z, x0.w + x1.w));
        const float2 d0 = twiddle<-1>(make_float2(x0.x - x1.x, x0.y - x1.y), w);
        const float2 d1 = twiddle<-1>(make_float2(x0.z - x1.z, x0.w - x1.w), w);
        g[HALF4 + f] = make_float4(d0.x, d0.y, d1.x, d1.y);
    }
    __syncthreads();
    // 2. the even frequencies, into y_e in the lower rows of the block
    fft_smem<T, N, L, -1>(X, twp, tid);
    __syncthreads();
    col_apply<N, H>(X, a.D, scol, a.col_slots, 0, tid);
    __syncthreads();
    fft_smem<T, N, L, 1>(X, twp, tid);
    __syncthreads();
#pragma unroll 4
    for (int q = 0; q < C::NP; ++q) {
        const int f = tid + q * T, k = 2 * f / N, n = 2 * f % N;
        const int o = xoff<L>(k);
        const float2 e0 = X[n * (L + 1) + o], e1 = X[(n + 1) * (L + 1) + o];
        g[f] = make_float4(e0.x, e0.y, e1.x, e1.y);
    }
    __syncthreads();
    // 3. the odd frequencies
#pragma unroll 4
    for (int q = 0; q < C::NP; ++q) {
        const int f = tid + q * T, k = 2 * f / N, n = 2 * f % N;
        const float4 v = g[HALF4 + f];
        put2<N, L>(X, k, n, make_float2(v.x, v.y), make_float2(v.z, v.w));
    }
    __syncthreads();
    fft_smem<T, N, L, -1>(X, twp, tid);
    __syncthreads();
    col_apply<N, H>(X, a.D, scol, a.col_slots, 1, tid);
    __syncthreads();
    fft_smem<T, N, L, 1>(X, twp, tid);
    __syncthreads();
    // 4. x_k = y_e + w^-k y_o, x_{k+L} = y_e - w^-k y_o
#pragma unroll 4
    for (int q = 0; q < C::NP; ++q) {
        const int f = tid + q * T, k = 2 * f / N, n = 2 * f % N;
        const int o = xoff<L>(k);
        const float2 w = tws[k];
        const float4 e = g[f];
        const float2 o0 = twiddle<1>(X[n * (L + 1) + o], w), o1 = twiddle<1>(X[(n + 1) * (L + 1) + o], w);
        g[f] = make_float4(e.x + o0.x, e.y + o0.y, e.z + o1.x, e.w + o1.y);
        g[HALF4 + f] = make_float4(e.x - o0.x, e.y - o0.y, e.z - o1.x, e.w - o1.y);
    }
}

template <int N, int H>
cudaError_t col_attr() {
    return cudaFuncSetAttribute(k_col_prop<N, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, ColCfg<N, H>::SMEM);
}

template <int N, int H>
cudaError_t col_launch(const ColArgs &a, cudaStream_t s) {
    cudaError_t e = col_attr<N, H>();
    if (e != cudaSuccess) return e;
    k_col_prop<N, H><<<a.Wc, ColCfg<N, H>::T, ColCfg<N, H>::SMEM, s>>>(a);
    return cudaGetLastError();
}

template <int N>
cudaError_t col_dispatch(int H, const ColArgs *a, cudaStream_t s) {
    switch (H) {
        case 64: return a ? col_launch<N, 64>(*a, s) : col_attr<N, 64>();
        case 128: return a ? col_launch<N, 128>(*a, s) : col_attr<N, 128>();
        case 256: return a ? col_launch<N, 256>(*a, s) : col_attr<N, 256>();
        case 512: return a ? col_launch<N, 512>(*a, s) : col_attr<N, 512>();
        case 1024: return a ? col_launch<N, 1024>(*a, s) : col_attr<N, 1024>();
        case 384: return a ? col_launch<N, 384>(*a, s) : col_attr<N, 384>();
        case 768: return a ? col_launch<N, 768>(*a, s) : col_attr<N, 768>();
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

}  // namespace se2n

bool se2n_col_supported(int N, int H) {
    return (N == 16 || N == 32) &&
           (H == 64 || H == 128 || H == 256 || H == 512 || H == 1024 || H == 384 || H == 768);
}

cudaError_t se2n_col_prepare(int N, int H) {
    if (!se2n_col_supported(N, H)) return cudaErrorInvalidValue;
    return N == 16 ? se2n::col_dispatch<16>(H, nullptr, nullptr) : se2n::col_dispatch<32>(H, nullptr, nullptr);
}

cudaError_t se2n_launch_col_prop(int N, const ColArgs &a, cudaStream_t s) {
    if (!se2n_col_supported(N, a.H)) return cudaErrorInvalidValue;
    return N == 16 ? se2n::col_dispatch<16>(a.H, &a, s) : se2n::col_dispatch<32>(a.H, &a, s);
}
