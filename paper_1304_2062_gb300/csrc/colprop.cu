// The column pass of one restoration interval on the Hermitian half of the
// spectrum, fused. Between intervals the volume is row-transformed: the DFT
// along x (index l) of every row of every angle plane, stored as complex
// [Wc][H][N] (rowfft.cu writes and reads it), so column l's H x N block is
// contiguous and a frequency's N angles are adjacent. For every column l:
//   1. the DFT along y (index k) of every angle plane (unnormalised), which
//      completes the two-dimensional DFT of the lifted volume;
//   2. x <- x + D_S x for the N-vector of every frequency (k, l), D_S the
//      S-step propagator of its class, stored by 16-byte chunks of its rows,
//      chunk-major (eq. (4.2), Theorem 2, integrated by S Crank-Nicolson
//      steps; see propagator.cu), with the angles reversed for rows H/2 + s
//      and H - s;
//   3. the inverse DFT along k,
// in shared memory, so the spectrum of the interval never goes through
// device memory.
//
// The four rows s, H/2 - s, H/2 + s, H - s of a class have the parity of s,
// so a first radix-2 step (decimation in frequency) splits each column into
// its even and odd frequencies, u_k = x_k + x_{k+H/2} and
// v_k = (x_k - x_{k+H/2}) w^k (w = exp(-2 pi i / H)), whose H/2-point DFTs
// are X_{2k} and X_{2k+1}: each half holds whole classes, and the column is
// put back by x_k = y_e,k + w^-k y_o,k, x_{k+H/2} = y_e,k - w^-k y_o,k.
//
// Two kernels. k_col_tma (wherever the column fits in shared memory: N H
// complex up to 192 KB) keeps the whole column in the rows of device memory
// ([k][n]), brought in and out by bulk asynchronous copies, with in-place
// transforms whose every access is a run of whole rows. k_col_prop (N = 32,
// H = 1024) keeps half a column in angle planes [n][k] (smem_fft.cuh), the
// halves one after the other, v and then the even half's result y_e held in
// the rows of the column's own block in device memory.
#include "diffuse_x2.cuh"
#include "prop_classes.cuh"
#include "se2n_internal.h"
#include "smem_fft.cuh"
#include "bulk_copy.cuh"
#include "rowdft.cuh"

namespace se2n {

// Set by a column pass whose bounded wait for its copy-in ran out (which would
// mean the device stopped making progress); read by se2n_col_fault().
__device__ int g_col_fault;

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

// ---------------------------------------------------------------------------
// The column pass with the whole column in shared memory (N H complex: up to
// H = 768 for N = 32 and H = 1024 for N = 16). Rows stay as they are in device
// memory, X[k N + n] (row k, angle n), so one bulk asynchronous copy brings
// the column in and one takes it back, and every access of the transforms
// (a row of all the angles) is one contiguous run of shared memory.
//
// The transforms along k are in place (rowdft.cuh): decimation in frequency
// forward (the half-column spectrum ends in digit-reversed order, rd_pos),
// decimation in time inverse (back to natural order). Rows 0 .. L-1 of the column hold the
// even half and rows L .. H-1 the odd half (L = H / 2); the radix-2 split is
// folded into the reads of the first forward pass and the recombination into
// the writes of the last inverse pass.

// x <- x + D_S x for every frequency of the column, classes s = 0 .. H/4
// (the even half for even s, the odd half for odd s): one class per N/2
// lanes, rows t and t + N/2 of D_S a lane in registers (drow), a class after
// another. x_j, x_{j+1} of one frequency are one 16-byte shared-memory
// broadcast for the lanes of a class; the classes of one warp take the
// columns j rotated by 16 / (classes a warp), so that their broadcasts fall
// on different banks (drow holds the rotated columns). Rows 0 and 1 take
// columns 2p, 2p + 1 at step p; the reversed rows 2 and 3 read angles
// -2p, -2p + 1 (adjacent in the row) for columns 2p, 2p - 1, except that
// column 0 is taken at step 0, column N/2 - 1 at the end of the first half,
// N/2 at the start of the second and N - 1 at the end (the order in which a
// row's terms are summed is fixed, so every run gives the same bits). The
// next class's rows are prefetched into L1 while this one is applied.
template <int T, int N, int H>
__device__ __forceinline__ void col_apply_rows(float2 *XA, float2 *XB, const float *D, int scol, int col_slots,
                                               int tid) {
    constexpr int L = H / 2, LPC = N / 2, CPW = 32 / LPC, WARPS = T / 32, ROT = 16 / CPW;
    constexpr int COUNT = H / 4 + 1, STRIDE = WARPS * CPW, NC = N / 4;  // NC: 16-byte chunks a row
    const int warp = tid >> 5, lane = tid & 31;
    const int g = lane / LPC, t = lane - g * LPC, rot = ROT * g;
    float drow[2][N];
    // chunks [c0, c0 + NC/2) of rows t, t + N/2 of class s (rotated columns);
    // chunk-major storage: D[r][4c .. 4c + 3] is float4 c N + r
    auto load_half = [&](int s, int c0) {
        const float4 *Dc = reinterpret_cast<const float4 *>(D + ((long long)s * col_slots + scol) * (N * N));
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int c = c0; c < c0 + NC / 2; ++c) {
                const float4 d = __ldg(Dc + ((c + rot / 4) & (NC - 1)) * N + t + q * LPC);
                drow[q][4 * c] = d.x;
                drow[q][4 * c + 1] = d.y;
                drow[q][4 * c + 2] = d.z;
                drow[q][4 * c + 3] = d.w;
            }
    };
    // classes are taken warp-uniformly so that every lane reaches each __syncwarp
    for (int i0 = warp * CPW; i0 < COUNT; i0 += STRIDE) {
        const int i = i0 + g;
        const bool live = i < COUNT, more = i + STRIDE < COUNT;
        const int s = live ? i : COUNT - 1;
        load_half(s, 0);
        load_half(s, NC / 2);
        // the class this lane takes next, into L1 while this one is applied
        if (more) {
            const char *Dn = reinterpret_cast<const char *>(D + ((long long)(i + STRIDE) * col_slots + scol) * (N * N));
#pragma unroll
            for (int c = 0; c < N / 16; ++c) asm volatile("prefetch.global.L1 [%0];" ::"l"(Dn + (t + c * LPC) * 128));
        }
        int k[4];
        bool kon[4];
        slot_rows(s, H, k, kon);
        float2 *Xh = (s & 1) ? XB : XA;
        int xo[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) xo[m] = rd_pos<L>(k[m] >> 1) * N;
        // shared-memory addresses: normal rows read angle 2p + rot, reversed
        // rows angle (N - rot - 2p) mod N; where N = 32 each wraps at one step
        // for every class of a warp (12 and 13), so each row has one address
        // before that step and one after, plus one for step 0 of a reversed row
        uint32_t a0[4], a1[4], az[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const uint32_t row = bulk::saddr(Xh + xo[m]);
            if (m < 2) {
                a0[m] = row + 8u * rot;
                a1[m] = a0[m] - 8u * N * (rot > 0);
                az[m] = 0;
            } else {
                a0[m] = row + 8u * (N - rot);
                a1[m] = a0[m] + 8u * N * (rot > 0);
                az[m] = row + 8u * ((N - rot) & (N - 1));
            }
        }
        auto xget = [&](int m, int p) -> float4 {
            float4 v;
            if constexpr (N == 32) {
                const uint32_t ad = m < 2 ? (p < 12 ? a0[m] : a1[m]) + 16u * p
                                          : (p == 0 ? az[m] : (p < 13 ? a0[m] : a1[m]) - 16u * p);
                asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                             : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                             : "r"(ad));
            } else {
                const int j = m < 2 ? (2 * p + rot) & (N - 1) : (N - rot - 2 * p) & (N - 1);
                v = *reinterpret_cast<const float4 *>(Xh + xo[m] + j);
            }
            return v;
        };
        f32x2 acc[2][4];
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int m = 0; m < 4; ++m) acc[q][m] = pk2(0.f, 0.f);
        auto fma_col = [&](int m, int col, f32x2 x) {
#pragma unroll
            for (int q = 0; q < 2; ++q) acc[q][m] = fma2(dup2(drow[q][col]), x, acc[q][m]);
        };
        f32x2 keep_last[2];  // angle -(N - 1) of the reversed rows, for column N - 1
        f32x2 keep_mid[2];   // angle -N/2 of the reversed rows, for column N/2
#pragma unroll
        for (int p = 0; p < N / 4; ++p) {
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const float4 v = xget(m, p);
                const f32x2 lo = pk2(v.x, v.y), hi = pk2(v.z, v.w);
                if (m < 2) {
                    fma_col(m, 2 * p, lo);
                    fma_col(m, 2 * p + 1, hi);
                } else if (p == 0) {
                    fma_col(m, 0, lo);
                    keep_last[m - 2] = hi;
                } else {
                    fma_col(m, 2 * p, lo);
                    fma_col(m, 2 * p - 1, hi);
                }
            }
        }
#pragma unroll
        for (int m = 2; m < 4; ++m) {
            const float4 v = xget(m, N / 4);
            fma_col(m, N / 2 - 1, pk2(v.z, v.w));
            keep_mid[m - 2] = pk2(v.x, v.y);
        }
#pragma unroll
        for (int m = 2; m < 4; ++m) fma_col(m, N / 2, keep_mid[m - 2]);
#pragma unroll
        for (int p = N / 4; p < N / 2; ++p) {
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                if (m >= 2 && p == N / 4) continue;  // taken above
                const float4 v = xget(m, p);
                const f32x2 lo = pk2(v.x, v.y), hi = pk2(v.z, v.w);
                if (m < 2) {
                    fma_col(m, 2 * p, lo);
                    fma_col(m, 2 * p + 1, hi);
                } else {
                    fma_col(m, 2 * p, lo);
                    fma_col(m, 2 * p - 1, hi);
                }
            }
        }
#pragma unroll
        for (int m = 2; m < 4; ++m) fma_col(m, N - 1, keep_last[m - 2]);
        __syncwarp();
        if (live) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int r = t + q * LPC, rr = (N - r) & (N - 1);
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    if (kon[m]) {
                        // slot r of a reversed row is angle -r
                        float2 &x = Xh[xo[m] + (m < 2 ? r : rr)];
                        x = make_float2(x.x + lo2(acc[q][m]), x.y + hi2(acc[q][m]));
                    }
            }
        }
        __syncwarp();
    }
}

template <int N, int H>
struct ColTmaCfg {
    static constexpr int L = H / 2;
    static constexpr int T = rd_threads<N, H / 2>();  // the first pass takes both halves at once
    static constexpr int HB = L * N * 8;   // bytes of half a column
    static constexpr int TWB = H * 8 + 16;  // w^m (m < H) and a barrier a half
    static constexpr int SMEM = 2 * HB + TWB;
    // blocks an SM the registers are shaped for: two where the column is
    // small (up to 128 registers a thread at T <= 256), else one
    static constexpr int MINB = T < 512 && 2 * SMEM <= 227 * 1024 ? 2 : 1;
};

template <int N, int H>
constexpr bool col_tma_fits() {
    return ColTmaCfg<N, H>::SMEM <= 227 * 1024;
}

// Column l of unit c: the two columns of a class are consecutive units, so
// they run side by side and share its propagators in L2.
__device__ __forceinline__ int col_of_unit(int c, int W) { return (c & 1) ? W / 2 - (c >> 1) : c >> 1; }

// Persistent: block x takes units x, x + gridDim.x, ... Each half of the
// column has its slot of shared memory (rows 0 .. L-1 and L .. H-1), its
// copy-in completing on the slot's barrier; the next column is copied in as
// soon as the copy-out of this one has read the slots. (A third slot, to copy
// the next column's even half in during the transforms, measured slower: the
// propagators' stream from device memory during the apply has no bandwidth
// to spare.) Every wait for a copy-in is bounded; one that runs out sets
// g_col_fault and returns once the copies in flight have landed (again
// bounded), leaving the unit's column as it was.
template <int N, int H>
__global__ void __launch_bounds__(ColTmaCfg<N, H>::T, ColTmaCfg<N, H>::MINB)
    k_col_tma(const __grid_constant__ ColArgs a) {
    using C = ColTmaCfg<N, H>;
    constexpr int L = C::L, T = C::T, HB = C::HB, HF = L * N;  // HF: complex a half
    extern __shared__ __align__(128) float2 ctm[];
    float2 *XA = ctm, *XB = ctm + HF;
    float2 *tws = ctm + 2 * HF;  // exp(-2 pi i m / H), m < H
    const uint32_t bar = bulk::saddr(tws + H), sa = bulk::saddr(XA), sb = bulk::saddr(XB);  // barriers at bar, bar + 8
    const int tid = threadIdx.x;
    int c = blockIdx.x;
    if (c >= a.Wc) return;
    if (tid == 0) {
        bulk::bar_init(bar, 1);
        bulk::bar_init(bar + 8, 1);
    }
    __syncthreads();
    auto copy_in = [&](int unit) {  // one thread
        const float2 *g = a.col + (long long)col_of_unit(unit, a.W) * (N * H);
        bulk::bar_expect(bar, HB);
        bulk::load(sa, g, HB, bar);
        bulk::bar_expect(bar + 8, HB);
        bulk::load(sb, g + HF, HB, bar + 8);
    };
    if (tid == 0) copy_in(c);
    for (int m = tid; m < H; m += T) tws[m] = a.tw[m];
    for (uint32_t ph = 0; c < a.Wc; c += gridDim.x, ph ^= 1u) {
        const int l = col_of_unit(c, a.W);
        const bool ok = bulk::bar_wait(bar, ph) && bulk::bar_wait(bar + 8, ph);
        if (!__syncthreads_and(ok)) {
            if (tid == 0) {
                atomicExch(&g_col_fault, 1);
                (void)bulk::bar_wait(bar, ph);
                (void)bulk::bar_wait(bar + 8, ph);
                bulk::store_commit_wait();
            }
            return;
        }
        rd_dif<T, N, L, -1, RD_SPLIT, RD_TWO>(XA, XB, tws, tid);
        __syncthreads();
        col_apply_rows<T, N, H>(XA, XB, a.D, half_col_slot(l, a.W), a.col_slots, tid);
        __syncthreads();
        rd_dit<T, N, L, 1, RD_TWO, RD_MERGE>(XA, XB, tws, tid);
        bulk::fence_to_async();
        __syncthreads();
        if (tid == 0) {
            float2 *g = a.col + (long long)l * (N * H);
            bulk::store(g, sa, HB);
            bulk::store(g + HF, sb, HB);
            bulk::store_commit();
            if (c + (int)gridDim.x < a.Wc) {
                bulk::store_wait_read();  // the copy-out has read both slots
                copy_in(c + gridDim.x);
            }
        }
    }
    if (tid == 0) bulk::store_commit_wait();
}

// persistent grid: the columns, at most the blocks resident at once
template <int N, int H>
int col_grid(const ColArgs &a) {
    static int per_sm = 0;  // per instantiation, the same on every GB300
    if (per_sm <= 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_col_tma<N, H>, ColTmaCfg<N, H>::T,
                                                                      ColTmaCfg<N, H>::SMEM) != cudaSuccess)
        per_sm = 0;
    const long long cap = (long long)(a.num_sms > 0 ? a.num_sms : 1) * (per_sm > 0 ? per_sm : 1);
    return (int)(a.Wc < cap ? a.Wc : cap);
}

// the whole-column kernel where the column fits in shared memory, else the
// kernel of half columns
template <int N, int H>
cudaError_t col_attr() {
    if constexpr (col_tma_fits<N, H>())
        return cudaFuncSetAttribute(k_col_tma<N, H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    ColTmaCfg<N, H>::SMEM);
    else
        return cudaFuncSetAttribute(k_col_prop<N, H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    ColCfg<N, H>::SMEM);
}

template <int N, int H>
cudaError_t col_launch(const ColArgs &a, cudaStream_t s) {
    cudaError_t e = col_attr<N, H>();
    if (e != cudaSuccess) return e;
    if constexpr (col_tma_fits<N, H>())
        k_col_tma<N, H><<<col_grid<N, H>(a), ColTmaCfg<N, H>::T, ColTmaCfg<N, H>::SMEM, s>>>(a);
    else
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

// N = 30: the 30-angle system in 32 slots (its propagators stored by slots)
bool se2n_col_supported(int N, int H) {
    return (N == 16 || N == 30 || N == 32) &&
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

cudaError_t se2n_col_fault(int *host_flag, bool reset) {
    cudaError_t e = cudaMemcpyFromSymbol(host_flag, se2n::g_col_fault, sizeof(int));
    if (e == cudaSuccess && reset && *host_flag) {
        const int zero = 0;
        e = cudaMemcpyToSymbol(se2n::g_col_fault, &zero, sizeof(int));
    }
    return e;
}
