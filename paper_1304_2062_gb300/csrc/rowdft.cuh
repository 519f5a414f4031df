// DFTs along the rows of a block [row][N] in shared memory (row k holds the
// N angles of one index, one angle a lane), the layout in which the
// row-transformed volume lies in device memory, so that a block is copied in
// and out whole and every access of a pass is a contiguous run of rows. The
// transforms are in place and self-sorting in pairs: decimation in frequency
// takes natural order to digit-reversed order (rd_pos), decimation in time
// takes it back, in either direction. Used by the column pass (colprop.cu,
// DFTs along y, the radix-2 split and recombination folded in).
#pragma once

#include "smem_fft.cuh"

namespace se2n {

// radices of a DFT of length L, first pass of the decimation in frequency
// first (R3 = 1: two passes); the first radix is small so that the first
// pass has many butterflies
template <int L>
struct RdPlan {
    static constexpr int R1 = L == 32 ? 4 : (L == 256 ? 16 : (L == 192 || L == 384 ? 3 : 8));
    static constexpr int R2 = L == 32 || L == 64 || L == 192 || L == 384 || L == 512 ? 8 : 16;
    static constexpr int R3 = L / (R1 * R2);
    static_assert(R1 * R2 * R3 == L && (R3 == 1 || R3 == 8 || R3 == 16), "radix plan");
};

// row holding index f after the decimation in frequency:
// f = f1 + R1 f2 + R1 R2 f3 sits at f1 L / R1 + f2 L / (R1 R2) + f3
template <int L>
__device__ __forceinline__ int rd_pos(int f) {
    using P = RdPlan<L>;
    const int f1 = f % P::R1, q = f / P::R1;
    const int f2 = q % P::R2, f3 = q / P::R2;
    return f1 * (L / P::R1) + f2 * (L / (P::R1 * P::R2)) + f3;
}

// the index held by row p after the decimation in frequency (rd_pos inverted)
template <int L>
__device__ __forceinline__ int rd_index(int p) {
    using P = RdPlan<L>;
    constexpr int S1 = L / P::R1, S2 = L / (P::R1 * P::R2);
    const int f1 = p / S1, r = p - f1 * S1;
    const int f2 = r / S2, f3 = r - f2 * S2;
    return f1 + P::R1 * (f2 + P::R2 * f3);
}

// RD_ONE: the block XA; RD_TWO: the blocks XA and XB; RD_SPLIT / RD_MERGE:
// XA and XB the even and odd halves of DFTs of length 2L, with the radix-2
// split u = x_k + x_{k+L}, v = (x_k - x_{k+L}) w^k (w = exp(-2 pi i / 2L))
// folded into the reads (first forward pass) or the recombination
// x_k = y_k + w^-k z_k, x_{k+L} = y_k - w^-k z_k into the writes (last
// inverse pass).
enum { RD_ONE = 0, RD_TWO = 1, RD_SPLIT = 2, RD_MERGE = 3 };

// One in-place radix-R pass over blocks of LS rows (S = LS / R): butterfly
// (block c, j < S) of angle n on rows c LS + j + m S, m < R. Decimation in
// frequency (DIF): the R-point DFT with exp(DIR 2 pi i / R), output r times
// w^{j r} (w = exp(DIR 2 pi i / LS)), back to row j + r S. Decimation in time:
// input r times w^{j r}, then the R-point DFT. tws[e] = exp(-2 pi i e / 2L),
// so w^{j r} is tws[j r 2L / LS] or its conjugate. Each butterfly reads and
// writes the same rows: no barrier inside a pass.
template <int T, int N, int L, int R, int LS, int DIR, bool DIF, int MODE>
__device__ __forceinline__ void rd_pass(float2 *XA, float2 *XB, const float2 *tws, int tid) {
    constexpr int S = LS / R, BLK = L / LS, TW = 2 * L / LS;
    constexpr int BF = BLK * S;  // butterflies of one block and angle
    constexpr bool PAIR = MODE == RD_SPLIT || MODE == RD_MERGE;
    constexpr int TASKS = (MODE == RD_TWO ? 2 : 1) * BF * N;
    static_assert(T % N == 0, "one angle a thread");
    static_assert(MODE != RD_SPLIT || (DIF && DIR < 0), "the split is the first forward pass");
    static_assert(MODE != RD_MERGE || (!DIF && DIR > 0), "the recombination is the last inverse pass");
    const int n = tid % N;
#pragma unroll
    for (int task = tid; task < TASKS; task += T) {
        const int u = task / N;
        const int half = MODE == RD_TWO ? u / BF : 0;
        const int rest = u - half * BF;
        const int c = rest / S, j = rest - c * S;
        float2 *Xa = (half ? XB : XA) + (c * LS + j) * N + n;  // row m of the butterfly: Xa[m S N]
        float2 *Xb = XB + (c * LS + j) * N + n;                // the same row of the odd half
        float2 p[R], q[PAIR ? R : 1];
        if constexpr (MODE == RD_SPLIT) {
#pragma unroll
            for (int m = 0; m < R; ++m) {
                const float2 x0 = Xa[m * S * N], x1 = Xb[m * S * N];
                p[m] = cadd(x0, x1);
                q[m] = twiddle<-1>(csub(x0, x1), tws[j + m * S]);
            }
        } else {
#pragma unroll
            for (int m = 0; m < R; ++m) {
                p[m] = Xa[m * S * N];
                if constexpr (MODE == RD_MERGE) q[m] = Xb[m * S * N];
            }
        }
        if constexpr (!DIF) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const float2 w = tws[j * r * TW];
                p[r] = twiddle<DIR>(p[r], w);
                if constexpr (PAIR) q[r] = twiddle<DIR>(q[r], w);
            }
        }
        dft_small<R, DIR>(p);
        if constexpr (PAIR) dft_small<R, DIR>(q);
        if constexpr (DIF) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const float2 w = tws[j * r * TW];
                p[r] = twiddle<DIR>(p[r], w);
                if constexpr (PAIR) q[r] = twiddle<DIR>(q[r], w);
            }
        }
        if constexpr (MODE == RD_MERGE) {
#pragma unroll
            for (int m = 0; m < R; ++m) {
                const float2 o = twiddle<1>(q[m], tws[j + m * S]);
                Xa[m * S * N] = cadd(p[m], o);
                Xb[m * S * N] = csub(p[m], o);
            }
        } else {
#pragma unroll
            for (int m = 0; m < R; ++m) {
                Xa[m * S * N] = p[m];
                if constexpr (MODE == RD_SPLIT) Xb[m * S * N] = q[m];
            }
        }
    }
}

// decimation in frequency, natural order in, digit-reversed out (FIRST: the
// first pass's mode, REST: the others'); the caller synchronises before and after
template <int T, int N, int L, int DIR, int FIRST, int REST>
__device__ __forceinline__ void rd_dif(float2 *XA, float2 *XB, const float2 *tws, int tid) {
    using P = RdPlan<L>;
    rd_pass<T, N, L, P::R1, L, DIR, true, FIRST>(XA, XB, tws, tid);
    __syncthreads();
    rd_pass<T, N, L, P::R2, L / P::R1, DIR, true, REST>(XA, XB, tws, tid);
    if constexpr (P::R3 > 1) {
        __syncthreads();
        rd_pass<T, N, L, P::R3, P::R3, DIR, true, REST>(XA, XB, tws, tid);
    }
}

// decimation in time, digit-reversed in, natural order out (LAST: the last
// pass's mode, REST: the others')
template <int T, int N, int L, int DIR, int REST, int LAST>
__device__ __forceinline__ void rd_dit(float2 *XA, float2 *XB, const float2 *tws, int tid) {
    using P = RdPlan<L>;
    if constexpr (P::R3 > 1) {
        rd_pass<T, N, L, P::R3, P::R3, DIR, false, REST>(XA, XB, tws, tid);
        __syncthreads();
    }
    rd_pass<T, N, L, P::R2, L / P::R1, DIR, false, REST>(XA, XB, tws, tid);
    __syncthreads();
    rd_pass<T, N, L, P::R1, L, DIR, false, LAST>(XA, XB, tws, tid);
}

// threads of a block whose first pass has (L / R1) N butterflies (one block,
// or both halves at once), 128 .. 512
template <int N, int L>
__host__ __device__ constexpr int rd_threads() {
    return (L / RdPlan<L>::R1) * N >= 512 ? 512 : (L / RdPlan<L>::R1) * N <= 128 ? 128 : (L / RdPlan<L>::R1) * N;
}

}  // namespace se2n
