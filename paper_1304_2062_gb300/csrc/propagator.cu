// The S-step propagator of the Crank-Nicolson integration of eq. (4.2).
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
// k and (H/2 - k) mod H and for columns l and (W/2 - l) mod W. Negating wy
// maps a_r to -a_{-r} (both angle grids: theta_{-r} is -theta_r or
// pi - theta_r), so the operator of rows H/2 + k and H - k is R L R, with R
// the reversal r -> -r mod N of the angles, and their propagator R D R: the
// apply reverses their vectors around the product. A class is one row slot
// s in [0, H/4] (rows s, H/2 - s as they are, H/2 + s, H - s reversed) times
// one column pair: up to eight frequencies share one propagator.
//
// Increment form. M is I plus a small matrix (of order beta dt), and its
// powers are near I for the slow modes; stored as such in FP32 they would
// lose the small part. Every matrix here is D_m = M^m - I instead:
//   D_1 = 2 A'^{-1} L            (one step, as the packed kernel takes it)
//   D_2m = 2 D_m + D_m D_m       (squaring)
//   D_a+b = D_a + D_b + D_a D_b  (combination)
// and the propagator is applied as x <- x + D_S x, so rounding is relative to
// the change of x, as in the step-by-step integration. D_S is reached by a
// program of squarings and combinations over two matrices with the fewest
// products (se2n_prop_chain): 11 for S = 500 where binary powering takes 13.
//
// Storage. B+ and B- are polynomials in one symmetric matrix, so M and D_S
// are symmetric. D_S is kept by cyclic diagonals, S_m[i] = D[i, (i + m) mod N]
// for m = 0 .. N/2 (the mean of the two mirrored FP32 entries): N (N/2 + 1)
// floats a class instead of N^2, and a lane i of the apply reads S_m[i] and
// S_m[i - m], both coalesced across the warp.
//
// One step in scaled form: A' = (1/c) I - L, c = beta dt / 2, L the operator
// divided by beta (diagonal -2 - a_r^2/beta, off-diagonals and corners 1);
// x_{n+1} = x_n + 2 A'^{-1} L x_n. D_1 is built column by column: column i
// is 2 A'^{-1} (Lap e_i) - 2 (a_i^2/beta) A'^{-1} e_i, with Lap the cyclic
// second difference, so the -2 and the a_i^2/beta never meet in one FP32
// number. A' is cyclic tridiagonal: Thomas elimination of its torn part plus
// one Sherman-Morrison correction.
#include <algorithm>
#include <unordered_map>
#include <vector>

#include "diffuse_x2.cuh"
#include "prop_classes.cuh"

namespace se2n {

namespace {

// The row slot and the column pair of class u.
__device__ __forceinline__ void class_slots(const PropArgs &a, long long u, int &srow, int &l, int &lb) {
    srow = (int)(u / a.col_slots);
    const int scol = (int)(u - (long long)srow * a.col_slots);
    if (a.half) {
        l = scol;
        lb = a.W / 2 - scol;
    } else {
        pair_row(scol, a.W, l, lb);
    }
}

// The class that build item w computes, and the class that receives it
// permuted (its transpose) or -1. Without sharing, item w is class w. With
// sharing (square planes, Hermitian half) the items are the n (n + 1) / 2
// slot pairs i <= j of the n x n grid of row and column slots, row by row:
// class (i, j) has wy = sin(2 pi i / H), wx = sin(2 pi j / W), and class
// (j, i) swaps them; a_r = wx cos th_r + wy sin th_r becomes a at the angle
// pi/2 - th_r, i.e. index perm_shift - r, so the transpose's operator is
// P A P with the permutation P: r -> (perm_shift - r) mod N (which keeps the
// cyclic second difference), and its propagator is P D_S P.
__device__ __forceinline__ long long build_class(const PropArgs &a, long long w, long long &partner) {
    if (!a.share_t) {
        partner = -1;
        return w;
    }
    const long long n = a.col_slots;
    // row i starts at item i n - i (i - 1) / 2
    const double b = 2.0 * (double)n + 1.0;
    long long i = (long long)((b - sqrt(b * b - 8.0 * (double)w)) * 0.5);
    if (i < 0) i = 0;
    while (i > 0 && i * n - i * (i - 1) / 2 > w) --i;
    while ((i + 1) * n - (i + 1) * i / 2 <= w) ++i;
    const long long j = i + (w - (i * n - i * (i - 1) / 2));
    partner = i != j ? j * n + i : -1;
    return i * n + j;
}

// Entry (i, j) of the stored matrix of class u: P D_S P for a transposed
// partner (shift = perm_shift), D_S itself (shift < 0). NE <= N angles are
// the system's; a padded index i >= NE stays where it is.
template <int N, int NE = N>
__device__ __forceinline__ int perm_index(int i, int shift) {
    if (shift < 0 || i >= NE) return i;
    const int v = shift - i;
    return v < 0 ? v + NE : v;
}

// x = A'^{-1} r and y = A'^{-1} s in place (N values each), with the torn
// factor's reciprocal pivots G and the Sherman-Morrison vector q = T^{-1} u:
// the two right-hand sides run through the same sweeps as independent chains.
template <int N>
__device__ __forceinline__ void prop_solve2(float (&x)[N], float (&y)[N], const float *G, const float *q,
                                            float inv_d0, float inv_den) {
#pragma unroll
    for (int j = 1; j < N; ++j) {
        x[j] = fmaf(G[j - 1], x[j - 1], x[j]);
        y[j] = fmaf(G[j - 1], y[j - 1], y[j]);
    }
    x[N - 1] *= G[N - 1];
    y[N - 1] *= G[N - 1];
#pragma unroll
    for (int j = N - 2; j >= 0; --j) {
        x[j] = (x[j] + x[j + 1]) * G[j];
        y[j] = (y[j] + y[j + 1]) * G[j];
    }
    const float wx = fmaf(x[N - 1], inv_d0, x[0]) * inv_den;
    const float wy = fmaf(y[N - 1], inv_d0, y[0]) * inv_den;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        x[j] = fmaf(-wx, q[j], x[j]);
        y[j] = fmaf(-wy, q[j], y[j]);
    }
}

// Lane 0 of a class: the torn factor of A' (reciprocal pivots G, diagonal
// d_j = 1/c + 2 + a_j^2/beta, with the corners folded into the first and last
// pivots) and q = T^{-1} u, u = (-d0, 0, ..., 0, -1), for the Sherman-Morrison
// correction; scal = (1/d0, 1/(1 + v.q)).
template <int N>
__device__ __forceinline__ void prop_factor(const PropArgs &a, float wx, float wy, float *G, float *q, float *scal) {
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

template <int N>
struct SymCfg;

// D_S of class u from a symmetric matrix in the layout of SymCfg<N>: as rows
// in 16-byte chunks, chunk-major (PROP_CHUNKS), row-major (PROP_ROWS) or by
// cyclic diagonals; lanes t of `lanes`. shift >= 0 stores the permuted matrix
// P D_S P of a transposed class, which PROP_ROWS leaves out (the tiled apply
// reads the built class).
template <int N, int NE = N>
__device__ __forceinline__ void prop_store(const PropArgs &a, const float *Rm, long long u, bool live, int t,
                                           int lanes, int shift = -1) {
    using C = SymCfg<N>;
    if (!live || u < 0) return;
    if (a.rows == PROP_ROWS) {
        if (shift >= 0) return;  // (N angles only: se2n_prop_apply_fmt)
        float4 *out = reinterpret_cast<float4 *>(a.D + u * (long long)(N * N));
        for (int e = t; e < N * N / 4; e += lanes) {
            const int i = e / (N / 4), c = e - i * (N / 4);
            out[e] = *reinterpret_cast<const float4 *>(Rm + C::at(i, 4 * c));
        }
    } else if (a.rows == PROP_CHUNKS) {
        // for the column pass: row i, columns 4c .. 4c + 3 as slots (an
        // NE-angle system at the slots of slot_of_angle)
        float4 *out = reinterpret_cast<float4 *>(a.D + u * (long long)(N * N));
        for (int e = t; e < N * N / 4; e += lanes) {
            const int c = e / N, i = e - c * N;
            if (shift < 0 && NE == N) {
                out[e] = *reinterpret_cast<const float4 *>(Rm + C::at(i, 4 * c));
            } else {
                const int pi = perm_index<N, NE>(angle_of_slot<N, NE>(i), shift);
                out[e] = make_float4(Rm[C::at(pi, perm_index<N, NE>(angle_of_slot<N, NE>(4 * c), shift))],
                                     Rm[C::at(pi, perm_index<N, NE>(angle_of_slot<N, NE>(4 * c + 1), shift))],
                                     Rm[C::at(pi, perm_index<N, NE>(angle_of_slot<N, NE>(4 * c + 2), shift))],
                                     Rm[C::at(pi, perm_index<N, NE>(angle_of_slot<N, NE>(4 * c + 3), shift))]);
            }
        }
    } else {
        float *out = a.D + u * (long long)((N / 2 + 1) * N);
        for (int e = t; e < (N / 2 + 1) * N; e += lanes) {
            const int m = e / N, i = e - m * N;
            out[e] = Rm[C::at(perm_index<N, NE>(i, shift), perm_index<N, NE>((i + m) & (N - 1), shift))];
        }
    }
}

// Build with symmetric products (N = 16, 32; N = 64 below). Every matrix of the powering
// is a function of the one symmetric operator of the class (D_1 = 2 A'^{-1} L
// with A' = I/c - L), so all of them are symmetric and commute, and so are
// the products D_m D_m and D_a D_b. A matrix is kept once, row-major (its
// rows are its columns), and a product is computed on the tiles of its upper
// triangle only and mirrored: 10 of 16 tiles of 8 x 8 at N = 32 (3 of 4 at
// N = 16), one lane a tile, 3 classes a warp at N = 32 and 10 at N = 16.
// The mirrored tile is exactly symmetric; for a diagonal tile the upper half
// is written and mirrored. D_1, built column by column by the solves, is
// symmetrised first (the mean of mirrored entries).
//
// Banks (N = 32). A 16-byte shared access is served 8 lanes at a time, and
// rows 8 apart (8 LD floats) fall on the same banks. The tiles' own rows
// (the epilogue's loads and stores) would collide whenever two lanes of one
// quarter-warp hold tiles in the same tile column (or, mirrored, the same
// tile row). So element (i, j) sits at i LD + ((j + SKEW(i / 8)) mod N), and
// lane t of a class takes tile TILE[t]: with the class bases 4 banks apart,
// every quarter-warp touches 8 different groups of 4 banks in every access
// of a product (the k steps, the tile rows and the mirrored rows), found by
// an exhaustive search over the skews and a random one over the tile orders.
template <int N>
struct SymCfg {
    static constexpr int WARPS = 4;
    static constexpr int NT = N / 8;                 // tiles a side
    static constexpr int TILES = NT * (NT + 1) / 2;  // upper-triangle tiles: lanes a class
    static constexpr int CPW = 32 / TILES;           // classes a warp
    // row stride, floats; at N = 64 columns 32 .. 63 sit 4 floats further
    // on, so that the 16-byte pieces at columns 8 b and 8 b + 4 (b = 0 .. 7)
    // that the eight lanes of a quarter-warp read in a product fall on
    // eight different groups of four banks
    static constexpr int LD = N == 64 ? 72 : N + 4;
    static constexpr int MAT = N * LD;
    static constexpr int CLASS_FLOATS = 2 * MAT + 2 * N + 4;  // P, R, pivots, q, scalars
    static constexpr int SMEM = WARPS * CPW * CLASS_FLOATS * 4;
    static constexpr int SBLK = (N / 2 + 1) * N;
    static_assert(N == 16 || N == 32 || N == 64, "8 x 8 tiles of 16, 32 or 64");
    static_assert(N != 32 || CLASS_FLOATS % 32 == 4, "class bases 4 banks apart");
    // SKEW(b) for b = 0 .. 3: 0, 20, 4, 24 floats (N = 32), none at N = 16
    static __device__ __forceinline__ int skew(int b) { return N == 32 ? (0x18041400u >> (8 * b)) & 0xff : 0; }
    static __device__ __forceinline__ int at(int i, int j) {
        return N == 64 ? i * LD + j + 4 * (j >> 5) : i * LD + ((j + skew(i >> 3)) & (N - 1));
    }
    // tile (bi, bj) = (TILE[t] / 4, TILE[t] mod 4) of lane t (N = 32), TILE =
    // 4 bi + bj of (2,3) (0,2) (1,2) (0,0) (2,2) (0,1) (1,3) (0,3) (3,3) (1,1),
    // four bits each
    static __device__ __forceinline__ void tile(int t, int &bi, int &bj) {
        if constexpr (N == 32) {
            const int v = (int)((0x5F371A062BULL >> (4 * (t < 10 ? t : 0))) & 0xF);
            bi = v >> 2;
            bj = v & 3;
        } else {
            // row order of the upper triangle
            bi = 0;
            int rem = t;
            while (rem >= NT - bi) {
                rem -= NT - bi;
                ++bi;
            }
            bj = bi + rem;
        }
    }
};

// out = two * X + Y + A B on the upper-triangle tile (bi, bj) of this lane,
// mirrored; A, B, X, Y, out symmetric N x N row-major (stride LD), Y may be
// null, out may be an input (the warp, or with BLOCK the block, synchronises
// between the reads and the writes; every lane of it calls this together).
template <int N, bool BLOCK = false>
__device__ __forceinline__ void sym_gemm(const float *A, const float *B, const float *X, float two, const float *Y,
                                         float *out, int bi, int bj, bool active) {
    using C = SymCfg<N>;
    const int r0 = 8 * bi, c0 = 8 * bj;
    f32x2 acc[8][4];  // [row][column pair]
    if (active) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 8; c += 4) {
                const float4 xv = *reinterpret_cast<const float4 *>(X + C::at(r0 + r, c0 + c));
                float4 yv = make_float4(0.f, 0.f, 0.f, 0.f);
                if (Y) yv = *reinterpret_cast<const float4 *>(Y + C::at(r0 + r, c0 + c));
                acc[r][c / 2] = pk2(fmaf(two, xv.x, yv.x), fmaf(two, xv.y, yv.y));
                acc[r][c / 2 + 1] = pk2(fmaf(two, xv.z, yv.z), fmaf(two, xv.w, yv.w));
            }
        // blocks of 8 rows k share their skew: the four slice offsets are
        // formed once a block and the rows are then fixed strides apart
#pragma unroll 1
        for (int kb = 0; kb < N; kb += 8) {
            const float *Ak0 = A + C::at(kb, r0), *Ak1 = A + C::at(kb, r0 + 4);
            const float *Bk0 = B + C::at(kb, c0), *Bk1 = B + C::at(kb, c0 + 4);
#pragma unroll 2
            for (int kk = 0; kk < 8; ++kk) {
                // A[r][k] = A[k][r]: row k of A, columns r0 .. r0 + 7
                const float4 a0 = *reinterpret_cast<const float4 *>(Ak0 + kk * C::LD);
                const float4 a1 = *reinterpret_cast<const float4 *>(Ak1 + kk * C::LD);
                const float4 b0 = *reinterpret_cast<const float4 *>(Bk0 + kk * C::LD);
                const float4 b1 = *reinterpret_cast<const float4 *>(Bk1 + kk * C::LD);
                const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const f32x2 bv[4] = {pk2(b0.x, b0.y), pk2(b0.z, b0.w), pk2(b1.x, b1.y), pk2(b1.z, b1.w)};
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const f32x2 s = dup2(av[r]);
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] = fma2(s, bv[c], acc[r][c]);
                }
            }
        }
    }
    if constexpr (BLOCK)
        __syncthreads();
    else
        __syncwarp();
    if (active) {
        float v[8][8];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                v[r][2 * c] = lo2(acc[r][c]);
                v[r][2 * c + 1] = hi2(acc[r][c]);
            }
        // a diagonal tile takes its upper half for the lower one
        if (bi == bj) {
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < r; ++c) v[r][c] = v[c][r];
        }
        // the tile and its transpose, as 16-byte rows
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            *reinterpret_cast<float4 *>(out + C::at(r0 + r, c0)) = make_float4(v[r][0], v[r][1], v[r][2], v[r][3]);
            *reinterpret_cast<float4 *>(out + C::at(r0 + r, c0 + 4)) =
                make_float4(v[r][4], v[r][5], v[r][6], v[r][7]);
        }
        if (bi != bj) {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                *reinterpret_cast<float4 *>(out + C::at(c0 + c, r0)) =
                    make_float4(v[0][c], v[1][c], v[2][c], v[3][c]);
                *reinterpret_cast<float4 *>(out + C::at(c0 + c, r0 + 4)) =
                    make_float4(v[4][c], v[5][c], v[6][c], v[7][c]);
            }
        }
    }
}

template <int N, int NE = N>
__global__ void __launch_bounds__(SymCfg<N>::WARPS * 32) k_prop_build_sym(const __grid_constant__ PropArgs a) {
    using C = SymCfg<N>;
    extern __shared__ __align__(16) float psm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / C::TILES, t = lane - g * C::TILES;
    const bool active = g < C::CPW;
    // this lane's tile (bi, bj), bi <= bj
    int bi, bj;
    C::tile(t, bi, bj);
    float *base = psm + (warp * C::CPW + (active ? g : 0)) * C::CLASS_FLOATS;
    float *P = base, *R = base + C::MAT;
    float *G = base + 2 * C::MAT;
    float *q = G + N;
    float *scal = q + N;  // 1/d0, 1/(1 + v.q)
    const long long stride = (long long)gridDim.x * C::WARPS * C::CPW;
    // classes are taken warp-uniformly so that every lane reaches each __syncwarp,
    // warp-major over the grid: where the classes do not divide evenly, the
    // warps that take one chunk more are spread over the blocks (and SMs)
    // instead of filling the first blocks
    for (long long u0 = ((long long)warp * gridDim.x + blockIdx.x) * C::CPW; u0 < a.items; u0 += stride) {
        const bool live = active && u0 + g < a.items;
        long long partner;
        const long long u = build_class(a, live ? u0 + g : a.items - 1, partner);
        int k, l, lb;
        class_slots(a, u, k, l, lb);
        const float wx = sin_2pi_frac(l, a.W), wy = sin_2pi_frac(k, a.H);
        if (active && t == 0) prop_factor<NE>(a, wx, wy, G, q, scal);
        __syncwarp();
        // D_1 column by column into R (R row c = column c), then P = (R + R^T) / 2.
        // A system of NE < N angles sits in the top-left NE x NE block, the
        // rest zero: the powering keeps the zero blocks zero (2 D + D D and
        // D_a + D_b + D_a D_b of block-diagonal matrices), so the block is the
        // NE-angle system's D_S.
        if (active) {
            const float inv_d0 = scal[0], inv_den = scal[1];
#pragma unroll 1
            for (int c = t; c < NE; c += C::TILES) {
                const float ar = fmaf(wx, a.cs[c], wy * a.sn[c]);
                const float e2 = ar * ar * a.inv_beta;
                const int cm = (c == 0) ? NE - 1 : c - 1, cp = (c == NE - 1) ? 0 : c + 1;
                float x[NE], y[NE];
#pragma unroll
                for (int j = 0; j < NE; ++j) {
                    x[j] = (j == c) ? 1.0f : 0.0f;
                    y[j] = (j == c) ? -2.0f : ((j == cm || j == cp) ? 1.0f : 0.0f);
                }
                prop_solve2<NE>(x, y, G, q, inv_d0, inv_den);
                float d[N];
#pragma unroll
                for (int j = NE; j < N; ++j) d[j] = 0.0f;
#pragma unroll
                for (int j = 0; j < NE; ++j) d[j] = fmaf(2.0f, y[j], -2.0f * e2 * x[j]);
#pragma unroll
                for (int j = 0; j < N; j += 4)
                    *reinterpret_cast<float4 *>(R + C::at(c, j)) = make_float4(d[j], d[j + 1], d[j + 2], d[j + 3]);
            }
            if constexpr (NE < N) {
#pragma unroll 1
                for (int c = NE + t; c < N; c += C::TILES)
#pragma unroll
                    for (int j = 0; j < N; j += 4)
                        *reinterpret_cast<float4 *>(R + C::at(c, j)) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
        }
        __syncwarp();
        // rows i of this lane: P[i][j] = (R[i][j] + R[j][i]) / 2, which gives
        // P[j][i] the same bits
        if (active) {
#pragma unroll 1
            for (int i = t; i < N; i += C::TILES)
#pragma unroll
                for (int j = 0; j < N; j += 4) {
                    const float4 ri = *reinterpret_cast<const float4 *>(R + C::at(i, j));
                    *reinterpret_cast<float4 *>(P + C::at(i, j)) =
                        make_float4(0.5f * (ri.x + R[C::at(j, i)]), 0.5f * (ri.y + R[C::at(j + 1, i)]),
                                    0.5f * (ri.z + R[C::at(j + 2, i)]), 0.5f * (ri.w + R[C::at(j + 3, i)]));
                }
        }
        __syncwarp();
        // the powering program: P starts as D_1, R empty
#pragma unroll 1
        for (int o = 0; o < a.chain_len; ++o) {
            const int op = a.chain[o];
            if (op != PROP_COPY) {
                // 2 P + P P into P, 2 R + R R into P, or R + P + R P into R
                // (one call site: the products share their registers)
                const bool add = op == PROP_ADD;
                const float *A = op == PROP_SQ_P ? P : R;
                sym_gemm<N>(A, add ? P : A, A, add ? 1.0f : 2.0f, add ? P : nullptr, add ? R : P, bi, bj, active);
            } else if (active) {
#pragma unroll 1
                for (int i = t; i < N; i += C::TILES)
#pragma unroll
                    for (int j = 0; j < N; j += 4)
                        *reinterpret_cast<float4 *>(R + i * C::LD + j) =
                            *reinterpret_cast<const float4 *>(P + i * C::LD + j);
            }
            __syncwarp();
        }
        prop_store<N, NE>(a, a.chain_in_r ? R : P, u, live, t, C::TILES);
        prop_store<N, NE>(a, a.chain_in_r ? R : P, partner, live, t, C::TILES, a.perm_shift);
        __syncwarp();
    }
}

// The symmetric build at N = 64: the 36 upper-triangle 8 x 8 tiles of a
// product take 36 lanes, so a class spans two warps; three classes a
// 128-thread block, synchronised block-wide. As at N = 16, 32, each matrix is
// kept once (its rows are its columns) and every tile is written with its
// transpose, so the result is exactly symmetric: two matrices a class
// instead of the three of a full product kept column- and row-major, and 36
// of the 64 tiles of a product computed.
template <int N>
struct SymWideCfg {
    using S = SymCfg<N>;
    static constexpr int THREADS = 128;
    static constexpr int LPC = S::TILES;           // lanes a class
    static constexpr int CPB = THREADS / LPC;      // classes a block
    static constexpr int SMEM = CPB * S::CLASS_FLOATS * 4;
};

template <int N>
__global__ void __launch_bounds__(SymWideCfg<N>::THREADS) k_prop_build_symw(const __grid_constant__ PropArgs a) {
    using S = SymCfg<N>;
    using C = SymWideCfg<N>;
    extern __shared__ __align__(16) float psm[];
    const int tid = threadIdx.x, cb = tid / C::LPC, t = tid - cb * C::LPC;
    const bool active = cb < C::CPB;
    int bi, bj;
    S::tile(active ? t : 0, bi, bj);
    float *base = psm + (active ? cb : 0) * S::CLASS_FLOATS;
    float *P = base, *R = base + S::MAT;
    float *G = base + 2 * S::MAT;
    float *q = G + N;
    float *scal = q + N;  // 1/d0, 1/(1 + v.q)
    const long long stride = (long long)gridDim.x * C::CPB;
    // classes are taken block-uniformly so that every thread reaches each barrier
    for (long long u0 = (long long)blockIdx.x * C::CPB; u0 < a.items; u0 += stride) {
        const bool live = active && u0 + cb < a.items;
        long long partner;
        const long long u = build_class(a, live ? u0 + cb : a.items - 1, partner);
        int k, l, lb;
        class_slots(a, u, k, l, lb);
        const float wx = sin_2pi_frac(l, a.W), wy = sin_2pi_frac(k, a.H);
        if (active && t == 0) prop_factor<N>(a, wx, wy, G, q, scal);
        __syncthreads();
        // D_1 column by column into R (R row c = column c); pivots and q are
        // read from shared memory (their 2 N values exceed the registers)
        if (active) {
            const float inv_d0 = scal[0], inv_den = scal[1];
#pragma unroll 1
            for (int c = t; c < N; c += C::LPC) {
                const float ar = fmaf(wx, a.cs[c], wy * a.sn[c]);
                const float e2 = ar * ar * a.inv_beta;
                const int cm = (c == 0) ? N - 1 : c - 1, cp = (c == N - 1) ? 0 : c + 1;
                float x[N], y[N];
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    x[j] = (j == c) ? 1.0f : 0.0f;
                    y[j] = (j == c) ? -2.0f : ((j == cm || j == cp) ? 1.0f : 0.0f);
                }
                prop_solve2<N>(x, y, G, q, inv_d0, inv_den);
#pragma unroll
                for (int j = 0; j < N; j += 4)
                    *reinterpret_cast<float4 *>(R + S::at(c, j)) =
                        make_float4(fmaf(2.0f, y[j], -2.0f * e2 * x[j]), fmaf(2.0f, y[j + 1], -2.0f * e2 * x[j + 1]),
                                    fmaf(2.0f, y[j + 2], -2.0f * e2 * x[j + 2]),
                                    fmaf(2.0f, y[j + 3], -2.0f * e2 * x[j + 3]));
            }
        }
        __syncthreads();
        // P = (R + R^T) / 2, rows of this lane (P[j][i] gets the same bits)
        if (active) {
#pragma unroll 1
            for (int i = t; i < N; i += C::LPC)
#pragma unroll 4
                for (int j = 0; j < N; j += 4) {
                    const float4 ri = *reinterpret_cast<const float4 *>(R + S::at(i, j));
                    *reinterpret_cast<float4 *>(P + S::at(i, j)) =
                        make_float4(0.5f * (ri.x + R[S::at(j, i)]), 0.5f * (ri.y + R[S::at(j + 1, i)]),
                                    0.5f * (ri.z + R[S::at(j + 2, i)]), 0.5f * (ri.w + R[S::at(j + 3, i)]));
                }
        }
        __syncthreads();
        // the powering program: P starts as D_1, R empty
#pragma unroll 1
        for (int o = 0; o < a.chain_len; ++o) {
            const int op = a.chain[o];
            if (op != PROP_COPY) {
                const bool add = op == PROP_ADD;
                const float *A = op == PROP_SQ_P ? P : R;
                sym_gemm<N, true>(A, add ? P : A, A, add ? 1.0f : 2.0f, add ? P : nullptr, add ? R : P, bi, bj,
                                  active);
            } else if (active) {
#pragma unroll 1
                for (int i = t; i < N; i += C::LPC)
#pragma unroll 4
                    for (int j = 0; j < S::LD; j += 4)
                        *reinterpret_cast<float4 *>(R + i * S::LD + j) =
                            *reinterpret_cast<const float4 *>(P + i * S::LD + j);
            }
            __syncthreads();
        }
        prop_store<N>(a, a.chain_in_r ? R : P, u, live, t, C::LPC);
        prop_store<N>(a, a.chain_in_r ? R : P, partner, live, t, C::LPC, a.perm_shift);
        __syncthreads();
    }
}

template <int N>
cudaError_t launch_build_wide(const PropArgs &a, int num_sms, cudaStream_t s) {
    using C = SymWideCfg<N>;
    cudaError_t e = cudaFuncSetAttribute(k_prop_build_symw<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_prop_build_symw<N>, C::THREADS, C::SMEM);
    if (e != cudaSuccess) return e;
    long long blocks = (a.items + C::CPB - 1) / C::CPB;
    const long long cap = (long long)num_sms * (per_sm > 0 ? per_sm : 1);
    if (blocks > cap) blocks = cap;
    k_prop_build_symw<N><<<(unsigned)blocks, C::THREADS, C::SMEM, s>>>(a);
    return cudaGetLastError();
}

// x <- x + D_S x for the (up to eight) frequencies of every class. A lane
// owns RPL rows of a class. It issues every global load it needs at once (its
// rows' diagonal entries, coalesced across the lanes of the class, and its
// rows of the eight frequencies' vectors), then expands the rows into a padded
// N x (N + 1) matrix in shared memory, reads them back into registers in
// column order, and for every column j loads x_j of the eight frequencies
// once (a shared-memory broadcast for all its rows) for RPL x 8 packed FMAs.
// The vectors of the reversed rows are stored reversed (angle r at slot -r),
// so slot r of every frequency receives row r of D x and goes back to the
// angle it came from.
template <int N>
struct ApplyCfg {
    static constexpr int WARPS = 4;
    static constexpr int RPL = N == 16 ? 1 : 2;  // rows a lane
    static constexpr int LPC = N / RPL;          // lanes a class: 16, 16 or 32
    static constexpr int CPW = 32 / LPC;         // classes a warp
    static constexpr int MEM = 8;                // frequencies a class
    static constexpr int DLD = N + 1;            // row stride of the expanded matrix
    static constexpr int DF = N * DLD;
    static constexpr int XF = 2 * MEM * N;       // x_j of the eight frequencies, (re, im) each
    // class regions 8 floats apart modulo 32 so that the classes of a warp
    // fall on different banks
    static constexpr int CLASS_FLOATS = ((DF + XF + 31) / 32) * 32 + 8;
    static constexpr int SBLK = (N / 2 + 1) * N;  // stored floats a class (cyclic diagonals)
    static constexpr int SMEM = WARPS * CPW * CLASS_FLOATS * 4;
    static_assert(XF % 4 == 0 && (CLASS_FLOATS % 4) == 0, "16-byte vectors");
};

// NE < N: a system of NE angles stored padded to N (the propagator's rows and
// columns NE .. N - 1 zero); only angles below NE are loaded and stored, and
// the reversal of rows 2 and 3 is modulo NE.
template <int N, int NE = N>
__global__ void __launch_bounds__(ApplyCfg<N>::WARPS * 32) k_prop_apply(const __grid_constant__ PropArgs a) {
    using C = ApplyCfg<N>;
    constexpr int M = C::MEM;
    extern __shared__ __align__(16) float asm_[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / C::LPC, t = lane - g * C::LPC;
    float *xs = asm_ + (warp * C::CPW + g) * C::CLASS_FLOATS;  // [N][2M], 16-byte aligned
    float *Df = xs + C::XF;                                     // [N][DLD]
    const long long stride = (long long)gridDim.x * C::WARPS * C::CPW;
    for (long long u0 = ((long long)blockIdx.x * C::WARPS + warp) * C::CPW; u0 < a.classes; u0 += stride) {
        const long long u = u0 + g;
        const bool live = u < a.classes;
        const long long uc = live ? u : a.classes - 1;
        int srow, l, lb;
        class_slots(a, uc, srow, l, lb);
        int k[4];
        bool kon[4];
        slot_rows(srow, a.H, k, kon);
        // frequency m = 2 (row) + (column); rows 2 and 3 reversed
        long long f[M];
        bool on[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            f[m] = (long long)k[m / 2] * a.Wc + ((m & 1) ? lb : l);
            on[m] = live && kon[m / 2] && (!(m & 1) || lb != l);
        }
        const float *Sc = a.D + uc * (long long)C::SBLK;
        // row r: D[r, r + d] = S_d[r] (d = 0 .. N/2), D[r, r - d] = S_d[r - d]
        // (d = 1 .. N/2 - 1); dv[i][d] and dv[i][N/2 + d] hold them
        float dv[C::RPL][N];
        float2 mine[M][C::RPL];
#pragma unroll
        for (int i = 0; i < C::RPL; ++i) {
            const int r = t + i * C::LPC;
#pragma unroll
            for (int d = 0; d <= N / 2; ++d) dv[i][d] = __ldg(Sc + d * N + r);
#pragma unroll
            for (int d = 1; d < N / 2; ++d) dv[i][N / 2 + d] = __ldg(Sc + d * N + ((r - d) & (N - 1)));
#pragma unroll
            for (int m = 0; m < M; ++m)
                mine[m][i] = on[m] && r < NE ? a.vol[(long long)r * a.HW + f[m]] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < C::RPL; ++i) {
            const int r = t + i * C::LPC;
            const int rr = r < NE ? (r == 0 ? 0 : NE - r) : r;
#pragma unroll
            for (int d = 0; d <= N / 2; ++d) Df[r * C::DLD + ((r + d) & (N - 1))] = dv[i][d];
#pragma unroll
            for (int d = 1; d < N / 2; ++d) Df[r * C::DLD + ((r - d) & (N - 1))] = dv[i][N / 2 + d];
#pragma unroll
            for (int m = 0; m < M; ++m) *reinterpret_cast<float2 *>(xs + (m < 4 ? r : rr) * (2 * M) + 2 * m) = mine[m][i];
        }
        __syncwarp();
        float drow[C::RPL][N];
#pragma unroll
        for (int i = 0; i < C::RPL; ++i)
#pragma unroll
            for (int j = 0; j < N; ++j) drow[i][j] = Df[(t + i * C::LPC) * C::DLD + j];
        f32x2 acc[C::RPL][M];
#pragma unroll
        for (int i = 0; i < C::RPL; ++i)
#pragma unroll
            for (int m = 0; m < M; ++m) acc[i][m] = pk2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            f32x2 xm[M];
#pragma unroll
            for (int q = 0; q < M / 2; ++q) {
                const float4 v = *reinterpret_cast<const float4 *>(xs + j * (2 * M) + 4 * q);
                xm[2 * q] = pk2(v.x, v.y);
                xm[2 * q + 1] = pk2(v.z, v.w);
            }
#pragma unroll
            for (int i = 0; i < C::RPL; ++i) {
                const f32x2 sd = dup2(drow[i][j]);
#pragma unroll
                for (int m = 0; m < M; ++m) acc[i][m] = fma2(sd, xm[m], acc[i][m]);
            }
        }
#pragma unroll
        for (int i = 0; i < C::RPL; ++i) {
            const int r = t + i * C::LPC;
            const int rr = r < NE ? (r == 0 ? 0 : NE - r) : r;
#pragma unroll
            for (int m = 0; m < M; ++m)
                if (on[m] && r < NE) {
                    // slot r holds the value of angle r (rows 0, 1) or -r (rows 2, 3)
                    const float2 x0 = *reinterpret_cast<const float2 *>(xs + r * (2 * M) + 2 * m);
                    a.vol[(long long)(m < 4 ? r : rr) * a.HW + f[m]] =
                        make_float2(x0.x + lo2(acc[i][m]), x0.y + hi2(acc[i][m]));
                }
        }
        __syncwarp();
    }
}

// The apply on the Hermitian half at N = 64, tile by tile. A tile is one row
// slot times CT = 16 consecutive column slots: 16 classes, 128 frequencies.
// Its vectors come in as runs of 16 consecutive columns of one row of one
// angle plane (128 bytes) and go back the same way, so every access to the
// volume is coalesced, where a class on its own touches 8 bytes in each of
// 512 places. In shared memory a class is [N slots][8 frequencies] complex,
// and the slot of angle r folds in the reversal of rows 2, 3 and, for a
// transposed class (share_t, row slot > column slot), the permutation P: such
// a class applies P D P with D the propagator of its transpose, built and
// stored once, as x + P D P x = P (P x + D (P x)). D_S is stored row-major;
// its row j is its column j (symmetric), so the eight lanes (rb) that hold
// rows 4 rb .. 4 rb + 3 and N/2 + 4 rb .. N/2 + 4 rb + 3 read column j of
// their rows as one 128-byte run. Rows of D come in four at a time (1 KB)
// by asynchronous copies into a ring of four slots a warp, three ahead of
// the rows in use, so that 48 KB of them are in flight on an SM at a time
// without registers to hold them. A warp applies one class: lane
// (rb, mp) accumulates its eight rows for frequencies 2 mp and 2 mp + 1, two
// rows a packed FMA, with x_j of both frequencies one 16-byte broadcast from
// shared memory; the sums run over j in slot order and x is added last.
// Tiles go in super-tiles of 16 x 16 classes (one tile wide), each (above
// the diagonal) followed by its transpose, so the transposed classes find
// their propagators in L2.
template <int N>
struct TileCfg {
    static constexpr int CT = 16;                  // column slots (classes) a tile
    static constexpr int WARPS = 8;                // a class a warp at a time
    static constexpr int THREADS = WARPS * 32;
    static constexpr int QF = 16 * N;              // floats a class: [N slots][8 frequencies] complex
    static constexpr int R = 4;                    // ring slots of 4 rows of D a warp
    static constexpr int SMEM = CT * QF * 4 + WARPS * R * 4 * N * 4;
    static constexpr int SUPER = 16;               // row and column slots a side of a super-tile
    static constexpr int SUPER_BLOCKS = SUPER * (SUPER / CT);
    static constexpr int GROUPS = THREADS / CT;    // runs loaded at once
    static constexpr int LOADS = 8 * N / GROUPS;   // (row, side, angle) runs a thread
    static_assert(N == 64, "eight rows a lane: 4 rb .. 4 rb + 3 and N/2 + 4 rb ..");
    static_assert(N % GROUPS == 0 && CT % WARPS == 0, "runs and classes");
};

__device__ __forceinline__ void cp_async16(float *dst, const float *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}

// Tile of block b: row slot srow, column slots c0 .. c0 + CT - 1; false for
// the padding blocks of the super-tile grid.
template <int N>
__device__ __forceinline__ bool tile_of_block(const PropArgs &a, long long b, int &srow, int &c0) {
    using C = TileCfg<N>;
    const int n = a.col_slots, nr = row_slots(a.H);
    if (!a.share_t) {
        const int tr = (n + C::CT - 1) / C::CT;
        srow = (int)(b / tr);
        c0 = (int)(b - (long long)srow * tr) * C::CT;
        return srow < nr;
    }
    // super-tiles column by column: (I, J) and (J, I) for I < J, then (J, J);
    // the J^2 super-tiles of columns < J come first
    const long long sg = b / C::SUPER_BLOCKS;
    const int w = (int)(b - sg * C::SUPER_BLOCKS);
    long long J = (long long)sqrt((double)sg);
    while (J * J > sg) --J;
    while ((J + 1) * (J + 1) <= sg) ++J;
    const long long p = sg - J * J;
    long long R = J, Cs = J;
    if (p < 2 * J) {
        if (p & 1) Cs = p >> 1;
        else R = p >> 1;
    }
    srow = (int)(R * C::SUPER) + w / (C::SUPER / C::CT);
    c0 = (int)(Cs * C::SUPER) + (w % (C::SUPER / C::CT)) * C::CT;
    return srow < nr && c0 < n;
}

// blocks of the launch: every tile, or the whole super-tile grid
template <int N>
long long tiled_blocks(const PropArgs &a) {
    using C = TileCfg<N>;
    const long long n = a.col_slots, nr = row_slots(a.H);
    if (!a.share_t) return nr * ((n + C::CT - 1) / C::CT);
    const long long sb = (n + C::SUPER - 1) / C::SUPER;
    return sb * sb * (long long)C::SUPER_BLOCKS;
}

template <int N>
__global__ void __launch_bounds__(TileCfg<N>::THREADS, 2) k_prop_apply_tiled(const __grid_constant__ PropArgs a) {
    using C = TileCfg<N>;
    extern __shared__ __align__(16) float tsm[];
    int srow, c0;
    if (!tile_of_block<N>(a, blockIdx.x, srow, c0)) return;
    const int tid = threadIdx.x, n = a.col_slots;
    int k[4];
    bool kon[4];
    slot_rows(srow, a.H, k, kon);
    // the propagator a class of the tile reads: its own, or its transpose's
    auto built = [&](int q) -> long long {
        const long long sc = c0 + q;
        return a.share_t && srow > sc ? sc * n + srow : (long long)srow * n + sc;
    };
    // into L2 while the vectors come in: 16 threads a class, 8 lines each
    {
        const int q = tid / (C::THREADS / C::CT), t = tid % (C::THREADS / C::CT);
        if (c0 + q < n) {
            const char *Dq = reinterpret_cast<const char *>(a.D + built(q) * (long long)(N * N));
#pragma unroll
            for (int i = 0; i < N * N * 4 / 128 / (C::THREADS / C::CT); ++i)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(Dq + (t + i * (C::THREADS / C::CT)) * 128));
        }
    }
    // Element (slot a, frequency m) of class q: 16-float row a ^ qh ^ (bit 2
    // of a), 16-byte unit ((m ^ qm) >> 1) ^ (bits 3, 4 of a), float pair
    // (m ^ qm) & 1, with qh = bit 3 of q and qm its low three bits. The 16
    // lanes of a run (one slot and m, 16 classes) fall on 16 different pairs
    // of banks, and the eight rows 4 rb + c (rb = 0 .. 7) of one unit that a
    // quarter-warp updates at the end on eight different groups of four.
    // m = 2 (row of the class) + side (0: column l, 1: column W/2 - l).
    const int q = tid % C::CT, g = tid / C::CT;
    const int sc = c0 + q, l = sc, lb = a.W / 2 - sc;
    const bool qlive = sc < n;
    const bool tq = a.share_t && srow > sc;
    const int qh = (q >> 3) & 1, qm = q & 7;
    float *xq = tsm + q * C::QF;
    auto xrow = [](int a, int h) { return a ^ h ^ ((a >> 2) & 1); };
    auto xunit = [](int a, int u) { return u ^ ((a >> 3) & 3); };
    auto xpos = [&](int a, int m, int h, int mm) {
        return xrow(a, h) * 16 + 4 * xunit(a, (m ^ mm) >> 1) + 2 * ((m ^ mm) & 1);
    };
    // run it of this thread: angle r = g + GROUPS (it mod (N / GROUPS)), m = it / (N / GROUPS)
    constexpr int RPM = N / C::GROUPS;
    auto run_ok = [&](int m) { return qlive && kon[m >> 1] && ((m & 1) == 0 || lb != l); };
    auto run_src = [&](int m, int r) -> long long {
        return (long long)r * a.HW + (long long)k[m >> 1] * a.Wc + ((m & 1) ? lb : l);
    };
    auto run_slot = [&](int m, int r) -> int {
        const bool neg = ((m >> 1) >= 2) != tq;
        return ((tq ? a.perm_shift : 0) + (neg ? -r : r)) & (N - 1);
    };
    {
        float2 v[C::LOADS];
#pragma unroll
        for (int it = 0; it < C::LOADS; ++it) {
            const int m = it / RPM, r = g + C::GROUPS * (it % RPM);
            v[it] = run_ok(m) ? a.vol[run_src(m, r)] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int it = 0; it < C::LOADS; ++it) {
            const int m = it / RPM, r = g + C::GROUPS * (it % RPM);
            *reinterpret_cast<float2 *>(xq + xpos(run_slot(m, r), m, qh, qm)) = v[it];
        }
    }
    __syncthreads();
    {
        const int warp = tid >> 5, lane = tid & 31, rb = lane & 7, mp = lane >> 3;
        float *ring = tsm + C::CT * C::QF + warp * (C::R * 4 * N);
#pragma unroll 1
        for (int cq = warp; cq < C::CT; cq += C::WARPS) {
            if (c0 + cq >= n) break;  // warp-uniform
            const int ch = (cq >> 3) & 1, cm = cq & 7;
            float *xc = tsm + cq * C::QF;
            const int uu = mp ^ (cm >> 1);  // the 16-byte unit of frequencies 2 mp, 2 mp + 1
            // rows 4 c .. 4 c + 3 of D (1 KB, contiguous) into ring slot c mod R,
            // 16 bytes a copy, one commit group a chunk (empty past the end)
            const float *Dq = a.D + built(cq) * (long long)(N * N);
            auto issue = [&](int c) {
                if (c < N / 4) {
#pragma unroll
                    for (int p = lane; p < N; p += 32) cp_async16(ring + (c % C::R) * (4 * N) + 4 * p, Dq + c * (4 * N) + 4 * p);
                }
                cp_async_commit();
            };
#pragma unroll
            for (int c = 0; c < C::R - 1; ++c) issue(c);
            // acc[h][p][f]: rows 4 (rb + 8 h) + 2 p, + 1 (a pair); f = the
            // unit's four floats (re, im of its two frequencies)
            f32x2 acc[2][2][4];
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int p = 0; p < 2; ++p)
#pragma unroll
                    for (int f = 0; f < 4; ++f) acc[h][p][f] = pk2(0.f, 0.f);
#pragma unroll 1
            for (int c = 0; c < N / 4; ++c) {
                cp_async_wait<C::R - 2>();  // this lane's copies of chunk c
                __syncwarp();               // everyone's, and chunk c - 1 read by all
                issue(c + C::R - 1);
                const float *dc = ring + (c % C::R) * (4 * N) + 4 * rb;
                // row 4 c + jj of x: 16-float row 4 c + (jj ^ e), e = ch ^ (c & 1)
                const float *xj = xc + 4 * c * 16 + 4 * xunit(4 * c, uu);
                const int ro = (ch ^ (c & 1)) * 16;
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const float4 xv = *reinterpret_cast<const float4 *>(xj + (jj & 2) * 16 + ((jj & 1) ? 16 - ro : ro));
                    const f32x2 xs[4] = {dup2(xv.x), dup2(xv.y), dup2(xv.z), dup2(xv.w)};
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        // column 4 c + jj of rows 4 (rb + 8 h) .. + 3 (D is symmetric)
                        const ulonglong2 dd = *reinterpret_cast<const ulonglong2 *>(dc + jj * N + 32 * h);
#pragma unroll
                        for (int f = 0; f < 4; ++f) {
                            acc[h][0][f] = fma2(dd.x, xs[f], acc[h][0][f]);
                            acc[h][1][f] = fma2(dd.y, xs[f], acc[h][1][f]);
                        }
                    }
                }
            }
            __syncwarp();
            // x <- x + D x on the lane's rows, in place
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int p = 0; p < 2; ++p)
#pragma unroll
                    for (int o = 0; o < 2; ++o) {
                        const int row = 4 * (rb + 8 * h) + 2 * p + o;
                        float4 *px = reinterpret_cast<float4 *>(xc + xrow(row, ch) * 16 + 4 * xunit(row, uu));
                        float4 x = *px;
                        x.x += o ? hi2(acc[h][p][0]) : lo2(acc[h][p][0]);
                        x.y += o ? hi2(acc[h][p][1]) : lo2(acc[h][p][1]);
                        x.z += o ? hi2(acc[h][p][2]) : lo2(acc[h][p][2]);
                        x.w += o ? hi2(acc[h][p][3]) : lo2(acc[h][p][3]);
                        *px = x;
                    }
            __syncwarp();
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < C::LOADS; ++it) {
        const int m = it / RPM, r = g + C::GROUPS * (it % RPM);
        if (run_ok(m))
            a.vol[run_src(m, r)] = *reinterpret_cast<const float2 *>(xq + xpos(run_slot(m, r), m, qh, qm));
    }
}

template <typename C, typename K>
cudaError_t launch_build_kernel(K kernel, const PropArgs &a, int num_sms, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, C::WARPS * 32, C::SMEM);
    if (e != cudaSuccess) return e;
    const long long per_block = (long long)C::WARPS * C::CPW;
    long long blocks = (a.items + per_block - 1) / per_block;
    // every block slot but one on an eighth of the SMs: the build runs on a
    // side stream beside the orientation and the first row pass, whose
    // kernels would otherwise wait for the build's blocks to leave
    const long long cap = (long long)num_sms * (per_sm > 0 ? per_sm : 1) - (per_sm > 1 ? num_sms / 8 : 0);
    if (blocks > cap) blocks = cap;
    kernel<<<(unsigned)blocks, C::WARPS * 32, C::SMEM, s>>>(a);
    return cudaGetLastError();
}

// symmetric products: N = 16, 32 (NE = 30 angles padded to 32) a class on
// 10 or 3 lanes, N = 64 a class on 36 lanes across two warps
template <int N, int NE = N>
cudaError_t launch_build(const PropArgs &a, int num_sms, cudaStream_t s) {
    if constexpr (N == 64)
        return launch_build_wide<N>(a, num_sms, s);
    else
        return launch_build_kernel<SymCfg<N>>(k_prop_build_sym<N, NE>, a, num_sms, s);
}

template <int N>
cudaError_t launch_apply_tiled(const PropArgs &a, cudaStream_t s) {
    using C = TileCfg<N>;
    cudaError_t e = cudaFuncSetAttribute(k_prop_apply_tiled<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    const long long blocks = tiled_blocks<N>(a);
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_prop_apply_tiled<N><<<(unsigned)blocks, C::THREADS, C::SMEM, s>>>(a);
    return cudaGetLastError();
}

template <int N, int NE = N>
cudaError_t launch_apply(const PropArgs &a, int num_sms, cudaStream_t s) {
    using C = ApplyCfg<N>;
    cudaError_t e = cudaFuncSetAttribute(k_prop_apply<N, NE>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    const long long per_block = (long long)C::WARPS * C::CPW;
    long long blocks = (a.classes + per_block - 1) / per_block;
    const long long cap = (long long)num_sms * 64;
    if (blocks > cap) blocks = cap;
    k_prop_apply<N, NE><<<(unsigned)blocks, C::WARPS * 32, C::SMEM, s>>>(a);
    return cudaGetLastError();
}

// Powering programs over two matrices. A state is the pair of exponents
// (p, r) of P and R (r = 0: R empty); an op costs CHAIN_PRODUCT a product
// and 1 a copy, so that the fewest products come first and the fewest copies
// second. The search is A* with the lower bound CHAIN_PRODUCT times the
// doublings from max(p, r) to S (no op more than doubles the largest
// exponent, so the bound never overestimates and never drops by more than
// an op costs), within the cost of binary powering.
constexpr int CHAIN_PRODUCT = 64;

int chain_bound(long long m, int S) {
    int d = 0;
    for (; m < S; m *= 2) ++d;
    return CHAIN_PRODUCT * d;
}

// binary powering, lowest bit first: P runs through D_1, D_2, D_4, ... and R
// collects the set bits
void chain_binary(int S, std::vector<unsigned char> &ops) {
    ops.clear();
    bool have_r = false;
    for (int s = S;;) {
        if (s & 1) {
            ops.push_back(have_r ? PROP_ADD : PROP_COPY);
            have_r = true;
        }
        s >>= 1;
        if (!s) break;
        ops.push_back(PROP_SQ_P);
    }
}

int chain_cost(const std::vector<unsigned char> &ops) {
    int c = 0;
    for (const unsigned char o : ops) c += o == PROP_COPY ? 1 : CHAIN_PRODUCT;
    return c;
}

bool chain_search(int S, int budget, std::vector<unsigned char> &ops, int &in_r) {
    struct Node {
        int g;
        long long pred;
        unsigned char op;
    };
    const long long W = (long long)S + 1;
    std::unordered_map<long long, Node> seen;
    std::vector<std::vector<long long>> bucket(budget + 1);
    auto visit = [&](int p, int r, int g, long long pred, unsigned char op) {
        const int f = g + chain_bound(std::max(p, r), S);
        if (f > budget) return;
        const long long key = p * W + r;
        const auto it = seen.find(key);
        if (it != seen.end() && it->second.g <= g) return;
        seen[key] = Node{g, pred, op};
        bucket[f].push_back(key);
    };
    visit(1, 0, 0, -1, 0);
    for (int f = 0; f <= budget; ++f) {
        for (size_t i = 0; i < bucket[f].size(); ++i) {
            const long long key = bucket[f][i];
            const int p = (int)(key / W), r = (int)(key % W);
            const int g = seen[key].g;
            if (g + chain_bound(std::max(p, r), S) != f) continue;  // reached again at a lower cost
            if (p == S || r == S) {
                in_r = p == S ? 0 : 1;
                ops.clear();
                for (long long k = key; seen[k].pred >= 0; k = seen[k].pred) ops.push_back(seen[k].op);
                std::reverse(ops.begin(), ops.end());
                return true;
            }
            if (2LL * p <= S) visit(2 * p, r, g + CHAIN_PRODUCT, key, PROP_SQ_P);
            if (r > 0 && 2LL * r <= S) visit(2 * r, r, g + CHAIN_PRODUCT, key, PROP_SQ_R);
            if (r > 0 && (long long)p + r <= S) visit(p, p + r, g + CHAIN_PRODUCT, key, PROP_ADD);
            if (r != p) visit(p, p, g + 1, key, PROP_COPY);
        }
    }
    return false;
}

}  // namespace

}  // namespace se2n

se2n_status se2n_prop_chain(int steps, unsigned char *ops, int cap, int *len, int *in_r) {
    if (steps < 1 || !ops || !len || !in_r) return SE2N_EINVAL;
    std::vector<unsigned char> prog, best;
    int r = 1, best_r = 1;
    se2n::chain_binary(steps, prog);
    if (steps <= 4096 && se2n::chain_search(steps, se2n::chain_cost(prog), best, best_r)) {
        prog.swap(best);
        r = best_r;
    }
    if ((int)prog.size() > cap) return SE2N_EINVAL;
    std::copy(prog.begin(), prog.end(), ops);
    *len = (int)prog.size();
    *in_r = r;
    return SE2N_OK;
}

bool se2n_prop_supported(int N) { return N == 16 || N == 30 || N == 32 || N == 64; }

// N = 30 is stored padded to 32 angles (zero rows and columns 30, 31)
int se2n_prop_dim(int N) { return N == 30 ? 32 : N; }

long long se2n_prop_floats(int N, int fmt) {
    const long long n = se2n_prop_dim(N);
    return fmt != PROP_DIAGONALS ? n * n : (n / 2 + 1) * n;
}

int se2n_prop_apply_fmt(int N, bool half) { return half && N == 64 ? PROP_ROWS : PROP_DIAGONALS; }

int se2n_prop_col_slots(int W, bool half) { return half ? W / 4 + 1 : se2n::pair_rows(W); }

long long se2n_prop_classes(int H, int W, bool half) {
    return (long long)se2n::row_slots(H) * se2n_prop_col_slots(W, half);
}

cudaError_t se2n_prop_prepare(int N) {
    switch (N) {
        case 16:
            return cudaFuncSetAttribute(se2n::k_prop_build_sym<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        se2n::SymCfg<16>::SMEM) == cudaSuccess
                       ? cudaFuncSetAttribute(se2n::k_prop_apply<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              se2n::ApplyCfg<16>::SMEM)
                       : cudaGetLastError();
        case 32:
            return cudaFuncSetAttribute(se2n::k_prop_build_sym<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        se2n::SymCfg<32>::SMEM) == cudaSuccess
                       ? cudaFuncSetAttribute(se2n::k_prop_apply<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              se2n::ApplyCfg<32>::SMEM)
                       : cudaGetLastError();
        case 30:
            return cudaFuncSetAttribute(se2n::k_prop_build_sym<32, 30>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        se2n::SymCfg<32>::SMEM) == cudaSuccess
                       ? cudaFuncSetAttribute(se2n::k_prop_apply<32, 30>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              se2n::ApplyCfg<32>::SMEM)
                       : cudaGetLastError();
        case 64:
            return cudaFuncSetAttribute(se2n::k_prop_build_symw<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        se2n::SymWideCfg<64>::SMEM) == cudaSuccess
                           && cudaFuncSetAttribute(se2n::k_prop_apply<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   se2n::ApplyCfg<64>::SMEM) == cudaSuccess
                       ? cudaFuncSetAttribute(se2n::k_prop_apply_tiled<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              se2n::TileCfg<64>::SMEM)
                       : cudaGetLastError();
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t se2n_launch_prop_build(int N, const PropArgs &a, int num_sms, cudaStream_t s) {
    switch (N) {
        case 16: return se2n::launch_build<16>(a, num_sms, s);
        case 32: return se2n::launch_build<32>(a, num_sms, s);
        case 30: return se2n::launch_build<32, 30>(a, num_sms, s);
        case 64: return se2n::launch_build<64>(a, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t se2n_launch_prop_apply(int N, const PropArgs &a, int num_sms, cudaStream_t s) {
    switch (N) {
        case 16: return se2n::launch_apply<16>(a, num_sms, s);
        case 32: return se2n::launch_apply<32>(a, num_sms, s);
        case 30: return se2n::launch_apply<32, 30>(a, num_sms, s);
        case 64:
            return a.rows == PROP_ROWS ? se2n::launch_apply_tiled<64>(a, s) : se2n::launch_apply<64>(a, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}
