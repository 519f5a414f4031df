// Batched complex DFTs in shared memory, the building block of the row and
// column passes (rowfft.cu, colprop.cu): N transforms of length L (a power
// of two, 32 .. 512, or 192 or 384) held as a block [N][L], transformed in
// place by mixed-radix Stockham (self-sorting) passes: radix 8 and then one
// pass of radix 2 or 4 where L is not a power of 8, two of radix 16 for 256,
// and a radix-3 pass first for 192 = 3 x 64 and 384 = 3 x 128:
//   pass with radix R over sub-transforms of length NS already done:
//   butterfly j reads elements j + r L / R (r < R), multiplies them by
//   exp(DIR 2 pi i r (j mod NS) / (NS R)), takes the R-point DFT, and writes
//   output r to (j / NS) NS R + (j mod NS) + r NS.
// Unnormalised; DIR = -1 forward, +1 inverse. Every read of a pass precedes
// its first write (a barrier in between), so each thread holds its
// butterflies' inputs in registers.
//
// Layout: element i of transform n at n (L + 1) + (i ^ s(i / 16)), with
// s(m) = (m mod 8) + 8 (bit 2 of m xor bit 3 of m): planes L + 1 apart put
// the N elements of one index on different banks (the per-frequency work
// between the transforms), and the XOR inside each run of 16 keeps the access
// patterns of the passes (consecutive; stride 8; stride 16; runs of 8 that
// are 64 apart) free of bank conflicts.
#pragma once

namespace se2n {

// position of element i inside a plane, and of element e = n L + i of the block
template <int L>
__device__ __forceinline__ int xoff(int i) {
    const int m = i >> 4;
    return i ^ ((m & 7) | (((m << 1) ^ m) & 8));
}
template <int L>
__device__ __forceinline__ int xsm(int e) {
    return (e / L) * (L + 1) + xoff<L>(e % L);
}

template <int N, int L>
struct SmemBlock {
    static constexpr int COMPLEX = N * (L + 1);
};

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
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// z times exp(DIR 2 pi i m / 16) for m = 1, 2, 3, 6, 9 (the inner twiddles of
// the 16-point DFT), from cos(pi / 8), sin(pi / 8) and cos(pi / 4)
template <int DIR, int M>
__device__ __forceinline__ float2 w16(float2 z) {
    constexpr float c8 = 0.92387953251128674f, s8 = 0.38268343236508977f, h = 0.70710678118654752f;
    constexpr float wr = M == 1 ? c8 : M == 2 ? h : M == 3 ? s8 : M == 6 ? -h : -c8;
    constexpr float wi = DIR * (M == 1 ? s8 : M == 2 ? h : M == 3 ? c8 : M == 6 ? h : -s8);
    return make_float2(fmaf(z.x, wr, -z.y * wi), fmaf(z.x, wi, z.y * wr));
}

// V_k = sum_n v_n exp(DIR 2 pi i n k / R), in place, for R = 2, 3, 4, 8, 16.
template <int R, int DIR>
__device__ __forceinline__ void dft_small(float2 (&v)[R]) {
    if constexpr (R == 3) {
        // w = exp(DIR 2 pi i / 3) = -1/2 + DIR i sqrt(3)/2: V_0 = a + (b + c),
        // V_1,2 = a - (b + c)/2 +- DIR i (sqrt(3)/2) (b - c)
        constexpr float h3 = 0.86602540378443865f;  // sqrt(3) / 2
        const float2 a = v[0], t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
        const float2 m = make_float2(fmaf(-0.5f, t1.x, a.x), fmaf(-0.5f, t1.y, a.y));
        const float2 n = DIR < 0 ? make_float2(h3 * t2.y, -h3 * t2.x) : make_float2(-h3 * t2.y, h3 * t2.x);
        v[0] = cadd(a, t1);
        v[1] = cadd(m, n);
        v[2] = csub(m, n);
    } else if constexpr (R == 2) {
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
    } else if constexpr (R == 16) {
        // n = a + 4 m, k = b + 4 c: 4-point DFTs over m, the twiddle
        // exp(DIR 2 pi i a b / 16), 4-point DFTs over a, output b + 4 c
        float2 u[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            float2 t[4] = {v[a], v[a + 4], v[a + 8], v[a + 12]};
            dft_small<4, DIR>(t);
#pragma unroll
            for (int b = 0; b < 4; ++b) u[a][b] = t[b];
        }
        u[1][1] = w16<DIR, 1>(u[1][1]);
        u[1][2] = w16<DIR, 2>(u[1][2]);
        u[1][3] = w16<DIR, 3>(u[1][3]);
        u[2][1] = w16<DIR, 2>(u[2][1]);
        u[2][2] = quarter<DIR>(u[2][2]);
        u[2][3] = w16<DIR, 6>(u[2][3]);
        u[3][1] = w16<DIR, 3>(u[3][1]);
        u[3][2] = w16<DIR, 6>(u[3][2]);
        u[3][3] = w16<DIR, 9>(u[3][3]);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            float2 t[4] = {u[0][b], u[1][b], u[2][b], u[3][b]};
            dft_small<4, DIR>(t);
#pragma unroll
            for (int c = 0; c < 4; ++c) v[b + 4 * c] = t[c];
        }
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

// One pass of T threads over the block X; twp[r NS + k] = exp(-2 pi i r k /
// (NS R)), this pass's twiddles (fft_twiddles below), read at consecutive
// entries by the lanes of consecutive k (free of bank conflicts).
template <int T, int N, int L, int R, int NS, int DIR>
__device__ __forceinline__ void fft_pass(float2 *X, const float2 *twp, int tid) {
    constexpr int M = L / R;  // butterflies a transform
    constexpr int NB = N * M;
    constexpr int BPT = (NB + T - 1) / T;
    // butterfly b = tid + q T: transform b / M, index j = b mod M. Where T is
    // a multiple of M, j = tid mod M for every q, so the positions and the
    // twiddles are formed once; otherwise (radix-3 lengths) once a butterfly.
    constexpr bool UNIFORM = T % M == 0;
    int ro[UNIFORM ? R : 1], wo[UNIFORM ? R : 1];
    float2 w[UNIFORM ? R : 1];
    if constexpr (UNIFORM) {
        const int j = tid % M, k = j % NS;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            ro[r] = xoff<L>(j + r * M);
            wo[r] = xoff<L>((j - k) * R + k + r * NS);
        }
    }
    float2 v[BPT][R];
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
        const int b = tid + q * T;
        if (NB % T == 0 || b < NB) {
            const float2 *Xn = X + (b / M) * (L + 1);
            const int j = b % M;
#pragma unroll
            for (int r = 0; r < R; ++r) v[q][r] = Xn[UNIFORM ? ro[r] : xoff<L>(j + r * M)];
        }
    }
    if constexpr (UNIFORM && NS > 1) {
        const int k = (tid % M) % NS;
#pragma unroll
        for (int r = 1; r < R; ++r) w[r] = twp[r * NS + k];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
        const int b = tid + q * T;
        if (NB % T == 0 || b < NB) {
            const int j = b % M, k = j % NS;
            if constexpr (NS > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) v[q][r] = twiddle<DIR>(v[q][r], UNIFORM ? w[r] : twp[r * NS + k]);
            }
            dft_small<R, DIR>(v[q]);
            float2 *Xn = X + (b / M) * (L + 1);
#pragma unroll
            for (int r = 0; r < R; ++r) Xn[UNIFORM ? wo[r] : xoff<L>((j - k) * R + k + r * NS)] = v[q][r];
        }
    }
}

// The passes with twiddles (NS > 1) of the DFTs of length L, and their
// tables: pass (R, NS) needs exp(-2 pi i r k / (NS R)) for r < R, k < NS,
// kept at twp[offset + r NS + k]. Lengths 32 = 8 x 4, 64 = 8 x 8,
// 128 = 8 x 8 x 2, 256 = 16 x 16, 512 = 8 x 8 x 8, 192 = 3 x 8 x 8,
// 384 = 3 x 8 x 8 x 2: up to three passes after the first (NS = 1).
template <int L>
struct FftTw {
    static constexpr bool TRI = L == 192 || L == 384;
    // (R, NS) of the second, third and fourth pass (R = 0 where there is none)
    static constexpr int R2 = L == 32 ? 4 : (L == 256 ? 16 : 8);
    static constexpr int NS2 = TRI ? 3 : (L == 256 ? 16 : 8);
    static constexpr int R3 = TRI ? 8 : (L == 128 ? 2 : (L == 512 ? 8 : 0));
    static constexpr int NS3 = TRI ? 24 : 64;
    static constexpr int R4 = L == 384 ? 2 : 0;
    static constexpr int NS4 = 192;
    static constexpr int OFF3 = R2 * NS2;
    static constexpr int OFF4 = OFF3 + R3 * NS3;
    static constexpr int SIZE = OFF4 + R4 * NS4;  // complex entries
};

// Fill the pass tables from tw[m TS] = exp(-2 pi i m / L) (a table of L TS
// entries); T threads. The caller synchronises after.
template <int T, int L, int TS>
__device__ __forceinline__ void fft_twiddles(float2 *twp, const float2 *tw, int tid) {
    using F = FftTw<L>;
    for (int e = tid; e < F::SIZE; e += T) {
        int r, k, step;
        if (e < F::OFF3) {
            r = e / F::NS2;
            k = e - r * F::NS2;
            step = L / (F::NS2 * F::R2);
        } else if (e < F::OFF4) {
            r = (e - F::OFF3) / F::NS3;
            k = (e - F::OFF3) - r * F::NS3;
            step = F::R3 ? L / (F::NS3 * F::R3) : 0;
        } else {
            r = (e - F::OFF4) / F::NS4;
            k = (e - F::OFF4) - r * F::NS4;
            step = F::R4 ? L / (F::NS4 * F::R4) : 0;
        }
        twp[e] = tw[r * k * step * TS];
    }
}

// The N DFTs of length L. twp: the pass tables of fft_twiddles. The caller
// synchronises before and after.
template <int T, int N, int L, int DIR>
__device__ __forceinline__ void fft_smem(float2 *X, const float2 *twp, int tid) {
    static_assert(L == 32 || L == 64 || L == 128 || L == 256 || L == 512 || L == 192 || L == 384,
                  "transform length");
    using F = FftTw<L>;
    if constexpr (L == 256) {
        fft_pass<T, N, L, 16, 1, DIR>(X, twp, tid);
        __syncthreads();
        fft_pass<T, N, L, 16, 16, DIR>(X, twp, tid);
        return;
    }
    if constexpr (F::TRI) {
        fft_pass<T, N, L, 3, 1, DIR>(X, twp, tid);
        __syncthreads();
        fft_pass<T, N, L, 8, 3, DIR>(X, twp, tid);
        __syncthreads();
        fft_pass<T, N, L, 8, 24, DIR>(X, twp + F::OFF3, tid);
        if constexpr (L == 384) {
            __syncthreads();
            fft_pass<T, N, L, 2, 192, DIR>(X, twp + F::OFF4, tid);
        }
        return;
    }
    fft_pass<T, N, L, 8, 1, DIR>(X, twp, tid);
    __syncthreads();
    if constexpr (L == 32) {
        fft_pass<T, N, L, 4, 8, DIR>(X, twp, tid);
    } else if constexpr (L == 64) {
        fft_pass<T, N, L, 8, 8, DIR>(X, twp, tid);
    } else {
        fft_pass<T, N, L, 8, 8, DIR>(X, twp, tid);
        __syncthreads();
        fft_pass<T, N, L, L / 64, 64, DIR>(X, twp + F::OFF3, tid);
    }
}

}  // namespace se2n
