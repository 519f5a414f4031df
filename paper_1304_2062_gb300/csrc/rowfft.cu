// The row pass of the Hermitian-half path with propagators: one block a row
// y, all N angles of it in shared memory. Between column passes (colprop.cu)
// the volume is row-transformed, complex [Wc][H][N] (Wc = W/2 + 1); a row
// pass
//   1. reads the row: from the lift (f on the pixel's bin, all bins if
//      flat), from the real volume, or from the row-transformed volume by
//      the inverse real DFT along x;
//   2. optionally applies the static restoration to every pixel (the rule of
//      restore.cuh, with h(t) the maximum over the angles);
//   3. writes the forward real DFT along x back to the row-transformed
//      volume, or the real row, or the projection over the angles (max or
//      mean, with the known pixels reinjected on request), or the image
//      value h = max over the angles and the angle of its first maximum
//      (the input of a growth step of dynamic restoration).
// So the restoration between two intervals (Section 5.2) costs one read and
// one write of the half spectrum, and the lift and the projection none.
//
// Real DFTs of length W by complex DFTs of length W/2 (smem_fft.cuh) on
// z_m = x_2m + i x_2m+1. Forward: E_l = (Z_l + conj Z_{W/2-l}) / 2 and
// O_l = -i (Z_l - conj Z_{W/2-l}) / 2 are the DFTs of the even and odd
// samples, and X_l = E_l + w^l O_l, X_{W/2-l} = conj(E_l - w^l O_l) with
// w = exp(-2 pi i / W). Inverse (unnormalised, as cuFFT's C2R, with the
// imaginary parts of X_0 and X_{W/2} ignored): Z_l = P + i Q and
// Z_{W/2-l} = conj P + i conj Q with P = X_l + conj X_{W/2-l} and
// Q = conj(w^l) (X_l - conj X_{W/2-l}), then z = inverse DFT of Z.
#include "prop_classes.cuh"
#include "restore.cuh"
#include "se2n_internal.h"
#include "smem_fft.cuh"

namespace se2n {

namespace {

// threads a block: 256, and 512 for rows of 768 and 1024 (transforms of
// length 384 and 512), which would otherwise hold too many values a thread
template <int W>
__host__ __device__ constexpr int row_threads() { return W >= 768 ? 512 : 256; }

template <int N, int W>
struct RowCfg {
    static constexpr int WH = W / 2;
    static constexpr int XF = SmemBlock<N, WH>::COMPLEX;
    static constexpr int SMEM = (XF + W + FftTw<WH>::SIZE) * 8;
};

// NE < N: an NE-angle system at the slots of slot_of_angle (prop_classes.cuh);
// the empty slots take no part in the maxima, means and argmaxima and stay zero
template <int N, int W, int NE = N>
__global__ void __launch_bounds__(row_threads<W>()) k_row(const __grid_constant__ RowArgs a) {
    constexpr int WH = W / 2, T = row_threads<W>();
    extern __shared__ __align__(16) float2 rsm[];
    float2 *Z = rsm;                       // [N][W/2]: z_m of every angle
    float2 *tws = rsm + RowCfg<N, W>::XF;  // exp(-2 pi i m / W)
    float2 *twp = tws + W;                 // the transforms' pass tables
    const int tid = threadIdx.x, y = blockIdx.x;
    const long long H = a.H;
    const long long row = (long long)y * W;  // first pixel of the row
    for (int m = tid; m < W; m += T) tws[m] = a.tw[m];
    fft_twiddles<T, WH, 2>(twp, a.tw, tid);  // from the table in device memory
    // 1. the row
    if (a.in_mode == SE2N_ROW_IN_LIFT) {
        for (int m = tid; m < WH; m += T) {
            const float2 fv = reinterpret_cast<const float2 *>(a.f + row)[m];
            const uchar2 mk = reinterpret_cast<const uchar2 *>(a.mask + row)[m];
            const uchar2 bn = reinterpret_cast<const uchar2 *>(a.bins + row)[m];
            const float a0 = mk.x ? fv.x : 0.0f, a1 = mk.y ? fv.y : 0.0f;
            float2 *Zm = Z + xoff<WH>(m);
#pragma unroll 8
            for (int n = 0; n < N; ++n) {
                const int an = angle_of_slot<N, NE>(n);
                const bool on0 = an < NE && ((bn.x == an) || (bn.x == SE2N_BIN_FLAT));
                const bool on1 = an < NE && ((bn.y == an) || (bn.y == SE2N_BIN_FLAT));
                Zm[n * (WH + 1)] = make_float2(on0 ? a0 : 0.0f, on1 ? a1 : 0.0f);
            }
        }
    } else if (a.in_mode == SE2N_ROW_IN_REAL) {
        for (int e = tid; e < N * WH; e += T) {
            const int n = e / WH, m = e - n * WH;
            Z[xsm<WH>(e)] = reinterpret_cast<const float2 *>(a.real_in + (n * H + y) * (W + 2))[m];
        }
    } else {
        // pairs (l, W/2 - l), l = 0 .. W/4: thread tid takes angle tid mod N
        // of pairs tid / N + i T / N (consecutive threads, consecutive angles
        // of one frequency), all its loads issued first
        constexpr int LP = WH / 2 + 1, TL = T / N, IT = (LP + TL - 1) / TL;
        static_assert(T % N == 0, "whole frequencies a block");
        const int n = tid % N, l0 = tid / N;
        float2 xl[IT], xb[IT];
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const int l = l0 + i * TL;
            if (LP % TL == 0 || l < LP) {
                xl[i] = __ldg(a.spec_in + ((long long)l * H + y) * N + n);
                xb[i] = __ldg(a.spec_in + ((long long)(WH - l) * H + y) * N + n);
            }
        }
        __syncthreads();  // twiddles
        float2 *Zn = Z + n * (WH + 1);
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const int l = l0 + i * TL;
            if (LP % TL == 0 || l < LP) {
                if (l == 0) {
                    xl[i].y = 0.0f;
                    xb[i].y = 0.0f;
                }
                const float2 P = cadd(xl[i], cconj(xb[i]));
                const float2 Q = twiddle<1>(csub(xl[i], cconj(xb[i])), tws[l]);
                Zn[xoff<WH>(l)] = make_float2(P.x - Q.y, P.y + Q.x);
                if (l != 0 && 2 * l != WH) Zn[xoff<WH>(WH - l)] = make_float2(P.x + Q.y, Q.x - P.y);
            }
        }
        __syncthreads();
        fft_smem<T, N, WH, 1>(Z, twp, tid);
    }
    __syncthreads();
    // 2. the restoration, one pixel pair (2m, 2m + 1) a thread
    if (a.mix) {
        for (int m = tid; m < WH; m += T) {
            float2 *Zm = Z + xoff<WH>(m);
            float ht0 = -INFINITY, ht1 = -INFINITY;
#pragma unroll 8
            for (int n = 0; n < N; ++n) {
                if (angle_of_slot<N, NE>(n) >= NE) continue;
                const float2 v = Zm[n * (WH + 1)];
                ht0 = fmaxf(ht0, v.x * a.scale);
                ht1 = fmaxf(ht1, v.y * a.scale);
            }
            const float2 fv = reinterpret_cast<const float2 *>(a.f + row)[m];
            const uchar2 mk = reinterpret_cast<const uchar2 *>(a.mask + row)[m];
            const uchar2 bn = reinterpret_cast<const uchar2 *>(a.bins + row)[m];
            const float a0 = mk.x ? fv.x : 0.0f, a1 = mk.y ? fv.y : 0.0f;
            const float h00 = (bn.x == SE2N_BIN_FLAT) ? a0 : fmaxf(a0, 0.0f);
            const float h01 = (bn.y == SE2N_BIN_FLAT) ? a1 : fmaxf(a1, 0.0f);
#pragma unroll 8
            for (int n = 0; n < N; ++n) {
                float2 &v = Zm[n * (WH + 1)];
                const int an = angle_of_slot<N, NE>(n);
                const float l0 = an < NE && ((bn.x == an) || (bn.x == SE2N_BIN_FLAT)) ? a0 : 0.0f;
                const float l1 = an < NE && ((bn.y == an) || (bn.y == SE2N_BIN_FLAT)) ? a1 : 0.0f;
                v = make_float2(sr_value(v.x * a.scale, h00, ht0, l0, mk.x != 0, a.eps, a.guard),
                                sr_value(v.y * a.scale, h01, ht1, l1, mk.y != 0, a.eps, a.guard));
            }
        }
        __syncthreads();
    }
    // 3. the output
    if (a.out_mode == SE2N_ROW_OUT_REAL) {
        for (int e = tid; e < N * WH; e += T) {
            const int n = e / WH, m = e - n * WH;
            reinterpret_cast<float2 *>(a.real_out + (n * H + y) * (W + 2))[m] = Z[xsm<WH>(e)];
        }
    } else if (a.out_mode == SE2N_ROW_OUT_PROJ) {
        for (int m = tid; m < WH; m += T) {
            const float2 *Zm = Z + xoff<WH>(m);
            float a0, a1;
            if (a.proj == SE2N_PROJ_MAX) {
                a0 = -INFINITY;
                a1 = -INFINITY;
#pragma unroll 8
                for (int n = 0; n < N; ++n) {
                    if (angle_of_slot<N, NE>(n) >= NE) continue;
                    const float2 v = Zm[n * (WH + 1)];
                    a0 = fmaxf(a0, v.x * a.scale_proj);
                    a1 = fmaxf(a1, v.y * a.scale_proj);
                }
            } else {
                a0 = 0.0f;
                a1 = 0.0f;
#pragma unroll 8
                for (int n = 0; n < N; ++n) {
                    const float2 v = Zm[n * (WH + 1)];
                    a0 += v.x * a.scale_proj;
                    a1 += v.y * a.scale_proj;
                }
                a0 /= (float)NE;  // the empty slots add zero
                a1 /= (float)NE;
            }
            if (a.reinject) {
                const float2 fv = reinterpret_cast<const float2 *>((a.rf ? a.rf : a.f) + row)[m];
                const uchar2 mk = reinterpret_cast<const uchar2 *>((a.rmask ? a.rmask : a.mask) + row)[m];
                if (mk.x) a0 = fv.x;
                if (mk.y) a1 = fv.y;
            }
            reinterpret_cast<float2 *>(a.proj_out + row)[m] = make_float2(a0, a1);
        }
    } else if (a.out_mode == SE2N_ROW_OUT_H) {
        for (int m = tid; m < WH; m += T) {
            const float2 *Zm = Z + xoff<WH>(m);
            float b0 = -INFINITY, b1 = -INFINITY;
            int r0 = 0, r1 = 0;
#pragma unroll 8
            for (int n = 0; n < N; ++n) {
                const int an = angle_of_slot<N, NE>(n);
                if (an >= NE) continue;
                const float2 v = Zm[n * (WH + 1)];
                const float v0 = v.x * a.scale, v1 = v.y * a.scale;
                // the slots run in angle order: the first maximum is the first angle
                if (v0 > b0) {
                    b0 = v0;
                    r0 = an;
                }
                if (v1 > b1) {
                    b1 = v1;
                    r1 = an;
                }
            }
            reinterpret_cast<float2 *>(a.h_out + row)[m] = make_float2(b0, b1);
            reinterpret_cast<uchar2 *>(a.amax_out + row)[m] = make_uchar2((uint8_t)r0, (uint8_t)r1);
        }
    } else {
        fft_smem<T, N, WH, -1>(Z, twp, tid);
        __syncthreads();
        constexpr int LP = WH / 2 + 1, TL = T / N, IT = (LP + TL - 1) / TL;
        const int n = tid % N, l0 = tid / N;
        const float2 *Zn = Z + n * (WH + 1);
#pragma unroll 4
        for (int i = 0; i < IT; ++i) {
            const int l = l0 + i * TL;
            if (LP % TL == 0 || l < LP) {
                const float2 zl = Zn[xoff<WH>(l)];
                const float2 zc = cconj(Zn[xoff<WH>(l == 0 ? 0 : WH - l)]);
                const float2 s = cadd(zl, zc), d = csub(zl, zc);
                const float2 E = make_float2(0.5f * s.x, 0.5f * s.y);
                const float2 O = make_float2(0.5f * d.y, -0.5f * d.x);  // -i d / 2
                const float2 B = twiddle<-1>(O, tws[l]);
                a.spec_out[((long long)l * H + y) * N + n] = cadd(E, B);
                if (2 * l != WH) a.spec_out[((long long)(WH - l) * H + y) * N + n] = cconj(csub(E, B));
            }
        }
    }
}

template <int N, int W, int NE>
cudaError_t row_attr() {
    return cudaFuncSetAttribute(k_row<N, W, NE>, cudaFuncAttributeMaxDynamicSharedMemorySize, RowCfg<N, W>::SMEM);
}

template <int N, int W, int NE>
cudaError_t row_launch(const RowArgs &a, cudaStream_t s) {
    // the real volume has NE planes, not N slots
    if (NE != N && (a.in_mode == SE2N_ROW_IN_REAL || a.out_mode == SE2N_ROW_OUT_REAL)) return cudaErrorInvalidValue;
    cudaError_t e = row_attr<N, W, NE>();
    if (e != cudaSuccess) return e;
    k_row<N, W, NE><<<a.H, row_threads<W>(), RowCfg<N, W>::SMEM, s>>>(a);
    return cudaGetLastError();
}

template <int N, int NE = N>
cudaError_t row_dispatch(int W, const RowArgs *a, cudaStream_t s) {
    switch (W) {
        case 64: return a ? row_launch<N, 64, NE>(*a, s) : row_attr<N, 64, NE>();
        case 128: return a ? row_launch<N, 128, NE>(*a, s) : row_attr<N, 128, NE>();
        case 256: return a ? row_launch<N, 256, NE>(*a, s) : row_attr<N, 256, NE>();
        case 512: return a ? row_launch<N, 512, NE>(*a, s) : row_attr<N, 512, NE>();
        case 1024: return a ? row_launch<N, 1024, NE>(*a, s) : row_attr<N, 1024, NE>();
        case 384: return a ? row_launch<N, 384, NE>(*a, s) : row_attr<N, 384, NE>();
        case 768: return a ? row_launch<N, 768, NE>(*a, s) : row_attr<N, 768, NE>();
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

}  // namespace se2n

// N = 30: the 30-angle system in 32 slots
bool se2n_row_supported(int N, int W) {
    return (N == 16 || N == 30 || N == 32) &&
           (W == 64 || W == 128 || W == 256 || W == 512 || W == 1024 || W == 384 || W == 768);
}

cudaError_t se2n_row_prepare(int N, int W) {
    if (!se2n_row_supported(N, W)) return cudaErrorInvalidValue;
    return N == 16   ? se2n::row_dispatch<16>(W, nullptr, nullptr)
           : N == 30 ? se2n::row_dispatch<32, 30>(W, nullptr, nullptr)
                     : se2n::row_dispatch<32>(W, nullptr, nullptr);
}

cudaError_t se2n_launch_row(int N, int W, const RowArgs &a, cudaStream_t s) {
    if (!se2n_row_supported(N, W)) return cudaErrorInvalidValue;
    return N == 16 ? se2n::row_dispatch<16>(W, &a, s)
           : N == 30 ? se2n::row_dispatch<32, 30>(W, &a, s)
                     : se2n::row_dispatch<32>(W, &a, s);
}
