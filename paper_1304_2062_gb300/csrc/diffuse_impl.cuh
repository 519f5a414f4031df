// Fused Crank-Nicolson diffusion of the decoupled Mathieu-type systems
// (eq. (4.2), Theorem 2; Crank-Nicolson as recommended in Section 4).
//
// Every DFT coefficient (k,l) of the lifted volume carries an N-vector psi
// with dpsi/dt = A psi, A = -diag(a_r^2) + beta L (L: cyclic second
// difference). One CN step is psi <- psi + dt (I - dt/2 A)^{-1} A psi, i.e.
// the increment is computed and added: slow modes then carry rounding
// relative to their (small) change, and the constant angular mode of the
// zero frequency is preserved exactly.
//
// Scaled form. With c = beta dt / 2 the left matrix divided by c is
//     B = diag(d_r) - (shift + shift^-1),   d_r = 1/c + E_r,   E_r = 2 + a_r^2 / beta,
// and the right-hand side divided by c is y_r = psi_{r-1} + psi_{r+1} - E_r psi_r,
// so the off-diagonals are exactly -1 and every recurrence is one FMA.
// Then psi_new = psi + 2 B^{-1} y.
//
// Work split. P threads (adjacent lanes) share one frequency; each holds
// K = N/P consecutive angles in registers. The cyclic matrix is cut
// ("torn") at Q = max(1, P/2) places into tridiagonal blocks; each block is
// eliminated from both ends at once by a pair of threads (twisted
// elimination, meeting in the middle), or by one thread (P = 1). The tears
// are added back by the Sherman-Morrison-Woodbury identity with tear vectors
//     u = -d_i e_i - e_j,   v = e_i + e_j / d_i
// for the coupled rows i (end of one block) and j (start of the next), which
// keeps the modified pivots 2 d_i and d_j + 1/d_i positive. A thread's local
// index 0 is always its tear row: even parts run upward from the start of
// their block, odd parts downward from its end.
//
// Per step and per real component each angle costs 6 FP32 instructions
// (add, 5 FMA; 7 when Q = 2), plus a few shuffles per thread.
//
// Split diagonal (SPLIT). E_r = 2 + a_r^2/beta held in one FP32 number
// quantises a_r^2/beta to ulp(2) = 2.4e-7, i.e. perturbs the decay rate of
// every mode by up to 1.2e-7 beta per unit time: negligible unless beta * T
// is large (the error grows as 1.2e-7 beta T on modes that survive). The
// SPLIT variant keeps e_r = a_r^2/beta alone and forms
// y_r = (psi_{r-1} + psi_{r+1} - 2 psi_r) - e_r psi_r, one more FMA per angle.
#pragma once

#include "se2n_internal.h"

namespace se2n {

__device__ __forceinline__ float xshfl(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ double xshfl(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }

// sin(2 pi l / W) with the argument reduced exactly in integers, so the
// FP32 sine sees an argument in [0, 1/2] (relative accuracy near Nyquist).
__device__ __forceinline__ float sin_2pi_frac(int l, int W) {
    int m = 2 * l;  // sin(pi m / W), 0 <= m < 2W
    float sgn = 1.0f;
    if (m >= W) { m -= W; sgn = -1.0f; }
    if (2 * m > W) m = W - m;
    return sgn * sinpif((float)m / (float)W);
}

// Butterfly sum over the P lanes of a frequency. Every lane gets the
// bitwise-identical total (each partial sum is formed from the same two
// operands in every lane, and FP addition is commutative).
template <int P, typename T>
__device__ __forceinline__ T group_sum(T v) {
    if constexpr (P >= 2) v += xshfl(v, 1);
    if constexpr (P >= 4) v += xshfl(v, 2);
    return v;
}

// Solve T' x = v for the torn (block-diagonal) matrix, in place: forward
// elimination, the 2x2 meeting of a pair (P >= 2), back substitution.
template <int K, int P, typename T>
__device__ __forceinline__ void torn_solve(T (&v)[K], const T (&G)[K], T M1, T M2) {
#pragma unroll
    for (int j = 1; j < K; ++j) v[j] = fma(G[j - 1], v[j - 1], v[j]);
    T xi;
    if constexpr (P == 1) {
        xi = v[K - 1];
    } else {
        const T q = xshfl(v[K - 1], 1);
        xi = fma(M1, v[K - 1], M2 * q);
    }
    v[K - 1] = G[K - 1] * xi;
#pragma unroll
    for (int j = K - 2; j >= 0; --j) {
        xi = fma(G[j + 1], xi, v[j]);
        v[j] = G[j] * xi;
    }
}

// Pivots of the torn matrix for one thread's rows: diag[0] already carries
// the tear modification. Returns G = 1/pivot and the pair-meeting factors.
template <int K, int P, typename T>
__device__ __forceinline__ void torn_factor(const T (&diag)[K], T (&G)[K], T &M1, T &M2) {
    T piv = diag[0];
    G[0] = T(1) / piv;
#pragma unroll
    for (int j = 1; j < K; ++j) {
        piv = diag[j] - G[j - 1];
        G[j] = T(1) / piv;
    }
    M1 = T(0);
    M2 = T(0);
    if constexpr (P >= 2) {
        const T pq = xshfl(piv, 1);
        const T prod = piv * pq;
        const T D = prod - T(1);
        M1 = prod / D;
        M2 = piv / D;
    }
}

// Tear bookkeeping for part p. Q tears; the part's local row 0 is on tear
// `tear`, on its i side (even p) or j side (odd p). For P == 1 the single
// corner tear has its i row at local 0 and its j row at local K-1.
template <int P>
struct TearInfo {
    static constexpr int Q = (P == 4) ? 2 : 1;
    int p, tear;
    bool iside;
    __device__ __forceinline__ explicit TearInfo(int p_) : p(p_) {
        iside = (p & 1) == 0;
        tear = (P == 4) ? ((p == 0 || p == 3) ? 0 : 1) : 0;
    }
};

// Correction setup in precision T: tear vectors Z = T'^{-1} U (returned
// doubled, for psi += 2 x), and the per-thread coefficients hc[q] such
// that alpha_q = sum over the group of hc[q] * xi(local 0) (+ hc1 * xi(K-1)
// for P == 1) is row q of (I + V^T Z)^{-1} V^T x~.
template <int K, int P, typename T>
__device__ __forceinline__ void tear_setup(const TearInfo<P> &ti, const T (&diag_mod)[K], T d_i, T d0,
                                           float (&Z2)[TearInfo<P>::Q][K], T (&hc)[TearInfo<P>::Q], T &hc1,
                                           T (&Gout)[K], T &M1, T &M2) {
    constexpr int Q = TearInfo<P>::Q;
    torn_factor<K, P, T>(diag_mod, Gout, M1, M2);
    T zl0[Q], zlK[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        T v[K];
#pragma unroll
        for (int j = 0; j < K; ++j) v[j] = T(0);
        if constexpr (P == 1) {
            v[0] = -d0;
            v[K - 1] = T(-1);
        } else if (ti.tear == q) {
            v[0] = ti.iside ? -d0 : T(-1);
        }
        torn_solve<K, P, T>(v, Gout, M1, M2);
#pragma unroll
        for (int j = 0; j < K; ++j) Z2[q][j] = (float)(T(2) * v[j]);
        zl0[q] = v[0];
        zlK[q] = v[K - 1];
    }
    // Capacitance C = I + V^T Z, row q gathered from the rows of tear q.
    const T w = (P == 1 || ti.iside) ? T(1) : T(1) / d_i;
    T C[Q][Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
#pragma unroll
        for (int qq = 0; qq < Q; ++qq) {
            T c;
            if constexpr (P == 1) {
                c = zl0[qq] + zlK[qq] / d0;
            } else {
                c = group_sum<P, T>(ti.tear == q ? w * zl0[qq] : T(0));
            }
            C[q][qq] = (q == qq ? T(1) : T(0)) + c;
        }
    }
    T Hm[Q][Q];
    if constexpr (Q == 1) {
        Hm[0][0] = T(1) / C[0][0];
    } else {
        const T det = C[0][0] * C[1][1] - C[0][1] * C[1][0];
        Hm[0][0] = C[1][1] / det;
        Hm[0][1] = -C[0][1] / det;
        Hm[1][0] = -C[1][0] / det;
        Hm[1][1] = C[0][0] / det;
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) hc[q] = (ti.tear == 0 ? Hm[q][0] : Hm[q][Q - 1]) * w * Gout[0];
    if constexpr (P == 1) {
        hc1 = Hm[0][0] * Gout[K - 1] / d0;
    } else {
        hc1 = T(0);
    }
}

// One frequency group: the P adjacent lanes of this warp integrate all
// steps of frequency fc of the H x W volume vol[N][H][W], loading and
// storing its N-vector. Every lane of the warp must call this together
// (shuffles); a lane with !active works on a valid frequency without storing.
template <int N, int P, bool FP64, bool SPLIT>
__device__ __forceinline__ void diffuse_group(const StepParams &sp, const float *cs, const float *sn,
    float2 *vol, int H, int W, int Wc, long long HW, long long fc, bool active, int k0 = 0) {
    constexpr int K = N / P;
    constexpr int Q = TearInfo<P>::Q;
    static_assert(P == 1 || P == 2 || P == 4, "threads per frequency");
    static_assert(N % P == 0 && K >= 2, "angles per thread");
    static_assert(P < 4 || (N % 4) == 0, "two pairs need N divisible by 4");

    const int lane = threadIdx.x & 31;
    const int p = (P == 1) ? 0 : (lane & (P - 1));
    const TearInfo<P> ti(p);
    constexpr int half = (P == 1) ? N : N / (P / 2);  // rows per tridiagonal block
    const int row0 = (P == 1) ? 0 : (ti.iside ? (p >> 1) * half : (p >> 1) * half + half - 1);
    const int rstep = (P == 1 || ti.iside) ? 1 : -1;

    // fc = k * Wc + l: Wc stored columns (W, or W/2 + 1 for the Hermitian half)
    const int k = (int)(fc / Wc);
    const int l = (int)(fc - (long long)k * Wc);
    const float wx = sin_2pi_frac(l, W);
    const float wy = sin_2pi_frac(k0 + k, H);  // k0: first row of a row shard
    float2 *col = vol + (long long)row0 * HW + fc;
    const long long stride = (long long)rstep * HW;

    float pr[K], pim[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const float2 v = col[j * stride];
        pr[j] = v.x;
        pim[j] = v.y;
    }

    // ---- per-frequency setup (once per launch) ----
    float E[K], dmod[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int r = row0 + rstep * j;
        const float ar = fmaf(wx, cs[r], wy * sn[r]);
        if constexpr (SPLIT) {
            E[j] = ar * ar * sp.inv_beta;
            dmod[j] = (sp.inv_c + 2.0f) + E[j];
        } else {
            E[j] = fmaf(ar * ar, sp.inv_beta, 2.0f);
            dmod[j] = sp.inv_c + E[j];
        }
    }
    const float d_loc0 = dmod[0];
    const float d_part = (P == 1) ? d_loc0 : xshfl(d_loc0, P - 1);  // the i row across my tear
    const float d_i = ti.iside ? d_loc0 : d_part;
    if constexpr (P == 1) {
        dmod[K - 1] = dmod[K - 1] + 1.0f / d_loc0;
        dmod[0] = 2.0f * d_loc0;
    } else if (ti.iside) {
        dmod[0] = 2.0f * d_loc0;
    } else {
        dmod[0] = d_loc0 + 1.0f / d_part;
    }

    float G[K], G2[K], Z2[Q][K], M1, M2;
    float hc[Q] = {}, hc1 = 0.0f;
    double hcd[Q] = {}, hcd1 = 0.0;
    if constexpr (FP64) {
        double dd[K], Gd[K], M1d, M2d;
        const double inv_c = sp.inv_c_d;
        double dE[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int r = row0 + rstep * j;
            const double ar = (double)wx * (double)cs[r] + (double)wy * (double)sn[r];
            dE[j] = 2.0 + ar * ar * sp.inv_beta_d;
            dd[j] = inv_c + dE[j];
        }
        const double dl0 = dd[0];
        const double dpart = (P == 1) ? dl0 : xshfl(dl0, P - 1);
        const double di = ti.iside ? dl0 : dpart;
        if constexpr (P == 1) {
            dd[K - 1] += 1.0 / dl0;
            dd[0] = 2.0 * dl0;
        } else if (ti.iside) {
            dd[0] = 2.0 * dl0;
        } else {
            dd[0] = dl0 + 1.0 / dpart;
        }
        tear_setup<K, P, double>(ti, dd, di, dl0, Z2, hcd, hcd1, Gd, M1d, M2d);
        torn_factor<K, P, float>(dmod, G, M1, M2);
    } else {
        tear_setup<K, P, float>(ti, dmod, d_i, d_loc0, Z2, hc, hc1, G, M1, M2);
    }
#pragma unroll
    for (int j = 0; j < K; ++j) G2[j] = 2.0f * G[j];

    // ---- the fused CN steps ----
#pragma unroll 1
    for (int s = 0; s < sp.steps; ++s) {
        float lr, li, rr, ri;
        if constexpr (P == 1) {
            lr = pr[K - 1]; li = pim[K - 1];
            rr = pr[0]; ri = pim[0];
        } else {
            lr = xshfl(pr[0], P - 1); li = xshfl(pim[0], P - 1);
            rr = xshfl(pr[K - 1], 1); ri = xshfl(pim[K - 1], 1);
        }
        float zr[K], zi[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const float Lr = (j == 0) ? lr : pr[j - 1];
            const float Li = (j == 0) ? li : pim[j - 1];
            const float Rr = (j == K - 1) ? rr : pr[j + 1];
            const float Ri = (j == K - 1) ? ri : pim[j + 1];
            float yr, yi;
            if constexpr (SPLIT) {
                yr = fmaf(-E[j], pr[j], fmaf(-2.0f, pr[j], Lr + Rr));
                yi = fmaf(-E[j], pim[j], fmaf(-2.0f, pim[j], Li + Ri));
            } else {
                yr = fmaf(-E[j], pr[j], Lr + Rr);
                yi = fmaf(-E[j], pim[j], Li + Ri);
            }
            if (j == 0) {
                zr[0] = yr;
                zi[0] = yi;
            } else {
                zr[j] = fmaf(G[j - 1], zr[j - 1], yr);
                zi[j] = fmaf(G[j - 1], zi[j - 1], yi);
            }
        }
        float xr, xi;
        if constexpr (P == 1) {
            xr = zr[K - 1];
            xi = zi[K - 1];
        } else {
            const float qr = xshfl(zr[K - 1], 1), qi = xshfl(zi[K - 1], 1);
            xr = fmaf(M1, zr[K - 1], M2 * qr);
            xi = fmaf(M1, zi[K - 1], M2 * qi);
        }
        const float xlr = xr, xli = xi;
        pr[K - 1] = fmaf(G2[K - 1], xr, pr[K - 1]);
        pim[K - 1] = fmaf(G2[K - 1], xi, pim[K - 1]);
#pragma unroll
        for (int j = K - 2; j >= 0; --j) {
            xr = fmaf(G[j + 1], xr, zr[j]);
            xi = fmaf(G[j + 1], xi, zi[j]);
            pr[j] = fmaf(G2[j], xr, pr[j]);
            pim[j] = fmaf(G2[j], xi, pim[j]);
        }
        float ar[Q], ai[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if constexpr (FP64) {
                double tr, tq;
                if constexpr (P == 1) {
                    tr = hcd[q] * (double)xr + hcd1 * (double)xlr;
                    tq = hcd[q] * (double)xi + hcd1 * (double)xli;
                } else {
                    tr = group_sum<P, double>(hcd[q] * (double)xr);
                    tq = group_sum<P, double>(hcd[q] * (double)xi);
                }
                ar[q] = (float)tr;
                ai[q] = (float)tq;
            } else if constexpr (P == 1) {
                ar[q] = fmaf(hc[q], xr, hc1 * xlr);
                ai[q] = fmaf(hc[q], xi, hc1 * xli);
            } else {
                ar[q] = group_sum<P, float>(hc[q] * xr);
                ai[q] = group_sum<P, float>(hc[q] * xi);
            }
        }
#pragma unroll
        for (int j = 0; j < K; ++j) {
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                pr[j] = fmaf(-ar[q], Z2[q][j], pr[j]);
                pim[j] = fmaf(-ai[q], Z2[q][j], pim[j]);
            }
        }
    }

    if (active) {
#pragma unroll
        for (int j = 0; j < K; ++j) col[j * stride] = make_float2(pr[j], pim[j]);
    }
}

template <int N, int P, bool FP64, bool SPLIT>
__global__ void __launch_bounds__(256) k_diffuse(const __grid_constant__ DiffuseArgs a) {
    const int lane = threadIdx.x & 31;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long slot = tid / P;
    const long long nslots = (long long)gridDim.x * blockDim.x / P;
    const long long warp_slot0 = (tid - lane) / P;
    // The loop bound is uniform across the warp (warp_slot0), so every lane
    // takes part in every shuffle; lanes past the end work on a clamped
    // frequency and do not store.
    for (long long base = 0; warp_slot0 + base < a.HW; base += nslots) {
        const long long f = slot + base;
        const bool active = f < a.HW;
        diffuse_group<N, P, FP64, SPLIT>(a.sp, a.cs, a.sn, a.vol, a.H, a.W, a.Wc, a.HW, active ? f : a.HW - 1,
                                         active, a.k0);
    }
}

}  // namespace se2n

// One instantiation per (N, P, fp64 correction, split diagonal): a table
// entry with the kernel pointer.
#define SE2N_DIFFUSE_ENTRY(N_, P_)                                                  \
    {N_, P_, false, false, (const void *)&se2n::k_diffuse<N_, P_, false, false>},   \
    {N_, P_, true, false, (const void *)&se2n::k_diffuse<N_, P_, true, false>},     \
    {N_, P_, false, true, (const void *)&se2n::k_diffuse<N_, P_, false, true>},     \
    {N_, P_, true, true, (const void *)&se2n::k_diffuse<N_, P_, true, true>}

struct DiffuseEntry {
    int N, P;
    bool fp64, split;
    const void *fn;
};
