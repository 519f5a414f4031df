// BF16 tensor-core GEMM with FP32 accumulation for the surrogate network's
// 3x3 convolutions, used as an implicit GEMM: the operand tiles are gathered
// from NHWC activations by loader functors, so no im2col buffer exists.
//
//   C[M][N] (+)= sum_k A(m, k) * B(k, n)
//
// A is "K-major" when its 8 consecutive k for one m are contiguous in memory
// (one 16-byte chunk), "M-major" when 8 consecutive m for one k are; the
// same for B with n. Each loader returns the address of the 16-byte chunk
// holding 8 consecutive elements along its contiguous dimension, or null
// for a chunk of zeros (outside the image or the matrix).
//
// CTA tile BM x BN x 32, four warps in a 2 x 2 arrangement, each computing a
// (BM/2) x (BN/2) tile with mma.sync.m16n8k16 (bf16 x bf16 -> f32).
// Global -> shared with cp.async (16 bytes, zero-filled when the loader
// says so), two stages; shared -> registers with ldmatrix (.trans for the
// operand that is not K-major). Rows of shared tiles are padded to 40
// elements (80 bytes) so the 8 rows an ldmatrix phase reads fall in
// distinct bank groups.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace se2n {
namespace nn {

constexpr int kBK = 32;
constexpr int kPad = 40;  // padded row length (elements) of K-major shared tiles

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const uint32_t s = smem_u32(smem);
    const int n = gmem ? 16 : 0;  // src-size 0: fill with zeros, read nothing
    const void *g = gmem ? gmem : smem;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(g), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int NPEND>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(NPEND)); }

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Shared-memory footprint of one stage.
template <int BM, int BN, bool A_KMAJOR, bool B_KMAJOR>
struct Smem {
    // K-major tiles: [rows][kPad]; M/N-major tiles: [kBK][cols + 8]
    static constexpr int A_ELEMS = A_KMAJOR ? BM * kPad : kBK * (BM + 8);
    static constexpr int B_ELEMS = B_KMAJOR ? BN * kPad : kBK * (BN + 8);
    static constexpr int STAGE = A_ELEMS + B_ELEMS;
    static constexpr int BYTES = 2 * STAGE * 2;
};

// Load one stage: every thread moves 16-byte chunks of A and B.
template <int BM, int BN, bool A_KMAJOR, bool B_KMAJOR, class LA, class LB>
__device__ __forceinline__ void load_stage(__nv_bfloat16 *sA, __nv_bfloat16 *sB, const LA &la, const LB &lb, int m0,
                                           int n0, int k0) {
    const int tid = threadIdx.x;
    if constexpr (A_KMAJOR) {
        // BM rows x 4 chunks of 8 k
#pragma unroll
        for (int c = tid; c < BM * 4; c += 128) {
            const int r = c >> 2, kc = (c & 3) * 8;
            cp_async16(sA + r * kPad + kc, la.chunk(m0 + r, k0 + kc));
        }
    } else {
        constexpr int CPR = BM / 8;  // chunks per k row
#pragma unroll
        for (int c = tid; c < kBK * CPR; c += 128) {
            const int kr = c / CPR, mc = (c % CPR) * 8;
            cp_async16(sA + kr * (BM + 8) + mc, la.chunk(k0 + kr, m0 + mc));
        }
    }
    if constexpr (B_KMAJOR) {
#pragma unroll
        for (int c = tid; c < BN * 4; c += 128) {
            const int r = c >> 2, kc = (c & 3) * 8;
            cp_async16(sB + r * kPad + kc, lb.chunk(n0 + r, k0 + kc));
        }
    } else {
        constexpr int CPR = BN / 8;
#pragma unroll
        for (int c = tid; c < kBK * CPR; c += 128) {
            const int kr = c / CPR, nc = (c % CPR) * 8;
            cp_async16(sB + kr * (BN + 8) + nc, lb.chunk(k0 + kr, n0 + nc));
        }
    }
}

// The GEMM main loop over k tiles [kt0, kt1); returns the warp's accumulators
// acc[MI][NI][4] for its (BM/2) x (BN/2) tile.
template <int BM, int BN, bool A_KMAJOR, bool B_KMAJOR, class LA, class LB>
__device__ __forceinline__ void gemm_mainloop(const LA &la, const LB &lb, int m0, int n0, int kt0, int kt1,
                                              __nv_bfloat16 *smem, float (&acc)[BM / 32][BN / 16][4]) {
    using S = Smem<BM, BN, A_KMAJOR, B_KMAJOR>;
    constexpr int MI = BM / 32;  // m16 tiles per warp
    constexpr int NI = BN / 16;  // n8 tiles per warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * (BM / 2), wn = (warp & 1) * (BN / 2);
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < NI; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;
    if (kt1 <= kt0) return;

    load_stage<BM, BN, A_KMAJOR, B_KMAJOR>(smem, smem + S::A_ELEMS, la, lb, m0, n0, kt0 * kBK);
    cp_async_commit();
    for (int kt = kt0; kt < kt1; ++kt) {
        const int cur = (kt - kt0) & 1;
        if (kt + 1 < kt1) {
            __nv_bfloat16 *nxt = smem + (cur ^ 1) * S::STAGE;
            load_stage<BM, BN, A_KMAJOR, B_KMAJOR>(nxt, nxt + S::A_ELEMS, la, lb, m0, n0, (kt + 1) * kBK);
        }
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const __nv_bfloat16 *sA = smem + cur * S::STAGE;
        const __nv_bfloat16 *sB = sA + S::A_ELEMS;
#pragma unroll
        for (int kk = 0; kk < kBK; kk += 16) {
            uint32_t af[MI][4];
#pragma unroll
            for (int i = 0; i < MI; ++i) {
                const int mb = wm + i * 16;
                const int mat = lane >> 3, rin = lane & 7;
                if constexpr (A_KMAJOR) {
                    const int r = mb + (mat & 1) * 8 + rin, c = kk + (mat >> 1) * 8;
                    ldsm_x4(af[i], sA + r * kPad + c);
                } else {
                    const int kr = kk + (mat >> 1) * 8 + rin, c = mb + (mat & 1) * 8;
                    ldsm_x4_t(af[i], sA + kr * (BM + 8) + c);
                }
            }
#pragma unroll
            for (int j = 0; j < NI; j += 2) {
                const int nb = wn + j * 8;
                const int mat = lane >> 3, rin = lane & 7;
                uint32_t bf[4];
                if constexpr (B_KMAJOR) {
                    const int r = nb + (mat >> 1) * 8 + rin, c = kk + (mat & 1) * 8;
                    ldsm_x4(bf, sB + r * kPad + c);
                } else {
                    const int kr = kk + (mat & 1) * 8 + rin, c = nb + (mat >> 1) * 8;
                    ldsm_x4_t(bf, sB + kr * (BN + 8) + c);
                }
#pragma unroll
                for (int i = 0; i < MI; ++i) {
                    mma_bf16(acc[i][j], af[i], bf[0], bf[1]);
                    mma_bf16(acc[i][j + 1], af[i], bf[2], bf[3]);
                }
            }
        }
        __syncthreads();
    }
    cp_async_wait<0>();
}

// Position of accumulator element q of tile (i, j) for this lane.
template <int BM, int BN>
__device__ __forceinline__ void acc_pos(int i, int j, int q, int &m, int &n) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * (BM / 2), wn = (warp & 1) * (BN / 2);
    m = wm + i * 16 + (lane >> 2) + ((q & 2) ? 8 : 0);
    n = wn + j * 8 + (lane & 3) * 2 + (q & 1);
}

}  // namespace nn
}  // namespace se2n
