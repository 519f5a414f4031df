// 3x3 convolution (padding 1, NHWC bf16) as an implicit GEMM on the
// fifth-generation tensor cores (tcgen05), FP32 accumulation in tensor
// memory:
//
//   D[m][n] = sum_k A(m, k) B(n, k),   m = output pixel, n = output channel,
//   k = tap * C + c (tap = (dy+1)*3 + (dx+1)),
//
// with A gathered from the activations by a loader functor (the same ones as
// the mma.sync path: padding, the nearest-upsampled half of a decoder
// concatenation and the mirrored taps of the data gradient are all in the
// loader) and B a K-major weight matrix.
//
// One CTA of 128 threads computes a 128 x BN tile of D. The K dimension runs
// in blocks of 64 (128 bytes of bf16 per row). For each block all threads
// copy their 16-byte chunks of A and B into a ring of STAGES shared-memory
// stages with cp.async, in the 128-byte-swizzled K-major layout the tensor
// core reads (row r, chunk j at r * 128 + ((j ^ (r & 7)) * 16); 8-row atoms
// of 1024 bytes). Thread 0 issues four tcgen05.mma (M = 128, N = BN, K = 16)
// per block into a BN-column FP32 accumulator in tensor memory, and a
// tcgen05.commit per block arrives on that stage's mbarrier once the tensor
// core has finished reading the stage. A stage is refilled only after that
// arrival; the copies run LAG blocks ahead of the MMAs, so that copies of
// LAG blocks and the MMAs of STAGES - LAG blocks are in flight together.
// The epilogue reads the accumulator with tcgen05.ld (each warp its 32 rows)
// and writes bf16.
//
// Every wait is bounded (2 s): a wait that runs out sets *err; the CTA stops
// copying and issuing, waits (bounded) for the MMAs it has issued, releases
// its tensor memory and returns, and CTAs that start after *err is set
// return at once.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "nn_gemm.cuh"

namespace se2n {
namespace nn {
namespace tc {

constexpr int BM = 128;
constexpr int BKC = 64;          // K elements per block (128 bytes)
constexpr int ROW_BYTES = 128;

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
    return t;
}

// 16-byte global -> shared copy (through L1: the 3x3 taps re-read the same
// input rows), or 16 zero bytes when there is nothing to read.
__device__ __forceinline__ void cp_async16_ca(uint32_t s, const void *gmem) {
    if (gmem)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
    else
        asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};\n" ::"r"(s), "r"(0));
}
__device__ __forceinline__ void cp_async16_cg(uint32_t s, const void *gmem) {
    if (gmem)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
    else
        asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};\n" ::"r"(s), "r"(0));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity), "r"(1000000u)
        : "memory");
    return done != 0;
}

// Wait for the completion of phase `parity`, bounded; false if it ran out
// (kWaitCycles SM cycles, about 2 s at the full clock and longer at lower
// ones) or (abort != null) another thread of the CTA already gave up. Each
// try_wait may suspend the thread in hardware for up to 1 ms, waking at the
// phase completion, so waiting threads do not take issue slots. The fast
// path is a single try_wait.
constexpr long long kWaitCycles = 4000000000LL;
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (abort && *abort) return false;
        if (clock64() - t0 > kWaitCycles) {
            if (abort) *abort = 1;
            return false;
        }
    }
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms
// 1024 bytes apart (stride byte offset); the leading byte offset is unused
// for this layout (set to 16 bytes); descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
template <int N>
__device__ __forceinline__ constexpr uint32_t idesc_bf16_f32() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

template <int BN>
struct Layout {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "tcgen05 M=128 needs N in [16, 256], N % 16 == 0");
    static constexpr int A_BYTES = BM * ROW_BYTES;
    static constexpr int B_BYTES = ((BN + 7) / 8) * 8 * ROW_BYTES;  // whole 8-row atoms
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int TMEM_COLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
};

template <int BN, int STAGES>
constexpr int smem_bytes() {
    return 1024 /* alignment slack */ + STAGES * Layout<BN>::STAGE + 256 /* barriers, tmem slot */;
}

// The 8 A rows a thread copies (rows i * 16 + tid / 8, chunk tid % 8 of
// every K-block), decoded once per tile.
struct RowCache {
    int b[8], y[8], x[8];
};

template <class LA>
__device__ __forceinline__ void decode_rows(const LA &la, int m0, RowCache &rc) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = m0 + i * 16 + (tid >> 3);
        if (m < la.M) {
            la.g.pix(m, rc.b[i], rc.y[i], rc.x[i]);
        } else {
            rc.b[i] = -1;
            rc.y[i] = rc.x[i] = 0;
        }
    }
}

// Copy K-block kb of A (rows m0..m0+127) and B (rows n0..n0+BN-1) into a stage.
template <int BN, class LA, class LB>
__device__ __forceinline__ void load_block(uint32_t sa, uint32_t sb, const LA &la, const LB &lb, const RowCache &rc,
                                           int n0, int kb) {
    const int tid = threadIdx.x;
    const int k0 = kb * BKC;
    // A: consecutive threads take consecutive 16-byte chunks of a row; the
    // chunk's k (hence its tap and channel) is the same for all 8 rows
    {
        const int j = tid & 7;
        const int k = k0 + j * 8;
        const bool kin = k < la.K;
        const int tap = kin ? k / la.C : 0, c = k - tap * la.C;
        int dy = tap / 3 - 1, dx = tap % 3 - 1;
        if (la.flip) {
            dy = -dy;
            dx = -dx;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = i * 16 + (tid >> 3);
            const void *src = nullptr;
            const int yy = rc.y[i] + dy, xx = rc.x[i] + dx;
            if (kin && rc.b[i] >= 0 && yy >= 0 && yy < la.g.H && xx >= 0 && xx < la.g.W)
                src = la.at(rc.b[i], yy, xx, c);
            cp_async16_ca(sa + r * ROW_BYTES + ((j ^ (r & 7)) << 4), src);
        }
    }
#pragma unroll
    for (int i = 0; i < (BN * 8 + 127) / 128; ++i) {
        const int c = i * 128 + tid;
        if (BN * 8 % 128 == 0 || c < BN * 8) {
            const int r = c >> 3, j = c & 7;
            cp_async16_cg(sb + r * ROW_BYTES + ((j ^ (r & 7)) << 4), lb.chunk(n0 + r, k0 + j * 8));
        }
    }
}

// Main loop plus accumulator hand-off. Returns (the same value in every
// thread) false if a wait ran out; the accumulator is then not valid, but
// every MMA that was issued has completed. tmem_base is the allocated column
// base; *issued counts the blocks whose MMAs thread 0 issued.
template <int BN, int STAGES, int LAG, class LA, class LB>
__device__ __forceinline__ bool mainloop(const LA &la, const LB &lb, const RowCache &rc, int n0, int KB,
                                         uint32_t smem_base, uint32_t bars, uint32_t tmem_base, volatile int *abort,
                                         volatile int *issued) {
    using L = Layout<BN>;
    static_assert(LAG >= 1 && LAG <= STAGES - 2, "copies must run ahead without waiting on the newest MMA");
    constexpr uint32_t IDESC = idesc_bf16_f32<BN>();
    bool ok = true;
    // iteration it: copy block it (if any), then issue the MMAs of block it - LAG
    for (int it = 0; it < KB + LAG; ++it) {
        if (it < KB) {
            const int s = it % STAGES;
            if (it >= STAGES) {
                // the MMAs of block it - STAGES read this stage
                const uint32_t parity = (uint32_t)((it / STAGES) - 1) & 1u;
                if (ok && !mbar_wait(bars + 8 * s, parity, abort)) ok = false;
            }
            if (ok)
                load_block<BN>(smem_base + s * L::STAGE, smem_base + s * L::STAGE + L::A_BYTES, la, lb, rc, n0, it);
        }
        asm volatile("cp.async.commit_group;\n" ::);
        const int c = it - LAG;
        if (c >= 0) {
            asm volatile("cp.async.wait_group %0;\n" ::"n"(LAG));
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncthreads();
            if (threadIdx.x == 0 && ok && !*abort) {
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const int s = c % STAGES;
                const uint32_t sa = smem_base + s * L::STAGE, sb = sa + L::A_BYTES;
#pragma unroll
                for (int kk = 0; kk < BKC / 16; ++kk)
                    mma_f16(tmem_base, smem_desc_sw128(sa + kk * 32), smem_desc_sw128(sb + kk * 32), IDESC,
                            (c > 0 || kk > 0) ? 1u : 0u);
                mma_commit(bars + 8 * s);
                *issued = c + 1;
            }
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
    __syncthreads();
    // The newest commit covers every MMA issued before it; wait for it (bounded,
    // even after an abort) so that the tensor memory is idle.
    const int n_issued = *issued;
    if (n_issued > 0) {
        const int last = n_issued - 1;
        if (!mbar_wait(bars + 8 * (last % STAGES), (uint32_t)(last / STAGES) & 1u, nullptr)) *abort = 1;
    }
    if (!ok || n_issued < KB) *abort = 1;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    __syncthreads();
    return *abort == 0;
}

// Kernel scaffold: shared memory carve-up, barrier init, tensor memory
// allocation, main loop, epilogue functor, release.
//   epi(row m, column n0 + j0, float v[16]) writes 16 consecutive outputs.
template <int BN, int STAGES, int LAG, class LA, class LB, class EPI>
__device__ __forceinline__ void conv_tile(const LA &la, const LB &lb, const EPI &epi, int *err) {
    using L = Layout<BN>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t smem_base = (raw + 1023u) & ~1023u;
    const uint32_t bars = smem_base + STAGES * L::STAGE;  // STAGES barriers, 8 bytes each
    const uint32_t tmem_slot = bars + 8 * STAGES;
    volatile int *abort = (volatile int *)(smem_raw + (tmem_slot + 4 - raw));
    volatile int *issued = abort + 1;
    const int warp = threadIdx.x >> 5;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int KB = (la.K + BKC - 1) / BKC;
    const int M = la.M;

    if (threadIdx.x == 0) {
        *abort = *(volatile int *)err;  // an earlier CTA gave up: do nothing
        *issued = 0;
        for (int s = 0; s < STAGES; ++s) mbar_init(bars + 8 * s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (*abort) return;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tmem_slot),
                     "r"((uint32_t)L::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    uint32_t tmem_base;
    asm volatile("ld.shared.u32 %0, [%1];\n" : "=r"(tmem_base) : "r"(tmem_slot));

    RowCache rc;
    decode_rows(la, m0, rc);
    const bool ok = mainloop<BN, STAGES, LAG>(la, lb, rc, n0, KB, smem_base, bars, tmem_base, abort, issued);
    if (!ok) {
        if (threadIdx.x == 0) atomicExch(err, 1);
    } else {
        // warp w owns accumulator rows (tensor-memory lanes) 32w .. 32w + 31
        const int m = m0 + warp * 32 + (threadIdx.x & 31);
        const uint32_t lane_base = tmem_base + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int j0 = 0; j0 < BN; j0 += 16) {
            uint32_t r[16];
            tmem_ld16(lane_base + (uint32_t)j0, r);
            if (m < M) {
                float v[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
                epi(m, n0 + j0, v);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem_base),
                     "r"((uint32_t)L::TMEM_COLS));
    }
}

}  // namespace tc
}  // namespace nn
}  // namespace se2n
