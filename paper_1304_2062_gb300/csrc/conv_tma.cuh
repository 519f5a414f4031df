// 3x3 convolution (padding 1, NHWC bf16) as a persistent, warp-specialised
// implicit GEMM on the tcgen05 tensor cores with TMA operand loads:
//
//   D[m][n] = sum_k A(m, k) B(n, k),  m = output pixel, n = output channel,
//   k = tap * C + c,  A(m, tap * C + c) = In[pixel m shifted by tap][c],
//   B = a K-major [N][9 C] weight matrix.
//
// Tiles of D are 128 pixels (a bw x bh rectangle of one image, bw * bh = 128)
// by BN channels. The K loop runs over (tap, CK-channel chunk) blocks; for
// each block one TMA box load brings the tile's 128 pixels shifted by the
// tap (the tensor map's out-of-bounds zero fill is the convolution's
// padding) and one brings the matching BN x CK weights, both in the
// swizzled K-major layout the tensor core reads (CK = 64: 128-byte swizzle;
// CK = 32: 64-byte swizzle).
//
// Roles (192 threads, one CTA per SM, tiles strided over CTAs):
//   warp 0, one thread   TMA producer: fills a ring of STAGES stages, each
//                        guarded by a "full" (transaction bytes) and an
//                        "empty" (tensor core done) mbarrier;
//   warp 1               allocates 2 x BN tensor-memory columns; one thread
//                        issues tcgen05.mma (M = 128, N = BN, K = 16) into
//                        one of two accumulators and commits to "empty" per
//                        stage and to "acc full" per tile;
//   warps 2-5            epilogue: tcgen05.ld of the accumulator rows their
//                        lane quarter may access, then the functor EPI, then
//                        "acc empty", so the next tile's MMAs overlap it.
//
// Every wait is bounded (about 2 s at the full clock). One that runs out sets *err and the
// shared abort flag; the CTA then stops, lets what it issued complete
// (bounded), releases its tensor memory and returns. CTAs that find *err
// set do nothing.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "conv_tc.cuh"

namespace se2n {
namespace nn {
namespace tma {

// Geometry of one convolution launch (passed by value).
struct ConvGeo {
    int B, H, W, C;      // A tensor: B images of H x W pixels, C channels
    int bw, bh;          // tile shape in pixels (bw * bh == 128)
    int tiles_x, tiles_y, mtiles, ntiles, tiles;
    int nchunk;          // C / CK
    int KB;              // 9 * nchunk
    int flip;            // 1: taps mirrored (data gradient)
};

template <int BN, int CK>
struct Cfg {
    static_assert(CK == 32 || CK == 64, "channel chunk of 32 (64-byte swizzle) or 64 (128-byte swizzle)");
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "tcgen05 M=128 needs N in [16, 256], N % 16 == 0");
    static constexpr int A_BYTES = 128 * CK * 2;
    static constexpr int B_BYTES = BN * CK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int STAGES = (196608 / STAGE) > 12 ? 12 : (196608 / STAGE);
    // two accumulators, each at a power-of-two column offset
    static constexpr int ACC_COLS = BN <= 16 ? 16 : BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
    static constexpr int TMEM_COLS = 2 * ACC_COLS < 32 ? 32 : 2 * ACC_COLS;
    static constexpr int SMEM = 1024 + STAGES * STAGE + 256;
    static constexpr uint32_t SBO = 8 * CK * 2;              // 8-row atom
    static constexpr uint64_t LAYOUT = CK == 64 ? 2 : 4;     // SWIZZLE_128B / SWIZZLE_64B
};

template <int BN, int CK>
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    using C = Cfg<BN, CK>;
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(C::SBO >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= C::LAYOUT << 61;
    return d;
}

__device__ __forceinline__ void arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];\n" ::"r"(dst),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tile_origin(const ConvGeo &g, int t, int &b, int &x0, int &y0, int &nt) {
    const int mt = t % g.mtiles;
    nt = t / g.mtiles;
    const int per_img = g.tiles_x * g.tiles_y;
    b = mt / per_img;
    const int r = mt - b * per_img;
    y0 = (r / g.tiles_x) * g.bh;
    x0 = (r % g.tiles_x) * g.bw;
}

// EPI provides
//   SMEM_FLOATS, prepare(sm, i, n)    constants copied to shared memory by the
//                                      epilogue threads i = 0..n-1 once per CTA
//   store(m, n, v[16], float &state, sm)  the 16 outputs of pixel m, columns n..n+15
//   finish(m, float state, sm)        after the last column group of pixel m
template <int BN, int CK, class EPI>
__global__ void __launch_bounds__(192, 1)
    k_conv_tma(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, const ConvGeo g,
               const EPI epi, int *err) {
    using Cf = Cfg<BN, CK>;
    constexpr int S = Cf::STAGES;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t bar_full = base + S * Cf::STAGE;
    const uint32_t bar_empty = bar_full + 8 * S;
    const uint32_t bar_afull = bar_empty + 8 * S;   // 2
    const uint32_t bar_aempty = bar_afull + 16;     // 2
    const uint32_t tmem_slot = bar_aempty + 16;
    volatile int *abort = (volatile int *)(smem_raw + (tmem_slot + 4 - raw));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        *abort = *(volatile int *)err;
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(bar_full + 8 * s, 1);
            tc::mbar_init(bar_empty + 8 * s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(bar_afull + 8 * a, 1);
            tc::mbar_init(bar_aempty + 8 * a, 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"((uint64_t)&mapA) : "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"((uint64_t)&mapB) : "memory");
    }
    __syncthreads();
    if (*abort) return;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tmem_slot),
                     "r"((uint32_t)Cf::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    uint32_t tmem_base;
    asm volatile("ld.shared.u32 %0, [%1];\n" : "=r"(tmem_base) : "r"(tmem_slot));

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int s = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < g.tiles && ok; t += gridDim.x) {
                int b, x0, y0, nt;
                tile_origin(g, t, b, x0, y0, nt);
                for (int kb = 0; kb < g.KB; ++kb) {
                    const int tap = kb / g.nchunk, ch = kb - tap * g.nchunk;
                    int dy = tap / 3 - 1, dx = tap % 3 - 1;
                    if (g.flip) {
                        dy = -dy;
                        dx = -dx;
                    }
                    if (!tc::mbar_wait(bar_empty + 8 * s, ph ^ 1u, abort)) {
                        ok = false;
                        break;
                    }
                    const uint32_t sa = base + s * Cf::STAGE, sb = sa + Cf::A_BYTES;
                    arrive_expect_tx(bar_full + 8 * s, Cf::STAGE);
                    tma_load_4d(sa, &mapA, ch * CK, x0 + dx, y0 + dy, b, bar_full + 8 * s);
                    tma_load_2d(sb, &mapB, tap * g.C + ch * CK, nt * BN, bar_full + 8 * s);
                    if (++s == S) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            if (!ok) {
                // loads already issued finish on their own within microseconds
                const long long t0 = clock64();
                while (clock64() - t0 < 200000LL) {
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            constexpr uint32_t IDESC = tc::idesc_bf16_f32<BN>();
            const uint64_t base_desc = sdesc<BN, CK>(base);
            int s = 0, acc = 0;
            uint32_t ph = 0, aph = 0;
            bool ok = true;
            uint32_t last_bar = 0, last_par = 0;
            for (int t = blockIdx.x; t < g.tiles && ok; t += gridDim.x) {
                if (!tc::mbar_wait(bar_aempty + 8 * acc, aph ^ 1u, abort)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t d = tmem_base + (uint32_t)(acc * Cf::ACC_COLS);
                for (int kb = 0; kb < g.KB; ++kb) {
                    if (!tc::mbar_wait(bar_full + 8 * s, ph, abort)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const uint32_t sa = base + s * Cf::STAGE, sb = sa + Cf::A_BYTES;
                    const uint64_t da = base_desc + ((sa - base) >> 4), db = base_desc + ((sb - base) >> 4);
#pragma unroll
                    for (int kk = 0; kk < CK / 16; ++kk)
                        tc::mma_f16(d, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), IDESC, (kb > 0 || kk > 0) ? 1u : 0u);
                    tc::mma_commit(bar_empty + 8 * s);
                    last_bar = bar_empty + 8 * s;
                    last_par = ph;
                    if (++s == S) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (!ok) break;
                tc::mma_commit(bar_afull + 8 * acc);
                if (++acc == 2) {
                    acc = 0;
                    aph ^= 1u;
                }
            }
            if (!ok && last_bar) tc::mbar_wait(last_bar, last_par, nullptr);  // tensor core idle before release
        }
    } else {
        // ---------------- epilogue (warps 2..5) ----------------
        __shared__ float epi_const[EPI::SMEM_FLOATS];
        epi.prepare(epi_const, threadIdx.x - 64, 128);
        asm volatile("bar.sync 1, 128;\n" ::: "memory");  // the four epilogue warps only
        const int q = warp & 3;  // lane quarter this warp may read
        int acc = 0;
        uint32_t aph = 0;
        for (int t = blockIdx.x; t < g.tiles; t += gridDim.x) {
            if (!tc::mbar_wait(bar_afull + 8 * acc, aph, abort)) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            int b, x0, y0, nt;
            tile_origin(g, t, b, x0, y0, nt);
            const int r = q * 32 + lane;
            const int y = y0 + r / g.bw, x = x0 + r % g.bw;
            const int m = (b * g.H + y) * g.W + x;
            const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * Cf::ACC_COLS);
            float state = 0.0f;
#pragma unroll 1
            for (int j0 = 0; j0 < BN; j0 += 16) {
                uint32_t v[16];
                tc::tmem_ld16(taddr + (uint32_t)j0, v);
                float f[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) f[i] = __uint_as_float(v[i]);
                epi.store(m, nt * BN + j0, f, state, epi_const);
            }
            epi.finish(m, state, epi_const);
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) arrive(bar_aempty + 8 * acc);
            if (++acc == 2) {
                acc = 0;
                aph ^= 1u;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && *abort) atomicExch(err, 1);
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem_base),
                     "r"((uint32_t)Cf::TMEM_COLS));
    }
}


// ---------------------------------------------------------------------------
// Narrow layers (BN <= 64): halo boxes and resident weights.
//
// Tiles are 16 x 8 pixels. For each channel block and each horizontal
// offset sx in {-1, 0, 1} one TMA box brings the 16 x 10 pixels (rows
// y0 - 1 .. y0 + 8) shifted by sx; the three vertical offsets sy are the
// same box read from row (sy + 1) * 16, a whole number of swizzle atoms, so
// one box feeds three taps (160 box rows instead of 3 x 128). All weights of
// the layer (9 C x BN) are loaded into shared memory once per CTA, so the
// K loop moves no weight rows at all.
// ---------------------------------------------------------------------------

constexpr int HBW = 16, HBH = 8;             // tile 16 x 8 pixels
constexpr int HROWS = HBW * (HBH + 2);        // 160 box rows

template <int BN, int CK>
struct HaloCfg {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 128, "narrow layers");
    static constexpr int A_BYTES = HROWS * CK * 2;
    static constexpr int BBLK = BN * CK * 2;   // one (tap, channel block) of weights
    static constexpr int ACC_COLS = BN <= 32 ? 32 : BN <= 64 ? 64 : 128;
    static constexpr int TMEM_COLS = 2 * ACC_COLS;
    static constexpr int SMEM_BUDGET = 196608;
};

template <int BN, int CK, class EPI>
__global__ void __launch_bounds__(192, 1)
    k_conv_halo(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, const ConvGeo g,
                const EPI epi, int S, int *err) {
    using Cf = HaloCfg<BN, CK>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const int nblk = 9 * g.nchunk;                       // resident weight blocks
    const uint32_t wres = base;                          // nblk x BBLK
    const uint32_t stages = wres + nblk * Cf::BBLK;      // S x A_BYTES
    const uint32_t bar_w = stages + S * Cf::A_BYTES;
    const uint32_t bar_full = bar_w + 8;
    const uint32_t bar_empty = bar_full + 8 * S;
    const uint32_t bar_afull = bar_empty + 8 * S;
    const uint32_t bar_aempty = bar_afull + 16;
    const uint32_t tmem_slot = bar_aempty + 16;
    volatile int *abort = (volatile int *)(smem_raw + (tmem_slot + 4 - raw));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tiles t = nt * mtiles + mt; CTA c takes n tile c % ntiles and every
    // (gridDim.x / ntiles)-th m tile from c / ntiles (gridDim.x % ntiles == 0)
    const int first_tile = (blockIdx.x % g.ntiles) * g.mtiles + blockIdx.x / g.ntiles;
    const int end_tile = (blockIdx.x % g.ntiles + 1) * g.mtiles;
    const int tile_step = gridDim.x / g.ntiles;

    if (threadIdx.x == 0) {
        *abort = *(volatile int *)err;
        tc::mbar_init(bar_w, 1);
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(bar_full + 8 * s, 1);
            tc::mbar_init(bar_empty + 8 * s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(bar_afull + 8 * a, 1);
            tc::mbar_init(bar_aempty + 8 * a, 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"((uint64_t)&mapA) : "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"((uint64_t)&mapB) : "memory");
    }
    __syncthreads();
    if (*abort) return;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tmem_slot),
                     "r"((uint32_t)Cf::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    uint32_t tmem_base;
    asm volatile("ld.shared.u32 %0, [%1];\n" : "=r"(tmem_base) : "r"(tmem_slot));

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            // this CTA's tiles all have the n tile blockIdx.x % ntiles: its weights stay resident
            const int nt0 = blockIdx.x % g.ntiles;
            arrive_expect_tx(bar_w, (uint32_t)(nblk * Cf::BBLK));
            for (int tap = 0; tap < 9; ++tap)
                for (int ch = 0; ch < g.nchunk; ++ch)
                    tma_load_2d(wres + (tap * g.nchunk + ch) * Cf::BBLK, &mapB, tap * g.C + ch * CK, nt0 * BN, bar_w);
            int s = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int t = first_tile; t < end_tile && ok; t += tile_step) {
                int b, x0, y0, nt;
                tile_origin(g, t, b, x0, y0, nt);
                for (int ch = 0; ch < g.nchunk && ok; ++ch)
                    for (int sxi = 0; sxi < 3; ++sxi) {
                        if (!tc::mbar_wait(bar_empty + 8 * s, ph ^ 1u, abort)) {
                            ok = false;
                            break;
                        }
                        arrive_expect_tx(bar_full + 8 * s, Cf::A_BYTES);
                        tma_load_4d(stages + s * Cf::A_BYTES, &mapA, ch * CK, x0 + sxi - 1, y0 - 1, b,
                                    bar_full + 8 * s);
                        if (++s == S) {
                            s = 0;
                            ph ^= 1u;
                        }
                    }
            }
            if (!ok) {
                const long long t0 = clock64();
                while (clock64() - t0 < 200000LL) {
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            constexpr uint32_t IDESC = tc::idesc_bf16_f32<BN>();
            const uint64_t a_desc0 = sdesc<BN, CK>(stages), w_desc0 = sdesc<BN, CK>(wres);
            int s = 0, acc = 0;
            uint32_t ph = 0, aph = 0;
            bool ok = tc::mbar_wait(bar_w, 0, abort);
            uint32_t last_bar = 0, last_par = 0;
            for (int t = first_tile; t < end_tile && ok; t += tile_step) {
                if (!tc::mbar_wait(bar_aempty + 8 * acc, aph ^ 1u, abort)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t d = tmem_base + (uint32_t)(acc * Cf::ACC_COLS);
                bool first = true;
                for (int ch = 0; ch < g.nchunk && ok; ++ch)
                    for (int sxi = 0; sxi < 3; ++sxi) {
                        if (!tc::mbar_wait(bar_full + 8 * s, ph, abort)) {
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                        const uint32_t sa = stages + s * Cf::A_BYTES;
#pragma unroll
                        for (int syi = 0; syi < 3; ++syi) {
                            // source offset (sy, sx) = (syi - 1, sxi - 1); the weight tap reads it
                            const int tap = g.flip ? (2 - syi) * 3 + (2 - sxi) : syi * 3 + sxi;
                            // descriptors = the base descriptors plus the offset in 16-byte units
                            const uint64_t da = a_desc0 + ((sa - stages + syi * HBW * CK * 2) >> 4);
                            const uint64_t dw = w_desc0 + (((tap * g.nchunk + ch) * Cf::BBLK) >> 4);
#pragma unroll
                            for (int kk = 0; kk < CK / 16; ++kk) {
                                tc::mma_f16(d, da + (uint64_t)(kk * 2), dw + (uint64_t)(kk * 2), IDESC,
                                            first ? 0u : 1u);
                                first = false;
                            }
                        }
                        tc::mma_commit(bar_empty + 8 * s);
                        last_bar = bar_empty + 8 * s;
                        last_par = ph;
                        if (++s == S) {
                            s = 0;
                            ph ^= 1u;
                        }
                    }
                if (!ok) break;
                tc::mma_commit(bar_afull + 8 * acc);
                if (++acc == 2) {
                    acc = 0;
                    aph ^= 1u;
                }
            }
            if (!ok && last_bar) tc::mbar_wait(last_bar, last_par, nullptr);
        }
    } else {
        // ---------------- epilogue (warps 2..5) ----------------
        __shared__ float epi_const[EPI::SMEM_FLOATS];
        epi.prepare(epi_const, threadIdx.x - 64, 128);
        asm volatile("bar.sync 1, 128;\n" ::: "memory");  // the four epilogue warps only
        const int q = warp & 3;
        int acc = 0;
        uint32_t aph = 0;
        for (int t = first_tile; t < end_tile; t += tile_step) {
            if (!tc::mbar_wait(bar_afull + 8 * acc, aph, abort)) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            int b, x0, y0, nt;
            tile_origin(g, t, b, x0, y0, nt);
            const int r = q * 32 + lane;
            const int y = y0 + r / HBW, x = x0 + r % HBW;
            const int m = (b * g.H + y) * g.W + x;
            const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * Cf::ACC_COLS);
            float state = 0.0f;
#pragma unroll 1
            for (int j0 = 0; j0 < BN; j0 += 16) {
                uint32_t v[16];
                tc::tmem_ld16(taddr + (uint32_t)j0, v);
                float f[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) f[i] = __uint_as_float(v[i]);
                epi.store(m, nt * BN + j0, f, state, epi_const);
            }
            epi.finish(m, state, epi_const);
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) arrive(bar_aempty + 8 * acc);
            if (++acc == 2) {
                acc = 0;
                aph ^= 1u;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && *abort) atomicExch(err, 1);
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem_base),
                     "r"((uint32_t)Cf::TMEM_COLS));
    }
}


// ---------------------------------------------------------------------------
// Weight gradient: dW[co][tap * C + ci] += sum over pixels p of
// In[p shifted by tap][ci] * gz[p][co], as D[m][n] with m = tap * C + ci
// (rows, M = 128 per tile), n = co (N = Cout), K = pixels. Both operands come
// from NHWC tensors, so they are MN-major in shared memory: a TMA box of MG
// channels x BKX pixels of one image row lands as BKX rows (one per pixel,
// the K index) of MG contiguous channels, the MN-major swizzled layout
// (MG = 64: 128-byte rows and swizzle; MG = 32: 64-byte). The tap shift
// moves the pixel coordinates, never the innermost (channel) one; rows of
// the M tile past 9 C are zero-filled by a box that starts out of range.
// A unit of work is (M tile, a range of pixel blocks); its partial D is
// added to dW with FP32 atomics by the epilogue, which overlaps the next
// unit's MMAs (two accumulators).
// ---------------------------------------------------------------------------

struct WgradGeo {
    int B, H, W, C, Cout;
    int bkx;            // pixels per K block (one image row segment), 16 / 32 / 64
    int xblocks;        // W / bkx
    int kblocks;        // B * H * xblocks
    int mtiles;         // ceil(9 C / 128)
    int ksplit;         // pixel ranges per M tile
    int units;          // mtiles * ksplit
};

template <int MG, int NG>
struct WgCfg {
    static_assert((MG == 32 || MG == 64) && (NG == 32 || NG == 64), "32- or 64-channel groups");
    static constexpr uint64_t LAYOUT_A = MG == 64 ? 2 : 4, LAYOUT_B = NG == 64 ? 2 : 4;
    static constexpr uint32_t SBO_A = 8 * MG * 2, SBO_B = 8 * NG * 2;
};

// MN-major matrix descriptor: leading byte offset = stride between MN groups,
// stride byte offset = stride between 8-row groups along K.
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint64_t layout) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= layout << 61;
    return d;
}

// kind::f16, D FP32, A and B BF16, both MN-major.
template <int N>
__device__ __forceinline__ constexpr uint32_t idesc_bf16_mn() {
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

template <int BN, int MG, int NG>
__global__ void __launch_bounds__(192, 1)
    k_wgrad_tma(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapG, const WgradGeo g,
                float *dw, int S, int *err) {
    using Cf = WgCfg<MG, NG>;
    constexpr int ACC = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
    constexpr int TMEM_COLS = 2 * ACC;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const int bkx = g.bkx;
    const uint32_t A_BYTES = 128u * bkx * 2, B_BYTES = (uint32_t)BN * bkx * 2, STAGE = A_BYTES + B_BYTES;
    const uint32_t bar_full = base + S * STAGE;
    const uint32_t bar_empty = bar_full + 8 * S;
    const uint32_t bar_afull = bar_empty + 8 * S;
    const uint32_t bar_aempty = bar_afull + 16;
    const uint32_t tmem_slot = bar_aempty + 16;
    volatile int *abort = (volatile int *)(smem_raw + (tmem_slot + 4 - raw));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m_total = 9 * g.C;

    if (threadIdx.x == 0) {
        *abort = *(volatile int *)err;
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(bar_full + 8 * s, 1);
            tc::mbar_init(bar_empty + 8 * s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(bar_afull + 8 * a, 1);
            tc::mbar_init(bar_aempty + 8 * a, 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"((uint64_t)&mapX) : "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"((uint64_t)&mapG) : "memory");
    }
    __syncthreads();
    if (*abort) return;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tmem_slot),
                     "r"((uint32_t)TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    uint32_t tmem_base;
    asm volatile("ld.shared.u32 %0, [%1];\n" : "=r"(tmem_base) : "r"(tmem_slot));

    // unit u = mt * ksplit + ks covers pixel blocks [kb0, kb1) of M tile mt
    auto unit_range = [&](int u, int &mt, int &kb0, int &kb1) {
        mt = u / g.ksplit;
        const int ks = u - mt * g.ksplit;
        const int per = (g.kblocks + g.ksplit - 1) / g.ksplit;
        kb0 = ks * per;
        kb1 = min(g.kblocks, kb0 + per);
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int s = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < g.units && ok; u += gridDim.x) {
                int mt, kb0, kb1;
                unit_range(u, mt, kb0, kb1);
                for (int kb = kb0; kb < kb1; ++kb) {
                    const int xb = kb % g.xblocks;
                    const int r = kb / g.xblocks;
                    const int y = r % g.H, b = r / g.H;
                    const int x0 = xb * bkx;
                    if (!tc::mbar_wait(bar_empty + 8 * s, ph ^ 1u, abort)) {
                        ok = false;
                        break;
                    }
                    const uint32_t sa = base + s * STAGE, sb = sa + A_BYTES;
                    arrive_expect_tx(bar_full + 8 * s, STAGE);
#pragma unroll
                    for (int gi = 0; gi < 128 / MG; ++gi) {
                        const int m0 = mt * 128 + gi * MG;
                        int c0 = g.C, dy = 0, dx = 0;  // past the last row: a box entirely out of range (zeros)
                        if (m0 < m_total) {
                            const int tap = m0 / g.C;
                            c0 = m0 - tap * g.C;
                            dy = tap / 3 - 1;
                            dx = tap % 3 - 1;
                        }
                        tma_load_4d(sa + gi * (uint32_t)(bkx * MG * 2), &mapX, c0, x0 + dx, y + dy, b,
                                    bar_full + 8 * s);
                    }
#pragma unroll
                    for (int gi = 0; gi < BN / NG; ++gi)
                        tma_load_4d(sb + gi * (uint32_t)(bkx * NG * 2), &mapG, gi * NG, x0, y, b, bar_full + 8 * s);
                    if (++s == S) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            if (!ok) {
                const long long t0 = clock64();
                while (clock64() - t0 < 200000LL) {
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            constexpr uint32_t IDESC = idesc_bf16_mn<BN>();
            const uint32_t lbo_a = (uint32_t)(bkx * MG * 2), lbo_b = (uint32_t)(bkx * NG * 2);
            int s = 0, acc = 0;
            uint32_t ph = 0, aph = 0;
            bool ok = true;
            uint32_t last_bar = 0, last_par = 0;
            for (int u = blockIdx.x; u < g.units && ok; u += gridDim.x) {
                int mt, kb0, kb1;
                unit_range(u, mt, kb0, kb1);
                if (!tc::mbar_wait(bar_aempty + 8 * acc, aph ^ 1u, abort)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t d = tmem_base + (uint32_t)(acc * ACC);
                bool first = true;
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!tc::mbar_wait(bar_full + 8 * s, ph, abort)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const uint32_t sa = base + s * STAGE, sb = sa + A_BYTES;
                    for (int kk = 0; kk < bkx / 16; ++kk) {
                        // 16 pixels = two 8-row groups along K
                        tc::mma_f16(d, sdesc_mn(sa + kk * 2 * Cf::SBO_A, lbo_a, Cf::SBO_A, Cf::LAYOUT_A),
                                    sdesc_mn(sb + kk * 2 * Cf::SBO_B, lbo_b, Cf::SBO_B, Cf::LAYOUT_B), IDESC,
                                    first ? 0u : 1u);
                        first = false;
                    }
                    tc::mma_commit(bar_empty + 8 * s);
                    last_bar = bar_empty + 8 * s;
                    last_par = ph;
                    if (++s == S) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (!ok) break;
                tc::mma_commit(bar_afull + 8 * acc);
                if (++acc == 2) {
                    acc = 0;
                    aph ^= 1u;
                }
            }
            if (!ok && last_bar) tc::mbar_wait(last_bar, last_par, nullptr);
        }
    } else {
        // ---------------- epilogue (warps 2..5): atomic adds into dW ----------------
        const int q = warp & 3;
        int acc = 0;
        uint32_t aph = 0;
        for (int u = blockIdx.x; u < g.units; u += gridDim.x) {
            int mt, kb0, kb1;
            unit_range(u, mt, kb0, kb1);
            if (!tc::mbar_wait(bar_afull + 8 * acc, aph, abort)) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const int m = mt * 128 + q * 32 + lane;
            const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * ACC);
#pragma unroll 1
            for (int j0 = 0; j0 < BN; j0 += 16) {
                uint32_t v[16];
                tc::tmem_ld16(taddr + (uint32_t)j0, v);
                if (m < m_total && kb1 > kb0) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) atomicAdd(dw + (long long)(j0 + i) * m_total + m, __uint_as_float(v[i]));
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) arrive(bar_aempty + 8 * acc);
            if (++acc == 2) {
                acc = 0;
                aph ^= 1u;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && *abort) atomicExch(err, 1);
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem_base),
                     "r"((uint32_t)TMEM_COLS));
    }
}

}  // namespace tma
}  // namespace nn
}  // namespace se2n
