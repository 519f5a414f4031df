// Host side of the TMA tensor-core convolutions (conv_tma.cuh): tensor-map
// encoding, shape checks, the epilogue functors and the launches for the
// forward convolution (optionally with the network's 1x1 head and input
// skip fused into the last layer) and the data gradient.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>

#include "conv_tma.cuh"
#include "nn.h"

using namespace se2n::nn;

// Set by a TMA convolution whose bounded wait ran out (never expected).
__device__ int g_tma_fault;

namespace {

__device__ __forceinline__ uint32_t pack2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *(const uint32_t *)&h;
}

__device__ __forceinline__ void store16(__nv_bfloat16 *dst, const float (&w)[16]) {
    uint32_t p[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) p[q] = pack2(w[2 * q], w[2 * q + 1]);
    uint4 *d4 = (uint4 *)dst;
    d4[0] = make_uint4(p[0], p[1], p[2], p[3]);
    d4[1] = make_uint4(p[4], p[5], p[6], p[7]);
}

// out[m][n..n+15] = relu?(v + bias) as bf16; pixel m's channels at out + m * N;
// nb bias values (the output channels).
struct FwdEpi {
    const float *bias;
    __nv_bfloat16 *out;
    int N, relu, nb;
    static constexpr int SMEM_FLOATS = 256;
    __device__ __forceinline__ void prepare(float *sm, int i, int n) const {
        for (int k = i; k < nb; k += n) sm[k] = bias[k];
    }
    __device__ __forceinline__ void store(int m, int n, const float (&v)[16], float &, const float *sm) const {
        float w[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            w[q] = v[q] + sm[n + q];
            if (relu) w[q] = fmaxf(w[q], 0.0f);
        }
        store16(out + (long long)m * N + n, w);
    }
    __device__ __forceinline__ void finish(int, float, const float *) const {}
};

// The last convolution (32 channels, ReLU) with the 1x1 head and the input
// skip: d[m][:] = bf16(relu(v + bias)) as FwdEpi (not stored when out is
// null: inference needs only y), and
// y[m] = f[m] (mask[m] != 0) + hb + sum_c hw[c] d[m][c] (FP32, c in order).
struct HeadEpi {
    const float *bias;
    __nv_bfloat16 *out;
    const float *hw, *hb, *f;
    const uint8_t *mask;
    float *y;
    static constexpr int SMEM_FLOATS = 65;  // bias[32], hw[32], hb
    __device__ __forceinline__ void prepare(float *sm, int i, int n) const {
        for (int k = i; k < 65; k += n) sm[k] = k < 32 ? bias[k] : k < 64 ? hw[k - 32] : hb[0];
    }
    __device__ __forceinline__ void store(int m, int n, const float (&v)[16], float &st, const float *sm) const {
        float w[16];
        if (n == 0) st = sm[64];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            w[q] = fmaxf(v[q] + sm[n + q], 0.0f);
            w[q] = __bfloat162float(__float2bfloat16_rn(w[q]));
            st = fmaf(sm[32 + n + q], w[q], st);
        }
        if (out) store16(out + (long long)m * 32 + n, w);
    }
    __device__ __forceinline__ void finish(int m, float st, const float *) const {
        y[m] = (mask[m] ? f[m] : 0.0f) + st;
    }
};

// Data gradient: columns < split go to din (times (act > 0) when act is
// given), the others to din2; N columns in all.
struct DgradEpi {
    const __nv_bfloat16 *act;
    __nv_bfloat16 *din, *din2;
    int split, N;
    static constexpr int SMEM_FLOATS = 1;
    __device__ __forceinline__ void prepare(float *, int, int) const {}
    __device__ __forceinline__ void store(int m, int n, const float (&v)[16], float &, const float *) const {
        float w[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) w[q] = v[q];
        if (n < split) {
            if (act) {
                const uint4 *a4 = (const uint4 *)(act + (long long)m * split + n);
                const uint4 a0 = a4[0], a1 = a4[1];
                const uint32_t aw[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const __nv_bfloat162 h = *(const __nv_bfloat162 *)&aw[q];
                    if (!(__bfloat162float(h.x) > 0.0f)) w[2 * q] = 0.0f;
                    if (!(__bfloat162float(h.y) > 0.0f)) w[2 * q + 1] = 0.0f;
                }
            }
            store16(din + (long long)m * split + n, w);
        } else {
            store16(din2 + (long long)m * (N - split) + (n - split), w);
        }
    }
    __device__ __forceinline__ void finish(int, float, const float *) const {}
};

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return (PFN_cuTensorMapEncodeTiled_v12000)p;
    }();
    return fn;
}

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return n;
}

int *fault_ptr() {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tma_fault) != cudaSuccess) return nullptr;
    return (int *)p;
}

// Tile shape: bw x bh = 128 pixels of one image.
bool tile_shape(int H, int W, int &bw, int &bh) {
    bw = W >= 128 ? 128 : W;
    if (bw < 1 || W % bw || 128 % bw) return false;
    bh = 128 / bw;
    return H % bh == 0;
}

template <int BN, int CK, class EPI>
cudaError_t launch(const __nv_bfloat16 *A, int B, int H, int W, int C, const __nv_bfloat16 *wmat, int N, int flip,
                   const EPI &epi, cudaStream_t s) {
    using Cf = tma::Cfg<BN, CK>;
    int bw, bh;
    if (!tile_shape(H, W, bw, bh) || C % CK || N % BN) return cudaErrorNotSupported;
    auto enc = encoder();
    const int nsm = sm_count();
    int *err = fault_ptr();
    if (!enc || nsm <= 0 || !err) return cudaErrorNotSupported;
    CUtensorMap ma, mb;
    {
        const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
        const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
        const cuuint32_t box[4] = {(cuuint32_t)CK, (cuuint32_t)bw, (cuuint32_t)bh, 1};
        const cuuint32_t es[4] = {1, 1, 1, 1};
        if (enc(&ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)A, dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CK == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        const cuuint64_t dims[2] = {(cuuint64_t)9 * C, (cuuint64_t)N};
        const cuuint64_t strides[1] = {(cuuint64_t)9 * C * 2};
        const cuuint32_t box[2] = {(cuuint32_t)CK, (cuuint32_t)BN};
        const cuuint32_t es[2] = {1, 1};
        if (enc(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)wmat, dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CK == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    tma::ConvGeo g;
    g.B = B;
    g.H = H;
    g.W = W;
    g.C = C;
    g.bw = bw;
    g.bh = bh;
    g.tiles_x = W / bw;
    g.tiles_y = H / bh;
    g.mtiles = B * g.tiles_x * g.tiles_y;
    g.ntiles = N / BN;
    g.tiles = g.mtiles * g.ntiles;
    g.nchunk = C / CK;
    g.KB = 9 * g.nchunk;
    g.flip = flip;
    auto *fn = &tma::k_conv_tma<BN, CK, EPI>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, Cf::SMEM);
    if (e != cudaSuccess) return e;
    const int grid = g.tiles < nsm ? g.tiles : nsm;
    fn<<<grid, 192, Cf::SMEM, s>>>(ma, mb, g, epi, err);
    return cudaGetLastError();
}

// Narrow layers: 16 x 8 tiles, halo boxes, weights resident in shared memory.
template <int BN, int CK, class EPI>
cudaError_t launch_halo(const __nv_bfloat16 *A, int B, int H, int W, int C, const __nv_bfloat16 *wmat, int N, int flip,
                        const EPI &epi, cudaStream_t s) {
    using Cf = tma::HaloCfg<BN, CK>;
    if (W % tma::HBW || H % tma::HBH || C % CK || N % BN) return cudaErrorNotSupported;
    const int nblk = 9 * (C / CK);
    const int wbytes = nblk * Cf::BBLK;
    int S = (Cf::SMEM_BUDGET - wbytes) / Cf::A_BYTES;
    if (S > 8) S = 8;
    if (S < 3) return cudaErrorNotSupported;
    auto enc = encoder();
    const int nsm = sm_count();
    int *err = fault_ptr();
    if (!enc || nsm <= 0 || !err) return cudaErrorNotSupported;
    CUtensorMap ma, mb;
    {
        const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
        const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
        const cuuint32_t box[4] = {(cuuint32_t)CK, (cuuint32_t)tma::HBW, (cuuint32_t)(tma::HBH + 2), 1};
        const cuuint32_t es[4] = {1, 1, 1, 1};
        if (enc(&ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)A, dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CK == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        const cuuint64_t dims[2] = {(cuuint64_t)9 * C, (cuuint64_t)N};
        const cuuint64_t strides[1] = {(cuuint64_t)9 * C * 2};
        const cuuint32_t box[2] = {(cuuint32_t)CK, (cuuint32_t)BN};
        const cuuint32_t es[2] = {1, 1};
        if (enc(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)wmat, dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CK == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    tma::ConvGeo g;
    g.B = B;
    g.H = H;
    g.W = W;
    g.C = C;
    g.bw = tma::HBW;
    g.bh = tma::HBH;
    g.tiles_x = W / tma::HBW;
    g.tiles_y = H / tma::HBH;
    g.mtiles = B * g.tiles_x * g.tiles_y;
    g.ntiles = N / BN;
    g.tiles = g.mtiles * g.ntiles;
    g.nchunk = C / CK;
    g.KB = 3 * g.nchunk;
    g.flip = flip;
    const int smem = 1024 + wbytes + S * Cf::A_BYTES + 256;
    auto *fn = &tma::k_conv_halo<BN, CK, EPI>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    // each CTA keeps one n tile's weights: a whole number of CTAs per n tile
    const int per = nsm / g.ntiles;
    if (per < 1) return cudaErrorNotSupported;
    const int grid = (g.mtiles < per ? g.mtiles : per) * g.ntiles;
    fn<<<grid, 192, smem, s>>>(ma, mb, g, epi, S, err);
    return cudaGetLastError();
}

// Weight gradient (k_wgrad_tma): x [B][H][W][C] and gz [B][H][W][Cout] NHWC, dw
// [Cout][9 C] FP32 (accumulated).
template <int BN, int MG, int NG>
cudaError_t launch_wgrad(const __nv_bfloat16 *x, int B, int H, int W, int C, const __nv_bfloat16 *gz, float *dw,
                         cudaStream_t s) {
    const int bkx = W >= 64 ? 64 : W;
    if (bkx < 16 || bkx % 16 || W % bkx || C % MG) return cudaErrorNotSupported;
    auto enc = encoder();
    const int nsm = sm_count();
    int *err = fault_ptr();
    if (!enc || nsm <= 0 || !err) return cudaErrorNotSupported;
    CUtensorMap mx, mg;
    {
        const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
        const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
        const cuuint32_t box[4] = {(cuuint32_t)MG, (cuuint32_t)bkx, 1, 1};
        const cuuint32_t es[4] = {1, 1, 1, 1};
        if (enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)x, dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, MG == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        const cuuint64_t dims[4] = {(cuuint64_t)BN, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
        const cuuint64_t strides[3] = {(cuuint64_t)BN * 2, (cuuint64_t)W * BN * 2, (cuuint64_t)H * W * BN * 2};
        const cuuint32_t box[4] = {(cuuint32_t)NG, (cuuint32_t)bkx, 1, 1};
        const cuuint32_t es[4] = {1, 1, 1, 1};
        if (enc(&mg, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)gz, dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, NG == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    tma::WgradGeo g;
    g.B = B;
    g.H = H;
    g.W = W;
    g.C = C;
    g.Cout = BN;
    g.bkx = bkx;
    g.xblocks = W / bkx;
    g.kblocks = B * H * g.xblocks;
    g.mtiles = (9 * C + 127) / 128;
    int ks = (2 * nsm + g.mtiles - 1) / g.mtiles;
    if (ks > g.kblocks) ks = g.kblocks;
    if (ks < 1) ks = 1;
    g.ksplit = ks;
    g.units = g.mtiles * ks;
    const int stage = (128 + BN) * bkx * 2;
    int S = 196608 / stage;
    if (S > 8) S = 8;
    const int smem = 1024 + S * stage + 256;
    auto *fn = &tma::k_wgrad_tma<BN, MG, NG>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int grid = g.units < nsm ? g.units : nsm;
    fn<<<grid, 192, smem, s>>>(mx, mg, g, dw, S, err);
    return cudaGetLastError();
}

}  // namespace

namespace se2n {
namespace nn {

cudaError_t conv_wgrad_tma(const __nv_bfloat16 *x, int B, int H, int W, int C, const __nv_bfloat16 *gz, int Cout,
                           float *dw, cudaStream_t s) {
    const bool m64 = C % 64 == 0;
    switch (Cout) {
        case 32: return m64 ? cudaErrorNotSupported : launch_wgrad<32, 32, 32>(x, B, H, W, C, gz, dw, s);
        case 64: return m64 ? launch_wgrad<64, 64, 64>(x, B, H, W, C, gz, dw, s)
                            : launch_wgrad<64, 32, 64>(x, B, H, W, C, gz, dw, s);
        case 128: return m64 ? launch_wgrad<128, 64, 64>(x, B, H, W, C, gz, dw, s) : cudaErrorNotSupported;
        case 256: return m64 ? launch_wgrad<256, 64, 64>(x, B, H, W, C, gz, dw, s) : cudaErrorNotSupported;
        default: return cudaErrorNotSupported;
    }
}

cudaError_t tma_fault(int *host_flag, bool reset) {
    cudaError_t e = cudaMemcpyFromSymbol(host_flag, g_tma_fault, sizeof(int));
    if (e == cudaSuccess && reset && *host_flag) {
        const int zero = 0;
        e = cudaMemcpyToSymbol(g_tma_fault, &zero, sizeof(int));
    }
    return e;
}

cudaError_t conv_forward_tma(const __nv_bfloat16 *in, int B, int H, int W, int Cin, const __nv_bfloat16 *w,
                             const float *bias, int Cout, int relu, __nv_bfloat16 *out, int ldo, const HeadArgs *head,
                             cudaStream_t s) {
    const bool ck64 = Cin % 64 == 0;
    if (head) {
        if (Cout != 32 || !relu || ldo != 32) return cudaErrorNotSupported;
        const HeadEpi epi{bias, out, head->hw, head->hb, head->f, head->mask, head->y};
        cudaError_t e = ck64 ? launch_halo<32, 64>(in, B, H, W, Cin, w, Cout, 0, epi, s)
                             : launch_halo<32, 32>(in, B, H, W, Cin, w, Cout, 0, epi, s);
        if (e != cudaErrorNotSupported) return e;
        return ck64 ? launch<32, 64>(in, B, H, W, Cin, w, Cout, 0, epi, s)
                    : launch<32, 32>(in, B, H, W, Cin, w, Cout, 0, epi, s);
    }
    const FwdEpi epi{bias, out, ldo, relu, Cout};
    if (Cout == 32 || Cout == 64) {
        cudaError_t e;
        if (Cout == 32)
            e = ck64 ? launch_halo<32, 64>(in, B, H, W, Cin, w, Cout, 0, epi, s)
                     : launch_halo<32, 32>(in, B, H, W, Cin, w, Cout, 0, epi, s);
        else
            e = ck64 ? launch_halo<64, 64>(in, B, H, W, Cin, w, Cout, 0, epi, s)
                     : launch_halo<64, 32>(in, B, H, W, Cin, w, Cout, 0, epi, s);
        if (e != cudaErrorNotSupported) return e;
    }
    switch (Cout) {
        case 32: return ck64 ? launch<32, 64>(in, B, H, W, Cin, w, Cout, 0, epi, s)
                             : launch<32, 32>(in, B, H, W, Cin, w, Cout, 0, epi, s);
        case 64: return ck64 ? launch<64, 64>(in, B, H, W, Cin, w, Cout, 0, epi, s)
                             : launch<64, 32>(in, B, H, W, Cin, w, Cout, 0, epi, s);
        case 128: return ck64 ? launch<128, 64>(in, B, H, W, Cin, w, Cout, 0, epi, s) : cudaErrorNotSupported;
        case 256: return ck64 ? launch<256, 64>(in, B, H, W, Cin, w, Cout, 0, epi, s) : cudaErrorNotSupported;
        default: return cudaErrorNotSupported;
    }
}

cudaError_t conv_dgrad_tma(const __nv_bfloat16 *gz, int B, int H, int W, int Cout, const __nv_bfloat16 *wt, int Cin,
                           const __nv_bfloat16 *act, __nv_bfloat16 *din, __nv_bfloat16 *din2, int split,
                           cudaStream_t s) {
    if (split % 16) return cudaErrorNotSupported;
    const bool ck64 = Cout % 64 == 0;
    const DgradEpi epi{act, din, din2, split, Cin};
    // A = gz (Cout channels, taps mirrored), B = wt [Cin][9 Cout]
    if (Cin == 32 || Cin == 64 || Cin == 96) {
        cudaError_t e = cudaErrorNotSupported;
        if (Cin == 32)
            e = ck64 ? launch_halo<32, 64>(gz, B, H, W, Cout, wt, Cin, 1, epi, s)
                     : launch_halo<32, 32>(gz, B, H, W, Cout, wt, Cin, 1, epi, s);
        else if (Cin == 64)
            e = ck64 ? launch_halo<64, 64>(gz, B, H, W, Cout, wt, Cin, 1, epi, s)
                     : launch_halo<64, 32>(gz, B, H, W, Cout, wt, Cin, 1, epi, s);
        else if (!ck64)
            e = launch_halo<96, 32>(gz, B, H, W, Cout, wt, Cin, 1, epi, s);
        if (e != cudaErrorNotSupported) return e;
    }
    if (!ck64) {
        if (Cin == 32) return launch<32, 32>(gz, B, H, W, Cout, wt, Cin, 1, epi, s);
        if (Cin == 96) return launch<96, 32>(gz, B, H, W, Cout, wt, Cin, 1, epi, s);
        return cudaErrorNotSupported;
    }
    switch (Cin) {
        case 32: return launch<32, 64>(gz, B, H, W, Cout, wt, Cin, 1, epi, s);
        case 64: return launch<64, 64>(gz, B, H, W, Cout, wt, Cin, 1, epi, s);
        case 128: return launch<128, 64>(gz, B, H, W, Cout, wt, Cin, 1, epi, s);
        case 192:
        case 384: return launch<192, 64>(gz, B, H, W, Cout, wt, Cin, 1, epi, s);
        case 256: return launch<256, 64>(gz, B, H, W, Cout, wt, Cin, 1, epi, s);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace nn
}  // namespace se2n
