// Diffusion of several transformed volumes that allocates nothing.
//
// Some callers cannot let a library call cudaMalloc: a host application that
// owns all device memory through its own pool or arena (a framework
// allocator, an embedded runtime with a fixed memory budget) must not have
// memory taken behind its back, and a latency-critical loop cannot afford
// the implicit device-wide synchronisation cudaMalloc and cudaFree may
// cause. For them, se2n_diffuse_many_noalloc runs the persistent diffusion
// over up to SE2N_NOALLOC_MAX_VOLUMES volumes using only the caller's
// volumes and the fixed scratch array below: the work counter, the volume
// records, the per-volume work-item prefix counts and the angle tables.
// The work items themselves are derived on the device from the prefix
// counts, so nothing else is needed. The per-frequency arithmetic is the
// single-image kernels' (diffuse_group / diffuse_group_x2).
#include <math.h>
#include <string.h>

#include "diffuse_x2.cuh"
#include "se2n_batch.h"

namespace {

constexpr int kMaxVolumes = SE2N_NOALLOC_MAX_VOLUMES;
constexpr int kPasses = 8;  // warp passes (32/P frequencies each) per work item

// The records of one call: built on the host and handed to the set-up kernel
// by value, as its launch parameter, so the call copies nothing from host
// memory and keeps no pointer to the host stack.
struct NoallocRecords {
    int count;                     // volumes in this call
    int tile[kMaxVolumes];         // frequencies per work item of volume i
    long long prefix[kMaxVolumes + 1];  // work items before volume i
    BatchImage vols[kMaxVolumes];
    float tables[2 * (16 + 32 + 64)];   // cos[N] then sin[N], for N = 16, 32, 64
};

struct StaticScratch {
    unsigned int counter;          // work items claimed; set to 0 by every call
    unsigned int pad[63];          // keeps the records 256 bytes apart from the counter
    NoallocRecords rec;
};

// The whole scratch of the entry point. Every GPU that loads the library
// holds these bytes until the process exits; every call shares them.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SE2N_NOALLOC_SCRATCH_BYTES];
static_assert(sizeof(StaticScratch) <= SE2N_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the stated size");
static_assert(sizeof(NoallocRecords) % 4 == 0 && sizeof(NoallocRecords) <= 16384, "records fit one launch parameter");

constexpr int table_offset(int N) { return N == 16 ? 0 : (N == 32 ? 2 * 16 : 2 * (16 + 32)); }

template <int N, int P, bool FAST, bool SPLIT>
__device__ __forceinline__ void static_item(const StepParams &sp, const float *tables, const BatchImage &im,
                                            long long first, int count, int lane) {
    constexpr int PER = 32 / P;
    const int slot = lane / P;
    const float *cs = tables + im.table;
    const float *sn = cs + N;
    for (int base = 0; base < count; base += PER) {
        const int o = base + slot;
        const bool active = o < count;
        const long long fc = first + (active ? o : 0);
        if constexpr (FAST) {
            se2n::diffuse_group_x2<N, P, SPLIT>(sp, cs, sn, im.vol, im.H, im.W, im.W, im.HW, fc, active);
        } else {
            se2n::diffuse_group<N, P, false, SPLIT>(sp, cs, sn, im.vol, im.H, im.W, im.W, im.HW, fc, active);
        }
    }
}

// Persistent: warps claim work items from the counter until all are done.
// Claims only grow and are bounded by the item count, so no warp waits on
// another.
template <bool FAST, bool SPLIT>
__global__ void __launch_bounds__(256) k_diffuse_static(const StepParams sp, StaticScratch *s) {
    const int lane = threadIdx.x & 31;
    const NoallocRecords &r = s->rec;
    const int count = r.count;
    const long long total = r.prefix[count];
    for (;;) {
        unsigned int it = 0;
        if (lane == 0) it = atomicAdd(&s->counter, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if ((long long)it >= total) return;
        int lo = 0, hi = count - 1;  // the volume i with prefix[i] <= it < prefix[i + 1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (r.prefix[mid] <= (long long)it) lo = mid;
            else hi = mid - 1;
        }
        const BatchImage im = r.vols[lo];
        const long long first = ((long long)it - r.prefix[lo]) * r.tile[lo];
        const int n = (int)min((long long)r.tile[lo], im.HW - first);
        if (im.N == 64) static_item<64, 4, FAST, SPLIT>(sp, r.tables, im, first, n, lane);
        else if (im.N == 32) static_item<32, 2, FAST, SPLIT>(sp, r.tables, im, first, n, lane);
        else static_item<16, 1, FAST, SPLIT>(sp, r.tables, im, first, n, lane);
    }
}

// Copies the call's records from the launch parameter into the scratch array
// and sets the work counter to zero. One block; it runs to completion before
// the diffusion launch that follows it on the same stream.
__global__ void __launch_bounds__(256) k_noalloc_setup(const __grid_constant__ NoallocRecords rec, StaticScratch *s) {
    const unsigned int *src = reinterpret_cast<const unsigned int *>(&rec);
    unsigned int *dst = reinterpret_cast<unsigned int *>(&s->rec);
    for (int i = threadIdx.x; i < (int)(sizeof(NoallocRecords) / 4); i += blockDim.x) dst[i] = src[i];
    if (threadIdx.x == 0) s->counter = 0u;
}

const void *static_kernel(bool fast, bool split) {
    if (fast) return split ? (const void *)&k_diffuse_static<true, true> : (const void *)&k_diffuse_static<true, false>;
    return split ? (const void *)&k_diffuse_static<false, true> : (const void *)&k_diffuse_static<false, false>;
}

bool device_ptr16(const void *p) {
    if (!p || ((uintptr_t)p % 16) != 0) return false;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// Device address of the scratch array on the current device. Host code
// cannot use the symbol itself as a device address; the lookup allocates
// nothing and is repeated on every call, so the address stays right if the
// device's context is ever created again.
se2n_status scratch_address(StaticScratch **out) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        (void)cudaGetLastError();
        return SE2N_ECUDA;
    }
    *out = (StaticScratch *)p;
    return SE2N_OK;
}

}  // namespace

extern "C" se2n_status se2n_diffuse_many_noalloc(const se2n_volume_desc *vols, int count, double beta, double T,
                                                 int steps, int angle_conv, int flags, void *stream) {
    if (!vols || count < 1 || count > kMaxVolumes) return SE2N_EINVAL;
    if (!(beta > 0.0) || !(T >= 0.0) || steps < 1 || !isfinite(beta) || !isfinite(T)) return SE2N_EINVAL;
    if ((angle_conv != 0 && angle_conv != 1) || (flags & ~(SE2N_DIFFUSE_SPLIT_DIAG | SE2N_DIFFUSE_FULL_CORRECTION)))
        return SE2N_EINVAL;
    for (int i = 0; i < count; ++i) {
        const se2n_volume_desc &v = vols[i];
        if (v.H < 2 || v.W < 2 || (v.H % 2) || (v.W % 2) || (long long)v.H * v.W > (1LL << 28)) return SE2N_EINVAL;
        if (v.N != 16 && v.N != 32 && v.N != 64) return SE2N_EUNSUPPORTED;
        if (!device_ptr16(v.vol_hat)) return SE2N_EINVAL;
    }
    if (T == 0.0) return SE2N_OK;
    const double bdt = beta * (T / steps);
    if (!(bdt >= 1e-30 && bdt <= 1e3)) return SE2N_ENUMERIC;
    const bool split = (flags & SE2N_DIFFUSE_SPLIT_DIAG) != 0 || beta * T > 8.0;
    const bool fast = !(flags & SE2N_DIFFUSE_FULL_CORRECTION) && se2n_diffuse_truncation_ok(bdt);

    int dev = -1, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SE2N_ECUDA;
    StaticScratch *d_scratch = nullptr;
    se2n_status st = scratch_address(&d_scratch);
    if (st != SE2N_OK) return st;

    // The call's records, passed by value to the set-up kernel (which also
    // sets the shared counter back to zero).
    NoallocRecords h;
    memset(&h, 0, sizeof(h));
    h.count = count;
    const int Ns[3] = {16, 32, 64};
    for (int t = 0; t < 3; ++t) {
        const int N = Ns[t];
        angle_table(N, angle_conv, h.tables + table_offset(N), h.tables + table_offset(N) + N, N);
    }
    h.prefix[0] = 0;
    for (int i = 0; i < count; ++i) {
        const se2n_volume_desc &v = vols[i];
        BatchImage &bi = h.vols[i];
        bi.vol = (float2 *)v.vol_hat;
        bi.H = v.H;
        bi.W = v.W;
        bi.HW = (long long)v.H * v.W;
        bi.N = v.N;
        bi.table = table_offset(v.N);
        const int P = v.N == 16 ? 1 : (v.N == 32 ? 2 : 4);
        h.tile[i] = (32 / P) * kPasses;
        h.prefix[i + 1] = h.prefix[i] + (bi.HW + h.tile[i] - 1) / h.tile[i];
    }
    cudaStream_t s = (cudaStream_t)stream;
    k_noalloc_setup<<<1, 256, 0, s>>>(h, d_scratch);
    cudaError_t e = cudaGetLastError();
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, static_kernel(fast, split), 256, 0);
    if (e == cudaSuccess) {
        const StepParams sp = step_params(beta, bdt, steps);
        void *args[] = {(void *)&sp, (void *)&d_scratch};
        e = cudaLaunchKernel(static_kernel(fast, split), dim3(sms * (per_sm > 0 ? per_sm : 1)), dim3(256), args, 0, s);
    }
    return e == cudaSuccess ? SE2N_OK : (e == cudaErrorMemoryAllocation ? SE2N_ENOMEM : SE2N_ECUDA);
}
