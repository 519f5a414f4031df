// Persistent diffusion kernel for a batch of images of uneven size and N.
//
// The batch's frequencies are cut into work items (image, first frequency,
// count); each warp claims items from one atomic counter until none are
// left, so a single launch keeps every SM busy across images of very
// different sizes. Items are ordered by decreasing cost (N = 64 first, then
// larger images), which lets the dynamic claiming approximate a
// longest-job-first schedule. The per-frequency arithmetic is exactly the
// single-image kernels' (diffuse_group / diffuse_group_x2), so a batched
// result is bitwise equal to the same image diffused on its own.
//
// The counter only grows and every claim is bounded by the item count: no
// warp waits on another, and the kernel cannot hang.
#include "diffuse_x2.cuh"
#include "se2n_batch.h"

namespace se2n {

template <int N, int P, bool FAST, bool SPLIT>
__device__ __forceinline__ void batch_item(const StepParams &sp, const float *tables, const BatchImage &im,
                                           const BatchItem &item, int lane) {
    constexpr int PER = 32 / P;  // frequencies per pass of the warp
    const int slot = lane / P;
    const float *cs = tables + im.table;
    const float *sn = cs + N;
    for (int base = 0; base < item.count; base += PER) {
        const int o = base + slot;
        const bool active = o < item.count;
        const long long fc = item.first + (active ? o : 0);
        if constexpr (FAST) {
            diffuse_group_x2<N, P, SPLIT>(sp, cs, sn, im.vol, im.H, im.W, im.Wc, im.HW, fc, active);
        } else {
            diffuse_group<N, P, false, SPLIT>(sp, cs, sn, im.vol, im.H, im.W, im.Wc, im.HW, fc, active);
        }
    }
}

template <int P16, int P32, int P64, bool FAST, bool SPLIT>
__global__ void __launch_bounds__(FAST ? kDiffuseMaxBlock : 256, 1) k_diffuse_batch(const StepParams sp, const float *__restrict__ tables,
                                                       const BatchImage *__restrict__ imgs,
                                                       const BatchItem *__restrict__ items, int n_items,
                                                       unsigned int *counter) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned int it = 0;
        if (lane == 0) it = atomicAdd(counter, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= (unsigned int)n_items) return;
        const BatchItem item = items[it];
        const BatchImage im = imgs[item.image];
        if (im.N == 64) {
            batch_item<64, P64, FAST, SPLIT>(sp, tables, im, item, lane);
        } else if (im.N == 32) {
            batch_item<32, P32, FAST, SPLIT>(sp, tables, im, item, lane);
        } else {
            batch_item<16, P16, FAST, SPLIT>(sp, tables, im, item, lane);
        }
    }
}

}  // namespace se2n

// Launch configurations the autotuner chooses among: threads per frequency
// for N = 16, 32, 64.
static const int kConfigs[][3] = {{1, 2, 4}, {2, 4, 4}};

template <int C, bool FAST, bool SPLIT>
static const void *pick() {
    if constexpr (C == 0) return (const void *)&se2n::k_diffuse_batch<1, 2, 4, FAST, SPLIT>;
    else return (const void *)&se2n::k_diffuse_batch<2, 4, 4, FAST, SPLIT>;
}

static const void *batch_kernel(int config, bool fast, bool split) {
    if (config == 0) {
        if (fast) return split ? pick<0, true, true>() : pick<0, true, false>();
        return split ? pick<0, false, true>() : pick<0, false, false>();
    }
    if (fast) return split ? pick<1, true, true>() : pick<1, true, false>();
    return split ? pick<1, false, true>() : pick<1, false, false>();
}

int se2n_batch_configs() { return (int)(sizeof(kConfigs) / sizeof(kConfigs[0])); }

int se2n_batch_config_P(int config, int N) {
    const int i = (N == 16) ? 0 : (N == 32) ? 1 : 2;
    return kConfigs[config][i];
}

cudaError_t se2n_batch_occupancy(int config, bool fast, bool split, int block, int *blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, batch_kernel(config, fast, split), block, 0);
}

cudaError_t se2n_launch_diffuse_batch(int config, bool fast, bool split, const StepParams &sp, const float *tables,
                                      const BatchImage *imgs, const BatchItem *items, int n_items,
                                      unsigned int *counter, int block, int blocks, cudaStream_t s) {
    void *args[] = {(void *)&sp, (void *)&tables, (void *)&imgs, (void *)&items, (void *)&n_items,
                    (void *)&counter};
    return cudaLaunchKernel(batch_kernel(config, fast, split), dim3(blocks), dim3(block), args, 0, s);
}
