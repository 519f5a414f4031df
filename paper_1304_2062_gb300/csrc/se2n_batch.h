// Device-side records of the batched diffusion (shared by batch_kern.cu and
// the host code that builds them).
#pragma once

#include "se2n_internal.h"

struct BatchImage {
    float2 *vol;       // [N][H][Wc] complex, the image's transformed volume
    long long HW;      // H * Wc frequencies per plane
    int H, W, N;
    int Wc;            // stored columns: W, or W/2 + 1 for the Hermitian half
    int table;         // offset of the image's angle table (cos[N] then sin[N]) in the table array
};

struct BatchItem {
    int image;         // index into the BatchImage array
    int count;         // frequencies in this item
    long long first;   // first frequency index k*Wc + l
};

int se2n_batch_configs();
int se2n_batch_config_P(int config, int N);
cudaError_t se2n_batch_occupancy(int config, bool fast, bool split, int block, int *blocks_per_sm);
cudaError_t se2n_launch_diffuse_batch(int config, bool fast, bool split, const StepParams &sp, const float *tables,
                                      const BatchImage *imgs, const BatchItem *items, int n_items,
                                      unsigned int *counter, int block, int blocks, cudaStream_t s);
