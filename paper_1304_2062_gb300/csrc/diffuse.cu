// Lookup and launch of the diffusion kernel instantiations.
#include "diffuse_x2.cuh"

#include <math.h>

#include <algorithm>
#include <climits>

extern const DiffuseEntry se2n_diffuse_tab_a[];
extern const int se2n_diffuse_tab_a_len;
extern const DiffuseEntry se2n_diffuse_tab_b[];
extern const int se2n_diffuse_tab_b_len;
extern const DiffuseEntry se2n_diffuse_tab_c[];
extern const int se2n_diffuse_tab_c_len;

extern const DiffuseX2Entry se2n_diffuse_x2_tab_a[];
extern const int se2n_diffuse_x2_tab_a_len;
extern const DiffuseX2Entry se2n_diffuse_x2_tab_b[];
extern const int se2n_diffuse_x2_tab_b_len;
extern const DiffuseX2Entry se2n_diffuse_x2_tab_c[];
extern const int se2n_diffuse_x2_tab_c_len;

static const void *find_x2(int N, int P, bool split) {
    const DiffuseX2Entry *tabs[3] = {se2n_diffuse_x2_tab_a, se2n_diffuse_x2_tab_b, se2n_diffuse_x2_tab_c};
    const int lens[3] = {se2n_diffuse_x2_tab_a_len, se2n_diffuse_x2_tab_b_len, se2n_diffuse_x2_tab_c_len};
    for (int t = 0; t < 3; ++t)
        for (int i = 0; i < lens[t]; ++i)
            if (tabs[t][i].N == N && tabs[t][i].P == P && tabs[t][i].split == split) return tabs[t][i].fn;
    return nullptr;
}

bool se2n_diffuse_truncation_ok(double beta_dt) {
    // decay per row of the tear vectors: 1/p with p the limiting pivot of the
    // scaled matrix at its smallest diagonal d_min = 2/(beta dt) + 2
    const double d = 2.0 / beta_dt + 2.0;
    const double p = 0.5 * (d + sqrt(d * d - 4.0));
    return pow(1.0 / p, (double)se2n::kTruncRows) <= 1e-9;
}

static const void *choose(int N, int P, bool fp64, bool split, bool fast);

static const void *find_kernel(int N, int P, bool fp64, bool split) {
    const DiffuseEntry *tabs[3] = {se2n_diffuse_tab_a, se2n_diffuse_tab_b, se2n_diffuse_tab_c};
    const int lens[3] = {se2n_diffuse_tab_a_len, se2n_diffuse_tab_b_len, se2n_diffuse_tab_c_len};
    for (int t = 0; t < 3; ++t)
        for (int i = 0; i < lens[t]; ++i)
            if (tabs[t][i].N == N && tabs[t][i].P == P && tabs[t][i].fp64 == fp64 && tabs[t][i].split == split)
                return tabs[t][i].fn;
    return nullptr;
}

bool se2n_diffuse_has(int N, int P) { return find_kernel(N, P, false, false) != nullptr; }

int se2n_diffuse_default_P(int N) {
    if (N <= 16) return 1;
    if (N <= 32) return 2;
    return 4;
}

static const void *choose(int N, int P, bool fp64, bool split, bool fast) {
    if (fast && !fp64) {
        const void *fn = find_x2(N, P, split);
        if (fn) return fn;
    }
    return find_kernel(N, P, fp64, split);
}

cudaError_t se2n_diffuse_occupancy(int N, int P, bool sm_fp64, bool split, bool fast, int block,
                                   int *blocks_per_sm, int *regs) {
    const void *fn = choose(N, P, sm_fp64, split, fast);
    if (!fn) return cudaErrorInvalidValue;
    cudaFuncAttributes attr;
    cudaError_t e = cudaFuncGetAttributes(&attr, fn);
    if (e != cudaSuccess) return e;
    if (regs) *regs = attr.numRegs;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, 0);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm) *blocks_per_sm = n;
    return cudaSuccess;
}

int se2n_diffuse_block_limit(int N, int P, bool sm_fp64, bool split, bool fast) {
    const void *fn = choose(N, P, sm_fp64, split, fast);
    cudaFuncAttributes attr;
    if (!fn || cudaFuncGetAttributes(&attr, fn) != cudaSuccess) return 256;
    return attr.maxThreadsPerBlock;
}

cudaError_t se2n_diffuse_shape(int N, int P, bool sm_fp64, bool split, bool fast, int tuned_block,
                               int tuned_blocks, int num_sms, long long freqs, int *block, int *blocks) {
    const bool packed = fast && !sm_fp64 && find_x2(N, P, split) != nullptr;
    int b = tuned_block, nb = tuned_blocks;
    bool all = false;
    if (b == 0) {
        if (packed && N < 48) {
            b = 128;
            all = true;
        } else {
            b = packed ? 384 : 256;
        }
        nb = 0;
    }
    b = std::min(b, se2n_diffuse_block_limit(N, P, sm_fp64, split, fast));
    const long long need = std::max((freqs * P + b - 1) / b, 1LL);
    if (all) {
        nb = (int)std::min(need, (long long)INT_MAX);
    } else if (nb <= 0) {
        int per_sm = 0;
        cudaError_t e = se2n_diffuse_occupancy(N, P, sm_fp64, split, fast, b, &per_sm, nullptr);
        if (e != cudaSuccess) return e;
        nb = num_sms * std::max(per_sm, 1);
    }
    if (nb > need) nb = (int)need;
    *block = b;
    *blocks = std::max(nb, 1);
    return cudaSuccess;
}

cudaError_t se2n_launch_diffuse(int N, int P, bool sm_fp64, bool split, bool fast, const DiffuseArgs &a,
                                int block, int blocks, cudaStream_t stream) {
    const void *fn = choose(N, P, sm_fp64, split, fast);
    if (!fn) return cudaErrorInvalidValue;
    void *args[] = {(void *)&a};
    return cudaLaunchKernel(fn, dim3(blocks), dim3(block), args, 0, stream);
}
