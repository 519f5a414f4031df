// Lookup and launch of the diffusion kernel instantiations.
#include "diffuse_impl.cuh"

extern const DiffuseEntry se2n_diffuse_tab_a[];
extern const int se2n_diffuse_tab_a_len;
extern const DiffuseEntry se2n_diffuse_tab_b[];
extern const int se2n_diffuse_tab_b_len;
extern const DiffuseEntry se2n_diffuse_tab_c[];
extern const int se2n_diffuse_tab_c_len;

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

cudaError_t se2n_diffuse_occupancy(int N, int P, bool sm_fp64, bool split, int block, int *blocks_per_sm,
                                   int *regs) {
    const void *fn = find_kernel(N, P, sm_fp64, split);
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

cudaError_t se2n_launch_diffuse(int N, int P, bool sm_fp64, bool split, const DiffuseArgs &a, int block,
                                int blocks, cudaStream_t stream) {
    const void *fn = find_kernel(N, P, sm_fp64, split);
    if (!fn) return cudaErrorInvalidValue;
    void *args[] = {(void *)&a};
    return cudaLaunchKernel(fn, dim3(blocks), dim3(block), args, 0, stream);
}
