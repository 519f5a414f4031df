// Diffusion kernel instantiations, small N (one thread or a pair per frequency).
#include "diffuse_x2.cuh"

extern const DiffuseEntry se2n_diffuse_tab_a[] = {
    SE2N_DIFFUSE_ENTRY(4, 1),  SE2N_DIFFUSE_ENTRY(8, 1),  SE2N_DIFFUSE_ENTRY(8, 2),
    SE2N_DIFFUSE_ENTRY(12, 1), SE2N_DIFFUSE_ENTRY(12, 2), SE2N_DIFFUSE_ENTRY(16, 1),
    SE2N_DIFFUSE_ENTRY(16, 2), SE2N_DIFFUSE_ENTRY(16, 4),
};
extern const int se2n_diffuse_tab_a_len = sizeof(se2n_diffuse_tab_a) / sizeof(se2n_diffuse_tab_a[0]);

// Packed fast path: P >= 2 needs K = N/P >= 6 angles per lane, so that the
// other tear's vector, at least K rows away, is below the truncation bound.
extern const DiffuseX2Entry se2n_diffuse_x2_tab_a[] = {SE2N_DIFFUSE_X2_ENTRY(4, 1), SE2N_DIFFUSE_X2_ENTRY(8, 1), SE2N_DIFFUSE_X2_ENTRY(12, 1), SE2N_DIFFUSE_X2_ENTRY(12, 2), SE2N_DIFFUSE_X2_ENTRY(16, 1), SE2N_DIFFUSE_X2_ENTRY(16, 2)};
extern const int se2n_diffuse_x2_tab_a_len = sizeof(se2n_diffuse_x2_tab_a) / sizeof(se2n_diffuse_x2_tab_a[0]);
