// Diffusion kernel instantiations, medium N (a pair or two pairs per frequency).
#include "diffuse_x2.cuh"

extern const DiffuseEntry se2n_diffuse_tab_b[] = {
    SE2N_DIFFUSE_ENTRY(24, 2), SE2N_DIFFUSE_ENTRY(24, 4), SE2N_DIFFUSE_ENTRY(30, 2),
    SE2N_DIFFUSE_ENTRY(32, 2), SE2N_DIFFUSE_ENTRY(32, 4),
};
extern const int se2n_diffuse_tab_b_len = sizeof(se2n_diffuse_tab_b) / sizeof(se2n_diffuse_tab_b[0]);

extern const DiffuseX2Entry se2n_diffuse_x2_tab_b[] = {SE2N_DIFFUSE_X2_ENTRY(24, 2), SE2N_DIFFUSE_X2_ENTRY(24, 4), SE2N_DIFFUSE_X2_ENTRY(30, 2), SE2N_DIFFUSE_X2_ENTRY(32, 2), SE2N_DIFFUSE_X2_ENTRY(32, 4)};
extern const int se2n_diffuse_x2_tab_b_len = sizeof(se2n_diffuse_x2_tab_b) / sizeof(se2n_diffuse_x2_tab_b[0]);
