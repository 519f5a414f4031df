// Diffusion kernel instantiations, large N (two pairs per frequency).
#include "diffuse_x2.cuh"

extern const DiffuseEntry se2n_diffuse_tab_c[] = {
    SE2N_DIFFUSE_ENTRY(48, 4), SE2N_DIFFUSE_ENTRY(64, 4),
};
extern const int se2n_diffuse_tab_c_len = sizeof(se2n_diffuse_tab_c) / sizeof(se2n_diffuse_tab_c[0]);

extern const DiffuseX2Entry se2n_diffuse_x2_tab_c[] = {SE2N_DIFFUSE_X2_ENTRY(48, 4), SE2N_DIFFUSE_X2_ENTRY(64, 4)};
extern const int se2n_diffuse_x2_tab_c_len = sizeof(se2n_diffuse_x2_tab_c) / sizeof(se2n_diffuse_x2_tab_c[0]);
