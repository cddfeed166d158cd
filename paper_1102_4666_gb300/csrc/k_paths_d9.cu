// k_paths_d9.cu -- instantiation of the path kernel for d = 9 assets.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(9)
