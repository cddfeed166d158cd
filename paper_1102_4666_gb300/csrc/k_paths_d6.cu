// k_paths_d6.cu -- instantiation of the path kernel for d = 6 assets.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(6)
