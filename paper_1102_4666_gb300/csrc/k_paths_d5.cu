// k_paths_d5.cu -- instantiation of the path kernel for d = 5 assets.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(5)
