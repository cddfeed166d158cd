// k_paths_d10.cu -- instantiation of the path kernel for d = 10 assets.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(10)
