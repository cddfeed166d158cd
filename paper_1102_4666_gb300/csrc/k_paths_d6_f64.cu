// k_paths_d6_f64.cu -- instantiation of the path kernel for d = 6 assets, FP64 paths.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(6, double, f64)
