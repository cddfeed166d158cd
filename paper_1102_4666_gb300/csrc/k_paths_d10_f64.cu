// k_paths_d10_f64.cu -- instantiation of the path kernel for d = 10 assets, FP64 paths.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(10, double, f64)
