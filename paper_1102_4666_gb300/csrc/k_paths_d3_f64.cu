// k_paths_d3_f64.cu -- instantiation of the path kernel for d = 3 assets, FP64 paths.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(3, double, f64)
