// k_paths_d8_f64.cu -- instantiation of the path kernel for d = 8 assets, FP64 paths.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE(8, double, f64)
