// k_paths_d3_tree.cu -- prefix-tree (dense, degree 4..6) evaluation kernels of the path kernel
// for d = 3 assets.
#include "k_paths.cuh"
BSDE_PATHS_INSTANTIATE_TREE(3)
