// k_paths_dispatch.cu -- choose the compiled path kernel for the number of
// assets d (the per-asset state is held in registers, so d is a template
// parameter of the kernel).
#include "k_paths.cuh"

#define DECL(DV)                                                                              \
  cudaError_t launch_paths_d##DV##_f32(const ModelHost&, const GridHost&, const ProblemDev&, int, \
                                       int, uint32_t, int, int, cudaStream_t);                \
  cudaError_t launch_paths_d##DV##_f64(const ModelHost&, const GridHost&, const ProblemDev&, int, \
                                       int, uint32_t, int, int, cudaStream_t);
DECL(1) DECL(2) DECL(3) DECL(4) DECL(5) DECL(6) DECL(7) DECL(8) DECL(9) DECL(10)
#undef DECL

int paths_supported_d(int d) { return d >= 1 && d <= 10; }

size_t paths_smem_bytes(int d, int p, int eta, int N, int tpb, bool mixed, bool dense) {
  // an upper bound for every volatility family and evaluation form: the tanh
  // families tabulate two coefficients per asset and step (rows padded to 16
  // bytes), and a dense evaluation with FP32 paths may keep its coefficients
  // twice and keep the states around the random time (copy_smem)
  return paths::smem_bytes(d, p, eta < 1 ? 1 : eta, N, tpb, mixed ? sizeof(float) : sizeof(double),
                           dense, (2 * (d < 3 ? 3 : d) + 3) & ~3, dense && mixed, dense && mixed);
}

cudaError_t launch_paths(const ModelHost& m, const GridHost& g, const ProblemDev& P, int M, int N,
                         uint32_t k, bool mixed, int tpb, int ppt, cudaStream_t st) {
#define CASE(DV)                                                                          \
  case DV:                                                                                \
    return mixed ? launch_paths_d##DV##_f32(m, g, P, M, N, k, tpb, ppt, st)               \
                 : launch_paths_d##DV##_f64(m, g, P, M, N, k, tpb, ppt, st);
  switch (m.d) {
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10)
    default: return cudaErrorInvalidValue;
  }
#undef CASE
}
