// tc_gemm.cu -- tcgen05 tensor-core products (placeholder until the kernels land).
#include "common.cuh"
#include "solver.h"

namespace prism {
bool tc_available() { return false; }
void launch_tc_gemm_P(const Dev&, cudaStream_t) {}
void launch_tc_gemm_x(const Dev&, cudaStream_t) {}
}  // namespace prism
