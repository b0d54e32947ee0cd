// Patch-solve kernel, FP32 instantiations (mixed path).
#include "k_sw.cuh"

namespace sem {
cudaError_t launch_schwarz_local_f32(const DevProblem& d, const double* r, float* wp, const PcgState* st,
                                     cudaStream_t s) {
  return launch_schwarz_local_t<float, double>(d, r, wp, st, s);
}
cudaError_t launch_schwarz_local_f32_in32(const DevProblem& d, const float* r, float* wp, const PcgState* st,
                                          cudaStream_t s) {
  return launch_schwarz_local_t<float, float>(d, r, wp, st, s);
}
cudaError_t launch_sw_diag_f32(const DevProblem& d, float* dg, cudaStream_t s) {
  return launch_sw_diag_t<float>(d, dg, s);
}
}  // namespace sem
