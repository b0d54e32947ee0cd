// Operator kernel, FP32 instantiations (mixed path).
#include "k_ax.cuh"

namespace sem {
cudaError_t launch_ax_local_f32(const DevProblem& d, const double* x, float* wl, const PcgState* st, cudaStream_t s) {
  return launch_ax_local_t<float, double>(d, x, wl, st, s);
}
cudaError_t launch_ax_local_f32_in32(const DevProblem& d, const float* x, float* wl, const PcgState* st,
                                     cudaStream_t s) {
  return launch_ax_local_t<float, float>(d, x, wl, st, s);
}
}  // namespace sem
