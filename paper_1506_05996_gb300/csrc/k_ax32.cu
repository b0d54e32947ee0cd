// Operator kernel, FP32 instantiations (mixed path).
#include "k_ax.cuh"

namespace sem {
cudaError_t launch_ax_local_f32(const DevProblem& d, const double* x, float* wl, const PcgState* st, cudaStream_t s) {
  return launch_ax_local_t<float, double, false>(d, x, wl, st, nullptr, s);
}
cudaError_t launch_ax_apply_f32(const DevProblem& d, const double* x, float* wl, double* y, cudaStream_t s) {
  return launch_ax_local_t<float, double, true>(d, x, wl, nullptr, y, s);
}
cudaError_t launch_ax_local_f32_in32(const DevProblem& d, const float* x, float* wl, const PcgState* st,
                                     cudaStream_t s) {
  return launch_ax_local_t<float, float, false>(d, x, wl, st, nullptr, s);
}
cudaError_t launch_ax_apply_f32io(const DevProblem& d, const float* x, float* wl, float* y, cudaStream_t s) {
  return launch_ax_local_t<float, float, true>(d, x, wl, nullptr, y, s);
}
}  // namespace sem
