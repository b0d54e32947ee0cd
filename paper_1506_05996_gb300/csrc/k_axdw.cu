// Operator kernel, double-FP32 instantiations: the FP64 interface's operator on the FP32
// pipe (stored factors as pairs, binary64 vectors in and out).
#include "k_ax.cuh"

namespace sem {
cudaError_t launch_ax_local_dw(const DevProblem& d, const double* x, double* wl, const PcgState* st, cudaStream_t s) {
  return launch_ax_local_t<dw, double, false>(d, x, wl, st, nullptr, s);
}
cudaError_t launch_ax_apply_dw(const DevProblem& d, const double* x, double* wl, double* y, cudaStream_t s) {
  return launch_ax_local_t<dw, double, true>(d, x, wl, nullptr, y, s);
}
bool ax_tile_ok_dw(int p, int epb) { return ax_tile_ok_t<dw>(p, epb); }
}  // namespace sem
