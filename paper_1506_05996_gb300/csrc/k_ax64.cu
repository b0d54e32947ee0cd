// Operator kernel, FP64 instantiations.
#include "k_ax.cuh"

namespace sem {
cudaError_t launch_ax_local(const DevProblem& d, const double* x, double* wl, const PcgState* st, cudaStream_t s) {
  return launch_ax_local_t<double, double, false>(d, x, wl, st, nullptr, s);
}
cudaError_t launch_ax_apply(const DevProblem& d, const double* x, double* wl, double* y, cudaStream_t s) {
  return launch_ax_local_t<double, double, true>(d, x, wl, nullptr, y, s);
}
// Whether the operator kernel exists for this order and elements per CTA, in either
// precision the handle may use.
bool ax_tile_ok(int p, int epb) { return ax_tile_ok_t<double>(p, epb) && ax_tile_ok_t<float>(p, epb); }
}  // namespace sem
