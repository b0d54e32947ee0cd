// Operator kernel, FP64 instantiations.
#include "k_ax.cuh"

namespace sem {
cudaError_t launch_ax_local_dw(const DevProblem& d, const double* x, double* wl, const PcgState* st, cudaStream_t s);
cudaError_t launch_ax_apply_dw(const DevProblem& d, const double* x, double* wl, double* y, cudaStream_t s);
bool ax_tile_ok_dw(int p, int epb);

// SEM_PREC_FP64: the double-FP32 kernel (d.dwk; stored or recomputed factors), else binary64.
cudaError_t launch_ax_local(const DevProblem& d, const double* x, double* wl, const PcgState* st, cudaStream_t s) {
  if (d.dwk) return launch_ax_local_dw(d, x, wl, st, s);
  return launch_ax_local_t<double, double, false>(d, x, wl, st, nullptr, s);
}
cudaError_t launch_ax_apply(const DevProblem& d, const double* x, double* wl, double* y, cudaStream_t s) {
  if (d.dwk) return launch_ax_apply_dw(d, x, wl, y, s);
  return launch_ax_local_t<double, double, true>(d, x, wl, nullptr, y, s);
}
// Whether the operator kernel exists for this order and elements per CTA, in every
// arithmetic the handle may use.
bool ax_tile_ok(int p, int epb) {
  return ax_tile_ok_t<double>(p, epb) && ax_tile_ok_t<float>(p, epb) && ax_tile_ok_dw(p, epb);
}
}  // namespace sem
