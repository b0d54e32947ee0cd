// Patch-solve kernel, FP64 instantiations.
#include "k_sw.cuh"

namespace sem {
cudaError_t launch_schwarz_local_dw(const DevProblem& d, const double* r, dw* wp, const PcgState* st,
                                    cudaStream_t s);
bool sw_tile_ok_dw(int P, int epb);

// SEM_PREC_FP64: the double-FP32 kernel (d.dwk; wp then holds pairs, read by the P-sum as
// such), else binary64.
cudaError_t launch_schwarz_local(const DevProblem& d, const double* r, double* wp, const PcgState* st, cudaStream_t s) {
  if (d.dwk) return launch_schwarz_local_dw(d, r, reinterpret_cast<dw*>(wp), st, s);
  return launch_schwarz_local_t<double, double>(d, r, wp, st, s);
}
cudaError_t launch_sw_diag(const DevProblem& d, double* dg, cudaStream_t s) {
  return launch_sw_diag_t<double>(d, dg, s);
}
bool sw_tile_ok(int P, int epb) {
  return sw_tile_ok_t<double>(P, epb) && sw_tile_ok_t<float>(P, epb) && sw_tile_ok_dw(P, epb);
}
}  // namespace sem
