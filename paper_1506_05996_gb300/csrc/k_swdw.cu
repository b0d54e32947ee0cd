// Patch-solve kernel, double-FP32 instantiation: the FP64 interface's P^f on the FP32 pipe
// (binary64 residual in, patch results as pairs for the P-sum).
#include "k_sw.cuh"

namespace sem {
cudaError_t launch_schwarz_local_dw(const DevProblem& d, const double* r, dw* wp, const PcgState* st,
                                    cudaStream_t s) {
  return launch_schwarz_local_t<dw, double>(d, r, wp, st, s);
}
bool sw_tile_ok_dw(int P, int epb) { return sw_tile_ok_t<dw>(P, epb); }
}  // namespace sem
