// sem_apply_A_noalloc: the operator apply y = A_D x for callers that must not
// allocate device memory.
//
// Why it exists: some callers cannot call cudaMalloc at all - code that runs
// while a stream is being captured into a CUDA graph (allocation is illegal
// there), code handed a fixed memory budget by a host framework that owns every
// allocation, or real-time loops where an allocator call is not allowed. They
// hold the mesh tables and vectors in memory they were given, and need the
// operator without the library allocating memory or creating CUDA objects.
//
// The two kernels of the ordinary apply are reused unchanged: the element kernel
// writes one FP64 value per local GLL node into scratch memory and the gather
// kernel sums those values per DOF. Here that scratch is the file-scope array
// g_noalloc_scratch below, of a fixed maximum size, which every GPU that loads
// the library holds until the process exits. The small GLL tables sit in a
// second static array.
#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sem.h"
#include "device.h"
#include "host_setup.h"

namespace {

constexpr int64_t kMaxLocal = SEM_NOALLOC_MAX_LOCAL_NODES;   // 2^21 doubles = 16 MiB
constexpr int kMinOrder = 2, kMaxOrder = 8, kMaxP = kMaxOrder + 1;
constexpr int kTabStride = kMaxP * kMaxP + 2 * kMaxP;        // D, then t, then rho
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kMaxLocal];
static __device__ __align__(256) double g_noalloc_tables[(kMaxOrder + 1) * kTabStride];

std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};
double* g_tables_ptr[kMaxDevices] = {nullptr};

int fail(int code, const std::string& msg) { return sem::report_error(code, msg); }

// Once per device, with that device current: resolve the device addresses of the
// static arrays (in host code their names are host-side stand-ins, not device
// addresses) and fill the GLL tables of every supported order.
int setup_device(int dev) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_scratch_ptr[dev] != nullptr) return SEM_OK;
  void* scratch = nullptr;
  void* tables = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&scratch, g_noalloc_scratch);
  if (e != cudaSuccess) return fail(SEM_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
  e = cudaGetSymbolAddress(&tables, g_noalloc_tables);
  if (e != cudaSuccess) return fail(SEM_ERR_CUDA, std::string("cudaGetSymbolAddress(tables): ") + cudaGetErrorString(e));
  double host[(kMaxOrder + 1) * kTabStride] = {0};
  for (int n = kMinOrder; n <= kMaxOrder; ++n) {
    std::vector<double> t, rho;
    sem::gll(n, t, rho);
    std::vector<double> D = sem::derivative_matrix(n, t);
    double* row = host + n * kTabStride;
    const int p = n + 1;
    for (int q = 0; q < p * p; ++q) row[q] = D[q];
    for (int q = 0; q < p; ++q) row[p * p + q] = t[q];
    for (int q = 0; q < p; ++q) row[p * p + p + q] = rho[q];
  }
  e = cudaMemcpyToSymbol(g_noalloc_tables, host, sizeof(host));
  if (e != cudaSuccess) return fail(SEM_ERR_CUDA, std::string("cudaMemcpyToSymbol(tables): ") + cudaGetErrorString(e));
  g_tables_ptr[dev] = (double*)tables;
  g_scratch_ptr[dev] = (double*)scratch;
  return SEM_OK;
}

}  // namespace

extern "C" int sem_apply_A_noalloc(int order, int64_t n_hex, int64_t n_dof, double lambda,
                                   const double* elem_xyz_dev, const int32_t* l2g_dev,
                                   const int32_t* g2l_off_dev, const int32_t* g2l_idx_dev,
                                   const uint8_t* mask_dev, const double* x_dev, double* y_dev,
                                   void* cuda_stream) {
  if (order < kMinOrder || order > kMaxOrder) return fail(SEM_ERR_ARG, "order must be in 2..8");
  if (n_hex < 1 || n_dof < 1) return fail(SEM_ERR_ARG, "n_hex and n_dof must be positive");
  const int p = order + 1;
  const int64_t L = n_hex * p * p * p;
  if (L > kMaxLocal)
    return fail(SEM_ERR_ARG, "sem_apply_A_noalloc: n_hex*(order+1)^3 = " + std::to_string(L) +
                                 " local nodes exceeds the static scratch of " + std::to_string(kMaxLocal));
  if (n_dof > L) return fail(SEM_ERR_ARG, "n_dof larger than the number of local nodes");
  if (!elem_xyz_dev || !l2g_dev || !g2l_off_dev || !g2l_idx_dev || !mask_dev || !x_dev || !y_dev || x_dev == y_dev)
    return fail(SEM_ERR_ARG, "NULL or aliased device pointer");
  if (!(lambda >= 0.0)) return fail(SEM_ERR_ARG, "lambda must be >= 0");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(SEM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(SEM_ERR_ARG, "device index out of range");
  if (int rc = setup_device(dev)) return rc;

  sem::DevProblem d;
  d.n = order; d.p = p; d.P = order + 3;
  d.ne = (int)n_hex; d.G = (int)n_dof;
  d.lambda = lambda;
  d.recompute = true;
  d.l2g = l2g_dev;
  d.exyz = elem_xyz_dev;
  const double* tab = g_tables_ptr[dev] + order * kTabStride;
  d.D = tab;
  d.tg = tab + p * p;
  d.rho = tab + p * p + p;
  d.mask = mask_dev;
  d.g2l_off = g2l_off_dev;
  d.g2l_idx = g2l_idx_dev;
  d.nblk = (int)std::min<int64_t>((n_dof + sem::kVecBlock - 1) / sem::kVecBlock, 152 * 8);
  double* scratch = g_scratch_ptr[dev];
  cudaStream_t s = (cudaStream_t)cuda_stream;
  e = sem::launch_ax_local(d, x_dev, scratch, nullptr, s);
  if (e == cudaSuccess) e = sem::launch_gather_identity(d, scratch, x_dev, y_dev, s);
  if (e != cudaSuccess) return fail(SEM_ERR_CUDA, std::string("sem_apply_A_noalloc launch: ") + cudaGetErrorString(e));
  return SEM_OK;
}
