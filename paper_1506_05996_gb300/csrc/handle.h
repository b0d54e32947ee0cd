// The library handle (sem_t of include/sem.h) and the per-handle profiler and iteration
// graph; shared by the C ABI translation units (api.cu, nn_api.cu).
#pragma once

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/sem.h"
#include "device.h"
#include "host_setup.h"
#include "nn.h"

// One PCG iteration (preconditioner, direction, operator, alpha, update) captured as a
// CUDA graph and replayed once per iteration; with profiling on, its timing events are
// graph nodes read back after each replay.
struct IterGraph {
  cudaGraphExec_t exec = nullptr;
  long key = -1;
  std::vector<cudaEvent_t> events;
  std::vector<int> pair_id, pair_idx;
  std::vector<uint64_t> pair_kernels;
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    key = -1;
    for (auto e : events) cudaEventDestroy(e);
    events.clear();
    pair_id.clear();
    pair_idx.clear();
    pair_kernels.clear();
  }
  ~IterGraph() { reset(); }
};

// A whole solve as one graph (device-driven loop): the initial steps, then a WHILE node
// around one iteration (with an IF node for the mixed path's residual replacement), so a
// solve is one graph launch with no host round trip per iteration.
struct LoopGraph {
  cudaGraphExec_t exec = nullptr;
  long key = -1;
  double rtol = -1.0;
  int maxit = -1;
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    key = -1;
    rtol = -1.0;
    maxit = -1;
  }
  ~LoopGraph() { reset(); }
};

constexpr int kGraphBase = 1 << 28;

// Per-kernel timing with CUDA events recorded on the handle's stream around each
// launch (enabled by sem_profile); accumulated when the stream is synchronised.
struct Profiler {
  IterGraph* cap = nullptr;   // set while an iteration graph is being captured
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, int>> pending;   // (kernel id, first event index)
  std::vector<uint64_t> pending_kernels;      // kernels launched inside each pending pair
  uint64_t count_at_begin = 0;
  int next = 0;
  std::vector<std::string> names;
  std::vector<double> total_ms;
  std::vector<int64_t> launches;

  int id(const char* name) {
    for (size_t i = 0; i < names.size(); ++i)
      if (names[i] == name) return (int)i;
    names.emplace_back(name);
    total_ms.push_back(0.0);
    launches.push_back(0);
    return (int)names.size() - 1;
  }
  int begin(cudaStream_t s) {
    if (!on) return -1;
    if (cap != nullptr) {
      cudaEvent_t a, b;
      if (cudaEventCreate(&a) != cudaSuccess) return -1;
      if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return -1; }
      cap->events.push_back(a);
      cap->events.push_back(b);
      // an external record becomes an event-record node, whose times can be read back
      cudaEventRecordWithFlags(a, s, cudaEventRecordExternal);
      count_at_begin = sem::kernel_launch_count();
      return kGraphBase + (int)cap->events.size() - 2;
    }
    while ((int)pool.size() < next + 2) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      pool.push_back(e);
    }
    int i = next;
    next += 2;
    cudaEventRecord(pool[i], s);
    count_at_begin = sem::kernel_launch_count();
    return i;
  }
  void end(int i, const char* name, cudaStream_t s) {
    if (i < 0) return;
    if (i >= kGraphBase) {
      const int k = i - kGraphBase;
      cudaEventRecordWithFlags(cap->events[k + 1], s, cudaEventRecordExternal);
      cap->pair_id.push_back(id(name));
      cap->pair_idx.push_back(k);
      cap->pair_kernels.push_back(sem::kernel_launch_count() - count_at_begin);
      return;
    }
    cudaEventRecord(pool[i + 1], s);
    pending.emplace_back(id(name), i);
    pending_kernels.push_back(sem::kernel_launch_count() - count_at_begin);
  }
  void collect() {   // stream must be synchronised
    for (size_t q = 0; q < pending.size(); ++q) {
      const auto& pr = pending[q];
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, pool[pr.second], pool[pr.second + 1]) == cudaSuccess) {
        total_ms[pr.first] += ms;
        launches[pr.first] += (int64_t)pending_kernels[q];
      }
    }
    pending.clear();
    pending_kernels.clear();
    next = 0;
  }
  void collect_graph(const IterGraph& g) {   // after a replay has completed
    for (size_t q = 0; q < g.pair_id.size(); ++q) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, g.events[g.pair_idx[q]], g.events[g.pair_idx[q] + 1]) == cudaSuccess) {
        total_ms[g.pair_id[q]] += ms;
        launches[g.pair_id[q]] += (int64_t)g.pair_kernels[q];
      } else {
        cudaGetLastError();   // a timing failure must not look like a later launch failure
      }
    }
  }
  void reset() {
    pending.clear();
    pending_kernels.clear();
    next = 0;
    names.clear();
    total_ms.clear();
    launches.clear();
  }
  ~Profiler() {
    for (auto e : pool) cudaEventDestroy(e);
  }
};

struct sem_s {
  Profiler prof;
  sem::DevProblem d;
  cudaStream_t stream = nullptr;
  // The coarse correction runs on a second, high-priority stream concurrently with the
  // fine patch solves (P = P^c + P^f are independent until they are summed).
  cudaStream_t coarse_stream = nullptr;
  cudaStream_t capture_stream = nullptr;   // graphs are captured here (not on a legacy stream)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int flags = 0;
  int precond = SEM_PRECOND_TWO_SCALE;
  sem::Numbering nb;
  sem::Csr A0full;
  std::vector<uint8_t> mask_host;
  std::vector<void*> allocs;        // freed at destroy
  std::vector<void*> coarse_allocs; // freed when the coarse space is rebuilt
  std::vector<sem::DevAmgLevel> levels;
  bool coarse_ok = false;
  std::string coarse_err;
  double *coords = nullptr, *mN = nullptr, *geo = nullptr;
  float* geo32 = nullptr;
  __nv_bfloat16* geo16 = nullptr;   // BF16 copy of the stored factors (SEM_MIXED)
  sem::dw* geodw = nullptr;         // pairs-of-FP32 copy of the stored factors (SEM_PREC_FP64)
  int precision = SEM_PREC_FP64;
  int amg_kind = 0;                 // SEM_COARSE_VCYCLE or SEM_COARSE_KCYCLE
  int overlap_sms = 48;             // FP32 patch solves leave this many SMs to the coarse branch
  uint8_t* mask = nullptr;
  uint8_t* pvar = nullptr;          // free sides of every element (see update_free_sides)
  double* swd = nullptr;             // patch-solve diagonals, scaled (update_free_sides)
  float* swd32 = nullptr;
  sem::dw* swddw = nullptr;          // the same as pairs of FP32 (double-FP32 patch solves)
  double* pw = nullptr;             // overlap weights of P^f (sem_set_weights)
  float* pw32 = nullptr;
  double *r = nullptr, *z = nullptr, *p = nullptr, *f = nullptr, *u = nullptr;
  IterGraph graph;
  LoopGraph loop;
  int loop_mode = SEM_LOOP_DEVICE;
  uint64_t epoch = 0;               // bumped whenever captured graphs become stale
  double* bbuf = nullptr;           // right-hand side copied in before a device-driven solve
  int* loop_guard = nullptr;        // iteration guard of the device-driven loop
  void invalidate() {
    graph.reset();
    loop.reset();
    ++epoch;
  }
  double* hist = nullptr;
  int hist_cap = 0;
  int kcap = 1;                      // right-hand sides the solver buffers hold (sem_solve_block)
  sem::PcgState* st_host = nullptr;  // pinned
  double *heat_b = nullptr, *heat_d = nullptr, *heat_norms = nullptr;   // sem_heat_step scratch
  // learned correction (not in the paper): attached network and its forward work space
  sem_net_t* net = nullptr;
  int nn_window = 8;        // stall rule of the flexible PCG (sem_set_learned)
  double nn_ratio = 0.5;
  double nn_theta = 0.25;   // per-iteration acceptance of the correction
  sem::NnWork nnws;
  std::vector<void*> nn_allocs;

  template <class T>
  cudaError_t alloc(T** ptr, size_t count, std::vector<void*>& list) {
    *ptr = nullptr;
    if (count == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc((void**)ptr, count * sizeof(T));
    if (e == cudaSuccess) list.push_back(*ptr);
    return e;
  }
  template <class T>
  cudaError_t upload(T** ptr, const std::vector<T>& v, std::vector<void*>& list) {
    cudaError_t e = alloc(ptr, v.size(), list);
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpyAsync(*ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, stream);
  }
  void free_list(std::vector<void*>& list) {
    for (void* q : list) cudaFree(q);
    list.clear();
  }
};

namespace sem {
// Learned correction of the attached network into d.nncorr (nn_api.cu); st != nullptr
// inside PCG (the kernels skip once the solve stopped or the network was switched off).
cudaError_t learned_correction(sem_t* h, const double* r, const PcgState* st, cudaStream_t s);
}  // namespace sem
