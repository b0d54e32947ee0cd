// C ABI (include/sem.h): handle creation, uploads, operator/preconditioner
// applications and the PCG driver of Algorithm 1.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sem.h"
#include "handle.h"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CK(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(e_ == cudaErrorMemoryAllocation ? SEM_ERR_OOM : SEM_ERR_CUDA,            \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                     \
  } while (0)

}  // namespace

namespace {

// The last batch graph of sem_solve_many (all its solves in one launch), kept while the
// same handles, in the same configuration, are solved again.
struct BatchGraph {
  std::vector<sem_t*> handles;
  std::vector<uint64_t> epochs;
  std::vector<long> keys;
  double rtol = -1.0;
  int maxit = -1;
  cudaGraphExec_t exec = nullptr;
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    handles.clear();
    epochs.clear();
    keys.clear();
  }
};
std::mutex g_batch_mutex;
BatchGraph g_batch;

}  // namespace

#define PROF_ON(h, strm, name, call)                 \
  do {                                                \
    int pi_ = (h)->prof.begin(strm);                  \
    CK(call);                                         \
    (h)->prof.end(pi_, name, strm);                   \
  } while (0)
#define PROF(h, name, call) PROF_ON(h, (h)->stream, name, call)

namespace {

// Coarse space on the free vertices and its AMG hierarchy (Sec. 4.1); rebuilt when
// the mask changes.
int build_coarse(sem_t* h) {
  cudaStreamSynchronize(h->stream);
  h->invalidate();
  h->free_list(h->coarse_allocs);
  h->levels.clear();
  sem::DevProblem& d = h->d;
  d.nlevels = 0;
  d.levels = nullptr;
  d.nfree = 0;
  h->coarse_ok = false;
  const sem::Numbering& nb = h->nb;
  std::vector<int> cvmap(nb.nv, -1), keep;
  for (int64_t v = 0; v < nb.nv; ++v) {
    int g = nb.vert_dof[v];
    if (g >= 0 && h->mask_host[g] == 0) { cvmap[v] = (int)keep.size(); keep.push_back((int)v); }
  }
  const int nfree = (int)keep.size();
  std::vector<int> ecv(8 * nb.ne);
  for (int64_t q = 0; q < 8 * nb.ne; ++q) ecv[q] = cvmap[nb.hexv[q]];
  std::vector<int> cv_off(nfree + 1, 0), cv_idx;
  for (int64_t q = 0; q < 8 * nb.ne; ++q)
    if (ecv[q] >= 0) cv_off[ecv[q] + 1]++;
  for (int i = 0; i < nfree; ++i) cv_off[i + 1] += cv_off[i];
  cv_idx.resize(cv_off[nfree]);
  {
    std::vector<int> fill(cv_off.begin(), cv_off.end() - 1);
    for (int64_t q = 0; q < 8 * nb.ne; ++q)
      if (ecv[q] >= 0) cv_idx[fill[ecv[q]]++] = (int)q;
  }
  int* tmp_i;
  CK(h->upload(&tmp_i, ecv, h->coarse_allocs)); d.ecv = tmp_i;
  CK(h->upload(&tmp_i, cv_off, h->coarse_allocs)); d.cv_off = tmp_i;
  CK(h->upload(&tmp_i, cv_idx, h->coarse_allocs)); d.cv_idx = tmp_i;
  d.nfree = nfree;
  if (nfree == 0) { h->coarse_ok = true; return SEM_OK; }
  sem::Csr A0 = sem::submatrix(h->A0full, keep);
  sem::Amg amg;
  d.amg_kind = h->amg_kind;
  std::string err = sem::build_amg(A0, amg, h->amg_kind == SEM_COARSE_KCYCLE ? sem::kAmgKcycle : sem::kAmgVcycle);
  if (!err.empty()) {
    h->coarse_err = err;
    d.nfree = 0;
    return SEM_OK;   // the operator still works; preconditioners needing P^c report it
  }
  auto up_csr = [&](const sem::Csr& A, sem::DevCsr& out) -> cudaError_t {
    out.n = A.n;
    out.nnz = (int)A.val.size();
    // about four entries per lane: 8 lanes for the 27-entry rows of the Q1 matrix, at most
    // a warp (wider groups measured slower on the long coarse-level rows)
    out.lanes = 4;
    while (out.lanes < 32 && 4 * out.lanes * (int64_t)A.n < (int64_t)out.nnz) out.lanes *= 2;
    cudaError_t e = h->upload(&out.ptr, A.ptr, h->coarse_allocs);
    if (e == cudaSuccess) e = h->upload(&out.col, A.col, h->coarse_allocs);
    if (e == cudaSuccess) e = h->upload(&out.val, A.val, h->coarse_allocs);
    return e;
  };
  h->levels.resize(amg.levels.size());
  for (size_t l = 0; l < amg.levels.size(); ++l) {
    const sem::AmgLevel& L = amg.levels[l];
    sem::DevAmgLevel& D = h->levels[l];
    CK(up_csr(L.A, D.A));
    CK(up_csr(L.P, D.P));
    CK(up_csr(L.R, D.R));
    if (h->amg_kind == SEM_COARSE_VCYCLE && L.M.val.empty()) {   // the V-cycle runs as M, N, Q
      h->coarse_err = "V-cycle level without its fused cycle matrices";
      d.nfree = 0;
      return SEM_OK;
    }
    if (!L.M.val.empty()) {
      CK(up_csr(L.M, D.M));
      CK(up_csr(L.N, D.N));
      CK(up_csr(L.Q, D.Q));
      const int64_t nnz = (int64_t)L.N.val.size() + (int64_t)L.Q.val.size();
      D.up_lanes = 4;
      while (D.up_lanes < 32 && 4 * D.up_lanes * (int64_t)L.N.n < nnz) D.up_lanes *= 2;
    }
    CK(h->upload(&D.dinv, L.dinv, h->coarse_allocs));
    // one slice per right-hand side of a block solve (h->kcap)
    CK(h->alloc(&D.b, (size_t)L.A.n * h->kcap, h->coarse_allocs));
    CK(h->alloc(&D.x, (size_t)L.A.n * h->kcap, h->coarse_allocs));
    CK(h->alloc(&D.t, (size_t)L.A.n * h->kcap, h->coarse_allocs));
    CK(h->alloc(&D.y, (size_t)L.A.n * h->kcap, h->coarse_allocs));
    if (h->amg_kind == SEM_COARSE_KCYCLE) {
      CK(h->alloc(&D.c1, L.A.n, h->coarse_allocs));
      CK(h->alloc(&D.c2, L.A.n, h->coarse_allocs));
      CK(h->alloc(&D.v1, L.A.n, h->coarse_allocs));
      CK(h->alloc(&D.v2, L.A.n, h->coarse_allocs));
      CK(h->alloc(&D.scal, 8, h->coarse_allocs));
    }
  }
  if (h->amg_kind == SEM_COARSE_KCYCLE && d.rprev == nullptr) CK(h->alloc(&d.rprev, (size_t)h->nb.G, h->allocs));
  double* tmp_d;
  CK(h->upload(&tmp_d, amg.coarsest_inv, h->coarse_allocs)); d.coarsest_inv = tmp_d;
  d.coarsest_n = amg.coarsest_n;
  const size_t kc = (size_t)h->kcap;
  CK(h->alloc(&d.cb, amg.coarsest_n * kc, h->coarse_allocs));
  CK(h->alloc(&d.cx, amg.coarsest_n * kc, h->coarse_allocs));
  CK(h->alloc(&d.cres, nfree * kc, h->coarse_allocs));
  CK(h->alloc(&d.Rc, nfree * kc, h->coarse_allocs));
  CK(h->alloc(&d.Zc, nfree * kc, h->coarse_allocs));
  CK(h->alloc(&d.Zce32, (size_t)8 * h->nb.ne * kc, h->coarse_allocs));
  CK(h->alloc(&d.Zce, (size_t)8 * h->nb.ne * kc, h->coarse_allocs));
  d.nlevels = (int)h->levels.size();
  d.levels = h->levels.data();
  CK(cudaStreamSynchronize(h->stream));
  h->coarse_ok = true;
  return SEM_OK;
}

// Pencil variant of every element side (natural boundary where a side has no neighbour
// and its face is not wholly masked); none anywhere -> d.pvar = null (the plain kernel path).
int update_free_sides(sem_t* h) {
  std::vector<uint8_t> fs = sem::free_sides(h->nb, h->mask_host);
  bool any = false;
  for (uint8_t v : fs) any = any || v != 0;
  CK(cudaMemcpyAsync(h->pvar, fs.data(), fs.size(), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->d.pvar = any ? h->pvar : nullptr;
  // the patch solves' diagonals depend on the pencils of each element
  CK(sem::launch_sw_diag(h->d, h->swd, h->stream));
  CK(sem::launch_sw_diag_f32(h->d, h->swd32, h->stream));
  CK(sem::launch_split_pairs((long long)h->nb.ne * h->d.P * h->d.P * h->d.P, h->swd, h->swddw, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->d.swd = h->swd;
  h->d.swd32 = h->swd32;
  h->d.swddw = h->swddw;
  h->invalidate();
  return SEM_OK;
}

int check_handle(const sem_t* h) {
  if (h == nullptr) return fail(SEM_ERR_ARG, "NULL handle");
  return SEM_OK;
}

// The FP32 paths' patch solves run in BF16 on the tensor cores (sem_set_patch_solver), unless
// some element side takes a natural-boundary pencil (the FP32 kernel serves those handles).
bool tc_active(const sem::DevProblem& d) { return d.tc && d.pfp32 && d.pvar == nullptr; }

// The BF16-factor operator's error, 2^-8 relative to |A|(|x|), is far larger relative to
// A x on the smooth error components that PCG leaves last, so the iteration stalls: BF16 is
// for operator and preconditioner applications only.
int check_solvable(const sem_t* h) {
  if (int rc = check_handle(h)) return rc;
  if (h->d.bf16) return fail(SEM_ERR_ARG, "SEM_PREC_BF16 is for sem_apply_A / sem_apply_P*; solve in FP32 or FP64");
  return SEM_OK;
}

// z = P r for the chosen parts; `pcg` adds the rz reduction / beta on the device.
int apply_precond(sem_t* h, int which, const double* r, double* z, bool pcg) {
  sem::DevProblem& d = h->d;
  const sem::PcgState* st = pcg ? d.st : nullptr;
  int mode = 0;
  const bool coarse = (which == SEM_PRECOND_TWO_SCALE || which == -1);
  if (coarse) {
    if (!h->coarse_ok || (d.nfree == 0 && !h->coarse_err.empty()))
      return fail(SEM_ERR_SINGULAR, "coarse space unavailable: " + h->coarse_err);
    // fork: AMG on the coarse stream, beside the patch solves. In FP64 the patch solves are
    // long enough to hide the restriction too, so it goes on the coarse stream; in FP32 the
    // restriction, slowed by sharing the SMs with them, would lengthen the critical path,
    // so it runs first, alone on the GPU, and only the latency-bound AMG kernels overlap.
    cudaStream_t cs = h->coarse_stream;
    const bool restrict_first = d.pfp32;
    if (restrict_first) {
      if (pcg && d.fp32)
        PROF(h, "coarse_restrict", sem::launch_coarse_restrict_f32(d, d.r32, st, h->stream));
      else
        PROF(h, "coarse_restrict", sem::launch_coarse_restrict(d, r, st, h->stream));
    }
    CK(cudaEventRecord(h->ev_fork, h->stream));
    CK(cudaStreamWaitEvent(cs, h->ev_fork, 0));
    if (!restrict_first) PROF_ON(h, cs, "coarse_restrict", sem::launch_coarse_restrict(d, r, st, cs));
    PROF_ON(h, cs, "coarse_amg", sem::launch_coarse_solve(d, st, cs));
    CK(cudaEventRecord(h->ev_join, cs));
    mode |= sem::PSUM_COARSE;
  }
  if (which == SEM_PRECOND_TWO_SCALE || which == SEM_PRECOND_FINE) {
    // FP32 patch solves leave h->overlap_sms SMs' worth of slots to the coarse branch
    sem::DevProblem dd = d;
    dd.sw_reserve_sms = (coarse && d.pfp32) ? h->overlap_sms : 0;
    if (tc_active(d) && d.fp32 && pcg)
      PROF(h, "schwarz_local", sem::launch_schwarz_tc_in32(dd, d.r32, reinterpret_cast<float*>(d.wp), st, h->stream));
    else if (tc_active(d))
      PROF(h, "schwarz_local", sem::launch_schwarz_tc(dd, r, reinterpret_cast<float*>(d.wp), st, h->stream));
    else if (d.fp32 && pcg)
      PROF(h, "schwarz_local", sem::launch_schwarz_local_f32_in32(dd, d.r32, reinterpret_cast<float*>(d.wp), st,
                                                                  h->stream));
    else if (d.pfp32)
      PROF(h, "schwarz_local", sem::launch_schwarz_local_f32(dd, r, reinterpret_cast<float*>(d.wp), st, h->stream));
    else
      PROF(h, "schwarz_local", sem::launch_schwarz_local(d, r, d.wp, st, h->stream));
    mode |= sem::PSUM_FINE;
  }
  if (coarse) CK(cudaStreamWaitEvent(h->stream, h->ev_join, 0));   // join
  if (which == SEM_PRECOND_NONE) mode = sem::PSUM_IDENT;
  // flexible PCG when P varies between applications: the K-cycle is nonlinear, and the
  // learned correction depends on r
  const bool learned = pcg && h->net != nullptr;
  // (the BF16 patch solves round between their contractions: P is then not exactly linear)
  const bool fine = which == SEM_PRECOND_TWO_SCALE || which == SEM_PRECOND_FINE;
  const bool flex = pcg && (learned || (coarse && d.amg_kind == SEM_COARSE_KCYCLE) || (fine && tc_active(d)));
  PROF(h, "psum", sem::launch_psum(d, mode, r, z, pcg && !flex, h->stream));
  if (learned) {
    // z = P r + N(r - A P r), flexible PCG; the operator application and the network skip
    // once the correction is switched off (d.st_nn->done), the combine keeps the dots. The
    // network's input needs no FP64: the FP32 operator runs whenever its factors exist.
    if (d.fp32 || d.recompute || d.geo32 != nullptr) {
      float* wl = reinterpret_cast<float*>(d.wl);
      PROF(h, "ax_local_flex", sem::launch_ax_local_f32(d, z, wl, d.st_nn, h->stream));
      PROF(h, "nn_residual", sem::launch_residual_of_f32(d, wl, r, d.nns, st, h->stream));
    } else {
      PROF(h, "ax_local_flex", sem::launch_ax_local(d, z, d.wl, d.st_nn, h->stream));
      PROF(h, "nn_residual", sem::launch_residual_of(d, d.wl, r, d.nns, st, h->stream));
    }
    PROF(h, "nn_correction", sem::learned_correction(h, d.nns, st, h->stream));
  }
  if (flex) PROF(h, "flex_combine", sem::launch_flex_combine(d, z, r, h->stream));
  return SEM_OK;
}

}  // namespace

static int create_impl(sem_t* h, const double* vert_xyz_host, int64_t n_vert, const int64_t* hex2vert_host,
                       int64_t n_hex, int order, double lambda, int flags);

int sem::report_error(int code, const std::string& msg) { return fail(code, msg); }

extern "C" {

const char* sem_last_error(void) { return g_err.c_str(); }

int sem_create(const double* vert_xyz_host, int64_t n_vert, const int64_t* hex2vert_host, int64_t n_hex,
               int order, double lambda, int flags, void* cuda_stream, sem_t** out) {
  g_err.clear();
  if (out == nullptr) return fail(SEM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (vert_xyz_host == nullptr || hex2vert_host == nullptr) return fail(SEM_ERR_ARG, "NULL mesh array");
  if (n_vert < 8 || n_hex < 1) return fail(SEM_ERR_ARG, "empty mesh");
  if (order < 2 || order > 8) return fail(SEM_ERR_ARG, "order must be in 2..8");
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) return fail(SEM_ERR_ARG, "lambda must be finite and >= 0");
  if (flags & ~(SEM_GEOM_RECOMPUTE | SEM_NEUMANN | SEM_MIXED | SEM_PATCH_FULL)) return fail(SEM_ERR_ARG, "unknown flag");
  for (int64_t i = 0; i < 3 * n_vert; ++i)
    if (!std::isfinite(vert_xyz_host[i])) return fail(SEM_ERR_ARG, "non-finite vertex coordinate");

  sem_t* h = new sem_t();
  h->stream = (cudaStream_t)cuda_stream;
  h->flags = flags;
  int rc = create_impl(h, vert_xyz_host, n_vert, hex2vert_host, n_hex, order, lambda, flags);
  if (rc != SEM_OK) {
    sem_destroy(h);
    return rc;
  }
  *out = h;
  return SEM_OK;
}

int sem_selfcheck_convert(const uint64_t* bits_dev, int64_t n, int64_t* mismatches_host) {
  if (n < 0 || (n > 0 && bits_dev == nullptr) || mismatches_host == nullptr)
    return fail(SEM_ERR_ARG, "bad arguments");
  unsigned long long* cnt = nullptr;
  if (cudaMalloc((void**)&cnt, sizeof(unsigned long long)) != cudaSuccess) return fail(SEM_ERR_OOM, "cudaMalloc failed");
  unsigned long long host = 0;
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(host), 0);
  if (e == cudaSuccess)
    e = sem::launch_convert_check(reinterpret_cast<const unsigned long long*>(bits_dev), (long long)n, cnt, 0);
  if (e == cudaSuccess) e = cudaMemcpy(&host, cnt, sizeof(host), cudaMemcpyDeviceToHost);
  cudaFree(cnt);
  if (e != cudaSuccess) return fail(SEM_ERR_CUDA, cudaGetErrorString(e));
  *mismatches_host = (int64_t)host;
  return SEM_OK;
}

int sem_profile(sem_t* h, int enable) {
  if (int rc = check_handle(h)) return rc;
  CK(cudaStreamSynchronize(h->stream));
  h->prof.reset();
  h->prof.on = enable != 0;
  return SEM_OK;
}

int sem_profile_read(sem_t* h, int max_kernels, char* names_host, int64_t* launches_host, double* total_ms_host,
                     int* n_kernels_host) {
  if (int rc = check_handle(h)) return rc;
  if (n_kernels_host == nullptr || max_kernels < 0) return fail(SEM_ERR_ARG, "bad profile arguments");
  CK(cudaStreamSynchronize(h->stream));
  h->prof.collect();
  const int nk = (int)h->prof.names.size();
  *n_kernels_host = nk;
  for (int i = 0; i < nk && i < max_kernels; ++i) {
    if (names_host) {
      std::strncpy(names_host + 64 * i, h->prof.names[i].c_str(), 63);
      names_host[64 * i + 63] = 0;
    }
    if (launches_host) launches_host[i] = h->prof.launches[i];
    if (total_ms_host) total_ms_host[i] = h->prof.total_ms[i];
  }
  return SEM_OK;
}

}  // extern "C"

static int create_impl(sem_t* h, const double* vert_xyz_host, int64_t n_vert, const int64_t* hex2vert_host,
                       int64_t n_hex, int order, double lambda, int flags) {
  auto bail = [&](int code) { return code; };

  std::string err = sem::number_mesh(vert_xyz_host, n_vert, hex2vert_host, n_hex, order, h->nb);
  if (!err.empty()) return bail(fail(err.find("range") != std::string::npos || err.find("repeated") != std::string::npos
                                         ? SEM_ERR_ARG : SEM_ERR_MESH, err));
  const sem::Numbering& nb = h->nb;
  const int n = order, p = n + 1, P = n + 3;
  const int64_t p3 = (int64_t)p * p * p, P3 = (int64_t)P * P * P;
  std::vector<double> t, rho;
  sem::gll(n, t, rho);
  std::vector<double> D = sem::derivative_matrix(n, t);
  std::vector<int> g2l_off, g2l_idx, owner;
  sem::gather_csr(nb, g2l_off, g2l_idx, owner);
  std::vector<int> ip = sem::patch_table(nb, (flags & SEM_PATCH_FULL) != 0);
  std::vector<int> pg_off(nb.G + 1, 0), pg_idx;
  for (size_t q = 0; q < ip.size(); ++q)
    if (ip[q] >= 0) pg_off[ip[q] + 1]++;
  for (int64_t g = 0; g < nb.G; ++g) pg_off[g + 1] += pg_off[g];
  pg_idx.resize(pg_off[nb.G]);
  {
    std::vector<int> fill(pg_off.begin(), pg_off.end() - 1);
    for (size_t q = 0; q < ip.size(); ++q)
      if (ip[q] >= 0) pg_idx[fill[ip[q]]++] = (int)q;
  }
  std::vector<double> S, ev;
  sem::pencil_tables(n, t, rho, D, S, ev);
  std::vector<double> hbox = sem::box_sizes(nb, vert_xyz_host);
  std::vector<double> coords = sem::dof_coords(nb, vert_xyz_host, t, owner);
  std::vector<double> exyz(24 * nb.ne);
  for (int64_t e = 0; e < nb.ne; ++e)
    for (int c = 0; c < 8; ++c)
      for (int a = 0; a < 3; ++a) exyz[24 * e + 3 * c + a] = vert_xyz_host[3 * nb.hexv[8 * e + c] + a];
  // Vandermonde B_{IJK,ijk} = Phi_I(t_i) Phi_J(t_j) Phi_K(t_k) (Sec. 4.1), node-major
  std::vector<double> Btab(8 * p3);
  for (int k = 0; k < p; ++k)
    for (int j = 0; j < p; ++j)
      for (int i = 0; i < p; ++i)
        for (int c = 0; c < 8; ++c) {
          auto phi = [](int bit, double x) { return bit ? 0.5 * (1.0 + x) : 0.5 * (1.0 - x); };
          Btab[8 * (i + p * (j + p * k)) + c] = phi(sem::kCornerBits[c][0], t[i]) * phi(sem::kCornerBits[c][1], t[j]) *
                                                 phi(sem::kCornerBits[c][2], t[k]);
        }
  h->mask_host.assign(nb.G, 0);
  if (!(flags & SEM_NEUMANN)) h->mask_host = nb.boundary;

  {
    int lo = 0, hi = 0;
    CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    CK(cudaStreamCreateWithPriority(&h->coarse_stream, cudaStreamNonBlocking, hi));
    CK(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  }
  sem::DevProblem& d = h->d;
  d.n = n; d.p = p; d.P = P;
  d.ne = (int)nb.ne; d.G = (int)nb.G; d.nv = (int)nb.nv; d.Gi = (int)nb.Gi;
  d.lambda = lambda;
  d.recompute = (flags & SEM_GEOM_RECOMPUTE) != 0;
  auto& A = h->allocs;
#define UP(field, vec, T) do { T* q_; CK(h->upload(&q_, vec, A)); d.field = q_; } while (0)
  UP(l2g, nb.l2g, int);
  UP(exyz, exyz, double);
  UP(D, D, double);
  UP(tg, t, double);
  UP(rho, rho, double);
  UP(g2l_off, g2l_off, int);
  UP(g2l_idx, g2l_idx, int);
  UP(owner, owner, int);
  UP(ip, ip, int);
  UP(pg_off, pg_off, int);
  UP(pg_idx, pg_idx, int);
  {
    // overlap weights c^-1/2 of P^f (used when sem_set_weights turns them on)
    std::vector<double> w(nb.G);
    std::vector<float> w32(nb.G);
    for (int64_t g = 0; g < nb.G; ++g) {
      const int c = pg_off[g + 1] - pg_off[g];
      w[g] = 1.0 / std::sqrt((double)(c > 0 ? c : 1));
      w32[g] = (float)w[g];
    }
    CK(h->upload(&h->pw, w, A));
    CK(h->upload(&h->pw32, w32, A));
  }
  UP(S, S, double);
  UP(ev, ev, double);
  {
    // pencils of element sides on a natural boundary: free low, free high, free both
    std::vector<double> Sv, evv;
    for (int v = 1; v <= 3; ++v) {
      std::vector<double> Sk, ek;
      sem::pencil_variant_tables(n, rho, D, (v & 1) != 0, (v & 2) != 0, Sk, ek);
      Sv.insert(Sv.end(), Sk.begin(), Sk.end());
      evv.insert(evv.end(), ek.begin(), ek.end());
    }
    UP(Sv, Sv, double);
    UP(evv, evv, double);
  }
  UP(hbox, hbox, double);
  UP(Btab, Btab, double);
  {
    std::vector<float> phi32(2 * p);
    for (int i = 0; i < p; ++i) {
      phi32[2 * i] = (float)(0.5 * (1.0 - t[i]));
      phi32[2 * i + 1] = (float)(0.5 * (1.0 + t[i]));
    }
    UP(phi32, phi32, float);
    std::vector<sem::dw> phi(2 * p);
    for (int i = 0; i < p; ++i) {
      phi[2 * i] = sem::dw_split_host(0.5 * (1.0 - t[i]));
      phi[2 * i + 1] = sem::dw_split_host(0.5 * (1.0 + t[i]));
    }
    UP(phidw, phi, sem::dw);
    std::vector<sem::dw> w3((size_t)p * p * p);
    for (int k = 0; k < p; ++k)
      for (int j = 0; j < p; ++j)
        for (int i = 0; i < p; ++i) w3[i + p * (j + p * k)] = sem::dw_split_host(rho[i] * rho[j] * rho[k]);
    UP(w3dw, w3, sem::dw);
  }
#undef UP
  CK(h->upload(&h->coords, coords, A));
  CK(h->upload(&h->mask, h->mask_host, A));
  d.mask = h->mask;
  CK(h->alloc(&h->pvar, (size_t)nb.ne, A));
  CK(h->alloc(&h->swd, (size_t)(nb.ne * P3), A));
  CK(h->alloc(&h->swd32, (size_t)(nb.ne * P3), A));
  CK(h->alloc(&h->swddw, (size_t)(nb.ne * P3), A));
  d.dwk = true;   // SEM_PREC_FP64 (the default) runs its element kernels in double-FP32
  if (int rc = update_free_sides(h)) return rc;
  CK(h->alloc(&d.wl, (size_t)(nb.ne * p3), A));
  CK(h->alloc(&d.wp, (size_t)(nb.ne * P3), A));
  CK(h->alloc(&d.Re, (size_t)(8 * nb.ne), A));
  CK(h->alloc(&h->mN, (size_t)nb.G, A));
  d.nblk = (int)std::min<int64_t>((nb.G + sem::kVecBlock - 1) / sem::kVecBlock, 152 * 8);
  if (d.nblk < 1) d.nblk = 1;
  CK(h->alloc(&d.partial, (size_t)(4 * d.nblk), A));
  CK(h->alloc(&d.st, 1, A));
  CK(cudaMemsetAsync(d.st, 0, sizeof(sem::PcgState), h->stream));
  CK(h->alloc(&d.wait_err, 1, A));
  CK(cudaMemsetAsync(d.wait_err, 0, sizeof(int), h->stream));
  CK(h->alloc(&h->r, (size_t)nb.G, A));
  CK(h->alloc(&h->z, (size_t)nb.G, A));
  CK(h->alloc(&h->p, (size_t)nb.G, A));
  CK(h->alloc(&h->f, (size_t)nb.G, A));
  CK(h->alloc(&h->u, (size_t)nb.G, A));
  CK(h->alloc(&d.p32, (size_t)nb.G, A));
  CK(h->alloc(&d.r32, (size_t)nb.G, A));
  {
    cudaError_t e = cudaMallocHost((void**)&h->st_host, sizeof(sem::PcgState));
    if (e != cudaSuccess) return bail(fail(SEM_ERR_OOM, "cudaMallocHost failed"));
  }

  // geometric factors (stored variant) and the assembled lumped mass
  if (!d.recompute) CK(h->alloc(&h->geo, (size_t)(7 * nb.ne * p3), A));
  if (!d.recompute) CK(h->alloc(&h->geodw, (size_t)(7 * nb.ne * p3), A));
  if (!d.recompute && (flags & SEM_MIXED)) {
    CK(h->alloc(&h->geo32, (size_t)(7 * nb.ne * p3), A));
    CK(h->alloc(&h->geo16, (size_t)(7 * nb.ne * p3), A));
  }
  d.geo = h->geo;
  d.geo32 = h->geo32;
  d.geo16 = h->geo16;
  int* bad;
  CK(h->alloc(&bad, 1, A));
  CK(cudaMemsetAsync(bad, 0, sizeof(int), h->stream));
  CK(sem::launch_geometry(d, h->geo, h->geo32, h->geo16, d.wl, bad, h->stream));
  CK(sem::launch_gather_plain(d, d.wl, h->mN, h->stream));
  if (h->geodw != nullptr) CK(sem::launch_split_pairs((long long)7 * nb.ne * p3, h->geo, h->geodw, h->stream));
  d.geodw = h->geodw;
  int bad_host = 0;
  CK(cudaMemcpyAsync(&bad_host, bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (bad_host) return bail(fail(SEM_ERR_JACOBIAN, "non-positive Jacobian at a GLL node"));

  h->A0full = sem::coarse_matrix(nb, vert_xyz_host, lambda);
  return build_coarse(h);
}

extern "C" {

void sem_destroy(sem_t* h) {
  if (h == nullptr) return;
  {
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    if (std::find(g_batch.handles.begin(), g_batch.handles.end(), h) != g_batch.handles.end()) g_batch.reset();
  }
  cudaStreamSynchronize(h->stream);
  if (h->coarse_stream) {
    cudaStreamSynchronize(h->coarse_stream);
    cudaStreamDestroy(h->coarse_stream);
  }
  h->invalidate();
  if (h->capture_stream) {
    cudaStreamSynchronize(h->capture_stream);
    cudaStreamDestroy(h->capture_stream);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  h->free_list(h->coarse_allocs);
  h->free_list(h->nn_allocs);
  h->free_list(h->allocs);
  if (h->hist) cudaFree(h->hist);
  if (h->st_host) cudaFreeHost(h->st_host);
  delete h;
}

int sem_set_stream(sem_t* h, void* cuda_stream) {
  if (int rc = check_handle(h)) return rc;
  h->stream = (cudaStream_t)cuda_stream;
  return SEM_OK;
}

int sem_num_dofs(const sem_t* h, int64_t* n_dof_host) {
  if (int rc = check_handle(h)) return rc;
  if (n_dof_host == nullptr) return fail(SEM_ERR_ARG, "NULL output");
  *n_dof_host = h->nb.G;
  return SEM_OK;
}

int sem_num_elements(const sem_t* h, int64_t* n_hex_host) {
  if (int rc = check_handle(h)) return rc;
  if (n_hex_host == nullptr) return fail(SEM_ERR_ARG, "NULL output");
  *n_hex_host = h->nb.ne;
  return SEM_OK;
}

int sem_dof_coords(const sem_t* h, double* xyz_dev) {
  if (int rc = check_handle(h)) return rc;
  if (xyz_dev == nullptr) return fail(SEM_ERR_ARG, "NULL output");
  CK(cudaMemcpyAsync(xyz_dev, h->coords, sizeof(double) * 3 * h->nb.G, cudaMemcpyDeviceToDevice, h->stream));
  return SEM_OK;
}

int sem_mass(const sem_t* h, double* m_dev) {
  if (int rc = check_handle(h)) return rc;
  if (m_dev == nullptr) return fail(SEM_ERR_ARG, "NULL output");
  CK(cudaMemcpyAsync(m_dev, h->mN, sizeof(double) * h->nb.G, cudaMemcpyDeviceToDevice, h->stream));
  return SEM_OK;
}

int sem_get_mask(const sem_t* h, uint8_t* mask_dev) {
  if (int rc = check_handle(h)) return rc;
  if (mask_dev == nullptr) return fail(SEM_ERR_ARG, "NULL output");
  CK(cudaMemcpyAsync(mask_dev, h->mask, h->nb.G, cudaMemcpyDeviceToDevice, h->stream));
  return SEM_OK;
}

int sem_boundary_mask(const sem_t* h, uint8_t* mask_dev) { return sem_get_mask(h, mask_dev); }

int sem_apply_mass(const sem_t* h, const double* s_dev, double* b_dev) {
  if (int rc = check_handle(h)) return rc;
  if (s_dev == nullptr || b_dev == nullptr) return fail(SEM_ERR_ARG, "NULL vector");
  CK(sem::launch_mass_load(h->d, h->mN, s_dev, b_dev, h->stream));
  return SEM_OK;
}

int sem_coarse_levels(const sem_t* h, int max_levels, int64_t* sizes_host, int* n_levels_host) {
  if (int rc = check_handle(h)) return rc;
  if (n_levels_host == nullptr || max_levels < 0 || (max_levels > 0 && sizes_host == nullptr))
    return fail(SEM_ERR_ARG, "bad output arguments");
  if (!h->coarse_ok || h->d.nfree == 0) {
    *n_levels_host = 0;
    return SEM_OK;
  }
  std::vector<int64_t> sz;
  for (const auto& L : h->levels) sz.push_back(L.A.n);
  sz.push_back(h->d.coarsest_n);
  for (int i = 0; i < (int)sz.size() && i < max_levels; ++i) sizes_host[i] = sz[i];
  *n_levels_host = (int)sz.size();
  return SEM_OK;
}

int sem_set_mask(sem_t* h, const uint8_t* mask_dev) {
  if (int rc = check_handle(h)) return rc;
  if (mask_dev == nullptr) return fail(SEM_ERR_ARG, "NULL mask");
  std::vector<uint8_t> m(h->nb.G);
  CK(cudaMemcpyAsync(m.data(), mask_dev, h->nb.G, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (auto& v : m) v = v ? 1 : 0;
  h->mask_host = m;
  CK(cudaMemcpyAsync(h->mask, h->mask_host.data(), h->nb.G, cudaMemcpyHostToDevice, h->stream));
  if (int rc = update_free_sides(h)) return rc;
  return build_coarse(h);
}

// SEM_ERR_CUDA (and the flag cleared) when a kernel's bounded wait on a barrier ran out since
// the last check; the caller has synchronised the handle's stream.
static int take_wait_error(sem_t* h) {
  int err = 0;
  CK(cudaMemcpy(&err, h->d.wait_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    CK(cudaMemset(h->d.wait_err, 0, sizeof(int)));
    return fail(SEM_ERR_CUDA, "a kernel gave up a bounded wait on a barrier (tensor-core MMAs or bulk copies)");
  }
  return SEM_OK;
}

int sem_status(sem_t* h) {
  if (int rc = check_handle(h)) return rc;
  CK(cudaStreamSynchronize(h->stream));
  return take_wait_error(h);
}

int sem_apply_A(sem_t* h, const double* x_dev, double* y_dev) {
  if (int rc = check_handle(h)) return rc;
  if (x_dev == nullptr || y_dev == nullptr || x_dev == y_dev) return fail(SEM_ERR_ARG, "bad vector arguments");
  // the element kernel writes the interior DOFs of y itself; the gather sums the rest
  if (h->d.fp32) {
    float* wl = reinterpret_cast<float*>(h->d.wl);
    PROF(h, "ax_local", sem::launch_ax_apply_f32(h->d, x_dev, wl, y_dev, h->stream));
    PROF(h, "gather", sem::launch_gather_shared_f32(h->d, wl, x_dev, y_dev, h->stream));
  } else {
    PROF(h, "ax_local", sem::launch_ax_apply(h->d, x_dev, h->d.wl, y_dev, h->stream));
    PROF(h, "gather", sem::launch_gather_shared(h->d, h->d.wl, x_dev, y_dev, h->stream));
  }
  return SEM_OK;
}

int sem_apply_A_f32(sem_t* h, const float* x_dev, float* y_dev) {
  if (int rc = check_handle(h)) return rc;
  if (x_dev == nullptr || y_dev == nullptr || (const void*)x_dev == (const void*)y_dev)
    return fail(SEM_ERR_ARG, "bad vector arguments");
  if (!h->d.recompute && h->geo32 == nullptr)
    return fail(SEM_ERR_ARG, "FP32 with stored geometry needs SEM_MIXED at sem_create");
  float* wl = reinterpret_cast<float*>(h->d.wl);
  PROF(h, "ax_local", sem::launch_ax_apply_f32io(h->d, x_dev, wl, y_dev, h->stream));
  PROF(h, "gather", sem::launch_gather_shared_f32io(h->d, wl, x_dev, y_dev, h->stream));
  return SEM_OK;
}

static int apply_P_common(sem_t* h, int which, const double* r_dev, double* z_dev) {
  if (int rc = check_handle(h)) return rc;
  if (r_dev == nullptr || z_dev == nullptr || r_dev == z_dev) return fail(SEM_ERR_ARG, "bad vector arguments");
  return apply_precond(h, which, r_dev, z_dev, false);
}

int sem_apply_P(sem_t* h, const double* r_dev, double* z_dev) {
  return apply_P_common(h, SEM_PRECOND_TWO_SCALE, r_dev, z_dev);
}
int sem_apply_Pf(sem_t* h, const double* r_dev, double* z_dev) {
  return apply_P_common(h, SEM_PRECOND_FINE, r_dev, z_dev);
}
int sem_apply_Pc(sem_t* h, const double* r_dev, double* z_dev) { return apply_P_common(h, -1, r_dev, z_dev); }

int sem_net_pair(sem_t* h, const double* b_dev, const double* x_star_dev, const double* x_k_dev, double* s_dev,
                 double* delta_dev, double* r_dev, double* z0_dev) {
  if (int rc = check_handle(h)) return rc;
  if (!b_dev || !x_star_dev || !x_k_dev || !s_dev || !delta_dev || s_dev == delta_dev)
    return fail(SEM_ERR_ARG, "bad vector arguments");
  for (const double* in : {b_dev, x_star_dev, x_k_dev})
    if (in == s_dev || in == delta_dev || in == r_dev || in == z0_dev)
      return fail(SEM_ERR_ARG, "outputs must not alias inputs");
  if ((r_dev && (r_dev == s_dev || r_dev == delta_dev || r_dev == z0_dev)) ||
      (z0_dev && (z0_dev == s_dev || z0_dev == delta_dev)))
    return fail(SEM_ERR_ARG, "outputs must not alias each other");
  sem::DevProblem& d = h->d;
  cudaStream_t s = h->stream;
  double* r = h->f;    // solver scratch, free between solves
  double* z0 = h->z;
  float* wl32 = reinterpret_cast<float*>(d.wl);
  // r = b - A x_k
  if (d.fp32) {
    PROF(h, "ax_local", sem::launch_ax_local_f32(d, x_k_dev, wl32, nullptr, s));
    PROF(h, "nn_residual", sem::launch_residual_of_f32(d, wl32, b_dev, r, nullptr, s));
  } else {
    PROF(h, "ax_local", sem::launch_ax_local(d, x_k_dev, d.wl, nullptr, s));
    PROF(h, "nn_residual", sem::launch_residual_of(d, d.wl, b_dev, r, nullptr, s));
  }
  // z0 = P r, s = r - A z0, delta = x_star - x_k - z0
  if (int rc = apply_precond(h, h->precond, r, z0, false)) return rc;
  if (d.fp32) {
    PROF(h, "ax_local", sem::launch_ax_local_f32(d, z0, wl32, nullptr, s));
    PROF(h, "nn_residual", sem::launch_residual_of_f32(d, wl32, r, s_dev, nullptr, s));
  } else {
    PROF(h, "ax_local", sem::launch_ax_local(d, z0, d.wl, nullptr, s));
    PROF(h, "nn_residual", sem::launch_residual_of(d, d.wl, r, s_dev, nullptr, s));
  }
  PROF(h, "nn_pair", sem::launch_pair_delta(d, x_star_dev, x_k_dev, z0, delta_dev, s));
  if (r_dev) CK(cudaMemcpyAsync(r_dev, r, sizeof(double) * h->nb.G, cudaMemcpyDeviceToDevice, s));
  if (z0_dev) CK(cudaMemcpyAsync(z0_dev, z0, sizeof(double) * h->nb.G, cudaMemcpyDeviceToDevice, s));
  return SEM_OK;
}

int sem_set_precision(sem_t* h, int precision) {
  if (int rc = check_handle(h)) return rc;
  if (precision != SEM_PREC_FP64 && precision != SEM_PREC_FP32 && precision != SEM_PREC_P32 &&
      precision != SEM_PREC_BF16 && precision != SEM_PREC_FP64_NATIVE)
    return fail(SEM_ERR_ARG, "unknown precision");
  if (precision == SEM_PREC_FP32 && !h->d.recompute && h->geo32 == nullptr)
    return fail(SEM_ERR_ARG, "FP32 with stored geometry needs SEM_MIXED at sem_create");
  if (precision == SEM_PREC_BF16 && (h->d.recompute || h->geo16 == nullptr))
    return fail(SEM_ERR_ARG, "BF16 needs stored geometry and SEM_MIXED at sem_create");
  h->precision = precision;
  h->d.fp32 = (precision == SEM_PREC_FP32 || precision == SEM_PREC_BF16);
  h->d.pfp32 = (precision != SEM_PREC_FP64 && precision != SEM_PREC_FP64_NATIVE);
  h->d.bf16 = (precision == SEM_PREC_BF16);
  // every FP64 element kernel (operator with stored factors, patch solve, the mixed path's
  // residual replacement) runs in double-FP32 unless binary64 is asked for
  h->d.dwk = (precision != SEM_PREC_FP64_NATIVE);
  return SEM_OK;
}

int sem_set_overlap(sem_t* h, int reserve_sms) {
  if (int rc = check_handle(h)) return rc;
  if (reserve_sms < 0 || reserve_sms > 1024) return fail(SEM_ERR_ARG, "reserve_sms out of range");
  h->overlap_sms = reserve_sms;
  h->invalidate();
  return SEM_OK;
}

int sem_set_patch_solver(sem_t* h, int kind) {
  if (int rc = check_handle(h)) return rc;
  if (kind != SEM_PATCH_SOLVE_FP32 && kind != SEM_PATCH_SOLVE_BF16_TC) return fail(SEM_ERR_ARG, "unknown patch solver");
  CK(cudaStreamSynchronize(h->stream));
  if (kind == SEM_PATCH_SOLVE_BF16_TC && h->d.rprev == nullptr) CK(h->alloc(&h->d.rprev, (size_t)h->nb.G, h->allocs));
  h->d.tc = kind == SEM_PATCH_SOLVE_BF16_TC;
  h->invalidate();
  return SEM_OK;
}

int sem_set_weights(sem_t* h, int weighted) {
  if (int rc = check_handle(h)) return rc;
  CK(cudaStreamSynchronize(h->stream));
  h->d.pw = weighted ? h->pw : nullptr;
  h->d.pw32 = weighted ? h->pw32 : nullptr;
  h->invalidate();
  return SEM_OK;
}

int sem_set_loop(sem_t* h, int mode) {
  if (int rc = check_handle(h)) return rc;
  if (mode != SEM_LOOP_HOST && mode != SEM_LOOP_DEVICE && mode != SEM_LOOP_EAGER)
    return fail(SEM_ERR_ARG, "unknown loop mode");
  h->loop_mode = mode;
  return SEM_OK;
}

int sem_set_coarse_solver(sem_t* h, int kind) {
  if (int rc = check_handle(h)) return rc;
  if (kind != SEM_COARSE_VCYCLE && kind != SEM_COARSE_KCYCLE) return fail(SEM_ERR_ARG, "unknown coarse solver");
  if (kind == h->amg_kind) return SEM_OK;
  h->amg_kind = kind;
  return build_coarse(h);
}

int sem_set_precond(sem_t* h, int which) {
  if (int rc = check_handle(h)) return rc;
  if (which < SEM_PRECOND_TWO_SCALE || which > SEM_PRECOND_NONE) return fail(SEM_ERR_ARG, "unknown preconditioner");
  h->precond = which;
  return SEM_OK;
}

}  // extern "C"

namespace {

// One PCG solve split into steps, so that sem_solve and sem_solve_many share them:
// begin (initial residual, preconditioner, first operator application, iteration graph),
// advance (read the device state; residual replacement if asked; replay the iteration
// graph), finish (true residual, copy out).
struct SolveCtx {
  const double* b = nullptr;
  double* x = nullptr;
  bool graph_pending = false;   // a replay whose profiling events are unread
  bool done = false;
  int rc = SEM_OK;
};

int ensure_hist(sem_t* h, int maxit) {
  if (maxit + 1 > h->hist_cap) {
    h->invalidate();
    if (h->hist) cudaFree(h->hist);
    h->hist = nullptr;
    h->hist_cap = 0;
    const int cap = std::max(maxit + 1, 1024);
    CK(cudaMalloc((void**)&h->hist, sizeof(double) * cap * h->kcap));
    h->hist_cap = cap;
  }
  return SEM_OK;
}

// The steps of Algorithm 1 as enqueue functions; work goes to h->stream (switched to the
// capture stream while capturing).
// Operator, alpha and update of one iteration, with the stop test on the device.
int enqueue_head(sem_t* h) {
  sem::DevProblem& d = h->d;
  cudaStream_t q = h->stream;
  if (d.fp32)
    PROF(h, "ax_local", sem::launch_ax_local_f32_in32(d, d.p32, reinterpret_cast<float*>(d.wl), d.st, q));
  else
    PROF(h, "ax_local", sem::launch_ax_local(d, h->p, d.wl, d.st, q));
  PROF(h, "pcg_gather_alpha", sem::launch_pcg_gather_alpha(d, h->p, h->f, q));
  PROF(h, "pcg_update", sem::launch_pcg_update(d, h->p, h->f, h->u, h->r, h->hist, q));
  return SEM_OK;
}

// Preconditioner and new direction, then the next iteration's head.
int enqueue_tail_head(sem_t* h) {
  if (int rc = apply_precond(h, h->precond, h->r, h->z, true)) return rc;
  PROF(h, "pcg_direction", sem::launch_pcg_direction(h->d, h->z, h->p, h->stream));
  return enqueue_head(h);
}

// Initial residual, preconditioner, first direction and the first head.
int enqueue_start(sem_t* h, const double* b, double rtol, int maxit) {
  sem::DevProblem& d = h->d;
  cudaStream_t s = h->stream;
  CK(cudaMemsetAsync(d.st, 0, sizeof(sem::PcgState) * d.nrhs, s));
  const int mixed = d.fp32 ? 1 : 0;
  const int learned = h->net != nullptr ? 1 : 0;
  const bool fine = h->precond == SEM_PRECOND_TWO_SCALE || h->precond == SEM_PRECOND_FINE;
  const int flexible = (learned || (d.amg_kind == SEM_COARSE_KCYCLE && h->precond == SEM_PRECOND_TWO_SCALE) ||
                        (fine && tc_active(d))) ? 1 : 0;
  if (learned) CK(cudaMemsetAsync(d.st_nn, 0, sizeof(sem::PcgState), s));
  PROF(h, "pcg_init", sem::launch_pcg_init(d, b, h->r, h->u, rtol, maxit, mixed, learned, flexible, h->nn_window,
                                           h->nn_ratio, h->nn_theta, h->hist, s));
  if (int rc = apply_precond(h, h->precond, h->r, h->z, true)) return rc;
  PROF(h, "pcg_direction", sem::launch_pcg_first_direction(d, h->z, h->p, s));
  return enqueue_head(h);
}

// Mixed path: the recursive residual replaced by b - A u with the FP64 operator.
int enqueue_replacement(sem_t* h, const double* b) {
  sem::DevProblem& d = h->d;
  PROF(h, "ax_local_fp64", sem::launch_ax_local(d, h->u, d.wl, d.st, h->stream));
  PROF(h, "pcg_replace", sem::launch_pcg_replace(d, b, d.wl, h->r, h->hist, h->stream));
  return SEM_OK;
}

// Configuration bits the captured graphs depend on.
long graph_key(const sem_t* h) {
  const sem::DevProblem& d = h->d;
  return (long)(d.fp32 ? 1 : 0) | ((long)(d.pfp32 ? 1 : 0) << 15) | ((long)h->precond << 1) | ((long)h->prof.on << 3) |
         ((long)d.epb_ax << 4) |
         ((long)d.epb_sw << 8) | ((long)(h->net != nullptr) << 12) | ((long)d.amg_kind << 13) |
         ((long)d.epb_ax32 << 16) | ((long)d.epb_sw32 << 20) | ((long)(d.bf16 ? 1 : 0) << 24) |
         ((long)(d.dwk ? 1 : 0) << 25) | ((long)d.epb_axdw << 26) | ((long)d.epb_swdw << 30) |
         ((long)(tc_active(d) ? 1 : 0) << 34) | ((long)d.nrhs << 35);
}

int solve_begin(sem_t* h, SolveCtx& c, double rtol, int maxit) {
  if (int rc = ensure_hist(h, maxit)) return rc;
  cudaStream_t s = h->stream;
  if (int rc = enqueue_start(h, c.b, rtol, maxit)) return rc;

  // capture the steady-state iteration once per configuration (not in the eager loop)
  const long key = graph_key(h);
  if (h->loop_mode != SEM_LOOP_EAGER && h->graph.key != key) {
    h->graph.reset();
    CK(cudaStreamSynchronize(s));
    if (h->prof.on) h->prof.collect();
    h->prof.cap = h->prof.on ? &h->graph : nullptr;
    cudaGraph_t g = nullptr;
    h->stream = h->capture_stream;
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    int rc = (e == cudaSuccess) ? enqueue_tail_head(h) : SEM_OK;
    cudaError_t e2 = (e == cudaSuccess) ? cudaStreamEndCapture(h->stream, &g) : cudaSuccess;
    h->stream = s;
    h->prof.cap = nullptr;
    if (rc != SEM_OK || e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      h->graph.reset();
      if (rc != SEM_OK) return rc;
      return fail(SEM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&h->graph.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      h->graph.reset();
      return fail(SEM_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    h->graph.key = key;
  }
  c.graph_pending = false;
  c.done = false;
  return SEM_OK;
}

// Enqueue the read-back of the device state (pinned host copy).
int solve_poll(sem_t* h) {
  CK(cudaMemcpyAsync(h->st_host, h->d.st, sizeof(sem::PcgState), cudaMemcpyDeviceToHost, h->stream));
  return SEM_OK;
}

// After the state read-back completed: stop, or replace the residual if asked, and
// replay the iteration graph.
int solve_advance(sem_t* h, SolveCtx& c) {
  sem::DevProblem& d = h->d;
  cudaStream_t s = h->stream;
  CK(cudaStreamSynchronize(s));
  if (c.graph_pending && h->prof.on) h->prof.collect_graph(h->graph);
  c.graph_pending = false;
  if (h->st_host->done) { c.done = true; return SEM_OK; }
  if (d.fp32 && h->st_host->replace) {
    if (int rc = enqueue_replacement(h, c.b)) return rc;
    CK(cudaMemcpyAsync(h->st_host, d.st, sizeof(sem::PcgState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h->st_host->done) { c.done = true; return SEM_OK; }
  }
  if (h->loop_mode == SEM_LOOP_EAGER) return enqueue_tail_head(h);   // the same work, launch by launch
  CK(cudaGraphLaunch(h->graph.exec, s));
  c.graph_pending = true;
  return SEM_OK;
}

int solve_finish(sem_t* h, SolveCtx& c, int* iters_host, double* res_hist_host, double* true_rel_res_host) {
  sem::DevProblem& d = h->d;
  cudaStream_t s = h->stream;
  // true residual ||b - A u|| / ||b|| on the free nodes, and the solution out
  PROF(h, "ax_local", sem::launch_ax_local(d, h->u, d.wl, nullptr, s));
  PROF(h, "true_residual", sem::launch_true_residual(d, c.b, d.wl, s));
  CK(cudaMemcpyAsync(c.x, h->u, sizeof(double) * h->nb.G, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(h->st_host, d.st, sizeof(sem::PcgState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  h->prof.collect();
  const sem::PcgState& st = *h->st_host;
  if (iters_host) *iters_host = st.iter;
  if (res_hist_host) {
    CK(cudaMemcpyAsync(res_hist_host, h->hist, sizeof(double) * (st.iter + 1), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  if (true_rel_res_host) *true_rel_res_host = st.bb > 0 ? std::sqrt(st.aux) / std::sqrt(st.bb) : 0.0;
  if (int rc = take_wait_error(h)) return rc;
  if (st.status == -4) return fail(SEM_ERR_CUDA, "a kernel of the solve gave up a bounded wait");
  if (st.status == -6) return fail(SEM_ERR_NAN, "NaN/Inf or non-positive curvature in PCG");
  if (!st.done) return fail(SEM_MAXIT, "maxit reached");
  return st.status == 1 ? SEM_MAXIT : SEM_OK;
}

// ---- device-driven solve loop --------------------------------------------------------
// Captures fn's work (h->stream switched to the capture stream; the coarse stream joins
// through its events) into graph g after the nodes deps; sinks receives the capture's last
// nodes, for the next node to depend on.
template <class F>
int capture_into(sem_t* h, cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps, F fn,
                 std::vector<cudaGraphNode_t>& sinks) {
  cudaStream_t saved = h->stream;
  h->stream = h->capture_stream;
  cudaError_t e = cudaStreamBeginCaptureToGraph(h->stream, g, deps.empty() ? nullptr : deps.data(), nullptr,
                                                deps.size(), cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    h->stream = saved;
    return fail(SEM_ERR_CUDA, std::string("cudaStreamBeginCaptureToGraph: ") + cudaGetErrorString(e));
  }
  const int rc = fn();
  cudaStreamCaptureStatus status;
  const cudaGraphNode_t* dl = nullptr;
  size_t nd = 0;
  const cudaError_t e1 = cudaStreamGetCaptureInfo(h->stream, &status, nullptr, nullptr, &dl, nullptr, &nd);
  if (e1 == cudaSuccess && dl != nullptr) sinks.assign(dl, dl + nd);
  else sinks.clear();
  cudaGraph_t out = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(h->stream, &out);
  h->stream = saved;
  if (rc != SEM_OK) return rc;
  if (e1 != cudaSuccess || e2 != cudaSuccess)
    return fail(SEM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
  return SEM_OK;
}

int add_conditional(cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps, cudaGraphConditionalHandle hc,
                    cudaGraphConditionalNodeType type, cudaGraphNode_t& node, cudaGraph_t& body) {
  cudaGraphNodeParams prm = {};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = hc;
  prm.conditional.type = type;
  prm.conditional.size = 1;
  CK(cudaGraphAddNode(&node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &prm));
  body = prm.conditional.phGraph_out[0];
  return SEM_OK;
}

// Appends one whole solve of handle h into graph g, independent of the graph's other
// nodes: the initial steps and the first head, then WHILE (not done, at most maxit + 2
// rounds) { preconditioner, direction, head }. The mixed path adds, after each head, an
// IF node with the FP64 residual replacement. The right-hand side is read from h->bbuf.
int build_loop(sem_t* h, cudaGraph_t g, double rtol, int maxit) {
  sem::DevProblem& d = h->d;
  const bool mixed = d.fp32;
  const int limit = maxit + 2;
  std::vector<cudaGraphNode_t> deps, tmp;
  cudaGraphConditionalHandle hw;
  CK(cudaGraphConditionalHandleCreate(&hw, g, 0, 0));
  auto set_loop = [&]() -> int {
    CK(sem::launch_loop_cond(d.st, d.nrhs, h->loop_guard, limit, hw, h->stream));
    return SEM_OK;
  };
  // IF (replacement requested) { FP64 residual replacement } inside graph gg after deps
  auto add_replacement = [&](cudaGraph_t gg, std::vector<cudaGraphNode_t>& dd) -> int {
    cudaGraphConditionalHandle hi;
    CK(cudaGraphConditionalHandleCreate(&hi, gg, 0, 0));
    if (int rc = capture_into(h, gg, dd, [&]() -> int {
          CK(sem::launch_replace_cond(d.st, hi, h->stream));
          return SEM_OK;
        }, dd)) return rc;
    cudaGraphNode_t node;
    cudaGraph_t body;
    if (int rc = add_conditional(gg, dd, hi, cudaGraphCondTypeIf, node, body)) return rc;
    if (int rc = capture_into(h, body, {}, [&]() { return enqueue_replacement(h, h->bbuf); }, tmp)) return rc;
    dd.assign(1, node);
    return SEM_OK;
  };
  if (int rc = capture_into(h, g, {}, [&]() -> int {
        CK(cudaMemsetAsync(h->loop_guard, 0, sizeof(int), h->stream));
        return enqueue_start(h, h->bbuf, rtol, maxit);
      }, deps)) return rc;
  if (mixed)
    if (int rc = add_replacement(g, deps)) return rc;
  if (int rc = capture_into(h, g, deps, set_loop, deps)) return rc;
  cudaGraphNode_t wnode;
  cudaGraph_t wbody;
  if (int rc = add_conditional(g, deps, hw, cudaGraphCondTypeWhile, wnode, wbody)) return rc;
  std::vector<cudaGraphNode_t> bd;
  if (int rc = capture_into(h, wbody, {}, [&]() { return enqueue_tail_head(h); }, bd)) return rc;
  if (mixed)
    if (int rc = add_replacement(wbody, bd)) return rc;
  return capture_into(h, wbody, bd, set_loop, bd);
}

int ensure_loop_buffers(sem_t* h) {
  if (h->bbuf == nullptr) CK(h->alloc(&h->bbuf, (size_t)h->nb.G * h->kcap, h->allocs));
  if (h->loop_guard == nullptr) CK(h->alloc(&h->loop_guard, 1, h->allocs));
  return SEM_OK;
}

// Grows the per-right-hand-side work buffers of the handle to k slices (block solves).
template <class T>
int regrow(sem_t* h, T** ptr, size_t count) {
  if (*ptr != nullptr) {
    auto it = std::find(h->allocs.begin(), h->allocs.end(), (void*)*ptr);
    if (it != h->allocs.end()) h->allocs.erase(it);
    cudaFree(*ptr);
    *ptr = nullptr;
  }
  CK(h->alloc(ptr, count, h->allocs));
  return SEM_OK;
}

int ensure_block(sem_t* h, int k) {
  if (k <= h->kcap) return SEM_OK;
  CK(cudaStreamSynchronize(h->stream));
  sem::DevProblem& d = h->d;
  const size_t G = (size_t)h->nb.G, ne = (size_t)h->nb.ne, kk = (size_t)k;
  const size_t p3 = (size_t)d.p * d.p * d.p, P3 = (size_t)d.P * d.P * d.P;
  h->kcap = k;
  if (int rc = regrow(h, &h->r, G * kk)) return rc;
  if (int rc = regrow(h, &h->z, G * kk)) return rc;
  if (int rc = regrow(h, &h->p, G * kk)) return rc;
  if (int rc = regrow(h, &h->f, G * kk)) return rc;
  if (int rc = regrow(h, &h->u, G * kk)) return rc;
  if (h->bbuf != nullptr)
    if (int rc = regrow(h, &h->bbuf, G * kk)) return rc;
  if (int rc = regrow(h, &d.wl, ne * p3 * kk)) return rc;
  if (int rc = regrow(h, &d.wp, ne * P3 * kk)) return rc;
  if (int rc = regrow(h, &d.Re, ne * 8 * kk)) return rc;
  if (int rc = regrow(h, &d.partial, (size_t)4 * d.nblk * kk)) return rc;
  if (int rc = regrow(h, &d.st, kk)) return rc;
  CK(cudaMemsetAsync(d.st, 0, sizeof(sem::PcgState) * kk, h->stream));
  if (h->st_host) cudaFreeHost(h->st_host);
  h->st_host = nullptr;
  CK(cudaMallocHost((void**)&h->st_host, sizeof(sem::PcgState) * kk));
  if (h->hist) cudaFree(h->hist);   // regrown by ensure_hist for kcap slices
  h->hist = nullptr;
  h->hist_cap = 0;
  return build_coarse(h);   // coarse vectors and AMG level work, kcap slices each
}


int instantiate(cudaGraph_t g, cudaGraphExec_t& exec) {
  cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
  if (e != cudaSuccess) {
    exec = nullptr;
    return fail(SEM_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  }
  return SEM_OK;
}

// One solve as one graph launch (no host round trip per iteration).
int solve_device_loop(sem_t* h, const double* b, double* x, double rtol, int maxit, int* iters_host,
                      double* res_hist_host, double* true_rel_res_host) {
  if (int rc = ensure_hist(h, maxit)) return rc;
  if (int rc = ensure_loop_buffers(h)) return rc;
  const long key = graph_key(h);
  if (h->loop.key != key || h->loop.rtol != rtol || h->loop.maxit != maxit) {
    h->loop.reset();
    CK(cudaStreamSynchronize(h->stream));
    cudaGraph_t g;
    CK(cudaGraphCreate(&g, 0));
    int rc = build_loop(h, g, rtol, maxit);
    if (rc == SEM_OK) rc = instantiate(g, h->loop.exec);
    cudaGraphDestroy(g);
    if (rc != SEM_OK) return rc;
    h->loop.key = key;
    h->loop.rtol = rtol;
    h->loop.maxit = maxit;
  }
  CK(cudaMemcpyAsync(h->bbuf, b, sizeof(double) * h->nb.G, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaGraphLaunch(h->loop.exec, h->stream));
  SolveCtx c;
  c.b = b;
  c.x = x;
  return solve_finish(h, c, iters_host, res_hist_host, true_rel_res_host);
}

bool batch_matches(int count, sem_t* const* hs, double rtol, int maxit) {
  if (g_batch.exec == nullptr || (int)g_batch.handles.size() != count || g_batch.rtol != rtol ||
      g_batch.maxit != maxit)
    return false;
  for (int i = 0; i < count; ++i)
    if (g_batch.handles[i] != hs[i] || g_batch.epochs[i] != hs[i]->epoch || g_batch.keys[i] != graph_key(hs[i]))
      return false;
  return true;
}

// Time `reps` launches of fn on the handle's stream with events (milliseconds per launch).
template <class F>
int time_launches(sem_t* h, F fn, int reps, float* ms_out) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  cudaError_t err = fn();   // warm-up (and validity of the configuration)
  if (err == cudaSuccess) {
    cudaEventRecord(e0, h->stream);
    for (int i = 0; i < reps && err == cudaSuccess; ++i) err = fn();
    cudaEventRecord(e1, h->stream);
    cudaEventSynchronize(e1);
  }
  float ms = 0.f;
  if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  *ms_out = ms / reps;
  return SEM_OK;
}

}  // namespace

extern "C" {

int sem_solve(sem_t* h, const double* b_dev, double* x_dev, double rtol, int maxit, int* iters_host,
              double* res_hist_host, double* true_rel_res_host) {
  if (int rc = check_solvable(h)) return rc;
  if (b_dev == nullptr || x_dev == nullptr || b_dev == x_dev) return fail(SEM_ERR_ARG, "bad vector arguments");
  if (!(rtol >= 0.0) || maxit < 0) return fail(SEM_ERR_ARG, "bad rtol or maxit");
  if (h->loop_mode == SEM_LOOP_DEVICE && !h->prof.on)
    return solve_device_loop(h, b_dev, x_dev, rtol, maxit, iters_host, res_hist_host, true_rel_res_host);
  SolveCtx c;
  c.b = b_dev;
  c.x = x_dev;
  if (int rc = solve_begin(h, c, rtol, maxit)) return rc;
  for (int guard = 0; guard <= maxit + 1 && !c.done; ++guard) {
    if (int rc = solve_poll(h)) return rc;
    if (int rc = solve_advance(h, c)) return rc;
  }
  return solve_finish(h, c, iters_host, res_hist_host, true_rel_res_host);
}

// Checks and buffers of a k-column block solve on h (sem_solve_block, sem_solve_many_block).
static int block_prepare(sem_t* h, int k, const double* b_dev, double* x_dev, int maxit) {
  if (int rc = check_handle(h)) return rc;
  sem::DevProblem& d = h->d;
  if (k < 1 || k > SEM_MAX_BLOCK || b_dev == nullptr || x_dev == nullptr || (const void*)b_dev == (const void*)x_dev)
    return fail(SEM_ERR_ARG, "bad block-solve arguments");
  if (h->precision != SEM_PREC_FP64 && h->precision != SEM_PREC_FP64_NATIVE)
    return fail(SEM_ERR_ARG, "block solves run in SEM_PREC_FP64 or SEM_PREC_FP64_NATIVE");
  if (h->net != nullptr || d.amg_kind == SEM_COARSE_KCYCLE)
    return fail(SEM_ERR_ARG, "block solves take the linear preconditioner (no network, V-cycle coarse solver)");
  if (int rc = check_solvable(h)) return rc;
  if (h->precond != SEM_PRECOND_FINE && h->precond != SEM_PRECOND_NONE &&
      (!h->coarse_ok || (d.nfree == 0 && !h->coarse_err.empty())))
    return fail(SEM_ERR_SINGULAR, "coarse space unavailable: " + h->coarse_err);
  if (int rc = ensure_block(h, k)) return rc;
  if (int rc = ensure_hist(h, maxit)) return rc;
  return ensure_loop_buffers(h);
}

// After a block solve's loop ran (d.nrhs = k): the true residuals ||b_j - A u_j|| and the
// solutions out, every right-hand side at once, then the states read back.
static int block_finish(sem_t* h, int k, double* x_dev, int* iters_host, int* status_host,
                        double* true_rel_res_host) {
  sem::DevProblem& d = h->d;
  cudaStream_t s = h->stream;
  const size_t G = (size_t)h->nb.G;
  PROF(h, "ax_local", sem::launch_ax_local(d, h->u, d.wl, nullptr, s));
  PROF(h, "true_residual", sem::launch_true_residual(d, h->bbuf, d.wl, s));
  CK(cudaMemcpyAsync(x_dev, h->u, sizeof(double) * G * k, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(h->st_host, d.st, sizeof(sem::PcgState) * k, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  h->prof.collect();
  int worst = SEM_OK;
  for (int j = 0; j < k; ++j) {
    const sem::PcgState& st = h->st_host[j];
    int rc = st.status == -6 ? SEM_ERR_NAN : (st.status == -4 ? SEM_ERR_CUDA : (!st.done || st.status == 1 ? SEM_MAXIT : SEM_OK));
    if (iters_host) iters_host[j] = st.iter;
    if (status_host) status_host[j] = rc;
    if (true_rel_res_host) true_rel_res_host[j] = st.bb > 0 ? std::sqrt(st.aux) / std::sqrt(st.bb) : 0.0;
    if (rc < 0 && (worst >= 0 || rc < worst)) worst = rc;
    else if (rc > 0 && worst == SEM_OK) worst = rc;
  }
  if (int rc = take_wait_error(h)) return rc;
  return worst;
}

int sem_solve_block(sem_t* h, int k, const double* b_dev, double* x_dev, double rtol, int maxit, int* iters_host,
                    int* status_host, double* true_rel_res_host) {
  if (int rc = block_prepare(h, k, b_dev, x_dev, maxit)) return rc;
  sem::DevProblem& d = h->d;
  cudaStream_t s = h->stream;
  const size_t G = (size_t)h->nb.G;
  d.nrhs = k;
  d.hist_stride = h->hist_cap;
  struct Restore {
    sem::DevProblem& d;
    ~Restore() { d.nrhs = 1; }
  } restore{d};
  const long key = graph_key(h);
  if (h->loop.key != key || h->loop.rtol != rtol || h->loop.maxit != maxit) {
    h->loop.reset();
    CK(cudaStreamSynchronize(s));
    cudaGraph_t g;
    CK(cudaGraphCreate(&g, 0));
    int rc = build_loop(h, g, rtol, maxit);
    if (rc == SEM_OK) rc = instantiate(g, h->loop.exec);
    cudaGraphDestroy(g);
    if (rc != SEM_OK) return rc;
    h->loop.key = key;
    h->loop.rtol = rtol;
    h->loop.maxit = maxit;
  }
  CK(cudaMemcpyAsync(h->bbuf, b_dev, sizeof(double) * G * k, cudaMemcpyDeviceToDevice, s));
  CK(cudaGraphLaunch(h->loop.exec, s));
  const int worst = block_finish(h, k, x_dev, iters_host, status_host, true_rel_res_host);
  if (worst < 0) return fail(worst, "a right-hand side of the block solve failed (see status_host)");
  return worst;
}

int sem_solve_many_block(int count, sem_t* const* handles, int k, const double* const* b_dev,
                         double* const* x_dev, double rtol, int maxit, int* iters_host, int* status_host) {
  if (count < 0 || (count > 0 && (handles == nullptr || b_dev == nullptr || x_dev == nullptr)))
    return fail(SEM_ERR_ARG, "bad arrays");
  if (!(rtol >= 0.0) || maxit < 0) return fail(SEM_ERR_ARG, "bad rtol or maxit");
  for (int i = 0; i < count; ++i) {
    if (handles[i] == nullptr) return fail(SEM_ERR_ARG, "bad handle at index " + std::to_string(i));
    for (int j = 0; j < i; ++j)
      if (handles[j] == handles[i]) return fail(SEM_ERR_ARG, "a handle appears twice");
    if (int rc = block_prepare(handles[i], k, b_dev[i], x_dev[i], maxit)) return rc;
  }
  if (count == 0) return SEM_OK;
  // every handle's block loop (k right-hand sides) is one branch of one graph, launched once
  std::lock_guard<std::mutex> lock(g_batch_mutex);
  struct Restore {
    int count;
    sem_t* const* hs;
    ~Restore() {
      for (int i = 0; i < count; ++i) hs[i]->d.nrhs = 1;
    }
  } restore{count, handles};
  for (int i = 0; i < count; ++i) {
    handles[i]->d.nrhs = k;
    handles[i]->d.hist_stride = handles[i]->hist_cap;
  }
  if (!batch_matches(count, handles, rtol, maxit)) {
    g_batch.reset();
    cudaGraph_t g;
    CK(cudaGraphCreate(&g, 0));
    int rc = SEM_OK;
    for (int i = 0; i < count && rc == SEM_OK; ++i) {
      cudaStreamSynchronize(handles[i]->stream);
      rc = build_loop(handles[i], g, rtol, maxit);
    }
    if (rc == SEM_OK) rc = instantiate(g, g_batch.exec);
    cudaGraphDestroy(g);
    if (rc != SEM_OK) return rc;
    for (int i = 0; i < count; ++i) {
      g_batch.handles.push_back(handles[i]);
      g_batch.epochs.push_back(handles[i]->epoch);
      g_batch.keys.push_back(graph_key(handles[i]));
    }
    g_batch.rtol = rtol;
    g_batch.maxit = maxit;
  }
  cudaStream_t s0 = handles[0]->stream;
  for (int i = 0; i < count; ++i) {
    sem_t* h = handles[i];
    if (h->stream != s0) CK(cudaStreamSynchronize(h->stream));   // the caller's work on b
    CK(cudaMemcpyAsync(h->bbuf, b_dev[i], sizeof(double) * h->nb.G * k, cudaMemcpyDeviceToDevice, s0));
  }
  CK(cudaGraphLaunch(g_batch.exec, s0));
  CK(cudaStreamSynchronize(s0));
  int worst = SEM_OK;
  for (int i = 0; i < count; ++i) {
    const int rc = block_finish(handles[i], k, x_dev[i], iters_host ? iters_host + (size_t)i * k : nullptr,
                                status_host ? status_host + (size_t)i * k : nullptr, nullptr);
    if (rc < 0 && (worst >= 0 || rc < worst)) worst = rc;
    else if (rc > 0 && worst == SEM_OK) worst = rc;
  }
  if (worst < 0) return fail(worst, "a right-hand side failed (see status_host)");
  return worst;
}

int sem_heat_step(sem_t* h, const double* u_prev_dev, const double* g_dev, double* u_dev, double rtol, int maxit,
                  int* iters_host, double* true_rel_res_host) {
  if (int rc = check_solvable(h)) return rc;
  if (!u_prev_dev || !g_dev || !u_dev || u_dev == g_dev) return fail(SEM_ERR_ARG, "bad vector arguments");
  if (!(rtol >= 0.0) || maxit < 0) return fail(SEM_ERR_ARG, "bad rtol or maxit");
  sem::DevProblem& d = h->d;
  cudaStream_t s = h->stream;
  const size_t G = (size_t)h->nb.G;
  if (h->heat_b == nullptr) {
    CK(h->alloc(&h->heat_b, G, h->allocs));
    CK(h->alloc(&h->heat_d, G, h->allocs));
    CK(h->alloc(&h->heat_norms, 2, h->allocs));
  }
  // b' = M (lambda u_prev + g) - A u_prev with the FP64 operator: the step solves for the
  // increment, so u_prev is the initial guess; the tolerance stays relative to the full
  // right-hand side M (lambda u_prev + g)
  PROF(h, "ax_local_fp64", sem::launch_ax_local(d, u_prev_dev, d.wl, nullptr, s));
  PROF(h, "heat_rhs", sem::launch_heat_rhs(d, d.wl, h->mN, u_prev_dev, g_dev, h->heat_b, h->heat_norms, s));
  double norms[2] = {0.0, 0.0};
  CK(cudaMemcpyAsync(norms, h->heat_norms, sizeof(norms), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (!std::isfinite(norms[0]) || !std::isfinite(norms[1])) return fail(SEM_ERR_NAN, "NaN/Inf in the heat step");
  if (norms[1] == 0.0 || norms[1] <= rtol * rtol * norms[0]) {
    if (u_dev != u_prev_dev) CK(cudaMemcpyAsync(u_dev, u_prev_dev, sizeof(double) * G, cudaMemcpyDeviceToDevice, s));
    if (iters_host) *iters_host = 0;
    if (true_rel_res_host) *true_rel_res_host = norms[0] > 0.0 ? std::sqrt(norms[1] / norms[0]) : 0.0;
    return SEM_OK;
  }
  const double scale = std::sqrt(norms[1] / norms[0]);   // ||b'|| / ||b||
  SolveCtx c;
  c.b = h->heat_b;
  c.x = h->heat_d;
  if (int rc = solve_begin(h, c, rtol / scale, maxit)) return rc;
  for (int guard = 0; guard <= maxit + 1 && !c.done; ++guard) {
    if (int rc = solve_poll(h)) return rc;
    if (int rc = solve_advance(h, c)) return rc;
  }
  double tr = 0.0;
  const int rc = solve_finish(h, c, iters_host, nullptr, &tr);
  if (rc < 0) return rc;
  PROF(h, "heat_update", sem::launch_add_vectors(d, u_prev_dev, h->heat_d, u_dev, s));
  if (true_rel_res_host) *true_rel_res_host = tr * scale;
  return rc;
}

int sem_solve_many(int count, sem_t* const* handles, const double* const* b_dev, double* const* x_dev,
                   double rtol, int maxit, int* iters_host, int* status_host) {
  if (count < 0 || (count > 0 && (handles == nullptr || b_dev == nullptr || x_dev == nullptr)))
    return fail(SEM_ERR_ARG, "bad arrays");
  if (!(rtol >= 0.0) || maxit < 0) return fail(SEM_ERR_ARG, "bad rtol or maxit");
  for (int i = 0; i < count; ++i) {
    if (handles[i] == nullptr || b_dev[i] == nullptr || x_dev[i] == nullptr || b_dev[i] == x_dev[i])
      return fail(SEM_ERR_ARG, "bad handle or vector at index " + std::to_string(i));
    if (int rc = check_solvable(handles[i])) return rc;
    for (int j = 0; j < i; ++j)
      if (handles[j] == handles[i]) return fail(SEM_ERR_ARG, "a handle appears twice");
  }
  std::vector<SolveCtx> ctx(count);
  bool device = count > 0;
  for (int i = 0; i < count; ++i) device = device && handles[i]->loop_mode == SEM_LOOP_DEVICE && !handles[i]->prof.on;
  if (device) {
    // every solve appended to one graph and launched once
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    for (int i = 0; i < count; ++i) {
      if (int rc = ensure_hist(handles[i], maxit)) return rc;
      if (int rc = ensure_loop_buffers(handles[i])) return rc;
    }
    if (!batch_matches(count, handles, rtol, maxit)) {
      g_batch.reset();
      cudaGraph_t g;
      CK(cudaGraphCreate(&g, 0));
      int rc = SEM_OK;
      for (int i = 0; i < count && rc == SEM_OK; ++i) {
        cudaStreamSynchronize(handles[i]->stream);
        rc = build_loop(handles[i], g, rtol, maxit);
      }
      if (rc == SEM_OK) rc = instantiate(g, g_batch.exec);
      cudaGraphDestroy(g);
      if (rc != SEM_OK) return rc;
      for (int i = 0; i < count; ++i) {
        g_batch.handles.push_back(handles[i]);
        g_batch.epochs.push_back(handles[i]->epoch);
        g_batch.keys.push_back(graph_key(handles[i]));
      }
      g_batch.rtol = rtol;
      g_batch.maxit = maxit;
    }
    cudaStream_t s0 = handles[0]->stream;
    for (int i = 0; i < count; ++i) {
      sem_t* h = handles[i];
      if (h->stream != s0) CK(cudaStreamSynchronize(h->stream));   // the caller's work on b
      CK(cudaMemcpyAsync(h->bbuf, b_dev[i], sizeof(double) * h->nb.G, cudaMemcpyDeviceToDevice, s0));
    }
    CK(cudaGraphLaunch(g_batch.exec, s0));
    CK(cudaStreamSynchronize(s0));
    int worst = SEM_OK;
    for (int i = 0; i < count; ++i) {
      ctx[i].b = b_dev[i];
      ctx[i].x = x_dev[i];
      int it = 0;
      const int rc = solve_finish(handles[i], ctx[i], &it, nullptr, nullptr);
      if (iters_host) iters_host[i] = it;
      if (status_host) status_host[i] = rc;
      if (rc < 0) worst = rc;
      else if (rc > 0 && worst == SEM_OK) worst = rc;
    }
    return worst;
  }
  for (int i = 0; i < count; ++i) {
    ctx[i].b = b_dev[i];
    ctx[i].x = x_dev[i];
    if (int rc = solve_begin(handles[i], ctx[i], rtol, maxit)) return rc;
  }
  // every round reads back all active states, then advances each solve on its own stream
  for (int guard = 0; guard <= maxit + 1; ++guard) {
    bool any = false;
    for (int i = 0; i < count; ++i)
      if (!ctx[i].done) {
        if (int rc = solve_poll(handles[i])) return rc;
        any = true;
      }
    if (!any) break;
    for (int i = 0; i < count; ++i)
      if (!ctx[i].done)
        if (int rc = solve_advance(handles[i], ctx[i])) return rc;
  }
  int worst = SEM_OK;
  for (int i = 0; i < count; ++i) {
    int it = 0;
    const int rc = solve_finish(handles[i], ctx[i], &it, nullptr, nullptr);
    if (iters_host) iters_host[i] = it;
    if (status_host) status_host[i] = rc;
    if (rc < 0) worst = rc;
    else if (rc > 0 && worst == SEM_OK) worst = rc;
  }
  return worst;
}

int sem_set_tiles(sem_t* h, int epb_ax, int epb_sw) {
  if (int rc = check_handle(h)) return rc;
  if (!sem::ax_tile_ok(h->d.p, epb_ax) || !sem::sw_tile_ok(h->d.P, epb_sw))
    return fail(SEM_ERR_ARG, "no kernel with that many elements per CTA for this order");
  h->d.epb_ax = h->d.epb_ax32 = epb_ax;
  h->d.epb_sw = h->d.epb_sw32 = h->d.epb_swdw = epb_sw;
  h->invalidate();
  return SEM_OK;
}

int sem_autotune(sem_t* h, int* epb_ax_host, int* epb_sw_host) {
  if (int rc = check_handle(h)) return rc;
  sem::DevProblem& d = h->d;
  CK(cudaMemsetAsync(h->p, 0, sizeof(double) * h->nb.G, h->stream));
  CK(cudaMemsetAsync(h->r, 0, sizeof(double) * h->nb.G, h->stream));
  CK(cudaMemsetAsync(d.p32, 0, sizeof(float) * h->nb.G, h->stream));
  CK(cudaMemsetAsync(d.r32, 0, sizeof(float) * h->nb.G, h->stream));
  // the kernels of the precision in use: the FP32 operator in the mixed path, the FP32
  // patch solve in the mixed and P32 paths, the FP64 kernels otherwise
  int& ax = d.fp32 ? d.epb_ax32 : (d.dwk ? d.epb_axdw : d.epb_ax);
  int& sw = d.pfp32 ? d.epb_sw32 : (d.dwk ? d.epb_swdw : d.epb_sw);
  auto fa = [&]() -> cudaError_t {
    return d.fp32 ? sem::launch_ax_local_f32_in32(d, d.p32, reinterpret_cast<float*>(d.wl), nullptr, h->stream)
                  : sem::launch_ax_local(d, h->p, d.wl, nullptr, h->stream);
  };
  auto fs = [&]() -> cudaError_t {
    float* wp32 = reinterpret_cast<float*>(d.wp);
    if (d.fp32) return sem::launch_schwarz_local_f32_in32(d, d.r32, wp32, nullptr, h->stream);
    if (d.pfp32) return sem::launch_schwarz_local_f32(d, h->r, wp32, nullptr, h->stream);
    return sem::launch_schwarz_local(d, h->r, d.wp, nullptr, h->stream);
  };
  const int cand[4] = {1, 2, 4, 8};
  int best_ax = 1, best_sw = 1;
  float t_ax = 1e30f, t_sw = 1e30f;
  for (int c : cand) {
    float ms;
    ax = sem::ax_tile_ok(d.p, c) ? c : 1;
    if (ax == c && time_launches(h, fa, 5, &ms) == SEM_OK && ms < t_ax) { t_ax = ms; best_ax = c; }
    sw = sem::sw_tile_ok(d.P, c) ? c : 1;
    if (sw == c && time_launches(h, fs, 5, &ms) == SEM_OK && ms < t_sw) { t_sw = ms; best_sw = c; }
  }
  ax = best_ax;
  sw = best_sw;
  h->invalidate();
  if (epb_ax_host) *epb_ax_host = best_ax;
  if (epb_sw_host) *epb_sw_host = best_sw;
  return SEM_OK;
}

}  // extern "C"
