// Device-side data of one problem and the kernel launchers (kernels.cu).
// Layouts (all device memory, element order = the library's order):
//   l2g   int32 [ne * p^3]       local node l = i + p (j + p k) of element e at e*p^3 + l
//   geo   f64 [ne][7][p^3]       G1..G6 (= w|J| J^-1 J^-T entries xx xy xz yy yz zz) and lambda m, m = w|J|
//   exyz  f64 [ne][8][3]         element vertex coordinates (VTK corner order)
//   g2l   CSR over DOFs -> local nodes (ascending), owner[g] = first local copy
//   ip    int32 [ne * P^3]       extended-box patch table, P = n + 3, -1 = absent
//   pg    CSR over DOFs -> patch entries e*P^3 + q (ascending)
//   ecv   int32 [ne][8]          coarse (free vertex) index of each corner or -1
//   cv    CSR over free vertices -> e*8 + corner
#pragma once

#include <cuda_bf16.h>

#include <cuda_runtime.h>
#include <cstdint>
#include <string>

#include "kdw.cuh"

namespace sem {

constexpr int kVecBlock = 256;          // threads per block of the vector kernels

// Scalars of one PCG solve, resident on the device (Algorithm 1).
constexpr int kMaxStallWindow = 8;

struct PcgState {
  double rz;        // z_k^T r_k
  double alpha, beta;
  double bb;        // ||b||^2
  double rtol;      // stop when ||r_k|| <= rtol ||b||
  double rr;        // ||r_k||^2
  double pf;        // p_k^T f
  double aux;       // spare reduction result (true residual)
  double rel_ref;   // ||r|| / ||b|| at the last residual replacement (mixed path)
  int iter;         // operator applications done
  int mixed;        // 1: FP32 operator/preconditioner, FP64 recurrences + replacement
  int replace;      // set by the update: the host runs a residual replacement next
  int replacements; // replacements done
  int done;         // 1 once converged / stopped
  int status;       // 0, SEM_MAXIT (1) or SEM_ERR_NAN (-6)
  int maxit;
  int learned;      // 1: the learned correction is added to z (flexible PCG)
  int flexible;     // 1: Polak-Ribiere beta (the K-cycle or the network make P vary)
  int nn_off;       // 1 once the learned correction was switched off for this solve
  int stall_window; // switch it off when ||r_k|| >= stall_ratio ||r_k-W|| (W = stall_window, 0 = never)
  double stall_ratio2;               // stall_ratio^2
  double nn_theta;  // the correction is used only if (z0 + c).r >= nn_theta z0.r
  int nn_use;       // 1: this iteration's direction includes the correction
  int nn_used;      // iterations that used it
  double rr_win[8];                  // ||r_j||^2 of the last 8 iterations, at j % 8
  unsigned int counter;   // blocks finished in the running reduction
};

struct DevCsr {
  int n = 0, nnz = 0;
  int lanes = 32;              // lanes per row in the AMG row kernels (4, 8, 16 or 32)
  int* ptr = nullptr;
  int* col = nullptr;
  double* val = nullptr;
};

struct DevAmgLevel {
  DevCsr A, P, R;
  DevCsr M, N, Q;              // the level's V(1,1) cycle as b_c = M b, x = N b + Q x_c (V-cycle kind)
  int up_lanes = 32;           // lanes per row of the N b + Q x_c kernel
  double* dinv = nullptr;
  double *b = nullptr, *x = nullptr, *t = nullptr, *y = nullptr;   // rhs, iterate, residual, output (size A.n)
  // K-cycle: the two inner directions c1, c2, their images A c1, A c2, and 8 scalars
  double *c1 = nullptr, *c2 = nullptr, *v1 = nullptr, *v2 = nullptr, *scal = nullptr;
};

struct DevProblem {
  int n = 0, p = 0, P = 0;
  // Block solves (sem_solve_block): nrhs right-hand sides advance together, each kernel of the
  // solve covering all of them (blockIdx.y = right-hand side). Right-hand side j's vectors,
  // local and patch results, coarse vectors, state and reduction partials sit at j times the
  // single-solve size after the first one's; its history at j * hist_stride.
  int nrhs = 1;
  int hist_stride = 0;
  int ne = 0, G = 0, nv = 0, nfree = 0;
  int Gi = 0;                       // DOFs 0..Gi-1 are element interiors, numbered e m^3 + a + m(b + m c)
                                    // for local node (a+1, b+1, c+1), m = n-1 (0: no such numbering)
  double lambda = 0.0;
  bool recompute = false;
  bool fp32 = false;                // operator and patch solves in FP32 (mixed path)
  bool pfp32 = false;               // preconditioner in FP32 (with fp32, or alone: FP64 operator)
  int sw_reserve_sms = 0;           // > 0: the patch-solve grid leaves this many SMs' worth of
                                    // slots free (for the coarse branch running beside it)
  int epb_ax = 1, epb_sw = 1;       // elements per CTA of the FP64 operator / patch-solve kernels
  int epb_ax32 = 1, epb_sw32 = 1;   // the same for the FP32 kernels (tuned separately)
  int epb_axdw = 1, epb_swdw = 1;   // and for the double-FP32 kernels of SEM_PREC_FP64
  bool tc = false;                  // the FP32 paths' patch solves in BF16 on the tensor cores
  int* wait_err = nullptr;          // set by a kernel whose bounded wait on a barrier ran out
  bool dwk = false;                 // SEM_PREC_FP64's element kernels in double-FP32 (kdw.cuh)
                                    // instead of binary64 (SEM_PREC_FP64_NATIVE)
                                    // (tile shapes picked by the autotuner; 1, 2, 4 or 8)
  const float* geo32 = nullptr;     // stored factors rounded to FP32 (same layout as geo)
  const __nv_bfloat16* geo16 = nullptr;   // the same rounded to BF16 (SEM_PREC_BF16)
  const dw* geodw = nullptr;        // the same as pairs of FP32 (h = fl32(G), l = fl32(G - h))
  bool bf16 = false;                // with fp32: the FP32 operator reads geo16
  // tables
  const int* l2g = nullptr;
  const double* geo = nullptr;
  const double* exyz = nullptr;
  const double* D = nullptr;        // p*p, Dhat[i*p + m] = phi_m'(t_i)
  const double* tg = nullptr;       // p GLL points
  const double* rho = nullptr;      // p GLL weights
  const uint8_t* mask = nullptr;
  const int* g2l_off = nullptr;
  const int* g2l_idx = nullptr;
  const int* owner = nullptr;
  const int* ip = nullptr;
  const int* pg_off = nullptr;
  const int* pg_idx = nullptr;
  const double* S = nullptr;        // P*P, S[row*P + mode]
  const double* ev = nullptr;       // P
  const uint8_t* pvar = nullptr;    // [ne] free sides (bit 2a low, 2a+1 high) or null if none
  const double* pw = nullptr;       // overlap weights c_N^-1/2 of P^f (null: unweighted, the paper's)
  const float* pw32 = nullptr;      // the same in FP32
  const double* Sv = nullptr;       // [3][P*P] pencils with a free low / high / both side(s)
  const double* evv = nullptr;      // [3][P]
  const double* hbox = nullptr;     // ne*3
  // per element patch, from hbox, the pencil eigenvalues and lambda (sw_diag_kernel): the
  // inverted diagonal of Eq. z times the scale 8/(hx hy hz), at [e][(b + P c) + P^2 a]
  const double* swd = nullptr;
  const float* swd32 = nullptr;
  const dw* swddw = nullptr;        // the same as pairs of FP32
  const double* Btab = nullptr;     // [p^3][8] Phi_I(t_i) Phi_J(t_j) Phi_K(t_k), VTK corner order
  const float* phi32 = nullptr;     // [p][2] (1 - t_i)/2 and (1 + t_i)/2 in FP32 (the 1D factors of Btab)
  const dw* phidw = nullptr;        // [p][2] (1 - t_i)/2 and (1 + t_i)/2 as pairs (the 1D factors of Btab)
  const dw* w3dw = nullptr;         // [p^3] (rho_i rho_j) rho_k in binary64 as pairs, node i + p (j + p k)
  dw* Zce = nullptr;                // [ne][8] coarse correction at each element's corners as pairs (0 where
                                    // the vertex is not free), for the double-FP32 P-sum
  const int* ecv = nullptr;
  const int* cv_off = nullptr;
  const int* cv_idx = nullptr;
  // AMG
  int nlevels = 0;
  int amg_kind = 0;                 // 0: three V(1,1) cycles (linear); 1: one K-cycle (nonlinear)
  DevAmgLevel* levels = nullptr;    // host array of device levels
  int coarsest_n = 0;
  const double* coarsest_inv = nullptr;
  double* cb = nullptr;             // coarsest rhs / solution work
  double* cx = nullptr;
  double* cres = nullptr;           // level-0 residual for repeated cycles
  // work
  double* wl = nullptr;             // ne*p^3 local results (FP32 view in the mixed path)
  double* wp = nullptr;             // ne*P^3 patch results (FP32 view in the mixed path)
  double* Re = nullptr;             // ne*8 element coarse residuals
  double* Rc = nullptr;             // nfree coarse residual
  double* Zc = nullptr;             // nfree coarse correction
  float* Zce32 = nullptr;           // [ne][8] the coarse correction at each element's corners in FP32
                                    // (0 where the vertex is not free), for the mixed path's P-sum
  float* p32 = nullptr;             // FP32 copies of the PCG direction and residual (mixed path)
  float* r32 = nullptr;
  double* nncorr = nullptr;         // learned correction N(s) (flexible PCG)
  double* nns = nullptr;            // its input s = r - A P r
  double* rprev = nullptr;          // r_{k-1} for the Polak-Ribiere beta (flexible PCG)
  double* partial = nullptr;        // reduction partials (4 * nblk)
  int nblk = 0;                     // blocks of the vector kernels
  PcgState* st = nullptr;
  PcgState* st_nn = nullptr;        // flexible PCG: done = 1 once the learned correction is off
};

// Records msg as this thread's sem_last_error() text and returns code (api.cu).
int report_error(int code, const std::string& msg);

// Number of kernels this thread has launched through the launchers below.
uint64_t kernel_launch_count();

// --- geometry set-up ---------------------------------------------------------
// Computes m_loc (ne*p^3) and, if geo != nullptr, the stored factors; sets *bad = 1
// if |J| <= 0 anywhere.
cudaError_t launch_geometry(const DevProblem& d, double* geo_out, float* geo32_out, __nv_bfloat16* geo16_out,
                            double* mloc, int* bad,
                            cudaStream_t s);

// Tile shapes (elements per CTA) compiled for an order: p = n+1 (operator), P = n+3 (patch).
bool ax_tile_ok(int p, int epb);
bool sw_tile_ok(int P, int epb);

// --- operator (Eq. R, Algorithm 2) -------------------------------------------
cudaError_t launch_ax_local(const DevProblem& d, const double* x, double* wl, const PcgState* st,
                            cudaStream_t s);
cudaError_t launch_ax_local_f32(const DevProblem& d, const double* x, float* wl, const PcgState* st,
                                cudaStream_t s);
// y = A x with the interior-first numbering (d.Gi > 0): interior DOFs written into y by the
// element kernel, the other local results into wl for launch_gather_shared*.
cudaError_t launch_ax_apply(const DevProblem& d, const double* x, double* wl, double* y, cudaStream_t s);
cudaError_t launch_ax_apply_f32(const DevProblem& d, const double* x, float* wl, double* y, cudaStream_t s);
cudaError_t launch_gather_shared(const DevProblem& d, const double* wl, const double* xin, double* y, cudaStream_t s);
// the same with FP32 vectors in and out (no conversions)
cudaError_t launch_ax_apply_f32io(const DevProblem& d, const float* x, float* wl, float* y, cudaStream_t s);
cudaError_t launch_gather_shared_f32io(const DevProblem& d, const float* wl, const float* xin, float* y,
                                       cudaStream_t s);
cudaError_t launch_gather_shared_f32(const DevProblem& d, const float* wl, const double* xin, double* y,
                                     cudaStream_t s);
cudaError_t launch_ax_local_f32_in32(const DevProblem& d, const float* x, float* wl, const PcgState* st,
                                     cudaStream_t s);
// y = gather(wl); masked rows take xin (identity) - sem_apply_A.
cudaError_t launch_gather_identity(const DevProblem& d, const double* wl, const double* xin, double* y,
                                   cudaStream_t s);
cudaError_t launch_gather_identity_f32(const DevProblem& d, const float* wl, const double* xin, double* y,
                                       cudaStream_t s);
// y = gather(wl) on all nodes, no mask (set-up: assembled mass).
cudaError_t launch_gather_plain(const DevProblem& d, const double* wl, double* y, cudaStream_t s);

// --- preconditioner (Sec. 4) -------------------------------------------------
cudaError_t launch_schwarz_local(const DevProblem& d, const double* r, double* wp, const PcgState* st,
                                 cudaStream_t s);
cudaError_t launch_schwarz_local_f32(const DevProblem& d, const double* r, float* wp, const PcgState* st,
                                     cudaStream_t s);
cudaError_t launch_schwarz_local_f32_in32(const DevProblem& d, const float* r, float* wp, const PcgState* st,
                                          cudaStream_t s);
cudaError_t launch_sw_diag(const DevProblem& d, double* dg, cudaStream_t s);
cudaError_t launch_convert_check(const unsigned long long* bits, long long n, unsigned long long* mismatches,
                                 cudaStream_t s);
cudaError_t launch_sw_diag_f32(const DevProblem& d, float* dg, cudaStream_t s);
// the same FP32 patch results from BF16 patch solves on the tensor cores (k_swtc.cu); needs
// d.pvar == null (no natural-boundary pencils)
cudaError_t launch_schwarz_tc(const DevProblem& d, const double* r, float* wp, const PcgState* st, cudaStream_t s);
cudaError_t launch_schwarz_tc_in32(const DevProblem& d, const float* r, float* wp, const PcgState* st,
                                   cudaStream_t s);
cudaError_t launch_coarse_restrict(const DevProblem& d, const double* r, const PcgState* st, cudaStream_t s);
cudaError_t launch_coarse_restrict_f32(const DevProblem& d, const float* r, const PcgState* st, cudaStream_t s);
cudaError_t launch_coarse_solve(const DevProblem& d, const PcgState* st, cudaStream_t s);
enum PsumMode { PSUM_FINE = 1, PSUM_COARSE = 2, PSUM_BOTH = 3, PSUM_IDENT = 4 };
// z = mask ? 0 : fine + coarse parts (or r itself with PSUM_IDENT); if pcg: rz reduction
// and beta on the device.
cudaError_t launch_psum(const DevProblem& d, int mode, const double* r, double* z, bool pcg,
                        cudaStream_t s);

// --- PCG (Algorithm 1) -------------------------------------------------------
cudaError_t launch_pcg_init(const DevProblem& d, const double* b, double* r, double* u, double rtol,
                            int maxit, int mixed, int learned, int flexible, int stall_window, double stall_ratio,
                            double nn_theta, double* hist, cudaStream_t s);
cudaError_t launch_pcg_first_direction(const DevProblem& d, const double* z, double* p, cudaStream_t s);
// f = gather(wl) (0 on masked; FP32 local results when d.fp32), pf = p.f, alpha = rz / pf.
cudaError_t launch_pcg_gather_alpha(const DevProblem& d, const double* p, double* f, cudaStream_t s);
cudaError_t launch_pcg_update(const DevProblem& d, const double* p, const double* f, double* u, double* r,
                              double* hist, cudaStream_t s);
cudaError_t launch_pcg_direction(const DevProblem& d, const double* z, double* p, cudaStream_t s);
// r = b - gather(wl) with FP64 local results; decides convergence on the true residual.
cudaError_t launch_pcg_replace(const DevProblem& d, const double* b, const double* wl, double* r, double* hist,
                               cudaStream_t s);
// --- learned correction in flexible PCG (not in the paper) ----------------------
// out = mask ? 0 : v - gather(wl); with st, skipped once the solve stopped or st->nn_off.
cudaError_t launch_residual_of(const DevProblem& d, const double* wl, const double* v, double* out,
                               const PcgState* st, cudaStream_t s);
cudaError_t launch_residual_of_f32(const DevProblem& d, const float* wl, const double* v, double* out,
                                   const PcgState* st, cudaStream_t s);
// decides whether this iteration uses d.nncorr (st->nn_use); rz and the Polak-Ribiere beta
cudaError_t launch_flex_combine(const DevProblem& d, const double* z, const double* r, cudaStream_t s);
// delta = mask ? 0 : xs - xk - z0
cudaError_t launch_pair_delta(const DevProblem& d, const double* xs, const double* xk, const double* z0,
                              double* delta, cudaStream_t s);

// --- backward-Euler heat step (Sec. 5) -------------------------------------------
// out = mask ? 0 : m (lambda u_prev + g) - gather(wl); norms = (||m (lambda u_prev + g)||^2,
// ||out||^2) over the free DOFs
cudaError_t launch_heat_rhs(const DevProblem& d, const double* wl, const double* mN, const double* u_prev,
                            const double* g, double* out, double* norms, cudaStream_t s);
// dst[i] = (fl32(src[i]), fl32(src[i] - fl32(src[i]))) for the double-FP32 kernels' tables
cudaError_t launch_split_pairs(long long n, const double* src, dw* dst, cudaStream_t s);
// b = mask ? 0 : mN * s (lumped GLL load)
cudaError_t launch_mass_load(const DevProblem& d, const double* mN, const double* sv, double* b, cudaStream_t s);
// y = a + b
cudaError_t launch_add_vectors(const DevProblem& d, const double* a, const double* b, double* y, cudaStream_t s);

// --- device-driven solve loop (graph conditional nodes) ----------------------------
// WHILE condition: !st->done and ++*guard <= limit; IF condition: st->replace && !st->done
cudaError_t launch_loop_cond(const PcgState* st, int nrhs, int* guard, int limit, cudaGraphConditionalHandle h,
                             cudaStream_t s);
cudaError_t launch_replace_cond(const PcgState* st, cudaGraphConditionalHandle h, cudaStream_t s);

// aux = ||b - f||^2 over free nodes
cudaError_t launch_true_residual(const DevProblem& d, const double* b, const double* wl, cudaStream_t s);

}  // namespace sem
