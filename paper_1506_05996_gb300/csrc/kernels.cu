// sm_103a kernels of the spectral-element solver, except the operator (k_ax*.cu) and
// the patch solve (k_sw*.cu). Gather and P-sum kernels are templated on the compute
// type T (double, or float for the mixed path); global vectors, dot products and the
// PCG recurrences are always FP64.
//
//  geometry_kernel      G1..G6 and m at every GLL node from the trilinear map (Sec. 2.3-2.4)
//  gather kernels       r_N = sum of local copies (Eq. gather), deterministic CSR order
//  coarse kernels       restriction C m^-1 r, AMG V-cycles, prolongation (Sec. 4.1, Eq. coarse)
//  pcg kernels          fused vector updates and dot products of Algorithm 1; alpha, beta
//                       and the stopping test are evaluated on the device
//
// Reductions are deterministic: fixed grid, fixed per-thread ranges, a fixed
// shuffle tree per block, and the last block to finish sums the block partials
// in index order (no spin-waits: a completion counter decides the last block).
#include <algorithm>
#include <cmath>

#include "kcommon.cuh"

namespace sem {

static thread_local uint64_t g_kernel_launches = 0;
uint64_t kernel_launch_count() { return g_kernel_launches; }
void count_launch() { ++g_kernel_launches; }

namespace {
using namespace sem;
// ----------------------------------------------------------------- geometry
template <int p>
__global__ void __launch_bounds__(p * p * p) geometry_kernel(const DevProblem d, double* geo, float* geo32,
                                                             __nv_bfloat16* geo16, double* mloc, int* bad) {
  constexpr int p3 = p * p * p;
  __shared__ double sx[24];
  const int e = blockIdx.x, t = threadIdx.x;
  if (t < 24) sx[t] = d.exyz[(size_t)e * 24 + t];
  __syncthreads();
  const int i = t % p, j = (t / p) % p, k = t / (p * p);
  double G[6], m, det;
  geom_point<double>(sx, d.tg[i], d.tg[j], d.tg[k], d.rho[i] * d.rho[j] * d.rho[k], G, m, det);
  if (!(det > 0.0)) *bad = 1;
  mloc[(size_t)e * p3 + t] = m;
  if (geo != nullptr) {
    double* gp = geo + (size_t)e * 7 * p3 + t;
#pragma unroll
    for (int c = 0; c < 6; ++c) gp[c * p3] = G[c];
    gp[6 * p3] = d.lambda * m;   // the c-term's factor lambda m, ready for the operator
  }
  if (geo32 != nullptr) {   // the same factors rounded to FP32 for the mixed path
    float* gp = geo32 + (size_t)e * 7 * p3 + t;
#pragma unroll
    for (int c = 0; c < 6; ++c) gp[c * p3] = (float)G[c];
    gp[6 * p3] = (float)(d.lambda * m);
  }
  if (geo16 != nullptr) {   // and to BF16 (one rounding from FP64, to nearest)
    __nv_bfloat16* gp = geo16 + (size_t)e * 7 * p3 + t;
#pragma unroll
    for (int c = 0; c < 6; ++c) gp[c * p3] = __double2bfloat16(G[c]);
    gp[6 * p3] = __double2bfloat16(d.lambda * m);
  }
}

// y = A x on DOFs g0..G-1 (g0 = 0, or d.Gi when the operator kernel wrote the interior
// DOFs itself): y = x on masked DOFs, else the sum of the local copies.
template <typename T, typename TY>
__global__ void gather_identity_kernel(const DevProblem d, const T* __restrict__ wl,
                                       const TY* __restrict__ xin, TY* __restrict__ y, int g0) {
  for (int g = g0 + blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    const bool mk = d.mask[g] != 0;   // applied after the gather's loads are issued
    const T s = gather_dof_ilp(d, wl, g);
    y[g] = mk ? xin[g] : (TY)s;
  }
}

__global__ void gather_plain_kernel(const DevProblem d, const double* __restrict__ wl, double* __restrict__ y) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    double s = 0.0;
    s = gather_dof(d, wl, g);
    y[g] = s;
  }
}

// ---------------------------------------------------------------- coarse
// Per element R_{IJK;e} = sum over the element's owned nodes of Phi_I(t_i) Phi_J(t_j)
// Phi_K(t_k) r_N; summed over elements this is C m^{-1} r (every node counted once, at
// its owner). Sum-factorised: one thread per (j, k) line contracts i, then (b0, k) pairs
// contract j, then the 8 corners contract k.
template <int p, typename T>
__global__ void __launch_bounds__(p * p) coarse_restrict_kernel(const DevProblem d, const T* __restrict__ r,
                                                                const PcgState* st) {
  st = st_rhs(st);
  if (stopped(st)) return;
  r += (size_t)blockIdx.y * d.G;                          // right-hand side blockIdx.y
  double* Re = d.Re + (size_t)blockIdx.y * d.ne * 8;
  constexpr int p3 = p * p * p;
  __shared__ T sl[2][p * p], sm[2][2][p], phi[2][p];
  const int e = blockIdx.x, t = threadIdx.x;
  if (t < p) {
    phi[0][t] = (T)(0.5 * (1.0 - d.tg[t]));
    phi[1][t] = (T)(0.5 * (1.0 + d.tg[t]));
  }
  __syncthreads();
  {   // thread (j, k): contract over i
    const int j = t % p, k = t / p;
    T a0 = 0, a1 = 0;
#pragma unroll
    for (int i = 0; i < p; ++i) {
      const int l = i + p * (j + p * k), gl = e * p3 + l;
      const int g = d.l2g[gl];
      const T rv = r[g];   // read with the owner and the mask, which select it after
      const T v = (d.owner[g] == gl && !d.mask[g]) ? rv : T(0);
      a0 += phi[0][i] * v;
      a1 += phi[1][i] * v;
    }
    sl[0][t] = a0;
    sl[1][t] = a1;
  }
  __syncthreads();
  if (t < 2 * p) {   // thread (b0, k): contract over j
    const int b0 = t / p, k = t % p;
    T c0 = 0, c1 = 0;
#pragma unroll
    for (int j = 0; j < p; ++j) {
      c0 += phi[0][j] * sl[b0][j + p * k];
      c1 += phi[1][j] * sl[b0][j + p * k];
    }
    sm[b0][0][k] = c0;
    sm[b0][1][k] = c1;
  }
  __syncthreads();
  if (t < 8) {   // VTK corner t: contract over k
    const int b0 = (t == 1 || t == 2 || t == 5 || t == 6), b1 = (t == 2 || t == 3 || t == 6 || t == 7), b2 = (t >= 4);
    T v = 0;
#pragma unroll
    for (int k = 0; k < p; ++k) v += phi[b2][k] * sm[b0][b1][k];
    Re[(size_t)e * 8 + t] = (double)v;
  }
}

__global__ void vertex_gather_kernel(const DevProblem d, const PcgState* st) {
  st = st_rhs(st);
  if (stopped(st)) return;
  const double* Re = d.Re + (size_t)blockIdx.y * d.ne * 8;
  double* Rc = d.Rc + (size_t)blockIdx.y * d.nfree;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < d.nfree; v += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = d.cv_off[v]; q < d.cv_off[v + 1]; ++q) s += Re[d.cv_idx[q]];
    Rc[v] = s;
  }
}

// AMG kernels. Sparse rows are handled by groups of LANES lanes (4..32, a power of two
// chosen per matrix from its mean row length, about four entries per lane): the lanes
// stride over the row, then a fixed shuffle tree. Short fine-level rows (27 entries) take
// 8 lanes instead of a warp. The groups step over the rows a warp at a time, so every lane
// reaches the shuffles of every step. (Groups of several warps per row, with partial sums
// meeting in shared memory, were measured slower for the long coarse-level rows; the
// block-wide form, a block stepping over rows, serves the dense coarsest matrix.)
__global__ void amg_jacobi0_kernel(int n, const double* __restrict__ dinv, const double* __restrict__ b,
                                   double* __restrict__ x, double omega, const PcgState* st) {
  if (stopped(st)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = omega * dinv[i] * b[i];
}

constexpr int kRowBlock = 256;   // block size of every row-group kernel

// Programmatic dependent launch of the coarse solve's kernel chain: a kernel launched with
// programmatic stream serialisation may be scheduled while its predecessor on the stream
// drains. Each kernel of the chain waits here, before reading anything, until that
// predecessor has completed and its writes are visible, and at once lets its own successor
// start launching (the successor waits in turn), so the chain pays no launch gap per kernel.
// Without the launch attribute both instructions have no effect.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// First row of this thread's group in the first step, the step (a warp covers 32 / LANES
// rows), and the thread's lane and group within the warp.
template <int LANES>
struct RowGroups {
  static_assert(LANES <= 32, "row groups are at most a warp");
  int first, step, lane, sub;
  __device__ __forceinline__ RowGroups() {
    lane = threadIdx.x & (LANES - 1);
    first = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 / LANES);
    step = ((gridDim.x * blockDim.x) >> 5) * (32 / LANES);
    sub = (threadIdx.x & 31) / LANES;
  }
};

// Sum over the LANES lanes of a group; every lane of the group gets it. LANES > 32 (the
// dense kernel's whole block) adds the warps' sums in shared memory, in warp order.
template <int LANES>
__device__ __forceinline__ double group_sum(double s) {
  constexpr int W = LANES < 32 ? LANES : 32;
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if constexpr (LANES > 32) {
    constexpr int NW = LANES / 32;
    __shared__ double red[kRowBlock / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    const int w0 = (threadIdx.x / LANES) * NW;
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < NW; ++k) t += red[w0 + k];
    __syncthreads();   // red is reused by the next step
    s = t;
  }
  return s;
}

// This lane's part of row `row` of A times x: entries lane, lane + LANES, ... in order. Four
// entries' column, value and x loads are issued together before their products are added
// (in the same order as one at a time, so the same bits): a lane of the long M and Q rows
// then waits for two memory latencies per four entries, not per entry.
template <int LANES>
__device__ __forceinline__ double row_dot(const DevCsr& A, int row, bool ok, const double* __restrict__ x, int lane) {
  double s = 0.0;
  if (ok) {
    const int q1 = A.ptr[row + 1];
    int q = A.ptr[row] + lane;
    for (; q + 3 * LANES < q1; q += 4 * LANES) {
      int c[4];
      double v[4], xv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        c[u] = A.col[q + u * LANES];
        v[u] = A.val[q + u * LANES];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) xv[u] = x[c[u]];
#pragma unroll
      for (int u = 0; u < 4; ++u) s += v[u] * xv[u];
    }
    for (; q < q1; q += LANES) s += A.val[q] * x[A.col[q]];
  }
  return s;
}

template <int LANES>
__global__ void __launch_bounds__(kRowBlock) amg_resid_kernel(DevCsr A, const double* __restrict__ b,
                                                             const double* __restrict__ x, double* __restrict__ t,
                                                             const PcgState* st) {
  pdl_enter();
  st = st_rhs(st);
  if (stopped(st)) return;
  const size_t o = (size_t)blockIdx.y * A.n;   // right-hand side blockIdx.y (square matrix)
  b += o;
  x += o;
  t += o;
  const RowGroups<LANES> g;
  for (int i0 = g.first; i0 < A.n; i0 += g.step) {
    const int i = i0 + g.sub;
    const bool ok = i < A.n;
    const double s = group_sum<LANES>(row_dot<LANES>(A, i, ok, x, g.lane));
    if (ok && g.lane == 0) t[i] = b[i] - s;
  }
}

template <int LANES>
__global__ void __launch_bounds__(kRowBlock) amg_spmv_kernel(DevCsr A, const double* __restrict__ x,
                                                            double* __restrict__ y, const PcgState* st, int sx) {
  pdl_enter();
  st = st_rhs(st);
  if (stopped(st)) return;
  x += (size_t)blockIdx.y * sx;                // right-hand side blockIdx.y: x has sx entries
  y += (size_t)blockIdx.y * A.n;
  const RowGroups<LANES> g;
  for (int i0 = g.first; i0 < A.n; i0 += g.step) {
    const int i = i0 + g.sub;
    const bool ok = i < A.n;
    const double s = group_sum<LANES>(row_dot<LANES>(A, i, ok, x, g.lane));
    if (ok && g.lane == 0) y[i] = s;
  }
}

template <int LANES>
__global__ void __launch_bounds__(kRowBlock) amg_prolong_add_kernel(DevCsr P, const double* __restrict__ xc,
                                                                   double* __restrict__ x, const PcgState* st) {
  if (stopped(st)) return;
  const RowGroups<LANES> g;
  for (int i0 = g.first; i0 < P.n; i0 += g.step) {
    const int i = i0 + g.sub;
    const bool ok = i < P.n;
    const double s = group_sum<LANES>(row_dot<LANES>(P, i, ok, xc, g.lane));
    if (ok && g.lane == 0) x[i] = x[i] + s;
  }
}

template <int LANES>
__global__ void __launch_bounds__(kRowBlock) amg_jacobi_post_kernel(DevCsr A, const double* __restrict__ dinv,
                                                                   const double* __restrict__ b,
                                                                   const double* __restrict__ x,
                                                                   double* __restrict__ xout, double omega,
                                                                   const PcgState* st) {
  if (stopped(st)) return;
  const RowGroups<LANES> g;
  for (int i0 = g.first; i0 < A.n; i0 += g.step) {
    const int i = i0 + g.sub;
    const bool ok = i < A.n;
    const double s = group_sum<LANES>(row_dot<LANES>(A, i, ok, x, g.lane));
    if (ok && g.lane == 0) xout[i] = x[i] + omega * dinv[i] * (b[i] - s);
  }
}

// x = z + N b + Q x_c (z may be null): the prolongation and post-smoothing of a V(1,1)
// cycle as one pass; both rows are summed by the same lanes, then one reduction.
template <int LANES>
__global__ void __launch_bounds__(kRowBlock) amg_up_kernel(DevCsr N, DevCsr Q, const double* __restrict__ b,
                                                          const double* __restrict__ xc, const double* z, double* out,
                                                          const PcgState* st, int sxc) {
  pdl_enter();
  st = st_rhs(st);
  if (stopped(st)) return;
  const size_t o = (size_t)blockIdx.y * N.n;   // right-hand side blockIdx.y; xc has sxc entries
  b += o;
  out += o;
  if (z != nullptr) z += o;
  xc += (size_t)blockIdx.y * sxc;
  const RowGroups<LANES> g;
  for (int i0 = g.first; i0 < N.n; i0 += g.step) {
    const int i = i0 + g.sub;
    const bool ok = i < N.n;
    const double s = group_sum<LANES>(row_dot<LANES>(N, i, ok, b, g.lane) + row_dot<LANES>(Q, i, ok, xc, g.lane));
    if (ok && g.lane == 0) out[i] = z != nullptr ? z[i] + s : s;   // z may alias out: same row
  }
}

// x = Ainv b at the dense coarsest level: one warp per row (Ainv row-major), each lane's
// entries lane, lane + 32, ... summed in order with their loads issued 4 at a time, then the
// warp's sum.
__global__ void __launch_bounds__(kRowBlock) dense_mv_kernel(int n, const double* __restrict__ Ainv,
                                                            const double* __restrict__ b, double* __restrict__ x,
                                                            const PcgState* st) {
  pdl_enter();
  st = st_rhs(st);
  if (stopped(st)) return;
  b += (size_t)blockIdx.y * n;
  x += (size_t)blockIdx.y * n;
  const int lane = threadIdx.x & 31;
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n; row += (gridDim.x * blockDim.x) >> 5) {
    const double* a = Ainv + (size_t)row * n;
    double s = 0.0;
    int c = lane;
    for (; c + 96 < n; c += 128) {
      double av[4], bv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        av[u] = a[c + 32 * u];
        bv[u] = b[c + 32 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) s += av[u] * bv[u];
    }
    for (; c < n; c += 32) s += a[c] * b[c];
    s = group_sum<32>(s);
    if (lane == 0) x[row] = s;
  }
}

// K-cycle (Sec. 4.1, the recursive cycle of the paper's AMG reference): two flexible-CG
// steps on a coarse level, c1 = K(r_c), c2 = K(r_c - (c1.r_c / c1.A c1) A c1), and the
// correction e_c = a c1 + b c2 that is A-orthogonal projection of A^-1 r_c onto
// span{c1, c2}: b = alpha2 / rho2, a = alpha1 / rho1 - gamma b / rho1 with
// rho1 = c1.A c1, alpha1 = c1.r_c, gamma = c2.A c1, beta = c2.A c2, alpha2 = c2.r2,
// rho2 = beta - gamma^2 / rho1 (one direction when rho2 <= 1e-14 beta). The level's
// vectors are small: one block sums them in a fixed order.
constexpr int kKcBlock = 512;
constexpr double kKcParallel = 1e-14;

// scal[0] = c1.v1 (rho1), scal[1] = c1.rc (alpha1)
__global__ void __launch_bounds__(kKcBlock) kc_dots1_kernel(int n, const double* __restrict__ c1,
                                                            const double* __restrict__ v1,
                                                            const double* __restrict__ rc, double* __restrict__ scal,
                                                            const PcgState* st) {
  if (stopped(st)) return;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += kKcBlock) {
    a += c1[i] * v1[i];
    b += c1[i] * rc[i];
  }
  a = block_sum<kKcBlock>(a);
  b = block_sum<kKcBlock>(b);
  if (threadIdx.x == 0) {
    scal[0] = a;
    scal[1] = b;
  }
}

// rc -= (alpha1 / rho1) v1 (rc becomes r2)
__global__ void kc_r2_kernel(int n, const double* __restrict__ v1, const double* __restrict__ scal,
                             double* __restrict__ rc, const PcgState* st) {
  if (stopped(st)) return;
  const double step = scal[0] > 0.0 ? scal[1] / scal[0] : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) rc[i] -= step * v1[i];
}

// scal[2] = c2.v1 (gamma), scal[3] = c2.v2 (beta), scal[4] = c2.r2 (alpha2)
__global__ void __launch_bounds__(kKcBlock) kc_dots2_kernel(int n, const double* __restrict__ c2,
                                                            const double* __restrict__ v1,
                                                            const double* __restrict__ v2,
                                                            const double* __restrict__ r2, double* __restrict__ scal,
                                                            const PcgState* st) {
  if (stopped(st)) return;
  double g = 0.0, b = 0.0, a = 0.0;
  for (int i = threadIdx.x; i < n; i += kKcBlock) {
    g += c2[i] * v1[i];
    b += c2[i] * v2[i];
    a += c2[i] * r2[i];
  }
  g = block_sum<kKcBlock>(g);
  b = block_sum<kKcBlock>(b);
  a = block_sum<kKcBlock>(a);
  if (threadIdx.x == 0) {
    scal[2] = g;
    scal[3] = b;
    scal[4] = a;
  }
}

// ec = a c1 + b c2 (the projection above)
__global__ void kc_combine_kernel(int n, const double* __restrict__ c1, const double* __restrict__ c2,
                                  const double* __restrict__ scal, double* __restrict__ ec, const PcgState* st) {
  if (stopped(st)) return;
  const double rho1 = scal[0], alpha1 = scal[1], gamma = scal[2], beta = scal[3], alpha2 = scal[4];
  double a = 0.0, b = 0.0;
  if (rho1 > 0.0) {
    const double rho2 = beta - gamma * gamma / rho1;
    if (rho2 <= kKcParallel * beta) {
      a = alpha1 / rho1;
    } else {
      b = alpha2 / rho2;
      a = alpha1 / rho1 - gamma * b / rho1;
    }
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) ec[i] = a * c1[i] + b * c2[i];
}

// ------------------------------------------------------------ P sum and PCG
template <typename T> __device__ __forceinline__ const T* wts_of(const DevProblem& d);
template <> __device__ __forceinline__ const double* wts_of<double>(const DevProblem& d) { return d.pw; }
template <> __device__ __forceinline__ const float* wts_of<float>(const DevProblem& d) { return d.pw32; }

// z = P r on the free nodes: the patch results summed over every patch containing the
// node (fine part) plus the trilinear interpolation of the coarse correction at the node
// (coarse part, Eq. coarse), accumulated in T; with PCG also z.r and beta (FP64). In FP32 the
// interpolation reads the element's 8 corner values (one contiguous 32-byte read, gathered
// once per corner by the coarse solve's last kernel) and is sum-factorised along i, j, k; in
// binary64 it is the 8-term sum over the corners' coarse DOFs.
template <bool PCG, typename T>
__global__ void __launch_bounds__(kVecBlock) psum_kernel(const DevProblem d, int mode, const T* __restrict__ wp,
                                                         const double* __restrict__ r, double* __restrict__ z) {
  PcgState* const pst = d.st + blockIdx.y;    // right-hand side blockIdx.y
  if (PCG && stopped(pst)) return;
  const int p = d.p, p3 = p * p * p;
  wp += (size_t)blockIdx.y * d.ne * d.P * d.P * d.P;
  r += (size_t)blockIdx.y * d.G;
  z += (size_t)blockIdx.y * d.G;
  double* const part = d.partial + (size_t)blockIdx.y * 4 * d.nblk;
  const double* __restrict__ Zc = d.Zc + (size_t)blockIdx.y * d.nfree;
  const T* __restrict__ Wt = wts_of<T>(d);
  double dot = 0.0;
  const bool coarse = (mode & PSUM_COARSE) && d.nfree > 0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    // the mask, the CSR range and the owner are read together (the mask is applied at the
    // end, so it adds no memory latency in front of the others)
    const bool mk = d.mask[g] != 0;
    const int q0 = d.pg_off[g], q1 = d.pg_off[g + 1];
    const int l = coarse ? d.owner[g] : 0;
    T v = 0;
    {
      if (mode & PSUM_IDENT) v += (T)r[g];
      if (mode & PSUM_FINE) {
        T vf = 0;
        for (int q = q0; q < q1; ++q) vf += wp[d.pg_idx[q]];
        if (Wt != nullptr) vf = vf * Wt[g];     // overlap-weighted P^f
        v += vf;
      }
      if (coarse) {
        const int e = l / p3, lr = l % p3;
        if constexpr (std::is_same<T, float>::value) {
          // corner values in VTK order at the owner node (i, j, k): along i, then j, then k
          const int i = lr % p, j = (lr / p) % p, k = lr / (p * p);
          const float4* Z4 = reinterpret_cast<const float4*>(d.Zce32 + ((size_t)blockIdx.y * d.ne + e) * 8);
          const float4 za = Z4[0], zb = Z4[1];
          const float a0 = d.phi32[2 * i], a1 = d.phi32[2 * i + 1];
          const float b0 = d.phi32[2 * j], b1 = d.phi32[2 * j + 1];
          const float c0 = d.phi32[2 * k], c1 = d.phi32[2 * k + 1];
          const float z00 = a0 * za.x + a1 * za.y, z10 = a0 * za.w + a1 * za.z;
          const float z01 = a0 * zb.x + a1 * zb.y, z11 = a0 * zb.w + a1 * zb.z;
          v += c0 * (b0 * z00 + b1 * z10) + c1 * (b0 * z01 + b1 * z11);
        } else {
          const int* ec = d.ecv + (size_t)e * 8;
          const double* B = d.Btab + 8 * lr;
          T zc = 0;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const int cv = ec[c];
            if (cv >= 0) zc += B[c] * Zc[cv];
          }
          v += zc;
        }
      }
    }
    const double vd = mk ? 0.0 : (double)v;
    z[g] = vd;
    if (PCG) dot += vd * r[g];
  }
  if (PCG) {
    double total;
    if (grid_reduce<kVecBlock>(dot, part, &pst->counter, total) && threadIdx.x == 0) {
      PcgState* st = pst;
      if (!isfinite(total)) { st->status = -6; st->done = 1; }
      if (st->iter > 0) st->beta = total / st->rz;
      st->rz = total;
    }
  }
}

// The coarse correction at the corners of every element in FP32 (the mixed path's P-sum),
// rounded to nearest by the integer routine (the FP64 converter runs on the FP64 pipe).
__global__ void coarse_corners_f32_kernel(const DevProblem d, const PcgState* st) {
  pdl_enter();
  if (stopped(st)) return;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < 8 * d.ne; q += gridDim.x * blockDim.x) {
    const int cv = d.ecv[q];
    d.Zce32[q] = cv >= 0 ? f64_to_f32(d.Zc[cv]) : 0.0f;
  }
}

// The coarse correction at the corners of every element, as pairs: one gather per corner
// instead of one per node of the P-sum (which then reads 8 contiguous pairs per node).
__global__ void coarse_corners_dw_kernel(const DevProblem d, const PcgState* st) {
  pdl_enter();
  st = st_rhs(st);
  if (stopped(st)) return;
  const double* Zc = d.Zc + (size_t)blockIdx.y * d.nfree;
  dw* Zce = d.Zce + (size_t)blockIdx.y * d.ne * 8;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < 8 * d.ne; q += gridDim.x * blockDim.x) {
    const int cv = d.ecv[q];
    Zce[q] = cv >= 0 ? dw_split(Zc[cv]) : dw_zero();
  }
}

// The P-sum of SEM_PREC_FP64 in double-FP32: the patch results (pairs, written by the
// double-FP32 patch solve) summed over the patches containing each node, plus the trilinear
// interpolation of the coarse correction (8 products per DOF), joined to binary64 once per
// DOF; the z.r reduction stays binary64.
template <bool PCG>
__global__ void __launch_bounds__(kVecBlock) psum_dw_kernel(const DevProblem d, int mode, const dw* __restrict__ wp,
                                                            const double* __restrict__ r, double* __restrict__ z) {
  PcgState* const pst = d.st + blockIdx.y;    // right-hand side blockIdx.y
  if (PCG && stopped(pst)) return;
  const int p = d.p, p3 = p * p * p;
  wp += (size_t)blockIdx.y * d.ne * d.P * d.P * d.P;
  r += (size_t)blockIdx.y * d.G;
  z += (size_t)blockIdx.y * d.G;
  double* const part = d.partial + (size_t)blockIdx.y * 4 * d.nblk;
  const dw* const Zce = d.Zce + (size_t)blockIdx.y * d.ne * 8;
  double dot = 0.0;
  const bool coarse = (mode & PSUM_COARSE) && d.nfree > 0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    // the mask, the CSR range and the owner are read together (the mask is applied at the
    // end, so it adds no memory latency in front of the others)
    const bool mk = d.mask[g] != 0;
    const int q0 = d.pg_off[g], q1 = d.pg_off[g + 1];
    const int l = coarse ? d.owner[g] : 0;
    dw v = dw_zero();
    {
      if (mode & PSUM_IDENT) v = dw_split(r[g]);
      if (mode & PSUM_FINE) {
        // the patch results in ascending patch-entry order, the first 8 loads issued together
        constexpr int U = 8;
        int ix[U];
#pragma unroll
        for (int c = 0; c < U; ++c) ix[c] = (q0 + c < q1) ? d.pg_idx[q0 + c] : 0;
        dw pv[U];
#pragma unroll
        for (int c = 0; c < U; ++c)
          if (q0 + c < q1) pv[c] = wp[ix[c]];
        dw vf = dw_zero();
#pragma unroll
        for (int c = 0; c < U; ++c)
          if (q0 + c < q1) vf = dw_add(vf, pv[c]);
        for (int q = q0 + U; q < q1; ++q) vf = dw_add(vf, wp[d.pg_idx[q]]);
        if (d.pw != nullptr) vf = dw_mul(vf, dw_split(d.pw[g]));   // overlap-weighted P^f
        v = dw_add(v, vf);
      }
      if (coarse) {
        // trilinear interpolation of the element's corner values (VTK order) at the owner
        // node (i, j, k), sum-factorised: along i, then j, then k
        const int e = l / p3, lr = l % p3;
        const int i = lr % p, j = (lr / p) % p, k = lr / (p * p);
        const dw* Z = Zce + (size_t)e * 8;
        const dw a0 = d.phidw[2 * i], a1 = d.phidw[2 * i + 1];
        const dw b0 = d.phidw[2 * j], b1 = d.phidw[2 * j + 1];
        const dw c0 = d.phidw[2 * k], c1 = d.phidw[2 * k + 1];
        auto lerp = [](dw f0, dw x0, dw f1, dw x1) { dw s = dw_mul(f0, x0); dw_mac(s, f1, x1); return s; };
        const dw z00 = lerp(a0, Z[0], a1, Z[1]), z10 = lerp(a0, Z[3], a1, Z[2]);
        const dw z01 = lerp(a0, Z[4], a1, Z[5]), z11 = lerp(a0, Z[7], a1, Z[6]);
        const dw w0 = lerp(b0, z00, b1, z10), w1 = lerp(b0, z01, b1, z11);
        v = dw_add(v, lerp(c0, w0, c1, w1));
      }
    }
    const double vd = mk ? 0.0 : dw_join(v);
    z[g] = vd;
    if (PCG) dot += vd * r[g];
  }
  if (PCG) {
    double total;
    if (grid_reduce<kVecBlock>(dot, part, &pst->counter, total) && threadIdx.x == 0) {
      PcgState* st = pst;
      if (!isfinite(total)) { st->status = -6; st->done = 1; }
      if (st->iter > 0) st->beta = total / st->rz;
      st->rz = total;
    }
  }
}


__global__ void __launch_bounds__(kVecBlock) pcg_init_kernel(const DevProblem d, const double* __restrict__ b,
                                                             double* __restrict__ r, double* __restrict__ u,
                                                             double rtol, int maxit, int mixed, int learned,
                                                             int flexible, int stall_window, double stall_ratio,
                                                             double nn_theta, double* hist) {
  PcgState* const pst = d.st + blockIdx.y;    // right-hand side blockIdx.y
  double* const part = d.partial + (size_t)blockIdx.y * 4 * d.nblk;
  b += (size_t)blockIdx.y * d.G;
  r += (size_t)blockIdx.y * d.G;
  u += (size_t)blockIdx.y * d.G;
  hist += (size_t)blockIdx.y * d.hist_stride;
  double dot = 0.0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    const double v = d.mask[g] ? 0.0 : b[g];
    r[g] = v;
    if (mixed) d.r32[g] = f64_to_f32(v);
    if (flexible) d.rprev[g] = 0.0;
    u[g] = 0.0;
    dot += v * v;
  }
  double total;
  if (grid_reduce<kVecBlock>(dot, part, &pst->counter, total) && threadIdx.x == 0) {
    PcgState* st = pst;
    st->bb = total;
    st->rtol = rtol;
    st->rr = total;
    st->iter = 0;
    st->maxit = maxit;
    st->status = 0;
    st->rz = 0.0;
    st->beta = 0.0;
    st->rel_ref = 1.0;
    st->mixed = mixed;
    st->replace = 0;
    st->replacements = 0;
    st->learned = learned;
    st->flexible = flexible;
    st->nn_off = learned ? 0 : 1;
    st->stall_window = stall_window;
    st->nn_theta = nn_theta;
    st->nn_use = 0;
    st->nn_used = 0;
    st->stall_ratio2 = stall_ratio * stall_ratio;
    st->rr_win[0] = total;
    hist[0] = (total > 0.0) ? 1.0 : 0.0;
    if (!isfinite(total)) { st->status = -6; st->done = 1; }
    else if (total == 0.0) st->done = 1;
    else if (maxit <= 0) { st->status = 1; st->done = 1; }
  }
}

__global__ void pcg_copy_kernel(const DevProblem d, const double* __restrict__ z, double* __restrict__ p) {
  PcgState* const pst = d.st + blockIdx.y;    // right-hand side blockIdx.y
  z += (size_t)blockIdx.y * d.G;
  p += (size_t)blockIdx.y * d.G;
  if (stopped(pst)) return;
  float* __restrict__ p32 = pst->mixed ? d.p32 : nullptr;
  const double* __restrict__ c = (pst->learned && pst->nn_use) ? d.nncorr : nullptr;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    const double pn = c ? z[g] + c[g] : z[g];
    p[g] = pn;
    if (p32) p32[g] = f64_to_f32(pn);
  }
}

template <typename T>
__global__ void __launch_bounds__(kVecBlock) pcg_gather_alpha_kernel(const DevProblem d, const T* __restrict__ wl,
                                                                     const double* __restrict__ p,
                                                                     double* __restrict__ f) {
  PcgState* const pst = d.st + blockIdx.y;    // right-hand side blockIdx.y
  double* const part = d.partial + (size_t)blockIdx.y * 4 * d.nblk;
  wl += (size_t)blockIdx.y * d.ne * d.p * d.p * d.p;
  p += (size_t)blockIdx.y * d.G;
  f += (size_t)blockIdx.y * d.G;
  if (stopped(pst)) return;
  double dot = 0.0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    const bool mk = d.mask[g] != 0;   // applied after the gather's loads are issued
    const T s = gather_dof(d, wl, g);
    const double sd = mk ? 0.0 : (double)s;
    f[g] = sd;
    dot += p[g] * sd;
  }
  double total;
  if (grid_reduce<kVecBlock>(dot, part, &pst->counter, total) && threadIdx.x == 0) {
    PcgState* st = pst;
    st->pf = total;
    if (!(total > 0.0) || !isfinite(total)) { st->status = -6; st->done = 1; }
    else st->alpha = st->rz / total;
  }
}

__global__ void __launch_bounds__(kVecBlock) pcg_update_kernel(const DevProblem d, const double* __restrict__ p,
                                                               const double* __restrict__ f, double* __restrict__ u,
                                                               double* __restrict__ r, double* hist) {
  PcgState* const pst = d.st + blockIdx.y;    // right-hand side blockIdx.y
  double* const part = d.partial + (size_t)blockIdx.y * 4 * d.nblk;
  p += (size_t)blockIdx.y * d.G;
  f += (size_t)blockIdx.y * d.G;
  u += (size_t)blockIdx.y * d.G;
  r += (size_t)blockIdx.y * d.G;
  hist += (size_t)blockIdx.y * d.hist_stride;
  if (stopped(pst)) return;
  const double alpha = pst->alpha;
  float* __restrict__ r32 = pst->mixed ? d.r32 : nullptr;
  double dot = 0.0;
  double* __restrict__ rprev = pst->flexible ? d.rprev : nullptr;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    u[g] = u[g] + alpha * p[g];
    const double ro = r[g];
    const double rn = ro - alpha * f[g];
    if (rprev) rprev[g] = ro;
    r[g] = rn;
    if (r32) r32[g] = f64_to_f32(rn);
    dot += rn * rn;
  }
  double total;
  if (grid_reduce<kVecBlock>(dot, part, &pst->counter, total) && threadIdx.x == 0) {
    PcgState* st = pst;
    st->rr = total;
    const int it = ++st->iter;
    if (st->learned) {
      // a correction under which the residual stops dropping over the window is switched
      // off for the rest of the solve
      const int W = st->stall_window;
      if (W > 0 && it >= W && total >= st->stall_ratio2 * st->rr_win[(it - W) % kMaxStallWindow]) {
        st->nn_off = 1;
        d.st_nn->done = 1;
      }
      st->rr_win[it % kMaxStallWindow] = total;
    }
    const double rel = sqrt(total) / sqrt(st->bb);
    hist[it] = rel;
    if (!isfinite(total)) { st->status = -6; st->done = 1; }
    else if (st->mixed) {
      // the recursive residual of the FP32 operator drifts from b - A u: confirm
      // convergence, or refresh r, with the FP64 operator (residual replacement)
      if (rel <= st->rtol || rel <= kReplaceFactor * st->rel_ref || it >= st->maxit) st->replace = 1;
    } else if (rel <= st->rtol) st->done = 1;
    else if (it >= st->maxit) { st->status = 1; st->done = 1; }
  }
}

// Residual replacement: r = b - A u with the FP64 operator (local results in wl),
// and the decision whether the true residual meets the tolerance.
__global__ void __launch_bounds__(kVecBlock) pcg_replace_kernel(const DevProblem d, const double* __restrict__ b,
                                                                const double* __restrict__ wl, double* __restrict__ r,
                                                                double* hist) {
  double dot = 0.0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    double res = 0.0;
    if (!d.mask[g]) {
      double s = 0.0;
      s = gather_dof(d, wl, g);
      res = b[g] - s;
    }
    r[g] = res;
    d.r32[g] = f64_to_f32(res);
    dot += res * res;
  }
  double total;
  if (grid_reduce<kVecBlock>(dot, d.partial, &d.st->counter, total) && threadIdx.x == 0) {
    PcgState* st = d.st;
    const double rel = sqrt(total) / sqrt(st->bb);
    st->rr = total;
    st->replacements += 1;
    hist[st->iter] = rel;
    st->replace = 0;
    if (!isfinite(total)) { st->status = -6; st->done = 1; }
    else if (rel <= st->rtol) st->done = 1;
    else if (st->iter >= st->maxit) { st->status = 1; st->done = 1; }
    else st->rel_ref = rel;
  }
}

__global__ void pcg_direction_kernel(const DevProblem d, const double* __restrict__ z, double* __restrict__ p) {
  PcgState* const pst = d.st + blockIdx.y;    // right-hand side blockIdx.y
  z += (size_t)blockIdx.y * d.G;
  p += (size_t)blockIdx.y * d.G;
  if (stopped(pst)) return;
  const double beta = pst->beta;
  float* __restrict__ p32 = pst->mixed ? d.p32 : nullptr;
  const double* __restrict__ c = (pst->learned && pst->nn_use) ? d.nncorr : nullptr;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    const double pn = (c ? z[g] + c[g] : z[g]) + beta * p[g];
    p[g] = pn;
    if (p32) p32[g] = f64_to_f32(pn);
  }
}

// out = mask ? 0 : v - gather(wl): the residual of an operator application (flexible PCG:
// s = r - A P r; training pairs: r = b - A x). Skipped inside PCG once the network is off.
template <typename T>
__global__ void __launch_bounds__(kVecBlock) residual_of_kernel(const DevProblem d, const T* __restrict__ wl,
                                                                const double* __restrict__ v, double* __restrict__ out,
                                                                const PcgState* st) {
  if (st != nullptr && (st->done || st->nn_off)) return;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    double res = 0.0;
    if (!d.mask[g]) {
      T s = 0;
      s = gather_dof(d, wl, g);
      res = v[g] - (double)s;
    }
    out[g] = res;
  }
}

// Flexible PCG with z0 = P r in z and the correction c in d.nncorr: the correction is used
// in this iteration (st->nn_use) only if it is on and keeps descent, (z0 + c).r >= theta z0.r;
// then rz = z.r and beta = z_k.(r_k - r_k-1) / (z_k-1.r_k-1) (Polak-Ribiere form) for the
// chosen z. z itself keeps z0; the direction kernels add c when st->nn_use.
__global__ void __launch_bounds__(kVecBlock) flex_combine_kernel(const DevProblem d, const double* __restrict__ z,
                                                                 const double* __restrict__ r) {
  if (stopped(d.st)) return;
  const bool on = d.st->nn_off == 0;
  double v[4] = {0.0, 0.0, 0.0, 0.0};   // z0.r, c.r, z0.rprev, c.rprev
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    const double zg = z[g], rg = r[g], rp = d.rprev[g];
    v[0] += zg * rg;
    v[2] += zg * rp;
    if (on) {
      const double cg = d.nncorr[g];
      v[1] += cg * rg;
      v[3] += cg * rp;
    }
  }
  double t[4];
  if (grid_reduce_n<kVecBlock, 4>(v, d.partial, &d.st->counter, t) && threadIdx.x == 0) {
    PcgState* st = d.st;
    const int use = (on && isfinite(t[1]) && isfinite(t[3]) && t[0] + t[1] >= st->nn_theta * t[0]) ? 1 : 0;
    const double zr = t[0] + (use ? t[1] : 0.0), zrp = t[2] + (use ? t[3] : 0.0);
    st->nn_use = use;
    st->nn_used += use;
    if (!isfinite(zr) || !isfinite(zrp)) { st->status = -6; st->done = 1; }
    if (st->iter > 0) st->beta = (zr - zrp) / st->rz;
    st->rz = zr;
  }
}

// Backward-Euler step (Sec. 5): out = mask ? 0 : m (lambda u_prev + g) - gather(wl), wl the FP64
// local results of A u_prev; norms[0] = ||m (lambda u_prev + g)||^2, norms[1] = ||out||^2
// over the free DOFs.
__global__ void __launch_bounds__(kVecBlock) heat_rhs_kernel(const DevProblem d, const double* __restrict__ wl,
                                                             const double* __restrict__ mN,
                                                             const double* __restrict__ u_prev,
                                                             const double* __restrict__ g, double* __restrict__ out,
                                                             double* __restrict__ norms) {
  double v[2] = {0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.G; i += gridDim.x * blockDim.x) {
    double res = 0.0;
    if (!d.mask[i]) {
      const double bf = mN[i] * (d.lambda * u_prev[i] + g[i]);
      double s = 0.0;
      s = gather_dof(d, wl, i);
      res = bf - s;
      v[0] += bf * bf;
      v[1] += res * res;
    }
    out[i] = res;
  }
  double t[2];
  if (grid_reduce_n<kVecBlock, 2>(v, d.partial, &d.st->counter, t) && threadIdx.x == 0) {
    norms[0] = t[0];
    norms[1] = t[1];
  }
}

// Lumped GLL load (Sec. 2.4, with the weak-form source read as s, reading A8):
// b_N = m_N s_N on free DOFs, 0 on Dirichlet DOFs.
__global__ void mass_load_kernel(const DevProblem d, const double* __restrict__ mN, const double* sv, double* b) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.G; i += gridDim.x * blockDim.x)
    b[i] = d.mask[i] ? 0.0 : mN[i] * sv[i];
}

// Pairs of FP32 from binary64 table entries, to nearest: h = fl32(v), l = fl32(v - h)
// (set-up of the double-FP32 kernels' stored factors and patch diagonals).
__global__ void split_pairs_kernel(long long n, const double* __restrict__ src, dw* __restrict__ dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = src[i];
    const float h = __double2float_rn(v);
    dst[i] = {h, __double2float_rn(v - (double)h)};
  }
}

// y = a + b
__global__ void add_vectors_kernel(int n, const double* __restrict__ a, const double* __restrict__ b,
                                   double* __restrict__ y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = a[i] + b[i];
}

// Device-driven solve loop (a CUDA graph WHILE node around one iteration): the loop runs
// while the solve is not done, and never more than `limit` times (an independent guard,
// so the graph ends whatever the solver state). One thread sets the condition.
__global__ void loop_cond_kernel(const PcgState* st, int nrhs, int* guard, int limit, cudaGraphConditionalHandle h) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int g = ++*guard;
    bool open = false;   // a block solve runs until each of its right-hand sides is done
    for (int j = 0; j < nrhs; ++j) open = open || st[j].done == 0;
    cudaGraphSetConditional(h, (open && g <= limit) ? 1u : 0u);
  }
}

// The IF node of the mixed path: run the FP64 residual replacement when the update asked.
__global__ void replace_cond_kernel(const PcgState* st, cudaGraphConditionalHandle h) {
  if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, (st->replace != 0 && st->done == 0) ? 1u : 0u);
}

// Training pair: delta = mask ? 0 : x_star - x_k - z0 (the error left after z0 = P r).
__global__ void pair_delta_kernel(const DevProblem d, const double* __restrict__ xs, const double* __restrict__ xk,
                                  const double* __restrict__ z0, double* __restrict__ delta) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x)
    delta[g] = d.mask[g] ? 0.0 : xs[g] - xk[g] - z0[g];
}

__global__ void __launch_bounds__(kVecBlock) true_residual_kernel(const DevProblem d, const double* __restrict__ b,
                                                                  const double* __restrict__ wl) {
  PcgState* const pst = d.st + blockIdx.y;    // right-hand side blockIdx.y
  double* const part = d.partial + (size_t)blockIdx.y * 4 * d.nblk;
  b += (size_t)blockIdx.y * d.G;
  wl += (size_t)blockIdx.y * d.ne * d.p * d.p * d.p;
  double dot = 0.0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    if (d.mask[g]) continue;
    double s = 0.0;
    s = gather_dof(d, wl, g);
    const double res = b[g] - s;
    dot += res * res;
  }
  double total;
  if (grid_reduce<kVecBlock>(dot, part, &pst->counter, total) && threadIdx.x == 0) pst->aux = total;
}

inline int grid_for(int n, int block, int cap) {
  int g = (n + block - 1) / block;
  return g < 1 ? 1 : (g > cap ? cap : g);
}

// Launches a row-group AMG kernel with the lane count of matrix M, one group per row
// (kRowBlock / lanes rows per block).
#define ROWS_LAUNCH(KERN, M, ...)                                                                   \
  do {                                                                                              \
    const int rows_ = (M).n;                                                                        \
    switch ((M).lanes) {                                                                            \
      case 4: KERN<4><<<dim3(grid_for(rows_, kRowBlock / 4, 8192), d.nrhs), kRowBlock, 0, s>>>(__VA_ARGS__); break;    \
      case 8: KERN<8><<<dim3(grid_for(rows_, kRowBlock / 8, 8192), d.nrhs), kRowBlock, 0, s>>>(__VA_ARGS__); break;    \
      case 16: KERN<16><<<dim3(grid_for(rows_, kRowBlock / 16, 8192), d.nrhs), kRowBlock, 0, s>>>(__VA_ARGS__); break; \
      default: KERN<32><<<dim3(grid_for(rows_, kRowBlock / 32, 8192), d.nrhs), kRowBlock, 0, s>>>(__VA_ARGS__); break; \
    }                                                                                               \
  } while (0)

constexpr double kOmega = 2.0 / 3.0;
constexpr int kCycles = 3;

// One launch of the coarse solve's kernel chain; pdl: with programmatic stream serialisation
// (every kernel of the chain but its first, whose predecessor may be on another stream).
template <typename... KArgs, typename... Args>
cudaError_t launch_chain(void (*kernel)(KArgs...), dim3 grid, int block, cudaStream_t s, bool pdl, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  ++g_kernel_launches;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ROWS_LAUNCH as a link of the chain (sets err; the next link is programmatic)
#define ROWS_CHAIN(KERN, M, ...)                                                                                \
  do {                                                                                                        \
    const int rows_ = (M).n;                                                                                  \
    switch ((M).lanes) {                                                                                      \
      case 4: err = launch_chain(KERN<4>, dim3(grid_for(rows_, kRowBlock / 4, 8192), d.nrhs), kRowBlock, s, pdl, __VA_ARGS__); break;   \
      case 8: err = launch_chain(KERN<8>, dim3(grid_for(rows_, kRowBlock / 8, 8192), d.nrhs), kRowBlock, s, pdl, __VA_ARGS__); break;   \
      case 16: err = launch_chain(KERN<16>, dim3(grid_for(rows_, kRowBlock / 16, 8192), d.nrhs), kRowBlock, s, pdl, __VA_ARGS__); break; \
      default: err = launch_chain(KERN<32>, dim3(grid_for(rows_, kRowBlock / 32, 8192), d.nrhs), kRowBlock, s, pdl, __VA_ARGS__); break; \
    }                                                                                                         \
    pdl = true;                                                                                               \
  } while (0)

// V(1,1) cycle at `level` as down and up passes (smoothed kind): b_c = M b, the next level
// (or the dense inverse), then out = z + N b + Q x_c (z null: out = V b). Two kernels per
// level instead of the cycle's five steps (pre-smoothing from zero, residual, restriction,
// prolongation, post-smoothing); the same linear map up to rounding.
cudaError_t vcycle_fused(const DevProblem& d, int level, const double* b, double* out, const double* z,
                         const PcgState* st, cudaStream_t s, bool& pdl) {
  cudaError_t err;
  if (level == d.nlevels) {
    err = launch_chain(dense_mv_kernel, dim3(grid_for(d.coarsest_n, kRowBlock / 32, 8192), d.nrhs), kRowBlock, s, pdl,
                       d.coarsest_n, d.coarsest_inv, b, out, st);
    pdl = true;
    return err;
  }
  const DevAmgLevel& L = d.levels[level];
  double* bc = (level + 1 == d.nlevels) ? d.cb : d.levels[level + 1].b;
  double* xc = (level + 1 == d.nlevels) ? d.cx : d.levels[level + 1].y;
  ROWS_CHAIN(amg_spmv_kernel, L.M, L.M, b, bc, st, L.A.n);
  if (err != cudaSuccess) return err;
  err = vcycle_fused(d, level + 1, bc, xc, nullptr, st, s, pdl);
  if (err != cudaSuccess) return err;
  const struct { int n, lanes; } up{L.N.n, L.up_lanes};   // N's rows, the level's lane count
  const int nc = (level + 1 == d.nlevels) ? d.coarsest_n : d.levels[level + 1].A.n;
  ROWS_CHAIN(amg_up_kernel, up, L.N, L.Q, b, xc, z, out, st, nc);
  return err;
}

// One K-cycle at `level` for right-hand side b, result in out (out != b).
cudaError_t kcycle(const DevProblem& d, int level, const double* b, double* out, const PcgState* st, cudaStream_t s) {
  if (level == d.nlevels) {
    dense_mv_kernel<<<dim3(grid_for(d.coarsest_n, kRowBlock / 32, 8192), d.nrhs), kRowBlock, 0, s>>>(d.coarsest_n, d.coarsest_inv, b,
                                                                                       out, st);
    ++g_kernel_launches;
    return cudaGetLastError();
  }
  const DevAmgLevel& L = d.levels[level];
  const int n = L.A.n, gb = grid_for(n, 256, 4096);
  amg_jacobi0_kernel<<<gb, 256, 0, s>>>(n, L.dinv, b, L.x, kOmega, st);
  ROWS_LAUNCH(amg_resid_kernel, L.A, L.A, b, L.x, L.t, st);
  g_kernel_launches += 2;
  const int nc = L.R.n;
  cudaError_t err;
  double* ec;
  if (level + 1 == d.nlevels) {
    ROWS_LAUNCH(amg_spmv_kernel, L.R, L.R, L.t, d.cb, st, L.A.n);
    ++g_kernel_launches;
    err = kcycle(d, level + 1, d.cb, d.cx, st, s);   // the dense level: exact
    if (err != cudaSuccess) return err;
    ec = d.cx;
  } else {
    const DevAmgLevel& N = d.levels[level + 1];
    const int gbc = grid_for(nc, 256, 4096);
    ROWS_LAUNCH(amg_spmv_kernel, L.R, L.R, L.t, N.b, st, L.A.n);
    ++g_kernel_launches;
    if ((err = kcycle(d, level + 1, N.b, N.c1, st, s)) != cudaSuccess) return err;
    ROWS_LAUNCH(amg_spmv_kernel, N.A, N.A, N.c1, N.v1, st, N.A.n);
    kc_dots1_kernel<<<1, kKcBlock, 0, s>>>(nc, N.c1, N.v1, N.b, N.scal, st);
    kc_r2_kernel<<<gbc, 256, 0, s>>>(nc, N.v1, N.scal, N.b, st);
    g_kernel_launches += 3;
    if ((err = kcycle(d, level + 1, N.b, N.c2, st, s)) != cudaSuccess) return err;
    ROWS_LAUNCH(amg_spmv_kernel, N.A, N.A, N.c2, N.v2, st, N.A.n);
    kc_dots2_kernel<<<1, kKcBlock, 0, s>>>(nc, N.c2, N.v1, N.v2, N.b, N.scal, st);
    kc_combine_kernel<<<gbc, 256, 0, s>>>(nc, N.c1, N.c2, N.scal, N.y, st);
    g_kernel_launches += 3;
    ec = N.y;
  }
  ROWS_LAUNCH(amg_prolong_add_kernel, L.P, L.P, ec, L.x, st);
  ROWS_LAUNCH(amg_jacobi_post_kernel, L.A, L.A, L.dinv, b, L.x, out, kOmega, st);
  g_kernel_launches += 2;
  return cudaGetLastError();
}
}  // namespace

// Self-check of the integer-op conversion against the conversion instruction, for each
// 64-bit pattern as a binary64; NaN matches NaN whatever the payload.
__global__ void convert_check_kernel(const unsigned long long* __restrict__ bits, long long n,
                                     unsigned long long* mismatches) {
  unsigned long long bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double x = __longlong_as_double((long long)bits[i]);
    const float a = f64_to_f32(x), b = __double2float_rn(x);
    if (!(__float_as_uint(a) == __float_as_uint(b) || (a != a && b != b))) ++bad;
  }
  if (bad) atomicAdd(mismatches, bad);
}

// ================================================================ launchers
cudaError_t launch_geometry(const DevProblem& d, double* geo_out, float* geo32_out, __nv_bfloat16* geo16_out,
                            double* mloc, int* bad,
                            cudaStream_t s) {
  switch (d.p) {
#define GEO_CASE(P_) case P_: geometry_kernel<P_><<<d.ne, P_ * P_ * P_, 0, s>>>(d, geo_out, geo32_out, geo16_out, mloc, bad); ++g_kernel_launches; break;
    GEO_CASE(2) GEO_CASE(3) GEO_CASE(4) GEO_CASE(5) GEO_CASE(6) GEO_CASE(7) GEO_CASE(8) GEO_CASE(9)
#undef GEO_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_gather_shared(const DevProblem& d, const double* wl, const double* xin, double* y, cudaStream_t s) {
  gather_identity_kernel<double, double><<<d.nblk, kVecBlock, 0, s>>>(d, wl, xin, y, d.Gi);
  ++g_kernel_launches;
  return cudaGetLastError();
}
cudaError_t launch_gather_shared_f32(const DevProblem& d, const float* wl, const double* xin, double* y,
                                     cudaStream_t s) {
  gather_identity_kernel<float, double><<<d.nblk, kVecBlock, 0, s>>>(d, wl, xin, y, d.Gi);
  ++g_kernel_launches;
  return cudaGetLastError();
}
cudaError_t launch_gather_shared_f32io(const DevProblem& d, const float* wl, const float* xin, float* y,
                                       cudaStream_t s) {
  gather_identity_kernel<float, float><<<d.nblk, kVecBlock, 0, s>>>(d, wl, xin, y, d.Gi);
  ++g_kernel_launches;
  return cudaGetLastError();
}
cudaError_t launch_gather_identity(const DevProblem& d, const double* wl, const double* xin, double* y, cudaStream_t s) {
  gather_identity_kernel<double, double><<<d.nblk, kVecBlock, 0, s>>>(d, wl, xin, y, 0);
  ++g_kernel_launches;
  return cudaGetLastError();
}
cudaError_t launch_gather_identity_f32(const DevProblem& d, const float* wl, const double* xin, double* y,
                                       cudaStream_t s) {
  gather_identity_kernel<float, double><<<d.nblk, kVecBlock, 0, s>>>(d, wl, xin, y, 0);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_gather_plain(const DevProblem& d, const double* wl, double* y, cudaStream_t s) {
  gather_plain_kernel<<<d.nblk, kVecBlock, 0, s>>>(d, wl, y);
  ++g_kernel_launches;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse_restrict_t(const DevProblem& d, const T* r, const PcgState* st, cudaStream_t s) {
  if (d.nfree == 0) return cudaSuccess;
  switch (d.p) {
#define RS_CASE(P_) case P_: coarse_restrict_kernel<P_, T><<<dim3(d.ne, d.nrhs), P_ * P_, 0, s>>>(d, r, st); ++g_kernel_launches; break;
    RS_CASE(3) RS_CASE(4) RS_CASE(5) RS_CASE(6) RS_CASE(7) RS_CASE(8) RS_CASE(9)
#undef RS_CASE
    default: return cudaErrorInvalidValue;
  }
  vertex_gather_kernel<<<dim3(grid_for(d.nfree, 256, 4096), d.nrhs), 256, 0, s>>>(d, st);
  ++g_kernel_launches;
  return cudaGetLastError();
}
cudaError_t launch_coarse_restrict(const DevProblem& d, const double* r, const PcgState* st, cudaStream_t s) {
  return launch_coarse_restrict_t<double>(d, r, st, s);
}
cudaError_t launch_coarse_restrict_f32(const DevProblem& d, const float* r, const PcgState* st, cudaStream_t s) {
  return launch_coarse_restrict_t<float>(d, r, st, s);
}

// Zc = P_0 Rc: kCycles stationary V(1,1) cycles from zero, or one K-cycle.
// The coarse solve (V-cycle kind: kCycles fused V-cycles, the later ones on the residual)
// as one chain of dependent launches on stream s, then the element-corner copy of the
// correction that the P-sum of the FP32 or double-FP32 path reads.
cudaError_t launch_coarse_solve(const DevProblem& d, const PcgState* st, cudaStream_t s) {
  if (d.nfree == 0) return cudaSuccess;
  bool pdl = false;
  cudaError_t err = d.amg_kind == 1 ? kcycle(d, 0, d.Rc, d.Zc, st, s)
                                    : vcycle_fused(d, 0, d.Rc, d.Zc, nullptr, st, s, pdl);
  if (err != cudaSuccess) return err;
  if (d.nlevels > 0 && d.amg_kind != 1) {
    const DevCsr& A0 = d.levels[0].A;
    for (int c = 1; c < kCycles; ++c) {   // Zc += V (Rc - A0 Zc), the add folded into the up pass
      ROWS_CHAIN(amg_resid_kernel, A0, A0, d.Rc, d.Zc, d.cres, st);
      if (err != cudaSuccess) return err;
      err = vcycle_fused(d, 0, d.cres, d.Zc, d.Zc, st, s, pdl);
      if (err != cudaSuccess) return err;
    }
  }
  if (d.pfp32)
    return launch_chain(coarse_corners_f32_kernel, dim3(grid_for(8 * d.ne, 256, 4096)), 256, s, pdl, d, st);
  if (d.dwk)
    return launch_chain(coarse_corners_dw_kernel, dim3(grid_for(8 * d.ne, 256, 4096), d.nrhs), 256, s, pdl, d, st);
  return cudaSuccess;
}

// Grid of a grid-stride vector kernel: at most cap CTAs (the reduction partials hold d.nblk)
// and no more than are resident at once, so that no CTA waits for a second wave.
template <typename K>
int resident_grid(K kernel, int block, int cap) {
  int dev = 0, nsm = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, block, 0) != cudaSuccess || nsm <= 0 || per <= 0)
    return cap;
  return nsm * per < cap ? nsm * per : cap;
}

cudaError_t launch_psum(const DevProblem& d, int mode, const double* r, double* z, bool pcg, cudaStream_t s) {
  if (d.pfp32) {
    const float* wp = reinterpret_cast<const float*>(d.wp);
    if (pcg) psum_kernel<true, float><<<dim3(d.nblk, d.nrhs), kVecBlock, 0, s>>>(d, mode, wp, r, z);
    else psum_kernel<false, float><<<dim3(d.nblk, d.nrhs), kVecBlock, 0, s>>>(d, mode, wp, r, z);
  } else if (d.dwk) {   // the patch results are pairs (double-FP32 patch solve)
    const dw* wp = reinterpret_cast<const dw*>(d.wp);
    // 48-60 registers: fewer CTAs are resident than d.nblk
    if (pcg)
      psum_dw_kernel<true><<<dim3(resident_grid(psum_dw_kernel<true>, kVecBlock, d.nblk), d.nrhs), kVecBlock, 0, s>>>(
          d, mode, wp, r, z);
    else
      psum_dw_kernel<false><<<dim3(resident_grid(psum_dw_kernel<false>, kVecBlock, d.nblk), d.nrhs), kVecBlock, 0, s>>>(
          d, mode, wp, r, z);
  } else {
    if (pcg) psum_kernel<true, double><<<dim3(d.nblk, d.nrhs), kVecBlock, 0, s>>>(d, mode, d.wp, r, z);
    else psum_kernel<false, double><<<dim3(d.nblk, d.nrhs), kVecBlock, 0, s>>>(d, mode, d.wp, r, z);
  }
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_pcg_init(const DevProblem& d, const double* b, double* r, double* u, double rtol, int maxit,
                            int mixed, int learned, int flexible, int stall_window, double stall_ratio,
                            double nn_theta, double* hist, cudaStream_t s) {
  pcg_init_kernel<<<dim3(d.nblk, d.nrhs), kVecBlock, 0, s>>>(d, b, r, u, rtol, maxit, mixed, learned, flexible, stall_window,
                                                stall_ratio, nn_theta, hist);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_pcg_first_direction(const DevProblem& d, const double* z, double* p, cudaStream_t s) {
  pcg_copy_kernel<<<dim3(d.nblk, d.nrhs), kVecBlock, 0, s>>>(d, z, p);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_pcg_gather_alpha(const DevProblem& d, const double* p, double* f, cudaStream_t s) {
  if (d.fp32) pcg_gather_alpha_kernel<float><<<dim3(d.nblk, d.nrhs), kVecBlock, 0, s>>>(d, reinterpret_cast<const float*>(d.wl), p, f);
  else pcg_gather_alpha_kernel<double><<<dim3(d.nblk, d.nrhs), kVecBlock, 0, s>>>(d, d.wl, p, f);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_pcg_update(const DevProblem& d, const double* p, const double* f, double* u, double* r, double* hist,
                              cudaStream_t s) {
  pcg_update_kernel<<<dim3(d.nblk, d.nrhs), kVecBlock, 0, s>>>(d, p, f, u, r, hist);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_pcg_direction(const DevProblem& d, const double* z, double* p, cudaStream_t s) {
  pcg_direction_kernel<<<dim3(d.nblk, d.nrhs), kVecBlock, 0, s>>>(d, z, p);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_convert_check(const unsigned long long* bits, long long n, unsigned long long* mismatches,
                                 cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  convert_check_kernel<<<grid_for((int)std::min<long long>(n, 1 << 30), 256, 4096), 256, 0, s>>>(bits, n, mismatches);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_pcg_replace(const DevProblem& d, const double* b, const double* wl, double* r, double* hist,
                               cudaStream_t s) {
  pcg_replace_kernel<<<d.nblk, kVecBlock, 0, s>>>(d, b, wl, r, hist);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_true_residual(const DevProblem& d, const double* b, const double* wl, cudaStream_t s) {
  true_residual_kernel<<<dim3(d.nblk, d.nrhs), kVecBlock, 0, s>>>(d, b, wl);
  ++g_kernel_launches;
  return cudaGetLastError();
}


cudaError_t launch_residual_of(const DevProblem& d, const double* wl, const double* v, double* out,
                               const PcgState* st, cudaStream_t s) {
  residual_of_kernel<double><<<d.nblk, kVecBlock, 0, s>>>(d, wl, v, out, st);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_residual_of_f32(const DevProblem& d, const float* wl, const double* v, double* out,
                                   const PcgState* st, cudaStream_t s) {
  residual_of_kernel<float><<<d.nblk, kVecBlock, 0, s>>>(d, wl, v, out, st);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_flex_combine(const DevProblem& d, const double* z, const double* r, cudaStream_t s) {
  flex_combine_kernel<<<d.nblk, kVecBlock, 0, s>>>(d, z, r);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_pair_delta(const DevProblem& d, const double* xs, const double* xk, const double* z0,
                              double* delta, cudaStream_t s) {
  pair_delta_kernel<<<d.nblk, kVecBlock, 0, s>>>(d, xs, xk, z0, delta);
  ++g_kernel_launches;
  return cudaGetLastError();
}


cudaError_t launch_heat_rhs(const DevProblem& d, const double* wl, const double* mN, const double* u_prev,
                            const double* g, double* out, double* norms, cudaStream_t s) {
  heat_rhs_kernel<<<d.nblk, kVecBlock, 0, s>>>(d, wl, mN, u_prev, g, out, norms);
  ++g_kernel_launches;
  return cudaGetLastError();
}


cudaError_t launch_mass_load(const DevProblem& d, const double* mN, const double* sv, double* b, cudaStream_t s) {
  mass_load_kernel<<<d.nblk, kVecBlock, 0, s>>>(d, mN, sv, b);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_split_pairs(long long n, const double* src, dw* dst, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long blocks = std::min<long long>((n + kVecBlock - 1) / kVecBlock, 65536);
  split_pairs_kernel<<<(int)blocks, kVecBlock, 0, s>>>(n, src, dst);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_add_vectors(const DevProblem& d, const double* a, const double* b, double* y, cudaStream_t s) {
  add_vectors_kernel<<<d.nblk, kVecBlock, 0, s>>>(d.G, a, b, y);
  ++g_kernel_launches;
  return cudaGetLastError();
}


cudaError_t launch_loop_cond(const PcgState* st, int nrhs, int* guard, int limit, cudaGraphConditionalHandle h,
                             cudaStream_t s) {
  loop_cond_kernel<<<1, 32, 0, s>>>(st, nrhs, guard, limit, h);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_replace_cond(const PcgState* st, cudaGraphConditionalHandle h, cudaStream_t s) {
  replace_cond_kernel<<<1, 32, 0, s>>>(st, h);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace sem
