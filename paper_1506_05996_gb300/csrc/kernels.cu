// sm_103a kernels of the spectral-element solver. The operator, gather, patch-solve and
// P-sum kernels are templated on the compute type T (double, or float for the mixed
// path); global vectors, dot products and the PCG recurrences are always FP64.
//
//  geometry_kernel      G1..G6 and m at every GLL node from the trilinear map (Sec. 2.3-2.4)
//  ax_local_kernel      local residual r_{ijk;e} of Eq. R / Algorithm 2 (stored or recomputed G)
//  gather kernels       r_N = sum of local copies (Eq. gather), deterministic CSR order
//  schwarz_local_kernel fast-diagonalisation patch solve of Eq. z (Sec. 4.2)
//  coarse kernels       restriction C m^-1 r, AMG V-cycles, prolongation (Sec. 4.1, Eq. coarse)
//  pcg kernels          fused vector updates and dot products of Algorithm 1; alpha, beta
//                       and the stopping test are evaluated on the device
//
// Reductions are deterministic: fixed grid, fixed per-thread ranges, a fixed
// shuffle tree per block, and the last block to finish sums the block partials
// in index order (no spin-waits: a completion counter decides the last block).
#include <cmath>

#include "device.h"

namespace sem {

static thread_local uint64_t g_kernel_launches = 0;
uint64_t kernel_launch_count() { return g_kernel_launches; }

namespace {

__device__ __forceinline__ bool stopped(const PcgState* st) { return st != nullptr && st->done != 0; }

// Mixed path: replace the recursive residual by b - A u (FP64 operator) whenever it has
// dropped by this factor since the last replacement, and before accepting convergence.
constexpr double kReplaceFactor = 1e-3;

// Sum over a block of BS threads; the result is valid in warp 0.
template <int BS>
__device__ __forceinline__ double block_sum(double v) {
  static_assert(BS % 32 == 0 && BS <= 1024, "block size");
  __shared__ double sh[BS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = (lane < BS / 32) ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;
}

// Grid reduction: every block writes its partial; the last block to arrive sums the
// partials in index order. Returns true in all threads of that last block, where
// `total` is valid in thread 0.
template <int BS>
__device__ __forceinline__ bool grid_reduce(double v, double* partial, unsigned int* counter, double& total) {
  __shared__ bool last;
  const double bs = block_sum<BS>(v);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = bs;
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double s = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += BS) s += __ldcg(&partial[i]);
  total = block_sum<BS>(s);
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// G = w |J| J^-1 J^-T (6 entries) and m = w |J| at reference point (a, b, c) from the
// 8 vertices xv[corner*3 + dim]. J[r][s] = d x_r / d xi_s of the trilinear map.
template <typename T>
__device__ __forceinline__ void geom_point(const T* xv, T a, T b, T c, T w, T G[6], T& m, T& det) {
  T J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  const T one = 1, half = 0.5;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const T sa = ((q == 1) | (q == 2) | (q == 5) | (q == 6)) ? one : -one;
    const T sb = ((q == 2) | (q == 3) | (q == 6) | (q == 7)) ? one : -one;
    const T sc = (q >= 4) ? one : -one;
    const T fa = half * (one + sa * a), fb = half * (one + sb * b), fc = half * (one + sc * c);
    const T d0 = half * sa * fb * fc, d1 = half * sb * fa * fc, d2 = half * sc * fa * fb;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const T x = xv[3 * q + r];
      J[r][0] += x * d0;
      J[r][1] += x * d1;
      J[r][2] += x * d2;
    }
  }
  T C[3][3];
  C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  C[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  C[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  C[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  C[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
  const T s = w / det;   // inv(J)[r][c] = C[c][r] / det
  G[0] = s * (C[0][0] * C[0][0] + C[1][0] * C[1][0] + C[2][0] * C[2][0]);
  G[1] = s * (C[0][0] * C[0][1] + C[1][0] * C[1][1] + C[2][0] * C[2][1]);
  G[2] = s * (C[0][0] * C[0][2] + C[1][0] * C[1][2] + C[2][0] * C[2][2]);
  G[3] = s * (C[0][1] * C[0][1] + C[1][1] * C[1][1] + C[2][1] * C[2][1]);
  G[4] = s * (C[0][1] * C[0][2] + C[1][1] * C[1][2] + C[2][1] * C[2][2]);
  G[5] = s * (C[0][2] * C[0][2] + C[1][2] * C[1][2] + C[2][2] * C[2][2]);
  m = w * det;
}

// ----------------------------------------------------------------- geometry
template <int p>
__global__ void __launch_bounds__(p * p * p) geometry_kernel(const DevProblem d, double* geo, float* geo32,
                                                             double* mloc, int* bad) {
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
    gp[6 * p3] = m;
  }
  if (geo32 != nullptr) {   // the same factors rounded to FP32 for the mixed path
    float* gp = geo32 + (size_t)e * 7 * p3 + t;
#pragma unroll
    for (int c = 0; c < 6; ++c) gp[c * p3] = (float)G[c];
    gp[6 * p3] = (float)m;
  }
}

template <typename T> __device__ __forceinline__ const T* geo_of(const DevProblem& d);
template <> __device__ __forceinline__ const double* geo_of<double>(const DevProblem& d) { return d.geo; }
template <> __device__ __forceinline__ const float* geo_of<float>(const DevProblem& d) { return d.geo32; }

// ----------------------------------------------------------------- operator
// D (the GLL differentiation matrix) is centro-antisymmetric, D[n-i][n-m] = -D[i][m], and so
// is D^T. With v = v_e + v_o split into its even and odd parts under m -> n-m,
//   a = D v_e is odd, s = D v_o is even:  (D v)[i] = a_i + s_i,  (D v)[n-i] = -a_i + s_i,
// and a_i, s_i need only the folded half-tables
//   Fp[i][m] = (D[i][m] + D[i][n-m]) / 2,   Fm[i][m] = (D[i][m] - D[i][n-m]) / 2   (m < h)
// applied to e_m = v[m] + v[n-m] and o_m = v[m] - v[n-m] (plus the middle column D[i][h]
// times v[h] when p is odd): about 3/4 of the multiply-adds of the plain product.
template <int p, typename T>
struct FoldedD {
  static constexpr int H = p / 2, ODD = p & 1, HM = H + ODD;
  T Fp[H * H > 0 ? H * H : 1], Fm[HM * H > 0 ? HM * H : 1], Fmid[H > 0 ? H : 1];
};

// Fill the folded tables of M (M = D for the gradient, D^T for the divergence) from
// Dhat[i*p + m] = phi_m'(t_i); called by one thread per entry.
template <int p, typename T>
__device__ __forceinline__ void fold_fill(FoldedD<p, T>& F, const double* __restrict__ D, bool transpose, int t) {
  constexpr int H = p / 2, ODD = p & 1, HM = H + ODD;
  constexpr int n = p - 1;
  auto M = [&](int i, int m) { return transpose ? D[m * p + i] : D[i * p + m]; };
  if (t < H * H) {
    const int i = t / H, m = t % H;
    F.Fp[t] = (T)(0.5 * (M(i, m) + M(i, n - m)));
  }
  if (t < HM * H) {
    const int i = t / H, m = t % H;
    F.Fm[t] = (T)(0.5 * (M(i, m) - M(i, n - m)));
  }
  if (ODD && t < H) F.Fmid[t] = (T)M(t, H);
}

template <int p, typename T>
__device__ __forceinline__ void fold_apply(const FoldedD<p, T>& F, const T (&v)[p], T (&out)[p]) {
  constexpr int H = p / 2, ODD = p & 1;
  constexpr int n = p - 1;
  T e[H], o[H];
#pragma unroll
  for (int m = 0; m < H; ++m) { e[m] = v[m] + v[n - m]; o[m] = v[m] - v[n - m]; }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    T a = ODD ? F.Fmid[i] * v[H] : T(0), sv = 0;
#pragma unroll
    for (int m = 0; m < H; ++m) {
      a += F.Fp[i * H + m] * e[m];
      sv += F.Fm[i * H + m] * o[m];
    }
    out[i] = sv + a;
    out[n - i] = sv - a;
  }
  if (ODD) {
    T sv = 0;
#pragma unroll
    for (int m = 0; m < H; ++m) sv += F.Fm[H * H + m] * o[m];
    out[H] = sv;
  }
}

// One CTA of p*p threads per element (Algorithm 2). Thread (x, y) owns the GLL nodes
// (x, y, k), k = 0..p-1, for the pointwise work, and one line per direction for the
// contractions: the gradient by D along i (line j=x, k=y), j (i=x, k=y) and k (i=x, j=y),
// A/B/C by the geometric factors, the divergence by D^T along the same lines, plus
// lambda m u.
template <int p, bool RECOMP, typename T, typename TX>
__global__ void __launch_bounds__(p * p) ax_local_kernel(const DevProblem d, const TX* __restrict__ x,
                                                         T* __restrict__ wl, const PcgState* st) {
  if (stopped(st)) return;
  constexpr int p2 = p * p, p3 = p * p * p;
  __shared__ FoldedD<p, T> Fg, Fd;
  __shared__ T su[p3], sA[p3], sB[p3], sC[p3];
  __shared__ T sx[24];
  const int e = blockIdx.x, tid = threadIdx.x;
  const int tx = tid % p, ty = tid / p;
  fold_fill<p, T>(Fg, d.D, false, tid);
  fold_fill<p, T>(Fd, d.D, true, tid);
  if (RECOMP)
    for (int q = tid; q < 24; q += p2) sx[q] = (T)d.exyz[(size_t)e * 24 + q];
  const int* l2ge = d.l2g + (size_t)e * p3;
  T uk[p], rk[p], line[p], res[p];
#pragma unroll
  for (int k = 0; k < p; ++k) {
    const int l = tx + p * (ty + p * k);
    const int g = l2ge[l];
    uk[k] = d.mask[g] ? T(0) : (T)x[g];
    su[l] = uk[k];
  }
  __syncthreads();
  // gradient: d/dxi on line (j=tx, k=ty), d/deta on line (i=tx, k=ty), d/dzeta on (i=tx, j=ty)
#pragma unroll
  for (int i = 0; i < p; ++i) line[i] = su[i + p * (tx + p * ty)];
  fold_apply<p, T>(Fg, line, res);
#pragma unroll
  for (int i = 0; i < p; ++i) sA[i + p * (tx + p * ty)] = res[i];
#pragma unroll
  for (int j = 0; j < p; ++j) line[j] = su[tx + p * (j + p * ty)];
  fold_apply<p, T>(Fg, line, res);
#pragma unroll
  for (int j = 0; j < p; ++j) sB[tx + p * (j + p * ty)] = res[j];
  fold_apply<p, T>(Fg, uk, res);
#pragma unroll
  for (int k = 0; k < p; ++k) sC[tx + p * (ty + p * k)] = res[k];
  __syncthreads();
  // pointwise: (A, B, C) = G grad u at the nodes (tx, ty, k); lambda m u kept in registers
  const T lam = (T)d.lambda;
#pragma unroll
  for (int k = 0; k < p; ++k) {
    const int l = tx + p * (ty + p * k);
    const T ur = sA[l], us = sB[l], ut = sC[l];
    T G[6], mm;
    if (!RECOMP) {
      const T* gp = geo_of<T>(d) + (size_t)e * 7 * p3 + l;
#pragma unroll
      for (int c = 0; c < 6; ++c) G[c] = gp[c * p3];
      mm = gp[6 * p3];
    } else {
      T det;
      geom_point<T>(sx, (T)d.tg[tx], (T)d.tg[ty], (T)d.tg[k], (T)(d.rho[tx] * d.rho[ty] * d.rho[k]), G, mm, det);
    }
    sA[l] = G[0] * ur + G[1] * us + G[2] * ut;
    sB[l] = G[1] * ur + G[3] * us + G[4] * ut;
    sC[l] = G[2] * ur + G[4] * us + G[5] * ut;
    rk[k] = lam * mm * uk[k];
  }
  __syncthreads();
  // divergence by D^T: the A lines (j=tx, k=ty) into su, then the B lines (i=tx, k=ty)
  // added into su, then the C line (i=tx, j=ty) and su added in registers
#pragma unroll
  for (int i = 0; i < p; ++i) line[i] = sA[i + p * (tx + p * ty)];
  fold_apply<p, T>(Fd, line, res);
#pragma unroll
  for (int i = 0; i < p; ++i) su[i + p * (tx + p * ty)] = res[i];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < p; ++j) line[j] = sB[tx + p * (j + p * ty)];
  fold_apply<p, T>(Fd, line, res);
#pragma unroll
  for (int j = 0; j < p; ++j) su[tx + p * (j + p * ty)] += res[j];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < p; ++k) line[k] = sC[tx + p * (ty + p * k)];
  fold_apply<p, T>(Fd, line, res);
  T* out = wl + (size_t)e * p3;
#pragma unroll
  for (int k = 0; k < p; ++k) {
    const int l = tx + p * (ty + p * k);
    out[l] = su[l] + res[k] + rk[k];
  }
}

template <typename T>
__global__ void gather_identity_kernel(const DevProblem d, const T* __restrict__ wl,
                                       const double* __restrict__ xin, double* __restrict__ y) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    if (d.mask[g]) { y[g] = xin[g]; continue; }
    T s = 0;
    for (int q = d.g2l_off[g]; q < d.g2l_off[g + 1]; ++q) s += wl[d.g2l_idx[q]];
    y[g] = (double)s;
  }
}

__global__ void gather_plain_kernel(const DevProblem d, const double* __restrict__ wl, double* __restrict__ y) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = d.g2l_off[g]; q < d.g2l_off[g + 1]; ++q) s += wl[d.g2l_idx[q]];
    y[g] = s;
  }
}

// ------------------------------------------------------------ fine Schwarz
// 1/d by Newton-Raphson (x <- x (2 - d x)) from the FP32 reciprocal: two steps take the
// 2^-24 seed error to below FP64 rounding; used for the per-node eigenvalue sums.
__device__ __forceinline__ double recip(double d) {
  double x = (double)(1.0f / (float)d);
  x = x * (2.0 - d * x);
  x = x * (2.0 - d * x);
  return x;
}
__device__ __forceinline__ float recip(float d) { return 1.0f / d; }

// Even/odd folded 1D contractions with the pencil eigenvectors S (P x P, modes 0..NE-1
// even and NE..P-1 odd under row -> P-1-row). fwd: modes t = S^T v; bwd: nodes v = S t.
template <int P, typename T>
__device__ __forceinline__ void pencil_fwd(const T* __restrict__ S, const T (&v)[P], T (&t)[P]) {
  constexpr int H = P / 2, ODD = P & 1, NE = H + ODD;
  T e[H], o[H];
#pragma unroll
  for (int k = 0; k < H; ++k) { e[k] = v[k] + v[P - 1 - k]; o[k] = v[k] - v[P - 1 - k]; }
#pragma unroll
  for (int c = 0; c < NE; ++c) {
    T a = ODD ? S[H * P + c] * v[H] : T(0);
#pragma unroll
    for (int k = 0; k < H; ++k) a += S[k * P + c] * e[k];
    t[c] = a;
  }
#pragma unroll
  for (int c = NE; c < P; ++c) {
    T a = 0;
#pragma unroll
    for (int k = 0; k < H; ++k) a += S[k * P + c] * o[k];
    t[c] = a;
  }
}

template <int P, typename T>
__device__ __forceinline__ void pencil_bwd(const T* __restrict__ S, const T (&t)[P], T (&v)[P]) {
  constexpr int H = P / 2, ODD = P & 1, NE = H + ODD;
#pragma unroll
  for (int k = 0; k < H; ++k) {
    T E = 0, O = 0;
#pragma unroll
    for (int c = 0; c < NE; ++c) E += S[k * P + c] * t[c];
#pragma unroll
    for (int c = NE; c < P; ++c) O += S[k * P + c] * t[c];
    v[k] = E + O;
    v[P - 1 - k] = E - O;
  }
  if (ODD) {
    T E = 0;
#pragma unroll
    for (int c = 0; c < NE; ++c) E += S[H * P + c] * t[c];
    v[H] = E;
  }
}

// One CTA of P*P threads per element (P = n + 3). Thread (x, y) owns one line of the
// extended box in each of the six tensor contractions of Eq. z:
//   t = (S^T x S^T x S^T) r',  t /= 4(l_a/hx^2 + l_b/hy^2 + l_c/hz^2) + lambda,
//   z = (S x S x S) t,        r' = 8/(hx hy hz) r.
template <int P, typename T, typename TR>
__global__ void __launch_bounds__(P * P) schwarz_local_kernel(const DevProblem d, const TR* __restrict__ r,
                                                              T* __restrict__ wp, const PcgState* st) {
  if (stopped(st)) return;
  constexpr int P2 = P * P, P3 = P * P * P;
  __shared__ T sS[P2], sev[P], s1[P3], s2[P3];
  const int e = blockIdx.x, tx = threadIdx.x;
  const int x = tx % P, y = tx / P;
  sS[tx] = (T)d.S[tx];
  if (tx < P) sev[tx] = (T)d.ev[tx];
  const double hxd = d.hbox[3 * e], hyd = d.hbox[3 * e + 1], hzd = d.hbox[3 * e + 2];
  const T ihx2 = (T)(1.0 / (hxd * hxd)), ihy2 = (T)(1.0 / (hyd * hyd)), ihz2 = (T)(1.0 / (hzd * hzd));
  const T scale = (T)(8.0 / (hxd * hyd * hzd));
  T col[P], out[P];
  const int* ipe = d.ip + (size_t)e * P3;
#pragma unroll
  for (int K = 0; K < P; ++K) {
    const int g = ipe[x + P * (y + P * K)];
    col[K] = (g >= 0 && !d.mask[g]) ? (T)r[g] * scale : T(0);
  }
  __syncthreads();
  // along K: line (I=x, J=y)
  pencil_fwd<P, T>(sS, col, out);
#pragma unroll
  for (int c = 0; c < P; ++c) s1[x + P * (y + P * c)] = out[c];
  __syncthreads();
  // along J: line (I=x, c=y)
#pragma unroll
  for (int J = 0; J < P; ++J) col[J] = s1[x + P * (J + P * y)];
  pencil_fwd<P, T>(sS, col, out);
#pragma unroll
  for (int b = 0; b < P; ++b) s2[x + P * (b + P * y)] = out[b];
  __syncthreads();
  // along I: line (b=x, c=y), eigenvalue scaling, and back along I
#pragma unroll
  for (int I = 0; I < P; ++I) col[I] = s2[I + P * (x + P * y)];
  pencil_fwd<P, T>(sS, col, out);
  {
    const T four = 4, lam = (T)d.lambda;
    const T lbc = sev[x] * ihy2 + sev[y] * ihz2;
#pragma unroll
    for (int a = 0; a < P; ++a) out[a] = out[a] * recip(four * (sev[a] * ihx2 + lbc) + lam);
  }
  pencil_bwd<P, T>(sS, out, col);
#pragma unroll
  for (int I = 0; I < P; ++I) s2[I + P * (x + P * y)] = col[I];
  __syncthreads();
  // back along J: line (I=x, c=y)
#pragma unroll
  for (int b = 0; b < P; ++b) out[b] = s2[x + P * (b + P * y)];
  pencil_bwd<P, T>(sS, out, col);
#pragma unroll
  for (int J = 0; J < P; ++J) s1[x + P * (J + P * y)] = col[J];
  __syncthreads();
  // back along K: line (I=x, J=y)
#pragma unroll
  for (int c = 0; c < P; ++c) out[c] = s1[x + P * (y + P * c)];
  pencil_bwd<P, T>(sS, out, col);
  T* outp = wp + (size_t)e * P3;
#pragma unroll
  for (int K = 0; K < P; ++K) outp[x + P * (y + P * K)] = col[K];
}

// ---------------------------------------------------------------- coarse
// Per element R_{IJK;e} = sum over the element's owned nodes of Phi_I(t_i) Phi_J(t_j)
// Phi_K(t_k) r_N; summed over elements this is C m^{-1} r (every node counted once, at
// its owner). Sum-factorised: one thread per (j, k) line contracts i, then (b0, k) pairs
// contract j, then the 8 corners contract k.
template <int p, typename T>
__global__ void __launch_bounds__(p * p) coarse_restrict_kernel(const DevProblem d, const T* __restrict__ r,
                                                                const PcgState* st) {
  if (stopped(st)) return;
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
      const T v = (d.owner[g] == gl && !d.mask[g]) ? r[g] : T(0);
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
    d.Re[(size_t)e * 8 + t] = (double)v;
  }
}

__global__ void vertex_gather_kernel(const DevProblem d, const PcgState* st) {
  if (stopped(st)) return;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < d.nfree; v += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = d.cv_off[v]; q < d.cv_off[v + 1]; ++q) s += d.Re[d.cv_idx[q]];
    d.Rc[v] = s;
  }
}

// AMG kernels. Sparse rows are handled by one warp each (lanes stride over the
// row, then a fixed shuffle tree), so long coarse-level rows do not serialise.
__global__ void amg_jacobi0_kernel(int n, const double* __restrict__ dinv, const double* __restrict__ b,
                                   double* __restrict__ x, double omega, const PcgState* st) {
  if (stopped(st)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = omega * dinv[i] * b[i];
}

__device__ __forceinline__ double warp_row_dot(const DevCsr& A, int row, const double* __restrict__ x, int lane) {
  double s = 0.0;
  for (int q = A.ptr[row] + lane; q < A.ptr[row + 1]; q += 32) s += A.val[q] * x[A.col[q]];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

#define WARP_ROWS(nrows)                                                              \
  const int lane = threadIdx.x & 31;                                                  \
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < (nrows); i += (gridDim.x * blockDim.x) >> 5)

__global__ void amg_resid_kernel(DevCsr A, const double* __restrict__ b, const double* __restrict__ x,
                                 double* __restrict__ t, const PcgState* st) {
  if (stopped(st)) return;
  WARP_ROWS(A.n) {
    const double s = warp_row_dot(A, i, x, lane);
    if (lane == 0) t[i] = b[i] - s;
  }
}

__global__ void amg_spmv_kernel(DevCsr A, const double* __restrict__ x, double* __restrict__ y, const PcgState* st) {
  if (stopped(st)) return;
  WARP_ROWS(A.n) {
    const double s = warp_row_dot(A, i, x, lane);
    if (lane == 0) y[i] = s;
  }
}

__global__ void amg_prolong_add_kernel(DevCsr P, const double* __restrict__ xc, double* __restrict__ x,
                                       const PcgState* st) {
  if (stopped(st)) return;
  WARP_ROWS(P.n) {
    const double s = warp_row_dot(P, i, xc, lane);
    if (lane == 0) x[i] = x[i] + s;
  }
}

__global__ void amg_jacobi_post_kernel(DevCsr A, const double* __restrict__ dinv, const double* __restrict__ b,
                                       const double* __restrict__ x, double* __restrict__ xout, double omega,
                                       const PcgState* st) {
  if (stopped(st)) return;
  WARP_ROWS(A.n) {
    const double s = warp_row_dot(A, i, x, lane);
    if (lane == 0) xout[i] = x[i] + omega * dinv[i] * (b[i] - s);
  }
}
#undef WARP_ROWS

__global__ void add_kernel(int n, double* __restrict__ x, const double* __restrict__ y, const PcgState* st) {
  if (stopped(st)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = x[i] + y[i];
}

// x = Ainv b, one warp per row (dense coarsest level).
__global__ void dense_mv_kernel(int n, const double* __restrict__ Ainv, const double* __restrict__ b,
                                double* __restrict__ x, const PcgState* st) {
  if (stopped(st)) return;
  const int lane = threadIdx.x & 31;
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n; row += (gridDim.x * blockDim.x) >> 5) {
    double s = 0.0;
    for (int c = lane; c < n; c += 32) s += Ainv[(size_t)row * n + c] * b[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[row] = s;
  }
}

// ------------------------------------------------------------ P sum and PCG
template <typename T> __device__ __forceinline__ const T* btab_of(const DevProblem& d);
template <> __device__ __forceinline__ const double* btab_of<double>(const DevProblem& d) { return d.Btab; }
template <> __device__ __forceinline__ const float* btab_of<float>(const DevProblem& d) { return d.Btab32; }
template <typename T> __device__ __forceinline__ const T* zc_of(const DevProblem& d);
template <> __device__ __forceinline__ const double* zc_of<double>(const DevProblem& d) { return d.Zc; }
template <> __device__ __forceinline__ const float* zc_of<float>(const DevProblem& d) { return d.Zc32; }

// z = P r on the free nodes: the patch results summed over every patch containing the
// node (fine part) plus the trilinear interpolation of the coarse correction at the node
// (coarse part, Eq. coarse), accumulated in T; with PCG also z.r and beta (FP64).
template <bool PCG, typename T>
__global__ void __launch_bounds__(kVecBlock) psum_kernel(const DevProblem d, int mode, const T* __restrict__ wp,
                                                         const double* __restrict__ r, double* __restrict__ z) {
  if (PCG && stopped(d.st)) return;
  const int p = d.p, p3 = p * p * p;
  const T* __restrict__ Bt = btab_of<T>(d);
  const T* __restrict__ Zc = zc_of<T>(d);
  double dot = 0.0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    T v = 0;
    if (!d.mask[g]) {
      if (mode & PSUM_IDENT) v += (T)r[g];
      if (mode & PSUM_FINE)
        for (int q = d.pg_off[g]; q < d.pg_off[g + 1]; ++q) v += wp[d.pg_idx[q]];
      if ((mode & PSUM_COARSE) && d.nfree > 0) {
        const int l = d.owner[g], e = l / p3, lr = l % p3;
        const int* ec = d.ecv + (size_t)e * 8;
        const T* B = Bt + 8 * lr;
        T zc = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int cv = ec[c];
          if (cv >= 0) zc += B[c] * Zc[cv];
        }
        v += zc;
      }
    }
    const double vd = (double)v;
    z[g] = vd;
    if (PCG) dot += vd * r[g];
  }
  if (PCG) {
    double total;
    if (grid_reduce<kVecBlock>(dot, d.partial, &d.st->counter, total) && threadIdx.x == 0) {
      PcgState* st = d.st;
      if (!isfinite(total)) { st->status = -6; st->done = 1; }
      if (st->iter > 0) st->beta = total / st->rz;
      st->rz = total;
    }
  }
}

__global__ void to_f32_kernel(int n, const double* __restrict__ a, float* __restrict__ b, const PcgState* st) {
  if (stopped(st)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = (float)a[i];
}

__global__ void __launch_bounds__(kVecBlock) pcg_init_kernel(const DevProblem d, const double* __restrict__ b,
                                                             double* __restrict__ r, double* __restrict__ u,
                                                             double rtol, int maxit, int mixed, double* hist) {
  double dot = 0.0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    const double v = d.mask[g] ? 0.0 : b[g];
    r[g] = v;
    if (mixed) d.r32[g] = (float)v;
    u[g] = 0.0;
    dot += v * v;
  }
  double total;
  if (grid_reduce<kVecBlock>(dot, d.partial, &d.st->counter, total) && threadIdx.x == 0) {
    PcgState* st = d.st;
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
    hist[0] = (total > 0.0) ? 1.0 : 0.0;
    if (!isfinite(total)) { st->status = -6; st->done = 1; }
    else if (total == 0.0) st->done = 1;
    else if (maxit <= 0) { st->status = 1; st->done = 1; }
  }
}

__global__ void pcg_copy_kernel(const DevProblem d, const double* __restrict__ z, double* __restrict__ p) {
  if (stopped(d.st)) return;
  float* __restrict__ p32 = d.st->mixed ? d.p32 : nullptr;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    p[g] = z[g];
    if (p32) p32[g] = (float)z[g];
  }
}

template <typename T>
__global__ void __launch_bounds__(kVecBlock) pcg_gather_alpha_kernel(const DevProblem d, const T* __restrict__ wl,
                                                                     const double* __restrict__ p,
                                                                     double* __restrict__ f) {
  if (stopped(d.st)) return;
  double dot = 0.0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    T s = 0;
    if (!d.mask[g])
      for (int q = d.g2l_off[g]; q < d.g2l_off[g + 1]; ++q) s += wl[d.g2l_idx[q]];
    const double sd = (double)s;
    f[g] = sd;
    dot += p[g] * sd;
  }
  double total;
  if (grid_reduce<kVecBlock>(dot, d.partial, &d.st->counter, total) && threadIdx.x == 0) {
    PcgState* st = d.st;
    st->pf = total;
    if (!(total > 0.0) || !isfinite(total)) { st->status = -6; st->done = 1; }
    else st->alpha = st->rz / total;
  }
}

__global__ void __launch_bounds__(kVecBlock) pcg_update_kernel(const DevProblem d, const double* __restrict__ p,
                                                               const double* __restrict__ f, double* __restrict__ u,
                                                               double* __restrict__ r, double* hist) {
  if (stopped(d.st)) return;
  const double alpha = d.st->alpha;
  float* __restrict__ r32 = d.st->mixed ? d.r32 : nullptr;
  double dot = 0.0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    u[g] = u[g] + alpha * p[g];
    const double rn = r[g] - alpha * f[g];
    r[g] = rn;
    if (r32) r32[g] = (float)rn;
    dot += rn * rn;
  }
  double total;
  if (grid_reduce<kVecBlock>(dot, d.partial, &d.st->counter, total) && threadIdx.x == 0) {
    PcgState* st = d.st;
    st->rr = total;
    const int it = ++st->iter;
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
      for (int q = d.g2l_off[g]; q < d.g2l_off[g + 1]; ++q) s += wl[d.g2l_idx[q]];
      res = b[g] - s;
    }
    r[g] = res;
    d.r32[g] = (float)res;
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
  if (stopped(d.st)) return;
  const double beta = d.st->beta;
  float* __restrict__ p32 = d.st->mixed ? d.p32 : nullptr;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    const double pn = z[g] + beta * p[g];
    p[g] = pn;
    if (p32) p32[g] = (float)pn;
  }
}

__global__ void __launch_bounds__(kVecBlock) true_residual_kernel(const DevProblem d, const double* __restrict__ b,
                                                                  const double* __restrict__ wl) {
  double dot = 0.0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    if (d.mask[g]) continue;
    double s = 0.0;
    for (int q = d.g2l_off[g]; q < d.g2l_off[g + 1]; ++q) s += wl[d.g2l_idx[q]];
    const double res = b[g] - s;
    dot += res * res;
  }
  double total;
  if (grid_reduce<kVecBlock>(dot, d.partial, &d.st->counter, total) && threadIdx.x == 0) d.st->aux = total;
}

inline int grid_for(int n, int block, int cap) {
  int g = (n + block - 1) / block;
  return g < 1 ? 1 : (g > cap ? cap : g);
}

constexpr double kOmega = 2.0 / 3.0;
constexpr int kCycles = 3;

// V(1,1) cycle at `level` for right-hand side b, result in out (out != b).
cudaError_t vcycle(const DevProblem& d, int level, const double* b, double* out, const PcgState* st, cudaStream_t s) {
  if (level == d.nlevels) {
    dense_mv_kernel<<<grid_for(d.coarsest_n * 32, 256, 4096), 256, 0, s>>>(d.coarsest_n, d.coarsest_inv, b, out, st);
    ++g_kernel_launches;
    return cudaGetLastError();
  }
  const DevAmgLevel& L = d.levels[level];
  const int n = L.A.n, gb = grid_for(n, 256, 4096), gw = grid_for(32 * n, 256, 8192);
  amg_jacobi0_kernel<<<gb, 256, 0, s>>>(n, L.dinv, b, L.x, kOmega, st);
  ++g_kernel_launches;
  amg_resid_kernel<<<gw, 256, 0, s>>>(L.A, b, L.x, L.t, st);
  ++g_kernel_launches;
  double* bc = (level + 1 == d.nlevels) ? d.cb : d.levels[level + 1].b;
  double* xc = (level + 1 == d.nlevels) ? d.cx : d.levels[level + 1].y;
  const int nc = L.R.n;
  amg_spmv_kernel<<<grid_for(32 * nc, 256, 8192), 256, 0, s>>>(L.R, L.t, bc, st);
  ++g_kernel_launches;
  cudaError_t err = vcycle(d, level + 1, bc, xc, st, s);
  if (err != cudaSuccess) return err;
  amg_prolong_add_kernel<<<gw, 256, 0, s>>>(L.P, xc, L.x, st);
  ++g_kernel_launches;
  amg_jacobi_post_kernel<<<gw, 256, 0, s>>>(L.A, L.dinv, b, L.x, out, kOmega, st);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace

// ================================================================ launchers
cudaError_t launch_geometry(const DevProblem& d, double* geo_out, float* geo32_out, double* mloc, int* bad,
                            cudaStream_t s) {
  switch (d.p) {
#define GEO_CASE(P_) case P_: geometry_kernel<P_><<<d.ne, P_ * P_ * P_, 0, s>>>(d, geo_out, geo32_out, mloc, bad); ++g_kernel_launches; break;
    GEO_CASE(2) GEO_CASE(3) GEO_CASE(4) GEO_CASE(5) GEO_CASE(6) GEO_CASE(7) GEO_CASE(8) GEO_CASE(9)
#undef GEO_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T, typename TX>
cudaError_t launch_ax_local_t(const DevProblem& d, const TX* x, T* wl, const PcgState* st, cudaStream_t s) {
  switch (d.p) {
#define AX_CASE(P_)                                                                           \
  case P_:                                                                                    \
    if (d.recompute) ax_local_kernel<P_, true, T, TX><<<d.ne, P_ * P_, 0, s>>>(d, x, wl, st);   \
    else ax_local_kernel<P_, false, T, TX><<<d.ne, P_ * P_, 0, s>>>(d, x, wl, st);              \
    ++g_kernel_launches;                                                                      \
    break;
    AX_CASE(3) AX_CASE(4) AX_CASE(5) AX_CASE(6) AX_CASE(7) AX_CASE(8) AX_CASE(9)
#undef AX_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_ax_local(const DevProblem& d, const double* x, double* wl, const PcgState* st, cudaStream_t s) {
  return launch_ax_local_t<double, double>(d, x, wl, st, s);
}
cudaError_t launch_ax_local_f32(const DevProblem& d, const double* x, float* wl, const PcgState* st, cudaStream_t s) {
  return launch_ax_local_t<float, double>(d, x, wl, st, s);
}
cudaError_t launch_ax_local_f32_in32(const DevProblem& d, const float* x, float* wl, const PcgState* st,
                                     cudaStream_t s) {
  return launch_ax_local_t<float, float>(d, x, wl, st, s);
}

cudaError_t launch_gather_identity(const DevProblem& d, const double* wl, const double* xin, double* y, cudaStream_t s) {
  gather_identity_kernel<double><<<d.nblk, kVecBlock, 0, s>>>(d, wl, xin, y);
  ++g_kernel_launches;
  return cudaGetLastError();
}
cudaError_t launch_gather_identity_f32(const DevProblem& d, const float* wl, const double* xin, double* y,
                                       cudaStream_t s) {
  gather_identity_kernel<float><<<d.nblk, kVecBlock, 0, s>>>(d, wl, xin, y);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_gather_plain(const DevProblem& d, const double* wl, double* y, cudaStream_t s) {
  gather_plain_kernel<<<d.nblk, kVecBlock, 0, s>>>(d, wl, y);
  ++g_kernel_launches;
  return cudaGetLastError();
}

template <typename T, typename TR>
cudaError_t launch_schwarz_local_t(const DevProblem& d, const TR* r, T* wp, const PcgState* st, cudaStream_t s) {
  switch (d.P) {
#define SW_CASE(P_) case P_: schwarz_local_kernel<P_, T, TR><<<d.ne, P_ * P_, 0, s>>>(d, r, wp, st); ++g_kernel_launches; break;
    SW_CASE(5) SW_CASE(6) SW_CASE(7) SW_CASE(8) SW_CASE(9) SW_CASE(10) SW_CASE(11)
#undef SW_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
cudaError_t launch_schwarz_local(const DevProblem& d, const double* r, double* wp, const PcgState* st, cudaStream_t s) {
  return launch_schwarz_local_t<double, double>(d, r, wp, st, s);
}
cudaError_t launch_schwarz_local_f32(const DevProblem& d, const double* r, float* wp, const PcgState* st,
                                     cudaStream_t s) {
  return launch_schwarz_local_t<float, double>(d, r, wp, st, s);
}
cudaError_t launch_schwarz_local_f32_in32(const DevProblem& d, const float* r, float* wp, const PcgState* st,
                                          cudaStream_t s) {
  return launch_schwarz_local_t<float, float>(d, r, wp, st, s);
}

template <typename T>
cudaError_t launch_coarse_restrict_t(const DevProblem& d, const T* r, const PcgState* st, cudaStream_t s) {
  if (d.nfree == 0) return cudaSuccess;
  switch (d.p) {
#define RS_CASE(P_) case P_: coarse_restrict_kernel<P_, T><<<d.ne, P_ * P_, 0, s>>>(d, r, st); ++g_kernel_launches; break;
    RS_CASE(3) RS_CASE(4) RS_CASE(5) RS_CASE(6) RS_CASE(7) RS_CASE(8) RS_CASE(9)
#undef RS_CASE
    default: return cudaErrorInvalidValue;
  }
  vertex_gather_kernel<<<grid_for(d.nfree, 256, 4096), 256, 0, s>>>(d, st);
  ++g_kernel_launches;
  return cudaGetLastError();
}
cudaError_t launch_coarse_restrict(const DevProblem& d, const double* r, const PcgState* st, cudaStream_t s) {
  return launch_coarse_restrict_t<double>(d, r, st, s);
}
cudaError_t launch_coarse_restrict_f32(const DevProblem& d, const float* r, const PcgState* st, cudaStream_t s) {
  return launch_coarse_restrict_t<float>(d, r, st, s);
}

// Zc = P_0 Rc: kCycles stationary V(1,1) cycles from zero.
cudaError_t launch_coarse_solve(const DevProblem& d, const PcgState* st, cudaStream_t s) {
  if (d.nfree == 0) return cudaSuccess;
  cudaError_t err = vcycle(d, 0, d.Rc, d.Zc, st, s);
  if (err != cudaSuccess) return err;
  if (d.nlevels == 0) {
    if (d.fp32) {
      to_f32_kernel<<<grid_for(d.nfree, 256, 4096), 256, 0, s>>>(d.nfree, d.Zc, d.Zc32, st);
      ++g_kernel_launches;
    }
    return cudaGetLastError();
  }
  const DevCsr& A0 = d.levels[0].A;
  const int gb = grid_for(A0.n, 256, 4096), gw = grid_for(32 * A0.n, 256, 8192);
  for (int c = 1; c < kCycles; ++c) {
    amg_resid_kernel<<<gw, 256, 0, s>>>(A0, d.Rc, d.Zc, d.cres, st);
    ++g_kernel_launches;
    err = vcycle(d, 0, d.cres, d.ctmp, st, s);
    if (err != cudaSuccess) return err;
    add_kernel<<<gb, 256, 0, s>>>(A0.n, d.Zc, d.ctmp, st);
    ++g_kernel_launches;
  }
  if (d.fp32) {
    to_f32_kernel<<<gb, 256, 0, s>>>(A0.n, d.Zc, d.Zc32, st);
    ++g_kernel_launches;
  }
  return cudaGetLastError();
}

cudaError_t launch_psum(const DevProblem& d, int mode, const double* r, double* z, bool pcg, cudaStream_t s) {
  if (d.fp32) {
    const float* wp = reinterpret_cast<const float*>(d.wp);
    if (pcg) psum_kernel<true, float><<<d.nblk, kVecBlock, 0, s>>>(d, mode, wp, r, z);
    else psum_kernel<false, float><<<d.nblk, kVecBlock, 0, s>>>(d, mode, wp, r, z);
  } else {
    if (pcg) psum_kernel<true, double><<<d.nblk, kVecBlock, 0, s>>>(d, mode, d.wp, r, z);
    else psum_kernel<false, double><<<d.nblk, kVecBlock, 0, s>>>(d, mode, d.wp, r, z);
  }
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_pcg_init(const DevProblem& d, const double* b, double* r, double* u, double rtol, int maxit,
                            int mixed, double* hist, cudaStream_t s) {
  pcg_init_kernel<<<d.nblk, kVecBlock, 0, s>>>(d, b, r, u, rtol, maxit, mixed, hist);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_pcg_first_direction(const DevProblem& d, const double* z, double* p, cudaStream_t s) {
  pcg_copy_kernel<<<d.nblk, kVecBlock, 0, s>>>(d, z, p);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_pcg_gather_alpha(const DevProblem& d, const double* p, double* f, cudaStream_t s) {
  if (d.fp32) pcg_gather_alpha_kernel<float><<<d.nblk, kVecBlock, 0, s>>>(d, reinterpret_cast<const float*>(d.wl), p, f);
  else pcg_gather_alpha_kernel<double><<<d.nblk, kVecBlock, 0, s>>>(d, d.wl, p, f);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_pcg_update(const DevProblem& d, const double* p, const double* f, double* u, double* r, double* hist,
                              cudaStream_t s) {
  pcg_update_kernel<<<d.nblk, kVecBlock, 0, s>>>(d, p, f, u, r, hist);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_pcg_direction(const DevProblem& d, const double* z, double* p, cudaStream_t s) {
  pcg_direction_kernel<<<d.nblk, kVecBlock, 0, s>>>(d, z, p);
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
  true_residual_kernel<<<d.nblk, kVecBlock, 0, s>>>(d, b, wl);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace sem
