// The fine patch-solve kernel (Eq. z): templates shared by k_sw64.cu and k_sw32.cu.
#pragma once

#include "kcommon.cuh"
#include "knum.cuh"

namespace sem {
namespace {

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
  for (int k = 0; k < H; ++k) { e[k] = num_add(v[k], v[P - 1 - k]); o[k] = num_sub(v[k], v[P - 1 - k]); }
#pragma unroll
  for (int c = 0; c < NE; ++c) {
    T a = ODD ? num_mul(S[H * P + c], v[H]) : num_zero<T>();
#pragma unroll
    for (int k = 0; k < H; ++k) num_mac(a, S[k * P + c], e[k]);
    t[c] = a;
  }
#pragma unroll
  for (int c = NE; c < P; ++c) {
    T a = num_zero<T>();
#pragma unroll
    for (int k = 0; k < H; ++k) num_mac(a, S[k * P + c], o[k]);
    t[c] = a;
  }
}

template <int P, typename T>
__device__ __forceinline__ void pencil_bwd(const T* __restrict__ S, const T (&t)[P], T (&v)[P]) {
  constexpr int H = P / 2, ODD = P & 1, NE = H + ODD;
#pragma unroll
  for (int k = 0; k < H; ++k) {
    T E = num_zero<T>(), O = num_zero<T>();
#pragma unroll
    for (int c = 0; c < NE; ++c) num_mac(E, S[k * P + c], t[c]);
#pragma unroll
    for (int c = NE; c < P; ++c) num_mac(O, S[k * P + c], t[c]);
    v[k] = num_add(E, O);
    v[P - 1 - k] = num_sub(E, O);
  }
  if (ODD) {
    T E = num_zero<T>();
#pragma unroll
    for (int c = 0; c < NE; ++c) num_mac(E, S[H * P + c], t[c]);
    v[H] = E;
  }
}

// v times the overlap weight of P^f at DOF g in the kernel's precision (v itself when
// unweighted, the paper's sum).
__device__ __forceinline__ double weighted(const DevProblem& d, double v, int g) {
  return d.pw != nullptr ? v * d.pw[g] : v;
}
__device__ __forceinline__ float weighted(const DevProblem& d, float v, int g) {
  return d.pw32 != nullptr ? v * d.pw32[g] : v;
}
__device__ __forceinline__ dw weighted(const DevProblem& d, dw v, int g) {
  return d.pw != nullptr ? dw_mul(v, dw_split(d.pw[g])) : v;
}

// Plain 1D contractions with a pencil that has no reflection symmetry (an element side on
// a natural boundary): fwd t = S^T v, bwd v = S t.
template <int P, typename T>
__device__ __forceinline__ void plain_fwd(const T* __restrict__ S, const T (&v)[P], T (&t)[P]) {
#pragma unroll
  for (int c = 0; c < P; ++c) {
    T a = num_zero<T>();
#pragma unroll
    for (int k = 0; k < P; ++k) num_mac(a, S[k * P + c], v[k]);
    t[c] = a;
  }
}

template <int P, typename T>
__device__ __forceinline__ void plain_bwd(const T* __restrict__ S, const T (&t)[P], T (&v)[P]) {
#pragma unroll
  for (int k = 0; k < P; ++k) {
    T a = num_zero<T>();
#pragma unroll
    for (int c = 0; c < P; ++c) num_mac(a, S[k * P + c], t[c]);
    v[k] = a;
  }
}

// The pencil of one axis: variant 0 (neighbours on both sides) folded, variants 1..3
// (free low, free high, free both) plain.
template <int P, typename T, bool VAR>
__device__ __forceinline__ void axis_fwd(int v, const T* sS, const T* sSv, const T (&x)[P], T (&t)[P]) {
  if (!VAR || v == 0) pencil_fwd<P, T>(sS, x, t);
  else plain_fwd<P, T>(sSv + (v - 1) * P * P, x, t);
}
template <int P, typename T, bool VAR>
__device__ __forceinline__ void axis_bwd(int v, const T* sS, const T* sSv, const T (&t)[P], T (&x)[P]) {
  if (!VAR || v == 0) pencil_bwd<P, T>(sS, t, x);
  else plain_bwd<P, T>(sSv + (v - 1) * P * P, t, x);
}

// Per-element tables of the patch solve, in the kernel's precision.
template <typename T> __device__ __forceinline__ const T* swd_of(const DevProblem& d);
template <> __device__ __forceinline__ const double* swd_of<double>(const DevProblem& d) { return d.swd; }
template <> __device__ __forceinline__ const float* swd_of<float>(const DevProblem& d) { return d.swd32; }
template <> __device__ __forceinline__ const dw* swd_of<dw>(const DevProblem& d) { return d.swddw; }

// The diagonal of the fast diagonalisation (Eq. z) of every element patch, inverted and
// times the patch scale 8/(hx hy hz): dg[e][(b + P c) + P^2 a] = (8/(hx hy hz)) / (4(l_a/hx^2 +
// l_b/hy^2 + l_c/hz^2) + lambda) with each axis' pencil eigenvalues. The scale commutes with
// the contractions, so it is applied here once instead of to every input node. One CTA of
// P*P threads per element; run once per handle (and again when the Dirichlet set changes
// the pencils), so that the patch kernels spend no divisions on it.
template <int P, typename T, bool VAR>
__global__ void __launch_bounds__(P * P) sw_diag_kernel(const DevProblem d, T* __restrict__ dg) {
  constexpr int P2 = P * P, P3 = P * P * P;
  const int e = blockIdx.x, tx = threadIdx.x, x = tx % P, y = tx / P;
  const double hxd = d.hbox[3 * e], hyd = d.hbox[3 * e + 1], hzd = d.hbox[3 * e + 2];
  const T ihx2 = (T)(1.0 / (hxd * hxd)), ihy2 = (T)(1.0 / (hyd * hyd)), ihz2 = (T)(1.0 / (hzd * hzd));
  const T scale = (T)(8.0 / (hxd * hyd * hzd));
  const int vb = VAR ? d.pvar[e] : 0;
  const int vx = vb & 3, vy = (vb >> 2) & 3, vz = (vb >> 4) & 3;
  const double* evx = vx ? d.evv + (vx - 1) * P : d.ev;
  const double* evy = vy ? d.evv + (vy - 1) * P : d.ev;
  const double* evz = vz ? d.evv + (vz - 1) * P : d.ev;
  const T four = 4, lam = (T)d.lambda;
  const T lbc = (T)evy[x] * ihy2 + (T)evz[y] * ihz2;
  T* out = dg + (size_t)e * P3 + tx;
#pragma unroll
  for (int a = 0; a < P; ++a) out[a * P2] = scale * recip(four * ((T)evx[a] * ihx2 + lbc) + lam);
}

// One CTA of P*P threads per element (P = n + 3). Thread (x, y) owns one line of the
// extended box in each of the six tensor contractions of Eq. z:
//   t = (S^T x S^T x S^T) r',  t /= 4(l_a/hx^2 + l_b/hy^2 + l_c/hz^2) + lambda,
//   z = (S x S x S) t,        r' = 8/(hx hy hz) r.
template <int P, typename T, int EPB>
constexpr int sw_smem_bytes() {
  return (int)((4 * P * P + EPB * 2 * P * P * P) * sizeof(T));
}

// VAR: some element sides lie on a natural boundary (d.pvar != null), so each axis picks its
// pencil; without, every axis takes the folded one (the same code as before variants).
// T = dw (the FP64 interface on the FP32 pipe) stores its patch results as pairs, which the
// P-sum adds in the same arithmetic.
// Resident CTAs per SM asked of the compiler for the double-FP32 kernels, whose pair
// arithmetic is latency-bound at the occupancy its register count would allow: at most 72
// registers a thread (the binary64 and FP32 instantiations keep the compiler's choice).
constexpr int dw_min_blocks(int threads) {
  return 65536 / (((threads + 31) / 32) * 32 * 72) > 0 ? 65536 / (((threads + 31) / 32) * 32 * 72) : 1;
}

template <int P, typename T, typename TR, int EPB, bool VAR>
__device__ __forceinline__ void schwarz_local_body(const DevProblem& d, const TR* __restrict__ r, T* __restrict__ wp,
                                                   const PcgState* st) {
  using TW = T;
  constexpr int P2 = P * P, P3 = P * P * P;
  if constexpr (!std::is_same<T, float>::value) {   // block solves run in the FP64 arithmetics only
    st = st_rhs(st);
    r += (size_t)blockIdx.y * d.G;                   // right-hand side blockIdx.y of a block solve
    wp += (size_t)blockIdx.y * d.ne * P3;
  }
  if (stopped(st)) return;
  __shared__ T sS[P2], sSv[3 * P2], s1_all[EPB * P3], s2_all[EPB * P3];
  // double-FP32: the element's inverted diagonal, copied asynchronously at the start of the
  // element so that its loads overlap the forward contractions (dynamic shared memory,
  // EPB P^3 pairs; none in the other instantiations)
  extern __shared__ __align__(16) unsigned char sw_dyn[];
  T* sdg_all = reinterpret_cast<T*>(sw_dyn);
  const int grp = threadIdx.x / P2, tx = threadIdx.x % P2;
  T* s1 = s1_all + grp * P3;
  T* s2 = s2_all + grp * P3;
  const int x = tx % P, y = tx / P;
  if (threadIdx.x < P2) sS[threadIdx.x] = num_const<T>(d.S[threadIdx.x]);
  if (VAR)
    for (int q = threadIdx.x; q < 3 * P2; q += blockDim.x) sSv[q] = num_const<T>(d.Sv[q]);
  // element groups strided over the grid (the grid may be capped below the group count to
  // leave SMs to the concurrent coarse branch); every thread of a CTA runs the same rounds
  const int ngroups = (d.ne + EPB - 1) / EPB;
  for (int blk = blockIdx.x; blk < ngroups; blk += gridDim.x) {
  const int e_raw = blk * EPB + grp;
  const bool active = e_raw < d.ne;            // a short last CTA recomputes its last element
  const int e = active ? e_raw : d.ne - 1;
  // pencil variant per axis (bit 2a: free low side, bit 2a+1: free high side)
  const int vb = VAR ? d.pvar[e] : 0;
  const int vx = vb & 3, vy = (vb >> 2) & 3, vz = (vb >> 4) & 3;
  T col[P], out[P];
  if constexpr (kIsDw<T>) {   // thread (x, y) copies the P entries it scales later
    const T* dge = swd_of<T>(d) + (size_t)e * P3 + tx;
    T* sdg = sdg_all + grp * P3 + tx;
#pragma unroll
    for (int a = 0; a < P; ++a)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(sdg + a * P2)),
                   "l"(dge + a * P2)
                   : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  const int* ipe = d.ip + (size_t)e * P3;
#pragma unroll
  for (int K = 0; K < P; ++K) {
    const int g = ipe[x + P * (y + P * K)];
    const int gs = g >= 0 ? g : 0;   // r and the mask read together, the mask applied after
    const TR rv = r[gs];
    const bool use = g >= 0 && !d.mask[gs];
    T v = use ? num_load<T>(rv) : num_zero<T>();
    if (g >= 0) v = weighted(d, v, g);
    col[K] = v;
  }
  __syncthreads();
  // along K: line (I=x, J=y)
  axis_fwd<P, T, VAR>(vz, sS, sSv, col, out);
#pragma unroll
  for (int c = 0; c < P; ++c) s1[x + P * (y + P * c)] = out[c];
  __syncthreads();
  // along J: line (I=x, c=y)
#pragma unroll
  for (int J = 0; J < P; ++J) col[J] = s1[x + P * (J + P * y)];
  axis_fwd<P, T, VAR>(vy, sS, sSv, col, out);
#pragma unroll
  for (int b = 0; b < P; ++b) s2[x + P * (b + P * y)] = out[b];
  __syncthreads();
  // along I: line (b=x, c=y), eigenvalue scaling, and back along I
#pragma unroll
  for (int I = 0; I < P; ++I) col[I] = s2[I + P * (x + P * y)];
  axis_fwd<P, T, VAR>(vx, sS, sSv, col, out);
  if constexpr (kIsDw<T>) {
    asm volatile("cp.async.wait_all;" ::: "memory");   // this thread's own copies
    const T* sdg = sdg_all + grp * P3 + tx;
#pragma unroll
    for (int a = 0; a < P; ++a) out[a] = num_mul(out[a], sdg[a * P2]);
  } else {
    const T* dge = swd_of<T>(d) + (size_t)e * P3 + tx;
#pragma unroll
    for (int a = 0; a < P; ++a) out[a] = num_mul(out[a], dge[a * P2]);
  }
  axis_bwd<P, T, VAR>(vx, sS, sSv, out, col);
#pragma unroll
  for (int I = 0; I < P; ++I) s2[I + P * (x + P * y)] = col[I];
  __syncthreads();
  // back along J: line (I=x, c=y)
#pragma unroll
  for (int b = 0; b < P; ++b) out[b] = s2[x + P * (b + P * y)];
  axis_bwd<P, T, VAR>(vy, sS, sSv, out, col);
#pragma unroll
  for (int J = 0; J < P; ++J) s1[x + P * (J + P * y)] = col[J];
  __syncthreads();
  // back along K: line (I=x, J=y)
#pragma unroll
  for (int c = 0; c < P; ++c) out[c] = s1[x + P * (y + P * c)];
  axis_bwd<P, T, VAR>(vz, sS, sSv, out, col);
  if (active) {
    TW* outp = wp + (size_t)e * P3;
#pragma unroll
    for (int K = 0; K < P; ++K) outp[x + P * (y + P * K)] = num_store<TW>(col[K]);
  }
  }
}


// The double-FP32 patch solve as a loop over its six line stages, in place in one shared
// buffer per element: a stage's lines partition the box, so every thread reads and rewrites
// only its own line, and a barrier separates the stages. Each contraction appears once in
// the code (the unrolled form of schwarz_local_body, six copies of the pair arithmetic,
// stalled on instruction fetch), and the shared memory is half. The arithmetic is the
// unrolled form's, in the same order.
//   stage s < 3 contracts axis K, J, I forward; stage s >= 3 the axis of stage 5 - s backward
//   axis K: line (I = x, J = y), nodes at x + P y + P^2 k
//   axis J: line (I = x, c = y), nodes at x + P^2 y + P k
//   axis I: line (b = x, c = y), nodes at P x + P^2 y + k
template <int P, typename TR, int EPB, bool VAR>
__device__ __forceinline__ void schwarz_dw_body(const DevProblem& d, const TR* __restrict__ r, dw* __restrict__ wp,
                                                const PcgState* st) {
  using T = dw;
  constexpr int P2 = P * P, P3 = P * P * P;
  st = st_rhs(st);
  r += (size_t)blockIdx.y * d.G;                   // right-hand side blockIdx.y of a block solve
  wp += (size_t)blockIdx.y * d.ne * P3;
  if (stopped(st)) return;
  __shared__ T sS[P2], sSv[3 * P2], sb_all[EPB * P3];
  extern __shared__ __align__(16) unsigned char sw_dyn[];   // the element's diagonal (EPB P^3 pairs)
  T* sdg_all = reinterpret_cast<T*>(sw_dyn);
  const int grp = threadIdx.x / P2, tx = threadIdx.x % P2;
  T* sb = sb_all + grp * P3;
  const int x = tx % P, y = tx / P;
  if (threadIdx.x < P2) sS[threadIdx.x] = num_const<T>(d.S[threadIdx.x]);
  if (VAR)
    for (int q = threadIdx.x; q < 3 * P2; q += blockDim.x) sSv[q] = num_const<T>(d.Sv[q]);
  const int ngroups = (d.ne + EPB - 1) / EPB;
  for (int blk = blockIdx.x; blk < ngroups; blk += gridDim.x) {
    const int e_raw = blk * EPB + grp;
    const bool active = e_raw < d.ne;            // a short last CTA recomputes its last element
    const int e = active ? e_raw : d.ne - 1;
    const int vb = VAR ? d.pvar[e] : 0;
    const int vx = vb & 3, vy = (vb >> 2) & 3, vz = (vb >> 4) & 3;
    {   // thread (x, y) copies the P diagonal entries it scales after the third stage
      const T* dge = d.swddw + (size_t)e * P3 + tx;
      T* sdg = sdg_all + grp * P3 + tx;
#pragma unroll
      for (int a = 0; a < P; ++a)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(sdg + a * P2)),
                     "l"(dge + a * P2)
                     : "memory");
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    T col[P], out[P];
    const int* ipe = d.ip + (size_t)e * P3;
#pragma unroll
    for (int K = 0; K < P; ++K) {
      const int g = ipe[x + P * (y + P * K)];
      const int gs = g >= 0 ? g : 0;   // r and the mask read together, the mask applied after
      const TR rv = r[gs];
      const bool use = g >= 0 && !d.mask[gs];
      T v = use ? num_load<T>(rv) : num_zero<T>();
      if (g >= 0) v = weighted(d, v, g);
      col[K] = v;
    }
    __syncthreads();   // sS ready (first group); the previous group's last reads of sb done
#pragma unroll 1
    for (int stg = 0; stg < 6; ++stg) {
      const int ax = stg < 3 ? stg : 5 - stg;   // 0: K, 1: J, 2: I
      const int base = ax == 0 ? x + P * y : (ax == 1 ? x + P2 * y : P * x + P2 * y);
      const int stride = ax == 0 ? P2 : (ax == 1 ? P : 1);
      const int v = ax == 0 ? vz : (ax == 1 ? vy : vx);
      if (stg > 0) {
        __syncthreads();
#pragma unroll
        for (int k = 0; k < P; ++k) col[k] = sb[base + stride * k];
      }
      if (stg < 3) axis_fwd<P, T, VAR>(v, sS, sSv, col, out);
      else axis_bwd<P, T, VAR>(v, sS, sSv, col, out);
      if (stg == 2) {   // the eigenvalue scaling (with the patch scale), line (b = x, c = y)
        asm volatile("cp.async.wait_all;" ::: "memory");   // this thread's own copies
        const T* sdg = sdg_all + grp * P3 + tx;
#pragma unroll
        for (int a = 0; a < P; ++a) out[a] = num_mul(out[a], sdg[a * P2]);
      }
      if (stg < 5) {
#pragma unroll
        for (int k = 0; k < P; ++k) sb[base + stride * k] = out[k];
      } else if (active) {
        T* outp = wp + (size_t)e * P3;
#pragma unroll
        for (int k = 0; k < P; ++k) outp[base + stride * k] = out[k];
      }
    }
  }
}

// The kernels: the binary64 and FP32 instantiations with the compiler's register choice,
// the double-FP32 one with at most 96 registers a thread (dw_min_blocks).
template <int P, typename T, typename TR, int EPB, bool VAR>
__global__ void __launch_bounds__(EPB * P * P) schwarz_local_kernel(const DevProblem d, const TR* __restrict__ r,
                                                                    T* __restrict__ wp, const PcgState* st) {
  schwarz_local_body<P, T, TR, EPB, VAR>(d, r, wp, st);
}
template <int P, typename T, typename TR, int EPB, bool VAR>
__global__ void __launch_bounds__(EPB * P * P, dw_min_blocks(EPB * P * P))
    schwarz_local_kernel_dw(const DevProblem d, const TR* __restrict__ r, T* __restrict__ wp, const PcgState* st) {
  if constexpr (kIsDw<T>) schwarz_dw_body<P, TR, EPB, VAR>(d, r, wp, st);
}

template <int P, typename T, int EPB>
constexpr bool sw_tile_supported() {
  return sw_smem_bytes<P, T, EPB>() <= 48 * 1024 && (EPB == 1 || EPB * P * P <= 256);
}

template <int P, typename T>
bool sw_tile_ok_P(int epb) {
  switch (epb) {
    case 1: return sw_tile_supported<P, T, 1>();
    case 2: return sw_tile_supported<P, T, 2>();
    case 4: return sw_tile_supported<P, T, 4>();
    case 8: return sw_tile_supported<P, T, 8>();
    default: return false;
  }
}

template <typename T>
bool sw_tile_ok_t(int P, int epb) {
  switch (P) {
    case 5: return sw_tile_ok_P<5, T>(epb);
    case 6: return sw_tile_ok_P<6, T>(epb);
    case 7: return sw_tile_ok_P<7, T>(epb);
    case 8: return sw_tile_ok_P<8, T>(epb);
    case 9: return sw_tile_ok_P<9, T>(epb);
    case 10: return sw_tile_ok_P<10, T>(epb);
    case 11: return sw_tile_ok_P<11, T>(epb);
    default: return false;
  }
}

template <int P, typename T, typename TR, int EPB>
cudaError_t launch_sw_epb(const DevProblem& d, const TR* r, T* wp, const PcgState* st, cudaStream_t s) {
  if constexpr (sw_tile_supported<P, T, EPB>()) {
    int grid = (d.ne + EPB - 1) / EPB;
    auto kernel = kIsDw<T> ? (d.pvar != nullptr ? schwarz_local_kernel_dw<P, T, TR, EPB, true>
                                                : schwarz_local_kernel_dw<P, T, TR, EPB, false>)
                           : (d.pvar != nullptr ? schwarz_local_kernel<P, T, TR, EPB, true>
                                                : schwarz_local_kernel<P, T, TR, EPB, false>);
    if (d.sw_reserve_sms > 0) {
      // as many CTAs as fit on all but sw_reserve_sms SMs, so that slots stay free
      int dev = 0, nsm = 0, per_sm = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, EPB * P * P,
                                                    kIsDw<T> ? EPB * P * P * P * (int)sizeof(T) : 0);
      const int cap = (nsm - d.sw_reserve_sms) * per_sm;
      if (cap > 0 && cap < grid) grid = cap;
    }
    constexpr int dyn = kIsDw<T> ? EPB * P * P * P * (int)sizeof(T) : 0;
    if (dyn > 0) {
      cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
      // all of the unified L1 / shared storage as shared memory, so that the shared memory of
      // the resident CTAs does not cap them below the register limit
      if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      if (e != cudaSuccess) return e;
    }
    kernel<<<dim3(grid, d.nrhs), EPB * P * P, dyn, s>>>(d, r, wp, st);
    count_launch();
    return cudaGetLastError();
  } else {
    return cudaErrorInvalidConfiguration;
  }
}

template <int P, typename T, typename TR>
cudaError_t launch_sw_P(const DevProblem& d, const TR* r, T* wp, const PcgState* st, cudaStream_t s) {
  switch (std::is_same<T, float>::value ? d.epb_sw32 : (kIsDw<T> ? d.epb_swdw : d.epb_sw)) {
    case 2: return launch_sw_epb<P, T, TR, 2>(d, r, wp, st, s);
    case 4: return launch_sw_epb<P, T, TR, 4>(d, r, wp, st, s);
    case 8: return launch_sw_epb<P, T, TR, 8>(d, r, wp, st, s);
    default: return launch_sw_epb<P, T, TR, 1>(d, r, wp, st, s);
  }
}

template <int P, typename T>
cudaError_t launch_sw_diag_P(const DevProblem& d, T* dg, cudaStream_t s) {
  if (d.pvar != nullptr) sw_diag_kernel<P, T, true><<<d.ne, P * P, 0, s>>>(d, dg);
  else sw_diag_kernel<P, T, false><<<d.ne, P * P, 0, s>>>(d, dg);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sw_diag_t(const DevProblem& d, T* dg, cudaStream_t s) {
  if (d.ne == 0) return cudaSuccess;
  switch (d.P) {
    case 5: return launch_sw_diag_P<5, T>(d, dg, s);
    case 6: return launch_sw_diag_P<6, T>(d, dg, s);
    case 7: return launch_sw_diag_P<7, T>(d, dg, s);
    case 8: return launch_sw_diag_P<8, T>(d, dg, s);
    case 9: return launch_sw_diag_P<9, T>(d, dg, s);
    case 10: return launch_sw_diag_P<10, T>(d, dg, s);
    case 11: return launch_sw_diag_P<11, T>(d, dg, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, typename TR>
cudaError_t launch_schwarz_local_t(const DevProblem& d, const TR* r, T* wp, const PcgState* st, cudaStream_t s) {
  switch (d.P) {
    case 5: return launch_sw_P<5, T, TR>(d, r, wp, st, s);
    case 6: return launch_sw_P<6, T, TR>(d, r, wp, st, s);
    case 7: return launch_sw_P<7, T, TR>(d, r, wp, st, s);
    case 8: return launch_sw_P<8, T, TR>(d, r, wp, st, s);
    case 9: return launch_sw_P<9, T, TR>(d, r, wp, st, s);
    case 10: return launch_sw_P<10, T, TR>(d, r, wp, st, s);
    case 11: return launch_sw_P<11, T, TR>(d, r, wp, st, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace
}  // namespace sem
