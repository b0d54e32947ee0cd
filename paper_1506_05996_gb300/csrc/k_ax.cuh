// The operator kernel (Eq. R, Algorithm 2): templates shared by k_ax64.cu and k_ax32.cu.
#pragma once

#include "kcommon.cuh"
#include "knum.cuh"

namespace sem {
namespace {

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
    F.Fp[t] = num_const<T>(0.5 * (M(i, m) + M(i, n - m)));
  }
  if (t < HM * H) {
    const int i = t / H, m = t % H;
    F.Fm[t] = num_const<T>(0.5 * (M(i, m) - M(i, n - m)));
  }
  if (ODD && t < H) F.Fmid[t] = num_const<T>(M(t, H));
}

template <int p, typename T>
__device__ __forceinline__ void fold_apply(const FoldedD<p, T>& F, const T (&v)[p], T (&out)[p]) {
  constexpr int H = p / 2, ODD = p & 1;
  constexpr int n = p - 1;
  T e[H], o[H];
#pragma unroll
  for (int m = 0; m < H; ++m) { e[m] = num_add(v[m], v[n - m]); o[m] = num_sub(v[m], v[n - m]); }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    T a = ODD ? num_mul(F.Fmid[i], v[H]) : num_zero<T>(), sv = num_zero<T>();
#pragma unroll
    for (int m = 0; m < H; ++m) {
      num_mac(a, F.Fp[i * H + m], e[m]);
      num_mac(sv, F.Fm[i * H + m], o[m]);
    }
    out[i] = num_add(sv, a);
    out[n - i] = num_sub(sv, a);
  }
  if (ODD) {
    T sv = num_zero<T>();
#pragma unroll
    for (int m = 0; m < H; ++m) num_mac(sv, F.Fm[H * H + m], o[m]);
    out[H] = sv;
  }
}

// One group of p*p threads per element (Algorithm 2), EPB elements per CTA (a tile shape
// chosen per order by the autotuner). Thread (x, y) owns the GLL nodes (x, y, k),
// k = 0..p-1, for the pointwise work, and one line per direction for the contractions:
// the gradient by D along i (line j=x, k=y), j (i=x, k=y) and k (i=x, j=y), A/B/C by the
// geometric factors, the divergence by D^T along the same lines, plus lambda m u.
// Shared-memory slab of one element: node (i, j, k) at i + RS j + PS k. A warp's 32 threads
// (x = 0..7, y = 0..3 at p = 8) read the rows along i at (q, x, y), along j at (x, q, y) and
// along k at (x, y, q). With the plain strides (8, 64) the rows along i start 32 bytes apart
// and fall into 4 bank groups (8-way conflicts for 4-byte words, 16-way for 8-byte ones), the
// rows along j into 8 (4-way); a row stride of 9 (PS = 72) makes i and j conflict-free for
// 4-byte words and 2 ways for 8-byte ones (the minimum), at 2 (4-byte) or 3 (8-byte) ways
// along k. Other orders keep the plain layout.
template <int p>
struct Slab {
  static constexpr int RS = (p == 8) ? p + 1 : p, PS = RS * p, N = PS * p;
  static __device__ __forceinline__ int at(int i, int j, int k) { return i + RS * j + PS * k; }
};

template <int p, typename T, int EPB>
constexpr int ax_smem_bytes() {
  return (int)(2 * sizeof(FoldedD<p, T>) + EPB * (4 * Slab<p>::N + 24) * sizeof(T));
}

// DIRECT (operator application y = A x with the interior-first numbering, d.Gi > 0): an
// element-interior node has one copy, so its result goes straight to y (x where masked) at
// its computed DOF, without an index read; only the other nodes go to wl for the gather.
// TG: the stored factors' type (T, or BF16 under SEM_PREC_BF16 with T = float).
// T = dw (the FP64 interface on the FP32 pipe) reads the factors as pairs and stores its
// local results joined to binary64 (TW = LocalOf<T>).
template <int p, bool RECOMP, typename T, typename TX, int EPB, bool DIRECT, typename TG>
__global__ void __launch_bounds__(EPB * p * p) ax_local_kernel(const DevProblem d, const TX* __restrict__ x,
                                                               typename LocalOf<T>::type* __restrict__ wl,
                                                               const PcgState* st, TX* __restrict__ yd) {
  using TW = typename LocalOf<T>::type;
  constexpr int p2 = p * p, p3 = p * p * p;
  if constexpr (!std::is_same<T, float>::value) {   // block solves run in the FP64 arithmetics only
    st = st_rhs(st);
    x += (size_t)blockIdx.y * d.G;                   // right-hand side blockIdx.y of a block solve
    wl += (size_t)blockIdx.y * d.ne * p3;
    if (DIRECT) yd += (size_t)blockIdx.y * d.G;
  }
  if (stopped(st)) return;
  __shared__ FoldedD<p, T> Fg, Fd;
  using SL = Slab<p>;
  __shared__ T su_all[EPB * SL::N], sA_all[EPB * SL::N], sB_all[EPB * SL::N], sC_all[EPB * SL::N];
  __shared__ T sx_all[EPB * 24];
  const int grp = threadIdx.x / p2, tid = threadIdx.x % p2;
  const int e_raw = blockIdx.x * EPB + grp;
  const bool active = e_raw < d.ne;            // a short last CTA recomputes its last element
  const int e = active ? e_raw : d.ne - 1;
  T* su = su_all + grp * SL::N;
  T* sA = sA_all + grp * SL::N;
  T* sB = sB_all + grp * SL::N;
  T* sC = sC_all + grp * SL::N;
  T* sx = sx_all + grp * 24;
  const int tx = tid % p, ty = tid / p;
  fold_fill<p, T>(Fg, d.D, false, threadIdx.x);
  fold_fill<p, T>(Fd, d.D, true, threadIdx.x);
  if constexpr (RECOMP)
    for (int q = tid; q < 24; q += p2) sx[q] = (T)d.exyz[(size_t)e * 24 + q];
  const int* l2ge = d.l2g + (size_t)e * p3;
  constexpr int m = p - 2;
  // interior line (tx, ty inside): DOF of node k is gi0 + m^2 (k - 1) for 1 <= k <= p - 2
  const bool inner_xy = DIRECT && tx >= 1 && tx <= p - 2 && ty >= 1 && ty <= p - 2;
  const int gi0 = e * m * m * m + (tx - 1) + m * (ty - 1);
  T uk[p], rk[p], line[p], res[p];
  unsigned masked = 0;
#pragma unroll
  for (int k = 0; k < p; ++k) {
    const int l = tx + p * (ty + p * k);
    const bool inner = inner_xy && k >= 1 && k <= p - 2;
    const int g = inner ? gi0 + m * m * (k - 1) : l2ge[l];
    const bool mk = d.mask[g] != 0;
    if (DIRECT && mk) masked |= 1u << k;
    uk[k] = mk ? num_zero<T>() : num_load<T>(x[g]);
    su[SL::at(tx, ty, k)] = uk[k];
  }
  __syncthreads();
  // gradient: d/dxi on line (j=tx, k=ty), d/deta on line (i=tx, k=ty), d/dzeta on (i=tx, j=ty)
#pragma unroll
  for (int i = 0; i < p; ++i) line[i] = su[SL::at(i, tx, ty)];
  fold_apply<p, T>(Fg, line, res);
#pragma unroll
  for (int i = 0; i < p; ++i) sA[SL::at(i, tx, ty)] = res[i];
#pragma unroll
  for (int j = 0; j < p; ++j) line[j] = su[SL::at(tx, j, ty)];
  fold_apply<p, T>(Fg, line, res);
#pragma unroll
  for (int j = 0; j < p; ++j) sB[SL::at(tx, j, ty)] = res[j];
  fold_apply<p, T>(Fg, uk, res);
#pragma unroll
  for (int k = 0; k < p; ++k) sC[SL::at(tx, ty, k)] = res[k];
  __syncthreads();
  // pointwise: (A, B, C) = G grad u at the nodes (tx, ty, k); lambda m u kept in registers
  const bool lam_zero = d.lambda == 0.0;
#pragma unroll
  for (int k = 0; k < p; ++k) {
    const int l = tx + p * (ty + p * k);
    const int ls = SL::at(tx, ty, k);
    const T ur = sA[ls], us = sB[ls], ut = sC[ls];
    T G[6], lm;   // lm: the c-term factor lambda m (stored as such; 0 skips the load)
    if constexpr (!RECOMP) {
      const TG* gp = geo_of<TG>(d) + (size_t)e * 7 * p3 + l;
#pragma unroll
      for (int c = 0; c < 6; ++c) G[c] = factor<T>(gp[c * p3]);
      lm = lam_zero ? num_zero<T>() : factor<T>(gp[6 * p3]);
    } else {
      T det, mm;
      geom_point<T>(sx, (T)d.tg[tx], (T)d.tg[ty], (T)d.tg[k], (T)(d.rho[tx] * d.rho[ty] * d.rho[k]), G, mm, det);
      lm = (T)d.lambda * mm;
    }
    sA[ls] = num_dot3(G[0], ur, G[1], us, G[2], ut);
    sB[ls] = num_dot3(G[1], ur, G[3], us, G[4], ut);
    sC[ls] = num_dot3(G[2], ur, G[4], us, G[5], ut);
    rk[k] = lm;
  }
  __syncthreads();
  // divergence by D^T: the A lines (j=tx, k=ty) into su, then the B lines (i=tx, k=ty)
  // added into su, then the C line (i=tx, j=ty) and su added in registers
#pragma unroll
  for (int i = 0; i < p; ++i) line[i] = sA[SL::at(i, tx, ty)];
  fold_apply<p, T>(Fd, line, res);
#pragma unroll
  for (int i = 0; i < p; ++i) su[SL::at(i, tx, ty)] = res[i];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < p; ++j) line[j] = sB[SL::at(tx, j, ty)];
  fold_apply<p, T>(Fd, line, res);
#pragma unroll
  for (int j = 0; j < p; ++j) su[SL::at(tx, j, ty)] = num_add(su[SL::at(tx, j, ty)], res[j]);
  __syncthreads();
#pragma unroll
  for (int k = 0; k < p; ++k) line[k] = sC[SL::at(tx, ty, k)];
  fold_apply<p, T>(Fd, line, res);
  if (!active) return;
  TW* out = wl + (size_t)e * p3;
#pragma unroll
  for (int k = 0; k < p; ++k) {
    const int l = tx + p * (ty + p * k);
    const T v = num_fma(rk[k], uk[k], num_add(su[SL::at(tx, ty, k)], res[k]));   // lambda m u + the divergence terms
    if (DIRECT && inner_xy && k >= 1 && k <= p - 2) {
      const int g = gi0 + m * m * (k - 1);
      yd[g] = (masked >> k) & 1u ? x[g] : num_store<TX>(v);   // y in x's type
    } else {
      out[l] = num_store<TW>(v);
    }
  }
}


// The double-FP32 operator with its six line contractions as two loops (gradient along i, j,
// k into A, B, C; divergence of A, B, C back into the sum), each contraction once in the code
// (the unrolled form of ax_local_kernel stalls on instruction fetch with the pair arithmetic).
// Same operations in the same order as the unrolled form.
//   axis i: line (j = tx, k = ty), nodes (q, tx, ty) of the slab
//   axis j: line (i = tx, k = ty), nodes (tx, q, ty)
//   axis k: line (i = tx, j = ty), nodes (tx, ty, q)
// RECOMP: the factors recomputed at every node from the element's vertices in pair arithmetic
// (geom_line_dw once per thread's line, geom_node_dw per node), the pointwise stage as a
// loop; the c-term lambda m u then starts the sum
// that the three divergence terms are added to: y = ((lambda m u + d_i) + d_j) + d_k.
template <int p, typename TX, int EPB, bool DIRECT, bool RECOMP = false>
__global__ void __launch_bounds__(EPB * p * p) ax_dw_kernel(const DevProblem d, const TX* __restrict__ x,
                                                            double* __restrict__ wl, const PcgState* st,
                                                            TX* __restrict__ yd) {
  using T = dw;
  constexpr int p2 = p * p, p3 = p * p * p;
  st = st_rhs(st);
  x += (size_t)blockIdx.y * d.G;                   // right-hand side blockIdx.y of a block solve
  wl += (size_t)blockIdx.y * d.ne * p3;
  if (DIRECT) yd += (size_t)blockIdx.y * d.G;
  if (stopped(st)) return;
  __shared__ FoldedD<p, T> Fg, Fd;
  using SL = Slab<p>;
  __shared__ T su_all[EPB * SL::N], sA_all[EPB * SL::N], sB_all[EPB * SL::N], sC_all[EPB * SL::N];
  const int grp = threadIdx.x / p2, tid = threadIdx.x % p2;
  const int e_raw = blockIdx.x * EPB + grp;
  const bool active = e_raw < d.ne;            // a short last CTA recomputes its last element
  const int e = active ? e_raw : d.ne - 1;
  T* su = su_all + grp * SL::N;
  T* const sA = sA_all + grp * SL::N;
  T* const sB = sB_all + grp * SL::N;
  T* const sC = sC_all + grp * SL::N;
  const int tx = tid % p, ty = tid / p;
  fold_fill<p, T>(Fg, d.D, false, threadIdx.x);
  fold_fill<p, T>(Fd, d.D, true, threadIdx.x);
  // RECOMP: the element's vertices as pairs, relative to corner 0. The derivatives of the
  // corner basis functions sum to zero, so J is unchanged in exact arithmetic, while the
  // binary64 differences (each within 2^-53 of itself) keep the pair sums at the element's
  // scale: summed from absolute coordinates, J would lose |x| / h of the pairs' 48 bits.
  __shared__ T sx_all[RECOMP ? EPB * 24 : 1];
  T* const sx = sx_all + (RECOMP ? grp * 24 : 0);
  if constexpr (RECOMP)
    for (int q = tid; q < 24; q += p2) {
      const double* xe = d.exyz + (size_t)e * 24;
      sx[q] = dw_split(xe[q] - xe[q % 3]);
    }
  const int* l2ge = d.l2g + (size_t)e * p3;
  constexpr int m = p - 2;
  // axis a's buffer, first node and node stride (selects, not arrays: no local memory)
  auto buf = [&](int a) { return a == 0 ? sA : (a == 1 ? sB : sC); };
  auto base = [&](int a) {
    return a == 0 ? SL::at(0, tx, ty) : (a == 1 ? SL::at(tx, 0, ty) : SL::at(tx, ty, 0));
  };
  auto stride = [&](int a) { return a == 0 ? 1 : (a == 1 ? SL::RS : SL::PS); };
  const bool inner_xy = DIRECT && tx >= 1 && tx <= p - 2 && ty >= 1 && ty <= p - 2;
  const int gi0 = e * m * m * m + (tx - 1) + m * (ty - 1);
  T uk[p], rk[p], line[p], res[p];
  unsigned masked = 0;
#pragma unroll
  for (int k = 0; k < p; ++k) {
    const int l = tx + p * (ty + p * k);
    const bool inner = inner_xy && k >= 1 && k <= p - 2;
    const int g = inner ? gi0 + m * m * (k - 1) : l2ge[l];
    const bool mk = d.mask[g] != 0;
    if (DIRECT && mk) masked |= 1u << k;
    uk[k] = mk ? num_zero<T>() : num_load<T>(x[g]);
    su[SL::at(tx, ty, k)] = uk[k];
  }
  __syncthreads();
#pragma unroll 1
  for (int a = 0; a < 3; ++a) {   // gradient along i, j, k
    const int b0 = base(a), st0 = stride(a);
    T* const dst = buf(a);
#pragma unroll
    for (int q = 0; q < p; ++q) line[q] = su[b0 + st0 * q];
    fold_apply<p, T>(Fg, line, res);
#pragma unroll
    for (int q = 0; q < p; ++q) dst[b0 + st0 * q] = res[q];
  }
  __syncthreads();
  const bool lam_zero = d.lambda == 0.0;
  if constexpr (RECOMP) {
    const dw lam = num_const<dw>(d.lambda);
    LineJ L;
    geom_line_dw(sx, d.phidw + 2 * tx, d.phidw + 2 * ty, L);
#pragma unroll 1
    for (int k = 0; k < p; ++k) {   // pointwise, factors recomputed; su = lambda m u
      const int ls = SL::at(tx, ty, k);
      const T ur = sA[ls], us = sB[ls], ut = sC[ls];
      T G[6], mm;
      geom_node_dw(L, d.phidw + 2 * k, d.w3dw[tx + p * (ty + p * k)], G, mm);
      sA[ls] = num_dot3(G[0], ur, G[1], us, G[2], ut);
      sB[ls] = num_dot3(G[1], ur, G[3], us, G[4], ut);
      sC[ls] = num_dot3(G[2], ur, G[4], us, G[5], ut);
      su[ls] = lam_zero ? num_zero<T>() : dw_mul(dw_mul(lam, mm), su[ls]);
    }
  }
#pragma unroll
  for (int k = 0; k < (RECOMP ? 0 : p); ++k) {   // pointwise: (A, B, C) = G grad u at the nodes (tx, ty, k)
    const int l = tx + p * (ty + p * k);
    const int ls = SL::at(tx, ty, k);
    const T ur = sA[ls], us = sB[ls], ut = sC[ls];
    const T* gp = d.geodw + (size_t)e * 7 * p3 + l;
    T G[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) G[c] = gp[c * p3];
    rk[k] = lam_zero ? num_zero<T>() : gp[6 * p3];
    sA[ls] = num_dot3(G[0], ur, G[1], us, G[2], ut);
    sB[ls] = num_dot3(G[1], ur, G[3], us, G[4], ut);
    sC[ls] = num_dot3(G[2], ur, G[4], us, G[5], ut);
  }
  __syncthreads();
#pragma unroll 1
  for (int a = 0; a < 3; ++a) {   // divergence by D^T along i (into su), j (added), k (output)
    const int b0 = base(a), st0 = stride(a);
    const T* const src = buf(a);
#pragma unroll
    for (int q = 0; q < p; ++q) line[q] = src[b0 + st0 * q];
    fold_apply<p, T>(Fd, line, res);
    if (a == 0) {
#pragma unroll
      for (int q = 0; q < p; ++q) su[b0 + q] = RECOMP ? num_add(su[b0 + q], res[q]) : res[q];
      __syncthreads();
    } else if (a == 1) {
#pragma unroll
      for (int q = 0; q < p; ++q) su[b0 + SL::RS * q] = num_add(su[b0 + SL::RS * q], res[q]);
      __syncthreads();
    }
  }
  if (!active) return;
  double* out = wl + (size_t)e * p3;
#pragma unroll
  for (int k = 0; k < p; ++k) {
    const int l = tx + p * (ty + p * k);
    // lambda m u + the divergence terms (RECOMP: lambda m u already in su)
    const T v = RECOMP ? num_add(su[SL::at(tx, ty, k)], res[k])
                       : num_fma(rk[k], uk[k], num_add(su[SL::at(tx, ty, k)], res[k]));
    if (DIRECT && inner_xy && k >= 1 && k <= p - 2) {
      const int g = gi0 + m * m * (k - 1);
      yd[g] = (masked >> k) & 1u ? x[g] : num_store<TX>(v);
    } else {
      out[l] = num_store<double>(v);
    }
  }
}

template <int p, typename T, int EPB>
constexpr bool ax_tile_supported() {
  return ax_smem_bytes<p, T, EPB>() <= 48 * 1024 && (EPB == 1 || EPB * p * p <= 256);
}

template <int p, typename T>
bool ax_tile_ok_p(int epb) {
  switch (epb) {
    case 1: return ax_tile_supported<p, T, 1>();
    case 2: return ax_tile_supported<p, T, 2>();
    case 4: return ax_tile_supported<p, T, 4>();
    case 8: return ax_tile_supported<p, T, 8>();
    default: return false;
  }
}

template <typename T>
bool ax_tile_ok_t(int p, int epb) {
  switch (p) {
    case 3: return ax_tile_ok_p<3, T>(epb);
    case 4: return ax_tile_ok_p<4, T>(epb);
    case 5: return ax_tile_ok_p<5, T>(epb);
    case 6: return ax_tile_ok_p<6, T>(epb);
    case 7: return ax_tile_ok_p<7, T>(epb);
    case 8: return ax_tile_ok_p<8, T>(epb);
    case 9: return ax_tile_ok_p<9, T>(epb);
    default: return false;
  }
}

template <int p, typename T, typename TX, int EPB, bool DIRECT>
cudaError_t launch_ax_epb(const DevProblem& d, const TX* x, typename LocalOf<T>::type* wl, const PcgState* st,
                          TX* yd, cudaStream_t s) {
  if constexpr (ax_tile_supported<p, T, EPB>()) {
    const int grid = (d.ne + EPB - 1) / EPB;
    constexpr bool kF32 = std::is_same<T, float>::value;
    if constexpr (kIsDw<T>) {   // stored factors as pairs, or the geometry recomputed in pairs
      if (d.recompute)
        ax_dw_kernel<p, TX, EPB, DIRECT, true><<<dim3(grid, d.nrhs), EPB * p * p, 0, s>>>(d, x, wl, st, yd);
      else if (d.geodw == nullptr)
        return cudaErrorInvalidValue;
      else
        ax_dw_kernel<p, TX, EPB, DIRECT, false><<<dim3(grid, d.nrhs), EPB * p * p, 0, s>>>(d, x, wl, st, yd);
    } else if (d.recompute) {
      ax_local_kernel<p, true, T, TX, EPB, DIRECT, T><<<dim3(grid, d.nrhs), EPB * p * p, 0, s>>>(d, x, wl, st, yd);
    } else if (kF32 && d.bf16) {
      if constexpr (kF32)
        ax_local_kernel<p, false, T, TX, EPB, DIRECT, __nv_bfloat16><<<dim3(grid, d.nrhs), EPB * p * p, 0, s>>>(d, x, wl, st, yd);
    } else {
      ax_local_kernel<p, false, T, TX, EPB, DIRECT, T><<<dim3(grid, d.nrhs), EPB * p * p, 0, s>>>(d, x, wl, st, yd);
    }
    count_launch();
    return cudaGetLastError();
  } else {
    return cudaErrorInvalidConfiguration;
  }
}

template <int p, typename T, typename TX, bool DIRECT>
cudaError_t launch_ax_p(const DevProblem& d, const TX* x, typename LocalOf<T>::type* wl, const PcgState* st,
                        TX* yd, cudaStream_t s) {
  switch (std::is_same<T, float>::value ? d.epb_ax32 : (kIsDw<T> ? d.epb_axdw : d.epb_ax)) {
    case 2: return launch_ax_epb<p, T, TX, 2, DIRECT>(d, x, wl, st, yd, s);
    case 4: return launch_ax_epb<p, T, TX, 4, DIRECT>(d, x, wl, st, yd, s);
    case 8: return launch_ax_epb<p, T, TX, 8, DIRECT>(d, x, wl, st, yd, s);
    default: return launch_ax_epb<p, T, TX, 1, DIRECT>(d, x, wl, st, yd, s);
  }
}

// Local results of every node into wl (DIRECT = false), or, for y = A x with the
// interior-first numbering, interior nodes into yd (in x's type) and the others into wl
// (DIRECT = true).
template <typename T, typename TX, bool DIRECT>
cudaError_t launch_ax_local_t(const DevProblem& d, const TX* x, typename LocalOf<T>::type* wl, const PcgState* st,
                              TX* yd, cudaStream_t s) {
  if (DIRECT && d.Gi == 0) return cudaErrorInvalidValue;
  switch (d.p) {
    case 3: return launch_ax_p<3, T, TX, DIRECT>(d, x, wl, st, yd, s);
    case 4: return launch_ax_p<4, T, TX, DIRECT>(d, x, wl, st, yd, s);
    case 5: return launch_ax_p<5, T, TX, DIRECT>(d, x, wl, st, yd, s);
    case 6: return launch_ax_p<6, T, TX, DIRECT>(d, x, wl, st, yd, s);
    case 7: return launch_ax_p<7, T, TX, DIRECT>(d, x, wl, st, yd, s);
    case 8: return launch_ax_p<8, T, TX, DIRECT>(d, x, wl, st, yd, s);
    case 9: return launch_ax_p<9, T, TX, DIRECT>(d, x, wl, st, yd, s);
    default: return cudaErrorInvalidValue;
  }
}


}  // namespace
}  // namespace sem
