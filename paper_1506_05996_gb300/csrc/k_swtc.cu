// Patch solves of P^f (Eq. z) in BF16 on the 5th-generation tensor cores (tcgen05), FP32
// accumulation in tensor memory: the preconditioner option SEM_PATCH_BF16 of the FP32 and
// P32 paths.
//
// The six 1D contractions of a patch solve are small dense products: along one axis every
// line of P = n+3 box nodes is multiplied by the P x P pencil eigenvector matrix S (or S^T).
// Lines of several elements are stacked into 128-row tiles, so one stage of a CTA's
// elements is a few MMAs D[128 x 16] = A[128 x 16] B[16 x 16] with A = the lines (nodes in
// the K dimension, zero padded to 16), B = S or S^T (zero padded) and D in TMEM. Between
// stages each thread reads its TMEM rows (tcgen05.ld), rounds them to BF16 and writes them
// into the next stage's A tile with the axes permuted, so that the next contraction runs
// along the next axis:
//   stage 1  rows (J,K), k = I  ->  modes a       (forward, B = S)
//   stage 2  rows (a,K), k = J  ->  modes b
//   stage 3  rows (a,b), k = K  ->  modes c, times the inverted diagonal d[a,b,c] (with the
//                                   patch scale 8/(hx hy hz)), in FP32 before rounding
//   stage 4  rows (a,b), k = c  ->  nodes K       (backward, B = S^T)
//   stage 5  rows (a,K), k = b  ->  nodes J
//   stage 6  rows (J,K), k = a  ->  nodes I, stored in FP32 for the P-sum.
// Operand tiles are K-major without swizzle: core matrices of 8 rows x 16 bytes, the two
// 8-wide k halves 128 bytes apart (leading byte offset), 8-row groups 256 bytes apart
// (stride byte offset). One thread issues the MMAs and commits them to an mbarrier; every
// wait on it is bounded, after which the kernel records an error, waits (bounded) once more
// and frees its tensor memory before returning.
//
// Rounding: the box values, S and every stage's input are rounded to BF16 (relative
// 2^-9 each), products are exact and accumulate in FP32, so a result errs by about
// 7 * 2^-9 of the all-absolute contraction |S||S^T|(|r|) (six roundings of the inputs and
// S, plus the diagonal's rounding), tested against that bound.
// Elements whose sides take natural-boundary pencils need a different S per axis and per
// element, so handles with such sides keep the FP32 patch kernel.
#include <cuda_bf16.h>
#include <cstdint>

#include "kcommon.cuh"

namespace sem {
namespace {

constexpr int kTcThreads = 256;          // 8 warps: two per TMEM lane quarter (even and odd tiles)
constexpr int kTcRows = 128;             // M of one MMA: 128 box lines
constexpr int kTcTileBytes = kTcRows * 16 * 2;   // 128 rows x 16 BF16
constexpr uint32_t kTcSpin = 1u << 22;   // bound of every wait on the MMA barrier

// Byte offset of (row, k) in a K-major, non-swizzled 16-column BF16 operand tile.
__device__ __forceinline__ int tc_off(int row, int k) {
  return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Shared-memory matrix descriptor of such a tile (start address, leading byte offset 128,
// stride byte offset 256, descriptor version 1, no swizzle).
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(256u >> 4) << 32) |
         ((uint64_t)1u << 46);
}

// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, N = 16, M = 128.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// D = A B (enable_input_d false: the tile's K = 16 is one instruction)
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(kTcIdesc), "r"(0));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

// Bounded wait for the given phase parity of the MMA barrier; false when the bound ran out.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
  for (uint32_t it = 0; it < kTcSpin; ++it) {
    uint32_t done = 0;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <int NCOL>
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "n"(NCOL)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
template <int NCOL>
__device__ __forceinline__ void tmem_free(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(NCOL) : "memory");
}

template <typename TR> __device__ __forceinline__ float to_f(TR v) { return (float)v; }

template <int P, int EPC>
struct TcShape {
  static constexpr int LINES = EPC * P * P;                       // box lines of the CTA's elements
  static constexpr int NT = (LINES + kTcRows - 1) / kTcRows;      // 128-row tiles per stage
  static constexpr int NCOL = NT * 16 <= 32 ? 32 : NT * 16 <= 64 ? 64 : NT * 16 <= 128 ? 128 : NT * 16 <= 256 ? 256 : 512;
  // A tiles, S and S^T tiles, barrier; at least 48 KB, so that no more than 4 CTAs share an
  // SM (their tensor memory, up to 128 columns each, then always fits)
  static constexpr int SMEM_USED = NT * kTcTileBytes + 2 * 512 + 64;
  static constexpr int SMEM = SMEM_USED > 49152 ? SMEM_USED : 49152;
};

// One CTA of 256 threads per group of EPC elements (groups strided over the grid). wp
// receives FP32 patch results in the layout of the FP32 patch kernel.
template <int P, typename TR, int EPC>
__global__ void __launch_bounds__(kTcThreads) schwarz_tc_kernel(const DevProblem d, const TR* __restrict__ r,
                                                                float* __restrict__ wp, const PcgState* st) {
  using Sh = TcShape<P, EPC>;
  constexpr int P2 = P * P, P3 = P * P * P, NT = Sh::NT, LINES = Sh::LINES;
  static_assert(Sh::NCOL <= 128 && NT * 16 <= Sh::NCOL, "tensor memory columns (4 CTAs per SM)");
  static_assert(P <= 16, "a line fits the 16-wide K of one MMA");
  if (stopped(st)) return;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* A = smem;                                   // NT tiles
  uint8_t* Bf = smem + NT * kTcTileBytes;              // (n = mode c, k = node):   S[k][c]
  uint8_t* Bb = Bf + 512;                              // (n = node k, k = mode c): S[k][c]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Bb + 512);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(Bb + 512 + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // zero the operand tiles (the padding k >= P and rows >= LINES stay zero), fill S, S^T
  for (int q = tid; q < (NT * kTcTileBytes + 1024) / 16; q += kTcThreads)
    reinterpret_cast<uint4*>(smem)[q] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  for (int q = tid; q < P2; q += kTcThreads) {
    const int k = q / P, c = q % P;                    // S[k][c] = d.S[k * P + c]
    const __nv_bfloat16 s = __float2bfloat16_rn((float)d.S[q]);
    *reinterpret_cast<__nv_bfloat16*>(Bf + tc_off(c, k)) = s;
    *reinterpret_cast<__nv_bfloat16*>(Bb + tc_off(k, c)) = s;
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc<Sh::NCOL>(smem_u32(tmem_slot));
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t a_base = smem_u32(A), mbar_a = smem_u32(mbar);
  const uint64_t bf_desc = tc_desc(smem_u32(Bf)), bb_desc = tc_desc(smem_u32(Bb));
  uint32_t phase = 0;
  bool ok = true;

  auto put = [&](int line, int k, float v) {
    *reinterpret_cast<__nv_bfloat16*>(A + (line / kTcRows) * kTcTileBytes + tc_off(line % kTcRows, k)) =
        __float2bfloat16_rn(v);
  };
  // the stage's MMAs (all tiles) by one thread, then every thread waits for them
  auto run_stage = [&](uint64_t bdesc) {
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      for (int t = 0; t < NT; ++t) tc_mma(tmem + 16u * t, tc_desc(a_base + t * kTcTileBytes), bdesc);
      tc_commit(mbar_a);
    }
    const bool waited = tc_wait(mbar_a, phase);
    ok = __syncthreads_and(ok && waited) != 0;   // uniform, so the warps stay converged
    phase ^= 1u;
    tc_fence_after();
  };

  const int ngroups = (d.ne + EPC - 1) / EPC;
  for (int blk = blockIdx.x; blk < ngroups && ok; blk += gridDim.x) {
    const int e0 = blk * EPC;
    // stage 1 input: row (J, K) of element el, k = I; four entries per thread in flight
    // (patch-table loads, then the residual and mask loads, then the stores)
    constexpr int NQ = EPC * P3, U = 4;
    for (int q0 = tid; q0 < NQ; q0 += kTcThreads * U) {
      int gi[U];
      float v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = q0 + u * kTcThreads, e = e0 + q / P3;
        gi[u] = (q < NQ && e < d.ne) ? d.ip[(size_t)e * P3 + q % P3] : -1;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        v[u] = 0.f;
        if (gi[u] >= 0) {
          const float rv = to_f(r[gi[u]]);
          const bool mk = d.mask[gi[u]] != 0;
          v[u] = mk ? 0.f : (d.pw32 != nullptr ? rv * d.pw32[gi[u]] : rv);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = q0 + u * kTcThreads;
        if (q < NQ) {
          const int el = q / P3, node = q % P3;
          put(el * P2 + node / P, node % P, v[u]);
        }
      }
    }
#pragma unroll 1
    for (int s = 0; s < 6; ++s) {
      run_stage(s < 3 ? bf_desc : bb_desc);
      if (!ok) break;
      // warp w reads TMEM lanes 32 (w % 4) + lane of the tiles t = w / 4, w / 4 + 2, ...:
      // line = 128 t + 32 (w % 4) + lane
      const int quarter = warp & 3;
      for (int t = warp >> 2; t < NT; t += 2) {
        float y[16];
        tc_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + 16u * t, y);
        const int line = t * kTcRows + 32 * quarter + lane;
        if (line >= LINES) continue;
        const int el = line / P2, lr = line % P2, al = lr % P, be = lr / P;   // row (alpha, beta)
        const int e = e0 + el;
        if (s == 5) {                       // rows (J, K), columns I: the patch result
          if (e < d.ne) {
            float* out = wp + (size_t)e * P3 + P * lr;
#pragma unroll
            for (int c = 0; c < P; ++c) out[c] = y[c];
          }
        } else if (s == 0 || s == 4) {      // (alpha, beta, gamma) -> row (gamma, beta), k = alpha
#pragma unroll
          for (int c = 0; c < P; ++c) put(el * P2 + c + P * be, al, y[c]);
        } else if (s == 1 || s == 3) {      // (alpha, beta, gamma) -> row (alpha, gamma), k = beta
#pragma unroll
          for (int c = 0; c < P; ++c) put(el * P2 + al + P * c, be, y[c]);
        } else {                            // s == 2: rows (a, b), modes c, times d[a, b, c]
          const float* dg = d.swd32 + (size_t)(e < d.ne ? e : d.ne - 1) * P3;
#pragma unroll
          for (int c = 0; c < P; ++c) put(line, c, y[c] * dg[(be + P * c) + P2 * al]);
        }
      }
      tc_fence_before();
    }
    __syncthreads();
  }
  if (!ok) {
    // a wait ran out: report it, give the MMAs in flight one more bounded wait, then free
    if (tid == 0 && st != nullptr) {
      PcgState* sw = const_cast<PcgState*>(st);
      sw->status = -4;
      sw->done = 1;
    }
    if (tid == 0 && d.wait_err != nullptr) atomicExch(d.wait_err, 1);
    tc_wait(mbar_a, phase);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_free<Sh::NCOL>(tmem);
  }
}

template <int P, typename TR>
cudaError_t launch_tc_P(const DevProblem& d, const TR* r, float* wp, const PcgState* st, cudaStream_t s) {
  constexpr int EPC = 8;
  using Sh = TcShape<P, EPC>;
  auto kernel = schwarz_tc_kernel<P, TR, EPC>;
  // the dynamic shared memory is above the default 48 KB limit
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM);
  if (e != cudaSuccess) return e;
  int grid = (d.ne + EPC - 1) / EPC;
  if (d.sw_reserve_sms > 0) {
    // 4 CTAs per SM (shared memory and tensor memory both hold 4) on all but the reserved SMs
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int cap = (nsm - d.sw_reserve_sms) * 4;
    if (cap > 0 && cap < grid) grid = cap;
  }
  kernel<<<grid, kTcThreads, Sh::SMEM, s>>>(d, r, wp, st);
  count_launch();
  return cudaGetLastError();
}

template <typename TR>
cudaError_t launch_tc_t(const DevProblem& d, const TR* r, float* wp, const PcgState* st, cudaStream_t s) {
  if (d.ne == 0) return cudaSuccess;
  switch (d.P) {
    case 5: return launch_tc_P<5, TR>(d, r, wp, st, s);
    case 6: return launch_tc_P<6, TR>(d, r, wp, st, s);
    case 7: return launch_tc_P<7, TR>(d, r, wp, st, s);
    case 8: return launch_tc_P<8, TR>(d, r, wp, st, s);
    case 9: return launch_tc_P<9, TR>(d, r, wp, st, s);
    case 10: return launch_tc_P<10, TR>(d, r, wp, st, s);
    case 11: return launch_tc_P<11, TR>(d, r, wp, st, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_schwarz_tc(const DevProblem& d, const double* r, float* wp, const PcgState* st, cudaStream_t s) {
  return launch_tc_t<double>(d, r, wp, st, s);
}
cudaError_t launch_schwarz_tc_in32(const DevProblem& d, const float* r, float* wp, const PcgState* st,
                                   cudaStream_t s) {
  return launch_tc_t<float>(d, r, wp, st, s);
}

}  // namespace sem
