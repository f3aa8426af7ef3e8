// BF16 GEMM on the fifth-generation tensor cores (tcgen05, accumulator in
// tensor memory) for the trace surrogate.
//
//   C[M x N] = alpha * op(A)[M x K] * op(B)[K x N] + beta * C
//
// A and B are BF16 row-major (op = transpose when TA / TB), C FP32 row-major.
// One CTA of four warps computes a 128 x 128 tile of C:
//  * warp 0 allocates 128 TMEM columns (the FP32 accumulator: TMEM lane m =
//    tile row m, column n = tile column n);
//  * per K chunk of 64 the four warps stage op(A) rows and op(B) columns in
//    shared memory in the no-swizzle K-major core-matrix layout (8 rows x 16
//    bytes per core matrix; core matrices 128 bytes apart along K, 1024 bytes
//    apart along M / N), zero-filling the ragged edges;
//  * one thread issues four tcgen05.mma (K = 16 each) and commits them to an
//    mbarrier; all threads wait (bounded) before the stage is overwritten;
//  * the epilogue reads the accumulator with tcgen05.ld (warp w reads TMEM
//    lanes 32 w .. 32 w + 31, 16 columns per load) and writes C.
// A wait that gives up sets bit 0 of the GEMM status word and skips the
// epilogue; the block then waits (bounded) once more for the MMAs it
// committed, and the TMEM columns are always freed.
#include "cwell_internal.cuh"
#include "tma_util.cuh"

namespace cwell {
namespace {

constexpr int TBM = 128, TBN = 128, TBK = 64;
// dynamic shared memory asked per CTA: caps residency at four CTAs per SM, so
// that four 128-column accumulators fill the SM's 512 TMEM columns exactly
constexpr int TC_SMEM = 56 * 1024;
constexpr int TILE_ELEMS = TBM * TBK;  // 128 x 64 BF16 = 16 KB per operand tile

__device__ int g_tc_status;

// shared-memory matrix descriptor: start address, leading (K-direction) and
// stride (M/N-direction) byte offsets between core matrices, descriptor
// version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = TBN, M = TBM
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TBN >> 3) << 17) |
                           ((uint32_t)(TBM >> 4) << 24);

// the first min(n, 8) BF16 values at src, zero-filled to 8, as one 16-byte word
__device__ __forceinline__ uint4 pack8(const __nv_bfloat16 *src, int n) {
  uint32_t w[4];
#pragma unroll
  for (int e = 0; e < 4; e++) {
    const uint32_t lo = 2 * e < n ? __bfloat16_as_ushort(src[2 * e]) : 0u;
    const uint32_t hi = 2 * e + 1 < n ? __bfloat16_as_ushort(src[2 * e + 1]) : 0u;
    w[e] = lo | (hi << 16);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// element (row, k) of a staged 128 x 64 tile in the core-matrix layout
__device__ __forceinline__ int cm_off(int row, int k) {
  return ((row >> 3) * (TBK / 8) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(128) gemm_tc(int M, int N, int K, const __nv_bfloat16 *__restrict__ A, int lda,
                                               const __nv_bfloat16 *__restrict__ B, int ldb, float *__restrict__ C,
                                               int ldc, float alpha, float beta) {
  extern __shared__ __align__(128) unsigned char smem[];
  __nv_bfloat16 *As = reinterpret_cast<__nv_bfloat16 *>(smem);
  __nv_bfloat16 *Bs = As + TILE_ELEMS;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 4 * TILE_ELEMS);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + 4 * TILE_ELEMS + 8);
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TBN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  const int nk = (K + TBK - 1) / TBK;
  // 16-byte loads along K need 16-byte aligned rows
  const bool vec_a = (lda % 8) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
  const bool vec_b = (ldb % 8) == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0;
  uint32_t phase = 0;
  for (int kc = 0; kc < nk; kc++) {
    const int k0 = kc * TBK;
    // stage op(A)[m0 + r][k0 + k] and op(B)[k0 + k][n0 + n].  Where K is the
    // contiguous dimension of the source, one 16-byte load fills one core-matrix
    // row (8 consecutive k); otherwise element by element, the fastest loop
    // index following the contiguous dimension.
    if (!TA) {
      for (int q = tid; q < TBM * (TBK / 8); q += 128) {
        const int r = q / (TBK / 8), k = (q % (TBK / 8)) * 8;
        const int m = m0 + r, kk = k0 + k;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (m < M) {
          const __nv_bfloat16 *src = A + (long long)m * lda + kk;
          if (vec_a && kk + 8 <= K) {
            v = __ldg(reinterpret_cast<const uint4 *>(src));
          } else {
            v = pack8(src, K - kk);
          }
        }
        *reinterpret_cast<uint4 *>(As + cm_off(r, k)) = v;
      }
    } else {
      for (int q = tid; q < TILE_ELEMS; q += 128) {
        const int r = q % TBM, k = q / TBM;
        const int m = m0 + r, kk = k0 + k;
        As[cm_off(r, k)] = (m < M && kk < K) ? A[(long long)kk * lda + m] : zero;
      }
    }
    if (TB) {
      for (int q = tid; q < TBN * (TBK / 8); q += 128) {
        const int c = q / (TBK / 8), k = (q % (TBK / 8)) * 8;
        const int n = n0 + c, kk = k0 + k;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (n < N) {
          const __nv_bfloat16 *src = B + (long long)n * ldb + kk;
          if (vec_b && kk + 8 <= K) {
            v = __ldg(reinterpret_cast<const uint4 *>(src));
          } else {
            v = pack8(src, K - kk);
          }
        }
        *reinterpret_cast<uint4 *>(Bs + cm_off(c, k)) = v;
      }
    } else {
      for (int q = tid; q < TILE_ELEMS; q += 128) {
        const int c = q % TBN, k = q / TBN;
        const int n = n0 + c, kk = k0 + k;
        Bs[cm_off(c, k)] = (n < N && kk < K) ? B[(long long)kk * ldb + n] : zero;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int ks = 0; ks < TBK / 16; ks++) {
        const uint64_t ad = smem_desc(smem_u32(As) + ks * 256, 128, 1024);
        const uint64_t bd = smem_desc(smem_u32(Bs) + ks * 256, 128, 1024);
        const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(bar))
                   : "memory");
    }
    if (!mbar_wait(bar, phase)) s_fail = 1;  // the MMAs of this stage have read the tiles
    phase ^= 1u;
    __syncthreads();
    if (s_fail) break;
  }
  // after a give-up the MMAs committed last may still be writing the
  // accumulator: wait (bounded) once more for that commit before the columns
  // are freed, so that a later CTA allocating them finds them quiet
  if (s_fail) (void)mbar_wait(bar, phase ^ 1u);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  if (!s_fail) {
    const int m = m0 + 32 * warp + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < TBN; c0 += 16) {
      uint32_t r[16];
      if (nk > 0) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
            "%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
#pragma unroll
        for (int c = 0; c < 16; c++) r[c] = 0u;  // K = 0: the product is zero
      }
      if (m < M) {
#pragma unroll
        for (int c = 0; c < 16; c++) {
          const int n = n0 + c0 + c;
          if (n < N) {
            float *cp = C + (long long)m * ldc + n;
            *cp = alpha * __uint_as_float(r[c]) + (beta != 0.f ? beta * *cp : 0.f);
          }
        }
      }
    }
  } else if (tid == 0) {
    atomicOr(&g_tc_status, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TBN) : "memory");
}

template <bool TA, bool TB>
cudaError_t launch_tc_t(int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb,
                        float *C, int ldc, float alpha, float beta, cudaStream_t s) {
  static bool attr_done[16] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 16) return cudaErrorInvalidDevice;
  if (!attr_done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(gemm_tc<TA, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    attr_done[dev] = true;
  }
  dim3 grd((N + TBN - 1) / TBN, (M + TBM - 1) / TBM);
  gemm_tc<TA, TB><<<grd, 128, TC_SMEM, s>>>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta);
  return cudaGetLastError();
}

}  // namespace

cudaError_t gemm_tcgen05(bool ta, bool tb, int M, int N, int K, const __nv_bfloat16 *A, int lda,
                         const __nv_bfloat16 *B, int ldb, float *C, int ldc, float alpha, float beta,
                         cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (K < 0 || (M + TBM - 1) / TBM > 65535) return cudaErrorInvalidValue;
  if (!ta && !tb) return launch_tc_t<false, false>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, s);
  if (!ta && tb) return launch_tc_t<false, true>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, s);
  if (ta && !tb) return launch_tc_t<true, false>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, s);
  return launch_tc_t<true, true>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, s);
}

// reads and clears the status word of the tcgen05 GEMM (bit 0: a bounded wait gave up)
cudaError_t gemm_tcgen05_status(int *out, cudaStream_t s) {
  cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_tc_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && *out) {
    const int z = 0;
    e = cudaMemcpyToSymbolAsync(g_tc_status, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  return e;
}

}  // namespace cwell
