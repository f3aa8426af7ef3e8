// TMA / mbarrier helpers and shared-memory accessors of the fused kernels.
#pragma once

#include <cuda.h>

#include "cwell_internal.cuh"

namespace cwell {

template <typename T>
struct Pad {
  static constexpr int HX = 16 / (int)sizeof(T);  // left z pad: keeps the TMA x coordinate 16-byte aligned
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// bounded parity wait: true when the phase completed, false after ~1 s
// (2^31 SM cycles) without completion
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  for (unsigned it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 31u) == 31u && (clock64() - t0 > (1LL << 31) || it > (1u << 26))) return false;
  }
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int x, int y, int z, int w,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ float sld(const float *p) { return *p; }
__device__ __forceinline__ float sld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ float sld(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ void gst(float *p, float v) { *p = v; }
__device__ __forceinline__ void gst(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void gst(__half *p, float v) { *p = __float2half_rn(v); }

}  // namespace cwell
