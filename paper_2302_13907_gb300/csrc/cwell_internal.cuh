// Internal definitions shared by the cased-well CUDA kernels and host code.
//
// Device layout (one GPU, everything resident in HBM):
//  * each of the nine fields is an array [nth][NR][NZp] of the storage type,
//    z fastest, NZp = NZ rounded up to 32 so every row starts on a 128-byte
//    boundary (float4 / 16-byte vector loads along z); the padding and the
//    wall / axis nodes that are not unknowns (v_r and s_rphi, s_rz at r = 0;
//    v_z, s_rz, s_phiz at the last z half-node) are held at zero;
//  * material IDs uint16 [nth][NR][NZp]; a float4 table {rho, lambda, mu,
//    1/mu} per ID (1/mu = +inf for a liquid, so the four-cell harmonic mean
//    4 / sum(1/mu) is exactly zero next to a liquid);
//  * PML memory variables only where the layers are: a radial slab
//    [12][nth][pml_r][NZp] (six radial differences, six 1/r groups) and a z
//    slab [6][nth][NR][2 pml_z], FP32.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace cwell {

enum { F_VR = 0, F_VP, F_VZ, F_SRR, F_SPP, F_SZZ, F_SRP, F_SPZ, F_SRZ, NF };
// radial-slab memory variables: radial differences (_R) and 1/r groups (_Q)
enum { R_VR = 0, R_VP, R_VZ, R_ERR, R_GRP, R_GRZ, Q_VR, Q_VP, Q_VZ, Q_EPP, Q_GRP, Q_GPZ, NPR };
// z-slab memory variables
enum { Z_VR = 0, Z_VP, Z_VZ, Z_EZZ, Z_GRZ, Z_GPZ, NPZ };

struct KParams {
  int nth, NR, NZ, NZp, nr, pml_r, pml_z;
  long long plane;  // NR * NZp
  float dtv;        // dt * (velocity scale / stress scale)
  float dts;        // dt * (stress scale / velocity scale)
  float inv_dr, inv_dz, inv_dth;
  const float *inv_ri;  // [NR] 1 / (i dr), 0 at i = 0
  const float *inv_rh;  // [NR] 1 / ((i + 1/2) dr)
  const float4 *ab_r;   // [NR] {a, b} at the integer node, {a, b} at the half node: radial difference
  const float4 *ab_q;   // [NR] the same for the 1/r group (integrated profile)
  const float4 *ab_z;   // [NZ] {a, b} at the cell centre, {a, b} at the half node
  const float4 *mat;    // [n_mat] {rho, lambda, mu, 1/mu}
  const float *m_rho;   // [n_mat] rho
  const float *m_imu;   // [n_mat] 1/mu (+inf for a liquid)
  const float2 *m_lam;  // [n_mat] {lambda, lambda + 2 mu}
  const uint16_t *id;   // [nth][NR][NZp]
  void *f[NF];          // field storage (type set by the kernel template)
  float *psr[NPR];      // [nth][pml_r][NZp]
  float *psz[NPZ];      // [nth][NR][2 pml_z]
  const float *wav;     // [n_wav] stress increment of the source at step n (scaled)
  int n_wav;
  int src_i, src_j, src_k;  // src_j < 0: all ring-0 cells
  int *step;                // device step counter
  int i_lo, i_hi;           // rows updated: i_lo <= i < i_hi (the rest are interface ghost rows)
  // z cells the split kernels update: k_lo <= k < k_hi (a z slab's own cells;
  // the rest are its ghost cells, filled by the neighbouring slabs)
  int k_lo = 0, k_hi = 1 << 30;
};

// Point forces and the torsion ring (source kinds 1-3): entry e adds
// w[e] * wav[step] to element off[e] of field fld[e] (stored units, so the
// weights carry dt, A, the node's 1 / (rho V) or 1 / V, the angular share and
// the storage scale); wav[n] = f(t) at the injection time of step n.
struct IParams {
  int n;
  const int *fld;
  const long long *off;
  const float *w;
  const float *wav;
  int n_wav;
  int *step;
  void *f[NF];
};

// Device watchdog (watchdog.cu): energy proxy of the owned cells every
// `every` steps; status bit 3 when it is not finite or exceeds WATCH_GROWTH
// times its first value after step n_quiet.  acc: [0] running sum,
// [1] last proxy, [2] reference, [3] step of the last check.
constexpr double WATCH_GROWTH = 100.0;
struct WParams {
  int nth, NR, NZp, k_lo, k_hi;
  int every, n_quiet;
  const void *f[NF];
  const uint16_t *id;
  const float *m_rho;
  const float2 *m_lam;
  double iv2, is2;  // 1 / (storage scale)^2 of the velocities and the stresses
  int *step, *status;
  double *acc;
};

struct RParams {
  int nth, NR, NZp, n_rec, cap;
  long long plane;
  const void *srr, *spp, *szz;
  const int *rec;        // [n_rec][3] i, j (-1: ring mean), k
  float scale;           // -1 / (3 * stress scale)
  float *traces;         // [n_rec][cap]
  int *step;
  int *status;           // bit 0: non-finite sample
};

// ---------------------------------------------------------------- storage
template <typename T>
struct St;

template <>
struct St<float> {
  static __device__ __forceinline__ float4 ld4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
  static __device__ __forceinline__ float ld1(const float *p) { return __ldg(p); }
  static __device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
};

template <>
struct St<__nv_bfloat16> {
  static __device__ __forceinline__ float4 ld4(const __nv_bfloat16 *p) {
    uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
    float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&u.x));
    float2 b = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
  }
  static __device__ __forceinline__ float ld1(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
  static __device__ __forceinline__ void st4(__nv_bfloat16 *p, float4 v) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
    uint2 u;
    u.x = *reinterpret_cast<unsigned *>(&a);
    u.y = *reinterpret_cast<unsigned *>(&b);
    *reinterpret_cast<uint2 *>(p) = u;
  }
};

template <>
struct St<__half> {
  static __device__ __forceinline__ float4 ld4(const __half *p) {
    uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
    float2 a = __half22float2(*reinterpret_cast<__half2 *>(&u.x));
    float2 b = __half22float2(*reinterpret_cast<__half2 *>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
  }
  static __device__ __forceinline__ float ld1(const __half *p) { return __half2float(__ldg(p)); }
  static __device__ __forceinline__ void st4(__half *p, float4 v) {
    __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
    uint2 u;
    u.x = *reinterpret_cast<unsigned *>(&a);
    u.y = *reinterpret_cast<unsigned *>(&b);
    *reinterpret_cast<uint2 *>(p) = u;
  }
};

// FP16 storage with stochastic rounding (storage mode 3): the same 16-bit
// format as __half, a distinct type so that the stencil kernels store it with
// stochastic rounding (hoist_body.cuh); every other reader and writer treats
// it as __half.
struct half_sr {
  __half h;
};

template <>
struct St<half_sr> {
  static __device__ __forceinline__ float4 ld4(const half_sr *p) { return St<__half>::ld4(reinterpret_cast<const __half *>(p)); }
  static __device__ __forceinline__ float ld1(const half_sr *p) { return St<__half>::ld1(reinterpret_cast<const __half *>(p)); }
};

template <typename T>
__device__ __forceinline__ float st_to_float(T x);
template <>
__device__ __forceinline__ float st_to_float<float>(float x) { return x; }
template <>
__device__ __forceinline__ float st_to_float<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <>
__device__ __forceinline__ float st_to_float<__half>(__half x) { return __half2float(x); }

__device__ __forceinline__ void f4_to(float (&a)[4], float4 v) {
  a[0] = v.x;
  a[1] = v.y;
  a[2] = v.z;
  a[3] = v.w;
}

__device__ __forceinline__ void ld_ids(const uint16_t *p, int (&o)[4]) {
  uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
  o[0] = u.x & 0xffff;
  o[1] = u.x >> 16;
  o[2] = u.y & 0xffff;
  o[3] = u.y >> 16;
}

// velocity coefficient 2 dt / (rho_a + rho_b) (two-cell mean density) and
// four-cell harmonic shear modulus 4 / sum(1/mu), by the fast division
// intrinsic (within 2 ulp; the coefficients need no more).  A liquid among the
// four cells makes the sum +inf and the modulus exactly 0.
__device__ __forceinline__ float vel_coef(float dtv, float rho_sum) { return __fdividef(2.f * dtv, rho_sum); }
__device__ __forceinline__ float mu_harm(float imu_sum) { return __fdividef(4.f, imu_sum); }

// convolutional memory variable: psi <- b psi + a D, returns D + psi
__device__ __forceinline__ float stretch(float *psi, float a, float b, float D) {
  float p = b * (*psi) + a * D;
  *psi = p;
  return D + p;
}

}  // namespace cwell

namespace cwell {
// TMA descriptors of the fused kernel: the nine fields of the buffer being
// read (field order F_*), and the material IDs; 4-D [case][nth][NR][NZp]
// tensors (one case for a single well).
struct FusedMaps {
  CUtensorMap f[NF];
  CUtensorMap id;
};
// Fused kernel parameters: k.f / k.psr / k.psz are the buffers read (step n),
// fo / psr_o / psz_o the buffers written (step n + 1).
struct FusedParams {
  KParams k;
  void *fo[NF];
  float *psr_o[NPR];
  float *psz_o[NPZ];
  int *status;  // bit 1: a bounded wait gave up
};

// launchers implemented in the .cu files (host side)
// parts: 1 = velocity kernel, 2 = stress kernel, 3 = both (velocity first)
cudaError_t launch_split(int storage, const KParams &p, cudaStream_t s, cudaEvent_t *ev, int parts = 3);
cudaError_t launch_receivers(int storage, const RParams &p, cudaStream_t s);
cudaError_t launch_inject(int storage, const IParams &p, cudaStream_t s);
cudaError_t launch_fused(int storage, int rt, const FusedMaps &maps, const FusedParams &fp, cudaStream_t s);
size_t fused_smem_bytes(int storage, int rt);
// upper bound on the work items of one case in either batched work list
long long split_items(int nth, int NR, int NZ);
// batched load-first kernels (interior and edge launches per half step): cases
// is a host array, launched in chunks of BATCH_MAX cases whose parameters
// travel in the kernel's parameter space; grid = persistent blocks per launch
constexpr int BATCH_MAX = 64;
cudaError_t launch_batch_split(int storage, bool vel, const KParams *cases, int n_cases, int grid, cudaStream_t s);
cudaError_t launch_batch_receivers(int storage, const RParams *rp, int n_cases, cudaStream_t s);

// Azimuthally refined grid: ghost rows filled from the neighbouring zone's
// row through a dense [n_out][n_in] interpolation matrix along theta, for
// every z cell: dst[jo * dst_plane + k] = sum_ji mat[jo][ji] src[ji * src_plane + k]
// (FP32 storage only).
constexpr int XFER_MAX = 24;
struct XferDesc {
  const float *src;
  float *dst;
  const float *mat;
  int n_in, n_out;
  long long src_plane, dst_plane;
};
struct XferParams {
  XferDesc d[XFER_MAX];
  int n, NZ;
};
cudaError_t launch_xfer(const XferParams &p, cudaStream_t s);
int fused_box_x(int storage);
cudaError_t launch_fused4(int storage, int rt, const FusedMaps &maps, const FusedParams &fp, cudaStream_t s);
size_t fused4_smem_bytes(int storage, int rt);
// fused path tile code: rt < 100 = scalar fused kernel with rt rows, rt >= 100 =
// vector fused kernel with rt - 100 rows
inline int tile_rows(int code) { return code % 100; }
int fused_pad_x(int storage);
// marching split path: tile code = 1000 + 100 * rows + planes per block
// (rows in {2, 4, 8}, planes 1 .. 99); TMA boxes {march_box_x, rows + 2} for
// the fields and {march_box_id, rows + 2} for the IDs
inline bool is_march(int code) { return code >= 1000 && code < 2000; }
inline int march_rows(int code) { return (code / 100) % 10; }
inline int march_planes(int code) { return code % 100; }
cudaError_t launch_march(int storage, int code, const FusedMaps &maps, const KParams &p, int *status, cudaStream_t s,
                         cudaEvent_t *ev, int parts = 3);
size_t march_smem_bytes(int storage, int code);
// split path: tile code 2000 = the kernels of stencil_split.cu; 2000 + 10 o + b
// = the load-first kernels of stencil_hoist.cu (four z cells per thread) with b
// resident blocks per SM asked of the register allocator (b = 3, 4 or 5) and
// block order o (0: theta fastest, 1: z fastest; b = 3 or 4 only); 2100 + b =
// the two-cells-per-thread variant, theta fastest (b = 6 or 8); 2200 + 10 c + b
// = interior / edge split launches (a lean-only interior kernel for b blocks per
// SM, the general kernel on the PML and end tiles): c = 1: two cells per thread
// in both (b = 6 or 8; edge for 6 blocks per SM); otherwise four cells per
// thread in the interior (b = 4 or 5) and an edge kernel with c = 0: four cells,
// 4 blocks per SM; c = 2: two cells, 4 blocks; c = 3: two cells, 6 blocks;
// c = 4: four cells, 3 blocks; c = 5: two cells in both (interior b = 6 or 8,
// edge for 4 blocks per SM); c = 6 / 7: as c = 2 / 4 with a persistent
// interior kernel that prefetches its next tile into L2; c = 8: plain
// interior, edge (four cells, 3 blocks) walked by a persistent prefetching
// kernel; c = 9: prefetching interior and prefetching edge (two cells, 4
// blocks); 2300 + 10 c + b = three-way split (interior, radial-PML rows with a
// body for interior z, z ends with the general body; persistent prefetching
// kernels for the last two): interior b = 5 plain, 4 prefetching, and c = 0:
// radial (four cells, 4 blocks per SM) + ends (four, 3); 1: (two, 5) + (two,
// 4); 2: (two, 4) + (two, 4); 3: (four, 3) + (four, 3).  A pair code
// v * 10000 + s runs the velocity kernel of split code v and the stress kernel
// of split code s (the autotuner times the two apart).
constexpr int SPLIT_CODE = 2000;
inline bool is_split_single(int code) { return code >= 2000 && code < 3000; }
inline bool is_split_pair(int code) {
  return code >= 10000 && is_split_single(code / 10000) && is_split_single(code % 10000);
}
inline bool is_split_family(int code) { return is_split_single(code) || is_split_pair(code); }
inline int split_vel_code(int code) { return code >= 10000 ? code / 10000 : code; }
inline int split_str_code(int code) { return code >= 10000 ? code % 10000 : code; }
inline bool is_hoist(int code) { return code > 2000 && code < 3000; }
inline int hoist_blocks(int code) { return code % 10; }
inline bool hoist_split(int code) { return (code / 100) % 10 == 2 || (code / 100) % 10 == 3; }
inline bool hoist_zfast(int code) { return !hoist_split(code) && (code / 10) % 10 == 1; }
inline int hoist_cells_per_thread(int code) {
  const int c = (code / 10) % 10;
  return ((code / 100) % 10 == 1 || ((code / 100) % 10 == 2 && (c == 1 || c == 5))) ? 2 : 4;
}
// FP16 stochastic rounding of n device values with the given 13-bit dithers
// (the rule of the FP16-SR stores), FP16 bit patterns out
cudaError_t launch_watchdog(int storage, const WParams &p, int blocks, cudaStream_t s);
cudaError_t launch_sr_round(const float *x, const unsigned *dither, unsigned short *out, long long n, cudaStream_t s);
cudaError_t launch_hoist(int storage, int code, const KParams &p, cudaStream_t s, cudaEvent_t *ev, int parts = 3);
// A second stream for the three-way split halves (23xx): while set on the
// calling thread, each half forks its radial-PML and z-end launches onto
// `side` (event `fork` recorded on the launching stream) and joins them back
// (event `join`) after the interior launch, so that the edge kernels fill
// the SMs the interior kernel leaves idle at its end; null = one stream.
// ghost cells a z slab keeps on each side it shares with another slab
constexpr int SLAB_GHOST = 4;

struct SideStream {
  cudaStream_t side;
  cudaEvent_t fork, join;
};
void set_side_stream(const SideStream *ss);
// single-pass sweep kernel (stencil_sweep.cu): tile code 3000 + 100 m + 10 e
// + b (b resident blocks per SM, general body in runs of e cells; m: z chunks
// of 32 or 64 cells, the lag of the stress items, an L2 prefetch of the next
// velocity item); vdone = sweep_chunks(NZ) ints (zeroed by the launcher
// before the kernel), status bit 1 = a bounded wait gave up; wait_limit in
// cycles (0: 2^31); withhold_chunk >= 0 is the test hook that makes one z
// chunk's velocity items never report
inline bool is_sweep(int code) { return code >= 3000 && code < 3600; }
int sweep_chunks(int NZ);
cudaError_t launch_sweep(int storage, int code, const KParams &p, int *vdone, int *status, long long wait_limit,
                         int withhold_chunk, cudaStream_t s);
// BF16 GEMM on the tcgen05 tensor cores (gemm_tc.cu); status bit 0: a
// bounded wait gave up (read and cleared by gemm_tcgen05_status)
cudaError_t gemm_tcgen05(bool ta, bool tb, int M, int N, int K, const __nv_bfloat16 *A, int lda,
                         const __nv_bfloat16 *B, int ldb, float *C, int ldc, float alpha, float beta,
                         cudaStream_t s);
cudaError_t gemm_tcgen05_status(int *out, cudaStream_t s);
int march_box_x(int storage);
int march_box_id();
}  // namespace cwell
