// Cell bodies of the load-first split kernels (one thread, NV consecutive z
// cells of one (theta, r) row): the velocity half-step (Eq. 1a) and the
// stress half-step (Eq. 1b) of the staggered cylindrical scheme, with every
// global load of the thread issued before its arithmetic and stores, the
// material lookups from the split tables {rho}, {1/mu}, {lambda, lambda + 2 mu},
// the PML memory variables fused in (reading R8), the volumetric source
// fused into the stress update (R6).  Shared by the split kernels
// (stencil_hoist.cu) and the single-pass sweep kernel (stencil_sweep.cu).
#pragma once

#include <type_traits>

#include "cwell_internal.cuh"

namespace cwell {
namespace {

__device__ __forceinline__ float4 z4() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// NV consecutive values of a row: 16-byte (four FP32) or 8-byte (two FP32,
// four 16-bit) vector loads and stores, converted to / from FP32
template <typename T, int NV>
struct Vec;
template <typename T>
struct Vec<T, 4> {
  static __device__ __forceinline__ void ld(float (&d)[4], const T *p) {
    const float4 v = St<T>::ld4(p);
    d[0] = v.x;
    d[1] = v.y;
    d[2] = v.z;
    d[3] = v.w;
  }
  static __device__ __forceinline__ void st(T *p, const float (&v)[4]) { St<T>::st4(p, make_float4(v[0], v[1], v[2], v[3])); }
};
template <>
struct Vec<float, 2> {
  static __device__ __forceinline__ void ld(float (&d)[2], const float *p) {
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    d[0] = v.x;
    d[1] = v.y;
  }
  static __device__ __forceinline__ void st(float *p, const float (&v)[2]) {
    *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
  }
};
template <>
struct Vec<__nv_bfloat16, 2> {
  static __device__ __forceinline__ void ld(float (&d)[2], const __nv_bfloat16 *p) {
    const unsigned u = __ldg(reinterpret_cast<const unsigned *>(p));
    const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u));
    d[0] = v.x;
    d[1] = v.y;
  }
  static __device__ __forceinline__ void st(__nv_bfloat16 *p, const float (&v)[2]) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
    *reinterpret_cast<unsigned *>(p) = *reinterpret_cast<const unsigned *>(&a);
  }
};
template <>
struct Vec<__half, 2> {
  static __device__ __forceinline__ void ld(float (&d)[2], const __half *p) {
    const unsigned u = __ldg(reinterpret_cast<const unsigned *>(p));
    const float2 v = __half22float2(*reinterpret_cast<const __half2 *>(&u));
    d[0] = v.x;
    d[1] = v.y;
  }
  static __device__ __forceinline__ void st(__half *p, const float (&v)[2]) {
    const __half2 a = __floats2half2_rn(v[0], v[1]);
    *reinterpret_cast<unsigned *>(p) = *reinterpret_cast<const unsigned *>(&a);
  }
};

// The same loads through L2 only (ld.global.cg, bypassing L1 and the
// read-only path), for values another block of the same launch may have
// written: the velocities the single-pass sweep kernel's stress items read.
template <typename T, int NV>
struct VecCG;
template <>
struct VecCG<float, 4> {
  static __device__ __forceinline__ void ld(float (&d)[4], const float *p) {
    const float4 v = __ldcg(reinterpret_cast<const float4 *>(p));
    d[0] = v.x;
    d[1] = v.y;
    d[2] = v.z;
    d[3] = v.w;
  }
};
template <>
struct VecCG<float, 2> {
  static __device__ __forceinline__ void ld(float (&d)[2], const float *p) {
    const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    d[0] = v.x;
    d[1] = v.y;
  }
};
__device__ __forceinline__ float2 u32_to_f2(unsigned u, const __nv_bfloat16 *) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u));
}
__device__ __forceinline__ float2 u32_to_f2(unsigned u, const __half *) {
  return __half22float2(*reinterpret_cast<const __half2 *>(&u));
}
__device__ __forceinline__ float2 u32_to_f2(unsigned u, const half_sr *) {
  return __half22float2(*reinterpret_cast<const __half2 *>(&u));
}
template <typename T>
struct VecCG<T, 4> {
  static __device__ __forceinline__ void ld(float (&d)[4], const T *p) {
    const uint2 u = __ldcg(reinterpret_cast<const uint2 *>(p));
    const float2 a = u32_to_f2(u.x, p), b = u32_to_f2(u.y, p);
    d[0] = a.x;
    d[1] = a.y;
    d[2] = b.x;
    d[3] = b.y;
  }
};
template <typename T>
struct VecCG<T, 2> {
  static __device__ __forceinline__ void ld(float (&d)[2], const T *p) {
    const float2 a = u32_to_f2(__ldcg(reinterpret_cast<const unsigned *>(p)), p);
    d[0] = a.x;
    d[1] = a.y;
  }
};
__device__ __forceinline__ float ld1cg(const float *p) { return __ldcg(p); }
__device__ __forceinline__ float ld1cg(const __nv_bfloat16 *p) {
  return __bfloat162float(__ushort_as_bfloat16(__ldcg(reinterpret_cast<const unsigned short *>(p))));
}
__device__ __forceinline__ float ld1cg(const __half *p) {
  return __half2float(__ushort_as_half(__ldcg(reinterpret_cast<const unsigned short *>(p))));
}
__device__ __forceinline__ float ld1cg(const half_sr *p) { return ld1cg(reinterpret_cast<const __half *>(p)); }
// Streaming loads and stores (ld/st.global.cs: lines allocated evict-first,
// so a last use does not push out lines that other items still need): the
// sweep kernel's stress items read their own stresses for the last time and
// write the new ones, which nothing reads again in the launch.
template <typename T, int NV>
struct VecCS;
template <>
struct VecCS<float, 4> {
  static __device__ __forceinline__ void ld(float (&d)[4], const float *p) {
    const float4 v = __ldcs(reinterpret_cast<const float4 *>(p));
    d[0] = v.x;
    d[1] = v.y;
    d[2] = v.z;
    d[3] = v.w;
  }
  static __device__ __forceinline__ void st(float *p, const float (&v)[4]) {
    __stcs(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
  }
};
template <>
struct VecCS<float, 2> {
  static __device__ __forceinline__ void ld(float (&d)[2], const float *p) {
    const float2 v = __ldcs(reinterpret_cast<const float2 *>(p));
    d[0] = v.x;
    d[1] = v.y;
  }
  static __device__ __forceinline__ void st(float *p, const float (&v)[2]) {
    __stcs(reinterpret_cast<float2 *>(p), make_float2(v[0], v[1]));
  }
};
__device__ __forceinline__ unsigned f2_to_u32(float a, float b, const __nv_bfloat16 *) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const unsigned *>(&h);
}
__device__ __forceinline__ unsigned f2_to_u32(float a, float b, const __half *) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const unsigned *>(&h);
}
template <typename T>
struct VecCS<T, 4> {
  static __device__ __forceinline__ void ld(float (&d)[4], const T *p) {
    const uint2 u = __ldcs(reinterpret_cast<const uint2 *>(p));
    const float2 a = u32_to_f2(u.x, p), b = u32_to_f2(u.y, p);
    d[0] = a.x;
    d[1] = a.y;
    d[2] = b.x;
    d[3] = b.y;
  }
  static __device__ __forceinline__ void st(T *p, const float (&v)[4]) {
    __stcs(reinterpret_cast<uint2 *>(p), make_uint2(f2_to_u32(v[0], v[1], p), f2_to_u32(v[2], v[3], p)));
  }
};
template <typename T>
struct VecCS<T, 2> {
  static __device__ __forceinline__ void ld(float (&d)[2], const T *p) {
    const float2 a = u32_to_f2(__ldcs(reinterpret_cast<const unsigned *>(p)), p);
    d[0] = a.x;
    d[1] = a.y;
  }
  static __device__ __forceinline__ void st(T *p, const float (&v)[2]) {
    __stcs(reinterpret_cast<unsigned *>(p), f2_to_u32(v[0], v[1], p));
  }
};
// CS selects the streaming loads and stores
template <typename T, int NV, bool CS>
__device__ __forceinline__ void ldown(float (&d)[NV], const T *p) {
  if (CS) VecCS<T, NV>::ld(d, p);
  else Vec<T, NV>::ld(d, p);
}
template <typename T, int NV, bool CS>
__device__ __forceinline__ void stown(T *p, const float (&v)[NV]) {
  if (CS) VecCS<T, NV>::st(p, v);
  else Vec<T, NV>::st(p, v);
}

// Stochastic rounding of the FP16 storage (mode 3).  The dither of field f
// of cell (j, i, k) in the update of step n is the 13-bit group
// (z >> 16 (k mod 4)) & 0x1fff of z = SplitMix64 mix of
// (key + 1) 0x9E3779B97F4A7C15, key = (((n * 9 + f) * nth + j) * NR + i) *
// ceil(NZ / 4) + floor(k / 4): one 64-bit hash per four cells.  A value x
// (the FP32 result) of magnitude a rounds away from zero when
// frac(a / u) * 8192 > dither, u the FP16 spacing at a (2^(E - 10), E the
// exponent of a, at least -14), so that E[rounded] = x; every step of this
// is exact in FP32.  Magnitudes beyond 65504 round to nearest.
// the key expanded: (n NF + f) S + (j NR + i) ngrp + floor(k0 / 4), S = nth NR
// ngrp (equal modulo 2^64); everything but f S is common to the nine fields
// of a cell, so a body takes it once, before its stores
struct SrKey {
  unsigned long long base, S;
  int k0;
};
__device__ __forceinline__ SrKey sr_key(const KParams &p, int n, int j, int i, int k0) {
  const unsigned long long ngrp = (unsigned long long)((p.NZ + 3) >> 2);
  const unsigned long long S = (unsigned long long)p.nth * (unsigned long long)p.NR * ngrp;
  return {(unsigned long long)n * NF * S + ((unsigned long long)j * p.NR + i) * ngrp + (unsigned long long)(k0 >> 2), S,
          k0};
}
__device__ __forceinline__ unsigned long long sr_hash(const SrKey &sk, int f) {
  unsigned long long z = (sk.base + (unsigned long long)f * sk.S + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }  // -126 <= k <= 127

__device__ __forceinline__ __half sr_round(float x, unsigned dither) {
  const float a = fabsf(x);
  // zero (whole warps of it ahead of the wavefront), beyond the format, not finite
  if (!(a <= 65504.f) || a == 0.f) return __float2half_rn(x);
  const int ex = (int)((__float_as_uint(a) >> 23) & 0xff) - 127;
  const int E = ex < -14 ? -14 : ex;
  const float q = a * pow2f(10 - E);  // a / u, exact
  const float fl = floorf(q);
  const float up = ((q - fl) * 8192.f > (float)dither) ? 1.f : 0.f;
  return __float2half_rn(copysignf((fl + up) * pow2f(E - 10), x));  // exact, a value of the format
}

// the NV values of field f at cells (j, i, k0 .. k0 + NV - 1) of step n (sk)
template <int NV>
__device__ __forceinline__ void sr_store(half_sr *p, const float (&v)[NV], const SrKey &sk, int f) {
  const unsigned long long z = sr_hash(sk, f);
  __half h[NV];
#pragma unroll
  for (int e = 0; e < NV; e++) h[e] = sr_round(v[e], (unsigned)(z >> (16 * ((sk.k0 + e) & 3))) & 0x1fffu);
  if (NV == 4) {
    uint2 u;
    u.x = (unsigned)__half_as_ushort(h[0]) | ((unsigned)__half_as_ushort(h[1 % NV]) << 16);
    u.y = (unsigned)__half_as_ushort(h[2 % NV]) | ((unsigned)__half_as_ushort(h[3 % NV]) << 16);
    *reinterpret_cast<uint2 *>(p) = u;
  } else {
    *reinterpret_cast<unsigned *>(p) =
        (unsigned)__half_as_ushort(h[0]) | ((unsigned)__half_as_ushort(h[1 % NV]) << 16);
  }
}

// the key of a body's stores: the step and the cell group (stochastic rounding only)
template <typename T>
__device__ __forceinline__ SrKey body_key(const KParams &p, int j, int i, int k0) {
  if constexpr (std::is_same<T, half_sr>::value) return sr_key(p, *p.step, j, i, k0);
  else return SrKey{0ull, 0ull, 0};
}

// store of a field's NV new values: stochastic rounding for half_sr, else
// the plain (CS = false) or streaming (CS = true) store
template <typename T, int NV, bool CS>
__device__ __forceinline__ void st_field(T *ptr, const float (&v)[NV], const SrKey &sk, int f) {
  if constexpr (std::is_same<T, half_sr>::value) sr_store<NV>(ptr, v, sk, f);
  else stown<T, NV, CS>(ptr, v);
}

// CG selects the L2-only loads
template <typename T, int NV, bool CG>
__device__ __forceinline__ void ldrow(float (&d)[NV], const T *p) {
  if (CG) VecCG<T, NV>::ld(d, p);
  else Vec<T, NV>::ld(d, p);
}
template <typename T, bool CG>
__device__ __forceinline__ float ldone(const T *p) {
  if (CG) return ld1cg(p);
  return St<T>::ld1(p);
}

template <>
struct Vec<half_sr, 2> {
  static __device__ __forceinline__ void ld(float (&d)[2], const half_sr *p) {
    Vec<__half, 2>::ld(d, reinterpret_cast<const __half *>(p));
  }
};

// PML memory variables: plain (not read-only path) vector loads and stores,
// since the thread that reads a memory variable rewrites it
template <int NV>
__device__ __forceinline__ void ldv(float (&d)[NV], const float *p);
template <>
__device__ __forceinline__ void ldv<4>(float (&d)[4], const float *p) {
  const float4 v = *reinterpret_cast<const float4 *>(p);
  d[0] = v.x;
  d[1] = v.y;
  d[2] = v.z;
  d[3] = v.w;
}
template <>
__device__ __forceinline__ void ldv<2>(float (&d)[2], const float *p) {
  const float2 v = *reinterpret_cast<const float2 *>(p);
  d[0] = v.x;
  d[1] = v.y;
}
template <int NV>
__device__ __forceinline__ void stv(float *p, const float (&v)[NV]);
template <>
__device__ __forceinline__ void stv<4>(float *p, const float (&v)[4]) {
  *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void stv<2>(float *p, const float (&v)[2]) {
  *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
}

// the memory-variable recursion of the stretched derivative on a register
// copy: psi <- b psi + a D, result D + psi (same arithmetic as stretch())
__device__ __forceinline__ float stretch_reg(float &psi, float a, float b, float D) {
  psi = b * psi + a * D;
  return D + psi;
}

template <int NV>
__device__ __forceinline__ void zero(float (&d)[NV]) {
#pragma unroll
  for (int e = 0; e < NV; e++) d[e] = 0.f;
}

// NV consecutive material IDs (8- or 4-byte load)
__device__ __forceinline__ void ldids(const uint16_t *p, int (&o)[4]) {
  const uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
  o[0] = u.x & 0xffff;
  o[1] = u.x >> 16;
  o[2] = u.y & 0xffff;
  o[3] = u.y >> 16;
}
__device__ __forceinline__ void ldids(const uint16_t *p, int (&o)[2]) {
  const unsigned u = __ldg(reinterpret_cast<const unsigned *>(p));
  o[0] = u & 0xffff;
  o[1] = u >> 16;
}
template <int NV>
__device__ __forceinline__ void zero_ids(int (&o)[NV]) {
#pragma unroll
  for (int e = 0; e < NV; e++) o[e] = 0;
}

// NV cells per thread (4 or 2).  ZIN: the NV cells and their +1 z neighbours
// lie inside NZ and outside the z PML (no z memory variable, no z bound
// check); by default the same as LEAN.  LEAN: the NV cells are interior (no PML
// memory variable, all inside NZ, k0 + NV < NZ); the kernels pick the lean
// body per thread, or run it alone on the interior tiles.
template <typename T, int NV, bool LEAN, bool PRE = false, bool ZIN = LEAN>
__device__ __forceinline__ void vel_hoist_body(const KParams &p, const int j, const int i, const int k0) {
  const int nth = p.nth, NR = p.NR, NZ = p.NZ;
  const long long NZp = p.NZp, pl = p.plane;
  const int jm = j == 0 ? nth - 1 : j - 1, jp = j == nth - 1 ? 0 : j + 1;
  const long long c = (long long)j * pl + i * NZp + k0;
  const long long cjm = (long long)jm * pl + i * NZp + k0;
  const long long cjp = (long long)jp * pl + i * NZp + k0;
  const T *srr = (const T *)p.f[F_SRR], *spp = (const T *)p.f[F_SPP], *szz = (const T *)p.f[F_SZZ];
  const T *srp = (const T *)p.f[F_SRP], *spz = (const T *)p.f[F_SPZ], *srz = (const T *)p.f[F_SRZ];
  T *vr = (T *)p.f[F_VR], *vp = (T *)p.f[F_VP], *vz = (T *)p.f[F_VZ];
  const bool im = i >= 1, ip = i + 1 < NR, k4 = ZIN || k0 + NV < NZ, km = k0 > 0;

  // ---- every load
  float a_srr[NV];
  Vec<T, NV>::ld(a_srr, srr + c);
  float a_spp[NV];
  Vec<T, NV>::ld(a_spp, spp + c);
  float a_srp[NV];
  Vec<T, NV>::ld(a_srp, srp + c);
  float a_srz[NV];
  Vec<T, NV>::ld(a_srz, srz + c);
  float a_spz[NV];
  Vec<T, NV>::ld(a_spz, spz + c);
  float a_szz[NV];
  Vec<T, NV>::ld(a_szz, szz + c);
  const float szz_k4 = k4 ? St<T>::ld1(szz + c + NV) : 0.f;
  const float srz_km = km ? St<T>::ld1(srz + c - 1) : 0.f, spz_km = km ? St<T>::ld1(spz + c - 1) : 0.f;
  float m_srr[NV];
  if (im) Vec<T, NV>::ld(m_srr, srr + c - NZp);
  else zero(m_srr);
  float m_spp[NV];
  if (im) Vec<T, NV>::ld(m_spp, spp + c - NZp);
  else zero(m_spp);
  float jm_srp[NV];
  Vec<T, NV>::ld(jm_srp, srp + cjm);
  float jm_spz[NV];
  Vec<T, NV>::ld(jm_spz, spz + cjm);
  float p_srp[NV];
  if (ip) Vec<T, NV>::ld(p_srp, srp + c + NZp);
  else zero(p_srp);
  float p_srz[NV];
  if (ip) Vec<T, NV>::ld(p_srz, srz + c + NZp);
  else zero(p_srz);
  float jp_spp[NV];
  Vec<T, NV>::ld(jp_spp, spp + cjp);
  float o_vr[NV];
  Vec<T, NV>::ld(o_vr, vr + c);
  float o_vp[NV];
  Vec<T, NV>::ld(o_vp, vp + c);
  float o_vz[NV];
  Vec<T, NV>::ld(o_vz, vz + c);
  int idc[NV], idj[NV], idm[NV];
  ldids(p.id + c, idc);
  ldids(p.id + cjp, idj);
  if (im) ldids(p.id + c - NZp, idm);
  else zero_ids(idm);
  int id_k4 = 0;
  if (k4) id_k4 = __ldg(p.id + c + NV);
  const bool rp = !LEAN && i >= p.nr;
  const float inv_ri = __ldg(p.inv_ri + i), inv_rh = __ldg(p.inv_rh + i);
  const float4 abr = __ldg(p.ab_r + i), abq = __ldg(p.ab_q + i);
  // PML memory variables of the NV cells (radial: one vector per array;
  // z: one value per cell inside the z PML), loaded before any arithmetic
  const long long cr = rp ? ((long long)j * p.pml_r + (i - p.nr)) * NZp + k0 : 0;
  const int pz = p.pml_z;
  const long long czrow = ((long long)j * NR + i) * (2 * pz);
  const bool zl = !ZIN && pz > 0 && (k0 < pz || k0 + NV - 1 >= NZ - pz);
  float ur_vr[NV], uq_vr[NV], ur_vp[NV], uq_vp[NV], ur_vz[NV], uq_vz[NV];
  if (PRE && rp) {
    ldv(ur_vr, p.psr[R_VR] + cr);
    ldv(uq_vr, p.psr[Q_VR] + cr);
    ldv(ur_vp, p.psr[R_VP] + cr);
    ldv(uq_vp, p.psr[Q_VP] + cr);
    ldv(ur_vz, p.psr[R_VZ] + cr);
    ldv(uq_vz, p.psr[Q_VZ] + cr);
  }
  float uz_vr[NV], uz_vp[NV], uz_vz[NV];
  if (PRE && zl) {
#pragma unroll
    for (int e = 0; e < NV; e++) {
      const int k = k0 + e;
      if (k < NZ && (k < pz || k >= NZ - pz)) {
        const long long q = czrow + (k < pz ? k : k - (NZ - 2 * pz));
        uz_vr[e] = p.psz[Z_VR][q];
        uz_vp[e] = p.psz[Z_VP][q];
        uz_vz[e] = p.psz[Z_VZ][q];
      }
    }
  }

  if (!k4) id_k4 = idc[NV - 1];
  float rho_c[NV + 1], rho_j[NV], rho_m[NV];
#pragma unroll
  for (int e = 0; e < NV; e++) {
    rho_c[e] = __ldg(p.m_rho + idc[e]);
    rho_j[e] = __ldg(p.m_rho + idj[e]);
    rho_m[e] = __ldg(p.m_rho + idm[e]);
  }
  rho_c[NV] = __ldg(p.m_rho + id_k4);

  const float dtv = p.dtv, idr = p.inv_dr, idz = p.inv_dz, idth = p.inv_dth;

  float out_r[NV], out_p[NV], out_z[NV];
#pragma unroll
  for (int e = 0; e < NV; e++) {
    out_r[e] = o_vr[e];
    out_p[e] = o_vp[e];
    out_z[e] = o_vz[e];
  }
#pragma unroll
  for (int e = 0; e < NV; e++) {
    const int k = k0 + e;
    if (!ZIN && k >= NZ) break;
    const bool zp = zl && (k < pz || k >= NZ - pz);
    const int kz = k < pz ? k : k - (NZ - 2 * pz);
    const float4 abz = zp ? __ldg(p.ab_z + k) : z4();
    const float srr_e = a_srr[e], spp_e = a_spp[e], srp_e = a_srp[e];
    const float srz_e = a_srz[e], spz_e = a_spz[e], szz_e = a_szz[e];
    const float srz_m1 = e ? a_srz[e - 1] : srz_km, spz_m1 = e ? a_spz[e - 1] : spz_km;
    // v_r at (r_i, theta_j, z_k), i >= 1
    if (im) {
      float Dr = (srr_e - m_srr[e]) * idr;
      float Q = (0.5f * (srr_e + m_srr[e]) - 0.5f * (spp_e + m_spp[e]) + (srp_e - jm_srp[e]) * idth) *
                inv_ri;
      float Dz = (srz_e - srz_m1) * idz;
      if (rp) {
        Dr = (PRE ? stretch_reg(ur_vr[e], abr.x, abr.y, Dr) : stretch(p.psr[R_VR] + cr + e, abr.x, abr.y, Dr));
        Q = (PRE ? stretch_reg(uq_vr[e], abq.x, abq.y, Q) : stretch(p.psr[Q_VR] + cr + e, abq.x, abq.y, Q));
      }
      if (zp) Dz = (PRE ? stretch_reg(uz_vr[e], abz.x, abz.y, Dz) : stretch(p.psz[Z_VR] + czrow + kz, abz.x, abz.y, Dz));
      out_r[e] += vel_coef(dtv, rho_m[e] + rho_c[e]) * (Dr + Q + Dz);
    }
    // v_phi at (r_{i+1/2}, theta_{j+1/2}, z_k)
    {
      const float s1 = p_srp[e];
      float Dr = (s1 - srp_e) * idr;
      float Q = ((s1 + srp_e) + (jp_spp[e] - spp_e) * idth) * inv_rh;
      float Dz = (spz_e - spz_m1) * idz;
      if (rp) {
        Dr = (PRE ? stretch_reg(ur_vp[e], abr.z, abr.w, Dr) : stretch(p.psr[R_VP] + cr + e, abr.z, abr.w, Dr));
        Q = (PRE ? stretch_reg(uq_vp[e], abq.z, abq.w, Q) : stretch(p.psr[Q_VP] + cr + e, abq.z, abq.w, Q));
      }
      if (zp) Dz = (PRE ? stretch_reg(uz_vp[e], abz.x, abz.y, Dz) : stretch(p.psz[Z_VP] + czrow + kz, abz.x, abz.y, Dz));
      out_p[e] += vel_coef(dtv, rho_c[e] + rho_j[e]) * (Dr + Q + Dz);
    }
    // v_z at (r_{i+1/2}, theta_j, z_{k+1/2}), k + 1 < NZ
    if (ZIN || k + 1 < NZ) {
      const float s1 = p_srz[e];
      float Dr = (s1 - srz_e) * idr;
      float Q = (0.5f * (s1 + srz_e) + (spz_e - jm_spz[e]) * idth) * inv_rh;
      float Dz = ((e < NV - 1 ? a_szz[e + 1] : szz_k4) - szz_e) * idz;
      if (rp) {
        Dr = (PRE ? stretch_reg(ur_vz[e], abr.z, abr.w, Dr) : stretch(p.psr[R_VZ] + cr + e, abr.z, abr.w, Dr));
        Q = (PRE ? stretch_reg(uq_vz[e], abq.z, abq.w, Q) : stretch(p.psr[Q_VZ] + cr + e, abq.z, abq.w, Q));
      }
      if (zp) Dz = (PRE ? stretch_reg(uz_vz[e], abz.z, abz.w, Dz) : stretch(p.psz[Z_VZ] + czrow + kz, abz.z, abz.w, Dz));
      out_z[e] += vel_coef(dtv, rho_c[e] + rho_c[e + 1]) * (Dr + Q + Dz);
    }
  }
  const SrKey sk = body_key<T>(p, j, i, k0);
  if (im) st_field<T, NV, false>(vr + c, out_r, sk, F_VR);
  st_field<T, NV, false>(vp + c, out_p, sk, F_VP);
  st_field<T, NV, false>(vz + c, out_z, sk, F_VZ);
  if (PRE && rp) {  // cells the loop skipped keep the values loaded
    stv(p.psr[R_VR] + cr, ur_vr);
    stv(p.psr[Q_VR] + cr, uq_vr);
    stv(p.psr[R_VP] + cr, ur_vp);
    stv(p.psr[Q_VP] + cr, uq_vp);
    stv(p.psr[R_VZ] + cr, ur_vz);
    stv(p.psr[Q_VZ] + cr, uq_vz);
  }
  if (PRE && zl) {
#pragma unroll
    for (int e = 0; e < NV; e++) {
      const int k = k0 + e;
      if (k < NZ && (k < pz || k >= NZ - pz)) {
        const long long q = czrow + (k < pz ? k : k - (NZ - 2 * pz));
        p.psz[Z_VR][q] = uz_vr[e];
        p.psz[Z_VP][q] = uz_vp[e];
        p.psz[Z_VZ][q] = uz_vz[e];
      }
    }
  }
}

// CG: the velocities are read through L2 only (ldrow / ldone), for a launch
// in which other blocks wrote them, and the cell's own stresses are read and
// written streaming (last use in the launch)
template <typename T, int NV, bool LEAN, bool PRE = false, bool ZIN = LEAN, bool CG = false>
__device__ __forceinline__ void str_hoist_body(const KParams &p, const int j, const int i, const int k0) {
  const int nth = p.nth, NR = p.NR, NZ = p.NZ;
  const long long NZp = p.NZp, pl = p.plane;
  const int jm = j == 0 ? nth - 1 : j - 1, jp = j == nth - 1 ? 0 : j + 1;
  const long long c = (long long)j * pl + i * NZp + k0;
  const long long cjm = (long long)jm * pl + i * NZp + k0;
  const long long cjp = (long long)jp * pl + i * NZp + k0;
  const T *vr = (const T *)p.f[F_VR], *vp = (const T *)p.f[F_VP], *vz = (const T *)p.f[F_VZ];
  T *srr = (T *)p.f[F_SRR], *spp = (T *)p.f[F_SPP], *szz = (T *)p.f[F_SZZ];
  T *srp = (T *)p.f[F_SRP], *spz = (T *)p.f[F_SPZ], *srz = (T *)p.f[F_SRZ];
  const bool im = i >= 1, ip = i + 1 < NR, k4 = ZIN || k0 + NV < NZ, km = k0 > 0;

  // ---- every load
  float a_vr[NV];
  ldrow<T, NV, CG>(a_vr, vr + c);
  float a_vp[NV];
  ldrow<T, NV, CG>(a_vp, vp + c);
  float a_vz[NV];
  ldrow<T, NV, CG>(a_vz, vz + c);
  const float vr_k4 = k4 ? ldone<T, CG>(vr + c + NV) : 0.f, vp_k4 = k4 ? ldone<T, CG>(vp + c + NV) : 0.f;
  const float vz_km = km ? ldone<T, CG>(vz + c - 1) : 0.f;
  float p_vr[NV];
  if (ip) ldrow<T, NV, CG>(p_vr, vr + c + NZp);
  else zero(p_vr);
  float jm_vp[NV];
  ldrow<T, NV, CG>(jm_vp, vp + cjm);
  float m_vp[NV];
  if (im) ldrow<T, NV, CG>(m_vp, vp + c - NZp);
  else zero(m_vp);
  float m_vz[NV];
  if (im) ldrow<T, NV, CG>(m_vz, vz + c - NZp);
  else zero(m_vz);
  float jp_vr[NV];
  ldrow<T, NV, CG>(jp_vr, vr + cjp);
  float jp_vz[NV];
  ldrow<T, NV, CG>(jp_vz, vz + cjp);
  float o_rr[NV];
  ldown<T, NV, CG>(o_rr, srr + c);
  float o_pp[NV];
  ldown<T, NV, CG>(o_pp, spp + c);
  float o_zz[NV];
  ldown<T, NV, CG>(o_zz, szz + c);
  float o_rp[NV];
  ldown<T, NV, CG>(o_rp, srp + c);
  float o_pz[NV];
  ldown<T, NV, CG>(o_pz, spz + c);
  float o_rz[NV];
  ldown<T, NV, CG>(o_rz, srz + c);
  int idc[NV], idj[NV], idm[NV], idjm[NV];
  ldids(p.id + c, idc);
  ldids(p.id + cjp, idj);
  if (im) {
    ldids(p.id + c - NZp, idm);
    ldids(p.id + cjp - NZp, idjm);
  } else {
    zero_ids(idm);
    zero_ids(idjm);
  }
  int idc4 = 0, idj4 = 0, idm4 = 0;
  if (k4) {
    idc4 = __ldg(p.id + c + NV);
    idj4 = __ldg(p.id + cjp + NV);
    if (im) idm4 = __ldg(p.id + c - NZp + NV);
  }
  const bool rp = !LEAN && i >= p.nr;
  const float inv_ri = __ldg(p.inv_ri + i), inv_rh = __ldg(p.inv_rh + i);
  const float4 abr = __ldg(p.ab_r + i), abq = __ldg(p.ab_q + i);
  // PML memory variables of the NV cells, loaded before any arithmetic
  const long long cr = rp ? ((long long)j * p.pml_r + (i - p.nr)) * NZp + k0 : 0;
  const int pz = p.pml_z;
  const long long czrow = ((long long)j * NR + i) * (2 * pz);
  const bool zl = !ZIN && pz > 0 && (k0 < pz || k0 + NV - 1 >= NZ - pz);
  float ur_rr[NV], uq_pp[NV], ur_rp[NV], uq_rp[NV], ur_rz[NV], uq_pz[NV];
  if (PRE && rp) {
    ldv(ur_rr, p.psr[R_ERR] + cr);
    ldv(uq_pp, p.psr[Q_EPP] + cr);
    ldv(ur_rp, p.psr[R_GRP] + cr);
    ldv(uq_rp, p.psr[Q_GRP] + cr);
    ldv(ur_rz, p.psr[R_GRZ] + cr);
    ldv(uq_pz, p.psr[Q_GPZ] + cr);
  }
  float uz_zz[NV], uz_rz[NV], uz_pz[NV];
  if (PRE && zl) {
#pragma unroll
    for (int e = 0; e < NV; e++) {
      const int k = k0 + e;
      if (k < NZ && (k < pz || k >= NZ - pz)) {
        const long long q = czrow + (k < pz ? k : k - (NZ - 2 * pz));
        uz_zz[e] = p.psz[Z_EZZ][q];
        uz_rz[e] = p.psz[Z_GRZ][q];
        uz_pz[e] = p.psz[Z_GPZ][q];
      }
    }
  }
  float src[NV] = {};
  if (i == p.src_i && (p.src_j < 0 || p.src_j == j) && p.src_k >= k0 && p.src_k < k0 + NV) {
    const int n = *p.step;
    src[p.src_k - k0] = n < p.n_wav ? __ldg(p.wav + n) : 0.f;
  }

  if (!k4) {
    idc4 = idc[NV - 1];
    idj4 = idj[NV - 1];
    idm4 = idm[NV - 1];
  }
  float imu_c[NV + 1], imu_j[NV + 1], imu_m[NV + 1], imu_jm[NV];
  float2 lam[NV];
#pragma unroll
  for (int e = 0; e < NV; e++) {
    imu_c[e] = __ldg(p.m_imu + idc[e]);
    imu_j[e] = __ldg(p.m_imu + idj[e]);
    imu_m[e] = __ldg(p.m_imu + idm[e]);
    imu_jm[e] = __ldg(p.m_imu + idjm[e]);
    lam[e] = __ldg(p.m_lam + idc[e]);
  }
  imu_c[NV] = __ldg(p.m_imu + idc4);
  imu_j[NV] = __ldg(p.m_imu + idj4);
  imu_m[NV] = __ldg(p.m_imu + idm4);

  const float dts = p.dts, idr = p.inv_dr, idz = p.inv_dz, idth = p.inv_dth;

  float orr[NV], opp[NV], ozz[NV], orp[NV], opz[NV], orz[NV];
#pragma unroll
  for (int e = 0; e < NV; e++) {
    orr[e] = o_rr[e];
    opp[e] = o_pp[e];
    ozz[e] = o_zz[e];
    orp[e] = o_rp[e];
    opz[e] = o_pz[e];
    orz[e] = o_rz[e];
  }
#pragma unroll
  for (int e = 0; e < NV; e++) {
    const int k = k0 + e;
    if (!ZIN && k >= NZ) break;
    const bool zp = zl && (k < pz || k >= NZ - pz);
    const int kz = k < pz ? k : k - (NZ - 2 * pz);
    const float4 abz = zp ? __ldg(p.ab_z + k) : z4();
    const float vr_e = a_vr[e], vp_e = a_vp[e], vz_e = a_vz[e];
    const float vr_e1 = e < NV - 1 ? a_vr[e + 1] : vr_k4, vp_e1 = e < NV - 1 ? a_vp[e + 1] : vp_k4;
    const float vz_m1 = e ? a_vz[e - 1] : vz_km;
    // normal stresses at the cell centre
    {
      const float vr1 = p_vr[e];
      float err = (vr1 - vr_e) * idr;
      float epp = ((vp_e - jm_vp[e]) * idth + 0.5f * (vr_e + vr1)) * inv_rh;
      float ezz = (vz_e - vz_m1) * idz;
      if (rp) {
        err = (PRE ? stretch_reg(ur_rr[e], abr.z, abr.w, err) : stretch(p.psr[R_ERR] + cr + e, abr.z, abr.w, err));
        epp = (PRE ? stretch_reg(uq_pp[e], abq.z, abq.w, epp) : stretch(p.psr[Q_EPP] + cr + e, abq.z, abq.w, epp));
      }
      if (zp) ezz = (PRE ? stretch_reg(uz_zz[e], abz.x, abz.y, ezz) : stretch(p.psz[Z_EZZ] + czrow + kz, abz.x, abz.y, ezz));
      const float l = lam[e].x, l2m = lam[e].y;
      orr[e] += dts * (l2m * err + l * (epp + ezz)) + src[e];
      opp[e] += dts * (l2m * epp + l * (err + ezz)) + src[e];
      ozz[e] += dts * (l2m * ezz + l * (err + epp)) + src[e];
    }
    if (im) {
      // s_rphi at (r_i, theta_{j+1/2}, z_k)
      {
        float gr = (vp_e - m_vp[e]) * idr;
        float Q = ((jp_vr[e] - vr_e) * idth - 0.5f * (vp_e + m_vp[e])) * inv_ri;
        if (rp) {
          gr = (PRE ? stretch_reg(ur_rp[e], abr.x, abr.y, gr) : stretch(p.psr[R_GRP] + cr + e, abr.x, abr.y, gr));
          Q = (PRE ? stretch_reg(uq_rp[e], abq.x, abq.y, Q) : stretch(p.psr[Q_GRP] + cr + e, abq.x, abq.y, Q));
        }
        const float mu = mu_harm(imu_m[e] + imu_c[e] + imu_jm[e] + imu_j[e]);
        orp[e] += dts * mu * (gr + Q);
      }
      // s_rz at (r_i, theta_j, z_{k+1/2})
      if (ZIN || k + 1 < NZ) {
        float gz = (vr_e1 - vr_e) * idz;
        float gr = (vz_e - m_vz[e]) * idr;
        if (zp) gz = (PRE ? stretch_reg(uz_rz[e], abz.z, abz.w, gz) : stretch(p.psz[Z_GRZ] + czrow + kz, abz.z, abz.w, gz));
        if (rp) gr = (PRE ? stretch_reg(ur_rz[e], abr.x, abr.y, gr) : stretch(p.psr[R_GRZ] + cr + e, abr.x, abr.y, gr));
        const float mu = mu_harm(imu_m[e] + imu_c[e] + imu_m[e + 1] + imu_c[e + 1]);
        orz[e] += dts * mu * (gz + gr);
      }
    }
    // s_phiz at (r_{i+1/2}, theta_{j+1/2}, z_{k+1/2})
    if (ZIN || k + 1 < NZ) {
      float Q = (jp_vz[e] - vz_e) * idth * inv_rh;
      float gz = (vp_e1 - vp_e) * idz;
      if (rp) Q = (PRE ? stretch_reg(uq_pz[e], abq.z, abq.w, Q) : stretch(p.psr[Q_GPZ] + cr + e, abq.z, abq.w, Q));
      if (zp) gz = (PRE ? stretch_reg(uz_pz[e], abz.z, abz.w, gz) : stretch(p.psz[Z_GPZ] + czrow + kz, abz.z, abz.w, gz));
      const float mu = mu_harm(imu_c[e] + imu_j[e] + imu_c[e + 1] + imu_j[e + 1]);
      opz[e] += dts * mu * (Q + gz);
    }
  }
  const SrKey sk = body_key<T>(p, j, i, k0);
  st_field<T, NV, CG>(srr + c, orr, sk, F_SRR);
  st_field<T, NV, CG>(spp + c, opp, sk, F_SPP);
  st_field<T, NV, CG>(szz + c, ozz, sk, F_SZZ);
  if (im) {
    st_field<T, NV, CG>(srp + c, orp, sk, F_SRP);
    st_field<T, NV, CG>(srz + c, orz, sk, F_SRZ);
  }
  st_field<T, NV, CG>(spz + c, opz, sk, F_SPZ);
  if (PRE && rp) {  // cells the loop skipped keep the values loaded
    stv(p.psr[R_ERR] + cr, ur_rr);
    stv(p.psr[Q_EPP] + cr, uq_pp);
    stv(p.psr[R_GRP] + cr, ur_rp);
    stv(p.psr[Q_GRP] + cr, uq_rp);
    stv(p.psr[R_GRZ] + cr, ur_rz);
    stv(p.psr[Q_GPZ] + cr, uq_pz);
  }
  if (PRE && zl) {
#pragma unroll
    for (int e = 0; e < NV; e++) {
      const int k = k0 + e;
      if (k < NZ && (k < pz || k >= NZ - pz)) {
        const long long q = czrow + (k < pz ? k : k - (NZ - 2 * pz));
        p.psz[Z_EZZ][q] = uz_zz[e];
        p.psz[Z_GRZ][q] = uz_rz[e];
        p.psz[Z_GPZ][q] = uz_pz[e];
      }
    }
  }
}

template <int NV>
__device__ __forceinline__ bool lean_cells(const KParams &p, int i, int k0) {
  return i < p.nr && k0 >= p.pml_z && k0 + NV < p.NZ - p.pml_z;
}

// PRE: the general body loads the PML memory variables of its cells with the
// fields and updates them in registers (for kernels with the registers to
// spare); otherwise it reads and rewrites each one where it is used
template <typename T, int NV, bool VEL, bool PRE = false, bool CG = false>
__device__ __forceinline__ void hoist_cells(const KParams &p, int j, int i, int k0) {
  if (lean_cells<NV>(p, i, k0)) {
    if (VEL) vel_hoist_body<T, NV, true>(p, j, i, k0);
    else str_hoist_body<T, NV, true, false, true, CG>(p, j, i, k0);
  } else {
    if (VEL) vel_hoist_body<T, NV, false, PRE>(p, j, i, k0);
    else str_hoist_body<T, NV, false, PRE, false, CG>(p, j, i, k0);
  }
}

// L2 prefetch of every 128-byte line a thread's cells at (j, i, k0) will load
// (fields and IDs of the cell and of its r and theta neighbours), issued by
// one lane per line; nothing is held in registers or shared memory.
__device__ __forceinline__ void prefetch_l2(const void *a) { asm volatile("prefetch.global.L2 [%0];" ::"l"(a)); }

template <typename T, int NV, bool VEL>
__device__ __forceinline__ void prefetch_tile(const KParams &p, int j, int i, int k0) {
  constexpr int LANES = 128 / (NV * (int)sizeof(T));  // threads per 128-byte line of a field row
  constexpr int LANES_ID = 128 / (NV * 2);
  const long long pl = p.plane, NZp = p.NZp;
  const int jm = j == 0 ? p.nth - 1 : j - 1, jp = j == p.nth - 1 ? 0 : j + 1;
  const long long c = (long long)j * pl + i * NZp + k0, cjm = (long long)jm * pl + i * NZp + k0,
                  cjp = (long long)jp * pl + i * NZp + k0;
  const bool im = i >= 1, ip = i + 1 < p.NR;
  if ((threadIdx.x & (LANES - 1)) == 0) {
    const T *const *f = (const T *const *)p.f;
    if (VEL) {
      for (int q = F_VR; q <= F_VZ; q++) prefetch_l2(f[q] + c);
      prefetch_l2(f[F_SRR] + c), prefetch_l2(f[F_SPP] + c), prefetch_l2(f[F_SZZ] + c);
      prefetch_l2(f[F_SRP] + c), prefetch_l2(f[F_SPZ] + c), prefetch_l2(f[F_SRZ] + c);
      if (im) prefetch_l2(f[F_SRR] + c - NZp), prefetch_l2(f[F_SPP] + c - NZp);
      if (ip) prefetch_l2(f[F_SRP] + c + NZp), prefetch_l2(f[F_SRZ] + c + NZp);
      prefetch_l2(f[F_SRP] + cjm), prefetch_l2(f[F_SPZ] + cjm), prefetch_l2(f[F_SPP] + cjp);
    } else {
      for (int q = F_SRR; q <= F_SRZ; q++) prefetch_l2(f[q] + c);
      prefetch_l2(f[F_VR] + c), prefetch_l2(f[F_VP] + c), prefetch_l2(f[F_VZ] + c);
      if (ip) prefetch_l2(f[F_VR] + c + NZp);
      if (im) prefetch_l2(f[F_VP] + c - NZp), prefetch_l2(f[F_VZ] + c - NZp);
      prefetch_l2(f[F_VP] + cjm), prefetch_l2(f[F_VR] + cjp), prefetch_l2(f[F_VZ] + cjp);
    }
  }
  if ((threadIdx.x & (LANES_ID - 1)) == 0) {
    prefetch_l2(p.id + c);
    prefetch_l2(p.id + cjp);
    if (im) {
      prefetch_l2(p.id + c - NZp);
      if (!VEL) prefetch_l2(p.id + cjp - NZp);
    }
  }
}

}  // namespace
}  // namespace cwell
