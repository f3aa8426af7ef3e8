// Split path, load-first variant: the velocity and stress kernels of
// stencil_split.cu with every global load of a thread issued before any of
// its arithmetic or stores (one round trip to memory per thread instead of
// one per component), and the material lookups from the split tables
// {rho}, {1/mu}, {lambda, lambda + 2 mu}.  Same thread layout (four z cells
// per thread, 16-byte loads, block = 32 x 4 threads, theta fastest across
// blocks), same arithmetic, same in-place update; variants with two z cells
// per thread (8-byte loads, fewer registers), and interior / edge split
// launches (a lean-only kernel on the interior tiles).
#include <algorithm>

#include "cwell_internal.cuh"

namespace cwell {
namespace {

constexpr int HB_X = 32;  // threads along z per block (NV cells each)
constexpr int HB_Y = 4;   // r rows per block

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
  if (im) Vec<T, NV>::st(vr + c, out_r);
  Vec<T, NV>::st(vp + c, out_p);
  Vec<T, NV>::st(vz + c, out_z);
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

template <typename T, int NV, bool LEAN, bool PRE = false, bool ZIN = LEAN>
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
  Vec<T, NV>::ld(a_vr, vr + c);
  float a_vp[NV];
  Vec<T, NV>::ld(a_vp, vp + c);
  float a_vz[NV];
  Vec<T, NV>::ld(a_vz, vz + c);
  const float vr_k4 = k4 ? St<T>::ld1(vr + c + NV) : 0.f, vp_k4 = k4 ? St<T>::ld1(vp + c + NV) : 0.f;
  const float vz_km = km ? St<T>::ld1(vz + c - 1) : 0.f;
  float p_vr[NV];
  if (ip) Vec<T, NV>::ld(p_vr, vr + c + NZp);
  else zero(p_vr);
  float jm_vp[NV];
  Vec<T, NV>::ld(jm_vp, vp + cjm);
  float m_vp[NV];
  if (im) Vec<T, NV>::ld(m_vp, vp + c - NZp);
  else zero(m_vp);
  float m_vz[NV];
  if (im) Vec<T, NV>::ld(m_vz, vz + c - NZp);
  else zero(m_vz);
  float jp_vr[NV];
  Vec<T, NV>::ld(jp_vr, vr + cjp);
  float jp_vz[NV];
  Vec<T, NV>::ld(jp_vz, vz + cjp);
  float o_rr[NV];
  Vec<T, NV>::ld(o_rr, srr + c);
  float o_pp[NV];
  Vec<T, NV>::ld(o_pp, spp + c);
  float o_zz[NV];
  Vec<T, NV>::ld(o_zz, szz + c);
  float o_rp[NV];
  Vec<T, NV>::ld(o_rp, srp + c);
  float o_pz[NV];
  Vec<T, NV>::ld(o_pz, spz + c);
  float o_rz[NV];
  Vec<T, NV>::ld(o_rz, srz + c);
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
  Vec<T, NV>::st(srr + c, orr);
  Vec<T, NV>::st(spp + c, opp);
  Vec<T, NV>::st(szz + c, ozz);
  if (im) {
    Vec<T, NV>::st(srp + c, orp);
    Vec<T, NV>::st(srz + c, orz);
  }
  Vec<T, NV>::st(spz + c, opz);
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
template <typename T, int NV, bool VEL, bool PRE = false>
__device__ __forceinline__ void hoist_cells(const KParams &p, int j, int i, int k0) {
  if (lean_cells<NV>(p, i, k0)) {
    if (VEL) vel_hoist_body<T, NV, true>(p, j, i, k0);
    else str_hoist_body<T, NV, true>(p, j, i, k0);
  } else {
    if (VEL) vel_hoist_body<T, NV, false, PRE>(p, j, i, k0);
    else str_hoist_body<T, NV, false, PRE>(p, j, i, k0);
  }
}

// Block order: ZF = false walks theta fastest (blockIdx.x = theta, y = r tile,
// z = z tile: co-resident blocks share theta-neighbour rows); ZF = true walks
// z fastest (x = z tile, y = r tile, z = theta: co-resident blocks stream
// whole rows, theta neighbours come back from L2).
template <bool ZF, int NV>
__device__ __forceinline__ void block_cell(int &j, int &i, int &k0) {
  const int zt = ZF ? blockIdx.x : blockIdx.z;
  j = ZF ? blockIdx.z : blockIdx.x;
  i = blockIdx.y * HB_Y + threadIdx.y;
  k0 = (zt * HB_X + threadIdx.x) * NV;
}

template <typename T, int NV, int MINB, bool ZF>
__global__ void __launch_bounds__(HB_X *HB_Y, MINB) vel_hoist(const KParams p) {
  int j, i, k0;
  block_cell<ZF, NV>(j, i, k0);
  if (i < p.NR && k0 < p.NZ) hoist_cells<T, NV, true>(p, j, i, k0);
}

template <typename T, int NV, int MINB, bool ZF>
__global__ void __launch_bounds__(HB_X *HB_Y, MINB) str_hoist(const KParams p) {
  int j, i, k0;
  block_cell<ZF, NV>(j, i, k0);
  if (i < p.NR && k0 < p.NZ) hoist_cells<T, NV, false>(p, j, i, k0);
}

// Interior / edge split: the interior tiles (every row outside the radial
// PML, every cell of the tile away from the z PML and the z end) run a kernel
// compiled with the lean body only, so it needs fewer registers and more
// blocks fit on an SM; the remaining tiles (radial-PML rows, the z ends) run
// the per-thread lean / general dispatch.  Both walk theta fastest.
struct Split2 {
  int nrt_in;              // r tiles whose rows are all outside the radial PML
  int zt_lo, zt_hi;        // interior z tiles: zt_lo <= zt < zt_hi (interior kernel's tiles)
  int nrt;                 // all r tiles
  int ez_lo, ez_hi, enzt;  // the same z bounds in the edge kernel's tiles; all edge z tiles
};

// NV: cells per thread of the interior kernel, NVE: of the edge kernel
template <int NV, int NVE>
Split2 split2(const KParams &p) {
  static_assert(NV % NVE == 0, "an interior tile spans whole edge tiles");
  const int W = NV * HB_X, WE = NVE * HB_X;
  Split2 q;
  q.nrt = (p.NR + HB_Y - 1) / HB_Y;
  q.nrt_in = p.nr / HB_Y;
  q.zt_lo = (p.pml_z + W - 1) / W;
  q.zt_hi = std::max(q.zt_lo, (p.NZ - p.pml_z - 1) / W);  // (zt + 1) W <= NZ - pml_z - 1
  q.ez_lo = q.zt_lo * (W / WE);
  q.ez_hi = q.zt_hi * (W / WE);
  q.enzt = (p.NZ + WE - 1) / WE;
  return q;
}

template <typename T, int NV, int MINB, bool VEL>
__global__ void __launch_bounds__(HB_X *HB_Y, MINB) hoist_interior(const KParams p, int zt_lo) {
  const int j = blockIdx.x, i = blockIdx.y * HB_Y + threadIdx.y;
  const int k0 = ((zt_lo + blockIdx.z) * HB_X + threadIdx.x) * NV;
  if (i < p.i_lo || i >= p.i_hi) return;
  if (VEL) vel_hoist_body<T, NV, true>(p, j, i, k0);
  else str_hoist_body<T, NV, true>(p, j, i, k0);
}

// Persistent interior kernel with an L2 prefetch of its next tile: one wave
// of resident blocks walks the interior tiles in the order above (theta
// fastest); before computing its tile a block asks L2 for every row its next
// tile will load (one prefetch per 128-byte line), so those loads find their
// lines in L2.  No register or shared memory holds the prefetched data.
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

template <typename T, int NV, int MINB, bool VEL>
__global__ void __launch_bounds__(HB_X *HB_Y, MINB)
    hoist_interior_pf(const KParams p, int zt_lo, int nrt_in, int ntiles) {
  auto cell = [&](int t, int &j, int &i, int &k0) {
    j = t % p.nth;
    t /= p.nth;
    i = (t % nrt_in) * HB_Y + threadIdx.y;
    k0 = ((zt_lo + t / nrt_in) * HB_X + threadIdx.x) * NV;
  };
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int j, i, k0;
    if (t + (int)gridDim.x < ntiles) {
      cell(t + gridDim.x, j, i, k0);
      prefetch_tile<T, NV, VEL>(p, j, i, k0);
    }
    cell(t, j, i, k0);
    if (i < p.i_lo || i >= p.i_hi) continue;
    if (VEL) vel_hoist_body<T, NV, true>(p, j, i, k0);
    else str_hoist_body<T, NV, true>(p, j, i, k0);
  }
}

// edge tile t (in edge-kernel tiles of NV * HB_X cells along z): first the r
// tiles nrt_in .. nrt-1 with every z tile, then the interior r tiles with the
// z tiles below ez_lo and from ez_hi on
__device__ __forceinline__ void edge_tile(const Split2 &q, int t, int &rt, int &zt) {
  const int a = (q.nrt - q.nrt_in) * q.enzt;
  if (t < a) {
    rt = q.nrt_in + t / q.enzt;
    zt = t % q.enzt;
  } else {
    t -= a;
    const int nz_edge = q.ez_lo + (q.enzt - q.ez_hi);
    rt = t / nz_edge;
    const int e = t % nz_edge;
    zt = e < q.ez_lo ? e : q.ez_hi + (e - q.ez_lo);
  }
}

inline long long edge_tiles(const Split2 &q) {
  return (long long)(q.nrt - q.nrt_in) * q.enzt + (long long)q.nrt_in * (q.ez_lo + q.enzt - q.ez_hi);
}

template <typename T, int NV, int MINB, bool VEL>
__global__ void __launch_bounds__(HB_X *HB_Y, MINB) hoist_edge(const KParams p, Split2 q) {
  int rt, zt;
  edge_tile(q, blockIdx.y, rt, zt);
  const int j = blockIdx.x, i = rt * HB_Y + threadIdx.y, k0 = (zt * HB_X + threadIdx.x) * NV;
  if (i >= p.i_lo && i < p.i_hi && k0 < p.NZ) hoist_cells<T, NV, VEL, true>(p, j, i, k0);
}

// the same edge tiles walked by one wave of resident blocks, each prefetching
// its next tile's rows into L2 (radial-PML memory variables included); only
// cells inside the grid are prefetched
template <typename T, int NV, int MINB, bool VEL>
__global__ void __launch_bounds__(HB_X *HB_Y, MINB) hoist_edge_pf(const KParams p, Split2 q, int ntiles) {
  auto cell = [&](int t, int &j, int &i, int &k0) {
    int rt, zt;
    j = t % p.nth;
    edge_tile(q, t / p.nth, rt, zt);
    i = rt * HB_Y + threadIdx.y;
    k0 = (zt * HB_X + threadIdx.x) * NV;
  };
  constexpr int LANES = 128 / (NV * 4);
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int j, i, k0;
    if (t + (int)gridDim.x < ntiles) {
      cell(t + gridDim.x, j, i, k0);
      if (i < p.NR && k0 < p.NZ) {
        prefetch_tile<T, NV, VEL>(p, j, i, k0);
        if (i >= p.nr && (threadIdx.x & (LANES - 1)) == 0) {
          const long long cr = ((long long)j * p.pml_r + (i - p.nr)) * p.NZp + k0;
          const int q0 = VEL ? R_VR : R_ERR, q1 = VEL ? Q_VR : Q_EPP;
          for (int u = 0; u < 3; u++) prefetch_l2(p.psr[q0 + u] + cr), prefetch_l2(p.psr[q1 + u] + cr);
        }
      }
    }
    cell(t, j, i, k0);
    if (i >= p.i_lo && i < p.i_hi && k0 < p.NZ) hoist_cells<T, NV, VEL, true>(p, j, i, k0);
  }
}

// Three-way split of a half step: interior tiles (above), the z-interior
// tiles of the other rows (in a well, the radial PML) with a body compiled
// for "radial PML, interior z" (no z memory variable, no z bound check), and
// the z-end tiles of every row with the general body.  Both walk their tiles
// as one wave of resident blocks that prefetch the next tile into L2.
template <typename T, int NV, bool VEL>
__device__ __forceinline__ void prefetch_edge_tile(const KParams &p, int j, int i, int k0) {
  constexpr int LANES = 128 / (NV * 4);
  if (i >= p.NR || k0 >= p.NZ) return;
  prefetch_tile<T, NV, VEL>(p, j, i, k0);
  if (i >= p.nr && (threadIdx.x & (LANES - 1)) == 0) {
    const long long cr = ((long long)j * p.pml_r + (i - p.nr)) * p.NZp + k0;
    const int q0 = VEL ? R_VR : R_ERR, q1 = VEL ? Q_VR : Q_EPP;
    for (int u = 0; u < 3; u++) prefetch_l2(p.psr[q0 + u] + cr), prefetch_l2(p.psr[q1 + u] + cr);
  }
}

template <typename T, int NV, int MINB, bool VEL>
__global__ void __launch_bounds__(HB_X *HB_Y, MINB) hoist_radial_pf(const KParams p, Split2 q, int ntiles) {
  const int nrr = q.nrt - q.nrt_in;
  auto cell = [&](int t, int &j, int &i, int &k0) {
    j = t % p.nth;
    t /= p.nth;
    i = (q.nrt_in + t % nrr) * HB_Y + threadIdx.y;
    k0 = ((q.ez_lo + t / nrr) * HB_X + threadIdx.x) * NV;
  };
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int j, i, k0;
    if (t + (int)gridDim.x < ntiles) {
      cell(t + gridDim.x, j, i, k0);
      prefetch_edge_tile<T, NV, VEL>(p, j, i, k0);
    }
    cell(t, j, i, k0);
    if (i < p.i_lo || i >= p.i_hi) continue;
    if (VEL) vel_hoist_body<T, NV, false, true, true>(p, j, i, k0);
    else str_hoist_body<T, NV, false, true, true>(p, j, i, k0);
  }
}

template <typename T, int NV, int MINB, bool VEL>
__global__ void __launch_bounds__(HB_X *HB_Y, MINB) hoist_ends_pf(const KParams p, Split2 q, int ntiles) {
  const int nzend = q.ez_lo + (q.enzt - q.ez_hi);
  auto cell = [&](int t, int &j, int &i, int &k0) {
    j = t % p.nth;
    t /= p.nth;
    const int e = t % nzend, zt = e < q.ez_lo ? e : q.ez_hi + (e - q.ez_lo);
    i = (t / nzend) * HB_Y + threadIdx.y;
    k0 = (zt * HB_X + threadIdx.x) * NV;
  };
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int j, i, k0;
    if (t + (int)gridDim.x < ntiles) {
      cell(t + gridDim.x, j, i, k0);
      prefetch_edge_tile<T, NV, VEL>(p, j, i, k0);
    }
    cell(t, j, i, k0);
    if (i >= p.i_lo && i < p.i_hi && k0 < p.NZ) hoist_cells<T, NV, VEL, true>(p, j, i, k0);
  }
}

// Batched scenarios: each half step is two persistent launches over the work
// lists of up to BATCH_MAX cases, one over every case's interior tiles (lean
// body only) and one over their edge tiles (radial-PML rows and z ends,
// general body); item = (case, theta, tile), theta fastest inside a case so
// that the theta neighbours a block reads are read by co-resident blocks too.
// The cases' parameters, their tile bounds and the prefix sum of the
// launch's items (start[c] = first item of case c, start[n] = total) travel in
// the kernel's parameter space, so a block reads its case's geometry and
// buffers from the constant bank.  The index inside a case is 32-bit (checked
// on the host); rows outside [i_lo, i_hi) are left alone (as in every
// split kernel: the ghost rows of an azimuthally refined grid's zones).  Cells per
// thread and blocks per SM: the velocity half takes
// interior (4, 5) and edge (4, 3), the stress half interior (4, 4) and edge
// (2, 4), the split launches the tuner picks for the single well.
struct BatchParams {
  KParams cases[BATCH_MAX];
  Split2 q[BATCH_MAX];
  long long start[BATCH_MAX + 1];
  int n;
};
static_assert(sizeof(BatchParams) <= 32000, "batch parameters exceed the kernel parameter space");

constexpr int BATCH_NV = 4;
template <bool VEL>
struct BatchCfg;
template <>
struct BatchCfg<true> {
  static constexpr int MINB_IN = 5, NVE = 4, MINB_E = 3;
  static constexpr bool PF = false;
};
template <>
struct BatchCfg<false> {
  static constexpr int MINB_IN = 4, NVE = 2, MINB_E = 4;
  // an L2 prefetch of the next item, which pays off in the one-wave interior
  // kernel, is slower here: the tuned grid is several waves deep
  static constexpr bool PF = false;
};

__device__ __forceinline__ int batch_case(const BatchParams &bp, long long item) {
  int lo = 0, hi = bp.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bp.start[mid] <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename T, bool VEL>
__global__ void __launch_bounds__(HB_X *HB_Y, BatchCfg<VEL>::MINB_IN)
    batch_interior(const __grid_constant__ BatchParams bp) {
  const long long total = bp.start[bp.n];
  auto cell = [&](long long item, int &c, int &j, int &i, int &k0) {
    c = batch_case(bp, item);
    const Split2 &q = bp.q[c];
    int t = (int)(item - bp.start[c]);
    j = t % bp.cases[c].nth;
    t /= bp.cases[c].nth;
    i = (t % q.nrt_in) * HB_Y + threadIdx.y;
    k0 = ((q.zt_lo + t / q.nrt_in) * HB_X + threadIdx.x) * BATCH_NV;
  };
  for (long long item = blockIdx.x; item < total; item += gridDim.x) {
    int c, j, i, k0;
    if (BatchCfg<VEL>::PF && item + gridDim.x < total) {
      cell(item + gridDim.x, c, j, i, k0);
      prefetch_tile<T, BATCH_NV, VEL>(bp.cases[c], j, i, k0);
    }
    cell(item, c, j, i, k0);
    const KParams &p = bp.cases[c];
    if (i < p.i_lo || i >= p.i_hi) continue;
    if (VEL) vel_hoist_body<T, BATCH_NV, true>(p, j, i, k0);
    else str_hoist_body<T, BATCH_NV, true>(p, j, i, k0);
  }
}

template <typename T, bool VEL>
__global__ void __launch_bounds__(HB_X *HB_Y, BatchCfg<VEL>::MINB_E) batch_edge(const __grid_constant__ BatchParams bp) {
  constexpr int NVE = BatchCfg<VEL>::NVE;
  const long long total = bp.start[bp.n];
  for (long long item = blockIdx.x; item < total; item += gridDim.x) {
    const int c = batch_case(bp, item);
    const KParams &p = bp.cases[c];
    int t = (int)(item - bp.start[c]), rt, zt;
    const int j = t % p.nth;
    edge_tile(bp.q[c], t / p.nth, rt, zt);
    const int i = rt * HB_Y + threadIdx.y, k0 = (zt * HB_X + threadIdx.x) * NVE;
    if (i >= p.i_lo && i < p.i_hi && k0 < p.NZ) hoist_cells<T, NVE, VEL, true>(p, j, i, k0);
  }
}

template <typename T, bool VEL>
cudaError_t launch_batch_t(const KParams *cases, int n_cases, int grid, cudaStream_t s) {
  using C = BatchCfg<VEL>;
  dim3 blk(HB_X, HB_Y);
  static thread_local BatchParams bp;  // large: kept off the stack
  for (int c0 = 0; c0 < n_cases; c0 += BATCH_MAX) {
    const int n = std::min(BATCH_MAX, n_cases - c0);
    bp.n = n;
    for (int c = 0; c < n; c++) {
      bp.cases[c] = cases[c0 + c];
      bp.q[c] = split2<BATCH_NV, C::NVE>(cases[c0 + c]);
    }
    // interior tiles
    bp.start[0] = 0;
    for (int c = 0; c < n; c++) {
      const Split2 &q = bp.q[c];
      bp.start[c + 1] = bp.start[c] + (long long)bp.cases[c].nth * q.nrt_in * (q.zt_hi - q.zt_lo);
    }
    if (bp.start[n] > 0)
      batch_interior<T, VEL><<<(int)std::min<long long>(grid, bp.start[n]), blk, 0, s>>>(bp);
    // edge tiles
    for (int c = 0; c < n; c++) bp.start[c + 1] = bp.start[c] + (long long)bp.cases[c].nth * edge_tiles(bp.q[c]);
    if (bp.start[n] > 0) batch_edge<T, VEL><<<(int)std::min<long long>(grid, bp.start[n]), blk, 0, s>>>(bp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n < 1) n = 1;
  }
  return n;
}

template <typename T, int NV, int MINB_IN, int NVE, int MINB_E, bool VEL, bool PF, bool PFE>
cudaError_t launch_split2_half(const KParams &p, const Split2 &q, cudaStream_t s) {
  dim3 blk(HB_X, HB_Y);
  const int nin = q.zt_hi - q.zt_lo;
  if (q.nrt_in > 0 && nin > 0) {
    if constexpr (PF) {  // one wave of resident blocks
      const long long tiles = (long long)p.nth * q.nrt_in * nin;
      if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
      const int grid = (int)std::min<long long>(tiles, (long long)sm_count() * MINB_IN);
      hoist_interior_pf<T, NV, MINB_IN, VEL><<<grid, blk, 0, s>>>(p, q.zt_lo, q.nrt_in, (int)tiles);
    } else {
      hoist_interior<T, NV, MINB_IN, VEL><<<dim3(p.nth, q.nrt_in, nin), blk, 0, s>>>(p, q.zt_lo);
    }
  }
  const long long nedge = (long long)(q.nrt - q.nrt_in) * q.enzt + (long long)q.nrt_in * (q.ez_lo + q.enzt - q.ez_hi);
  if (nedge > 65535 || p.nth > 65535) return cudaErrorInvalidValue;
  if (nedge > 0) {
    if constexpr (PFE) {
      const long long tiles = (long long)p.nth * nedge;
      const int grid = (int)std::min<long long>(tiles, (long long)sm_count() * MINB_E);
      hoist_edge_pf<T, NVE, MINB_E, VEL><<<grid, blk, 0, s>>>(p, q, (int)tiles);
    } else {
      hoist_edge<T, NVE, MINB_E, VEL><<<dim3(p.nth, (unsigned)nedge), blk, 0, s>>>(p, q);
    }
  }
  return cudaGetLastError();
}

// three-way split half step: interior (plain or prefetching), radial tiles
// (NVE cells per thread, MINB_R blocks per SM), z-end tiles (NVE, MINB_E)
template <typename T, int NV, int MINB_IN, bool PF, int NVE, int MINB_R, int MINB_E, bool VEL>
cudaError_t launch_split3_half(const KParams &p, const Split2 &q, cudaStream_t s) {
  dim3 blk(HB_X, HB_Y);
  const int nin = q.zt_hi - q.zt_lo;
  if (q.nrt_in > 0 && nin > 0) {
    if constexpr (PF) {
      const long long tiles = (long long)p.nth * q.nrt_in * nin;
      if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
      const int grid = (int)std::min<long long>(tiles, (long long)sm_count() * MINB_IN);
      hoist_interior_pf<T, NV, MINB_IN, VEL><<<grid, blk, 0, s>>>(p, q.zt_lo, q.nrt_in, (int)tiles);
    } else {
      hoist_interior<T, NV, MINB_IN, VEL><<<dim3(p.nth, q.nrt_in, nin), blk, 0, s>>>(p, q.zt_lo);
    }
  }
  const long long rad = (long long)p.nth * (q.nrt - q.nrt_in) * (q.ez_hi - q.ez_lo);
  const long long ends = (long long)p.nth * q.nrt * (q.ez_lo + q.enzt - q.ez_hi);
  if (rad > 0x7fffffffLL || ends > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (rad > 0)
    hoist_radial_pf<T, NVE, MINB_R, VEL>
        <<<(int)std::min<long long>(rad, (long long)sm_count() * MINB_R), blk, 0, s>>>(p, q, (int)rad);
  if (ends > 0)
    hoist_ends_pf<T, NVE, MINB_E, VEL>
        <<<(int)std::min<long long>(ends, (long long)sm_count() * MINB_E), blk, 0, s>>>(p, q, (int)ends);
  return cudaGetLastError();
}

template <typename T, int NV, int MINB_IN, bool PF, int NVE, int MINB_R, int MINB_E>
cudaError_t launch_split3_t(const KParams &p, cudaStream_t s, cudaEvent_t *ev, int parts) {
  const Split2 q = split2<NV, NVE>(p);
  cudaError_t e = cudaSuccess;
  if (parts & 1) {
    if (ev) cudaEventRecord(ev[0], s);
    e = launch_split3_half<T, NV, MINB_IN, PF, NVE, MINB_R, MINB_E, true>(p, q, s);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], s);
  }
  if (parts & 2) {
    e = launch_split3_half<T, NV, MINB_IN, PF, NVE, MINB_R, MINB_E, false>(p, q, s);
    if (ev) cudaEventRecord(ev[2], s);
  }
  return e;
}

template <typename T, int NV, int MINB_IN, int NVE, int MINB_E, bool PF = false, bool PFE = false>
cudaError_t launch_split2_t(const KParams &p, cudaStream_t s, cudaEvent_t *ev, int parts) {
  const Split2 q = split2<NV, NVE>(p);
  if (q.zt_hi - q.zt_lo > 65535) return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
  if (parts & 1) {
    if (ev) cudaEventRecord(ev[0], s);
    e = launch_split2_half<T, NV, MINB_IN, NVE, MINB_E, true, PF, PFE>(p, q, s);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], s);
  }
  if (parts & 2) {
    e = launch_split2_half<T, NV, MINB_IN, NVE, MINB_E, false, PF, PFE>(p, q, s);
    if (ev) cudaEventRecord(ev[2], s);
  }
  return e;
}

template <typename T, int NV, int MINB, bool ZF>
cudaError_t launch_hoist_t(const KParams &p, cudaStream_t s, cudaEvent_t *ev, int parts) {
  dim3 blk(HB_X, HB_Y);
  const int nzt = (p.NZ + NV * HB_X - 1) / (NV * HB_X), nrt = (p.NR + HB_Y - 1) / HB_Y;
  if (nzt > 65535 || p.nth > 65535) return cudaErrorInvalidValue;
  dim3 grd = ZF ? dim3(nzt, nrt, p.nth) : dim3(p.nth, nrt, nzt);
  if (parts & 1) {
    if (ev) cudaEventRecord(ev[0], s);
    vel_hoist<T, NV, MINB, ZF><<<grd, blk, 0, s>>>(p);
    if (ev) cudaEventRecord(ev[1], s);
  }
  if (parts & 2) {
    str_hoist<T, NV, MINB, ZF><<<grd, blk, 0, s>>>(p);
    if (ev) cudaEventRecord(ev[2], s);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_hoist_st(int nv, int minb, bool zf, bool split, int edge, const KParams &p, cudaStream_t s,
                            cudaEvent_t *ev, int parts, bool split3 = false) {
  if (split3) {  // interior b = 5 plain, 4 prefetching; c = radial / ends configuration
    switch (edge * 10 + minb) {
      case 4: return launch_split3_t<T, 4, 4, true, 4, 4, 3>(p, s, ev, parts);
      case 5: return launch_split3_t<T, 4, 5, false, 4, 4, 3>(p, s, ev, parts);
      case 14: return launch_split3_t<T, 4, 4, true, 2, 5, 4>(p, s, ev, parts);
      case 15: return launch_split3_t<T, 4, 5, false, 2, 5, 4>(p, s, ev, parts);
      case 24: return launch_split3_t<T, 4, 4, true, 2, 4, 4>(p, s, ev, parts);
      case 25: return launch_split3_t<T, 4, 5, false, 2, 4, 4>(p, s, ev, parts);
      case 34: return launch_split3_t<T, 4, 4, true, 4, 3, 3>(p, s, ev, parts);
      case 35: return launch_split3_t<T, 4, 5, false, 4, 3, 3>(p, s, ev, parts);
    }
    return cudaErrorInvalidValue;
  }
  if (split) {  // interior kernel for minb blocks per SM; edge kernel config c (cells per thread, blocks per SM)
    switch (edge * 10 + minb) {
      case 4: return launch_split2_t<T, 4, 4, 4, 4>(p, s, ev, parts);
      case 5: return launch_split2_t<T, 4, 5, 4, 4>(p, s, ev, parts);
      case 16: return launch_split2_t<T, 2, 6, 2, 6>(p, s, ev, parts);
      case 18: return launch_split2_t<T, 2, 8, 2, 6>(p, s, ev, parts);
      case 24: return launch_split2_t<T, 4, 4, 2, 4>(p, s, ev, parts);
      case 25: return launch_split2_t<T, 4, 5, 2, 4>(p, s, ev, parts);
      case 34: return launch_split2_t<T, 4, 4, 2, 6>(p, s, ev, parts);
      case 35: return launch_split2_t<T, 4, 5, 2, 6>(p, s, ev, parts);
      case 44: return launch_split2_t<T, 4, 4, 4, 3>(p, s, ev, parts);
      case 45: return launch_split2_t<T, 4, 5, 4, 3>(p, s, ev, parts);
      case 56: return launch_split2_t<T, 2, 6, 2, 4>(p, s, ev, parts);
      case 58: return launch_split2_t<T, 2, 8, 2, 4>(p, s, ev, parts);
      case 64: return launch_split2_t<T, 4, 4, 2, 4, true>(p, s, ev, parts);
      case 65: return launch_split2_t<T, 4, 5, 2, 4, true>(p, s, ev, parts);
      case 74: return launch_split2_t<T, 4, 4, 4, 3, true>(p, s, ev, parts);
      case 75: return launch_split2_t<T, 4, 5, 4, 3, true>(p, s, ev, parts);
      case 84: return launch_split2_t<T, 4, 4, 4, 3, false, true>(p, s, ev, parts);
      case 85: return launch_split2_t<T, 4, 5, 4, 3, false, true>(p, s, ev, parts);
      case 94: return launch_split2_t<T, 4, 4, 2, 4, true, true>(p, s, ev, parts);
      case 95: return launch_split2_t<T, 4, 5, 2, 4, true, true>(p, s, ev, parts);
    }
    return cudaErrorInvalidValue;
  }
  if (nv == 2) {
    switch (minb) {
      case 6: return launch_hoist_t<T, 2, 6, false>(p, s, ev, parts);
      case 8: return launch_hoist_t<T, 2, 8, false>(p, s, ev, parts);
    }
    return cudaErrorInvalidValue;
  }
  switch (minb * 2 + (zf ? 1 : 0)) {
    case 6: return launch_hoist_t<T, 4, 3, false>(p, s, ev, parts);
    case 7: return launch_hoist_t<T, 4, 3, true>(p, s, ev, parts);
    case 8: return launch_hoist_t<T, 4, 4, false>(p, s, ev, parts);
    case 9: return launch_hoist_t<T, 4, 4, true>(p, s, ev, parts);
    case 10: return launch_hoist_t<T, 4, 5, false>(p, s, ev, parts);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

long long split_items(int nth, int NR, int NZ) {  // bound on the items of either list: two-cell tiles
  return (long long)nth * ((NR + HB_Y - 1) / HB_Y) * ((NZ + 2 * HB_X - 1) / (2 * HB_X));
}

cudaError_t launch_batch_split(int storage, bool vel, const KParams *cases, int n_cases, int grid, cudaStream_t s) {
  if (grid < 1 || n_cases < 1) return cudaErrorInvalidValue;
  switch (storage * 2 + (vel ? 1 : 0)) {
    case 0: return launch_batch_t<float, false>(cases, n_cases, grid, s);
    case 1: return launch_batch_t<float, true>(cases, n_cases, grid, s);
    case 2: return launch_batch_t<__nv_bfloat16, false>(cases, n_cases, grid, s);
    case 3: return launch_batch_t<__nv_bfloat16, true>(cases, n_cases, grid, s);
    case 4: return launch_batch_t<__half, false>(cases, n_cases, grid, s);
    case 5: return launch_batch_t<__half, true>(cases, n_cases, grid, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_hoist(int storage, int code, const KParams &p, cudaStream_t s, cudaEvent_t *ev, int parts) {
  const int minb = hoist_blocks(code), nv = hoist_cells_per_thread(code);
  const bool zf = hoist_zfast(code), split = hoist_split(code), split3 = (code / 100) % 10 == 3;
  const int edge = (code / 10) % 10;
  switch (storage) {
    case 0: return launch_hoist_st<float>(nv, minb, zf, split, edge, p, s, ev, parts, split3);
    case 1: return launch_hoist_st<__nv_bfloat16>(nv, minb, zf, split, edge, p, s, ev, parts, split3);
    case 2: return launch_hoist_st<__half>(nv, minb, zf, split, edge, p, s, ev, parts, split3);
  }
  return cudaErrorInvalidValue;
}

}  // namespace cwell
