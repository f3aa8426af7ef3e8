// Split path, load-first variant: the velocity and stress kernels of
// stencil_split.cu with every global load of a thread issued before any of
// its arithmetic or stores (one round trip to memory per thread instead of
// one per component), and the material lookups from the split tables
// {rho}, {1/mu}, {lambda, lambda + 2 mu}.  Same thread layout (four z cells
// per thread, 16-byte loads, block = 32 quads x 4 rows, theta fastest across
// blocks), same arithmetic, same in-place update.
#include <algorithm>

#include "cwell_internal.cuh"

namespace cwell {
namespace {

constexpr int HB_X = 32;  // z-quads per block
constexpr int HB_Y = 4;   // r rows per block

__device__ __forceinline__ float4 z4() { return make_float4(0.f, 0.f, 0.f, 0.f); }

__device__ __forceinline__ void ids4(uint2 u, int (&o)[4]) {
  o[0] = u.x & 0xffff;
  o[1] = u.x >> 16;
  o[2] = u.y & 0xffff;
  o[3] = u.y >> 16;
}

__device__ __forceinline__ uint2 ldid(const uint16_t *p) { return __ldg(reinterpret_cast<const uint2 *>(p)); }

#define E4(v, e) ((e) == 0 ? (v).x : (e) == 1 ? (v).y : (e) == 2 ? (v).z : (v).w)

// LEAN: the four cells are interior (no PML memory variable, all inside NZ,
// k0 + 4 < NZ); the kernels pick the lean body per thread.
template <typename T, bool LEAN>
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
  const bool im = i >= 1, ip = i + 1 < NR, k4 = LEAN || k0 + 4 < NZ, km = k0 > 0;

  // ---- every load
  const float4 a_srr = St<T>::ld4(srr + c), a_spp = St<T>::ld4(spp + c), a_srp = St<T>::ld4(srp + c);
  const float4 a_srz = St<T>::ld4(srz + c), a_spz = St<T>::ld4(spz + c), a_szz = St<T>::ld4(szz + c);
  const float szz_k4 = k4 ? St<T>::ld1(szz + c + 4) : 0.f;
  const float srz_km = km ? St<T>::ld1(srz + c - 1) : 0.f, spz_km = km ? St<T>::ld1(spz + c - 1) : 0.f;
  const float4 m_srr = im ? St<T>::ld4(srr + c - NZp) : z4(), m_spp = im ? St<T>::ld4(spp + c - NZp) : z4();
  const float4 jm_srp = St<T>::ld4(srp + cjm), jm_spz = St<T>::ld4(spz + cjm);
  const float4 p_srp = ip ? St<T>::ld4(srp + c + NZp) : z4(), p_srz = ip ? St<T>::ld4(srz + c + NZp) : z4();
  const float4 jp_spp = St<T>::ld4(spp + cjp);
  const float4 o_vr = St<T>::ld4(vr + c), o_vp = St<T>::ld4(vp + c), o_vz = St<T>::ld4(vz + c);
  const uint2 u_c = ldid(p.id + c), u_j = ldid(p.id + cjp), u_m = im ? ldid(p.id + c - NZp) : make_uint2(0, 0);
  int id_k4 = 0;
  if (k4) id_k4 = __ldg(p.id + c + 4);
  const bool rp = !LEAN && i >= p.nr;
  const float inv_ri = __ldg(p.inv_ri + i), inv_rh = __ldg(p.inv_rh + i);
  const float4 abr = __ldg(p.ab_r + i), abq = __ldg(p.ab_q + i);

  int idc[4], idj[4], idm[4];
  ids4(u_c, idc);
  ids4(u_j, idj);
  ids4(u_m, idm);
  if (!k4) id_k4 = idc[3];
  float rho_c[5], rho_j[4], rho_m[4];
#pragma unroll
  for (int e = 0; e < 4; e++) {
    rho_c[e] = __ldg(p.m_rho + idc[e]);
    rho_j[e] = __ldg(p.m_rho + idj[e]);
    rho_m[e] = __ldg(p.m_rho + idm[e]);
  }
  rho_c[4] = __ldg(p.m_rho + id_k4);

  const long long cr = rp ? ((long long)j * p.pml_r + (i - p.nr)) * NZp + k0 : 0;
  const float dtv = p.dtv, idr = p.inv_dr, idz = p.inv_dz, idth = p.inv_dth;
  const int pz = p.pml_z;
  const long long czrow = ((long long)j * NR + i) * (2 * pz);
  const bool zl = !LEAN && pz > 0 && (k0 < pz || k0 + 3 >= NZ - pz);

  float out_r[4], out_p[4], out_z[4];
#pragma unroll
  for (int e = 0; e < 4; e++) {
    out_r[e] = E4(o_vr, e);
    out_p[e] = E4(o_vp, e);
    out_z[e] = E4(o_vz, e);
  }
#pragma unroll
  for (int e = 0; e < 4; e++) {
    const int k = k0 + e;
    if (!LEAN && k >= NZ) break;
    const bool zp = zl && (k < pz || k >= NZ - pz);
    const int kz = k < pz ? k : k - (NZ - 2 * pz);
    const float4 abz = zp ? __ldg(p.ab_z + k) : z4();
    const float srr_e = E4(a_srr, e), spp_e = E4(a_spp, e), srp_e = E4(a_srp, e);
    const float srz_e = E4(a_srz, e), spz_e = E4(a_spz, e), szz_e = E4(a_szz, e);
    const float srz_m1 = e ? E4(a_srz, e - 1) : srz_km, spz_m1 = e ? E4(a_spz, e - 1) : spz_km;
    // v_r at (r_i, theta_j, z_k), i >= 1
    if (im) {
      float Dr = (srr_e - E4(m_srr, e)) * idr;
      float Q = (0.5f * (srr_e + E4(m_srr, e)) - 0.5f * (spp_e + E4(m_spp, e)) + (srp_e - E4(jm_srp, e)) * idth) *
                inv_ri;
      float Dz = (srz_e - srz_m1) * idz;
      if (rp) {
        Dr = stretch(p.psr[R_VR] + cr + e, abr.x, abr.y, Dr);
        Q = stretch(p.psr[Q_VR] + cr + e, abq.x, abq.y, Q);
      }
      if (zp) Dz = stretch(p.psz[Z_VR] + czrow + kz, abz.x, abz.y, Dz);
      out_r[e] += vel_coef(dtv, rho_m[e] + rho_c[e]) * (Dr + Q + Dz);
    }
    // v_phi at (r_{i+1/2}, theta_{j+1/2}, z_k)
    {
      const float s1 = E4(p_srp, e);
      float Dr = (s1 - srp_e) * idr;
      float Q = ((s1 + srp_e) + (E4(jp_spp, e) - spp_e) * idth) * inv_rh;
      float Dz = (spz_e - spz_m1) * idz;
      if (rp) {
        Dr = stretch(p.psr[R_VP] + cr + e, abr.z, abr.w, Dr);
        Q = stretch(p.psr[Q_VP] + cr + e, abq.z, abq.w, Q);
      }
      if (zp) Dz = stretch(p.psz[Z_VP] + czrow + kz, abz.x, abz.y, Dz);
      out_p[e] += vel_coef(dtv, rho_c[e] + rho_j[e]) * (Dr + Q + Dz);
    }
    // v_z at (r_{i+1/2}, theta_j, z_{k+1/2}), k + 1 < NZ
    if (LEAN || k + 1 < NZ) {
      const float s1 = E4(p_srz, e);
      float Dr = (s1 - srz_e) * idr;
      float Q = (0.5f * (s1 + srz_e) + (spz_e - E4(jm_spz, e)) * idth) * inv_rh;
      float Dz = ((e < 3 ? E4(a_szz, e + 1) : szz_k4) - szz_e) * idz;
      if (rp) {
        Dr = stretch(p.psr[R_VZ] + cr + e, abr.z, abr.w, Dr);
        Q = stretch(p.psr[Q_VZ] + cr + e, abq.z, abq.w, Q);
      }
      if (zp) Dz = stretch(p.psz[Z_VZ] + czrow + kz, abz.z, abz.w, Dz);
      out_z[e] += vel_coef(dtv, rho_c[e] + rho_c[e + 1]) * (Dr + Q + Dz);
    }
  }
  if (im) St<T>::st4(vr + c, make_float4(out_r[0], out_r[1], out_r[2], out_r[3]));
  St<T>::st4(vp + c, make_float4(out_p[0], out_p[1], out_p[2], out_p[3]));
  St<T>::st4(vz + c, make_float4(out_z[0], out_z[1], out_z[2], out_z[3]));
}

template <typename T, bool LEAN>
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
  const bool im = i >= 1, ip = i + 1 < NR, k4 = LEAN || k0 + 4 < NZ, km = k0 > 0;

  // ---- every load
  const float4 a_vr = St<T>::ld4(vr + c), a_vp = St<T>::ld4(vp + c), a_vz = St<T>::ld4(vz + c);
  const float vr_k4 = k4 ? St<T>::ld1(vr + c + 4) : 0.f, vp_k4 = k4 ? St<T>::ld1(vp + c + 4) : 0.f;
  const float vz_km = km ? St<T>::ld1(vz + c - 1) : 0.f;
  const float4 p_vr = ip ? St<T>::ld4(vr + c + NZp) : z4();
  const float4 jm_vp = St<T>::ld4(vp + cjm);
  const float4 m_vp = im ? St<T>::ld4(vp + c - NZp) : z4(), m_vz = im ? St<T>::ld4(vz + c - NZp) : z4();
  const float4 jp_vr = St<T>::ld4(vr + cjp), jp_vz = St<T>::ld4(vz + cjp);
  const float4 o_rr = St<T>::ld4(srr + c), o_pp = St<T>::ld4(spp + c), o_zz = St<T>::ld4(szz + c);
  const float4 o_rp = St<T>::ld4(srp + c), o_pz = St<T>::ld4(spz + c), o_rz = St<T>::ld4(srz + c);
  const uint2 u_c = ldid(p.id + c), u_j = ldid(p.id + cjp);
  const uint2 u_m = im ? ldid(p.id + c - NZp) : make_uint2(0, 0), u_jm = im ? ldid(p.id + cjp - NZp) : make_uint2(0, 0);
  int idc4 = 0, idj4 = 0, idm4 = 0;
  if (k4) {
    idc4 = __ldg(p.id + c + 4);
    idj4 = __ldg(p.id + cjp + 4);
    if (im) idm4 = __ldg(p.id + c - NZp + 4);
  }
  const bool rp = !LEAN && i >= p.nr;
  const float inv_ri = __ldg(p.inv_ri + i), inv_rh = __ldg(p.inv_rh + i);
  const float4 abr = __ldg(p.ab_r + i), abq = __ldg(p.ab_q + i);
  float src[4] = {0.f, 0.f, 0.f, 0.f};
  if (i == p.src_i && (p.src_j < 0 || p.src_j == j) && p.src_k >= k0 && p.src_k < k0 + 4) {
    const int n = *p.step;
    src[p.src_k - k0] = n < p.n_wav ? __ldg(p.wav + n) : 0.f;
  }

  int idc[4], idj[4], idm[4], idjm[4];
  ids4(u_c, idc);
  ids4(u_j, idj);
  ids4(u_m, idm);
  ids4(u_jm, idjm);
  if (!k4) {
    idc4 = idc[3];
    idj4 = idj[3];
    idm4 = idm[3];
  }
  float imu_c[5], imu_j[5], imu_m[5], imu_jm[4];
  float2 lam[4];
#pragma unroll
  for (int e = 0; e < 4; e++) {
    imu_c[e] = __ldg(p.m_imu + idc[e]);
    imu_j[e] = __ldg(p.m_imu + idj[e]);
    imu_m[e] = __ldg(p.m_imu + idm[e]);
    imu_jm[e] = __ldg(p.m_imu + idjm[e]);
    lam[e] = __ldg(p.m_lam + idc[e]);
  }
  imu_c[4] = __ldg(p.m_imu + idc4);
  imu_j[4] = __ldg(p.m_imu + idj4);
  imu_m[4] = __ldg(p.m_imu + idm4);

  const long long cr = rp ? ((long long)j * p.pml_r + (i - p.nr)) * NZp + k0 : 0;
  const float dts = p.dts, idr = p.inv_dr, idz = p.inv_dz, idth = p.inv_dth;
  const int pz = p.pml_z;
  const long long czrow = ((long long)j * NR + i) * (2 * pz);
  const bool zl = !LEAN && pz > 0 && (k0 < pz || k0 + 3 >= NZ - pz);

  float orr[4], opp[4], ozz[4], orp[4], opz[4], orz[4];
#pragma unroll
  for (int e = 0; e < 4; e++) {
    orr[e] = E4(o_rr, e);
    opp[e] = E4(o_pp, e);
    ozz[e] = E4(o_zz, e);
    orp[e] = E4(o_rp, e);
    opz[e] = E4(o_pz, e);
    orz[e] = E4(o_rz, e);
  }
#pragma unroll
  for (int e = 0; e < 4; e++) {
    const int k = k0 + e;
    if (!LEAN && k >= NZ) break;
    const bool zp = zl && (k < pz || k >= NZ - pz);
    const int kz = k < pz ? k : k - (NZ - 2 * pz);
    const float4 abz = zp ? __ldg(p.ab_z + k) : z4();
    const float vr_e = E4(a_vr, e), vp_e = E4(a_vp, e), vz_e = E4(a_vz, e);
    const float vr_e1 = e < 3 ? E4(a_vr, e + 1) : vr_k4, vp_e1 = e < 3 ? E4(a_vp, e + 1) : vp_k4;
    const float vz_m1 = e ? E4(a_vz, e - 1) : vz_km;
    // normal stresses at the cell centre
    {
      const float vr1 = E4(p_vr, e);
      float err = (vr1 - vr_e) * idr;
      float epp = ((vp_e - E4(jm_vp, e)) * idth + 0.5f * (vr_e + vr1)) * inv_rh;
      float ezz = (vz_e - vz_m1) * idz;
      if (rp) {
        err = stretch(p.psr[R_ERR] + cr + e, abr.z, abr.w, err);
        epp = stretch(p.psr[Q_EPP] + cr + e, abq.z, abq.w, epp);
      }
      if (zp) ezz = stretch(p.psz[Z_EZZ] + czrow + kz, abz.x, abz.y, ezz);
      const float l = lam[e].x, l2m = lam[e].y;
      orr[e] += dts * (l2m * err + l * (epp + ezz)) + src[e];
      opp[e] += dts * (l2m * epp + l * (err + ezz)) + src[e];
      ozz[e] += dts * (l2m * ezz + l * (err + epp)) + src[e];
    }
    if (im) {
      // s_rphi at (r_i, theta_{j+1/2}, z_k)
      {
        float gr = (vp_e - E4(m_vp, e)) * idr;
        float Q = ((E4(jp_vr, e) - vr_e) * idth - 0.5f * (vp_e + E4(m_vp, e))) * inv_ri;
        if (rp) {
          gr = stretch(p.psr[R_GRP] + cr + e, abr.x, abr.y, gr);
          Q = stretch(p.psr[Q_GRP] + cr + e, abq.x, abq.y, Q);
        }
        const float mu = mu_harm(imu_m[e] + imu_c[e] + imu_jm[e] + imu_j[e]);
        orp[e] += dts * mu * (gr + Q);
      }
      // s_rz at (r_i, theta_j, z_{k+1/2})
      if (LEAN || k + 1 < NZ) {
        float gz = (vr_e1 - vr_e) * idz;
        float gr = (vz_e - E4(m_vz, e)) * idr;
        if (zp) gz = stretch(p.psz[Z_GRZ] + czrow + kz, abz.z, abz.w, gz);
        if (rp) gr = stretch(p.psr[R_GRZ] + cr + e, abr.x, abr.y, gr);
        const float mu = mu_harm(imu_m[e] + imu_c[e] + imu_m[e + 1] + imu_c[e + 1]);
        orz[e] += dts * mu * (gz + gr);
      }
    }
    // s_phiz at (r_{i+1/2}, theta_{j+1/2}, z_{k+1/2})
    if (LEAN || k + 1 < NZ) {
      float Q = (E4(jp_vz, e) - vz_e) * idth * inv_rh;
      float gz = (vp_e1 - vp_e) * idz;
      if (rp) Q = stretch(p.psr[Q_GPZ] + cr + e, abq.z, abq.w, Q);
      if (zp) gz = stretch(p.psz[Z_GPZ] + czrow + kz, abz.z, abz.w, gz);
      const float mu = mu_harm(imu_c[e] + imu_j[e] + imu_c[e + 1] + imu_j[e + 1]);
      opz[e] += dts * mu * (Q + gz);
    }
  }
  St<T>::st4(srr + c, make_float4(orr[0], orr[1], orr[2], orr[3]));
  St<T>::st4(spp + c, make_float4(opp[0], opp[1], opp[2], opp[3]));
  St<T>::st4(szz + c, make_float4(ozz[0], ozz[1], ozz[2], ozz[3]));
  if (im) {
    St<T>::st4(srp + c, make_float4(orp[0], orp[1], orp[2], orp[3]));
    St<T>::st4(srz + c, make_float4(orz[0], orz[1], orz[2], orz[3]));
  }
  St<T>::st4(spz + c, make_float4(opz[0], opz[1], opz[2], opz[3]));
}

__device__ __forceinline__ bool lean_quad(const KParams &p, int i, int k0) {
  return i < p.nr && k0 >= p.pml_z && k0 + 4 < p.NZ - p.pml_z;
}

template <typename T, bool VEL>
__device__ __forceinline__ void hoist_quad(const KParams &p, int j, int i, int k0) {
  if (lean_quad(p, i, k0)) {
    if (VEL) vel_hoist_body<T, true>(p, j, i, k0);
    else str_hoist_body<T, true>(p, j, i, k0);
  } else {
    if (VEL) vel_hoist_body<T, false>(p, j, i, k0);
    else str_hoist_body<T, false>(p, j, i, k0);
  }
}

// Block order: ZF = false walks theta fastest (blockIdx.x = theta, y = r tile,
// z = z tile: co-resident blocks share theta-neighbour rows); ZF = true walks
// z fastest (x = z tile, y = r tile, z = theta: co-resident blocks stream
// whole rows, theta neighbours come back from L2).
template <bool ZF>
__device__ __forceinline__ void block_cell(int &j, int &i, int &k0) {
  const int zt = ZF ? blockIdx.x : blockIdx.z;
  j = ZF ? blockIdx.z : blockIdx.x;
  i = blockIdx.y * HB_Y + threadIdx.y;
  k0 = (zt * HB_X + threadIdx.x) * 4;
}

template <typename T, int MINB, bool ZF>
__global__ void __launch_bounds__(HB_X *HB_Y, MINB) vel_hoist(const KParams p) {
  int j, i, k0;
  block_cell<ZF>(j, i, k0);
  if (i < p.NR && k0 < p.NZ) hoist_quad<T, true>(p, j, i, k0);
}

template <typename T, int MINB, bool ZF>
__global__ void __launch_bounds__(HB_X *HB_Y, MINB) str_hoist(const KParams p) {
  int j, i, k0;
  block_cell<ZF>(j, i, k0);
  if (i < p.NR && k0 < p.NZ) hoist_quad<T, false>(p, j, i, k0);
}

// Batched scenarios: the blocks walk the work list of up to BATCH_MAX cases,
// item = (case, theta, r tile, z tile), theta fastest inside a case so that
// the theta neighbours a block reads are read by co-resident blocks too.  The
// cases' parameters and the prefix sum of their items (start[c] = first item
// of case c, start[n] = total) travel in the kernel's parameter space, so a
// block reads its case's geometry and buffers from the constant bank.  The
// index inside a case is 32-bit (checked on the host).
struct BatchParams {
  KParams cases[BATCH_MAX];
  long long start[BATCH_MAX + 1];
  int n;
};
static_assert(sizeof(BatchParams) <= 32000, "batch parameters exceed the kernel parameter space");

template <typename T, bool VEL, int MINB>
__global__ void __launch_bounds__(HB_X *HB_Y, MINB) batch_hoist(const __grid_constant__ BatchParams bp) {
  const long long total = bp.start[bp.n];
  for (long long item = blockIdx.x; item < total; item += gridDim.x) {
    int lo = 0, hi = bp.n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (bp.start[mid] <= item) lo = mid;
      else hi = mid - 1;
    }
    const KParams &p = bp.cases[lo];
    int q = (int)(item - bp.start[lo]);
    const int nth = p.nth, nrt = (p.NR + HB_Y - 1) / HB_Y;
    const int j = q % nth;
    q /= nth;
    const int i = (q % nrt) * HB_Y + threadIdx.y, k0 = ((q / nrt) * HB_X + threadIdx.x) * 4;
    if (i < p.NR && k0 < p.NZ) hoist_quad<T, VEL>(p, j, i, k0);
  }
}

template <typename T, int MINB, bool ZF>
cudaError_t launch_hoist_t(const KParams &p, cudaStream_t s, cudaEvent_t *ev, int parts) {
  dim3 blk(HB_X, HB_Y);
  const int nzt = (p.NZ + 4 * HB_X - 1) / (4 * HB_X), nrt = (p.NR + HB_Y - 1) / HB_Y;
  if (nzt > 65535 || p.nth > 65535) return cudaErrorInvalidValue;
  dim3 grd = ZF ? dim3(nzt, nrt, p.nth) : dim3(p.nth, nrt, nzt);
  if (parts & 1) {
    if (ev) cudaEventRecord(ev[0], s);
    vel_hoist<T, MINB, ZF><<<grd, blk, 0, s>>>(p);
    if (ev) cudaEventRecord(ev[1], s);
  }
  if (parts & 2) {
    str_hoist<T, MINB, ZF><<<grd, blk, 0, s>>>(p);
    if (ev) cudaEventRecord(ev[2], s);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_hoist_st(int minb, bool zf, const KParams &p, cudaStream_t s, cudaEvent_t *ev, int parts) {
  switch (minb * 2 + (zf ? 1 : 0)) {
    case 6: return launch_hoist_t<T, 3, false>(p, s, ev, parts);
    case 7: return launch_hoist_t<T, 3, true>(p, s, ev, parts);
    case 8: return launch_hoist_t<T, 4, false>(p, s, ev, parts);
    case 9: return launch_hoist_t<T, 4, true>(p, s, ev, parts);
    case 10: return launch_hoist_t<T, 5, false>(p, s, ev, parts);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

long long split_items(int nth, int NR, int NZ) {
  return (long long)nth * ((NR + HB_Y - 1) / HB_Y) * ((NZ + 4 * HB_X - 1) / (4 * HB_X));
}

constexpr int BATCH_MINB = 4;  // the load-first bodies at four resident blocks per SM

cudaError_t launch_batch_split(int storage, bool vel, const KParams *cases, const long long *start, int n_cases,
                               int grid, cudaStream_t s) {
  dim3 blk(HB_X, HB_Y);
  if (grid < 1 || n_cases < 1) return cudaErrorInvalidValue;
  static thread_local BatchParams bp;  // large: kept off the stack
  for (int c0 = 0; c0 < n_cases; c0 += BATCH_MAX) {
    const int n = std::min(BATCH_MAX, n_cases - c0);
    bp.n = n;
    for (int c = 0; c < n; c++) {
      bp.cases[c] = cases[c0 + c];
      bp.start[c] = start[c0 + c] - start[c0];
    }
    bp.start[n] = start[c0 + n] - start[c0];
    if (bp.start[n] < 1) continue;
    const int g = (int)std::min<long long>(grid, bp.start[n]);
    switch (storage * 2 + (vel ? 1 : 0)) {
      case 0: batch_hoist<float, false, BATCH_MINB><<<g, blk, 0, s>>>(bp); break;
      case 1: batch_hoist<float, true, BATCH_MINB><<<g, blk, 0, s>>>(bp); break;
      case 2: batch_hoist<__nv_bfloat16, false, BATCH_MINB><<<g, blk, 0, s>>>(bp); break;
      case 3: batch_hoist<__nv_bfloat16, true, BATCH_MINB><<<g, blk, 0, s>>>(bp); break;
      case 4: batch_hoist<__half, false, BATCH_MINB><<<g, blk, 0, s>>>(bp); break;
      case 5: batch_hoist<__half, true, BATCH_MINB><<<g, blk, 0, s>>>(bp); break;
      default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_hoist(int storage, int code, const KParams &p, cudaStream_t s, cudaEvent_t *ev, int parts) {
  const int minb = hoist_blocks(code);
  const bool zf = hoist_zfast(code);
  switch (storage) {
    case 0: return launch_hoist_st<float>(minb, zf, p, s, ev, parts);
    case 1: return launch_hoist_st<__nv_bfloat16>(minb, zf, p, s, ev, parts);
    case 2: return launch_hoist_st<__half>(minb, zf, p, s, ev, parts);
  }
  return cudaErrorInvalidValue;
}

}  // namespace cwell
