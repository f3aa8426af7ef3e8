// Marching split path: the velocity and the stress kernels of stencil_split.cu
// (same arithmetic, same in-place update, one launch each per leapfrog step),
// with the fields a kernel reads staged in shared memory by TMA.
//
// A block owns an (RT x 128) tile of (r, z) and marches a run of NJ theta
// planes.  Each plane of the fields it reads (six stresses and the material
// IDs for the velocity kernel, three velocities and the IDs for the stress
// kernel) arrives as one (RT + 2) x (128 + 2 HX) box per field, halo row and
// 16-byte halo column on each side, in a ring of four slots.  Planes j - 1,
// j and j + 1 are resident while plane j is updated and plane j + 2 is in
// flight, so every plane of a field is fetched once per block, and the
// theta differences read the neighbouring slots.
//
// Warp roles: warps 0 .. RT-1 compute, warp w owning tile row w; lane l owns
// the four z cells k0 + 4 l .. k0 + 4 l + 3 (16-byte shared loads; the z
// neighbours outside the quad are single loads from the halo).  Warp RT
// issues the TMA copies.  Slot hand-off uses two mbarriers per slot: `full`
// (TMA bytes landed) and `empty` (every compute warp has finished with the
// plane).  The fields a kernel updates (v for the velocity kernel, the six
// stresses for the stress kernel) are read with 16-byte global loads one
// plane ahead and written back with 16-byte stores.  Every wait is bounded:
// a wait that gives up sets bit 1 of the status word, the block stops
// computing, waits (bounded) for the copies it issued and returns.
#include "tma_util.cuh"

namespace cwell {
namespace {

constexpr int MZT = 128;  // z cells per tile: 32 quads, one warp per tile row
constexpr int MNS = 4;    // ring slots

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <typename T>
__device__ __forceinline__ float4 ld4s(const T *p);
template <>
__device__ __forceinline__ float4 ld4s<float>(const float *p) { return *reinterpret_cast<const float4 *>(p); }
template <>
__device__ __forceinline__ float4 ld4s<__nv_bfloat16>(const __nv_bfloat16 *p) {
  const uint2 u = *reinterpret_cast<const uint2 *>(p);
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}
template <>
__device__ __forceinline__ float4 ld4s<__half>(const __half *p) {
  const uint2 u = *reinterpret_cast<const uint2 *>(p);
  const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ void ids4s(const uint16_t *p, int (&o)[4]) {
  const uint2 u = *reinterpret_cast<const uint2 *>(p);
  o[0] = u.x & 0xffff;
  o[1] = u.x >> 16;
  o[2] = u.y & 0xffff;
  o[3] = u.y >> 16;
}

__device__ __forceinline__ void to4(float *a, float4 v) {  // a[0 .. 3]
  a[0] = v.x;
  a[1] = v.y;
  a[2] = v.z;
  a[3] = v.w;
}

template <typename T, int RT, bool VEL>
struct MSmem {
  static constexpr int HX = Pad<T>::HX;
  static constexpr int BR = RT + 2;
  static constexpr int BW = MZT + 2 * HX;
  static constexpr int BWI = MZT + 16;
  static constexpr int NFLD = VEL ? 6 : 3;
  static constexpr int BOXB = (BR * BW * (int)sizeof(T) + 127) / 128 * 128;
  static constexpr int IDB = (BR * BWI * 2 + 127) / 128 * 128;
  static constexpr int SLOT = NFLD * BOXB + IDB;
  static constexpr size_t BAR_OFF = (size_t)MNS * SLOT;
  static constexpr size_t BYTES = BAR_OFF + 2 * MNS * 8 + 128;  // + base alignment slack
  static constexpr uint32_t TX = (uint32_t)(NFLD * BR * BW * sizeof(T) + BR * BWI * 2);
  static constexpr int NT = 32 * (RT + 1);
};

// velocity half-step of the quad (row r of the box, column x) of plane j:
// stresses and IDs of planes j - 1, j, j + 1 in slots sm1, s0, sp1
template <typename T, int RT>
__device__ __forceinline__ void vel_quad(const KParams &p, const unsigned char *ring, int sm1, int s0, int sp1,
                                         int r, int x, int xi, int i, int j, int kq, float4 (&v)[3]) {
  using SM = MSmem<T, RT, true>;
  constexpr int BW = SM::BW, BWI = SM::BWI;
  auto F = [&](int s, int f) { return reinterpret_cast<const T *>(ring + (size_t)s * SM::SLOT + (size_t)f * SM::BOXB); };
  auto I = [&](int s) { return reinterpret_cast<const uint16_t *>(ring + (size_t)s * SM::SLOT + 6 * SM::BOXB); };
  const int NR = p.NR, NZ = p.NZ, pz = p.pml_z;
  const long long NZp = p.NZp;
  const float dtv = p.dtv, idr = p.inv_dr, idz = p.inv_dz, idth = p.inv_dth;
  const int o = r * BW + x, oi = r * BWI + xi;
  // slot fields: 0 s_rr, 1 s_pp, 2 s_zz, 3 s_rp, 4 s_pz, 5 s_rz
  float srr[4], spp[4], srp[4], srz[4], spz[4], szz[5];
  to4(srr, ld4s(F(s0, 0) + o));
  to4(spp, ld4s(F(s0, 1) + o));
  to4(srp, ld4s(F(s0, 3) + o));
  to4(srz, ld4s(F(s0, 5) + o));
  to4(spz, ld4s(F(s0, 4) + o));
  to4(szz, ld4s(F(s0, 2) + o));
  szz[4] = sld(F(s0, 2) + o + 4);
  const float srz_km = sld(F(s0, 5) + o - 1), spz_km = sld(F(s0, 4) + o - 1);
  int idc[4], idj[4];
  ids4s(I(s0) + oi, idc);
  ids4s(I(sp1) + oi, idj);
  const int id_k4 = I(s0)[oi + 4];
  float rho_c[5];
#pragma unroll
  for (int e = 0; e < 4; e++) rho_c[e] = __ldg(p.m_rho + idc[e]);
  rho_c[4] = __ldg(p.m_rho + id_k4);

  const bool rp = i >= p.nr;
  const long long cr = rp ? ((long long)j * p.pml_r + (i - p.nr)) * NZp + kq : 0;
  const float inv_ri = __ldg(p.inv_ri + i), inv_rh = __ldg(p.inv_rh + i);
  const float4 abr = __ldg(p.ab_r + i), abq = __ldg(p.ab_q + i);
  const long long czrow = ((long long)j * NR + i) * (2 * pz);
  const bool zl = pz > 0 && (kq < pz || kq + 3 >= NZ - pz);

  // ---- v_r at (r_i, theta_j, z_k), i >= 1
  if (i >= 1) {
    float srr_m[4], spp_m[4], srp_jm[4];
    to4(srr_m, ld4s(F(s0, 0) + o - BW));
    to4(spp_m, ld4s(F(s0, 1) + o - BW));
    to4(srp_jm, ld4s(F(sm1, 3) + o));
    int idm[4];
    ids4s(I(s0) + oi - BWI, idm);
    float out[4];
    to4(out, v[0]);
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int k = kq + e;
      if (k >= NZ) break;
      float Dr = (srr[e] - srr_m[e]) * idr;
      float Q = (0.5f * (srr[e] + srr_m[e]) - 0.5f * (spp[e] + spp_m[e]) + (srp[e] - srp_jm[e]) * idth) * inv_ri;
      float Dz = (srz[e] - (e ? srz[e - 1] : srz_km)) * idz;
      if (rp) {
        Dr = stretch(p.psr[R_VR] + cr + e, abr.x, abr.y, Dr);
        Q = stretch(p.psr[Q_VR] + cr + e, abq.x, abq.y, Q);
      }
      if (zl && (k < pz || k >= NZ - pz)) {
        const int kz = k < pz ? k : k - (NZ - 2 * pz);
        const float4 abz = __ldg(p.ab_z + k);
        Dz = stretch(p.psz[Z_VR] + czrow + kz, abz.x, abz.y, Dz);
      }
      out[e] += vel_coef(dtv, __ldg(p.m_rho + idm[e]) + rho_c[e]) * (Dr + Q + Dz);
    }
    v[0] = make_float4(out[0], out[1], out[2], out[3]);
  }
  // ---- v_phi at (r_{i+1/2}, theta_{j+1/2}, z_k)
  {
    float srp_ip[4], spp_jp[4];
    to4(srp_ip, ld4s(F(s0, 3) + o + BW));  // zero beyond the last row (TMA fill)
    to4(spp_jp, ld4s(F(sp1, 1) + o));
    float out[4];
    to4(out, v[1]);
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int k = kq + e;
      if (k >= NZ) break;
      float Dr = (srp_ip[e] - srp[e]) * idr;
      float Q = ((srp_ip[e] + srp[e]) + (spp_jp[e] - spp[e]) * idth) * inv_rh;
      float Dz = (spz[e] - (e ? spz[e - 1] : spz_km)) * idz;
      if (rp) {
        Dr = stretch(p.psr[R_VP] + cr + e, abr.z, abr.w, Dr);
        Q = stretch(p.psr[Q_VP] + cr + e, abq.z, abq.w, Q);
      }
      if (zl && (k < pz || k >= NZ - pz)) {
        const int kz = k < pz ? k : k - (NZ - 2 * pz);
        const float4 abz = __ldg(p.ab_z + k);
        Dz = stretch(p.psz[Z_VP] + czrow + kz, abz.x, abz.y, Dz);
      }
      out[e] += vel_coef(dtv, rho_c[e] + __ldg(p.m_rho + idj[e])) * (Dr + Q + Dz);
    }
    v[1] = make_float4(out[0], out[1], out[2], out[3]);
  }
  // ---- v_z at (r_{i+1/2}, theta_j, z_{k+1/2}), k + 1 < NZ
  {
    float srz_ip[4], spz_jm[4];
    to4(srz_ip, ld4s(F(s0, 5) + o + BW));
    to4(spz_jm, ld4s(F(sm1, 4) + o));
    float out[4];
    to4(out, v[2]);
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int k = kq + e;
      if (k + 1 >= NZ) break;
      float Dr = (srz_ip[e] - srz[e]) * idr;
      float Q = (0.5f * (srz_ip[e] + srz[e]) + (spz[e] - spz_jm[e]) * idth) * inv_rh;
      float Dz = (szz[e + 1] - szz[e]) * idz;
      if (rp) {
        Dr = stretch(p.psr[R_VZ] + cr + e, abr.z, abr.w, Dr);
        Q = stretch(p.psr[Q_VZ] + cr + e, abq.z, abq.w, Q);
      }
      if (zl && (k < pz || k >= NZ - pz)) {
        const int kz = k < pz ? k : k - (NZ - 2 * pz);
        const float4 abz = __ldg(p.ab_z + k);
        Dz = stretch(p.psz[Z_VZ] + czrow + kz, abz.z, abz.w, Dz);
      }
      out[e] += vel_coef(dtv, rho_c[e] + rho_c[e + 1]) * (Dr + Q + Dz);
    }
    v[2] = make_float4(out[0], out[1], out[2], out[3]);
  }
  (void)NR;
}

// stress step of the quad of plane j: velocities and IDs of planes j - 1, j,
// j + 1 in slots sm1, s0, sp1; s = {s_rr, s_pp, s_zz, s_rp, s_pz, s_rz}
template <typename T, int RT>
__device__ __forceinline__ void str_quad(const KParams &p, const unsigned char *ring, int sm1, int s0, int sp1, int r,
                                         int x, int xi, int i, int j, int kq, float4 (&s)[6]) {
  using SM = MSmem<T, RT, false>;
  constexpr int BW = SM::BW, BWI = SM::BWI;
  auto F = [&](int sl, int f) { return reinterpret_cast<const T *>(ring + (size_t)sl * SM::SLOT + (size_t)f * SM::BOXB); };
  auto I = [&](int sl) { return reinterpret_cast<const uint16_t *>(ring + (size_t)sl * SM::SLOT + 3 * SM::BOXB); };
  const int NR = p.NR, NZ = p.NZ, pz = p.pml_z;
  const long long NZp = p.NZp;
  const float dts = p.dts, idr = p.inv_dr, idz = p.inv_dz, idth = p.inv_dth;
  const int o = r * BW + x, oi = r * BWI + xi;
  // slot fields: 0 v_r, 1 v_phi, 2 v_z
  float vr[5], vp[5], vz[4];
  to4(vr, ld4s(F(s0, 0) + o));
  vr[4] = sld(F(s0, 0) + o + 4);
  to4(vp, ld4s(F(s0, 1) + o));
  vp[4] = sld(F(s0, 1) + o + 4);
  to4(vz, ld4s(F(s0, 2) + o));
  const float vz_km = sld(F(s0, 2) + o - 1);
  int idc[5], idj[5];
  {
    int t[4];
    ids4s(I(s0) + oi, t);
    idc[0] = t[0]; idc[1] = t[1]; idc[2] = t[2]; idc[3] = t[3];
    idc[4] = I(s0)[oi + 4];
    ids4s(I(sp1) + oi, t);
    idj[0] = t[0]; idj[1] = t[1]; idj[2] = t[2]; idj[3] = t[3];
    idj[4] = I(sp1)[oi + 4];
  }
  float imu_c[5], imu_j[5];
#pragma unroll
  for (int e = 0; e < 5; e++) {
    imu_c[e] = __ldg(p.m_imu + idc[e]);
    imu_j[e] = __ldg(p.m_imu + idj[e]);
  }
  const bool rp = i >= p.nr;
  const long long cr = rp ? ((long long)j * p.pml_r + (i - p.nr)) * NZp + kq : 0;
  const float inv_ri = __ldg(p.inv_ri + i), inv_rh = __ldg(p.inv_rh + i);
  const float4 abr = __ldg(p.ab_r + i), abq = __ldg(p.ab_q + i);
  const long long czrow = ((long long)j * NR + i) * (2 * pz);
  const bool zl = pz > 0 && (kq < pz || kq + 3 >= NZ - pz);
  float src[4] = {0.f, 0.f, 0.f, 0.f};
  if (i == p.src_i && (p.src_j < 0 || p.src_j == j) && p.src_k >= kq && p.src_k < kq + 4) {
    const int n = *p.step;
    src[p.src_k - kq] = n < p.n_wav ? __ldg(p.wav + n) : 0.f;
  }

  // ---- normal stresses at the cell centre
  {
    float vr_ip[4], vp_jm[4];
    to4(vr_ip, ld4s(F(s0, 0) + o + BW));  // zero beyond the last row (TMA fill)
    to4(vp_jm, ld4s(F(sm1, 1) + o));
    float orr[4], opp[4], ozz[4];
    to4(orr, s[0]);
    to4(opp, s[1]);
    to4(ozz, s[2]);
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int k = kq + e;
      if (k >= NZ) break;
      float err = (vr_ip[e] - vr[e]) * idr;
      float epp = ((vp[e] - vp_jm[e]) * idth + 0.5f * (vr[e] + vr_ip[e])) * inv_rh;
      float ezz = (vz[e] - (e ? vz[e - 1] : vz_km)) * idz;
      if (rp) {
        err = stretch(p.psr[R_ERR] + cr + e, abr.z, abr.w, err);
        epp = stretch(p.psr[Q_EPP] + cr + e, abq.z, abq.w, epp);
      }
      if (zl && (k < pz || k >= NZ - pz)) {
        const int kz = k < pz ? k : k - (NZ - 2 * pz);
        const float4 abz = __ldg(p.ab_z + k);
        ezz = stretch(p.psz[Z_EZZ] + czrow + kz, abz.x, abz.y, ezz);
      }
      const float2 lm = __ldg(p.m_lam + idc[e]);  // {lambda, lambda + 2 mu}
      orr[e] += dts * (lm.y * err + lm.x * (epp + ezz)) + src[e];
      opp[e] += dts * (lm.y * epp + lm.x * (err + ezz)) + src[e];
      ozz[e] += dts * (lm.y * ezz + lm.x * (err + epp)) + src[e];
    }
    s[0] = make_float4(orr[0], orr[1], orr[2], orr[3]);
    s[1] = make_float4(opp[0], opp[1], opp[2], opp[3]);
    s[2] = make_float4(ozz[0], ozz[1], ozz[2], ozz[3]);
  }
  if (i >= 1) {
    int idm[5], idjm[4];
    {
      int t[4];
      ids4s(I(s0) + oi - BWI, t);
      idm[0] = t[0]; idm[1] = t[1]; idm[2] = t[2]; idm[3] = t[3];
      idm[4] = I(s0)[oi - BWI + 4];
      ids4s(I(sp1) + oi - BWI, idjm);
    }
    float vp_im[4], vz_im[4];
    to4(vp_im, ld4s(F(s0, 1) + o - BW));
    to4(vz_im, ld4s(F(s0, 2) + o - BW));
    // ---- s_rphi at (r_i, theta_{j+1/2}, z_k)
    {
      float vr_jp[4];
      to4(vr_jp, ld4s(F(sp1, 0) + o));
      float out[4];
      to4(out, s[3]);
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const int k = kq + e;
        if (k >= NZ) break;
        float gr = (vp[e] - vp_im[e]) * idr;
        float Q = ((vr_jp[e] - vr[e]) * idth - 0.5f * (vp[e] + vp_im[e])) * inv_ri;
        if (rp) {
          gr = stretch(p.psr[R_GRP] + cr + e, abr.x, abr.y, gr);
          Q = stretch(p.psr[Q_GRP] + cr + e, abq.x, abq.y, Q);
        }
        const float mu = mu_harm(__ldg(p.m_imu + idm[e]) + imu_c[e] + __ldg(p.m_imu + idjm[e]) + imu_j[e]);
        out[e] += dts * mu * (gr + Q);
      }
      s[3] = make_float4(out[0], out[1], out[2], out[3]);
    }
    // ---- s_rz at (r_i, theta_j, z_{k+1/2})
    {
      float out[4];
      to4(out, s[5]);
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const int k = kq + e;
        if (k + 1 >= NZ) break;
        float gz = (vr[e + 1] - vr[e]) * idz;
        float gr = (vz[e] - vz_im[e]) * idr;
        if (zl && (k < pz || k >= NZ - pz)) {
          const int kz = k < pz ? k : k - (NZ - 2 * pz);
          const float4 abz = __ldg(p.ab_z + k);
          gz = stretch(p.psz[Z_GRZ] + czrow + kz, abz.z, abz.w, gz);
        }
        if (rp) gr = stretch(p.psr[R_GRZ] + cr + e, abr.x, abr.y, gr);
        const float mu =
            mu_harm(__ldg(p.m_imu + idm[e]) + imu_c[e] + __ldg(p.m_imu + idm[e + 1]) + imu_c[e + 1]);
        out[e] += dts * mu * (gz + gr);
      }
      s[5] = make_float4(out[0], out[1], out[2], out[3]);
    }
  }
  // ---- s_phiz at (r_{i+1/2}, theta_{j+1/2}, z_{k+1/2})
  {
    float vz_jp[4];
    to4(vz_jp, ld4s(F(sp1, 2) + o));
    float out[4];
    to4(out, s[4]);
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int k = kq + e;
      if (k + 1 >= NZ) break;
      float Q = (vz_jp[e] - vz[e]) * idth * inv_rh;
      float gz = (vp[e + 1] - vp[e]) * idz;
      if (rp) Q = stretch(p.psr[Q_GPZ] + cr + e, abq.z, abq.w, Q);
      if (zl && (k < pz || k >= NZ - pz)) {
        const int kz = k < pz ? k : k - (NZ - 2 * pz);
        const float4 abz = __ldg(p.ab_z + k);
        gz = stretch(p.psz[Z_GPZ] + czrow + kz, abz.z, abz.w, gz);
      }
      const float mu = mu_harm(imu_c[e] + imu_j[e] + imu_c[e + 1] + imu_j[e + 1]);
      out[e] += dts * mu * (Q + gz);
    }
    s[4] = make_float4(out[0], out[1], out[2], out[3]);
  }
  (void)NR;
}

// One block's work: tile (rtile, ztile) of (r, z), planes seg * nj .. of one
// well.  VEL: velocity kernel (reads the six stresses, updates v_r, v_phi,
// v_z); otherwise the stress kernel (reads the velocities, updates the six
// stresses).
template <typename T, int RT, bool VEL>
__device__ __forceinline__ void march_block(const FusedMaps &maps, const KParams &p, int nj, int *status, int seg,
                                            int rtile, int ztile) {
  using SM = MSmem<T, RT, VEL>;
  constexpr int NOUT = VEL ? 3 : 6;
  constexpr int F0 = VEL ? F_SRR : F_VR;   // first field staged in the ring
  constexpr int U0 = VEL ? F_VR : F_SRR;   // first field updated
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *ring = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  uint64_t *full = reinterpret_cast<uint64_t *>(ring + SM::BAR_OFF);
  uint64_t *empty = full + MNS;
  __shared__ int s_fail, s_issued;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nth = p.nth, NR = p.NR;
  const int j0 = seg * nj;
  const int np = min(nj, nth - j0);  // planes this block updates (>= 1)
  const int i0 = rtile * RT, k0 = ztile * MZT;
  const int nq = np + 2;             // planes loaded: j0 - 1 .. j0 + np

  if (threadIdx.x == 0) {
    for (int s = 0; s < MNS; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], RT);
    }
    s_fail = 0;
    s_issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == RT) {
    // ---------------- producer: one lane issues the copies
    if (lane == 0) {
      int q = 0;
      for (; q < nq; q++) {
        const int s = q % MNS;
        if (q >= MNS && !mbar_wait(&empty[s], (uint32_t)((q / MNS) - 1) & 1u)) {
          s_fail = 1;
          break;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const int plane = (j0 - 1 + q + nth) % nth;
        unsigned char *dst = ring + (size_t)s * SM::SLOT;
        mbar_expect_tx(&full[s], SM::TX);
#pragma unroll
        for (int f = 0; f < SM::NFLD; f++)
          tma_load_4d(dst + f * SM::BOXB, &maps.f[F0 + f], k0 - SM::HX, i0 - 1, plane, 0, &full[s]);
        tma_load_4d(dst + SM::NFLD * SM::BOXB, &maps.id, k0 - 8, i0 - 1, plane, 0, &full[s]);
      }
      s_issued = q;
    }
  } else {
    // ---------------- compute warps
    const int r = warp + 1, i = i0 + warp;
    const int kq = k0 + 4 * lane;
    const bool live = i < NR && kq < p.NZp;  // whole quad inside the padded row (NZp is a multiple of 32)
    const int x = SM::HX + 4 * lane, xi = 8 + 4 * lane;
    const long long pl = p.plane, cb = (long long)i * p.NZp + kq;
    T *u[NOUT];  // the updated fields, in the order of vel_quad / str_quad
#pragma unroll
    for (int c = 0; c < NOUT; c++) u[c] = (T *)p.f[U0 + c];
    float4 cur[NOUT], nxt[NOUT];
    auto load = [&](int t, float4 (&d)[NOUT]) {
      const long long cg = (long long)(j0 + t) * pl + cb;
#pragma unroll
      for (int c = 0; c < NOUT; c++) d[c] = live ? St<T>::ld4(u[c] + cg) : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    load(0, cur);
    int waited = 0;
    bool ok = true;
    for (int t = 0; t < np; t++) {
      if (t + 1 < np) load(t + 1, nxt);
      while (ok && waited < t + 3) {
        if (mbar_wait(&full[waited % MNS], (uint32_t)(waited / MNS) & 1u)) waited++;
        else ok = false;
      }
      if (!ok) {
        s_fail = 1;
        break;
      }
      if (live) {
        const int j = j0 + t;
        if constexpr (VEL)
          vel_quad<T, RT>(p, ring, t % MNS, (t + 1) % MNS, (t + 2) % MNS, r, x, xi, i, j, kq, cur);
        else
          str_quad<T, RT>(p, ring, t % MNS, (t + 1) % MNS, (t + 2) % MNS, r, x, xi, i, j, kq, cur);
        const long long cg = (long long)j * pl + cb;
#pragma unroll
        for (int c = 0; c < NOUT; c++) St<T>::st4(u[c] + cg, cur[c]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[t % MNS]);  // plane j - 1 is no longer read
#pragma unroll
      for (int c = 0; c < NOUT; c++) cur[c] = nxt[c];
    }
  }
  __syncthreads();
  if (s_fail && threadIdx.x == 0) {
    // a wait gave up: report, and wait (bounded) for the copies still in flight
    atomicOr(status, 2);
    for (int q = max(0, s_issued - MNS); q < s_issued; q++) mbar_wait(&full[q % MNS], (uint32_t)(q / MNS) & 1u);
  }
  __syncthreads();
}

// one well: grid (theta runs, r tiles, z tiles)
template <typename T, int RT, bool VEL>
__global__ void __launch_bounds__(MSmem<T, RT, VEL>::NT) march_step(const __grid_constant__ FusedMaps maps,
                                                                     const __grid_constant__ KParams p, int nj,
                                                                     int *status) {
  march_block<T, RT, VEL>(maps, p, nj, status, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <typename T, int RT, bool VEL>
cudaError_t launch_march_t(const FusedMaps &maps, const KParams &p, int nj, int *status, cudaStream_t s) {
  using SM = MSmem<T, RT, VEL>;
  auto kern = march_step<T, RT, VEL>;
  static bool attr_done[16] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 16) return cudaErrorInvalidDevice;
  if (!attr_done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::BYTES);
    if (e != cudaSuccess) return e;
    attr_done[dev] = true;
  }
  dim3 grd((p.nth + nj - 1) / nj, (p.NR + RT - 1) / RT, (p.NZ + MZT - 1) / MZT);
  kern<<<grd, SM::NT, SM::BYTES, s>>>(maps, p, nj, status);
  return cudaGetLastError();
}

template <typename T, int RT>
cudaError_t launch_march_rt(const FusedMaps &maps, const KParams &p, int nj, int *status, cudaStream_t s,
                            cudaEvent_t *ev, int parts) {
  cudaError_t e = cudaSuccess;
  if (parts & 1) {
    if (ev) cudaEventRecord(ev[0], s);
    e = launch_march_t<T, RT, true>(maps, p, nj, status, s);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], s);
  }
  if (parts & 2) {
    e = launch_march_t<T, RT, false>(maps, p, nj, status, s);
    if (ev) cudaEventRecord(ev[2], s);
  }
  return e;
}

template <typename T>
cudaError_t launch_march_st(int rt, const FusedMaps &m, const KParams &p, int nj, int *status, cudaStream_t s,
                            cudaEvent_t *ev, int parts) {
  switch (rt) {
    case 2: return launch_march_rt<T, 2>(m, p, nj, status, s, ev, parts);
    case 4: return launch_march_rt<T, 4>(m, p, nj, status, s, ev, parts);
    case 8: return launch_march_rt<T, 8>(m, p, nj, status, s, ev, parts);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
size_t march_bytes_t(int rt) {
  auto mx = [](size_t a, size_t b) { return a > b ? a : b; };
  switch (rt) {
    case 2: return mx(MSmem<T, 2, true>::BYTES, MSmem<T, 2, false>::BYTES);
    case 4: return mx(MSmem<T, 4, true>::BYTES, MSmem<T, 4, false>::BYTES);
    case 8: return mx(MSmem<T, 8, true>::BYTES, MSmem<T, 8, false>::BYTES);
  }
  return 0;
}

}  // namespace

cudaError_t launch_march(int storage, int code, const FusedMaps &maps, const KParams &p, int *status, cudaStream_t s,
                         cudaEvent_t *ev, int parts) {
  const int rt = march_rows(code), nj = march_planes(code);
  if (nj < 1) return cudaErrorInvalidValue;
  switch (storage) {
    case 0: return launch_march_st<float>(rt, maps, p, nj, status, s, ev, parts);
    case 1: return launch_march_st<__nv_bfloat16>(rt, maps, p, nj, status, s, ev, parts);
    case 2: return launch_march_st<__half>(rt, maps, p, nj, status, s, ev, parts);
  }
  return cudaErrorInvalidValue;
}

size_t march_smem_bytes(int storage, int code) {
  const int rt = march_rows(code);
  if (storage == 0) return march_bytes_t<float>(rt);
  if (storage == 1) return march_bytes_t<__nv_bfloat16>(rt);
  return march_bytes_t<__half>(rt);
}

int march_box_x(int storage) { return MZT + 2 * (storage == 0 ? 4 : 8); }
int march_box_id() { return MZT + 16; }

}  // namespace cwell
