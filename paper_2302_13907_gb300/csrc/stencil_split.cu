// Split path: one velocity kernel and one stress kernel per leapfrog step.
//
// Each thread updates four consecutive z cells of one (theta, r) row with
// 16-byte vector loads along z; a warp covers 128 contiguous z values, so
// every global access is a full 128-byte line.  Block = 32 z-quads x 4 r rows;
// blockIdx.x walks theta fastest so that the theta neighbours a block reads
// are the rows its co-resident blocks read too (L2 reuse), then r tiles,
// then z tiles.
//
// Per cell (cylindrical velocity-stress system, Eq. 1; staggering and
// readings as in the header of the C-ABI):
//   v_r   += dt/rho_r   * ( d_r s_rr + [(s_rr - s_pp) + d_th s_rp] / r + d_z s_rz )
//   v_phi += dt/rho_p   * ( d_r s_rp + [2 s_rp + d_th s_pp] / r + d_z s_pz )
//   v_z   += dt/rho_z   * ( d_r s_rz + [s_rz + d_th s_pz] / r + d_z s_zz )
//   e_rr = d_r v_r, e_pp = [d_th v_p + v_r] / r, e_zz = d_z v_z
//   s_ii += dt * ((lambda + 2 mu) e_ii + lambda (e_jj + e_kk))
//   s_rp += dt * mu_rp * ( d_r v_p + [d_th v_r - v_p] / r )
//   s_rz += dt * mu_rz * ( d_r v_z + d_z v_r )
//   s_pz += dt * mu_pz * ( [d_th v_z] / r + d_z v_p )
// with two-cell density means and four-cell harmonic shear moduli; radial
// differences, 1/r groups and z differences are stretched by convolutional
// PML memory variables inside the layers.
#include "cwell_internal.cuh"

namespace cwell {

constexpr int SB_X = 32;  // z-quads per block
constexpr int SB_Y = 4;   // r rows per block
constexpr int SB_MINB = 6;  // resident blocks per SM asked of the register allocator

// velocity half-step of the four z cells k0 .. k0+3 of row (j, i)
template <typename T>
__device__ __forceinline__ void vel_body(const KParams &p, const int j, const int i, const int k0) {
  const int nth = p.nth, NR = p.NR, NZ = p.NZ;
  const long long NZp = p.NZp, pl = p.plane;
  const int jm = j == 0 ? nth - 1 : j - 1, jp = j == nth - 1 ? 0 : j + 1;
  const long long c = (long long)j * pl + i * NZp + k0;
  const long long cjm = (long long)jm * pl + i * NZp + k0;
  const long long cjp = (long long)jp * pl + i * NZp + k0;
  const T *srr = (const T *)p.f[F_SRR], *spp = (const T *)p.f[F_SPP], *szz = (const T *)p.f[F_SZZ];
  const T *srp = (const T *)p.f[F_SRP], *spz = (const T *)p.f[F_SPZ], *srz = (const T *)p.f[F_SRZ];
  T *vr = (T *)p.f[F_VR], *vp = (T *)p.f[F_VP], *vz = (T *)p.f[F_VZ];

  float a_srr[4], a_spp[4], a_srp[4], a_srz[4], a_spz[4], a_szz[5];
  f4_to(a_srr, St<T>::ld4(srr + c));
  f4_to(a_spp, St<T>::ld4(spp + c));
  f4_to(a_srp, St<T>::ld4(srp + c));
  f4_to(a_srz, St<T>::ld4(srz + c));
  f4_to(a_spz, St<T>::ld4(spz + c));
  {
    float4 t = St<T>::ld4(szz + c);
    a_szz[0] = t.x; a_szz[1] = t.y; a_szz[2] = t.z; a_szz[3] = t.w;
    a_szz[4] = (k0 + 4 < NZ) ? St<T>::ld1(szz + c + 4) : 0.f;
  }
  const float srz_km = k0 > 0 ? St<T>::ld1(srz + c - 1) : 0.f;
  const float spz_km = k0 > 0 ? St<T>::ld1(spz + c - 1) : 0.f;
  int idc[4];
  ld_ids(p.id + c, idc);
  const int id_k4 = (k0 + 4 < NZ) ? __ldg(p.id + c + 4) : idc[3];
  float rho_c[5];
#pragma unroll
  for (int e = 0; e < 4; e++) rho_c[e] = __ldg(&p.mat[idc[e]]).x;
  rho_c[4] = __ldg(&p.mat[id_k4]).x;

  const bool rp = i >= p.nr;  // inside the radial layer
  const long long cr = rp ? ((long long)j * p.pml_r + (i - p.nr)) * NZp + k0 : 0;
  const float inv_ri = __ldg(p.inv_ri + i), inv_rh = __ldg(p.inv_rh + i);
  const float4 abr = __ldg(p.ab_r + i), abq = __ldg(p.ab_q + i);
  const float dtv = p.dtv, idr = p.inv_dr, idz = p.inv_dz, idth = p.inv_dth;
  const int pz = p.pml_z;
  const long long czrow = ((long long)j * NR + i) * (2 * pz);

  // ---- v_r at (r_i, theta_j, z_k), i >= 1
  if (i >= 1) {
    float b_srr[4], b_spp[4], b_srp[4];
    const long long cm = c - NZp;
    f4_to(b_srr, St<T>::ld4(srr + cm));
    f4_to(b_spp, St<T>::ld4(spp + cm));
    f4_to(b_srp, St<T>::ld4(srp + cjm));
    int idm[4];
    ld_ids(p.id + cm, idm);
    float out[4];
    f4_to(out, St<T>::ld4(vr + c));
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int k = k0 + e;
      if (k >= NZ) break;
      float Dr = (a_srr[e] - b_srr[e]) * idr;
      float Q = (0.5f * (a_srr[e] + b_srr[e]) - 0.5f * (a_spp[e] + b_spp[e]) + (a_srp[e] - b_srp[e]) * idth) * inv_ri;
      float Dz = (a_srz[e] - (e ? a_srz[e - 1] : srz_km)) * idz;
      if (rp) {
        Dr = stretch(p.psr[R_VR] + cr + e, abr.x, abr.y, Dr);
        Q = stretch(p.psr[Q_VR] + cr + e, abq.x, abq.y, Q);
      }
      if (k < pz || k >= NZ - pz) {
        const int kz = k < pz ? k : k - (NZ - 2 * pz);
        const float4 abz = __ldg(p.ab_z + k);
        Dz = stretch(p.psz[Z_VR] + czrow + kz, abz.x, abz.y, Dz);
      }
      const float rm = __ldg(&p.mat[idm[e]]).x;
      out[e] += vel_coef(dtv, rm + rho_c[e]) * (Dr + Q + Dz);
    }
    St<T>::st4(vr + c, make_float4(out[0], out[1], out[2], out[3]));
  }
  // ---- v_phi at (r_{i+1/2}, theta_{j+1/2}, z_k)
  {
    float b_srp[4] = {0.f, 0.f, 0.f, 0.f}, b_spp[4];
    if (i + 1 < NR) f4_to(b_srp, St<T>::ld4(srp + c + NZp));
    f4_to(b_spp, St<T>::ld4(spp + cjp));
    int idj[4];
    ld_ids(p.id + cjp, idj);
    float out[4];
    f4_to(out, St<T>::ld4(vp + c));
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int k = k0 + e;
      if (k >= NZ) break;
      const float s1 = b_srp[e], s0 = a_srp[e];
      float Dr = (s1 - s0) * idr;
      float Q = ((s1 + s0) + (b_spp[e] - a_spp[e]) * idth) * inv_rh;
      float Dz = (a_spz[e] - (e ? a_spz[e - 1] : spz_km)) * idz;
      if (rp) {
        Dr = stretch(p.psr[R_VP] + cr + e, abr.z, abr.w, Dr);
        Q = stretch(p.psr[Q_VP] + cr + e, abq.z, abq.w, Q);
      }
      if (k < pz || k >= NZ - pz) {
        const int kz = k < pz ? k : k - (NZ - 2 * pz);
        const float4 abz = __ldg(p.ab_z + k);
        Dz = stretch(p.psz[Z_VP] + czrow + kz, abz.x, abz.y, Dz);
      }
      const float rj = __ldg(&p.mat[idj[e]]).x;
      out[e] += vel_coef(dtv, rho_c[e] + rj) * (Dr + Q + Dz);
    }
    St<T>::st4(vp + c, make_float4(out[0], out[1], out[2], out[3]));
  }
  // ---- v_z at (r_{i+1/2}, theta_j, z_{k+1/2}), k + 1 < NZ
  {
    float b_srz[4] = {0.f, 0.f, 0.f, 0.f}, b_spz[4];
    if (i + 1 < NR) f4_to(b_srz, St<T>::ld4(srz + c + NZp));
    f4_to(b_spz, St<T>::ld4(spz + cjm));
    float out[4];
    f4_to(out, St<T>::ld4(vz + c));
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int k = k0 + e;
      if (k + 1 >= NZ) break;
      const float s1 = b_srz[e], s0 = a_srz[e];
      float Dr = (s1 - s0) * idr;
      float Q = (0.5f * (s1 + s0) + (a_spz[e] - b_spz[e]) * idth) * inv_rh;
      float Dz = (a_szz[e + 1] - a_szz[e]) * idz;
      if (rp) {
        Dr = stretch(p.psr[R_VZ] + cr + e, abr.z, abr.w, Dr);
        Q = stretch(p.psr[Q_VZ] + cr + e, abq.z, abq.w, Q);
      }
      if (k < pz || k >= NZ - pz) {
        const int kz = k < pz ? k : k - (NZ - 2 * pz);
        const float4 abz = __ldg(p.ab_z + k);
        Dz = stretch(p.psz[Z_VZ] + czrow + kz, abz.z, abz.w, Dz);
      }
      out[e] += vel_coef(dtv, rho_c[e] + rho_c[e + 1]) * (Dr + Q + Dz);
    }
    St<T>::st4(vz + c, make_float4(out[0], out[1], out[2], out[3]));
  }
}

// stress step of the four z cells k0 .. k0+3 of row (j, i)
template <typename T>
__device__ __forceinline__ void str_body(const KParams &p, const int j, const int i, const int k0) {
  const int nth = p.nth, NR = p.NR, NZ = p.NZ;
  const long long NZp = p.NZp, pl = p.plane;
  const int jm = j == 0 ? nth - 1 : j - 1, jp = j == nth - 1 ? 0 : j + 1;
  const long long c = (long long)j * pl + i * NZp + k0;
  const long long cjm = (long long)jm * pl + i * NZp + k0;
  const long long cjp = (long long)jp * pl + i * NZp + k0;
  const T *vr = (const T *)p.f[F_VR], *vp = (const T *)p.f[F_VP], *vz = (const T *)p.f[F_VZ];
  T *srr = (T *)p.f[F_SRR], *spp = (T *)p.f[F_SPP], *szz = (T *)p.f[F_SZZ];
  T *srp = (T *)p.f[F_SRP], *spz = (T *)p.f[F_SPZ], *srz = (T *)p.f[F_SRZ];

  float a_vr[5], a_vp[5], a_vz[4];
  {
    float4 t = St<T>::ld4(vr + c);
    a_vr[0] = t.x; a_vr[1] = t.y; a_vr[2] = t.z; a_vr[3] = t.w;
    a_vr[4] = (k0 + 4 < NZ) ? St<T>::ld1(vr + c + 4) : 0.f;
    t = St<T>::ld4(vp + c);
    a_vp[0] = t.x; a_vp[1] = t.y; a_vp[2] = t.z; a_vp[3] = t.w;
    a_vp[4] = (k0 + 4 < NZ) ? St<T>::ld1(vp + c + 4) : 0.f;
  }
  f4_to(a_vz, St<T>::ld4(vz + c));
  const float vz_km = k0 > 0 ? St<T>::ld1(vz + c - 1) : 0.f;
  int idc[5];
  {
    int t[4];
    ld_ids(p.id + c, t);
    idc[0] = t[0]; idc[1] = t[1]; idc[2] = t[2]; idc[3] = t[3];
    idc[4] = (k0 + 4 < NZ) ? __ldg(p.id + c + 4) : t[3];
  }
  int idj[5];
  {
    int t[4];
    ld_ids(p.id + cjp, t);
    idj[0] = t[0]; idj[1] = t[1]; idj[2] = t[2]; idj[3] = t[3];
    idj[4] = (k0 + 4 < NZ) ? __ldg(p.id + cjp + 4) : t[3];
  }
  const bool rp = i >= p.nr;
  const long long cr = rp ? ((long long)j * p.pml_r + (i - p.nr)) * NZp + k0 : 0;
  const float inv_ri = __ldg(p.inv_ri + i), inv_rh = __ldg(p.inv_rh + i);
  const float4 abr = __ldg(p.ab_r + i), abq = __ldg(p.ab_q + i);
  const float dts = p.dts, idr = p.inv_dr, idz = p.inv_dz, idth = p.inv_dth;
  const int pz = p.pml_z;
  const long long czrow = ((long long)j * NR + i) * (2 * pz);
  float imu_c[5], imu_j[5];
#pragma unroll
  for (int e = 0; e < 5; e++) {
    imu_c[e] = __ldg(&p.mat[idc[e]]).w;
    imu_j[e] = __ldg(&p.mat[idj[e]]).w;
  }
  // source: step-indexed increment of the three normal stresses
  float src[4] = {0.f, 0.f, 0.f, 0.f};
  if (i == p.src_i && (p.src_j < 0 || p.src_j == j) && p.src_k >= k0 && p.src_k < k0 + 4) {
    const int n = *p.step;
    src[p.src_k - k0] = n < p.n_wav ? __ldg(p.wav + n) : 0.f;
  }

  // ---- normal stresses at the cell centre
  {
    float b_vr[4] = {0.f, 0.f, 0.f, 0.f}, b_vp[4];
    if (i + 1 < NR) f4_to(b_vr, St<T>::ld4(vr + c + NZp));
    f4_to(b_vp, St<T>::ld4(vp + cjm));
    float o_rr[4], o_pp[4], o_zz[4];
    f4_to(o_rr, St<T>::ld4(srr + c));
    f4_to(o_pp, St<T>::ld4(spp + c));
    f4_to(o_zz, St<T>::ld4(szz + c));
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int k = k0 + e;
      if (k >= NZ) break;
      const float vr0 = a_vr[e], vr1 = b_vr[e];
      float err = (vr1 - vr0) * idr;
      float epp = ((a_vp[e] - b_vp[e]) * idth + 0.5f * (vr0 + vr1)) * inv_rh;
      float ezz = (a_vz[e] - (e ? a_vz[e - 1] : vz_km)) * idz;
      if (rp) {
        err = stretch(p.psr[R_ERR] + cr + e, abr.z, abr.w, err);
        epp = stretch(p.psr[Q_EPP] + cr + e, abq.z, abq.w, epp);
      }
      if (k < pz || k >= NZ - pz) {
        const int kz = k < pz ? k : k - (NZ - 2 * pz);
        const float4 abz = __ldg(p.ab_z + k);
        ezz = stretch(p.psz[Z_EZZ] + czrow + kz, abz.x, abz.y, ezz);
      }
      const float4 m = __ldg(&p.mat[idc[e]]);
      const float l = m.y, l2m = m.y + 2.f * m.z;
      o_rr[e] += dts * (l2m * err + l * (epp + ezz)) + src[e];
      o_pp[e] += dts * (l2m * epp + l * (err + ezz)) + src[e];
      o_zz[e] += dts * (l2m * ezz + l * (err + epp)) + src[e];
    }
    St<T>::st4(srr + c, make_float4(o_rr[0], o_rr[1], o_rr[2], o_rr[3]));
    St<T>::st4(spp + c, make_float4(o_pp[0], o_pp[1], o_pp[2], o_pp[3]));
    St<T>::st4(szz + c, make_float4(o_zz[0], o_zz[1], o_zz[2], o_zz[3]));
  }
  if (i >= 1) {
    const long long cm = c - NZp;
    int idm[5], idjm[5];
    {
      int t[4];
      ld_ids(p.id + cm, t);
      idm[0] = t[0]; idm[1] = t[1]; idm[2] = t[2]; idm[3] = t[3];
      idm[4] = (k0 + 4 < NZ) ? __ldg(p.id + cm + 4) : t[3];
      ld_ids(p.id + cjp - NZp, t);
      idjm[0] = t[0]; idjm[1] = t[1]; idjm[2] = t[2]; idjm[3] = t[3];
    }
    // ---- s_rphi at (r_i, theta_{j+1/2}, z_k)
    {
      float b_vp[4], j_vr[4];
      f4_to(b_vp, St<T>::ld4(vp + cm));
      f4_to(j_vr, St<T>::ld4(vr + cjp));
      float o[4];
      f4_to(o, St<T>::ld4(srp + c));
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const int k = k0 + e;
        if (k >= NZ) break;
        float gr = (a_vp[e] - b_vp[e]) * idr;
        float Q = ((j_vr[e] - a_vr[e]) * idth - 0.5f * (a_vp[e] + b_vp[e])) * inv_ri;
        if (rp) {
          gr = stretch(p.psr[R_GRP] + cr + e, abr.x, abr.y, gr);
          Q = stretch(p.psr[Q_GRP] + cr + e, abq.x, abq.y, Q);
        }
        const float mu = mu_harm(__ldg(&p.mat[idm[e]]).w + imu_c[e] + __ldg(&p.mat[idjm[e]]).w + imu_j[e]);
        o[e] += dts * mu * (gr + Q);
      }
      St<T>::st4(srp + c, make_float4(o[0], o[1], o[2], o[3]));
    }
    // ---- s_rz at (r_i, theta_j, z_{k+1/2})
    {
      float b_vz[4];
      f4_to(b_vz, St<T>::ld4(vz + cm));
      float o[4];
      f4_to(o, St<T>::ld4(srz + c));
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const int k = k0 + e;
        if (k + 1 >= NZ) break;
        float gz = (a_vr[e + 1] - a_vr[e]) * idz;
        float gr = (a_vz[e] - b_vz[e]) * idr;
        if (k < pz || k >= NZ - pz) {
          const int kz = k < pz ? k : k - (NZ - 2 * pz);
          const float4 abz = __ldg(p.ab_z + k);
          gz = stretch(p.psz[Z_GRZ] + czrow + kz, abz.z, abz.w, gz);
        }
        if (rp) gr = stretch(p.psr[R_GRZ] + cr + e, abr.x, abr.y, gr);
        const float mu = mu_harm(__ldg(&p.mat[idm[e]]).w + imu_c[e] + __ldg(&p.mat[idm[e + 1]]).w + imu_c[e + 1]);
        o[e] += dts * mu * (gz + gr);
      }
      St<T>::st4(srz + c, make_float4(o[0], o[1], o[2], o[3]));
    }
  }
  // ---- s_phiz at (r_{i+1/2}, theta_{j+1/2}, z_{k+1/2})
  {
    float j_vz[4];
    f4_to(j_vz, St<T>::ld4(vz + cjp));
    float o[4];
    f4_to(o, St<T>::ld4(spz + c));
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int k = k0 + e;
      if (k + 1 >= NZ) break;
      float Q = (j_vz[e] - a_vz[e]) * idth * inv_rh;
      float gz = (a_vp[e + 1] - a_vp[e]) * idz;
      if (rp) Q = stretch(p.psr[Q_GPZ] + cr + e, abq.z, abq.w, Q);
      if (k < pz || k >= NZ - pz) {
        const int kz = k < pz ? k : k - (NZ - 2 * pz);
        const float4 abz = __ldg(p.ab_z + k);
        gz = stretch(p.psz[Z_GPZ] + czrow + kz, abz.z, abz.w, gz);
      }
      const float mu = mu_harm(imu_c[e] + imu_j[e] + imu_c[e + 1] + imu_j[e + 1]);
      o[e] += dts * mu * (Q + gz);
    }
    St<T>::st4(spz + c, make_float4(o[0], o[1], o[2], o[3]));
  }
  (void)cjm;
  (void)nth;
}

template <typename T>
__global__ void __launch_bounds__(SB_X *SB_Y, SB_MINB) vel_split(const KParams p) {
  const int i = blockIdx.y * SB_Y + threadIdx.y, k0 = (blockIdx.z * SB_X + threadIdx.x) * 4;
  if (i < p.NR && k0 < p.NZ) vel_body<T>(p, blockIdx.x, i, k0);
}

template <typename T>
__global__ void __launch_bounds__(SB_X *SB_Y, SB_MINB) str_split(const KParams p) {
  const int i = blockIdx.y * SB_Y + threadIdx.y, k0 = (blockIdx.z * SB_X + threadIdx.x) * 4;
  if (i < p.NR && k0 < p.NZ) str_body<T>(p, blockIdx.x, i, k0);
}


// Pressure at the receivers after the stress update; one block, fixed
// summation order over theta; advances the device step counter.
template <typename T>
__device__ __forceinline__ void receivers_body(const RParams &p) {
  const int n = *p.step;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T *srr = (const T *)p.srr, *spp = (const T *)p.spp, *szz = (const T *)p.szz;
  for (int r = warp; r < p.n_rec; r += blockDim.x >> 5) {
    const int i = p.rec[3 * r], jr = p.rec[3 * r + 1], k = p.rec[3 * r + 2];
    if (k < 0) {  // a receiver of another z slab: recorded as zero here
      if (lane == 0 && n < p.cap) p.traces[(long long)r * p.cap + n] = 0.f;
      continue;
    }
    const int j0 = jr < 0 ? 0 : jr, j1 = jr < 0 ? p.nth : jr + 1;
    double acc = 0.0;
    for (int j = j0 + lane; j < j1; j += 32) {
      const long long c = (long long)j * p.plane + (long long)i * p.NZp + k;
      acc += (double)st_to_float<T>(srr[c]) + (double)st_to_float<T>(spp[c]) + (double)st_to_float<T>(szz[c]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const float v = (float)(acc / (double)(j1 - j0) * (double)p.scale);
      if (!isfinite(v)) atomicOr(p.status, 1);
      if (n < p.cap) p.traces[(long long)r * p.cap + n] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *p.step = n + 1;
}

// Point forces / torsion ring: one thread per injection point, after the
// velocity (forces) or the stress (torsion) kernel of the step.
template <typename T>
__device__ __forceinline__ T to_store(float v);
template <>
__device__ __forceinline__ float to_store<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half to_store<__half>(float v) { return __float2half_rn(v); }

template <typename T>
__global__ void __launch_bounds__(128) inject_kernel(const IParams p) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p.n) return;
  const int n = *p.step;
  if (n < 0 || n >= p.n_wav) return;
  T *x = (T *)p.f[p.fld[e]] + p.off[e];
  *x = to_store<T>(st_to_float<T>(*x) + p.w[e] * __ldg(p.wav + n));
}

template <typename T>
__global__ void __launch_bounds__(256) receivers_kernel(const RParams p) {
  receivers_body<T>(p);
}

// one block per case
template <typename T>
__global__ void __launch_bounds__(256) receivers_batch(const RParams *rp) {
  receivers_body<T>(rp[blockIdx.x]);
}

template <typename T>
static cudaError_t launch_split_t(const KParams &p, cudaStream_t s, cudaEvent_t *ev, int parts) {
  dim3 blk(SB_X, SB_Y);
  dim3 grd(p.nth, (p.NR + SB_Y - 1) / SB_Y, (p.NZ + 4 * SB_X - 1) / (4 * SB_X));
  if (parts & 1) {
    if (ev) cudaEventRecord(ev[0], s);
    vel_split<T><<<grd, blk, 0, s>>>(p);
    if (ev) cudaEventRecord(ev[1], s);
  }
  if (parts & 2) {
    str_split<T><<<grd, blk, 0, s>>>(p);
    if (ev) cudaEventRecord(ev[2], s);
  }
  return cudaGetLastError();
}

cudaError_t launch_split(int storage, const KParams &p, cudaStream_t s, cudaEvent_t *ev, int parts) {
  switch (storage) {
    case 0: return launch_split_t<float>(p, s, ev, parts);
    case 1: return launch_split_t<__nv_bfloat16>(p, s, ev, parts);
    case 2: return launch_split_t<__half>(p, s, ev, parts);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_batch_receivers(int storage, const RParams *rp, int n_cases, cudaStream_t s) {
  switch (storage) {
    case 0: receivers_batch<float><<<n_cases, 256, 0, s>>>(rp); break;
    case 1: receivers_batch<__nv_bfloat16><<<n_cases, 256, 0, s>>>(rp); break;
    case 2: receivers_batch<__half><<<n_cases, 256, 0, s>>>(rp); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_inject(int storage, const IParams &p, cudaStream_t s) {
  if (p.n < 1) return cudaSuccess;
  const int blocks = (p.n + 127) / 128;
  switch (storage) {
    case 0: inject_kernel<float><<<blocks, 128, 0, s>>>(p); break;
    case 1: inject_kernel<__nv_bfloat16><<<blocks, 128, 0, s>>>(p); break;
    case 2: inject_kernel<__half><<<blocks, 128, 0, s>>>(p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_receivers(int storage, const RParams &p, cudaStream_t s) {
  switch (storage) {
    case 0: receivers_kernel<float><<<1, 256, 0, s>>>(p); break;
    case 1: receivers_kernel<__nv_bfloat16><<<1, 256, 0, s>>>(p); break;
    case 2: receivers_kernel<__half><<<1, 256, 0, s>>>(p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace cwell
