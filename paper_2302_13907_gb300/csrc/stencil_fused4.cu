// Fused path, vector variant: the time-skewed theta-marching step of
// stencil_fused.cu with four consecutive z cells per thread.
//
// Per block: an (RT x 64) tile of (r, z), NT = 16 (RT + 2) threads, thread
// (row, quad) owns z cells k0 + 4 quad .. k0 + 4 quad + 3 of one tile row in
// both passes.  The six stresses and the material IDs of planes m-1 .. m+2
// sit in the 4-slot TMA ring; the thread's own v^{n-1/2} comes from one
// 16-byte global load per component, issued one plane ahead; shared-memory
// reads are 16-byte vectors; z neighbours inside the quad come from
// registers.  Halo columns (v_z at k0-1, v_r and v_phi at k0+64) are computed
// by the edge quads of each row.  Same arithmetic, same bounded waits, same
// double buffering as the scalar fused kernel.
#include "tma_util.cuh"

namespace cwell {

template <typename T>
__device__ __forceinline__ float4 sld4(const T *p);
template <>
__device__ __forceinline__ float4 sld4<float>(const float *p) { return *reinterpret_cast<const float4 *>(p); }
template <>
__device__ __forceinline__ float4 sld4<__nv_bfloat16>(const __nv_bfloat16 *p) {
  const uint2 u = *reinterpret_cast<const uint2 *>(p);
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}
template <>
__device__ __forceinline__ float4 sld4<__half>(const __half *p) {
  const uint2 u = *reinterpret_cast<const uint2 *>(p);
  const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ void ids4(const uint16_t *p, int (&o)[4]) {
  const uint2 u = *reinterpret_cast<const uint2 *>(p);
  o[0] = u.x & 0xffff;
  o[1] = u.x >> 16;
  o[2] = u.y & 0xffff;
  o[3] = u.y >> 16;
}

#define F4(v, e) ((e) == 0 ? (v).x : (e) == 1 ? (v).y : (e) == 2 ? (v).z : (v).w)

template <typename T, int RT>
struct F4Smem {
  static constexpr int ZT = 64;
  static constexpr int HX = Pad<T>::HX;
  static constexpr int BR = RT + 2;
  static constexpr int BW = ZT + 2 * HX;
  static constexpr int BWI = ZT + 16;
  static constexpr int VW = ZT + 8;  // velocity ring: z from k0-4 (16-byte aligned quads)
  static constexpr int NT = 16 * BR;
  static constexpr int BOXB = (BR * BW * (int)sizeof(T) + 127) / 128 * 128;
  static constexpr int BOX_ELEMS = BOXB / (int)sizeof(T);
  static constexpr int IDB = (BR * BWI * 2 + 127) / 128 * 128;
  static constexpr int SLOT_BYTES = 6 * BOXB + IDB;  // six stresses + IDs of one plane
  static constexpr size_t RING_BYTES = (size_t)4 * SLOT_BYTES;
  static constexpr int VPL = 3 * BR * VW;  // floats per velocity plane
  static constexpr size_t V_BYTES = (size_t)4 * VPL * 4;
  static constexpr size_t BAR_OFF = (RING_BYTES + V_BYTES + 127) / 128 * 128;
  static constexpr size_t BYTES = BAR_OFF + 4 * 8 + 128;
  static constexpr uint32_t TX = (uint32_t)(6 * BR * BW * sizeof(T) + BR * BWI * 2);
};

template <typename T, int RT>
__global__ void __launch_bounds__(F4Smem<T, RT>::NT) fused4_step(const __grid_constant__ FusedMaps maps,
                                                                  const __grid_constant__ FusedParams fp) {
  using SM = F4Smem<T, RT>;
  constexpr int ZT = SM::ZT, HX = SM::HX, BR = SM::BR, BW = SM::BW, BWI = SM::BWI, VW = SM::VW, NT = SM::NT,
                VPL = SM::VPL;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  float *vring = reinterpret_cast<float *>(smem + SM::RING_BYTES);
  float *vsave = vring + 3 * VPL;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + SM::BAR_OFF);

  const KParams &p = fp.k;
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * RT, k0 = blockIdx.y * ZT;
  const int nth = p.nth, NR = p.NR, NZ = p.NZ, NZp = p.NZp, pz = p.pml_z, nr_p = p.nr;
  const long long pl = p.plane;
  const int row = tid >> 4, qd = tid & 15;
  const int i = i0 - 1 + row;    // radial index of this thread's row
  const int kq = k0 + 4 * qd;    // first z cell of this thread's quad
  const int x = row * BW + 4 * qd + HX;     // quad in a field box
  const int xi = row * BWI + 4 * qd + 8;    // quad in an ID box
  const int xv = row * VW + 4 * qd + 4;     // quad in a velocity plane

  if (tid == 0) {
    for (int s = 0; s < 4; s++) mbar_init(&bar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // stresses of ring slot s (field 0 .. 5 = s_rr, s_pp, s_zz, s_rp, s_pz, s_rz)
  auto SF = [&](int s, int f) -> const T * {
    return reinterpret_cast<const T *>(smem + (size_t)s * SM::SLOT_BYTES + (size_t)f * SM::BOXB);
  };
  auto SI = [&](int s) -> const uint16_t * {
    return reinterpret_cast<const uint16_t *>(smem + (size_t)s * SM::SLOT_BYTES + 6 * SM::BOXB);
  };
  uint32_t phase = 0;
  auto issue = [&](int q) {
    const int s = q & 3, plane = ((q % nth) + nth) % nth;
    mbar_expect_tx(&bar[s], SM::TX);
    unsigned char *base = smem + (size_t)s * SM::SLOT_BYTES;
    for (int f = 0; f < 6; f++)
      tma_load_4d(base + f * SM::BOXB, &maps.f[F_SRR + f], k0 - HX, i0 - 1, plane, 0, &bar[s]);
    tma_load_4d(base + 6 * SM::BOXB, &maps.id, k0 - 8, i0 - 1, plane, 0, &bar[s]);
  };
  int issued_hi, waited_hi = -3;
  bool ok = true, failed = false;
  auto wait_q = [&](int q) {
    const int s = q & 3;
    const bool w = mbar_wait(&bar[s], (phase >> s) & 1u);
    if (w) {
      phase ^= 1u << s;
      waited_hi = q;
    }
    return w;
  };
  if (tid == 0)
    for (int q = -2; q <= 1; q++) issue(q);
  issued_hi = 1;
  ok = wait_q(-2);
  if (ok) ok = wait_q(-1);

  // ---- per-thread constants (fixed along the march)
  const bool row_ok = i >= 0 && i < NR;
  const int ic = min(max(i, 0), NR - 1);
  const float inv_ri = __ldg(p.inv_ri + ic), inv_rh = __ldg(p.inv_rh + ic);
  const float4 ab = __ldg(p.ab_r + ic), aq = __ldg(p.ab_q + ic);
  const bool rp = row_ok && i >= nr_p;
  const long long crb = rp ? (long long)(i - nr_p) * NZp + kq : 0;  // radial slab, plane term added per plane
  const long long pr_plane = (long long)p.pml_r * NZp, pz_plane = (long long)NR * 2 * pz;
  const bool quad_in = kq < NZp;  // whole quad inside the padded row (NZp is a multiple of 32)
  const bool any_zp = pz > 0 && (kq < pz || kq + 3 >= NZ - pz);
  const float dtv = p.dtv, dts = p.dts, idr = p.inv_dr, idz = p.inv_dz, idth = p.inv_dth;
  const float *m_rho = p.m_rho, *m_imu = p.m_imu;
  const float2 *m_lam = p.m_lam;
  const T *vcur_g[3] = {(const T *)p.f[F_VR], (const T *)p.f[F_VP], (const T *)p.f[F_VZ]};
  T *vnxt[3] = {(T *)fp.fo[F_VR], (T *)fp.fo[F_VP], (T *)fp.fo[F_VZ]};
  T *so[6] = {(T *)fp.fo[F_SRR], (T *)fp.fo[F_SPP], (T *)fp.fo[F_SZZ],
              (T *)fp.fo[F_SRP], (T *)fp.fo[F_SPZ], (T *)fp.fo[F_SRZ]};
  const long long cb = (long long)ic * NZp + kq;  // this quad's offset inside a plane

  // v^{n-1/2} of this quad: registers, loaded one plane ahead
  float4 vold[3], vpre[3];
  auto load_vold = [&](int m, float4 (&dst)[3]) {
    const int plane = ((m % nth) + nth) % nth;
    for (int c = 0; c < 3; c++)
      dst[c] = (row_ok && quad_in) ? St<T>::ld4(vcur_g[c] + plane * pl + cb) : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  load_vold(-1, vold);

  // scalar velocity of component c at (tile row r, depth k) for the halo columns
  auto vel_scalar = [&](int c, int r, int k, int plane, int sm1, int s0, int sp1) -> float {
    const int ii = i0 - 1 + r;
    if (ii < 0 || ii >= NR || k < 0 || k >= NZ || (c == 0 && ii < 1) || (c == 2 && k + 1 >= NZ)) return 0.f;
    const int xx = r * BW + (k - k0 + HX), xx_i = r * BWI + (k - k0 + 8);
    const uint16_t *I0 = SI(s0);
    const long long cc = (long long)plane * pl + (long long)ii * NZp + k;
    const bool rpx = ii >= nr_p;
    const long long cr = rpx ? ((long long)plane * p.pml_r + (ii - nr_p)) * NZp + k : 0;
    const bool zpx = k < pz || k >= NZ - pz;
    const long long cz = ((long long)plane * NR + ii) * (2 * pz) + (k < pz ? k : k - (NZ - 2 * pz));
    const float4 abx = __ldg(p.ab_r + ii), aqx = __ldg(p.ab_q + ii);
    const float4 abz = zpx ? __ldg(p.ab_z + k) : make_float4(0.f, 1.f, 0.f, 1.f);
    float Dr, Q, Dz, rho;
    if (c == 0) {
      const float a = sld(SF(s0, 0) + xx), am = sld(SF(s0, 0) + xx - BW), b = sld(SF(s0, 1) + xx),
                  bm = sld(SF(s0, 1) + xx - BW);
      Dr = (a - am) * idr;
      Q = (0.5f * (a + am) - 0.5f * (b + bm) + (sld(SF(s0, 3) + xx) - sld(SF(sm1, 3) + xx)) * idth) * __ldg(p.inv_ri + ii);
      Dz = (sld(SF(s0, 5) + xx) - sld(SF(s0, 5) + xx - 1)) * idz;
      if (rpx) {
        Dr += abx.y * p.psr[R_VR][cr] + abx.x * Dr;
        Q += aqx.y * p.psr[Q_VR][cr] + aqx.x * Q;
      }
      if (zpx) Dz += abz.y * p.psz[Z_VR][cz] + abz.x * Dz;
      rho = __ldg(m_rho + I0[xx_i]) + __ldg(m_rho + I0[xx_i - BWI]);
    } else if (c == 1) {
      const float s1 = sld(SF(s0, 3) + xx + BW), s0v = sld(SF(s0, 3) + xx);
      Dr = (s1 - s0v) * idr;
      Q = ((s1 + s0v) + (sld(SF(sp1, 1) + xx) - sld(SF(s0, 1) + xx)) * idth) * __ldg(p.inv_rh + ii);
      Dz = (sld(SF(s0, 4) + xx) - sld(SF(s0, 4) + xx - 1)) * idz;
      if (rpx) {
        Dr += abx.w * p.psr[R_VP][cr] + abx.z * Dr;
        Q += aqx.w * p.psr[Q_VP][cr] + aqx.z * Q;
      }
      if (zpx) Dz += abz.y * p.psz[Z_VP][cz] + abz.x * Dz;
      rho = __ldg(m_rho + I0[xx_i]) + __ldg(m_rho + SI(sp1)[xx_i]);
    } else {
      const float s1 = sld(SF(s0, 5) + xx + BW), s0v = sld(SF(s0, 5) + xx);
      Dr = (s1 - s0v) * idr;
      Q = (0.5f * (s1 + s0v) + (sld(SF(s0, 4) + xx) - sld(SF(sm1, 4) + xx)) * idth) * __ldg(p.inv_rh + ii);
      Dz = (sld(SF(s0, 2) + xx + 1) - sld(SF(s0, 2) + xx)) * idz;
      if (rpx) {
        Dr += abx.w * p.psr[R_VZ][cr] + abx.z * Dr;
        Q += aqx.w * p.psr[Q_VZ][cr] + aqx.z * Q;
      }
      if (zpx) Dz += abz.w * p.psz[Z_VZ][cz] + abz.z * Dz;
      rho = __ldg(m_rho + I0[xx_i]) + __ldg(m_rho + I0[xx_i + 1]);
    }
    return St<T>::ld1(vcur_g[c] + cc) + vel_coef(dtv, rho) * (Dr + Q + Dz);
  };

  for (int m = -1; m <= nth; m++) {
    if (m + 2 <= nth && m + 2 > issued_hi) {
      if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(m + 2);
      }
      issued_hi = m + 2;
    }
    if (m + 1 <= nth - 1) load_vold(m + 1, vpre);  // next plane's v^{n-1/2}, one plane ahead
    if (ok && m + 1 <= nth && m + 1 > waited_hi) ok = wait_q(m + 1);
    const int sm1 = (m - 1) & 3, s0 = m & 3, sp1 = (m + 1) & 3;

    if (m <= nth - 1) {
      // ---------------- velocity half-step of plane m (quad of this thread + halo columns)
      const int plane = ((m % nth) + nth) % nth;
      float *V = vring + (((m % 3) + 3) % 3) * VPL;
      const long long cr = plane * pr_plane + crb;
      const bool own = m >= 0 && row >= 1 && row <= RT && row_ok && quad_in;
      float4 vr4 = make_float4(0.f, 0.f, 0.f, 0.f), vp4 = vr4, vz4 = vr4;
      if (row_ok && quad_in) {
        const T *Srr = SF(s0, 0), *Spp = SF(s0, 1), *Szz = SF(s0, 2), *Srp = SF(s0, 3), *Spz = SF(s0, 4),
                *Srz = SF(s0, 5);
        int idc[4], idm[4], idj[4];
        ids4(SI(s0) + xi, idc);
        const float4 rp0 = sld4(Srp + x), pp0 = sld4(Spp + x), rz0 = sld4(Srz + x), pz0 = sld4(Spz + x);
        const float rz_km = sld(Srz + x - 1), pz_km = sld(Spz + x - 1);
        // v_r (rows 1 .. RT+1, i >= 1)
        if (row >= 1 && i >= 1) {
          ids4(SI(s0) + xi - BWI, idm);
          const float4 rr0 = sld4(Srr + x), rrm = sld4(Srr + x - BW), ppm = sld4(Spp + x - BW),
                       rpj = sld4(SF(sm1, 3) + x);
          float o[4];
#pragma unroll
          for (int e = 0; e < 4; e++) {
            const int k = kq + e;
            float Dr = (F4(rr0, e) - F4(rrm, e)) * idr;
            float Q = (0.5f * (F4(rr0, e) + F4(rrm, e)) - 0.5f * (F4(pp0, e) + F4(ppm, e)) +
                       (F4(rp0, e) - F4(rpj, e)) * idth) * inv_ri;
            float Dz = (F4(rz0, e) - (e ? F4(rz0, e - 1) : rz_km)) * idz;
            if (rp) {
              const float ps = ab.y * p.psr[R_VR][cr + e] + ab.x * Dr;
              const float qs = aq.y * p.psr[Q_VR][cr + e] + aq.x * Q;
              if (own) {
                fp.psr_o[R_VR][cr + e] = ps;
                fp.psr_o[Q_VR][cr + e] = qs;
              }
              Dr += ps;
              Q += qs;
            }
            if (any_zp && (k < pz || (k >= NZ - pz && k < NZ))) {
              const long long cz = plane * pz_plane + (long long)i * (2 * pz) + (k < pz ? k : k - (NZ - 2 * pz));
              const float4 abz = __ldg(p.ab_z + k);
              const float ps = abz.y * p.psz[Z_VR][cz] + abz.x * Dz;
              if (own) fp.psz_o[Z_VR][cz] = ps;
              Dz += ps;
            }
            const float rho = __ldg(m_rho + idc[e]) + __ldg(m_rho + idm[e]);
            o[e] = k < NZ ? F4(vold[0], e) + vel_coef(dtv, rho) * (Dr + Q + Dz) : 0.f;
          }
          vr4 = make_float4(o[0], o[1], o[2], o[3]);
        }
        if (row <= RT) {
          // v_phi
          ids4(SI(sp1) + xi, idj);
          const float4 rp1 = sld4(Srp + x + BW), ppj = sld4(SF(sp1, 1) + x);
          float o[4];
#pragma unroll
          for (int e = 0; e < 4; e++) {
            const int k = kq + e;
            float Dr = (F4(rp1, e) - F4(rp0, e)) * idr;
            float Q = ((F4(rp1, e) + F4(rp0, e)) + (F4(ppj, e) - F4(pp0, e)) * idth) * inv_rh;
            float Dz = (F4(pz0, e) - (e ? F4(pz0, e - 1) : pz_km)) * idz;
            if (rp) {
              const float ps = ab.w * p.psr[R_VP][cr + e] + ab.z * Dr;
              const float qs = aq.w * p.psr[Q_VP][cr + e] + aq.z * Q;
              if (own) {
                fp.psr_o[R_VP][cr + e] = ps;
                fp.psr_o[Q_VP][cr + e] = qs;
              }
              Dr += ps;
              Q += qs;
            }
            if (any_zp && (k < pz || (k >= NZ - pz && k < NZ))) {
              const long long cz = plane * pz_plane + (long long)i * (2 * pz) + (k < pz ? k : k - (NZ - 2 * pz));
              const float4 abz = __ldg(p.ab_z + k);
              const float ps = abz.y * p.psz[Z_VP][cz] + abz.x * Dz;
              if (own) fp.psz_o[Z_VP][cz] = ps;
              Dz += ps;
            }
            const float rho = __ldg(m_rho + idc[e]) + __ldg(m_rho + idj[e]);
            o[e] = k < NZ ? F4(vold[1], e) + vel_coef(dtv, rho) * (Dr + Q + Dz) : 0.f;
          }
          vp4 = make_float4(o[0], o[1], o[2], o[3]);
          // v_z
          const float4 rz1 = sld4(Srz + x + BW), pzj = sld4(SF(sm1, 4) + x), zz0 = sld4(Szz + x);
          const float zz4 = sld(Szz + x + 4);
          const int id4 = SI(s0)[xi + 4];
#pragma unroll
          for (int e = 0; e < 4; e++) {
            const int k = kq + e;
            float Dr = (F4(rz1, e) - F4(rz0, e)) * idr;
            float Q = (0.5f * (F4(rz1, e) + F4(rz0, e)) + (F4(pz0, e) - F4(pzj, e)) * idth) * inv_rh;
            float Dz = ((e < 3 ? F4(zz0, e + 1) : zz4) - F4(zz0, e)) * idz;
            if (rp) {
              const float ps = ab.w * p.psr[R_VZ][cr + e] + ab.z * Dr;
              const float qs = aq.w * p.psr[Q_VZ][cr + e] + aq.z * Q;
              if (own) {
                fp.psr_o[R_VZ][cr + e] = ps;
                fp.psr_o[Q_VZ][cr + e] = qs;
              }
              Dr += ps;
              Q += qs;
            }
            if (any_zp && (k < pz || (k >= NZ - pz && k < NZ))) {
              const long long cz = plane * pz_plane + (long long)i * (2 * pz) + (k < pz ? k : k - (NZ - 2 * pz));
              const float4 abz = __ldg(p.ab_z + k);
              const float ps = abz.w * p.psz[Z_VZ][cz] + abz.z * Dz;
              if (own) fp.psz_o[Z_VZ][cz] = ps;
              Dz += ps;
            }
            const float rho = __ldg(m_rho + idc[e]) + __ldg(m_rho + (e < 3 ? idc[e + 1] : id4));
            o[e] = k + 1 < NZ ? F4(vold[2], e) + vel_coef(dtv, rho) * (Dr + Q + Dz) : 0.f;
          }
          vz4 = make_float4(o[0], o[1], o[2], o[3]);
        }
      }
      *reinterpret_cast<float4 *>(V + 0 * BR * VW + xv) = vr4;
      *reinterpret_cast<float4 *>(V + 1 * BR * VW + xv) = vp4;
      *reinterpret_cast<float4 *>(V + 2 * BR * VW + xv) = vz4;
      if (own) {
        const long long cg = (long long)plane * pl + cb;
        St<T>::st4(vnxt[0] + cg, vr4);
        St<T>::st4(vnxt[1] + cg, vp4);
        St<T>::st4(vnxt[2] + cg, vz4);
      }
      // halo columns (recomputed, never written): v_z at k0-1 by quad 0, v_r and v_phi at k0+64 by quad 15
      if (qd == 0) {
        V[2 * BR * VW + row * VW + 3] = row <= RT ? vel_scalar(2, row, k0 - 1, plane, sm1, s0, sp1) : 0.f;
      } else if (qd == 15) {
        V[0 * BR * VW + row * VW + 4 + ZT] = row >= 1 ? vel_scalar(0, row, k0 + ZT, plane, sm1, s0, sp1) : 0.f;
        V[1 * BR * VW + row * VW + 4 + ZT] = row <= RT ? vel_scalar(1, row, k0 + ZT, plane, sm1, s0, sp1) : 0.f;
      }
      if (m == 0) {
        __syncthreads();
        for (int q = tid; q < VPL; q += NT) vsave[q] = V[q];
      }
    }
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }

    if (m >= 1 && row >= 1 && row <= RT && row_ok && quad_in) {
      // ---------------- stress step of plane m-1, four cells per thread
      const int plane = m - 1;
      const float *Va = vring + (((m - 2) % 3 + 3) % 3) * VPL, *Vb = vring + ((m - 1) % 3) * VPL;
      const float *Vc = (m == nth) ? vsave : vring + (m % 3) * VPL;
      const float *Vbr = Vb, *Vbp = Vb + BR * VW, *Vbz = Vb + 2 * BR * VW;
      const float4 vr0 = *reinterpret_cast<const float4 *>(Vbr + xv), vr1 = *reinterpret_cast<const float4 *>(Vbr + xv + VW);
      const float vr_k4 = Vbr[xv + 4];
      const float4 vp0 = *reinterpret_cast<const float4 *>(Vbp + xv), vpm = *reinterpret_cast<const float4 *>(Vbp + xv - VW);
      const float4 vpa = *reinterpret_cast<const float4 *>(Va + BR * VW + xv);
      const float vp_k4 = Vbp[xv + 4];
      const float4 vz0 = *reinterpret_cast<const float4 *>(Vbz + xv), vzm = *reinterpret_cast<const float4 *>(Vbz + xv - VW);
      const float vz_km = Vbz[xv - 1];
      const float4 vrc = *reinterpret_cast<const float4 *>(Vc + xv), vzc = *reinterpret_cast<const float4 *>(Vc + 2 * BR * VW + xv);
      float4 o4[6];
#pragma unroll
      for (int f = 0; f < 6; f++) o4[f] = sld4(SF(sm1, f) + x);
      int im[4], imm[4], ij[4], ijm[4];
      ids4(SI(sm1) + xi, im);
      ids4(SI(sm1) + xi - BWI, imm);
      ids4(SI(s0) + xi, ij);
      ids4(SI(s0) + xi - BWI, ijm);
      const int im4 = SI(sm1)[xi + 4], imm4 = SI(sm1)[xi - BWI + 4], ij4 = SI(s0)[xi + 4];
      float mu_c[5], mu_m[5], mu_j[5], mu_jm[4];
#pragma unroll
      for (int e = 0; e < 4; e++) {
        mu_c[e] = __ldg(m_imu + im[e]);
        mu_m[e] = __ldg(m_imu + imm[e]);
        mu_j[e] = __ldg(m_imu + ij[e]);
        mu_jm[e] = __ldg(m_imu + ijm[e]);
      }
      mu_c[4] = __ldg(m_imu + im4);
      mu_m[4] = __ldg(m_imu + imm4);
      mu_j[4] = __ldg(m_imu + ij4);
      const long long cr = plane * pr_plane + crb;
      float o[6][4];
#pragma unroll
      for (int f = 0; f < 6; f++) {
        o[f][0] = o4[f].x;
        o[f][1] = o4[f].y;
        o[f][2] = o4[f].z;
        o[f][3] = o4[f].w;
      }
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const int k = kq + e;
        if (k >= NZ) break;
        const bool zpm = any_zp && (k < pz || k >= NZ - pz);
        const long long cz = plane * pz_plane + (long long)i * (2 * pz) + (k < pz ? k : k - (NZ - 2 * pz));
        const float4 abz = zpm ? __ldg(p.ab_z + k) : make_float4(0.f, 1.f, 0.f, 1.f);
        {
          float err = (F4(vr1, e) - F4(vr0, e)) * idr;
          float epp = ((F4(vp0, e) - F4(vpa, e)) * idth + 0.5f * (F4(vr0, e) + F4(vr1, e))) * inv_rh;
          float ezz = (F4(vz0, e) - (e ? F4(vz0, e - 1) : vz_km)) * idz;
          if (rp) {
            const float ps = ab.w * p.psr[R_ERR][cr + e] + ab.z * err;
            const float qs = aq.w * p.psr[Q_EPP][cr + e] + aq.z * epp;
            fp.psr_o[R_ERR][cr + e] = ps;
            fp.psr_o[Q_EPP][cr + e] = qs;
            err += ps;
            epp += qs;
          }
          if (zpm) {
            const float ps = abz.y * p.psz[Z_EZZ][cz] + abz.x * ezz;
            fp.psz_o[Z_EZZ][cz] = ps;
            ezz += ps;
          }
          const float2 ll = __ldg(m_lam + im[e]);
          float src = 0.f;
          if (i == p.src_i && k == p.src_k && (p.src_j < 0 || p.src_j == plane)) {
            const int n = *p.step;
            src = n < p.n_wav ? __ldg(p.wav + n) : 0.f;
          }
          o[0][e] += dts * (ll.y * err + ll.x * (epp + ezz)) + src;
          o[1][e] += dts * (ll.y * epp + ll.x * (err + ezz)) + src;
          o[2][e] += dts * (ll.y * ezz + ll.x * (err + epp)) + src;
        }
        if (i >= 1) {
          float gr = (F4(vp0, e) - F4(vpm, e)) * idr;
          float Q = ((F4(vrc, e) - F4(vr0, e)) * idth - 0.5f * (F4(vp0, e) + F4(vpm, e))) * inv_ri;
          if (rp) {
            const float ps = ab.y * p.psr[R_GRP][cr + e] + ab.x * gr;
            const float qs = aq.y * p.psr[Q_GRP][cr + e] + aq.x * Q;
            fp.psr_o[R_GRP][cr + e] = ps;
            fp.psr_o[Q_GRP][cr + e] = qs;
            gr += ps;
            Q += qs;
          }
          const float mu = mu_harm(mu_m[e] + mu_c[e] + mu_jm[e] + mu_j[e]);
          o[3][e] += dts * mu * (gr + Q);
        }
        if (k + 1 < NZ) {
          if (i >= 1) {
            float gz = ((e < 3 ? F4(vr0, e + 1) : vr_k4) - F4(vr0, e)) * idz;
            float gr = (F4(vz0, e) - F4(vzm, e)) * idr;
            if (zpm) {
              const float ps = abz.w * p.psz[Z_GRZ][cz] + abz.z * gz;
              fp.psz_o[Z_GRZ][cz] = ps;
              gz += ps;
            }
            if (rp) {
              const float ps = ab.y * p.psr[R_GRZ][cr + e] + ab.x * gr;
              fp.psr_o[R_GRZ][cr + e] = ps;
              gr += ps;
            }
            const float mu = mu_harm(mu_m[e] + mu_c[e] + mu_m[e + 1] + mu_c[e + 1]);
            o[5][e] += dts * mu * (gz + gr);
          }
          float Q = (F4(vzc, e) - F4(vz0, e)) * idth * inv_rh;
          float gz = ((e < 3 ? F4(vp0, e + 1) : vp_k4) - F4(vp0, e)) * idz;
          if (rp) {
            const float qs = aq.w * p.psr[Q_GPZ][cr + e] + aq.z * Q;
            fp.psr_o[Q_GPZ][cr + e] = qs;
            Q += qs;
          }
          if (zpm) {
            const float ps = abz.w * p.psz[Z_GPZ][cz] + abz.z * gz;
            fp.psz_o[Z_GPZ][cz] = ps;
            gz += ps;
          }
          const float mu = mu_harm(mu_c[e] + mu_j[e] + mu_c[e + 1] + mu_j[e + 1]);
          o[4][e] += dts * mu * (Q + gz);
        }
      }
      const long long cg = (long long)plane * pl + cb;
#pragma unroll
      for (int f = 0; f < 6; f++) St<T>::st4(so[f] + cg, make_float4(o[f][0], o[f][1], o[f][2], o[f][3]));
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 3; c++) vold[c] = vpre[c];
  }
  if (failed) {
    if (tid == 0) atomicOr(fp.status, 2);
    for (int q = waited_hi + 1; q <= issued_hi; q++) {
      const int s = q & 3;
      if (mbar_wait(&bar[s], (phase >> s) & 1u)) phase ^= 1u << s;
    }
    __syncthreads();
  }
}

template <typename T, int RT>
static cudaError_t launch_fused4_t(const FusedMaps &maps, const FusedParams &fp, cudaStream_t s) {
  using SM = F4Smem<T, RT>;
  auto kern = fused4_step<T, RT>;
  static bool attr_done[16] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 16 && !attr_done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::BYTES);
    if (e != cudaSuccess) return e;
    attr_done[dev] = true;
  }
  dim3 grd((fp.k.NR + RT - 1) / RT, (fp.k.NZ + SM::ZT - 1) / SM::ZT);
  kern<<<grd, SM::NT, SM::BYTES, s>>>(maps, fp);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_fused4_rt(int rt, const FusedMaps &maps, const FusedParams &fp, cudaStream_t s) {
  switch (rt) {
    case 6: return launch_fused4_t<T, 6>(maps, fp, s);
    case 10: return launch_fused4_t<T, 10>(maps, fp, s);
    case 14: return launch_fused4_t<T, 14>(maps, fp, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_fused4(int storage, int rt, const FusedMaps &maps, const FusedParams &fp, cudaStream_t s) {
  switch (storage) {
    case 0: return launch_fused4_rt<float>(rt, maps, fp, s);
    case 1: return launch_fused4_rt<__nv_bfloat16>(rt, maps, fp, s);
    case 2: return launch_fused4_rt<__half>(rt, maps, fp, s);
  }
  return cudaErrorInvalidValue;
}

size_t fused4_smem_bytes(int storage, int rt) {
  auto pick = [&](auto tag) -> size_t {
    using T = decltype(tag);
    switch (rt) {
      case 6: return F4Smem<T, 6>::BYTES;
      case 10: return F4Smem<T, 10>::BYTES;
      case 14: return F4Smem<T, 14>::BYTES;
    }
    return 0;
  };
  if (storage == 0) return pick(float{});
  if (storage == 1) return pick(__nv_bfloat16{});
  return pick(__half{});
}

}  // namespace cwell
