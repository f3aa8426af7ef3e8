// Fused path: one kernel per leapfrog step (velocity half-step and stress
// step together), double-buffered state.
//
// A block owns an (r, z) tile of RT rows x ZT cells and marches over all
// nth azimuthal planes.  For march index m it
//   1. has the nine fields of step n (and the material IDs) of planes m-1, m,
//      m+1 in a 4-slot shared-memory ring (tile plus one cell of halo in r
//      and z), brought in by TMA (cp.async.bulk.tensor, mbarrier completion)
//      one plane ahead;
//   2. computes v^{n+1/2} of plane m on the tile plus halo (halo values are
//      recomputed here instead of exchanged between blocks), keeps it in a
//      3-plane ring and writes the owned part with its PML memory variables;
//   3. computes s^{n+1} of plane m-1 from the velocity planes m-2, m-1, m and
//      writes it, with the source increment and PML memory variables.
// The march starts at m = -1 so the periodic neighbour of plane 0 exists;
// velocity plane 0 is kept for the last stress plane.  Reads come from the
// "cur" buffers, writes go to "nxt", so recomputed halos never race with the
// owners' writes.  DRAM traffic per cell-update is the minimum: every field
// read once and written once, plus the material ID.
//
// Threads: NT = 64 (RT + 2); thread (row, lane) owns one z column of one
// tile row in both passes, so every shared-memory access of a warp is 32
// consecutive words.  The tensors are 4-D [case][nth][NR][NZp] so the same
// body serves one well and a batch of wells.
//
// Every mbarrier wait is bounded; a wait that gives up sets bit 1 of the
// status word, waits (bounded) for the block's copies still in flight and
// returns, so a broken launch reports SIM_ETIMEOUT instead of hanging.
#include "tma_util.cuh"

namespace cwell {

template <typename T, int RT, int ZT>
struct FusedSmem {
  static constexpr int HX = Pad<T>::HX;
  static constexpr int BR = RT + 2;       // rows i0-1 .. i0+RT
  static constexpr int BW = ZT + 2 * HX;  // z from k0-HX
  static constexpr int BWI = ZT + 16;     // IDs: z from k0-8
  static constexpr int VW = ZT + 2;       // velocity ring: z from k0-1
  static constexpr int NT = 64 * BR;      // threads: one z column of one row each
  // resident blocks per SM the register allocator is asked to allow (shared
  // memory allows 3 / 2 / 2 / 1 blocks of the 2 / 4 / 6 / 8-row tiles)
  static constexpr int MINB = RT == 2 ? 3 : (RT <= 6 ? 2 : 1);
  // every TMA destination starts on a 128-byte boundary
  static constexpr int BOXB = (BR * BW * (int)sizeof(T) + 127) / 128 * 128;
  static constexpr int IDB = (BR * BWI * 2 + 127) / 128 * 128;
  static constexpr int BOX_ELEMS = BOXB / (int)sizeof(T);
  static constexpr int SLOT_BYTES = 9 * BOXB + IDB;  // nine fields + IDs of one plane
  static constexpr size_t RING_BYTES = (size_t)4 * SLOT_BYTES;
  static constexpr size_t V_BYTES = (size_t)4 * 3 * BR * VW * 4;  // 3 ring planes + saved plane 0
  static constexpr size_t BAR_OFF = (RING_BYTES + V_BYTES + 127) / 128 * 128;
  static constexpr size_t BYTES = BAR_OFF + 4 * 8 + 128;  // + slack for aligning the base
  static constexpr uint32_t TX = (uint32_t)(9 * BR * BW * sizeof(T) + BR * BWI * 2);
  static_assert(ZT == 64, "thread mapping assumes 64 z columns per tile");
};

// One fused step of the tile (i0, k0) of case `cs` (4th TMA coordinate).
template <typename T, int RT, int ZT>
__device__ __forceinline__ void fused_tile(const FusedMaps &maps, const FusedParams &fp, int cs, int i0, int k0,
                                           unsigned char *smem, uint64_t *bar, uint32_t &phase) {
  using SM = FusedSmem<T, RT, ZT>;
  constexpr int HX = SM::HX, BR = SM::BR, BW = SM::BW, BWI = SM::BWI, VW = SM::VW, NT = SM::NT;
  const KParams &p = fp.k;
  const int tid = threadIdx.x;
  const int nth = p.nth, NR = p.NR, NZ = p.NZ, NZp = p.NZp;
  const long long pl = p.plane;
  const int pz = p.pml_z, nr_p = p.nr;
  float *vr_ring = reinterpret_cast<float *>(smem + SM::RING_BYTES);
  float *vsave = vr_ring + 3 * 3 * BR * VW;

  // thread -> (row, z column) of the tile plus halo rows
  const int row = tid >> 6, lane = tid & 63;

  auto slot_field = [&](int s, int f) -> const T * {
    return reinterpret_cast<const T *>(smem + (size_t)s * SM::SLOT_BYTES + (size_t)f * SM::BOXB);
  };
  auto slot_ids = [&](int s) -> const uint16_t * {
    return reinterpret_cast<const uint16_t *>(smem + (size_t)s * SM::SLOT_BYTES + 9 * SM::BOXB);
  };
  auto issue = [&](int q) {  // march index q -> ring slot q & 3
    const int s = q & 3, plane = ((q % nth) + nth) % nth;
    mbar_expect_tx(&bar[s], SM::TX);
    unsigned char *base = smem + (size_t)s * SM::SLOT_BYTES;
    for (int f = 0; f < 9; f++) tma_load_4d(base + f * SM::BOXB, &maps.f[f], k0 - HX, i0 - 1, plane, cs, &bar[s]);
    tma_load_4d(base + 9 * SM::BOXB, &maps.id, k0 - 8, i0 - 1, plane, cs, &bar[s]);
  };
  int issued_hi, waited_hi = -3;
  bool ok = true, failed = false;
  auto wait_q = [&](int q) {  // only a completed wait advances the bookkeeping
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

  const float dtv = p.dtv, dts = p.dts, idr = p.inv_dr, idz = p.inv_dz, idth = p.inv_dth;
  const float *m_rho = p.m_rho, *m_imu = p.m_imu;
  const float2 *m_lam = p.m_lam;
  T *vnxt[3] = {(T *)fp.fo[F_VR], (T *)fp.fo[F_VP], (T *)fp.fo[F_VZ]};
  const int i = i0 - 1 + row;  // this thread's radial index

  // Per-point constants of a velocity point at tile row r, depth k: they do
  // not change along the theta march, so each thread builds them once.
  struct VCtx {
    int ii, k, x, xi;     // radial index, depth, offsets in a field box / ID box
    long long cb, crb, czb;  // global, radial-slab and z-slab offsets without the plane term
    int kz;
    bool rp, zp;
    float inv_ri, inv_rh;
    float4 ab, aq, abz;
  };
  auto make_ctx = [&](int r, int k) {
    VCtx v;
    v.ii = i0 - 1 + r;
    v.k = k;
    v.x = r * BW + (k - k0 + HX);
    v.xi = r * BWI + (k - k0 + 8);
    const int iic = min(max(v.ii, 0), NR - 1), kc = min(max(k, 0), NZ - 1);
    v.cb = (long long)v.ii * NZp + k;
    v.rp = v.ii >= nr_p && v.ii < NR;
    v.crb = v.rp ? (long long)(v.ii - nr_p) * NZp + k : 0;
    v.zp = (k >= 0 && k < pz) || (k >= NZ - pz && k < NZ);
    v.kz = k < pz ? k : k - (NZ - 2 * pz);
    v.czb = (long long)iic * (2 * pz) + v.kz;
    v.inv_ri = __ldg(p.inv_ri + iic);
    v.inv_rh = __ldg(p.inv_rh + iic);
    v.ab = __ldg(p.ab_r + iic);
    v.aq = __ldg(p.ab_q + iic);
    v.abz = v.zp ? __ldg(p.ab_z + kc) : make_float4(0.f, 1.f, 0.f, 1.f);
    return v;
  };
  const long long pr_plane = (long long)p.pml_r * NZp, pz_plane = (long long)NR * 2 * pz;

  // velocity component c at the point of `v` in plane `plane`, with ring slots
  // (sm1, s0, sp1) = planes (m-1, m, m+1); writes the owned value and memory
  // variables, returns the new value (0 at walls and outside the grid).
  auto vel_point = [&](int c, const VCtx &v, int plane, bool own, int sm1, int s0, int sp1) -> float {
    const int ii = v.ii, k = v.k, x = v.x, xi = v.xi;
    const long long cr = plane * pr_plane + v.crb, cz = plane * pz_plane + v.czb;
    const T *S0 = slot_field(s0, 0);
    const int F = SM::BOX_ELEMS;  // stride between field boxes of one slot
    const uint16_t *I0 = slot_ids(s0);
    float out;
    if (c == 0) {  // v_r at (r_i, theta_j, z_k): i >= 1
      if (ii < 1 || ii >= NR || k >= NZ) return 0.f;
      const float srr_c = sld(S0 + 3 * F + x), srr_m = sld(S0 + 3 * F + x - BW);
      const float spp_c = sld(S0 + 4 * F + x), spp_m = sld(S0 + 4 * F + x - BW);
      float Dr = (srr_c - srr_m) * idr;
      float Q = (0.5f * (srr_c + srr_m) - 0.5f * (spp_c + spp_m) + (sld(S0 + 6 * F + x) - sld(slot_field(sm1, 6) + x)) * idth) *
                v.inv_ri;
      float Dz = (sld(S0 + 8 * F + x) - sld(S0 + 8 * F + x - 1)) * idz;
      if (v.rp) {
        const float ps = v.ab.y * p.psr[R_VR][cr] + v.ab.x * Dr;
        const float qs = v.aq.y * p.psr[Q_VR][cr] + v.aq.x * Q;
        if (own) {
          fp.psr_o[R_VR][cr] = ps;
          fp.psr_o[Q_VR][cr] = qs;
        }
        Dr += ps;
        Q += qs;
      }
      if (v.zp) {
        const float ps = v.abz.y * p.psz[Z_VR][cz] + v.abz.x * Dz;
        if (own) fp.psz_o[Z_VR][cz] = ps;
        Dz += ps;
      }
      const float rho = __ldg(m_rho + I0[xi]) + __ldg(m_rho + I0[xi - BWI]);
      out = sld(S0 + x) + vel_coef(dtv, rho) * (Dr + Q + Dz);
    } else if (c == 1) {  // v_phi at (r_{i+1/2}, theta_{j+1/2}, z_k)
      if (ii < 0 || ii >= NR || k >= NZ) return 0.f;
      const float s1 = sld(S0 + 6 * F + x + BW), s0v = sld(S0 + 6 * F + x);
      float Dr = (s1 - s0v) * idr;
      float Q = ((s1 + s0v) + (sld(slot_field(sp1, 4) + x) - sld(S0 + 4 * F + x)) * idth) * v.inv_rh;
      float Dz = (sld(S0 + 7 * F + x) - sld(S0 + 7 * F + x - 1)) * idz;
      if (v.rp) {
        const float ps = v.ab.w * p.psr[R_VP][cr] + v.ab.z * Dr;
        const float qs = v.aq.w * p.psr[Q_VP][cr] + v.aq.z * Q;
        if (own) {
          fp.psr_o[R_VP][cr] = ps;
          fp.psr_o[Q_VP][cr] = qs;
        }
        Dr += ps;
        Q += qs;
      }
      if (v.zp) {
        const float ps = v.abz.y * p.psz[Z_VP][cz] + v.abz.x * Dz;
        if (own) fp.psz_o[Z_VP][cz] = ps;
        Dz += ps;
      }
      const float rho = __ldg(m_rho + I0[xi]) + __ldg(m_rho + slot_ids(sp1)[xi]);
      out = sld(S0 + F + x) + vel_coef(dtv, rho) * (Dr + Q + Dz);
    } else {  // v_z at (r_{i+1/2}, theta_j, z_{k+1/2}); the last half-node is a wall
      if (ii < 0 || ii >= NR || k < 0 || k + 1 >= NZ) return 0.f;
      const float s1 = sld(S0 + 8 * F + x + BW), s0v = sld(S0 + 8 * F + x);
      float Dr = (s1 - s0v) * idr;
      float Q = (0.5f * (s1 + s0v) + (sld(S0 + 7 * F + x) - sld(slot_field(sm1, 7) + x)) * idth) * v.inv_rh;
      float Dz = (sld(S0 + 5 * F + x + 1) - sld(S0 + 5 * F + x)) * idz;
      if (v.rp) {
        const float ps = v.ab.w * p.psr[R_VZ][cr] + v.ab.z * Dr;
        const float qs = v.aq.w * p.psr[Q_VZ][cr] + v.aq.z * Q;
        if (own) {
          fp.psr_o[R_VZ][cr] = ps;
          fp.psr_o[Q_VZ][cr] = qs;
        }
        Dr += ps;
        Q += qs;
      }
      if (v.zp) {
        const float ps = v.abz.w * p.psz[Z_VZ][cz] + v.abz.z * Dz;
        if (own) fp.psz_o[Z_VZ][cz] = ps;
        Dz += ps;
      }
      const float rho = __ldg(m_rho + I0[xi]) + __ldg(m_rho + I0[xi + 1]);
      out = sld(S0 + 2 * F + x) + vel_coef(dtv, rho) * (Dr + Q + Dz);
    }
    if (own && k < NZp) gst(vnxt[c] + plane * pl + v.cb, out);
    return out;
  };
  // this thread's main point and, for the row's edge lanes, its halo point
  const VCtx vmain = make_ctx(row, k0 + lane);
  const VCtx vhalo = make_ctx(row, lane == 0 ? k0 - 1 : k0 + ZT);

  for (int m = -1; m <= nth; m++) {
    // prefetch plane m + 2 into the slot freed at the end of the previous iteration
    if (m + 2 <= nth && m + 2 > issued_hi) {
      if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(m + 2);
      }
      issued_hi = m + 2;
    }
    if (ok && m + 1 <= nth && m + 1 > waited_hi) ok = wait_q(m + 1);

    const int sm1 = (m - 1) & 3, s0 = m & 3, sp1 = (m + 1) & 3;
    if (m <= nth - 1) {
      // ---------------- velocity half-step of plane m on the tile plus halo
      const int plane = ((m % nth) + nth) % nth;
      const bool own_plane = m >= 0;
      float *V = vr_ring + (((m % 3) + 3) % 3) * 3 * BR * VW;
      {
        const bool own_rz = own_plane && row >= 1 && row <= RT;
        // v_r on rows 1 .. RT+1, v_phi and v_z on rows 0 .. RT
        V[(0 * BR + row) * VW + lane + 1] = row >= 1 ? vel_point(0, vmain, plane, own_rz, sm1, s0, sp1) : 0.f;
        V[(1 * BR + row) * VW + lane + 1] = row <= RT ? vel_point(1, vmain, plane, own_rz, sm1, s0, sp1) : 0.f;
        V[(2 * BR + row) * VW + lane + 1] = row <= RT ? vel_point(2, vmain, plane, own_rz, sm1, s0, sp1) : 0.f;
        // halo columns, one row per warp pair: v_z at k0-1 by lane 0, v_r and
        // v_phi at k0+ZT by lane 63 (recomputed, never written)
        if (lane == 0) {
          V[(2 * BR + row) * VW + 0] = row <= RT ? vel_point(2, vhalo, plane, false, sm1, s0, sp1) : 0.f;
        } else if (lane == 63) {
          V[(0 * BR + row) * VW + ZT + 1] = row >= 1 ? vel_point(0, vhalo, plane, false, sm1, s0, sp1) : 0.f;
          V[(1 * BR + row) * VW + ZT + 1] = row <= RT ? vel_point(1, vhalo, plane, false, sm1, s0, sp1) : 0.f;
        }
      }
      if (m == 0) {
        __syncthreads();
        for (int q = tid; q < 3 * BR * VW; q += NT) vsave[q] = V[q];
      }
    }
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }

    if (m >= 1 && row >= 1 && row <= RT && i < NR) {
      // ---------------- stress step of plane m-1 on the owned tile (one column per thread)
      const int plane = m - 1;
      const int k = k0 + lane;
      const float *Va = vr_ring + (((m - 2) % 3 + 3) % 3) * 3 * BR * VW;      // plane m-2
      const float *Vb = vr_ring + ((m - 1) % 3) * 3 * BR * VW;                // plane m-1
      const float *Vc = (m == nth) ? vsave : vr_ring + (m % 3) * 3 * BR * VW;  // plane m (0 at the end)
      const int v = row * VW + lane + 1;  // (row, k) in the velocity ring
      const int x = row * BW + lane + HX, xi = row * BWI + lane + 8;
      if (k < NZp) {
        const long long c = (long long)plane * pl + (long long)i * NZp + k;
        float o[6];
#pragma unroll
        for (int f = 0; f < 6; f++) o[f] = sld(slot_field(sm1, 3 + f) + x);  // s^n of plane m-1
        if (k < NZ) {
          const uint16_t *Im = slot_ids(sm1), *Ij = slot_ids(s0);
          const bool rpm = vmain.rp, zpm = vmain.zp;
          const long long cr = plane * pr_plane + vmain.crb, cz = plane * pz_plane + vmain.czb;
          const float inv_rh = vmain.inv_rh, inv_ri = vmain.inv_ri;
          const float4 ab = vmain.ab, aq = vmain.aq, abz = vmain.abz;
          const float imu_c = __ldg(m_imu + Im[xi]), imu_m = __ldg(m_imu + Im[xi - BWI]);
          // normal stresses
          {
            const float vr0 = Vb[v], vr1 = Vb[v + VW];
            float err = (vr1 - vr0) * idr;
            float epp = ((Vb[BR * VW + v] - Va[BR * VW + v]) * idth + 0.5f * (vr0 + vr1)) * inv_rh;
            float ezz = (Vb[2 * BR * VW + v] - Vb[2 * BR * VW + v - 1]) * idz;
            if (rpm) {
              const float ps = ab.w * p.psr[R_ERR][cr] + ab.z * err;
              const float qs = aq.w * p.psr[Q_EPP][cr] + aq.z * epp;
              fp.psr_o[R_ERR][cr] = ps;
              fp.psr_o[Q_EPP][cr] = qs;
              err += ps;
              epp += qs;
            }
            if (zpm) {
              const float ps = abz.y * p.psz[Z_EZZ][cz] + abz.x * ezz;
              fp.psz_o[Z_EZZ][cz] = ps;
              ezz += ps;
            }
            const float2 ll = __ldg(m_lam + Im[xi]);  // {lambda, lambda + 2 mu}
            float src = 0.f;
            if (i == p.src_i && k == p.src_k && (p.src_j < 0 || p.src_j == plane)) {
              const int n = *p.step;
              src = n < p.n_wav ? __ldg(p.wav + n) : 0.f;
            }
            o[0] += dts * (ll.y * err + ll.x * (epp + ezz)) + src;
            o[1] += dts * (ll.y * epp + ll.x * (err + ezz)) + src;
            o[2] += dts * (ll.y * ezz + ll.x * (err + epp)) + src;
          }
          if (i >= 1) {
            // s_rphi at (r_i, theta_{j+1/2}, z_k)
            float gr = (Vb[BR * VW + v] - Vb[BR * VW + v - VW]) * idr;
            float Q = ((Vc[v] - Vb[v]) * idth - 0.5f * (Vb[BR * VW + v] + Vb[BR * VW + v - VW])) * inv_ri;
            if (rpm) {
              const float ps = ab.y * p.psr[R_GRP][cr] + ab.x * gr;
              const float qs = aq.y * p.psr[Q_GRP][cr] + aq.x * Q;
              fp.psr_o[R_GRP][cr] = ps;
              fp.psr_o[Q_GRP][cr] = qs;
              gr += ps;
              Q += qs;
            }
            const float mu = mu_harm(imu_m + imu_c + __ldg(m_imu + Ij[xi - BWI]) + __ldg(m_imu + Ij[xi]));
            o[3] += dts * mu * (gr + Q);
          }
          if (k + 1 < NZ) {
            const float imu_c1 = __ldg(m_imu + Im[xi + 1]);
            if (i >= 1) {
              // s_rz at (r_i, theta_j, z_{k+1/2})
              float gz = (Vb[v + 1] - Vb[v]) * idz;
              float gr = (Vb[2 * BR * VW + v] - Vb[2 * BR * VW + v - VW]) * idr;
              if (zpm) {
                const float ps = abz.w * p.psz[Z_GRZ][cz] + abz.z * gz;
                fp.psz_o[Z_GRZ][cz] = ps;
                gz += ps;
              }
              if (rpm) {
                const float ps = ab.y * p.psr[R_GRZ][cr] + ab.x * gr;
                fp.psr_o[R_GRZ][cr] = ps;
                gr += ps;
              }
              const float mu = mu_harm(imu_m + imu_c + __ldg(m_imu + Im[xi - BWI + 1]) + imu_c1);
              o[5] += dts * mu * (gz + gr);
            }
            // s_phiz at (r_{i+1/2}, theta_{j+1/2}, z_{k+1/2})
            {
              float Q = (Vc[2 * BR * VW + v] - Vb[2 * BR * VW + v]) * idth * inv_rh;
              float gz = (Vb[BR * VW + v + 1] - Vb[BR * VW + v]) * idz;
              if (rpm) {
                const float qs = aq.w * p.psr[Q_GPZ][cr] + aq.z * Q;
                fp.psr_o[Q_GPZ][cr] = qs;
                Q += qs;
              }
              if (zpm) {
                const float ps = abz.w * p.psz[Z_GPZ][cz] + abz.z * gz;
                fp.psz_o[Z_GPZ][cz] = ps;
                gz += ps;
              }
              const float mu = mu_harm(imu_c + __ldg(m_imu + Ij[xi]) + imu_c1 + __ldg(m_imu + Ij[xi + 1]));
              o[4] += dts * mu * (Q + gz);
            }
          }
        }
        T *so[6] = {(T *)fp.fo[F_SRR], (T *)fp.fo[F_SPP], (T *)fp.fo[F_SZZ],
                    (T *)fp.fo[F_SRP], (T *)fp.fo[F_SPZ], (T *)fp.fo[F_SRZ]};
#pragma unroll
        for (int f = 0; f < 6; f++) gst(so[f] + c, o[f]);
      }
    }
    __syncthreads();
  }
  if (failed) {
    if (tid == 0) atomicOr(fp.status, 2);
    // drain the copies this block still has in flight (bounded) before leaving
    for (int q = waited_hi + 1; q <= issued_hi; q++) {
      const int s = q & 3;
      if (mbar_wait(&bar[s], (phase >> s) & 1u)) phase ^= 1u << s;
    }
    __syncthreads();
  }
}

template <typename T, int RT, int ZT>
__global__ void __launch_bounds__(FusedSmem<T, RT, ZT>::NT, FusedSmem<T, RT, ZT>::MINB) fused_step(const __grid_constant__ FusedMaps maps,
                                                                       const __grid_constant__ FusedParams fp) {
  using SM = FusedSmem<T, RT, ZT>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + SM::BAR_OFF);
  if (threadIdx.x == 0) {
    for (int s = 0; s < 4; s++) mbar_init(&bar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t phase = 0;  // bit s: parity of the next completion of slot s
  fused_tile<T, RT, ZT>(maps, fp, 0, blockIdx.x * RT, blockIdx.y * ZT, smem, bar, phase);
}

template <typename T, int RT, int ZT>
static cudaError_t launch_fused_t(const FusedMaps &maps, const FusedParams &fp, cudaStream_t s) {
  using SM = FusedSmem<T, RT, ZT>;
  auto kern = fused_step<T, RT, ZT>;
  static bool attr_done[16] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 16 && !attr_done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::BYTES);
    if (e != cudaSuccess) return e;
    attr_done[dev] = true;
  }
  dim3 grd((fp.k.NR + RT - 1) / RT, (fp.k.NZ + ZT - 1) / ZT);
  kern<<<grd, SM::NT, SM::BYTES, s>>>(maps, fp);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_fused_rt(int rt, const FusedMaps &maps, const FusedParams &fp, cudaStream_t s) {
  switch (rt) {
    case 2: return launch_fused_t<T, 2, 64>(maps, fp, s);
    case 4: return launch_fused_t<T, 4, 64>(maps, fp, s);
    case 6: return launch_fused_t<T, 6, 64>(maps, fp, s);
    case 8: return launch_fused_t<T, 8, 64>(maps, fp, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_fused(int storage, int rt, const FusedMaps &maps, const FusedParams &fp, cudaStream_t s) {
  switch (storage) {
    case 0: return launch_fused_rt<float>(rt, maps, fp, s);
    case 1: return launch_fused_rt<__nv_bfloat16>(rt, maps, fp, s);
    case 2: return launch_fused_rt<__half>(rt, maps, fp, s);
  }
  return cudaErrorInvalidValue;
}

size_t fused_smem_bytes(int storage, int rt) {
  auto pick = [&](auto tag) -> size_t {
    using T = decltype(tag);
    switch (rt) {
      case 2: return FusedSmem<T, 2, 64>::BYTES;
      case 4: return FusedSmem<T, 4, 64>::BYTES;
      case 6: return FusedSmem<T, 6, 64>::BYTES;
      case 8: return FusedSmem<T, 8, 64>::BYTES;
    }
    return 0;
  };
  if (storage == 0) return pick(float{});
  if (storage == 1) return pick(__nv_bfloat16{});
  return pick(__half{});
}

int fused_box_x(int storage) { return storage == 0 ? 64 + 8 : 64 + 16; }
int fused_pad_x(int storage) { return storage == 0 ? 4 : 8; }

}  // namespace cwell
