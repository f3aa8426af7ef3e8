// Fused path: one kernel per leapfrog step (velocity half-step and stress
// step together), double-buffered state.
//
// A block owns an (r, z) tile of RT rows x ZT cells and marches over all
// nth azimuthal planes.  For march index m it
//   1. has the stress state s^n of planes m-1, m, m+1 in a 4-slot shared
//      memory ring (tile plus one cell of halo in r and z), brought in by TMA
//      (cp.async.bulk.tensor, mbarrier completion) one plane ahead;
//   2. computes v^{n+1/2} of plane m on the tile plus halo (the halo values
//      are recomputed here instead of exchanged), keeps it in a 3-plane
//      ring, and writes the owned part (and the owned PML memory variables);
//   3. computes s^{n+1} of plane m-1 from the velocity planes m-2, m-1, m and
//      writes it (plus the source increment and PML memory variables).
// The march starts at m = -1 so the periodic neighbour of plane 0 exists;
// velocity plane 0 is kept for the last stress plane.  Reads come from the
// "cur" buffers, writes go to "nxt", so recomputed halos never race with the
// owners' writes.  DRAM traffic per cell-update is the minimum: every field
// read once and written once, plus the material ID.
//
// Every mbarrier wait is bounded; a wait that gives up sets bit 1 of the
// status word, waits (bounded) for the block's copies still in flight and
// returns, so a broken launch reports SIM_ETIMEOUT instead of hanging.
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

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ float sld(const float *p) { return *p; }
__device__ __forceinline__ float sld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ float sld(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ void gst(float *p, float v) { *p = v; }
__device__ __forceinline__ void gst(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void gst(__half *p, float v) { *p = __float2half_rn(v); }

template <typename T, int RT, int ZT>
struct FusedSmem {
  static constexpr int HX = Pad<T>::HX;
  static constexpr int BR = RT + 2;         // rows i0-1 .. i0+RT
  static constexpr int BW = ZT + 2 * HX;    // z from k0-HX
  static constexpr int BWI = ZT + 16;       // IDs: z from k0-8
  static constexpr int VW = ZT + 2;         // velocity ring: z from k0-1
  // every TMA destination starts on a 128-byte boundary
  static constexpr int BOXB = (BR * BW * (int)sizeof(T) + 127) / 128 * 128;
  static constexpr int IDB = (BR * BWI * 2 + 127) / 128 * 128;
  static constexpr int SIG_SLOT = 6 * BOXB / (int)sizeof(T);  // elements of T per ring slot
  static constexpr int BOX_ELEMS = BOXB / (int)sizeof(T);
  static constexpr size_t SIG_BYTES = (size_t)4 * 6 * BOXB;
  static constexpr size_t ID_BYTES = (size_t)4 * IDB;
  static constexpr size_t V_BYTES = (size_t)4 * 3 * BR * VW * 4;  // 3 ring slots + saved plane 0
  static constexpr size_t BAR_OFF = (SIG_BYTES + ID_BYTES + V_BYTES + 127) / 128 * 128;
  static constexpr size_t BYTES = BAR_OFF + 4 * 8 + 128;  // + slack for aligning the base
  static constexpr uint32_t TX = (uint32_t)(6 * BR * BW * sizeof(T) + BR * BWI * 2);
};

template <typename T, int RT, int ZT, int NT>
__global__ void __launch_bounds__(NT) fused_step(const __grid_constant__ FusedMaps maps,
                                                 const __grid_constant__ FusedParams fp) {
  using SM = FusedSmem<T, RT, ZT>;
  constexpr int HX = SM::HX, BR = SM::BR, BW = SM::BW, BWI = SM::BWI, VW = SM::VW;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  T *sig = reinterpret_cast<T *>(smem);
  uint16_t *ids = reinterpret_cast<uint16_t *>(smem + SM::SIG_BYTES);
  float *vr_ring = reinterpret_cast<float *>(smem + SM::SIG_BYTES + SM::ID_BYTES);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + SM::BAR_OFF);

  const KParams &p = fp.k;
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * RT, k0 = blockIdx.y * ZT;
  const int nth = p.nth, NR = p.NR, NZ = p.NZ, NZp = p.NZp;
  const long long pl = p.plane;
  const int pz = p.pml_z;

  auto S = [&](int slot, int f, int r, int k) -> float {
    return sld(sig + (size_t)slot * SM::SIG_SLOT + f * SM::BOX_ELEMS + r * BW + (k - k0 + HX));
  };
  auto ID = [&](int slot, int r, int k) -> int { return ids[slot * (SM::IDB / 2) + r * BWI + (k - k0 + 8)]; };
  auto V = [&](int slot, int c, int r, int k) -> float & {
    return vr_ring[((slot * 3 + c) * BR + r) * VW + (k - k0 + 1)];
  };
  const T *vcur[3] = {(const T *)p.f[F_VR], (const T *)p.f[F_VP], (const T *)p.f[F_VZ]};
  T *vnxt[3] = {(T *)fp.fo[F_VR], (T *)fp.fo[F_VP], (T *)fp.fo[F_VZ]};

  if (tid == 0) {
    for (int s = 0; s < 4; s++) mbar_init(&bar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  uint32_t phase = 0;  // bit s: parity of the next completion of slot s
  auto issue = [&](int q) {  // march index q -> slot q & 3
    const int s = q & 3, plane = ((q % nth) + nth) % nth;
    mbar_expect_tx(&bar[s], SM::TX);
    for (int f = 0; f < 6; f++)
      tma_load_3d(sig + (size_t)s * SM::SIG_SLOT + f * SM::BOX_ELEMS, &maps.sig[f], k0 - HX, i0 - 1, plane, &bar[s]);
    tma_load_3d(ids + (size_t)s * (SM::IDB / 2), &maps.id, k0 - 8, i0 - 1, plane, &bar[s]);
  };
  int issued_hi = -3;  // highest march index issued
  int waited_hi = -3;  // highest march index waited
  if (tid == 0) {
    for (int q = -2; q <= 1; q++) issue(q);
  }
  issued_hi = 1;
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
  ok = wait_q(-2);
  if (ok) ok = wait_q(-1);

  const float dtv = p.dtv, dts = p.dts, idr = p.inv_dr, idz = p.inv_dz, idth = p.inv_dth;
  const int nr_p = p.nr;
  float *vsave = vr_ring + 3 * 3 * BR * VW;

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
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }

    const int sm1 = (m - 1) & 3, s0 = m & 3, sp1 = (m + 1) & 3;
    if (m <= nth - 1) {
      // ---------------- velocity half-step of plane m on the tile plus halo
      const int plane = ((m % nth) + nth) % nth;
      const bool own_plane = m >= 0;
      const int vs = ((m % 3) + 3) % 3;
      // v_r: rows r' = 1 .. RT+1 (i = i0 .. i0+RT), z k0 .. k0+ZT
      for (int q = tid; q < (RT + 1) * (ZT + 1); q += NT) {
        const int r = 1 + q / (ZT + 1), k = k0 + q % (ZT + 1), i = i0 - 1 + r;
        float out = 0.f;
        if (i >= 1 && i < NR && k < NZ) {
          const long long c = (long long)plane * pl + (long long)i * NZp + k;
          const float srr_c = S(s0, 0, r, k), srr_m = S(s0, 0, r - 1, k);
          const float spp_c = S(s0, 1, r, k), spp_m = S(s0, 1, r - 1, k);
          float Dr = (srr_c - srr_m) * idr;
          float Q = (0.5f * (srr_c + srr_m) - 0.5f * (spp_c + spp_m) + (S(s0, 3, r, k) - S(sm1, 3, r, k)) * idth) *
                    __ldg(p.inv_ri + i);
          float Dz = (S(s0, 5, r, k) - S(s0, 5, r, k - 1)) * idz;
          const bool own = own_plane && r <= RT && k < k0 + ZT;
          if (i >= nr_p) {
            const long long cr = ((long long)plane * p.pml_r + (i - nr_p)) * NZp + k;
            const float4 ab = __ldg(p.ab_r + i), aq = __ldg(p.ab_q + i);
            float ps = ab.y * p.psr[R_VR][cr] + ab.x * Dr;
            float qs = aq.y * p.psr[Q_VR][cr] + aq.x * Q;
            if (own) {
              fp.psr_o[R_VR][cr] = ps;
              fp.psr_o[Q_VR][cr] = qs;
            }
            Dr += ps;
            Q += qs;
          }
          if (k < pz || k >= NZ - pz) {
            const int kz = k < pz ? k : k - (NZ - 2 * pz);
            const long long cz = ((long long)plane * NR + i) * (2 * pz) + kz;
            const float4 abz = __ldg(p.ab_z + k);
            float ps = abz.y * p.psz[Z_VR][cz] + abz.x * Dz;
            if (own) fp.psz_o[Z_VR][cz] = ps;
            Dz += ps;
          }
          const float rho = __ldg(p.mat + ID(s0, r, k)).x + __ldg(p.mat + ID(s0, r - 1, k)).x;
          out = St<T>::ld1(vcur[0] + c) + 2.f * dtv / rho * (Dr + Q + Dz);
        }
        V(vs, 0, r, k) = out;
        if (own_plane && r <= RT && i < NR && k < NZp && k < k0 + ZT)
          gst(vnxt[0] + (long long)plane * pl + (long long)i * NZp + k, out);
      }
      // v_phi: rows r' = 0 .. RT (i = i0-1 .. i0+RT-1), z k0 .. k0+ZT
      for (int q = tid; q < (RT + 1) * (ZT + 1); q += NT) {
        const int r = q / (ZT + 1), k = k0 + q % (ZT + 1), i = i0 - 1 + r;
        float out = 0.f;
        if (i >= 0 && i < NR && k < NZ) {
          const long long c = (long long)plane * pl + (long long)i * NZp + k;
          const float s1 = S(s0, 3, r + 1, k), s0v = S(s0, 3, r, k);
          float Dr = (s1 - s0v) * idr;
          float Q = ((s1 + s0v) + (S(sp1, 1, r, k) - S(s0, 1, r, k)) * idth) * __ldg(p.inv_rh + i);
          float Dz = (S(s0, 4, r, k) - S(s0, 4, r, k - 1)) * idz;
          const bool own = own_plane && r >= 1 && k < k0 + ZT;
          if (i >= nr_p) {
            const long long cr = ((long long)plane * p.pml_r + (i - nr_p)) * NZp + k;
            const float4 ab = __ldg(p.ab_r + i), aq = __ldg(p.ab_q + i);
            float ps = ab.w * p.psr[R_VP][cr] + ab.z * Dr;
            float qs = aq.w * p.psr[Q_VP][cr] + aq.z * Q;
            if (own) {
              fp.psr_o[R_VP][cr] = ps;
              fp.psr_o[Q_VP][cr] = qs;
            }
            Dr += ps;
            Q += qs;
          }
          if (k < pz || k >= NZ - pz) {
            const int kz = k < pz ? k : k - (NZ - 2 * pz);
            const long long cz = ((long long)plane * NR + i) * (2 * pz) + kz;
            const float4 abz = __ldg(p.ab_z + k);
            float ps = abz.y * p.psz[Z_VP][cz] + abz.x * Dz;
            if (own) fp.psz_o[Z_VP][cz] = ps;
            Dz += ps;
          }
          const float rho = __ldg(p.mat + ID(s0, r, k)).x + __ldg(p.mat + ID(sp1, r, k)).x;
          out = St<T>::ld1(vcur[1] + c) + 2.f * dtv / rho * (Dr + Q + Dz);
        }
        V(vs, 1, r, k) = out;
        if (own_plane && r >= 1 && i < NR && k < NZp && k < k0 + ZT)
          gst(vnxt[1] + (long long)plane * pl + (long long)i * NZp + k, out);
      }
      // v_z: rows r' = 0 .. RT, z k0-1 .. k0+ZT-1
      for (int q = tid; q < (RT + 1) * (ZT + 1); q += NT) {
        const int r = q / (ZT + 1), k = k0 - 1 + q % (ZT + 1), i = i0 - 1 + r;
        float out = 0.f;
        if (i >= 0 && i < NR && k >= 0 && k + 1 < NZ) {
          const long long c = (long long)plane * pl + (long long)i * NZp + k;
          const float s1 = S(s0, 5, r + 1, k), s0v = S(s0, 5, r, k);
          float Dr = (s1 - s0v) * idr;
          float Q = (0.5f * (s1 + s0v) + (S(s0, 4, r, k) - S(sm1, 4, r, k)) * idth) * __ldg(p.inv_rh + i);
          float Dz = (S(s0, 2, r, k + 1) - S(s0, 2, r, k)) * idz;
          const bool own = own_plane && r >= 1 && k >= k0;
          if (i >= nr_p) {
            const long long cr = ((long long)plane * p.pml_r + (i - nr_p)) * NZp + k;
            const float4 ab = __ldg(p.ab_r + i), aq = __ldg(p.ab_q + i);
            float ps = ab.w * p.psr[R_VZ][cr] + ab.z * Dr;
            float qs = aq.w * p.psr[Q_VZ][cr] + aq.z * Q;
            if (own) {
              fp.psr_o[R_VZ][cr] = ps;
              fp.psr_o[Q_VZ][cr] = qs;
            }
            Dr += ps;
            Q += qs;
          }
          if (k < pz || k >= NZ - pz) {
            const int kz = k < pz ? k : k - (NZ - 2 * pz);
            const long long cz = ((long long)plane * NR + i) * (2 * pz) + kz;
            const float4 abz = __ldg(p.ab_z + k);
            float ps = abz.w * p.psz[Z_VZ][cz] + abz.z * Dz;
            if (own) fp.psz_o[Z_VZ][cz] = ps;
            Dz += ps;
          }
          const float rho = __ldg(p.mat + ID(s0, r, k)).x + __ldg(p.mat + ID(s0, r, k + 1)).x;
          out = St<T>::ld1(vcur[2] + c) + 2.f * dtv / rho * (Dr + Q + Dz);
        }
        V(vs, 2, r, k) = out;
        if (own_plane && r >= 1 && k >= k0 && i < NR && k < NZp)
          gst(vnxt[2] + (long long)plane * pl + (long long)i * NZp + k, out);
      }
      if (m == 0) {
        __syncthreads();
        for (int q = tid; q < 3 * BR * VW; q += NT) vsave[q] = vr_ring[vs * 3 * BR * VW + q];
      }
    }
    __syncthreads();

    if (m >= 1) {
      // ---------------- stress step of plane m-1 on the owned tile
      const int plane = m - 1;
      const int va = ((m - 2) % 3 + 3) % 3, vb = (m - 1) % 3, vcx = m % 3;
      float *vslot_c = (m == nth) ? vsave : vr_ring + vcx * 3 * BR * VW;  // plane m (0 at the end)
      auto Vc = [&](int c, int r, int k) -> float { return vslot_c[(c * BR + r) * VW + (k - k0 + 1)]; };
      const int n = *p.step;
      for (int q = tid; q < RT * ZT; q += NT) {
        const int r = 1 + q / ZT, k = k0 + q % ZT, i = i0 - 1 + r;
        if (i >= NR || k >= NZp) continue;
        const long long c = (long long)plane * pl + (long long)i * NZp + k;
        float o[6];
#pragma unroll
        for (int f = 0; f < 6; f++) o[f] = S(sm1, f, r, k);  // s^n of plane m-1
        if (k < NZ) {
          const bool rpm = i >= nr_p;
          const long long cr = rpm ? ((long long)plane * p.pml_r + (i - nr_p)) * NZp + k : 0;
          const bool zpm = k < pz || k >= NZ - pz;
          const int kz = k < pz ? k : k - (NZ - 2 * pz);
          const long long cz = ((long long)plane * NR + i) * (2 * pz) + kz;
          const float4 ab = __ldg(p.ab_r + i), aq = __ldg(p.ab_q + i);
          const float4 abz = __ldg(p.ab_z + k);
          const float inv_rh = __ldg(p.inv_rh + i), inv_ri = __ldg(p.inv_ri + i);
          // normal stresses
          {
            const float vr0 = V(vb, 0, r, k), vr1 = V(vb, 0, r + 1, k);
            float err = (vr1 - vr0) * idr;
            float epp = ((V(vb, 1, r, k) - V(va, 1, r, k)) * idth + 0.5f * (vr0 + vr1)) * inv_rh;
            float ezz = (V(vb, 2, r, k) - V(vb, 2, r, k - 1)) * idz;
            if (rpm) {
              float ps = ab.w * p.psr[R_ERR][cr] + ab.z * err;
              float qs = aq.w * p.psr[Q_EPP][cr] + aq.z * epp;
              fp.psr_o[R_ERR][cr] = ps;
              fp.psr_o[Q_EPP][cr] = qs;
              err += ps;
              epp += qs;
            }
            if (zpm) {
              float ps = abz.y * p.psz[Z_EZZ][cz] + abz.x * ezz;
              fp.psz_o[Z_EZZ][cz] = ps;
              ezz += ps;
            }
            const float4 mt = __ldg(p.mat + ID(sm1, r, k));
            const float l = mt.y, l2m = mt.y + 2.f * mt.z;
            float src = 0.f;
            if (i == p.src_i && k == p.src_k && (p.src_j < 0 || p.src_j == plane))
              src = n < p.n_wav ? __ldg(p.wav + n) : 0.f;
            o[0] += dts * (l2m * err + l * (epp + ezz)) + src;
            o[1] += dts * (l2m * epp + l * (err + ezz)) + src;
            o[2] += dts * (l2m * ezz + l * (err + epp)) + src;
          }
          if (i >= 1) {
            // s_rphi
            float gr = (V(vb, 1, r, k) - V(vb, 1, r - 1, k)) * idr;
            float Q = ((Vc(0, r, k) - V(vb, 0, r, k)) * idth - 0.5f * (V(vb, 1, r, k) + V(vb, 1, r - 1, k))) * inv_ri;
            if (rpm) {
              float ps = ab.y * p.psr[R_GRP][cr] + ab.x * gr;
              float qs = aq.y * p.psr[Q_GRP][cr] + aq.x * Q;
              fp.psr_o[R_GRP][cr] = ps;
              fp.psr_o[Q_GRP][cr] = qs;
              gr += ps;
              Q += qs;
            }
            const float mu = 4.f / (__ldg(p.mat + ID(sm1, r - 1, k)).w + __ldg(p.mat + ID(sm1, r, k)).w +
                                    __ldg(p.mat + ID(s0, r - 1, k)).w + __ldg(p.mat + ID(s0, r, k)).w);
            o[3] += dts * mu * (gr + Q);
          }
          if (k + 1 < NZ) {
            if (i >= 1) {
              // s_rz
              float gz = (V(vb, 0, r, k + 1) - V(vb, 0, r, k)) * idz;
              float gr = (V(vb, 2, r, k) - V(vb, 2, r - 1, k)) * idr;
              if (zpm) {
                float ps = abz.w * p.psz[Z_GRZ][cz] + abz.z * gz;
                fp.psz_o[Z_GRZ][cz] = ps;
                gz += ps;
              }
              if (rpm) {
                float ps = ab.y * p.psr[R_GRZ][cr] + ab.x * gr;
                fp.psr_o[R_GRZ][cr] = ps;
                gr += ps;
              }
              const float mu = 4.f / (__ldg(p.mat + ID(sm1, r - 1, k)).w + __ldg(p.mat + ID(sm1, r, k)).w +
                                      __ldg(p.mat + ID(sm1, r - 1, k + 1)).w + __ldg(p.mat + ID(sm1, r, k + 1)).w);
              o[5] += dts * mu * (gz + gr);
            }
            // s_phiz
            {
              float Q = (Vc(2, r, k) - V(vb, 2, r, k)) * idth * inv_rh;
              float gz = (V(vb, 1, r, k + 1) - V(vb, 1, r, k)) * idz;
              if (rpm) {
                float qs = aq.w * p.psr[Q_GPZ][cr] + aq.z * Q;
                fp.psr_o[Q_GPZ][cr] = qs;
                Q += qs;
              }
              if (zpm) {
                float ps = abz.w * p.psz[Z_GPZ][cz] + abz.z * gz;
                fp.psz_o[Z_GPZ][cz] = ps;
                gz += ps;
              }
              const float mu = 4.f / (__ldg(p.mat + ID(sm1, r, k)).w + __ldg(p.mat + ID(s0, r, k)).w + __ldg(p.mat + ID(sm1, r, k + 1)).w +
                                      __ldg(p.mat + ID(s0, r, k + 1)).w);
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
    // drain the copies this block still has in flight (bounded) before exiting
    for (int q = waited_hi + 1; q <= issued_hi; q++) {
      const int s = q & 3;
      if (mbar_wait(&bar[s], (phase >> s) & 1u)) phase ^= 1u << s;
    }
  }

}

template <typename T, int RT, int ZT, int NT>
static cudaError_t launch_fused_t(const FusedMaps &maps, const FusedParams &fp, cudaStream_t s) {
  using SM = FusedSmem<T, RT, ZT>;
  auto kern = fused_step<T, RT, ZT, NT>;
  static bool attr_done[8] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 8 && !attr_done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::BYTES);
    if (e != cudaSuccess) return e;
    attr_done[dev] = true;
  }
  dim3 grd((fp.k.NR + RT - 1) / RT, (fp.k.NZ + ZT - 1) / ZT);
  kern<<<grd, NT, SM::BYTES, s>>>(maps, fp);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_fused_rt(int rt, const FusedMaps &maps, const FusedParams &fp, cudaStream_t s) {
  switch (rt) {
    case 4: return launch_fused_t<T, 4, 64, 256>(maps, fp, s);
    case 8: return launch_fused_t<T, 8, 64, 256>(maps, fp, s);
    case 12: return launch_fused_t<T, 12, 64, 256>(maps, fp, s);
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
      case 4: return FusedSmem<T, 4, 64>::BYTES;
      case 8: return FusedSmem<T, 8, 64>::BYTES;
      case 12: return FusedSmem<T, 12, 64>::BYTES;
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
