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

#include "hoist_body.cuh"

namespace cwell {
namespace {

constexpr int HB_X = 32;  // threads along z per block (NV cells each)
constexpr int HB_Y = 4;   // r rows per block

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
  if (i < p.i_lo || i >= p.i_hi || k0 < p.k_lo || k0 >= p.k_hi) return;
  if (VEL) vel_hoist_body<T, NV, true>(p, j, i, k0);
  else str_hoist_body<T, NV, true>(p, j, i, k0);
}

// Persistent interior kernel with an L2 prefetch of its next tile: one wave
// of resident blocks walks the interior tiles in the order above (theta
// fastest); before computing its tile a block asks L2 for every row its next
// tile will load (one prefetch per 128-byte line), so those loads find their
// lines in L2.  No register or shared memory holds the prefetched data.
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
    if (i < p.i_lo || i >= p.i_hi || k0 < p.k_lo || k0 >= p.k_hi) continue;
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
  if (i >= p.i_lo && i < p.i_hi && k0 < p.NZ && k0 >= p.k_lo && k0 < p.k_hi) hoist_cells<T, NV, VEL, true>(p, j, i, k0);
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
    if (i >= p.i_lo && i < p.i_hi && k0 < p.NZ && k0 >= p.k_lo && k0 < p.k_hi) hoist_cells<T, NV, VEL, true>(p, j, i, k0);
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
    if (i < p.i_lo || i >= p.i_hi || k0 < p.k_lo || k0 >= p.k_hi) continue;
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
    if (i >= p.i_lo && i < p.i_hi && k0 < p.NZ && k0 >= p.k_lo && k0 < p.k_hi) hoist_cells<T, NV, VEL, true>(p, j, i, k0);
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

thread_local const SideStream *g_side = nullptr;

// fork / join of the edge launches of a half onto the side stream (when one
// is set and the half has both kinds of tiles); returns the edge stream
inline cudaError_t side_fork(bool fork, cudaStream_t s, cudaStream_t *se) {
  *se = s;
  if (!fork) return cudaSuccess;
  cudaError_t e = cudaEventRecord(g_side->fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(g_side->side, g_side->fork, 0);
  if (e == cudaSuccess) *se = g_side->side;
  return e;
}
inline cudaError_t side_join(bool fork, cudaStream_t s) {
  if (!fork) return cudaSuccess;
  cudaError_t e = cudaEventRecord(g_side->join, g_side->side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, g_side->join, 0);
  return e;
}

template <typename T, int NV, int MINB_IN, int NVE, int MINB_E, bool VEL, bool PF, bool PFE>
cudaError_t launch_split2_half(const KParams &p, const Split2 &q, cudaStream_t s) {
  dim3 blk(HB_X, HB_Y);
  const int nin = q.zt_hi - q.zt_lo;
  const long long nedge = (long long)(q.nrt - q.nrt_in) * q.enzt + (long long)q.nrt_in * (q.ez_lo + q.enzt - q.ez_hi);
  if (nedge > 65535 || p.nth > 65535) return cudaErrorInvalidValue;
  const bool interior = q.nrt_in > 0 && nin > 0;
  const bool fork = g_side && interior && nedge > 0;  // the edge launch beside the interior one
  cudaStream_t se;
  cudaError_t e = side_fork(fork, s, &se);
  if (e != cudaSuccess) return e;
  if (nedge > 0) {
    if constexpr (PFE) {
      const long long tiles = (long long)p.nth * nedge;
      const int grid = (int)std::min<long long>(tiles, (long long)sm_count() * MINB_E);
      hoist_edge_pf<T, NVE, MINB_E, VEL><<<grid, blk, 0, se>>>(p, q, (int)tiles);
    } else {
      hoist_edge<T, NVE, MINB_E, VEL><<<dim3(p.nth, (unsigned)nedge), blk, 0, se>>>(p, q);
    }
  }
  if (interior) {
    if constexpr (PF) {  // one wave of resident blocks
      const long long tiles = (long long)p.nth * q.nrt_in * nin;
      if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
      const int grid = (int)std::min<long long>(tiles, (long long)sm_count() * MINB_IN);
      hoist_interior_pf<T, NV, MINB_IN, VEL><<<grid, blk, 0, s>>>(p, q.zt_lo, q.nrt_in, (int)tiles);
    } else {
      hoist_interior<T, NV, MINB_IN, VEL><<<dim3(p.nth, q.nrt_in, nin), blk, 0, s>>>(p, q.zt_lo);
    }
  }
  if ((e = side_join(fork, s)) != cudaSuccess) return e;
  return cudaGetLastError();
}


// three-way split half step: interior (plain or prefetching), radial tiles
// (NVE cells per thread, MINB_R blocks per SM), z-end tiles (NVE, MINB_E).
// The three update disjoint cells from inputs no launch of the half writes,
// so with a side stream the edge launches run beside the interior launch.
template <typename T, int NV, int MINB_IN, bool PF, int NVE, int MINB_R, int MINB_E, bool VEL>
cudaError_t launch_split3_half(const KParams &p, const Split2 &q, cudaStream_t s) {
  dim3 blk(HB_X, HB_Y);
  const int nin = q.zt_hi - q.zt_lo;
  const long long rad = (long long)p.nth * (q.nrt - q.nrt_in) * (q.ez_hi - q.ez_lo);
  const long long ends = (long long)p.nth * q.nrt * (q.ez_lo + q.enzt - q.ez_hi);
  if (rad > 0x7fffffffLL || ends > 0x7fffffffLL) return cudaErrorInvalidValue;
  const bool interior = q.nrt_in > 0 && nin > 0;
  const bool fork = g_side && interior && (rad > 0 || ends > 0);
  cudaStream_t se;  // stream of the edge launches
  cudaError_t e = side_fork(fork, s, &se);
  if (e != cudaSuccess) return e;
  if (rad > 0)
    hoist_radial_pf<T, NVE, MINB_R, VEL>
        <<<(int)std::min<long long>(rad, (long long)sm_count() * MINB_R), blk, 0, se>>>(p, q, (int)rad);
  if (ends > 0)
    hoist_ends_pf<T, NVE, MINB_E, VEL>
        <<<(int)std::min<long long>(ends, (long long)sm_count() * MINB_E), blk, 0, se>>>(p, q, (int)ends);
  if (interior) {
    if constexpr (PF) {
      const long long tiles = (long long)p.nth * q.nrt_in * nin;
      if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
      const int grid = (int)std::min<long long>(tiles, (long long)sm_count() * MINB_IN);
      hoist_interior_pf<T, NV, MINB_IN, VEL><<<grid, blk, 0, s>>>(p, q.zt_lo, q.nrt_in, (int)tiles);
    } else {
      hoist_interior<T, NV, MINB_IN, VEL><<<dim3(p.nth, q.nrt_in, nin), blk, 0, s>>>(p, q.zt_lo);
    }
  }
  if ((e = side_join(fork, s)) != cudaSuccess) return e;
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

void set_side_stream(const SideStream *ss) { g_side = ss; }

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

namespace {
// the stochastic rounding of the FP16-SR stores, element by element
__global__ void __launch_bounds__(256) sr_round_kernel(const float *x, const unsigned *dither, unsigned short *out,
                                                       long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    out[q] = __half_as_ushort(sr_round(x[q], dither[q] & 0x1fffu));
}
}  // namespace

cudaError_t launch_sr_round(const float *x, const unsigned *dither, unsigned short *out, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int grid = (int)std::min<long long>((n + 255) / 256, 152LL * 8);
  sr_round_kernel<<<grid, 256, 0, s>>>(x, dither, out, n);
  return cudaGetLastError();
}

cudaError_t launch_hoist(int storage, int code, const KParams &p, cudaStream_t s, cudaEvent_t *ev, int parts) {
  const int minb = hoist_blocks(code), nv = hoist_cells_per_thread(code);
  const bool zf = hoist_zfast(code), split = hoist_split(code), split3 = (code / 100) % 10 == 3;
  const int edge = (code / 10) % 10;
  switch (storage) {
    case 0: return launch_hoist_st<float>(nv, minb, zf, split, edge, p, s, ev, parts, split3);
    case 1: return launch_hoist_st<__nv_bfloat16>(nv, minb, zf, split, edge, p, s, ev, parts, split3);
    case 2: return launch_hoist_st<__half>(nv, minb, zf, split, edge, p, s, ev, parts, split3);
    case 3:  // FP16 with stochastic rounding: the three-way split codes only
      if (!split3) return cudaErrorInvalidValue;
      switch (edge * 10 + minb) {
        case 4: return launch_split3_t<half_sr, 4, 4, true, 4, 4, 3>(p, s, ev, parts);
        case 5: return launch_split3_t<half_sr, 4, 5, false, 4, 4, 3>(p, s, ev, parts);
        case 14: return launch_split3_t<half_sr, 4, 4, true, 2, 5, 4>(p, s, ev, parts);
        case 15: return launch_split3_t<half_sr, 4, 5, false, 2, 5, 4>(p, s, ev, parts);
        case 24: return launch_split3_t<half_sr, 4, 4, true, 2, 4, 4>(p, s, ev, parts);
        case 25: return launch_split3_t<half_sr, 4, 5, false, 2, 4, 4>(p, s, ev, parts);
        case 34: return launch_split3_t<half_sr, 4, 4, true, 4, 3, 3>(p, s, ev, parts);
        case 35: return launch_split3_t<half_sr, 4, 5, false, 4, 3, 3>(p, s, ev, parts);
      }
      return cudaErrorInvalidValue;
  }
  return cudaErrorInvalidValue;
}

}  // namespace cwell
