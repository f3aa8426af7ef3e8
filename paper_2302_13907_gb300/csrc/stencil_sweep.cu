// Single-pass sweep step (tile codes 3000 + 100 m + 10 e + b): one persistent
// launch per leapfrog step that performs both halves of the staggered scheme
// (Eq. 1a, then Eq. 1b) while the velocities it has just written and the
// stresses it has just read are still in L2.
//
// The launch sweeps z in chunks of ZC cells (32 or 64) that span every
// (theta, r) row.  The velocity update of chunk c reads the stresses of
// chunk c and one cell of each z neighbour chunk; the stress update of chunk
// c reads the velocities of chunk c and one cell of each neighbour, and
// overwrites stresses that only the velocity updates of chunks c - 1 .. c + 1
// read.  So the stress items of chunk c may run once the velocity items of
// chunks c - 1 .. c + 1 have finished, and nothing else orders the launch.
// Velocity items are handed out chunk by chunk; stress items follow them
// with a lag of L chunks, the two streams alternating item by item, so that
// at any time the launch reads fresh chunks from DRAM (velocity items) while
// it reuses chunks L behind from L2 (stress items).  L2 holds about L + 1
// chunks of fields and IDs (38 B per cell in FP32: 15 MB for ZC = 32 on the
// 20 m well), and every field crosses DRAM once per step: 18 values and an
// ID per cell (74 B in FP32) plus the PML memory variables, against 120 B
// for the two split launches.
//
// Items: an item is 512 cells, four cells per thread: ZC / 4 lanes per row
// segment, 512 / ZC consecutive (theta, r) rows (flattened, theta slowest).
// A block of 128 threads processes items blockIdx.x, blockIdx.x + gridDim.x,
// ... in order, with one wave of resident blocks of odd size, so that every
// block alternates velocity and stress items.  Interior cells run the lean
// bodies; PML rows, z-PML cells and the z ends the general bodies with the
// memory variables in registers, in runs of e cells per call (e = 4 or 2,
// fewer registers).  Every warp of a velocity item reports to its chunk's
// counter (a release reduction after its stores); a stress item's warp checks
// (lane 0, acquire loads, bounded) that the counters of its three chunks are
// complete, once per chunk, and reads the velocities through L2 only, since
// blocks of the same launch wrote them; they read their own stresses and
// write the new ones streaming (evict-first: last use in the launch).  m
// selects the chunk, the lag and an L2 prefetch of each block's next
// velocity item (launch_sweep_st).
//
// Order and progress: an item waits only on items handed out before it, and
// every block is resident, so the lowest unfinished item can always finish.
// A wait that passes its cycle limit sets status bit 1 and the warp skips its
// cells; once the bit is set, every later wait gives up at once (the step's
// result is then void and sim_sync reports SIM_ETIMEOUT).
#include <algorithm>

#include "hoist_body.cuh"

namespace cwell {
namespace {

constexpr int SW_THREADS = 128;  // four warps
constexpr int SW_NV = 4;         // z cells per thread
constexpr int SW_ITEM = SW_THREADS * SW_NV;  // cells per item

struct SweepParams {
  int *vdone;            // [nchunk] velocity warps finished per chunk (zeroed before the launch)
  int *status;           // bit 1: a bounded wait gave up
  int nrows;             // nth * NR
  int nchunk;            // ceil(NZ / ZC)
  int items_chunk;       // items per chunk and half: ceil(nrows / (512 / ZC))
  long long nv;          // velocity items: nchunk * items_chunk (as many stress items)
  long long lag;         // velocity items handed out before the first stress item
  long long total;       // 2 * nv
  long long wait_limit;  // clock cycles a stress warp waits for its chunks
  int withhold_chunk;    // velocity items of this chunk never report (-1: none); a test of the give-up path
};

// item it -> (velocity or stress, index in its stream): velocity items 0 ..
// lag-1 first, then alternating velocity item u and stress item u - lag,
// then the remaining stress items
__device__ __forceinline__ void sweep_item(const SweepParams &q, long long it, bool &vel, long long &idx) {
  if (it < q.lag) {
    vel = true;
    idx = it;
    return;
  }
  it -= q.lag;
  const long long pairs = q.nv - q.lag;
  if (it < 2 * pairs) {
    vel = (it & 1) == 0;
    idx = vel ? q.lag + (it >> 1) : (it >> 1);
    return;
  }
  vel = false;
  idx = pairs + (it - 2 * pairs);
}

__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(int *p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// lane 0: have the velocity items of chunks c-1 .. c+1 all reported (four
// warps each)?  Bounded: gives up after q.wait_limit cycles, or at once when
// another wait has given up.
__device__ __noinline__ bool sweep_ready(const SweepParams &q, int c) {
  const int lo = c > 0 ? c - 1 : 0, hi = c + 1 < q.nchunk ? c + 1 : q.nchunk - 1;
  const int full = 4 * q.items_chunk;
  long long t0 = 0;
  for (unsigned it = 0;; ++it) {
    bool ok = true;
    for (int r = lo; r <= hi && ok; r++) ok = ld_acquire(q.vdone + r) >= full;
    if (ok) return true;
    if (it == 0) {
      t0 = clock64();
      continue;
    }
    if ((it & 7u) == 7u) {
      if (*(volatile int *)q.status & 2) return false;
      if (clock64() - t0 > q.wait_limit) {
        atomicOr(q.status, 2);
        return false;
      }
    }
    __nanosleep(200);
  }
}

// the four cells of one thread: the lean bodies inside, the general bodies in
// runs of NVE cells elsewhere
template <typename T, int NVE, bool VEL>
__device__ __forceinline__ void sweep_cells(const KParams &p, int j, int i, int k0) {
  if (lean_cells<SW_NV>(p, i, k0)) {
    if (VEL) vel_hoist_body<T, SW_NV, true>(p, j, i, k0);
    else str_hoist_body<T, SW_NV, true, false, true, true>(p, j, i, k0);
  } else {
#pragma unroll 1
    for (int h = 0; h < SW_NV; h += NVE) {
      const int k = k0 + h;
      if (k >= p.NZ) break;
      if (VEL) vel_hoist_body<T, NVE, false, true>(p, j, i, k);
      else str_hoist_body<T, NVE, false, true, false, true>(p, j, i, k);
    }
  }
}

template <typename T, int ZC, int MINB, int NVE, bool PF>
__global__ void __launch_bounds__(SW_THREADS, MINB) sweep_step(const KParams p, const SweepParams q) {
  constexpr int LPR = ZC / SW_NV;    // lanes per row segment
  constexpr int RPI = SW_ITEM / ZC;  // rows per item
  const int lane = threadIdx.x & 31;
  const int row_in_item = threadIdx.x / LPR, kk = (threadIdx.x % LPR) * SW_NV;
  int ready = -1;  // the last chunk whose three velocity chunks this warp found complete
  // (chunk, theta, r, first z cell) of this thread's cells in item `idx` of a
  // stream; false when they lie outside the grid
  auto place = [&](long long idx, int &c, int &j, int &i, int &k0) {
    c = (int)(idx / q.items_chunk);
    const int row = (int)(idx - (long long)c * q.items_chunk) * RPI + row_in_item;
    j = row / p.NR;
    i = row - j * p.NR;
    k0 = c * ZC + kk;
    return row < q.nrows && k0 < p.NZ;
  };
  for (long long it = blockIdx.x; it < q.total; it += gridDim.x) {
    bool vel;
    long long idx;
    sweep_item(q, it, vel, idx);
    if (PF && it + gridDim.x < q.total) {  // the block's next item, if a velocity item: its lines into L2
      bool v2;
      long long i2;
      sweep_item(q, it + gridDim.x, v2, i2);
      int c2, j2, r2, k2;
      if (v2 && place(i2, c2, j2, r2, k2)) prefetch_tile<T, SW_NV, true>(p, j2, r2, k2);
    }
    int c, j, i, k0;
    const bool inside = place(idx, c, j, i, k0);
    const bool active = inside && i >= p.i_lo && i < p.i_hi;
    if (vel) {
      if (active) sweep_cells<T, NVE, true>(p, j, i, k0);
      __syncwarp();  // the warp's stores precede its report
      if (lane == 0 && c != q.withhold_chunk) red_release_add(q.vdone + c, 1);
    } else {
      int ok = 1;
      if (c != ready) {
        if (lane == 0) ok = sweep_ready(q, c);
        __syncwarp();  // orders the warp's loads after lane 0's acquire
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (ok) ready = c;
      }
      if (ok && active) sweep_cells<T, NVE, false>(p, j, i, k0);
    }
  }
}

int sm_count_sw() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n < 1) n = 1;
  }
  return n;
}

template <typename T, int ZC, int MINB, int NVE, bool PF>
cudaError_t launch_sweep_t(const KParams &p, SweepParams q, int lag_half_chunks, cudaStream_t s) {
  static int resident[16] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 16) return cudaErrorInvalidDevice;
  if (!resident[dev]) {
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_step<T, ZC, MINB, NVE, PF>, SW_THREADS, 0);
    if (e != cudaSuccess) return e;
    if (n < 1) return cudaErrorInvalidConfiguration;
    resident[dev] = std::min(n, MINB);
  }
  q.nchunk = (p.NZ + ZC - 1) / ZC;
  q.items_chunk = (q.nrows + SW_ITEM / ZC - 1) / (SW_ITEM / ZC);
  q.nv = (long long)q.nchunk * q.items_chunk;
  q.lag = std::min<long long>(q.nv, (long long)lag_half_chunks * q.items_chunk / 2);
  q.total = 2 * q.nv;
  // one wave: every block resident, so that an item's wait on earlier items
  // ends; an odd count, so that each block alternates velocity and stress items
  long long grid = std::min<long long>(q.total, (long long)resident[dev] * sm_count_sw());
  if (grid > 1 && (grid & 1) == 0) grid--;
  if (grid < 1) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(q.vdone, 0, (size_t)q.nchunk * sizeof(int), s);
  if (e != cudaSuccess) return e;
  sweep_step<T, ZC, MINB, NVE, PF><<<(int)grid, SW_THREADS, 0, s>>>(p, q);
  return cudaGetLastError();
}

// m: 0, 1 chunks of 32 cells, lag 3 chunks (1: with prefetch); 2, 3 chunks of
// 64, lag 2.5 (3: with prefetch); 4, 5 chunks of 32, lag 2.5 and 2
template <typename T>
cudaError_t launch_sweep_st(int code, const KParams &p, const SweepParams &q, cudaStream_t s) {
  switch (code) {
    case 3043: return launch_sweep_t<T, 32, 3, 4, false>(p, q, 6, s);
    case 3024: return launch_sweep_t<T, 32, 4, 2, false>(p, q, 6, s);
    case 3143: return launch_sweep_t<T, 32, 3, 4, true>(p, q, 6, s);
    case 3124: return launch_sweep_t<T, 32, 4, 2, true>(p, q, 6, s);
    case 3243: return launch_sweep_t<T, 64, 3, 4, false>(p, q, 5, s);
    case 3224: return launch_sweep_t<T, 64, 4, 2, false>(p, q, 5, s);
    case 3343: return launch_sweep_t<T, 64, 3, 4, true>(p, q, 5, s);
    case 3324: return launch_sweep_t<T, 64, 4, 2, true>(p, q, 5, s);
    case 3443: return launch_sweep_t<T, 32, 3, 4, false>(p, q, 5, s);
    case 3424: return launch_sweep_t<T, 32, 4, 2, false>(p, q, 5, s);
    case 3543: return launch_sweep_t<T, 32, 3, 4, false>(p, q, 4, s);
    case 3524: return launch_sweep_t<T, 32, 4, 2, false>(p, q, 4, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

int sweep_chunks(int NZ) { return (NZ + 31) / 32; }

cudaError_t launch_sweep(int storage, int code, const KParams &p, int *vdone, int *status, long long wait_limit,
                         int withhold_chunk, cudaStream_t s) {
  if (!vdone || !status || p.NR < 1 || p.nth < 1 || p.NZ < 1) return cudaErrorInvalidValue;
  const long long nrows = (long long)p.nth * p.NR;
  if (nrows > 0x7fffffffLL / 16) return cudaErrorInvalidValue;
  SweepParams q{};
  q.vdone = vdone;
  q.status = status;
  q.nrows = (int)nrows;
  q.wait_limit = wait_limit > 0 ? wait_limit : (1LL << 31);
  q.withhold_chunk = withhold_chunk;
  switch (storage) {
    case 0: return launch_sweep_st<float>(code, p, q, s);
    case 1: return launch_sweep_st<__nv_bfloat16>(code, p, q, s);
    case 2: return launch_sweep_st<__half>(code, p, q, s);
    case 3: return launch_sweep_st<half_sr>(code, p, q, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace cwell
