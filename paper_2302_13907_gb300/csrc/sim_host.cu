// Host side of the C-ABI: validation, FP64 set-up (time step, material
// table, PML profiles, source wavelet, receiver nodes), device allocation,
// CUDA-graph stepping, traces, checkpoints.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "sim_state.cuh"

using namespace cwell;

thread_local std::string cwell::g_create_err;

static int dev_alloc(sim_t *h, void **p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  if (h->mem_cap && h->bytes + bytes > h->mem_cap)
    return fail(h, SIM_ENOMEM, "device memory cap exceeded (" + std::to_string(h->bytes + bytes) + " > " +
                                   std::to_string(h->mem_cap) + " bytes)");
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, SIM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  h->allocs.push_back(*p);
  h->bytes += bytes;
  e = cudaMemsetAsync(*p, 0, bytes, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync");
  return SIM_OK;
}

// Ricker pulse, dominant frequency f0, delay 2/f0 (Sec. 2 of the paper)
double cwell::ricker(double t, double f0) {
  double a = M_PI * f0 * (t - 2.0 / f0);
  a = a * a;
  return (1.0 - 2.0 * a) * exp(-a);
}

void cwell::cpml(double d, double al, double dt, float *a, float *b) {
  if (!(d > 0.0)) {
    *a = 0.f;
    *b = 1.f;
    return;
  }
  double bb = exp(-(d + al) * dt);
  *b = (float)bb;
  *a = (float)(d * (bb - 1.0) / (d + al));
}

int cwell::validate_inputs(const sim_grid_t *g, const sim_medium_t *m, const sim_source_t *s,
                           const sim_receivers_t *r, const sim_opts_t *o) {
  if (!g || !m || !s || !r || !o) return fail(nullptr, SIM_EINVAL, "null argument");
  if (g->nr < 2 || g->nth < 4 || (g->nth & 1) || g->nz < 2 || g->pml_r < 0 || g->pml_z < 0)
    return fail(nullptr, SIM_EINVAL, "grid: need nr >= 2, nth >= 4 and even, nz >= 2, pml >= 0");
  if (!(g->dr > 0) || !(g->dz > 0) || !isfinite(g->dr) || !isfinite(g->dz))
    return fail(nullptr, SIM_EINVAL, "grid: dr, dz must be positive and finite");
  if (!(g->dt > 0) && !(g->cfl > 0)) return fail(nullptr, SIM_EINVAL, "grid: need dt > 0 or cfl > 0");
  long long cells = (long long)g->nth * (g->nr + g->pml_r) * (g->nz + 2 * g->pml_z);
  if (cells > (1LL << 40)) return fail(nullptr, SIM_EINVAL, "grid too large");
  if (m->n_mat < 1 || m->n_mat > 65536 || !m->rho || !m->vp || !m->vs || !m->cell_id)
    return fail(nullptr, SIM_EINVAL, "medium: need 1 <= n_mat <= 65536 and non-null arrays");
  for (int q = 0; q < m->n_mat; q++)
    if (!(m->rho[q] > 0) || !(m->vp[q] > 0) || !(m->vs[q] >= 0) || m->vp[q] * m->vp[q] < 2.0 * m->vs[q] * m->vs[q] ||
        !isfinite(m->rho[q]) || !isfinite(m->vp[q]))
      return fail(nullptr, SIM_EINVAL, "medium: material " + std::to_string(q) + " needs rho, vp > 0, vs >= 0, vp^2 >= 2 vs^2");
  if (s->kind < 0 || s->kind > 3) return fail(nullptr, SIM_EINVAL, "source: kind must be 0 .. 3");
  if (s->kind != 0 && (o->kernel == SIM_KERNEL_FUSED || o->kernel == SIM_KERNEL_FUSED_VEC))
    return fail(nullptr, SIM_EUNSUPPORTED, "source: point forces and torsion run on the split and marching paths only");
  if ((s->kind == 1 || s->kind == 2) && o->kernel == SIM_KERNEL_SWEEP)
    return fail(nullptr, SIM_EUNSUPPORTED, "source: point forces act between the half-steps, which the sweep kernel fuses");
  if (!(s->f0 > 0) || !isfinite(s->amplitude)) return fail(nullptr, SIM_EINVAL, "source: need f0 > 0, finite amplitude");
  if (!(s->r >= 0) || s->r >= g->nr * g->dr) return fail(nullptr, SIM_EINVAL, "source: r outside the interior");
  long ks = lround(s->z / g->dz);
  if (!isfinite(s->z) || ks < 0 || ks >= g->nz) return fail(nullptr, SIM_EINVAL, "source: z outside the interior");
  if (s->kind != 0) {  // the nodes of a point force or of the torsion ring
    const int NR = g->nr + g->pml_r, NZ = g->nz + 2 * g->pml_z, nth = g->nth;
    const long k = ks + g->pml_z;
    const int i_int = (int)lround(s->r / g->dr), i_half = (int)floor(s->r / g->dr);
    if (s->kind == 1 && s->r >= g->dr && (i_int < 1 || i_int >= NR))
      return fail(nullptr, SIM_EINVAL, "source: the transverse force's v_r node falls outside the grid");
    if ((s->kind == 2 || s->kind == 3) && k + 1 >= NZ)
      return fail(nullptr, SIM_EINVAL, "source: the node above the force / torsion depth falls outside the grid");
    if (s->kind == 3) {
      if (i_int < 1 || i_int >= NR) return fail(nullptr, SIM_EINVAL, "source: the torsion ring needs 1 <= r / dr < NR");
      auto solid = [&](int j, int i, long kk) { return m->vs[m->cell_id[((size_t)j * NR + i) * NZ + kk]] > 0.0; };
      for (int j = 0; j < nth; j++) {
        const int jp = (j + 1) % nth;
        if (!(solid(j, i_int - 1, k) && solid(j, i_int, k) && solid(jp, i_int - 1, k) && solid(jp, i_int, k) &&
              solid(j, i_half, k) && solid(jp, i_half, k) && solid(j, i_half, k + 1) && solid(jp, i_half, k + 1)))
          return fail(nullptr, SIM_EUNSUPPORTED, "source: the torsion ring needs a solid at both shear nodes");
      }
    }
  }
  if (r->n < 0 || (r->n > 0 && (!r->r || !r->theta || !r->z)) || r->quantity != 0)
    return fail(nullptr, SIM_EINVAL, "receivers: bad count, arrays or quantity");
  for (int q = 0; q < r->n; q++) {
    long kr = lround(r->z[q] / g->dz);
    if (!isfinite(r->z[q]) || kr < 0 || kr >= g->nz || !(r->r[q] >= 0) || r->r[q] >= g->nr * g->dr)
      return fail(nullptr, SIM_EINVAL, "receiver " + std::to_string(q) + " outside the interior");
  }
  if (o->storage < 0 || o->storage > 3) return fail(nullptr, SIM_EINVAL, "opts: storage must be 0 .. 3");
  if (o->watchdog_every < 0) return fail(nullptr, SIM_EINVAL, "opts: watchdog_every < 0");
  if (o->storage == SIM_STORAGE_F16_SR) {
    if (!(o->kernel == SIM_KERNEL_AUTO || o->kernel == SIM_KERNEL_SPLIT || o->kernel == SIM_KERNEL_SWEEP))
      return fail(nullptr, SIM_EUNSUPPORTED, "storage: stochastic rounding runs on the split and sweep kernels only");
    if (s->kind != 0)
      return fail(nullptr, SIM_EUNSUPPORTED, "storage: stochastic rounding with the volumetric source only");
    if (o->tile != 0 && !(o->tile >= 2300 && o->tile < 2400) && !is_sweep(o->tile) &&
        !(is_split_pair(o->tile) && split_vel_code(o->tile) / 100 == 23 && split_str_code(o->tile) / 100 == 23))
      return fail(nullptr, SIM_EUNSUPPORTED, "storage: stochastic rounding runs on the 23xx split and the sweep codes");
  }
  if (o->kernel < 0 || o->kernel > 5) return fail(nullptr, SIM_EINVAL, "opts: kernel must be 0 .. 5");
  if (o->tile != 0) {  // the family of the code must match the kernel asked for; the code itself is checked later
    const int t = o->tile;
    const bool ok = t > 0 && ((o->kernel == SIM_KERNEL_SPLIT && is_split_family(t)) ||
                              (o->kernel == SIM_KERNEL_FUSED && t < 100) ||
                              (o->kernel == SIM_KERNEL_FUSED_VEC && t >= 100 && t < 1000) ||
                              (o->kernel == SIM_KERNEL_MARCH && is_march(t)) ||
                              (o->kernel == SIM_KERNEL_SWEEP && is_sweep(t)) ||
                              (o->kernel == SIM_KERNEL_AUTO && (t < 3000 || is_split_pair(t) || is_sweep(t))));
    if (!ok) return fail(nullptr, SIM_EINVAL, "opts: tile " + std::to_string(t) + " is not a tile code of the kernel asked for");
  }
  if (o->max_steps < 0) return fail(nullptr, SIM_EINVAL, "opts: max_steps < 0");
  return SIM_OK;
}

// Reading R7: dt = cfl * min over cells 1 / (Vp sqrt(1/dr^2 + 1/(r dth)^2 +
// 1/dz^2)), r the cell centre; grid.dt > 0 overrides it.  Host only.
static double grid_time_step(const sim_grid_t &g, const sim_medium_t *medium) {
  if (g.dt > 0) return g.dt;
  const int NR = g.nr + g.pml_r, NZ = g.nz + 2 * g.pml_z, nth = g.nth;
  const double dth = 2.0 * M_PI / nth;
  const uint16_t *cid = medium->cell_id;
  double best = INFINITY;
  for (int i = 0; i < NR; i++) {
    double cmax = 0.0;
    for (int j = 0; j < nth; j++) {
      const uint16_t *row = cid + ((size_t)j * NR + i) * NZ;
      for (int k = 0; k < NZ; k++) cmax = std::max(cmax, medium->vp[row[k]]);
    }
    const double rc = (i + 0.5) * g.dr;
    const double s = sqrt(1.0 / (g.dr * g.dr) + 1.0 / ((rc * dth) * (rc * dth)) + 1.0 / (g.dz * g.dz));
    best = std::min(best, 1.0 / (cmax * s));
  }
  return g.cfl * best;
}

extern "C" int sim_time_step(const sim_grid_t *grid, const sim_medium_t *medium, double *dt) {
  if (!grid || !medium || !dt || !medium->cell_id || !medium->vp) return fail(nullptr, SIM_EINVAL, "null argument");
  if (grid->nr < 1 || grid->nth < 1 || grid->nz < 1 || grid->pml_r < 0 || grid->pml_z < 0 || !(grid->dr > 0) ||
      !(grid->dz > 0) || (!(grid->dt > 0) && !(grid->cfl > 0)))
    return fail(nullptr, SIM_EINVAL, "grid: need positive sizes and steps, and dt > 0 or cfl > 0");
  const size_t ncell = (size_t)grid->nth * (grid->nr + grid->pml_r) * (grid->nz + 2 * grid->pml_z);
  for (size_t c = 0; c < ncell; c++)
    if (medium->cell_id[c] >= medium->n_mat) return fail(nullptr, SIM_EINVAL, "medium: cell_id out of range");
  *dt = grid_time_step(*grid, medium);
  return SIM_OK;
}

extern "C" int sim_round_f16_sr(const float *x, const unsigned *dither, unsigned short *out, long long n,
                                void *cuda_stream) {
  if (n < 0 || (n > 0 && (!x || !dither || !out))) return fail(nullptr, SIM_EINVAL, "null pointer or n < 0");
  const cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaError_t e = launch_sr_round(x, dither, out, n, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(nullptr, SIM_ECUDA, std::string("sim_round_f16_sr: ") + cudaGetErrorString(e));
  return SIM_OK;
}

// RAII: the handle's side stream for the three-way split halves while in scope
struct SideScope {
  explicit SideScope(const sim_t *h) { set_side_stream(h->side.side ? &h->side : nullptr); }
  ~SideScope() { set_side_stream(nullptr); }
};

static void release(sim_t *h) {
  if (!h) return;
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->side.fork) cudaEventDestroy(h->side.fork);
  if (h->side.join) cudaEventDestroy(h->side.join);
  if (h->side.side) cudaStreamDestroy(h->side.side);
  for (auto &e : h->ev)
    if (e) cudaEventDestroy(e);
  for (void *p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

// ---------------------------------------------------------------- TMA descriptors
static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

// 4-D tiled descriptor of an [1][nth][NR][NZp] array, box {bx, rows, 1, 1};
// loads outside the array read zeros.
static int make_map(sim_t *h, CUtensorMap *m, void *base, CUtensorMapDataType dt, int elem, int bx, int rows) {
  auto enc = tmap_encoder();
  if (!enc) return fail(h, SIM_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  cuuint64_t dims[4] = {(cuuint64_t)h->NZp, (cuuint64_t)h->NR, (cuuint64_t)h->grid.nth, 1};
  cuuint64_t strides[3] = {(cuuint64_t)h->NZp * elem, (cuuint64_t)h->NZp * h->NR * elem,
                           (cuuint64_t)h->NZp * h->NR * h->grid.nth * elem};
  cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)rows, 1, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = enc(m, dt, 4, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(h, SIM_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return SIM_OK;
}

static int build_maps(sim_t *h, int code) {
  const int rt = tile_rows(code);
  const CUtensorMapDataType dt = h->storage == 0   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : h->storage == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                   : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  for (int par = 0; par < 2; par++) {
    void **src = par == 0 ? h->f : h->f2;
    for (int q = 0; q < NF; q++) {
      int rc = make_map(h, &h->maps[par].f[q], src[q], dt, (int)h->elem, fused_box_x(h->storage), rt + 2);
      if (rc) return rc;
    }
    int rc = make_map(h, &h->maps[par].id, h->id, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, 64 + 16, rt + 2);
    if (rc) return rc;
  }
  return SIM_OK;
}

// descriptors of the marching kernels: the nine fields of the first buffer
// set (updated in place) and the IDs, boxes of rows + 2 rows
static int build_march_maps(sim_t *h, int code) {
  const int rt = march_rows(code);
  const CUtensorMapDataType dt = h->storage == 0   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : h->storage == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                   : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  for (int q = 0; q < NF; q++) {
    int rc = make_map(h, &h->mmaps.f[q], h->f[q], dt, (int)h->elem, march_box_x(h->storage), rt + 2);
    if (rc) return rc;
  }
  return make_map(h, &h->mmaps.id, h->id, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, march_box_id(), rt + 2);
}

// Autotuner: time each tile height on the still-zero state with the source
// disabled (the state stays zero), keep the fastest; cached per grid shape.
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int, int, int>, int> g_tune;

static cudaError_t launch_fused_any(int storage, int code, const FusedMaps &maps, const FusedParams &fp,
                                    cudaStream_t s) {
  return code >= 100 ? launch_fused4(storage, code - 100, maps, fp, s) : launch_fused(storage, code, maps, fp, s);
}

// Candidates: the fused kernels with each tile height that fits in shared
// memory, the marching split kernels with each tile height and theta run, and
// the split kernels (plain and load-first), as far as the requested kernel allows.
static cudaError_t launch_split_one(int storage, int code, const KParams &p, cudaStream_t s, cudaEvent_t *ev,
                                    int parts) {
  return is_hoist(code) ? launch_hoist(storage, code, p, s, ev, parts) : launch_split(storage, p, s, ev, parts);
}

// a pair code runs the velocity half of one split code and the stress half of another
static cudaError_t launch_split_family(int storage, int code, const KParams &p, cudaStream_t s, cudaEvent_t *ev,
                                       int parts = 3) {
  const int v = split_vel_code(code), c = split_str_code(code);
  if (v == c) return launch_split_one(storage, v, p, s, ev, parts);
  cudaError_t e = cudaSuccess;
  if (parts & 1) e = launch_split_one(storage, v, p, s, ev, 1);
  if (e == cudaSuccess && (parts & 2)) e = launch_split_one(storage, c, p, s, ev, 2);
  return e;
}

// one or both halves of a handle's step with the split code its tuner chose
// (the batch drives its large cases this way, on the batch's stream)
cudaError_t cwell::sim_split_halves(const sim_t *h, const KParams &p, cudaStream_t s, int parts) {
  if (!is_split_family(h->tile_rt)) return cudaErrorInvalidValue;
  return launch_split_family(h->stencil_storage, h->tile_rt, p, s, nullptr, parts);
}

static int autotune(sim_t *h, int kernel, int forced, int *best_rt) {
  SideScope side_scope(h);
  const bool allow_split = kernel == SIM_KERNEL_AUTO || kernel == SIM_KERNEL_SPLIT;
  int dev = h->device, maxsm = 0;
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // point forces rule out the sweep kernel: they key a separate choice
  const bool force = h->src_kind == 1 || h->src_kind == 2;
  auto key = std::make_tuple(dev, h->grid.nth, h->NR, h->NZ, h->stencil_storage * 8 + kernel,
                             (h->kp.pml_r > 0 ? 1 : 0) + (force ? 2 : 0));
  if (!forced) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      *best_rt = it->second;
      return SIM_OK;
    }
  }
  const int cand[] = {2,    4,    6,    8,    106,  110,  114,  1216, 1232, 1264, 1416, 1432, 1464, 1816, 1832,
                      1864, 2003, 2004, 2005, 2013, 2014, 2106, 2108, 2204, 2205, 2216, 2218, 2224, 2225,
                      2234, 2235, 2244, 2245, 2256, 2258, 2264, 2265, 2274, 2275,
                      2284, 2285, 2294, 2295, 2304, 2305, 2314, 2315, 2324, 2325, 2334, 2335, SPLIT_CODE,
                      3043, 3024, 3143, 3124, 3243, 3224, 3343, 3324, 3443, 3424, 3543, 3524};
  cudaEvent_t a, b, c3;
  CK(h, cudaEventCreate(&a));
  CK(h, cudaEventCreate(&b));
  CK(h, cudaEventCreate(&c3));
  float best = INFINITY, best_v = INFINITY, best_s = INFINITY;
  int pick = -1, pick_v = -1, pick_s = -1;
  std::vector<std::pair<float, int>> times_v, times_s;  // every split code's half-step times
  if (forced && is_split_pair(forced) && allow_split) {  // both halves must be split candidates; nothing to fit
    bool v = false, c = false;
    for (int rt : cand) v |= rt == split_vel_code(forced), c |= rt == split_str_code(forced);
    if (v && c) pick = forced;
  }
  for (int rt : cand) {
    cudaError_t e = cudaSuccess;
    const bool fused_code = rt < 1000;
    if (kernel == SIM_KERNEL_FUSED && (!fused_code || rt >= 100)) continue;
    if (kernel == SIM_KERNEL_FUSED_VEC && (!fused_code || rt < 100)) continue;
    if (kernel == SIM_KERNEL_MARCH && !is_march(rt)) continue;
    if (kernel == SIM_KERNEL_SPLIT && !is_split_family(rt)) continue;
    if (kernel == SIM_KERNEL_SWEEP && !is_sweep(rt)) continue;
    if (is_sweep(rt) && (force || !(kernel == SIM_KERNEL_AUTO || kernel == SIM_KERNEL_SWEEP))) continue;
    if (is_split_family(rt) && !allow_split) continue;
    if (!h->fused && fused_code) continue;  // no second buffer set for the fused kernels
    // a slab: the interior / edge split codes, whose kernels honour its z range
    if (h->slab && !(rt >= 2200 && rt < 2400)) continue;
    // stochastic rounding: the three-way split codes and the sweep kernel only
    if (h->stencil_storage == SIM_STORAGE_F16_SR && !(rt >= 2300 && rt < 2400) && !is_sweep(rt)) continue;
    if (forced && rt != forced) continue;
    if (forced) {  // a tile asked for by the caller: check that it fits, time nothing
      const size_t need = is_split_family(rt) || is_sweep(rt) ? 1
                          : is_march(rt)      ? march_smem_bytes(h->storage, rt)
                          : rt >= 100         ? fused4_smem_bytes(h->storage, rt - 100)
                                              : fused_smem_bytes(h->storage, rt);
      if (need == 0 || need > (size_t)maxsm) continue;
      pick = rt;
      break;
    }
    if (is_split_family(rt)) {  // each half timed on its own: the best velocity and stress kernels may differ
      KParams dry = h->kp;
      dry.src_i = -1;  // no source: zero state stays zero
      for (int w = 0; w < 2 && e == cudaSuccess; w++)
        e = launch_split_family(h->stencil_storage, rt, dry, h->stream, nullptr);
      cudaEventRecord(a, h->stream);
      for (int w = 0; w < 3 && e == cudaSuccess; w++)
        e = launch_split_family(h->stencil_storage, rt, dry, h->stream, nullptr, 1);
      cudaEventRecord(b, h->stream);
      for (int w = 0; w < 3 && e == cudaSuccess; w++)
        e = launch_split_family(h->stencil_storage, rt, dry, h->stream, nullptr, 2);
      cudaEventRecord(c3, h->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(c3);
      if (e != cudaSuccess) {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        cudaEventDestroy(c3);
        return cuda_fail(h, e, "autotune launch");
      }
      float mv = 0, ms = 0;
      cudaEventElapsedTime(&mv, a, b);
      cudaEventElapsedTime(&ms, b, c3);
      if (mv < best_v) best_v = mv, pick_v = rt;
      if (ms < best_s) best_s = ms, pick_s = rt;
      times_v.push_back({mv, rt});
      times_s.push_back({ms, rt});
      continue;
    } else if (is_sweep(rt)) {
      KParams dry = h->kp;
      dry.src_i = -1;
      for (int w = 0; w < 2 && e == cudaSuccess; w++)
        e = launch_sweep(h->stencil_storage, rt, dry, h->vdone, h->status, 0, -1, h->stream);
      cudaEventRecord(a, h->stream);
      for (int w = 0; w < 3 && e == cudaSuccess; w++)
        e = launch_sweep(h->stencil_storage, rt, dry, h->vdone, h->status, 0, -1, h->stream);
      cudaEventRecord(b, h->stream);
    } else if (is_march(rt)) {
      const size_t need = march_smem_bytes(h->storage, rt);
      if (need == 0 || need > (size_t)maxsm) continue;
      if (march_planes(rt) > 16 && march_planes(rt) / 2 >= h->grid.nth) continue;  // same launch as a shorter run
      int rc = build_march_maps(h, rt);
      if (rc) return rc;
      KParams dry = h->kp;
      dry.src_i = -1;
      for (int w = 0; w < 2 && e == cudaSuccess; w++)
        e = launch_march(h->storage, rt, h->mmaps, dry, h->status, h->stream, nullptr);
      cudaEventRecord(a, h->stream);
      for (int w = 0; w < 3 && e == cudaSuccess; w++)
        e = launch_march(h->storage, rt, h->mmaps, dry, h->status, h->stream, nullptr);
      cudaEventRecord(b, h->stream);
    } else {
      const size_t need = rt >= 100 ? fused4_smem_bytes(h->storage, rt - 100) : fused_smem_bytes(h->storage, rt);
      if (need == 0 || need > (size_t)maxsm) continue;
      int rc = build_maps(h, rt);
      if (rc) return rc;
      FusedParams dry = h->fp[0];
      dry.k.src_i = -1;
      for (int w = 0; w < 2 && e == cudaSuccess; w++) e = launch_fused_any(h->storage, rt, h->maps[0], dry, h->stream);
      cudaEventRecord(a, h->stream);
      for (int w = 0; w < 3 && e == cudaSuccess; w++) e = launch_fused_any(h->storage, rt, h->maps[0], dry, h->stream);
      cudaEventRecord(b, h->stream);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e != cudaSuccess) {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      cudaEventDestroy(c3);
      return cuda_fail(h, e, "autotune launch");
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    if (ms < best) {
      best = ms;
      pick = rt;
    }
  }
  if (!forced && pick_v >= 0 && best_v + best_s < best) {  // the split family's best halves win
    pick = pick_v == pick_s ? pick_v : pick_v * 10000 + pick_s;
    // the halves within 3 % of the best ones, paired and timed again as they
    // run: whole steps in a captured graph, the edge launches on the side
    // stream (the times above are of separate launches, three at a time)
    auto near = [](std::vector<std::pair<float, int>> t, float b) {
      std::sort(t.begin(), t.end());
      std::vector<int> out;
      for (size_t q = 0; q < t.size() && out.size() < 3; q++)
        if (t[q].first <= 1.03f * b) out.push_back(t[q].second);
      return out;
    };
    const std::vector<int> nv = near(times_v, best_v), ns = near(times_s, best_s);
    if (nv.size() * ns.size() > 1) {
      KParams dry = h->kp;
      dry.src_i = -1;
      float best_pair = INFINITY;
      for (int v : nv)
        for (int c : ns) {
          const int code = v == c ? v : v * 10000 + c;
          cudaGraph_t graph = nullptr;
          cudaGraphExec_t exec = nullptr;
          cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
          for (int r = 0; r < 4 && e == cudaSuccess; r++)
            e = launch_split_family(h->stencil_storage, code, dry, h->stream, nullptr);
          cudaError_t e2 = cudaStreamEndCapture(h->stream, &graph);
          if (e == cudaSuccess) e = e2;
          if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
          if (e == cudaSuccess) e = cudaGraphLaunch(exec, h->stream);
          if (e == cudaSuccess) e = cudaEventRecord(a, h->stream);
          for (int r = 0; r < 3 && e == cudaSuccess; r++) e = cudaGraphLaunch(exec, h->stream);
          if (e == cudaSuccess) e = cudaEventRecord(b, h->stream);
          if (e == cudaSuccess) e = cudaEventSynchronize(b);
          if (exec) cudaGraphExecDestroy(exec);
          if (graph) cudaGraphDestroy(graph);
          if (e != cudaSuccess) {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            cudaEventDestroy(c3);
            return cuda_fail(h, e, "autotune graph");
          }
          float ms = 0;
          cudaEventElapsedTime(&ms, a, b);
          if (ms < best_pair) best_pair = ms, pick = code;
        }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaEventDestroy(c3);
  if (pick < 0 && forced)
    return fail(h, SIM_EINVAL, "opts.tile " + std::to_string(forced) + " is not a tile of the requested kernel that fits");
  if (pick < 0) return fail(h, SIM_EUNSUPPORTED, "no tile of the requested kernel fits in shared memory");
  if (!forced) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[key] = pick;
  }
  *best_rt = pick;
  return SIM_OK;
}

// slab == nullptr: the whole well; otherwise {s0, s1}: the z slab of stored
// cells s0 <= k < s1 (sim_create_slab)
static int create_impl(const sim_grid_t *grid, const sim_medium_t *medium, const sim_source_t *source,
                       const sim_receivers_t *receivers, const sim_opts_t *opts, const int *slab, sim_t **out) {
  if (!out) return fail(nullptr, SIM_EINVAL, "out is null");
  *out = nullptr;
  int rc = validate_inputs(grid, medium, source, receivers, opts);
  if (rc) return rc;
  const sim_grid_t &g = *grid;
  const int NR = g.nr + g.pml_r, NZg = g.nz + 2 * g.pml_z, nth = g.nth;
  // the stored z cells this handle holds: l0 <= k < l1 of the well (all of
  // them, or a slab with SLAB_GHOST ghost cells on each inner side)
  int l0 = 0, l1 = NZg, s0 = 0, s1 = NZg;
  if (slab) {
    s0 = slab[0];
    s1 = slab[1];
    if (s0 < 0 || s1 > NZg || s1 - s0 < 2 * SLAB_GHOST || (s0 % 4) || (s1 < NZg && (s1 % 4)))
      return fail(nullptr, SIM_EINVAL, "slab: need 0 <= s0 < s1 <= NZ, s1 - s0 >= 8, inner bounds multiples of 4");
    if (opts->storage != 0 || !(opts->kernel == SIM_KERNEL_AUTO || opts->kernel == SIM_KERNEL_SPLIT))
      return fail(nullptr, SIM_EUNSUPPORTED, "slab: FP32 storage on the split kernels only");
    l0 = std::max(0, s0 - SLAB_GHOST);
    l1 = std::min(NZg, s1 + SLAB_GHOST);
    if (g.pml_z > 0 && l1 - l0 < 2 * g.pml_z + 8)
      return fail(nullptr, SIM_EINVAL, "slab: fewer cells than two z layers and eight more");
  }
  const int NZ = l1 - l0;
  const int NZp = (NZ + 31) / 32 * 32;
  const size_t ncell = (size_t)nth * NR * NZg;
  const uint16_t *cid = medium->cell_id;
  // material IDs in range; ring 0 (the axis cells) must be a liquid
  for (size_t c = 0; c < ncell; c++)
    if (cid[c] >= medium->n_mat) return fail(nullptr, SIM_EINVAL, "medium: cell_id out of range at " + std::to_string(c));
  for (int j = 0; j < nth; j++)
    for (int k = 0; k < NZg; k++)
      if (medium->vs[cid[((size_t)j * NR) * NZg + k]] != 0.0)
        return fail(nullptr, SIM_EUNSUPPORTED, "medium: ring 0 (next to the axis) must be a liquid");

  sim_t *h = new sim_t();
  h->grid = g;
  h->NR = NR;
  h->NZ = NZ;
  h->NZp = NZp;
  h->slab = slab != nullptr;
  h->l0 = l0;
  h->s0 = s0;
  h->s1 = s1;
  h->stencil_storage = opts->storage;
  h->storage = opts->storage == SIM_STORAGE_F16_SR ? SIM_STORAGE_F16 : opts->storage;  // the stored format
  h->elem = opts->storage == 0 ? 4 : 2;
  // AUTO prepares the fused path and lets the autotuner fall back to the split
  // or marching kernels; the split and marching paths update one buffer set in place
  h->kernel = opts->kernel == SIM_KERNEL_SPLIT || slab ? SIM_KERNEL_SPLIT
              : opts->kernel == SIM_KERNEL_MARCH ? SIM_KERNEL_MARCH
              : opts->kernel == SIM_KERNEL_SWEEP ? SIM_KERNEL_SWEEP
                                                 : SIM_KERNEL_FUSED;
  h->src_kind = source->kind;
  // point forces and torsion are injected between the half-steps: in-place paths only
  if (h->src_kind != 0 && h->kernel == SIM_KERNEL_FUSED) h->kernel = SIM_KERNEL_AUTO;
  h->fused = h->kernel == SIM_KERNEL_FUSED;

  h->graph_chunk = opts->graph_chunk == 0 ? 64 : opts->graph_chunk;
  h->timing = opts->timing;
  h->mem_cap = opts->mem_cap;
  h->n_mat = medium->n_mat;
  h->n_rec = receivers->n;
  h->cap = opts->max_steps ? opts->max_steps : 65536;
  h->device = opts->device;
  auto bail = [&](int code) {
    if (code != SIM_OK) {
      g_create_err = h->err;
      release(h);
      delete h;
    }
    return code;
  };
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return bail(cuda_fail(h, e, "cudaSetDevice"));
  if (opts->cuda_stream) {
    h->stream = (cudaStream_t)opts->cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "cudaStreamCreate"));
    h->own_stream = true;
  }
  if ((e = cudaStreamCreateWithFlags(&h->side.side, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&h->side.fork, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&h->side.join, cudaEventDisableTiming)) != cudaSuccess)
    return bail(cuda_fail(h, e, "side stream"));

  // --- time step (reading R7)
  const double dth = 2.0 * M_PI / nth;
  h->dt = grid_time_step(g, medium);
  const double dt = h->dt;

  // --- storage scales (FP16 needs the velocities lifted by an impedance)
  long ks = lround(source->z / g.dz) + g.pml_z;
  int is = source->r < g.dr ? 0 : (int)floor(source->r / g.dr);
  int js = source->r < g.dr ? -1 : (int)(((lround(source->theta / dth) % nth) + nth) % nth);
  if (h->storage == 2) {
    int m0 = cid[((size_t)(js < 0 ? 0 : js) * NR + is) * NZg + ks];
    h->sscale = source->amplitude != 0 ? 1.0 / fabs(source->amplitude) : 1.0;
    h->vscale = h->sscale * medium->rho[m0] * medium->vp[m0];
  }

  // --- material table {rho, lambda, mu, 1/mu}; Lame from the cell-centre values
  std::vector<float4> mat(h->n_mat);
  std::vector<float> m_rho(h->n_mat), m_imu(h->n_mat);
  std::vector<float2> m_lam(h->n_mat);
  double vpmax = 0;
  for (int q = 0; q < h->n_mat; q++) {
    double rho = medium->rho[q], mu = rho * medium->vs[q] * medium->vs[q];
    double lam = rho * medium->vp[q] * medium->vp[q] - 2.0 * mu;
    mat[q] = make_float4((float)rho, (float)lam, (float)mu, mu > 0 ? (float)(1.0 / mu) : INFINITY);
    m_rho[q] = mat[q].x;
    m_imu[q] = mat[q].w;
    m_lam[q] = make_float2(mat[q].y, mat[q].y + 2.f * mat[q].z);
    vpmax = std::max(vpmax, medium->vp[q]);
  }
  // --- radius tables
  std::vector<float> inv_ri(NR), inv_rh(NR);
  for (int i = 0; i < NR; i++) {
    inv_ri[i] = i > 0 ? (float)(1.0 / (i * g.dr)) : 0.f;
    inv_rh[i] = (float)(1.0 / ((i + 0.5) * g.dr));
  }
  // --- PML: d(x) = d0 (x/L)^2, alpha = pi f0, dbar = (1/r) int d for the 1/r group
  const bool pml = !opts->pml_off;
  const double al = M_PI * source->f0;
  const double Lr = g.pml_r * g.dr, Lz = g.pml_z * g.dz;
  const double d0r = Lr > 0 ? -3.0 * vpmax * log(1e-3) / (2.0 * Lr) : 0.0;
  const double d0z = Lz > 0 ? -3.0 * vpmax * log(1e-3) / (2.0 * Lz) : 0.0;
  auto prof = [](double x, double L, double d0) { return (x > 0 && L > 0) ? d0 * (x / L) * (x / L) : 0.0; };
  auto profbar = [](double x, double r, double L, double d0) {
    return (x > 0 && L > 0 && r > 0) ? d0 * x * x * x / (3.0 * L * L) / r : 0.0;
  };
  std::vector<float4> ab_r(NR), ab_q(NR), ab_z(NZ);
  for (int i = 0; i < NR; i++) {
    double xi = pml ? (i - g.nr) * g.dr : 0.0, xh = pml ? (i + 0.5 - g.nr) * g.dr : 0.0;
    cpml(prof(xi, Lr, d0r), al, dt, &ab_r[i].x, &ab_r[i].y);
    cpml(prof(xh, Lr, d0r), al, dt, &ab_r[i].z, &ab_r[i].w);
    cpml(profbar(xi, i * g.dr, Lr, d0r), al, dt, &ab_q[i].x, &ab_q[i].y);
    cpml(profbar(xh, (i + 0.5) * g.dr, Lr, d0r), al, dt, &ab_q[i].z, &ab_q[i].w);
  }
  for (int k = 0; k < NZ; k++) {
    const int kg = k + l0;  // the well's stored index (a slab's profile is the well's)
    double xi = std::max((g.pml_z - 0.5 - kg) * g.dz, (kg - (g.pml_z + g.nz - 0.5)) * g.dz);
    double xh = std::max((g.pml_z - 1.0 - kg) * g.dz, (kg + 1.0 - g.pml_z - g.nz) * g.dz);
    if (!pml) xi = xh = 0.0;
    cpml(prof(xi, Lz, d0z), al, dt, &ab_z[k].x, &ab_z[k].y);
    cpml(prof(xh, Lz, d0z), al, dt, &ab_z[k].z, &ab_z[k].w);
  }
  // --- source wavelet: per-step increment dt * A * f(t_{n+1/2}) / V of the normal stresses
  const double vol = js < 0 ? M_PI * g.dr * g.dr * g.dz : (is + 0.5) * g.dr * g.dr * dth * g.dz;
  int n_pulse = (int)std::min<double>(ceil(8.0 / (source->f0 * dt)) + 1.0, 1e8);
  h->n_wav = std::max(1, std::min(n_pulse, std::max(h->cap, 1)));
  if (n_pulse > h->n_wav) h->n_wav = n_pulse;  // the pulse always fits
  std::vector<float> wav(h->n_wav);
  for (int n = 0; n < h->n_wav; n++)
    wav[n] = (float)(dt * source->amplitude * ricker((n + 0.5) * dt, source->f0) / vol * h->sscale);
  // --- point forces (R12) and the torsion ring (R13): injection points in stored units,
  // weight = dt * A * share / (rho_node V) (forces) or dt * A / (2 pi r dr dz) (torsion),
  // times the storage scale; wav2[n] = f(t_n) (forces) or f(t_{n+1/2}) (torsion)
  std::vector<int> ifld;
  std::vector<long long> ioff;
  std::vector<float> iw, iwav;
  if (source->kind != 0) {
    const bool axis = source->r < g.dr;
    const int jsrc = (int)(((lround(source->theta / dth) % nth) + nth) % nth);
    const double A = source->amplitude, dr = g.dr, dz = g.dz;
    auto hc = [&](int j, int i, long k) { return ((size_t)j * NR + i) * NZg + (size_t)k; };  // host cell
    auto dc = [&](int j, int i, long k) { return ((long long)j * NR + i) * NZp + (k - l0); };  // device element
    auto rho2 = [&](size_t a, size_t b) { return 0.5 * (medium->rho[cid[a]] + medium->rho[cid[b]]); };
    auto solid = [&](size_t c) { return medium->vs[cid[c]] > 0.0; };
    // every point of a source sits at depth k = ks; a slab that does not own
    // it injects nothing (the owner does, and the planes it sends carry it)
    const bool own_src = ks >= s0 && ks < s1;
    auto add = [&](int fld, long long off, double w) {
      if (!own_src) return;
      ifld.push_back(fld);
      ioff.push_back(off);
      iw.push_back((float)(dt * A * w * (fld <= F_VZ ? h->vscale : h->sscale)));
    };
    bool bad = false;
    const long k = ks;
    if (source->kind == 1) {
      if (axis) {
        for (int j = 0; j < nth; j++)
          add(F_VR, dc(j, 1, k), 2.0 * cos(j * dth - source->theta) / nth / (rho2(hc(j, 0, k), hc(j, 1, k)) * dr * dr * dth * dz));
      } else {
        const int i = (int)lround(source->r / dr);
        if (i < 1 || i >= NR) bad = true;
        else add(F_VR, dc(jsrc, i, k), 1.0 / (rho2(hc(jsrc, i - 1, k), hc(jsrc, i, k)) * i * dr * dr * dth * dz));
      }
    } else if (source->kind == 2) {
      if (k + 1 >= NZg) bad = true;
      else if (axis) {
        for (int j = 0; j < nth; j++)
          add(F_VZ, dc(j, 0, k), 1.0 / (rho2(hc(j, 0, k), hc(j, 0, k + 1)) * M_PI * dr * dr * dz));
      } else {
        const int i = (int)floor(source->r / dr);
        add(F_VZ, dc(jsrc, i, k), 1.0 / (rho2(hc(jsrc, i, k), hc(jsrc, i, k + 1)) * (i + 0.5) * dr * dr * dth * dz));
      }
    } else {
      const int i = (int)lround(source->r / dr), ih = (int)floor(source->r / dr);
      if (i < 1 || i >= NR || ih + 1 > NR || k + 1 >= NZg) bad = true;
      for (int j = 0; j < nth && !bad; j++) {
        const int jp = (j + 1) % nth;
        if (!(solid(hc(j, i - 1, k)) && solid(hc(j, i, k)) && solid(hc(jp, i - 1, k)) && solid(hc(jp, i, k)) &&
              solid(hc(j, ih, k)) && solid(hc(jp, ih, k)) && solid(hc(j, ih, k + 1)) && solid(hc(jp, ih, k + 1))))
          return bail(fail(h, SIM_EUNSUPPORTED, "source: the torsion ring needs a solid at both shear nodes"));
        add(F_SRP, dc(j, i, k), 1.0 / (2.0 * M_PI * i * dr * dr * dz));
        add(F_SPZ, dc(j, ih, k), 1.0 / (2.0 * M_PI * (ih + 0.5) * dr * dr * dz));
      }
    }
    if (bad) return bail(fail(h, SIM_EINVAL, "source: the force / torsion node falls outside the grid"));
    const bool force = source->kind != 3;
    iwav.resize(h->n_wav);
    for (int n = 0; n < h->n_wav; n++) iwav[n] = (float)ricker((force ? n : n + 0.5) * dt, source->f0);
  }
  // --- receivers
  std::vector<int> rec(3 * std::max(1, h->n_rec));
  for (int q = 0; q < h->n_rec; q++) {
    bool axis = receivers->r[q] < g.dr;
    rec[3 * q] = axis ? 0 : (int)floor(receivers->r[q] / g.dr);
    rec[3 * q + 1] = axis ? -1 : (int)(((lround(receivers->theta[q] / dth) % nth) + nth) % nth);
    const int kr = (int)(lround(receivers->z[q] / g.dz) + g.pml_z);
    rec[3 * q + 2] = (kr >= s0 && kr < s1) ? kr - l0 : -1;  // -1: another slab records it
  }

  // --- device memory
  const size_t fbytes = (size_t)nth * NR * NZp * h->elem;
  for (int q = 0; q < NF; q++)
    if ((rc = dev_alloc(h, &h->f[q], fbytes))) return bail(rc);
  h->psr_elems = (size_t)nth * g.pml_r * NZp;
  h->psz_elems = (size_t)nth * NR * 2 * g.pml_z;
  if (pml) {
    for (int q = 0; q < NPR; q++)
      if ((rc = dev_alloc(h, (void **)&h->psr[q], h->psr_elems * 4))) return bail(rc);
    for (int q = 0; q < NPZ; q++)
      if ((rc = dev_alloc(h, (void **)&h->psz[q], h->psz_elems * 4))) return bail(rc);
  }
  if (h->fused) {
    for (int q = 0; q < NF; q++)
      if ((rc = dev_alloc(h, &h->f2[q], fbytes))) return bail(rc);
    if (pml) {
      for (int q = 0; q < NPR; q++)
        if ((rc = dev_alloc(h, (void **)&h->psr2[q], h->psr_elems * 4))) return bail(rc);
      for (int q = 0; q < NPZ; q++)
        if ((rc = dev_alloc(h, (void **)&h->psz2[q], h->psz_elems * 4))) return bail(rc);
    }
  }
  if ((rc = dev_alloc(h, (void **)&h->id, (size_t)nth * NR * NZp * 2))) return bail(rc);
  if ((rc = dev_alloc(h, (void **)&h->mat, mat.size() * sizeof(float4)))) return bail(rc);
  if ((rc = dev_alloc(h, (void **)&h->m_rho, mat.size() * 4))) return bail(rc);
  if ((rc = dev_alloc(h, (void **)&h->m_imu, mat.size() * 4))) return bail(rc);
  if ((rc = dev_alloc(h, (void **)&h->m_lam, mat.size() * 8))) return bail(rc);
  if ((rc = dev_alloc(h, (void **)&h->ab_r, NR * sizeof(float4)))) return bail(rc);
  if ((rc = dev_alloc(h, (void **)&h->ab_q, NR * sizeof(float4)))) return bail(rc);
  if ((rc = dev_alloc(h, (void **)&h->ab_z, NZ * sizeof(float4)))) return bail(rc);
  if ((rc = dev_alloc(h, (void **)&h->inv_ri, NR * 4))) return bail(rc);
  if ((rc = dev_alloc(h, (void **)&h->inv_rh, NR * 4))) return bail(rc);
  if ((rc = dev_alloc(h, (void **)&h->wav, wav.size() * 4))) return bail(rc);
  if ((rc = dev_alloc(h, (void **)&h->rec, rec.size() * 4))) return bail(rc);
  if ((rc = dev_alloc(h, (void **)&h->traces, (size_t)std::max(1, h->n_rec) * h->cap * 4))) return bail(rc);
  if ((rc = dev_alloc(h, (void **)&h->step, 16))) return bail(rc);
  if ((rc = dev_alloc(h, (void **)&h->status, 16))) return bail(rc);
  if ((rc = dev_alloc(h, (void **)&h->vdone, (size_t)sweep_chunks(NZ) * sizeof(int)))) return bail(rc);
  int *d_ifld = nullptr;
  long long *d_ioff = nullptr;
  float *d_iw = nullptr, *d_iwav = nullptr;
  if (!ifld.empty()) {
    if ((rc = dev_alloc(h, (void **)&d_ifld, ifld.size() * 4))) return bail(rc);
    if ((rc = dev_alloc(h, (void **)&d_ioff, ioff.size() * 8))) return bail(rc);
    if ((rc = dev_alloc(h, (void **)&d_iw, iw.size() * 4))) return bail(rc);
    if ((rc = dev_alloc(h, (void **)&d_iwav, iwav.size() * 4))) return bail(rc);
  }

  cudaStream_t st = h->stream;
#define UP(dst, src, n) \
  if ((e = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, st)) != cudaSuccess) return bail(cuda_fail(h, e, "upload"))
  e = cudaMemcpy2DAsync(h->id, NZp * 2, cid + l0, NZg * 2, NZ * 2, (size_t)nth * NR, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return bail(cuda_fail(h, e, "upload cell_id"));
  UP(h->mat, mat.data(), mat.size() * sizeof(float4));
  UP(h->m_rho, m_rho.data(), mat.size() * 4);
  UP(h->m_imu, m_imu.data(), mat.size() * 4);
  UP(h->m_lam, m_lam.data(), mat.size() * 8);
  UP(h->ab_r, ab_r.data(), NR * sizeof(float4));
  UP(h->ab_q, ab_q.data(), NR * sizeof(float4));
  UP(h->ab_z, ab_z.data(), NZ * sizeof(float4));
  UP(h->inv_ri, inv_ri.data(), NR * 4);
  UP(h->inv_rh, inv_rh.data(), NR * 4);
  UP(h->wav, wav.data(), wav.size() * 4);
  UP(h->rec, rec.data(), rec.size() * 4);
  if (!ifld.empty()) {
    UP(d_ifld, ifld.data(), ifld.size() * 4);
    UP(d_ioff, ioff.data(), ioff.size() * 8);
    UP(d_iw, iw.data(), iw.size() * 4);
    UP(d_iwav, iwav.data(), iwav.size() * 4);
  }
#undef UP
  // pageable host sources: make the upload complete before the host vectors go away
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return bail(cuda_fail(h, e, "cudaStreamSynchronize"));

  KParams &p = h->kp;
  p.nth = nth;
  p.NR = NR;
  p.NZ = NZ;
  p.NZp = NZp;
  p.nr = g.nr;
  p.pml_r = pml ? g.pml_r : 0;
  p.pml_z = pml ? g.pml_z : 0;
  if (!pml) p.nr = NR;  // no radial layer at all
  p.plane = (long long)NR * NZp;
  p.dtv = (float)(dt * h->vscale / h->sscale);
  p.dts = (float)(dt * h->sscale / h->vscale);
  p.inv_dr = (float)(1.0 / g.dr);
  p.inv_dz = (float)(1.0 / g.dz);
  p.inv_dth = (float)(1.0 / dth);
  p.inv_ri = h->inv_ri;
  p.inv_rh = h->inv_rh;
  p.ab_r = h->ab_r;
  p.ab_q = h->ab_q;
  p.ab_z = h->ab_z;
  p.mat = h->mat;
  p.m_rho = h->m_rho;
  p.m_imu = h->m_imu;
  p.m_lam = h->m_lam;
  p.id = h->id;
  for (int q = 0; q < NF; q++) p.f[q] = h->f[q];
  for (int q = 0; q < NPR; q++) p.psr[q] = h->psr[q];
  for (int q = 0; q < NPZ; q++) p.psz[q] = h->psz[q];
  p.wav = h->wav;
  p.n_wav = h->n_wav;
  // the stress kernels inject only the volumetric source, and only in the
  // cells this handle owns
  p.src_i = (source->kind == 0 && ks >= s0 && ks < s1) ? is : -1;
  p.src_j = js;
  p.src_k = (int)ks - l0;
  p.k_lo = s0 - l0;
  p.k_hi = s1 - l0;
  p.step = h->step;
  p.i_lo = 0;
  p.i_hi = NR;
  h->ip.n = (int)ifld.size();
  h->ip.fld = d_ifld;
  h->ip.off = d_ioff;
  h->ip.w = d_iw;
  h->ip.wav = d_iwav;
  h->ip.n_wav = h->n_wav;
  h->ip.step = h->step;
  for (int q = 0; q < NF; q++) h->ip.f[q] = h->f[q];
  RParams &r = h->rp;
  r.nth = nth;
  r.NR = NR;
  r.NZp = NZp;
  r.n_rec = h->n_rec;
  r.cap = h->cap;
  r.plane = p.plane;
  r.srr = h->f[F_SRR];
  r.spp = h->f[F_SPP];
  r.szz = h->f[F_SZZ];
  r.rec = h->rec;
  r.scale = (float)(-1.0 / (3.0 * h->sscale));
  r.traces = h->traces;
  r.step = h->step;
  r.status = h->status;
  if (opts->watchdog_every > 0) {
    h->watch_every = opts->watchdog_every;
    if ((rc = dev_alloc(h, (void **)&h->watch_acc, 4 * sizeof(double)))) return bail(rc);
    if ((e = cudaMemsetAsync(h->watch_acc, 0, 4 * sizeof(double), st)) != cudaSuccess)
      return bail(cuda_fail(h, e, "watchdog"));
    int dev_sms = 0;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, h->device);
    h->watch_blocks = std::max(1, std::min(nth * NR, 4 * std::max(dev_sms, 1)));
    for (int par = 0; par < 2; par++) {
      WParams &w = h->wp[par];
      w.nth = nth;
      w.NR = NR;
      w.NZp = NZp;
      w.k_lo = std::max(0, s0 - l0);
      w.k_hi = std::min(NZ, s1 - l0);
      w.every = h->watch_every;
      // the last step of the source's wavelet tables: no injection after it
      w.n_quiet = std::max(h->n_wav, h->ip.n_wav);
      // the state after a step of parity par (the fused path writes the other set)
      void **cur = (h->fused && par == 0) ? h->f2 : h->f;
      for (int q = 0; q < NF; q++) w.f[q] = cur[q];
      w.id = h->id;
      w.m_rho = h->m_rho;
      w.m_lam = h->m_lam;
      w.iv2 = 1.0 / (h->vscale * h->vscale);
      w.is2 = 1.0 / (h->sscale * h->sscale);
      w.step = h->step;
      w.status = h->status;
      w.acc = h->watch_acc;
    }
  }
  if (h->fused) {
    for (int par = 0; par < 2; par++) {
      FusedParams &f = h->fp[par];
      f.k = p;
      void **cur = par == 0 ? h->f : h->f2, **nxt = par == 0 ? h->f2 : h->f;
      float **pc = par == 0 ? h->psr : h->psr2, **pn = par == 0 ? h->psr2 : h->psr;
      float **zc = par == 0 ? h->psz : h->psz2, **zn = par == 0 ? h->psz2 : h->psz;
      for (int q = 0; q < NF; q++) {
        f.k.f[q] = cur[q];
        f.fo[q] = nxt[q];
      }
      for (int q = 0; q < NPR; q++) {
        f.k.psr[q] = pc[q];
        f.psr_o[q] = pn[q];
      }
      for (int q = 0; q < NPZ; q++) {
        f.k.psz[q] = zc[q];
        f.psz_o[q] = zn[q];
      }
      f.status = h->status;
      // the stresses of step n + 1 are in the buffer this parity writes
      h->rp2[par] = r;
      h->rp2[par].srr = nxt[F_SRR];
      h->rp2[par].spp = nxt[F_SPP];
      h->rp2[par].szz = nxt[F_SZZ];
    }
    if ((rc = autotune(h, opts->kernel, opts->tile, &h->tile_rt))) return bail(rc);
    if (is_split_family(h->tile_rt)) {  // the split kernels won: run in place on the first buffer set
      h->fused = false;
      h->kernel = SIM_KERNEL_SPLIT;
    } else if (is_sweep(h->tile_rt)) {  // the sweep kernel won: in place as well
      h->fused = false;
      h->kernel = SIM_KERNEL_SWEEP;
    } else if (is_march(h->tile_rt)) {  // the marching kernels won: in place as well
      h->fused = false;
      h->kernel = SIM_KERNEL_MARCH;
    } else if ((rc = build_maps(h, h->tile_rt))) {
      return bail(rc);
    }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "autotune"));
  } else {  // the marching or the split kernels (asked for by name, or the in-place paths of AUTO)
    if ((rc = autotune(h, h->kernel, opts->tile, &h->tile_rt))) return bail(rc);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "autotune"));
    h->kernel = is_march(h->tile_rt) ? SIM_KERNEL_MARCH : is_sweep(h->tile_rt) ? SIM_KERNEL_SWEEP : SIM_KERNEL_SPLIT;
  }
  h->sweep = h->kernel == SIM_KERNEL_SWEEP;
  if (h->kernel == SIM_KERNEL_MARCH) {
    h->march = true;
    if ((rc = build_march_maps(h, h->tile_rt))) return bail(rc);
  }
  if (h->timing)
    for (auto &ev : h->ev)
      if ((e = cudaEventCreate(&ev)) != cudaSuccess) return bail(cuda_fail(h, e, "cudaEventCreate"));
  *out = h;
  return SIM_OK;
}

extern "C" int sim_create(const sim_grid_t *grid, const sim_medium_t *medium, const sim_source_t *source,
                          const sim_receivers_t *receivers, const sim_opts_t *opts, sim_t **out) {
  return create_impl(grid, medium, source, receivers, opts, nullptr, out);
}

extern "C" int sim_create_slab(const sim_grid_t *grid, const sim_medium_t *medium, const sim_source_t *source,
                               const sim_receivers_t *receivers, const sim_opts_t *opts, int s0, int s1,
                               sim_t **out) {
  const int slab[2] = {s0, s1};
  return create_impl(grid, medium, source, receivers, opts, slab, out);
}

// Enqueue one step; `parity` = index of the step mod 2 (fused path buffers).
static cudaError_t enqueue_step(sim_t *h, int parity, bool timed) {
  SideScope side_scope(h);
  cudaError_t e;
  if (h->fused) {
    if (timed) cudaEventRecord(h->ev[0], h->stream);
    e = launch_fused_any(h->storage, h->tile_rt, h->maps[parity], h->fp[parity], h->stream);
    if (e != cudaSuccess) return e;
    if (timed) {
      cudaEventRecord(h->ev[1], h->stream);
      cudaEventRecord(h->ev[2], h->stream);
    }
    e = launch_receivers(h->storage, h->rp2[parity], h->stream);
  } else if (h->sweep) {
    if (timed) cudaEventRecord(h->ev[0], h->stream);
    e = launch_sweep(h->stencil_storage, h->tile_rt, h->kp, h->vdone, h->status, h->wait_cycles, h->withhold_chunk,
                     h->stream);
    if (e != cudaSuccess) return e;
    if (timed) {
      cudaEventRecord(h->ev[1], h->stream);
      cudaEventRecord(h->ev[2], h->stream);
    }
    if (h->src_kind == 3) e = launch_inject(h->storage, h->ip, h->stream);  // the torsion ring after the step
    if (e == cudaSuccess) e = launch_receivers(h->storage, h->rp, h->stream);
  } else {
    // point forces act after the velocity kernel, the torsion ring after the stress kernel
    cudaEvent_t *ev = timed ? h->ev : nullptr;
    const bool force = h->src_kind == 1 || h->src_kind == 2;
    auto half = [&](int parts) {
      return h->march ? launch_march(h->storage, h->tile_rt, h->mmaps, h->kp, h->status, h->stream, ev, parts)
                      : launch_split_family(h->stencil_storage, h->tile_rt, h->kp, h->stream, ev, parts);
    };
    if (force) {
      e = half(1);
      if (e == cudaSuccess) e = launch_inject(h->storage, h->ip, h->stream);
      if (e == cudaSuccess) e = half(2);
    } else {
      e = half(3);
      if (e == cudaSuccess && h->src_kind == 3) e = launch_inject(h->storage, h->ip, h->stream);
    }
    if (e != cudaSuccess) return e;
    e = launch_receivers(h->storage, h->rp, h->stream);
  }
  if (e != cudaSuccess) return e;
  if (h->watch_every > 0) {
    e = launch_watchdog(h->storage, h->wp[parity], h->watch_blocks, h->stream);
    if (e != cudaSuccess) return e;
  }
  if (timed) {
    cudaEventRecord(h->ev[3], h->stream);
    e = cudaEventSynchronize(h->ev[3]);
    if (e != cudaSuccess) return e;
    float a = 0, b = 0, c = 0;
    cudaEventElapsedTime(&a, h->ev[0], h->ev[1]);
    cudaEventElapsedTime(&b, h->ev[1], h->ev[2]);
    cudaEventElapsedTime(&c, h->ev[2], h->ev[3]);
    h->kms[0] += a;
    h->kms[1] += b;
    h->kms[2] += c;
    h->kcount[0]++;
    h->kcount[1]++;
    h->kcount[2]++;
  }
  return cudaSuccess;
}

extern "C" int sim_step(sim_t *h, int nsteps) {
  if (!h) return SIM_EINVAL;
  if (nsteps < 0) return fail(h, SIM_EINVAL, "nsteps < 0");
  CK(h, cudaSetDevice(h->device));
  int left = nsteps;
  auto direct = [&]() -> int {
    cudaError_t e = enqueue_step(h, h->steps_done & 1, h->timing != 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "kernel launch");
    h->steps_done++;
    left--;
    return SIM_OK;
  };
  // a captured chunk starts on an even step (fused buffers alternate) and has even length
  int chunk = h->graph_chunk;
  if (h->fused && chunk > 0 && (chunk & 1)) chunk++;
  if (!h->timing && chunk > 0 && left >= chunk + (h->steps_done & 1)) {
    if (h->steps_done & 1) {
      int rc = direct();
      if (rc) return rc;
    }
    if (!h->gexec) {
      cudaGraph_t graph;
      CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = cudaSuccess;
      for (int q = 0; q < chunk && e == cudaSuccess; q++) e = enqueue_step(h, q & 1, false);
      cudaError_t e2 = cudaStreamEndCapture(h->stream, &graph);
      if (e != cudaSuccess) return cuda_fail(h, e, "kernel launch during capture");
      if (e2 != cudaSuccess) return cuda_fail(h, e2, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&h->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
      h->gsteps = chunk;
    }
    while (left >= h->gsteps) {
      CK(h, cudaGraphLaunch(h->gexec, h->stream));
      left -= h->gsteps;
      h->steps_done += h->gsteps;
    }
  }
  while (left > 0) {
    int rc = direct();
    if (rc) return rc;
  }
  return SIM_OK;
}

// buffers holding the current state (the fused path alternates two sets)
static void **cur_fields(sim_t *h) { return (h->fused && (h->steps_done & 1)) ? h->f2 : h->f; }
static float **cur_psr(sim_t *h) { return (h->fused && (h->steps_done & 1)) ? h->psr2 : h->psr; }
static float **cur_psz(sim_t *h) { return (h->fused && (h->steps_done & 1)) ? h->psz2 : h->psz; }

extern "C" int sim_half_step(sim_t *h, int which) {
  if (!h) return SIM_EINVAL;
  if (which != 0 && which != 1) return fail(h, SIM_EINVAL, "which must be 0 (velocity) or 1 (stress)");
  if (h->fused || h->march || h->sweep) return fail(h, SIM_EUNSUPPORTED, "half steps run on the split kernels only");
  CK(h, cudaSetDevice(h->device));
  SideScope side_scope(h);
  const bool force = h->src_kind == 1 || h->src_kind == 2;
  cudaError_t e = launch_split_family(h->stencil_storage, h->tile_rt, h->kp, h->stream, nullptr, which == 0 ? 1 : 2);
  if (e == cudaSuccess && ((which == 0 && force) || (which == 1 && h->src_kind == 3)))
    e = launch_inject(h->storage, h->ip, h->stream);
  if (e == cudaSuccess && which == 1) e = launch_receivers(h->storage, h->rp, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "half step");
  if (which == 1) h->steps_done++;
  return SIM_OK;
}

extern "C" int sim_slab_info(const sim_t *h, int *l0, int *s0, int *s1, int *nz_local) {
  if (!h) return SIM_EINVAL;
  if (l0) *l0 = h->l0;
  if (s0) *s0 = h->slab ? h->s0 : 0;
  if (s1) *s1 = h->slab ? h->s1 : h->NZ;
  if (nz_local) *nz_local = h->NZ;
  return SIM_OK;
}

// planes k0 <= k < k1 (the well's stored z index) of the velocities (group 0)
// or the stresses (group 1) to / from buf [field][nth * NR][k1 - k0]
static int copy_planes(sim_t *h, int group, int k0, int k1, void *buf, bool out) {
  if (!h) return SIM_EINVAL;
  if ((group != 0 && group != 1) || !buf) return fail(h, SIM_EINVAL, "group must be 0 or 1, buffer non-null");
  if (k0 < h->l0 || k1 > h->l0 + h->NZ || k0 >= k1)
    return fail(h, SIM_EINVAL, "planes outside the cells the handle holds");
  if (h->fused) return fail(h, SIM_EUNSUPPORTED, "plane copies run on the in-place paths");
  CK(h, cudaSetDevice(h->device));
  const int q0 = group == 0 ? F_VR : F_SRR, q1 = group == 0 ? F_SRR : NF;
  const size_t w = (size_t)(k1 - k0) * h->elem, rows = (size_t)h->grid.nth * h->NR;
  for (int q = q0; q < q1; q++) {
    char *f = (char *)h->f[q] + (size_t)(k0 - h->l0) * h->elem;
    char *b = (char *)buf + (size_t)(q - q0) * rows * w;
    cudaError_t e = out ? cudaMemcpy2DAsync(b, w, f, (size_t)h->NZp * h->elem, w, rows, cudaMemcpyDefault, h->stream)
                        : cudaMemcpy2DAsync(f, (size_t)h->NZp * h->elem, b, w, w, rows, cudaMemcpyDefault, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "plane copy");
  }
  return SIM_OK;
}

extern "C" int sim_get_planes(sim_t *h, int group, int k0, int k1, void *dst) {
  return copy_planes(h, group, k0, k1, dst, true);
}

extern "C" int sim_put_planes(sim_t *h, int group, int k0, int k1, const void *src) {
  return copy_planes(h, group, k0, k1, const_cast<void *>(src), false);
}

extern "C" int sim_sync(sim_t *h) {
  if (!h) return SIM_EINVAL;
  CK(h, cudaSetDevice(h->device));
  CK(h, cudaStreamSynchronize(h->stream));
  int st = 0;
  CK(h, cudaMemcpy(&st, h->status, 4, cudaMemcpyDeviceToHost));
  // a wait that gave up voids the state: report it first
  if (st & 2) return fail(h, SIM_ETIMEOUT, "a bounded device wait gave up");
  if (st & 1) return fail(h, SIM_EUNSTABLE, "non-finite value in the receiver traces");
  if (st & 8)
    return fail(h, SIM_EUNSTABLE, "watchdog: the energy proxy is not finite or grew past " +
                                      std::to_string((int)WATCH_GROWTH) + " times its value after the source");
  return SIM_OK;
}

extern "C" int sim_watchdog(sim_t *h, double *energy, double *reference, int *step) {
  if (!h) return SIM_EINVAL;
  if (h->watch_every <= 0) return fail(h, SIM_EINVAL, "the watchdog is off (opts.watchdog_every = 0)");
  CK(h, cudaSetDevice(h->device));
  CK(h, cudaStreamSynchronize(h->stream));
  double a[4];
  CK(h, cudaMemcpy(a, h->watch_acc, sizeof(a), cudaMemcpyDeviceToHost));
  if (energy) *energy = a[1];
  if (reference) *reference = a[2];
  if (step) *step = (int)a[3];
  return SIM_OK;
}

extern "C" int sim_traces(sim_t *h, float *out, size_t cap, int *n_rec, int *n_steps) {
  if (!h) return SIM_EINVAL;
  int rc = sim_sync(h);
  if (rc && rc != SIM_EUNSTABLE) return rc;
  int ns = std::min(h->steps_done, h->cap);
  if (n_rec) *n_rec = h->n_rec;
  if (n_steps) *n_steps = ns;
  if (!out) return rc;
  if (cap < (size_t)h->n_rec * ns) return fail(h, SIM_EINVAL, "output buffer too small");
  if (h->n_rec > 0 && ns > 0)
    CK(h, cudaMemcpy2D(out, (size_t)ns * 4, h->traces, (size_t)h->cap * 4, (size_t)ns * 4, h->n_rec,
                       cudaMemcpyDeviceToHost));
  return rc;
}

template <typename T>
__global__ void to_f32(const T *in, float *out, long long n, float scale) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q < n) out[q] = st_to_float<T>(in[q]) * scale;
}
template <typename T>
__global__ void from_f32(const float *in, T *out, long long n, float scale);
template <>
__global__ void from_f32<float>(const float *in, float *out, long long n, float scale) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q < n) out[q] = in[q] * scale;
}
template <>
__global__ void from_f32<__nv_bfloat16>(const float *in, __nv_bfloat16 *out, long long n, float scale) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q < n) out[q] = __float2bfloat16_rn(in[q] * scale);
}
template <>
__global__ void from_f32<__half>(const float *in, __half *out, long long n, float scale) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q < n) out[q] = __float2half_rn(in[q] * scale);
}

static double field_scale(const sim_t *h, int which) { return which <= F_VZ ? h->vscale : h->sscale; }

extern "C" int sim_read_field(sim_t *h, int which, float *out, size_t n) {
  if (!h) return SIM_EINVAL;
  if (which < 0 || which >= NF || !out) return fail(h, SIM_EINVAL, "bad field index or buffer");
  const size_t rows = (size_t)h->grid.nth * h->NR, need = rows * h->NZ;
  if (n < need) return fail(h, SIM_EINVAL, "output buffer too small");
  CK(h, cudaSetDevice(h->device));
  CK(h, cudaStreamSynchronize(h->stream));
  const long long tot = (long long)rows * h->NZp;
  float *tmp = nullptr;
  CK(h, cudaMalloc(&tmp, tot * 4));
  const float sc = (float)(1.0 / field_scale(h, which));
  int blocks = (int)((tot + 255) / 256);
  switch (h->storage) {
    case 0: to_f32<float><<<blocks, 256, 0, h->stream>>>((const float *)cur_fields(h)[which], tmp, tot, sc); break;
    case 1: to_f32<__nv_bfloat16><<<blocks, 256, 0, h->stream>>>((const __nv_bfloat16 *)cur_fields(h)[which], tmp, tot, sc); break;
    default: to_f32<__half><<<blocks, 256, 0, h->stream>>>((const __half *)cur_fields(h)[which], tmp, tot, sc); break;
  }
  cudaError_t e = cudaMemcpy2DAsync(out, h->NZ * 4, tmp, h->NZp * 4, h->NZ * 4, rows, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(h, e, "read field");
  return SIM_OK;
}

// ---------------------------------------------------------------------------
// Field read-back without allocation.  Same result as sim_read_field, but the
// storage-to-FP32 conversion is staged in this fixed device array instead of a
// buffer obtained from cudaMalloc.  The array lives in device memory of every
// GPU that loads the library, until the process exits.  In host code its name
// is only a stand-in for the symbol: the kernel gets the device address that
// cudaGetSymbolAddress returns for the current device.
#define SIM_NOALLOC_SCRATCH_FLOATS (4u << 20) /* 16 MiB: fields of up to 4 Mi padded cells */
static __device__ __align__(256) float g_field_scratch[SIM_NOALLOC_SCRATCH_FLOATS];
static std::mutex g_scratch_mu;
static float *g_scratch_addr[64] = {};

// device address of the scratch array on the current device, looked up once per device
static int scratch_address(sim_t *h, float **out) {
  std::lock_guard<std::mutex> g(g_scratch_mu);
  if (h->device < 0 || h->device >= 64) return fail(h, SIM_EINVAL, "device ordinal out of range for the scratch table");
  if (!g_scratch_addr[h->device]) {
    float *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&p, g_field_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(h, e, "cudaGetSymbolAddress(g_field_scratch)");
    g_scratch_addr[h->device] = p;
  }
  *out = g_scratch_addr[h->device];
  return SIM_OK;
}

extern "C" int sim_read_field_noalloc(sim_t *h, int which, float *out, size_t n) {
  if (!h) return SIM_EINVAL;
  if (which < 0 || which >= NF || !out) return fail(h, SIM_EINVAL, "bad field index or buffer");
  const size_t rows = (size_t)h->grid.nth * h->NR, need = rows * h->NZ;
  if (n < need) return fail(h, SIM_EINVAL, "output buffer too small");
  const long long tot = (long long)rows * h->NZp;
  if (tot > (long long)SIM_NOALLOC_SCRATCH_FLOATS)
    return fail(h, SIM_EINVAL, "field of " + std::to_string(tot) + " padded cells exceeds the " +
                                   std::to_string(SIM_NOALLOC_SCRATCH_FLOATS) + "-float scratch of sim_read_field_noalloc");
  CK(h, cudaSetDevice(h->device));
  float *tmp = nullptr;
  int rc = scratch_address(h, &tmp);
  if (rc) return rc;
  CK(h, cudaStreamSynchronize(h->stream));
  const float sc = (float)(1.0 / field_scale(h, which));
  const int blocks = (int)((tot + 255) / 256);
  switch (h->storage) {  // every element the copy reads is written here: nothing needs clearing
    case 0: to_f32<float><<<blocks, 256, 0, h->stream>>>((const float *)cur_fields(h)[which], tmp, tot, sc); break;
    case 1: to_f32<__nv_bfloat16><<<blocks, 256, 0, h->stream>>>((const __nv_bfloat16 *)cur_fields(h)[which], tmp, tot, sc); break;
    default: to_f32<__half><<<blocks, 256, 0, h->stream>>>((const __half *)cur_fields(h)[which], tmp, tot, sc); break;
  }
  CK(h, cudaGetLastError());
  CK(h, cudaMemcpy2DAsync(out, h->NZ * 4, tmp, h->NZp * 4, h->NZ * 4, rows, cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return SIM_OK;
}

extern "C" int sim_write_field(sim_t *h, int which, const float *in, size_t n) {
  if (!h) return SIM_EINVAL;
  if (which < 0 || which >= NF || !in) return fail(h, SIM_EINVAL, "bad field index or buffer");
  const size_t rows = (size_t)h->grid.nth * h->NR, need = rows * h->NZ;
  if (n < need) return fail(h, SIM_EINVAL, "input buffer too small");
  CK(h, cudaSetDevice(h->device));
  const long long tot = (long long)rows * h->NZp;
  float *tmp = nullptr;
  CK(h, cudaMalloc(&tmp, tot * 4));
  cudaError_t e = cudaMemsetAsync(tmp, 0, tot * 4, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(tmp, h->NZp * 4, in, h->NZ * 4, h->NZ * 4, rows, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) {
    const float sc = (float)field_scale(h, which);
    int blocks = (int)((tot + 255) / 256);
    switch (h->storage) {
      case 0: from_f32<float><<<blocks, 256, 0, h->stream>>>(tmp, (float *)cur_fields(h)[which], tot, sc); break;
      case 1: from_f32<__nv_bfloat16><<<blocks, 256, 0, h->stream>>>(tmp, (__nv_bfloat16 *)cur_fields(h)[which], tot, sc); break;
      default: from_f32<__half><<<blocks, 256, 0, h->stream>>>(tmp, (__half *)cur_fields(h)[which], tot, sc); break;
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(h, e, "write field");
  return SIM_OK;
}

extern "C" double sim_dt(const sim_t *h) { return h ? h->dt : 0.0; }
extern "C" int sim_steps_done(const sim_t *h) { return h ? h->steps_done : -1; }
extern "C" size_t sim_device_bytes(const sim_t *h) { return h ? h->bytes : 0; }

extern "C" int sim_config(const sim_t *h, int *kernel, int *tile_rows) {
  if (!h) return SIM_EINVAL;
  if (kernel) *kernel = h->kernel;
  if (tile_rows) *tile_rows = h->tile_rt;
  return SIM_OK;
}

extern "C" int sim_set_wait_test(sim_t *h, long long wait_cycles, int withhold_chunk) {
  if (!h) return SIM_EINVAL;
  if (wait_cycles < 0 || withhold_chunk < -1 || withhold_chunk >= sweep_chunks(h->NZ))
    return fail(h, SIM_EINVAL, "wait_cycles >= 0 and -1 <= withhold_chunk < ceil(NZ / 32) required");
  CK(h, cudaSetDevice(h->device));
  CK(h, cudaStreamSynchronize(h->stream));
  h->wait_cycles = wait_cycles;
  h->withhold_chunk = withhold_chunk;
  if (h->gexec) {  // the captured steps carry the old values
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  return SIM_OK;
}

extern "C" int sim_kernel_time(sim_t *h, int q, double *ms, long *launches) {
  if (!h) return SIM_EINVAL;
  if (q < 0 || q > 2) return fail(h, SIM_EINVAL, "kernel slot out of range");
  if (!h->timing) return fail(h, SIM_EINVAL, "handle was created without opts.timing");
  CK(h, cudaStreamSynchronize(h->stream));
  if (ms) *ms = h->kms[q];
  if (launches) *launches = h->kcount[q];
  return SIM_OK;
}

// checkpoint file: magic, sizes, step counter, raw device arrays in order
static const char kMagic[8] = {'C', 'W', 'E', 'L', 'L', 'C', 'K', '1'};

extern "C" int sim_save(sim_t *h, const char *path) {
  if (!h) return SIM_EINVAL;
  if (!path) return fail(h, SIM_EINVAL, "null path");
  CK(h, cudaSetDevice(h->device));
  CK(h, cudaStreamSynchronize(h->stream));
  FILE *fp = fopen(path, "wb");
  if (!fp) return fail(h, SIM_EINVAL, std::string("cannot open ") + path);
  long long hdr[8] = {h->grid.nth, h->NR, h->NZp, (long long)h->elem, (long long)h->psr_elems,
                      (long long)h->psz_elems, h->steps_done, (long long)h->n_rec * h->cap};
  bool ok = fwrite(kMagic, 1, 8, fp) == 8 && fwrite(hdr, sizeof(hdr), 1, fp) == 1;
  std::vector<char> buf;
  auto dump = [&](const void *dptr, size_t bytes) {
    if (!ok || !dptr) return;
    buf.resize(bytes);
    ok = cudaMemcpy(buf.data(), dptr, bytes, cudaMemcpyDeviceToHost) == cudaSuccess &&
         fwrite(buf.data(), 1, bytes, fp) == bytes;
  };
  const size_t fbytes = (size_t)h->grid.nth * h->NR * h->NZp * h->elem;
  for (int q = 0; q < NF; q++) dump(cur_fields(h)[q], fbytes);
  for (int q = 0; q < NPR; q++) dump(cur_psr(h)[q], h->psr_elems * 4);
  for (int q = 0; q < NPZ; q++) dump(cur_psz(h)[q], h->psz_elems * 4);
  dump(h->traces, (size_t)h->n_rec * h->cap * 4);
  dump(h->step, 4);
  if (fclose(fp) != 0) ok = false;
  return ok ? SIM_OK : fail(h, SIM_EINVAL, "checkpoint write failed");
}

extern "C" int sim_load(sim_t *h, const char *path) {
  if (!h) return SIM_EINVAL;
  if (!path) return fail(h, SIM_EINVAL, "null path");
  CK(h, cudaSetDevice(h->device));
  CK(h, cudaStreamSynchronize(h->stream));
  FILE *fp = fopen(path, "rb");
  if (!fp) return fail(h, SIM_EINVAL, std::string("cannot open ") + path);
  char mg[8];
  long long hdr[8];
  bool ok = fread(mg, 1, 8, fp) == 8 && memcmp(mg, kMagic, 8) == 0 && fread(hdr, sizeof(hdr), 1, fp) == 1;
  ok = ok && hdr[0] == h->grid.nth && hdr[1] == h->NR && hdr[2] == h->NZp && hdr[3] == (long long)h->elem &&
       hdr[4] == (long long)h->psr_elems && hdr[5] == (long long)h->psz_elems &&
       hdr[7] == (long long)h->n_rec * h->cap;
  if (!ok) {
    fclose(fp);
    return fail(h, SIM_EINVAL, "checkpoint does not match this handle");
  }
  const int prev_steps = h->steps_done;
  h->steps_done = (int)hdr[6];
  std::vector<char> buf;
  auto load = [&](void *dptr, size_t bytes) {
    if (!ok || !dptr) return;
    buf.resize(bytes);
    ok = fread(buf.data(), 1, bytes, fp) == bytes &&
         cudaMemcpy(dptr, buf.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  const size_t fbytes = (size_t)h->grid.nth * h->NR * h->NZp * h->elem;
  for (int q = 0; q < NF; q++) load(cur_fields(h)[q], fbytes);
  for (int q = 0; q < NPR; q++) load(cur_psr(h)[q], h->psr_elems * 4);
  for (int q = 0; q < NPZ; q++) load(cur_psz(h)[q], h->psz_elems * 4);
  load(h->traces, (size_t)h->n_rec * h->cap * 4);
  load(h->step, 4);
  fclose(fp);
  // the watchdog takes its reference again from the restored run
  if (ok && h->watch_acc) ok = cudaMemset(h->watch_acc, 0, 4 * sizeof(double)) == cudaSuccess;
  if (!ok) {
    h->steps_done = prev_steps;
    return fail(h, SIM_EINVAL, "checkpoint read failed");
  }
  return SIM_OK;
}

extern "C" void sim_destroy(sim_t *h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  release(h);
  delete h;
}

extern "C" const char *sim_last_error(const sim_t *h) { return h ? h->err.c_str() : g_create_err.c_str(); }

extern "C" const char *sim_error_string(int code) {
  switch (code) {
    case SIM_OK: return "ok";
    case SIM_EINVAL: return "invalid argument";
    case SIM_ENOMEM: return "out of device memory";
    case SIM_ECUDA: return "CUDA error";
    case SIM_EUNSTABLE: return "unstable (non-finite field)";
    case SIM_ETIMEOUT: return "device wait timed out";
    case SIM_EUNSUPPORTED: return "unsupported";
  }
  return "unknown error";
}
