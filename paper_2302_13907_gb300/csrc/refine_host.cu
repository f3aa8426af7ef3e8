// Azimuthally refined grid (paper Sec. 3, "Azimuth grid refinement"): the
// rows form M radial zones, zone m with nth / 2^(M-1-m) azimuthal nodes (the
// node count doubles at each interface going outward).  Every zone is stored
// as a uniform grid of its own, [nth_m][rows + ghost rows][NZp] per field,
// with one ghost row below (m > 0: the coarser zone's last row at this zone's
// nodes) and one above (m < M-1: the finer zone's first row at this zone's
// nodes).  A step is
//   velocity half of every zone (the single well's interior / edge split
//   launches, zone by zone, ghost rows excluded) -> point force -> ghost rows
//   of the velocities -> stress half of every zone (volumetric source
//   inside) -> ghost rows of the stresses -> receivers (one block per zone,
//   which also advances the zone's step counter).
// Ghost rows: coarse -> fine by the trigonometric interpolant (the paper's
// FFT zero-padding, here as its matrix: the periodic Dirichlet kernel with
// the Nyquist term halved), fine -> coarse by its adjoint
// (dtheta_fine / dtheta_coarse) P^T, so that the scheme's discrete energy
// is exact across the interface.  Fields on half-integer azimuth nodes
// (v_phi, s_rphi, s_phiz) use the interpolant evaluated half a fine step
// off the coarse nodes.  Materials of a ghost row below: fine node j takes
// the coarse cell floor(j / 2).  FP32 storage; the four source kinds.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "sim_state.cuh"

namespace {

struct RZone {
  int row = 0, rows = 0, nth = 0, g_lo = 0, g_hi = 0, NR = 0;  // first global row, own rows, nodes, ghost rows, stored rows
  int n_rec = 0, rec0 = 0;                                      // its receivers: trace rows rec0 ..
  float *f[NF] = {};
  float *psr[NPR] = {};
  float *psz[NPZ] = {};
  uint16_t *id = nullptr;
  float4 *ab_r = nullptr, *ab_q = nullptr;
  float *inv_ri = nullptr, *inv_rh = nullptr;
  int *rec = nullptr, *step = nullptr;
  KParams kp{};
  RParams rp{};
};

thread_local std::string g_refine_err;

}  // namespace

struct simr_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // streams of the zones other than the largest in each half (forked from
  // `stream` by zfork, joined back by zjoin): the zones of a half update
  // disjoint arrays from inputs no launch of the half writes
  static constexpr int MAX_ZSTREAMS = 7;
  cudaStream_t zs[MAX_ZSTREAMS] = {};
  cudaEvent_t zfork = nullptr, zjoin[MAX_ZSTREAMS] = {};
  int big_zone = 0;
  bool zone_streams = false;
  int vel_code = 0, str_code = 0;  // split codes of every zone's halves
  sim_grid_t grid{};
  int NR = 0, NZ = 0, NZp = 0, M = 0;
  double dt = 0;
  int n_rec = 0, cap = 0, steps_done = 0, graph_chunk = 64, src_kind = 0;
  std::vector<RZone> z;
  std::vector<int> trace_row;  // device trace row of each receiver
  std::vector<KParams> kps;
  float4 *mat = nullptr, *ab_z = nullptr;
  float *m_rho = nullptr, *m_imu = nullptr, *wav = nullptr, *traces = nullptr, *mats = nullptr;
  float2 *m_lam = nullptr;
  int *status = nullptr;
  int n_wav = 0;
  RParams *d_rp = nullptr;
  IParams ip{};
  XferParams xv{}, xs{};
  size_t bytes = 0, mem_cap = 0;
  std::vector<void *> allocs;
  cudaGraphExec_t gexec = nullptr;
  int gsteps = 0;
  std::string err;
};

namespace {

int rfail(simr_t *h, int code, const std::string &msg) {
  if (h) h->err = msg;
  else g_refine_err = msg;
  return code;
}
int rcuda(simr_t *h, cudaError_t e, const char *what) {
  return rfail(h, SIM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int ralloc(simr_t *h, void **p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  if (h->mem_cap && h->bytes + bytes > h->mem_cap)
    return rfail(h, SIM_ENOMEM, "device memory cap exceeded (" + std::to_string(h->bytes + bytes) + " bytes)");
  // stream-ordered: freeing a handle then waits for nothing but its own
  // stream, so handles on other streams keep running
  cudaError_t e = cudaMallocAsync(p, bytes, h->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return rfail(h, SIM_ENOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
  }
  h->allocs.push_back(*p);
  h->bytes += bytes;
  e = cudaMemsetAsync(*p, 0, bytes, h->stream);
  if (e != cudaSuccess) return rcuda(h, e, "cudaMemsetAsync");
  return SIM_OK;
}

void rrelease(simr_t *h) {
  if (!h) return;
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  for (void *p : h->allocs) cudaFreeAsync(p, h->stream);
  h->allocs.clear();
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (int k = 0; k < simr_t::MAX_ZSTREAMS; k++) {
    if (h->zs[k]) cudaStreamDestroy(h->zs[k]);
    if (h->zjoin[k]) cudaEventDestroy(h->zjoin[k]);
  }
  if (h->zfork) cudaEventDestroy(h->zfork);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

// periodic interpolation kernel of N samples with the Nyquist term halved:
// D(t) = (1/N) [1 + 2 sum_{m=1}^{N/2-1} cos(m t) + cos(N t / 2)]
double dirichlet(int N, double t) {
  double s = 1.0 + cos(0.5 * N * t);
  for (int m = 1; m < N / 2; m++) s += 2.0 * cos(m * t);
  return s / N;
}

bool pow2_in(int n) { return n == 4 || n == 8 || n == 16 || n == 32 || n == 64; }

// split codes each zone's halves run with, the fastest pairs measured: plain
// interior + prefetching edge for the velocities; for the stresses on a grid
// whose largest zone fills the GPU (the 20 m well) the three-way split with
// the zones on parallel streams, on a smaller one (a 1.6 m crop, several
// handles side by side) the prefetching interior and edge kernels with the
// zones one after another, whose fewer launches pay there
constexpr int REFINED_VEL_CODE = 2285, REFINED_STR_CODE = 2324, REFINED_STR_CODE_SMALL = 2294;
constexpr long long ZONE_STREAM_CELLS = 8LL << 20;
// opts.tile of a refined handle: 0, or a split code or pair code whose halves
// are interior / edge (22xx) or three-way (23xx) split codes
bool refined_tile_ok(int t) {
  auto ok = [](int c) { return c >= 2200 && c < 2400; };
  return t == 0 || (is_split_single(t) && ok(t)) || (is_split_pair(t) && ok(split_vel_code(t)) && ok(split_str_code(t)));
}

// one half of every zone: the largest zone on the handle's stream, each other
// zone on a stream of its own forked from it, all joined back before the
// interface transfer that follows.  Only where the largest zone fills the GPU
// by itself (ZONE_STREAM_CELLS): on small grids the zones run one after
// another, since several such handles usually run side by side already and the
// extra streams there cost more than they overlap.
cudaError_t zones_half(simr_t *h, int code, int parts) {
  const int nz = h->zone_streams ? (int)h->kps.size() : 1;
  if (!h->zone_streams) {  // one after another on the handle's stream
    cudaError_t e = cudaSuccess;
    for (size_t m = 0; m < h->kps.size() && e == cudaSuccess; m++) e = launch_hoist(0, code, h->kps[m], h->stream, nullptr, parts);
    return e;
  }
  cudaError_t e = cudaSuccess;
  if (nz > 1) {
    e = cudaEventRecord(h->zfork, h->stream);
    for (int k = 0; k < nz - 1 && e == cudaSuccess; k++) e = cudaStreamWaitEvent(h->zs[k], h->zfork, 0);
  }
  for (int m = 0, k = 0; m < nz && e == cudaSuccess; m++) {
    const cudaStream_t st = m == h->big_zone ? h->stream : h->zs[k++];
    e = launch_hoist(0, code, h->kps[m], st, nullptr, parts);
  }
  for (int k = 0; k < nz - 1 && e == cudaSuccess; k++) {
    e = cudaEventRecord(h->zjoin[k], h->zs[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->zjoin[k], 0);
  }
  return e;
}

cudaError_t enqueue_refined_step(simr_t *h) {
  cudaError_t e = cudaSuccess;
  const bool force = h->src_kind == 1 || h->src_kind == 2;
  e = zones_half(h, h->vel_code, 1);
  if (e == cudaSuccess && force) e = launch_inject(0, h->ip, h->stream);
  if (e == cudaSuccess) e = launch_xfer(h->xv, h->stream);
  if (e == cudaSuccess) e = zones_half(h, h->str_code, 2);
  if (e == cudaSuccess && h->src_kind == 3) e = launch_inject(0, h->ip, h->stream);
  if (e == cudaSuccess) e = launch_xfer(h->xs, h->stream);
  if (e == cudaSuccess) e = launch_batch_receivers(0, h->d_rp, (int)h->kps.size(), h->stream);
  return e;
}

}  // namespace

extern "C" int simr_interface_matrix(int n_coarse, int half, int fine_to_coarse, double *out) {
  if (!out || n_coarse < 4 || (n_coarse & 1)) return SIM_EINVAL;
  const int na = n_coarse, nb = 2 * na;
  const double hb = 2.0 * M_PI / nb;
  for (int jb = 0; jb < nb; jb++)
    for (int ja = 0; ja < na; ja++) {
      const double d = dirichlet(na, (jb - 2 * ja - (half ? 0.5 : 0.0)) * hb);
      if (fine_to_coarse) out[(size_t)ja * nb + jb] = 0.5 * d;  // (dtheta_fine / dtheta_coarse) P^T
      else out[(size_t)jb * na + ja] = d;
    }
  return SIM_OK;
}

extern "C" int simr_create(const sim_grid_t *grid, const simr_zones_t *zones, const sim_medium_t *medium,
                           const sim_source_t *source, const sim_receivers_t *receivers, const sim_opts_t *opts,
                           simr_t **out) {
  if (!out) return rfail(nullptr, SIM_EINVAL, "out is null");
  *out = nullptr;
  if (!zones) return rfail(nullptr, SIM_EINVAL, "zones is null");
  int rc = validate_inputs(grid, medium, source, receivers, opts);
  if (rc) return rfail(nullptr, rc, g_create_err);
  const sim_grid_t &g = *grid;
  const int M = zones->n_zones, NR = g.nr + g.pml_r, NZ = g.nz + 2 * g.pml_z, NZp = (NZ + 31) / 32 * 32;
  if (opts->storage != 0) return rfail(nullptr, SIM_EUNSUPPORTED, "refined grid: FP32 storage only");
  if (opts->watchdog_every != 0)
    return rfail(nullptr, SIM_EUNSUPPORTED, "refined grid: no device watchdog (uniform-grid handles only)");
  if (opts->kernel != SIM_KERNEL_AUTO && opts->kernel != SIM_KERNEL_SPLIT)
    return rfail(nullptr, SIM_EUNSUPPORTED, "refined grid: the split kernels only");
  if (!refined_tile_ok(opts->tile))
    return rfail(nullptr, SIM_EINVAL, "refined grid: opts.tile must be 0 or a 22xx / 23xx split code or pair");
  if (M < 1 || M > 5 || (M > 1 && !zones->row0)) return rfail(nullptr, SIM_EINVAL, "zones: 1 to 5 zones");
  const int nth0 = g.nth >> (M - 1);
  if (nth0 < 4 || (nth0 << (M - 1)) != g.nth || (nth0 & 1))
    return rfail(nullptr, SIM_EINVAL, "zones: nth / 2^(M-1) must be an even integer >= 4");
  if (M > 1 && !pow2_in(g.nth)) return rfail(nullptr, SIM_EINVAL, "zones: nth must be 8, 16, 32 or 64 with interfaces");
  std::vector<int> row0(M + 1);
  row0[0] = 0;
  row0[M] = NR;
  for (int m = 1; m < M; m++) {
    row0[m] = zones->row0[m - 1];
    if (row0[m] < row0[m - 1] + 2 || row0[m] > g.nr - 2)
      return rfail(nullptr, SIM_EINVAL, "zones: interface rows increasing, 2 rows per zone, radial PML in the last zone");
  }
  const size_t ncell = (size_t)g.nth * NR * NZ;
  const uint16_t *cid = medium->cell_id;
  for (size_t c = 0; c < ncell; c++)
    if (cid[c] >= medium->n_mat) return rfail(nullptr, SIM_EINVAL, "medium: cell_id out of range");
  for (int j = 0; j < g.nth; j++)
    for (int k = 0; k < NZ; k++)
      if (medium->vs[cid[((size_t)j * NR) * NZ + k]] != 0.0)
        return rfail(nullptr, SIM_EUNSUPPORTED, "medium: ring 0 (next to the axis) must be a liquid");
  auto zone_of = [&](int i) {
    int m = 0;
    while (m + 1 < M && i >= row0[m + 1]) m++;
    return m;
  };
  auto fine = [&](int j, int i, int k) { return cid[((size_t)j * NR + i) * NZ + k]; };  // finest-grid cell ID
  auto zone_id = [&](int m, int j, int i, int k) { return fine(j << (M - 1 - m), i, k); };  // zone m's cell j
  if ((source->kind == 1 || source->kind == 3) && source->r >= g.dr) {
    const int i = (int)lround(source->r / g.dr);
    if (i >= 1 && i < NR && zone_of(i - 1) != zone_of(i))
      return rfail(nullptr, SIM_EUNSUPPORTED, "source: the force's v_r node or the torsion ring's s_rphi row is the first row of a zone");
  }

  simr_t *h = new simr_t();
  h->grid = g;
  h->NR = NR;
  h->NZ = NZ;
  h->NZp = NZp;
  h->M = M;
  h->device = opts->device;
  h->mem_cap = opts->mem_cap;
  h->graph_chunk = opts->graph_chunk == 0 ? 64 : opts->graph_chunk;
  h->n_rec = receivers->n;
  h->cap = opts->max_steps ? opts->max_steps : 65536;
  h->src_kind = source->kind;
  auto bail = [&](int code) {
    g_refine_err = h->err;
    rrelease(h);
    delete h;
    return code;
  };
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return bail(rcuda(h, e, "cudaSetDevice"));
  if (opts->cuda_stream) {
    h->stream = (cudaStream_t)opts->cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(rcuda(h, e, "cudaStreamCreate"));
    h->own_stream = true;
  }

  // --- time step: R7 with each row's own azimuthal step
  if (g.dt > 0) {
    h->dt = g.dt;
  } else {
    double best = INFINITY;
    for (int i = 0; i < NR; i++) {
      const int m = zone_of(i), n = g.nth >> (M - 1 - m);
      double cmax = 0.0;
      for (int j = 0; j < n; j++)
        for (int k = 0; k < NZ; k++) cmax = std::max(cmax, medium->vp[zone_id(m, j, i, k)]);
      const double rc = (i + 0.5) * g.dr, dth = 2.0 * M_PI / n;
      const double s = sqrt(1.0 / (g.dr * g.dr) + 1.0 / ((rc * dth) * (rc * dth)) + 1.0 / (g.dz * g.dz));
      best = std::min(best, 1.0 / (cmax * s));
    }
    h->dt = g.cfl * best;
  }
  const double dt = h->dt;

  // --- material table, z PML profile (as the uniform grid)
  std::vector<float4> mat(medium->n_mat);
  std::vector<float> m_rho(medium->n_mat), m_imu(medium->n_mat);
  std::vector<float2> m_lam(medium->n_mat);
  double vpmax = 0;
  for (int q = 0; q < medium->n_mat; q++) {
    double rho = medium->rho[q], mu = rho * medium->vs[q] * medium->vs[q];
    double lam = rho * medium->vp[q] * medium->vp[q] - 2.0 * mu;
    mat[q] = make_float4((float)rho, (float)lam, (float)mu, mu > 0 ? (float)(1.0 / mu) : INFINITY);
    m_rho[q] = mat[q].x;
    m_imu[q] = mat[q].w;
    m_lam[q] = make_float2(mat[q].y, mat[q].y + 2.f * mat[q].z);
    vpmax = std::max(vpmax, medium->vp[q]);
  }
  const bool pml = !opts->pml_off;
  const double al = M_PI * source->f0;
  const double Lr = g.pml_r * g.dr, Lz = g.pml_z * g.dz;
  const double d0r = Lr > 0 ? -3.0 * vpmax * log(1e-3) / (2.0 * Lr) : 0.0;
  const double d0z = Lz > 0 ? -3.0 * vpmax * log(1e-3) / (2.0 * Lz) : 0.0;
  auto prof = [](double x, double L, double d0) { return (x > 0 && L > 0) ? d0 * (x / L) * (x / L) : 0.0; };
  auto profbar = [](double x, double r, double L, double d0) {
    return (x > 0 && L > 0 && r > 0) ? d0 * x * x * x / (3.0 * L * L) / r : 0.0;
  };
  std::vector<float4> ab_z(NZ);
  for (int k = 0; k < NZ; k++) {
    double xi = std::max((g.pml_z - 0.5 - k) * g.dz, (k - (g.pml_z + g.nz - 0.5)) * g.dz);
    double xh = std::max((g.pml_z - 1.0 - k) * g.dz, (k + 1.0 - g.pml_z - g.nz) * g.dz);
    if (!pml) xi = xh = 0.0;
    cpml(prof(xi, Lz, d0z), al, dt, &ab_z[k].x, &ab_z[k].y);
    cpml(prof(xh, Lz, d0z), al, dt, &ab_z[k].z, &ab_z[k].w);
  }
#define ALLOC(ptr, bytes)                                    \
  if ((rc = ralloc(h, (void **)&(ptr), (bytes))) != SIM_OK) \
    return bail(rc)
#define UP(dst, src, n)                                                                   \
  if ((e = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess) \
    return bail(rcuda(h, e, "upload"))
  ALLOC(h->mat, mat.size() * sizeof(float4));
  ALLOC(h->m_rho, mat.size() * 4);
  ALLOC(h->m_imu, mat.size() * 4);
  ALLOC(h->m_lam, mat.size() * 8);
  ALLOC(h->ab_z, NZ * sizeof(float4));
  ALLOC(h->status, 16);
  ALLOC(h->traces, (size_t)std::max(1, h->n_rec) * h->cap * 4);
  UP(h->mat, mat.data(), mat.size() * sizeof(float4));
  UP(h->m_rho, m_rho.data(), mat.size() * 4);
  UP(h->m_imu, m_imu.data(), mat.size() * 4);
  UP(h->m_lam, m_lam.data(), mat.size() * 8);
  UP(h->ab_z, ab_z.data(), NZ * sizeof(float4));

  // --- source
  const long ks = lround(source->z / g.dz) + g.pml_z;
  const bool axis = source->r < g.dr;
  int src_zone = 0, src_i = -1, src_j = -1;
  double vol = M_PI * g.dr * g.dr * g.dz;
  if (source->kind == 0 && !axis) {
    const int i = (int)floor(source->r / g.dr);
    src_zone = zone_of(i);
    const int n = g.nth >> (M - 1 - src_zone);
    const double dth = 2.0 * M_PI / n;
    src_i = i;
    src_j = (int)(((lround(source->theta / dth) % n) + n) % n);
    vol = (i + 0.5) * g.dr * g.dr * dth * g.dz;
  } else if (source->kind == 0) {
    src_i = 0;
  }
  int n_pulse = (int)std::min<double>(ceil(8.0 / (source->f0 * dt)) + 1.0, 1e8);
  h->n_wav = std::max(n_pulse, 1);
  std::vector<float> wav(h->n_wav);
  for (int n = 0; n < h->n_wav; n++)  // volumetric: the stress increment; forces f(t_n); torsion f(t_{n+1/2})
    wav[n] = source->kind == 0 ? (float)(dt * source->amplitude * ricker((n + 0.5) * dt, source->f0) / vol)
             : source->kind == 3 ? (float)ricker((n + 0.5) * dt, source->f0)
                                 : (float)ricker(n * dt, source->f0);
  ALLOC(h->wav, wav.size() * 4);
  UP(h->wav, wav.data(), wav.size() * 4);

  // --- receivers: grouped by zone
  std::vector<int> rz(h->n_rec), ri(h->n_rec), rj(h->n_rec), rk(h->n_rec);
  for (int q = 0; q < h->n_rec; q++) {
    const bool ax = receivers->r[q] < g.dr;
    const int i = ax ? 0 : (int)floor(receivers->r[q] / g.dr);
    rz[q] = zone_of(i);
    const int n = g.nth >> (M - 1 - rz[q]);
    ri[q] = i;
    rj[q] = ax ? -1 : (int)(((lround(receivers->theta[q] / (2.0 * M_PI / n)) % n) + n) % n);
    rk[q] = (int)(lround(receivers->z[q] / g.dz) + g.pml_z);
  }
  h->trace_row.assign(h->n_rec, 0);

  // --- zones
  std::vector<float> host_f;
  h->z.resize(M);
  int trow = 0;
  for (int m = 0; m < M; m++) {
    RZone &Z = h->z[m];
    Z.row = row0[m];
    Z.rows = row0[m + 1] - row0[m];
    Z.nth = g.nth >> (M - 1 - m);
    Z.g_lo = m > 0 ? 1 : 0;
    Z.g_hi = m < M - 1 ? 1 : 0;
    Z.NR = Z.g_lo + Z.rows + Z.g_hi;
    const int nthm = Z.nth, NRm = Z.NR, base = Z.row - Z.g_lo;  // global row of local row 0
    const bool outer = m == M - 1;
    const size_t fbytes = (size_t)nthm * NRm * NZp * 4;
    for (int q = 0; q < NF; q++) ALLOC(Z.f[q], fbytes);
    ALLOC(Z.id, (size_t)nthm * NRm * NZp * 2);
    if (pml && outer && g.pml_r > 0)
      for (int q = 0; q < NPR; q++) ALLOC(Z.psr[q], (size_t)nthm * g.pml_r * NZp * 4);
    if (pml && g.pml_z > 0)
      for (int q = 0; q < NPZ; q++) ALLOC(Z.psz[q], (size_t)nthm * NRm * 2 * g.pml_z * 4);
    ALLOC(Z.ab_r, NRm * sizeof(float4));
    ALLOC(Z.ab_q, NRm * sizeof(float4));
    ALLOC(Z.inv_ri, NRm * 4);
    ALLOC(Z.inv_rh, NRm * 4);
    ALLOC(Z.step, 16);
    // IDs: own rows sampled at this zone's nodes; the ghost row below holds the
    // coarser zone's cell floor(j / 2); the one above (never read) this zone's nodes
    std::vector<uint16_t> id((size_t)nthm * NRm * NZp, 0);
    for (int j = 0; j < nthm; j++)
      for (int l = 0; l < NRm; l++) {
        const int gi = base + l;
        for (int k = 0; k < NZ; k++)
          id[((size_t)j * NRm + l) * NZp + k] =
              (l == 0 && Z.g_lo) ? zone_id(m - 1, j / 2, gi, k) : zone_id(m, j, gi, k);
      }
    UP(Z.id, id.data(), id.size() * 2);
    std::vector<float4> ab_r(NRm), ab_q(NRm);
    std::vector<float> inv_ri(NRm), inv_rh(NRm);
    for (int l = 0; l < NRm; l++) {
      const int i = base + l;
      inv_ri[l] = i > 0 ? (float)(1.0 / (i * g.dr)) : 0.f;
      inv_rh[l] = (float)(1.0 / ((i + 0.5) * g.dr));
      double xi = pml ? (i - g.nr) * g.dr : 0.0, xh = pml ? (i + 0.5 - g.nr) * g.dr : 0.0;
      cpml(prof(xi, Lr, d0r), al, dt, &ab_r[l].x, &ab_r[l].y);
      cpml(prof(xh, Lr, d0r), al, dt, &ab_r[l].z, &ab_r[l].w);
      cpml(profbar(xi, i * g.dr, Lr, d0r), al, dt, &ab_q[l].x, &ab_q[l].y);
      cpml(profbar(xh, (i + 0.5) * g.dr, Lr, d0r), al, dt, &ab_q[l].z, &ab_q[l].w);
    }
    UP(Z.ab_r, ab_r.data(), NRm * sizeof(float4));
    UP(Z.ab_q, ab_q.data(), NRm * sizeof(float4));
    UP(Z.inv_ri, inv_ri.data(), NRm * 4);
    UP(Z.inv_rh, inv_rh.data(), NRm * 4);
    // its receivers
    std::vector<int> rec;
    Z.rec0 = trow;
    for (int q = 0; q < h->n_rec; q++)
      if (rz[q] == m) {
        rec.push_back(ri[q] - base);
        rec.push_back(rj[q]);
        rec.push_back(rk[q]);
        h->trace_row[q] = trow++;
      }
    Z.n_rec = (int)rec.size() / 3;
    ALLOC(Z.rec, std::max<size_t>(rec.size(), 3) * 4);
    if (!rec.empty()) UP(Z.rec, rec.data(), rec.size() * 4);
    // kernel parameters
    KParams &p = Z.kp;
    p.nth = nthm;
    p.NR = NRm;
    p.NZ = NZ;
    p.NZp = NZp;
    p.nr = (pml && outer) ? g.nr - base : NRm;
    p.pml_r = (pml && outer) ? g.pml_r : 0;
    p.pml_z = pml ? g.pml_z : 0;
    p.plane = (long long)NRm * NZp;
    p.dtv = (float)dt;
    p.dts = (float)dt;
    p.inv_dr = (float)(1.0 / g.dr);
    p.inv_dz = (float)(1.0 / g.dz);
    p.inv_dth = (float)(nthm / (2.0 * M_PI));
    p.inv_ri = Z.inv_ri;
    p.inv_rh = Z.inv_rh;
    p.ab_r = Z.ab_r;
    p.ab_q = Z.ab_q;
    p.ab_z = h->ab_z;
    p.mat = h->mat;
    p.m_rho = h->m_rho;
    p.m_imu = h->m_imu;
    p.m_lam = h->m_lam;
    p.id = Z.id;
    for (int q = 0; q < NF; q++) p.f[q] = Z.f[q];
    for (int q = 0; q < NPR; q++) p.psr[q] = Z.psr[q];
    for (int q = 0; q < NPZ; q++) p.psz[q] = Z.psz[q];
    p.wav = h->wav;
    p.n_wav = h->n_wav;
    p.src_i = (source->kind == 0 && m == src_zone) ? src_i - base : -1;
    p.src_j = src_j;
    p.src_k = (int)ks;
    p.step = Z.step;
    p.i_lo = Z.g_lo;
    p.i_hi = NRm - Z.g_hi;
    RParams &r = Z.rp;
    r.nth = nthm;
    r.NR = NRm;
    r.NZp = NZp;
    r.n_rec = Z.n_rec;
    r.cap = h->cap;
    r.plane = p.plane;
    r.srr = Z.f[F_SRR];
    r.spp = Z.f[F_SPP];
    r.szz = Z.f[F_SZZ];
    r.rec = Z.rec;
    r.scale = (float)(-1.0 / 3.0);
    r.traces = h->traces + (size_t)Z.rec0 * h->cap;
    r.step = Z.step;
    r.status = h->status;
    h->kps.push_back(p);
  }
  // the zones' streams: the largest zone stays on the handle's stream
  {
    long long most = -1;
    for (int m = 0; m < M; m++) {
      const long long cells = (long long)h->kps[m].nth * (h->kps[m].i_hi - h->kps[m].i_lo) * NZ;
      if (cells > most) most = cells, h->big_zone = m;
    }
    h->zone_streams = M > 1 && most >= ZONE_STREAM_CELLS;
    for (int k = 0; k < M - 1; k++) {
      if ((e = cudaStreamCreateWithFlags(&h->zs[k], cudaStreamNonBlocking)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&h->zjoin[k], cudaEventDisableTiming)) != cudaSuccess)
        return bail(rcuda(h, e, "zone streams"));
    }
    if (M > 1 && (e = cudaEventCreateWithFlags(&h->zfork, cudaEventDisableTiming)) != cudaSuccess)
      return bail(rcuda(h, e, "zone streams"));
  }
  // the zones' split codes; a forced one is tried once per half on the still
  // zero state of zone 0 with the source off (the state stays zero)
  h->vel_code = opts->tile ? split_vel_code(opts->tile) : REFINED_VEL_CODE;
  h->str_code = opts->tile            ? split_str_code(opts->tile)
                : h->zone_streams ? REFINED_STR_CODE
                                  : REFINED_STR_CODE_SMALL;
  if (opts->tile) {
    KParams dry = h->kps[0];
    dry.src_i = -1;
    e = launch_hoist(0, h->vel_code, dry, h->stream, nullptr, 1);
    if (e == cudaSuccess) e = launch_hoist(0, h->str_code, dry, h->stream, nullptr, 2);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e == cudaErrorInvalidValue) return bail(rfail(h, SIM_EINVAL, "opts.tile: no such split code"));
    if (e != cudaSuccess) return bail(rcuda(h, e, "opts.tile"));
  }
  {
    std::vector<RParams> rp(M);
    for (int m = 0; m < M; m++) rp[m] = h->z[m].rp;
    ALLOC(h->d_rp, M * sizeof(RParams));
    UP(h->d_rp, rp.data(), M * sizeof(RParams));
  }

  // --- point forces (R12) and the torsion ring (R13) on the zone's own nodes
  if (source->kind != 0) {
    std::vector<int> ifld;
    std::vector<long long> ioff;
    std::vector<float> iw;
    const int mz = axis ? 0 : zone_of(source->kind == 2 ? (int)floor(source->r / g.dr) : (int)lround(source->r / g.dr));
    const RZone &Z = h->z[mz];
    const int n = Z.nth, base = Z.row - Z.g_lo;
    const double dth = 2.0 * M_PI / n, dr = g.dr, dz = g.dz, A = source->amplitude;
    auto rho2 = [&](int a, int b) { return 0.5 * (medium->rho[a] + medium->rho[b]); };
    auto dc = [&](int j, int l) { return ((long long)j * Z.NR + l) * NZp + ks; };
    auto mu = [&](int a) { return medium->rho[a] * medium->vs[a] * medium->vs[a]; };
    if (source->kind == 2) {  // longitudinal force: v_z nodes, the cells above and below in one row
      if (ks + 1 >= NZ) return bail(rfail(h, SIM_EINVAL, "source: the force node falls outside the grid"));
      if (axis) {
        for (int j = 0; j < n; j++) {
          ifld.push_back(F_VZ);
          ioff.push_back(dc(j, 0));
          iw.push_back((float)(dt * A / (rho2(zone_id(0, j, 0, ks), zone_id(0, j, 0, ks + 1)) * M_PI * dr * dr * dz)));
        }
      } else {
        const int i = (int)floor(source->r / dr);
        const int js = (int)(((lround(source->theta / dth) % n) + n) % n);
        ifld.push_back(F_VZ);
        ioff.push_back(dc(js, i - base));
        iw.push_back((float)(dt * A / (rho2(zone_id(mz, js, i, ks), zone_id(mz, js, i, ks + 1)) * (i + 0.5) * dr * dr * dth * dz)));
      }
    } else if (source->kind == 3) {  // torsion ring on every node of its zone
      const int i = (int)lround(source->r / dr), ih = (int)floor(source->r / dr);
      if (i < 1 || i >= NR || ks + 1 >= NZ)
        return bail(rfail(h, SIM_EINVAL, "source: the torsion ring falls outside the grid"));
      for (int j = 0; j < n; j++) {
        const int jp = (j + 1) % n;
        if (!(mu(zone_id(mz, j, i - 1, ks)) > 0 && mu(zone_id(mz, j, i, ks)) > 0 && mu(zone_id(mz, jp, i - 1, ks)) > 0 &&
              mu(zone_id(mz, jp, i, ks)) > 0 && mu(zone_id(mz, j, ih, ks)) > 0 && mu(zone_id(mz, jp, ih, ks)) > 0 &&
              mu(zone_id(mz, j, ih, ks + 1)) > 0 && mu(zone_id(mz, jp, ih, ks + 1)) > 0))
          return bail(rfail(h, SIM_EUNSUPPORTED, "source: the torsion ring needs a solid at both shear nodes"));
        ifld.push_back(F_SRP);
        ioff.push_back(dc(j, i - base));
        iw.push_back((float)(dt * A / (2.0 * M_PI * i * dr * dr * dz)));
        ifld.push_back(F_SPZ);
        ioff.push_back(dc(j, ih - base));
        iw.push_back((float)(dt * A / (2.0 * M_PI * (ih + 0.5) * dr * dr * dz)));
      }
    } else if (axis) {  // transverse force on the axis: the ring-1 v_r nodes
      for (int j = 0; j < n; j++) {
        ifld.push_back(F_VR);
        ioff.push_back(dc(j, 1));
        iw.push_back((float)(dt * A * 2.0 * cos(j * dth - source->theta) / n /
                             (rho2(zone_id(0, j, 0, ks), zone_id(0, j, 1, ks)) * dr * dr * dth * dz)));
      }
    } else {
      const int i = (int)lround(source->r / dr);
      if (i < 1 || i >= NR) return bail(rfail(h, SIM_EINVAL, "source: the force node falls outside the grid"));
      const int js = (int)(((lround(source->theta / dth) % n) + n) % n);
      ifld.push_back(F_VR);
      ioff.push_back(dc(js, i - base));
      iw.push_back((float)(dt * A / (rho2(zone_id(mz, js, i - 1, ks), zone_id(mz, js, i, ks)) * i * dr * dr * dth * dz)));
    }
    int *d_ifld;
    long long *d_ioff;
    float *d_iw;
    ALLOC(d_ifld, ifld.size() * 4);
    ALLOC(d_ioff, ioff.size() * 8);
    ALLOC(d_iw, iw.size() * 4);
    UP(d_ifld, ifld.data(), ifld.size() * 4);
    UP(d_ioff, ioff.data(), ioff.size() * 8);
    UP(d_iw, iw.data(), iw.size() * 4);
    h->ip.n = (int)ifld.size();
    h->ip.fld = d_ifld;
    h->ip.off = d_ioff;
    h->ip.w = d_iw;
    h->ip.wav = h->wav;
    h->ip.n_wav = h->n_wav;
    h->ip.step = Z.step;
    for (int q = 0; q < NF; q++) h->ip.f[q] = Z.f[q];
  }

  // --- interface matrices and the ghost-row transfers of each half step
  h->xv.NZ = h->xs.NZ = NZ;
  if (M > 1) {
    std::vector<float> mats;
    std::vector<size_t> at(4 * M, 0);  // per interface: P_int, P_half, R_int, R_half offsets
    for (int m = 1; m < M; m++) {
      const int na = h->z[m - 1].nth;
      std::vector<double> mat(2 * (size_t)na * na);
      for (int k = 0; k < 4; k++) {  // P_int, P_half, R_int, R_half
        simr_interface_matrix(na, k & 1, k >> 1, mat.data());
        at[4 * m + k] = mats.size();
        for (double v : mat) mats.push_back((float)v);
      }
    }
    ALLOC(h->mats, mats.size() * 4);
    UP(h->mats, mats.data(), mats.size() * 4);
    auto add = [&](XferParams &X, int m, int q, bool up) {
      const RZone &A = h->z[m - 1], &B = h->z[m];
      const bool half = q == F_VP || q == F_SRP || q == F_SPZ;
      XferDesc &d = X.d[X.n++];
      if (up) {  // coarse A's last row -> ghost row below B
        d.src = A.f[q] + (long long)(A.g_lo + A.rows - 1) * NZp;
        d.src_plane = (long long)A.NR * NZp;
        d.dst = B.f[q];
        d.dst_plane = (long long)B.NR * NZp;
        d.n_in = A.nth;
        d.n_out = B.nth;
        d.mat = h->mats + at[4 * m + (half ? 1 : 0)];
      } else {  // fine B's first row -> ghost row above A
        d.src = B.f[q] + (long long)B.g_lo * NZp;
        d.src_plane = (long long)B.NR * NZp;
        d.dst = A.f[q] + (long long)(A.NR - 1) * NZp;
        d.dst_plane = (long long)A.NR * NZp;
        d.n_in = B.nth;
        d.n_out = A.nth;
        d.mat = h->mats + at[4 * m + 2 + (half ? 1 : 0)];
      }
    };
    for (int m = 1; m < M; m++) {
      add(h->xv, m, F_VP, true);
      add(h->xv, m, F_VZ, true);
      add(h->xv, m, F_VR, false);
      add(h->xs, m, F_SRR, true);
      add(h->xs, m, F_SPP, true);
      add(h->xs, m, F_SRP, false);
      add(h->xs, m, F_SRZ, false);
    }
  }
#undef ALLOC
#undef UP
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return bail(rcuda(h, e, "upload"));

  *out = h;
  return SIM_OK;
}

extern "C" int simr_step(simr_t *h, int nsteps) {
  if (!h) return SIM_EINVAL;
  if (nsteps < 0) return rfail(h, SIM_EINVAL, "nsteps < 0");
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return rcuda(h, e, "cudaSetDevice");
  int left = nsteps;
  if (h->graph_chunk > 0 && left >= h->graph_chunk) {
    if (!h->gexec) {
      cudaGraph_t graph;
      if ((e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return rcuda(h, e, "cudaStreamBeginCapture");
      cudaError_t e1 = cudaSuccess;
      for (int q = 0; q < h->graph_chunk && e1 == cudaSuccess; q++) e1 = enqueue_refined_step(h);
      e = cudaStreamEndCapture(h->stream, &graph);
      if (e1 != cudaSuccess) return rcuda(h, e1, "kernel launch during capture");
      if (e != cudaSuccess) return rcuda(h, e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&h->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return rcuda(h, e, "cudaGraphInstantiate");
      h->gsteps = h->graph_chunk;
    }
    while (left >= h->gsteps) {
      if ((e = cudaGraphLaunch(h->gexec, h->stream)) != cudaSuccess) return rcuda(h, e, "cudaGraphLaunch");
      left -= h->gsteps;
    }
  }
  for (; left > 0; left--)
    if ((e = enqueue_refined_step(h)) != cudaSuccess) return rcuda(h, e, "kernel launch");
  h->steps_done += nsteps;
  return SIM_OK;
}

extern "C" int simr_sync(simr_t *h) {
  if (!h) return SIM_EINVAL;
  cudaError_t e = cudaSetDevice(h->device);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return rcuda(h, e, "cudaStreamSynchronize");
  int st = 0;
  e = cudaMemcpy(&st, h->status, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return rcuda(h, e, "cudaMemcpy");
  if (st & 1) return rfail(h, SIM_EUNSTABLE, "non-finite value in the receiver traces");
  return SIM_OK;
}

extern "C" int simr_traces(simr_t *h, float *out, size_t cap, int *n_rec, int *n_steps) {
  if (!h) return SIM_EINVAL;
  int rc = simr_sync(h);
  if (rc && rc != SIM_EUNSTABLE) return rc;
  const int ns = std::min(h->steps_done, h->cap);
  if (n_rec) *n_rec = h->n_rec;
  if (n_steps) *n_steps = ns;
  if (!out) return rc;
  if (cap < (size_t)h->n_rec * ns) return rfail(h, SIM_EINVAL, "output buffer too small");
  for (int q = 0; q < h->n_rec && ns > 0; q++) {
    cudaError_t e = cudaMemcpy(out + (size_t)q * ns, h->traces + (size_t)h->trace_row[q] * h->cap, (size_t)ns * 4,
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return rcuda(h, e, "cudaMemcpy traces");
  }
  return rc;
}

extern "C" int simr_zone(const simr_t *h, int zone, int *row, int *rows, int *nth) {
  if (!h || zone < 0 || zone >= h->M) return SIM_EINVAL;
  if (row) *row = h->z[zone].row;
  if (rows) *rows = h->z[zone].rows;
  if (nth) *nth = h->z[zone].nth;
  return SIM_OK;
}

extern "C" int simr_read_field(simr_t *h, int field, int zone, float *out, size_t n) {
  if (!h) return SIM_EINVAL;
  if (field < 0 || field >= NF || zone < 0 || zone >= h->M || !out)
    return rfail(h, SIM_EINVAL, "simr_read_field: bad field, zone or buffer");
  const RZone &Z = h->z[zone];
  if (n < (size_t)Z.nth * Z.rows * h->NZ) return rfail(h, SIM_EINVAL, "simr_read_field: buffer too small");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  for (int j = 0; j < Z.nth && e == cudaSuccess; j++)
    e = cudaMemcpy2D(out + (size_t)j * Z.rows * h->NZ, (size_t)h->NZ * 4,
                     Z.f[field] + ((size_t)j * Z.NR + Z.g_lo) * h->NZp, (size_t)h->NZp * 4, (size_t)h->NZ * 4, Z.rows,
                     cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return rcuda(h, e, "simr_read_field");
  return SIM_OK;
}

extern "C" double simr_dt(const simr_t *h) { return h ? h->dt : 0.0; }
extern "C" int simr_steps_done(const simr_t *h) { return h ? h->steps_done : 0; }
extern "C" size_t simr_cells(const simr_t *h) {
  if (!h) return 0;
  size_t c = 0;
  for (const RZone &Z : h->z) c += (size_t)Z.nth * Z.rows * h->NZ;
  return c;
}

extern "C" void simr_destroy(simr_t *h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  rrelease(h);
  delete h;
}

extern "C" const char *simr_last_error(const simr_t *h) { return h ? h->err.c_str() : g_refine_err.c_str(); }
