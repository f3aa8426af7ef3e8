// Batched scenarios: many wells advanced together.  Every case is a regular
// simulator handle (same validation and set-up as sim_create, buffers updated
// in place by the load-first split bodies).  Small cases share one interior
// and one edge launch per half step (their kernel parameters travel as kernel
// parameters, up to 64 cases per launch); a case large enough to fill the GPU
// runs its own tuned split launches, the large cases spread over parallel
// streams (branches of the captured graph) so that one case's launch tails
// overlap another's work.  The steps are captured in a CUDA graph.
#include <algorithm>
#include <string>
#include <vector>

#include "sim_state.cuh"

struct simb_s {
  int device = 0, storage = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<sim_t *> cases;
  std::vector<KParams> kp;        // the cases' kernel parameters (host: they travel as kernel parameters)
  std::vector<int> shared, own;   // cases in the shared persistent launches / on their own tuned launches
  RParams *d_rp = nullptr;
  long long total = 0;  // bound on the items of one work list of the shared cases
  int grid = 0, graph_chunk = 64, steps_done = 0;
  // parallel streams for the own-launch cases: case own[q] runs on branch[q % nbranch]
  static constexpr int MAX_BRANCH = 4;
  cudaStream_t branch[MAX_BRANCH] = {};
  cudaEvent_t fork = nullptr, join[MAX_BRANCH] = {};
  int nbranch = 1;
  bool fixed_branches = false;
  cudaGraphExec_t gexec = nullptr;
  int gsteps = 0;
  std::string err;
};

static thread_local std::string g_batch_err;

static int bfail(simb_t *b, int code, const std::string &msg) {
  if (b) b->err = msg;
  else g_batch_err = msg;
  return code;
}

static int bcuda(simb_t *b, cudaError_t e, const char *what) {
  return bfail(b, SIM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

static void brelease(simb_t *b) {
  if (!b) return;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  for (int k = 0; k < simb_t::MAX_BRANCH; k++) {
    if (b->branch[k]) cudaStreamDestroy(b->branch[k]);
    if (b->join[k]) cudaEventDestroy(b->join[k]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  for (sim_t *h : b->cases) sim_destroy(h);
  b->cases.clear();
  if (b->d_rp) cudaFree(b->d_rp);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

// Small cases share the persistent batched launches (one case cannot fill the
// GPU); a case of at least OWN_CELLS cells fills it alone and runs its own
// split launches with the code its tuner chose (the prefetching kernels), in
// the same stream and graph.
constexpr long long OWN_CELLS = 4LL << 20;

// One step of every case.  The shared cases run on the batch's stream; the
// own-launch cases on nbranch streams forked from it and joined back (each
// case's two halves stay in order on its branch; cases share nothing).
static cudaError_t batch_step(simb_t *b, const KParams *cases) {
  cudaError_t e = cudaSuccess;
  std::vector<KParams> sh;
  for (int c : b->shared) sh.push_back(cases[c]);
  const int nb = b->own.size() > 1 ? std::min<int>(b->nbranch, (int)b->own.size()) : 1;
  auto stream_of = [&](size_t q) { return nb > 1 ? b->branch[q % nb] : b->stream; };
  if (nb > 1) {
    e = cudaEventRecord(b->fork, b->stream);
    for (int k = 0; k < nb && e == cudaSuccess; k++) e = cudaStreamWaitEvent(b->branch[k], b->fork, 0);
  }
  for (int half = 1; half <= 2 && e == cudaSuccess; half++) {
    if (!sh.empty()) e = launch_batch_split(b->storage, half == 1, sh.data(), (int)sh.size(), b->grid, b->stream);
    for (size_t q = 0; q < b->own.size() && e == cudaSuccess; q++)
      e = sim_split_halves(b->cases[b->own[q]], cases[b->own[q]], stream_of(q), half);
  }
  if (nb > 1)
    for (int k = 0; k < nb && e == cudaSuccess; k++) {
      e = cudaEventRecord(b->join[k], b->branch[k]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join[k], 0);
    }
  return e;
}

// time persistent grids of several sizes (and one block per item) on the
// still-zero state with every source disabled; keep the fastest
static int tune_grid(simb_t *b) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  const int n = (int)b->cases.size();
  std::vector<KParams> dry(n);
  for (int c = 0; c < n; c++) {
    dry[c] = b->cases[c]->kp;
    dry[c].src_i = -1;
  }
  cudaError_t e = cudaSuccess;
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  const long long cand[5] = {(long long)sms * 6, (long long)sms * 12, (long long)sms * 24, (long long)sms * 48,
                             b->total};
  float best = INFINITY;
  int pick = (int)std::min<long long>(b->total, (long long)sms * 12);
  for (long long g : cand) {
    if (e != cudaSuccess) break;
    b->grid = (int)std::max<long long>(1, std::min<long long>(g, std::min<long long>(b->total, 1LL << 30)));
    e = batch_step(b, dry.data());
    cudaEventRecord(t0, b->stream);
    for (int w = 0; w < 3 && e == cudaSuccess; w++) e = batch_step(b, dry.data());
    cudaEventRecord(t1, b->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0;
    cudaEventElapsedTime(&ms, t0, t1);
    if (e == cudaSuccess && ms < best) {
      best = ms;
      pick = b->grid;
    }
  }
  b->grid = pick;
  // branches of the own-launch cases: 1, 2 or 4 parallel streams
  int pick_b = 1;
  if (e == cudaSuccess && b->own.size() > 1 && !b->fixed_branches) {
    float best_b = INFINITY;
    for (int nb : {1, 2, 4}) {
      if (nb > (int)b->own.size() || e != cudaSuccess) break;
      b->nbranch = nb;
      e = batch_step(b, dry.data());
      cudaEventRecord(t0, b->stream);
      for (int w = 0; w < 3 && e == cudaSuccess; w++) e = batch_step(b, dry.data());
      cudaEventRecord(t1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      float ms = 0;
      cudaEventElapsedTime(&ms, t0, t1);
      if (e == cudaSuccess && ms < best_b) {
        best_b = ms;
        pick_b = nb;
      }
    }
    b->nbranch = pick_b;
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (e != cudaSuccess) return bcuda(b, e, "batch autotune");
  return SIM_OK;
}

extern "C" int simb_create(int n, const sim_grid_t *grids, const sim_medium_t *media, const sim_source_t *sources,
                           const sim_receivers_t *receivers, const sim_opts_t *opts, simb_t **out) {
  if (!out) return bfail(nullptr, SIM_EINVAL, "out is null");
  *out = nullptr;
  if (n < 1 || !grids || !media || !sources || !receivers || !opts)
    return bfail(nullptr, SIM_EINVAL, "need n >= 1 and non-null arrays");
  if (opts->storage == SIM_STORAGE_F16_SR)
    return bfail(nullptr, SIM_EUNSUPPORTED, "batches store FP32, BF16 or FP16 rounded to nearest");
  if (opts->watchdog_every != 0)
    return bfail(nullptr, SIM_EUNSUPPORTED, "batches: no device watchdog (single handles only)");
  if (opts->tile != 0 && opts->tile != 1 && opts->tile != -1 && opts->tile != -2 && opts->tile != -4)
    return bfail(nullptr, SIM_EINVAL, "opts.tile of a batch: 0, 1 (all shared) or -1, -2, -4 (branches)");
  sim_opts_t vo = *opts;  // the batch's own use of opts.tile is not a tile code
  vo.tile = 0;
  for (int c = 0; c < n; c++) {  // host-side checks of every case before any device work
    int rc = validate_inputs(&grids[c], &media[c], &sources[c], &receivers[c], &vo);
    if (rc) return bfail(nullptr, rc, "case " + std::to_string(c) + ": " + g_create_err);
    if (sources[c].kind != 0)
      return bfail(nullptr, SIM_EUNSUPPORTED, "case " + std::to_string(c) + ": batches run the volumetric source only");
  }
  simb_t *b = new simb_t();
  b->device = opts->device;
  b->storage = opts->storage;
  b->graph_chunk = opts->graph_chunk == 0 ? 64 : opts->graph_chunk;
  auto bail = [&](int code) {
    g_batch_err = b->err;
    brelease(b);
    delete b;
    return code;
  };
  cudaError_t e = cudaSetDevice(b->device);
  if (e != cudaSuccess) return bail(bcuda(b, e, "cudaSetDevice"));
  if (opts->cuda_stream) {
    b->stream = (cudaStream_t)opts->cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(bcuda(b, e, "cudaStreamCreate"));
    b->own_stream = true;
  }
  if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess)
    return bail(bcuda(b, e, "cudaEventCreate"));
  for (int k = 0; k < simb_t::MAX_BRANCH; k++)
    if ((e = cudaStreamCreateWithFlags(&b->branch[k], cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming)) != cudaSuccess)
      return bail(bcuda(b, e, "batch branches"));
  // opts.tile of a batch: 1 = every case in the shared persistent launches,
  // -b (b = 1, 2, 4) = b branches for the own-launch cases; 0 = tuned
  const bool all_shared = opts->tile == 1;
  if (opts->tile < 0) {
    b->nbranch = std::min(simb_t::MAX_BRANCH, -opts->tile);
    b->fixed_branches = true;
  }
  sim_opts_t o = *opts;
  o.kernel = SIM_KERNEL_SPLIT;
  o.cuda_stream = b->stream;
  o.graph_chunk = -1;
  o.timing = 0;
  size_t used = 0;
  for (int c = 0; c < n; c++) {
    if (opts->mem_cap) o.mem_cap = opts->mem_cap > used ? opts->mem_cap - used : 1;
    const long long cells =
        (long long)grids[c].nth * (grids[c].nr + grids[c].pml_r) * (grids[c].nz + 2 * grids[c].pml_z);
    const bool own = cells >= OWN_CELLS && !all_shared;
    o.tile = own ? 0 : SPLIT_CODE;  // a large case is tuned (split family); the shared ones take the plain code
    (own ? b->own : b->shared).push_back(c);
    sim_t *h = nullptr;
    int rc = sim_create(&grids[c], &media[c], &sources[c], &receivers[c], &o, &h);
    if (rc) return bail(bfail(b, rc, "case " + std::to_string(c) + ": " + sim_last_error(nullptr)));
    b->cases.push_back(h);
    used += sim_device_bytes(h);
    const long long items = split_items(grids[c].nth, grids[c].nr + grids[c].pml_r, grids[c].nz + 2 * grids[c].pml_z);
    if (!own && items > 0x7fffffffLL)
      return bail(bfail(b, SIM_EINVAL, "case " + std::to_string(c) + ": more work items than a 32-bit index holds"));
    if (!own) b->total += items;  // work items of the shared launches
  }
  b->kp.resize(n);
  std::vector<RParams> rp(n);
  for (int c = 0; c < n; c++) {
    b->kp[c] = b->cases[c]->kp;
    rp[c] = b->cases[c]->rp;
  }
  if ((e = cudaMalloc(&b->d_rp, n * sizeof(RParams))) != cudaSuccess) {
    cudaGetLastError();
    return bail(bfail(b, SIM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)));
  }
  if ((e = cudaMemcpy(b->d_rp, rp.data(), n * sizeof(RParams), cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(bcuda(b, e, "upload batch tables"));
  int rc = tune_grid(b);
  if (rc) return bail(rc);
  *out = b;
  return SIM_OK;
}

static cudaError_t enqueue_batch_step(simb_t *b) {
  cudaError_t e = batch_step(b, b->kp.data());
  if (e == cudaSuccess) e = launch_batch_receivers(b->storage, b->d_rp, (int)b->cases.size(), b->stream);
  return e;
}

extern "C" int simb_run(simb_t *b, int nsteps) {
  if (!b) return SIM_EINVAL;
  if (nsteps < 0) return bfail(b, SIM_EINVAL, "nsteps < 0");
  cudaError_t e = cudaSetDevice(b->device);
  if (e != cudaSuccess) return bcuda(b, e, "cudaSetDevice");
  int left = nsteps;
  if (b->graph_chunk > 0 && left >= b->graph_chunk) {
    if (!b->gexec) {
      cudaGraph_t graph;
      if ((e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return bcuda(b, e, "cudaStreamBeginCapture");
      cudaError_t e1 = cudaSuccess;
      for (int q = 0; q < b->graph_chunk && e1 == cudaSuccess; q++) e1 = enqueue_batch_step(b);
      e = cudaStreamEndCapture(b->stream, &graph);
      if (e1 != cudaSuccess) return bcuda(b, e1, "kernel launch during capture");
      if (e != cudaSuccess) return bcuda(b, e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&b->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return bcuda(b, e, "cudaGraphInstantiate");
      b->gsteps = b->graph_chunk;
    }
    while (left >= b->gsteps) {
      if ((e = cudaGraphLaunch(b->gexec, b->stream)) != cudaSuccess) return bcuda(b, e, "cudaGraphLaunch");
      left -= b->gsteps;
    }
  }
  for (; left > 0; left--)
    if ((e = enqueue_batch_step(b)) != cudaSuccess) return bcuda(b, e, "kernel launch");
  b->steps_done += nsteps;
  for (sim_t *h : b->cases) sim_advance(h, nsteps);
  return SIM_OK;
}

extern "C" int simb_sync(simb_t *b) {
  if (!b) return SIM_EINVAL;
  for (size_t c = 0; c < b->cases.size(); c++) {
    int rc = sim_sync(b->cases[c]);
    if (rc) return bfail(b, rc, "case " + std::to_string(c) + ": " + sim_last_error(b->cases[c]));
  }
  return SIM_OK;
}

extern "C" int simb_traces(simb_t *b, int which, float *out, size_t cap, int *n_rec, int *n_steps) {
  if (!b) return SIM_EINVAL;
  if (which < 0 || which >= (int)b->cases.size()) return bfail(b, SIM_EINVAL, "case index out of range");
  int rc = sim_traces(b->cases[which], out, cap, n_rec, n_steps);
  if (rc) bfail(b, rc, sim_last_error(b->cases[which]));
  return rc;
}

extern "C" int simb_read_field(simb_t *b, int which, int field, float *out, size_t n) {
  if (!b) return SIM_EINVAL;
  if (which < 0 || which >= (int)b->cases.size()) return bfail(b, SIM_EINVAL, "case index out of range");
  int rc = sim_read_field(b->cases[which], field, out, n);
  if (rc) bfail(b, rc, sim_last_error(b->cases[which]));
  return rc;
}

extern "C" int simb_config(const simb_t *b, int *n_cases, long long *work_items, int *grid_blocks) {
  if (!b) return SIM_EINVAL;
  if (n_cases) *n_cases = (int)b->cases.size();
  if (work_items) *work_items = b->total;
  if (grid_blocks) *grid_blocks = b->grid;
  return SIM_OK;
}

extern "C" int simb_layout(const simb_t *b, int *own_cases, int *branches) {
  if (!b) return SIM_EINVAL;
  if (own_cases) *own_cases = (int)b->own.size();
  if (branches) *branches = b->own.size() > 1 ? std::min<int>(b->nbranch, (int)b->own.size()) : 1;
  return SIM_OK;
}

extern "C" void simb_destroy(simb_t *b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  brelease(b);
  delete b;
}

extern "C" const char *simb_last_error(const simb_t *b) { return b ? b->err.c_str() : g_batch_err.c_str(); }
