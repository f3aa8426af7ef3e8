// Internal state of a simulator handle, shared by the single-well and batch
// host code.
#pragma once

#include <cudaTypedefs.h>

#include <string>
#include <vector>

#include "../../include/cwell.h"
#include "cwell_internal.cuh"

// the handle type is declared at global scope by cwell.h
using namespace cwell;

struct sim_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  sim_grid_t grid{};
  int NR = 0, NZ = 0, NZp = 0;
  double dt = 0, vscale = 1, sscale = 1;
  // storage: the stored format (0 FP32, 1 BF16, 2 FP16); stencil_storage:
  // what the stencil kernels write (also 3 = FP16 with stochastic rounding)
  int storage = 0, stencil_storage = 0, kernel = SIM_KERNEL_SPLIT, graph_chunk = 64, timing = 0;
  int n_mat = 0, n_rec = 0, cap = 0;
  size_t elem = 4;
  void *f[NF] = {};
  float *psr[NPR] = {};
  float *psz[NPZ] = {};
  uint16_t *id = nullptr;
  float4 *mat = nullptr, *ab_r = nullptr, *ab_q = nullptr, *ab_z = nullptr;
  float *m_rho = nullptr, *m_imu = nullptr;
  float2 *m_lam = nullptr;
  float *inv_ri = nullptr, *inv_rh = nullptr, *wav = nullptr, *traces = nullptr;
  int *rec = nullptr, *step = nullptr, *status = nullptr;
  int n_wav = 0;
  KParams kp{};
  RParams rp{};
  // fused path: second buffer set, TMA descriptors and parameters per step parity
  bool fused = false;
  int tile_rt = 0;
  void *f2[NF] = {};
  float *psr2[NPR] = {};
  float *psz2[NPZ] = {};
  FusedMaps maps[2];
  // point forces / torsion ring (source kinds 1-3): injection points
  int src_kind = 0;
  IParams ip{};
  // single-pass sweep path (in place on the first buffer set): per-chunk
  // counters of finished velocity items, the wait limit and the test hook
  bool sweep = false;
  int *vdone = nullptr;
  long long wait_cycles = 0;
  int withhold_chunk = -1;
  // marching split path (in place on the first buffer set): TMA descriptors
  bool march = false;
  FusedMaps mmaps;
  FusedParams fp[2];
  RParams rp2[2];
  // second stream and fork / join events of the three-way split halves
  SideStream side{};
  // device watchdog (opts.watchdog_every > 0): parameters per step parity
  // (the fused path's state alternates between the buffer sets)
  int watch_every = 0, watch_blocks = 0;
  double *watch_acc = nullptr;
  WParams wp[2]{};
  // z slab (sim_create_slab): the handle holds the well's stored z cells
  // l0 .. l0 + NZ - 1 and owns s0 .. s1 - 1 of them
  bool slab = false;
  int l0 = 0, s0 = 0, s1 = 0;
  int steps_done = 0;
  size_t bytes = 0, mem_cap = 0, psr_elems = 0, psz_elems = 0;
  std::vector<void *> allocs;
  cudaGraphExec_t gexec = nullptr;
  int gsteps = 0;
  cudaEvent_t ev[4] = {};
  double kms[3] = {0, 0, 0};
  long kcount[3] = {0, 0, 0};
  std::string err;
};

namespace cwell {
extern thread_local std::string g_create_err;

inline int fail(sim_t *h, int code, const std::string &msg) {
  if (h) h->err = msg;
  else g_create_err = msg;
  return code;
}

inline int cuda_fail(sim_t *h, cudaError_t e, const char *what) {
  return fail(h, SIM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, call)                                  \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)


// host-only argument checks of sim_create (no device call); message in g_create_err
int validate_inputs(const sim_grid_t *g, const sim_medium_t *m, const sim_source_t *s, const sim_receivers_t *r,
                    const sim_opts_t *o);

// Ricker pulse with delay 2/f0 (Sec. 2) and the C-PML recursion coefficients
double ricker(double t, double f0);
void cpml(double d, double al, double dt, float *a, float *b);

// the split halves (parts: 1 velocity, 2 stress) of a handle on the split
// path with its chosen code, parameters p, on stream s
cudaError_t sim_split_halves(const sim_t *h, const KParams &p, cudaStream_t s, int parts);

// steps enqueued on the handle (the batch advances its cases directly)
inline void sim_advance(sim_t *h, int n) { h->steps_done += n; }

}  // namespace cwell
