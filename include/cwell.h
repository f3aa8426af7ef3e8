/*
 * cwell.h -- C-ABI of the GB300 cased-well acoustic simulator.
 *
 * The library advances the first-order velocity-stress system of elasticity
 * in cylindrical coordinates (r, theta, z) -- Eq. 1 of "Parallel Modeling of
 * the Acoustic Signal Propagation in a Cased Well" (arXiv 2302.13907), with
 * zero initial data (Eq. 2), a liquid modelled by a vanishing shear modulus
 * (Sec. 2), medium parameters attached to the cell centre of a staggered
 * grid (Sec. 3), a PML at the outer radius and at both z ends (Sec. 1,
 * Sec. 6), a volumetric point source with a Ricker pulse delayed by 2/f0
 * (Sec. 2) -- on one GPU, with hand-written sm_103a CUDA kernels.
 *
 * Conventions shared by every call:
 *  - Cell (i, j, k): r = (i + 1/2) dr, theta = j * 2 pi / nth, depth
 *    z = (k - pml_z) dz; i in [0, NR), j in [0, nth), k in [0, NZ) with
 *    NR = nr + pml_r and NZ = nz + 2 pml_z.  Host arrays are [theta][r][z]
 *    with z fastest.  SI units throughout.
 *  - Staggering of the nine unknowns (field index in brackets):
 *    [0] v_r (i, j, k)     [1] v_phi (i+1/2, j+1/2, k)   [2] v_z (i+1/2, j, k+1/2)
 *    [3] s_rr, [4] s_phiphi, [5] s_zz at the cell centre (i+1/2, j, k)
 *    [6] s_rphi (i, j+1/2, k)  [7] s_phiz (i+1/2, j+1/2, k+1/2)  [8] s_rz (i, j, k+1/2)
 *    where an integer r index i means r = i dr.
 *  - Return codes: 0 on success, a negative SIM_E* code otherwise; the
 *    message of the last failure of a handle is sim_last_error(handle).
 *    No call aborts, traps or exits the process.
 *  - Ownership: every input is deep-copied by the create calls; the caller
 *    keeps its host buffers.  Device memory belongs to the handle and is
 *    released by the destroy calls.
 *  - Asynchrony: the step/run calls enqueue work on the handle's CUDA
 *    stream and return; errors raised on the device (non-finite field,
 *    a bounded wait that gave up) are reported by the next sync/traces call.
 */
#ifndef CWELL_H
#define CWELL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SIM_OK 0
#define SIM_EINVAL (-1)      /* invalid argument, checked on the host before any device work */
#define SIM_ENOMEM (-2)      /* device allocation failed or opts.mem_cap exceeded */
#define SIM_ECUDA (-3)       /* a CUDA runtime call failed */
#define SIM_EUNSTABLE (-4)   /* non-finite value in the receiver traces, or the watchdog tripped */
#define SIM_ETIMEOUT (-5)    /* a bounded device-side wait gave up */
#define SIM_EUNSUPPORTED (-6) /* e.g. a solid (mu > 0) cell in ring 0 next to the axis */

#define SIM_FIELD_VR 0
#define SIM_FIELD_VPHI 1
#define SIM_FIELD_VZ 2
#define SIM_FIELD_SRR 3
#define SIM_FIELD_SPHIPHI 4
#define SIM_FIELD_SZZ 5
#define SIM_FIELD_SRPHI 6
#define SIM_FIELD_SPHIZ 7
#define SIM_FIELD_SRZ 8

#define SIM_STORAGE_F32 0
#define SIM_STORAGE_BF16 1
#define SIM_STORAGE_F16 2
#define SIM_STORAGE_F16_SR 3  /* FP16 written with stochastic rounding by the stencil kernels (see sim_opts_t) */

#define SIM_KERNEL_AUTO 0     /* fastest path for the storage type */
#define SIM_KERNEL_SPLIT 1    /* separate velocity and stress kernels */
#define SIM_KERNEL_FUSED 2    /* one time-skewed kernel per step, one cell per thread */
#define SIM_KERNEL_FUSED_VEC 3 /* the time-skewed kernel with four z cells per thread */
#define SIM_KERNEL_MARCH 4     /* velocity and stress kernels marching theta over TMA-staged planes */
#define SIM_KERNEL_SWEEP 5     /* one persistent launch per step sweeping z in chunks: both half-steps,
                                  each chunk's velocities and stresses reused from L2 */

/* Grid (Sec. 3): interior cell counts, PML widths in cells, steps in metres.
 * nth must be even and >= 4; nr >= 2; nz >= 2.  dt > 0 fixes the time step;
 * otherwise dt = cfl * min over cells of 1 / (Vp sqrt(1/dr^2 + 1/(r dtheta)^2 + 1/dz^2)). */
typedef struct {
  int nr, nth, nz, pml_r, pml_z;
  double dr, dz;
  double cfl;
  double dt;
} sim_grid_t;

/* Medium (Sec. 2-3): per-material density [kg/m^3], P and S speeds [m/s]
 * (vs = 0 is a liquid, mu = 0); cell_id[nth][NR][NZ] (z fastest) indexes
 * the material table.  Requires vp^2 >= 2 vs^2 and rho, vp > 0. */
typedef struct {
  int n_mat;
  const double *rho, *vp, *vs;
  const uint16_t *cell_id;
} sim_medium_t;

/* Point source (Sec. 2, the four source types), f the Ricker pulse with
 * dominant frequency f0 and delay 2/f0, A = amplitude, V the node's volume.
 *  kind 0, volumetric: the three normal stresses receive dt * A f(t_{n+1/2}) / V
 *    per step; r < dr places it on the axis, shared by all ring-0 cells of the
 *    nearest depth (V = pi dr^2 dz).
 *  kind 1, transverse point force (direction theta): after the velocity
 *    update v_r += dt * A f(t_n) / (rho V) at the nearest v_r node; on the
 *    axis a horizontal force spread over the ring-1 v_r nodes with the share
 *    2 cos(theta_j - theta) / Ntheta each.
 *  kind 2, longitudinal point force: the same on v_z (on the axis every
 *    ring-0 v_z node, V = pi dr^2 dz).
 *  kind 3, torsion: s_rphi and s_phiz += dt * A f(t_{n+1/2}) / (2 pi r dr dz)
 *    on the whole ring at radius r (a torque about the axis); both shear
 *    nodes must lie in a solid, else SIM_EUNSUPPORTED.
 * Kinds 1-3 run on the split and marching paths, kind 3 on the sweep path
 * too (SIM_EUNSUPPORTED when the fused kernels, or for kinds 1-2 the sweep
 * kernel, are asked for; AUTO picks among the others) and not in batches. */
typedef struct {
  int kind;
  double r, theta, z, f0, amplitude;
} sim_source_t;

/* Receivers: quantity 0 = pressure -(s_rr + s_phiphi + s_zz)/3 at the
 * nearest cell centre; r < dr records the mean over the ring-0 cells. */
typedef struct {
  int n;
  const double *r, *theta, *z;
  int quantity;
} sim_receivers_t;

/* Options.  Zero-initialised options are valid defaults. */
typedef struct {
  int storage;        /* SIM_STORAGE_*: field storage; arithmetic is FP32.  SIM_STORAGE_F16_SR stores
                         FP16 (the FP16 scales) rounded stochastically: field f of cell (j, i, k)
                         at step n rounds up with probability frac(|x| / u), u the FP16 spacing,
                         against a 13-bit dither from SplitMix64 of the counter
                         ((((n * 9 + f) * nth + j) * NR + i) * ceil(NZ / 4) + k / 4), bits
                         16 (k mod 4) .. 16 (k mod 4) + 12; the split (23xx) and sweep kernels and
                         the volumetric source only (SIM_EUNSUPPORTED otherwise) */
  int pml_off;        /* 1: rigid walls with no PML (energy-conserving closure) */
  int graph_chunk;    /* steps per captured CUDA graph; 0 = 64; < 0 = no graph */
  void *cuda_stream;  /* cudaStream_t to enqueue on; NULL = a stream owned by the handle */
  size_t mem_cap;     /* bytes of device memory the handle may take; 0 = no cap */
  int max_steps;      /* trace capacity in steps; 0 = 65536 */
  int kernel;         /* SIM_KERNEL_* */
  int timing;         /* 1: bracket each kernel launch with CUDA events (no graph) */
  int device;         /* CUDA device ordinal */
  int tile;           /* 0: the autotuner picks the tile; otherwise the tile code
                         (see sim_config) of the requested kernel to run,
                         SIM_EINVAL if that kernel has no such tile or it does
                         not fit in shared memory */
  int watchdog_every; /* K > 0: a device watchdog after every K-th full step (sim_step) sums the
                         energy proxy 1/2 sum [rho |v|^2 + (s_rr^2 + s_pp^2 + s_zz^2 + 2 (s_rp^2 +
                         s_pz^2 + s_rz^2)) / (lambda + 2 mu)] over the owned cells (physical units,
                         each cell's material); it trips when the proxy is not finite, or exceeds 100
                         times its first value once the source wavelet has ended (the energy of
                         Eq. 1 with the PML cannot grow then; the proxy stays within a factor of
                         about 0.3 to 3 of it), and sim_sync then returns SIM_EUNSTABLE.  Two
                         launches per step that return at once on the other steps.  0 = off;
                         < 0 SIM_EINVAL; batches and the refined grid: SIM_EUNSUPPORTED */
} sim_opts_t;

typedef struct sim_s sim_t;

/* Build the device state: validates, computes dt, the material table, PML
 * profiles and the wavelet on the host in FP64, allocates and uploads.
 * *out is NULL on failure. */
int sim_create(const sim_grid_t *grid, const sim_medium_t *medium, const sim_source_t *source,
               const sim_receivers_t *receivers, const sim_opts_t *opts, sim_t **out);

/* Enqueue nsteps leapfrog steps (velocity to t_{n+1/2}, stress to t_{n+1},
 * source, receivers; Eq. 1a then Eq. 1b).  nsteps >= 0. */
int sim_step(sim_t *h, int nsteps);

/* ------------------------------------------------------------------------
 * Z slabs of one well (Sec. 4 of the paper: each processing unit owns a
 * contiguous range of z planes and swaps the planes next to its boundaries
 * with its neighbours after each half-step), one handle per slab, e.g. one
 * per GPU.
 *
 * sim_create_slab takes the whole well (grid, medium, source, receivers as
 * for sim_create) and the slab's stored z cells s0 <= k < s1 (k = the
 * well's index, PML cells included; inner bounds multiples of 4, at least 8
 * cells).  The handle holds those cells and 4 ghost cells on each side shared
 * with another slab, updates only its own cells, injects the source only if
 * it owns its depth, records only its own receivers (the others read zero)
 * and takes the well's time step and PML profile, so that its cells evolve
 * exactly as in the undivided well once the ghost cells are refilled after
 * every half-step: FP32 storage, split kernels (interior / edge codes).
 *
 * A step of a slab is sim_half_step(h, 0) (velocity half-step and point
 * forces), the velocity swap, sim_half_step(h, 1) (stress half-step,
 * volumetric or torsion source, receivers), the stress swap.  A swap copies
 * the slab's 4 own cells next to each inner boundary (sim_get_planes) to the
 * neighbour's ghost cells (sim_put_planes).  sim_step also works on a slab
 * (without swaps: its ghost cells then stay as they are).
 * ------------------------------------------------------------------------ */
int sim_create_slab(const sim_grid_t *grid, const sim_medium_t *medium, const sim_source_t *source,
                    const sim_receivers_t *receivers, const sim_opts_t *opts, int s0, int s1, sim_t **out);

/* One half of a leapfrog step: which = 0 velocity half-step (and point
 * forces), which = 1 stress half-step (volumetric or torsion source) and the
 * receivers; enqueued on the handle's stream.  Split kernels only. */
int sim_half_step(sim_t *h, int which);

/* Stored z cells the handle holds (l0 .. l0 + nz_local - 1 of the well) and
 * owns (s0 .. s1 - 1); a whole-well handle gives 0, 0, NZ, NZ. */
int sim_slab_info(const sim_t *h, int *l0, int *s0, int *s1, int *nz_local);

/* Copy the planes k0 <= k < k1 (the well's stored index, within the cells the
 * handle holds) of the velocities (group 0: v_r, v_phi, v_z) or the stresses
 * (group 1: the six in field order) to / from buf, laid out
 * [field][nth * NR][k1 - k0] in the storage type; buf may be device or host
 * memory.  Enqueued on the handle's stream (asynchronous). */
int sim_get_planes(sim_t *h, int group, int k0, int k1, void *dst);
int sim_put_planes(sim_t *h, int group, int k0, int k1, const void *src);

/* Wait for the handle's stream; reports device-side failures. */
int sim_sync(sim_t *h);

/* Copy the recorded traces to host memory out[n_rec][n_steps] (row-major,
 * sample m = value after step m, time (m + 1) dt); cap = capacity of out in
 * floats.  Synchronises.  *n_rec, *n_steps receive the shape. */
int sim_traces(sim_t *h, float *out, size_t cap, int *n_rec, int *n_steps);

/* Host copy of field `which` (SIM_FIELD_*) as FP32 [nth][NR][NZ]; n = capacity. */
int sim_read_field(sim_t *h, int which, float *out, size_t n);

/* The same read-back as sim_read_field with no device allocation, for callers
 * that cannot call cudaMalloc / cudaFree: a process whose device memory is
 * fully reserved by a caching allocator (a new cudaMalloc would fail), or a
 * monitoring thread beside running graph replays (cudaFree synchronises the
 * whole device).  The paper has no counterpart; this is a library service.
 * The FP32 conversion is staged in one fixed device array of 4 Mi floats
 * (16 MiB) that every GPU loading the library holds until the process exits;
 * a field of more than 4 Mi padded cells (nth * NR * NZ rounded up to 32 in z)
 * is rejected with SIM_EINVAL.  The first call on a device looks up the
 * array's device address, so make it before any stream capture.  All calls
 * share the array: calls that overlap on the GPU (two threads, two handles
 * at once) race; serialise them.  Synchronises the handle's stream. */
int sim_read_field_noalloc(sim_t *h, int which, float *out, size_t n);

/* Overwrite field `which` from host FP32 [nth][NR][NZ] (initial conditions). */
int sim_write_field(sim_t *h, int which, const float *in, size_t n);

/* The time step sim_create would take for this grid and medium (reading R7
 * of the scheme, Sec. 3: cfl * min over cells 1 / (Vp sqrt(1/dr^2 +
 * 1/(r dtheta)^2 + 1/dz^2)), r the cell centre; grid->dt when > 0), computed
 * on the host without any device call.  SIM_EINVAL for a malformed grid or
 * an out-of-range material ID; the message is sim_last_error(NULL). */
int sim_time_step(const sim_grid_t *grid, const sim_medium_t *medium, double *dt);

/* The device watchdog's last energy proxy, its reference (the first proxy
 * after the source wavelet ended; 0 until then) and the step of the last
 * check (see opts.watchdog_every).  Synchronises the handle's stream; any
 * output pointer may be NULL.  SIM_EINVAL when the watchdog is off.
 * sim_load restarts the reference. */
int sim_watchdog(sim_t *h, double *energy, double *reference, int *step);

/* The stochastic rounding of the FP16-SR storage (SIM_STORAGE_F16_SR) applied
 * to n FP32 values, for checking it value by value: out[q] = the FP16 bit
 * pattern of x[q] rounded up in magnitude when the 13 bits that FP16 drops
 * below its spacing u, read as frac(|x| / u) * 8192, exceed dither[q] & 0x1fff
 * (u = 2^-24 below 2^-14, the same rule on the exact frac there); zero,
 * non-finite values and magnitudes beyond 65504 round to nearest.  x, dither
 * and out are DEVICE pointers of n elements, owned by the caller;
 * cuda_stream: the stream to run on (NULL = the default stream), synchronised
 * before return.  SIM_EINVAL for n < 0 or a null pointer with n > 0,
 * SIM_ECUDA for a launch failure. */
int sim_round_f16_sr(const float *x, const unsigned *dither, unsigned short *out, long long n, void *cuda_stream);

/* Time step in seconds, steps done so far, device bytes held. */
double sim_dt(const sim_t *h);
int sim_steps_done(const sim_t *h);
size_t sim_device_bytes(const sim_t *h);

/* Path the handle runs: *kernel = SIM_KERNEL_SPLIT, SIM_KERNEL_FUSED or
 * SIM_KERNEL_MARCH; *tile_rows = the tile code chosen by the autotuner (or
 * forced by opts.tile): r (< 100) for the fused kernel with r rows per block,
 * 100 + r for its four-cells-per-thread variant; 1000 + 100 r + J for the
 * marching kernels with r rows per block and runs of J theta planes; 2000 for
 * the split kernels, 2000 + b for their load-first variant (four z cells per
 * thread) compiled for b resident blocks per SM (b = 3, 4, 5; blocks walk theta
 * fastest), 2010 + b for the same with the blocks walking z fastest (b = 3, 4),
 * 2100 + b for two z cells per thread (b = 6, 8), 2200 + 10 c + b for interior /
 * edge split launches (a kernel with the interior body only on the tiles away
 * from every PML and end, compiled for b blocks per SM, and the general kernel
 * on the rest; interior four cells per thread, b = 4, 5, with edge c = 0 (four
 * cells, 4 blocks/SM), 2 (two, 4), 3 (two, 6), 4 (four, 3); interior two
 * cells, b = 6, 8, with edge c = 1 (two, 6) or 5 (two, 4); c = 6, 7 as 2, 4
 * with a persistent interior kernel prefetching its next tile into L2; c = 8
 * as 4 and c = 9 as 6, each with the edge tiles walked by a persistent
 * prefetching kernel); 2300 + 10 c + b for a three-way split (interior; the
 * radial-PML rows' interior z tiles with a body for interior z; the z ends),
 * interior b = 5 plain or 4 prefetching, c = 0 to 3 the radial / end kernels'
 * cells per thread and blocks per SM;
 * v * 10000 + s (a pair code) for the velocity kernel of split code v with the
 * stress kernel of split code s; 3000 + 100 m + 10 e + b for the single-pass
 * sweep kernel (kernel = SIM_KERNEL_SWEEP: four z cells per thread, b resident
 * blocks per SM, the general body in runs of e cells; (b, e) = (3, 4) or
 * (4, 2); m = 0, 1: z chunks of 32 cells with stress items 3 chunks behind,
 * m = 2, 3: chunks of 64 cells 2.5 chunks behind, m = 4, 5: chunks of 32
 * cells 2.5 and 2 chunks behind; m = 1, 3 add an L2 prefetch of each block's
 * next velocity item).
 * opts.tile accepts every code listed here. */
int sim_config(const sim_t *h, int *kernel, int *tile_rows);

/* Test hook of the failure path of the sweep kernel (SIM_KERNEL_SWEEP), the
 * one kernel whose blocks wait on one another: the stress items of a z chunk
 * wait, bounded, for the velocity items of that chunk and its two
 * neighbours.  wait_cycles > 0 sets the limit of one wait in SM clock cycles
 * (0 restores the default 2^31, about 1 s); withhold_chunk >= 0 makes the
 * velocity items of that chunk (cells 32 c .. 32 c + 31 along z for the
 * 32-cell chunks, 64 c .. for the 64-cell ones) never report, so that the
 * waits on it run out: the kernel sets the status word, the warps that gave
 * up skip their cells, every later wait gives up at once, and the next
 * sim_sync returns SIM_ETIMEOUT (the state is then void; destroy the
 * handle).  -1 turns the withholding off; SIM_EINVAL unless -1 <=
 * withhold_chunk < ceil(NZ / 32).  Other paths ignore both.  The paper has no
 * counterpart. */
int sim_set_wait_test(sim_t *h, long long wait_cycles, int withhold_chunk);

/* Kernel timings gathered with opts.timing = 1: for kernel slot q
 * (0 = fused or sweep kernel, or the velocity kernel of the split and marching paths,
 * 1 = their stress kernel, 2 = receivers), total milliseconds and launch count so far.
 * Synchronises. */
int sim_kernel_time(sim_t *h, int q, double *ms, long *launches);

/* Checkpoint: write / read fields, PML memory variables, step counter and
 * traces to / from a file.  sim_load needs a handle created with the same
 * grid, medium, source, receivers and options. */
int sim_save(sim_t *h, const char *path);
int sim_load(sim_t *h, const char *path);

void sim_destroy(sim_t *h);
const char *sim_last_error(const sim_t *h);
const char *sim_error_string(int code);

/* ------------------------------------------------------------------------
 * Batched scenarios: n independent wells (e.g. cement-hardening cases of
 * uneven length) advanced together in one stream and one captured graph.
 * Each case is defined exactly as for sim_create (grid, medium, source,
 * receivers; shapes may differ between cases); opts is shared (storage,
 * stream, device, mem_cap applied to the batch total, graph_chunk,
 * max_steps; opts.kernel is ignored).  Cases of fewer than 4 Mi cells share
 * one interior and one edge launch per half step of the load-first split
 * bodies, driven by blocks that walk a work list of (case, theta, r tile, z
 * tile) items; the number of blocks is chosen by timing candidates at create
 * time.  A larger case fills the GPU alone and runs its own split launches
 * with the code its tuner picks (as sim_create with kernel SIM_KERNEL_SPLIT);
 * those cases are spread over 1, 2 or 4 parallel streams (branches of the
 * captured graph, the count timed at create time), so that one case's launch
 * tails overlap another's work.  opts.tile: 0 = as above; 1 = every case in
 * the shared launches, whatever its size; -1, -2, -4 = that many branches.  Every case computes what its own sim_create handle on
 * the split path computes, to FP32 rounding.  SIM_EINVAL for a shared case
 * of more than 2^31 - 1 items.
 * ------------------------------------------------------------------------ */
typedef struct simb_s simb_t;

/* Arrays hold n entries.  On failure *out is NULL and simb_last_error(NULL)
 * names the failing case. */
int simb_create(int n, const sim_grid_t *grids, const sim_medium_t *media, const sim_source_t *sources,
                const sim_receivers_t *receivers, const sim_opts_t *opts, simb_t **out);

/* Enqueue nsteps leapfrog steps of every case (nsteps >= 0). */
int simb_run(simb_t *b, int nsteps);

/* Wait for the batch; reports device-side failures of any case. */
int simb_sync(simb_t *b);

/* Traces of case `which` as sim_traces; field of case `which` as sim_read_field. */
int simb_traces(simb_t *b, int which, float *out, size_t cap, int *n_rec, int *n_steps);
int simb_read_field(simb_t *b, int which, int field, float *out, size_t n);

/* Number of cases, work items of the shared launches, persistent blocks per shared launch. */
int simb_config(const simb_t *b, int *n_cases, long long *work_items, int *grid_blocks);
/* Cases on their own launches and the parallel streams they run on. */
int simb_layout(const simb_t *b, int *own_cases, int *branches);

void simb_destroy(simb_t *b);
const char *simb_last_error(const simb_t *b);

/* ------------------------------------------------------------------------
 * Azimuthally refined grid (paper Sec. 3, "Azimuth grid refinement": the
 * azimuthal step halves each time the radius doubles).  The rows form
 * n_zones radial zones; zone m starts at row row0[m - 1] (zone 0 at row 0)
 * and has grid.nth / 2^(n_zones - 1 - m) azimuthal nodes, so the outermost
 * zone has grid.nth.  Inside a zone the scheme is the uniform grid's.  Where
 * a stencil crosses an interface it reads the other zone's row at its own
 * nodes: coarse -> fine by trigonometric (FFT zero-padding) interpolation,
 * the Nyquist coefficient split; fine -> coarse by its adjoint
 * (dtheta_fine / dtheta_coarse) P^T, which keeps the discrete energy exact.
 * dt follows the CFL rule with each row's own azimuthal step, so coarse
 * zones near the axis allow a larger dt than the uniform grid.
 *
 * Arguments as sim_create; the medium is given on the finest azimuthal grid
 * [grid.nth][nr + pml_r][nz + 2 pml_z] and zone m samples it at its nodes
 * (cell j of zone m = cell j 2^(n_zones - 1 - m)).  Restrictions (SIM_EINVAL
 * or SIM_EUNSUPPORTED): 1 to 5 zones; with interfaces grid.nth in {8, 16, 32,
 * 64} and nth / 2^(n_zones - 1) >= 4; interface rows increasing, at least two
 * rows per zone, the radial PML inside the last zone (row0 <= nr - 2); FP32
 * storage; any source kind, placed on the nodes of the zone that holds it
 * (the transverse force off the axis and the torsion ring not on a zone's
 * first row, SIM_EUNSUPPORTED).  Every zone runs the split kernels, velocity
 * code 2285 and stress code 2324 (largest zone of at least 8 Mi cells; the
 * zones of a half then run on parallel streams) or 2294 (smaller grids, zones
 * one after another) unless opts.tile names a 22xx / 23xx split code or pair
 * code (SIM_EINVAL otherwise).
 * Ownership and errors as sim_create; simr_last_error(NULL) after a failed create.
 * ------------------------------------------------------------------------ */
typedef struct {
  int n_zones;
  const int *row0; /* n_zones - 1 interface rows */
} simr_zones_t;
typedef struct simr_s simr_t;

/* The interface maps in FP64 (host only, no device call): coarse -> fine
 * (fine_to_coarse = 0) the [2n][n] trigonometric interpolation matrix of n
 * coarse azimuthal nodes, for the integer (half = 0) or half-integer (half = 1)
 * nodes; fine -> coarse (fine_to_coarse = 1) its adjoint [n][2n] = P^T / 2.
 * out holds 2 n^2 doubles, row-major.  The refined grid applies them in FP32.
 * SIM_EINVAL for n < 4, odd n or a null out. */
int simr_interface_matrix(int n_coarse, int half, int fine_to_coarse, double *out);

int simr_create(const sim_grid_t *grid, const simr_zones_t *zones, const sim_medium_t *medium,
                const sim_source_t *source, const sim_receivers_t *receivers, const sim_opts_t *opts, simr_t **out);
/* Enqueue nsteps leapfrog steps (CUDA-graph chunks of opts.graph_chunk steps). */
int simr_step(simr_t *h, int nsteps);
/* Wait; SIM_EUNSTABLE if a receiver sample was not finite. */
int simr_sync(simr_t *h);
/* Traces [n_rec][n_steps] in the order of the receivers given at create. */
int simr_traces(simr_t *h, float *out, size_t cap, int *n_rec, int *n_steps);
/* Zone geometry: first row, rows, azimuthal nodes. */
int simr_zone(const simr_t *h, int zone, int *row, int *rows, int *nth);
/* Field (F order of sim_read_field) of one zone: [nth_zone][rows][nz + 2 pml_z] FP32, n floats. */
int simr_read_field(simr_t *h, int field, int zone, float *out, size_t n);
double simr_dt(const simr_t *h);
int simr_steps_done(const simr_t *h);
/* Cells updated per step (every zone's own rows). */
size_t simr_cells(const simr_t *h);
void simr_destroy(simr_t *h);
const char *simr_last_error(const simr_t *h);

/* ------------------------------------------------------------------------
 * Trace surrogate: maps the six case parameters of a cement-hardening
 * scenario to its 8 receiver traces over the reflected window.  The paper
 * has no learned component; this network is trained on traces the simulator
 * itself produces and the simulator remains the fallback.
 *
 *   h1 = gelu(x W1 + b1), h2 = gelu(h1 W2 + b2),
 *   a0 = gelu(reshape(h2 W3 + b3, [l0][chans[0]])),
 *   a_{l+1} = gelu(convT(a_l)) for l < n_up (kernel 4, stride 2, padding 1),
 *   y = a_{n_up} Wf + bf  -> output [out_ch][l0 * 2^n_up]
 * with gelu(x) = x/2 (1 + tanh(sqrt(2/pi)(x + 0.044715 x^3))), inputs
 * normalised as (x - mean) / scale and outputs multiplied by y_scale.  BF16 weights and activations at every
 * GEMM, FP32 accumulation, FP32 Adam master weights.  Parameters are one
 * FP32 vector in the order W1 [in][h1], b1, W2 [h1][h2], b2, W3 [h2][l0*c0],
 * b3, then (T_l [c_l][c_{l+1}][4], t_l) per transposed convolution, then
 * Wf [c_n][out_ch], bf.  Host buffers are row-major FP32.
 * ------------------------------------------------------------------------ */
typedef struct {
  int in_dim, h1, h2, l0, n_up;
  int chans[9];       /* chans[0]: channels of the reshaped dense output; chans[l+1]: after convT l */
  int out_ch;
  int max_batch;      /* samples per device pass */
  unsigned long long seed;  /* initial weights: uniform +-sqrt(6/(fan_in+fan_out)), biases 0 */
} sur_cfg_t;

typedef struct sur_s sur_t;

int sur_create(const sur_cfg_t *cfg, const sim_opts_t *opts, sur_t **out);  /* opts: device, stream */
int sur_param_count(const sur_t *s, long long *n);
int sur_get_params(sur_t *s, float *out, size_t n);
int sur_set_params(sur_t *s, const float *in, size_t n);   /* also resets the Adam moments */
/* inputs enter as (x - x_mean) / x_scale; outputs and targets are in units of
 * y_scale (the network works on y / y_scale) */
int sur_set_normalization(sur_t *s, const float *x_mean, const float *x_scale, float y_scale);
/* Y[n][out_ch][l0 * 2^n_up] from raw inputs X[n][in_dim]. */
int sur_forward(sur_t *s, const float *X, int n, float *Y);
/* Mean-square loss of the normalised output against Y[n][out_ch][L] / y_scale
 * and its gradient (n <= max_batch). */
int sur_loss_grad(sur_t *s, const float *X, const float *Y, int n, float *loss, float *grad, size_t ngrad);
/* Adam (beta 0.9 / 0.999, eps 1e-8), cosine learning-rate decay from lr over
 * all steps, minibatches of `batch` drawn by a seeded shuffle each epoch;
 * epoch_loss[epochs] receives the mean minibatch loss per epoch (may be NULL). */
int sur_train(sur_t *s, const float *X, const float *Y, int n, int epochs, int batch, float lr,
              unsigned long long seed, float *epoch_loss);
/* Fallback gate: fit on validation inputs and their relative errors; a query
 * is accepted when the largest error among its k nearest validation inputs
 * (normalised distance) is <= tol, else the caller runs the simulator. */
int sur_gate_fit(sur_t *s, const float *X, const float *err, int n);
int sur_gate(sur_t *s, const float *X, int n, int k, float tol, int *accept);
/* Local sensitivity of the network at each of the n host inputs X[n][in_dim]:
 * sens[q] = max over input dimensions d of ||f(x_q + step scale_d e_d) -
 * f(x_q)|| / ||f(x_q)|| (L2 over the whole output; step in normalised input
 * units, scale_d the normalisation's scale), from (in_dim + 1) forward passes
 * per query on the device.  A second gate signal: an answer whose output
 * swings under a small move of its inputs sits where the network is least
 * trustworthy.  step > 0; sens is a host array of n floats (infinity where
 * f(x_q) = 0). */
int sur_sensitivity(sur_t *s, const float *X, int n, float step, float *sens);
void sur_destroy(sur_t *s);
const char *sur_last_error(const sur_t *s);

/* Tensor-core GEMM of the surrogate on host buffers: C[M][N] = op(A) op(B),
 * A and B BF16 bit patterns (row-major, op = transpose when trans_* != 0),
 * C FP32; for testing the kernel against an FP64 product of the same inputs.
 * Products of at least 128 rows run on the tcgen05 kernel (accumulator in
 * tensor memory), narrower ones on the mma.sync kernel, as in training. */
int cw_gemm_bf16(int trans_a, int trans_b, int M, int N, int K, const uint16_t *A, int lda, const uint16_t *B,
                 int ldb, float *C, int ldc);

/* The same with the kernel named: path 0 = by shape (as above), 1 = the
 * mma.sync kernel, 2 = the tcgen05 kernel for any shape.  SIM_ETIMEOUT if a
 * bounded wait of the tcgen05 kernel gave up (the TMEM it held is freed). */
int cw_gemm_bf16_path(int path, int trans_a, int trans_b, int M, int N, int K, const uint16_t *A, int lda,
                      const uint16_t *B, int ldb, float *C, int ldc);

#ifdef __cplusplus
}
#endif
#endif /* CWELL_H */
