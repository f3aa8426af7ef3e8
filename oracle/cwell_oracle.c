/*
 * FP64 CPU oracle of the cased-well velocity-stress scheme.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * reference the CUDA simulator is checked against.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * simulator never does.  It shares no code with the CUDA path.
 *
 * What it computes (paper: "Parallel Modeling of the Acoustic Signal
 * Propagation in a Cased Well", arXiv 2302.13907):
 *
 *   rho du/dt  = A ds/dr + (1/r) B ds/dphi + C ds/dz + (1/r)(A - D) s + F   (Eq. 1a)
 *   M ds/dt    = A^T du/dr + (1/r) B^T du/dphi + C^T du/dz + (1/r) D^T u + G (Eq. 1b)
 *
 * with u = (u_r, u_phi, u_z), s = (s_rr, s_phiphi, s_zz, s_rphi, s_phiz, s_rz),
 * the selector matrices A, B, C, D and the isotropic compliance M of Sec. 2,
 * zero initial data (Eq. 2), a liquid modelled as mu = 0 (Sec. 2), medium
 * parameters attached to the cell centre (Sec. 3), a staggered (Virieux-type)
 * grid in cylindrical coordinates (Sec. 3), a PML at the outer radius and at
 * both z ends without splitting in azimuth (Sec. 1, Sec. 6), a volumetric
 * point source with a Ricker wavelet delayed by 2/f0 (Sec. 2).
 *
 * Readings where the printed paper is garbled or silent (each one is listed
 * with its justification in the design notes of the repository):
 *  R1  Eq. 1 as printed drops the B and C terms of the velocity equation and
 *      writes A^T du/dz where the structure needs A^T du/dr; D is the
 *      transpose of the printed 6x3 matrix.  Written out this gives
 *        rho du_r/dt   = ds_rr/dr + (1/r) ds_rphi/dphi + ds_rz/dz + (s_rr - s_phiphi)/r
 *        rho du_phi/dt = ds_rphi/dr + (1/r) ds_phiphi/dphi + ds_phiz/dz + 2 s_rphi/r
 *        rho du_z/dt   = ds_rz/dr + (1/r) ds_phiz/dphi + ds_zz/dz + s_rz/r
 *      and engineering strain rates e_rr = du_r/dr, e_phiphi = (1/r)du_phi/dphi
 *      + u_r/r, e_zz = du_z/dz, g_rphi = du_phi/dr + (1/r)du_r/dphi - u_phi/r,
 *      g_phiz = (1/r)du_z/dphi + du_phi/dz, g_rz = du_z/dr + du_r/dz.
 *  R2  M is singular for mu = 0, so the stress is advanced in stiffness form
 *      ds/dt = C e with C = M^{-1} (Lame form) for mu > 0 and its lambda-only
 *      limit for a liquid.  The printed M_22 entry is read as (l+m)/(3l+2m).
 *  R3  staggering: normal stresses at (i+1/2, j, k), v_r at (i, j, k),
 *      v_phi at (i+1/2, j+1/2, k), v_z at (i+1/2, j, k+1/2), s_rphi at
 *      (i, j+1/2, k), s_rz at (i, j, k+1/2), s_phiz at (i+1/2, j+1/2, k+1/2),
 *      with r_i = i dr and flux-form radial differences so that the discrete
 *      velocity operator is minus the r-weighted adjoint of the strain-rate
 *      operator (discrete energy conservation).
 *  R4  axis: v_r, s_rphi, s_rz at r = 0 are not unknowns (held zero); ring 0
 *      must be liquid.
 *  R5  density at a velocity node: arithmetic mean of its two cells; shear
 *      modulus at a shear node: harmonic mean of its four cells, zero when
 *      any of them is zero.
 *  R6  volumetric source: the printed normalisation is singular in a liquid;
 *      read as an isotropic moment-rate source s_ii += dt * A f(t_{n+1/2})
 *      * delta_h, delta_h = 1 / (cell volume) (on the axis 1/(pi dr^2 dz)
 *      shared by all ring-0 nodes).
 *  R7  dt = CFL * min over cells of 1 / (Vp sqrt(1/dr^2 + 1/(r dphi)^2 + 1/dz^2)).
 *  R8  PML (cited by the paper, Sec. 1, without formulas): complex stretching
 *      of r and z in convolutional form.  Every radial difference is
 *      stretched by s_r = 1 + d_r/(alpha + i w) and every 1/r term (hoop,
 *      azimuthal and axis terms) by r/r~, r~ = r + int d_r/(alpha + i w),
 *      whose memory variable uses the integrated profile
 *      dbar(r) = (1/r) int_{r_pml}^{r} d_r; every z difference by s_z.  The
 *      azimuthal derivative is never split off ("no splitting of variables in
 *      the azimuth direction", Sec. 6).  Memory variables: psi <- b psi + a D,
 *      D <- D + psi, b = exp(-(d + alpha) dt), a = d (b - 1) / (d + alpha),
 *      d(x) = d0 (x/L)^2, d0 = -3 Vp_max ln(R0) / (2 L), R0 = 1e-3,
 *      alpha = pi f0 (constant, so that s_r = dr~/dr holds exactly).
 *      Outside the PML the walls are rigid.
 *  R9  closed walls: v_r = s_rphi = s_rz = 0 at r = NR dr; v_z = s_rz =
 *      s_phiz = 0 at the z half-nodes -1/2 and NZ - 1/2; theta periodic.
 *  R12 point forces (the paper's transverse and longitudinal point impacts,
 *      F = (1,0,0) f and (0,0,1) f; the printed normalisation is singular in
 *      a liquid): v += dt * A f(t_n) / (rho_node * V_node) after the velocity
 *      half-step, t_n = n dt, rho_node the two-cell mean of R5.  Longitudinal
 *      on the axis: every ring-0 v_z node, V = pi dr^2 dz (as R6).
 *      Transverse on the axis (a horizontal force in direction phi0): the
 *      ring-1 v_r nodes, each with the share 2 cos(theta_j - phi0) / Ntheta
 *      of the force, V = dr^2 dphi dz, so that the momentum put in along phi0
 *      is dt A f.  Off the axis: the nearest v_r (v_z) node, V = r dr dphi dz.
 *  R13 torsion source (printed G = (0,0,0,1,1,0) f): an axisymmetric torque
 *      about the well axis, s_rphi and s_phiz += dt * A f(t_{n+1/2}) /
 *      (2 pi r dr dz) on every theta node of the ring at r0 (s_rphi at
 *      r_i = i dr, i = round(r0 / dr); s_phiz at r_{i'+1/2}, i' = floor(r0 /
 *      dr)); both nodes must have a non-zero shear modulus.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)
#define OR_EUNSUPPORTED (-6)

enum { F_VR, F_VP, F_VZ, F_SRR, F_SPP, F_SZZ, F_SRP, F_SPZ, F_SRZ, NFIELD };
/* memory variables: _R radial difference, _Q 1/r group, _Z z difference */
enum {
  P_VR_R, P_VP_R, P_VZ_R, P_VR_Z, P_VP_Z, P_VZ_Z,
  P_ERR_R, P_GRP_R, P_GRZ_R, P_EZZ_Z, P_GRZ_Z, P_GPZ_Z,
  P_VR_Q, P_VP_Q, P_VZ_Q, P_EPP_Q, P_GRP_Q, P_GPZ_Q, NPSI
};

typedef struct {
  int nr, nth, nz, pml_r, pml_z, NR, NZ;
  double dr, dz, dth, dt, f0;
  int pml_on;
  size_t ncell;
  uint16_t *id;
  int n_mat;
  double *rho, *lam, *mu;
  double *f[NFIELD];
  double *psi[NPSI];
  /* 1-D PML coefficients: r at integer / half nodes (radial difference and
     1/r group), z at integer / half nodes */
  double *ar_i, *br_i, *ar_h, *br_h, *aq_i, *bq_i, *aq_h, *bq_h, *az_i, *bz_i, *az_h, *bz_h;
  /* source: injection points (field, cell, weight per unit f(t)) */
  int src_kind, src_n;
  int *src_field;
  size_t *src_cell;
  double *src_w;
  /* receivers */
  int n_rec, *rec_i, *rec_j, *rec_k; /* rec_j = -1: mean over ring 0 */
  int cap, steps_done;
  double *traces;
  int threads;
  /* storage rounding (precision variant): 0 none, 1 BF16, 2 FP16, 3 FP16
     with stochastic rounding; stored value = round(value * scale), scale
     st_sv (velocities), st_ss (stresses) */
  int storage;
  double st_sv, st_ss;
  /* z range the updates, the sources and the receivers cover (a z slab of
     a decomposed run: the cells outside are the neighbours' and arrive by
     exchange); 0 .. NZ by default */
  int k_lo, k_hi;
} or_sim;

/* Ricker pulse with dominant frequency f0 and delay 2/f0 (Sec. 2). */
double or_ricker(double t, double f0) {
  double a = M_PI * f0 * (t - 2.0 / f0);
  a = a * a;
  return (1.0 - 2.0 * a) * exp(-a);
}

/*
 * Storage rounding of the precision variant (FP32 arithmetic on fields kept
 * in a 16-bit format; the paper computes in full precision, so this is a
 * property of the storage format, written from the IEEE 754 definitions):
 * the value is first rounded to binary32 (the arithmetic precision of the
 * variant), then to the format with p significant bits, minimum normal
 * exponent emin and largest finite value maxf, both steps round to nearest,
 * ties to even.  Below 2^emin the spacing stays 2^(emin - p + 1) (gradual
 * underflow); a result beyond maxf is an infinity.
 *   BF16: p = 8,  emin = -126, maxf = (2 - 2^-7) 2^127
 *   FP16: p = 11, emin = -14,  maxf = 65504
 */
static double round_format(double x, int p, int emin, double maxf) {
  if (x == 0.0 || !isfinite(x)) return x;
  int e;
  frexp(x, &e);              /* |x| in [2^(e-1), 2^e) */
  int E = e - 1;
  if (E < emin) E = emin;
  const double ulp = ldexp(1.0, E - (p - 1));
  const double q = nearbyint(x / ulp) * ulp; /* exact scaling, round half to even */
  if (fabs(q) > maxf) return copysign(INFINITY, x);
  return q;
}

double or_round_storage(double x, int mode) {
  const double f = (double)(float)x; /* binary32 first */
  if (mode == 1) return round_format(f, 8, -126, 0x1.fep127);
  if (mode == 2) return round_format(f, 11, -14, 65504.0);
  return x;
}

/*
 * Stochastic rounding to FP16 (storage mode 3): the binary32 value x of
 * magnitude a is rounded down to the FP16 grid, a_lo = floor(a / u) u with
 * u = 2^(E - 10) the grid spacing (E the exponent of a, at least -14), and
 * up to a_lo + u when frac(a / u) * 2^13 > d, d a 13-bit dither, so that the
 * expected result is x.  Beyond 65504 (and for zero) round to nearest.
 */
double or_round_stochastic_f16(double x, unsigned d) {
  const double f = (double)(float)x;
  const double a = fabs(f);
  if (!(a <= 65504.0) || a == 0.0) return round_format(f, 11, -14, 65504.0);
  int e;
  frexp(a, &e);
  int E = e - 1;
  if (E < -14) E = -14;
  const double q = ldexp(a, 10 - E), fl = floor(q);
  const double m = ldexp(fl + ((q - fl) * 8192.0 > (double)d ? 1.0 : 0.0), E - 10);
  return copysign(m, f);
}

/* SplitMix64 (Steele, Lea and Flood, 2014): the output for counter value
   key, i.e. the mix of state (key + 1) * 0x9E3779B97F4A7C15. */
uint64_t or_splitmix64(uint64_t key) {
  uint64_t z = (key + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* The 13-bit dither of field q of cell (j, i, k) in the update of step n:
   one SplitMix64 output per group of four cells along z, 16 bits per cell. */
unsigned or_sr_dither(int n, int q, int j, int i, int k, int nth, int NR, int NZ) {
  const uint64_t ngrp = (uint64_t)((NZ + 3) / 4);
  const uint64_t key = ((((uint64_t)n * 9u + (uint64_t)q) * (uint64_t)nth + (uint64_t)j) * (uint64_t)NR +
                        (uint64_t)i) * ngrp + (uint64_t)(k / 4);
  return (unsigned)((or_splitmix64(key) >> (16 * (k % 4))) & 0x1fffu);
}

/* Reading R7 of the time step. */
double or_cfl_dt(int nth, int NR, int NZ, double dr, double dz, const uint16_t *id, const double *vp, double cfl) {
  double dth = 2.0 * M_PI / nth, best = INFINITY;
  for (int j = 0; j < nth; j++)
    for (int i = 0; i < NR; i++) {
      double rc = (i + 0.5) * dr;
      double s = sqrt(1.0 / (dr * dr) + 1.0 / ((rc * dth) * (rc * dth)) + 1.0 / (dz * dz));
      for (int k = 0; k < NZ; k++) {
        double c = vp[id[((size_t)j * NR + i) * NZ + k]];
        if (c > 0) {
          double t = 1.0 / (c * s);
          if (t < best) best = t;
        }
      }
    }
  return cfl * best;
}

/* recursive-convolution coefficients for damping d and frequency shift alpha */
void cpml_ab(double d, double al, double dt, double *a, double *b) {
  if (!(d > 0.0)) {
    *a = 0.0;
    *b = 1.0;
    return;
  }
  *b = exp(-(d + al) * dt);
  *a = d * (*b - 1.0) / (d + al);
}

/* profile d(x) = d0 (x/L)^2 at depth x into a layer of thickness L */
double pml_d(double x, double L, double d0) {
  if (x <= 0.0 || L <= 0.0) return 0.0;
  return d0 * (x / L) * (x / L);
}

/* dbar(r) = (1/r) int_0^x d, the damping of the stretched radius r~ */
double pml_dbar(double x, double r, double L, double d0) {
  if (x <= 0.0 || L <= 0.0 || r <= 0.0) return 0.0;
  return d0 * x * x * x / (3.0 * L * L) / r;
}

void or_destroy(or_sim *s) {
  if (!s) return;
  free(s->id);
  free(s->rho);
  free(s->lam);
  free(s->mu);
  for (int q = 0; q < NFIELD; q++) free(s->f[q]);
  for (int q = 0; q < NPSI; q++) free(s->psi[q]);
  free(s->ar_i); free(s->br_i); free(s->ar_h); free(s->br_h);
  free(s->aq_i); free(s->bq_i); free(s->aq_h); free(s->bq_h);
  free(s->az_i); free(s->bz_i); free(s->az_h); free(s->bz_h);
  free(s->rec_i); free(s->rec_j); free(s->rec_k);
  free(s->src_field); free(s->src_cell); free(s->src_w);
  free(s->traces);
  free(s);
}

#define IX(j, i, k) (((size_t)(j) * NR + (i)) * NZ + (k))

/* R5 averages */
static inline double rho_avg2(const or_sim *s, size_t c1, size_t c2) {
  return 0.5 * (s->rho[s->id[c1]] + s->rho[s->id[c2]]);
}
static inline double mu_harm4(const or_sim *s, size_t c1, size_t c2, size_t c3, size_t c4) {
  double m1 = s->mu[s->id[c1]], m2 = s->mu[s->id[c2]], m3 = s->mu[s->id[c3]], m4 = s->mu[s->id[c4]];
  if (m1 == 0.0 || m2 == 0.0 || m3 == 0.0 || m4 == 0.0) return 0.0;
  return 4.0 / (1.0 / m1 + 1.0 / m2 + 1.0 / m3 + 1.0 / m4);
}

/*
 * Create the oracle state.  Arrays are copied.  dt_override > 0 replaces the
 * CFL rule.  Returns NULL and sets *err on failure.
 */
or_sim *or_create(int nr, int nth, int nz, int pml_r, int pml_z, double dr, double dz,
                  int n_mat, const double *rho, const double *vp, const double *vs,
                  const uint16_t *cell_id, double cfl, double dt_override, int pml_on,
                  int src_kind, double src_r, double src_theta, double src_z, double f0, double src_amp,
                  int n_rec, const double *rec_r, const double *rec_theta, const double *rec_z,
                  int max_steps, int *err) {
  *err = OR_EINVAL;
  if (nr < 1 || nth < 4 || (nth & 1) || nz < 2 || pml_r < 0 || pml_z < 0 || !(dr > 0) || !(dz > 0) ||
      n_mat < 1 || n_rec < 0 || max_steps < 0 || src_kind < 0 || src_kind > 3)
    return NULL;
  or_sim *s = (or_sim *)calloc(1, sizeof(or_sim));
  if (!s) { *err = OR_ENOMEM; return NULL; }
  s->nr = nr; s->nth = nth; s->nz = nz; s->pml_r = pml_r; s->pml_z = pml_z;
  s->NR = nr + pml_r; s->NZ = nz + 2 * pml_z;
  s->dr = dr; s->dz = dz; s->dth = 2.0 * M_PI / nth; s->f0 = f0; s->pml_on = pml_on;
  s->ncell = (size_t)nth * s->NR * s->NZ;
  s->threads = 0;
  s->storage = 0;
  s->st_sv = s->st_ss = 1.0;
  s->k_lo = 0;
  s->k_hi = nz + 2 * pml_z;
  int NR = s->NR, NZ = s->NZ;
  s->id = (uint16_t *)malloc(s->ncell * sizeof(uint16_t));
  s->n_mat = n_mat;
  s->rho = (double *)malloc(n_mat * sizeof(double));
  s->lam = (double *)malloc(n_mat * sizeof(double));
  s->mu = (double *)malloc(n_mat * sizeof(double));
  for (int q = 0; q < NFIELD; q++) s->f[q] = (double *)calloc(s->ncell, sizeof(double));
  for (int q = 0; q < NPSI; q++) s->psi[q] = (double *)calloc(s->ncell, sizeof(double));
  s->ar_i = malloc(NR * sizeof(double)); s->br_i = malloc(NR * sizeof(double));
  s->ar_h = malloc(NR * sizeof(double)); s->br_h = malloc(NR * sizeof(double));
  s->aq_i = malloc(NR * sizeof(double)); s->bq_i = malloc(NR * sizeof(double));
  s->aq_h = malloc(NR * sizeof(double)); s->bq_h = malloc(NR * sizeof(double));
  s->az_i = malloc(NZ * sizeof(double)); s->bz_i = malloc(NZ * sizeof(double));
  s->az_h = malloc(NZ * sizeof(double)); s->bz_h = malloc(NZ * sizeof(double));
  s->n_rec = n_rec;
  s->rec_i = malloc((n_rec + 1) * sizeof(int));
  s->rec_j = malloc((n_rec + 1) * sizeof(int));
  s->rec_k = malloc((n_rec + 1) * sizeof(int));
  s->cap = max_steps;
  s->traces = (double *)calloc((size_t)(n_rec + 1) * (max_steps + 1), sizeof(double));
  int ok = s->id && s->rho && s->lam && s->mu && s->ar_i && s->br_i && s->ar_h && s->br_h && s->az_i &&
           s->aq_i && s->bq_i && s->aq_h && s->bq_h &&
           s->bz_i && s->az_h && s->bz_h && s->rec_i && s->rec_j && s->rec_k && s->traces;
  for (int q = 0; q < NFIELD; q++) ok = ok && s->f[q];
  for (int q = 0; q < NPSI; q++) ok = ok && s->psi[q];
  if (!ok) { or_destroy(s); *err = OR_ENOMEM; return NULL; }

  /* Lame parameters from the cell-centre values (Sec. 3): mu = rho Vs^2,
     lambda = rho Vp^2 - 2 mu; a liquid has mu = 0 (Sec. 2). */
  double vpmax = 0.0;
  for (int m = 0; m < n_mat; m++) {
    if (!(rho[m] > 0) || !(vp[m] > 0) || vs[m] < 0 || vp[m] * vp[m] < 2.0 * vs[m] * vs[m]) {
      or_destroy(s); return NULL;
    }
    s->rho[m] = rho[m];
    s->mu[m] = rho[m] * vs[m] * vs[m];
    s->lam[m] = rho[m] * vp[m] * vp[m] - 2.0 * s->mu[m];
    if (vp[m] > vpmax) vpmax = vp[m];
  }
  for (size_t c = 0; c < s->ncell; c++) {
    if (cell_id[c] >= n_mat) { or_destroy(s); return NULL; }
    s->id[c] = cell_id[c];
  }
  /* R4: ring 0 must be a liquid */
  for (int j = 0; j < nth; j++)
    for (int k = 0; k < NZ; k++)
      if (s->mu[s->id[((size_t)j * NR + 0) * NZ + k]] != 0.0) {
        or_destroy(s); *err = OR_EUNSUPPORTED; return NULL;
      }

  s->dt = dt_override > 0 ? dt_override : or_cfl_dt(nth, NR, NZ, dr, dz, s->id, vp, cfl);

  /* R8: PML profiles at the staggered positions. */
  double Lr = pml_r * dr, Lz = pml_z * dz;
  double d0r = Lr > 0 ? -3.0 * vpmax * log(1e-3) / (2.0 * Lr) : 0.0;
  double d0z = Lz > 0 ? -3.0 * vpmax * log(1e-3) / (2.0 * Lz) : 0.0;
  const double al = M_PI * f0;
  for (int i = 0; i < NR; i++) {
    double xi = pml_on ? (i - nr) * dr : 0.0;
    double xh = pml_on ? (i + 0.5 - nr) * dr : 0.0;
    cpml_ab(pml_d(xi, Lr, d0r), al, s->dt, &s->ar_i[i], &s->br_i[i]);
    cpml_ab(pml_d(xh, Lr, d0r), al, s->dt, &s->ar_h[i], &s->br_h[i]);
    cpml_ab(pml_dbar(xi, i * dr, Lr, d0r), al, s->dt, &s->aq_i[i], &s->bq_i[i]);
    cpml_ab(pml_dbar(xh, (i + 0.5) * dr, Lr, d0r), al, s->dt, &s->aq_h[i], &s->bq_h[i]);
  }
  for (int k = 0; k < NZ; k++) {
    double lo_i = (pml_z - 0.5 - k) * dz, hi_i = (k - (pml_z + nz - 0.5)) * dz;
    double lo_h = (pml_z - 1.0 - k) * dz, hi_h = (k + 1.0 - pml_z - nz) * dz;
    double xi = pml_on ? fmax(lo_i, hi_i) : 0.0;
    double xh = pml_on ? fmax(lo_h, hi_h) : 0.0;
    cpml_ab(pml_d(xi, Lz, d0z), al, s->dt, &s->az_i[k], &s->bz_i[k]);
    cpml_ab(pml_d(xh, Lz, d0z), al, s->dt, &s->az_h[k], &s->bz_h[k]);
  }

  /* R6, R12, R13: source injection points */
  s->src_kind = src_kind;
  {
    const int k = (int)lround(src_z / dz) + pml_z;
    if (k < pml_z || k >= pml_z + nz || src_r < 0 || src_r >= nr * dr) { or_destroy(s); return NULL; }
    const int axis = src_r < dr;
    const int js = (int)(((long)lround(src_theta / s->dth) % nth + nth) % nth);
    const double dth = s->dth;
    s->src_field = malloc(2 * nth * sizeof(int));
    s->src_cell = malloc(2 * nth * sizeof(size_t));
    s->src_w = malloc(2 * nth * sizeof(double));
    if (!s->src_field || !s->src_cell || !s->src_w) { or_destroy(s); *err = OR_ENOMEM; return NULL; }
    int n = 0, bad = 0;
#define ADD(fld, cell, w) (s->src_field[n] = (fld), s->src_cell[n] = (cell), s->src_w[n] = (w), n++)
    if (src_kind == 0) { /* volumetric, R6: the three normal stresses */
      if (axis) {
        for (int j = 0; j < nth; j++) ADD(F_SRR, IX(j, 0, k), src_amp / (M_PI * dr * dr * dz));
      } else {
        const int i = (int)floor(src_r / dr);
        ADD(F_SRR, IX(js, i, k), src_amp / ((i + 0.5) * dr * dr * dth * dz));
      }
    } else if (src_kind == 1) { /* transverse point force, R12 */
      if (axis) {
        if (NR < 2) bad = 1;
        for (int j = 0; j < nth && !bad; j++) {
          const double w = 2.0 * cos(j * dth - src_theta) / nth;
          ADD(F_VR, IX(j, 1, k), src_amp * w / (rho_avg2(s, IX(j, 0, k), IX(j, 1, k)) * dr * dr * dth * dz));
        }
      } else {
        const int i = (int)lround(src_r / dr);
        if (i < 1 || i >= NR) bad = 1;
        else ADD(F_VR, IX(js, i, k), src_amp / (rho_avg2(s, IX(js, i - 1, k), IX(js, i, k)) * i * dr * dr * dth * dz));
      }
    } else if (src_kind == 2) { /* longitudinal point force, R12 */
      if (k + 1 >= NZ) bad = 1;
      else if (axis) {
        for (int j = 0; j < nth; j++)
          ADD(F_VZ, IX(j, 0, k), src_amp / (rho_avg2(s, IX(j, 0, k), IX(j, 0, k + 1)) * M_PI * dr * dr * dz));
      } else {
        const int i = (int)floor(src_r / dr);
        ADD(F_VZ, IX(js, i, k), src_amp / (rho_avg2(s, IX(js, i, k), IX(js, i, k + 1)) * (i + 0.5) * dr * dr * dth * dz));
      }
    } else { /* torsion ring, R13 */
      const int i = (int)lround(src_r / dr), ih = (int)floor(src_r / dr);
      if (i < 1 || i >= NR || ih + 1 > NR || k + 1 >= NZ) bad = 1;
      for (int j = 0; j < nth && !bad; j++) {
        const int jp = (j + 1) % nth;
        if (mu_harm4(s, IX(j, i - 1, k), IX(j, i, k), IX(jp, i - 1, k), IX(jp, i, k)) == 0.0 ||
            mu_harm4(s, IX(j, ih, k), IX(jp, ih, k), IX(j, ih, k + 1), IX(jp, ih, k + 1)) == 0.0) {
          or_destroy(s); *err = OR_EUNSUPPORTED; return NULL;
        }
        ADD(F_SRP, IX(j, i, k), src_amp / (2.0 * M_PI * i * dr * dr * dz));
        ADD(F_SPZ, IX(j, ih, k), src_amp / (2.0 * M_PI * (ih + 0.5) * dr * dr * dz));
      }
    }
#undef ADD
    if (bad) { or_destroy(s); return NULL; }
    s->src_n = n;
  }
  for (int n = 0; n < n_rec; n++) {
    s->rec_k[n] = (int)lround(rec_z[n] / dz) + pml_z;
    if (s->rec_k[n] < pml_z || s->rec_k[n] >= pml_z + nz || rec_r[n] < 0 || rec_r[n] >= nr * dr) {
      or_destroy(s); return NULL;
    }
    if (rec_r[n] < dr) { s->rec_i[n] = 0; s->rec_j[n] = -1; }
    else {
      s->rec_i[n] = (int)floor(rec_r[n] / dr);
      s->rec_j[n] = (int)(((long)lround(rec_theta[n] / s->dth) % nth + nth) % nth);
    }
  }
  *err = OR_OK;
  return s;
}


/* stretch a difference D with its memory variable psi (R8) */
static inline double stretch(int on, double *psi, double a, double b, double D) {
  if (!on) return D;
  *psi = b * (*psi) + a * D;
  return D + *psi;
}

static void set_threads(const or_sim *s) {
#ifdef _OPENMP
  if (s->threads > 0) omp_set_num_threads(s->threads);
#else
  (void)s;
#endif
}

/* Velocity half-step v^{n-1/2} -> v^{n+1/2} from s^n (Eq. 1a, R1, R3-R5, R8). */
void or_velocity_update(or_sim *s) {
  const int NR = s->NR, NZ = s->NZ, nth = s->nth, on = s->pml_on;
  const double dr = s->dr, dz = s->dz, dth = s->dth, dt = s->dt;
  double *vr = s->f[F_VR], *vp = s->f[F_VP], *vz = s->f[F_VZ];
  const double *srr = s->f[F_SRR], *spp = s->f[F_SPP], *szz = s->f[F_SZZ];
  const double *srp = s->f[F_SRP], *spz = s->f[F_SPZ], *srz = s->f[F_SRZ];
  set_threads(s);
#pragma omp parallel for collapse(2) schedule(static)
  for (int j = 0; j < nth; j++)
    for (int i = 0; i < NR; i++) {
      const int jm = (j + nth - 1) % nth, jp = (j + 1) % nth;
      const double ri = i * dr, rh = (i + 0.5) * dr;
      for (int k = s->k_lo; k < s->k_hi; k++) {
        const size_t c = IX(j, i, k);
        /* v_r at (r_i, theta_j, z_k); r = 0 is not an unknown (R4).
           ds_rr/dr + [(s_rr - s_phiphi) + ds_rphi/dphi] / r + ds_rz/dz */
        if (i >= 1) {
          const size_t cm = IX(j, i - 1, k);
          double Dr = (srr[c] - srr[cm]) / dr;
          double Q = (0.5 * (srr[c] + srr[cm]) - 0.5 * (spp[c] + spp[cm]) + (srp[c] - srp[IX(jm, i, k)]) / dth) / ri;
          double Dz = (srz[c] - (k > 0 ? srz[IX(j, i, k - 1)] : 0.0)) / dz;
          Dr = stretch(on, &s->psi[P_VR_R][c], s->ar_i[i], s->br_i[i], Dr);
          Q = stretch(on, &s->psi[P_VR_Q][c], s->aq_i[i], s->bq_i[i], Q);
          Dz = stretch(on, &s->psi[P_VR_Z][c], s->az_i[k], s->bz_i[k], Dz);
          vr[c] += dt / rho_avg2(s, cm, c) * (Dr + Q + Dz);
        }
        /* v_phi at (r_{i+1/2}, theta_{j+1/2}, z_k):
           ds_rphi/dr + [2 s_rphi + ds_phiphi/dphi] / r + ds_phiz/dz */
        {
          double s1 = (i + 1 < NR) ? srp[IX(j, i + 1, k)] : 0.0, s0 = srp[c];
          double Dr = (s1 - s0) / dr;
          double Q = ((s1 + s0) + (spp[IX(jp, i, k)] - spp[c]) / dth) / rh;
          double Dz = (spz[c] - (k > 0 ? spz[IX(j, i, k - 1)] : 0.0)) / dz;
          Dr = stretch(on, &s->psi[P_VP_R][c], s->ar_h[i], s->br_h[i], Dr);
          Q = stretch(on, &s->psi[P_VP_Q][c], s->aq_h[i], s->bq_h[i], Q);
          Dz = stretch(on, &s->psi[P_VP_Z][c], s->az_i[k], s->bz_i[k], Dz);
          vp[c] += dt / rho_avg2(s, c, IX(jp, i, k)) * (Dr + Q + Dz);
        }
        /* v_z at (r_{i+1/2}, theta_j, z_{k+1/2}); the last half-node is a wall (R9):
           ds_rz/dr + [s_rz + ds_phiz/dphi] / r + ds_zz/dz */
        if (k + 1 < NZ) {
          double s1 = (i + 1 < NR) ? srz[IX(j, i + 1, k)] : 0.0, s0 = srz[c];
          double Dr = (s1 - s0) / dr;
          double Q = (0.5 * (s1 + s0) + (spz[c] - spz[IX(jm, i, k)]) / dth) / rh;
          double Dz = (szz[IX(j, i, k + 1)] - szz[c]) / dz;
          Dr = stretch(on, &s->psi[P_VZ_R][c], s->ar_h[i], s->br_h[i], Dr);
          Q = stretch(on, &s->psi[P_VZ_Q][c], s->aq_h[i], s->bq_h[i], Q);
          Dz = stretch(on, &s->psi[P_VZ_Z][c], s->az_h[k], s->bz_h[k], Dz);
          vz[c] += dt / rho_avg2(s, c, IX(j, i, k + 1)) * (Dr + Q + Dz);
        }
      }
    }
}

/* Stress step s^n -> s^{n+1} from v^{n+1/2} (Eq. 1b, R1-R5, R8). */
void or_stress_update(or_sim *s) {
  const int NR = s->NR, NZ = s->NZ, nth = s->nth, on = s->pml_on;
  const double dr = s->dr, dz = s->dz, dth = s->dth, dt = s->dt;
  const double *vr = s->f[F_VR], *vp = s->f[F_VP], *vz = s->f[F_VZ];
  double *srr = s->f[F_SRR], *spp = s->f[F_SPP], *szz = s->f[F_SZZ];
  double *srp = s->f[F_SRP], *spz = s->f[F_SPZ], *srz = s->f[F_SRZ];
  set_threads(s);
#pragma omp parallel for collapse(2) schedule(static)
  for (int j = 0; j < nth; j++)
    for (int i = 0; i < NR; i++) {
      const int jm = (j + nth - 1) % nth, jp = (j + 1) % nth;
      const double ri = i * dr, rh = (i + 0.5) * dr;
      for (int k = s->k_lo; k < s->k_hi; k++) {
        const size_t c = IX(j, i, k);
        /* normal stresses at the cell centre (r_{i+1/2}, theta_j, z_k):
           e_rr = du_r/dr, e_phiphi = [du_phi/dphi + u_r] / r, e_zz = du_z/dz */
        {
          double vr0 = (i >= 1) ? vr[c] : 0.0;
          double vr1 = (i + 1 < NR) ? vr[IX(j, i + 1, k)] : 0.0;
          double err = (vr1 - vr0) / dr;
          double epp = ((vp[c] - vp[IX(jm, i, k)]) / dth + 0.5 * (vr0 + vr1)) / rh;
          double ezz = (vz[c] - (k > 0 ? vz[IX(j, i, k - 1)] : 0.0)) / dz;
          err = stretch(on, &s->psi[P_ERR_R][c], s->ar_h[i], s->br_h[i], err);
          epp = stretch(on, &s->psi[P_EPP_Q][c], s->aq_h[i], s->bq_h[i], epp);
          ezz = stretch(on, &s->psi[P_EZZ_Z][c], s->az_i[k], s->bz_i[k], ezz);
          const double l = s->lam[s->id[c]], m = s->mu[s->id[c]];
          srr[c] += dt * ((l + 2.0 * m) * err + l * (epp + ezz));
          spp[c] += dt * ((l + 2.0 * m) * epp + l * (err + ezz));
          szz[c] += dt * ((l + 2.0 * m) * ezz + l * (err + epp));
        }
        /* s_rphi at (r_i, theta_{j+1/2}, z_k):
           g_rphi = du_phi/dr + [du_r/dphi - u_phi] / r */
        if (i >= 1) {
          const size_t cm = IX(j, i - 1, k);
          double gr = (vp[c] - vp[cm]) / dr;
          double Q = ((vr[IX(jp, i, k)] - vr[c]) / dth - 0.5 * (vp[c] + vp[cm])) / ri;
          gr = stretch(on, &s->psi[P_GRP_R][c], s->ar_i[i], s->br_i[i], gr);
          Q = stretch(on, &s->psi[P_GRP_Q][c], s->aq_i[i], s->bq_i[i], Q);
          double m = mu_harm4(s, cm, c, IX(jp, i - 1, k), IX(jp, i, k));
          srp[c] += dt * m * (gr + Q);
        }
        if (k + 1 < NZ) {
          /* s_rz at (r_i, theta_j, z_{k+1/2}): g_rz = du_z/dr + du_r/dz */
          if (i >= 1) {
            double gz = (vr[IX(j, i, k + 1)] - vr[c]) / dz;
            double gr = (vz[c] - vz[IX(j, i - 1, k)]) / dr;
            gz = stretch(on, &s->psi[P_GRZ_Z][c], s->az_h[k], s->bz_h[k], gz);
            gr = stretch(on, &s->psi[P_GRZ_R][c], s->ar_i[i], s->br_i[i], gr);
            double m = mu_harm4(s, IX(j, i - 1, k), c, IX(j, i - 1, k + 1), IX(j, i, k + 1));
            srz[c] += dt * m * (gz + gr);
          }
          /* s_phiz at (r_{i+1/2}, theta_{j+1/2}, z_{k+1/2}):
             g_phiz = [du_z/dphi] / r + du_phi/dz */
          {
            double Q = (vz[IX(jp, i, k)] - vz[c]) / (rh * dth);
            double gz = (vp[IX(j, i, k + 1)] - vp[c]) / dz;
            Q = stretch(on, &s->psi[P_GPZ_Q][c], s->aq_h[i], s->bq_h[i], Q);
            gz = stretch(on, &s->psi[P_GPZ_Z][c], s->az_h[k], s->bz_h[k], gz);
            double m = mu_harm4(s, c, IX(jp, i, k), IX(j, i, k + 1), IX(jp, i, k + 1));
            spz[c] += dt * m * (Q + gz);
          }
        }
      }
    }
}

/* Source of step n (Sec. 2, R6, R12, R13): point forces (kinds 1, 2) act on
   the velocities with f(t_n) after the velocity half-step; the volumetric
   source (kind 0, all three normal stresses) and the torsion ring (kind 3)
   on the stresses with f(t_{n+1/2}) after the stress half-step. */
void or_inject_source(or_sim *s, int n) {
  const int force = s->src_kind == 1 || s->src_kind == 2;
  const double f = or_ricker((force ? n : n + 0.5) * s->dt, s->f0);
  for (int q = 0; q < s->src_n; q++) {
    const double add = s->dt * s->src_w[q] * f;
    const size_t c = s->src_cell[q];
    const int kc = (int)(c % (size_t)s->NZ);
    if (kc < s->k_lo || kc >= s->k_hi) continue; /* another slab's cell */
    if (s->src_kind == 0) {
      s->f[F_SRR][c] += add;
      s->f[F_SPP][c] += add;
      s->f[F_SZZ][c] += add;
    } else {
      s->f[s->src_field[q]][c] += add;
    }
  }
}

/* Pressure p = -(s_rr + s_phiphi + s_zz)/3 at each receiver (ring-0 mean on the axis). */
void or_sample(or_sim *s, int n) {
  const int NR = s->NR, NZ = s->NZ;
  for (int r = 0; r < s->n_rec; r++) {
    if (s->rec_k[r] < s->k_lo || s->rec_k[r] >= s->k_hi) continue; /* another slab's receiver */
    int j0 = s->rec_j[r] < 0 ? 0 : s->rec_j[r], j1 = s->rec_j[r] < 0 ? s->nth : s->rec_j[r] + 1;
    double acc = 0.0;
    for (int j = j0; j < j1; j++) {
      size_t c = IX(j, s->rec_i[r], s->rec_k[r]);
      acc += -(s->f[F_SRR][c] + s->f[F_SPP][c] + s->f[F_SZZ][c]) / 3.0;
    }
    if (n < s->cap) s->traces[(size_t)r * s->cap + n] = acc / (j1 - j0);
  }
}

/* Storage rounding of the fields q0 .. q1-1 with scale sc: the stored
   representation is round(value * sc), the value it stands for that over sc. */
static void round_fields(or_sim *s, int q0, int q1, double sc, int step) {
  if (!s->storage) return;
  set_threads(s);
  const int NR = s->NR, NZ = s->NZ, nth = s->nth;
  for (int q = q0; q < q1; q++) {
    double *f = s->f[q];
    const long long n = (long long)s->ncell;
    if (s->storage == 3) {
#pragma omp parallel for schedule(static)
      for (long long c = 0; c < n; c++) {
        const int k = (int)(c % NZ), i = (int)((c / NZ) % NR), j = (int)(c / ((long long)NZ * NR));
        f[c] = or_round_stochastic_f16(f[c] * sc, or_sr_dither(step, q, j, i, k, nth, NR, NZ)) / sc;
      }
    } else {
#pragma omp parallel for schedule(static)
      for (long long c = 0; c < n; c++) f[c] = or_round_storage(f[c] * sc, s->storage) / sc;
    }
  }
}

/* Select storage rounding: mode 0 none (FP64 fields), 1 BF16, 2 FP16 (round
   to nearest even), 3 FP16 with stochastic rounding, with velocity and
   stress scales sv, ss (> 0).  The present fields are rounded to nearest. */
int or_set_storage(or_sim *s, int mode, double sv, double ss) {
  if (!s || mode < 0 || mode > 3 || !(sv > 0) || !(ss > 0)) return OR_EINVAL;
  s->storage = mode == 3 ? 2 : mode;
  s->st_sv = sv;
  s->st_ss = ss;
  round_fields(s, F_VR, F_SRR, sv, 0);
  round_fields(s, F_SRR, NFIELD, ss, 0);
  s->storage = mode;
  return OR_OK;
}

/* Advance n leapfrog steps: velocity, stress, source, receivers.  With
   storage rounding the fields are rounded where the reduced-precision
   variant stores them: velocities after the velocity half-step (and again
   after a point force), stresses after the stress half-step with the
   volumetric source (and again after the torsion ring). */
int or_step(or_sim *s, int n) {
  if (!s || n < 0) return OR_EINVAL;
  for (int q = 0; q < n; q++) {
    int m = s->steps_done;
    const int force = s->src_kind == 1 || s->src_kind == 2;
    or_velocity_update(s);
    round_fields(s, F_VR, F_SRR, s->st_sv, m);
    if (force) {
      or_inject_source(s, m);
      round_fields(s, F_VR, F_SRR, s->st_sv, m);
    }
    or_stress_update(s);
    if (s->src_kind == 0) or_inject_source(s, m);
    round_fields(s, F_SRR, NFIELD, s->st_ss, m);
    if (s->src_kind == 3) {
      or_inject_source(s, m);
      round_fields(s, F_SRR, NFIELD, s->st_ss, m);
    }
    or_sample(s, m);
    s->steps_done++;
  }
  return OR_OK;
}

/* Restrict the updates, sources and receivers to stored z cells
   k_lo <= k < k_hi (a slab of a z decomposition). */
int or_set_zrange(or_sim *s, int k_lo, int k_hi) {
  if (!s || k_lo < 0 || k_hi > s->NZ || k_lo >= k_hi) return OR_EINVAL;
  s->k_lo = k_lo;
  s->k_hi = k_hi;
  return OR_OK;
}

void or_set_steps_done(or_sim *s, int n) { s->steps_done = n; }

double or_dt(const or_sim *s) { return s->dt; }
int or_steps_done(const or_sim *s) { return s->steps_done; }
double *or_field(or_sim *s, int q) { return (q >= 0 && q < NFIELD) ? s->f[q] : NULL; }
double *or_psi(or_sim *s, int q) { return (q >= 0 && q < NPSI) ? s->psi[q] : NULL; }
const double *or_traces(const or_sim *s) { return s->traces; }
int or_trace_capacity(const or_sim *s) { return s->cap; }
void or_set_threads(or_sim *s, int t) { s->threads = t; }
int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
/* PML tables: 0 a_r(int) 1 b_r(int) 2 a_r(half) 3 b_r(half) 4..7 the same for
   the 1/r group, 8..11 the same in z */
const double *or_pml_table(const or_sim *s, int q) {
  const double *t[12] = {s->ar_i, s->br_i, s->ar_h, s->br_h, s->aq_i, s->bq_i, s->aq_h, s->bq_h,
                         s->az_i, s->bz_i, s->az_h, s->bz_h};
  return (q >= 0 && q < 12) ? t[q] : NULL;
}
