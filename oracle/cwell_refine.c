/*
 * FP64 CPU oracle of the azimuthally refined grid.
 *
 * TEST INFRASTRUCTURE ONLY.  Like cwell_oracle.c, this file is the plain,
 * slow reference the CUDA simulator is checked against; only the test-suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code with the CUDA path.
 *
 * What it computes (paper, Sec. 3, "Azimuth grid refinement"): the grid of
 * cwell_oracle.c with the azimuthal step halved each time the radius doubles.
 * The rows form M radial zones; zone m covers rows [row0[m], row0[m+1]) and
 * has Ntheta_m = nth / 2^(M-1-m) azimuthal nodes, so the outermost zone has
 * the grid's nth.  Inside a zone the scheme is the uniform one of
 * cwell_oracle.c (readings R1-R13, same formulas, same order of operations).
 * Where a stencil reaches across an interface it uses the other zone's row
 * brought to its own azimuthal nodes:
 *
 *  R14 coarse zone A -> fine zone B (the paper's procedure): the coarse row's
 *      trigonometric interpolant at the fine nodes, in three steps: forward
 *      DFT of the Ntheta_A samples; the spectrum padded with zeros to
 *      Ntheta_B coefficients (the Nyquist coefficient split equally between
 *      the frequencies +Ntheta_A/2 and -Ntheta_A/2); inverse DFT.  Fields on
 *      half-integer azimuth nodes (v_phi, s_rphi, s_phiz) sit at
 *      (j + 1/2) dtheta_A on A and (j' + 1/2) dtheta_B on B, which do not
 *      coincide: the padded spectrum is first multiplied by the phase of a
 *      shift of -dtheta_B / 2, i.e. the interpolant is evaluated at the fine
 *      half nodes.  The map is linear; the oracle applies the three steps to
 *      each unit vector once and keeps the resulting matrix P.
 *      Fine zone B -> coarse zone A (the paper does not say): R =
 *      (dtheta_B / dtheta_A) P^T, the adjoint of P in the azimuthal
 *      quadrature of each zone, so that the discrete energy of the uniform
 *      scheme stays exact across the interface (R is the truncation of the
 *      fine spectrum to the coarse one with the two Nyquist terms averaged).
 *      Materials of the coarse row seen from fine node j: coarse cell
 *      floor(j / 2).  Zone m samples the medium given on the finest azimuthal
 *      grid at its own nodes: cell j of zone m is finest cell j 2^(M-1-m).
 *      dt: reading R7 with each row's own azimuthal step.
 *      The radial PML lies in the outermost zone.  Sources: all four kinds,
 *      on the nodes of the zone holding the source row; the transverse
 *      force's v_r node and the torsion ring's s_rphi row must not be the
 *      first row of a zone other than zone 0 (their cells would straddle
 *      the interface).
 *
 * Storage: every field is a ragged array, row i holding Ntheta(i) x NZ
 * values (theta, then z fastest) from offset off[i]; zone m is therefore a
 * contiguous block [rows][Ntheta_m][NZ].
 */
#include <complex.h>
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
enum {
  P_VR_R, P_VP_R, P_VZ_R, P_VR_Z, P_VP_Z, P_VZ_Z,
  P_ERR_R, P_GRP_R, P_GRZ_R, P_EZZ_Z, P_GRZ_Z, P_GPZ_Z,
  P_VR_Q, P_VP_Q, P_VZ_Q, P_EPP_Q, P_GRP_Q, P_GPZ_Q, NPSI
};

double or_ricker(double t, double f0);
void cpml_ab(double d, double al, double dt, double *a, double *b);
double pml_d(double x, double L, double d0);
double pml_dbar(double x, double r, double L, double d0);

/* fields on half-integer azimuth nodes */
static int half_theta(int q) { return q == F_VP || q == F_SRP || q == F_SPZ; }

typedef struct {
  int M, nth, nr, nz, pml_r, pml_z, NR, NZ;
  int *row0;    /* M + 1 */
  int *ntz;     /* Ntheta of each zone */
  int *zone;    /* zone of each row */
  size_t *off;  /* NR + 1 */
  size_t ntot;
  double dr, dz, dt, f0;
  int pml_on;
  uint16_t *id;
  int n_mat;
  double *rho, *lam, *mu;
  double *f[NFIELD];
  double *psi[NPSI];
  double *ar_i, *br_i, *ar_h, *br_h, *aq_i, *bq_i, *aq_h, *bq_h, *az_i, *bz_i, *az_h, *bz_h;
  /* interface m = 1 .. M-1 (between zones m-1 and m): P of each staggering
     [Ntheta_m][Ntheta_{m-1}], the coarse row at fine nodes (up) and the fine
     row at coarse nodes (dn), per field */
  double **P_int, **P_half;
  double **up, **dn; /* [(m * NFIELD) + q] */
  int src_kind, src_n;
  int *src_field;
  size_t *src_cell;
  double *src_w;
  int n_rec, *rec_i, *rec_j, *rec_k;
  int cap, steps_done;
  double *traces;
  int threads;
} ref_sim;

#define RX(i, j, k) (s->off[i] + (size_t)(j) * NZ + (size_t)(k))

/*
 * The paper's three steps on one coarse array a[NA] (R14): forward DFT,
 * zero padding to NB coefficients with the Nyquist coefficient split, phase
 * shift by `shift` fine steps, inverse DFT; the real part goes to b[NB].
 */
static void fft_interp(const double *a, int NA, int NB, double shift, double *b) {
  double complex *c = malloc(NA * sizeof(double complex)), *d = calloc(NB, sizeof(double complex));
  for (int m = 0; m < NA; m++) {
    double complex acc = 0;
    for (int j = 0; j < NA; j++) acc += a[j] * cexp(-2.0 * M_PI * I * (double)m * j / NA);
    c[m] = acc / NA;
  }
  for (int m = 0; m < NA; m++) {
    if (m < NA / 2) d[m] += c[m];
    else if (m > NA / 2) d[NB - (NA - m)] += c[m];
    else {
      d[NA / 2] += 0.5 * c[m];
      d[NB - NA / 2] += 0.5 * c[m];
    }
  }
  const double hB = 2.0 * M_PI / NB;
  for (int m = 0; m < NB; m++) {
    const int fm = m <= NB / 2 ? m : m - NB;
    d[m] *= cexp(I * (double)fm * shift * hB);
  }
  for (int j = 0; j < NB; j++) {
    double complex acc = 0;
    for (int m = 0; m < NB; m++) acc += d[m] * cexp(2.0 * M_PI * I * (double)m * j / NB);
    b[j] = creal(acc);
  }
  free(c);
  free(d);
}

/* matrix of the procedure: column ja = fft_interp(e_ja) */
static double *interp_matrix(int NA, int NB, double shift) {
  double *P = malloc((size_t)NB * NA * sizeof(double)), *e = calloc(NA, sizeof(double)),
         *col = malloc(NB * sizeof(double));
  for (int ja = 0; ja < NA; ja++) {
    memset(e, 0, NA * sizeof(double));
    e[ja] = 1.0;
    fft_interp(e, NA, NB, shift, col);
    for (int jb = 0; jb < NB; jb++) P[(size_t)jb * NA + ja] = col[jb];
  }
  free(e);
  free(col);
  return P;
}

/* exposed for the pins: the coarse-to-fine map of one staggering */
void or_ref_interp(const double *a, int NA, int NB, int half, double *b) {
  fft_interp(a, NA, NB, half ? -0.5 : 0.0, b);
}

void or_ref_destroy(ref_sim *s) {
  if (!s) return;
  free(s->row0); free(s->ntz); free(s->zone); free(s->off);
  free(s->id); free(s->rho); free(s->lam); free(s->mu);
  for (int q = 0; q < NFIELD; q++) free(s->f[q]);
  for (int q = 0; q < NPSI; q++) free(s->psi[q]);
  free(s->ar_i); free(s->br_i); free(s->ar_h); free(s->br_h);
  free(s->aq_i); free(s->bq_i); free(s->aq_h); free(s->bq_h);
  free(s->az_i); free(s->bz_i); free(s->az_h); free(s->bz_h);
  if (s->P_int && s->P_half)
    for (int m = 0; m < s->M; m++) { free(s->P_int[m]); free(s->P_half[m]); }
  free(s->P_int); free(s->P_half);
  if (s->up && s->dn)
    for (int t = 0; t < s->M * NFIELD; t++) { free(s->up[t]); free(s->dn[t]); }
  free(s->up); free(s->dn);
  free(s->src_field); free(s->src_cell); free(s->src_w);
  free(s->rec_i); free(s->rec_j); free(s->rec_k);
  free(s->traces);
  free(s);
}

/* row i of field q at the azimuthal nodes of row `at` (|i - at| <= 1) */
static const double *row_seen(const ref_sim *s, int q, int i, int at) {
  const int zi = s->zone[i], za = s->zone[at];
  if (zi == za) return s->f[q] + s->off[i];
  if (zi < za) return s->up[za * NFIELD + q]; /* coarse row seen from the fine zone */
  return s->dn[zi * NFIELD + q];              /* fine row seen from the coarse zone */
}

/* material ID of cell (i, j, k), j counted on row `at`'s azimuthal nodes */
static int id_seen(const ref_sim *s, int i, int at, int j, int k) {
  const int NZ = s->NZ;
  const int zi = s->zone[i], za = s->zone[at];
  const int jj = zi == za ? j : (zi < za ? j / 2 : 2 * j);
  return s->id[RX(i, jj, k)];
}

static double rho2(const ref_sim *s, int a, int b) { return 0.5 * (s->rho[a] + s->rho[b]); }
static double muh4(const ref_sim *s, int a, int b, int c, int d) {
  double m1 = s->mu[a], m2 = s->mu[b], m3 = s->mu[c], m4 = s->mu[d];
  if (m1 == 0.0 || m2 == 0.0 || m3 == 0.0 || m4 == 0.0) return 0.0;
  return 4.0 / (1.0 / m1 + 1.0 / m2 + 1.0 / m3 + 1.0 / m4);
}

/* interface rows of field q: coarse last row -> fine nodes, fine first row -> coarse nodes */
static void exchange(ref_sim *s, int q) {
  const int NZ = s->NZ;
  for (int m = 1; m < s->M; m++) {
    const int NA = s->ntz[m - 1], NB = s->ntz[m], ib = s->row0[m];
    const double *P = half_theta(q) ? s->P_half[m] : s->P_int[m];
    const double *a = s->f[q] + s->off[ib - 1], *b = s->f[q] + s->off[ib];
    double *up = s->up[m * NFIELD + q], *dn = s->dn[m * NFIELD + q];
    const double w = (double)NA / NB; /* dtheta_B / dtheta_A */
    for (int jb = 0; jb < NB; jb++)
      for (int k = 0; k < NZ; k++) {
        double acc = 0.0;
        for (int ja = 0; ja < NA; ja++) acc += P[(size_t)jb * NA + ja] * a[(size_t)ja * NZ + k];
        up[(size_t)jb * NZ + k] = acc;
      }
    for (int ja = 0; ja < NA; ja++)
      for (int k = 0; k < NZ; k++) {
        double acc = 0.0;
        for (int jb = 0; jb < NB; jb++) acc += w * P[(size_t)jb * NA + ja] * b[(size_t)jb * NZ + k];
        dn[(size_t)ja * NZ + k] = acc;
      }
  }
}

/* Reading R7 per row: dt = cfl * min 1 / (Vp sqrt(1/dr^2 + 1/(r dtheta_row)^2 + 1/dz^2)) */
static double ref_cfl_dt(const ref_sim *s, const double *vp, double cfl) {
  const int NZ = s->NZ;
  double best = INFINITY;
  for (int i = 0; i < s->NR; i++) {
    const int N = s->ntz[s->zone[i]];
    const double dth = 2.0 * M_PI / N, rc = (i + 0.5) * s->dr;
    const double sq = sqrt(1.0 / (s->dr * s->dr) + 1.0 / ((rc * dth) * (rc * dth)) + 1.0 / (s->dz * s->dz));
    for (int j = 0; j < N; j++)
      for (int k = 0; k < NZ; k++) {
        const double c = vp[s->id[RX(i, j, k)]];
        if (c > 0 && 1.0 / (c * sq) < best) best = 1.0 / (c * sq);
      }
  }
  return cfl * best;
}

/*
 * Create.  `row0` holds the M - 1 interface rows (zone m starts at
 * row0[m - 1]); cell_id is given on the finest azimuthal grid [nth][NR][NZ].
 */
ref_sim *or_ref_create(int nr, int nth, int nz, int pml_r, int pml_z, double dr, double dz, int M,
                       const int *row0, int n_mat, const double *rho, const double *vp, const double *vs,
                       const uint16_t *cell_id, double cfl, double dt_override, int pml_on, int src_kind,
                       double src_r, double src_theta, double src_z, double f0, double src_amp, int n_rec,
                       const double *rec_r, const double *rec_theta, const double *rec_z, int max_steps,
                       int *err) {
  *err = OR_EINVAL;
  const int NR = nr + pml_r, NZ = nz + 2 * pml_z;
  if (nr < 1 || nth < 4 || (nth & 1) || nz < 2 || pml_r < 0 || pml_z < 0 || !(dr > 0) || !(dz > 0) || M < 1 ||
      n_mat < 1 || n_rec < 0 || max_steps < 0 || src_kind < 0 || src_kind > 3)
    return NULL;
  if ((nth >> (M - 1)) < 4 || ((nth >> (M - 1)) << (M - 1)) != nth || ((nth >> (M - 1)) & 1)) return NULL;
  for (int m = 0; m + 1 < M; m++) {
    const int lo = m == 0 ? 0 : row0[m - 1];
    if (row0[m] < lo + 2 || row0[m] > nr - 2) return NULL; /* two rows per zone; PML in the last zone */
  }
  if (M > 1 && NR - row0[M - 2] < 2) return NULL;
  ref_sim *s = calloc(1, sizeof(ref_sim));
  if (!s) { *err = OR_ENOMEM; return NULL; }
  s->M = M; s->nth = nth; s->nr = nr; s->nz = nz; s->pml_r = pml_r; s->pml_z = pml_z; s->NR = NR; s->NZ = NZ;
  s->dr = dr; s->dz = dz; s->f0 = f0; s->pml_on = pml_on;
  s->row0 = malloc((M + 1) * sizeof(int));
  s->ntz = malloc(M * sizeof(int));
  s->zone = malloc(NR * sizeof(int));
  s->off = malloc((NR + 1) * sizeof(size_t));
  if (!s->row0 || !s->ntz || !s->zone || !s->off) { or_ref_destroy(s); *err = OR_ENOMEM; return NULL; }
  s->row0[0] = 0;
  for (int m = 1; m < M; m++) s->row0[m] = row0[m - 1];
  s->row0[M] = NR;
  for (int m = 0; m < M; m++) s->ntz[m] = nth >> (M - 1 - m);
  s->off[0] = 0;
  for (int m = 0; m < M; m++)
    for (int i = s->row0[m]; i < s->row0[m + 1]; i++) {
      s->zone[i] = m;
      s->off[i + 1] = s->off[i] + (size_t)s->ntz[m] * NZ;
    }
  s->ntot = s->off[NR];
  s->id = malloc(s->ntot * sizeof(uint16_t));
  s->n_mat = n_mat;
  s->rho = malloc(n_mat * sizeof(double));
  s->lam = malloc(n_mat * sizeof(double));
  s->mu = malloc(n_mat * sizeof(double));
  int ok = s->id && s->rho && s->lam && s->mu;
  for (int q = 0; q < NFIELD; q++) ok = ok && (s->f[q] = calloc(s->ntot, sizeof(double)));
  for (int q = 0; q < NPSI; q++) ok = ok && (s->psi[q] = calloc(s->ntot, sizeof(double)));
  double **tabs[12] = {&s->ar_i, &s->br_i, &s->ar_h, &s->br_h, &s->aq_i, &s->bq_i,
                       &s->aq_h, &s->bq_h, &s->az_i, &s->bz_i, &s->az_h, &s->bz_h};
  for (int t = 0; t < 12; t++) ok = ok && (*tabs[t] = malloc((t < 8 ? NR : NZ) * sizeof(double)));
  s->P_int = calloc(M, sizeof(double *));
  s->P_half = calloc(M, sizeof(double *));
  s->up = calloc((size_t)M * NFIELD, sizeof(double *));
  s->dn = calloc((size_t)M * NFIELD, sizeof(double *));
  ok = ok && s->P_int && s->P_half && s->up && s->dn;
  for (int m = 1; m < M && ok; m++) {
    const int NA = s->ntz[m - 1], NB = s->ntz[m];
    s->P_int[m] = interp_matrix(NA, NB, 0.0);
    s->P_half[m] = interp_matrix(NA, NB, -0.5);
    for (int q = 0; q < NFIELD; q++) {
      s->up[m * NFIELD + q] = calloc((size_t)NB * NZ, sizeof(double));
      s->dn[m * NFIELD + q] = calloc((size_t)NA * NZ, sizeof(double));
      ok = ok && s->up[m * NFIELD + q] && s->dn[m * NFIELD + q];
    }
    ok = ok && s->P_int[m] && s->P_half[m];
  }
  s->n_rec = n_rec;
  s->rec_i = malloc((n_rec + 1) * sizeof(int));
  s->rec_j = malloc((n_rec + 1) * sizeof(int));
  s->rec_k = malloc((n_rec + 1) * sizeof(int));
  s->cap = max_steps;
  s->traces = calloc((size_t)(n_rec + 1) * (max_steps + 1), sizeof(double));
  s->src_field = malloc(2 * nth * sizeof(int));
  s->src_cell = malloc(2 * nth * sizeof(size_t));
  s->src_w = malloc(2 * nth * sizeof(double));
  ok = ok && s->rec_i && s->rec_j && s->rec_k && s->traces && s->src_field && s->src_cell && s->src_w;
  if (!ok) { or_ref_destroy(s); *err = OR_ENOMEM; return NULL; }

  double vpmax = 0.0;
  for (int m = 0; m < n_mat; m++) {
    if (!(rho[m] > 0) || !(vp[m] > 0) || vs[m] < 0 || vp[m] * vp[m] < 2.0 * vs[m] * vs[m]) {
      or_ref_destroy(s); return NULL;
    }
    s->rho[m] = rho[m];
    s->mu[m] = rho[m] * vs[m] * vs[m];
    s->lam[m] = rho[m] * vp[m] * vp[m] - 2.0 * s->mu[m];
    if (vp[m] > vpmax) vpmax = vp[m];
  }
  /* zone m samples the finest grid at its own nodes */
  for (int i = 0; i < NR; i++) {
    const int m = s->zone[i], stride = nth / s->ntz[m];
    for (int j = 0; j < s->ntz[m]; j++)
      for (int k = 0; k < NZ; k++) {
        const uint16_t c = cell_id[((size_t)(j * stride) * NR + i) * NZ + k];
        if (c >= n_mat) { or_ref_destroy(s); return NULL; }
        s->id[RX(i, j, k)] = c;
      }
  }
  for (int j = 0; j < s->ntz[0]; j++) /* R4 */
    for (int k = 0; k < NZ; k++)
      if (s->mu[s->id[RX(0, j, k)]] != 0.0) { or_ref_destroy(s); *err = OR_EUNSUPPORTED; return NULL; }

  s->dt = dt_override > 0 ? dt_override : ref_cfl_dt(s, vp, cfl);

  double Lr = pml_r * dr, Lz = pml_z * dz;
  double d0r = Lr > 0 ? -3.0 * vpmax * log(1e-3) / (2.0 * Lr) : 0.0;
  double d0z = Lz > 0 ? -3.0 * vpmax * log(1e-3) / (2.0 * Lz) : 0.0;
  const double al = M_PI * f0;
  for (int i = 0; i < NR; i++) {
    double xi = pml_on ? (i - nr) * dr : 0.0, xh = pml_on ? (i + 0.5 - nr) * dr : 0.0;
    cpml_ab(pml_d(xi, Lr, d0r), al, s->dt, &s->ar_i[i], &s->br_i[i]);
    cpml_ab(pml_d(xh, Lr, d0r), al, s->dt, &s->ar_h[i], &s->br_h[i]);
    cpml_ab(pml_dbar(xi, i * dr, Lr, d0r), al, s->dt, &s->aq_i[i], &s->bq_i[i]);
    cpml_ab(pml_dbar(xh, (i + 0.5) * dr, Lr, d0r), al, s->dt, &s->aq_h[i], &s->bq_h[i]);
  }
  for (int k = 0; k < NZ; k++) {
    double lo_i = (pml_z - 0.5 - k) * dz, hi_i = (k - (pml_z + nz - 0.5)) * dz;
    double lo_h = (pml_z - 1.0 - k) * dz, hi_h = (k + 1.0 - pml_z - nz) * dz;
    double xi = pml_on ? fmax(lo_i, hi_i) : 0.0, xh = pml_on ? fmax(lo_h, hi_h) : 0.0;
    cpml_ab(pml_d(xi, Lz, d0z), al, s->dt, &s->az_i[k], &s->bz_i[k]);
    cpml_ab(pml_d(xh, Lz, d0z), al, s->dt, &s->az_h[k], &s->bz_h[k]);
  }

  /* R6, R12 injection points, on the azimuthal nodes of the source's zone */
  s->src_kind = src_kind;
  {
    const int k = (int)lround(src_z / dz) + pml_z;
    if (k < pml_z || k >= pml_z + nz || src_r < 0 || src_r >= nr * dr) { or_ref_destroy(s); return NULL; }
    const int axis = src_r < dr;
    int n = 0, bad = 0;
    if (src_kind == 0) {
      if (axis) {
        for (int j = 0; j < s->ntz[0]; j++) {
          s->src_field[n] = F_SRR; s->src_cell[n] = RX(0, j, k); s->src_w[n++] = src_amp / (M_PI * dr * dr * dz);
        }
      } else {
        const int i = (int)floor(src_r / dr), N = s->ntz[s->zone[i]];
        const double dth = 2.0 * M_PI / N;
        const int js = (int)(((long)lround(src_theta / dth) % N + N) % N);
        s->src_field[n] = F_SRR; s->src_cell[n] = RX(i, js, k);
        s->src_w[n++] = src_amp / ((i + 0.5) * dr * dr * dth * dz);
      }
    } else if (src_kind == 2) { /* longitudinal force, R12: v_z nodes, cells of one row */
      if (k + 1 >= NZ) bad = 1;
      else if (axis) {
        for (int j = 0; j < s->ntz[0]; j++) {
          s->src_field[n] = F_VZ; s->src_cell[n] = RX(0, j, k);
          s->src_w[n++] = src_amp / (rho2(s, s->id[RX(0, j, k)], s->id[RX(0, j, k + 1)]) * M_PI * dr * dr * dz);
        }
      } else {
        const int i = (int)floor(src_r / dr), N = s->ntz[s->zone[i]];
        const double dth = 2.0 * M_PI / N;
        const int js = (int)(((long)lround(src_theta / dth) % N + N) % N);
        s->src_field[n] = F_VZ; s->src_cell[n] = RX(i, js, k);
        s->src_w[n++] = src_amp / (rho2(s, s->id[RX(i, js, k)], s->id[RX(i, js, k + 1)]) * (i + 0.5) * dr * dr * dth * dz);
      }
    } else if (src_kind == 3) { /* torsion ring, R13, on every node of its zone */
      const int i = (int)lround(src_r / dr), ih = (int)floor(src_r / dr);
      if (axis || i < 1 || i >= NR || ih + 1 > NR || k + 1 >= NZ || s->zone[i - 1] != s->zone[i]) bad = 1;
      const int N = bad ? 0 : s->ntz[s->zone[i]];
      for (int j = 0; j < N && !bad; j++) {
        const int jp = (j + 1) % N;
        if (muh4(s, s->id[RX(i - 1, j, k)], s->id[RX(i, j, k)], s->id[RX(i - 1, jp, k)], s->id[RX(i, jp, k)]) == 0.0 ||
            muh4(s, s->id[RX(ih, j, k)], s->id[RX(ih, jp, k)], s->id[RX(ih, j, k + 1)], s->id[RX(ih, jp, k + 1)]) == 0.0) {
          bad = 1;
          break;
        }
        s->src_field[n] = F_SRP; s->src_cell[n] = RX(i, j, k);
        s->src_w[n++] = src_amp / (2.0 * M_PI * i * dr * dr * dz);
        s->src_field[n] = F_SPZ; s->src_cell[n] = RX(ih, j, k);
        s->src_w[n++] = src_amp / (2.0 * M_PI * (ih + 0.5) * dr * dr * dz);
      }
    } else {
      if (axis) {
        const int N = s->ntz[0];
        const double dth = 2.0 * M_PI / N;
        if (s->zone[1] != 0) bad = 1;
        for (int j = 0; j < N && !bad; j++) {
          const double w = 2.0 * cos(j * dth - src_theta) / N;
          s->src_field[n] = F_VR; s->src_cell[n] = RX(1, j, k);
          s->src_w[n++] = src_amp * w / (rho2(s, s->id[RX(0, j, k)], s->id[RX(1, j, k)]) * dr * dr * dth * dz);
        }
      } else {
        const int i = (int)lround(src_r / dr);
        if (i < 1 || i >= NR || s->zone[i - 1] != s->zone[i]) bad = 1;
        else {
          const int N = s->ntz[s->zone[i]];
          const double dth = 2.0 * M_PI / N;
          const int js = (int)(((long)lround(src_theta / dth) % N + N) % N);
          s->src_field[n] = F_VR; s->src_cell[n] = RX(i, js, k);
          s->src_w[n++] = src_amp / (rho2(s, s->id[RX(i - 1, js, k)], s->id[RX(i, js, k)]) * i * dr * dr * dth * dz);
        }
      }
    }
    if (bad) { or_ref_destroy(s); *err = OR_EUNSUPPORTED; return NULL; }
    s->src_n = n;
  }
  for (int q = 0; q < n_rec; q++) {
    s->rec_k[q] = (int)lround(rec_z[q] / dz) + pml_z;
    if (s->rec_k[q] < pml_z || s->rec_k[q] >= pml_z + nz || rec_r[q] < 0 || rec_r[q] >= nr * dr) {
      or_ref_destroy(s); return NULL;
    }
    if (rec_r[q] < dr) {
      s->rec_i[q] = 0; s->rec_j[q] = -1;
    } else {
      const int i = (int)floor(rec_r[q] / dr), N = s->ntz[s->zone[i]];
      s->rec_i[q] = i;
      s->rec_j[q] = (int)(((long)lround(rec_theta[q] / (2.0 * M_PI / N)) % N + N) % N);
    }
  }
  *err = OR_OK;
  return s;
}

static inline double stretch(int on, double *psi, double a, double b, double D) {
  if (!on) return D;
  *psi = b * (*psi) + a * D;
  return D + *psi;
}

static void set_threads(const ref_sim *s) {
#ifdef _OPENMP
  if (s->threads > 0) omp_set_num_threads(s->threads);
#else
  (void)s;
#endif
}

/* Velocity half-step, the formulas of cwell_oracle.c row by row on each row's own nodes. */
void or_ref_velocity_update(ref_sim *s) {
  exchange(s, F_SRR);
  exchange(s, F_SPP);
  exchange(s, F_SRP);
  exchange(s, F_SRZ);
  const int NR = s->NR, NZ = s->NZ, on = s->pml_on;
  const double dr = s->dr, dz = s->dz, dt = s->dt;
  set_threads(s);
#pragma omp parallel for schedule(dynamic)
  for (int i = 0; i < NR; i++) {
    const int N = s->ntz[s->zone[i]];
    const double dth = 2.0 * M_PI / N, ri = i * dr, rh = (i + 0.5) * dr;
    const size_t o = s->off[i];
    const double *srr = s->f[F_SRR] + o, *spp = s->f[F_SPP] + o, *szz = s->f[F_SZZ] + o;
    const double *srp = s->f[F_SRP] + o, *spz = s->f[F_SPZ] + o, *srz = s->f[F_SRZ] + o;
    double *vr = s->f[F_VR] + o, *vp = s->f[F_VP] + o, *vz = s->f[F_VZ] + o;
    const double *srr_m = i >= 1 ? row_seen(s, F_SRR, i - 1, i) : NULL;
    const double *spp_m = i >= 1 ? row_seen(s, F_SPP, i - 1, i) : NULL;
    const double *srp_p = i + 1 < NR ? row_seen(s, F_SRP, i + 1, i) : NULL;
    const double *srz_p = i + 1 < NR ? row_seen(s, F_SRZ, i + 1, i) : NULL;
    for (int j = 0; j < N; j++) {
      const int jm = (j + N - 1) % N, jp = (j + 1) % N;
      for (int k = 0; k < NZ; k++) {
        const size_t c = (size_t)j * NZ + k, g = o + c;
        const int idc = s->id[g];
        if (i >= 1) {
          double Dr = (srr[c] - srr_m[c]) / dr;
          double Q = (0.5 * (srr[c] + srr_m[c]) - 0.5 * (spp[c] + spp_m[c]) + (srp[c] - srp[(size_t)jm * NZ + k]) / dth) / ri;
          double Dz = (srz[c] - (k > 0 ? srz[c - 1] : 0.0)) / dz;
          Dr = stretch(on, &s->psi[P_VR_R][g], s->ar_i[i], s->br_i[i], Dr);
          Q = stretch(on, &s->psi[P_VR_Q][g], s->aq_i[i], s->bq_i[i], Q);
          Dz = stretch(on, &s->psi[P_VR_Z][g], s->az_i[k], s->bz_i[k], Dz);
          vr[c] += dt / rho2(s, id_seen(s, i - 1, i, j, k), idc) * (Dr + Q + Dz);
        }
        {
          double s1 = srp_p ? srp_p[c] : 0.0, s0 = srp[c];
          double Dr = (s1 - s0) / dr;
          double Q = ((s1 + s0) + (spp[(size_t)jp * NZ + k] - spp[c]) / dth) / rh;
          double Dz = (spz[c] - (k > 0 ? spz[c - 1] : 0.0)) / dz;
          Dr = stretch(on, &s->psi[P_VP_R][g], s->ar_h[i], s->br_h[i], Dr);
          Q = stretch(on, &s->psi[P_VP_Q][g], s->aq_h[i], s->bq_h[i], Q);
          Dz = stretch(on, &s->psi[P_VP_Z][g], s->az_i[k], s->bz_i[k], Dz);
          vp[c] += dt / rho2(s, idc, s->id[o + (size_t)jp * NZ + k]) * (Dr + Q + Dz);
        }
        if (k + 1 < NZ) {
          double s1 = srz_p ? srz_p[c] : 0.0, s0 = srz[c];
          double Dr = (s1 - s0) / dr;
          double Q = (0.5 * (s1 + s0) + (spz[c] - spz[(size_t)jm * NZ + k]) / dth) / rh;
          double Dz = (szz[c + 1] - szz[c]) / dz;
          Dr = stretch(on, &s->psi[P_VZ_R][g], s->ar_h[i], s->br_h[i], Dr);
          Q = stretch(on, &s->psi[P_VZ_Q][g], s->aq_h[i], s->bq_h[i], Q);
          Dz = stretch(on, &s->psi[P_VZ_Z][g], s->az_h[k], s->bz_h[k], Dz);
          vz[c] += dt / rho2(s, idc, s->id[g + 1]) * (Dr + Q + Dz);
        }
      }
    }
  }
}

/* Stress step, the formulas of cwell_oracle.c row by row on each row's own nodes. */
void or_ref_stress_update(ref_sim *s) {
  exchange(s, F_VR);
  exchange(s, F_VP);
  exchange(s, F_VZ);
  const int NR = s->NR, NZ = s->NZ, on = s->pml_on;
  const double dr = s->dr, dz = s->dz, dt = s->dt;
  set_threads(s);
#pragma omp parallel for schedule(dynamic)
  for (int i = 0; i < NR; i++) {
    const int N = s->ntz[s->zone[i]];
    const double dth = 2.0 * M_PI / N, ri = i * dr, rh = (i + 0.5) * dr;
    const size_t o = s->off[i];
    const double *vr = s->f[F_VR] + o, *vp = s->f[F_VP] + o, *vz = s->f[F_VZ] + o;
    double *srr = s->f[F_SRR] + o, *spp = s->f[F_SPP] + o, *szz = s->f[F_SZZ] + o;
    double *srp = s->f[F_SRP] + o, *spz = s->f[F_SPZ] + o, *srz = s->f[F_SRZ] + o;
    const double *vr_p = i + 1 < NR ? row_seen(s, F_VR, i + 1, i) : NULL;
    const double *vp_m = i >= 1 ? row_seen(s, F_VP, i - 1, i) : NULL;
    const double *vz_m = i >= 1 ? row_seen(s, F_VZ, i - 1, i) : NULL;
    for (int j = 0; j < N; j++) {
      const int jm = (j + N - 1) % N, jp = (j + 1) % N;
      for (int k = 0; k < NZ; k++) {
        const size_t c = (size_t)j * NZ + k, g = o + c;
        const int idc = s->id[g];
        {
          double vr0 = (i >= 1) ? vr[c] : 0.0;
          double vr1 = vr_p ? vr_p[c] : 0.0;
          double err = (vr1 - vr0) / dr;
          double epp = ((vp[c] - vp[(size_t)jm * NZ + k]) / dth + 0.5 * (vr0 + vr1)) / rh;
          double ezz = (vz[c] - (k > 0 ? vz[c - 1] : 0.0)) / dz;
          err = stretch(on, &s->psi[P_ERR_R][g], s->ar_h[i], s->br_h[i], err);
          epp = stretch(on, &s->psi[P_EPP_Q][g], s->aq_h[i], s->bq_h[i], epp);
          ezz = stretch(on, &s->psi[P_EZZ_Z][g], s->az_i[k], s->bz_i[k], ezz);
          const double l = s->lam[idc], m = s->mu[idc];
          srr[c] += dt * ((l + 2.0 * m) * err + l * (epp + ezz));
          spp[c] += dt * ((l + 2.0 * m) * epp + l * (err + ezz));
          szz[c] += dt * ((l + 2.0 * m) * ezz + l * (err + epp));
        }
        if (i >= 1) {
          double gr = (vp[c] - vp_m[c]) / dr;
          double Q = ((vr[(size_t)jp * NZ + k] - vr[c]) / dth - 0.5 * (vp[c] + vp_m[c])) / ri;
          gr = stretch(on, &s->psi[P_GRP_R][g], s->ar_i[i], s->br_i[i], gr);
          Q = stretch(on, &s->psi[P_GRP_Q][g], s->aq_i[i], s->bq_i[i], Q);
          double m = muh4(s, id_seen(s, i - 1, i, j, k), idc, id_seen(s, i - 1, i, jp, k), s->id[o + (size_t)jp * NZ + k]);
          srp[c] += dt * m * (gr + Q);
        }
        if (k + 1 < NZ) {
          if (i >= 1) {
            double gz = (vr[c + 1] - vr[c]) / dz;
            double gr = (vz[c] - vz_m[c]) / dr;
            gz = stretch(on, &s->psi[P_GRZ_Z][g], s->az_h[k], s->bz_h[k], gz);
            gr = stretch(on, &s->psi[P_GRZ_R][g], s->ar_i[i], s->br_i[i], gr);
            double m = muh4(s, id_seen(s, i - 1, i, j, k), idc, id_seen(s, i - 1, i, j, k + 1), s->id[g + 1]);
            srz[c] += dt * m * (gz + gr);
          }
          {
            double Q = (vz[(size_t)jp * NZ + k] - vz[c]) / (rh * dth);
            double gz = (vp[c + 1] - vp[c]) / dz;
            Q = stretch(on, &s->psi[P_GPZ_Q][g], s->aq_h[i], s->bq_h[i], Q);
            gz = stretch(on, &s->psi[P_GPZ_Z][g], s->az_h[k], s->bz_h[k], gz);
            double m = muh4(s, idc, s->id[o + (size_t)jp * NZ + k], s->id[g + 1], s->id[o + (size_t)jp * NZ + k + 1]);
            spz[c] += dt * m * (Q + gz);
          }
        }
      }
    }
  }
}

void or_ref_inject_source(ref_sim *s, int n) {
  const int force = s->src_kind == 1 || s->src_kind == 2;
  const double f = or_ricker((force ? n : n + 0.5) * s->dt, s->f0);
  for (int q = 0; q < s->src_n; q++) {
    const double add = s->dt * s->src_w[q] * f;
    const size_t c = s->src_cell[q];
    if (s->src_kind == 0) {
      s->f[F_SRR][c] += add;
      s->f[F_SPP][c] += add;
      s->f[F_SZZ][c] += add;
    } else {
      s->f[s->src_field[q]][c] += add;
    }
  }
}

void or_ref_sample(ref_sim *s, int n) {
  const int NZ = s->NZ;
  for (int r = 0; r < s->n_rec; r++) {
    const int i = s->rec_i[r], N = s->ntz[s->zone[i]];
    const int j0 = s->rec_j[r] < 0 ? 0 : s->rec_j[r], j1 = s->rec_j[r] < 0 ? N : s->rec_j[r] + 1;
    double acc = 0.0;
    for (int j = j0; j < j1; j++) {
      const size_t c = RX(i, j, s->rec_k[r]);
      acc += -(s->f[F_SRR][c] + s->f[F_SPP][c] + s->f[F_SZZ][c]) / 3.0;
    }
    if (n < s->cap) s->traces[(size_t)r * s->cap + n] = acc / (j1 - j0);
  }
}

int or_ref_step(ref_sim *s, int n) {
  if (!s || n < 0) return OR_EINVAL;
  for (int q = 0; q < n; q++) {
    const int m = s->steps_done, force = s->src_kind == 1 || s->src_kind == 2;
    or_ref_velocity_update(s);
    if (force) or_ref_inject_source(s, m);
    or_ref_stress_update(s);
    if (!force) or_ref_inject_source(s, m);
    or_ref_sample(s, m);
    s->steps_done++;
  }
  return OR_OK;
}

double or_ref_dt(const ref_sim *s) { return s->dt; }
int or_ref_steps_done(const ref_sim *s) { return s->steps_done; }
double *or_ref_field(ref_sim *s, int q) { return (q >= 0 && q < NFIELD) ? s->f[q] : NULL; }
const double *or_ref_traces(const ref_sim *s) { return s->traces; }
void or_ref_set_threads(ref_sim *s, int t) { s->threads = t; }
/* zone m: first row, rows, Ntheta, element offset of its block */
void or_ref_zone(const ref_sim *s, int m, int *row, int *rows, int *nth, long long *off) {
  *row = s->row0[m];
  *rows = s->row0[m + 1] - s->row0[m];
  *nth = s->ntz[m];
  *off = (long long)s->off[s->row0[m]];
}
/* interface matrix of interface m (1 .. M-1), staggering half: [Ntheta_m][Ntheta_{m-1}] */
const double *or_ref_matrix(const ref_sim *s, int m, int half) {
  if (m < 1 || m >= s->M) return NULL;
  return half ? s->P_half[m] : s->P_int[m];
}
