/*
 * irs_oracle.c -- plain, slow, FP64 CPU oracle for inverse ray-shooting.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * What it computes (Zheng, Chen, Li & Chen, "An Improved GPU-Based
 * Ray-Shooting Code For Gravitational Microlensing", arXiv:2204.10871):
 *
 *   sizing ...................... flow chart, "Protective Border" and level-3
 *                                 resolution (Sec. 2.4 item list)
 *   rectangular negative sheet .. Appendix A, the two closed-form integrals
 *   deflection, rectangular plane Eq. (alpha1) = Eq. 6 with the sheet above
 *   deflection, circular plane .. Eq. (alpha) = Eq. 4
 *   lens equation ............... beta = theta - alpha(theta)  (Eq. 3)
 *   binning + magnification ..... "Calculate the magnification of each pixel",
 *                                 Mag_ij = N_ij * S_I / S_S
 *
 * Every ray is summed over ALL lenses (brute force), with Neumaier-compensated
 * FP64 sums so that the oracle's own rounding is far below the tolerances it
 * judges.  Threads split the ray lattice by rows; each thread owns a private
 * count map, merged at the end (integer adds, order-independent).
 *
 * Readings of points the paper leaves open are numbered R1.. and listed in
 * the design notes; the ones used here:
 *   R1  the appendix integral is the deflection of a POSITIVE sheet, so the
 *       negative sheet of Eq. (alpha1) is its negation;
 *   R2  the matrix term uses kappa = kappa_s + kappa_*^act and the sheet uses
 *       kappa_*^act = pi * sum(m) / area, the density of the lenses actually
 *       passed in (declared kappa_* only sizes the plane);
 *   R3  Delta x3 = sqrt(s_x s_y / N_av) with N_av the rays per UNLENSED source
 *       pixel; the ray count per axis is ceil(I / Delta x3) and the plane is
 *       widened to that whole number of rays;
 *   R6  rays sit at cell centres (i + 1/2) Delta x3; the rectangle is centred
 *       on the image of the source-region centre under the mean lens map;
 *   R7  pixel = floor((beta - lo) / s) per axis, kept if inside [0, npix);
 *   R8  a lens exactly on a ray (r^2 == 0) contributes nothing;
 *   circle plane: alpha = diag(k_s+g, k_s-g) theta + k_*^act theta_c + sum,
 *       i.e. Eq. (alpha1) with the circular sheet -k_*(theta - theta_c) of
 *       Eq. (alphapart) centred on the plane centre theta_c, and
 *       kappa_*^act = sum(m) / R_c^2 for the circumscribed circle R_c.
 *
 * Parity pins (tests marked "not gpu"): 2-D quadrature of the sheet, the
 * sheet's divergence and far-field limit, Paczynski's point-lens
 * magnification, the lens-free sheet's exact lattice counts, ray
 * conservation, the mean magnification, and the paper's printed lens count.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PLANE_RECT 0
#define OR_PLANE_CIRCLE 1

typedef struct {
  double kappa_star, kappa_s, gamma;
  double src_x0, src_x1, src_y0, src_y1;
  int32_t npix_x, npix_y;
  double rays_per_pixel;
  double border; /* < 0: the paper's rule P = 10 sqrt(kappa_*) */
  int32_t plane;
  int32_t pad_;
} or_params;

typedef struct {
  double kappa;             /* kappa_s + declared kappa_* */
  double border;            /* P */
  double lambda1, lambda2;  /* 1 - kappa - gamma, 1 - kappa + gamma */
  double ix0, iy0;          /* paper I_xscale, I_yscale */
  double sx, sy;            /* source pixel sides */
  double dx3;               /* ray spacing (level-3 resolution) */
  double ix, iy;            /* plane sides after widening to whole rays */
  double cx, cy;            /* plane centre */
  double a1, a2, b1, b2;    /* plane rectangle */
  int64_t nrx, nry, n_rays; /* ray lattice */
  double circle_r;          /* circumscribed circle radius */
  double n_star_paper;      /* kappa_* * area / pi, mean mass 1 */
} or_plan;

/* --- sizing: flow-chart items "Input parameters", "Protective Border",
 *     level-3 resolution (with reading R3) ------------------------------- */
int or_size(const or_params* p, or_plan* q) {
  memset(q, 0, sizeof(*q));
  if (!(p->npix_x > 0 && p->npix_y > 0)) return 1;
  if (!(p->rays_per_pixel > 0)) return 1;
  if (!(p->src_x1 > p->src_x0 && p->src_y1 > p->src_y0)) return 1;
  if (!(p->kappa_star >= 0 && p->kappa_s >= 0)) return 1;
  q->kappa = p->kappa_s + p->kappa_star;
  q->border = p->border < 0 ? 10.0 * sqrt(p->kappa_star) : p->border;
  q->lambda1 = 1.0 - q->kappa - p->gamma;
  q->lambda2 = 1.0 - q->kappa + p->gamma;
  if (fabs(q->lambda1) < 1e-6 || fabs(q->lambda2) < 1e-6) return 2;
  double S_x = p->src_x1 - p->src_x0, S_y = p->src_y1 - p->src_y0;
  q->ix0 = (S_x + 2.0 * q->border) / fabs(q->lambda1);
  q->iy0 = (S_y + 2.0 * q->border) / fabs(q->lambda2);
  q->sx = S_x / p->npix_x;
  q->sy = S_y / p->npix_y;
  q->dx3 = sqrt(q->sx * q->sy / p->rays_per_pixel);
  q->nrx = (int64_t)ceil(q->ix0 / q->dx3 - 1e-9);
  q->nry = (int64_t)ceil(q->iy0 / q->dx3 - 1e-9);
  if (q->nrx < 1) q->nrx = 1;
  if (q->nry < 1) q->nry = 1;
  q->n_rays = q->nrx * q->nry;
  q->ix = (double)q->nrx * q->dx3;
  q->iy = (double)q->nry * q->dx3;
  q->cx = 0.5 * (p->src_x0 + p->src_x1) / q->lambda1;
  q->cy = 0.5 * (p->src_y0 + p->src_y1) / q->lambda2;
  q->a1 = q->cx - 0.5 * q->ix;
  q->a2 = q->cx + 0.5 * q->ix;
  q->b1 = q->cy - 0.5 * q->iy;
  q->b2 = q->cy + 0.5 * q->iy;
  q->circle_r = 0.5 * sqrt(q->ix * q->ix + q->iy * q->iy);
  if (p->plane == OR_PLANE_CIRCLE)
    q->n_star_paper = p->kappa_star * q->circle_r * q->circle_r;
  else
    q->n_star_paper = p->kappa_star * q->ix * q->iy / M_PI;
  return 0;
}

/* x * atan(y / x), continued by its limit 0 at x == 0 (the appendix terms
 * (theta1 - a) * arctan(...) vanish there). */
static double x_atan_ratio(double x, double y) {
  if (x == 0.0) return 0.0;
  return x * atan(y / x);
}

/* y * ln(num / den), continued by 0 where the prefactor vanishes. */
static double y_log_ratio(double y, double num, double den) {
  if (y == 0.0) return 0.0;
  return y * log(num / den);
}

/* --- Appendix A: deflection of a uniform POSITIVE sheet of density
 *     kappa over [a1,a2] x [b1,b2], A = kappa / pi, written out term by term
 *     as the appendix prints alpha_1 and alpha_2.  Reading R1: the negative
 *     sheet of Eq. (alpha1) is minus this. ------------------------------- */
void or_sheet_positive(double a1, double a2, double b1, double b2, double kappa,
                       double t1, double t2, double* out1, double* out2) {
  const double A = kappa / M_PI;
  const double u2 = t1 - a2, u1 = t1 - a1; /* theta_1 - a_2, theta_1 - a_1 */
  const double v2 = t2 - b2, v1 = t2 - b1; /* theta_2 - b_2, theta_2 - b_1 */
  const double r22 = u2 * u2 + v2 * v2;   /* corner (a2, b2) */
  const double r12 = u1 * u1 + v2 * v2;   /* corner (a1, b2) */
  const double r21 = u2 * u2 + v1 * v1;   /* corner (a2, b1) */
  const double r11 = u1 * u1 + v1 * v1;   /* corner (a1, b1) */
  /* alpha_1: two log terms in theta_2 - b, four arctan terms */
  double s1 = 0.5 * y_log_ratio(v2, r22, r12) - 0.5 * y_log_ratio(v1, r21, r11);
  s1 += x_atan_ratio(u2, v2) - x_atan_ratio(u2, v1);
  s1 += x_atan_ratio(u1, v1) - x_atan_ratio(u1, v2);
  /* alpha_2: two log terms in theta_1 - a, four arctan terms */
  double s2 = 0.5 * y_log_ratio(u2, r22, r21) - 0.5 * y_log_ratio(u1, r12, r11);
  s2 += x_atan_ratio(v2, u2) - x_atan_ratio(v2, u1);
  s2 += x_atan_ratio(v1, u1) - x_atan_ratio(v1, u2);
  *out1 = A * s1;
  *out2 = A * s2;
}

/* Neumaier (improved Kahan) accumulator. */
typedef struct { double s, c; } nsum;
static inline void nsum_add(nsum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x))
    a->c += (a->s - t) + x;
  else
    a->c += (x - t) + a->s;
  a->s = t;
}
static inline double nsum_get(const nsum* a) { return a->s + a->c; }

/* kappa_*^act (reading R2): density of the lenses actually passed in. */
double or_kappa_star_actual(const or_params* p, const or_plan* q, const double* mass, int64_t n) {
  nsum m = {0, 0};
  for (int64_t i = 0; i < n; ++i) nsum_add(&m, mass[i]);
  double M = nsum_get(&m);
  if (p->plane == OR_PLANE_CIRCLE) return M / (q->circle_r * q->circle_r);
  return M_PI * M / (q->ix * q->iy);
}

/* --- Eq. (alpha1) for the rectangular plane, Eq. (alpha) for the circular
 *     one.  xy holds lens positions interleaved (x0, y0, x1, y1, ...). ---- */
void or_deflection(const or_params* p, const or_plan* q, const double* xy, const double* mass,
                   int64_t n, double kstar_act, double t1, double t2, double* al1, double* al2) {
  nsum s1 = {0, 0}, s2 = {0, 0};
  for (int64_t i = 0; i < n; ++i) {
    double d1 = t1 - xy[2 * i], d2 = t2 - xy[2 * i + 1];
    double r2 = d1 * d1 + d2 * d2;
    if (r2 == 0.0) continue; /* reading R8 */
    nsum_add(&s1, mass[i] * d1 / r2);
    nsum_add(&s2, mass[i] * d2 / r2);
  }
  if (p->plane == OR_PLANE_CIRCLE) {
    /* Eq. (alpha): diag(k_s + g, k_s - g) theta + sum, plus k_* theta_c for
     * a plane not centred on the origin */
    nsum_add(&s1, (p->kappa_s + p->gamma) * t1);
    nsum_add(&s2, (p->kappa_s - p->gamma) * t2);
    nsum_add(&s1, kstar_act * q->cx);
    nsum_add(&s2, kstar_act * q->cy);
  } else {
    /* Eq. (alpha1): diag(k + g, k - g) theta + sum + alpha_{-k_*} */
    double kap = p->kappa_s + kstar_act;
    double sh1, sh2;
    or_sheet_positive(q->a1, q->a2, q->b1, q->b2, kstar_act, t1, t2, &sh1, &sh2);
    nsum_add(&s1, (kap + p->gamma) * t1);
    nsum_add(&s2, (kap - p->gamma) * t2);
    nsum_add(&s1, -sh1);
    nsum_add(&s2, -sh2);
  }
  *al1 = nsum_get(&s1);
  *al2 = nsum_get(&s2);
}

/* ray (i, j) of the lattice, reading R6 */
static inline void ray_pos(const or_plan* q, int64_t i, int64_t j, double* t1, double* t2) {
  *t1 = q->a1 + ((double)i + 0.5) * q->dx3;
  *t2 = q->b1 + ((double)j + 0.5) * q->dx3;
}

/* pixel of a source position, reading R7; returns -1 when outside */
static inline int64_t pixel_of(const or_params* p, const or_plan* q, double b1, double b2) {
  double fx = floor((b1 - p->src_x0) / q->sx);
  double fy = floor((b2 - p->src_y0) / q->sy);
  if (!(fx >= 0 && fx < p->npix_x && fy >= 0 && fy < p->npix_y)) return -1;
  return (int64_t)fy * p->npix_x + (int64_t)fx;
}

/* Per-ray lens equation for a list of flat ray indices (idx = j * nrx + i):
 * writes alpha and beta (2 doubles each) and the pixel index (or -1). */
void or_shoot_rays(const or_params* p, const or_plan* q, const double* xy, const double* mass,
                   int64_t n, double kstar_act, const int64_t* idx, int64_t nidx, double* alpha,
                   double* beta, int64_t* pixel) {
  for (int64_t k = 0; k < nidx; ++k) {
    int64_t i = idx[k] % q->nrx, j = idx[k] / q->nrx;
    double t1, t2, a1, a2;
    ray_pos(q, i, j, &t1, &t2);
    or_deflection(p, q, xy, mass, n, kstar_act, t1, t2, &a1, &a2);
    double b1 = t1 - a1, b2 = t2 - a2; /* Eq. (3) */
    if (alpha) { alpha[2 * k] = a1; alpha[2 * k + 1] = a2; }
    if (beta) { beta[2 * k] = b1; beta[2 * k + 1] = b2; }
    if (pixel) pixel[k] = pixel_of(p, q, b1, b2);
  }
}

typedef struct {
  const or_params* p;
  const or_plan* q;
  const double* xy;
  const double* mass;
  int64_t n;
  double kstar;
  int64_t row0, row1; /* rows [row0, row1) of the lattice */
  int64_t col0, col1; /* columns [col0, col1) */
  uint32_t* counts;   /* private map */
  int64_t landed;
} or_job;

static void* map_worker(void* arg) {
  or_job* J = (or_job*)arg;
  const or_plan* q = J->q;
  for (int64_t j = J->row0; j < J->row1; ++j)
    for (int64_t i = J->col0; i < J->col1; ++i) {
      double t1, t2, a1, a2;
      ray_pos(q, i, j, &t1, &t2);
      or_deflection(J->p, q, J->xy, J->mass, J->n, J->kstar, t1, t2, &a1, &a2);
      int64_t pix = pixel_of(J->p, q, t1 - a1, t2 - a2);
      if (pix >= 0) { J->counts[pix] += 1u; J->landed += 1; }
    }
  return NULL;
}

/* Count map over the rays with rows in [row0, row1) and columns in
 * [col0, col1) of the lattice (the full map: 0, nry, 0, nrx).  counts must
 * hold npix_x * npix_y zeros on entry; mag (may be NULL) receives
 * Mag_ij = N_ij * S_I / S_S.  Returns the number of rays that landed. */
int64_t or_make_map(const or_params* p, const or_plan* q, const double* xy, const double* mass,
                    int64_t n, int64_t row0, int64_t row1, int64_t col0, int64_t col1,
                    int nthreads, uint32_t* counts, double* mag) {
  const int64_t npix = (int64_t)p->npix_x * p->npix_y;
  double kstar = or_kappa_star_actual(p, q, mass, n);
  if (nthreads < 1) nthreads = 1;
  int64_t rows = row1 - row0;
  if (rows < nthreads) nthreads = rows > 0 ? (int)rows : 1;
  or_job* jobs = (or_job*)calloc((size_t)nthreads, sizeof(or_job));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].p = p; jobs[t].q = q; jobs[t].xy = xy; jobs[t].mass = mass; jobs[t].n = n;
    jobs[t].kstar = kstar;
    jobs[t].row0 = row0 + rows * t / nthreads;
    jobs[t].row1 = row0 + rows * (t + 1) / nthreads;
    jobs[t].col0 = col0; jobs[t].col1 = col1;
    jobs[t].counts = (uint32_t*)calloc((size_t)npix, sizeof(uint32_t));
    pthread_create(&th[t], NULL, map_worker, &jobs[t]);
  }
  int64_t landed = 0;
  for (int t = 0; t < nthreads; ++t) {
    pthread_join(th[t], NULL);
    for (int64_t k = 0; k < npix; ++k) counts[k] += jobs[t].counts[k];
    landed += jobs[t].landed;
    free(jobs[t].counts);
  }
  free(jobs);
  free(th);
  if (mag) {
    const double ratio = q->dx3 * q->dx3 / (q->sx * q->sy); /* S_I / S_S */
    for (int64_t k = 0; k < npix; ++k) mag[k] = (double)counts[k] * ratio;
  }
  return landed;
}
