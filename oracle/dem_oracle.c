/*
 * dem_oracle.c -- plain, slow FP64 CPU oracle for one DEM time step.
 *
 * TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this.  It shares no code with the CUDA path.
 * Build: gcc -O2 -std=c99 -ffp-contract=off -fPIC -shared (oracle/build.py).
 * -ffp-contract=off matters: the single-precision predicate below must round
 * every product and sum separately, exactly as written.
 *
 * Each function names the passage of Nakahara & Washizawa (arXiv 1503.03553)
 * it follows.  Where the paper leaves a passage open, the comment states the
 * reading taken.
 *
 * Built with -fopenmp -DORC_OPENMP (liboracle_omp.so) the particle and pair
 * loops run on all host cores: each particle's contacts are found in the
 * serial order, each pair's force is computed on its own, and each
 * particle's contributions are added in the serial order (ascending pair
 * index), so the results are bit for bit those of the serial build.
 */
#include "dem_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef ORC_OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                     */
/* ------------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }

/* ------------------------------------------------------------------------ */
/* alpha(epsilon): Sec. 2 names alpha "a function of the coefficient of      */
/* restitution" without giving it.                                           */
/* Reading: alpha is the exact inverse of the restitution of the paper's own */
/* normal law.  For two spheres, m* d'' = -k_n d^{3/2} - eta_n d', with      */
/* eta_n = alpha sqrt(m* k_n sqrt(d)).  Scaling d = d0 x, t = t0 tau with     */
/* d0 = (m* v0^2 / k_n)^{2/5}, t0 = d0 / v0 gives                           */
/*     x'' = -x^{3/2} - alpha x^{1/4} x',   x(0) = 0, x'(0) = 1,             */
/* so e = -x'(tau_end) at the first return to x = 0 depends on alpha only.   */
/* The contact ends when the overlap returns to zero (no tensile clamp).     */
/* ------------------------------------------------------------------------ */
static void ode_rhs(double alpha, double x, double u, double* dx, double* du) {
  double xp = x > 0.0 ? x : 0.0;
  *dx = u;
  *du = -pow(xp, 1.5) - alpha * pow(xp, 0.25) * u;
}

static void rk4(double alpha, double h, double x, double u, double* xo,
                double* uo) {
  double k1x, k1u, k2x, k2u, k3x, k3u, k4x, k4u;
  ode_rhs(alpha, x, u, &k1x, &k1u);
  ode_rhs(alpha, x + 0.5 * h * k1x, u + 0.5 * h * k1u, &k2x, &k2u);
  ode_rhs(alpha, x + 0.5 * h * k2x, u + 0.5 * h * k2u, &k3x, &k3u);
  ode_rhs(alpha, x + h * k3x, u + h * k3u, &k4x, &k4u);
  *xo = x + h / 6.0 * (k1x + 2.0 * k2x + 2.0 * k3x + k4x);
  *uo = u + h / 6.0 * (k1u + 2.0 * k2u + 2.0 * k3u + k4u);
}

double orc_restitution(double alpha) {
  /* RK4 with a graded step: x^{1/4} is not smooth at x = 0, so the step
   * shrinks in proportion to x near both ends of the contact. */
  double x = 0.0, u = 1.0, tau = 0.0;
  long k;
  for (k = 0; k < 50000000L; ++k) {
    double x1, u1, h;
    h = 0.05 * x / (fabs(u) > 1e-3 ? fabs(u) : 1e-3);
    if (h > 1e-4) h = 1e-4;
    if (h < 1e-9) h = 1e-9;
    rk4(alpha, h, x, u, &x1, &u1);
    if (k > 0 && x1 <= 0.0) {
      /* The return to x = 0 lies inside this step: find the partial step
       * length s with x(s) = 0 by bisection and report -x'(s). */
      double a = 0.0, b = h;
      int it;
      for (it = 0; it < 200; ++it) {
        double s = 0.5 * (a + b), xs, us;
        rk4(alpha, s, x, u, &xs, &us);
        if (xs > 0.0) a = s; else b = s;
        if (b - a < 1e-20) break;
      }
      {
        double xs, us;
        rk4(alpha, 0.5 * (a + b), x, u, &xs, &us);
        return -us;
      }
    }
    tau += h;
    if (tau > 200.0) return 0.0; /* no rebound within 60 contact times */
    x = x1;
    u = u1;
  }
  return 0.0;
}

double orc_alpha(double e) {
  static double cached_e = -1.0, cached_alpha = 0.0;
  double lo = 0.0, hi = 4.0; /* e(4) < 1e-3 */
  int it;
  if (e >= 1.0) return 0.0;
  if (e <= 0.0) return hi;
  if (e == cached_e) return cached_alpha;
  /* e(alpha) decreases monotonically in alpha. */
  for (it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (orc_restitution(mid) > e) lo = mid; else hi = mid;
    if (hi - lo < 1e-13) break;
  }
  cached_e = e;
  cached_alpha = 0.5 * (lo + hi);
  return cached_alpha;
}

/* ------------------------------------------------------------------------ */
/* Coefficients, Sec. 2:                                                     */
/*   k_n = 4/3 sqrt(r1 r2/(r1+r2)) ((c(s1))/E1 + (c(s2))/E2)^-1               */
/*   k_t = 8 sqrt(r1 r2/(r1+r2) dn) ((2-s1)/G1 + (2-s2)/G2)^-1                */
/* The printed numerator of k_n is 2 - sigma^2; Hertz theory has            */
/* 1 - sigma^2, which is read as meant and taken as the default;             */
/* kn_literal = 1 selects the printed form.                                  */
/* Both bodies share one material.  A wall (r2 <= 0) has infinite radius,    */
/* so r1 r2/(r1+r2) -> r1.                                                   */
/* ------------------------------------------------------------------------ */
static double reduced_radius(double r1, double r2) {
  return r2 > 0.0 ? r1 * r2 / (r1 + r2) : r1;
}

double orc_kn(const orc_params* p, double r1, double r2) {
  double s = p->poisson;
  double c = p->kn_literal ? (2.0 - s * s) : (1.0 - s * s);
  double inv = c / p->E + c / p->E;
  return 4.0 / 3.0 * sqrt(reduced_radius(r1, r2)) / inv;
}

static double kt_of(const orc_params* p, double r1, double r2, double dn) {
  double s = p->poisson;
  double G = p->E / (2.0 * (1.0 + s)); /* transverse modulus G = E/(2(1+s)) */
  double inv = (2.0 - s) / G + (2.0 - s) / G;
  return 8.0 * sqrt(reduced_radius(r1, r2) * dn) / inv;
}

static double mass_of(const orc_params* p, double r) {
  return p->density * 4.0 / 3.0 * M_PI * r * r * r;
}

/* ------------------------------------------------------------------------ */
/* One contact: Eq. (1), Eq. (vt), Eq. (dt), the Coulomb cap of Eq. (sliding */
/* friction) with the delta_t reset that follows it, and T = r (n x F).      */
/* Particle 1 is the lower id; n points from 1 to 2 (Sec. 2); v = v1 - v2.   */
/* delta_t is advanced (with this step's v_t dt) before the force, then the  */
/* cap, then the torque: the order of Algorithm 1.  The projection of        */
/* delta_t,old in Eq. (dt) keeps its tangential part without rescaling, and  */
/* the cap uses F_t including its damping part, both as printed.             */
/* ------------------------------------------------------------------------ */
static void contact_force(const orc_params* p, double alpha,
                          const double n[3], double dn,
                          double r1, double r2, double m1, double m2,
                          const double v1[3], const double v2[3],
                          const double w1[3], const double w2[3],
                          const double dt_old[3], double dt_new[3],
                          orc_contact_info* out) {
  int a;
  double v[3], vn[3], vt[3], rot[3], rxn[3], Fn[3], Ft[3], F[3];
  double vn_s, dd, kn, kt, mstar, eta, fn_el, absFn, absFt;
  memset(out, 0, sizeof(*out));
  out->delta_n = dn;
  if (!(dn > 0.0)) {
    /* listed by a single-precision predicate but not overlapping in FP64:
     * no force, history cleared */
    dt_new[0] = dt_new[1] = dt_new[2] = 0.0;
    return;
  }
  for (a = 0; a < 3; ++a) v[a] = v1[a] - v2[a];
  vn_s = dot3(v, n);
  for (a = 0; a < 3; ++a) vn[a] = vn_s * n[a];
  /* Eq. (vt): v_t = v - (v.n) n + (r1 w1 + r2 w2) x n */
  for (a = 0; a < 3; ++a) rot[a] = r1 * w1[a] + (r2 > 0.0 ? r2 * w2[a] : 0.0);
  cross3(rot, n, rxn);
  for (a = 0; a < 3; ++a) vt[a] = v[a] - vn[a] + rxn[a];
  /* Eq. (dt): delta_t = delta_t,old - (delta_t,old . n) n + v_t dt */
  dd = dot3(dt_old, n);
  for (a = 0; a < 3; ++a) dt_new[a] = dt_old[a] - dd * n[a] + vt[a] * p->dt;
  /* coefficients */
  kn = orc_kn(p, r1, r2);
  kt = kt_of(p, r1, r2, dn);
  mstar = r2 > 0.0 ? m1 * m2 / (m1 + m2) : m1;
  eta = alpha * sqrt(mstar * kn * sqrt(dn)); /* eta_n = eta_t */
  /* Eq. (1), split into normal and tangential parts */
  fn_el = kn * pow(dn, 1.5);
  for (a = 0; a < 3; ++a) Fn[a] = -fn_el * n[a] - eta * vn[a];
  for (a = 0; a < 3; ++a) Ft[a] = -kt * dt_new[a] - eta * vt[a];
  /* the size of the terms whose float sum forms F (the error scale of the
   * parity tests): Eq. (1)'s terms, with eta v_t counted by the terms of
   * Eq. (vt), |v| + r1 |w1| + r2 |w2|: in a rolling contact the
   * translational and rotational parts of v_t nearly cancel, and a float
   * evaluation of v_t errs by the unit roundoff times those parts */
  out->scale = fn_el + eta * fabs(vn_s) + kt * norm3(dt_new) +
               eta * (norm3(v) + r1 * norm3(w1) + (r2 > 0.0 ? r2 * norm3(w2) : 0.0));
  absFn = norm3(Fn);
  absFt = norm3(Ft);
  out->ratio = (p->mu_d * absFn > 0.0) ? absFt / (p->mu_d * absFn)
                                        : (absFt > 0.0 ? INFINITY : 0.0);
  /* Eq. (sliding friction): cap |F_t| at mu_D |F_n|, then reset delta_t so
   * that F_t,new = -k_t delta_t */
  if (absFt > p->mu_d * absFn) {
    double s = p->mu_d * absFn / absFt;
    for (a = 0; a < 3; ++a) Ft[a] *= s;
    for (a = 0; a < 3; ++a) dt_new[a] = -Ft[a] / kt;
    out->capped = 1;
  }
  for (a = 0; a < 3; ++a) F[a] = Fn[a] + Ft[a];
  for (a = 0; a < 3; ++a) out->F[a] = F[a];
  for (a = 0; a < 3; ++a) out->n[a] = n[a];
  out->kt = kt;
  cross3(n, F, out->nF);
}

/* ------------------------------------------------------------------------ */
/* Cell rules and contact predicates.  Sec. 2 defines contact as a positive  */
/* normal overlap; the cell method (Sec. 2, last paragraph) only finds the   */
/* candidates.  The three predicate variants fix how the comparison          */
/* |d|^2 < (r1+r2)^2 is rounded so that a GPU mode can be checked bit for    */
/* bit.                                                                       */
/* ------------------------------------------------------------------------ */
#define FIXQ_SHIFT 60 /* fixed-point quantum q = 2^-60 m */

static int64_t to_fixed(double x) { return llround(ldexp(x, FIXQ_SHIFT)); }

static int64_t floor_div64(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
  return q;
}

static int32_t clampi(int64_t c, int32_t n) {
  if (c < 0) return 0;
  if (c > n - 1) return n - 1;
  return (int32_t)c;
}

/* Cell coordinate of one position component on axis a. */
static int32_t cell_coord(const orc_params* p, int a, double x) {
  int32_t n = p->ncell[a];
  if (p->predicate == ORC_PRED_FIXED_F32) {
    int64_t Lq = to_fixed(p->L[a]);
    int64_t H = Lq / n;
    return clampi(floor_div64(to_fixed(x), H), n);
  } else if (p->predicate == ORC_PRED_ABS_F32) {
    float inv_h = (float)((double)n / p->L[a]);
    float t = (float)x * inv_h;
    return clampi((int64_t)floorf(t), n);
  } else {
    double inv_h = (double)n / p->L[a];
    return clampi((int64_t)floor(x * inv_h), n);
  }
}

/* Single-precision offset of a position from its cell origin (fixed rule). */
static float fixed_offset(const orc_params* p, int a, double x, int32_t c) {
  int64_t Lq = to_fixed(p->L[a]);
  int64_t H = Lq / p->ncell[a];
  int64_t O = to_fixed(x) - (int64_t)c * H;
  return (float)O * 0x1p-60f;
}

static int stencil_of(const orc_params* p) {
  return p->stencil > 0 ? p->stencil : 1;
}

/* Geometric cell step from ci to cj on axis a: in [-w, w] (w = stencil), or
 * w + 1 when the two cells are not within the stencil.  *image receives the
 * periodic image (-1, 0, +1) in units of the box length that places cell cj
 * at that step from ci. */
static int cell_step(const orc_params* p, int a, int32_t ci, int32_t cj,
                     int* image) {
  int32_t n = p->ncell[a];
  int32_t d = cj - ci;
  int w = stencil_of(p);
  *image = 0;
  if (d >= -w && d <= w) return d;
  if (p->periodic[a]) {
    if (d - n >= -w && d - n <= w) { *image = -1; return d - n; }
    if (d + n >= -w && d + n <= w) { *image = 1; return d + n; }
  }
  return w + 1;
}

/* Per-particle data the predicates need, computed once per call: cell
 * coordinates under the predicate's cell rule and, for the fixed-point rule,
 * the single-precision offsets from the cell origin. */
typedef struct {
  int32_t* cc;   /* n x 3 cell coordinates        */
  float* off;    /* n x 3 offsets (fixed rule)     */
  int64_t Lq[3]; /* box length in quanta           */
  int64_t H[3];  /* cell edge in quanta            */
} pred_data;

static int pred_init(const orc_params* p, int64_t n, const double* x,
                     pred_data* pd) {
  int64_t i;
  int a;
  pd->cc = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(n > 0 ? n : 1));
  pd->off = (float*)malloc(sizeof(float) * 3 * (size_t)(n > 0 ? n : 1));
  if (!pd->cc || !pd->off) { free(pd->cc); free(pd->off); return 1; }
  for (a = 0; a < 3; ++a) {
    pd->Lq[a] = to_fixed(p->L[a]);
    pd->H[a] = pd->Lq[a] / p->ncell[a];
  }
  for (i = 0; i < n; ++i)
    for (a = 0; a < 3; ++a) {
      int32_t c = cell_coord(p, a, x[3 * i + a]);
      pd->cc[3 * i + a] = c;
      pd->off[3 * i + a] = p->predicate == ORC_PRED_FIXED_F32
                               ? fixed_offset(p, a, x[3 * i + a], c) : 0.0f;
    }
  return 0;
}

static void pred_free(pred_data* pd) {
  free(pd->cc);
  free(pd->off);
}

/* Is (i, j) a contact?  x holds FP64 positions, r radii. */
static int is_contact(const orc_params* p, const pred_data* pd,
                      const double* x, const double* r, int64_t i,
                      int64_t j) {
  int a;
  const double* xi = &x[3 * i];
  const double* xj = &x[3 * j];
  if (p->predicate == ORC_PRED_FP64) {
    double d[3], d2, R;
    for (a = 0; a < 3; ++a) {
      d[a] = xj[a] - xi[a];
      if (p->periodic[a]) {
        double hl = 0.5 * p->L[a];
        if (d[a] > hl) d[a] -= p->L[a];
        else if (d[a] < -hl) d[a] += p->L[a];
      }
    }
    d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
    R = r[i] + r[j];
    return d2 < R * R;
  } else if (p->predicate == ORC_PRED_FIXED_F32) {
    /* Offsets from the cell origins in FP32, plus the exact cell shift
     * rounded once: dx = (o_j - o_i) + (float)((cj - ci) H + image L). */
    float d[3], d2, R;
    for (a = 0; a < 3; ++a) {
      int image;
      int32_t ci = pd->cc[3 * i + a];
      int32_t cj = pd->cc[3 * j + a];
      int step = cell_step(p, a, ci, cj, &image);
      int64_t S;
      float s;
      if (step > stencil_of(p)) return 0;
      S = (int64_t)(cj - ci) * pd->H[a] + (int64_t)image * pd->Lq[a];
      s = (float)S * 0x1p-60f;
      d[a] = (pd->off[3 * j + a] - pd->off[3 * i + a]) + s;
    }
    d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
    R = (float)r[i] + (float)r[j];
    return d2 < R * R;
  } else {
    float d[3], d2, R;
    for (a = 0; a < 3; ++a) {
      d[a] = (float)xj[a] - (float)xi[a];
      if (p->periodic[a]) {
        float Lf = (float)p->L[a];
        float hl = 0.5f * Lf;
        if (d[a] > hl) d[a] -= Lf;
        else if (d[a] < -hl) d[a] += Lf;
      }
    }
    d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
    R = (float)r[i] + (float)r[j];
    return d2 < R * R;
  }
}

/* ------------------------------------------------------------------------ */
/* Sort order by (Morton code of the cell, id).  The paper sorts particle    */
/* data by cell every step (Sec. 4.2, "BitonicSort" and                       */
/* "FindCellBoundsAndReorder"); the key here interleaves the cell            */
/* coordinates' bits (x lowest) and breaks ties by id.                        */
/* ------------------------------------------------------------------------ */
static uint64_t morton3(uint32_t x, uint32_t y, uint32_t z) {
  uint64_t code = 0;
  int b;
  for (b = 0; b < 21; ++b) {
    code |= (uint64_t)((x >> b) & 1u) << (3 * b);
    code |= (uint64_t)((y >> b) & 1u) << (3 * b + 1);
    code |= (uint64_t)((z >> b) & 1u) << (3 * b + 2);
  }
  return code;
}

typedef struct { uint64_t key; int32_t id; } key_id;

static int cmp_key_id(const void* a, const void* b) {
  const key_id* x = (const key_id*)a;
  const key_id* y = (const key_id*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return (x->id > y->id) - (x->id < y->id);
}

int orc_order(const orc_params* p, int64_t n, const double* x, int32_t* cell,
              int32_t* order) {
  int64_t i;
  key_id* k = (key_id*)malloc(sizeof(key_id) * (size_t)(n > 0 ? n : 1));
  if (!k) return 1;
  for (i = 0; i < n; ++i) {
    int32_t c[3];
    int a;
    for (a = 0; a < 3; ++a) c[a] = cell_coord(p, a, x[3 * i + a]);
    if (cell)
      cell[i] = (c[2] * p->ncell[1] + c[1]) * p->ncell[0] + c[0];
    k[i].key = morton3((uint32_t)c[0], (uint32_t)c[1], (uint32_t)c[2]);
    k[i].id = (int32_t)i;
  }
  qsort(k, (size_t)n, sizeof(key_id), cmp_key_id);
  for (i = 0; i < n; ++i) order[i] = k[i].id;
  free(k);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Contact search: the cell method of Sec. 2 (27 neighbour cells, Algorithm  */
/* 1 loops) or O(N^2) brute force.  Each pair is recorded once, lo < hi.     */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t lo, hi; } pair32;

static int cmp_pair(const void* a, const void* b) {
  const pair32* x = (const pair32*)a;
  const pair32* y = (const pair32*)b;
  if (x->lo != y->lo) return (x->lo > y->lo) - (x->lo < y->lo);
  return (x->hi > y->hi) - (x->hi < y->hi);
}

/* The contacts (i, j), j > i, of particle i found through the linked cells
 * (Sec. 2, last paragraph: the neighbour cells of i's cell), in the order of
 * the neighbour cells (dz, dy, dx) and of each cell's list; up to lim of
 * them are written to out (out may be NULL).  Returns how many there are. */
static int64_t scan_particle(const orc_params* p, const pred_data* pd, const double* x,
                             const double* r, const int64_t* head, const int64_t* next,
                             int64_t i, pair32* out, int64_t lim) {
  int32_t nx = p->ncell[0], ny = p->ncell[1];
  const int32_t* cc = pd->cc;
  int64_t nb[125], j, got = 0;
  int nnb = 0, dx, dy, dz, q;
  const int w = stencil_of(p);
  /* distinct neighbour cells (a periodic axis with few cells repeats) */
  for (dz = -w; dz <= w; ++dz)
    for (dy = -w; dy <= w; ++dy)
      for (dx = -w; dx <= w; ++dx) {
        int32_t c[3];
        int d[3], a, ok = 1, seen = 0;
        int64_t lin;
        d[0] = dx; d[1] = dy; d[2] = dz;
        for (a = 0; a < 3; ++a) {
          int32_t v = cc[3 * i + a] + d[a];
          if (v < 0 || v >= p->ncell[a]) {
            if (!p->periodic[a]) { ok = 0; break; }
            v = ((v % p->ncell[a]) + p->ncell[a]) % p->ncell[a];
          }
          c[a] = v;
        }
        if (!ok) continue;
        lin = ((int64_t)c[2] * ny + c[1]) * nx + c[0];
        for (q = 0; q < nnb; ++q) if (nb[q] == lin) seen = 1;
        if (!seen) nb[nnb++] = lin;
      }
  for (q = 0; q < nnb; ++q) {
    for (j = head[nb[q]]; j >= 0; j = next[j]) {
      if (j <= i) continue;
      if (is_contact(p, pd, x, r, i, j)) {
        if (out && got < lim) {
          out[got].lo = (int32_t)i;
          out[got].hi = (int32_t)j;
        }
        ++got;
      }
    }
  }
  return got;
}

static int64_t find_pairs(const orc_params* p, int64_t n, const double* x,
                          const double* r, int64_t cap, pair32* out) {
  int64_t cnt = 0, i, j;
  pred_data pd;
  if (pred_init(p, n, x, &pd)) return -2;
  if (p->brute_force) {
    for (i = 0; i < n; ++i)
      for (j = i + 1; j < n; ++j)
        if (is_contact(p, &pd, x, r, i, j)) {
          if (cnt >= cap) { pred_free(&pd); return -1; }
          out[cnt].lo = (int32_t)i;
          out[cnt].hi = (int32_t)j;
          ++cnt;
        }
  } else {
    int32_t nx = p->ncell[0], ny = p->ncell[1], nz = p->ncell[2];
    int64_t M = (int64_t)nx * ny * nz;
    int64_t* head = (int64_t*)malloc(sizeof(int64_t) * (size_t)M);
    int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    const int32_t* cc = pd.cc;
    if (!head || !next) { free(head); free(next); pred_free(&pd); return -2; }
    for (i = 0; i < M; ++i) head[i] = -1;
    /* build linked cells; inserting in descending id keeps lists ascending */
    for (i = n - 1; i >= 0; --i) {
      int64_t lin = ((int64_t)cc[3 * i + 2] * ny + cc[3 * i + 1]) * nx + cc[3 * i + 0];
      next[i] = head[lin];
      head[lin] = i;
    }
#ifdef ORC_OPENMP
    {
      /* count each particle's contacts, then write them at the serial
       * positions (the same order as the loop below) */
      int64_t* off = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
      if (!off) { free(head); free(next); pred_free(&pd); return -2; }
#pragma omp parallel for schedule(dynamic, 256)
      for (i = 0; i < n; ++i)
        off[i + 1] = scan_particle(p, &pd, x, r, head, next, i, NULL, 0);
      for (i = 0; i < n; ++i) off[i + 1] += off[i];
      cnt = off[n];
      if (cnt > cap) { free(off); free(head); free(next); pred_free(&pd); return -1; }
#pragma omp parallel for schedule(dynamic, 256)
      for (i = 0; i < n; ++i)
        scan_particle(p, &pd, x, r, head, next, i, out + off[i], off[i + 1] - off[i]);
      free(off);
    }
#else
    for (i = 0; i < n; ++i) {
      int64_t got = scan_particle(p, &pd, x, r, head, next, i, out + cnt, cap - cnt);
      if (got > cap - cnt) { free(head); free(next); pred_free(&pd); return -1; }
      cnt += got;
    }
#endif
    free(head);
    free(next);
  }
  pred_free(&pd);
  qsort(out, (size_t)cnt, sizeof(pair32), cmp_pair);
  return cnt;
}

int64_t orc_contacts(const orc_params* p, int64_t n, const double* x,
                     const double* r, int64_t cap, int32_t* lo, int32_t* hi) {
  pair32* pr = (pair32*)malloc(sizeof(pair32) * (size_t)(cap > 0 ? cap : 1));
  int64_t cnt, k;
  if (!pr) return -2;
  cnt = find_pairs(p, n, x, r, cap, pr);
  for (k = 0; k < cnt; ++k) { lo[k] = pr[k].lo; hi[k] = pr[k].hi; }
  free(pr);
  return cnt;
}

/* History lookup: binary search of (lo, hi) in a list sorted by (lo, hi). */
static int64_t find_history(int64_t nc, const int32_t* lo, const int32_t* hi,
                            int32_t a, int32_t b) {
  int64_t l = 0, u = nc - 1;
  while (l <= u) {
    int64_t m = l + (u - l) / 2;
    if (lo[m] == a && hi[m] == b) return m;
    if (lo[m] < a || (lo[m] == a && hi[m] < b)) l = m + 1; else u = m - 1;
  }
  return -1;
}

/* Overlap of a particle (centre c, radius r) with a rectangle or line wall:
 * q = the wall's point closest to c (coordinates along the edges clamped to
 * [0, 1]), n = (q - c) / |q - c| (from the particle to the wall), returns
 * r - |q - c|.  A centre lying on the wall has no normal: no contact. */
static double wall_overlap(const orc_wall* wl, const double c[3], double r,
                           double n[3]) {
  double d[3], q[3], e[3], s, t = 0.0, dist;
  int a;
  for (a = 0; a < 3; ++a) d[a] = c[a] - wl->p[a];
  s = dot3(d, wl->u) / dot3(wl->u, wl->u);
  s = s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s);
  if (wl->kind == ORC_WALL_RECT) {
    t = dot3(d, wl->v) / dot3(wl->v, wl->v);
    t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
  }
  for (a = 0; a < 3; ++a) {
    q[a] = wl->p[a] + s * wl->u[a] + (wl->kind == ORC_WALL_RECT ? t * wl->v[a] : 0.0);
    e[a] = q[a] - c[a];
  }
  dist = norm3(e);
  if (!(dist > 0.0)) {
    n[0] = n[1] = n[2] = 0.0;
    return 0.0;
  }
  for (a = 0; a < 3; ++a) n[a] = e[a] / dist;
  return r - dist;
}

/* Periodic wrap into [0, L). */
static double wrap(double x, double L) {
  while (x >= L) x -= L;
  while (x < 0.0) x += L;
  return x;
}

/* One pair (1 = lower id): geometry with the minimum image on periodic axes,
 * n from 1 to 2 and the overlap dn = r1 + r2 - |d| (Sec. 2), the history of
 * the pair (zero for a new contact, Sec. 4.2 InitializeContactIDs) and the
 * contact law; dtn receives the new delta_t. */
static void pair_force(const orc_params* p, double alpha, const double* x, const double* v,
                       const double* w, const double* r, int64_t nc_in, const int32_t* lo_in,
                       const int32_t* hi_in, const double* dt_in, int32_t i1, int32_t i2,
                       double dtn[3], orc_contact_info* ci) {
  double d[3], nrm[3], dist, dn, m1, m2, dto[3] = {0.0, 0.0, 0.0};
  int64_t h;
  int a;
  for (a = 0; a < 3; ++a) {
    d[a] = x[3 * i2 + a] - x[3 * i1 + a];
    if (p->periodic[a]) {
      double hl = 0.5 * p->L[a];
      if (d[a] > hl) d[a] -= p->L[a];
      else if (d[a] < -hl) d[a] += p->L[a];
    }
  }
  dist = norm3(d);
  for (a = 0; a < 3; ++a) nrm[a] = dist > 0.0 ? d[a] / dist : 0.0;
  dn = r[i1] + r[i2] - dist; /* normal overlap, Sec. 2 */
  h = find_history(nc_in, lo_in, hi_in, i1, i2);
  if (h >= 0) for (a = 0; a < 3; ++a) dto[a] = dt_in[3 * h + a];
  m1 = mass_of(p, r[i1]);
  m2 = mass_of(p, r[i2]);
  contact_force(p, alpha, nrm, dn, r[i1], r[i2], m1, m2, &v[3 * i1], &v[3 * i2], &w[3 * i1],
                &w[3 * i2], dto, dtn, ci);
}

/* ------------------------------------------------------------------------ */
/* One step.  The paper leaves the integrator unstated; it is read as       */
/* symplectic Euler.  Order: wrap, contact set, forces (Algorithm 1          */
/* per pair, evaluated once per pair with the action-reaction law), floor    */
/* wall, gravity, then symplectic Euler: v += F/m dt, w += T/I dt,           */
/* x += v dt, with I = 2/5 m r^2.                                             */
/* ------------------------------------------------------------------------ */
int orc_step(const orc_params* p, int64_t n, double* x, double* v, double* w,
             const double* r,
             int64_t nc_in, const int32_t* lo_in, const int32_t* hi_in,
             const double* dt_in, double* wall_dt,
             int64_t cap, int64_t* nc_out, int32_t* lo_out, int32_t* hi_out,
             double* dt_out, orc_contact_info* info, double* F, double* T) {
  int64_t i, k, nc;
  int a;
  double alpha = orc_alpha(p->restitution);
  double* Fp = (double*)calloc((size_t)(3 * (n > 0 ? n : 1)), sizeof(double));
  double* Tp = (double*)calloc((size_t)(3 * (n > 0 ? n : 1)), sizeof(double));
  pair32* pr = (pair32*)malloc(sizeof(pair32) * (size_t)(cap > 0 ? cap : 1));
  if (!Fp || !Tp || !pr) { free(Fp); free(Tp); free(pr); return 1; }

#ifdef ORC_OPENMP
#pragma omp parallel for schedule(static) private(a)
#endif
  for (i = 0; i < n; ++i)
    for (a = 0; a < 3; ++a)
      if (p->periodic[a]) x[3 * i + a] = wrap(x[3 * i + a], p->L[a]);

  nc = find_pairs(p, n, x, r, cap, pr);
  if (nc < 0) { free(Fp); free(Tp); free(pr); return 4; }

#ifdef ORC_OPENMP
  {
    /* every pair's force on its own, then each particle's contributions in
     * ascending pair index: the serial loop's order of additions */
    orc_contact_info* cis = (orc_contact_info*)malloc(sizeof(orc_contact_info) *
                                                      (size_t)(nc > 0 ? nc : 1));
    int64_t* roff = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t* rlist = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * nc > 0 ? 2 * nc : 1));
    if (!cis || !roff || !rlist) {
      free(cis); free(roff); free(rlist); free(Fp); free(Tp); free(pr);
      return 1;
    }
#pragma omp parallel for schedule(static)
    for (k = 0; k < nc; ++k) {
      int32_t i1 = pr[k].lo, i2 = pr[k].hi;
      pair_force(p, alpha, x, v, w, r, nc_in, lo_in, hi_in, dt_in, i1, i2, &dt_out[3 * k],
                 &cis[k]);
      lo_out[k] = i1;
      hi_out[k] = i2;
      if (info) info[k] = cis[k];
    }
    for (k = 0; k < nc; ++k) {
      roff[pr[k].lo + 1]++;
      roff[pr[k].hi + 1]++;
    }
    for (i = 0; i < n; ++i) roff[i + 1] += roff[i];
    {
      int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
      if (!fill) {
        free(cis); free(roff); free(rlist); free(Fp); free(Tp); free(pr);
        return 1;
      }
      memcpy(fill, roff, sizeof(int64_t) * (size_t)n);
      for (k = 0; k < nc; ++k) {
        rlist[fill[pr[k].lo]++] = k;
        rlist[fill[pr[k].hi]++] = k;
      }
      free(fill);
    }
#pragma omp parallel for schedule(static) private(a)
    for (i = 0; i < n; ++i) {
      int64_t e;
      for (e = roff[i]; e < roff[i + 1]; ++e) {
        const int64_t q = rlist[e];
        const int lo = pr[q].lo == i;
        for (a = 0; a < 3; ++a) {
          if (lo) Fp[3 * i + a] += cis[q].F[a];
          else Fp[3 * i + a] -= cis[q].F[a];
          Tp[3 * i + a] += r[i] * cis[q].nF[a];
        }
      }
    }
    free(cis);
    free(roff);
    free(rlist);
  }
#else
  for (k = 0; k < nc; ++k) {
    int32_t i1 = pr[k].lo, i2 = pr[k].hi;
    orc_contact_info ci;
    pair_force(p, alpha, x, v, w, r, nc_in, lo_in, hi_in, dt_in, i1, i2, &dt_out[3 * k], &ci);
    for (a = 0; a < 3; ++a) {
      Fp[3 * i1 + a] += ci.F[a];
      Fp[3 * i2 + a] -= ci.F[a];
      /* torque on 1: arm r1 n, force F; on 2: arm -r2 n, force -F */
      Tp[3 * i1 + a] += r[i1] * ci.nF[a];
      Tp[3 * i2 + a] += r[i2] * ci.nF[a];
    }
    lo_out[k] = i1;
    hi_out[k] = i2;
    if (info) info[k] = ci;
  }
#endif
  *nc_out = nc;

  /* walls: the floor z = 0, then rectangles and lines, each a particle of
   * infinite radius and mass at rest touching the particle at the wall's
   * point closest to its centre (Sec. 3.3 item 5) */
  {
    static const double zero3[3] = {0.0, 0.0, 0.0};
    const int nw = (p->floor_wall ? 1 : 0) + p->nwalls;
    int wi;
    for (wi = 0; wi < nw; ++wi) {
      const int floor = p->floor_wall && wi == 0;
      const orc_wall* wl = floor ? NULL : &p->walls[wi - (p->floor_wall ? 1 : 0)];
#ifdef ORC_OPENMP
#pragma omp parallel for schedule(static) private(a)
#endif
      for (i = 0; i < n; ++i) {
        double nwall[3], dn;
        double* hist = wall_dt ? &wall_dt[3 * (i * nw + wi)] : NULL;
        if (floor) {
          nwall[0] = 0.0;
          nwall[1] = 0.0;
          nwall[2] = -1.0;
          dn = r[i] - x[3 * i + 2];
        } else {
          dn = wall_overlap(wl, &x[3 * i], r[i], nwall);
        }
        if (dn > 0.0) {
          double dto[3], dtn[3];
          orc_contact_info ci;
          for (a = 0; a < 3; ++a) dto[a] = hist ? hist[a] : 0.0;
          contact_force(p, alpha, nwall, dn, r[i], 0.0, mass_of(p, r[i]), 0.0,
                        &v[3 * i], zero3, &w[3 * i], zero3, dto, dtn, &ci);
          for (a = 0; a < 3; ++a) {
            Fp[3 * i + a] += ci.F[a];
            Tp[3 * i + a] += r[i] * ci.nF[a];
            if (hist) hist[a] = dtn[a];
          }
        } else if (hist) {
          for (a = 0; a < 3; ++a) hist[a] = 0.0;
        }
      }
    }
  }

  /* gravity, Sec. 4.2 "ForceGravity" */
#ifdef ORC_OPENMP
#pragma omp parallel for schedule(static) private(a)
#endif
  for (i = 0; i < n; ++i) {
    double m = mass_of(p, r[i]);
    for (a = 0; a < 3; ++a) Fp[3 * i + a] += m * p->g[a];
  }

  if (F) memcpy(F, Fp, sizeof(double) * 3 * (size_t)n);
  if (T) memcpy(T, Tp, sizeof(double) * 3 * (size_t)n);

  /* symplectic Euler, Sec. 4.2 "Integrate" */
#ifdef ORC_OPENMP
#pragma omp parallel for schedule(static) private(a)
#endif
  for (i = 0; i < n; ++i) {
    double m = mass_of(p, r[i]);
    double I = 0.4 * m * r[i] * r[i];
    for (a = 0; a < 3; ++a) {
      v[3 * i + a] += Fp[3 * i + a] / m * p->dt;
      w[3 * i + a] += Tp[3 * i + a] / I * p->dt;
      x[3 * i + a] += v[3 * i + a] * p->dt;
      if (p->periodic[a]) x[3 * i + a] = wrap(x[3 * i + a], p->L[a]);
    }
  }
  free(Fp);
  free(Tp);
  free(pr);
  return 0;
}
