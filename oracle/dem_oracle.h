/*
 * dem_oracle.h -- plain, slow FP64 CPU oracle for one DEM time step of
 * Nakahara & Washizawa, "Accelerating DEM simulations on GPUs by reducing
 * the impact of warp divergences" (arXiv 1503.03553).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * What it computes (Sec. 2 of the paper, read as documented per item):
 *   contact set    pairs with |d| < r1 + r2 (Sec. 2, the overlap definition
 *                  of delta_n); optionally with the single-precision
 *                  predicate the GPU path uses, reproduced bit for bit
 *   per contact    Eq. (1) force, Eq. (vt) tangential velocity, Eq. (dt)
 *                  tangential displacement update, k_n / k_t / eta_n = eta_t
 *                  definitions, Eq. (sliding friction) Coulomb cap and the
 *                  delta_t reset, torque T = r (n x F)
 *   history        delta_t kept per pair and erased when a pair separates
 *                  (Sec. 4.2, kernel "InitializeContactIDs")
 *   walls          flat floor z = 0, rectangles and straight line segments,
 *                  each treated like a particle of infinite radius and mass
 *                  at rest (Sec. 3.3 item 5; kernels "CollideRectangle" and
 *                  "CollideLine" of Sec. 4.2)
 *   gravity        m g (Sec. 4.2, "ForceGravity")
 *   integration    symplectic Euler (Sec. 4.2 "Integrate"; scheme unstated)
 *   alpha(eps)     exact inversion of the restitution of the paper's own
 *                  normal force law (alpha is named but not given, Sec. 2)
 *
 * Pinned by tests/test_oracle_*.py against: O(N^2) brute force and a k-d
 * tree library search, the closed-form Hertz contact time and maximum
 * overlap, an independent library ODE solve of the restitution, the textbook
 * sliding-to-rolling transition of a sphere on a floor, momentum
 * conservation, the Coulomb inequality and hand-derived single-contact
 * forces.
 */
#ifndef DEM_ORACLE_H
#define DEM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Contact predicate / cell rule variants (the "reading" the GPU mode uses). */
enum {
  ORC_PRED_FP64 = 0,       /* d.d < (r1+r2)^2 in FP64, minimum image      */
  ORC_PRED_FIXED_F32 = 1,  /* 2^-60 m fixed-point position, FP32 offsets  */
  ORC_PRED_ABS_F32 = 2     /* FP32 absolute position, FP32 minimum image  */
};

/* A wall (Sec. 3.3 item 5: rectangles and straight lines).
 *   ORC_WALL_RECT  the rectangle p + s u + t v, s, t in [0, 1], u and v
 *                  perpendicular; a particle touches its closest point
 *                  (face, edge or corner)
 *   ORC_WALL_LINE  the segment p + s u, s in [0, 1]
 * Walls are not repeated across periodic boundaries. */
enum { ORC_WALL_RECT = 0, ORC_WALL_LINE = 1 };
typedef struct {
  int32_t kind;
  int32_t pad;
  double p[3], u[3], v[3];
} orc_wall;

typedef struct {
  double L[3];          /* box edge lengths [m]; box is [0, L)            */
  double g[3];          /* gravitational acceleration [m/s^2]            */
  double dt;            /* time step [s]                                  */
  double E;             /* Young's modulus [Pa]                           */
  double poisson;       /* Poisson ratio sigma                            */
  double density;       /* [kg/m^3]                                       */
  double restitution;   /* coefficient of restitution epsilon             */
  double mu_d;          /* sliding friction coefficient                   */
  int32_t periodic[3];  /* 1 = periodic axis                              */
  int32_t floor_wall;   /* 1 = flat wall at z = 0                         */
  int32_t ncell[3];     /* cell grid used for sort order and predicates   */
  int32_t predicate;    /* ORC_PRED_*                                     */
  int32_t kn_literal;   /* 1 = k_n with the printed (2 - sigma^2)/E term  */
  int32_t brute_force;  /* 1 = O(N^2) pair search instead of cells        */
  int32_t stencil;      /* neighbour cells searched per axis: +-stencil   */
                        /* (cells at least 2 r_max / stencil wide; 0 = 1) */
  int32_t nwalls;       /* rectangle and line walls                       */
  const orc_wall* walls;
} orc_params;

/* Per-contact diagnostics, one record per contact of the new list. */
typedef struct {
  double F[3];      /* force on the lower-id particle                     */
  double nF[3];     /* n x F                                              */
  double n[3];      /* unit normal from the lower-id particle to the other */
  double kt;        /* tangential stiffness k_t                            */
  double scale;     /* k_n dn^1.5 + eta|v_n| + k_t|delta_t|                 */
                    /* + eta (|v| + r1|w1| + r2|w2|): Eq. (1)'s terms, v_t  */
                    /* counted by the terms of Eq. (vt)                      */
  double delta_n;   /* normal overlap                                     */
  double ratio;     /* |F_t| / (mu |F_n|) before the cap                  */
  int32_t capped;   /* 1 if the Coulomb cap fired                          */
  int32_t pad;
} orc_contact_info;

/* Restitution coefficient e(alpha) of the paper's normal law.  The paper
 * does not give alpha(eps); alpha is read as the exact inverse of the
 * rebound of its own two-body normal law x'' = -x^{3/2} - alpha x^{1/4} x',
 * x(0) = 0, x'(0) = 1, e = -x'(end) (independent of speed and size). */
double orc_restitution(double alpha);
/* alpha(e): inverse of orc_restitution by bisection. */
double orc_alpha(double e);

/* Normal stiffness k_n for radii r1, r2 (r2 <= 0 means a wall). */
double orc_kn(const orc_params* p, double r1, double r2);

/* Cell of each particle under the predicate's cell rule (linear index
 * (cz*ny + cy)*nx + cx) and the sort order by (Morton code of the cell, id). */
int orc_order(const orc_params* p, int64_t n, const double* x,
              int32_t* cell, int32_t* order);

/* Contact set, pairs (lo < hi) sorted by (lo, hi).  Returns the count, or -1
 * when more than cap pairs exist. */
int64_t orc_contacts(const orc_params* p, int64_t n, const double* x,
                     const double* r, int64_t cap, int32_t* lo, int32_t* hi);

/* One time step in place on x, v, w (n x 3 each, id order).
 *   in:  contact history (nc_in pairs sorted by (lo, hi)) with delta_t
 *        (nc_in x 3); wall_dt (n x nw x 3 with nw = floor_wall + nwalls,
 *        the floor first, then the walls in order; may be NULL when nw = 0)
 *   out: new contact list and delta_t (sorted by (lo, hi)), per-contact
 *        info (may be NULL), per-particle force F and torque T used in the
 *        step (n x 3 each, may be NULL).
 * Returns 0, or 4 when the new list needs more than cap entries. */
int orc_step(const orc_params* p, int64_t n, double* x, double* v, double* w,
             const double* r,
             int64_t nc_in, const int32_t* lo_in, const int32_t* hi_in,
             const double* dt_in, double* wall_dt,
             int64_t cap, int64_t* nc_out, int32_t* lo_out, int32_t* hi_out,
             double* dt_out, orc_contact_info* info, double* F, double* T);

#ifdef __cplusplus
}
#endif
#endif
