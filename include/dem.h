/*
 * dem.h -- C ABI of the GB300 DEM library (libdem_gb300.so).
 *
 * One time step of the discrete element method of Nakahara & Washizawa,
 * "Accelerating DEM simulations on GPUs by reducing the impact of warp
 * divergences" (arXiv 1503.03553), run on one GPU:
 *   - cell binning and a Morton-ordered counting sort (Sec. 4.2, kernels
 *     CalcHash, BitonicSort, FindCellBoundsAndReorder),
 *   - contact detection over the 27 neighbour cells (Sec. 2, last
 *     paragraph; Algorithm 1) into a candidate list kept between re-sorts
 *     (pairs within a skin of contact), the contact rule applied to every
 *     candidate each step, and warp-level compaction of the true contacts
 *     for the force (the paper's two-loop split, Sec. 3.4 and Sec. 4.3,
 *     carried to a global list),
 *   - carry-over of the tangential displacement history between steps
 *     (Sec. 2 "condensed format of a sparse matrix"; Sec. 4.2
 *     InitializeContactIDs),
 *   - Hertz-Mindlin contact force and torque, Eq. (1), Eq. (vt), Eq. (dt),
 *     the k_n, k_t, eta definitions and the Coulomb cap Eq. (sliding
 *     friction) with its delta_t reset,
 *   - floor wall (Sec. 3.3 item 5; CollideRectangle) and gravity
 *     (ForceGravity),
 *   - a deterministic per-particle force sum and symplectic Euler
 *     integration (Sec. 4.2, Integrate).
 *
 * Conventions for every entry point
 *   Units are SI.  Particle arrays are in id order: element k (or row k of
 *   an n x 3 array, row-major) belongs to particle id k of that box.
 *   A `where` argument says whether caller pointers are host (DEM_HOST) or
 *   device (DEM_DEVICE) memory of the context's GPU.  Caller memory is only
 *   read or written during the call; the library never keeps a caller
 *   pointer.  The library owns all device state; it allocates it in
 *   dem_create through the caller's allocator hook (or cudaMallocAsync when
 *   the hook is NULL) and frees it in dem_destroy.  All work is ordered on
 *   the configuration's CUDA stream.  Calls on one context must not run
 *   concurrently from several host threads.
 *   Errors are returned as dem_status codes; nothing aborts and no C++
 *   exception crosses the ABI.  A device-side error (capacity overflow,
 *   non-finite state, failed internal consistency check) is recorded in a
 *   status word that dem_step returns; it stays set until dem_destroy.
 *   dem_last_error gives a one-line description of the last failure.
 */
#ifndef DEM_GB300_H
#define DEM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DEM_ABI_VERSION 5

typedef enum {
  DEM_OK = 0,
  DEM_ERR_ARG = 1,        /* invalid argument (null, out of range, bad box) */
  DEM_ERR_ALLOC = 2,      /* device allocation failed                      */
  DEM_ERR_CUDA = 3,       /* a CUDA runtime call failed                     */
  DEM_ERR_CAPACITY = 4,   /* a contact row or the contact list overflowed   */
  DEM_ERR_NONFINITE = 5,  /* a position, velocity or force became NaN/Inf   */
  DEM_ERR_TIMEOUT = 6,    /* reserved: no kernel of this library waits on   */
                          /* another, so no wait can time out               */
  DEM_ERR_STATE = 7       /* call out of order (e.g. step before particles) */
} dem_status;

/* Arithmetic of the force path.
 *   DEM_FP64  : everything in FP64 (the plain form).
 *   DEM_MIXED : FP32 force arithmetic; master positions in 64-bit fixed
 *               point (quantum 2^-60 m), overlap from an exact position
 *               difference, tangential history accumulated as a float-float
 *               pair.
 *   DEM_FP32  : FP32 everywhere (positions, history, forces). */
typedef enum { DEM_FP64 = 0, DEM_MIXED = 1, DEM_FP32 = 2 } dem_precision;

typedef enum { DEM_HOST = 0, DEM_DEVICE = 1 } dem_where;

/* Contact-force kernel layout.
 *   DEM_COLLIDE_COMPACT : the contact search writes a candidate list (the
 *                         contacts plus, with a skin, the pairs within the
 *                         skin of contact); every step the contact rule is
 *                         applied to each candidate, the contacts are
 *                         compacted by warp ballots and one thread per
 *                         contact computes the force; a per-particle pass
 *                         sums it in partner-id order (no float atomics).
 *   DEM_COLLIDE_FUSED   : Algorithm 1 of the paper: one thread per particle
 *                         searches and computes the force of each contact as
 *                         it is found (each pair evaluated from both sides).
 *   DEM_COLLIDE_TWOLOOP : the paper's improved Collide (Sec. 3.4): one thread
 *                         per particle first finds and keeps all its contact
 *                         partners, then computes their forces in a second
 *                         loop.  Same results as DEM_COLLIDE_FUSED, bit for
 *                         bit (same summation order). */
typedef enum {
  DEM_COLLIDE_COMPACT = 0,
  DEM_COLLIDE_FUSED = 1,
  DEM_COLLIDE_TWOLOOP = 2
} dem_collide;

/* One material (Sec. 2: sigma, G, E, m via density; alpha from epsilon).
 * The transverse modulus is G = E / (2 (1 + poisson)). */
typedef struct {
  double E;            /* Young's modulus [Pa]                  */
  double poisson;      /* Poisson ratio                         */
  double density;      /* [kg/m^3]                              */
  double restitution;  /* coefficient of restitution, (0, 1]    */
  double mu_d;         /* sliding friction coefficient, >= 0    */
} dem_material;

/* A wall (Sec. 3.3 item 5: rectangles and straight lines; Sec. 4.2 kernels
 * CollideRectangle and CollideLine).  A wall is a body of infinite radius
 * and mass at rest of the box's material; a particle touches it at the
 * wall's point closest to its centre, and the force is that of a
 * particle-particle contact with R* = r and m* = m.  Each particle keeps a
 * tangential history per wall.  Walls are not repeated across periodic
 * boundaries.
 *   DEM_WALL_RECT : the rectangle p + s u + t v, s and t in [0, 1]; u and v
 *                   must be perpendicular (|u.v| <= 1e-9 |u||v|)
 *   DEM_WALL_LINE : the segment p + s u, s in [0, 1] (v unused) */
typedef enum { DEM_WALL_RECT = 0, DEM_WALL_LINE = 1 } dem_wall_kind;
typedef struct {
  int32_t kind;        /* dem_wall_kind                                */
  int32_t pad;
  double p[3];         /* corner / first end [m]                       */
  double u[3];         /* first edge / segment [m], non-zero           */
  double v[3];         /* second edge [m] (rectangles)                 */
} dem_wall;

/* One independent box.  Periodic axes wrap positions into [0, L).
 * Non-periodic axes are open; floor_wall adds a flat wall at z = 0, walls
 * adds rectangles and lines (at most 15 per box, floor included). */
typedef struct {
  double L[3];            /* edge lengths [m], > 0                        */
  int32_t periodic[3];    /* 1 = periodic                                 */
  int32_t floor_wall;     /* 1 = wall at z = 0 (z must be non-periodic)    */
  double g[3];            /* gravity [m/s^2]                              */
  double dt;              /* time step [s]                                */
  int32_t material;       /* index into dem_config.materials              */
  int32_t ncell[3];       /* cell grid; 0 = largest grid with cells at     */
                          /* least 2 r_max (1 + 1e-5) wide (see r_split)   */
  int64_t max_particles;  /* capacity of the box                          */
  double r_max;           /* largest radius the box will hold [m]         */
  int32_t nwalls;         /* rectangle and line walls (0 = none)           */
  const dem_wall* walls;  /* nwalls entries, read during dem_create        */
  double r_split;         /* size-binned contact search (0 = off; Sec. 3.3 */
                          /* cell-size trade-off), for polydisperse boxes: */
                          /* a particle of radius                          */
                          /* above r_split searches the +-2 neighbour      */
                          /* cells for all its partners, the others search */
                          /* +-1 cells for partners of radius up to        */
                          /* r_split.  Cells then need only be             */
                          /* max(2 r_split, r_max) (1 + 1e-5) wide (ncell  */
                          /* 0 picks the largest such grid) and periodic   */
                          /* axes at least 5 cells.  Same contacts as the  */
                          /* single-class search.  DEM_COLLIDE_COMPACT only */
  double skin;            /* candidate-list skin [m] (0 = search every     */
                          /* step).  The cell search at a re-sort keeps    */
                          /* every pair within r_i + r_j + skin; each step */
                          /* then applies the contact rule to those pairs  */
                          /* only, and the next re-sort comes as soon as a */
                          /* particle has moved about skin / 2 since the   */
                          /* last one (Sec. 2 cell method; the paper       */
                          /* searches every step).  Same contacts and      */
                          /* results, bit for bit, whatever the skin.      */
                          /* Cells must then be (2 r_max + skin) (1 +      */
                          /* 1e-5) wide (max(2 r_split + skin, r_max +     */
                          /* skin / 2) (1 + 1e-5) size-binned).            */
                          /* DEM_COLLIDE_COMPACT only.                     */
} dem_box;

typedef struct {
  int32_t nboxes;
  const dem_box* boxes;
  int32_t nmaterials;
  const dem_material* materials;
  int32_t precision;          /* dem_precision                              */
  int32_t collide;            /* dem_collide                                */
  int32_t kn_literal;         /* 1 = k_n with the printed (2 - sigma^2)/E    */
                              /* term of Sec. 2 instead of Hertz 1 - sigma^2 */
  int32_t row_capacity;       /* max contacts of one particle; 0 = 32;      */
                              /* rounded up to a multiple of 4, at least 8 */
  int32_t graph_steps;        /* steps per captured CUDA graph; 0 = 16,     */
                              /* -1 = launch kernels directly.  With       */
                              /* DEM_COLLIDE_COMPACT the steps of a call   */
                              /* beyond a multiple of it run as one-step   */
                              /* graphs; the other forms launch them       */
                              /* directly                                  */
  int32_t block;              /* threads per block of per-particle kernels; */
                              /* 0 = 128                                   */
  int32_t l2_fetch;           /* L2 fetch granularity in bytes set on the   */
                              /* CUDA context at creation (the runtime's    */
                              /* cudaLimitMaxL2FetchGranularity, a hint):   */
                              /* 0 = 64, or 32, 64, 128; -1 = leave the     */
                              /* context's limit alone.  The limit holds for */
                              /* every kernel of the context (other         */
                              /* libraries' too) until it is set again.  64 */
                              /* keeps the per-particle sum's scattered     */
                              /* 32-byte reads from fetching more; the pair */
                              /* kernel asks for 128-byte fetches on its    */
                              /* own loads of partner state                 */
  void* stream;               /* cudaStream_t; NULL = legacy default stream */
  void* (*alloc)(size_t bytes, void* ctx);  /* device allocator or NULL     */
  void (*free)(void* ptr, void* ctx);
  void* alloc_ctx;
} dem_config;

typedef struct dem_ctx dem_ctx;

/* Create a context on the current CUDA device and allocate all device state
 * for cfg (copied; cfg need not outlive the call; the walls are read during
 * the call).  On success *out holds the context; on failure *out is NULL and
 * the status says why (dem_last_error(NULL) describes it).
 * DEM_ERR_ARG: inconsistent configuration (a periodic axis with fewer than 3
 * cells, cells narrower than 2 r_max, bad material index, floor on a
 * periodic z axis, a bad wall or more than 15 per box, r_split outside
 * [0, r_max], a size-binned box with a per-particle Collide form or a
 * periodic axis of fewer than 5 cells, ...).  DEM_ERR_ALLOC: the allocator
 * returned NULL.  DEM_ERR_CUDA: no device, or a CUDA call failed. */
dem_status dem_create(const dem_config* cfg, dem_ctx** out);

/* Replace the particles of one box (Sec. 4.2: the CPU only creates the
 * initial configuration).  n <= max_particles; x, v, omega: n x 3; radius:
 * n, each in (0, r_max].  Clears the box's contact history.  In DEM_MIXED
 * and DEM_FP32 radii are stored as float32 and positions are rounded to the
 * mode's representation.  DEM_ERR_ARG: bad box, n above the capacity, a
 * NULL array, a radius outside (0, r_max] or a non-finite value (host
 * arrays are checked before any copy). */
dem_status dem_set_particles(dem_ctx* ctx, int32_t box, int64_t n,
                             const double* x, const double* v,
                             const double* omega, const double* radius,
                             int32_t where);

/* Overwrite positions, velocities and angular velocities (n x 3 each, any
 * may be NULL to keep it) of the particles already in a box, keeping radii
 * and the contact history.  Host arrays are read by the time the call
 * returns.  A non-finite value is reported by the next dem_step
 * (DEM_ERR_NONFINITE).  With DEM_COLLIDE_COMPACT new positions are taken
 * like those of a step: the next step re-sorts only if a particle moved
 * beyond its box's skin limit since the last re-sort (the results do not
 * depend on when re-sorts happen). */
dem_status dem_set_state(dem_ctx* ctx, int32_t box, const double* x,
                         const double* v, const double* omega, int32_t where);

/* Advance every box by nsteps >= 0 steps (Sec. 4.2's kernel sequence;
 * Algorithm 1; Eq. (1), Eq. (vt), Eq. (dt), the coefficients of Sec. 2 and
 * the sliding-friction cap).  Each step: find contacts (with
 * DEM_COLLIDE_COMPACT, a re-sort first when one is due: sort by cell,
 * candidate search, delta_t history carried to the new list), compute
 * forces and torques, walls and gravity, integrate.  The decision to
 * re-sort is taken on the device; with CUDA graphs the re-sort kernels sit
 * in a conditional node and do not launch in other steps.  Returns after the work is enqueued and the device status
 * word is read (one stream synchronisation per call).  DEM_ERR_CAPACITY:
 * a particle's contacts exceeded row_capacity or the list its capacity;
 * DEM_ERR_NONFINITE: a non-finite or out-of-range state; DEM_ERR_STATE:
 * no particles set, or an internal consistency check failed.  Device
 * errors are sticky: later calls return them until dem_destroy. */
dem_status dem_step(dem_ctx* ctx, int64_t nsteps);

/* Read the state of one box in id order: x, v, omega (n x 3); force and
 * torque (n x 3): the totals used in the last step (Eq. (1) and
 * T = r (n x F) summed over contacts, walls and gravity).  Any pointer may
 * be NULL.  The caller owns the arrays; they are written by the time the
 * call returns. */
dem_status dem_get_state(dem_ctx* ctx, int32_t box, double* x, double* v,
                         double* omega, double* force, double* torque,
                         int32_t where);

/* Number of particles currently in a box. */
dem_status dem_get_count(dem_ctx* ctx, int32_t box, int64_t* n);

/* Contact list of one box after the last step (host pointers), sorted by
 * (id_lo, id_hi), id_lo < id_hi: the pairs found in that step and their
 * tangential displacement delta_t (cap x 3) after the step's update, as
 * stored for the next step (Sec. 2: delta_t kept per contact, in a
 * condensed sparse format; Sec. 4.2 InitializeContactIDs).  *n receives
 * the count; DEM_ERR_CAPACITY if it exceeds cap (nothing written then). */
dem_status dem_get_contacts(dem_ctx* ctx, int32_t box, int64_t cap,
                            int64_t* n, int32_t* id_lo, int32_t* id_hi,
                            double* delta_t);

/* Per-contact force of the last step (host pointers), in the order of
 * dem_get_contacts: F (cap x 3) is the force on particle id_lo from Eq. (1)
 * after the Coulomb cap; nF (cap x 3) is n x F with n the unit normal from
 * id_lo to id_hi, so the torques are T_lo = r_lo nF and T_hi = r_hi nF.
 * Either output may be NULL.  DEM_ERR_CAPACITY if the count exceeds cap. */
dem_status dem_get_contact_forces(dem_ctx* ctx, int32_t box, int64_t cap,
                                  int64_t* n, int32_t* id_lo, int32_t* id_hi,
                                  double* F, double* nF);

/* Replace the contact history of one box (host pointers, any order,
 * id_lo < id_hi < count) so that the next step starts from it
 * (checkpoint restore of Sec. 2's per-contact delta_t).  DEM_ERR_ARG: an
 * id out of range, not ordered or a pair given twice; DEM_ERR_CAPACITY:
 * more pairs than the list holds. */
dem_status dem_set_contacts(dem_ctx* ctx, int32_t box, int64_t n,
                            const int32_t* id_lo, const int32_t* id_hi,
                            const double* delta_t);

/* Sort order used in the last step (host pointers, n entries each, may be
 * NULL; Sec. 4.2 BitonicSort / FindCellBoundsAndReorder: particle data
 * kept in cell order): the particle id held by each storage slot, and the
 * linear cell (cz*ny + cy)*nx + cx of that slot.  Slots are ordered by
 * (Morton code of the cell, id). */
dem_status dem_get_order(dem_ctx* ctx, int32_t box, int32_t* id_by_slot,
                         int32_t* cell_by_slot);

/* Cell grid of a box (Sec. 2, last paragraph: the cells of the contact
 * search): cells per axis. */
dem_status dem_get_grid(dem_ctx* ctx, int32_t box, int32_t ncell[3]);

#define DEM_NSTATS 10
/* Diagnostics of one box from the current state and the last step's
 * contacts, reduced in FP64 in a fixed order:
 *   [0] translational kinetic energy   [1] rotational kinetic energy
 *   [2..4] total momentum              [5] number of contacts
 *   [6] mean coordination 2 C / n      [7] max overlap / smaller radius
 *   [8] max |F_t| / (mu |F_n|) before the cap   [9] particles in the box */
dem_status dem_get_stats(dem_ctx* ctx, int32_t box, double out[DEM_NSTATS]);

/* Milliseconds of device time per step phase, averaged over the steps of
 * the last dem_step call run with timing on (dem_set_timing; kernels are
 * then launched one by one and a step that does not re-sort still launches
 * the re-sort kernels, which return at once).  Phases:
 * [0] sort (scan, scatter, cell order, reorder)  [1] contact search
 * [2] candidate rows and history carry-over  [3] contact rule and force
 * [4] sum + integrate + bin (+ rectangle and line walls).
 * Returns the number of phases written (<= cap). */
int32_t dem_get_phase_times(dem_ctx* ctx, double* ms, int32_t cap);
dem_status dem_set_timing(dem_ctx* ctx, int32_t on);

/* Autotuner (orchestration): times every combination of the per-particle
 * kernels' block size {128, 256, 512} and the CUDA-graph length {8, 16, 32}
 * on the live state, `steps` steps each (at least 4), and keeps the fastest
 * for this context.  The timed steps advance the simulation like dem_step.
 * best_ms (may be NULL) receives the best time per step in milliseconds;
 * block and graph_steps (may be NULL) the chosen values. */
dem_status dem_autotune(dem_ctx* ctx, int64_t steps, double* best_ms,
                        int32_t* block, int32_t* graph_steps);

/* Layout tuner (orchestration).  Searches, on the live particles, the
 * candidate-list skin (per box a multiple of r_max: 0, 0.5 %, 1.5 % or 4 %),
 * the cell grid (the finest legal cells, 8 % and 18 % wider; Sec. 3.3: the
 * cell size trades the length of each particle's candidate loop against the
 * divergence of a warp and the cells it visits), the size split r_split (0,
 * or the box's 90 % or 97 % radius quantile), then the block size
 * {128, 256, 512} and the CUDA-graph length {8, 16, 32}, one parameter
 * after the other, keeping the best of each.  The re-sort interval follows
 * from the skin (a re-sort comes when a particle has moved about half of
 * it).  Each candidate runs `steps` steps (at least 4) from the state the
 * call started with, the first step's re-sort included; that state
 * (positions, velocities, spins, pair history) is put back after every
 * trial and at the end, so the call does not advance the simulation; wall
 * histories restart from zero.  The context keeps the fastest
 * configuration (dem_get_layout reads it per box).  The per-particle Collide
 * forms search only the block size and graph length.  out (may be NULL)
 * receives the choice. */
typedef struct {
  double ms_per_step;       /* device time per step of the chosen one      */
  double skin_over_rmax;    /* skin / r_max                                */
  double cell_scale;        /* cell edge / finest legal cell edge          */
  double rsplit_quantile;   /* 0 = one size class                          */
  int32_t block;
  int32_t graph_steps;
  int32_t trials;           /* configurations timed                        */
  int32_t pad;
} dem_tuning;
dem_status dem_autotune_layout(dem_ctx* ctx, int64_t steps, dem_tuning* out);

/* Measured arithmetic peaks of the current GPU (a measurement utility with
 * no counterpart in the paper): the FP32 and FP64 fused multiply-add rates,
 * 2 flops each, of a kernel that keeps eight independent FMA chains per
 * thread on eight 256-thread blocks per SM, timed with CUDA events on
 * `stream` after a warm-up launch.  They are the denominators of the
 * rooflines of arithmetic-bound kernels (the FP64 force path in
 * particular).  Synchronises the stream; allocates nothing. */
dem_status dem_measure_fma_rates(double* fp32_tflops, double* fp64_tflops, void* stream);

/* The layout of one box now in use: cells per axis, skin [m], r_split [m]. */
dem_status dem_get_layout(dem_ctx* ctx, int32_t box, int32_t ncell[3], double* skin,
                          double* r_split);

/* Kernel launches issued by a step that does not re-sort in a CUDA graph
 * (DEM_COLLIDE_COMPACT) or by any step (the per-particle forms re-sort
 * every step). */
int32_t dem_launches_per_step(const dem_ctx* ctx);

/* Re-sort statistics of the contact-list pipeline (DEM_COLLIDE_COMPACT):
 * out[0] re-sorts since dem_create, out[1] kernel launches a re-sort adds to
 * its step, out[2] candidate pairs in the current list, out[3] steps since
 * dem_create.  Zeros for the per-particle forms. */
dem_status dem_get_resort_stats(dem_ctx* ctx, int64_t out[4]);

/* Block until all queued work of the context finished; returns the sticky
 * device status. */
dem_status dem_sync(dem_ctx* ctx);

/* Description of the last failure on ctx (or of the last dem_create failure
 * when ctx is NULL).  The string lives until the next call on ctx. */
const char* dem_last_error(const dem_ctx* ctx);

/* Release all device memory and the context.  NULL is allowed. */
dem_status dem_destroy(dem_ctx* ctx);

int32_t dem_abi_version(void);

/* Contact detection for one small box without any device allocation.
 * (The paper has no counterpart: this is a library service.)
 *
 * Who needs it: callers that cannot allocate device memory when they need a
 * contact list -- code running inside another framework's memory pool or
 * under a fixed memory budget, code that must not grow its footprint after
 * start-up, or latency-critical code that must not call cudaMalloc (it can
 * synchronise the device).  dem_create allocates; this call does not: it
 * runs the same binning, sorting and search kernels as dem_step with all
 * scratch carved from one file-scope device array of 6,000,000 bytes that
 * every GPU loading this library holds until the process exits.  It calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *
 * Inputs (device memory of the current GPU; host pointers and memory of
 * another GPU are rejected with DEM_ERR_ARG): x (n x 3 FP64 positions [m]),
 * radius (n, each in (0, h/2] with h the narrowest cell edge L[a]/ncell[a];
 * DEM_ERR_ARG otherwise).  A non-finite position gives DEM_ERR_NONFINITE.
 * Host arrays: box lengths L, periodic flags and the cell grid ncell
 * (periodic axes need >= 3 cells).  The contact rule is DEM_MIXED's: the
 * position is rounded to 2^-60 m fixed point and a pair is in contact when
 * the single-precision test of dem_step accepts it.
 * Output: pairs (device, cap x 2 int32, 8-byte aligned) receives
 * (id_lo, id_hi) of every contact, id_lo < id_hi, each pair once, in an
 * order fixed by the cell grid (sort them for a canonical order); *count
 * (host) the number of contacts.
 * Limits: n <= 8192, ncell[0] * ncell[1] * ncell[2] <= 32768, at most
 * 131072 contacts (fewer if cap is smaller), and at most 32 partners found
 * by one particle in its half of the neighbour cells (its own cell's later
 * slots and the 13 cells after it); larger sizes are rejected with
 * DEM_ERR_ARG (sizes) or DEM_ERR_CAPACITY (contacts).
 * Runs on `stream` (cudaStream_t, NULL = legacy default) and returns after
 * synchronising it.  The first call on a device looks up the array's device
 * address (once per device, with that device current); make that first call
 * before any stream capture.  All calls share the one array, which keeps
 * the previous call's contents (each call clears what must start at zero):
 * calls that overlap on the GPU, from several streams or threads, race.
 * Errors are described by dem_last_error(NULL). */
dem_status dem_contacts_static(int64_t n, const double* x, const double* radius,
                               const double L[3], const int32_t periodic[3],
                               const int32_t ncell[3], int64_t cap,
                               int32_t* pairs, int64_t* count, void* stream);

/* Restitution parameter (Sec. 2: eta_n = eta_t = alpha(eps) sqrt(m* k_n
 * sqrt(dn)), alpha "a function of the coefficient of restitution", not
 * given in the paper).  The library defines alpha as the exact inverse of
 * the rebound of its own normal law: the scaled two-body equation
 * x'' = -x^{3/2} - alpha x^{1/4} x', x(0) = 0, x'(0) = 1, rebounds with
 * speed eps whatever the impact speed, mass or size.  Host-only functions;
 * they need no GPU.  dem_alpha_of_restitution(eps) for eps in (0, 1]
 * (NaN outside, or when eps is below the rebound of alpha = 4);
 * dem_restitution_of_alpha(alpha) for alpha >= 0 (0 = no rebound). */
double dem_alpha_of_restitution(double eps);
double dem_restitution_of_alpha(double alpha);

#ifdef __cplusplus
}
#endif
#endif /* DEM_GB300_H */
