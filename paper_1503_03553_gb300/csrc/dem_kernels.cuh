// dem_kernels.cuh -- CUDA kernels of one DEM time step (sm_103a).
//
// Per step (Nakahara & Washizawa, arXiv 1503.03553, Sec. 4.2 kernel list,
// re-laid out for one GB300):
//   scan of cell counts        -> cell starts          (CalcHash/BitonicSort)
//   k_scatter                  -> permutation by (Morton cell, id)
//   k_reorder                  -> state in sorted order (FindCellBoundsAndReorder)
//   k_candidates               -> search over half the neighbour cells (the
//                                 loops of Algorithm 1; the paper's first loop,
//                                 Sec. 3.4) for every pair within r_i + r_j +
//                                 skin: the candidate list (Sec. 3.4 split,
//                                 global)
//   k_rows                     -> each particle's candidates in partner-id
//                                 order
//   k_carry                    -> delta_t history carried to the new list
//                                 (InitializeContactIDs)
//   k_commit                   -> the sorted state and list become current
//   (the kernels above run only in a step that re-sorts: the first one, and
//    then whenever a particle has moved far enough for a pair outside the
//    list to reach contact; k_decide makes that call on the device)
//   k_pairs                    -> the contact rule on every candidate, ballot
//                                 compaction of the contacts, one lane per
//                                 contact: Eq. (1), Eq. (vt), Eq. (dt),
//                                 Coulomb cap (Collide)
//   k_gather_integrate         -> per-particle sum in partner-id order, floor
//                                 wall (CollideRectangle), gravity
//                                 (ForceGravity), symplectic Euler
//                                 (Integrate), next binning, skin test
#pragma once

#include <climits>

#include <type_traits>

#include "dem_common.cuh"

namespace dem {

// ---------------------------------------------------------------------------
// precision traits
// ---------------------------------------------------------------------------
template <int M> struct Tr;
template <> struct Tr<kMIXED> {
  using P = long long;  // fixed-point position (quanta)
  using R = float;      // force arithmetic
  using V4 = float4;    // (v, m) and (w, r)
  using PR = float4;    // predicate record: offset from the cell origin + r
  using DT = float2;    // one delta_t component as (hi, lo)
};
template <> struct Tr<kFP64> {
  using P = double;
  using R = double;
  using V4 = d4;
  using PR = d4;        // absolute position + radius
  using DT = double;
};
template <> struct Tr<kFP32> {
  using P = float;
  using R = float;
  using V4 = float4;
  using PR = float4;
  using DT = float;
};

// One parity of the per-slot particle state (slots sorted by cell).
struct PState {
  void* px;
  void* py;
  void* pz;
  void* vel;    // V4 (vx, vy, vz, m)
  void* omg;    // V4 (wx, wy, wz, r)
  void* posr;   // PR
  int* id;      // global id = box slot base + id within the box
  int* cellc;   // packed cell coordinates of the current position (set by
                // the sort and kept up to date by the integrator)
  int* cellx;   // packed cell coordinates at the last sort
  int* cellg;   // rank-space cell of the current position
  void* wx;     // floor-wall delta_t (DT); null when no box has a floor
  void* wy;
  void* wz;
};

// The candidate list of the contact-list pipeline: every pair within
// r_i + r_j + skin at the last re-sort (each pair once, in the block of the
// slot that found it), with the pair's tangential history.  A pair is in
// contact in a step when the contact rule accepts it then; between re-sorts
// the list is a superset of the contacts (the re-sort comes before any
// particle can have moved half the skin).  Two of them: the current one and
// the one a re-sort builds.
struct VList {
  int2* pair;   // storage slots (lower-id member, higher-id member)
  int2* hid;    // ids (lo, hi), lo < hi; written only when not null
  void* dx;     // delta_t after the last step, per component (DT), of a
  void* dy;     // pair in contact in that step
  void* dz;
  unsigned char* flag;  // 1: in contact in the last step (the history dx,
                        // dy, dz of a pair without it is not read)
  int* hs;      // by slot: first entry of the pairs the slot found ...
  int* oc;      // ... and how many (the slot's block of the list)
  int* count;   // entries (device scalar)
};

// One parity of the contact list of the per-particle Collide forms: the
// pairs of one step.
struct CList {
  int2* pair;   // storage slots (lo, hi) of that step
  int2* hid;    // global ids (lo, hi), lo < hi
  void* dx;     // delta_t after the step, per component (DT)
  void* dy;
  void* dz;
  int* hs;      // by slot: first entry of the contacts the slot found ...
  int* oc;      // ... and how many (the slot's block of the list)
  int* count;   // number of contacts (device scalar)
};

struct Dev {
  const BoxDev* boxes;
  const WallDev* walls;  // all boxes' rectangle and line walls
  int nwh;               // wall histories per slot (floor + walls, largest box)
  const int* slot_box;
  int N;         // slots over all boxes
  int K;         // row capacity per particle
  int Cmax;      // contact list capacity
  int M_lin;     // cells over all boxes
  int M_rank;    // cells + one free-slot cell per box
  int nbox;      // boxes (1: every slot is in box 0, no lookup needed)
  const int* rank_of_lin;  // box-local Morton rank of each linear cell
  const int* lin_of_rank;  // global linear cell of each rank cell, -1 = free
  int* ccount;   // per rank cell: particles in it (kept up to date by movers)
  int* cstart;   // per rank cell: first slot in the order being built
  const int* cstart_old;  // per rank cell: first slot in the current order
  int* ccur;     // per rank cell: scatter cursor of a cell that changed
  const unsigned char* chg;    // per rank cell: members changed since the
                               // last sort (set by the cell scan of a sort)
  unsigned char* collect;      // the same, collected by the integrator for
                               // the next sort
  int2* crange;  // per linear cell: (first slot, count)
  float4* cellbox;  // per linear cell, 2 entries: (lo.xyz, largest radius),
                    // (hi.xyz, 0): the bounding box of the members' centres
                    // as offsets from the cell origin; radius -1 if empty
  int* perm;     // scatter position -> old slot (cell order, not yet by id)
  int* pcell;    // scatter position -> linear cell
  int* row;      // N x K: partner slots a slot found (the search); the
                 // partner ids of its candidate row (contact-list pipeline,
                 // after the search)
  int* large;    // slots of the large particles of size-binned boxes (the
                 // search appends them; null when no box is size-binned)
  int* nlarge;   // their number (device scalar, reset by the reorder)
  int* icnt;     // contacts in which a slot was found by its partner
  int* prev;     // slot of each particle before this step's reorder
  int* next;     // the inverse: new slot of each slot before the reorder
                 // (contact-list pipeline; null otherwise)
  int2* inrow;   // N x K: the contacts in which a slot was found by its
                 // partner (any order): (list entry, partner id << 1 |
                 // 1 if this slot is the lower-id member)
  void* Fc;      // 2 V4 per contact (one record: 32 bytes in FP32, 64 in
                 // FP64): the force on the lower-id particle, then n x F
  void* Ffused;  // V4 per slot: contact force sum of the fused layout
  void* Tfused;  // V4 per slot: contact torque sum of the fused layout
  void* Fwall;   // V4 per slot: rectangle and line walls' force (k_walls)
  void* Twall;   // V4 per slot: their torque
  void* Fout;    // V4 per slot: total force of the last step
  void* Tout;    // V4 per slot: total torque of the last step
  // contact-list pipeline
  int* frow;     // N x K: every candidate pair of a slot (entry << 1 | 1 if
                 // the slot is the lower-id member), in increasing partner id
  int* fcnt;     // their number per slot
  void* xb;      // P per slot: position at the last re-sort (skin test);
  void* yb;      // null for the per-particle Collide forms
  void* zb;
  unsigned* vctl;        // control words (kCtl*)
  const unsigned* gate;  // re-sort kernels run only when *gate != 0 (null:
                         // always)
  unsigned* status;
  unsigned* diag;  // per box: max overlap / r_min, max |F_t| / (mu |F_n|)
  int* scan_bsum;
};

__device__ __forceinline__ void flag(unsigned* st, unsigned bit) {
  atomicOr(st, bit);
}

// a re-sort kernel whose gate is closed does nothing this step
__device__ __forceinline__ bool gated_off(const unsigned* gate) {
  return gate != nullptr && *(const volatile unsigned*)gate == 0u;
}

// ---------------------------------------------------------------------------
// small 3-vectors
// ---------------------------------------------------------------------------
template <typename R> struct v3 {
  R x, y, z;
};
template <typename R>
__device__ __forceinline__ v3<R> operator+(v3<R> a, v3<R> b) {
  return {a.x + b.x, a.y + b.y, a.z + b.z};
}
template <typename R>
__device__ __forceinline__ v3<R> operator-(v3<R> a, v3<R> b) {
  return {a.x - b.x, a.y - b.y, a.z - b.z};
}
template <typename R>
__device__ __forceinline__ v3<R> operator*(R s, v3<R> a) {
  return {s * a.x, s * a.y, s * a.z};
}
template <typename R>
__device__ __forceinline__ v3<R> operator*(v3<R> a, R s) {
  return {a.x * s, a.y * s, a.z * s};
}
template <typename R>
__device__ __forceinline__ R dot(v3<R> a, v3<R> b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <typename R>
__device__ __forceinline__ v3<R> cross(v3<R> a, v3<R> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename R>
__device__ __forceinline__ R norm(v3<R> a) {
  return sqrt(dot(a, a));
}
template <typename V>
__device__ __forceinline__ auto xyz(V v) -> v3<decltype(v.x)> {
  return {v.x, v.y, v.z};
}

// ---------------------------------------------------------------------------
// cell rule: exact floor division in fixed point; floor(x n / L) otherwise
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ int cell_coord(const BoxDev& B, int a,
                                          typename Tr<M>::P x);
template <>
__device__ __forceinline__ int cell_coord<kMIXED>(const BoxDev& B, int a,
                                                  long long X) {
  return clampi(floor_div64(X, B.Hq[a]), B.n[a]);
}
template <>
__device__ __forceinline__ int cell_coord<kFP64>(const BoxDev& B, int a,
                                                 double x) {
  return clampi((long long)floor(__dmul_rn(x, B.inv_h[a])), B.n[a]);
}
template <>
__device__ __forceinline__ int cell_coord<kFP32>(const BoxDev& B, int a,
                                                 float x) {
  return clampi((long long)floorf(__fmul_rn(x, B.inv_hf[a])), B.n[a]);
}

__device__ __forceinline__ int rank_cell(const Dev& d, const BoxDev& B, int cx,
                                         int cy, int cz) {
  int lin = (cz * B.n[1] + cy) * B.n[0] + cx;
  return B.rank_base + d.rank_of_lin[B.lin_base + lin];
}

template <int M>
__device__ __forceinline__ typename Tr<M>::P wrap_pos(const BoxDev& B, int a,
                                                      typename Tr<M>::P x);
template <>
__device__ __forceinline__ long long wrap_pos<kMIXED>(const BoxDev& B, int a,
                                                      long long X) {
  if (!B.periodic[a]) return X;
  long long L = B.Lq[a];
  if (X >= L || X < 0) X -= floor_div64(X, L) * L;
  return X;
}
template <>
__device__ __forceinline__ double wrap_pos<kFP64>(const BoxDev& B, int a,
                                                  double x) {
  if (!B.periodic[a]) return x;
  double L = B.L[a];
  int guard = 0;
  while (x >= L && guard++ < 64) x -= L;
  while (x < 0.0 && guard++ < 128) x += L;
  return x;
}
template <>
__device__ __forceinline__ float wrap_pos<kFP32>(const BoxDev& B, int a,
                                                 float x) {
  if (!B.periodic[a]) return x;
  float L = B.Lf[a];
  int guard = 0;
  while (x >= L && guard++ < 64) x -= L;
  while (x < 0.0f && guard++ < 128) x += L;
  return x;
}

template <int M>
__device__ __forceinline__ typename Tr<M>::R pos_metres(typename Tr<M>::P p) {
  return (typename Tr<M>::R)p;
}

// ---------------------------------------------------------------------------
// set particles: id order -> slots pbase + id; initial binning
// ---------------------------------------------------------------------------
template <int M>
__global__ void k_set_particles(Dev d, PState s, int box, int n,
                                const double* __restrict__ x,
                                const double* __restrict__ v,
                                const double* __restrict__ w,
                                const double* __restrict__ r) {
  using T = Tr<M>;
  using P = typename T::P;
  using R = typename T::R;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const BoxDev& B = d.boxes[box];
  int slot = B.pbase + k;
  P p[3];
  int c[3];
  bool bad = false;
  for (int a = 0; a < 3; ++a) {
    double xa = x[3 * k + a];
    if (!isfinite(xa)) bad = true;
    if (M == kMIXED) {
      double sx = xa * 0x1p60;
      if (!(fabs(sx) < 0x1p62)) { bad = true; sx = 0.0; }
      p[a] = (P)wrap_pos<kMIXED>(B, a, __double2ll_rn(sx));
    } else if (M == kFP64) {
      p[a] = (P)wrap_pos<kFP64>(B, a, bad ? 0.0 : xa);
    } else {
      p[a] = (P)wrap_pos<kFP32>(B, a, bad ? 0.0f : (float)xa);
    }
    c[a] = cell_coord<M>(B, a, p[a]);
  }
  if (bad) flag(d.status, kStNonFinite);
  ((P*)s.px)[slot] = p[0];
  ((P*)s.py)[slot] = p[1];
  ((P*)s.pz)[slot] = p[2];
  double rr = r[k];
  double m = B.density * (4.0 / 3.0) * 3.14159265358979323846 * rr * rr * rr;
  using V4 = typename T::V4;
  st4((V4*)s.vel + slot, mk4<R>((R)v[3 * k], (R)v[3 * k + 1], (R)v[3 * k + 2], (R)m));
  st4((V4*)s.omg + slot, mk4<R>((R)w[3 * k], (R)w[3 * k + 1], (R)w[3 * k + 2], (R)rr));
  s.id[slot] = slot;
  s.cellc[slot] = pack_cell(c[0], c[1], c[2]);
  s.cellx[slot] = pack_cell(c[0], c[1], c[2]);
  int g = rank_cell(d, B, c[0], c[1], c[2]);
  s.cellg[slot] = g;
  atomicAdd(&d.ccount[g], 1);
  if (s.wx) {
    using DT = typename T::DT;
    for (int q = 0; q < d.nwh; ++q) {
      const size_t h = (size_t)slot * d.nwh + q;
      ((DT*)s.wx)[h] = DT{};
      ((DT*)s.wy)[h] = DT{};
      ((DT*)s.wz)[h] = DT{};
    }
  }
}

// The contact rule's record of a particle at position p in cell c: its
// offset from the cell's origin (DEM_MIXED, rounded as the sort rounds it) or
// its position, and its radius r.
template <int M>
__device__ __forceinline__ typename Tr<M>::PR pos_record(const BoxDev& B,
                                                         const typename Tr<M>::P* p,
                                                         const int* c, typename Tr<M>::R r) {
  typename Tr<M>::PR pr;
  if (M == kMIXED) {
    pr.x = __fmul_rn(i64_to_f32_rn((long long)p[0] - (long long)c[0] * B.Hq[0]), kQ);
    pr.y = __fmul_rn(i64_to_f32_rn((long long)p[1] - (long long)c[1] * B.Hq[1]), kQ);
    pr.z = __fmul_rn(i64_to_f32_rn((long long)p[2] - (long long)c[2] * B.Hq[2]), kQ);
  } else {
    pr.x = p[0];
    pr.y = p[1];
    pr.z = p[2];
  }
  pr.w = r;
  return pr;
}

// Skin test: whether a particle now at p moved farther than the box's limit
// since the last re-sort, where it was at q (the squared displacement
// rounded up); the caller checks that the box keeps a skin.
template <int M>
__device__ __forceinline__ bool skin_exceeded(const BoxDev& B, const typename Tr<M>::P* p,
                                              const typename Tr<M>::P* q) {
  float d2;
  if (M == kMIXED) {
    float acc = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      long long D = (long long)p[a] - (long long)q[a];
      if (B.periodic[a]) {
        const long long L = B.Lq[a], h = L >> 1;
        if (D > h) D -= L;
        else if (D < -h) D += L;
      }
      const float f = __fmul_rn(i64_to_f32_rn(D), kQ);
      acc = __fmaf_ru(f, f, acc);
    }
    d2 = __fmul_ru(acc, 1.000001f);
  } else {
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double D = (double)p[a] - (double)q[a];
      if (B.periodic[a]) {
        if (D > B.half_L[a]) D -= B.L[a];
        else if (D < -B.half_L[a]) D += B.L[a];
      }
      acc += D * D;
    }
    d2 = __fmul_ru(__double2float_ru(acc), 1.000001f);
  }
  return d2 > B.disp2_lim;
}

// whether slot i's box runs the skin test (a candidate list with a skin)
__device__ __forceinline__ bool has_skin_test(const Dev& d, const BoxDev& B) {
  return d.xb && B.disp2_lim >= 0.0f;
}

// Overwrite x / v / w of live particles (id order), keep everything else.
// New positions (track = 1, the contact-list pipeline) are handled as the
// integrator handles a step's: the contact rule's record and the current
// cell follow them, a particle that changed cell updates the counts and
// flags both cells for the next sort, and one that moved beyond the skin
// limit asks for a re-sort; otherwise (the per-particle forms, which sort
// every step) the next sort starts from every cell.
template <int M>
__global__ void k_set_state(Dev d, PState s, int box, int n,
                            const double* __restrict__ x,
                            const double* __restrict__ v,
                            const double* __restrict__ w, int track) {
  using T = Tr<M>;
  using P = typename T::P;
  using R = typename T::R;
  using V4 = typename T::V4;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  const BoxDev& B = d.boxes[box];
  if (t >= B.nlive) return;
  int slot = B.pbase + t;
  int k = s.id[slot] - B.pbase;  // id held by this slot
  if (x) {
    P p[3];
    int c[3];
    for (int a = 0; a < 3; ++a) {
      double xa = x[3 * k + a];
      if (M == kMIXED) {
        double sx = xa * 0x1p60;
        if (!(fabs(sx) < 0x1p62)) { flag(d.status, kStNonFinite); sx = 0.0; }
        p[a] = (P)wrap_pos<kMIXED>(B, a, __double2ll_rn(sx));
      } else if (M == kFP64) {
        p[a] = (P)wrap_pos<kFP64>(B, a, xa);
      } else {
        p[a] = (P)wrap_pos<kFP32>(B, a, (float)xa);
      }
      c[a] = cell_coord<M>(B, a, p[a]);
    }
    ((P*)s.px)[slot] = p[0];
    ((P*)s.py)[slot] = p[1];
    ((P*)s.pz)[slot] = p[2];
    int old = s.cellg[slot];
    int g = rank_cell(d, B, c[0], c[1], c[2]);
    if (g != old) {
      atomicSub(&d.ccount[old], 1);
      atomicAdd(&d.ccount[g], 1);
      if (track) {
        d.collect[old] = 1;
        d.collect[g] = 1;
      }
    }
    s.cellg[slot] = g;
    s.cellc[slot] = pack_cell(c[0], c[1], c[2]);
    if (track) {
      using PR = typename T::PR;
      st4((PR*)s.posr + slot, pos_record<M>(B, p, c, (R)((const V4*)s.omg)[slot].w));
      if (has_skin_test(d, B)) {
        const P q[3] = {((const P*)d.xb)[slot], ((const P*)d.yb)[slot], ((const P*)d.zb)[slot]};
        if (skin_exceeded<M>(B, p, q)) d.vctl[kCtlRequest] = 1u;
      }
    } else {
      s.cellx[slot] = pack_cell(c[0], c[1], c[2]);
    }
  }
  if (v) {
    V4 q = ((V4*)s.vel)[slot];
    q.x = (R)v[3 * k];
    q.y = (R)v[3 * k + 1];
    q.z = (R)v[3 * k + 2];
    st4((V4*)s.vel + slot, q);
  }
  if (w) {
    V4 q = ((V4*)s.omg)[slot];
    q.x = (R)w[3 * k];
    q.y = (R)w[3 * k + 1];
    q.z = (R)w[3 * k + 2];
    st4((V4*)s.omg + slot, q);
  }
}

// ---------------------------------------------------------------------------
// device-wide exclusive scan (three passes, deterministic)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;  // 1024
constexpr int kScanTopThreads = 1024;
constexpr int kScanTopItems = 16;                    // <= 16384 tiles

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// block-wide exclusive scan of one value per thread; returns the prefix and
// the block total in *total
template <int NT, typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* total) {
  __shared__ T wsum[NT / 32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T inc = warp_incl_scan(v);
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T s = lane < NT / 32 ? wsum[lane] : T(0);
    T si = warp_incl_scan(s);
    if (lane < NT / 32) wsum[lane] = si - s;
    if (lane == NT / 32 - 1) *total = si;
  }
  __syncthreads();
  T r = wsum[wid] + inc - v;
  __syncthreads();
  return r;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(const T* __restrict__ in, int n, T* __restrict__ bsum, const unsigned* gate) {
  if (gated_off(gate)) return;
  int base = blockIdx.x * kScanTile;
  T s = 0;
  for (int k = threadIdx.x; k < kScanTile; k += kScanThreads) {
    int idx = base + k;
    if (idx < n) s += in[idx];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ T ws[kScanThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    T t = 0;
    for (int q = 0; q < kScanThreads / 32; ++q) t += ws[q];
    bsum[blockIdx.x] = t;
  }
}

// Exclusive scan of the tile sums in place.  *total gets the grand total
// (low 32 bits for packed 64-bit counts), clamped to cap (a larger total sets
// status bit over_bit).
template <typename T>
__global__ void __launch_bounds__(kScanTopThreads)
k_scan_top(T* bsum, int nb, int* total, int cap, unsigned* status,
           unsigned over_bit, const unsigned* gate) {
  if (gated_off(gate)) return;
  __shared__ T tot;
  T v[kScanTopItems];
  T s = 0;
  int base = threadIdx.x * kScanTopItems;
#pragma unroll
  for (int q = 0; q < kScanTopItems; ++q) {
    int idx = base + q;
    v[q] = idx < nb ? bsum[idx] : T(0);
    s += v[q];
  }
  T pre = block_excl_scan<kScanTopThreads, T>(s, &tot);
#pragma unroll
  for (int q = 0; q < kScanTopItems; ++q) {
    int idx = base + q;
    if (idx < nb) bsum[idx] = pre;
    pre += v[q];
  }
  if (threadIdx.x == 0 && total) {
    long long t = (long long)(tot & T(0xffffffffu));
    if (t > cap) {
      atomicOr(status, over_bit);
      t = cap;
    }
    *total = (int)t;
  }
}

// Per tile: coalesced load to shared memory, kScanItems consecutive items
// per thread, block scan, then the epilogue is called once per item
// epi(index, count, exclusive_prefix) with coalesced indices.
template <typename T, class Epi>
__global__ void __launch_bounds__(kScanThreads)
k_scan_apply(const T* __restrict__ in, int n, const T* __restrict__ bsum,
             Epi epi, const unsigned* gate) {
  if (gated_off(gate)) return;
  __shared__ T buf[kScanTile];
  __shared__ T tot;
  int base = blockIdx.x * kScanTile;
  for (int k = threadIdx.x; k < kScanTile; k += kScanThreads) {
    int idx = base + k;
    buf[k] = idx < n ? in[idx] : T(0);
  }
  __syncthreads();
  T v[kScanItems];
  T s = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    v[q] = buf[threadIdx.x * kScanItems + q];
    s += v[q];
  }
  T pre = block_excl_scan<kScanThreads, T>(s, &tot) + bsum[blockIdx.x];
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    buf[threadIdx.x * kScanItems + q] = pre;
    pre += v[q];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kScanTile; k += kScanThreads) {
    int idx = base + k;
    if (idx < n) epi(idx, in[idx], buf[k]);
  }
}

// cell counts -> cell starts (rank order) and (start, count) by linear cell
// For a cell whose members changed since the last sort (flag collected by
// the integrator) it marks the cell changed for this sort and zeroes the
// scatter cursor; it clears the collected flag and resets the cell's box.
struct CellEpi {
  int* cstart;
  int2* crange;
  float4* cellbox;  // reset for the reorder's atomics (may be null)
  const int* lin_of_rank;
  unsigned char* collect;  // changed since the last sort (read and cleared)
  unsigned char* chg;      // changed, for this sort's scatter and reorder
  int* ccur;
  __device__ void operator()(int g, int cnt, int pre) const {
    cstart[g] = pre;
    const bool changed = collect[g] != 0;
    chg[g] = changed ? 1 : 0;
    if (changed) {
      ccur[g] = 0;
      collect[g] = 0;
    }
    int lin = lin_of_rank[g];
    if (lin >= 0) {
      crange[lin] = make_int2(pre, cnt);
      if (cellbox) {
        cellbox[2 * lin] = make_float4(INFINITY, INFINITY, INFINITY, -1.0f);
        cellbox[2 * lin + 1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      }
    }
  }
};

// ---------------------------------------------------------------------------
// counting sort, pass 1: each particle takes a position in its cell's range
// and records its old slot and its cell there.  A cell whose members did not
// change since the last sort keeps their order (sorted by id): position =
// new start + old position in the cell, no atomics.  Particles of a changed
// cell take positions in atomic order; pass 2 sorts those.
// ---------------------------------------------------------------------------
__global__ void k_scatter(Dev d, PState a) {
  if (gated_off(d.gate)) return;
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.N) return;
  const BoxDev& B = d.boxes[d.slot_box[s]];
  if (s - B.pbase >= B.nlive) return;
  const int g = a.cellg[s];
  int pos;
  if (!d.chg[g]) {
    pos = d.cstart[g] + (s - d.cstart_old[g]);
  } else {
    const int cnt = d.ccount[g];  // loaded beside the atomic, not after it
    const int k = atomicAdd(&d.ccur[g], 1);
    if (k >= cnt) {  // counts out of step: report
      flag(d.status, kStInconsistent);
      return;
    }
    pos = d.cstart[g] + k;
  }
  if (pos < 0 || pos >= d.N) {
    flag(d.status, kStInconsistent);
    return;
  }
  d.perm[pos] = s;
  d.pcell[pos] = g;
}

// ---------------------------------------------------------------------------
// counting sort, pass 2: in a changed cell each particle's final slot is the
// cell's start plus the number of cell-mates with a smaller id, so the slot
// order is (Morton rank of the cell, id) whatever the atomic order of pass 1;
// in an unchanged cell pass 1 already placed it.  The state moves there and
// the predicate record is built.
// ---------------------------------------------------------------------------
template <int M>
__global__ void k_reorder(Dev d, PState a, PState b, int* cursor) {
  using T = Tr<M>;
  using P = typename T::P;
  using V4 = typename T::V4;
  using PR = typename T::PR;
  if (gated_off(d.gate)) return;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // scatter position
  if (q == 0 && cursor) *cursor = 0;  // the search allocates list entries
  if (q == 0 && d.nlarge) *d.nlarge = 0;  // ... and appends large particles
  if (q < d.N && d.icnt) d.icnt[q] = 0;  // the search counts into it
  // this particle's contribution to its cell's box: offset from the cell
  // origin (lo) and (hi), radius; identities for lanes without a particle
  int lin = -1;
  float blo[3] = {INFINITY, INFINITY, INFINITY}, bhi[3] = {0.0f, 0.0f, 0.0f};
  float brad = -1.0f;
  if (q < d.N) {
    const BoxDev& B = d.boxes[d.slot_box[q]];
    if (q - B.pbase < B.nlive) {
      const int s = d.perm[q];
      const int g = d.pcell[q];
      lin = d.lin_of_rank[g];
      const bool changed = d.chg[g] != 0;
      const int key = a.id[s];
      int t = q;  // final slot
      if (changed) {
        // the cell-mates' ids, eight at a time: their scatter entries, then
        // their ids, each batch of loads in flight together
        const int2 rg = d.crange[lin];
        const int end = rg.x + rg.y;
        int rank = 0;
        for (int u0 = rg.x; u0 < end; u0 += 8) {
          int pu[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) pu[k] = u0 + k < end ? d.perm[u0 + k] : -1;
#pragma unroll
          for (int k = 0; k < 8; ++k) rank += (pu[k] >= 0 && a.id[pu[k]] < key) ? 1 : 0;
        }
        t = rg.x + rank;
      }
      if (d.prev) d.prev[t] = s;
      if (d.next) d.next[s] = t;
      P x = ((const P*)a.px)[s], y = ((const P*)a.py)[s], z = ((const P*)a.pz)[s];
      ((P*)b.px)[t] = x;
      ((P*)b.py)[t] = y;
      ((P*)b.pz)[t] = z;
      V4 vel = ld4((const V4*)a.vel + s);
      V4 om = ld4((const V4*)a.omg + s);
      st4((V4*)b.vel + t, vel);
      st4((V4*)b.omg + t, om);
      b.id[t] = key;
      const int cc = a.cellc[s];  // the current cell, kept by the integrator
      b.cellc[t] = cc;
      b.cellx[t] = cc;            // the cell this sort used
      b.cellg[t] = g;
      if (a.wx) {
        using DT = typename T::DT;
        for (int w = 0; w < d.nwh; ++w) {
          const size_t hs = (size_t)s * d.nwh + w, ht = (size_t)t * d.nwh + w;
          ((DT*)b.wx)[ht] = ((const DT*)a.wx)[hs];
          ((DT*)b.wy)[ht] = ((const DT*)a.wy)[hs];
          ((DT*)b.wz)[ht] = ((const DT*)a.wz)[hs];
        }
      }
      int cx, cy, cz;
      unpack_cell(cc, cx, cy, cz);
      PR pr;
      float o[3];
      if (M == kMIXED) {
        long long X = (long long)x, Y = (long long)y, Z = (long long)z;
        pr.x = __fmul_rn(i64_to_f32_rn(X - (long long)cx * B.Hq[0]), kQ);
        pr.y = __fmul_rn(i64_to_f32_rn(Y - (long long)cy * B.Hq[1]), kQ);
        pr.z = __fmul_rn(i64_to_f32_rn(Z - (long long)cz * B.Hq[2]), kQ);
        o[0] = pr.x;
        o[1] = pr.y;
        o[2] = pr.z;
      } else {
        pr.x = x;
        pr.y = y;
        pr.z = z;
        o[0] = (float)((double)x - (double)cx * B.h[0]);
        o[1] = (float)((double)y - (double)cy * B.h[1]);
        o[2] = (float)((double)z - (double)cz * B.h[2]);
      }
      pr.w = om.w;
      st4((PR*)b.posr + t, pr);
      // a negative offset (a centre outside its clamped cell on an open
      // axis) leaves that side of the box open: -inf below, 0 above
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        blo[c] = o[c] >= 0.0f ? o[c] : -INFINITY;
        bhi[c] = o[c] >= 0.0f ? o[c] : 0.0f;
      }
      brad = (float)om.w;
    }
  }
  if (!d.cellbox) return;
  // The cell boxes for the search's pruning: a reduction over each run of
  // lanes in the same cell (scatter positions of a cell are consecutive),
  // then one set of atomics per run.  All stored values are non-negative
  // floats or -inf, which order like their bit patterns as signed ints.
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  unsigned same = 0u;  // bit k: the lane 2^k ahead is in the same cell
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int o = 1 << k;
    const int other = __shfl_down_sync(full, lin, o);
    if (lane + o < 32 && other == lin) same |= 1u << k;
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int o = 1 << k;
    const bool take = (same >> k) & 1u;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float l2 = __shfl_down_sync(full, blo[c], o);
      const float h2 = __shfl_down_sync(full, bhi[c], o);
      if (take) {
        blo[c] = fminf(blo[c], l2);
        bhi[c] = fmaxf(bhi[c], h2);
      }
    }
    const float r2 = __shfl_down_sync(full, brad, o);
    if (take) brad = fmaxf(brad, r2);
  }
  const int prev_lin = __shfl_up_sync(full, lin, 1);
  if (lin >= 0 && (lane == 0 || prev_lin != lin)) {
    int* box = (int*)(d.cellbox + 2 * lin);
    atomicMin(box + 0, __float_as_int(blo[0]));
    atomicMin(box + 1, __float_as_int(blo[1]));
    atomicMin(box + 2, __float_as_int(blo[2]));
    atomicMax(box + 3, __float_as_int(brad));
    atomicMax(box + 4, __float_as_int(bhi[0]));
    atomicMax(box + 5, __float_as_int(bhi[1]));
    atomicMax(box + 6, __float_as_int(bhi[2]));
  }
}

// ---------------------------------------------------------------------------
// contact predicates (must match the oracle's rounding bit for bit)
// ---------------------------------------------------------------------------
// fixed rule: dx = (o_j - o_i) + shift, |d|^2 = (dx dx + dy dy) + dz dz
__device__ __forceinline__ bool pred_fixed(float4 pi, float4 pj, float sx,
                                           float sy, float sz) {
  float dx = __fadd_rn(__fsub_rn(pj.x, pi.x), sx);
  float dy = __fadd_rn(__fsub_rn(pj.y, pi.y), sy);
  float dz = __fadd_rn(__fsub_rn(pj.z, pi.z), sz);
  float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)),
                       __fmul_rn(dz, dz));
  float R = __fadd_rn(pi.w, pj.w);
  return d2 < __fmul_rn(R, R);
}

// The same rule on the packed FP32x2 path (two lanes of one instruction,
// each rounded as its scalar counterpart): (dx, dy) = ((x_j, y_j) +
// (-x_i, -y_i)) + (sx, sy) and (dz, R) = ((z_j, r_j) + (-z_i, r_i)) +
// (sz, skin), then the squares, (dx^2 + dy^2) + dz^2 < R^2.  a - b is
// a + (-b) exactly, r_j + r_i = r_i + r_j, and R + 0 = R for R >= 0: with
// skin = 0 bit for bit pred_fixed; with skin > 0 the reach r_i + r_j + skin
// of a re-sort's candidate test, which accepts every pair pred_fixed accepts
// (the same d^2 against a square that is at least as large).
__device__ __forceinline__ bool pred_fixed_packed(float4 pj, float2 nxy, float2 nzw,
                                                  float2 sxy, float2 sz0) {
  const float2 u = __fadd2_rn(__fadd2_rn(make_float2(pj.x, pj.y), nxy), sxy);
  const float2 t = __fadd2_rn(__fadd2_rn(make_float2(pj.z, pj.w), nzw), sz0);
  const float2 uu = __fmul2_rn(u, u);
  const float2 tt = __fmul2_rn(t, t);
  return __fadd_rn(__fadd_rn(uu.x, uu.y), tt.x) < tt.y;
}

__device__ __forceinline__ double min_image(double d, const BoxDev& B, int a) {
  if (B.periodic[a]) {
    if (d > B.half_L[a]) d = __dsub_rn(d, B.L[a]);
    else if (d < -B.half_L[a]) d = __dadd_rn(d, B.L[a]);
  }
  return d;
}
__device__ __forceinline__ float min_image(float d, const BoxDev& B, int a) {
  if (B.periodic[a]) {
    if (d > B.half_Lf[a]) d = __fsub_rn(d, B.Lf[a]);
    else if (d < -B.half_Lf[a]) d = __fadd_rn(d, B.Lf[a]);
  }
  return d;
}
// absolute-position rule (DEM_FP64, DEM_FP32); skin > 0 widens the reach to
// r_i + r_j + skin (the candidate test of a re-sort; skin = 0 is the
// contact rule itself)
__device__ __forceinline__ bool pred_abs(const d4& pi, const d4& pj,
                                         const BoxDev& B, float skin = 0.0f) {
  double dx = min_image(__dsub_rn(pj.x, pi.x), B, 0);
  double dy = min_image(__dsub_rn(pj.y, pi.y), B, 1);
  double dz = min_image(__dsub_rn(pj.z, pi.z), B, 2);
  double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                        __dmul_rn(dz, dz));
  double R = __dadd_rn(__dadd_rn(pi.w, pj.w), (double)skin);
  return d2 < __dmul_rn(R, R);
}
__device__ __forceinline__ bool pred_abs(const float4& pi, const float4& pj,
                                         const BoxDev& B, float skin = 0.0f) {
  float dx = min_image(__fsub_rn(pj.x, pi.x), B, 0);
  float dy = min_image(__fsub_rn(pj.y, pi.y), B, 1);
  float dz = min_image(__fsub_rn(pj.z, pi.z), B, 2);
  float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)),
                       __fmul_rn(dz, dz));
  float R = __fadd_rn(__fadd_rn(pi.w, pj.w), skin);
  return d2 < __fmul_rn(R, R);
}

// Neighbour cell at step s (|s| <= w) along axis a from cell c: false when
// it lies outside a non-periodic box.  *shift gets the fixed-rule shift in
// metres, (float)((cn - c) H + image L) with image = -1 / +1 when the step
// wraps below 0 / above n - 1 (the oracle's rounding, exactly).
__device__ __forceinline__ bool axis_step(const BoxDev& B, int a, int c, int s,
                                          int& cn, float& shift) {
  const int n = B.n[a];
  cn = c + s;
  int k = s + 1;  // fixed-rule shift (cn - c) H + image L, tabulated per box
  if (cn < 0) {
    if (!B.periodic[a]) return false;
    cn += n;
    k = 3;
  } else if (cn >= n) {
    if (!B.periodic[a]) return false;
    cn -= n;
    k = 4;
  }
  shift = B.shift[a][k];
  return true;
}

// ---------------------------------------------------------------------------
// contact search: one thread per particle over half of the 27 neighbour
// cells (Algorithm 1 loops, each pair tested once): its own cell from the
// next slot on and the 13 cells after it in (dz, dy, dx) order.  With at
// least 3 cells on every periodic axis each pair of distinct cells is then
// one step apart in exactly one direction, and the predicate is exactly
// antisymmetric, so the pairs found are the pairs of the full stencil.
// Found partners go into the particle's row.  The same kernel then writes
// the dense contact list: each warp takes a block of list entries for all
// its particles' contacts with one atomic add on the list length (the
// warp's position in the list depends on timing, the content of every
// entry does not) and a warp scan places each particle's contacts there.
// Each contact's entry index also goes into the partner's incoming row, at
// a position taken from the partner's incoming count.
// Pass 1 decides, with independent loads, which neighbour cells can hold a
// contact: a cell is skipped when its nearest point is farther than r_i plus
// the largest radius in that cell (0.1 % margin, far above rounding).
// Pass 2 tests the candidates of the kept cells in (dz, dy, dx) order, eight
// at a time so that eight loads are in flight.
// ---------------------------------------------------------------------------

// Size classes of a size-binned box: a particle is large when its radius,
// rounded to FP32, exceeds the box's r_split (every kernel decides it with
// this one expression).
__device__ __forceinline__ bool is_large(float r, float rs) { return r > rs; }
__device__ __forceinline__ bool is_large(double r, float rs) { return (float)r > rs; }

// the search of one live slot: partners into its row, returns how many.
// kSplit: the slot is small in a size-binned box; large candidates are
// skipped (the large particles find those pairs) and the pruning bounds the
// partners' radii by r_split.
template <int M, bool kSplit>
__device__ __forceinline__ int search_row(const Dev& d, const PState& b, const BoxDev& B,
                                          int i) {
  using T = Tr<M>;
  using PR = typename T::PR;
  const PR* __restrict__ posr = (const PR*)b.posr;
  const int2* __restrict__ crange = d.crange;
  const float4* __restrict__ cellbox = d.cellbox;
  const PR pi = ld4(posr + i);
  int c[3];
  unpack_cell(b.cellc[i], c[0], c[1], c[2]);
  // Per axis: squared gaps from the particle to the lower and upper
  // neighbour cell, the neighbour cells' offsets in the linear cell index
  // and their fixed-rule shifts (only the steps the half stencil takes:
  // z 0/+1, y and x -1/0/+1); invalid steps (out of an open box) clear bits
  // of 'valid' (bit 3a + st for step st - 1 along axis a).
  float g2lo[3], g2hi[3], oi[3];
  unsigned valid = 0u;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float o, hc = c[a] == B.n[a] - 1 ? B.hcell[a][1] : B.hcell[a][0];
    if (M == kMIXED) o = (float)(a == 0 ? pi.x : a == 1 ? pi.y : pi.z);
    else o = (float)((double)(a == 0 ? pi.x : a == 1 ? pi.y : pi.z) - (double)c[a] * B.h[a]);
    oi[a] = o;
    const float gl = fmaxf(o, 0.0f), gh = fmaxf(hc - o, 0.0f);
    g2lo[a] = gl * gl;
    g2hi[a] = gh * gh;
    const bool per = B.periodic[a] != 0;
    valid |= (per || c[a] > 0 ? 1u : 0u) << (3 * a);
    valid |= 1u << (3 * a + 1);
    valid |= (per || c[a] < B.n[a] - 1 ? 1u : 0u) << (3 * a + 2);
  }
  const int n0 = B.n[0], n01 = B.n[0] * B.n[1];
  const bool xw0 = c[0] == 0, xw2 = c[0] == B.n[0] - 1;
  const bool yw0 = c[1] == 0, yw2 = c[1] == B.n[1] - 1;
  const bool zw2 = c[2] == B.n[2] - 1;
  const int X0 = xw0 ? B.n[0] - 1 : c[0] - 1, X1 = c[0], X2 = xw2 ? 0 : c[0] + 1;
  const int Y0 = (yw0 ? B.n[1] - 1 : c[1] - 1) * n0, Y1 = c[1] * n0,
            Y2 = (yw2 ? 0 : c[1] + 1) * n0;
  const int Z1 = B.lin_base + c[2] * n01, Z2 = B.lin_base + (zw2 ? 0 : c[2] + 1) * n01;
  const float ri = (float)pi.w;
  // Pass 1: a neighbour cell is kept when it holds particles and the bounding
  // box of their centres lies within r_i plus the largest radius in it
  // (0.1 % margin, far above the rounding of these FP32 gaps); the box's
  // largest radius screens cells by the cell faces first, before any load,
  // and the loads left are independent of one another.
  // the largest radius a partner can have
  const float rp = kSplit ? fminf(B.rmax_f, B.rsplit_f) : B.rmax_f;
  const float skin = B.skin_f;
  const float rb = 1.001f * (ri + rp + skin);
  const float rb2 = rb * rb;
  unsigned keep = 0u;
#pragma unroll
  for (int k = 13; k < 27; ++k) {
    const int kz = k / 9, ky = (k / 3) % 3, kx = k % 3;
    const float g2 = (kz == 2 ? g2hi[2] : 0.0f) + (ky == 0 ? g2lo[1] : ky == 2 ? g2hi[1] : 0.0f) +
                     (kx == 0 ? g2lo[0] : kx == 2 ? g2hi[0] : 0.0f);
    if (((valid >> (6 + kz)) & (valid >> (3 + ky)) & (valid >> kx) & 1u) && g2 <= rb2) {
      const int lin = (kz == 2 ? Z2 : Z1) + (ky == 0 ? Y0 : ky == 1 ? Y1 : Y2) +
                      (kx == 0 ? X0 : kx == 1 ? X1 : X2);
      const float4 blo = __ldg(cellbox + 2 * lin), bhi = __ldg(cellbox + 2 * lin + 1);
      // the neighbour cell's origin relative to this particle's cell origin
      float sh[3];
      if (M == kMIXED) {
        sh[2] = kz == 2 ? B.shift[2][zw2 ? 4 : 2] : 0.0f;
        sh[1] = ky == 1 ? 0.0f : (ky == 0 ? B.shift[1][yw0 ? 3 : 0] : B.shift[1][yw2 ? 4 : 2]);
        sh[0] = kx == 1 ? 0.0f : (kx == 0 ? B.shift[0][xw0 ? 3 : 0] : B.shift[0][xw2 ? 4 : 2]);
      } else {
        sh[2] = (float)(kz - 1) * (float)B.h[2];
        sh[1] = (float)(ky - 1) * (float)B.h[1];
        sh[0] = (float)(kx - 1) * (float)B.h[0];
      }
      const float b_lo[3] = {blo.x, blo.y, blo.z}, b_hi[3] = {bhi.x, bhi.y, bhi.z};
      float gb2 = 0.0f;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float gap = fmaxf(fmaxf(b_lo[a] + sh[a] - oi[a], oi[a] - (b_hi[a] + sh[a])), 0.0f);
        gb2 += gap * gap;
      }
      const float reach = 1.001f * (ri + (kSplit ? fminf(blo.w, rp) : blo.w) + skin);  // blo.w < 0: empty
      if (blo.w >= 0.0f && gb2 <= reach * reach) keep |= 1u << k;
    }
  }
  int own = 0;
  const int K = d.K;
  int* rowp = d.row + (size_t)i * K;
  bool over = false;
  // Pass 2, warp-uniform: each iteration every lane tests its next eight
  // candidates, first moving on to its next kept cell when the current one is
  // exhausted; one reconvergence point per iteration keeps the lanes of a
  // warp testing together (iterations ~ the largest per-lane candidate count).
  const unsigned wmask = __activemask();
  int j = 0, e = 0;
  float sx = 0.f, sy = 0.f, sz = 0.f;
  while (__any_sync(wmask, j < e || keep != 0u)) {
    if (j >= e && keep != 0u) {
      const int k = __ffs(keep) - 1;
      keep &= keep - 1u;
      const int kz = k >= 18 ? 2 : 1, r9 = k - 9 * kz;
      const int ky = r9 >= 6 ? 2 : (r9 >= 3 ? 1 : 0), kx = r9 - 3 * ky;
      const int lin = (kz == 2 ? Z2 : Z1) + (ky == 0 ? Y0 : ky == 1 ? Y1 : Y2) +
                      (kx == 0 ? X0 : kx == 1 ? X1 : X2);
      const int2 cr = __ldg(crange + lin);
      j = k == 13 ? i + 1 : cr.x;  // own cell: later slots only
      e = cr.x + cr.y;
      if (M == kMIXED) {
        sz = kz == 2 ? B.shift[2][zw2 ? 4 : 2] : 0.0f;
        sy = ky == 1 ? 0.0f : (ky == 0 ? B.shift[1][yw0 ? 3 : 0] : B.shift[1][yw2 ? 4 : 2]);
        sx = kx == 1 ? 0.0f : (kx == 0 ? B.shift[0][xw0 ? 3 : 0] : B.shift[0][xw2 ? 4 : 2]);
      }
    }
    if (j < e) {
      const int m = e - j;
      unsigned hm = 0u;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const PR pu = ld4(posr + j + (u < m ? u : 0));
        bool h;
        if (M == kMIXED) {
          const float4& q = *(const float4*)&pi;
          const float2 nxy = make_float2(-q.x, -q.y), nzw = make_float2(-q.z, q.w);
          const float2 sxy = make_float2(sx, sy), sz0 = make_float2(sz, skin);
          h = pred_fixed_packed(*(const float4*)&pu, nxy, nzw, sxy, sz0);
        } else {
          h = pred_abs(pi, pu, B, skin);
        }
        hm |= (unsigned)h << u;
        if (kSplit && is_large(pu.w, B.rsplit_f)) hm &= ~(1u << u);
      }
      hm &= (m >= 8) ? 0xFFu : ((1u << m) - 1u);
      while (hm) {
        const int jj = j + __ffs(hm) - 1;
        hm &= hm - 1u;
        if (own >= K) {
          over = true;
        } else {
          rowp[own++] = jj;
        }
      }
      j += 8;
    }
    __syncwarp(wmask);
  }
  if (over) flag(d.status, kStRowOverflow);
  return own;
}

// The dense list entries of a warp's particles: slot i (-1: none) found
// `own` partners, in its row.  One atomic add per warp on the list length
// takes the warp's block (its position depends on timing, the content of
// every entry does not), a warp scan places each particle's pairs there,
// oriented (lower id, higher id), and each entry index also goes into the
// partner's incoming row at a position taken from its incoming count.
__device__ __forceinline__ void write_list(const Dev& d, const PState& b, const VList& cn, int i,
                                           int own) {
  const int lane = threadIdx.x & 31;
  const int incl = warp_incl_scan(own);
  int base = 0;
  if (lane == 31 && incl > 0) base = atomicAdd(cn.count, incl);
  base = __shfl_sync(0xffffffffu, base, 31);
  if (i < 0) return;
  const long long pre = (long long)base + incl - own;
  int n = own;
  if (pre + n > d.Cmax) {
    flag(d.status, kStListOverflow);
    n = (int)max(0ll, (long long)d.Cmax - pre);
  }
  const int hs = (int)min(pre, (long long)d.Cmax);
  cn.hs[i] = hs;
  cn.oc[i] = n;
  const int idi = b.id[i];
  const int K = d.K;
  int* rowp = d.row + (size_t)i * K;
  for (int k = 0; k < n; k += 4) {
    int jj[4], pos[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) jj[u] = k + u < n ? rowp[k + u] : -1;
    // incoming positions of four partners, issued before any result is used
#pragma unroll
    for (int u = 0; u < 4; ++u) pos[u] = (d.inrow && jj[u] >= 0) ? atomicAdd(d.icnt + jj[u], 1) : K;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (jj[u] < 0) continue;
      const int j = jj[u], c = hs + k + u;
      const int idj = b.id[j];
      cn.pair[c] = idi < idj ? make_int2(i, j) : make_int2(j, i);
      if (cn.hid) cn.hid[c] = idi < idj ? make_int2(idi, idj) : make_int2(idj, idi);
      if (pos[u] < K) d.inrow[(size_t)j * K + pos[u]] = make_int2(c, (idi << 1) | (idj < idi ? 1 : 0));
      rowp[k + u] = idj;  // the row now holds the partners' ids (the keys of k_rows)
    }
  }
}

// kSplit: some box is size-binned; its large particles are not searched
// here but appended to d.large for k_candidates_large.
template <int M, bool kSplit>
__global__ void __launch_bounds__(256, 4)
k_candidates(Dev d, PState b, VList cn) {
  if (gated_off(d.gate)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // whole warps run
  int own = 0;
  bool live = false, large = false;
  if (i < d.N) {
    const BoxDev& B = d.boxes[d.slot_box[i]];
    live = i - B.pbase < B.nlive;
    if (kSplit && live) large = is_large(ld4((const typename Tr<M>::PR*)b.posr + i).w, B.rsplit_f);
    if (live && !large) own = kSplit ? search_row<M, true>(d, b, B, i) : search_row<M, false>(d, b, B, i);
  }
  __syncwarp();
  const int lane = threadIdx.x & 31;
  if (kSplit) {
    // append the warp's large particles (one atomic per warp)
    const unsigned lb = __ballot_sync(0xffffffffu, large);
    if (lb) {
      const int leader = __ffs(lb) - 1;
      int lbase = 0;
      if (lane == leader) lbase = atomicAdd(d.nlarge, __popc(lb));
      lbase = __shfl_sync(0xffffffffu, lbase, leader);
      if (large) d.large[lbase + __popc(lb & ((1u << lane) - 1u))] = i;
    }
  }
  if (!live && i < d.N) {
    cn.hs[i] = 0;
    cn.oc[i] = 0;
  }
  write_list(d, b, cn, live ? i : -1, own);
}

// ---------------------------------------------------------------------------
// size-binned search, large particles.  One cell size trades the cost of
// each particle's candidate loop against the number of cells it visits
// (Sec. 3.3); in a polydisperse box cells sized for the largest particle
// give every small particle a long loop.  A size-binned box (r_split > 0)
// sizes its cells for the small particles instead (at least 2 r_split and
// r_max wide): a small particle's partners of radius <= r_split lie within
// +-1 cell and any partner of a large particle within +-2 cells.  The small
// search above keeps its half stencil and skips large candidates; here the
// 125 cells of a large particle's +-2 neighbourhood go through the same two
// passes (face gaps with the box's largest radius, then the cell's bounding
// box and largest radius; then the kept cells' members four at a time,
// warp-uniform).  A large particle takes every small partner and the large
// partners in later slots, so each pair is found once.
// Periodic axes need at least 5 cells (the 5 cells of a step are distinct).
// ---------------------------------------------------------------------------

// Step st (-2..2) along axis a from cell c of a particle at offset o (cell
// width hc): false outside an open box; else the neighbour cell cc, the
// fixed-rule shift of its origin, (float)((cc - c) H + image L) exactly as
// the contact rule rounds it (DEM_MIXED) or st * h, and the squared gap
// from the particle to the cell's near face (whole cells in between count
// the ordinary width, which no cell undercuts).
template <int M>
__device__ __forceinline__ bool axis_step2(const BoxDev& B, int a, int c, int st, float o,
                                           float hc, int& cc, float& sh, float& g2) {
  const int n = B.n[a];
  cc = c + st;
  int image = 0;
  if (cc < 0) {
    if (!B.periodic[a]) return false;
    cc += n;
    image = -1;
  } else if (cc >= n) {
    if (!B.periodic[a]) return false;
    cc -= n;
    image = 1;
  }
  const float H = B.hcell[a][0];
  const float gap = st > 0 ? (hc - o) + (float)(st - 1) * H
                           : (st < 0 ? o + (float)(-st - 1) * H : 0.0f);
  const float gp = fmaxf(gap, 0.0f);
  g2 = gp * gp;
  if (M == kMIXED) {
    const long long S = (long long)(cc - c) * B.Hq[a] + (long long)image * B.Lq[a];
    sh = __fmul_rn(i64_to_f32_rn(S), kQ);
  } else {
    sh = (float)st * (float)B.h[a];
  }
  return true;
}

// Five lanes per large particle, six particles per warp (lanes 30 and 31
// idle): lane s of a group takes the 25 cells of z step s - 2.  Hits of a
// group go into the particle's row in (iteration, candidate, lane) order by
// ballots; the group then writes the particle's block of the list (one
// atomic per warp) and the partners' incoming rows, five entries at a time.
template <int M>
__global__ void __launch_bounds__(256)
k_candidates_large(Dev d, PState b, VList cn) {
  if (gated_off(d.gate)) return;
  using T = Tr<M>;
  using PR = typename T::PR;
  const PR* __restrict__ posr = (const PR*)b.posr;
  const float4* __restrict__ cellbox = d.cellbox;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int grp = lane / 5, s = lane - 5 * grp;  // grp 6: lanes 30, 31
  const unsigned gmask = grp < 6 ? 0x1Fu << (5 * grp) : 0u;
  const unsigned lt = (1u << lane) - 1u;
  const int K = d.K;
  const int nl = *d.nlarge;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int w0 = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); 6 * w0 < nl; w0 += nwarps) {
    const int t = 6 * w0 + grp;
    const bool has = grp < 6 && t < nl;
    const int i = has ? d.large[t] : 0;
    const BoxDev& B = d.boxes[d.slot_box[i]];
    const PR pi = ld4(posr + i);
    int c[3];
    unpack_cell(b.cellc[i], c[0], c[1], c[2]);
    float oi[3], hc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      hc[a] = c[a] == B.n[a] - 1 ? B.hcell[a][1] : B.hcell[a][0];
      if (M == kMIXED) oi[a] = (float)(a == 0 ? pi.x : a == 1 ? pi.y : pi.z);
      else oi[a] = (float)((double)(a == 0 ? pi.x : a == 1 ? pi.y : pi.z) - (double)c[a] * B.h[a]);
    }
    const float ri = (float)pi.w;
    const float skin = B.skin_f;
    const float rb = 1.001f * (ri + B.rmax_f + skin);
    const float rb2 = rb * rb;
    // Pass 1: keep bit ky 5 + kx of the lane's 25 cells
    unsigned keep = 0u;
    int cz = 0;
    float shz = 0.0f, gz2 = 0.0f;
    if (has && axis_step2<M>(B, 2, c[2], s - 2, oi[2], hc[2], cz, shz, gz2) && gz2 <= rb2) {
      unsigned xok = 0u;
      int xc[5];
      float xsh[5], xg2[5];
#pragma unroll
      for (int kx = 0; kx < 5; ++kx)
        if (axis_step2<M>(B, 0, c[0], kx - 2, oi[0], hc[0], xc[kx], xsh[kx], xg2[kx])) xok |= 1u << kx;
#pragma unroll
      for (int ky = 0; ky < 5; ++ky) {
        int cy;
        float shy, gy2;
        if (!axis_step2<M>(B, 1, c[1], ky - 2, oi[1], hc[1], cy, shy, gy2)) continue;
        const float gzy = gz2 + gy2;
        if (gzy > rb2) continue;
        const int row = B.lin_base + (cz * B.n[1] + cy) * B.n[0];
#pragma unroll
        for (int kx = 0; kx < 5; ++kx) {
          if (!((xok >> kx) & 1u) || gzy + xg2[kx] > rb2) continue;
          const int lin = row + xc[kx];
          const float4 blo = __ldg(cellbox + 2 * lin), bhi = __ldg(cellbox + 2 * lin + 1);
          const float gx = fmaxf(fmaxf(blo.x + xsh[kx] - oi[0], oi[0] - (bhi.x + xsh[kx])), 0.0f);
          const float gy = fmaxf(fmaxf(blo.y + shy - oi[1], oi[1] - (bhi.y + shy)), 0.0f);
          const float gz = fmaxf(fmaxf(blo.z + shz - oi[2], oi[2] - (bhi.z + shz)), 0.0f);
          const float reach = 1.001f * (ri + blo.w + skin);
          if (blo.w >= 0.0f && gx * gx + gy * gy + gz * gz <= reach * reach) keep |= 1u << (ky * 5 + kx);
        }
      }
    }
    // Pass 2, warp-uniform: every lane its next four candidates per
    // iteration; the group's hits are counted by ballot
    int* rowp = d.row + (size_t)i * K;
    const float rs = B.rsplit_f;
    int own = 0;
    int j = 0, e = 0;
    float sx = 0.f, sy = 0.f;
    // the next kept cell's range is loaded one cell ahead of its use
    bool nxt = false;
    int2 crn = make_int2(0, 0);
    float nsx = 0.f, nsy = 0.f;
    auto take = [&]() {
      nxt = keep != 0u;
      if (!nxt) return;
      const int idx = __ffs(keep) - 1;
      keep &= keep - 1u;
      int cx, cy;
      float g2;
      axis_step2<M>(B, 0, c[0], idx % 5 - 2, oi[0], hc[0], cx, nsx, g2);
      axis_step2<M>(B, 1, c[1], idx / 5 - 2, oi[1], hc[1], cy, nsy, g2);
      crn = __ldg(d.crange + B.lin_base + (cz * B.n[1] + cy) * B.n[0] + cx);
    };
    take();
    while (__any_sync(full, j < e || nxt)) {
      if (j >= e && nxt) {
        j = crn.x;
        e = crn.x + crn.y;
        sx = nsx;
        sy = nsy;
        take();
      }
      unsigned hm = 0u;
      if (j < e) {
        const int m = e - j;
        const PR p0 = ld4(posr + j);
        const PR p1 = m > 1 ? ld4(posr + j + 1) : p0;
        const PR p2 = m > 2 ? ld4(posr + j + 2) : p0;
        const PR p3 = m > 3 ? ld4(posr + j + 3) : p0;
        if (M == kMIXED) {
          const float4& q = *(const float4*)&pi;
          const float2 nxy = make_float2(-q.x, -q.y), nzw = make_float2(-q.z, q.w);
          const float2 sxy = make_float2(sx, sy), sz0 = make_float2(shz, skin);
          hm = (unsigned)pred_fixed_packed(*(const float4*)&p0, nxy, nzw, sxy, sz0) |
               ((unsigned)pred_fixed_packed(*(const float4*)&p1, nxy, nzw, sxy, sz0) << 1) |
               ((unsigned)pred_fixed_packed(*(const float4*)&p2, nxy, nzw, sxy, sz0) << 2) |
               ((unsigned)pred_fixed_packed(*(const float4*)&p3, nxy, nzw, sxy, sz0) << 3);
        } else {
          hm = (unsigned)pred_abs(pi, p0, B, skin) | ((unsigned)pred_abs(pi, p1, B, skin) << 1) |
               ((unsigned)pred_abs(pi, p2, B, skin) << 2) | ((unsigned)pred_abs(pi, p3, B, skin) << 3);
        }
        hm &= (m >= 4) ? 0xFu : ((1u << m) - 1u);
        // not the particle itself, nor a large partner in an earlier slot
        // (that partner's own search finds the pair)
        hm &= ~((unsigned)(j == i || (j < i && is_large(p0.w, rs))) |
                ((unsigned)(j + 1 == i || (j + 1 < i && is_large(p1.w, rs))) << 1) |
                ((unsigned)(j + 2 == i || (j + 2 < i && is_large(p2.w, rs))) << 2) |
                ((unsigned)(j + 3 == i || (j + 3 < i && is_large(p3.w, rs))) << 3));
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const bool hit = (hm >> v) & 1u;
        const unsigned bal = __ballot_sync(full, hit) & gmask;
        const int pos = own + __popc(bal & lt);
        if (hit && pos < K) rowp[pos] = j + v;
        own += __popc(bal);
      }
      j += 4;
    }
    __syncwarp();
    // the group's particle: its block of the list, one atomic per warp
    int n = own;
    if (n > K) {
      if (has && s == 0) flag(d.status, kStRowOverflow);
      n = K;
    }
    const int incl = warp_incl_scan((has && s == 0) ? n : 0);
    int base = 0;
    if (lane == 31 && incl > 0) base = atomicAdd(cn.count, incl);
    base = __shfl_sync(full, base, 31);
    const int gincl = __shfl_sync(full, incl, 5 * min(grp, 5));
    if (has) {
      const long long pre = (long long)base + gincl - n;
      if (pre + n > d.Cmax) {
        if (s == 0) flag(d.status, kStListOverflow);
        n = (int)max(0ll, (long long)d.Cmax - pre);
      }
      const int hs = (int)min(pre, (long long)d.Cmax);
      if (s == 0) {
        cn.hs[i] = hs;
        cn.oc[i] = n;
      }
      const int idi = b.id[i];
      for (int k = s; k < n; k += 5) {
        const int j2 = rowp[k], c2 = hs + k;
        const int pos = d.inrow ? atomicAdd(d.icnt + j2, 1) : K;
        const int idj = b.id[j2];
        cn.pair[c2] = idi < idj ? make_int2(i, j2) : make_int2(j2, i);
        if (cn.hid) cn.hid[c2] = idi < idj ? make_int2(idi, idj) : make_int2(idj, idi);
        if (pos < K) d.inrow[(size_t)j2 * K + pos] = make_int2(c2, (idi << 1) | (idj < idi ? 1 : 0));
        rowp[k] = idj;  // the row now holds the partners' ids (the keys of k_rows)
      }
    }
  }
}

// ---------------------------------------------------------------------------
// contact geometry: unit normal n (from 1 to 2) and overlap dn
// ---------------------------------------------------------------------------
// Fixed point: the position difference D is an exact integer (quanta), the
// radii are float32 values and therefore exact integers of quanta too, so
// R^2 - |D|^2 is formed exactly in 128-bit integers.  The overlap
// dn = (R^2 - |D|^2) / (R + |D|) then has FP32 relative accuracy however
// small it is (Eq. (1) has eta ~ dn^{1/4}, which amplifies any absolute
// error of a near-zero overlap without bound).
struct u128 {
  unsigned long long hi, lo;
};
__device__ __forceinline__ void u128_add_sq(u128& a, unsigned long long x) {
  unsigned long long l = x * x, h = __umul64hi(x, x);
  a.lo += l;
  a.hi += h + (a.lo < l ? 1ull : 0ull);
}
__device__ __forceinline__ bool u128_less(u128 a, u128 b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ u128 u128_sub(u128 a, u128 b) {  // a >= b
  u128 r;
  r.lo = a.lo - b.lo;
  r.hi = a.hi - b.hi - (a.lo < b.lo ? 1ull : 0ull);
  return r;
}
// to float without the FP64 pipe: top 32 significant bits, truncated
// (relative error below 2^-31), then one rounding to float and an exact
// power-of-two scale
__device__ __forceinline__ float u128_to_f32(u128 a) {
  if (a.hi == 0 && (a.lo >> 32) == 0) return __uint2float_rn((unsigned)a.lo);
  int bits = a.hi ? 128 - __clzll((long long)a.hi) : 64 - __clzll((long long)a.lo);
  int sh = bits - 32;  // > 0
  unsigned m;
  if (sh >= 64) m = (unsigned)(a.hi >> (sh - 64));
  else m = (unsigned)((a.hi << (64 - sh)) | (a.lo >> sh));
  float f = __uint2float_rn(m);
  return __fmul_rn(f, __int_as_float((127 + sh) << 23));  // sh <= 96
}

__device__ __forceinline__ void geom_fixed(const BoxDev& B, long long X1,
                                           long long Y1, long long Z1,
                                           long long X2, long long Y2,
                                           long long Z2, float r1, float r2,
                                           v3<float>& n, float& dn) {
  long long D[3] = {X2 - X1, Y2 - Y1, Z2 - Z1};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (B.periodic[a]) {
      long long L = B.Lq[a], h = L >> 1;
      if (D[a] > h) D[a] -= L;
      else if (D[a] < -h) D[a] += L;
    }
  }
  u128 S = {0ull, 0ull};
#pragma unroll
  for (int a = 0; a < 3; ++a)
    u128_add_sq(S, (unsigned long long)(D[a] < 0 ? -D[a] : D[a]));
  unsigned bad = 0;
  long long Rq = f32_to_i64_rn(__fmul_rn(r1, kInvQ), &bad) +
                 f32_to_i64_rn(__fmul_rn(r2, kInvQ), &bad);
  u128 R2 = {0ull, 0ull};
  u128_add_sq(R2, (unsigned long long)Rq);
  float distq = fsqrt(u128_to_f32(S));
  if (u128_less(S, R2)) {
    float num = u128_to_f32(u128_sub(R2, S));
    dn = __fmul_rn(fdiv(num, i64_to_f32_rn(Rq) + distq), kQ);
  } else {
    dn = 0.0f;
  }
  if (distq > 0.0f) {
    float inv = frcp(distq);
    n = {i64_to_f32_rn(D[0]) * inv, i64_to_f32_rn(D[1]) * inv,
         i64_to_f32_rn(D[2]) * inv};
  } else {
    n = {0.0f, 0.0f, 0.0f};
  }
}

template <typename R>
__device__ __forceinline__ void geom_abs(const BoxDev& B, R x1, R y1, R z1,
                                         R x2, R y2, R z2, R r1, R r2,
                                         v3<R>& n, R& dn) {
  v3<R> dd = {min_image(x2 - x1, B, 0), min_image(y2 - y1, B, 1),
              min_image(z2 - z1, B, 2)};
  R dist = norm(dd);
  if (dist > R(0)) n = (R(1) / dist) * dd;
  else n = {R(0), R(0), R(0)};
  dn = (r1 + r2) - dist;
}

// ---------------------------------------------------------------------------
// the contact law (Sec. 2): Eq. (vt), Eq. (dt), Eq. (1), coefficients,
// Coulomb cap with the delta_t reset.  Particle 1 is the lower id; v is
// v1 - v2; n points from 1 to 2.
// ---------------------------------------------------------------------------
template <typename R>
struct ContactOut {
  v3<R> F;      // force on particle 1
  v3<R> nF;     // n x F
  v3<R> dt;     // new delta_t (plain part)
  R ratio;      // |F_t| / (mu |F_n|) before the cap
  bool capped;
};

template <typename R>
__device__ __forceinline__ void contact_law(
    R kn_c, R kt_c, R alpha, R mu, R dtstep, v3<R> n, R dn, R r1, R r2,
    R m1, R m2, v3<R> v1, v3<R> v2, v3<R> w1, v3<R> w2, v3<R> dt_old,
    bool wall, ContactOut<R>& o, v3<R>& dt_delta) {
  v3<R> v = v1 - v2;
  R vns = dot(v, n);
  v3<R> vn = vns * n;
  v3<R> rot = wall ? r1 * w1 : (r1 * w1 + r2 * w2);
  v3<R> vt = v - vn + cross(rot, n);                      // Eq. (vt)
  R dd = dot(dt_old, n);
  dt_delta = (dtstep * vt) - (dd * n);                     // Eq. (dt) increment
  v3<R> dtn = dt_old + dt_delta;
  R Rs = wall ? r1 : fdiv(r1 * r2, r1 + r2);
  R ms = wall ? m1 : fdiv(m1 * m2, m1 + m2);
  R sdn = fsqrt(dn);
  R kn = kn_c * fsqrt(Rs);
  R kt = kt_c * fsqrt(Rs * dn);
  R eta = alpha * fsqrt(ms * kn * sdn);                     // eta_n = eta_t
  R fel = kn * dn * sdn;
  v3<R> Fn = (-fel) * n - eta * vn;                        // Eq. (1), normal
  v3<R> Ft = (-kt) * dtn - eta * vt;                       // Eq. (1), tangential
  R aFn = fsqrt(dot(Fn, Fn)), aFt = fsqrt(dot(Ft, Ft));
  R lim = mu * aFn;
  o.ratio = lim > R(0) ? fdiv(aFt, lim) : (aFt > R(0) ? R(1e30) : R(0));
  o.capped = aFt > lim;
  if (o.capped) {                                          // Eq. (sliding friction)
    R s = fdiv(lim, aFt);
    Ft = s * Ft;
    dtn = (-frcp(kt)) * Ft;                                // F_t,new = -k_t delta_t
  }
  o.dt = dtn;
  o.F = Fn + Ft;
  o.nF = cross(n, o.F);
}

__device__ __forceinline__ void atomic_max_pos(unsigned* p, float v) {
  if (v > 0.0f && isfinite(v)) atomicMax(p, __float_as_uint(v));
}

// ---------------------------------------------------------------------------
// one pair: history lookup (InitializeContactIDs) and the contact law.  i is
// the slot of the lower-id particle, j of the higher; idlo / idhi their ids.
// ---------------------------------------------------------------------------
template <int M>
struct PairOut {
  typename Tr<M>::V4 F4, N4;      // force on the lower particle, n x F
  typename Tr<M>::DT nx, ny, nz;  // delta_t after the step
  float ov, ratio;                // overlap / r_min, Coulomb ratio (0 if none)
};

// The contact law of one listed pair from its tangential history (ox, oy,
// oz: delta_t after the previous step, zero for a new contact): geometry from
// the exact positions, Eq. (vt), Eq. (dt), Eq. (1), the Coulomb cap, the new
// delta_t (a float-float sum in DEM_MIXED unless the cap reset it).  i is the
// slot of the lower-id particle, j of the higher.  A listed pair whose
// overlap in the force arithmetic is not positive gets no force and loses
// its history.
template <int M>
__device__ __forceinline__ void pair_law(const PState& b, const BoxDev& B, int i, int j,
                                         typename Tr<M>::DT ox, typename Tr<M>::DT oy,
                                         typename Tr<M>::DT oz, PairOut<M>& out) {
  using T = Tr<M>;
  using P = typename T::P;
  using R = typename T::R;
  using V4 = typename T::V4;
  using DT = typename T::DT;
  const P* __restrict__ px = (const P*)b.px;
  const P* __restrict__ py = (const P*)b.py;
  const P* __restrict__ pz = (const P*)b.pz;
  const V4* __restrict__ vel = (const V4*)b.vel;
  const V4* __restrict__ omg = (const V4*)b.omg;
  V4 v1 = ld4_fetch128(vel + i), v2 = ld4_fetch128(vel + j);
  V4 w1 = ld4_fetch128(omg + i), w2 = ld4_fetch128(omg + j);
  R r1 = w1.w, r2 = w2.w;
  v3<R> n;
  R dn;
  if (M == kMIXED) {
    float fn_dn;
    v3<float> fn_n;
    geom_fixed(B, (long long)ld_fetch128(px + i), (long long)ld_fetch128(py + i),
               (long long)ld_fetch128(pz + i), (long long)ld_fetch128(px + j),
               (long long)ld_fetch128(py + j), (long long)ld_fetch128(pz + j),
               (float)r1, (float)r2, fn_n, fn_dn);
    n = {(R)fn_n.x, (R)fn_n.y, (R)fn_n.z};
    dn = (R)fn_dn;
  } else {
    geom_abs<R>(B, (R)ld_fetch128(px + i), (R)ld_fetch128(py + i), (R)ld_fetch128(pz + i),
                (R)ld_fetch128(px + j), (R)ld_fetch128(py + j), (R)ld_fetch128(pz + j), r1, r2,
                n, dn);
  }
  out.F4 = V4{};
  out.N4 = V4{};
  out.nx = out.ny = out.nz = DT{};
  out.ov = out.ratio = 0.0f;
  if (!(dn > R(0))) return;
  v3<R> dold;
  if (M == kMIXED) {
    const float2 *fx = (const float2*)&ox, *fy = (const float2*)&oy,
                 *fz = (const float2*)&oz;
    dold = {(R)(fx->x + fx->y), (R)(fy->x + fy->y), (R)(fz->x + fz->y)};
  } else {
    dold = {*(const R*)&ox, *(const R*)&oy, *(const R*)&oz};
  }
  ContactOut<R> o;
  v3<R> inc;
  R kn_c = M == kFP64 ? (R)B.kn_c : (R)B.kn_cf;
  R kt_c = M == kFP64 ? (R)B.kt_c : (R)B.kt_cf;
  R al = M == kFP64 ? (R)B.alpha : (R)B.alpha_f;
  R mu = M == kFP64 ? (R)B.mu : (R)B.mu_f;
  R dts = M == kFP64 ? (R)B.dt : (R)B.dt_f;
  contact_law<R>(kn_c, kt_c, al, mu, dts, n, dn, r1, r2, (R)v1.w, (R)v2.w,
                 xyz(v1), xyz(v2), xyz(w1), xyz(w2), dold, false, o, inc);
  if (M == kMIXED) {
    // carry delta_t as a float-float sum unless the cap reset it
    float2* qx = (float2*)&out.nx;
    float2* qy = (float2*)&out.ny;
    float2* qz = (float2*)&out.nz;
    if (o.capped) {
      *qx = make_float2((float)o.dt.x, 0.f);
      *qy = make_float2((float)o.dt.y, 0.f);
      *qz = make_float2((float)o.dt.z, 0.f);
    } else {
      const float2 *fx = (const float2*)&ox, *fy = (const float2*)&oy,
                   *fz = (const float2*)&oz;
      ff ax = ff_add_f({fx->x, fx->y}, (float)inc.x);
      ff ay = ff_add_f({fy->x, fy->y}, (float)inc.y);
      ff az = ff_add_f({fz->x, fz->y}, (float)inc.z);
      *qx = make_float2(ax.hi, ax.lo);
      *qy = make_float2(ay.hi, ay.lo);
      *qz = make_float2(az.hi, az.lo);
    }
  } else {
    *(R*)&out.nx = o.dt.x;
    *(R*)&out.ny = o.dt.y;
    *(R*)&out.nz = o.dt.z;
  }
  out.F4 = mk4<R>(o.F.x, o.F.y, o.F.z, R(0));
  out.N4 = mk4<R>(o.nF.x, o.nF.y, o.nF.z, R(0));
  R rmin = r1 < r2 ? r1 : r2;
  out.ov = (float)fdiv(dn, rmin);
  out.ratio = (float)o.ratio;
}


// one pair of the per-particle Collide forms: history lookup
// (InitializeContactIDs) in the previous step's list, then the contact law.
// i is the slot of the lower-id particle, j of the higher.
template <int M>
__device__ __forceinline__ void pair_force(const Dev& d, const PState& b,
                                           const CList& co, const BoxDev& B,
                                           int i, int j, PairOut<M>& out) {
  using DT = typename Tr<M>::DT;
  // the pair is listed, by the slots the two particles had then, in the
  // block of the one that found it, which may be either
  int found = -1;
  {
    const int si = d.prev[i], sj = d.prev[j];
    const int os1 = co.hs[si], on1 = co.oc[si];
    const int os2 = co.hs[sj], on2 = co.oc[sj];
    for (int k = 0; k < on1; ++k) {
      const int2 h = co.pair[os1 + k];
      if (h.x == si && h.y == sj) {
        found = os1 + k;
        break;
      }
    }
    if (found < 0) {
      for (int k = 0; k < on2; ++k) {
        const int2 h = co.pair[os2 + k];
        if (h.x == si && h.y == sj) {
          found = os2 + k;
          break;
        }
      }
    }
  }
  DT ox = {}, oy = {}, oz = {};
  if (found >= 0) {
    ox = ((const DT*)co.dx)[found];
    oy = ((const DT*)co.dy)[found];
    oz = ((const DT*)co.dz)[found];
  }
  pair_law<M>(b, B, i, j, ox, oy, oz, out);
}

// warp-level max of the per-box diagnostics held in registers; every lane
// of the warp must call this
__device__ __forceinline__ void flush_diag(const Dev& d, int mbox, float m_ov,
                                           float m_ratio) {
  const unsigned full = 0xffffffffu;
  int b0 = __reduce_max_sync(full, mbox);
  if (__all_sync(full, mbox == b0 || mbox < 0)) {
    unsigned u_ov = __reduce_max_sync(full, mbox >= 0 ? __float_as_uint(m_ov) : 0u);
    unsigned u_ra = __reduce_max_sync(full, mbox >= 0 ? __float_as_uint(m_ratio) : 0u);
    if ((threadIdx.x & 31) == 0 && b0 >= 0) {
      if (u_ov) atomicMax(d.diag + 2 * b0, u_ov);
      if (u_ra) atomicMax(d.diag + 2 * b0 + 1, u_ra);
    }
  } else if (mbox >= 0) {
    atomic_max_pos(d.diag + 2 * mbox, m_ov);
    atomic_max_pos(d.diag + 2 * mbox + 1, m_ratio);
  }
}

__device__ __forceinline__ void track_diag(const Dev& d, int box, float ov,
                                           float ratio, int& mbox, float& m_ov,
                                           float& m_ratio) {
  if (box != mbox) {
    if (mbox >= 0) {
      atomic_max_pos(d.diag + 2 * mbox, m_ov);
      atomic_max_pos(d.diag + 2 * mbox + 1, m_ratio);
    }
    mbox = box;
    m_ov = m_ratio = 0.0f;
  }
  if (isfinite(ov)) m_ov = fmaxf(m_ov, ov);
  if (isfinite(ratio)) m_ratio = fmaxf(m_ratio, ratio);
}

// ---------------------------------------------------------------------------
// contact-list pipeline, every step: the contact rule on each candidate pair
// from the particles' current cells, then the force of the pairs in contact
// ---------------------------------------------------------------------------

// Fixed-rule shift of cell cj relative to cell ci along axis a for a pair the
// cell search tests: the step st, |st| <= w, with wrap(ci + st) = cj (unique:
// periodic axes have at least 2 w + 1 cells); the shift is that of the
// search, (float)((cj - ci) H + image L) with image -1 / +1 when the step
// wraps below 0 / above n - 1.  false when the cells are farther apart: the
// cell search never tests such a pair.
template <int M>
__device__ __forceinline__ bool pair_shift(const BoxDev& B, int a, int ci, int cj, int w,
                                           float& sh) {
  const int n = B.n[a];
  const int dc = cj - ci;
  int image = 0;
  if (dc < -w || dc > w) {
    if (!B.periodic[a]) return false;
    if (dc - n >= -w && dc - n <= w) image = -1;
    else if (dc + n >= -w && dc + n <= w) image = 1;
    else return false;
  }
  if (M != kMIXED) {
    sh = 0.0f;  // the absolute-position rule needs no shift
  } else if (w == 1) {
    // the search's table: -H, 0, +H, wrap below, wrap above
    sh = B.shift[a][image == 0 ? dc + 1 : (image < 0 ? 3 : 4)];
  } else {
    const long long S = (long long)dc * B.Hq[a] + (long long)image * B.Lq[a];
    sh = __fmul_rn(i64_to_f32_rn(S), kQ);
  }
  return true;
}

// The contact rule of the cell search (pred_fixed in DEM_MIXED, the
// absolute-position rule otherwise) on a listed pair, from both particles'
// current cells and predicate records: the same decision the search takes
// when it meets the pair (the rule is exactly antisymmetric, so the order of
// i and j does not matter).
template <int M>
__device__ __forceinline__ bool pair_in_contact(const BoxDev& B, const PState& b, int i, int j) {
  using PR = typename Tr<M>::PR;
  const int w = B.rsplit_f < INFINITY ? 2 : 1;  // size-binned boxes: +-2 cells
  int ci[3], cj[3];
  unpack_cell(ld_fetch128(b.cellc + i), ci[0], ci[1], ci[2]);
  unpack_cell(ld_fetch128(b.cellc + j), cj[0], cj[1], cj[2]);
  float sh[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (!pair_shift<M>(B, a, ci[a], cj[a], w, sh[a])) return false;
  const PR pi = ld4_fetch128((const PR*)b.posr + i), pj = ld4_fetch128((const PR*)b.posr + j);
  if (M == kMIXED) return pred_fixed(*(const float4*)&pi, *(const float4*)&pj, sh[0], sh[1], sh[2]);
  return pred_abs(pi, pj, B);
}

// One warp takes kPairTile candidates: each lane tests kPairU of them (their
// loads in flight together), the pairs in contact are compacted by ballot into
// a warp-local queue in shared memory (entry, history bit and both slots), and
// the warp then computes their forces 32 at a time with every lane busy.  A
// pair that left contact loses its history.  Every output is written at the
// pair's own list entry.  kOne: the context holds one box, whose constants
// come in B0 (a kernel parameter, read through the constant cache; its
// particle count is not valid there and is not read).
constexpr int kPairU = 2;
constexpr int kPairTile = 32 * kPairU;
constexpr int kPairWarps = 8;

template <bool kOne>
__device__ __forceinline__ const BoxDev& box_of(const Dev& d, const BoxDev& B0, int slot) {
  return kOne ? B0 : d.boxes[d.nbox == 1 ? 0 : d.slot_box[slot]];
}

template <int M, bool kOne>
__global__ void __launch_bounds__(32 * kPairWarps, M == kFP64 ? 2 : 4)
k_pairs(Dev d, PState b, VList vl, const __grid_constant__ BoxDev B0) {
  using T = Tr<M>;
  using V4 = typename T::V4;
  using DT = typename T::DT;
  __shared__ int qcb[kPairWarps][kPairTile + 32];
  __shared__ int2 qpb[kPairWarps][kPairTile + 32];
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  int* qc_ = qcb[wi];
  int2* qp = qpb[wi];
  // the sum kernel after this one may start on the SMs this kernel's blocks
  // leave (it waits for this kernel's results before it reads them)
  pdl_launch_dependents();
  const int nc = min(*vl.count, d.Cmax);
  const int nw = gridDim.x * kPairWarps;
  int mbox = -1;
  float m_ov = 0.0f, m_ratio = 0.0f;
  // qn pairs wait in the queue.  After each tile the whole groups of 32 are
  // computed and the rest (fewer than 32) waits for the next tile's, so that
  // every lane computes a force but in the warp's last group; one pass past
  // the warp's last tile computes what is left.  (The force is computed at
  // one place in the code, so that a pair's result does not depend on which
  // group it falls in.)
  int qn = 0;
  for (int t0 = (blockIdx.x * kPairWarps + wi) * kPairTile;; t0 += nw * kPairTile) {
    const bool more = t0 < nc;
    if (more) {
      int2 pr[kPairU];
      unsigned char fl[kPairU];
#pragma unroll
      for (int u = 0; u < kPairU; ++u) {
        const int c = t0 + u * 32 + lane;
        pr[u] = c < nc ? vl.pair[c] : make_int2(-1, -1);
        fl[u] = c < nc ? vl.flag[c] : 0;
      }
#pragma unroll
      for (int u = 0; u < kPairU; ++u) {
        const int c = t0 + u * 32 + lane;
        bool hit = false;
        if (pr[u].x >= 0) {
          const BoxDev& B = box_of<kOne>(d, B0, pr[u].x);
          hit = pair_in_contact<M>(B, b, pr[u].x, pr[u].y);
          if (!hit && fl[u]) vl.flag[c] = 0;  // left contact: no history any more
        }
        const unsigned bal = __ballot_sync(full, hit);
        if (hit) {
          const int at = qn + __popc(bal & lt);
          qc_[at] = (c << 1) | (fl[u] ? 1 : 0);
          qp[at] = pr[u];
        }
        qn += __popc(bal);
      }
    }
    __syncwarp();
    const int upto = more ? (qn & ~31) : qn;
    for (int k = 0; k < upto; k += 32) {
      if (k + lane < upto) {
        const int qc = qc_[k + lane];
        const int c = qc >> 1;
        const int2 p = qp[k + lane];
        const int box = kOne ? 0 : (d.nbox == 1 ? 0 : d.slot_box[p.x]);
        const BoxDev& B = box_of<kOne>(d, B0, p.x);
        // a pair in contact in the last step has a history; a new one starts
        // from zero (the stored values of a pair without the flag mean nothing)
        DT ox = {}, oy = {}, oz = {};
        if (qc & 1) {
          ox = ((const DT*)vl.dx)[c];
          oy = ((const DT*)vl.dy)[c];
          oz = ((const DT*)vl.dz)[c];
        }
        PairOut<M> o;
        pair_law<M>(b, B, p.x, p.y, ox, oy, oz, o);
        ((DT*)vl.dx)[c] = o.nx;
        ((DT*)vl.dy)[c] = o.ny;
        ((DT*)vl.dz)[c] = o.nz;
        vl.flag[c] = 1;
        st4((V4*)d.Fc + 2 * (size_t)c, o.F4);
        st4((V4*)d.Fc + 2 * (size_t)c + 1, o.N4);
        if (o.ov > 0.0f) track_diag(d, box, o.ov, o.ratio, mbox, m_ov, m_ratio);
      }
    }
    if (!more) break;
    __syncwarp();
    // the rest moves to the front of the queue
    if (lane < qn - upto) {
      qc_[lane] = qc_[upto + lane];
      qp[lane] = qp[upto + lane];
    }
    qn -= upto;
    __syncwarp();
  }
  flush_diag(d, mbox, m_ov, m_ratio);  // every lane of the warp gets here
}

// ---------------------------------------------------------------------------
// contact-list pipeline, at a re-sort (after the search wrote the new
// candidate list vn in the new slot order of b): each slot's row of all its
// candidate pairs, ordered by partner id (the order of the force sum, which
// then does not depend on slots, re-sorts or timing).  The row's entries go
// to d.frow and the partner ids beside them to d.row (where the search left
// the ids of the slot's own partners), where k_carry looks pairs up.  Every
// input is the slot's own: no partner's record is read.  A row of up to 16 entries is loaded into
// registers and ordered there by a bitonic sorting network (Batcher, 1968):
// 8 wide when every row of the warp fits, else 16 wide, unused places
// holding the largest key; a longer row is ordered by insertion in place.
// The new entries start without history (k_carry brings it).
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ void bitonic_sort(int (&key)[16], int (&val)[16]) {
#pragma unroll
  for (int k = 2; k <= W; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
      for (int u = 0; u < W; ++u) {
        const int v = u ^ j;
        if (v > u) {
          const bool up = (u & k) == 0;  // this pair's run ascends
          const bool sw = up ? key[u] > key[v] : key[u] < key[v];
          const int ku = key[u], kv = key[v], vu = val[u], vv = val[v];
          key[u] = sw ? kv : ku;
          key[v] = sw ? ku : kv;
          val[u] = sw ? vv : vu;
          val[v] = sw ? vu : vv;
        }
      }
    }
  }
}

template <int M>
__global__ void __launch_bounds__(256)
k_rows(Dev d, PState b, VList vn) {
  if (gated_off(d.gate)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.N) return;
  const BoxDev& B = d.boxes[d.nbox == 1 ? 0 : d.slot_box[i]];
  if (i - B.pbase >= B.nlive) {
    d.fcnt[i] = 0;
    return;
  }
  const int K = d.K;
  const int own = vn.oc[i], hs = vn.hs[i];
  const int inc = min(d.icnt[i], K);
  if (own + inc > K) flag(d.status, kStRowOverflow);
  const int n = min(own + inc, K);
  const int idi = b.id[i];
  // the search left the partners' ids of the slot's own pairs in its row
  // (the entry of the k-th is hs + k) and the incoming pairs as (entry,
  // partner id << 1 | lower-id bit)
  int* kr = d.row + (size_t)i * K;
  int* vr = d.frow + (size_t)i * K;
  const int2* in = d.inrow + (size_t)i * K;
  for (int k = 0; k < own; ++k) vn.flag[hs + k] = 0;
  if (n <= 16) {
    int key[16], val[16];
    // the row's inputs in 16-byte loads; the own entries fill the first
    // places, the incoming ones the last (entry m at place W - 1 - m), the
    // places between hold the largest key: every register index is fixed
    const int ninc = n - own;
    int4 ko[4], ic[8];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      ko[q] = 4 * q < own ? *(const int4*)(kr + 4 * q) : make_int4(0, 0, 0, 0);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      ic[q] = 2 * q < ninc ? *(const int4*)(in + 2 * q) : make_int4(0, 0, 0, 0);
    const bool w8 = __all_sync(__activemask(), n <= 8);  // W = 8, else 16
#pragma unroll
    for (int s = 0; s < 16; ++s) {
      const int4 o4 = ko[s >> 2];
      const int oid = (s & 3) == 0 ? o4.x : (s & 3) == 1 ? o4.y : (s & 3) == 2 ? o4.z : o4.w;
      int id = INT_MAX, v = 0;
      if (s < own) {
        id = oid;
        v = ((hs + s) << 1) | (idi < id ? 1 : 0);
      }
      key[s] = id;
      val[s] = v;
    }
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int4 c4 = ic[m >> 1];
      const int ex = (m & 1) ? c4.z : c4.x, ey = (m & 1) ? c4.w : c4.y;
      if (m < ninc) {
        if (w8) {
          if (m < 8) {
            key[7 - m] = ey >> 1;
            val[7 - m] = (ex << 1) | (ey & 1);
          }
        } else {
          key[15 - m] = ey >> 1;
          val[15 - m] = (ex << 1) | (ey & 1);
        }
      }
    }
    if (w8) bitonic_sort<8>(key, val);
    else bitonic_sort<16>(key, val);
#pragma unroll
    for (int k = 0; k < 16; k += 4) {
      if (k < n) {
        *(int4*)(kr + k) = make_int4(key[k], key[k + 1], key[k + 2], key[k + 3]);
        *(int4*)(vr + k) = make_int4(val[k], val[k + 1], val[k + 2], val[k + 3]);
      }
    }
  } else {
    // the own entries in place first, then the incoming ones inserted
    for (int k = 0; k < own; ++k) vr[k] = ((hs + k) << 1) | (idi < kr[k] ? 1 : 0);
    auto insert = [&](int m, int key, int val) {
      int pos = m;
      while (pos > 0 && kr[pos - 1] > key) {
        kr[pos] = kr[pos - 1];
        vr[pos] = vr[pos - 1];
        --pos;
      }
      kr[pos] = key;
      vr[pos] = val;
    };
    for (int m = 1; m < own; ++m) insert(m, kr[m], vr[m]);
    for (int m = own; m < n; ++m) {
      const int2 e = in[m - own];
      insert(m, e.y >> 1, (e.x << 1) | (e.y & 1));
    }
  }
  d.fcnt[i] = n;
}

// History carried over at a re-sort: each pair of the current list vo that
// was in contact in the last step (its flag) is looked up in the new row of
// its lower-id member (new slot from the reorder's map d.next; the partner
// found by id among the row's keys), and its delta_t goes to the new entry
// there, which gets the flag.  A pair that is no longer a candidate loses
// its history.  Four entries per thread, their loads in flight together.
constexpr int kCarryU = 4;

template <int M>
__global__ void __launch_bounds__(256)
k_carry(Dev d, PState a, VList vo, VList vn) {
  if (gated_off(d.gate)) return;
  using DT = typename Tr<M>::DT;
  const int nc = min(*vo.count, d.Cmax);
  const int K = d.K;
  const int stride = gridDim.x * blockDim.x;
  for (int c0 = blockIdx.x * blockDim.x + threadIdx.x; c0 < nc; c0 += kCarryU * stride) {
    int c[kCarryU], ni[kCarryU], idj[kCarryU], e[kCarryU];
    bool f[kCarryU];
#pragma unroll
    for (int u = 0; u < kCarryU; ++u) {
      c[u] = c0 + u * stride;
      // every listed pair holds two valid slots: the map and id loads need
      // not wait for the flag
      int2 p = make_int2(0, 0);
      unsigned char fl = 0;
      if (c[u] < nc) {
        fl = vo.flag[c[u]];
        p = vo.pair[c[u]];
      }
      ni[u] = d.next[p.x];
      idj[u] = a.id[p.y];
      f[u] = fl != 0;
    }
#pragma unroll
    for (int u = 0; u < kCarryU; ++u) {
      e[u] = -1;
      if (!f[u]) continue;
      const int* kr = d.row + (size_t)ni[u] * K;
      const int n = min(d.fcnt[ni[u]], K);
      const int4 q0 = *(const int4*)kr, q1 = *(const int4*)(kr + 4);
      const int q[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
      int at = -1;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k < n && q[k] == idj[u]) at = k;
      for (int k = 8; at < 0 && k < n; ++k)
        if (kr[k] == idj[u]) at = k;
      if (at >= 0) e[u] = d.frow[(size_t)ni[u] * K + at] >> 1;
    }
#pragma unroll
    for (int u = 0; u < kCarryU; ++u) {
      if (e[u] < 0) continue;
      ((DT*)vn.dx)[e[u]] = ((const DT*)vo.dx)[c[u]];
      ((DT*)vn.dy)[e[u]] = ((const DT*)vo.dy)[c[u]];
      ((DT*)vn.dz)[e[u]] = ((const DT*)vo.dz)[c[u]];
      vn.flag[e[u]] = 1;
    }
  }
}

// A box given new particles keeps no history: the contact flags of the
// entries in its slots' blocks of the current list are cleared.
__global__ void k_clear_flags(VList vo, int pbase, int cap) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= cap) return;
  const int hs = vo.hs[pbase + s], oc = vo.oc[pbase + s];
  for (int k = 0; k < oc; ++k) vo.flag[hs + k] = 0;
}

// The re-sorted state b and list vn become the current a and vo (the state
// stays in one place between re-sorts, where the integrator updates it); the
// positions of this sort are kept for the skin test, and the new cell starts
// become the current order's.
template <int M>
__global__ void k_commit(Dev d, PState a, PState b, VList vo, VList vn, const int* cs_new,
                         int* cs_cur) {
  if (gated_off(d.gate)) return;
  using T = Tr<M>;
  using P = typename T::P;
  using V4 = typename T::V4;
  using PR = typename T::PR;
  using DT = typename T::DT;
  const int nc = min(*vn.count, d.Cmax);
  const int top = max(max(d.N, nc), d.M_rank);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < top; k += gridDim.x * blockDim.x) {
    if (k < d.N) {
      const BoxDev& B = d.boxes[d.slot_box[k]];
      if (k - B.pbase < B.nlive) {
        const P x = ((const P*)b.px)[k], y = ((const P*)b.py)[k], z = ((const P*)b.pz)[k];
        ((P*)a.px)[k] = x;
        ((P*)a.py)[k] = y;
        ((P*)a.pz)[k] = z;
        ((P*)d.xb)[k] = x;
        ((P*)d.yb)[k] = y;
        ((P*)d.zb)[k] = z;
        st4((V4*)a.vel + k, ld4((const V4*)b.vel + k));
        st4((V4*)a.omg + k, ld4((const V4*)b.omg + k));
        st4((PR*)a.posr + k, ld4((const PR*)b.posr + k));
        a.id[k] = b.id[k];
        a.cellc[k] = b.cellc[k];
        a.cellx[k] = b.cellx[k];
        a.cellg[k] = b.cellg[k];
        if (a.wx) {
          for (int w = 0; w < d.nwh; ++w) {
            const size_t h = (size_t)k * d.nwh + w;
            ((DT*)a.wx)[h] = ((const DT*)b.wx)[h];
            ((DT*)a.wy)[h] = ((const DT*)b.wy)[h];
            ((DT*)a.wz)[h] = ((const DT*)b.wz)[h];
          }
        }
      }
      vo.hs[k] = vn.hs[k];
      vo.oc[k] = vn.oc[k];
    }
    if (k < nc) {
      vo.pair[k] = vn.pair[k];
      const unsigned char f = vn.flag[k];
      vo.flag[k] = f;
      if (f) {  // only a pair with the flag has a history
        ((DT*)vo.dx)[k] = ((const DT*)vn.dx)[k];
        ((DT*)vo.dy)[k] = ((const DT*)vn.dy)[k];
        ((DT*)vo.dz)[k] = ((const DT*)vn.dz)[k];
      }
    }
    if (k < d.M_rank) cs_cur[k] = cs_new[k];
    if (k == 0) *vo.count = nc;
  }
}

// Whether this step re-sorts: when a particle moved far enough since the
// last re-sort for a pair outside the candidate list to reach contact (the
// integrator's skin test), when the host asked for it (new particles,
// positions or history), or every step when some box keeps no skin.  In a
// CUDA graph the decision also opens or closes the conditional node that
// holds the re-sort kernels; launched directly, those kernels read it.
__global__ void k_decide(unsigned* vctl, int always, cudaGraphConditionalHandle h,
                         int set_handle) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const unsigned r = (always || vctl[kCtlRequest] != 0u) ? 1u : 0u;
  vctl[kCtlResort] = r;
  vctl[kCtlRequest] = 0u;
  vctl[kCtlResorts] += r;
  if (set_handle) cudaGraphSetConditional(h, r);
}

// ---------------------------------------------------------------------------
// The paper's per-particle Collide forms: one thread per particle scans its
// 27 neighbour cells; no contact list, no action-reaction (each pair is
// evaluated by both of its particles, in the same orientation, so the two
// results are exact negatives).  The lower-id particle stores the pair's
// delta_t in its slot's block of ko entries of the next list.
//   kTwoLoop = false (DEM_COLLIDE_FUSED): Algorithm 1 as printed, the force
//     of each contact computed as soon as the contact is found.
//   kTwoLoop = true (DEM_COLLIDE_TWOLOOP): the paper's improvement (Sec. 3.4):
//     a first loop only tests candidates and keeps the partners in contact
//     (here in the particle's row), a second loop computes their forces.
// Both sum the contacts in the same order, so their results are identical.
// ---------------------------------------------------------------------------
template <int M, bool kTwoLoop>
__global__ void __launch_bounds__(256)
k_collide_per_particle(Dev d, PState b, CList co, CList cn, int ko) {
  using T = Tr<M>;
  using PR = typename T::PR;
  using V4 = typename T::V4;
  using DT = typename T::DT;
  using R = typename T::R;
  int mbox = -1;
  float m_ov = 0.0f, m_ratio = 0.0f;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool live = false;
  if (i < d.N) {
    const BoxDev& B0 = d.boxes[d.slot_box[i]];
    live = i - B0.pbase < B0.nlive;
    if (!live) {
      cn.hs[i] = 0;
      cn.oc[i] = 0;
    }
  }
  if (live) {
    const int box = d.slot_box[i];
    const BoxDev& B = d.boxes[box];
    const PR* __restrict__ posr = (const PR*)b.posr;
    const int* __restrict__ ids = b.id;
    const PR pi = ld4(posr + i);
    const int idi = ids[i];
    int c[3];
    unpack_cell(b.cellc[i], c[0], c[1], c[2]);
    v3<R> F = {R(0), R(0), R(0)}, Ns = {R(0), R(0), R(0)};
    int own = 0;
    bool over = false;
    auto force_with = [&](int j) {
      const int idj = ids[j];
      const bool lo = idi < idj;
      PairOut<M> o;
      if (lo) pair_force<M>(d, b, co, B, i, j, o);
      else pair_force<M>(d, b, co, B, j, i, o);
      if (lo) {
        F = F + xyz(o.F4);
        if (own < ko) {
          const int cc = i * ko + own;
          cn.pair[cc] = make_int2(i, j);
          cn.hid[cc] = make_int2(idi, idj);
          ((DT*)cn.dx)[cc] = o.nx;
          ((DT*)cn.dy)[cc] = o.ny;
          ((DT*)cn.dz)[cc] = o.nz;
          st4((V4*)d.Fc + 2 * (size_t)cc, o.F4);
          st4((V4*)d.Fc + 2 * (size_t)cc + 1, o.N4);
          ++own;
        } else {
          over = true;
        }
        if (o.ov > 0.0f) track_diag(d, box, o.ov, o.ratio, mbox, m_ov, m_ratio);
      } else {
        F = F - xyz(o.F4);
      }
      Ns = Ns + xyz(o.N4);
    };
    int* rowp = d.row + (size_t)i * d.K;
    int nfound = 0;
    bool row_over = false;
    for (int dz = -1; dz <= 1; ++dz) {
      int czn;
      float sz;
      if (!axis_step(B, 2, c[2], dz, czn, sz)) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        int cyn;
        float sy;
        if (!axis_step(B, 1, c[1], dy, cyn, sy)) continue;
        for (int dx = -1; dx <= 1; ++dx) {
          int cxn;
          float sx;
          if (!axis_step(B, 0, c[0], dx, cxn, sx)) continue;
          const int2 rg = d.crange[B.lin_base + (czn * B.n[1] + cyn) * B.n[0] + cxn];
          for (int j = rg.x; j < rg.x + rg.y; ++j) {
            if (j == i) continue;
            const PR pj = ld4(posr + j);
            bool hit;
            if (M == kMIXED)
              hit = pred_fixed(*(const float4*)&pi, *(const float4*)&pj, sx, sy, sz);
            else
              hit = pred_abs(pi, pj, B);
            if (!hit) continue;
            if (kTwoLoop) {
              if (nfound < d.K) rowp[nfound++] = j;
              else row_over = true;
            } else {
              force_with(j);
            }
          }
        }
      }
    }
    if (kTwoLoop)
      for (int k = 0; k < nfound; ++k) force_with(rowp[k]);
    if (row_over) flag(d.status, kStRowOverflow);
    if (over) flag(d.status, kStListOverflow);
    const R r = (R)pi.w;
    st4((V4*)d.Ffused + i, mk4<R>(F.x, F.y, F.z, R(0)));
    st4((V4*)d.Tfused + i, mk4<R>(r * Ns.x, r * Ns.y, r * Ns.z, R(0)));
    cn.hs[i] = i * ko;
    cn.oc[i] = own;
  }
  flush_diag(d, mbox, m_ov, m_ratio);
}

// ---------------------------------------------------------------------------
// walls: one particle-wall contact of Eq. (1) with the wall as a body of
// infinite radius and mass at rest, its delta_t kept in the particle's slot
// h of the wall histories (float-float in DEM_MIXED)
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void wall_force(const Dev& d, const PState& b, const BoxDev& B,
                                           size_t h, v3<typename Tr<M>::R> nw,
                                           typename Tr<M>::R dn, const typename Tr<M>::V4& vm,
                                           const typename Tr<M>::V4& wr,
                                           v3<typename Tr<M>::R>& F, v3<typename Tr<M>::R>& Tq) {
  using T = Tr<M>;
  using R = typename T::R;
  using DT = typename T::DT;
  DT* wx = (DT*)b.wx;
  DT* wy = (DT*)b.wy;
  DT* wz = (DT*)b.wz;
  const R m = vm.w, r = wr.w;
  v3<R> dold;
  DT ox = wx[h], oy = wy[h], oz = wz[h];
  if (M == kMIXED) {
    const float2 *fx = (const float2*)&ox, *fy = (const float2*)&oy, *fz = (const float2*)&oz;
    dold = {(R)(fx->x + fx->y), (R)(fy->x + fy->y), (R)(fz->x + fz->y)};
  } else {
    dold = {*(const R*)&ox, *(const R*)&oy, *(const R*)&oz};
  }
  v3<R> zero = {R(0), R(0), R(0)};
  ContactOut<R> o;
  v3<R> incd;
  R kn_c = M == kFP64 ? (R)B.kn_c : (R)B.kn_cf;
  R kt_c = M == kFP64 ? (R)B.kt_c : (R)B.kt_cf;
  R al = M == kFP64 ? (R)B.alpha : (R)B.alpha_f;
  R mu = M == kFP64 ? (R)B.mu : (R)B.mu_f;
  R dts = M == kFP64 ? (R)B.dt : (R)B.dt_f;
  contact_law<R>(kn_c, kt_c, al, mu, dts, nw, dn, r, R(0), m, R(0), xyz(vm), zero, xyz(wr),
                 zero, dold, true, o, incd);
  F = F + o.F;
  Tq = Tq + r * o.nF;
  if (M == kMIXED) {
    float2 qx, qy, qz;
    if (o.capped) {
      qx = make_float2((float)o.dt.x, 0.f);
      qy = make_float2((float)o.dt.y, 0.f);
      qz = make_float2((float)o.dt.z, 0.f);
    } else {
      const float2 *fx = (const float2*)&ox, *fy = (const float2*)&oy, *fz = (const float2*)&oz;
      ff ax = ff_add_f({fx->x, fx->y}, (float)incd.x);
      ff ay = ff_add_f({fy->x, fy->y}, (float)incd.y);
      ff az = ff_add_f({fz->x, fz->y}, (float)incd.z);
      qx = make_float2(ax.hi, ax.lo);
      qy = make_float2(ay.hi, ay.lo);
      qz = make_float2(az.hi, az.lo);
    }
    wx[h] = *(DT*)&qx;
    wy[h] = *(DT*)&qy;
    wz[h] = *(DT*)&qz;
  } else {
    R tx = o.dt.x, ty = o.dt.y, tz = o.dt.z;
    wx[h] = *(DT*)&tx;
    wy[h] = *(DT*)&ty;
    wz[h] = *(DT*)&tz;
  }
}

template <int M>
__device__ __forceinline__ void wall_clear(const PState& b, size_t h) {
  using DT = typename Tr<M>::DT;
  ((DT*)b.wx)[h] = DT{};
  ((DT*)b.wy)[h] = DT{};
  ((DT*)b.wz)[h] = DT{};
}

// Rectangle and line walls (CollideRectangle, CollideLine), one thread per
// particle of a box that has them: the contact point is the wall's point
// closest to the particle's centre, found first in FP32 (a conservative
// cull: a particle farther than r + slack cannot touch) and then, for the
// particles that pass, in the oracle's FP64 arithmetic (FP32 in DEM_FP32).
// The sum of the walls' forces and torques goes to Fwall / Twall.
template <int M>
__global__ void k_walls(Dev d, PState b) {
  using T = Tr<M>;
  using P = typename T::P;
  using R = typename T::R;
  using V4 = typename T::V4;
  using G = typename std::conditional<M == kFP32, float, double>::type;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.N) return;
  const BoxDev& B = d.boxes[d.slot_box[i]];
  if (i - B.pbase >= B.nlive || B.nwalls == 0) return;
  const P x = ((const P*)b.px)[i], y = ((const P*)b.py)[i], z = ((const P*)b.pz)[i];
  const V4 vm = ld4((const V4*)b.vel + i), wr = ld4((const V4*)b.omg + i);
  const R r = wr.w;
  float cf[3];
  if (M == kMIXED) {
    cf[0] = __fmul_rn(i64_to_f32_rn((long long)x), kQ);
    cf[1] = __fmul_rn(i64_to_f32_rn((long long)y), kQ);
    cf[2] = __fmul_rn(i64_to_f32_rn((long long)z), kQ);
  } else {
    cf[0] = (float)x;
    cf[1] = (float)y;
    cf[2] = (float)z;
  }
  v3<R> F = {R(0), R(0), R(0)}, Tq = {R(0), R(0), R(0)};
  const size_t hbase = (size_t)i * d.nwh + (B.floor_wall ? 1 : 0);
  for (int k = 0; k < B.nwalls; ++k) {
    const WallDev& Wl = d.walls[B.wall_base + k];
    const size_t h = hbase + k;
    float e2f;
    {
      float df[3], qf[3];
      for (int a = 0; a < 3; ++a) df[a] = cf[a] - Wl.pf[a];
      float sf = (df[0] * Wl.uf[0] + df[1] * Wl.uf[1] + df[2] * Wl.uf[2]) * Wl.inv_uuf;
      sf = fminf(fmaxf(sf, 0.0f), 1.0f);
      float tf = 0.0f;
      if (Wl.kind == 0) {
        tf = (df[0] * Wl.vf[0] + df[1] * Wl.vf[1] + df[2] * Wl.vf[2]) * Wl.inv_vvf;
        tf = fminf(fmaxf(tf, 0.0f), 1.0f);
      }
      for (int a = 0; a < 3; ++a) qf[a] = Wl.pf[a] + sf * Wl.uf[a] + tf * Wl.vf[a] - cf[a];
      e2f = qf[0] * qf[0] + qf[1] * qf[1] + qf[2] * qf[2];
    }
    const float reachf = (float)r + Wl.slack;
    if (!(e2f <= reachf * reachf)) {
      wall_clear<M>(b, h);
      continue;
    }
    G c[3];
    if (M == kMIXED) {
      c[0] = (G)__ll2double_rn((long long)x) * 0x1p-60;
      c[1] = (G)__ll2double_rn((long long)y) * 0x1p-60;
      c[2] = (G)__ll2double_rn((long long)z) * 0x1p-60;
    } else {
      c[0] = (G)x;
      c[1] = (G)y;
      c[2] = (G)z;
    }
    G dd[3], e[3];
    for (int a = 0; a < 3; ++a) dd[a] = c[a] - (G)Wl.p[a];
    G sw = (dd[0] * (G)Wl.u[0] + dd[1] * (G)Wl.u[1] + dd[2] * (G)Wl.u[2]) * (G)Wl.inv_uu;
    sw = sw < G(0) ? G(0) : (sw > G(1) ? G(1) : sw);
    G tw = G(0);
    if (Wl.kind == 0) {
      tw = (dd[0] * (G)Wl.v[0] + dd[1] * (G)Wl.v[1] + dd[2] * (G)Wl.v[2]) * (G)Wl.inv_vv;
      tw = tw < G(0) ? G(0) : (tw > G(1) ? G(1) : tw);
    }
    for (int a = 0; a < 3; ++a) e[a] = (G)Wl.p[a] + sw * (G)Wl.u[a] + tw * (G)Wl.v[a] - c[a];
    const G dist = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    const G dnw = (G)r - dist;
    if (dist > G(0) && dnw > G(0)) {
      const G inv = G(1) / dist;
      wall_force<M>(d, b, B, h, {(R)(e[0] * inv), (R)(e[1] * inv), (R)(e[2] * inv)}, (R)dnw,
                    vm, wr, F, Tq);
    } else {
      wall_clear<M>(b, h);
    }
  }
  st4((V4*)d.Fwall + i, mk4<R>(F.x, F.y, F.z, R(0)));
  st4((V4*)d.Twall + i, mk4<R>(Tq.x, Tq.y, Tq.z, R(0)));
}

// ---------------------------------------------------------------------------
// per-particle sum (fixed order), floor wall, gravity, symplectic Euler,
// then binning for the next step
// (kOne: one box, its constants in B0 as in k_pairs; the particle count is
// read from the box array)
// ---------------------------------------------------------------------------
template <int M, bool kOne>
__global__ void __launch_bounds__(256, M == kFP64 ? 2 : 4)
k_gather_integrate(Dev d, PState b, const unsigned char* __restrict__ vl_flag, int store_ft,
                   const __grid_constant__ BoxDev B0) {
  using T = Tr<M>;
  using P = typename T::P;
  using R = typename T::R;
  using V4 = typename T::V4;
  using DT = typename T::DT;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.N) return;
  const int bi = kOne ? 0 : d.slot_box[i];
  const BoxDev& B = kOne ? B0 : d.boxes[bi];
  if (i - B.pbase >= d.boxes[bi].nlive) return;
  const V4* Fc = (const V4*)d.Fc;
  v3<R> F = {R(0), R(0), R(0)}, Ns = {R(0), R(0), R(0)};
  // Launched as a dependent of the pair kernel, this kernel may start while
  // that kernel finishes: before waiting for it, it reads only what the pair
  // kernel does not write (the row, written at the last re-sort) and writes
  // nothing.  (Asking L2 for the slot's own state there as well measured
  // slower.)
  const int* row = d.Ffused ? nullptr : d.frow + (size_t)i * d.K;
  const int nrow = d.Ffused ? 0 : min(d.fcnt[i], d.K);
  int4 ea = make_int4(0, 0, 0, 0), eb = ea;
  if (!d.Ffused) {
    ea = *(const int4*)row;
    eb = *(const int4*)(row + 4);
  }
  pdl_wait();
  if (!d.Ffused) {
    // the slot's candidate pairs in increasing partner id (the first eight,
    // then four at a time): their contact flags first, then the forces of
    // the pairs in contact; Fc is the force on the pair's lower-id member:
    // added when this slot is that member, subtracted otherwise; n x F
    // enters with the same sign for both
    {
      // the first eight entries (a row holds at least eight): their flags in
      // one batch, then the records of those in contact
      const int e[8] = {ea.x, ea.y, ea.z, ea.w, eb.x, eb.y, eb.z, eb.w};
      unsigned mask = 0u;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (u < nrow && vl_flag[e[u] >> 1]) mask |= 1u << u;
#pragma unroll
      for (int g = 0; g < 8; g += 4) {
        V4 fv[4], qv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (mask & (1u << (g + u))) {
            fv[u] = ld4(Fc + 2 * (size_t)(e[g + u] >> 1));
            qv[u] = ld4(Fc + 2 * (size_t)(e[g + u] >> 1) + 1);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (!(mask & (1u << (g + u)))) continue;
          if (e[g + u] & 1) F = F + xyz(fv[u]);
          else F = F - xyz(fv[u]);
          Ns = Ns + xyz(qv[u]);
        }
      }
    }
    for (int k = 8; k < nrow; k += 4) {
      const int4 e4 = *(const int4*)(row + k);
      const int e[4] = {e4.x, e4.y, e4.z, e4.w};
      unsigned char f[4];
      V4 fv[4], qv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) f[u] = k + u < nrow ? vl_flag[e[u] >> 1] : 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (f[u]) {
          fv[u] = ld4(Fc + 2 * (size_t)(e[u] >> 1));
          qv[u] = ld4(Fc + 2 * (size_t)(e[u] >> 1) + 1);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (!f[u]) continue;
        if (e[u] & 1) F = F + xyz(fv[u]);
        else F = F - xyz(fv[u]);
        Ns = Ns + xyz(qv[u]);
      }
    }
  }
  V4 vm = ((const V4*)b.vel)[i];
  V4 wr = ((const V4*)b.omg)[i];
  // the position of the last re-sort, for the skin test at the end (loaded
  // here, before the stores, so that its latency overlaps the integration)
  const bool skin_test = has_skin_test(d, B);
  P q[3] = {P(0), P(0), P(0)};
  if (skin_test) {
    q[0] = ((const P*)d.xb)[i];
    q[1] = ((const P*)d.yb)[i];
    q[2] = ((const P*)d.zb)[i];
  }
  R m = vm.w, r = wr.w;
  v3<R> Tq = r * Ns;  // T = r (n x F), same sign for both members of a pair
  if (d.Ffused) {
    F = xyz(ld4((const V4*)d.Ffused + i));
    Tq = xyz(ld4((const V4*)d.Tfused + i));
  }
  P x = ((P*)b.px)[i], y = ((P*)b.py)[i], z = ((P*)b.pz)[i];
  // Walls (Sec. 3.3 item 5): the floor z = 0 here; rectangles and lines
  // were summed by k_walls into Fwall / Twall.  Each is a body of infinite
  // radius and mass at rest (R* = r, m* = m); the particle keeps one delta_t
  // per wall (the floor first).
  const size_t hbase = (size_t)i * d.nwh;
  if (B.floor_wall) {
    R dn;
    if (M == kMIXED) {
      // overlap r - z from the exact fixed-point height: r (a float) is an
      // exact count of quanta, so only the final conversion rounds
      unsigned badr = 0;
      long long rq = f32_to_i64_rn(__fmul_rn((float)r, kInvQ), &badr);
      dn = (R)__fmul_rn(i64_to_f32_rn(rq - (long long)z), kQ);
    } else {
      dn = r - (R)z;
    }
    if (dn > R(0)) wall_force<M>(d, b, B, hbase, {R(0), R(0), R(-1)}, dn, vm, wr, F, Tq);
    else wall_clear<M>(b, hbase);
  }
  if (d.Fwall && B.nwalls > 0) {
    F = F + xyz(ld4((const V4*)d.Fwall + i));
    Tq = Tq + xyz(ld4((const V4*)d.Twall + i));
  }
  // gravity (ForceGravity)
  if (M == kFP64) F = F + m * v3<R>{(R)B.g[0], (R)B.g[1], (R)B.g[2]};
  else F = F + m * v3<R>{(R)B.g_f[0], (R)B.g_f[1], (R)B.g_f[2]};
  if (store_ft) {
    st4((V4*)d.Fout + i, mk4<R>(F.x, F.y, F.z, R(0)));
    st4((V4*)d.Tout + i, mk4<R>(Tq.x, Tq.y, Tq.z, R(0)));
  }
  // symplectic Euler: v += F/m dt, w += T/I dt, x += v dt, I = 2/5 m r^2
  R dts = M == kFP64 ? (R)B.dt : (R)B.dt_f;
  R am = dts / m;
  R aw = dts / (R(0.4) * m * r * r);
  vm.x += F.x * am;
  vm.y += F.y * am;
  vm.z += F.z * am;
  wr.x += Tq.x * aw;
  wr.y += Tq.y * aw;
  wr.z += Tq.z * aw;
  bool finite = isfinite(vm.x) && isfinite(vm.y) && isfinite(vm.z) &&
                isfinite(wr.x) && isfinite(wr.y) && isfinite(wr.z);
  if (!finite) {
    flag(d.status, kStNonFinite);
    vm.x = vm.y = vm.z = R(0);
    wr.x = wr.y = wr.z = R(0);
  }
  st4((V4*)b.vel + i, vm);
  st4((V4*)b.omg + i, wr);
  int c[3];
  int cc = b.cellc[i];
  unpack_cell(cc, c[0], c[1], c[2]);
  P p[3] = {x, y, z};
  R vv[3] = {vm.x, vm.y, vm.z};
  unsigned bad = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (M == kMIXED) {
      long long X = (long long)p[a];
      long long D = f32_to_i64_rn(__fmul_rn((float)vv[a], B.dtq_f), &bad);
      X += D;
      int ca = c[a];
      const long long H = B.Hq[a];
      const int n = B.n[a];
      if (B.periodic[a]) {
        const long long L = B.Lq[a];
        if (X >= L) {
          X -= L;
          ca = 0;
        } else if (X < 0) {
          X += L;
          ca = n - 1;
        }
        if (X < 0 || X >= L) {  // moved more than a box length
          X = wrap_pos<kMIXED>(B, a, X);
          ca = cell_coord<kMIXED>(B, a, X);
        }
      }
      // step to the containing cell (particles move far less than a cell)
      int guard = 0;
      while (ca > 0 && X < (long long)ca * H && guard++ < 4) --ca;
      while (ca < n - 1 && X >= (long long)(ca + 1) * H && guard++ < 8) ++ca;
      if (guard >= 4) ca = cell_coord<kMIXED>(B, a, X);
      p[a] = (P)X;
      c[a] = ca;
    } else {
      P xa = p[a] + (P)(vv[a] * dts);
      xa = wrap_pos<M>(B, a, xa);
      p[a] = xa;
      c[a] = cell_coord<M>(B, a, xa);
    }
  }
  if (bad) flag(d.status, kStRange);
  ((P*)b.px)[i] = p[0];
  ((P*)b.py)[i] = p[1];
  ((P*)b.pz)[i] = p[2];
  const int cnew = pack_cell(c[0], c[1], c[2]);
  b.cellc[i] = cnew;
  // the contact rule's record for the next step, then the skin test
  st4((typename T::PR*)b.posr + i, pos_record<M>(B, p, c, wr.w));
  if (skin_test && skin_exceeded<M>(B, p, q)) d.vctl[kCtlRequest] = 1u;
  if (cnew != cc) {
    // moved to another cell: counts and the changed-cell flags of both
    const int g0 = b.cellg[i];
    const int g = rank_cell(d, B, c[0], c[1], c[2]);
    b.cellg[i] = g;
    atomicSub(&d.ccount[g0], 1);
    atomicAdd(&d.ccount[g], 1);
    d.collect[g0] = 1;
    d.collect[g] = 1;
  }
}

// ---------------------------------------------------------------------------
// state out (id order, FP64)
// ---------------------------------------------------------------------------
template <int M>
__global__ void k_get_state(Dev d, PState b, int box, double* x, double* v,
                            double* w, double* F, double* Tq, int have_ft) {
  using T = Tr<M>;
  using P = typename T::P;
  using V4 = typename T::V4;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  const BoxDev& B = d.boxes[box];
  if (t >= B.nlive) return;
  int slot = B.pbase + t;
  int k = b.id[slot] - B.pbase;
  if (x) {
    P p[3] = {((P*)b.px)[slot], ((P*)b.py)[slot], ((P*)b.pz)[slot]};
    for (int a = 0; a < 3; ++a) {
      if (M == kMIXED) x[3 * k + a] = (double)(long long)p[a] * 0x1p-60;
      else x[3 * k + a] = (double)p[a];
    }
  }
  if (v) {
    V4 q = ((const V4*)b.vel)[slot];
    v[3 * k] = q.x;
    v[3 * k + 1] = q.y;
    v[3 * k + 2] = q.z;
  }
  if (w) {
    V4 q = ((const V4*)b.omg)[slot];
    w[3 * k] = q.x;
    w[3 * k + 1] = q.y;
    w[3 * k + 2] = q.z;
  }
  if (F) {
    V4 q = {};
    if (have_ft) q = ((const V4*)d.Fout)[slot];
    F[3 * k] = q.x;
    F[3 * k + 1] = q.y;
    F[3 * k + 2] = q.z;
  }
  if (Tq) {
    V4 q = {};
    if (have_ft) q = ((const V4*)d.Tout)[slot];
    Tq[3 * k] = q.x;
    Tq[3 * k + 1] = q.y;
    Tq[3 * k + 2] = q.z;
  }
}

// radii in id order (the layout tuner's snapshot)
template <int M>
__global__ void k_get_radius(Dev d, PState b, int box, double* r) {
  using V4 = typename Tr<M>::V4;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const BoxDev& B = d.boxes[box];
  if (t >= B.nlive) return;
  const int slot = B.pbase + t;
  r[b.id[slot] - B.pbase] = (double)((const V4*)b.omg)[slot].w;
}

__global__ void k_get_order(Dev d, PState b, int box, int* id_by_slot,
                            int* cell_by_slot) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  const BoxDev& B = d.boxes[box];
  if (t >= B.nlive) return;
  int slot = B.pbase + t;
  if (id_by_slot) id_by_slot[t] = b.id[slot] - B.pbase;
  if (cell_by_slot) {
    int cx, cy, cz;
    unpack_cell(b.cellx[slot], cx, cy, cz);
    cell_by_slot[t] = (cz * B.n[1] + cy) * B.n[0] + cx;
  }
}

// per-box FP64 reductions in a fixed order (one block per box)
// Box statistics in FP64: each block sums a strided share of the box's
// slots into part[block][6]; k_stats_final adds the parts in block order
// (a fixed order: the result does not depend on timing).
template <int M>
__global__ void k_stats(Dev d, PState b, const int* hs, const int* oc,
                        const unsigned char* flag, int box, double* part) {
  using T = Tr<M>;
  using V4 = typename T::V4;
  const BoxDev& B = d.boxes[box];
  double acc[6] = {0, 0, 0, 0, 0, 0};  // KEt, KEr, Px, Py, Pz, contacts
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < B.nlive;
       t += gridDim.x * blockDim.x) {
    int s = B.pbase + t;
    V4 vm = ((const V4*)b.vel)[s];
    V4 wr = ((const V4*)b.omg)[s];
    double m = vm.w, r = wr.w;
    double vx = vm.x, vy = vm.y, vz = vm.z;
    double wx = wr.x, wy = wr.y, wz = wr.z;
    acc[0] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
    acc[1] += 0.5 * 0.4 * m * r * r * (wx * wx + wy * wy + wz * wz);
    acc[2] += m * vx;
    acc[3] += m * vy;
    acc[4] += m * vz;
    if (flag) {  // candidate list: the pairs in contact in the last step
      int nin = 0;
      for (int k = 0; k < oc[s]; ++k) nin += flag[hs[s] + k] ? 1 : 0;
      acc[5] += (double)nin;
    } else {
      acc[5] += (double)oc[s];
    }
  }
  __shared__ double sh[6][256];
  for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 6; ++q) part[6 * blockIdx.x + q] = sh[q][0];
}

__global__ void k_stats_final(const double* part, int nparts, double* out) {
  const int q = threadIdx.x;
  if (q >= 6) return;
  double s = 0.0;
  for (int k = 0; k < nparts; ++k) s += part[6 * k + q];
  out[q] = s;
}

}  // namespace dem
