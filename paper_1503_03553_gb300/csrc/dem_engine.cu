// dem_engine.cu -- host engine and C ABI of the GB300 DEM library.
//
// Owns the device state of all boxes (flat arrays; box b holds storage slots
// [pbase_b, pbase_b + cap_b) and cells [lin_base_b, lin_base_b + ncells_b)),
// orders one time step as a fixed sequence of kernels on one stream, and
// replays G steps at a time from a captured CUDA graph.
#include <algorithm>
#include <array>
#include <climits>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/dem.h"
#include "dem_kernels.cuh"

using namespace dem;

namespace {

constexpr int kPhases = 5;
thread_local std::string g_create_error;

// Per-phase timing: a ring of event sets, one set per step, read back when
// the ring is full and at the end of dem_step (no synchronisation per step).
constexpr int kRing = 64;
struct Timing {
  bool on = false;
  bool made = false;
  cudaEvent_t ev[kRing][kPhases + 1] = {};
  int used = 0;  // sets recorded since the last read
  double acc[kPhases] = {};
  int steps = 0;
};

}  // namespace

struct dem_ctx {
  dem_config cfg{};
  std::vector<dem_box> boxes;
  std::vector<dem_material> mats;
  int mode = kMIXED;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // host transfers of dem_set_state / dem_get_state: copies on their own
  // stream, overlapped with the per-array kernels on the context's stream
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t xfer_ev[6] = {};
  int device = 0;
  int nsm = 152;
  int pairs_grid = 0;  // blocks of the pair kernel: one wave (set at set-up)
  int N = 0, K = 32, Cmax = 0, M_lin = 0, M_rank = 0;
  int block = 256;
  int graph_steps = 16;
  int max_cap = 0;
  bool fused = false;  // a per-particle Collide form: no contact list
  bool twoloop = false;  // DEM_COLLIDE_TWOLOOP: the paper's two-loop form
  bool split = false;    // some box is size-binned (r_split > 0)
  int ko = 8;          // fused: stored contacts per particle
  std::vector<BoxDev> hbox;
  std::vector<void*> allocs;
  Dev dev{};
  // Particle state.  DEM_COLLIDE_COMPACT keeps it in ps[0] between re-sorts
  // (a re-sort orders it into ps[1] and commits it back; parity stays 0);
  // the per-particle Collide forms sort every step from one to the other.
  PState ps[2]{};
  CList cl[2]{};               // contact lists of the per-particle forms
  VList vl[2]{};               // candidate lists: [0] current, [1] a re-sort's
  int* cs_cur = nullptr;       // cell starts of the current order
  int* cs_new = nullptr;       // cell starts of the order being built
  unsigned char* collect = nullptr;  // cells changed since the last sort
  unsigned char* chg = nullptr;      // ... as seen by the sort running now
  bool always_resort = false;  // some box keeps no skin: re-sort every step
  cudaStream_t body_stream = nullptr;  // captures the re-sort kernels of a graph
  int parity = 0;
  int nwh = 0;                   // wall histories per slot (largest box)
  std::vector<WallDev> hwalls;   // all boxes' rectangle and line walls
  std::vector<std::vector<dem_wall>> wall_src;  // the caller's walls, copied
  bool have_particles = false;
  bool have_ft = false;
  unsigned* h_status = nullptr;  // pinned
  int* h_count = nullptr;        // pinned
  double* staging = nullptr;     // device, max_cap x 16 doubles
  int* staging_i = nullptr;      // device, max_cap x 2 ints
  std::string err;
  unsigned sticky = 0;
  // graphs of graph_steps steps by starting parity ([0], [1]); for the
  // contact-list pipeline also one step without ([2]) and with ([3]) the
  // force output, which take the steps left over
  cudaGraphExec_t gexec[4] = {nullptr, nullptr, nullptr, nullptr};
  Timing tm;
  double phase_ms[kPhases] = {};
  int64_t steps_done = 0;
};

namespace {

dem_status fail(dem_ctx* c, dem_status s, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_error = msg;
  return s;
}

#define CK(call)                                                          \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess)                                                \
      return fail(ctx, DEM_ERR_CUDA,                                      \
                  std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)

void* dalloc(dem_ctx* ctx, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (ctx->cfg.alloc) {
    p = ctx->cfg.alloc(bytes, ctx->cfg.alloc_ctx);
  } else if (cudaMallocAsync(&p, bytes, ctx->stream) != cudaSuccess) {
    p = nullptr;
  }
  if (p) ctx->allocs.push_back(p);
  return p;
}

void free_all(dem_ctx* ctx) {
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (void* p : ctx->allocs) {
    if (ctx->cfg.free) ctx->cfg.free(p, ctx->cfg.alloc_ctx);
    else if (!ctx->cfg.alloc) cudaFreeAsync(p, ctx->stream);
  }
  ctx->allocs.clear();
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
}

uint64_t morton3(uint32_t x, uint32_t y, uint32_t z) {
  // spread 21 bits of each coordinate three apart (magic-number form)
  auto spread = [](uint64_t v) {
    v &= 0x1fffff;
    v = (v | v << 32) & 0x1f00000000ffffull;
    v = (v | v << 16) & 0x1f0000ff0000ffull;
    v = (v | v << 8) & 0x100f00f00f00f00full;
    v = (v | v << 4) & 0x10c30c30c30c30c3ull;
    v = (v | v << 2) & 0x1249249249249249ull;
    return v;
  };
  return spread(x) | (spread(y) << 1) | (spread(z) << 2);
}

// kernels of a step that does not re-sort (DEM_COLLIDE_COMPACT: decide,
// pairs, sum + integrate; the per-particle forms sort every step)
int launches_per_step(const dem_ctx* ctx) {
  if (ctx->fused) return 7 + (ctx->hwalls.empty() ? 0 : 1);
  return 3 + (ctx->hwalls.empty() ? 0 : 1);
}
// kernels a re-sort adds (cell scan x3, scatter, reorder, search, rows,
// history, commit)
int launches_per_resort(const dem_ctx* ctx) { return ctx->fused ? 0 : 9 + (ctx->split ? 1 : 0); }

size_t pos_bytes(int mode) { return mode == kMIXED ? 8 : (mode == kFP64 ? 8 : 4); }
size_t v4_bytes(int mode) { return mode == kFP64 ? 32 : 16; }
size_t dt_bytes(int mode) { return mode == kMIXED ? 8 : (mode == kFP64 ? 8 : 4); }

int blocks_for(long long n, int b) { return (int)((n + b - 1) / b); }

// --------------------------------------------------------------------------
// one step, enqueued on ctx->stream
// --------------------------------------------------------------------------
// Box 0's constants as a kernel parameter for the one-box kernels (read
// through the constant cache, and fixed in a captured graph).  Its particle
// count changes with dem_set_particles, so the copy carries an impossible
// value there and the kernels read the count from the device array.
BoxDev box0_param(const dem_ctx* ctx) {
  BoxDev B = ctx->hbox[0];
  B.nlive = INT_MIN;
  return B;
}

// The per-particle Collide forms (Algorithm 1 and its two-loop form): sort
// every step from state p into state q, then the per-particle kernel.
template <int M>
void enqueue_fused(dem_ctx* ctx, int p, bool store_ft) {
  const int q = 1 - p;
  Dev d = ctx->dev;
  d.cstart = ctx->cs_new;
  d.cstart_old = ctx->cs_cur;
  d.chg = ctx->chg;
  d.collect = ctx->collect;
  d.cellbox = nullptr;  // the per-particle forms do not prune
  d.gate = nullptr;
  cudaStream_t s = ctx->stream;
  const int bs = ctx->block;
  const bool tm = ctx->tm.on;
  cudaEvent_t* ev = ctx->tm.ev[ctx->tm.used % kRing];
  if (tm) cudaEventRecord(ev[0], s);
  // 1. cell counts -> starts (rank order) and ranges (linear cells)
  int nbc = blocks_for(d.M_rank, kScanTile);
  k_scan_reduce<<<nbc, kScanThreads, 0, s>>>(d.ccount, d.M_rank, d.scan_bsum, d.gate);
  k_scan_top<<<1, kScanTopThreads, 0, s>>>(d.scan_bsum, nbc, nullptr, 0, d.status, 0u, d.gate);
  k_scan_apply<<<nbc, kScanThreads, 0, s>>>(
      d.ccount, d.M_rank, d.scan_bsum,
      CellEpi{d.cstart, d.crange, d.cellbox, d.lin_of_rank, d.collect, ctx->chg, d.ccur}, d.gate);
  // 2. counting sort by (Morton cell, id) and reorder into parity q
  k_scatter<<<blocks_for(d.N, bs), bs, 0, s>>>(d, ctx->ps[p]);
  k_reorder<M><<<blocks_for(d.N, bs), bs, 0, s>>>(d, ctx->ps[p], ctx->ps[q], nullptr);
  cudaMemcpyAsync(ctx->cs_cur, ctx->cs_new, sizeof(int) * std::max(1, d.M_rank),
                  cudaMemcpyDeviceToDevice, s);
  if (tm) cudaEventRecord(ev[1], s);
  // Algorithm 1: search and force in one pass, no contact list
  if (ctx->twoloop)
    k_collide_per_particle<M, true><<<blocks_for(d.N, bs), bs, 0, s>>>(
        d, ctx->ps[q], ctx->cl[p], ctx->cl[q], ctx->ko);
  else
    k_collide_per_particle<M, false><<<blocks_for(d.N, bs), bs, 0, s>>>(
        d, ctx->ps[q], ctx->cl[p], ctx->cl[q], ctx->ko);
  if (tm) {
    cudaEventRecord(ev[2], s);
    cudaEventRecord(ev[3], s);
    cudaEventRecord(ev[4], s);
  }
  const int bsg = bs < 256 ? bs : 256;  // compiled for at most 256 threads
  if (d.Fwall) k_walls<M><<<blocks_for(d.N, bs), bs, 0, s>>>(d, ctx->ps[q]);
  const BoxDev B0 = box0_param(ctx);
  if (ctx->hbox.size() == 1)
    k_gather_integrate<M, true><<<blocks_for(d.N, bsg), bsg, 0, s>>>(
        d, ctx->ps[q], nullptr, store_ft ? 1 : 0, B0);
  else
    k_gather_integrate<M, false><<<blocks_for(d.N, bsg), bsg, 0, s>>>(
        d, ctx->ps[q], nullptr, store_ft ? 1 : 0, B0);
  if (tm) cudaEventRecord(ev[5], s);
}

// The contact-list pipeline (DEM_COLLIDE_COMPACT).  The re-sort kernels
// (cell scan, counting sort, reorder, candidate search, rows with the
// history carried over, commit) go on stream rs: the step's own stream when
// launched directly, where they read the decision from the device and return
// at once when it is "no"; a capture stream into the body of a conditional
// graph node otherwise, which runs them only when the decision is "yes".
template <int M>
void enqueue_resort(dem_ctx* ctx, cudaStream_t rs, bool tm, cudaEvent_t* ev) {
  Dev d = ctx->dev;
  d.cstart = ctx->cs_new;
  d.cstart_old = ctx->cs_cur;
  d.chg = ctx->chg;
  d.collect = ctx->collect;
  d.gate = d.vctl + kCtlResort;
  const int bs = ctx->block;
  int nbc = blocks_for(d.M_rank, kScanTile);
  k_scan_reduce<<<nbc, kScanThreads, 0, rs>>>(d.ccount, d.M_rank, d.scan_bsum, d.gate);
  k_scan_top<<<1, kScanTopThreads, 0, rs>>>(d.scan_bsum, nbc, nullptr, 0, d.status, 0u, d.gate);
  k_scan_apply<<<nbc, kScanThreads, 0, rs>>>(
      d.ccount, d.M_rank, d.scan_bsum,
      CellEpi{d.cstart, d.crange, d.cellbox, d.lin_of_rank, d.collect, ctx->chg, d.ccur}, d.gate);
  k_scatter<<<blocks_for(d.N, bs), bs, 0, rs>>>(d, ctx->ps[0]);
  k_reorder<M><<<blocks_for(d.N, bs), bs, 0, rs>>>(d, ctx->ps[0], ctx->ps[1], ctx->vl[1].count);
  if (tm) cudaEventRecord(ev[1], rs);
  // the search kernel is compiled for at most 256 threads per block
  const int bs_search = bs < 256 ? bs : 256;
  if (ctx->split) {
    k_candidates<M, true><<<blocks_for(d.N, bs_search), bs_search, 0, rs>>>(d, ctx->ps[1], ctx->vl[1]);
    // large particles of size-binned boxes: one warp each, persistent grid
    k_candidates_large<M><<<ctx->nsm * 8, 256, 0, rs>>>(d, ctx->ps[1], ctx->vl[1]);
  } else {
    k_candidates<M, false><<<blocks_for(d.N, bs_search), bs_search, 0, rs>>>(d, ctx->ps[1], ctx->vl[1]);
  }
  if (tm) cudaEventRecord(ev[2], rs);
  k_rows<M><<<blocks_for(d.N, 256), 256, 0, rs>>>(d, ctx->ps[1], ctx->vl[1]);
  k_carry<M><<<ctx->nsm * 8, 256, 0, rs>>>(d, ctx->ps[0], ctx->vl[0], ctx->vl[1]);
  k_commit<M><<<ctx->nsm * 8, 256, 0, rs>>>(d, ctx->ps[0], ctx->ps[1], ctx->vl[0], ctx->vl[1],
                                            ctx->cs_new, ctx->cs_cur);
}

template <int M>
void enqueue_tail(dem_ctx* ctx, bool store_ft, bool tm, cudaEvent_t* ev) {
  Dev d = ctx->dev;
  d.gate = nullptr;
  d.collect = ctx->collect;
  cudaStream_t s = ctx->stream;
  // the sum + integrate kernel is compiled for at most 256 threads per block
  const int bs = ctx->block < 256 ? ctx->block : 256;
  if (tm) cudaEventRecord(ev[3], s);
  const BoxDev B0 = box0_param(ctx);
  const bool one = ctx->hbox.size() == 1;
  // the pair kernel runs as one wave of resident blocks (its warps stride
  // over the candidate tiles), which measured faster than more,
  // shorter-lived blocks
  const int pgrid = ctx->pairs_grid;
  if (one)
    k_pairs<M, true><<<pgrid, 32 * kPairWarps, 0, s>>>(d, ctx->ps[0], ctx->vl[0], B0);
  else
    k_pairs<M, false><<<pgrid, 32 * kPairWarps, 0, s>>>(d, ctx->ps[0], ctx->vl[0], B0);
  if (tm) cudaEventRecord(ev[4], s);
  if (d.Fwall) k_walls<M><<<blocks_for(d.N, bs), bs, 0, s>>>(d, ctx->ps[0]);
  // the sum kernel as a programmatic dependent of the kernel before it: its
  // blocks start on the SMs the pair kernel's blocks leave, read their rows
  // and wait there for the pair kernel's results
  cudaLaunchConfig_t lc{};
  lc.gridDim = dim3(blocks_for(d.N, bs));
  lc.blockDim = dim3(bs);
  lc.dynamicSmemBytes = 0;
  lc.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  const int sft = store_ft ? 1 : 0;
  const unsigned char* flag = ctx->vl[0].flag;
  if (one)
    cudaLaunchKernelEx(&lc, k_gather_integrate<M, true>, d, ctx->ps[0], flag, sft, B0);
  else
    cudaLaunchKernelEx(&lc, k_gather_integrate<M, false>, d, ctx->ps[0], flag, sft, B0);
  if (tm) cudaEventRecord(ev[5], s);
}

// one step launched directly (no graph)
template <int M>
void enqueue_compact(dem_ctx* ctx, bool store_ft) {
  cudaStream_t s = ctx->stream;
  const bool tm = ctx->tm.on;
  cudaEvent_t* ev = ctx->tm.ev[ctx->tm.used % kRing];
  if (tm) cudaEventRecord(ev[0], s);
  k_decide<<<1, 32, 0, s>>>(ctx->dev.vctl, ctx->always_resort ? 1 : 0, 0, 0);
  enqueue_resort<M>(ctx, s, tm, ev);
  enqueue_tail<M>(ctx, store_ft, tm, ev);
}

// one step launched directly; returns the parity after it
int enqueue(dem_ctx* ctx, int p, bool store_ft) {
  if (ctx->fused) {
    switch (ctx->mode) {
      case kFP64: enqueue_fused<kFP64>(ctx, p, store_ft); break;
      case kMIXED: enqueue_fused<kMIXED>(ctx, p, store_ft); break;
      default: enqueue_fused<kFP32>(ctx, p, store_ft); break;
    }
    return 1 - p;
  }
  switch (ctx->mode) {
    case kFP64: enqueue_compact<kFP64>(ctx, store_ft); break;
    case kMIXED: enqueue_compact<kMIXED>(ctx, store_ft); break;
    default: enqueue_compact<kFP32>(ctx, store_ft); break;
  }
  return p;
}

void enqueue_resort_any(dem_ctx* ctx, cudaStream_t rs) {
  switch (ctx->mode) {
    case kFP64: enqueue_resort<kFP64>(ctx, rs, false, nullptr); break;
    case kMIXED: enqueue_resort<kMIXED>(ctx, rs, false, nullptr); break;
    default: enqueue_resort<kFP32>(ctx, rs, false, nullptr); break;
  }
}

void enqueue_tail_any(dem_ctx* ctx, bool store_ft) {
  switch (ctx->mode) {
    case kFP64: enqueue_tail<kFP64>(ctx, store_ft, false, nullptr); break;
    case kMIXED: enqueue_tail<kMIXED>(ctx, store_ft, false, nullptr); break;
    default: enqueue_tail<kFP32>(ctx, store_ft, false, nullptr); break;
  }
}

dem_status check_box(dem_ctx* ctx, int32_t box) {
  if (!ctx) return fail(ctx, DEM_ERR_ARG, "null context");
  if (box < 0 || box >= (int)ctx->boxes.size())
    return fail(ctx, DEM_ERR_ARG, "box index out of range");
  return DEM_OK;
}

dem_status upload_box(dem_ctx* ctx, int b) {
  CK(cudaMemcpyAsync((void*)(ctx->dev.boxes + b), &ctx->hbox[b], sizeof(BoxDev),
                     cudaMemcpyHostToDevice, ctx->stream));
  return DEM_OK;
}

dem_status read_status(dem_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->h_status, ctx->dev.status, sizeof(unsigned),
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->sticky |= *ctx->h_status;
  unsigned st = ctx->sticky;
  if (st & (kStRowOverflow | kStListOverflow))
    return fail(ctx, DEM_ERR_CAPACITY,
                (st & kStRowOverflow) ? "a particle has more contacts than row_capacity"
                                      : "contact list longer than its capacity");
  if (st & (kStNonFinite | kStRange))
    return fail(ctx, DEM_ERR_NONFINITE, "non-finite or out-of-range particle state");
  if (st & kStInconsistent)
    return fail(ctx, DEM_ERR_STATE, "contact seen by one member of a pair only");
  return DEM_OK;
}

}  // namespace

// ==========================================================================
// C ABI
// ==========================================================================
extern "C" {

int32_t dem_abi_version(void) { return DEM_ABI_VERSION; }

const char* dem_last_error(const dem_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

int32_t dem_launches_per_step(const dem_ctx* ctx) {
  return ctx ? launches_per_step(ctx) : 0;
}

// Device state for ctx->boxes from scratch: per-box geometry, cell grids and
// material constants, every device array, their initial contents.  Used by
// dem_create and by the layout tuner (which re-creates it for other grids,
// skins and size splits).  On failure *msg says why and nothing stays
// allocated.
// resident blocks per SM of the context's pair kernel
static cudaError_t pairs_per_sm(const dem_ctx* ctx, int* per_sm) {
  const bool one = ctx->hbox.size() == 1;
  const int nt = 32 * kPairWarps;
  switch (ctx->mode) {
    case kFP64:
      return one ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_pairs<kFP64, true>, nt, 0)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_pairs<kFP64, false>, nt, 0);
    case kMIXED:
      return one ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_pairs<kMIXED, true>, nt, 0)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_pairs<kMIXED, false>, nt, 0);
    default:
      return one ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_pairs<kFP32, true>, nt, 0)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_pairs<kFP32, false>, nt, 0);
  }
}

static dem_status setup_device(dem_ctx* ctx, std::string* msg) {
  auto bail = [&](dem_status s, const std::string& m) {
    *msg = m;
    free_all(ctx);
    return s;
  };
  // derived state of a previous set-up
  for (auto& g : ctx->gexec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  free_all(ctx);
  ctx->hbox.clear();
  ctx->hwalls.clear();
  ctx->nwh = 0;
  ctx->split = false;
  ctx->always_resort = false;
  ctx->dev = Dev{};
  for (int p = 0; p < 2; ++p) {
    ctx->ps[p] = PState{};
    ctx->cl[p] = CList{};
    ctx->vl[p] = VList{};
  }
  ctx->cs_cur = ctx->cs_new = nullptr;
  ctx->collect = ctx->chg = nullptr;
  ctx->staging = nullptr;
  ctx->staging_i = nullptr;
  ctx->parity = 0;
  ctx->sticky = 0;
  ctx->have_particles = false;
  ctx->have_ft = false;
  // ---- boxes: geometry, cell grids, material constants --------------------
  long long N = 0, Mlin = 0, Mrank = 0;
  int max_cap = 0;
  std::vector<std::vector<int>> rank_tab(ctx->boxes.size());
  for (size_t b = 0; b < ctx->boxes.size(); ++b) {
    const dem_box& bx = ctx->boxes[b];
    BoxDev B{};
    if (bx.material < 0 || bx.material >= (int)ctx->mats.size())
      return bail(DEM_ERR_ARG, "box material index out of range");
    const dem_material& mt = ctx->mats[bx.material];
    if (!(mt.E > 0) || !(mt.poisson > -1 && mt.poisson < 0.5) || !(mt.density > 0) ||
        !(mt.restitution > 0 && mt.restitution <= 1) || !(mt.mu_d >= 0))
      return bail(DEM_ERR_ARG, "material parameters out of range");
    if (!(bx.r_max > 0) || !(bx.dt > 0) || bx.max_particles < 0 ||
        bx.max_particles > (1ll << 30))
      return bail(DEM_ERR_ARG, "box needs r_max > 0, dt > 0, capacity in [0, 2^30]");
    if (bx.floor_wall && bx.periodic[2])
      return bail(DEM_ERR_ARG, "floor wall needs a non-periodic z axis");
    if (!(bx.r_split >= 0) || bx.r_split > bx.r_max)
      return bail(DEM_ERR_ARG, "r_split outside [0, r_max]");
    const bool split = bx.r_split > 0;
    if (split && ctx->fused)
      return bail(DEM_ERR_ARG, "a size-binned box (r_split > 0) needs DEM_COLLIDE_COMPACT");
    if (!(bx.skin >= 0) || !std::isfinite(bx.skin))
      return bail(DEM_ERR_ARG, "skin must be finite and >= 0");
    if (bx.skin > 0 && ctx->fused)
      return bail(DEM_ERR_ARG, "a skin needs DEM_COLLIDE_COMPACT (the per-particle forms search every step)");
    const double skin = bx.skin;
    ctx->split = ctx->split || split;
    long long ncell = 1;
    for (int a = 0; a < 3; ++a) {
      if (!(bx.L[a] > 0) || bx.L[a] * 0x1p60 >= 0x1p62)
        return bail(DEM_ERR_ARG, "box length out of range (0, 4 m)");
      int n = bx.ncell[a];
      // candidate pairs (reach r_i + r_j + skin) of small particles within
      // +-1 cell; with r_split, those of large ones within +-2
      const double hmin = (split ? std::max(2.0 * bx.r_split + skin, bx.r_max + 0.5 * skin)
                                 : 2.0 * bx.r_max + skin) * (1.0 + 1e-5);
      if (n <= 0) n = std::max(1, (int)std::floor(bx.L[a] / hmin));
      if (bx.L[a] / n < hmin)
        return bail(DEM_ERR_ARG, split ? "cells narrower than max(2 r_split + skin, r_max + skin / 2) (1 + 1e-5)"
                                       : "cells narrower than (2 r_max + skin) (1 + 1e-5)");
      if (bx.periodic[a] && n < (split ? 5 : 3))
        return bail(DEM_ERR_ARG, split ? "a periodic axis of a size-binned box needs at least 5 cells"
                                       : "a periodic axis needs at least 3 cells");
      if (n > kMaxAxisCells) return bail(DEM_ERR_ARG, "more than 1024 cells on an axis");
      B.n[a] = n;
      B.periodic[a] = bx.periodic[a] ? 1 : 0;
      B.Lq[a] = std::llround(std::ldexp(bx.L[a], kFixShift));
      B.Hq[a] = B.Lq[a] / n;
      B.L[a] = bx.L[a];
      B.half_L[a] = 0.5 * bx.L[a];
      B.inv_h[a] = (double)n / bx.L[a];
      B.Lf[a] = (float)bx.L[a];
      B.half_Lf[a] = 0.5f * B.Lf[a];
      B.inv_hf[a] = (float)((double)n / bx.L[a]);
      long long H = B.Hq[a], L = B.Lq[a];
      long long S[5] = {-H, 0, H, (long long)(n - 1) * H - L, L - (long long)(n - 1) * H};
      for (int k = 0; k < 5; ++k) B.shift[a][k] = (float)S[k] * 0x1p-60f;
      B.h[a] = bx.L[a] / n;
      if (ctx->mode == kMIXED) {
        B.hcell[a][0] = (float)H * 0x1p-60f;
        B.hcell[a][1] = B.periodic[a] ? (float)(L - (long long)(n - 1) * H) * 0x1p-60f : INFINITY;
      } else {
        B.hcell[a][0] = (float)B.h[a];
        B.hcell[a][1] = B.periodic[a] ? (float)B.h[a] : INFINITY;
      }
      ncell *= n;
    }
    if (ncell > (1ll << 30)) return bail(DEM_ERR_ARG, "too many cells");
    B.floor_wall = bx.floor_wall ? 1 : 0;
    B.rmax_f = (float)bx.r_max;
    B.rsplit_f = split ? (float)bx.r_split : INFINITY;
    // The skin test.  A pair left out of the candidate list at a re-sort was
    // at least r_i + r_j + skin apart, less the FP32 rounding of that test
    // (far below 1e-5 of the reach); the contact rule accepts nothing
    // farther than r_i + r_j plus its own rounding (the same bound).  So no
    // pair outside the list can touch while every particle has moved less
    // than half of skin - 1e-5 (4 r_max + skin), less in DEM_FP32 the
    // rounding of its float positions (a few units of the last place of
    // the box length) in the tests and in the displacement itself.
    {
      double lim = skin - 1e-5 * (4.0 * bx.r_max + skin);
      if (ctx->mode == kFP32) {
        const double Lmax = std::max(bx.L[0], std::max(bx.L[1], bx.L[2]));
        const double ulp = std::ldexp(1.0, std::ilogb(Lmax) - 23);
        lim -= 20.0 * ulp;
      }
      lim *= 0.5;
      B.skin_f = (float)skin;
      B.disp2_lim = lim > 0 ? std::nextafter((float)(lim * lim * (1.0 - 1e-6)), 0.0f) : -1.0f;
      if (B.disp2_lim < 0.0f) ctx->always_resort = true;
    }
    // rectangle and line walls
    if (bx.nwalls < 0 || (bx.nwalls > 0 && !bx.walls) || B.floor_wall + bx.nwalls > 15)
      return bail(DEM_ERR_ARG, "a box holds 0 to 15 walls (floor included), listed in walls");
    B.nwalls = bx.nwalls;
    B.wall_base = (int)ctx->hwalls.size();
    for (int k = 0; k < bx.nwalls; ++k) {
      const dem_wall& w = bx.walls[k];
      auto dot = [](const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
      const double uu = dot(w.u, w.u), vv = dot(w.v, w.v);
      const bool ok_kind = w.kind == DEM_WALL_RECT || w.kind == DEM_WALL_LINE;
      const bool finite = std::isfinite(uu) && std::isfinite(vv) && std::isfinite(dot(w.p, w.p));
      if (!ok_kind || !finite || !(uu > 0) ||
          (w.kind == DEM_WALL_RECT && (!(vv > 0) || std::fabs(dot(w.u, w.v)) > 1e-9 * std::sqrt(uu * vv))))
        return bail(DEM_ERR_ARG, "wall: kind RECT or LINE, non-zero edges, rectangle edges perpendicular");
      WallDev W{};
      W.kind = w.kind == DEM_WALL_RECT ? 0 : 1;
      for (int a = 0; a < 3; ++a) {
        W.p[a] = w.p[a];
        W.u[a] = w.u[a];
        W.v[a] = W.kind == 0 ? w.v[a] : 0.0;
        W.pf[a] = (float)W.p[a];
        W.uf[a] = (float)W.u[a];
        W.vf[a] = (float)W.v[a];
      }
      W.inv_uu = 1.0 / uu;
      W.inv_vv = W.kind == 0 ? 1.0 / vv : 0.0;
      W.inv_uuf = (float)W.inv_uu;
      W.inv_vvf = (float)W.inv_vv;
      // FP32 geometry errs by a few ulps of the coordinates involved
      const double span = std::sqrt(dot(w.p, w.p)) + std::sqrt(uu) + (W.kind == 0 ? std::sqrt(vv) : 0.0) +
                          std::max(bx.L[0], std::max(bx.L[1], bx.L[2]));
      W.slack = (float)(1e-5 * span + 1e-3 * bx.r_max);
      ctx->hwalls.push_back(W);
    }
    ctx->nwh = std::max(ctx->nwh, B.floor_wall + B.nwalls);
    B.ncells = (int)ncell;
    B.lin_base = (int)Mlin;
    B.rank_base = (int)Mrank;
    B.pbase = (int)N;
    B.cap = (int)bx.max_particles;
    B.nlive = 0;
    B.dt = bx.dt;
    B.dt_f = (float)bx.dt;
    B.dtq_f = (float)std::ldexp(bx.dt, kFixShift);
    for (int a = 0; a < 3; ++a) {
      B.g[a] = bx.g[a];
      B.g_f[a] = (float)bx.g[a];
    }
    double s = mt.poisson;
    double cn = ctx->cfg.kn_literal ? (2.0 - s * s) : (1.0 - s * s);
    double G = mt.E / (2.0 * (1.0 + s));
    B.kn_c = 4.0 / 3.0 / (cn / mt.E + cn / mt.E);
    B.kt_c = 8.0 / ((2.0 - s) / G + (2.0 - s) / G);
    B.alpha = dem_alpha_of_restitution(mt.restitution);
    if (!std::isfinite(B.alpha)) return bail(DEM_ERR_ARG, "restitution too small");
    B.mu = mt.mu_d;
    B.kn_cf = (float)B.kn_c;
    B.kt_cf = (float)B.kt_c;
    B.alpha_f = (float)B.alpha;
    B.mu_f = (float)B.mu;
    B.density = mt.density;
    // box-local Morton rank of every cell (dense)
    std::vector<std::pair<uint64_t, int>> codes((size_t)ncell);
    for (int cz = 0, l = 0; cz < B.n[2]; ++cz)
      for (int cy = 0; cy < B.n[1]; ++cy)
        for (int cx = 0; cx < B.n[0]; ++cx, ++l)
          codes[l] = {morton3(cx, cy, cz), l};
    std::sort(codes.begin(), codes.end());
    rank_tab[b].resize((size_t)ncell);
    for (long long r = 0; r < ncell; ++r) rank_tab[b][codes[r].second] = (int)r;
    N += bx.max_particles;
    Mlin += ncell;
    Mrank += ncell + 1;
    max_cap = std::max(max_cap, (int)bx.max_particles);
    ctx->hbox.push_back(B);
  }
  const long long scan_limit = (long long)kScanTile * kScanTopThreads * kScanTopItems;
  if (N > scan_limit || Mrank > scan_limit)
    return bail(DEM_ERR_ARG, "more than 2^24 slots or cells in one context");
  ctx->N = (int)N;
  ctx->M_lin = (int)Mlin;
  ctx->M_rank = (int)Mrank;
  ctx->max_cap = max_cap;
  // dense list: 8 contacts per particle on average is ample (dense
  // packings hold 1-3); the fused layout needs a block per particle of the
  // most contacts one particle may own
  long long cmax = (long long)N * (ctx->fused ? std::max(4, ctx->K / 2) : std::max(4, ctx->K / 4));
  if (cmax > (1ll << 31) - 1) cmax = (1ll << 31) - 1;
  ctx->Cmax = (int)std::max(1ll, cmax);
  ctx->ko = (int)std::max(1ll, cmax / std::max(1ll, N));

  // ---- device allocations ----------------------------------------------------
  const int M = ctx->mode;
  const size_t n = (size_t)std::max(1, ctx->N);
  Dev& d = ctx->dev;
  d.N = ctx->N;
  d.K = ctx->K;
  d.Cmax = ctx->Cmax;
  d.M_lin = ctx->M_lin;
  d.M_rank = ctx->M_rank;
  d.nbox = (int)ctx->hbox.size();
  bool ok = true;
  auto A = [&](size_t bytes) {
    void* p = dalloc(ctx, bytes);
    ok = ok && p;
    return p;
  };
  d.boxes = (const BoxDev*)A(sizeof(BoxDev) * ctx->hbox.size());
  d.walls = ctx->hwalls.empty() ? nullptr : (const WallDev*)A(sizeof(WallDev) * ctx->hwalls.size());
  d.nwh = ctx->nwh;
  d.slot_box = (const int*)A(sizeof(int) * n);
  d.rank_of_lin = (const int*)A(sizeof(int) * std::max(1, ctx->M_lin));
  d.lin_of_rank = (const int*)A(sizeof(int) * std::max(1, ctx->M_rank));
  d.ccount = (int*)A(sizeof(int) * std::max(1, ctx->M_rank));
  d.ccur = (int*)A(sizeof(int) * std::max(1, ctx->M_rank));
  ctx->cs_cur = (int*)A(sizeof(int) * std::max(1, ctx->M_rank));
  ctx->cs_new = (int*)A(sizeof(int) * std::max(1, ctx->M_rank));
  ctx->collect = (unsigned char*)A(std::max(1, ctx->M_rank));
  ctx->chg = (unsigned char*)A(std::max(1, ctx->M_rank));
  d.crange = (int2*)A(sizeof(int2) * std::max(1, ctx->M_lin));
  d.cellbox = (float4*)A(2 * sizeof(float4) * std::max(1, ctx->M_lin));
  d.perm = (int*)A(sizeof(int) * n);
  d.pcell = (int*)A(sizeof(int) * n);
  d.row = (int*)A(sizeof(int) * n * ctx->K);
  if (ctx->split) {
    d.large = (int*)A(sizeof(int) * n);
    d.nlarge = (int*)A(sizeof(int));
  }
  d.icnt = (int*)A(sizeof(int) * n);
  d.prev = (int*)A(sizeof(int) * n);
  d.Fc = A(2 * v4_bytes(M) * ctx->Cmax);
  if (ctx->fused) {
    d.Ffused = A(v4_bytes(M) * n);
    d.Tfused = A(v4_bytes(M) * n);
  } else {
    d.inrow = (int2*)A(sizeof(int2) * n * ctx->K);
    d.frow = (int*)A(sizeof(int) * n * ctx->K);
    d.fcnt = (int*)A(sizeof(int) * n);
    d.next = (int*)A(sizeof(int) * n);
    d.xb = A(pos_bytes(M) * n);
    d.yb = A(pos_bytes(M) * n);
    d.zb = A(pos_bytes(M) * n);
  }
  d.vctl = (unsigned*)A(sizeof(unsigned) * kCtlWords);
  if (!ctx->hwalls.empty()) {
    d.Fwall = A(v4_bytes(M) * n);
    d.Twall = A(v4_bytes(M) * n);
  }
  d.Fout = A(v4_bytes(M) * n);
  d.Tout = A(v4_bytes(M) * n);
  d.status = (unsigned*)A(sizeof(unsigned));
  d.diag = (unsigned*)A(sizeof(unsigned) * 2 * ctx->hbox.size());
  d.scan_bsum = (int*)A(sizeof(unsigned long long) * kScanTopThreads * kScanTopItems);
  for (int p = 0; p < 2; ++p) {
    PState& s = ctx->ps[p];
    s.px = A(pos_bytes(M) * n);
    s.py = A(pos_bytes(M) * n);
    s.pz = A(pos_bytes(M) * n);
    s.vel = A(v4_bytes(M) * n);
    s.omg = A(v4_bytes(M) * n);
    s.posr = A(v4_bytes(M) * n);
    s.id = (int*)A(sizeof(int) * n);
    s.cellc = (int*)A(sizeof(int) * n);
    s.cellx = (int*)A(sizeof(int) * n);
    s.cellg = (int*)A(sizeof(int) * n);
    if (ctx->nwh > 0) {
      s.wx = A(dt_bytes(M) * n * ctx->nwh);
      s.wy = A(dt_bytes(M) * n * ctx->nwh);
      s.wz = A(dt_bytes(M) * n * ctx->nwh);
    }
    if (ctx->fused) {
      CList& c = ctx->cl[p];
      c.pair = (int2*)A(sizeof(int2) * ctx->Cmax);
      c.hid = (int2*)A(sizeof(int2) * ctx->Cmax);
      c.dx = A(dt_bytes(M) * ctx->Cmax);
      c.dy = A(dt_bytes(M) * ctx->Cmax);
      c.dz = A(dt_bytes(M) * ctx->Cmax);
      c.hs = (int*)A(sizeof(int) * n);
      c.oc = (int*)A(sizeof(int) * n);
      c.count = (int*)A(sizeof(int));
    } else {
      VList& c = ctx->vl[p];
      c.pair = (int2*)A(sizeof(int2) * ctx->Cmax);
      c.hid = nullptr;  // ids come from the slots' ids when they are read
      c.dx = A(dt_bytes(M) * ctx->Cmax);
      c.dy = A(dt_bytes(M) * ctx->Cmax);
      c.dz = A(dt_bytes(M) * ctx->Cmax);
      c.flag = (unsigned char*)A(ctx->Cmax);
      c.hs = (int*)A(sizeof(int) * n);
      c.oc = (int*)A(sizeof(int) * n);
      c.count = (int*)A(sizeof(int));
    }
  }
  ctx->staging = (double*)A(sizeof(double) * 16 * (size_t)std::max(1, max_cap));
  ctx->staging_i = (int*)A(sizeof(int) * 2 * (size_t)std::max(1, max_cap));
  if (!ok) return bail(DEM_ERR_ALLOC, "device allocation failed");

  // ---- initial contents --------------------------------------------------------
  std::vector<int> slot_box(n, 0), rol(std::max(1, ctx->M_lin)),
      lor(std::max(1, ctx->M_rank)), cnt(std::max(1, ctx->M_rank), 0);
  for (size_t b = 0; b < ctx->hbox.size(); ++b) {
    const BoxDev& B = ctx->hbox[b];
    for (int k = 0; k < B.cap; ++k) slot_box[B.pbase + k] = (int)b;
    for (int l = 0; l < B.ncells; ++l) {
      int r = rank_tab[b][l];
      rol[B.lin_base + l] = r;
      lor[B.rank_base + r] = B.lin_base + l;
    }
    lor[B.rank_base + B.ncells] = -1;
    cnt[B.rank_base + B.ncells] = B.cap;  // all slots free
  }
  cudaStream_t s = ctx->stream;
  auto H2D = [&](const void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync((void*)dst, src, bytes, cudaMemcpyHostToDevice, s);
  };
  cudaError_t e = cudaSuccess;
  if (!e) e = H2D(d.boxes, ctx->hbox.data(), sizeof(BoxDev) * ctx->hbox.size());
  if (!e && !ctx->hwalls.empty())
    e = H2D(d.walls, ctx->hwalls.data(), sizeof(WallDev) * ctx->hwalls.size());
  if (!e) e = H2D(d.slot_box, slot_box.data(), sizeof(int) * n);
  if (!e) e = H2D(d.rank_of_lin, rol.data(), sizeof(int) * rol.size());
  if (!e) e = H2D(d.lin_of_rank, lor.data(), sizeof(int) * lor.size());
  if (!e) e = H2D(d.ccount, cnt.data(), sizeof(int) * cnt.size());
  if (!e) e = cudaMemsetAsync(d.status, 0, sizeof(unsigned), s);
  if (!e) e = cudaMemsetAsync(d.diag, 0, sizeof(unsigned) * 2 * ctx->hbox.size(), s);
  if (!e) e = cudaMemsetAsync(d.icnt, 0, sizeof(int) * n, s);
  if (!e) e = cudaMemsetAsync(ctx->collect, 1, std::max(1, ctx->M_rank), s);
  if (!e) e = cudaMemsetAsync(ctx->chg, 1, std::max(1, ctx->M_rank), s);
  if (!e) e = cudaMemsetAsync(ctx->cs_cur, 0, sizeof(int) * std::max(1, ctx->M_rank), s);
  if (!e) e = cudaMemsetAsync(ctx->cs_new, 0, sizeof(int) * std::max(1, ctx->M_rank), s);
  if (!e) e = cudaMemsetAsync(d.vctl, 0, sizeof(unsigned) * kCtlWords, s);
  for (int p = 0; p < 2 && !e; ++p) {
    int* oc = ctx->fused ? ctx->cl[p].oc : ctx->vl[p].oc;
    int* hs = ctx->fused ? ctx->cl[p].hs : ctx->vl[p].hs;
    int* cnt = ctx->fused ? ctx->cl[p].count : ctx->vl[p].count;
    e = cudaMemsetAsync(oc, 0, sizeof(int) * n, s);
    if (!e) e = cudaMemsetAsync(hs, 0, sizeof(int) * n, s);
    if (!e) e = cudaMemsetAsync(cnt, 0, sizeof(int), s);
  }
  if (!e && !ctx->fused) e = cudaMemsetAsync(d.fcnt, 0, sizeof(int) * n, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (e) return bail(DEM_ERR_CUDA, std::string("initialisation: ") + cudaGetErrorString(e));
  // the pair kernel runs as one wave: as many blocks as the GPU holds at
  // once (queried here, outside any stream capture)
  int per_sm = 0;
  e = pairs_per_sm(ctx, &per_sm);
  if (e || per_sm < 1)
    return bail(DEM_ERR_CUDA, std::string("pair kernel occupancy: ") + cudaGetErrorString(e));
  ctx->pairs_grid = ctx->nsm * per_sm;
  return DEM_OK;
}

static dem_status prepare_graphs(dem_ctx* ctx);

dem_status dem_create(const dem_config* cfg, dem_ctx** out) {
  dem_ctx* ctx = nullptr;
  if (!out) return fail(nullptr, DEM_ERR_ARG, "out is null");
  *out = nullptr;
  if (!cfg || cfg->nboxes <= 0 || !cfg->boxes || cfg->nmaterials <= 0 ||
      !cfg->materials)
    return fail(nullptr, DEM_ERR_ARG, "config needs boxes and materials");
  if (cfg->precision < 0 || cfg->precision > 2)
    return fail(nullptr, DEM_ERR_ARG, "bad precision");
  if (cfg->collide != DEM_COLLIDE_COMPACT && cfg->collide != DEM_COLLIDE_FUSED &&
      cfg->collide != DEM_COLLIDE_TWOLOOP)
    return fail(nullptr, DEM_ERR_ARG,
                "collide must be DEM_COLLIDE_COMPACT, DEM_COLLIDE_FUSED or DEM_COLLIDE_TWOLOOP");
  if (!!cfg->alloc != !!cfg->free)
    return fail(nullptr, DEM_ERR_ARG, "alloc and free hooks go together");
  ctx = new dem_ctx();
  ctx->cfg = *cfg;
  ctx->boxes.assign(cfg->boxes, cfg->boxes + cfg->nboxes);
  ctx->mats.assign(cfg->materials, cfg->materials + cfg->nmaterials);
  ctx->cfg.boxes = nullptr;
  ctx->cfg.materials = nullptr;
  ctx->mode = cfg->precision == DEM_FP64 ? kFP64
              : cfg->precision == DEM_MIXED ? kMIXED : kFP32;
  ctx->K = cfg->row_capacity > 0 ? cfg->row_capacity : 32;
  ctx->fused = cfg->collide == DEM_COLLIDE_FUSED || cfg->collide == DEM_COLLIDE_TWOLOOP;
  ctx->twoloop = cfg->collide == DEM_COLLIDE_TWOLOOP;
  ctx->block = cfg->block > 0 ? cfg->block : 128;  // the tuners' usual pick
  ctx->graph_steps = cfg->graph_steps == 0 ? 16 : cfg->graph_steps;
  if (ctx->graph_steps > 0 && (ctx->graph_steps & 1)) ctx->graph_steps += 1;
  auto bail = [&](dem_status s, const std::string& m) {
    g_create_error = m;
    if (ctx) {
      free_all(ctx);
      if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
      if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
      if (ctx->body_stream) cudaStreamDestroy(ctx->body_stream);
      for (cudaEvent_t& e : ctx->xfer_ev)
        if (e) cudaEventDestroy(e);
      if (ctx->h_status) cudaFreeHost(ctx->h_status);
      if (ctx->h_count) cudaFreeHost(ctx->h_count);
      delete ctx;
    }
    return s;
  };
  if (ctx->K < 2 || ctx->K > 1024) return bail(DEM_ERR_ARG, "row_capacity out of range");
  // rows are read four entries at a time, the first eight at once
  ctx->K = std::max(8, (ctx->K + 3) & ~3);
  if (ctx->block < 32 || ctx->block > 1024 || (ctx->block & 31))
    return bail(DEM_ERR_ARG, "block must be a multiple of 32 in [32, 1024]");
  const int l2f = cfg->l2_fetch == 0 ? 64 : cfg->l2_fetch;
  if (l2f != -1 && l2f != 32 && l2f != 64 && l2f != 128)
    return bail(DEM_ERR_ARG, "l2_fetch must be -1, 0, 32, 64 or 128");
  if (cudaGetDevice(&ctx->device) != cudaSuccess)
    return bail(DEM_ERR_CUDA, "no CUDA device");
  // the context's L2 fetch granularity: the per-particle sum reads scattered
  // 32-byte records, which a larger fetch would bring in with neighbours it
  // does not use (measured at 1 M particles: 71 against 76 us per launch)
  if (l2f > 0 && cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)l2f) != cudaSuccess)
    return bail(DEM_ERR_CUDA, "cannot set the L2 fetch granularity");
  cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->device);
  if (cfg->stream) {
    ctx->stream = (cudaStream_t)cfg->stream;
  } else {
    if (cudaStreamCreate(&ctx->stream) != cudaSuccess)
      return bail(DEM_ERR_CUDA, "stream creation failed");
    ctx->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->body_stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(DEM_ERR_CUDA, "stream creation failed");
  for (cudaEvent_t& e : ctx->xfer_ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return bail(DEM_ERR_CUDA, "event creation failed");

  // the walls are read during the call: keep copies for later set-ups
  ctx->wall_src.resize(ctx->boxes.size());
  for (size_t b = 0; b < ctx->boxes.size(); ++b) {
    dem_box& bx = ctx->boxes[b];
    if (bx.nwalls > 0 && bx.walls && bx.nwalls <= 15)
      ctx->wall_src[b].assign(bx.walls, bx.walls + bx.nwalls);
    bx.walls = ctx->wall_src[b].empty() ? nullptr : ctx->wall_src[b].data();
    if (bx.nwalls > 0 && ctx->wall_src[b].empty()) bx.walls = nullptr;
  }
  if (cudaMallocHost(&ctx->h_status, sizeof(unsigned)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_count, sizeof(int)) != cudaSuccess)
    return bail(DEM_ERR_ALLOC, "pinned host allocation failed");
  std::string msg;
  const dem_status st = setup_device(ctx, &msg);
  if (st) return bail(st, msg);
  *out = ctx;
  return prepare_graphs(ctx);
}

dem_status dem_destroy(dem_ctx* ctx) {
  if (!ctx) return DEM_OK;
  for (auto& g : ctx->gexec)
    if (g) cudaGraphExecDestroy(g);
  if (ctx->tm.made)
    for (auto& set : ctx->tm.ev)
      for (auto& ev : set) cudaEventDestroy(ev);
  free_all(ctx);
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  if (ctx->h_count) cudaFreeHost(ctx->h_count);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->body_stream) cudaStreamDestroy(ctx->body_stream);
  for (cudaEvent_t& e : ctx->xfer_ev)
    if (e) cudaEventDestroy(e);
  delete ctx;
  return DEM_OK;
}

dem_status dem_set_particles(dem_ctx* ctx, int32_t box, int64_t n,
                             const double* x, const double* v,
                             const double* omega, const double* radius,
                             int32_t where) {
  dem_status st = check_box(ctx, box);
  if (st) return st;
  BoxDev& B = ctx->hbox[box];
  if (n < 0 || n > B.cap) return fail(ctx, DEM_ERR_ARG, "n exceeds the box capacity");
  if (n > 0 && (!x || !v || !omega || !radius))
    return fail(ctx, DEM_ERR_ARG, "x, v, omega and radius are required");
  if (where != DEM_HOST && where != DEM_DEVICE) return fail(ctx, DEM_ERR_ARG, "bad where");
  const double rmax = ctx->boxes[box].r_max;
  if (where == DEM_HOST) {
    for (int64_t k = 0; k < n; ++k) {
      double r = radius[k];
      if (!(r > 0.0) || r > rmax)
        return fail(ctx, DEM_ERR_ARG, "radius outside (0, r_max]");
      for (int a = 0; a < 3; ++a)
        if (!std::isfinite(x[3 * k + a]) || !std::isfinite(v[3 * k + a]) ||
            !std::isfinite(omega[3 * k + a]))
          return fail(ctx, DEM_ERR_ARG, "non-finite particle state");
    }
  }
  cudaStream_t s = ctx->stream;
  const int p = ctx->parity;
  // clear the box's cell counts; all unused slots go to its free-slot cell
  CK(cudaMemsetAsync(ctx->dev.ccount + B.rank_base, 0, sizeof(int) * B.ncells, s));
  int freec = B.cap - (int)n;
  CK(cudaMemcpyAsync(ctx->dev.ccount + B.rank_base + B.ncells, &freec, sizeof(int),
                     cudaMemcpyHostToDevice, s));
  B.nlive = (int)n;
  st = upload_box(ctx, box);
  if (st) return st;
  // the box's history is empty: no slot of the box holds a stored contact
  if (!ctx->fused && B.cap > 0)
    k_clear_flags<<<blocks_for(B.cap, 256), 256, 0, s>>>(ctx->vl[0], B.pbase, B.cap);
  for (int q = 0; q < 2; ++q)
    CK(cudaMemsetAsync((ctx->fused ? ctx->cl[q].oc : ctx->vl[q].oc) + B.pbase, 0,
                       sizeof(int) * B.cap, s));
  // the next sort starts from the order the particles were given in, and
  // the next step re-sorts
  CK(cudaMemsetAsync(ctx->collect, 1, std::max(1, ctx->M_rank), s));
  CK(cudaMemsetAsync(ctx->dev.vctl + kCtlRequest, 1, sizeof(unsigned), s));
  if (n > 0) {
    const double *dx = x, *dv = v, *dw = omega, *dr = radius;
    if (where == DEM_HOST) {
      double* stg = ctx->staging;
      CK(cudaMemcpyAsync(stg, x, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(stg + 3 * n, v, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(stg + 6 * n, omega, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(stg + 9 * n, radius, sizeof(double) * n, cudaMemcpyHostToDevice, s));
      dx = stg;
      dv = stg + 3 * n;
      dw = stg + 6 * n;
      dr = stg + 9 * n;
    }
    int nb = blocks_for(n, 256);
    switch (ctx->mode) {
      case kFP64: k_set_particles<kFP64><<<nb, 256, 0, s>>>(ctx->dev, ctx->ps[p], box, (int)n, dx, dv, dw, dr); break;
      case kMIXED: k_set_particles<kMIXED><<<nb, 256, 0, s>>>(ctx->dev, ctx->ps[p], box, (int)n, dx, dv, dw, dr); break;
      default: k_set_particles<kFP32><<<nb, 256, 0, s>>>(ctx->dev, ctx->ps[p], box, (int)n, dx, dv, dw, dr); break;
    }
    CK(cudaGetLastError());
  }
  ctx->have_particles = true;
  ctx->have_ft = false;
  return read_status(ctx);
}

dem_status dem_set_state(dem_ctx* ctx, int32_t box, const double* x,
                         const double* v, const double* omega, int32_t where) {
  dem_status st = check_box(ctx, box);
  if (st) return st;
  const BoxDev& B = ctx->hbox[box];
  int n = B.nlive;
  if (where != DEM_HOST && where != DEM_DEVICE) return fail(ctx, DEM_ERR_ARG, "bad where");
  if (n == 0) return DEM_OK;
  cudaStream_t s = ctx->stream, cs = ctx->copy_stream;
  const int nb = blocks_for(n, 256);
  const int p = ctx->parity;
  // one array at a time: its copy (host data) on the copy stream, then its
  // kernel on the context's stream, so that copies and kernels overlap
  const double* in[3] = {x, v, omega};
  if (where == DEM_HOST) {
    // the staging buffer is free once the context's earlier work is done
    CK(cudaEventRecord(ctx->xfer_ev[5], s));
    CK(cudaStreamWaitEvent(cs, ctx->xfer_ev[5], 0));
  }
  for (int k = 0; k < 3; ++k) {
    if (!in[k]) continue;
    const double* dk = in[k];
    if (where == DEM_HOST) {
      double* stg = ctx->staging + (size_t)3 * n * k;
      CK(cudaMemcpyAsync(stg, in[k], sizeof(double) * 3 * n, cudaMemcpyHostToDevice, cs));
      CK(cudaEventRecord(ctx->xfer_ev[k], cs));
      CK(cudaStreamWaitEvent(s, ctx->xfer_ev[k], 0));
      dk = stg;
    }
    const double* a0 = k == 0 ? dk : nullptr;
    const double* a1 = k == 1 ? dk : nullptr;
    const double* a2 = k == 2 ? dk : nullptr;
    // the contact-list pipeline tracks new positions like a step's (cells,
    // records, skin test); the per-particle forms sort every step anyway
    Dev dd = ctx->dev;
    dd.collect = ctx->collect;
    const int track = ctx->fused ? 0 : 1;
    switch (ctx->mode) {
      case kFP64: k_set_state<kFP64><<<nb, 256, 0, s>>>(dd, ctx->ps[p], box, n, a0, a1, a2, track); break;
      case kMIXED: k_set_state<kMIXED><<<nb, 256, 0, s>>>(dd, ctx->ps[p], box, n, a0, a1, a2, track); break;
      default: k_set_state<kFP32><<<nb, 256, 0, s>>>(dd, ctx->ps[p], box, n, a0, a1, a2, track); break;
    }
    CK(cudaGetLastError());
  }
  // the per-particle forms: new positions may have changed cells, the next
  // sort starts from every cell
  if (x && ctx->fused) {
    CK(cudaMemsetAsync(ctx->collect, 1, std::max(1, ctx->M_rank), s));
    CK(cudaMemsetAsync(ctx->dev.vctl + kCtlRequest, 1, sizeof(unsigned), s));
  }
  // the caller's host arrays are read by the time the call returns
  if (where == DEM_HOST) CK(cudaStreamSynchronize(cs));
  return DEM_OK;
}

// G steps in one CUDA graph.  The per-particle forms alternate the state
// parity and need one graph per starting parity.  The contact-list pipeline
// keeps its state in place: each step is a decision kernel, a conditional
// node whose body holds the re-sort kernels (run only when the decision says
// so), and the pair and integration kernels.
static dem_status build_graph(dem_ctx* ctx, int p, int nsteps, bool store_last,
                              cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  int q = p;
  cudaError_t e = cudaSuccess;
  const char* where = "";
  for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
    const bool last = k == nsteps - 1 && store_last;
    if (ctx->fused) {
      q = enqueue(ctx, q, last);
      continue;
    }
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t ndeps = 0;
    where = "capture info";
    e = cudaStreamGetCaptureInfo(ctx->stream, &cst, nullptr, &cg, &deps, &edges, &ndeps);
    cudaGraphConditionalHandle h{};
    if (e == cudaSuccess) {
      where = "conditional handle";
      e = cudaGraphConditionalHandleCreate(&h, cg, 0, 0);
    }
    if (e != cudaSuccess) break;
    k_decide<<<1, 32, 0, ctx->stream>>>(ctx->dev.vctl, ctx->always_resort ? 1 : 0, h, 1);
    e = cudaStreamGetCaptureInfo(ctx->stream, &cst, nullptr, &cg, &deps, &edges, &ndeps);
    if (e != cudaSuccess) break;
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    where = "conditional node";
    e = cudaGraphAddNode(&node, cg, deps, edges, ndeps, &cp);
    if (e == cudaSuccess)
      e = cudaStreamUpdateCaptureDependencies(ctx->stream, &node, nullptr, 1,
                                              cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) break;
    where = "re-sort body";
    e = cudaStreamBeginCaptureToGraph(ctx->body_stream, cp.conditional.phGraph_out[0], nullptr,
                                      nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) break;
    enqueue_resort_any(ctx, ctx->body_stream);
    cudaGraph_t body = nullptr;
    e = cudaStreamEndCapture(ctx->body_stream, &body);
    if (e != cudaSuccess) break;
    where = "step kernels";
    enqueue_tail_any(ctx, last);
  }
  cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return fail(ctx, DEM_ERR_CUDA, std::string("graph capture (") + where + "): " +
                                       cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(ctx, DEM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return DEM_OK;
}

// The graphs dem_step launches, instantiated ahead of the first step (at
// creation and after a tuner changed the launch configuration), so that a
// step never pays for a capture: G steps from the current parity (both
// parities for the per-particle forms) and, for the contact-list pipeline,
// the one-step graphs of the steps left over.
static dem_status prepare_graphs(dem_ctx* ctx) {
  if (ctx->graph_steps <= 0) return DEM_OK;
  if (ctx->fused) {
    for (int p = 0; p < 2; ++p)
      if (!ctx->gexec[p]) {
        dem_status st = build_graph(ctx, p, ctx->graph_steps, true, &ctx->gexec[p]);
        if (st) return st;
      }
    return DEM_OK;
  }
  const int p = ctx->parity;
  if (!ctx->gexec[p]) {
    dem_status st = build_graph(ctx, p, ctx->graph_steps, true, &ctx->gexec[p]);
    if (st) return st;
  }
  for (int k = 2; k < 4; ++k)
    if (!ctx->gexec[k]) {
      dem_status st = build_graph(ctx, p, 1, k == 3, &ctx->gexec[k]);
      if (st) return st;
    }
  return DEM_OK;
}

dem_status dem_step(dem_ctx* ctx, int64_t nsteps) {
  if (!ctx) return fail(ctx, DEM_ERR_ARG, "null context");
  if (nsteps < 0) return fail(ctx, DEM_ERR_ARG, "nsteps < 0");
  if (!ctx->have_particles) return fail(ctx, DEM_ERR_STATE, "no particles set");
  if (ctx->sticky) return read_status(ctx);
  if (nsteps == 0) return DEM_OK;
  cudaStream_t s = ctx->stream;
  CK(cudaMemsetAsync(ctx->dev.diag, 0, sizeof(unsigned) * 2 * ctx->hbox.size(), s));
  int64_t left = nsteps;
  const bool timing = ctx->tm.on;
  if (timing) {
    for (double& a : ctx->tm.acc) a = 0.0;
    ctx->tm.steps = 0;
  }
  if (ctx->graph_steps > 0 && !timing) {
    while (left >= ctx->graph_steps) {
      int p = ctx->parity;
      if (!ctx->gexec[p]) {
        dem_status st = build_graph(ctx, p, ctx->graph_steps, true, &ctx->gexec[p]);
        if (st) return st;
      }
      CK(cudaGraphLaunch(ctx->gexec[p], s));
      left -= ctx->graph_steps;  // an even number of steps: parity unchanged
    }
    // the contact-list pipeline keeps its state in place: the steps left over
    // go through one-step graphs (the re-sort kernels skipped, not launched,
    // in a step that does not re-sort)
    while (!ctx->fused && left > 0) {
      const int k = left == 1 ? 3 : 2;
      if (!ctx->gexec[k]) {
        dem_status st = build_graph(ctx, ctx->parity, 1, k == 3, &ctx->gexec[k]);
        if (st) return st;
      }
      CK(cudaGraphLaunch(ctx->gexec[k], s));
      --left;
    }
  }
  auto drain = [&]() -> dem_status {
    if (!ctx->tm.used) return DEM_OK;
    CK(cudaEventSynchronize(ctx->tm.ev[(ctx->tm.used - 1) % kRing][kPhases]));
    for (int u = 0; u < ctx->tm.used; ++u)
      for (int k = 0; k < kPhases; ++k) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ctx->tm.ev[u][k], ctx->tm.ev[u][k + 1]);
        ctx->tm.acc[k] += ms;
      }
    ctx->tm.steps += ctx->tm.used;
    ctx->tm.used = 0;
    return DEM_OK;
  };
  while (left > 0) {
    ctx->parity = enqueue(ctx, ctx->parity, left == 1);
    CK(cudaGetLastError());
    if (timing && ++ctx->tm.used == kRing) {
      dem_status st = drain();
      if (st) return st;
    }
    --left;
  }
  if (timing) {
    dem_status st = drain();
    if (st) return st;
  }
  if (timing && ctx->tm.steps)
    for (int k = 0; k < kPhases; ++k) ctx->phase_ms[k] = ctx->tm.acc[k] / ctx->tm.steps;
  ctx->have_ft = true;
  ctx->steps_done += nsteps;
  return read_status(ctx);
}

dem_status dem_autotune(dem_ctx* ctx, int64_t steps, double* best_ms,
                        int32_t* block, int32_t* graph_steps) {
  if (!ctx) return fail(ctx, DEM_ERR_ARG, "null context");
  if (!ctx->have_particles) return fail(ctx, DEM_ERR_STATE, "no particles set");
  if (steps < 4) steps = 4;
  const int blocks[3] = {128, 256, 512};
  const int graphs[3] = {8, 16, 32};
  const bool was_timing = ctx->tm.on;
  ctx->tm.on = false;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double best = 1e300;
  int bb = ctx->block, bg = ctx->graph_steps;
  for (int gb : blocks)
    for (int gg : graphs) {
      ctx->block = gb;
      ctx->graph_steps = gg;
      for (auto& g : ctx->gexec)
        if (g) {
          cudaGraphExecDestroy(g);
          g = nullptr;
        }
      // one untimed graph-length of warm-up, then the timed steps
      dem_status st = dem_step(ctx, gg);
      if (st) break;
      const int64_t k = std::max<int64_t>(steps / gg, 1) * gg;
      CK(cudaEventRecord(e0, ctx->stream));
      st = dem_step(ctx, k);
      CK(cudaEventRecord(e1, ctx->stream));
      CK(cudaEventSynchronize(e1));
      if (st) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return st;
      }
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      const double per = ms / (double)k;
      if (per < best) {
        best = per;
        bb = gb;
        bg = gg;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->block = bb;
  ctx->graph_steps = bg;
  for (auto& g : ctx->gexec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  ctx->tm.on = was_timing;
  if (best_ms) *best_ms = best;
  if (block) *block = bb;
  if (graph_steps) *graph_steps = bg;
  dem_status st = prepare_graphs(ctx);
  if (st) return st;
  return read_status(ctx);
}

}  // extern "C"

// ---- layout tuner ------------------------------------------------------------
namespace {

// the particles and pair history of every box, in id order (host)
struct Snapshot {
  std::vector<std::vector<double>> x, v, w, r, dt;
  std::vector<std::vector<int32_t>> lo, hi;
};

dem_status take_snapshot(dem_ctx* ctx, Snapshot& sn) {
  const size_t nb = ctx->boxes.size();
  sn = Snapshot{};
  sn.x.resize(nb); sn.v.resize(nb); sn.w.resize(nb); sn.r.resize(nb);
  sn.lo.resize(nb); sn.hi.resize(nb); sn.dt.resize(nb);
  for (size_t b = 0; b < nb; ++b) {
    const int n = ctx->hbox[b].nlive;
    sn.x[b].resize(3 * (size_t)n); sn.v[b].resize(3 * (size_t)n); sn.w[b].resize(3 * (size_t)n);
    sn.r[b].resize((size_t)n);
    if (n == 0) continue;
    dem_status st = dem_get_state(ctx, (int32_t)b, sn.x[b].data(), sn.v[b].data(),
                                  sn.w[b].data(), nullptr, nullptr, DEM_HOST);
    if (st) return st;
    double* dr = ctx->staging;
    const int p = ctx->parity;
    switch (ctx->mode) {
      case kFP64: k_get_radius<kFP64><<<blocks_for(n, 256), 256, 0, ctx->stream>>>(ctx->dev, ctx->ps[p], (int)b, dr); break;
      case kMIXED: k_get_radius<kMIXED><<<blocks_for(n, 256), 256, 0, ctx->stream>>>(ctx->dev, ctx->ps[p], (int)b, dr); break;
      default: k_get_radius<kFP32><<<blocks_for(n, 256), 256, 0, ctx->stream>>>(ctx->dev, ctx->ps[p], (int)b, dr); break;
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(sn.r[b].data(), dr, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    int64_t nc = 0;
    st = dem_get_contacts(ctx, (int32_t)b, 0, &nc, nullptr, nullptr, nullptr);
    if (st && st != DEM_ERR_CAPACITY) return st;
    sn.lo[b].resize((size_t)nc); sn.hi[b].resize((size_t)nc); sn.dt[b].resize(3 * (size_t)nc);
    st = dem_get_contacts(ctx, (int32_t)b, nc, &nc, sn.lo[b].data(), sn.hi[b].data(), sn.dt[b].data());
    if (st) return st;
  }
  return DEM_OK;
}

dem_status restore_snapshot(dem_ctx* ctx, const Snapshot& sn) {
  for (size_t b = 0; b < ctx->boxes.size(); ++b) {
    const int64_t n = (int64_t)sn.r[b].size();
    dem_status st = dem_set_particles(ctx, (int32_t)b, n, sn.x[b].data(), sn.v[b].data(),
                                      sn.w[b].data(), sn.r[b].data(), DEM_HOST);
    if (st) return st;
    if (!sn.lo[b].empty()) {
      st = dem_set_contacts(ctx, (int32_t)b, (int64_t)sn.lo[b].size(), sn.lo[b].data(),
                            sn.hi[b].data(), sn.dt[b].data());
      if (st) return st;
    }
  }
  return DEM_OK;
}

// the finest legal cell count per axis of a box for a skin and size split
int finest_cells(const dem_box& bx, int a, double skin, double rsplit) {
  const bool split = rsplit > 0;
  const double hmin = (split ? std::max(2.0 * rsplit + skin, bx.r_max + 0.5 * skin)
                             : 2.0 * bx.r_max + skin) * (1.0 + 1e-5);
  return std::max(1, (int)std::floor(bx.L[a] / hmin));
}

struct Layout {
  double skin_rel = 0.0, scale = 1.0, rq = 0.0;
};

// the boxes of a layout (per box: skin = skin_rel r_max, cells scale times
// the finest legal edge, r_split the rq quantile of its radii)
std::vector<dem_box> layout_boxes(const std::vector<dem_box>& base, const Snapshot& sn,
                                  const Layout& lay) {
  std::vector<dem_box> out = base;
  for (size_t b = 0; b < out.size(); ++b) {
    dem_box& bx = out[b];
    bx.skin = lay.skin_rel * bx.r_max;
    bx.r_split = 0.0;
    if (lay.rq > 0 && !sn.r[b].empty()) {
      std::vector<double> r = sn.r[b];
      const size_t k = std::min(r.size() - 1, (size_t)(lay.rq * (double)(r.size() - 1)));
      std::nth_element(r.begin(), r.begin() + (ptrdiff_t)k, r.end());
      if (r[k] > 0 && r[k] < bx.r_max) bx.r_split = r[k];
    }
    for (int a = 0; a < 3; ++a)
      bx.ncell[a] = std::max(1, (int)std::floor(finest_cells(bx, a, bx.skin, bx.r_split) / lay.scale));
  }
  return out;
}

// device ms per step of `steps` steps from the snapshot (graphs built by an
// untimed run first); a negative value when the configuration is refused
dem_status time_trial(dem_ctx* ctx, const Snapshot& sn, int64_t steps, cudaEvent_t e0,
                      cudaEvent_t e1, double* ms) {
  *ms = -1.0;
  dem_status st = restore_snapshot(ctx, sn);
  if (st) return st;
  st = dem_step(ctx, std::max<int64_t>(ctx->graph_steps, 1));
  if (st) return st;
  st = restore_snapshot(ctx, sn);
  if (st) return st;
  CK(cudaEventRecord(e0, ctx->stream));
  st = dem_step(ctx, steps);
  CK(cudaEventRecord(e1, ctx->stream));
  CK(cudaEventSynchronize(e1));
  if (st) return st;
  float t = 0.f;
  CK(cudaEventElapsedTime(&t, e0, e1));
  *ms = t / (double)steps;
  return DEM_OK;
}

}  // namespace

// ---- arithmetic peak probe -----------------------------------------------------
namespace {

// Eight independent fused multiply-add chains per thread (enough in flight
// to keep the pipe busy); the result is stored, to a file-scope sink, only
// under a condition the compiler cannot rule out (the chains stay in [0, 1]
// and their sum is never negative), so the chains are not removed.
__device__ double g_fma_sink;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_rate(int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) x[u] = (T)(threadIdx.x + u) * (T)1e-3;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = fma(x[u], a, b);
  }
  T sum = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) sum += x[u];
  if (sum < (T)0) g_fma_sink = (double)sum;
}

template <typename T>
dem_status fma_rate(cudaStream_t s, int nsm, int iters, double* tflops) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) || cudaEventCreate(&e1)) return DEM_ERR_CUDA;
  const int blocks = nsm * 8;
  k_fma_rate<T><<<blocks, 256, 0, s>>>(iters / 8, (T)0.999999, (T)1e-6);  // warm-up
  cudaEventRecord(e0, s);
  k_fma_rate<T><<<blocks, 256, 0, s>>>(iters, (T)0.999999, (T)1e-6);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e || ms <= 0.f) return DEM_ERR_CUDA;
  const double flops = 2.0 * 8.0 * (double)iters * 256.0 * (double)blocks;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return DEM_OK;
}

}  // namespace

extern "C" dem_status dem_measure_fma_rates(double* fp32_tflops, double* fp64_tflops,
                                            void* stream) {
  if (!fp32_tflops || !fp64_tflops) return fail(nullptr, DEM_ERR_ARG, "null output");
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev))
    return fail(nullptr, DEM_ERR_CUDA, "no CUDA device");
  cudaStream_t s = (cudaStream_t)stream;
  dem_status st = fma_rate<float>(s, nsm, 1 << 14, fp32_tflops);
  if (!st) st = fma_rate<double>(s, nsm, 1 << 10, fp64_tflops);
  if (st) return fail(nullptr, st, "dem_measure_fma_rates: kernel timing failed");
  return DEM_OK;
}

extern "C" dem_status dem_autotune_layout(dem_ctx* ctx, int64_t steps, dem_tuning* out) {
  if (!ctx) return fail(ctx, DEM_ERR_ARG, "null context");
  if (!ctx->have_particles) return fail(ctx, DEM_ERR_STATE, "no particles set");
  if (ctx->sticky) return read_status(ctx);
  if (steps < 4) steps = 4;
  Snapshot sn;
  dem_status st = take_snapshot(ctx, sn);
  if (st) return st;
  const bool was_timing = ctx->tm.on;
  ctx->tm.on = false;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const std::vector<dem_box> base = ctx->boxes;
  Layout best_lay;
  for (const dem_box& bx : base) {  // the layout the context starts with
    best_lay.skin_rel = std::max(best_lay.skin_rel, bx.skin / bx.r_max);
  }
  int trials = 0;
  double best = 1e300;
  int best_block = ctx->block, best_graph = ctx->graph_steps;
  auto apply = [&](const Layout& lay, std::string* msg) -> dem_status {
    if (ctx->fused) return DEM_OK;
    ctx->boxes = layout_boxes(base, sn, lay);
    return setup_device(ctx, msg);
  };
  auto trial = [&](const Layout& lay, int block, int graph, double* ms) -> dem_status {
    *ms = -1.0;
    ctx->block = block;
    ctx->graph_steps = graph;
    std::string msg;
    dem_status s2 = apply(lay, &msg);
    if (s2 == DEM_ERR_ARG) return DEM_OK;  // not a legal layout for these boxes
    if (s2) return fail(ctx, s2, msg);
    s2 = time_trial(ctx, sn, steps, e0, e1, ms);
    if (s2 == DEM_ERR_CAPACITY) {  // rows too short for this skin: not a candidate
      *ms = -1.0;
      return DEM_OK;
    }
    ++trials;
    return s2;
  };
  auto consider = [&](const Layout& lay, int block, int graph) -> dem_status {
    double ms;
    dem_status s2 = trial(lay, block, graph, &ms);
    if (s2) return s2;
    if (ms > 0 && ms < best) {
      best = ms;
      best_lay = lay;
      best_block = block;
      best_graph = graph;
    }
    return DEM_OK;
  };
  st = consider(best_lay, best_block, best_graph);  // the starting point
  if (!st && !ctx->fused) {
    for (double sk : {0.0, 0.005, 0.015, 0.04}) {
      Layout l = best_lay;
      l.skin_rel = sk;
      l.scale = 1.0;
      l.rq = 0.0;
      if ((st = consider(l, best_block, best_graph))) break;
    }
    for (double sc : {1.08, 1.18}) {
      if (st) break;
      Layout l = best_lay;
      l.scale = sc;
      st = consider(l, best_block, best_graph);
    }
    for (double q : {0.90, 0.97}) {
      if (st) break;
      Layout l = best_lay;
      l.rq = q;
      st = consider(l, best_block, best_graph);
    }
  }
  for (int bl : {128, 256, 512}) {
    if (st) break;
    if (bl != best_block) st = consider(best_lay, bl, best_graph);
  }
  for (int gs : {8, 16, 32}) {
    if (st) break;
    if (gs != best_graph) st = consider(best_lay, best_block, gs);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // keep the best and put the starting state back
  dem_status st2 = DEM_OK;
  {
    ctx->block = best_block;
    ctx->graph_steps = best_graph;
    std::string msg;
    st2 = apply(best_lay, &msg);
    if (st2) st2 = fail(ctx, st2, msg);
    if (!st2) st2 = restore_snapshot(ctx, sn);
  }
  ctx->tm.on = was_timing;
  if (st) return st;
  if (st2) return st2;
  if (out) {
    out->ms_per_step = best;
    out->skin_over_rmax = best_lay.skin_rel;
    out->cell_scale = best_lay.scale;
    out->rsplit_quantile = best_lay.rq;
    out->block = best_block;
    out->graph_steps = best_graph;
    out->trials = trials;
    out->pad = 0;
  }
  st = prepare_graphs(ctx);
  if (st) return st;
  return read_status(ctx);
}

extern "C" dem_status dem_get_layout(dem_ctx* ctx, int32_t box, int32_t ncell[3], double* skin,
                                     double* r_split) {
  dem_status st = check_box(ctx, box);
  if (st) return st;
  if (ncell)
    for (int a = 0; a < 3; ++a) ncell[a] = ctx->hbox[box].n[a];
  if (skin) *skin = ctx->boxes[box].skin;
  if (r_split) *r_split = ctx->boxes[box].r_split;
  return DEM_OK;
}

extern "C" {

dem_status dem_set_timing(dem_ctx* ctx, int32_t on) {
  if (!ctx) return fail(ctx, DEM_ERR_ARG, "null context");
  if (on && !ctx->tm.made) {
    for (auto& set : ctx->tm.ev)
      for (auto& ev : set) CK(cudaEventCreate(&ev));
    ctx->tm.made = true;
  }
  ctx->tm.used = 0;
  ctx->tm.on = on != 0;
  return DEM_OK;
}

int32_t dem_get_phase_times(dem_ctx* ctx, double* ms, int32_t cap) {
  if (!ctx || !ms) return 0;
  int k = std::min(cap, kPhases);
  for (int q = 0; q < k; ++q) ms[q] = ctx->phase_ms[q];
  return k;
}

dem_status dem_get_resort_stats(dem_ctx* ctx, int64_t out[4]) {
  if (!ctx || !out) return fail(ctx, DEM_ERR_ARG, "null argument");
  for (int k = 0; k < 4; ++k) out[k] = 0;
  if (ctx->fused) return DEM_OK;
  unsigned ctl[kCtlWords] = {};
  int cnt = 0;
  CK(cudaMemcpyAsync(ctl, ctx->dev.vctl, sizeof(ctl), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&cnt, ctx->vl[0].count, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  out[0] = ctl[kCtlResorts];
  out[1] = launches_per_resort(ctx);
  out[2] = std::min(cnt, ctx->Cmax);
  out[3] = ctx->steps_done;
  return DEM_OK;
}

dem_status dem_sync(dem_ctx* ctx) {
  if (!ctx) return fail(ctx, DEM_ERR_ARG, "null context");
  return read_status(ctx);
}

dem_status dem_get_count(dem_ctx* ctx, int32_t box, int64_t* n) {
  dem_status st = check_box(ctx, box);
  if (st) return st;
  if (!n) return fail(ctx, DEM_ERR_ARG, "n is null");
  *n = ctx->hbox[box].nlive;
  return DEM_OK;
}

dem_status dem_get_grid(dem_ctx* ctx, int32_t box, int32_t ncell[3]) {
  dem_status st = check_box(ctx, box);
  if (st) return st;
  if (!ncell) return fail(ctx, DEM_ERR_ARG, "ncell is null");
  for (int a = 0; a < 3; ++a) ncell[a] = ctx->hbox[box].n[a];
  return DEM_OK;
}

dem_status dem_get_state(dem_ctx* ctx, int32_t box, double* x, double* v,
                         double* omega, double* force, double* torque,
                         int32_t where) {
  dem_status st = check_box(ctx, box);
  if (st) return st;
  if (where != DEM_HOST && where != DEM_DEVICE) return fail(ctx, DEM_ERR_ARG, "bad where");
  const BoxDev& B = ctx->hbox[box];
  int n = B.nlive;
  if (n == 0) return DEM_OK;
  cudaStream_t s = ctx->stream, cs = ctx->copy_stream;
  double* outs[5] = {x, v, omega, force, torque};
  const int nb = blocks_for(n, 256);
  const int p = ctx->parity;
  const int hf = ctx->have_ft ? 1 : 0;
  // one array at a time: its kernel (id order, into staging) on the
  // context's stream, then its copy to the host on the copy stream
  for (int k = 0; k < 5; ++k) {
    if (!outs[k]) continue;
    double* dk = where == DEM_HOST ? ctx->staging + (size_t)3 * n * k : outs[k];
    double* o[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    o[k] = dk;
    switch (ctx->mode) {
      case kFP64: k_get_state<kFP64><<<nb, 256, 0, s>>>(ctx->dev, ctx->ps[p], box, o[0], o[1], o[2], o[3], o[4], hf); break;
      case kMIXED: k_get_state<kMIXED><<<nb, 256, 0, s>>>(ctx->dev, ctx->ps[p], box, o[0], o[1], o[2], o[3], o[4], hf); break;
      default: k_get_state<kFP32><<<nb, 256, 0, s>>>(ctx->dev, ctx->ps[p], box, o[0], o[1], o[2], o[3], o[4], hf); break;
    }
    CK(cudaGetLastError());
    if (where == DEM_HOST) {
      CK(cudaEventRecord(ctx->xfer_ev[k], s));
      CK(cudaStreamWaitEvent(cs, ctx->xfer_ev[k], 0));
      CK(cudaMemcpyAsync(outs[k], dk, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, cs));
    }
  }
  CK(cudaStreamSynchronize(s));
  if (where == DEM_HOST) CK(cudaStreamSynchronize(cs));
  return DEM_OK;
}

dem_status dem_get_order(dem_ctx* ctx, int32_t box, int32_t* id_by_slot,
                         int32_t* cell_by_slot) {
  dem_status st = check_box(ctx, box);
  if (st) return st;
  const BoxDev& B = ctx->hbox[box];
  int n = B.nlive;
  if (n == 0) return DEM_OK;
  cudaStream_t s = ctx->stream;
  int* a = ctx->staging_i;
  int* c = ctx->staging_i + n;
  k_get_order<<<blocks_for(n, 256), 256, 0, s>>>(ctx->dev, ctx->ps[ctx->parity], box, a, c);
  CK(cudaGetLastError());
  if (id_by_slot) CK(cudaMemcpyAsync(id_by_slot, a, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
  if (cell_by_slot) CK(cudaMemcpyAsync(cell_by_slot, c, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return DEM_OK;
}

// Download the current contact list of all boxes as host vectors, walking
// each particle's (start, count) index: works for the dense list, the fused
// layout's per-slot blocks and a list restored by dem_set_contacts.
// Optional per-contact force and n x F.
static dem_status download_list(dem_ctx* ctx, std::vector<int2>& hid,
                                std::vector<double>& dts,
                                std::vector<double>* F = nullptr,
                                std::vector<double>* nF = nullptr) {
  cudaStream_t s = ctx->stream;
  // the per-particle forms' list of the last step, or the candidate list
  // (its pairs in contact in the last step carry flag 1)
  const int* c_hs = ctx->fused ? ctx->cl[ctx->parity].hs : ctx->vl[0].hs;
  const int* c_oc = ctx->fused ? ctx->cl[ctx->parity].oc : ctx->vl[0].oc;
  // ids: the per-particle forms store them; the candidate list stores slots
  // (lower id first), whose ids are read here
  const int2* c_hid = ctx->fused ? ctx->cl[ctx->parity].hid : ctx->vl[0].pair;
  void* const comps[3] = {ctx->fused ? ctx->cl[ctx->parity].dx : ctx->vl[0].dx,
                          ctx->fused ? ctx->cl[ctx->parity].dy : ctx->vl[0].dy,
                          ctx->fused ? ctx->cl[ctx->parity].dz : ctx->vl[0].dz};
  const unsigned char* c_flag = ctx->fused ? nullptr : ctx->vl[0].flag;
  const int N = ctx->N;
  std::vector<int> rs(N), rc(N);
  hid.clear();
  dts.clear();
  if (N == 0) return DEM_OK;
  CK(cudaMemcpyAsync(rs.data(), c_hs, sizeof(int) * N, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(rc.data(), c_oc, sizeof(int) * N, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  long long top = 0;
  for (const BoxDev& B : ctx->hbox)
    for (int g = B.pbase; g < B.pbase + B.nlive; ++g)
      if (rc[g] > 0) top = std::max(top, (long long)rs[g] + rc[g]);
  top = std::min<long long>(top, ctx->Cmax);
  std::vector<int2> h(top);
  std::vector<int> slot_id;
  if (!ctx->fused) {
    slot_id.resize(N);
    CK(cudaMemcpyAsync(slot_id.data(), ctx->ps[ctx->parity].id, sizeof(int) * N,
                       cudaMemcpyDeviceToHost, s));
  }
  const size_t eb = dt_bytes(ctx->mode), vb = v4_bytes(ctx->mode);
  std::vector<unsigned char> raw[3], fr, fl(std::max(1ll, top), 1);
  for (int a = 0; a < 3; ++a) raw[a].resize(eb * std::max(1ll, top));
  if (top > 0) {
    CK(cudaMemcpyAsync(h.data(), c_hid, sizeof(int2) * top, cudaMemcpyDeviceToHost, s));
    for (int a = 0; a < 3; ++a)
      CK(cudaMemcpyAsync(raw[a].data(), comps[a], eb * top, cudaMemcpyDeviceToHost, s));
    if (c_flag) CK(cudaMemcpyAsync(fl.data(), c_flag, top, cudaMemcpyDeviceToHost, s));
    if (F) {
      fr.resize(2 * vb * top);  // per contact: F, then n x F
      CK(cudaMemcpyAsync(fr.data(), ctx->dev.Fc, 2 * vb * top, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
  }
  auto dtval = [&](int a, long long k) {
    double val;
    if (ctx->mode == kMIXED) {
      float hl[2];
      std::memcpy(hl, raw[a].data() + 8 * k, 8);
      val = (double)hl[0] + (double)hl[1];
    } else if (ctx->mode == kFP64) {
      std::memcpy(&val, raw[a].data() + 8 * k, 8);
    } else {
      float f;
      std::memcpy(&f, raw[a].data() + 4 * k, 4);
      val = f;
    }
    return val;
  };
  auto v4val = [&](const std::vector<unsigned char>& buf, long long k, int a) {
    if (ctx->mode == kFP64) {
      double v;
      std::memcpy(&v, buf.data() + 32 * k + 8 * a, 8);
      return v;
    }
    float v;
    std::memcpy(&v, buf.data() + 16 * k + 4 * a, 4);
    return (double)v;
  };
  // the two vectors of a contact's record
  for (const BoxDev& B : ctx->hbox)
    for (int g = B.pbase; g < B.pbase + B.nlive; ++g)
      for (int k = 0; k < rc[g]; ++k) {
        long long e = (long long)rs[g] + k;
        if (e >= top) break;
        if (!fl[e]) continue;  // a candidate pair not in contact
        hid.push_back(ctx->fused ? h[e] : make_int2(slot_id[h[e].x], slot_id[h[e].y]));
        for (int a = 0; a < 3; ++a) dts.push_back(dtval(a, e));
        if (F)
          for (int a = 0; a < 3; ++a) {
            F->push_back(v4val(fr, 2 * e, a));
            nF->push_back(v4val(fr, 2 * e + 1, a));
          }
      }
  return DEM_OK;
}

dem_status dem_get_contacts(dem_ctx* ctx, int32_t box, int64_t cap, int64_t* n,
                            int32_t* id_lo, int32_t* id_hi, double* delta_t) {
  dem_status st = check_box(ctx, box);
  if (st) return st;
  if (!n) return fail(ctx, DEM_ERR_ARG, "n is null");
  std::vector<int2> hid;
  std::vector<double> dts;
  st = download_list(ctx, hid, dts);
  if (st) return st;
  const BoxDev& B = ctx->hbox[box];
  std::vector<int> sel;
  for (size_t k = 0; k < hid.size(); ++k)
    if (hid[k].x >= B.pbase && hid[k].x < B.pbase + B.nlive) sel.push_back((int)k);
  std::sort(sel.begin(), sel.end(), [&](int a, int b) {
    return hid[a].x != hid[b].x ? hid[a].x < hid[b].x : hid[a].y < hid[b].y;
  });
  *n = (int64_t)sel.size();
  if ((int64_t)sel.size() > cap) return fail(ctx, DEM_ERR_CAPACITY, "cap smaller than the contact count");
  for (size_t q = 0; q < sel.size(); ++q) {
    int k = sel[q];
    if (id_lo) id_lo[q] = hid[k].x - B.pbase;
    if (id_hi) id_hi[q] = hid[k].y - B.pbase;
    if (delta_t)
      for (int a = 0; a < 3; ++a) delta_t[3 * q + a] = dts[(size_t)3 * k + a];
  }
  return DEM_OK;
}

dem_status dem_get_contact_forces(dem_ctx* ctx, int32_t box, int64_t cap,
                                  int64_t* n, int32_t* id_lo, int32_t* id_hi,
                                  double* F, double* nF) {
  dem_status st = check_box(ctx, box);
  if (st) return st;
  if (!n) return fail(ctx, DEM_ERR_ARG, "n is null");
  std::vector<int2> hid;
  std::vector<double> dts, f, q;
  st = download_list(ctx, hid, dts, &f, &q);
  if (st) return st;
  const BoxDev& B = ctx->hbox[box];
  std::vector<int> sel;
  for (size_t k = 0; k < hid.size(); ++k)
    if (hid[k].x >= B.pbase && hid[k].x < B.pbase + B.nlive) sel.push_back((int)k);
  std::sort(sel.begin(), sel.end(), [&](int a, int b) {
    return hid[a].x != hid[b].x ? hid[a].x < hid[b].x : hid[a].y < hid[b].y;
  });
  *n = (int64_t)sel.size();
  if ((int64_t)sel.size() > cap) return fail(ctx, DEM_ERR_CAPACITY, "cap smaller than the contact count");
  for (size_t t = 0; t < sel.size(); ++t) {
    int k = sel[t];
    if (id_lo) id_lo[t] = hid[k].x - B.pbase;
    if (id_hi) id_hi[t] = hid[k].y - B.pbase;
    for (int a = 0; a < 3; ++a) {
      if (F) F[3 * t + a] = f[3 * (size_t)k + a];
      if (nF) nF[3 * t + a] = q[3 * (size_t)k + a];
    }
  }
  return DEM_OK;
}

dem_status dem_set_contacts(dem_ctx* ctx, int32_t box, int64_t n,
                            const int32_t* id_lo, const int32_t* id_hi,
                            const double* delta_t) {
  dem_status st = check_box(ctx, box);
  if (st) return st;
  const BoxDev& B = ctx->hbox[box];
  if (n < 0 || (n > 0 && (!id_lo || !id_hi || !delta_t)))
    return fail(ctx, DEM_ERR_ARG, "bad contact arrays");
  for (int64_t k = 0; k < n; ++k)
    if (id_lo[k] < 0 || id_hi[k] >= B.nlive || id_lo[k] >= id_hi[k])
      return fail(ctx, DEM_ERR_ARG, "contact ids must satisfy 0 <= lo < hi < count");
  std::vector<int2> hid;
  std::vector<double> dts;
  st = download_list(ctx, hid, dts);
  if (st) return st;
  // keep other boxes' entries, replace this box's
  std::vector<std::pair<int2, std::array<double, 3>>> all;
  for (size_t k = 0; k < hid.size(); ++k)
    if (!(hid[k].x >= B.pbase && hid[k].x < B.pbase + B.cap))
      all.push_back({hid[k], {dts[3 * k], dts[3 * k + 1], dts[3 * k + 2]}});
  for (int64_t k = 0; k < n; ++k)
    all.push_back({make_int2(B.pbase + id_lo[k], B.pbase + id_hi[k]),
                   {delta_t[3 * k], delta_t[3 * k + 1], delta_t[3 * k + 2]}});
  std::sort(all.begin(), all.end(), [](const auto& a, const auto& b) {
    return a.first.x != b.first.x ? a.first.x < b.first.x : a.first.y < b.first.y;
  });
  for (size_t k = 1; k < all.size(); ++k)
    if (all[k].first.x == all[k - 1].first.x && all[k].first.y == all[k - 1].first.y)
      return fail(ctx, DEM_ERR_ARG, "duplicate contact");
  if ((long long)all.size() > ctx->Cmax) return fail(ctx, DEM_ERR_CAPACITY, "contact list capacity");
  const int nc = (int)all.size();
  // the list is indexed by the slots the particles hold now: each contact
  // goes into the block of its lower-id member's slot
  cudaStream_t s = ctx->stream;
  const int N = ctx->N;
  std::vector<int> id_of(N), slot_of(N, -1);
  CK(cudaMemcpyAsync(id_of.data(), ctx->ps[ctx->parity].id, sizeof(int) * N,
                     cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (const BoxDev& Bx : ctx->hbox)
    for (int g = Bx.pbase; g < Bx.pbase + Bx.nlive; ++g)
      if (id_of[g] >= 0 && id_of[g] < N) slot_of[id_of[g]] = g;
  std::vector<int2> slots(nc);
  for (int k = 0; k < nc; ++k) {
    slots[k] = make_int2(slot_of[all[k].first.x], slot_of[all[k].first.y]);
    if (slots[k].x < 0 || slots[k].y < 0)
      return fail(ctx, DEM_ERR_STATE, "contact of a particle that holds no slot");
  }
  std::vector<int> order(nc);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return slots[a].x < slots[b].x; });
  std::vector<int> rs(N, 0), rc(N, 0);
  std::vector<int2> h2(nc), p2(nc);
  const size_t eb = dt_bytes(ctx->mode);
  std::vector<unsigned char> comp[3];
  for (int a = 0; a < 3; ++a) comp[a].resize(eb * std::max(1, nc));
  for (int k = 0; k < nc; ++k) {
    const int src = order[k];
    h2[k] = all[src].first;
    p2[k] = slots[src];
    const int lo = p2[k].x;
    if (rc[lo] == 0) rs[lo] = k;
    rc[lo]++;
    for (int a = 0; a < 3; ++a) {
      double val = all[src].second[a];
      if (ctx->mode == kMIXED) {
        float hl[2];
        hl[0] = (float)val;
        hl[1] = (float)(val - (double)hl[0]);
        std::memcpy(comp[a].data() + 8 * k, hl, 8);
      } else if (ctx->mode == kFP64) {
        std::memcpy(comp[a].data() + 8 * k, &val, 8);
      } else {
        float f = (float)val;
        std::memcpy(comp[a].data() + 4 * k, &f, 4);
      }
    }
  }
  // the per-particle forms read it as the previous step's list; the
  // contact-list pipeline as its current candidate list (every pair in
  // contact), carried into the list of the re-sort the next step makes
  int2* c_hid = ctx->fused ? ctx->cl[ctx->parity].hid : ctx->vl[0].hid;
  int2* c_pair = ctx->fused ? ctx->cl[ctx->parity].pair : ctx->vl[0].pair;
  void* const c_d[3] = {ctx->fused ? ctx->cl[ctx->parity].dx : ctx->vl[0].dx,
                        ctx->fused ? ctx->cl[ctx->parity].dy : ctx->vl[0].dy,
                        ctx->fused ? ctx->cl[ctx->parity].dz : ctx->vl[0].dz};
  int* c_hs = ctx->fused ? ctx->cl[ctx->parity].hs : ctx->vl[0].hs;
  int* c_oc = ctx->fused ? ctx->cl[ctx->parity].oc : ctx->vl[0].oc;
  int* c_count = ctx->fused ? ctx->cl[ctx->parity].count : ctx->vl[0].count;
  if (nc > 0) {
    if (c_hid) CK(cudaMemcpyAsync(c_hid, h2.data(), sizeof(int2) * nc, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c_pair, p2.data(), sizeof(int2) * nc, cudaMemcpyHostToDevice, s));
    for (int a = 0; a < 3; ++a)
      CK(cudaMemcpyAsync(c_d[a], comp[a].data(), eb * nc, cudaMemcpyHostToDevice, s));
    if (!ctx->fused) CK(cudaMemsetAsync(ctx->vl[0].flag, 1, nc, s));
  }
  CK(cudaMemcpyAsync(c_hs, rs.data(), sizeof(int) * N, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c_oc, rc.data(), sizeof(int) * N, cudaMemcpyHostToDevice, s));
  *ctx->h_count = nc;
  CK(cudaMemcpyAsync(c_count, ctx->h_count, sizeof(int), cudaMemcpyHostToDevice, s));
  if (!ctx->fused) CK(cudaMemsetAsync(ctx->dev.vctl + kCtlRequest, 1, sizeof(unsigned), s));
  CK(cudaStreamSynchronize(s));
  return DEM_OK;
}

dem_status dem_get_stats(dem_ctx* ctx, int32_t box, double out[DEM_NSTATS]) {
  dem_status st = check_box(ctx, box);
  if (st) return st;
  if (!out) return fail(ctx, DEM_ERR_ARG, "out is null");
  cudaStream_t s = ctx->stream;
  double* dout = ctx->staging;
  double* part = ctx->staging + 8;
  const int nparts = std::max(1, std::min(512, blocks_for(ctx->hbox[box].nlive, 256)));
  const int p = ctx->parity;
  const int* hs = ctx->fused ? ctx->cl[p].hs : ctx->vl[0].hs;
  const int* oc = ctx->fused ? ctx->cl[p].oc : ctx->vl[0].oc;
  const unsigned char* fl = ctx->fused ? nullptr : ctx->vl[0].flag;
  switch (ctx->mode) {
    case kFP64: k_stats<kFP64><<<nparts, 256, 0, s>>>(ctx->dev, ctx->ps[p], hs, oc, fl, box, part); break;
    case kMIXED: k_stats<kMIXED><<<nparts, 256, 0, s>>>(ctx->dev, ctx->ps[p], hs, oc, fl, box, part); break;
    default: k_stats<kFP32><<<nparts, 256, 0, s>>>(ctx->dev, ctx->ps[p], hs, oc, fl, box, part); break;
  }
  k_stats_final<<<1, 32, 0, s>>>(part, nparts, dout);
  CK(cudaGetLastError());
  double h[6];
  unsigned dg[2];
  CK(cudaMemcpyAsync(h, dout, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(dg, ctx->dev.diag + 2 * box, sizeof(dg), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int n = ctx->hbox[box].nlive;
  float f0, f1;
  std::memcpy(&f0, &dg[0], 4);
  std::memcpy(&f1, &dg[1], 4);
  out[0] = h[0];
  out[1] = h[1];
  out[2] = h[2];
  out[3] = h[3];
  out[4] = h[4];
  out[5] = h[5];
  out[6] = n > 0 ? 2.0 * h[5] / n : 0.0;
  out[7] = f0;
  out[8] = f1;
  out[9] = n;
  return DEM_OK;
}

}  // extern "C"

// ==========================================================================
// Contact detection without device allocation (dem_contacts_static).
//
// Some callers cannot allocate device memory at the moment they need a
// contact list: code running inside another framework's memory pool or
// under a fixed memory budget, code that must not grow its footprint once
// it is running, or code that must not call cudaMalloc (which may
// synchronise the device) on a latency-critical path.  For them this entry
// point runs the same search kernels as dem_step on one small box, with all
// of its scratch carved from one file-scope device array of fixed size.
// The array (6,000,000 bytes) exists on every GPU that loads this library
// until the process exits.
// ==========================================================================
namespace {

constexpr int kStaticMaxParticles = 8192;
constexpr int kStaticMaxCells = 32768;
constexpr int kStaticMaxContacts = 131072;
constexpr int kStaticK = 32;

// layout of the scratch array (every part 256-byte aligned)
struct StaticLayout {
  size_t box, slot_box, rol, lor, ccount, cstart, ccur, dirty, chg, crange, cellbox, perm, pcell, row,
      icnt, bsum, status, count, pair, rs, rc, state[2][10], total;
};

constexpr size_t al(size_t v) { return (v + 255) & ~size_t(255); }

StaticLayout static_layout() {
  StaticLayout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = al(o + bytes);
    return at;
  };
  const size_t N = kStaticMaxParticles, M = kStaticMaxCells;
  L.box = take(sizeof(BoxDev));
  L.slot_box = take(4 * N);
  L.rol = take(4 * M);
  L.lor = take(4 * (M + 1));
  L.ccount = take(4 * (M + 1));
  L.cstart = take(4 * (M + 1));
  L.ccur = take(4 * (M + 1));
  L.dirty = take(M + 1);
  L.chg = take(M + 1);
  L.crange = take(8 * M);
  L.cellbox = take(32 * M);
  L.perm = take(4 * N);
  L.pcell = take(4 * N);
  L.row = take(4 * N * kStaticK);
  L.icnt = take(4 * N);
  L.bsum = take(4 * 16384);
  L.status = take(4);
  L.count = take(4);
  L.pair = take(8 * (size_t)kStaticMaxContacts);
  L.rs = take(4 * N);
  L.rc = take(4 * N);
  for (int p = 0; p < 2; ++p) {
    const size_t sz[10] = {8 * N, 8 * N, 8 * N, 16 * N, 16 * N, 16 * N, 4 * N, 4 * N, 4 * N, 4 * N};
    for (int k = 0; k < 10; ++k) L.state[p][k] = take(sz[k]);
  }
  L.total = o;
  return L;
}

// Upper bound of the layout above (checked at set-up).
constexpr size_t kStaticScratchBytes = 6000000;

}  // namespace

// The scratch itself.  In host code this name is only a stand-in for the
// symbol; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_dem_static_scratch[kStaticScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
unsigned char* g_static_addr[kMaxDevices] = {};

__global__ void k_static_iota(int* rank_of_lin, int* lin_of_rank, int M) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < M) {
    rank_of_lin[l] = l;
    lin_of_rank[l] = l;
  } else if (l == M) {
    lin_of_rank[M] = -1;
  }
}

// status bits of the radius check
constexpr unsigned kStStaticRadiusLarge = 0x100u;  // above half the narrowest cell
constexpr unsigned kStStaticRadiusBad = 0x200u;    // zero, negative or not finite

// a radius above half the narrowest cell would let contacts skip a cell
__global__ void k_static_check_radius(const double* r, int n, double hmin,
                                      unsigned* status) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double rk = r[k];
  if (!(rk > 0.0) || !isfinite(rk)) atomicOr(status, kStStaticRadiusBad);
  else if (!(2.0 * rk * (1.0 + 1e-5) <= hmin)) atomicOr(status, kStStaticRadiusLarge);
}

// true when p is memory of device dev that kernels can read (device or
// managed memory); host and unregistered pointers are rejected
bool static_device_pointer(const void* p, int dev) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the error this query may leave behind
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" dem_status dem_contacts_static(int64_t n, const double* x,
                                          const double* radius,
                                          const double L[3],
                                          const int32_t periodic[3],
                                          const int32_t ncell[3], int64_t cap,
                                          int32_t* pairs, int64_t* count,
                                          void* stream) {
  dem_ctx* ctx = nullptr;  // errors go to the create-error string
  if (!count) return fail(ctx, DEM_ERR_ARG, "count is null");
  *count = 0;
  if (n < 0 || n > kStaticMaxParticles)
    return fail(ctx, DEM_ERR_ARG, "dem_contacts_static: n must be in [0, 8192]");
  if (!L || !periodic || !ncell || cap < 0 || (cap > 0 && !pairs) ||
      (n > 0 && (!x || !radius)))
    return fail(ctx, DEM_ERR_ARG, "dem_contacts_static: null or negative argument");
  if (((uintptr_t)pairs & 7) != 0)
    return fail(ctx, DEM_ERR_ARG, "dem_contacts_static: pairs must be 8-byte aligned");
  long long M = 1;
  double hmin = 1e300;
  for (int a = 0; a < 3; ++a) {
    if (!(L[a] > 0) || L[a] * 0x1p60 >= 0x1p62)
      return fail(ctx, DEM_ERR_ARG, "dem_contacts_static: box length out of range (0, 4 m)");
    if (ncell[a] < 1 || ncell[a] > kMaxAxisCells || (periodic[a] && ncell[a] < 3))
      return fail(ctx, DEM_ERR_ARG, "dem_contacts_static: bad cell grid (periodic axes need >= 3 cells)");
    M *= ncell[a];
    hmin = std::min(hmin, L[a] / ncell[a]);
  }
  if (M > kStaticMaxCells)
    return fail(ctx, DEM_ERR_ARG, "dem_contacts_static: more than 32768 cells");
  if (n == 0) return DEM_OK;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(ctx, DEM_ERR_CUDA, "dem_contacts_static: no usable current device");
  const StaticLayout lay = static_layout();
  unsigned char* base = nullptr;
  {
    // set-up, once per device, with that device current
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
      if (lay.total > kStaticScratchBytes)
        return fail(ctx, DEM_ERR_ALLOC, "dem_contacts_static: scratch layout exceeds the array");
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_dem_static_scratch);
      if (e != cudaSuccess || !p)
        return fail(ctx, DEM_ERR_CUDA, std::string("dem_contacts_static: cudaGetSymbolAddress: ") +
                                           cudaGetErrorString(e));
      g_static_addr[dev] = (unsigned char*)p;
    }
    base = g_static_addr[dev];
  }
  if (!static_device_pointer(x, dev) || !static_device_pointer(radius, dev) ||
      (cap > 0 && !static_device_pointer(pairs, dev)))
    return fail(ctx, DEM_ERR_ARG,
                "dem_contacts_static: x, radius and pairs must be device memory of the current GPU");
  cudaStream_t s = (cudaStream_t)stream;
  const int N = (int)n;

  BoxDev B{};
  for (int a = 0; a < 3; ++a) {
    int nc = ncell[a];
    B.n[a] = nc;
    B.periodic[a] = periodic[a] ? 1 : 0;
    B.Lq[a] = std::llround(std::ldexp(L[a], kFixShift));
    B.Hq[a] = B.Lq[a] / nc;
    B.L[a] = L[a];
    B.half_L[a] = 0.5 * L[a];
    B.inv_h[a] = (double)nc / L[a];
    B.Lf[a] = (float)L[a];
    B.half_Lf[a] = 0.5f * B.Lf[a];
    B.inv_hf[a] = (float)((double)nc / L[a]);
    long long H = B.Hq[a], Lq = B.Lq[a];
    long long S[5] = {-H, 0, H, (long long)(nc - 1) * H - Lq, Lq - (long long)(nc - 1) * H};
    for (int k = 0; k < 5; ++k) B.shift[a][k] = (float)S[k] * 0x1p-60f;
    B.h[a] = L[a] / nc;
    B.hcell[a][0] = (float)H * 0x1p-60f;
    B.hcell[a][1] = B.periodic[a] ? (float)(Lq - (long long)(nc - 1) * H) * 0x1p-60f : INFINITY;
  }
  B.ncells = (int)M;
  B.cap = N;
  B.nlive = N;
  B.density = 1.0;
  B.rmax_f = (float)(0.5 * hmin);
  B.rsplit_f = INFINITY;  // one size class

  Dev d{};
  d.nbox = 1;
  d.boxes = (const BoxDev*)(base + lay.box);
  d.slot_box = (const int*)(base + lay.slot_box);
  d.N = N;
  d.K = kStaticK;
  d.Cmax = (int)std::min<int64_t>(cap, kStaticMaxContacts);
  d.M_lin = (int)M;
  d.M_rank = (int)M + 1;
  d.rank_of_lin = (const int*)(base + lay.rol);
  d.lin_of_rank = (const int*)(base + lay.lor);
  d.ccount = (int*)(base + lay.ccount);
  d.cstart = (int*)(base + lay.cstart);
  d.cstart_old = d.cstart;
  d.ccur = (int*)(base + lay.ccur);
  d.collect = (unsigned char*)(base + lay.dirty);
  d.chg = (const unsigned char*)(base + lay.chg);
  d.crange = (int2*)(base + lay.crange);
  d.cellbox = (float4*)(base + lay.cellbox);
  d.perm = (int*)(base + lay.perm);
  d.pcell = (int*)(base + lay.pcell);
  d.row = (int*)(base + lay.row);
  d.icnt = (int*)(base + lay.icnt);
  d.status = (unsigned*)(base + lay.status);
  d.scan_bsum = (int*)(base + lay.bsum);
  PState ps[2];
  for (int p = 0; p < 2; ++p) {
    const size_t* o = lay.state[p];
    ps[p] = PState{base + o[0], base + o[1], base + o[2], base + o[3], base + o[4], base + o[5],
                   (int*)(base + o[6]), (int*)(base + o[7]), (int*)(base + o[8]),
                   (int*)(base + o[9]), nullptr, nullptr, nullptr};
  }
  VList cn{};
  cn.pair = (int2*)(base + lay.pair);
  cn.hid = (int2*)pairs;
  cn.hs = (int*)(base + lay.rs);
  cn.oc = (int*)(base + lay.rc);
  cn.count = (int*)(base + lay.count);

  // The array keeps the previous call's contents: clear what must start at
  // zero (cell counts, box index of every slot, status, count) and mark
  // every cell changed (no order to keep from a previous call).
  auto ck = [&](cudaError_t e, const char* what) -> dem_status {
    if (e == cudaSuccess) return DEM_OK;
    return fail(ctx, DEM_ERR_CUDA, std::string("dem_contacts_static: ") + what + ": " +
                                       cudaGetErrorString(e));
  };
  dem_status st;
  if ((st = ck(cudaMemcpyAsync(base + lay.box, &B, sizeof(BoxDev), cudaMemcpyHostToDevice, s), "box")))
    return st;
  if ((st = ck(cudaMemsetAsync(d.ccount, 0, 4 * (size_t)(M + 1), s), "counts"))) return st;
  if ((st = ck(cudaMemsetAsync(base + lay.dirty, 1, (size_t)(M + 1), s), "cell flags"))) return st;
  if ((st = ck(cudaMemsetAsync((void*)d.slot_box, 0, 4 * (size_t)N, s), "slots"))) return st;
  if ((st = ck(cudaMemsetAsync(d.status, 0, 4, s), "status"))) return st;
  if ((st = ck(cudaMemsetAsync(cn.count, 0, 4, s), "count"))) return st;
  k_static_iota<<<blocks_for(M + 1, 256), 256, 0, s>>>((int*)d.rank_of_lin, (int*)d.lin_of_rank, (int)M);
  k_static_check_radius<<<blocks_for(N, 256), 256, 0, s>>>(radius, N, hmin, d.status);
  // bin, sort, search, compact: the DEM_MIXED kernels of dem_step
  k_set_particles<kMIXED><<<blocks_for(N, 256), 256, 0, s>>>(d, ps[0], 0, N, x, x, x, radius);
  int nbc = blocks_for(d.M_rank, kScanTile);
  k_scan_reduce<<<nbc, kScanThreads, 0, s>>>(d.ccount, d.M_rank, d.scan_bsum, nullptr);
  k_scan_top<<<1, kScanTopThreads, 0, s>>>(d.scan_bsum, nbc, nullptr, 0, d.status, 0u, nullptr);
  k_scan_apply<<<nbc, kScanThreads, 0, s>>>(d.ccount, d.M_rank, d.scan_bsum,
                                            CellEpi{d.cstart, d.crange, d.cellbox, d.lin_of_rank,
                                                    d.collect, (unsigned char*)d.chg, d.ccur},
                                            nullptr);
  k_scatter<<<blocks_for(N, 256), 256, 0, s>>>(d, ps[0]);
  k_reorder<kMIXED><<<blocks_for(N, 256), 256, 0, s>>>(d, ps[0], ps[1], cn.count);
  k_candidates<kMIXED, false><<<blocks_for(N, 256), 256, 0, s>>>(d, ps[1], cn);
  if ((st = ck(cudaGetLastError(), "launch"))) return st;
  int hcount = 0;
  unsigned hstatus = 0;
  if ((st = ck(cudaMemcpyAsync(&hcount, cn.count, 4, cudaMemcpyDeviceToHost, s), "count read")))
    return st;
  if ((st = ck(cudaMemcpyAsync(&hstatus, d.status, 4, cudaMemcpyDeviceToHost, s), "status read")))
    return st;
  if ((st = ck(cudaStreamSynchronize(s), "synchronise"))) return st;
  *count = std::min(hcount, d.Cmax);
  if (hstatus & kStStaticRadiusBad)
    return fail(ctx, DEM_ERR_ARG, "dem_contacts_static: a radius is zero, negative or not finite");
  if (hstatus & kStStaticRadiusLarge)
    return fail(ctx, DEM_ERR_ARG,
                "dem_contacts_static: a radius exceeds half the narrowest cell edge");
  if (hstatus & kStNonFinite) return fail(ctx, DEM_ERR_NONFINITE, "dem_contacts_static: non-finite position");
  if (hstatus & (kStRowOverflow | kStListOverflow))
    return fail(ctx, DEM_ERR_CAPACITY, "dem_contacts_static: contacts exceed cap, 131072, or 32 per particle");
  if (hstatus) return fail(ctx, DEM_ERR_STATE, "dem_contacts_static: internal consistency check failed");
  return DEM_OK;
}
