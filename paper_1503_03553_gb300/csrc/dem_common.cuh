// dem_common.cuh -- device types and arithmetic helpers of the GB300 DEM path.
//
// Positions in DEM_MIXED are signed 64-bit fixed point with quantum 2^-60 m
// (range +-8 m).  On GB300 the FP64 pipe and the int64<->float conversions
// issue at under 2 per clock per SM (about 1/70 of FP32), so every
// conversion here is built from 32-bit integer/float operations and one
// fused multiply-add, which round exactly like the single correctly rounded
// conversion they replace.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dem {

constexpr int kFixShift = 60;
constexpr float kQ = 0x1p-60f;        // 2^-60 m, one quantum
constexpr float kInvQ = 0x1p60f;      // 2^60 / m
constexpr int kMaxAxisCells = 1024;   // packed cell coordinates: 10 bits each

enum Mode : int { kFP64 = 0, kMIXED = 1, kFP32 = 2 };

// device status word bits (sticky)
enum : unsigned {
  kStRowOverflow = 1u,     // a particle has more contacts than a row holds
  kStListOverflow = 2u,    // contact list longer than its capacity
  kStNonFinite = 4u,       // NaN/Inf in position, velocity or force
  kStInconsistent = 8u,    // contact seen by one member of a pair only
  kStRange = 16u,          // fixed-point position out of range
};

// control words of the candidate-list pipeline (device, per context)
enum : int {
  kCtlResort = 0,     // this step re-sorts and rebuilds the candidate list
  kCtlRequest = 1,    // a re-sort is asked for (displacement or host call)
  kCtlResorts = 2,    // re-sorts so far (statistics)
  kCtlWords = 4
};

// A rectangle (p + s u + t v) or line (p + s u) wall, s, t in [0, 1]: the
// geometry in FP64 for the contact and in FP32 for a conservative cull.
struct WallDev {
  int kind;             // 0 rectangle, 1 line
  double p[3], u[3], v[3];
  double inv_uu, inv_vv;  // 1 / u.u, 1 / v.v (0 for a line)
  float pf[3], uf[3], vf[3];
  float inv_uuf, inv_vvf;
  float slack;          // cull margin [m]: far above the FP32 geometry error
};

// Per-box constants, filled on the host at creation.
struct BoxDev {
  long long Lq[3];      // box length in quanta
  long long Hq[3];      // cell edge in quanta (last cell takes the rest)
  double L[3];          // box length [m]
  double half_L[3];
  double inv_h[3];      // ncell / L
  float Lf[3];
  float half_Lf[3];
  float inv_hf[3];
  float shift[3][5];    // fixed-rule cell shifts: -H, 0, +H, wrap low, wrap high
  float hcell[3][2];    // cell edge [m]: ordinary cell, last cell (inf when open)
  double h[3];          // L / ncell [m]
  float rmax_f;         // largest radius the box may hold [m]
  float rsplit_f;       // size-binned search: a particle is large when its
                        // FP32 radius exceeds this (+inf: one class)
  float skin_f;         // candidate-list skin [m]: pairs within r_i + r_j +
                        // skin are kept between re-sorts (0: re-sort and
                        // search every step)
  float disp2_lim;      // a particle displaced more than sqrt(disp2_lim)
                        // since the last re-sort asks for the next one
                        // (-1: every step)
  int n[3];             // cells per axis
  int periodic[3];
  int floor_wall;
  int nwalls;           // rectangle and line walls
  int wall_base;        // first of them in the context's wall array
  int lin_base;         // first cell of this box in linear-cell space
  int rank_base;        // first cell in rank space (ncells + 1: last is the
                        // box's "free slot" cell holding unused capacity)
  int ncells;
  int pbase;            // first storage slot
  int cap;              // storage slots
  int nlive;            // particles present
  double dt;
  float dt_f;
  float dtq_f;          // dt * 2^60, displacement to quanta
  double g[3];
  float g_f[3];
  // Sec. 2 coefficients, one material per box:
  //   k_n = kn_c sqrt(R*),  k_t = kt_c sqrt(R* dn),  eta = alpha sqrt(m* k_n sqrt(dn))
  double kn_c, kt_c, alpha, mu;
  float kn_cf, kt_cf, alpha_f, mu_f;
  double density;
};

// ---------------------------------------------------------------------------
// float-float (hi + lo) arithmetic: Knuth's TwoSum, Dekker's Fast2Sum and an
// FMA-based exact product.  Plain float adds/subs are never contracted or
// reassociated by nvcc; products use explicit rounding intrinsics.
// ---------------------------------------------------------------------------
struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ ff two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}
// (hi, lo) + b, renormalised
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  ff s = two_sum(a.hi, b);
  float lo = __fadd_rn(s.lo, a.lo);
  return fast_two_sum(s.hi, lo);
}

// Correctly rounded int64 -> float using 32-bit conversions: with
// O = a 2^24 + b, b in [0, 2^24) and |a| < 2^24 both parts are exact floats
// and one fma rounds the exact sum once.
__device__ __forceinline__ float i64_to_f32_rn(long long O) {
  long long a = O >> 24;
  if (a >= -(1ll << 24) && a < (1ll << 24)) {
    float fa = __int2float_rn((int)a);
    float fb = __int2float_rn((int)(O & 0xFFFFFFll));
    return __fmaf_rn(fa, 16777216.0f, fb);
  }
  return __ll2float_rn(O);  // beyond 2^48 quanta: rare slow path
}

// Exact float-float of an int64 (|D| < 2^48): hi + lo == D.
__device__ __forceinline__ ff i64_to_ff(long long D) {
  long long a = D >> 24;
  if (a >= -(1ll << 24) && a < (1ll << 24)) {
    float fa = __fmul_rn(__int2float_rn((int)a), 16777216.0f);
    float fb = __int2float_rn((int)(D & 0xFFFFFFll));
    return two_sum(fa, fb);
  }
  float hi = __ll2float_rn(D);
  float lo = __ll2float_rn(D - __float2ll_rn(hi));
  return {hi, lo};
}

// Round a float holding a count of quanta to the nearest int64 without the
// FP64 pipe: values below 2^31 use the 32-bit conversion; larger floats are
// integers already and are rebuilt from their mantissa and exponent.
__device__ __forceinline__ long long f32_to_i64_rn(float f, unsigned* bad) {
  if (fabsf(f) < 2147483648.0f) return (long long)__float2int_rn(f);
  int bits = __float_as_int(f);
  int e = ((bits >> 23) & 0xFF) - 127;
  long long m = (long long)((bits & 0x7FFFFF) | 0x800000);
  if (e > 62) {  // beyond +-2^62 quanta (includes Inf/NaN)
    *bad = 1u;
    return 0;
  }
  long long v = m << (e - 23);
  return bits < 0 ? -v : v;
}

// Division, reciprocal and square root in the contact force: in FP32 the
// hardware approximations of PTX (div.approx.f32 within 2 ulp; rcp.approx
// and sqrt.approx.f32 within about 1 ulp), orders of magnitude inside the
// force tolerance and several instructions cheaper each than the correctly
// rounded forms; FP64 keeps the correctly rounded operations.
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float frcp(float a) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ double frcp(double a) { return 1.0 / a; }
__device__ __forceinline__ float fsqrt(float a) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ double fsqrt(double a) { return sqrt(a); }

__device__ __forceinline__ long long floor_div64(long long a, long long b) {
  long long q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

__device__ __forceinline__ int clampi(long long c, int n) {
  return c < 0 ? 0 : (c > n - 1 ? n - 1 : (int)c);
}

__device__ __forceinline__ int pack_cell(int cx, int cy, int cz) {
  return cx | (cy << 10) | (cz << 20);
}
__device__ __forceinline__ void unpack_cell(int p, int& cx, int& cy, int& cz) {
  cx = p & 1023;
  cy = (p >> 10) & 1023;
  cz = (p >> 20) & 1023;
}

// 4-wide vectors for velocity (v, m) and spin (w, r); FP64 uses 32-byte
// records loaded as two 16-byte halves.
struct __align__(16) d4 {
  double x, y, z, w;
};
__device__ __forceinline__ float4 ld4(const float4* p) { return __ldg(p); }
__device__ __forceinline__ d4 ld4(const d4* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  double2 a = __ldg(q), b = __ldg(q + 1);
  return {a.x, a.y, b.x, b.y};
}
// Read-only loads with a 128-byte L2 fetch hint (PTX ld.global.nc with
// .L2::128B), for gathers whose neighbouring slots the same warp reads soon
// after (the pair kernel's loads of both members' state: a warp's pairs lie in
// a few neighbouring cells), whatever fetch granularity the context sets for
// the other loads.
__device__ __forceinline__ float4 ld4_fetch128(const float4* p) {
  float4 v;
  asm("ld.global.nc.L2::128B.v4.f32 {%0, %1, %2, %3}, [%4];"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ d4 ld4_fetch128(const d4* p) {
  d4 v;
  asm("ld.global.nc.L2::128B.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
  asm("ld.global.nc.L2::128B.v2.f64 {%0, %1}, [%2];"
      : "=d"(v.z), "=d"(v.w) : "l"(reinterpret_cast<const double*>(p) + 2));
  return v;
}
__device__ __forceinline__ long long ld_fetch128(const long long* p) {
  long long v;
  asm("ld.global.nc.L2::128B.s64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double ld_fetch128(const double* p) {
  double v;
  asm("ld.global.nc.L2::128B.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_fetch128(const float* p) {
  float v;
  asm("ld.global.nc.L2::128B.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ int ld_fetch128(const int* p) {
  int v;
  asm("ld.global.nc.L2::128B.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
// Programmatic dependent launch (PTX griddepcontrol): a kernel launched with
// the programmatic stream serialization attribute may start while the kernel
// before it in the stream is still running, once that kernel's blocks have
// all signalled (or exited); it must wait (pdl_wait: until that kernel has
// completed and its writes are visible) before it reads what that kernel
// writes or writes what it reads.  Both are no-ops for a kernel launched
// without the attribute.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void st4(float4* p, float4 v) { *p = v; }
__device__ __forceinline__ void st4(d4* p, d4 v) {
  double2* q = reinterpret_cast<double2*>(p);
  q[0] = make_double2(v.x, v.y);
  q[1] = make_double2(v.z, v.w);
}

template <typename R> struct vec4_of;
template <> struct vec4_of<float> { using type = float4; };
template <> struct vec4_of<double> { using type = d4; };

template <typename R>
__device__ __forceinline__ typename vec4_of<R>::type mk4(R x, R y, R z, R w) {
  return {x, y, z, w};
}

}  // namespace dem
