// dg_device.cuh — device building blocks of the RKDG jump-filter kernels (sm_103a).
//
// Basis (Eq. GLbasisequation): Legendre P_l on [-1,1], tabulated at compile time from
// dg_tables.cuh; endpoint derivatives from the closed form
//   P_l^{(r)}(+1) = (l+r)! / (2^r r! (l-r)!),   P_l^{(r)}(-1) = (-1)^{l+r} P_l^{(r)}(+1).
// Physics: Burgers f = u^2/2, linear advection f = a u, Euler (Section 3.1, 3.2) with
// p = (gamma-1)(E - |m|^2/(2 rho)), wave speed |u_n| + c, enthalpy H = (E + p)/rho.
// Numerical flux: local Lax–Friedrichs (Section 3).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "dg_tables.cuh"

namespace dgk {

enum { EQ_ADV = 0, EQ_BURG = 1, EQ_EULER = 2 };
enum { BASIS_Q = 0, BASIS_P = 1 };
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1 };

// The stage kernels' filter switch: off, or the damping coefficients of DG_FILTER_JUMP,
// DG_FILTER_GLOBAL, DG_FILTER_OEDG (include/dg.h) plus one.
enum { FILT_OFF = 0, FILT_JUMP = 1, FILT_GLOBAL = 2, FILT_OEDG = 3 };

// Error bits of DevScalars::err.
enum : unsigned { ERRB_NONPHYS = 1u, ERRB_RATE = 2u };

// Device-resident step control shared by the stage kernels of one solver.
struct DevScalars {
  double t;                       // current time
  double T_end;                   // stop time (inf for unclipped stepping)
  double dt;                      // step size of the step in progress (written by stage 0)
  unsigned long long rate_bits[2];  // CFL rate max (bits of a non-negative double), by step parity
  long long step;                 // completed steps
  long long max_step;             // stop when step reaches this
  unsigned int done;              // 1: t >= T_end or step >= max_step; stage kernels do nothing
  unsigned int err;               // ERRB_* bits; stage kernels do nothing
  unsigned int blocks_done;       // last-block counter of the final stage
  unsigned int is_last;           // current step is clipped to land on T_end
};

// Hybrid limiter (Algorithm 1) of one solver: the stage kernel stores the unfiltered DG solution
// and, per output cell, the jump indicator eta and the filter factors exp(-sigma^l dt), l >= 1; it
// appends the troubled cells (eta > 1) to `list` and maxes eta into `max_bits`. The blend kernel
// then rescales the higher modes of the listed cells and clears the scalars for the next stage.
struct HybridScalars {
  unsigned long long max_bits;    // max eta over the stage (bits of a non-negative double)
  unsigned int count;             // troubled cells listed
  unsigned int blocks;            // last-block counter of the blend kernel
};
struct HybridOut {
  void* eta;                      // [ncell], stage arithmetic type
  void* fac;                      // [LMAX][ncell], factor of total degree l = 1..LMAX
  int* list;                      // [ncell] troubled cells
  HybridScalars* sc;
};

// OEDG damping (DG_FILTER_OEDG, Section 2.1): the stage kernel stores the unfiltered stage solution
// and, per output cell, variable v and total degree l, the jump sum A_v(l) of the coefficient
// (the beta-weighted, h-scaled sums of the edge jumps with the weights (2m+1)/m!); it also reduces,
// per variable, the sum of the cell averages and the largest and smallest value at the volume Gauss
// points. The OEDG filter kernel then forms sigma^l = max_v A_v(l) / (2 (2k-1) ||u_v - avg u_v||_inf)
// and rescales the modes.
struct OedgScalars {
  double sum[4];                          // sum of the cell averages per variable
  unsigned long long maxb[4];             // largest point value per variable (ordered_bits)
  unsigned long long nminb[4];            // smallest point value per variable (~ordered_bits)
  unsigned int active;                    // the stage kernel ran (else the filter kernel does nothing)
  unsigned int blocks;                    // last-block counter of the filter kernel
};
struct OedgOut {
  void* A;                                // [NV][LMAX][ncell], stage arithmetic type
  OedgScalars* sc;
};
// Order-preserving map of a double to 64 bits (atomicMax on signed values); all-zero scalars are
// the empty max (maxb) and the empty min (nminb).
__host__ __device__ inline unsigned long long ordered_bits(double x) {
#ifdef __CUDA_ARCH__
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  memcpy(&b, &x, sizeof(b));
#endif
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__host__ __device__ inline double from_ordered_bits(unsigned long long o) {
  const unsigned long long b = (o >> 63) ? (o & 0x7fffffffffffffffull) : ~o;
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  memcpy(&x, &b, sizeof(x));
  return x;
#endif
}

__host__ __device__ constexpr double cfact(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

// d^r P_l at -1 (side 0) or +1 (side 1), closed form.
__host__ __device__ constexpr double dend(int side, int l, int r) {
  return r > l ? 0.0
               : ((side == 0 && ((l + r) & 1)) ? -1.0 : 1.0) * cfact(l + r) /
                     (double)(1 << r) / cfact(r) / cfact(l - r);
}

// Mode enumeration: q outer, p inner; P^k drops p + q > k.
template <int K, int BASIS>
struct Modes {
  static constexpr int NM = BASIS == BASIS_Q ? (K + 1) * (K + 1) : (K + 1) * (K + 2) / 2;
  static constexpr int LMAX = BASIS == BASIS_Q ? 2 * K : K;
  __host__ __device__ static constexpr int p(int m) {
    if (BASIS == BASIS_Q) return m % (K + 1);
    int idx = 0;
    for (int q = 0; q <= K; ++q)
      for (int pp = 0; pp + q <= K; ++pp) {
        if (idx == m) return pp;
        ++idx;
      }
    return -1;
  }
  __host__ __device__ static constexpr int q(int m) {
    if (BASIS == BASIS_Q) return m / (K + 1);
    int idx = 0;
    for (int qq = 0; qq <= K; ++qq)
      for (int pp = 0; pp + qq <= K; ++pp) {
        if (idx == m) return qq;
        ++idx;
      }
    return -1;
  }
  // Multi-indices alpha = (a1, a2) with nonzero derivatives: a1, a2 <= K (and a1 + a2 <= K for P^k).
  static constexpr int NA = BASIS == BASIS_Q ? (K + 1) * (K + 1) : (K + 1) * (K + 2) / 2;
  __host__ __device__ static constexpr int a1(int a) { return p(a); }
  __host__ __device__ static constexpr int a2(int a) { return q(a); }
};

// Small constexpr array usable in device code (tables are built by the compiler front end and the
// unrolled loops read them at constant indices).
template <class V, int N>
struct carr {
  V v[N];
  __host__ __device__ constexpr V operator[](int i) const { return v[i]; }
  __host__ __device__ constexpr V& operator[](int i) { return v[i]; }
};

// Compile-time loop: f(cint<0>{}), ..., f(cint<N-1>{}). Inside f the index is a constant
// expression (decltype(i)::value), so table entries it selects are folded by the front end and
// `if constexpr` can drop zero terms; nothing depends on the optimiser unrolling a loop.
template <int I>
struct cint {
  static constexpr int value = I;
};
template <int I, int N, class F>
__device__ __forceinline__ void sfor_from(F& f) {
  if constexpr (I < N) {
    f(cint<I>{});
    sfor_from<I + 1, N>(f);
  }
}
template <int N, class F>
__device__ __forceinline__ void sfor(F&& f) {
  sfor_from<0, N>(f);
}

template <int EQ, int DIM>
struct NVars {
  static constexpr int value = EQ == EQ_EULER ? (DIM == 1 ? 3 : 4) : 1;
};

// Physical constants handed to the kernels.
struct PhysConst {
  double gamma, ax, ay;
};

// Reciprocal and square root of the fluxes' primitive variables: in FP32 the hardware
// approximations without the full-range and denormal handling of the compiler's approximate division
// and square root (one MUFU instruction each; the same values for the normal, positive densities and
// pressures of the FP32 form; NaN for a negative square-root argument, which the callers rely on to
// report a non-physical trace); correctly rounded in FP64. 2048^2 Q2 FP32 form: 0.662 -> 0.629 ms
// per stage launch, bit for bit the same states.
__device__ __forceinline__ float arcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double arcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float asqrt(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double asqrt(double x) { return sqrt(x); }

// ---- fluxes ------------------------------------------------------------------------------
// 1D flux of u (NV = 1 or 3).
template <int EQ, class T>
__device__ __forceinline__ void flux1d(const T* u, T* f, T gm1, T ax) {
  if constexpr (EQ == EQ_ADV) {
    f[0] = ax * u[0];
  } else if constexpr (EQ == EQ_BURG) {
    f[0] = T(0.5) * u[0] * u[0];
  } else {
    T vel = u[1] * arcp(u[0]);
    T p = gm1 * (u[2] - T(0.5) * u[1] * vel);
    f[0] = u[1];
    f[1] = u[1] * vel + p;
    f[2] = vel * (u[2] + p);
  }
}

template <int EQ, class T>
__device__ __forceinline__ T speed1d(const T* u, T gamma, T gm1, T ax) {
  if constexpr (EQ == EQ_ADV) {
    return fabs(ax);
  } else if constexpr (EQ == EQ_BURG) {
    return fabs(u[0]);
  } else {
    const T inv = arcp(u[0]);
    T vel = u[1] * inv;
    T p = gm1 * (u[2] - T(0.5) * u[1] * vel);
    return fabs(vel) + asqrt(gamma * p * inv);
  }
}

// 2D flux in direction DIR (0 = x, 1 = y).
template <int EQ, int DIR, class T>
__device__ __forceinline__ void flux2d(const T* u, T* f, T gm1, T ax, T ay) {
  if constexpr (EQ == EQ_ADV) {
    f[0] = (DIR == 0 ? ax : ay) * u[0];
  } else if constexpr (EQ == EQ_BURG) {
    f[0] = T(0.5) * u[0] * u[0];
  } else {
    T inv = arcp(u[0]);
    T vx = u[1] * inv, vy = u[2] * inv;
    T p = gm1 * (u[3] - T(0.5) * (u[1] * vx + u[2] * vy));
    T vn = DIR == 0 ? vx : vy;
    f[0] = DIR == 0 ? u[1] : u[2];                 // rho u_n is the momentum component itself
    f[1] = u[1] * vn + (DIR == 0 ? p : T(0));
    f[2] = u[2] * vn + (DIR == 1 ? p : T(0));
    f[3] = vn * (u[3] + p);
  }
}

// Both directional fluxes at a volume point (shares the primitive variables).
template <int EQ, class T>
__device__ __forceinline__ void flux2d_xy(const T* u, T* fx, T* fy, T gm1, T ax, T ay) {
  if constexpr (EQ == EQ_ADV) {
    fx[0] = ax * u[0];
    fy[0] = ay * u[0];
  } else if constexpr (EQ == EQ_BURG) {
    fx[0] = T(0.5) * u[0] * u[0];
    fy[0] = fx[0];
  } else {
    T inv = arcp(u[0]);
    T vx = u[1] * inv, vy = u[2] * inv;
    T p = gm1 * (u[3] - T(0.5) * (u[1] * vx + u[2] * vy));
    T ep = u[3] + p;
    fx[0] = u[1];
    fx[1] = u[1] * vx + p;
    fx[2] = u[2] * vx;
    fx[3] = vx * ep;
    fy[0] = u[2];
    fy[1] = u[1] * vy;
    fy[2] = u[2] * vy + p;
    fy[3] = vy * ep;
  }
}

template <int EQ, int DIR, class T>
__device__ __forceinline__ T speed2d(const T* u, T gamma, T gm1, T ax, T ay) {
  if constexpr (EQ == EQ_ADV) {
    return fabs(DIR == 0 ? ax : ay);
  } else if constexpr (EQ == EQ_BURG) {
    return fabs(u[0]);
  } else {
    T inv = arcp(u[0]);
    T vx = u[1] * inv, vy = u[2] * inv;
    T p = gm1 * (u[3] - T(0.5) * (u[1] * vx + u[2] * vy));
    return fabs(DIR == 0 ? vx : vy) + asqrt(gamma * p * inv);
  }
}

// max that keeps a NaN: a non-physical trace (p < 0 gives a NaN sound speed) must reach the cell
// averages and be reported, not be hidden by the other side's wave speed.
template <class T>
__device__ __forceinline__ T nan_max(T a, T b) {
  return (a > b || a != a) ? a : b;
}
// FP32: the same in one instruction (max.NaN returns NaN if either operand is NaN)
__device__ __forceinline__ float nan_max(float a, float b) {
  float r;
  asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}

// Local Lax–Friedrichs flux for a 1D face: fh = 1/2 (f(uL) + f(uR)) - 1/2 alpha (uR - uL).
template <int EQ, class T>
__device__ __forceinline__ void llf1d(const T* uL, const T* uR, T* fh, T gamma, T gm1, T ax) {
  constexpr int NV = EQ == EQ_EULER ? 3 : 1;
  T fL[NV], fR[NV];
  flux1d<EQ>(uL, fL, gm1, ax);
  flux1d<EQ>(uR, fR, gm1, ax);
  T a = nan_max(speed1d<EQ>(uL, gamma, gm1, ax), speed1d<EQ>(uR, gamma, gm1, ax));
#pragma unroll
  for (int v = 0; v < NV; ++v) fh[v] = T(0.5) * (fL[v] + fR[v]) - T(0.5) * a * (uR[v] - uL[v]);
}

template <int EQ, int DIR, class T>
__device__ __forceinline__ void llf2d(const T* uL, const T* uR, T* fh, T gamma, T gm1, T ax, T ay) {
  constexpr int NV = EQ == EQ_EULER ? 4 : 1;
  T fL[NV], fR[NV];
  flux2d<EQ, DIR>(uL, fL, gm1, ax, ay);
  flux2d<EQ, DIR>(uR, fR, gm1, ax, ay);
  T a = nan_max(speed2d<EQ, DIR>(uL, gamma, gm1, ax, ay), speed2d<EQ, DIR>(uR, gamma, gm1, ax, ay));
#pragma unroll
  for (int v = 0; v < NV; ++v) fh[v] = T(0.5) * (fL[v] + fR[v]) - T(0.5) * a * (uR[v] - uL[v]);
}

// Cell-average quantities for the filter and the CFL rate: beta^x, beta^y, 1/Hbar.
template <int EQ, int DIM, class T>
__device__ __forceinline__ void avg_params(const T* ub, T gamma, T gm1, T ax, T ay, T& bx, T& by,
                                           T& invH, bool& physical) {
  if constexpr (EQ == EQ_ADV) {
    bx = fabs(ax);
    by = fabs(ay);
    invH = T(1);
    physical = isfinite(ub[0]);
  } else if constexpr (EQ == EQ_BURG) {
    bx = fabs(ub[0]);
    by = bx;
    invH = T(1);
    physical = isfinite(ub[0]);
  } else if constexpr (DIM == 1) {
    const T inv = arcp(ub[0]);
    T vel = ub[1] * inv;
    T p = gm1 * (ub[2] - T(0.5) * ub[1] * vel);
    T c = asqrt(gamma * p * inv);
    bx = fabs(vel) + c;
    by = T(0);
    invH = ub[0] * arcp(ub[2] + p);
    physical = (ub[0] > T(0)) && (p > T(0)) && isfinite(bx) && isfinite(invH);
  } else {
    T inv = arcp(ub[0]);
    T vx = ub[1] * inv, vy = ub[2] * inv;
    T p = gm1 * (ub[3] - T(0.5) * (ub[1] * vx + ub[2] * vy));
    T c = asqrt(gamma * p * inv);
    bx = fabs(vx) + c;
    by = fabs(vy) + c;
    invH = ub[0] * arcp(ub[3] + p);
    physical = (ub[0] > T(0)) && (p > T(0)) && isfinite(bx) && isfinite(by) && isfinite(invH);
  }
}

// ---- positivity-preserving limiter (Zhang & Shu 2010), Euler ----------------------------------
// Pressure of a conservative state (1D: NV = 3, 2D: NV = 4).
template <int NV, class T>
__device__ __forceinline__ T pressure_of(const T* w, T gm1) {
  if constexpr (NV == 3) return gm1 * (w[2] - T(0.5) * w[1] * w[1] / w[0]);
  else return gm1 * (w[3] - T(0.5) * (w[1] * w[1] + w[2] * w[2]) / w[0]);
}

// Largest t in [0, 1] with p(ub + t (w - ub)) >= eps, by bisection (the admissible set is convex,
// so p - eps changes sign once on the segment; p(ub) >= eps, p(w) < eps on entry).
template <int NV, class T>
__device__ __noinline__ T pp_segment(const T* ub, const T* w, T eps, T gm1) {
  T lo = T(0), hi = T(1);
  const int iters = sizeof(T) == 8 ? 60 : 30;
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
    const T mid = T(0.5) * (lo + hi);
    T x[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = ub[v] + mid * (w[v] - ub[v]);
    if (pressure_of<NV>(x, gm1) >= eps) lo = mid; else hi = mid;
  }
  return lo;
}

// ---- storage of the FP32 form ---------------------------------------------------------------
// Word index (4-byte words from the state's base) of coefficient (v, m) of cell c, m = NM meaning the
// low word of the double-float cell average.
//   plain layout (an odd number of variables): float2 planes (hi, lo) of the averages per variable,
//     then one float plane per (variable, mode >= 1);
//   paired layout (an even number of variables, 2D Euler): per pair of variables a region of float4
//     planes over the cells, {hi v0, hi v1, lo v0, lo v1}, then {v0[m], v1[m], v0[m+1], v1[m+1]} for
//     m = 1, 3, ..., and a float2 plane {v0[m], v1[m]} for a last single mode; each region a multiple
//     of 16 bytes. A warp reads a pair's two variables, two modes at a time, with 128-bit loads, and
//     the values land in the register pairs of the packed two-lane FP32 arithmetic.
struct F32Layout {
  long long ncell;
  int nv, nm;
  __host__ __device__ bool paired() const { return (nv & 1) == 0; }
  // words of one pair's region
  __host__ __device__ long long region_words() const { return ((ncell * (4 + 2LL * (nm - 1)) + 3) / 4) * 4; }
  __host__ __device__ long long word(int v, int m, long long c) const {
    if (!paired()) {
      if (m == 0 || m == nm) return 2LL * ((long long)v * ncell + c) + (m == nm ? 1 : 0);
      return 2LL * nv * ncell + ((long long)v * (nm - 1) + m - 1) * ncell + c;
    }
    const long long base = (long long)(v >> 1) * region_words();
    const int j = v & 1;
    if (m == 0) return base + 4 * c + j;
    if (m == nm) return base + 4 * c + 2 + j;
    const int i = m - 1, q = i >> 1;
    if (q < (nm - 1) / 2) return base + 4 * ncell * (1 + q) + 4 * c + 2 * (i & 1) + j;
    return base + 4 * ncell * (1 + (nm - 1) / 2) + 2 * c + j;
  }
  __host__ __device__ size_t bytes() const {
    return paired() ? sizeof(float) * (size_t)(nv / 2) * (size_t)region_words()
                    : (sizeof(float2) + sizeof(float) * (size_t)(nm - 1)) * (size_t)nv * (size_t)ncell;
  }
};

// ---- double-float arithmetic (error-free transformations; Dekker / Knuth) -------------------
struct df {
  float hi, lo;
};
__device__ __forceinline__ df df_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = df_two_sum(a.hi, b.hi);
  df t = df_two_sum(a.lo, b.lo);
  float c = __fadd_rn(s.lo, t.hi);
  df v = df_fast_two_sum(s.hi, c);
  float w = __fadd_rn(t.lo, v.lo);
  return df_fast_two_sum(v.hi, w);
}
__device__ __forceinline__ df df_mul(df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
  float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return df_fast_two_sum(p, e);
}
// Running double-float sum: each float term is added to hi by an error-free two-sum and the
// rounding error (with the low parts of df terms and products) is collected in lo; one fast
// two-sum renormalises at the end. The error is a few units of 2^-48 times the sum of the terms'
// magnitudes, which is what conservation of the cell averages needs (the flux terms of a face are
// formed bitwise alike on its two sides).
struct df_acc {
  float hi, lo;
  __device__ __forceinline__ void add(float x) {
    const float s = __fadd_rn(hi, x);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ void add(df x) {
    add(x.hi);
    lo = __fadd_rn(lo, x.lo);
  }
  // + a * b: a.hi * b exactly as p + e (FMA), a.lo * b rounded
  __device__ __forceinline__ void add_prod(df a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    add(p);
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ df result() const { return df_fast_two_sum(hi, lo); }
};

__host__ __device__ inline df df_from_double(double x) {
  float hi = (float)x;
  float lo = (float)(x - (double)hi);
  return {hi, lo};
}

// ---- two FP32 lanes in one register pair (the packed FP32 instructions of sm_100 and later) ----
// Each lane is rounded to nearest exactly like the scalar instruction, so a sum of products
// formed lane-wise with vmad equals the scalar FMA chain bit for bit (the sign of a zero sum
// aside: packed sums start at +0, scalar ones at -0).
struct f2 {
  float x, y;
};
__device__ __forceinline__ float2 f2v(f2 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ f2 f2of(float2 a) { return f2{a.x, a.y}; }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2of(__fadd2_rn(f2v(a), f2v(b))); }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) {
  f2 d;
  asm("{\n\t.reg .b64 pa, pb, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ f2 operator-(f2 a) { return f2{-a.x, -a.y}; }

__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return f2of(__fmul2_rn(f2v(a), f2v(b))); }
__device__ __forceinline__ f2 vfma(f2 a, f2 b, f2 c) { return f2of(__ffma2_rn(f2v(a), f2v(b), f2v(c))); }

// Two double-float values (two variables) in register pairs; every lane performs exactly the
// operations of the scalar df functions and df_acc below, so the results are bitwise the same.
struct df2 {
  f2 hi, lo;
};
__device__ __forceinline__ df2 df2_fast_two_sum(f2 a, f2 b) {
  const f2 s = a + b;
  return {s, b - (s - a)};
}
// a (one double-float for both lanes) times b
__device__ __forceinline__ df2 df2_mul(df a, df2 b) {
  const f2 ah{a.hi, a.hi}, al{a.lo, a.lo};
  const f2 p = ah * b.hi;
  f2 e = vfma(ah, b.hi, -p);
  e = vfma(ah, b.lo, e);
  e = vfma(al, b.hi, e);
  return df2_fast_two_sum(p, e);
}
struct df2_acc {
  f2 hi, lo;
  __device__ __forceinline__ void add(f2 x) {
    const f2 s = hi + x;
    const f2 bb = s - hi;
    const f2 e = (hi - (s - bb)) + (x - bb);
    hi = s;
    lo = lo + e;
  }
  __device__ __forceinline__ void add(df2 x) {
    add(x.hi);
    lo = lo + x.lo;
  }
  // + a * b: a.hi * b exactly as p + e (FMA), a.lo * b rounded
  __device__ __forceinline__ void add_prod(df a, f2 b) {
    const f2 ah{a.hi, a.hi}, al{a.lo, a.lo};
    const f2 p = ah * b;
    f2 e = vfma(ah, b, -p);
    e = vfma(al, b, e);
    add(p);
    lo = lo + e;
  }
  __device__ __forceinline__ df2 result() const { return df2_fast_two_sum(hi, lo); }
};

// value-type generic arithmetic for the sum-factorised kernels: T = float, double or f2
template <class V>
struct vtraits {
  using S = V;
  static __device__ __forceinline__ V zero() { return V(-0.0); }   // additive identity
};
template <>
struct vtraits<f2> {
  using S = float;
  static __device__ __forceinline__ f2 zero() { return f2{0.f, 0.f}; }
};
__device__ __forceinline__ float vmad(float x, float c, float acc) { return acc + x * c; }
__device__ __forceinline__ double vmad(double x, double c, double acc) { return acc + x * c; }
__device__ __forceinline__ f2 vmad(f2 x, float c, f2 acc) {
  return f2of(__ffma2_rn(f2v(x), make_float2(c, c), f2v(acc)));
}
__device__ __forceinline__ float vabs(float x) { return fabsf(x); }
__device__ __forceinline__ double vabs(double x) { return fabs(x); }
__device__ __forceinline__ f2 vabs(f2 x) { return f2{fabsf(x.x), fabsf(x.y)}; }
// max(|a|, |b|), lane by lane
__device__ __forceinline__ float vmaxabs(float a, float b) { return fmaxf(fabsf(a), fabsf(b)); }
__device__ __forceinline__ double vmaxabs(double a, double b) { return fmax(fabs(a), fabs(b)); }
__device__ __forceinline__ f2 vmaxabs(f2 a, f2 b) {
  return f2{fmaxf(fabsf(a.x), fabsf(b.x)), fmaxf(fabsf(a.y), fabsf(b.y))};
}
__device__ __forceinline__ float vscale(float x, float c) { return x * c; }
__device__ __forceinline__ double vscale(double x, double c) { return x * c; }
__device__ __forceinline__ f2 vscale(f2 x, float c) { return f2of(__fmul2_rn(f2v(x), make_float2(c, c))); }
// A sum whose first term is taken as it is (no add to a zero): in the fully unrolled callers the
// flag is a compile-time constant at every use.
template <class V>
struct vsum {
  V s;
  bool any = false;
  __device__ __forceinline__ void add(V x) {
    s = any ? s + x : x;
    any = true;
  }
  __device__ __forceinline__ V get() const { return any ? s : vtraits<V>::zero(); }
};
__device__ __forceinline__ float shfl_down_v(float x, int d) { return __shfl_down_sync(0xffffffffu, x, d); }
__device__ __forceinline__ double shfl_down_v(double x, int d) { return __shfl_down_sync(0xffffffffu, x, d); }
__device__ __forceinline__ f2 shfl_down_v(f2 x, int d) {
  return f2{__shfl_down_sync(0xffffffffu, x.x, d), __shfl_down_sync(0xffffffffu, x.y, d)};
}
__device__ __forceinline__ float shfl_up_v(float x, int d) { return __shfl_up_sync(0xffffffffu, x, d); }
__device__ __forceinline__ double shfl_up_v(double x, int d) { return __shfl_up_sync(0xffffffffu, x, d); }
__device__ __forceinline__ f2 shfl_up_v(f2 x, int d) {
  return f2{__shfl_up_sync(0xffffffffu, x.x, d), __shfl_up_sync(0xffffffffu, x.y, d)};
}

// Atomic max of a non-negative double through its bit pattern (monotone for x >= 0; NaN sorts
// above +inf, so a NaN rate is kept and reported).
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double x) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(x));
}

__device__ __forceinline__ double warp_max(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double y = __shfl_xor_sync(0xffffffffu, x, o);
    x = (y > x || y != y) ? y : x;
  }
  return x;
}

}  // namespace dgk
