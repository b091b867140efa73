// stage2d.cuh — fused 2D SSP-RK3 stage with the jump filter (one launch per stage).
//
// What one launch computes, per cell K_ij (Section 2.2 weak form, Section 3 choices):
//   R = M^{-1} [ (F(u), grad phi)_K - <F^ . n, phi>_{dK} ]          (volume + LLF edge fluxes)
//   u~ = c0 u^n + c1 (u^(s) + dt R)                                  (Shu–Osher, Eq. rkdg1)
//   u^{p,q} <- exp(-sigma_l dt) u~^{p,q},  l = p + q >= 1           (Eq. para:2ddamp)
//   sigma_l = max_v (1/Hbar) [ beta^x (J^V_0 + sum_{m=1..l} m(m+1) h_x^m S^V_m)
//                             + beta^y (J^H_0 + sum_{m=1..l} m(m+1) h_y^m S^H_m) ]
// which is Eqs. (para:damp22d)-(para:damp22d1) with (c_fx, c_fy) = (h_y beta^x, h_x beta^y) /
// (4 lambda_{p,q} Hbar) of Section 3.2 substituted (lambda_{p,q} and the (2/h)^2 factor cancel), the
// max over components of Section 2.3, S_m = sum_{|alpha| = m} of the edge-averaged absolute jumps of
// d^alpha u, each edge average taken by the trapezoidal rule over the edge's two corners.
//
// Parallel structure (GB300): a warp owns a strip of 32 consecutive columns (28 output columns plus
// a 2-column halo on each side) and a chunk of rows; lane L owns column x0 + L and marches upwards.
//   - x-neighbours: warp shuffles (face traces, face fluxes, corner derivatives, jump sums); each
//     vertical face flux is computed once, by its left cell, and shuffled to the right cell.
//   - y-neighbours: the previous row's top traces live in registers; three per-lane shared-memory
//     slots hold the stage values u~ of rows t, t-1, t-2. Each horizontal face flux and face jump
//     is computed once per column. No row is computed twice except the 2 halo rows per chunk.
//   - coalescing: the state is structure-of-arrays u[v][m][cell] with x fastest, so a warp's load
//     of one coefficient of one row is 32 consecutive words.
// Face fluxes and jumps at tile seams are recomputed by both tiles with the same operands in the
// same order, so both sides see bitwise-equal values and conservation holds to roundoff.
#pragma once
#include <type_traits>

#include "stage_common.cuh"

namespace dgk {

// Mesh and physics constants of a 2D stage, computed once by stage2d_consts (on the host for a
// single solve, so that the kernel reads them from its parameter space instead of holding them in
// registers): powers of 2/h for physical derivatives, the filter's per-order jump weights (the jump
// filter's m(m+1) h^m, or the OEDG form's (2m+1)/m! h^(m-1), with the trapezoid's 1/2), 1/h, gamma,
// gamma - 1 and the advection velocity.
template <class T>
struct Consts2D {
  T px[4], py[4], wx[7], wy[7];
  T pxy[16], pxy2[16];   // (2/h_x)^a1 (2/h_y)^a2 at [a1 * 4 + a2], and twice that
  T ihx, ihy, gam, gm1, ax, ay;
};

struct Stage2DArgs {
  const void* uin;   // u^(s), the stage input
  const void* un;    // u^n
  void* uout;        // output (never aliases uin or un)
  int nx, ny;
  long long ncell;
  double hx, hy;
  int bcx, bcy;      // BC_PERIODIC or BC_OUTFLOW (both sides of an axis alike)
  double c0, c1;     // u~ = c0 u^n + c1 (u^(s) + dt R)
  int stage;         // 0, 1, 2
  int filter_on;      // FILT_OFF, FILT_JUMP or FILT_GLOBAL
  double gamma, ax, ay, cfl;
  int H;             // rows per chunk
  int nstrips, nchunks;
  int positivity;    // Euler: Zhang-Shu limiter after the filter
  int hybrid;        // hybrid limiter (Algorithm 1): store u^DG, eta and the filter factors
  HybridOut hyb;
  OedgOut oe;        // OEDG damping (kernels instantiated with OE = true)
  DevScalars* sc;
  Consts2D<float> cf;  // stage2d_consts
  Consts2D<double> cd;
};

template <class T>
__host__ __device__ inline void consts2d_fill(Consts2D<T>& c, double hx, double hy, double gamma, double ax,
                                              double ay, bool oedg) {
  c.ihx = (T)(1.0 / hx);
  c.ihy = (T)(1.0 / hy);
  c.gam = (T)gamma;
  c.gm1 = (T)(gamma - 1.0);
  c.ax = (T)ax;
  c.ay = (T)ay;
  double px[4], py[4];
  px[0] = py[0] = 1.0;
  for (int r = 1; r < 4; ++r) {
    px[r] = px[r - 1] * (2.0 / hx);
    py[r] = py[r - 1] * (2.0 / hy);
  }
  for (int r = 0; r < 4; ++r) {
    c.px[r] = (T)px[r];
    c.py[r] = (T)py[r];
  }
  for (int a1 = 0; a1 < 4; ++a1)
    for (int a2 = 0; a2 < 4; ++a2) {
      c.pxy[a1 * 4 + a2] = (T)(px[a1] * py[a2]);
      c.pxy2[a1 * 4 + a2] = (T)(2.0 * px[a1] * py[a2]);
    }
  double hmx = 1.0, hmy = 1.0, fm = 1.0;        // h^m, m!
  for (int m = 0; m < 7; ++m) {
    if (m > 0) fm *= m;
    if (!oedg) {
      c.wx[m] = (T)(m == 0 ? 0.5 : 0.5 * m * (m + 1) * hmx);
      c.wy[m] = (T)(m == 0 ? 0.5 : 0.5 * m * (m + 1) * hmy);
    } else {
      c.wx[m] = (T)(0.5 * (2 * m + 1) / fm * hmx / hx);
      c.wy[m] = (T)(0.5 * (2 * m + 1) / fm * hmy / hy);
    }
    hmx *= hx;
    hmy *= hy;
  }
}
// Fill a.cf and a.cd from a.hx, a.hy, a.gamma, a.ax, a.ay and the filter kind.
__host__ __device__ inline void stage2d_consts(Stage2DArgs& a) {
  const bool oedg = a.filter_on == FILT_OEDG;
  consts2d_fill(a.cf, a.hx, a.hy, a.gamma, a.ax, a.ay, oedg);
  consts2d_fill(a.cd, a.hx, a.hy, a.gamma, a.ax, a.ay, oedg);
}

constexpr int STRIP_OUT = 28;  // output columns per warp

// Storage policies. FP64: one double plane per (v, m). FP32 mixed: F32Layout (the cell average of
// each variable a double-float hi/lo pair; with an even number of variables, pairs of variables in
// float4 planes).
struct PrecF64 {
  using T = double;
  static constexpr bool MIXED = false;
};
struct PrecF32M {
  using T = float;
  static constexpr bool MIXED = true;
};

// COH = true: coherent loads through L2 (ld.global.cg) instead of the read-only path, for kernels that
// read states written earlier by other blocks of the same launch (the persistent batched kernel).
template <class PR, int NV, int NM, bool COH = false>
struct Store {
  using T = typename PR::T;
  template <class V>
  static __device__ __forceinline__ V ld(const V* p) {
    if constexpr (COH) return __ldcg(p);
    else return __ldg(p);
  }
  // the FP32 form with an even number of variables keeps them in pairs (F32Layout)
  static constexpr bool PAIRED = PR::MIXED && (NV % 2) == 0;
  // load u[v][m] (and the low word of the mode-0 double-float in lo0[v]).
  static __device__ __forceinline__ void load(const void* base, long long ncell, long long c,
                                              T (&u)[NV][NM], T (&lo0)[NV]) {
    if constexpr (!PR::MIXED) {
      const double* b = (const double*)base;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
#pragma unroll
        for (int m = 0; m < NM; ++m) u[v][m] = ld(b + (long long)(v * NM + m) * ncell + c);
        lo0[v] = T(0);
      }
    } else if constexpr (PAIRED) {
      const F32Layout L{ncell, NV, NM};
#pragma unroll
      for (int pr = 0; pr < NV / 2; ++pr) {
        const float* r = (const float*)base + pr * L.region_words();
        const float4 a = ld((const float4*)r + c);
        u[2 * pr][0] = a.x;
        u[2 * pr + 1][0] = a.y;
        lo0[2 * pr] = a.z;
        lo0[2 * pr + 1] = a.w;
#pragma unroll
        for (int q = 0; q < (NM - 1) / 2; ++q) {
          const float4 x = ld((const float4*)r + ncell * (1 + q) + c);
          u[2 * pr][1 + 2 * q] = x.x;
          u[2 * pr + 1][1 + 2 * q] = x.y;
          u[2 * pr][2 + 2 * q] = x.z;
          u[2 * pr + 1][2 + 2 * q] = x.w;
        }
        if constexpr (((NM - 1) & 1) != 0) {
          const float2 y = ld((const float2*)(r + 4 * ncell * (1 + (NM - 1) / 2)) + c);
          u[2 * pr][NM - 1] = y.x;
          u[2 * pr + 1][NM - 1] = y.y;
        }
      }
    } else {
      const float2* b0 = (const float2*)base;
      const float* bh = (const float*)((const char*)base + sizeof(float2) * (size_t)NV * ncell);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        float2 a = ld(b0 + (long long)v * ncell + c);
        u[v][0] = a.x;
        lo0[v] = a.y;
#pragma unroll
        for (int m = 1; m < NM; ++m) u[v][m] = ld(bh + (long long)(v * (NM - 1) + m - 1) * ncell + c);
      }
    }
  }
  // L2 prefetch of cell c's words (paired FP32 layout): issued a row ahead of the load, it takes the
  // DRAM latency off the row march (2048^2 Q2: 0.686 -> 0.661 ms per stage launch)
  static __device__ __forceinline__ void prefetch(const void* base, long long ncell, long long c) {
    if constexpr (PAIRED) {
      const F32Layout L{ncell, NV, NM};
#pragma unroll
      for (int pr = 0; pr < NV / 2; ++pr) {
        const float* r = (const float*)base + pr * L.region_words();
#pragma unroll
        for (int q = 0; q <= (NM - 1) / 2; ++q)
          asm volatile("prefetch.global.L2 [%0];" ::"l"((const float4*)r + ncell * q + c));
        if constexpr (((NM - 1) & 1) != 0)
          asm volatile("prefetch.global.L2 [%0];" ::"l"((const float2*)(r + 4 * ncell * (1 + (NM - 1) / 2)) + c));
      }
    }
  }
  static __device__ __forceinline__ void store(void* base, long long ncell, long long c,
                                               const T (&u)[NV][NM], const T (&lo0)[NV]) {
    if constexpr (!PR::MIXED) {
      double* b = (double*)base;
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int m = 0; m < NM; ++m) b[(long long)(v * NM + m) * ncell + c] = u[v][m];
    } else if constexpr (PAIRED) {
      const F32Layout L{ncell, NV, NM};
#pragma unroll
      for (int pr = 0; pr < NV / 2; ++pr) {
        float* r = (float*)base + pr * L.region_words();
        ((float4*)r)[c] = make_float4(u[2 * pr][0], u[2 * pr + 1][0], lo0[2 * pr], lo0[2 * pr + 1]);
#pragma unroll
        for (int q = 0; q < (NM - 1) / 2; ++q)
          ((float4*)r)[ncell * (1 + q) + c] =
              make_float4(u[2 * pr][1 + 2 * q], u[2 * pr + 1][1 + 2 * q], u[2 * pr][2 + 2 * q], u[2 * pr + 1][2 + 2 * q]);
        if constexpr (((NM - 1) & 1) != 0)
          ((float2*)(r + 4 * ncell * (1 + (NM - 1) / 2)))[c] = make_float2(u[2 * pr][NM - 1], u[2 * pr + 1][NM - 1]);
      }
    } else {
      float2* b0 = (float2*)base;
      float* bh = (float*)((char*)base + sizeof(float2) * (size_t)NV * ncell);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        b0[(long long)v * ncell + c] = make_float2(u[v][0], lo0[v]);
#pragma unroll
        for (int m = 1; m < NM; ++m) bh[(long long)(v * (NM - 1) + m - 1) * ncell + c] = u[v][m];
      }
    }
  }
};

// OE = true: the OEDG form of the damping (DG_FILTER_OEDG): the kernel stores u~ unfiltered with the
// jump sums A_v(l) and the reductions of OedgOut, and the OEDG filter kernel applies the damping.
// LIM = false: no positivity or hybrid limiter code (a.positivity and a.hybrid are ignored); a
// smaller loop body for the solves that use neither (2048^2 Q2, FP32 form: 0.748 -> 0.702 ms).
// COH = true: state loads through L2 (Store), for the persistent batched kernel.
template <int K, int EQ, int BASIS, class PR, bool OE = false, bool LIM = true, bool COH = false>
struct Stage2D {
  using T = typename PR::T;
  using MB = Modes<K, BASIS>;
  static constexpr int NM = MB::NM;
  static constexpr int NV = NVars<EQ, 2>::value;
  static constexpr int NQ = K + 1;
  static constexpr int LMAX = MB::LMAX;
  static constexpr int NA = MB::NA;
  static constexpr int NME = NM + (PR::MIXED ? 1 : 0);  // slot words per variable (+ mode-0 low word)
  // FP32 form with an even number of variables: the linear (sum-factorised) parts run on pairs of
  // variables in register pairs (packed FP32 instructions), each lane computing the scalar chain.
  // Edge traces and the double-float cell averages run packed as well at degrees 1-2 (traces) and
  // 2-3 (averages). Measured on GB300 at 2048^2 Q2 with the paired HBM layout, whose loads land in
  // the register pairs: 0.788 ms per stage launch scalar, 0.786 with packed traces, 0.798 with packed
  // averages, 0.764 with both. At degree 1 the packed averages were slower (1024^2: 0.155 -> 0.166
  // ms), at degree 3 faster (0.851 -> 0.820 ms, traces scalar).
  static constexpr bool PACK = PR::MIXED && (NV % 2) == 0;
  static constexpr bool PACK_TRACES = PACK && K <= 2;
  static constexpr bool PACK_DF = PACK && K >= 2;
  using GR = GaussRule<NQ>;
  using ST = Store<PR, NV, NM, COH>;
  using TB = Tab2D<K, BASIS>;

  // Row slots of u~ (rows t, t-1, t-2). Packed FP32 form: per lane, one contiguous block per (slot,
  // pair of variables) of NMEP pair words {v0[m], v1[m]} (m = NM: the low words of the two cell
  // averages), read and written with 128-bit shared-memory instructions; the lane stride LS is
  // 4 (mod 8) words, so the 8 lanes of each phase of a 128-bit access hit distinct banks. Otherwise
  // one row of 32 lanes per (slot, v, m).
  static constexpr int NMEP = (NME + 1) & ~1;
  static constexpr int PW = 3 * (NV / 2) * NMEP * 2;
  static constexpr int LS = PW + (12 - PW % 8) % 8;
  static constexpr int SLOT_WORDS = PACK ? 32 * LS : 3 * NV * NME * 32;
  // per-warp shared memory: the row slots, the partial damping Q[v][l-1] of one row and the partial
  // jump indicator of one row (hybrid limiter)
  static constexpr size_t warp_bytes() { return sizeof(T) * (SLOT_WORDS + (NV * LMAX + 1) * 32); }
  static constexpr size_t slot_bytes_per_warp() { return warp_bytes(); }

  // ---- compile-time tables of the positivity limiter's points (evaluated by the front end) ----
  __host__ __device__ static constexpr carr<int, NM> tab_p() {
    carr<int, NM> t{};
    for (int m = 0; m < NM; ++m) t[m] = MB::p(m);
    return t;
  }
  __host__ __device__ static constexpr carr<int, NM> tab_q() {
    carr<int, NM> t{};
    for (int m = 0; m < NM; ++m) t[m] = MB::q(m);
    return t;
  }
  // traces on the horizontal edge eta = -1 (side 0) / +1 (side 1) at Gauss point g: P_p(x_g) P_q(+-1)
  __host__ __device__ static constexpr carr<double, 2 * NQ * NM> tab_trace_h() {
    carr<double, 2 * NQ * NM> t{};
    for (int sd = 0; sd < 2; ++sd)
      for (int g = 0; g < NQ; ++g)
        for (int m = 0; m < NM; ++m) t[(sd * NQ + g) * NM + m] = GR::P(MB::p(m), g) * dend(sd, MB::q(m), 0);
    return t;
  }
  // traces on the vertical edge xi = -1 / +1: P_p(+-1) P_q(x_g)
  __host__ __device__ static constexpr carr<double, 2 * NQ * NM> tab_trace_v() {
    carr<double, 2 * NQ * NM> t{};
    for (int sd = 0; sd < 2; ++sd)
      for (int g = 0; g < NQ; ++g)
        for (int m = 0; m < NM; ++m) t[(sd * NQ + g) * NM + m] = dend(sd, MB::p(m), 0) * GR::P(MB::q(m), g);
    return t;
  }
  // volume point values P_p(x_a) P_q(x_b)
  __host__ __device__ static constexpr carr<double, NQ * NQ * NM> tab_vol(int) {
    carr<double, NQ * NQ * NM> t{};
    for (int qa = 0; qa < NQ; ++qa)
      for (int qb = 0; qb < NQ; ++qb)
        for (int m = 0; m < NM; ++m) t[(qa * NQ + qb) * NM + m] = GR::P(MB::p(m), qa) * GR::P(MB::q(m), qb);
    return t;
  }

  // Zhang and Shu's Gauss-Lobatto mid-lines: their positivity of the averages uses the Gauss nodes
  // crossed with the N-point Lobatto nodes, 2N - 3 >= k; for k = 3 (N = 3) the Lobatto node 0 is
  // not a Gauss node, so the points (0, x_g) and (x_g, 0) are checked as well (P_l(0) is the
  // 1-point Gauss rule's value table).
  static constexpr int NMID = (K >= 2 && NQ % 2 == 0) ? 2 * NQ : 0;
  __host__ __device__ static constexpr carr<double, (NMID > 0 ? NMID : 1) * NM> tab_mid() {
    carr<double, (NMID > 0 ? NMID : 1) * NM> t{};
    for (int g = 0; g < NQ && NMID > 0; ++g)
      for (int m = 0; m < NM; ++m) {
        t[(2 * g) * NM + m] = GaussRule<1>::P(MB::p(m), 0) * GR::P(MB::q(m), g);
        t[(2 * g + 1) * NM + m] = GR::P(MB::p(m), g) * GaussRule<1>::P(MB::q(m), 0);
      }
    return t;
  }
  // the limiter's points: volume Gauss points, Gauss points of the edges, Lobatto mid-lines
  static constexpr int NP_LIM = NQ * NQ + 4 * NQ + NMID;
  // value of mode m at limiter point i (folds to an immediate for constant i, m)
  static __device__ __forceinline__ double lim_coef(int i, int m) {
    constexpr carr<double, NQ * NQ * NM> VE = tab_vol(0);
    constexpr carr<double, 2 * NQ * NM> TH = tab_trace_h();
    constexpr carr<double, 2 * NQ * NM> TV = tab_trace_v();
    constexpr carr<double, (NMID > 0 ? NMID : 1) * NM> TM = tab_mid();
    return i < NQ * NQ ? VE[i * NM + m]
                       : (i < NQ * NQ + 2 * NQ ? TH[(i - NQ * NQ) * NM + m]
                                               : (i < NQ * NQ + 4 * NQ ? TV[(i - NQ * NQ - 2 * NQ) * NM + m]
                                                                       : TM[(i - NQ * NQ - 4 * NQ) * NM + m]));
  }

  // row slot of row r (rows >= -2 occur; keep the index in 0..2)
  static __device__ __forceinline__ int slot_of(int r) { return ((r % 3) + 3) % 3; }
  // r mod n for r in [-2, n + 1] and n >= 1 (the rows and columns a tile touches), without division
  static __device__ __forceinline__ int wrap_near(int r, int n) {
    r += r < 0 ? n : 0;
    r += r < 0 ? n : 0;
    r -= r >= n ? n : 0;
    r -= r >= n ? n : 0;
    return r;
  }
  static __device__ __forceinline__ T* slot_ptr(T* ws, int s, int v, int m, int lane) {
    if constexpr (PACK) return ws + lane * LS + ((s * (NV / 2) + v / 2) * NMEP + m) * 2 + (v & 1);
    else return ws + (((s * NV + v) * NME + m) << 5) + lane;
  }
  // packed form: the block of a pair of variables, and its NMEP pair words in registers
  static __device__ __forceinline__ float4* pblock(T* ws, int s, int vp, int lane) {
    return (float4*)(ws + lane * LS + (s * (NV / 2) + vp) * NMEP * 2);
  }
  static __device__ __forceinline__ void pload(const float4* b, f2 (&w)[NMEP]) {
#pragma unroll
    for (int i = 0; i < NMEP / 2; ++i) {
      const float4 x = b[i];
      w[2 * i] = f2{x.x, x.y};
      w[2 * i + 1] = f2{x.z, x.w};
    }
  }
  static __device__ __forceinline__ void pstore(float4* b, const f2 (&w)[NMEP]) {
#pragma unroll
    for (int i = 0; i < NMEP / 2; ++i) b[i] = make_float4(w[2 * i].x, w[2 * i].y, w[2 * i + 1].x, w[2 * i + 1].y);
  }
  // variable groups of the filter's linear parts: pairs in packed FP32 (VG = f2), else single
  static constexpr int GW = PACK ? 2 : 1;
  static constexpr int NG = NV / GW;
  using VG = typename std::conditional<PACK, f2, T>::type;
  static __device__ __forceinline__ VG vzero() {
    if constexpr (PACK) return f2{0.f, 0.f};
    else return T(0);
  }
  template <int G>
  static __device__ __forceinline__ VG gslot(T* ws, int s, int m, int lane) {
    if constexpr (PACK) return f2{*slot_ptr(ws, s, 2 * G, m, lane), *slot_ptr(ws, s, 2 * G + 1, m, lane)};
    else return *slot_ptr(ws, s, G, m, lane);
  }
  template <int J>
  static __device__ __forceinline__ T comp(const VG& x) {
    if constexpr (PACK) return J == 0 ? x.x : x.y;
    else return x;
  }
  static __device__ __forceinline__ const Consts2D<T>& consts_of(const Stage2DArgs& a) {
    if constexpr (PR::MIXED) return a.cf;
    else return a.cd;
  }
  static __device__ __forceinline__ T shfl_down_t(T x, int d) { return __shfl_down_sync(0xffffffffu, x, d); }
  static __device__ __forceinline__ T shfl_up_t(T x, int d) { return __shfl_up_sync(0xffffffffu, x, d); }

  // ---- sum factorisation on the tensor-product modes (all coefficients are immediates) ----
  // Sums start at -0, the additive identity (-0 + x == x for every x), so their first add folds away.

  // f[g] = sum_{l=0..K} c[l] P_l(x_g) at the NQ Gauss nodes. P_l has the parity of l and the nodes
  // are symmetric, so f[g] = E(x_g) + O(x_g) and f[NQ-1-g] = E(x_g) - O(x_g) with E, O the even- and
  // odd-degree parts; the middle node of an odd rule sees only E.
  template <class VT>
  static __device__ __forceinline__ void gauss_values(const VT (&c)[K + 1], VT (&f)[NQ]) {
    using S = typename vtraits<VT>::S;
    sfor<NQ / 2>([&](auto G) {
      constexpr int g = decltype(G)::value;
      VT ev = c[0], od = vtraits<VT>::zero();
      sfor<K + 1>([&](auto L) {
        constexpr int l = decltype(L)::value;
        constexpr double w = TB::GP[l * NQ + g];
        if constexpr (l >= 1 && w != 0.0) {
          if constexpr ((l & 1) != 0) od = vmad(c[l], (S)w, od);
          else ev = vmad(c[l], (S)w, ev);
        }
      });
      f[g] = ev + od;
      f[NQ - 1 - g] = ev - od;
    });
    if constexpr ((NQ & 1) != 0) {
      VT ev = c[0];
      sfor<K + 1>([&](auto L) {
        constexpr int l = decltype(L)::value;
        constexpr double w = TB::GP[l * NQ + NQ / 2];
        if constexpr (l >= 2 && (l & 1) == 0 && w != 0.0) ev = vmad(c[l], (S)w, ev);
      });
      f[NQ / 2] = ev;
    }
  }

  // M[l] = sum_g w_g phi_l(x_g) F[g], l = 0..K, phi_l = P_l (DERIV = 0) or P_l' (DERIV = 1), from the
  // node-pair sums F[g] + F[NQ-1-g] (phi_l even) and differences (phi_l odd). M[0] = 0 for DERIV = 1.
  // HALF: the moments of F / 2 (the weights halved, which is exact), for the LLF fluxes formed as
  // twice their value.
  template <int DERIV, class VT, bool HALF = false>
  static __device__ __forceinline__ void gauss_moments(const VT (&F)[NQ], VT (&M)[K + 1]) {
    using S = typename vtraits<VT>::S;
    VT s[NQ / 2], d[NQ / 2];
#pragma unroll
    for (int g = 0; g < NQ / 2; ++g) {
      s[g] = F[g] + F[NQ - 1 - g];
      d[g] = F[g] - F[NQ - 1 - g];
    }
    sfor<K + 1>([&](auto L) {
      constexpr int l = decltype(L)::value;
      constexpr bool even = ((l + DERIV) & 1) == 0;
      VT acc = vtraits<VT>::zero();
      sfor<NQ / 2>([&](auto G) {
        constexpr int g = decltype(G)::value;
        constexpr double w = (DERIV ? TB::WD[l * NQ + g] : TB::WP[l * NQ + g]) * (HALF ? 0.5 : 1.0);
        if constexpr (w != 0.0) {
          if constexpr (even) acc = vmad(s[g], (S)w, acc);
          else acc = vmad(d[g], (S)w, acc);
        }
      });
      if constexpr ((NQ & 1) != 0 && even) {
        constexpr double w = (DERIV ? TB::WD[l * NQ + NQ / 2] : TB::WP[l * NQ + NQ / 2]) * (HALF ? 0.5 : 1.0);
        if constexpr (w != 0.0) acc = vmad(F[NQ / 2], (S)w, acc);
      }
      M[l] = acc;
    });
  }

  // Twice the LLF flux at one face point, f(uL) + f(uR) - alpha (uR - uL), alpha the larger spectral
  // radius, with the combination on pairs of variables (packed form): fh[vp] = 2 {fh_2vp, fh_2vp+1}.
  // The halving goes into the moments' weights (gauss_moments<.., true>); scaling by 2 commutes with
  // rounding, so the moments are bitwise those of the flux itself.
  template <int DIR>
  static __device__ __forceinline__ void llf_pairs(const T (&uL)[NV], const T (&uR)[NV], f2 (&fh)[NV / 2], T gam,
                                                   T gm1, T ax, T ay) {
    T fL[NV], fR[NV];
    flux2d<EQ, DIR>(uL, fL, gm1, ax, ay);
    flux2d<EQ, DIR>(uR, fR, gm1, ax, ay);
    const T na = -nan_max(speed2d<EQ, DIR>(uL, gam, gm1, ax, ay), speed2d<EQ, DIR>(uR, gam, gm1, ax, ay));
#pragma unroll
    for (int vp = 0; vp < NV / 2; ++vp) {
      const f2 sum = f2{fL[2 * vp], fL[2 * vp + 1]} + f2{fR[2 * vp], fR[2 * vp + 1]};
      const f2 dif = f2{uR[2 * vp], uR[2 * vp + 1]} - f2{uL[2 * vp], uL[2 * vp + 1]};
      fh[vp] = vfma(dif, f2{na, na}, sum);
    }
  }

  // Traces of u on the vertical edges xi = -1 (tl) and xi = +1 (tr) at the edge Gauss points:
  // collapse p with P_p(+-1) = (+-1)^p, then evaluate the q-expansions at the nodes.
  static __device__ __forceinline__ void edge_traces_v(const T (&u)[NV][NM], T (&tl)[NQ][NV], T (&tr)[NQ][NV]) {
    if constexpr (PACK_TRACES) {
      sfor<NV / 2>([&](auto VP) {
        constexpr int v0 = 2 * decltype(VP)::value, v1 = v0 + 1;
        f2 cl[K + 1], cr[K + 1];
        sfor<K + 1>([&](auto Q) {
          constexpr int q = decltype(Q)::value;
          f2 e{u[v0][TB::MIX[q]], u[v1][TB::MIX[q]]};
          vsum<f2> o;
          sfor<K + 1>([&](auto P) {
            constexpr int p = decltype(P)::value;
            constexpr int m = TB::MIX[p * (K + 1) + q];
            if constexpr (p >= 1 && m >= 0) {
              if constexpr ((p & 1) != 0) o.add(f2{u[v0][m], u[v1][m]});
              else e = e + f2{u[v0][m], u[v1][m]};
            }
          });
          if constexpr (TB::any_p_par(q, 1)) {
            cr[q] = e + o.get();
            cl[q] = e - o.get();
          } else {
            cr[q] = e;
            cl[q] = e;
          }
        });
        f2 fl[NQ], fr[NQ];
        gauss_values(cl, fl);
        gauss_values(cr, fr);
#pragma unroll
        for (int g = 0; g < NQ; ++g) {
          tl[g][v0] = fl[g].x;
          tl[g][v1] = fl[g].y;
          tr[g][v0] = fr[g].x;
          tr[g][v1] = fr[g].y;
        }
      });
      return;
    }
    sfor<NV>([&](auto V) {
      constexpr int v = decltype(V)::value;
      T cl[K + 1], cr[K + 1];
      sfor<K + 1>([&](auto Q) {
        constexpr int q = decltype(Q)::value;
        T e = u[v][TB::MIX[q]], o = T(-0.0);
        sfor<K + 1>([&](auto P) {
          constexpr int p = decltype(P)::value;
          constexpr int m = TB::MIX[p * (K + 1) + q];
          if constexpr (p >= 1 && m >= 0) {
            if constexpr ((p & 1) != 0) o += u[v][m];
            else e += u[v][m];
          }
        });
        if constexpr (TB::any_p_par(q, 1)) {
          cr[q] = e + o;
          cl[q] = e - o;
        } else {
          cr[q] = e;
          cl[q] = e;
        }
      });
      T fl[NQ], fr[NQ];
      gauss_values(cl, fl);
      gauss_values(cr, fr);
#pragma unroll
      for (int g = 0; g < NQ; ++g) {
        tl[g][v] = fl[g];
        tr[g][v] = fr[g];
      }
    });
  }

  // Traces of u on the horizontal edges eta = -1 (bot) and eta = +1 (top).
  static __device__ __forceinline__ void edge_traces_h(const T (&u)[NV][NM], T (&bot)[NQ][NV], T (&top)[NQ][NV]) {
    if constexpr (PACK_TRACES) {
      sfor<NV / 2>([&](auto VP) {
        constexpr int v0 = 2 * decltype(VP)::value, v1 = v0 + 1;
        f2 cb[K + 1], ct[K + 1];
        sfor<K + 1>([&](auto P) {
          constexpr int p = decltype(P)::value;
          f2 e{u[v0][TB::MIX[p * (K + 1)]], u[v1][TB::MIX[p * (K + 1)]]};
          vsum<f2> o;
          sfor<K + 1>([&](auto Q) {
            constexpr int q = decltype(Q)::value;
            constexpr int m = TB::MIX[p * (K + 1) + q];
            if constexpr (q >= 1 && m >= 0) {
              if constexpr ((q & 1) != 0) o.add(f2{u[v0][m], u[v1][m]});
              else e = e + f2{u[v0][m], u[v1][m]};
            }
          });
          if constexpr (TB::any_q_par(p, 1)) {
            ct[p] = e + o.get();
            cb[p] = e - o.get();
          } else {
            ct[p] = e;
            cb[p] = e;
          }
        });
        f2 fb[NQ], ft[NQ];
        gauss_values(cb, fb);
        gauss_values(ct, ft);
#pragma unroll
        for (int g = 0; g < NQ; ++g) {
          bot[g][v0] = fb[g].x;
          bot[g][v1] = fb[g].y;
          top[g][v0] = ft[g].x;
          top[g][v1] = ft[g].y;
        }
      });
      return;
    }
    sfor<NV>([&](auto V) {
      constexpr int v = decltype(V)::value;
      T cb[K + 1], ct[K + 1];
      sfor<K + 1>([&](auto P) {
        constexpr int p = decltype(P)::value;
        T e = u[v][TB::MIX[p * (K + 1)]], o = T(-0.0);
        sfor<K + 1>([&](auto Q) {
          constexpr int q = decltype(Q)::value;
          constexpr int m = TB::MIX[p * (K + 1) + q];
          if constexpr (q >= 1 && m >= 0) {
            if constexpr ((q & 1) != 0) o += u[v][m];
            else e += u[v][m];
          }
        });
        if constexpr (TB::any_q_par(p, 1)) {
          ct[p] = e + o;
          cb[p] = e - o;
        } else {
          ct[p] = e;
          cb[p] = e;
        }
      });
      T fb[NQ], ft[NQ];
      gauss_values(cb, fb);
      gauss_values(ct, ft);
#pragma unroll
      for (int g = 0; g < NQ; ++g) {
        bot[g][v] = fb[g];
        top[g][v] = ft[g];
      }
    });
  }

  // Volume integral (F(u), grad phi) of one cell, sum-factorised column by column of Gauss points:
  // for node x_a the q-coefficients C[q] = sum_p u[p,q] P_p(x_a) give the values at (x_a, y_b) for
  // all b; the fluxes there are reduced to the moments Gx[q] = sum_b w_b P_q(y_b) f^x and
  // Gy[q] = sum_b w_b P_q'(y_b) f^y, and acc[p,q] += w_a P_p'(x_a) sx Gx[q] + w_a P_p(x_a) sy Gy[q].
  static __device__ __forceinline__ void volume(const T (&u)[NV][NM], T (&acc)[NV][NM], T sx, T sy, T gm1,
                                                T ax, T ay) {
    sfor<NQ>([&](auto A) {
      constexpr int qa = decltype(A)::value;
      T FX[NV][NQ], FY[NV][NQ];
      {
        T uq[NV][NQ];
        if constexpr (PACK) {
          sfor<NV / 2>([&](auto VP) {
            constexpr int v0 = 2 * decltype(VP)::value, v1 = v0 + 1;
            f2 c[K + 1];
            sfor<K + 1>([&](auto Q) {
              constexpr int q = decltype(Q)::value;
              f2 s{u[v0][TB::MIX[q]], u[v1][TB::MIX[q]]};
              sfor<K + 1>([&](auto P) {
                constexpr int p = decltype(P)::value;
                constexpr int m = TB::MIX[p * (K + 1) + q];
                constexpr double w = TB::GP[p * NQ + qa];
                if constexpr (p >= 1 && m >= 0 && w != 0.0) s = vmad(f2{u[v0][m], u[v1][m]}, (T)w, s);
              });
              c[q] = s;
            });
            f2 f[NQ];
            gauss_values(c, f);
#pragma unroll
            for (int g = 0; g < NQ; ++g) {
              uq[v0][g] = f[g].x;
              uq[v1][g] = f[g].y;
            }
          });
        } else {
          sfor<NV>([&](auto V) {
            constexpr int v = decltype(V)::value;
            T c[K + 1];
            sfor<K + 1>([&](auto Q) {
              constexpr int q = decltype(Q)::value;
              T s = u[v][TB::MIX[q]];
              sfor<K + 1>([&](auto P) {
                constexpr int p = decltype(P)::value;
                constexpr int m = TB::MIX[p * (K + 1) + q];
                constexpr double w = TB::GP[p * NQ + qa];
                if constexpr (p >= 1 && m >= 0 && w != 0.0) s += u[v][m] * (T)w;
              });
              c[q] = s;
            });
            gauss_values(c, uq[v]);
          });
        }
#pragma unroll
        for (int qb = 0; qb < NQ; ++qb) {
          T w[NV], fx[NV], fy[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) w[v] = uq[v][qb];
          flux2d_xy<EQ>(w, fx, fy, gm1, ax, ay);
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            FX[v][qb] = fx[v];
            FY[v][qb] = fy[v];
          }
        }
      }
      if constexpr (PACK) {
        sfor<NV / 2>([&](auto VP) {
          constexpr int v0 = 2 * decltype(VP)::value, v1 = v0 + 1;
          f2 fx[NQ], fy[NQ], gx[K + 1], gy[K + 1];
#pragma unroll
          for (int g = 0; g < NQ; ++g) {
            fx[g] = f2{FX[v0][g], FX[v1][g]};
            fy[g] = f2{FY[v0][g], FY[v1][g]};
          }
          gauss_moments<0>(fx, gx);
          gauss_moments<1>(fy, gy);
#pragma unroll
          for (int q = 0; q <= K; ++q) {
            gx[q] = vscale(gx[q], sx);
            gy[q] = vscale(gy[q], sy);
          }
          sfor<NM>([&](auto Mi) {
            constexpr int m = decltype(Mi)::value;
            constexpr int p = TB::PP[m], q = TB::QQ[m];
            constexpr double kx = TB::WD[p * NQ + qa], ky = TB::WP[p * NQ + qa];
            f2 a{acc[v0][m], acc[v1][m]};
            if constexpr (kx != 0.0) a = vmad(gx[q], (T)kx, a);
            if constexpr (q >= 1 && ky != 0.0) a = vmad(gy[q], (T)ky, a);
            acc[v0][m] = a.x;
            acc[v1][m] = a.y;
          });
        });
      } else {
        sfor<NV>([&](auto V) {
          constexpr int v = decltype(V)::value;
          T gx[K + 1], gy[K + 1];
          gauss_moments<0>(FX[v], gx);
          gauss_moments<1>(FY[v], gy);
#pragma unroll
          for (int q = 0; q <= K; ++q) {
            gx[q] *= sx;
            gy[q] *= sy;
          }
          sfor<NM>([&](auto Mi) {
            constexpr int m = decltype(Mi)::value;
            constexpr int p = TB::PP[m], q = TB::QQ[m];
            constexpr double kx = TB::WD[p * NQ + qa], ky = TB::WP[p * NQ + qa];
            if constexpr (kx != 0.0) acc[v][m] += (T)kx * gx[q];
            if constexpr (q >= 1 && ky != 0.0) acc[v][m] += (T)ky * gy[q];
          });
        });
      }
    });
  }

  // ---- the filter's jumps, edge by edge ----
  // Across an edge the jump of d^(a1,a2) u at the edge's two corners is a derivative of a jump
  // polynomial along the edge. For a vertical edge (between this cell and its right neighbour) and
  // normal order a1: W[q] = sum_p (w_R[p,q] P_p^{(a1)}(-1) - w[p,q] P_p^{(a1)}(+1)), a polynomial
  // in eta with Legendre coefficients W[q]; its a2-th eta-derivative at eta = -1, +1 is the jump of
  // d^(a1,a2) at the two corners (the reference scaling (2/h_x)^a1 (2/h_y)^a2 is the positive
  // factor f applied with the absolute values). P_l^{(r)}(-1) = (-1)^{l+r} P_l^{(r)}(+1), so each
  // end sum is formed once from its even- and odd-degree parts. Horizontal edges are the same with
  // the roles of (p, xi) and (q, eta) exchanged.

  // Compile-time structure: the end sum over p of order a1 at fixed q has terms of parity par.
  static constexpr bool xe(int a1, int q, int par) {
    for (int pp = a1; pp <= K; ++pp)
      if ((pp & 1) == par && TB::has(pp, q) && TB::DE[pp * (K + 1) + a1] != 0.0) return true;
    return false;
  }
  static constexpr bool ye(int a2, int pp, int par) { return TB::hq(pp, a2, par); }
  // the jump polynomial coefficient of order a1 (x-normal) / a2 (y-normal) exists
  static constexpr bool xw(int a1, int q) { return xe(a1, q, 0) || xe(a1, q, 1); }
  static constexpr bool yw(int a2, int pp) { return ye(a2, pp, 0) || ye(a2, pp, 1); }
  // its tangential derivative of order r at +-1 has terms of parity par (over the coefficient index)
  static constexpr bool xt(int a1, int r, int par) {
    for (int q = r; q <= K; ++q)
      if ((q & 1) == par && xw(a1, q) && TB::DE[q * (K + 1) + r] != 0.0) return true;
    return false;
  }
  static constexpr bool yt(int a2, int r, int par) {
    for (int pp = r; pp <= K; ++pp)
      if ((pp & 1) == par && yw(a2, pp) && TB::DE[pp * (K + 1) + r] != 0.0) return true;
    return false;
  }

  // The end sums of one cell (or a pair of variables, VT = f2) along x: at xi = +1 (xp) and -1 (xm)
  // for order a1 and coefficient q of the eta-expansion.
  template <int A1, int Q, class VT>
  static __device__ __forceinline__ void x_end(const VT (&w)[NM], VT& xp, VT& xm) {
    using S = typename vtraits<VT>::S;
    constexpr bool he = xe(A1, Q, 0), ho = xe(A1, Q, 1);
    VT ev = vtraits<VT>::zero(), od = vtraits<VT>::zero();
    sfor<K + 1>([&](auto P) {
      constexpr int pp = decltype(P)::value;
      constexpr int m = TB::MIX[pp * (K + 1) + Q];
      constexpr double c = TB::DE[pp * (K + 1) + A1];
      if constexpr (pp >= A1 && m >= 0 && c != 0.0) {
        if constexpr ((pp & 1) != 0) od = vmad(w[m], (S)c, od);
        else ev = vmad(w[m], (S)c, ev);
      }
    });
    if constexpr (he && ho) {
      xp = ev + od;
      xm = (A1 & 1) ? od - ev : ev - od;
    } else if constexpr (he) {
      xp = ev;
      xm = (A1 & 1) ? -ev : ev;
    } else {
      xp = od;
      xm = (A1 & 1) ? od : -od;
    }
  }
  // along y: at eta = +1 (yp) and -1 (ym) for order a2 and coefficient p of the xi-expansion
  template <int A2, int PD, class VT>
  static __device__ __forceinline__ void y_end(const VT (&w)[NM], VT& yp, VT& ym) {
    using S = typename vtraits<VT>::S;
    constexpr bool he = ye(A2, PD, 0), ho = ye(A2, PD, 1);
    VT ev = vtraits<VT>::zero(), od = vtraits<VT>::zero();
    sfor<K + 1>([&](auto Q) {
      constexpr int q = decltype(Q)::value;
      constexpr int m = TB::MIX[PD * (K + 1) + q];
      constexpr double c = TB::DE[q * (K + 1) + A2];
      if constexpr (q >= A2 && m >= 0 && c != 0.0) {
        if constexpr ((q & 1) != 0) od = vmad(w[m], (S)c, od);
        else ev = vmad(w[m], (S)c, ev);
      }
    });
    if constexpr (he && ho) {
      yp = ev + od;
      ym = (A2 & 1) ? od - ev : ev - od;
    } else if constexpr (he) {
      yp = ev;
      ym = (A2 & 1) ? -ev : ev;
    } else {
      yp = od;
      ym = (A2 & 1) ? od : -od;
    }
  }

  // |value at +1| + |value at -1| of the R-th derivative of the jump polynomial with coefficients
  // c[0..K] of normal order NO across an x-edge (DIR = 0) or a y-edge (DIR = 1), times f, into acc.
  template <int DIR, int NO, int R, class VT>
  static __device__ __forceinline__ void corner_pair(const VT (&c)[K + 1], typename vtraits<VT>::S f,
                                                     typename vtraits<VT>::S f2x, VT& acc) {
    using S = typename vtraits<VT>::S;
    constexpr bool HE = DIR == 0 ? xt(NO, R, 0) : yt(NO, R, 0);
    constexpr bool HO = DIR == 0 ? xt(NO, R, 1) : yt(NO, R, 1);
    VT ev = vtraits<VT>::zero(), od = vtraits<VT>::zero();
    sfor<K + 1>([&](auto Q) {
      constexpr int q = decltype(Q)::value;
      constexpr double d = TB::DE[q * (K + 1) + R];
      constexpr bool present = DIR == 0 ? xw(NO, q) : yw(NO, q);
      if constexpr (q >= R && d != 0.0 && present) {
        if constexpr ((q & 1) != 0) od = vmad(c[q], (S)d, od);
        else ev = vmad(c[q], (S)d, ev);
      }
    });
    if constexpr (HE && HO) {
      // |e + o| + |e - o| = 2 max(|e|, |o|): the two corners' magnitudes without forming them
      // (2048^2 Q2 FP32 form: -2.5 % per stage launch)
      acc = vmad(vmaxabs(ev, od), f2x, acc);
    } else if constexpr (HE) {
      acc = vmad(vabs(ev), f2x, acc);        // the same magnitude at both corners
    } else if constexpr (HO) {
      acc = vmad(vabs(od), f2x, acc);
    }
  }

  // Right vertical edge of the cell w: per total order m, sum over |alpha| = m of
  // f_alpha (|jump at the bottom corner| + |jump at the top corner|) into sv[m].
  template <class VT>
  static __device__ __forceinline__ void vertical_jumps(const VT (&w)[NM], VT (&sv)[LMAX + 1], const T* pxy,
                                                        const T* pxy2) {
    sfor<K + 1>([&](auto A1_) {
      constexpr int a1 = decltype(A1_)::value;
      VT W[K + 1];
      sfor<K + 1>([&](auto Q) {
        constexpr int q = decltype(Q)::value;
        if constexpr (xw(a1, q)) {
          VT xp, xm;
          x_end<a1, q>(w, xp, xm);
          W[q] = shfl_down_v(xm, 1) - xp;           // the right neighbour's end minus this cell's
        }
      });
      sfor<K + 1>([&](auto A2_) {
        constexpr int a2 = decltype(A2_)::value;
        if constexpr (TB::alpha_ok(a1, a2) && (xt(a1, a2, 0) || xt(a1, a2, 1)))
          corner_pair<0, a1, a2>(W, pxy[a1 * 4 + a2], pxy2[a1 * 4 + a2], sv[a1 + a2]);
      });
    });
  }

  // The horizontal edge between the cell below (wb, its top) and the cell above (wa, its bottom).
  template <class VT>
  static __device__ __forceinline__ void horizontal_jumps(const VT (&wa)[NM], const VT (&wb)[NM], VT (&sh)[LMAX + 1],
                                                          const T* pxy, const T* pxy2) {
    sfor<K + 1>([&](auto A2_) {
      constexpr int a2 = decltype(A2_)::value;
      VT V[K + 1];
      sfor<K + 1>([&](auto P) {
        constexpr int pp = decltype(P)::value;
        if constexpr (yw(a2, pp)) {
          VT ap, am, bp, bm;
          y_end<a2, pp>(wa, ap, am);
          y_end<a2, pp>(wb, bp, bm);
          V[pp] = am - bp;                          // above at eta = -1 minus below at eta = +1
        }
      });
      sfor<K + 1>([&](auto A1_) {
        constexpr int a1 = decltype(A1_)::value;
        if constexpr (TB::alpha_ok(a1, a2) && (yt(a2, a1, 0) || yt(a2, a1, 1)))
          corner_pair<1, a2, a1>(V, pxy[a1 * 4 + a2], pxy2[a1 * 4 + a2], sh[a1 + a2]);
      });
    });
  }

  // One tile item: strip `strip` (28 output columns) and row chunk `chunk` of one instance, with step
  // size dtd. ws: this warp's row slots and Q area in shared memory. The output cells' max CFL rate
  // and physicality are folded into my_rate (FP64 form) / my_rate_t (FP32 form) and my_ok.
  static __device__ void item(const Stage2DArgs& a, double dtd, int strip, int chunk, T* ws,
                              double& my_rate, T& my_rate_t, bool& my_ok) {
    constexpr carr<int, NM> PP = TB::PP;
    constexpr carr<int, NM> QQ = TB::QQ;
    constexpr carr<double, NM> MINV = TB::MINV;

    const T dt = (T)dtd;
    const int lane = threadIdx.x & 31;
    T* wq = ws + SLOT_WORDS;                                      // Q[v][l-1] of the next row to filter
    T* weta = wq + NV * LMAX * 32;                                // hybrid: eta of the next row, partial
    T my_eta = T(0);
    const int nx = a.nx, ny = a.ny;
    // mesh and physics constants from the kernel parameters (stage2d_consts)
    const Consts2D<T>& KC = consts_of(a);
    const T gam = KC.gam, gm1 = KC.gm1, ax = KC.ax, ay = KC.ay;
    const double ihx = 1.0 / a.hx, ihy = 1.0 / a.hy, c1dt = a.c1 * dtd;
    const T inv_hx = KC.ihx, inv_hy = KC.ihy;
    // u~ = u + c0 (u^n - u) + c1 dt R: the edge and volume integrals enter through c1 dt / h
    const T sx = (T)(c1dt * ihx), sy = (T)(c1dt * ihy), c0 = (T)a.c0;
    // double-float coefficients of the cell-average update (computed once, off the cell loop)
    const df dfx = df_from_double(0.5 * c1dt * ihx);
    const df dfy = df_from_double(0.5 * c1dt * ihy);
    const df dfc0 = df_from_double(a.c0);
    // powers of 2/h for physical derivatives; weights of the m-th derivative jumps (with the 1/2 of
    // the trapezoidal rule over an edge's two corners): the jump filter's m(m+1) h^m, or the OEDG
    // form's (2m+1)/m! h^m, each direction divided by its own h (Section 2.1's form)
    const T* px = KC.px;
    const T* py = KC.py;
    const T* wx = KC.wx;
    const T* wy = KC.wy;
    // OEDG reductions of this lane's output cells: sum of the averages, largest / smallest value at
    // the volume Gauss points, per variable
    constexpr int NVO = OE ? NV : 1;
    double osum[NVO];
    T omax[NVO], omin[NVO];
#pragma unroll
    for (int v = 0; v < NVO; ++v) {
      osum[v] = 0.0;
      omax[v] = -INFINITY;
      omin[v] = INFINITY;
    }
    {
      const int x = strip * STRIP_OUT - 2 + lane;
      const bool perx = a.bcx == BC_PERIODIC, pery = a.bcy == BC_PERIODIC;
      const int xc = perx ? ((x % nx) + nx) % nx : (x < 0 ? 0 : (x >= nx ? nx - 1 : x));
      // outflow: columns and rows outside the mesh are ghost cells holding the constant state equal
      // to the adjacent interior cell's average (stage input for the fluxes, u~ for the jumps)
      const bool gcol = !perx && (x < 0 || x >= nx);
      const int xw = strip * STRIP_OUT - 2;                     // column of lane 0
      const bool edge_strip = !perx && (xw < 0 || xw + 31 >= nx);
      const bool out_lane = lane >= 2 && lane < 2 + STRIP_OUT && x >= 0 && x < nx;
      const int yb = chunk * a.H;
      const int ye = min(yb + a.H, ny);

      T topPrev[NQ][NV];
#pragma unroll
      for (int g = 0; g < NQ; ++g)
#pragma unroll
        for (int v = 0; v < NV; ++v) topPrev[g][v] = T(0);
      // cell-average quantities of the row filtered next (row t-2 at iteration t)
      T bx2 = T(0), by2 = T(0), invH2 = T(0);
      bool phys2 = true;

      // row slots of rows t, t-1, t-2, rotated once per row (row r in slot r mod 3)
      int sl0 = slot_of(yb - 2), sl1 = slot_of(yb - 3), sl2 = slot_of(yb - 4);
#pragma unroll 1
      for (int t = yb - 2; t <= ye + 1; ++t) {
        const bool grow = !pery && (t < 0 || t >= ny);
        const int ty = pery ? wrap_near(t, ny) : (t < 0 ? 0 : (t >= ny ? ny - 1 : t));
        const long long cell = (long long)ty * nx + xc;
        T u[NV][NM], lo0[NV];
        ST::load(a.uin, a.ncell, cell, u, lo0);
        if constexpr (ST::PAIRED) {
          // the next row of the stage input, and this row of u^n (read after the volume integral)
          const int tn = t + 1;
          const int tyn = pery ? (ty + 1 >= ny ? ty + 1 - ny : ty + 1) : (tn < 0 ? 0 : (tn >= ny ? ny - 1 : tn));
          ST::prefetch(a.uin, a.ncell, (long long)tyn * nx + xc);
          if (a.stage > 0) ST::prefetch(a.un, a.ncell, cell);
        }
        if (grow || gcol) {
#pragma unroll
          for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int m = 1; m < NM; ++m) u[v][m] = T(0);
        }

        // ---- horizontal face between rows t-1 and t (once per column) ----
        // Mh[v][p] = sum_g w_g P_p(x_g) F^_v(x_g): the face's flux moments, used by both rows
        T Mh[NV][K + 1];
        {
          T bot[NQ][NV], top[NQ][NV];
          edge_traces_h(u, bot, top);
          if (PACK || t >= yb - 1) {   // (packed form: unguarded, see the filter)
            if constexpr (PACK) {
              f2 Fh2[NQ][NV / 2];
#pragma unroll
              for (int g = 0; g < NQ; ++g) llf_pairs<1>(topPrev[g], bot[g], Fh2[g], gam, gm1, ax, ay);
#pragma unroll
              for (int vp = 0; vp < NV / 2; ++vp) {
                f2 F[NQ], M[K + 1];
#pragma unroll
                for (int g = 0; g < NQ; ++g) F[g] = Fh2[g][vp];
                gauss_moments<0, f2, true>(F, M);
#pragma unroll
                for (int p = 0; p <= K; ++p) {
                  Mh[2 * vp][p] = M[p].x;
                  Mh[2 * vp + 1][p] = M[p].y;
                }
              }
            } else {
              T Fh[NQ][NV];
#pragma unroll
              for (int g = 0; g < NQ; ++g) llf2d<EQ, 1>(topPrev[g], bot[g], Fh[g], gam, gm1, ax, ay);
#pragma unroll
              for (int v = 0; v < NV; ++v) {
                T F[NQ];
#pragma unroll
                for (int g = 0; g < NQ; ++g) F[g] = Fh[g][v];
                gauss_moments<0>(F, Mh[v]);
              }
            }
            // finalise u~ of row t-1 with its top-face term (P_q(+1) = 1)
            if (PACK || (t - 1 >= yb - 1 && t - 1 <= ye)) {
              const int s = sl1;
#pragma unroll
              for (int v = 0; v < NV; ++v) {
                if constexpr (PR::MIXED && !PACK) {
                  df_acc acc0{*slot_ptr(ws, s, v, 0, lane), *slot_ptr(ws, s, v, NM, lane)};
                  acc0.add_prod(dfy, -Mh[v][0]);
                  const df r0 = acc0.result();
                  *slot_ptr(ws, s, v, 0, lane) = r0.hi;
                  *slot_ptr(ws, s, v, NM, lane) = r0.lo;
                }
                if constexpr (!PACK) {
                  T ms[K + 1];
#pragma unroll
                  for (int p = 0; p <= K; ++p) ms[p] = sy * Mh[v][p];
#pragma unroll
                  for (int m = PR::MIXED ? 1 : 0; m < NM; ++m)
                    *slot_ptr(ws, s, v, m, lane) -= (T)MINV[m] * ms[PP[m]];
                }
              }
              if constexpr (PACK) {
#pragma unroll
                for (int vp = 0; vp < NV / 2; ++vp) {
                  const int v0 = 2 * vp, v1 = v0 + 1;
                  f2 blk[NMEP];
                  pload(pblock(ws, s, vp, lane), blk);
                  if constexpr (PACK_DF) {
                    df2_acc acc0{blk[0], blk[NM]};
                    acc0.add_prod(dfy, -f2{Mh[v0][0], Mh[v1][0]});
                    const df2 r0 = acc0.result();
                    blk[0] = r0.hi;
                    blk[NM] = r0.lo;
                  } else {
                    // the scalar double-float update of each of the two averages
                    df_acc a0{blk[0].x, blk[NM].x}, a1{blk[0].y, blk[NM].y};
                    a0.add_prod(dfy, -Mh[v0][0]);
                    a1.add_prod(dfy, -Mh[v1][0]);
                    const df r0 = a0.result(), r1 = a1.result();
                    blk[0] = f2{r0.hi, r1.hi};
                    blk[NM] = f2{r0.lo, r1.lo};
                  }
                  f2 ms[K + 1];
#pragma unroll
                  for (int p = 0; p <= K; ++p) ms[p] = vscale(f2{Mh[v0][p], Mh[v1][p]}, sy);
#pragma unroll
                  for (int m = 1; m < NM; ++m) blk[m] = vmad(ms[PP[m]], -(T)MINV[m], blk[m]);
                  pstore(pblock(ws, s, vp, lane), blk);
                }
              }
            }
          }
#pragma unroll
          for (int g = 0; g < NQ; ++g)
#pragma unroll
            for (int v = 0; v < NV; ++v) topPrev[g][v] = top[g][v];
        }

        // ---- partial u~ of row t: bottom face, vertical faces, volume, RK combination ----
        if (t >= yb - 1 && t <= ye) {
          // vertical faces: F^ at xi = +1 by this lane, the one at xi = -1 from the left lane
          T MR[NV][K + 1], ML[NV][K + 1];
          {
            T tl[NQ][NV], tr[NQ][NV];
            edge_traces_v(u, tl, tr);
            if constexpr (PACK) {
              f2 FR2[NQ][NV / 2], FL2[NQ][NV / 2];
#pragma unroll
              for (int g = 0; g < NQ; ++g) {
                T nb[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) nb[v] = shfl_down_t(tl[g][v], 1);
                llf_pairs<0>(tr[g], nb, FR2[g], gam, gm1, ax, ay);
#pragma unroll
                for (int vp = 0; vp < NV / 2; ++vp) FL2[g][vp] = shfl_up_v(FR2[g][vp], 1);
              }
#pragma unroll
              for (int vp = 0; vp < NV / 2; ++vp) {
                const int v0 = 2 * vp, v1 = v0 + 1;
                f2 FRv[NQ], FLv[NQ], MRp[K + 1], MLp[K + 1];
#pragma unroll
                for (int g = 0; g < NQ; ++g) {
                  FRv[g] = FR2[g][vp];
                  FLv[g] = FL2[g][vp];
                }
                gauss_moments<0, f2, true>(FRv, MRp);
                gauss_moments<0, f2, true>(FLv, MLp);
#pragma unroll
                for (int p = 0; p <= K; ++p) {
                  MR[v0][p] = MRp[p].x;
                  MR[v1][p] = MRp[p].y;
                  ML[v0][p] = MLp[p].x;
                  ML[v1][p] = MLp[p].y;
                }
              }
            } else {
              T FR[NQ][NV], FL[NQ][NV];
#pragma unroll
              for (int g = 0; g < NQ; ++g) {
                T nb[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) nb[v] = shfl_down_t(tl[g][v], 1);
                llf2d<EQ, 0>(tr[g], nb, FR[g], gam, gm1, ax, ay);
#pragma unroll
                for (int v = 0; v < NV; ++v) FL[g][v] = shfl_up_t(FR[g][v], 1);
              }
#pragma unroll
              for (int v = 0; v < NV; ++v) {
                T FRv[NQ], FLv[NQ];
#pragma unroll
                for (int g = 0; g < NQ; ++g) {
                  FRv[g] = FR[g][v];
                  FLv[g] = FL[g][v];
                }
                gauss_moments<0>(FRv, MR[v]);
                gauss_moments<0>(FLv, ML[v]);
              }
            }
          }
          // edge terms: acc[p,q] = sy (-1)^q Mh[p] - sx (MR[q] - (-1)^p ML[q])
          T acc[NV][NM];
          if constexpr (PACK) {
#pragma unroll
            for (int vp = 0; vp < NV / 2; ++vp) {
              const int v0 = 2 * vp, v1 = v0 + 1;
              f2 mh[K + 1], dq[K + 1], sq[K + 1];
#pragma unroll
              for (int i = 0; i <= K; ++i) {
                const f2 l2{ML[v0][i], ML[v1][i]}, r2{MR[v0][i], MR[v1][i]};
                mh[i] = vscale(f2{Mh[v0][i], Mh[v1][i]}, sy);
                dq[i] = vscale(l2 - r2, sx);
                sq[i] = vscale(l2 + r2, -sx);
              }
#pragma unroll
              for (int m = 0; m < NM; ++m) {
                const f2 e = (PP[m] & 1) ? sq[QQ[m]] : dq[QQ[m]];
                const f2 r = (QQ[m] & 1) ? e - mh[PP[m]] : mh[PP[m]] + e;
                acc[v0][m] = r.x;
                acc[v1][m] = r.y;
              }
            }
          } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              T mh[K + 1], dq[K + 1], sq[K + 1];
#pragma unroll
              for (int i = 0; i <= K; ++i) {
                mh[i] = sy * Mh[v][i];
                dq[i] = sx * (ML[v][i] - MR[v][i]);
                sq[i] = -sx * (ML[v][i] + MR[v][i]);
              }
#pragma unroll
              for (int m = 0; m < NM; ++m) {
                const T hb = (QQ[m] & 1) ? -mh[PP[m]] : mh[PP[m]];
                acc[v][m] = hb + ((PP[m] & 1) ? sq[QQ[m]] : dq[QQ[m]]);
              }
            }
          }
          volume(u, acc, sx, sy, gm1, ax, ay);

          const int s = sl0;
          T un_[NV][NM], unlo[NV];
          if (a.stage > 0) ST::load(a.un, a.ncell, cell, un_, unlo);
          // cell average in double-float from the edge integrals, each formed once per edge:
          // u0 + c0 (un0 - u0) + c1 dt/(2h) (Phi_L - Phi_R + Phi_B [- Phi_T at the next row])
          auto df_average = [&](auto v) -> df {          // (instantiated by the FP32 form only)
            df_acc m0{u[v][0], lo0[v]};
            if (a.stage > 0) {
              df_acc d{un_[v][0], unlo[v]};
              d.add(df{-u[v][0], -lo0[v]});
              const df dd = d.result();
              m0.add(df_mul(dfc0, dd));
            }
            m0.add_prod(dfx, ML[v][0]);
            m0.add_prod(dfx, -MR[v][0]);
            m0.add_prod(dfy, Mh[v][0]);
            return m0.result();
          };
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            if constexpr (PR::MIXED && !PACK) {
              const df r0 = df_average(v);
              *slot_ptr(ws, s, v, 0, lane) = r0.hi;
              *slot_ptr(ws, s, v, NM, lane) = r0.lo;
            }
            if constexpr (!PACK) {
#pragma unroll
              for (int m = PR::MIXED ? 1 : 0; m < NM; ++m) {
                // u + c0 (u^n - u) + c1 dt R  (= c0 u^n + c1 (u + dt R) with c0 + c1 = 1 kept exact)
                T val = u[v][m];
                if (a.stage > 0) val += c0 * (un_[v][m] - u[v][m]);
                val += (T)MINV[m] * acc[v][m];
                *slot_ptr(ws, s, v, m, lane) = val;
              }
            }
          }
          if constexpr (PACK) {
#pragma unroll
            for (int vp = 0; vp < NV / 2; ++vp) {
              const int v0 = 2 * vp, v1 = v0 + 1;
              f2 blk[NMEP];
              if constexpr (PACK_DF) {
                // the double-float cell averages of the scalar branch, two variables per pair
                const f2 uh{u[v0][0], u[v1][0]}, ul{lo0[v0], lo0[v1]};
                df2_acc m0{uh, ul};
                if (a.stage > 0) {
                  df2_acc d{f2{un_[v0][0], un_[v1][0]}, f2{unlo[v0], unlo[v1]}};
                  d.add(df2{-uh, -ul});
                  m0.add(df2_mul(dfc0, d.result()));
                }
                m0.add_prod(dfx, f2{ML[v0][0], ML[v1][0]});
                m0.add_prod(dfx, -f2{MR[v0][0], MR[v1][0]});
                m0.add_prod(dfy, f2{Mh[v0][0], Mh[v1][0]});
                const df2 r0 = m0.result();
                blk[0] = r0.hi;
                blk[NM] = r0.lo;
              } else {
                const df r0 = df_average(v0), r1 = df_average(v1);
                blk[0] = f2{r0.hi, r1.hi};
                blk[NM] = f2{r0.lo, r1.lo};
              }
#pragma unroll
              for (int m = 1; m < NM; ++m) {
                f2 val{u[v0][m], u[v1][m]};
                if (a.stage > 0) val = vmad(f2{un_[v0][m], un_[v1][m]} - val, c0, val);
                blk[m] = vmad(f2{acc[v0][m], acc[v1][m]}, (T)MINV[m], val);
              }
#pragma unroll
              for (int m = NM + 1; m < NMEP; ++m) blk[m] = f2{0.f, 0.f};
              pstore(pblock(ws, s, vp, lane), blk);
            }
          }
        }

        // ---- jumps of u~; the filter of row t-2 ----
        // Row t-1 is final. Its vertical-face jumps and the jump of the face (t-2 | t-1) give, per
        // variable v and total degree l, Q_v(l) = beta^x AV_v(l) + beta^y SH_v(l) for row t-1 (kept
        // in shared memory until its top face is known) and the top-face term of row t-2.
        const bool r1 = (t - 1 >= yb - 1 && t - 1 <= ye);
        const bool g1 = !pery && (t - 1 < 0 || t - 1 >= ny);   // row t-1 is a ghost row
        const bool g2 = !pery && (t - 2 < 0 || t - 2 >= ny);
        const bool filt_row = (t - 2 >= yb && t - 2 < ye);
        const bool need_v = (t - 1 >= yb && t - 1 < ye);      // row t-1 is filtered next iteration
        T bx1 = T(0), by1 = T(0), invH1 = T(0);
        bool phys1 = true;
        if (PACK || r1) {
          T ub[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            if constexpr (PACK) {
              if ((v & 1) == 0) {
                const float4 x = pblock(ws, sl1, v / 2, lane)[0];   // {v, v+1} of mode 0 (and 1)
                ub[v] = x.x;
                ub[v + 1] = x.y;
              }
            } else {
              ub[v] = *slot_ptr(ws, sl1, v, 0, lane);
            }
          }
          avg_params<EQ, 2>(ub, gam, gm1, ax, ay, bx1, by1, invH1, phys1);
        }
        const int ty2 = t - 2;   // used only while row t-2 is filtered, a row of the chunk
        const long long cell2 = (long long)ty2 * nx + xc;       // the cell filtered in this iteration
        T sig[LMAX + 1];
#pragma unroll
        for (int l = 0; l <= LMAX; ++l) sig[l] = T(0);
        T eta2 = T(0);                                            // hybrid: eta of row t-2
        if (a.filter_on && (PACK || need_v || filt_row)) {
          T eta_v = T(0), eta_h = T(0);
          const int s1 = sl1, s2 = sl2;
          // groups of variables (pairs in packed FP32, else one variable): the jumps are linear in
          // the modes, each group's chain is the scalar chain of every variable in it
          sfor<NG>([&](auto G_) {
            constexpr int g = decltype(G_)::value;
            const VG z = vzero();
            VG w1[NM], w2[NM];
            if constexpr (PACK) {
              f2 b1[NMEP], b2[NMEP];
              pload(pblock(ws, s1, g, lane), b1);
              pload(pblock(ws, s2, g, lane), b2);
#pragma unroll
              for (int m = 0; m < NM; ++m) {
                w1[m] = b1[m];
                w2[m] = b2[m];
              }
            } else {
#pragma unroll
              for (int m = 0; m < NM; ++m) {
                w1[m] = gslot<g>(ws, s1, m, lane);
                w2[m] = gslot<g>(ws, s2, m, lane);
              }
            }
            // ghost rows and columns: the constant state of the adjacent interior cell's u~ average
            if (g1) {
              w1[0] = w2[0];
#pragma unroll
              for (int m = 1; m < NM; ++m) w1[m] = z;
            }
            if (g2) {
              w2[0] = w1[0];
#pragma unroll
              for (int m = 1; m < NM; ++m) w2[m] = z;
            }
            if (edge_strip) {                                   // warp-uniform: a strip at an outflow side
              const VG v_r = shfl_down_v(w1[0], 1), v_l = shfl_up_v(w1[0], 1);
              const VG w_r = shfl_down_v(w2[0], 1), w_l = shfl_up_v(w2[0], 1);
              if (gcol) {
                w1[0] = x < 0 ? v_r : v_l;
                w2[0] = x < 0 ? w_r : w_l;
#pragma unroll
                for (int m = 1; m < NM; ++m) w1[m] = w2[m] = z;
              }
            }
            // per total order m: sum over |alpha| = m of the scaled corner jumps, the right vertical
            // edge of row t-1 (sv) and the face (t-2 | t-1) (sh)
            VG sv[LMAX + 1], sh[LMAX + 1];
#pragma unroll
            for (int l = 0; l <= LMAX; ++l) sv[l] = sh[l] = z;
            // In the packed form the row's filter work runs unguarded: the conditions are uniform,
            // a row that is not filtered next only wastes work on values nobody reads, and the
            // straight code schedules better (2048^2 Q2: 0.555 -> 0.505 ms per stage launch; the
            // horizontal face, the top-face update of row t-1 and its average parameters likewise,
            // whose guards fail only in the first iteration: -> 0.482 ms. Those writes go to a row
            // slot that the partial stage value of row yb overwrites before it is read. Unguarding
            // the partial stage value itself as well was slower, 0.497 ms)
            if (PACK || need_v) vertical_jumps(w1, sv, KC.pxy, KC.pxy2);
            horizontal_jumps(w1, w2, sh, KC.pxy, KC.pxy2);
            VG av = z, shc = z;
#pragma unroll
            for (int l = 0; l <= LMAX; ++l) {
              shc = vmad(sh[l], wy[l], shc);
              if (PACK || need_v) av = vmad(shfl_up_v(sv[l], 1) + sv[l], wx[l], av);
              if (l == 0) {
                // density: edge-averaged value jumps, J^V / (2 h_x) and the face (t-2 | t-1) / (2 h_y)
                if ((LIM && a.hybrid) && g == 0) {
                  eta_v = comp<0>(av) * T(0.5) * inv_hx;
                  eta_h = comp<0>(shc) * T(0.5) * inv_hy;
                }
                continue;
              }
              if constexpr (PACK && !OE) {
                // Q of the pair's two variables in one 64-bit word per lane
                f2* q2 = (f2*)wq + ((g * LMAX + (l - 1)) << 5) + lane;
                // Q of row t-2 + its top face (sig is read only when row t-2 is filtered), then Q of
                // row t-1 (rows are visited in order, so the Q read here is the one written for
                // row t-2 in the previous iteration)
                const f2 x = vfma(shc, f2{by2, by2}, *q2);
                sig[l] = fmax(fmax(sig[l], x.x), x.y);
                *q2 = vfma(shc, f2{by1, by1}, vscale(av, bx1));
                continue;
              }
              sfor<GW>([&](auto J_) {
                constexpr int j = decltype(J_)::value, v = g * GW + j;
                T* q = wq + ((v * LMAX + (l - 1)) << 5) + lane;
                if constexpr (OE) {
                  // A_v(l) of row t-2, stored for the OEDG filter kernel
                  if (filt_row && out_lane) ((T*)a.oe.A)[(long long)(v * LMAX + l - 1) * a.ncell + cell2] = *q + by2 * comp<j>(shc);
                } else {
                  // Q of row t-2 + its top face; a plain max: a NaN jump comes from NaN modes, which the
                  // filter keeps NaN whatever the factor, so the cell is still reported
                  if (filt_row) sig[l] = fmax(sig[l], *q + by2 * comp<j>(shc));
                }
                if (need_v) *q = bx1 * comp<j>(av) + by1 * comp<j>(shc);          // Q of row t-1 (bottom face)
              });
            }
          });
          if ((LIM && a.hybrid)) {
            if (filt_row) eta2 = weta[lane] + eta_h;             // row t-2: + its top face
            if (need_v) weta[lane] = eta_v + eta_h;               // row t-1: vertical faces + bottom face
          }
        }
        if (filt_row) {
          const int s2 = sl2;
          T uo[NV][NM], lo[NV];
          if constexpr (PACK) {
#pragma unroll
            for (int vp = 0; vp < NV / 2; ++vp) {
              f2 blk[NMEP];
              pload(pblock(ws, s2, vp, lane), blk);
#pragma unroll
              for (int m = 0; m < NM; ++m) {
                uo[2 * vp][m] = blk[m].x;
                uo[2 * vp + 1][m] = blk[m].y;
              }
              lo[2 * vp] = blk[NM].x;
              lo[2 * vp + 1] = blk[NM].y;
            }
          } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
#pragma unroll
              for (int m = 0; m < NM; ++m) uo[v][m] = *slot_ptr(ws, s2, v, m, lane);
              if constexpr (PR::MIXED) lo[v] = *slot_ptr(ws, s2, v, NM, lane);
              else lo[v] = T(0);
            }
          }
          if constexpr (OE) {
            // u~ is stored as it is; the reductions for the OEDG coefficient
            if (out_lane) {
              auto coef = [](int i, int m) -> double { return lim_coef(i, m); };
#pragma unroll
              for (int v = 0; v < NV; ++v) osum[v] += (double)uo[v][0] + (double)lo[v];
#pragma unroll
              for (int i = 0; i < NQ * NQ; ++i) {               // the volume Gauss points
                T w[NV];
                point_w(uo, i, coef, w);
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                  omax[v] = fmax(omax[v], w[v]);
                  omin[v] = fmin(omin[v], w[v]);
                }
              }
            }
          } else if (a.filter_on) {
            T fac[LMAX + 1];
            if constexpr (PR::MIXED) {
              // exp(-sigma dt) as 2^(-sigma dt log2 e) by the hardware's approximate exponential
              // (about 2 ulp; a damping factor in (0, 1])
              const T dtl = dt * T(1.4426950408889634);
#pragma unroll
              for (int l = 1; l <= LMAX; ++l) {
                const float x = -(sig[l] * invH2) * dtl;
                float f;
                asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(f) : "f"(x));
                fac[l] = f;
              }
            } else {
#pragma unroll
              for (int l = 1; l <= LMAX; ++l) fac[l] = exp(-(sig[l] * invH2) * dt);
            }
            if (a.filter_on == FILT_GLOBAL) {
              // one coefficient for every mode, from the jumps of all derivative orders (Eq. para:damp)
#pragma unroll
              for (int l = 1; l < LMAX; ++l) fac[l] = fac[LMAX];
            }
            if ((LIM && a.hybrid)) {
              // u^DG is stored as it is; the blend kernel limits the troubled cells
              hybrid_record<T, LMAX>(a.hyb, a.ncell, cell2, out_lane, eta2, fac);
              if (out_lane) my_eta = nan_max(eta2, my_eta);
            } else if constexpr (PACK) {
#pragma unroll
              for (int vp = 0; vp < NV / 2; ++vp)
#pragma unroll
                for (int m = 1; m < NM; ++m) {
                  const f2 r = vscale(f2{uo[2 * vp][m], uo[2 * vp + 1][m]}, fac[PP[m] + QQ[m]]);
                  uo[2 * vp][m] = r.x;
                  uo[2 * vp + 1][m] = r.y;
                }
            } else {
#pragma unroll
              for (int v = 0; v < NV; ++v)
#pragma unroll
                for (int m = 1; m < NM; ++m) uo[v][m] *= fac[PP[m] + QQ[m]];
            }
          }
          T rate_pts = T(0);
          if constexpr (K >= 3) {
            if ((LIM && a.positivity) && out_lane) rate_pts = limit_and_rate(uo, gam, gm1, a.hx, a.hy);
          } else {
            if ((LIM && a.positivity) && out_lane) positivity_limit(uo, gm1);
          }
          if (out_lane) {
            ST::store(a.uout, a.ncell, cell2, uo, lo);
            if (!phys2) my_ok = false;
            if constexpr (PR::MIXED) {
              const T r = bx2 * inv_hx + by2 * inv_hy;
              my_rate_t = nan_max(r, my_rate_t);
              if constexpr (K >= 3) {
                if ((LIM && a.positivity)) my_rate_t = nan_max(rate_pts, my_rate_t);
              } else {
                if ((LIM && a.positivity)) my_rate_t = nan_max(point_rate(uo, gam, gm1, a.hx, a.hy), my_rate_t);
              }
            } else {
              const double r = (double)bx2 / a.hx + (double)by2 / a.hy;
              my_rate = (r > my_rate || r != r) ? r : my_rate;
              if ((LIM && a.positivity)) {
                const double rp = K >= 3 ? (double)rate_pts : (double)point_rate(uo, gam, gm1, a.hx, a.hy);
                my_rate = (rp > my_rate || rp != rp) ? rp : my_rate;
              }
            }
          }
        }
        // carry to the next row
        bx2 = bx1;
        by2 = by1;
        invH2 = invH1;
        phys2 = phys1;
        const int sfree = sl2;
        sl2 = sl1;
        sl1 = sl0;
        sl0 = sfree;
      }
    }
    if ((LIM && a.hybrid)) hybrid_max(a.hyb, my_eta);
    if constexpr (OE) oedg_reduce<NV>(a.oe, osum, omax, omin);
  }

  // All variables of a cell at limiter point i, w[v] = sum_m coef(i, m) uo[v][m] (the coefficients
  // fold to immediates in the unrolled callers); pairs of variables in packed FP32 (PACK).
  template <class CF>
  static __device__ __forceinline__ void point_w(const T (&uo)[NV][NM], int i, const CF& coef, T (&w)[NV]) {
    if constexpr (PACK) {
#pragma unroll
      for (int vp = 0; vp < NV / 2; ++vp) {
        f2 x{0.f, 0.f};
#pragma unroll
        for (int m = 0; m < NM; ++m) {
          const double c = coef(i, m);
          if (c != 0.0) x = vmad(f2{uo[2 * vp][m], uo[2 * vp + 1][m]}, (T)c, x);
        }
        w[2 * vp] = x.x;
        w[2 * vp + 1] = x.y;
      }
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T x = T(0);
#pragma unroll
        for (int m = 0; m < NM; ++m) {
          const double c = coef(i, m);
          if (c != 0.0) x += (T)c * uo[v][m];
        }
        w[v] = x;
      }
    }
  }

  // Max CFL rate beta^x / hx + beta^y / hy over the positivity limiter's points of one cell: with
  // the limiter on, Zhang and Shu's positivity result for the averages needs the CFL bound on the
  // wave speeds at those points, not only at the average.
  static __device__ T point_rate(const T (&uo)[NV][NM], T gam, T gm1, double hx, double hy) {
    T best = T(0);
    if constexpr (EQ == EQ_EULER) {
      constexpr int NP = NP_LIM;
      const T thx = (T)hx, thy = (T)hy;
      auto coef = [](int i, int m) -> double { return lim_coef(i, m); };
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T w[NV];
        point_w(uo, i, coef, w);
        T bx, by, invH;
        bool ph;
        avg_params<EQ, 2>(w, gam, gm1, T(0), T(0), bx, by, invH, ph);
        best = nan_max(bx / thx + by / thy, best);
      }
    }
    return best;
  }

  // Zhang-Shu positivity-preserving limiter on one cell (after the filter, as in Section 3.2 of the
  // paper): density first (theta_1), then pressure (theta_2), checked at the volume and edge Gauss
  // points where the scheme evaluates the polynomial. Cell averages are not touched.
  static __device__ void positivity_limit(T (&uo)[NV][NM], T gm1) {
    if constexpr (EQ == EQ_EULER) {
      constexpr int NP = NP_LIM;
      T ub[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) ub[v] = uo[v][0];
      const T pbar = pressure_of<NV>(ub, gm1);
      // admissibility margins, relative to the cell average in both precisions (as the oracle):
      // rho(x) >= 1e-3 rho_bar and p(x) >= min(1e-3 (rho_bar + |E_bar|), rho_bar, p_bar). Relative
      // margins keep the velocity at a limited point bounded (an absolute 1e-10 let it grow until
      // the CFL rate over the limiter's points collapsed dt), and in the FP32 form they keep a
      // limited point positive when the next stage re-evaluates it in a different order
      T eps_r = T(1e-3) * ub[0];
      T eps = T(1e-3) * (ub[0] + fabs(ub[NV - 1]));
      eps_r = ub[0] < eps_r ? ub[0] : eps_r;
      eps = ub[0] < eps ? ub[0] : eps;
      eps = pbar < eps ? pbar : eps;
      if (!(eps > T(0)) || !(eps_r > T(0))) return;
      auto coef = [](int i, int m) -> double { return lim_coef(i, m); };
      T rmin = ub[0];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T r = T(0);
#pragma unroll
        for (int m = 0; m < NM; ++m) {
          const double c = coef(i, m);
          if (c != 0.0) r += (T)c * uo[0][m];
        }
        rmin = r < rmin ? r : rmin;
      }
      if (rmin < eps_r) {
        const T th1 = (ub[0] - eps_r) / (ub[0] - rmin);
#pragma unroll
        for (int m = 1; m < NM; ++m) uo[0][m] *= th1;
      }
      T th2 = T(1);
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T w[NV];
        point_w(uo, i, coef, w);
        if (pressure_of<NV>(w, gm1) < eps) {
          const T t = pp_segment<NV>(ub, w, eps, gm1);
          th2 = t < th2 ? t : th2;
        }
      }
      if (th2 < T(1)) {
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
          for (int m = 1; m < NM; ++m) uo[v][m] *= th2;
      }
    }
  }

  // The limiter of positivity_limit with the CFL rate of point_rate taken in its pressure pass (the
  // point values there are the final ones unless theta_2 < 1, in which case the limited cell is
  // evaluated once more). Used from degree 3, where the points are many (NQ^2 + 4 NQ = 32).
  static __device__ T limit_and_rate(T (&uo)[NV][NM], T gam, T gm1, double hx, double hy) {
    if constexpr (EQ != EQ_EULER) {
      return T(0);
    } else {
      constexpr int NP = NP_LIM;
      T ub[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) ub[v] = uo[v][0];
      const T pbar = pressure_of<NV>(ub, gm1);
      // the same admissibility margins as positivity_limit
      T eps_r = T(1e-3) * ub[0];
      T eps = T(1e-3) * (ub[0] + fabs(ub[NV - 1]));
      eps_r = ub[0] < eps_r ? ub[0] : eps_r;
      eps = ub[0] < eps ? ub[0] : eps;
      eps = pbar < eps ? pbar : eps;
      if (!(eps > T(0)) || !(eps_r > T(0))) return point_rate(uo, gam, gm1, hx, hy);
      const T thx = (T)hx, thy = (T)hy;
      auto coef = [](int i, int m) -> double { return lim_coef(i, m); };
      T rmin = ub[0];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T r = T(0);
#pragma unroll
        for (int m = 0; m < NM; ++m) {
          const double c = coef(i, m);
          if (c != 0.0) r += (T)c * uo[0][m];
        }
        rmin = r < rmin ? r : rmin;
      }
      if (rmin < eps_r) {
        const T th1 = (ub[0] - eps_r) / (ub[0] - rmin);
#pragma unroll
        for (int m = 1; m < NM; ++m) uo[0][m] *= th1;
      }
      T th2 = T(1), rate = T(0);
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T w[NV];
        point_w(uo, i, coef, w);
        if (pressure_of<NV>(w, gm1) < eps) {
          const T t = pp_segment<NV>(ub, w, eps, gm1);
          th2 = t < th2 ? t : th2;
        }
        T bx, by, invH;
        bool ph;
        avg_params<EQ, 2>(w, gam, gm1, T(0), T(0), bx, by, invH, ph);
        rate = nan_max(bx / thx + by / thy, rate);
      }
      if (th2 < T(1)) {
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
          for (int m = 1; m < NM; ++m) uo[v][m] *= th2;
        rate = point_rate(uo, gam, gm1, hx, hy);
      }
      return rate;
    }
  }

  // Single-instance stage: one warp per tile item, step control on the instance's DevScalars.
  static __device__ void run(const Stage2DArgs& a, unsigned char* smem) {
    const StageCtl ctl = stage_begin(a.sc, a.stage, a.cfl);
    if (!ctl.run) return;
    if constexpr (OE) {
      if (blockIdx.x == 0 && threadIdx.x == 0) a.oe.sc->active = 1u;
    }
    const int wib = threadIdx.x >> 5;
    double* red = (double*)smem;                                  // 32 doubles for stage_end
    T* ws = (T*)(smem + 256 + warp_bytes() * wib);
    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + wib;
    double my_rate = 0.0;
    T my_rate_t = T(0);
    bool my_ok = true;
    if (gw < (long long)a.nstrips * a.nchunks)
      item(a, ctl.dt, (int)(gw % a.nstrips), (int)(gw / a.nstrips), ws, my_rate, my_rate_t, my_ok);
    if constexpr (PR::MIXED) my_rate = (double)my_rate_t;
    stage_end(a.sc, a.stage, my_rate, my_ok, red);
  }
};

template <int K, int EQ, int BASIS, class PR, bool OE = false, bool LIM = true>
__global__ void __launch_bounds__(256) stage2d_kernel(const Stage2DArgs a) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  Stage2D<K, EQ, BASIS, PR, OE, LIM>::run(a, dyn_smem);
}

}  // namespace dgk
