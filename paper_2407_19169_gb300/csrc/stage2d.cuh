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
#include "stage_common.cuh"

namespace dgk {

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
  int filter_on;
  double gamma, ax, ay, cfl;
  int H;             // rows per chunk
  int nstrips, nchunks;
  int positivity;    // Euler: Zhang-Shu limiter after the filter
  DevScalars* sc;
};

constexpr int STRIP_OUT = 28;  // output columns per warp

// Storage policies. FP64: one double plane per (v, m). FP32 mixed: a float2 (hi, lo) plane per v for
// the cell average (mode 0, a double-float value), then float planes for modes 1..NM-1.
struct PrecF64 {
  using T = double;
  static constexpr bool MIXED = false;
};
struct PrecF32M {
  using T = float;
  static constexpr bool MIXED = true;
};

template <class PR, int NV, int NM>
struct Store {
  using T = typename PR::T;
  // load u[v][m] (and the low word of the mode-0 double-float in lo0[v]).
  static __device__ __forceinline__ void load(const void* base, long long ncell, long long c,
                                              T (&u)[NV][NM], T (&lo0)[NV]) {
    if constexpr (!PR::MIXED) {
      const double* b = (const double*)base;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
#pragma unroll
        for (int m = 0; m < NM; ++m) u[v][m] = __ldg(b + (long long)(v * NM + m) * ncell + c);
        lo0[v] = T(0);
      }
    } else {
      const float2* b0 = (const float2*)base;
      const float* bh = (const float*)((const char*)base + sizeof(float2) * (size_t)NV * ncell);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        float2 a = __ldg(b0 + (long long)v * ncell + c);
        u[v][0] = a.x;
        lo0[v] = a.y;
#pragma unroll
        for (int m = 1; m < NM; ++m) u[v][m] = __ldg(bh + (long long)(v * (NM - 1) + m - 1) * ncell + c);
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

template <int K, int EQ, int BASIS, class PR>
struct Stage2D {
  using T = typename PR::T;
  using MB = Modes<K, BASIS>;
  static constexpr int NM = MB::NM;
  static constexpr int NV = NVars<EQ, 2>::value;
  static constexpr int NQ = K + 1;
  static constexpr int LMAX = MB::LMAX;
  static constexpr int NA = MB::NA;
  static constexpr int NME = NM + (PR::MIXED ? 1 : 0);  // slot words per variable (+ mode-0 low word)
  using GR = GaussRule<NQ>;
  using ST = Store<PR, NV, NM>;

  // per-warp shared memory: 3 row slots of u~ plus the partial damping Q[v][l-1] of one row
  static constexpr size_t warp_bytes() { return sizeof(T) * (3 * NV * NME + NV * LMAX) * 32; }
  static constexpr size_t slot_bytes_per_warp() { return warp_bytes(); }

  // ---- compile-time tables (evaluated by the front end) ----
  // mode degrees and total degree l = p + q
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
  // volume point values P_p(x_a) P_q(x_b) and the weighted test-function derivatives
  __host__ __device__ static constexpr carr<double, NQ * NQ * NM> tab_vol(int which) {
    carr<double, NQ * NQ * NM> t{};
    for (int qa = 0; qa < NQ; ++qa)
      for (int qb = 0; qb < NQ; ++qb)
        for (int m = 0; m < NM; ++m) {
          const int pp = MB::p(m), qq = MB::q(m);
          const double w = GR::w(qa) * GR::w(qb);
          double v = 0.0;
          if (which == 0) v = GR::P(pp, qa) * GR::P(qq, qb);
          if (which == 1) v = w * GR::dP(pp, qa) * GR::P(qq, qb);
          if (which == 2) v = w * GR::P(pp, qa) * GR::dP(qq, qb);
          t[(qa * NQ + qb) * NM + m] = v;
        }
    return t;
  }
  // edge quadrature against the test function: vertical edges w_g P_q(x_g), horizontal w_g P_p(x_g)
  __host__ __device__ static constexpr carr<double, NQ * NM> tab_face(int horizontal) {
    carr<double, NQ * NM> t{};
    for (int g = 0; g < NQ; ++g)
      for (int m = 0; m < NM; ++m) t[g * NM + m] = GR::w(g) * GR::P(horizontal ? MB::p(m) : MB::q(m), g);
    return t;
  }
  // corner derivative coefficients d^a1 P_p(sx) d^a2 P_q(sy), corner index c = 2 sx + sy
  __host__ __device__ static constexpr carr<double, 4 * NA * NM> tab_corner() {
    carr<double, 4 * NA * NM> t{};
    for (int c = 0; c < 4; ++c)
      for (int a = 0; a < NA; ++a)
        for (int m = 0; m < NM; ++m)
          t[(c * NA + a) * NM + m] = dend(c >> 1, MB::p(m), MB::a1(a)) * dend(c & 1, MB::q(m), MB::a2(a));
    return t;
  }
  __host__ __device__ static constexpr carr<int, NA> tab_a(int which) {
    carr<int, NA> t{};
    for (int a = 0; a < NA; ++a) t[a] = which == 0 ? MB::a1(a) : MB::a2(a);
    return t;
  }

  // row slot of row r (rows >= -2 occur; keep the index in 0..2)
  static __device__ __forceinline__ int slot_of(int r) { return ((r % 3) + 3) % 3; }
  static __device__ __forceinline__ T* slot_ptr(T* ws, int s, int v, int m, int lane) {
    return ws + (((s * NV + v) * NME + m) << 5) + lane;
  }
  static __device__ __forceinline__ T shfl_down_t(T x, int d) { return __shfl_down_sync(0xffffffffu, x, d); }
  static __device__ __forceinline__ T shfl_up_t(T x, int d) { return __shfl_up_sync(0xffffffffu, x, d); }

  // Traces of all variables at Gauss point g of one edge.
  static __device__ __forceinline__ void trace_at(const T (&u)[NV][NM], const double* tab, int g, T (&tr)[NV]) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T s = T(0);
#pragma unroll
      for (int m = 0; m < NM; ++m) {
        const double c = tab[g * NM + m];
        if (c != 0.0) s += u[v][m] * (T)c;
      }
      tr[v] = s;
    }
  }

  // One tile item: strip `strip` (28 output columns) and row chunk `chunk` of one instance, with step
  // size dtd. ws: this warp's row slots and Q area in shared memory. The output cells' max CFL rate
  // and physicality are folded into my_rate (FP64 form) / my_rate_t (FP32 form) and my_ok.
  static __device__ void item(const Stage2DArgs& a, double dtd, int strip, int chunk, T* ws,
                              double& my_rate, T& my_rate_t, bool& my_ok) {
    constexpr carr<int, NM> PP = tab_p();
    constexpr carr<int, NM> QQ = tab_q();
    constexpr carr<double, 2 * NQ * NM> TH = tab_trace_h();
    constexpr carr<double, 2 * NQ * NM> TV = tab_trace_v();
    constexpr carr<double, NQ * NQ * NM> VE = tab_vol(0);
    constexpr carr<double, NQ * NQ * NM> VX = tab_vol(1);
    constexpr carr<double, NQ * NQ * NM> VY = tab_vol(2);
    constexpr carr<double, NQ * NM> FXT = tab_face(0);
    constexpr carr<double, NQ * NM> FYT = tab_face(1);
    constexpr carr<double, 4 * NA * NM> CT = tab_corner();
    constexpr carr<int, NA> A1 = tab_a(0);
    constexpr carr<int, NA> A2 = tab_a(1);

    const T dt = (T)dtd;
    const int lane = threadIdx.x & 31;
    T* wq = ws + 3 * NV * NME * 32;                               // Q[v][l-1] of the next row to filter
    const int nx = a.nx, ny = a.ny;
    const T gam = (T)a.gamma, gm1 = (T)(a.gamma - 1.0), ax = (T)a.ax, ay = (T)a.ay;
    const T inv_hx = (T)(1.0 / a.hx), inv_hy = (T)(1.0 / a.hy);
    const T c1dt = (T)(a.c1 * dtd), c0 = (T)a.c0;
    // double-float coefficients of the cell-average update (computed once, off the cell loop)
    const df dfx = df_from_double(a.c1 * dtd * 0.5 / a.hx);
    const df dfy = df_from_double(a.c1 * dtd * 0.5 / a.hy);
    const df dfc0 = df_from_double(a.c0);
    // powers of 2/h for physical derivatives; weights m(m+1) h^m of the m-th derivative jumps
    T px[K + 1], py[K + 1], wx[LMAX + 1], wy[LMAX + 1];
    {
      double sx = 1.0, sy = 1.0;
#pragma unroll
      for (int r = 0; r <= K; ++r) {
        px[r] = (T)sx;
        py[r] = (T)sy;
        sx *= 2.0 / a.hx;
        sy *= 2.0 / a.hy;
      }
      double hx = 1.0, hy = 1.0;
#pragma unroll
      for (int m = 0; m <= LMAX; ++m) {
        wx[m] = (T)(m == 0 ? 1.0 : m * (m + 1) * hx);
        wy[m] = (T)(m == 0 ? 1.0 : m * (m + 1) * hy);
        hx *= a.hx;
        hy *= a.hy;
      }
    }
    {
      const int x = strip * STRIP_OUT - 2 + lane;
      const bool perx = a.bcx == BC_PERIODIC, pery = a.bcy == BC_PERIODIC;
      const int xc = perx ? ((x % nx) + nx) % nx : (x < 0 ? 0 : (x >= nx ? nx - 1 : x));
      // outflow: columns and rows outside the mesh are ghost cells holding the constant state equal
      // to the adjacent interior cell's average (stage input for the fluxes, u~ for the jumps)
      const bool gcol = !perx && (x < 0 || x >= nx);
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

#pragma unroll 1
      for (int t = yb - 2; t <= ye + 1; ++t) {
        const bool grow = !pery && (t < 0 || t >= ny);
        const int ty = pery ? ((t % ny) + ny) % ny : (t < 0 ? 0 : (t >= ny ? ny - 1 : t));
        const long long cell = (long long)ty * nx + xc;
        T u[NV][NM], lo0[NV];
        ST::load(a.uin, a.ncell, cell, u, lo0);
        if (grow || gcol) {
#pragma unroll
          for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int m = 1; m < NM; ++m) u[v][m] = T(0);
        }

        // ---- horizontal face between rows t-1 and t (once per column) ----
        T Fh[NQ][NV];
        if (t >= yb - 1) {
#pragma unroll
          for (int g = 0; g < NQ; ++g) {
            T bot[NV];
            trace_at(u, &TH.v[0], g, bot);
            llf2d<EQ, 1>(topPrev[g], bot, Fh[g], gam, gm1, ax, ay);
          }
          // finalise u~ of row t-1 with its top-face term
          if (t - 1 >= yb - 1 && t - 1 <= ye) {
            const int s = slot_of(t - 1);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              if constexpr (PR::MIXED) {
                T phi = T(0);
#pragma unroll
                for (int g = 0; g < NQ; ++g) phi += (T)GR::w(g) * Fh[g][v];
                df acc0{*slot_ptr(ws, s, v, 0, lane), *slot_ptr(ws, s, v, NM, lane)};
                acc0 = df_add(acc0, df_mul_f(dfy, -phi));
                *slot_ptr(ws, s, v, 0, lane) = acc0.hi;
                *slot_ptr(ws, s, v, NM, lane) = acc0.lo;
              }
#pragma unroll
              for (int m = PR::MIXED ? 1 : 0; m < NM; ++m) {
                T sum = T(0);
#pragma unroll
                for (int g = 0; g < NQ; ++g) {
                  const double c = FYT[g * NM + m];
                  if (c != 0.0) sum += (T)c * Fh[g][v];
                }
                *slot_ptr(ws, s, v, m, lane) -= (T)(0.5 * (2 * PP[m] + 1) * (2 * QQ[m] + 1)) * c1dt * inv_hy * sum;
              }
            }
          }
        }

        // ---- partial u~ of row t: bottom face, vertical faces, volume, RK combination ----
        if (t >= yb - 1 && t <= ye) {
          T acc[NV][NM];
          T phiR[NV], phiL[NV], phiB[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            phiR[v] = phiL[v] = phiB[v] = T(0);
#pragma unroll
            for (int m = 0; m < NM; ++m) {
              T sum = T(0);
#pragma unroll
              for (int g = 0; g < NQ; ++g) {
                const double c = FYT[g * NM + m] * ((QQ[m] & 1) ? -1.0 : 1.0);
                if (c != 0.0) sum += (T)c * Fh[g][v];
              }
              acc[v][m] = sum * inv_hy;
            }
#pragma unroll
            for (int g = 0; g < NQ; ++g) phiB[v] += (T)GR::w(g) * Fh[g][v];
          }
          // vertical faces, one Gauss point at a time: F^_R by this lane, F^_L from the left lane
#pragma unroll
          for (int g = 0; g < NQ; ++g) {
            T tl[NV], tr[NV], nb[NV], FR[NV], FL[NV];
            trace_at(u, &TV.v[0], g, tl);
            trace_at(u, &TV.v[NQ * NM], g, tr);
#pragma unroll
            for (int v = 0; v < NV; ++v) nb[v] = shfl_down_t(tl[v], 1);
            llf2d<EQ, 0>(tr, nb, FR, gam, gm1, ax, ay);
#pragma unroll
            for (int v = 0; v < NV; ++v) FL[v] = shfl_up_t(FR[v], 1);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              phiR[v] += (T)GR::w(g) * FR[v];
              phiL[v] += (T)GR::w(g) * FL[v];
#pragma unroll
              for (int m = 0; m < NM; ++m) {
                const double c = FXT[g * NM + m];
                if (c != 0.0)
                  acc[v][m] -= inv_hx * (T)c * (FR[v] - ((PP[m] & 1) ? -FL[v] : FL[v]));
              }
            }
          }
          // volume integral at the NQ x NQ Gauss points
#pragma unroll
          for (int qa = 0; qa < NQ; ++qa)
#pragma unroll
            for (int qb = 0; qb < NQ; ++qb) {
              const int base = (qa * NQ + qb) * NM;
              T uq[NV], fx[NV], fy[NV];
#pragma unroll
              for (int v = 0; v < NV; ++v) {
                T sacc = T(0);
#pragma unroll
                for (int m = 0; m < NM; ++m) {
                  const double c = VE[base + m];
                  if (c != 0.0) sacc += u[v][m] * (T)c;
                }
                uq[v] = sacc;
              }
              flux2d_xy<EQ>(uq, fx, fy, gm1, ax, ay);
#pragma unroll
              for (int v = 0; v < NV; ++v) {
                const T fxs = fx[v] * inv_hx, fys = fy[v] * inv_hy;
#pragma unroll
                for (int m = 0; m < NM; ++m) {
                  const double cx = VX[base + m], cy = VY[base + m];
                  if (cx != 0.0) acc[v][m] += fxs * (T)cx;
                  if (cy != 0.0) acc[v][m] += fys * (T)cy;
                }
              }
            }
          const int s = slot_of(t);
          T un_[NV][NM], unlo[NV];
          if (a.stage > 0) ST::load(a.un, a.ncell, cell, un_, unlo);
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            if constexpr (PR::MIXED) {
              // cell average in double-float from the edge integrals, each computed once per edge:
              // u0 + c0 (un0 - u0) + c1 dt/(2h) (Phi_L - Phi_R + Phi_B - Phi_T)
              df m0{u[v][0], lo0[v]};
              if (a.stage > 0) {
                const df d = df_add(df{un_[v][0], unlo[v]}, df{-u[v][0], -lo0[v]});
                m0 = df_add(m0, df_mul(dfc0, d));
              }
              m0 = df_add(m0, df_mul_f(dfx, phiL[v]));
              m0 = df_add(m0, df_mul_f(dfx, -phiR[v]));
              m0 = df_add(m0, df_mul_f(dfy, phiB[v]));
              *slot_ptr(ws, s, v, 0, lane) = m0.hi;
              *slot_ptr(ws, s, v, NM, lane) = m0.lo;
            }
#pragma unroll
            for (int m = PR::MIXED ? 1 : 0; m < NM; ++m) {
              const T R = (T)(0.5 * (2 * PP[m] + 1) * (2 * QQ[m] + 1)) * acc[v][m];
              // u + c0 (u^n - u) + c1 dt R  (= c0 u^n + c1 (u + dt R) with c0 + c1 = 1 kept exact)
              T val = u[v][m] + c1dt * R;
              if (a.stage > 0) val += c0 * (un_[v][m] - u[v][m]);
              *slot_ptr(ws, s, v, m, lane) = val;
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
        if (r1) {
          T ub[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) ub[v] = *slot_ptr(ws, slot_of(t - 1), v, 0, lane);
          avg_params<EQ, 2>(ub, gam, gm1, ax, ay, bx1, by1, invH1, phys1);
        }
        T sig[LMAX + 1];
#pragma unroll
        for (int l = 0; l <= LMAX; ++l) sig[l] = T(0);
        if (a.filter_on && (need_v || filt_row)) {
          const int s1 = slot_of(t - 1), s2 = slot_of(t - 2);
#pragma unroll 1
          for (int v = 0; v < NV; ++v) {
            T uv[NM], u2[NM];
#pragma unroll
            for (int m = 0; m < NM; ++m) {
              uv[m] = *slot_ptr(ws, s1, v, m, lane);
              u2[m] = *slot_ptr(ws, s2, v, m, lane);
            }
            // ghost rows and columns: the constant state of the adjacent interior cell's u~ average
            if (g1) {
              uv[0] = u2[0];
#pragma unroll
              for (int m = 1; m < NM; ++m) uv[m] = T(0);
            }
            if (g2) {
              u2[0] = uv[0];
#pragma unroll
              for (int m = 1; m < NM; ++m) u2[m] = T(0);
            }
            {
              const T v_r = shfl_down_t(uv[0], 1), v_l = shfl_up_t(uv[0], 1);
              const T w_r = shfl_down_t(u2[0], 1), w_l = shfl_up_t(u2[0], 1);
              if (gcol) {
                uv[0] = x < 0 ? v_r : v_l;
                u2[0] = x < 0 ? w_r : w_l;
#pragma unroll
                for (int m = 1; m < NM; ++m) uv[m] = u2[m] = T(0);
              }
            }
            T svr[LMAX + 1], sh[LMAX + 1];
#pragma unroll
            for (int l = 0; l <= LMAX; ++l) svr[l] = sh[l] = T(0);
#pragma unroll
            for (int aa = 0; aa < NA; ++aa) {
              // corner values of d^alpha u~: c00 = (xi,eta) = (-1,-1), c01 = (-1,+1), c10, c11
              T c00 = T(0), c01 = T(0), c10 = T(0), c11 = T(0), t01 = T(0), t11 = T(0);
#pragma unroll
              for (int m = 0; m < NM; ++m) {
                const double k00 = CT[(0 * NA + aa) * NM + m], k01 = CT[(1 * NA + aa) * NM + m];
                const double k10 = CT[(2 * NA + aa) * NM + m], k11 = CT[(3 * NA + aa) * NM + m];
                if (k00 != 0.0) c00 += uv[m] * (T)k00;
                if (k01 != 0.0) { c01 += uv[m] * (T)k01; t01 += u2[m] * (T)k01; }
                if (k10 != 0.0) c10 += uv[m] * (T)k10;
                if (k11 != 0.0) { c11 += uv[m] * (T)k11; t11 += u2[m] * (T)k11; }
              }
              const T f = px[A1[aa]] * py[A2[aa]];
              c00 *= f; c01 *= f; c10 *= f; c11 *= f; t01 *= f; t11 *= f;
              const int l = A1[aa] + A2[aa];
              if (need_v) {
                const T n0 = shfl_down_t(c00, 1), n1 = shfl_down_t(c01, 1);
                svr[l] += T(0.5) * (fabs(c10 - n0) + fabs(c11 - n1));
              }
              sh[l] += T(0.5) * (fabs(c00 - t01) + fabs(c10 - t11));
            }
            T av = T(0), shc = T(0);
#pragma unroll
            for (int l = 0; l <= LMAX; ++l) {
              shc += wy[l] * sh[l];
              if (need_v) av += wx[l] * (shfl_up_t(svr[l], 1) + svr[l]);
              if (l == 0) continue;
              T* q = wq + ((v * LMAX + (l - 1)) << 5) + lane;
              if (filt_row) sig[l] = nan_max(sig[l], *q + by2 * shc);   // Q of row t-2 + its top face
              if (need_v) *q = bx1 * av + by1 * shc;                      // Q of row t-1 (bottom face)
            }
          }
        }
        if (filt_row) {
          const int s2 = slot_of(t - 2);
          const int ty2 = pery ? ((t - 2) % ny + ny) % ny : t - 2;
          const long long cell2 = (long long)ty2 * nx + xc;
          T uo[NV][NM], lo[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
#pragma unroll
            for (int m = 0; m < NM; ++m) uo[v][m] = *slot_ptr(ws, s2, v, m, lane);
            if constexpr (PR::MIXED) lo[v] = *slot_ptr(ws, s2, v, NM, lane);
            else lo[v] = T(0);
          }
          if (a.filter_on) {
            T fac[LMAX + 1];
#pragma unroll
            for (int l = 1; l <= LMAX; ++l) fac[l] = exp(-(sig[l] * invH2) * dt);
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
              for (int m = 1; m < NM; ++m) uo[v][m] *= fac[PP[m] + QQ[m]];
          }
          if (a.positivity && out_lane) positivity_limit(uo, gm1);
          if (out_lane) {
            ST::store(a.uout, a.ncell, cell2, uo, lo);
            if (!phys2) my_ok = false;
            if constexpr (PR::MIXED) {
              const T r = bx2 * inv_hx + by2 * inv_hy;
              my_rate_t = nan_max(r, my_rate_t);
              if (a.positivity) my_rate_t = nan_max(point_rate(uo, gam, gm1, a.hx, a.hy), my_rate_t);
            } else {
              const double r = (double)bx2 / a.hx + (double)by2 / a.hy;
              my_rate = (r > my_rate || r != r) ? r : my_rate;
              if (a.positivity) {
                const double rp = (double)point_rate(uo, gam, gm1, a.hx, a.hy);
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
#pragma unroll
        for (int g = 0; g < NQ; ++g) trace_at(u, &TH.v[NQ * NM], g, topPrev[g]);
      }
    }
  }

  // Max CFL rate beta^x / hx + beta^y / hy over the positivity limiter's points of one cell: with
  // the limiter on, Zhang and Shu's positivity result for the averages needs the CFL bound on the
  // wave speeds at those points, not only at the average.
  static __device__ T point_rate(const T (&uo)[NV][NM], T gam, T gm1, double hx, double hy) {
    T best = T(0);
    if constexpr (EQ == EQ_EULER) {
      constexpr carr<double, NQ * NQ * NM> VE = tab_vol(0);
      constexpr carr<double, 2 * NQ * NM> TH = tab_trace_h();
      constexpr carr<double, 2 * NQ * NM> TV = tab_trace_v();
      constexpr int NP = NQ * NQ + 4 * NQ;
      const T thx = (T)hx, thy = (T)hy;
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T w[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          T x = T(0);
#pragma unroll
          for (int m = 0; m < NM; ++m) {
            const double c = i < NQ * NQ ? VE[i * NM + m]
                                         : (i < NQ * NQ + 2 * NQ ? TH[(i - NQ * NQ) * NM + m]
                                                                 : TV[(i - NQ * NQ - 2 * NQ) * NM + m]);
            if (c != 0.0) x += (T)c * uo[v][m];
          }
          w[v] = x;
        }
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
      constexpr carr<double, NQ * NQ * NM> VE = tab_vol(0);
      constexpr carr<double, 2 * NQ * NM> TH = tab_trace_h();
      constexpr carr<double, 2 * NQ * NM> TV = tab_trace_v();
      constexpr int NP = NQ * NQ + 4 * NQ;
      T ub[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) ub[v] = uo[v][0];
      const T pbar = pressure_of<NV>(ub, gm1);
      // admissibility margins: 1e-10 in FP64 (as the oracle). In the FP32 form point values of rho
      // and |m|^2 / (2 rho) lose digits to cancellation when rho(x) << rho_bar, so the margins are
      // relative: rho(x) >= 1e-3 rho_bar and p(x) >= 1e-3 (rho_bar + E_bar), which keeps a limited
      // point positive when the next stage re-evaluates it in a different order
      T eps_r = sizeof(T) == 8 ? T(1e-10) : T(1e-3) * ub[0];
      T eps = sizeof(T) == 8 ? T(1e-10) : T(1e-3) * (ub[0] + fabs(ub[NV - 1]));
      eps_r = ub[0] < eps_r ? ub[0] : eps_r;
      eps = ub[0] < eps ? ub[0] : eps;
      eps = pbar < eps ? pbar : eps;
      if (!(eps > T(0)) || !(eps_r > T(0))) return;
      auto coef = [&](int i, int m) -> double {
        return i < NQ * NQ ? VE[i * NM + m]
                           : (i < NQ * NQ + 2 * NQ ? TH[(i - NQ * NQ) * NM + m] : TV[(i - NQ * NQ - 2 * NQ) * NM + m]);
      };
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

  // Single-instance stage: one warp per tile item, step control on the instance's DevScalars.
  static __device__ void run(const Stage2DArgs& a, unsigned char* smem) {
    const StageCtl ctl = stage_begin(a.sc, a.stage, a.cfl);
    if (!ctl.run) return;
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

template <int K, int EQ, int BASIS, class PR>
__global__ void __launch_bounds__(256) stage2d_kernel(const Stage2DArgs a) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  Stage2D<K, EQ, BASIS, PR>::run(a, dyn_smem);
}

}  // namespace dgk
