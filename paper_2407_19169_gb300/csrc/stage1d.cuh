// stage1d.cuh — fused 1D SSP-RK3 stage with the jump filter (one launch per stage).
//
// Per cell K_j (Section 2.1):
//   R^l = (2l+1)/h [ sum_q w_q f(u_h(xi_q)) P_l'(xi_q) - f^_{j+1/2} + (-1)^l f^_{j-1/2} ]   (Eq. scheme:DG)
//   u~ = c0 u^n + c1 (u^(s) + dt R)                                                          (Eq. rkdg1)
//   u^l <- exp(-sigma^l dt) u~^l,  sigma^l = beta/(h Hbar) max_v (J_0 + sum_{m=1..l} m(m+1) h^m J_m)
// the last line being Eqs. (para:damp2)-(para:damp21) with c_f^l = beta/(4 l(l+1)) (1/Hbar for
// Euler, Section 3.1) substituted, the max over components of Eq. (para:dampsystems1d), and
// J_m = |[d^m u]_{j-1/2}| + |[d^m u]_{j+1/2}| with physical derivatives.
//
// Parallel structure: a warp owns 32 consecutive cells and writes the middle 28 (2-cell halo per
// side); traces, face fluxes, end derivatives and face jumps move between lanes by shuffles. Each
// face flux and face jump is computed once, by the face's left cell. Outflow boundaries: lanes
// outside the mesh are ghost cells holding the constant state of the adjacent interior cell's
// average (for the fluxes that of the stage input, for the jumps that of u~).
#pragma once
#include "stage2d.cuh"

namespace dgk {

struct Stage1DArgs {
  const void* uin;
  const void* un;
  void* uout;
  int nx;
  long long ncell;
  double h;
  int bc;            // BC_PERIODIC or BC_OUTFLOW (both ends alike)
  double c0, c1;
  int stage;
  int filter_on;      // FILT_OFF, FILT_JUMP or FILT_GLOBAL
  double gamma, ax, cfl;
  int nwarps;
  int positivity;    // Euler: Zhang-Shu limiter after the filter
  int hybrid;        // hybrid limiter (Algorithm 1): store u^DG, eta and the filter factors
  HybridOut hyb;
  OedgOut oe;        // OEDG damping (kernels instantiated with OE = true)
  DevScalars* sc;
  // mesh constants computed once on the host (stage1d_consts): 1/h, 2/h and the jump weights
  // m(m+1) h^m (1 for m = 0), and the OEDG weights (2m+1)/m! h^m, in both arithmetic types; c0 as
  // a double-float
  double inv_h_d, scl_d, wpow_d[4], wpoe_d[4];
  float inv_h_f, scl_f, wpow_f[4], wpoe_f[4];
  float c0_hi, c0_lo;
};

// Fill the host-side constants of a Stage1DArgs from its h and c0 (no FP64 division on the GPU).
inline void stage1d_consts(Stage1DArgs& a) {
  a.inv_h_d = 1.0 / a.h;
  a.scl_d = 2.0 / a.h;
  a.inv_h_f = (float)a.inv_h_d;
  a.scl_f = (float)a.scl_d;
  double hp = 1.0;
  double fm = 1.0;
  for (int m = 0; m < 4; ++m) {
    a.wpow_d[m] = m == 0 ? 1.0 : m * (m + 1) * hp;
    a.wpow_f[m] = (float)a.wpow_d[m];
    if (m > 0) fm *= m;
    a.wpoe_d[m] = (2 * m + 1) / fm * hp;
    a.wpoe_f[m] = (float)a.wpoe_d[m];
    hp *= a.h;
  }
  a.c0_hi = (float)a.c0;
  a.c0_lo = (float)(a.c0 - (double)a.c0_hi);
}

// OE = true: the OEDG form of the damping (the kernel stores u~ unfiltered with the jump sums A_v(l)
// and the reductions of OedgOut; the OEDG filter kernel applies the damping).
// COH = true: state loads through L2 (Store), for the persistent batched kernel.
template <int K, int EQ, class PR, bool OE = false, bool COH = false>
struct Stage1D {
  using T = typename PR::T;
  static constexpr int NM = K + 1;
  static constexpr int NV = NVars<EQ, 1>::value;
  static constexpr int NQ = K + 1;
  using GR = GaussRule<NQ>;
  using ST = Store<PR, NV, NM, COH>;
  // FP32 form, Euler (three variables): the double-float cell averages of variables 0 and 1 in one
  // register pair (packed FP32 instructions, bitwise the same results). Degrees 1 and 2 only
  // (4 M cells: k = 1 0.108 -> 0.105 ms per launch, k = 2 -1 %; k = 3 +0.4 %).
  static constexpr bool PACK_DF = PR::MIXED && NV == 3 && K <= 2;
  using TB = Tab2D<K, BASIS_Q>;        // the 1D mode l is the x-degree p of the tables

  static __device__ __forceinline__ T sd(T x, int d) { return __shfl_down_sync(0xffffffffu, x, d); }
  static __device__ __forceinline__ T su(T x, int d) { return __shfl_up_sync(0xffffffffu, x, d); }

  // One tile item: the 32-cell strip `strip` (28 output cells) of one instance, step size dtd. The
  // output cells' max CFL rate and physicality are folded into my_rate / my_rate_t and my_ok.
  static __device__ void item(const Stage1DArgs& a, double dtd, long long strip, double& my_rate,
                              T& my_rate_t, bool& my_ok) {
    const T dt = (T)dtd;
    const int lane = threadIdx.x & 31;
    const int nx = a.nx;
    const T gam = (T)a.gamma, gm1 = (T)(a.gamma - 1.0), ax = (T)a.ax;
    T inv_h, scl, wpow[NM];
    if constexpr (PR::MIXED) {
      inv_h = a.inv_h_f;
      scl = a.scl_f;
#pragma unroll
      for (int m = 0; m < NM; ++m) wpow[m] = OE ? a.wpoe_f[m] : a.wpow_f[m];
    } else {
      inv_h = a.inv_h_d;
      scl = a.scl_d;
#pragma unroll
      for (int m = 0; m < NM; ++m) wpow[m] = OE ? a.wpoe_d[m] : a.wpow_d[m];
    }
    constexpr int NVO = OE ? NV : 1;
    double osum[NVO];
    T omax[NVO], omin[NVO];
#pragma unroll
    for (int v = 0; v < NVO; ++v) {
      osum[v] = 0.0;
      omax[v] = -INFINITY;
      omin[v] = INFINITY;
    }
    const T c1dt = (T)(a.c1 * dtd), c0 = (T)a.c0;
    // double-float coefficients of the cell-average update (once per item, off the cell path)
    const df dcf = df_from_double(a.c1 * dtd * a.inv_h_d);
    const df dc0 = df{a.c0_hi, a.c0_lo};
    T my_eta = T(0);
    {
      const int x = (int)strip * STRIP_OUT - 2 + lane;
      const bool per = a.bc == BC_PERIODIC;
      const int xc = per ? ((x % nx) + nx) % nx : (x < 0 ? 0 : (x >= nx ? nx - 1 : x));
      // outflow: a lane left or right of the mesh is a ghost cell holding the constant state equal
      // to the adjacent interior cell's average
      const bool ghost = !per && (x < 0 || x >= nx);
      const bool out_lane = lane >= 2 && lane < 2 + STRIP_OUT && x >= 0 && x < nx;
      T u[NV][NM], lo0[NV];
      ST::load(a.uin, a.ncell, xc, u, lo0);
      if (ghost) {
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
          for (int l = 1; l < NM; ++l) u[v][l] = T(0);
      }
      // traces at xi = -1 and +1
      T tl[NV], tr[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T sl = T(0), sr = T(0);
#pragma unroll
        for (int l = 0; l < NM; ++l) {
          sr += u[v][l];
          sl += (l & 1) ? -u[v][l] : u[v][l];
        }
        tl[v] = sl;
        tr[v] = sr;
      }
      // face fluxes: right face by this lane, left face from the left lane
      T nb[NV], FR[NV], FL[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) nb[v] = sd(tl[v], 1);
      llf1d<EQ>(tr, nb, FR, gam, gm1, ax);
#pragma unroll
      for (int v = 0; v < NV; ++v) FL[v] = su(FR[v], 1);
      // volume integral
      T acc[NV][NM];
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int l = 0; l < NM; ++l) acc[v][l] = T(0);
      sfor<NQ>([&](auto Q_) {
        constexpr int q = decltype(Q_)::value;
        T uq[NV], fq[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          T s = u[v][0];
          sfor<NM>([&](auto L_) {
            constexpr int l = decltype(L_)::value;
            constexpr double c = TB::GP[l * NQ + q];
            if constexpr (l >= 1 && c != 0.0) s += u[v][l] * (T)c;
          });
          uq[v] = s;
        }
        flux1d<EQ>(uq, fq, gm1, ax);
#pragma unroll
        for (int v = 0; v < NV; ++v)
          sfor<NM>([&](auto L_) {
            constexpr int l = decltype(L_)::value;
            constexpr double c = TB::WD[l * NQ + q];
            if constexpr (l >= 1 && c != 0.0) acc[v][l] += fq[v] * (T)c;
          });
      });
      T un_[NV][NM], unlo[NV];
      if (a.stage > 0) ST::load(a.un, a.ncell, xc, un_, unlo);
      T ut[NV][NM], ulo[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
#pragma unroll
        for (int l = 0; l < NM; ++l) {
          const T R = (T)(2 * l + 1) * inv_h * (acc[v][l] - FR[v] + ((l & 1) ? -FL[v] : FL[v]));
          if (PR::MIXED && l == 0) continue;
          // u~ = u + c0 (u^n - u) + c1 dt R: equal to c0 u^n + c1 (u + dt R) when c0 + c1 = 1, and
          // it keeps that identity exact whatever the rounding of c0 and c1
          T val = u[v][l] + c1dt * R;
          if (a.stage > 0) val += c0 * (un_[v][l] - u[v][l]);
          ut[v][l] = val;
        }
        ulo[v] = T(0);
        if constexpr (PR::MIXED && !PACK_DF) {
          // cell average in double-float: u0 + c0 (un0 - u0) + c1 dt/h (F_L - F_R)
          // (a cascaded double-float sum; the face terms are formed bitwise alike on both sides)
          df_acc m0{u[v][0], lo0[v]};
          if (a.stage > 0) {
            df_acc d{un_[v][0], unlo[v]};
            d.add(df{-u[v][0], -lo0[v]});
            m0.add(df_mul(dc0, d.result()));
          }
          m0.add_prod(dcf, FL[v]);
          m0.add_prod(dcf, -FR[v]);
          const df r0 = m0.result();
          ut[v][0] = r0.hi;
          ulo[v] = r0.lo;
        }
      }
      if constexpr (PACK_DF) {
        // the same double-float cell averages with variables 0 and 1 in one register pair (each
        // lane performs the scalar operations), variable 2 scalar
        {
          const f2 uh{u[0][0], u[1][0]}, ul{lo0[0], lo0[1]};
          df2_acc m0{uh, ul};
          if (a.stage > 0) {
            df2_acc d{f2{un_[0][0], un_[1][0]}, f2{unlo[0], unlo[1]}};
            d.add(df2{-uh, -ul});
            m0.add(df2_mul(dc0, d.result()));
          }
          m0.add_prod(dcf, f2{FL[0], FL[1]});
          m0.add_prod(dcf, -f2{FR[0], FR[1]});
          const df2 r0 = m0.result();
          ut[0][0] = r0.hi.x;
          ut[1][0] = r0.hi.y;
          ulo[0] = r0.lo.x;
          ulo[1] = r0.lo.y;
        }
        {
          df_acc m0{u[2][0], lo0[2]};
          if (a.stage > 0) {
            df_acc d{un_[2][0], unlo[2]};
            d.add(df{-u[2][0], -lo0[2]});
            m0.add(df_mul(dc0, d.result()));
          }
          m0.add_prod(dcf, FL[2]);
          m0.add_prod(dcf, -FR[2]);
          const df r0 = m0.result();
          ut[2][0] = r0.hi;
          ulo[2] = r0.lo;
        }
      }
      T ub[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) ub[v] = ut[v][0];
      T bx, by, invH;
      bool phys;
      avg_params<EQ, 1>(ub, gam, gm1, ax, ax, bx, by, invH, phys);
      if (a.filter_on) {
        // ghost cells take the constant state of the adjacent interior cell's u~ average
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const T from_right = sd(ut[v][0], 1), from_left = su(ut[v][0], 1);
          if (ghost) {
            ut[v][0] = x < 0 ? from_right : from_left;
#pragma unroll
            for (int l = 1; l < NM; ++l) ut[v][l] = T(0);
          }
        }
        // end derivatives d^r u~ at xi = -1, +1 and the jump at the right face
        T J[NV][NM];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          T jr[NM];
          T f = T(1);                              // (2/h)^r
          sfor<NM>([&](auto R_) {
            constexpr int r = decltype(R_)::value;
            // d^r u~ at xi = +1 and -1: P_l^{(r)}(-1) = (-1)^{l+r} P_l^{(r)}(+1)
            T ev = T(-0.0), od = T(-0.0);
            sfor<NM>([&](auto L_) {
              constexpr int l = decltype(L_)::value;
              constexpr double c = TB::DE[l * (K + 1) + r];
              if constexpr (l >= r && c != 0.0) {
                if constexpr ((l & 1) != 0) od += ut[v][l] * (T)c;
                else ev += ut[v][l] * (T)c;
              }
            });
            T dr = ev + od, dl = ((r & 1) != 0) ? od - ev : ev - od;
            if constexpr (r > 0) f *= scl;
            dl *= f;
            dr *= f;
            const T nbl = sd(dl, 1);
            jr[r] = fabs(nbl - dr);
          });
#pragma unroll
          for (int r = 0; r < NM; ++r) J[v][r] = su(jr[r], 1) + jr[r];
        }
        // sigma^l = beta / (h Hbar) max_v (J_0 + sum_{m<=l} m(m+1) h^m J_m)
        T run[NV], facs[NM];
#pragma unroll
        for (int v = 0; v < NV; ++v) run[v] = J[v][0];
#pragma unroll
        for (int l = 1; l < NM; ++l) {
          T best = T(0);
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            run[v] += wpow[l] * J[v][l];
            best = (run[v] > best || run[v] != run[v]) ? run[v] : best;
            if constexpr (OE) {
              // A_v(l) = beta / h (J_0 + sum_{m<=l} (2m+1)/m! h^m J_m) for the OEDG filter kernel
              if (out_lane) ((T*)a.oe.A)[(long long)(v * K + l - 1) * a.ncell + xc] = bx * inv_h * run[v];
            }
          }
          facs[l] = exp(-(bx * inv_h * invH * best) * dt);
        }
        if (a.filter_on == FILT_GLOBAL) {
          // one coefficient for every mode, from the jumps of all derivative orders (Eq. para:damp)
#pragma unroll
          for (int l = 1; l < NM - 1; ++l) facs[l] = facs[NM - 1];
        }
        if constexpr (OE) {
          // u~ is stored as it is; the reductions for the OEDG coefficient
          if (out_lane) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              osum[v] += (double)ut[v][0] + (double)ulo[v];
#pragma unroll
              for (int g = 0; g < NQ; ++g) {
                T w = T(0);
#pragma unroll
                for (int l = 0; l < NM; ++l) w += ut[v][l] * (T)GR::P(l, g);
                omax[v] = fmax(omax[v], w);
                omin[v] = fmin(omin[v], w);
              }
            }
          }
        } else if (!a.hybrid) {
#pragma unroll
          for (int l = 1; l < NM; ++l)
#pragma unroll
            for (int v = 0; v < NV; ++v) ut[v][l] *= facs[l];
        }
        if (a.hybrid) {
          // Algorithm 1: eta = (|[rho]_{j-1/2}| + |[rho]_{j+1/2}|) / (2 h); u^DG stored as it is
          const T eta = J[0][0] * T(0.5) * inv_h;
          hybrid_record<T, K>(a.hyb, a.ncell, xc, out_lane, eta, facs);
          if (out_lane) my_eta = nan_max(eta, my_eta);
        }
      }
      if constexpr (EQ == EQ_EULER) {
        if (a.positivity && out_lane) positivity_limit(ut, gm1);
      }
      if (out_lane) {
        ST::store(a.uout, a.ncell, xc, ut, ulo);
        if (!phys) my_ok = false;
        if constexpr (PR::MIXED) {
          my_rate_t = nan_max(bx * inv_h, my_rate_t);
          if (a.positivity) my_rate_t = nan_max(point_rate(ut, gam, gm1, a.h), my_rate_t);
        } else {
          const double r = (double)bx / a.h;
          my_rate = (r > my_rate || r != r) ? r : my_rate;
          if (a.positivity) {
            const double rp = (double)point_rate(ut, gam, gm1, a.h);
            my_rate = (rp > my_rate || rp != rp) ? rp : my_rate;
          }
        }
      }
    }
    if (a.hybrid) hybrid_max(a.hyb, my_eta);
    if constexpr (OE) oedg_reduce<NV>(a.oe, osum, omax, omin);
  }

  // The limiter's points: the Gauss points, both ends and, for k = 3, the node 0 of the 3-point
  // Gauss-Lobatto rule (Zhang and Shu's positivity of the averages uses the Lobatto nodes with
  // 2N - 3 >= k; for k = 2 the node 0 is a Gauss node already). Value of P_l at point i.
  static constexpr int NP_LIM = NQ + 2 + ((K >= 2 && NQ % 2 == 0) ? 1 : 0);
  static __device__ __forceinline__ double lim_coef(int i, int l) {
    constexpr carr<double, (K + 1) * NQ> GPT = TB::GP;
    return i < NQ ? GPT[l * NQ + i] : (i == NQ ? ((l & 1) ? -1.0 : 1.0) : (i == NQ + 1 ? 1.0 : GaussRule<1>::P(l, 0)));
  }

  // Max CFL rate beta / h over the positivity limiter's points of one cell: with the limiter on,
  // Zhang and Shu's positivity result for the averages needs the CFL bound on the wave speeds at
  // those points.
  static __device__ T point_rate(const T (&ut)[NV][NM], T gam, T gm1, double h) {
    T best = T(0);
    if constexpr (EQ == EQ_EULER) {
      constexpr int NP = NP_LIM;
      const T th = (T)h;
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T w[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          T x = T(0);
#pragma unroll
          for (int l = 0; l < NM; ++l) {
            const double c = lim_coef(i, l);
            x += (T)c * ut[v][l];
          }
          w[v] = x;
        }
        T bx, by, invH;
        bool ph;
        avg_params<EQ, 1>(w, gam, gm1, T(0), T(0), bx, by, invH, ph);
        best = nan_max(bx / th, best);
      }
    }
    return best;
  }

  // Zhang-Shu positivity-preserving limiter on one cell (after the filter, Section 3.2 of the
  // paper), checked at the limiter's points (lim_coef); averages untouched.
  static __device__ void positivity_limit(T (&ut)[NV][NM], T gm1) {
    if constexpr (EQ == EQ_EULER) {
      constexpr int NP = NP_LIM;
      T ub[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) ub[v] = ut[v][0];
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
      auto coef = [](int i, int l) -> double { return lim_coef(i, l); };
      T rmin = ub[0];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T r = T(0);
#pragma unroll
        for (int l = 0; l < NM; ++l) r += (T)coef(i, l) * ut[0][l];
        rmin = r < rmin ? r : rmin;
      }
      if (rmin < eps_r) {
        const T th1 = (ub[0] - eps_r) / (ub[0] - rmin);
#pragma unroll
        for (int l = 1; l < NM; ++l) ut[0][l] *= th1;
      }
      T th2 = T(1);
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T w[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          T x = T(0);
#pragma unroll
          for (int l = 0; l < NM; ++l) x += (T)coef(i, l) * ut[v][l];
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
          for (int l = 1; l < NM; ++l) ut[v][l] *= th2;
      }
    }
  }

  // Single-instance stage: one warp per strip, step control on the instance's DevScalars.
  static __device__ void run(const Stage1DArgs& a, unsigned char* smem) {
    const StageCtl ctl = stage_begin(a.sc, a.stage, a.cfl);
    if (!ctl.run) return;
    if constexpr (OE) {
      if (blockIdx.x == 0 && threadIdx.x == 0) a.oe.sc->active = 1u;
    }
    double* red = (double*)smem;
    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nwt = (long long)gridDim.x * (blockDim.x >> 5);
    double my_rate = 0.0;
    T my_rate_t = T(0);
    bool my_ok = true;
    // a bounded grid: each warp takes strips gw, gw + nwt, ... so the per-block step control and
    // rate reduction are paid once per block, not once per 28 cells
    for (long long w = gw; w < a.nwarps; w += nwt) item(a, ctl.dt, w, my_rate, my_rate_t, my_ok);
    if constexpr (PR::MIXED) my_rate = (double)my_rate_t;
    stage_end(a.sc, a.stage, my_rate, my_ok, red);
  }
};

template <int K, int EQ, class PR, bool OE = false>
__global__ void __launch_bounds__(256) stage1d_kernel(const Stage1DArgs a) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  Stage1D<K, EQ, PR, OE>::run(a, dyn_smem);
}

}  // namespace dgk
