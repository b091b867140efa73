// stage_common.cuh — step control shared by the 1D and 2D stage kernels.
//
// One SSP-RK3 step (Shu–Osher form, Eq. rkdg1 / err_rk1) is three stage launches:
//   stage 0: u1 = F(u^n + dt L(u^n))
//   stage 1: u2 = F(3/4 u^n + 1/4 (u1 + dt L(u1)))
//   stage 2: u^{n+1} = F(1/3 u^n + 2/3 (u2 + dt L(u2)))
// with F the jump filter (Eq. err_rk2). dt = CFL / (max rate over cells at cell averages of u^n)
// (the CFL condition of Theorem 2.1), clipped so that the last step lands on T_end. The rate max of
// u^{n+1} is reduced inside stage 2 (the filter leaves cell averages unchanged), so the next step's
// dt never travels to the host.
//
// Protocol on DevScalars (no spin-waits anywhere):
//   - every stage kernel returns at once if done or err is set (values fixed during the launch);
//   - stage 0: all threads compute the same dt from (t, T_end, rate_bits[step & 1]); block 0
//     publishes dt and is_last, clears rate_bits[(step + 1) & 1] and the last-block counter;
//   - stage 2: every block atomically maxes its rate into rate_bits[(step + 1) & 1], then counts
//     itself done; the last block (threadfence reduction) advances t and step, and sets done.
#pragma once
#include "dg_device.cuh"

namespace dgk {

// Compile-time tables of the tensor-product sum factorisation for degree K, basis BASIS (P^k drops
// the modes p + q > k). All are evaluated by the compiler front end and read only in constant
// expressions, so every coefficient the kernels multiply by is an immediate.
template <int K, int BASIS>
struct Tab2DBuild {
  using MB = Modes<K, BASIS>;
  using GR = GaussRule<K + 1>;
  static constexpr int NQ = K + 1;
  static constexpr int NM = MB::NM;

  static constexpr carr<int, (K + 1) * (K + 1)> mi() {
    carr<int, (K + 1) * (K + 1)> t{};
    for (int i = 0; i < (K + 1) * (K + 1); ++i) t[i] = -1;
    for (int m = 0; m < NM; ++m) t[MB::p(m) * (K + 1) + MB::q(m)] = m;
    return t;
  }
  static constexpr carr<int, NM> pq(int which) {
    carr<int, NM> t{};
    for (int m = 0; m < NM; ++m) t[m] = which == 0 ? MB::p(m) : MB::q(m);
    return t;
  }
  // [l * NQ + g]: P_l(x_g) (0), w_g P_l(x_g) (1), w_g P_l'(x_g) (2)
  static constexpr carr<double, (K + 1) * NQ> gauss(int which) {
    carr<double, (K + 1) * NQ> t{};
    for (int l = 0; l <= K; ++l)
      for (int g = 0; g < NQ; ++g)
        t[l * NQ + g] = which == 0 ? GR::P(l, g) : (which == 1 ? GR::w(g) * GR::P(l, g) : GR::w(g) * GR::dP(l, g));
    return t;
  }
  // [l * (K + 1) + r]: P_l^{(r)}(+1), zero for r > l
  static constexpr carr<double, (K + 1) * (K + 1)> ends() {
    carr<double, (K + 1) * (K + 1)> t{};
    for (int l = 0; l <= K; ++l)
      for (int r = 0; r <= K; ++r) t[l * (K + 1) + r] = dend(1, l, r);
    return t;
  }
  static constexpr carr<double, NM> minv() {
    carr<double, NM> t{};
    for (int m = 0; m < NM; ++m) t[m] = 0.5 * (2 * MB::p(m) + 1) * (2 * MB::q(m) + 1);
    return t;
  }
};

template <int K, int BASIS>
struct Tab2D {
  using B = Tab2DBuild<K, BASIS>;
  static constexpr int NQ = K + 1;
  static constexpr int NM = B::NM;
  static constexpr carr<int, (K + 1) * (K + 1)> MIX = B::mi();
  static constexpr carr<int, NM> PP = B::pq(0);
  static constexpr carr<int, NM> QQ = B::pq(1);
  static constexpr carr<double, (K + 1) * NQ> GP = B::gauss(0);
  static constexpr carr<double, (K + 1) * NQ> WP = B::gauss(1);
  static constexpr carr<double, (K + 1) * NQ> WD = B::gauss(2);
  static constexpr carr<double, (K + 1) * (K + 1)> DE = B::ends();
  static constexpr carr<double, NM> MINV = B::minv();

  static constexpr bool has(int p, int q) { return p <= K && q <= K && MIX[p * (K + 1) + q] >= 0; }
  // a mode (p, q) with q of parity `par` (p fixed) / p of parity `par` (q fixed), index >= 1
  static constexpr bool any_q_par(int p, int par) {
    for (int q = 1; q <= K; ++q)
      if ((q & 1) == par && has(p, q)) return true;
    return false;
  }
  static constexpr bool any_p_par(int q, int par) {
    for (int p = 1; p <= K; ++p)
      if ((p & 1) == par && has(p, q)) return true;
    return false;
  }
  // sum_q u[p,q] P_q^{(a2)}(+1) has terms of parity par in q (q >= a2)
  static constexpr bool hq(int p, int a2, int par) {
    for (int q = a2; q <= K; ++q)
      if ((q & 1) == par && has(p, q) && DE[q * (K + 1) + a2] != 0.0) return true;
    return false;
  }
  // the x-polynomial H[p][a2] exists (some q >= a2 with mode (p, q))
  static constexpr bool hh(int p, int a2) { return hq(p, a2, 0) || hq(p, a2, 1); }
  // sum_p H[p][a2] P_p^{(a1)}(+1) has terms of parity par in p
  static constexpr bool hp(int a1, int a2, int par) {
    for (int p = a1; p <= K; ++p)
      if ((p & 1) == par && hh(p, a2) && DE[p * (K + 1) + a1] != 0.0) return true;
    return false;
  }
  // derivative multi-indices alpha = (a1, a2) that can be nonzero
  static constexpr bool alpha_ok(int a1, int a2) { return BASIS == BASIS_Q ? true : a1 + a2 <= K; }
};


struct StageCtl {
  bool run;
  double dt;
};

__device__ __forceinline__ StageCtl stage_begin(DevScalars* sc, int stage, double cfl) {
  volatile DevScalars* vs = sc;
  StageCtl c{false, 0.0};
  if (vs->done | vs->err) return c;
  if (stage == 0) {
    long long step = vs->step;
    double rate = __longlong_as_double((long long)vs->rate_bits[step & 1]);
    if (!(rate > 0.0) || !isfinite(rate)) {
      if (threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0) atomicOr(&sc->err, ERRB_RATE);
      return c;
    }
    double t = vs->t, T = vs->T_end;
    double dtc = cfl / rate;
    bool last = (t + dtc >= T);
    c.dt = last ? T - t : dtc;
    if (threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0) {
      sc->dt = c.dt;
      sc->is_last = last ? 1u : 0u;
      sc->rate_bits[(step + 1) & 1] = 0ull;
      sc->blocks_done = 0u;
    }
  } else {
    c.dt = vs->dt;
  }
  c.run = true;
  return c;
}

// Block-level end of a stage: publish non-physical flags; in the final stage also the rate max
// and the last-block step advance. Every thread of the block must call it (uses __syncthreads).
__device__ __forceinline__ void stage_end(DevScalars* sc, int stage, double my_rate, bool my_ok,
                                          double* red_buf /* >= 32 doubles of shared memory */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  double r = warp_max(my_rate);
  unsigned bad = __ballot_sync(0xffffffffu, !my_ok);
  __shared__ unsigned s_bad;
  __shared__ bool s_last;
  if (threadIdx.x == 0) s_bad = 0u;
  __syncthreads();
  if (lane == 0) {
    red_buf[wid] = r;
    if (bad) atomicOr(&s_bad, 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < nw; ++w) m = (red_buf[w] > m || red_buf[w] != red_buf[w]) ? red_buf[w] : m;
    if (s_bad) atomicOr(&sc->err, ERRB_NONPHYS);
    s_last = false;
    if (stage == 2) {
      long long step = ((volatile DevScalars*)sc)->step;
      atomic_max_nonneg(&sc->rate_bits[(step + 1) & 1], m);
      __threadfence();
      unsigned nblocks = gridDim.x * gridDim.y;
      unsigned prev = atomicAdd(&sc->blocks_done, 1u);
      s_last = (prev == nblocks - 1);
    }
  }
  __syncthreads();
  if (stage == 2 && s_last && threadIdx.x == 0) {
    __threadfence();
    volatile DevScalars* vs = sc;
    if (vs->err == 0u) {
      double t = vs->t;
      double tn = vs->is_last ? vs->T_end : t + vs->dt;
      long long st = vs->step + 1;
      vs->t = tn;
      vs->step = st;
      vs->done = (tn >= vs->T_end || st >= vs->max_step) ? 1u : 0u;
    }
  }
}

// Hybrid limiter (Algorithm 1), one row of output cells of a warp: eta and the filter factors of the
// lanes that own an output cell go to the scratch arrays, the troubled ones (eta > 1) are appended
// to the list. Called by every lane of the warp (ballot).
template <class T, int LMAX>
__device__ __forceinline__ void hybrid_record(const HybridOut& h, long long ncell, long long cell, bool active,
                                              T eta, const T (&fac)[LMAX + 1]) {
  const int lane = threadIdx.x & 31;
  if (active) {
    ((T*)h.eta)[cell] = eta;
#pragma unroll
    for (int l = 1; l <= LMAX; ++l) ((T*)h.fac)[(long long)(l - 1) * ncell + cell] = fac[l];
  }
  const bool tr = active && eta > T(1);
  const unsigned mask = __ballot_sync(0xffffffffu, tr);
  if (mask) {
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(&h.sc->count, (unsigned)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (tr) h.list[base + __popc(mask & ((1u << lane) - 1u))] = (int)cell;
  }
}

// OEDG: the warp's sums of cell averages and its largest / smallest point values into the stage's
// reductions (called by every lane; lanes without output cells hold 0, -inf, +inf).
template <int NV, class T>
__device__ __forceinline__ void oedg_reduce(const OedgOut& o, const double (&sum)[NV], const T (&mx)[NV],
                                            const T (&mn)[NV]) {
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double s = sum[v], a = (double)mx[v], b = (double)mn[v];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      s += __shfl_xor_sync(0xffffffffu, s, off);
      a = fmax(a, __shfl_xor_sync(0xffffffffu, a, off));
      b = fmin(b, __shfl_xor_sync(0xffffffffu, b, off));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&o.sc->sum[v], s);
      atomicMax(&o.sc->maxb[v], ordered_bits(a));
      atomicMax(&o.sc->nminb[v], ~ordered_bits(b));
    }
  }
}

// The warp's largest eta into the stage maximum (called by every lane).
template <class T>
__device__ __forceinline__ void hybrid_max(const HybridOut& h, T my_eta) {
  const double m = warp_max((double)my_eta);
  if ((threadIdx.x & 31) == 0 && !(m <= 0.0)) atomic_max_nonneg(&h.sc->max_bits, m);
}

}  // namespace dgk
