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

// The warp's largest eta into the stage maximum (called by every lane).
template <class T>
__device__ __forceinline__ void hybrid_max(const HybridOut& h, T my_eta) {
  const double m = warp_max((double)my_eta);
  if ((threadIdx.x & 31) == 0 && !(m <= 0.0)) atomic_max_nonneg(&h.sc->max_bits, m);
}

}  // namespace dgk
