// dg_batch.cu — batched stepping of many uneven solves (dg_batch_run).
//
// Work decomposition: every solver is an instance; the tile items of an instance are its warp
// strips (1D) or (strip, row-chunk) tiles (2D), exactly the items its own stage kernel would run.
// Instances of one (dimension, degree) class share one grid-stride work-list kernel per stage: a
// warp takes the next item of the class, finds its instance by binary search over the instances'
// first-item offsets, and runs the same item() body as the single-solve kernel with that instance's
// dt and buffers. 2D classes are split by the positivity limiter, so that every instance runs the
// instantiation it runs alone (the one without the limiter code when the limiter is off). Large and small instances therefore share the GPU in proportion to their work.
//
// Step control per instance, without inter-block waits: a begin kernel computes each instance's
// dt from its CFL rate max (clipped to its T_end), the three stage launches follow, and an end
// kernel advances t and the step count. A whole step — begin, the classes' stage kernels as
// parallel graph branches, end — is captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "../../include/dg_probes.h"
#include "solver.h"
#include "stage1d.cuh"

namespace dgk {

struct BatchInst {
  void* buf[3];
  DevScalars* sc;
  long long ncell;
  long long item0;     // first work item of this instance within its class
  int nx, ny, bcx, bcy, H, nstrips, nchunks, filter_on, positivity;
  double hx, hy, gamma, ax, ay, cfl;
  // 1D mesh constants from the host (stage1d_consts)
  double inv_h_d, scl_d, wpow_d[4];
  float inv_h_f, scl_f, wpow_f[4];
  // 2D mesh constants from the host (stage2d_consts)
  Consts2D<float> cf;
  Consts2D<double> cd;
};

struct BatchArgs {
  const BatchInst* inst;   // the class's instances, item0 ascending
  int ninst;
  long long nitems;
  int stage;
  float c0_hi, c0_lo;      // the stage's c0 as a double-float
};

__device__ __forceinline__ int find_inst(const BatchInst* inst, int n, long long w) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (inst[mid].item0 <= w) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Fold one item's rate max and physicality into its instance (lane 0 of the warp).
__device__ __forceinline__ void item_end(const BatchInst& I, int stage, long long step, double r, bool ok) {
  r = warp_max(r);
  const unsigned bad = __ballot_sync(0xffffffffu, !ok);
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicOr(&I.sc->err, ERRB_NONPHYS);
    if (stage == 2) atomic_max_nonneg(&I.sc->rate_bits[(step + 1) & 1], r);
  }
  __syncwarp();
}

// LIM = false: the instantiation without the limiter code, the one a solve without the positivity
// limiter runs alone, so that its batched results equal its solo results bit for bit.
template <int K, int EQ, int B, class PR, bool LIM>
__global__ void __launch_bounds__(256) batch2d_kernel(const BatchArgs b) {
  using S = Stage2D<K, EQ, B, PR, false, LIM>;
  using T = typename PR::T;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  const int wib = threadIdx.x >> 5;
  T* ws = (T*)(dyn_smem + S::warp_bytes() * wib);
  const long long nwt = (long long)gridDim.x * (blockDim.x >> 5);
  // each warp takes a contiguous range of items, so consecutive items mostly belong to one
  // instance and its rate / physicality are folded once per run of items, not once per item
  const long long per = (b.nitems + nwt - 1) / nwt;
  const long long w0 = ((long long)blockIdx.x * (blockDim.x >> 5) + wib) * per;
  const long long w1 = w0 + per < b.nitems ? w0 + per : b.nitems;
  int cur = -1;
  long long cur_step = 0;
  double racc = 0.0;
  bool okacc = true;
  for (long long w = w0; w < w1; ++w) {
    const int ii = find_inst(b.inst, b.ninst, w);
    if (ii != cur) {
      if (cur >= 0) item_end(b.inst[cur], b.stage, cur_step, racc, okacc);
      cur = ii;
      cur_step = ((volatile DevScalars*)b.inst[ii].sc)->step;
      racc = 0.0;
      okacc = true;
    }
    const BatchInst& I = b.inst[ii];
    volatile DevScalars* vs = I.sc;
    if (vs->done | vs->err) continue;
    const long long step = vs->step;
    const double dt = vs->dt;
    const int p = (int)(step & 1);
    Stage2DArgs a;
    a.uin = b.stage == 0 ? I.buf[p] : (b.stage == 1 ? I.buf[1 - p] : I.buf[2]);
    a.un = I.buf[p];
    a.uout = b.stage == 1 ? I.buf[2] : I.buf[1 - p];
    a.nx = I.nx;
    a.ny = I.ny;
    a.ncell = I.ncell;
    a.hx = I.hx;
    a.hy = I.hy;
    a.bcx = I.bcx;
    a.bcy = I.bcy;
    a.c0 = b.stage == 0 ? 0.0 : (b.stage == 1 ? 0.75 : 1.0 / 3.0);
    a.c1 = b.stage == 0 ? 1.0 : (b.stage == 1 ? 0.25 : 2.0 / 3.0);
    a.stage = b.stage;
    a.filter_on = I.filter_on;
    a.gamma = I.gamma;
    a.ax = I.ax;
    a.ay = I.ay;
    a.cfl = I.cfl;
    a.H = I.H;
    a.nstrips = I.nstrips;
    a.nchunks = I.nchunks;
    a.positivity = I.positivity;
    a.hybrid = 0;
    a.hyb = HybridOut{};
    a.sc = I.sc;
    a.cf = I.cf;
    a.cd = I.cd;
    const long long local = w - I.item0;
    double r = 0.0;
    T rt = T(0);
    bool ok = true;
    S::item(a, dt, (int)(local % I.nstrips), (int)(local / I.nstrips), ws, r, rt, ok);
    if constexpr (PR::MIXED) r = (double)rt;
    racc = (r > racc || r != r) ? r : racc;
    okacc = okacc && ok;
  }
  if (cur >= 0) item_end(b.inst[cur], b.stage, cur_step, racc, okacc);
}

template <int K, int EQ, class PR>
__global__ void __launch_bounds__(256) batch1d_kernel(const BatchArgs b) {
  using S = Stage1D<K, EQ, PR>;
  using T = typename PR::T;
  const long long nwt = (long long)gridDim.x * (blockDim.x >> 5);
  // each warp takes a contiguous range of items, so consecutive items mostly belong to one
  // instance and its rate / physicality are folded once per run of items, not once per item
  const long long per = (b.nitems + nwt - 1) / nwt;
  const long long w0 = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * per;
  const long long w1 = w0 + per < b.nitems ? w0 + per : b.nitems;
  int cur = -1;
  long long cur_step = 0;
  double racc = 0.0;
  bool okacc = true;
  for (long long w = w0; w < w1; ++w) {
    const int ii = find_inst(b.inst, b.ninst, w);
    if (ii != cur) {
      if (cur >= 0) item_end(b.inst[cur], b.stage, cur_step, racc, okacc);
      cur = ii;
      cur_step = ((volatile DevScalars*)b.inst[ii].sc)->step;
      racc = 0.0;
      okacc = true;
    }
    const BatchInst& I = b.inst[ii];
    volatile DevScalars* vs = I.sc;
    if (vs->done | vs->err) continue;
    const long long step = vs->step;
    const double dt = vs->dt;
    const int p = (int)(step & 1);
    Stage1DArgs a;
    a.uin = b.stage == 0 ? I.buf[p] : (b.stage == 1 ? I.buf[1 - p] : I.buf[2]);
    a.un = I.buf[p];
    a.uout = b.stage == 1 ? I.buf[2] : I.buf[1 - p];
    a.nx = I.nx;
    a.ncell = I.ncell;
    a.h = I.hx;
    a.bc = I.bcx;
    a.c0 = b.stage == 0 ? 0.0 : (b.stage == 1 ? 0.75 : 1.0 / 3.0);
    a.c1 = b.stage == 0 ? 1.0 : (b.stage == 1 ? 0.25 : 2.0 / 3.0);
    a.stage = b.stage;
    a.filter_on = I.filter_on;
    a.gamma = I.gamma;
    a.ax = I.ax;
    a.cfl = I.cfl;
    a.nwarps = I.nstrips;
    a.positivity = I.positivity;
    a.hybrid = 0;
    a.hyb = HybridOut{};
    a.sc = I.sc;
    a.inv_h_d = I.inv_h_d;
    a.scl_d = I.scl_d;
    a.inv_h_f = I.inv_h_f;
    a.scl_f = I.scl_f;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      a.wpow_d[m] = I.wpow_d[m];
      a.wpow_f[m] = I.wpow_f[m];
    }
    a.c0_hi = b.c0_hi;
    a.c0_lo = b.c0_lo;
    double r = 0.0;
    T rt = T(0);
    bool ok = true;
    S::item(a, dt, w - I.item0, r, rt, ok);
    if constexpr (PR::MIXED) r = (double)rt;
    racc = (r > racc || r != r) ? r : racc;
    okacc = okacc && ok;
  }
  if (cur >= 0) item_end(b.inst[cur], b.stage, cur_step, racc, okacc);
}

#ifndef DG_BATCH_K
// Per-instance dt at the start of a step (the same rule as the single-solve stage 0).
__global__ void batch_begin_kernel(const BatchInst* inst, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  DevScalars* sc = inst[i].sc;
  if (sc->done | sc->err) return;
  const long long step = sc->step;
  const double rate = __longlong_as_double((long long)sc->rate_bits[step & 1]);
  if (!(rate > 0.0) || !isfinite(rate)) {
    sc->err |= ERRB_RATE;
    return;
  }
  const double t = sc->t, T = sc->T_end, dtc = inst[i].cfl / rate;
  const bool last = (t + dtc >= T);
  sc->dt = last ? T - t : dtc;
  sc->is_last = last ? 1u : 0u;
  sc->rate_bits[(step + 1) & 1] = 0ull;
}

// Per-instance step advance at the end of a step (the single-solve last-block rule).
__global__ void batch_end_kernel(const BatchInst* inst, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  DevScalars* sc = inst[i].sc;
  if (sc->done | sc->err) return;
  const double tn = sc->is_last ? sc->T_end : sc->t + sc->dt;
  const long long st = sc->step + 1;
  sc->t = tn;
  sc->step = st;
  sc->done = (tn >= sc->T_end || st >= sc->max_step) ? 1u : 0u;
}


#endif  // !DG_BATCH_K
// ---- persistent batched stepping (dg_batch_run_persistent) ----
// One launch per class runs every step of its instances. The class's work is a queue of items in the
// order (step, stage, instance, item); a warp takes the next queue index with one atomic, waits until
// every item of the instance's earlier stages has finished (a per-instance release counter), runs the
// item and arrives. The last item of an instance's stage releases the next stage; the last of its
// final stage also advances the instance's step (t, step, done) and sets the next step's dt, the work
// of the graph path's end and begin kernels. A wait only ever depends on queue indices taken before
// its own, by warps that are running, so the queue order itself rules out a deadlock; the launch is
// cooperative all the same, and every wait gives up after a bounded number of polls, sets a status
// bit and makes all warps leave.

// Per-instance barrier state (zeroed before the launch).
struct PersistCtl {
  unsigned long long arrived;   // items of this run finished
  unsigned int released;        // stages (phases) of this run whose items have all finished
  unsigned int pad;
};

enum : unsigned { PERSIST_TIMEOUT = 1u };

struct PersistArgs {
  const BatchInst* inst;        // the class's instances, item0 ascending
  PersistCtl* ctl;              // one per instance
  int ninst;
  long long nitems;             // items of one phase (one stage of every instance)
  long long total;              // nitems * 3 * steps
  long long steps;
  unsigned long long* queue;    // next queue index (zeroed)
  unsigned int* status;         // PERSIST_TIMEOUT when a wait gave up
  unsigned int poll_limit;      // polls of a wait before it gives up
};

// Wait until `phase` stages of the instance have finished. False if the wait gave up (or another
// warp's did): the caller leaves.
__device__ __forceinline__ bool persist_wait(const PersistCtl* C, long long phase, unsigned* status,
                                             unsigned poll_limit) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0 && phase > 0) {
    unsigned polls = 0;
    while (*(const volatile unsigned*)&C->released < (unsigned)phase) {
      if (*(volatile unsigned*)status) {
        ok = 0;
        break;
      }
      if (++polls > poll_limit) {
        atomicOr(status, PERSIST_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(256);
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __threadfence();   // the released stage's stores before this item's loads
  return ok != 0;
}

// End of the step of one instance (the graph path's end kernel) and, if another step follows in this
// run, the start of the next (its begin kernel).
__device__ __forceinline__ void persist_step_advance(const BatchInst& I, bool next) {
  volatile DevScalars* sc = I.sc;
  if (sc->done | sc->err) return;
  const double tn = sc->is_last ? sc->T_end : sc->t + sc->dt;
  const long long st = sc->step + 1;
  sc->t = tn;
  sc->step = st;
  const bool done = (tn >= sc->T_end || st >= sc->max_step);
  sc->done = done ? 1u : 0u;
  if (done || !next) return;
  const double rate = __longlong_as_double((long long)sc->rate_bits[st & 1]);
  if (!(rate > 0.0) || !isfinite(rate)) {
    atomicOr(&I.sc->err, ERRB_RATE);
    return;
  }
  const double T = sc->T_end, dtc = I.cfl / rate;
  const bool last = (tn + dtc >= T);
  sc->dt = last ? T - tn : dtc;
  sc->is_last = last ? 1u : 0u;
  sc->rate_bits[(st + 1) & 1] = 0ull;
}

// Arrival of one finished (or skipped) item; the last item of an instance's stage releases it.
__device__ __forceinline__ void persist_arrive(const PersistArgs& P, const BatchInst& I, PersistCtl* C,
                                               long long phase) {
  __threadfence();   // this lane's stores before the arrival
  __syncwarp();
  if ((threadIdx.x & 31) == 0) {
    __threadfence();
    const unsigned long long items = (unsigned long long)I.nstrips * (unsigned long long)I.nchunks;
    const unsigned long long prev = atomicAdd(&C->arrived, 1ull);
    if (prev + 1 == (unsigned long long)(phase + 1) * items) {
      if (phase % 3 == 2) persist_step_advance(I, phase / 3 + 1 < P.steps);
      __threadfence();
      atomicExch(&C->released, (unsigned)(phase + 1));
    }
  }
  __syncwarp();
}

// The queue index a warp takes next (P.total when the queue is empty or a wait gave up).
__device__ __forceinline__ long long persist_take(const PersistArgs& P) {
  long long k = 0;
  if ((threadIdx.x & 31) == 0)
    k = *(volatile unsigned*)P.status ? P.total : (long long)atomicAdd(P.queue, 1ull);
  return __shfl_sync(0xffffffffu, k, 0);
}

template <int K, bool LIM>
__global__ void __launch_bounds__(256) persist2d_kernel(const PersistArgs P) {
  using S = Stage2D<K, EQ_EULER, BASIS_Q, PrecF32M, false, LIM, true>;
  using T = float;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  T* ws = (T*)(dyn_smem + S::warp_bytes() * (threadIdx.x >> 5));
  for (;;) {
    const long long k = persist_take(P);
    if (k >= P.total) break;
    const long long phase = k / P.nitems, w = k - phase * P.nitems;
    const int ii = find_inst(P.inst, P.ninst, w);
    const BatchInst& I = P.inst[ii];
    PersistCtl* C = P.ctl + ii;
    if (!persist_wait(C, phase, P.status, P.poll_limit)) break;
    const int stage = (int)(phase % 3);
    volatile DevScalars* vs = I.sc;
    if (!(vs->done | vs->err)) {
      const long long step = vs->step;
      const double dt = vs->dt;
      const int p = (int)(step & 1);
      Stage2DArgs a;
      a.uin = stage == 0 ? I.buf[p] : (stage == 1 ? I.buf[1 - p] : I.buf[2]);
      a.un = I.buf[p];
      a.uout = stage == 1 ? I.buf[2] : I.buf[1 - p];
      a.nx = I.nx;
      a.ny = I.ny;
      a.ncell = I.ncell;
      a.hx = I.hx;
      a.hy = I.hy;
      a.bcx = I.bcx;
      a.bcy = I.bcy;
      a.c0 = stage == 0 ? 0.0 : (stage == 1 ? 0.75 : 1.0 / 3.0);
      a.c1 = stage == 0 ? 1.0 : (stage == 1 ? 0.25 : 2.0 / 3.0);
      a.stage = stage;
      a.filter_on = I.filter_on;
      a.gamma = I.gamma;
      a.ax = I.ax;
      a.ay = I.ay;
      a.cfl = I.cfl;
      a.H = I.H;
      a.nstrips = I.nstrips;
      a.nchunks = I.nchunks;
      a.positivity = I.positivity;
      a.hybrid = 0;
      a.hyb = HybridOut{};
      a.sc = I.sc;
      a.cf = I.cf;
      a.cd = I.cd;
      const long long local = w - I.item0;
      double r = 0.0;
      T rt = T(0);
      bool ok = true;
      S::item(a, dt, (int)(local % I.nstrips), (int)(local / I.nstrips), ws, r, rt, ok);
      item_end(I, stage, step, (double)rt, ok);
    }
    persist_arrive(P, I, C, phase);
  }
}

template <int K>
__global__ void __launch_bounds__(256) persist1d_kernel(const PersistArgs P) {
  using S = Stage1D<K, EQ_EULER, PrecF32M, false, true>;
  using T = float;
  for (;;) {
    const long long k = persist_take(P);
    if (k >= P.total) break;
    const long long phase = k / P.nitems, w = k - phase * P.nitems;
    const int ii = find_inst(P.inst, P.ninst, w);
    const BatchInst& I = P.inst[ii];
    PersistCtl* C = P.ctl + ii;
    if (!persist_wait(C, phase, P.status, P.poll_limit)) break;
    const int stage = (int)(phase % 3);
    volatile DevScalars* vs = I.sc;
    if (!(vs->done | vs->err)) {
      const long long step = vs->step;
      const double dt = vs->dt;
      const int p = (int)(step & 1);
      Stage1DArgs a;
      a.uin = stage == 0 ? I.buf[p] : (stage == 1 ? I.buf[1 - p] : I.buf[2]);
      a.un = I.buf[p];
      a.uout = stage == 1 ? I.buf[2] : I.buf[1 - p];
      a.nx = I.nx;
      a.ncell = I.ncell;
      a.h = I.hx;
      a.bc = I.bcx;
      a.c0 = stage == 0 ? 0.0 : (stage == 1 ? 0.75 : 1.0 / 3.0);
      a.c1 = stage == 0 ? 1.0 : (stage == 1 ? 0.25 : 2.0 / 3.0);
      a.stage = stage;
      a.filter_on = I.filter_on;
      a.gamma = I.gamma;
      a.ax = I.ax;
      a.cfl = I.cfl;
      a.nwarps = I.nstrips;
      a.positivity = I.positivity;
      a.hybrid = 0;
      a.hyb = HybridOut{};
      a.sc = I.sc;
      a.inv_h_d = I.inv_h_d;
      a.scl_d = I.scl_d;
      a.inv_h_f = I.inv_h_f;
      a.scl_f = I.scl_f;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        a.wpow_d[m] = I.wpow_d[m];
        a.wpow_f[m] = I.wpow_f[m];
      }
      {
        const double c0 = a.c0;
        a.c0_hi = (float)c0;
        a.c0_lo = (float)(c0 - (double)a.c0_hi);
      }
      double r = 0.0;
      T rt = T(0);
      bool ok = true;
      S::item(a, dt, w - I.item0, r, rt, ok);
      item_end(I, stage, step, (double)rt, ok);
    }
    persist_arrive(P, I, C, phase);
  }
}

struct BatchLauncher {
  cudaError_t (*launch)(const BatchArgs&, unsigned grid, unsigned block, size_t smem, cudaStream_t s);
  cudaError_t (*set_smem)(size_t bytes);
  size_t warp_bytes;
  int (*blocks_per_sm)(unsigned block, size_t smem);  // 2D: resident blocks per SM
};

// The persistent kernel of a class and the row-slot bytes per warp it needs (2D; 1D: 0).
struct PersistLauncher {
  const void* fn;
  size_t warp_bytes;
};
// The 2D kernels of degree K (graph path and persistent path, without / with the limiter code) are
// compiled in units of their own (this file with -DDG_BATCH_K=K), in parallel; the main unit reaches
// them through these specialisations.
template <int K, bool LIM>
BatchLauncher make_b2();
template <int K, bool LIM>
PersistLauncher make_p2();
#define DG_BATCH_DECLARE(K)          \
  template <>                        \
  BatchLauncher make_b2<K, false>(); \
  template <>                        \
  BatchLauncher make_b2<K, true>();  \
  template <>                        \
  PersistLauncher make_p2<K, false>(); \
  template <>                        \
  PersistLauncher make_p2<K, true>();
DG_BATCH_DECLARE(1)
DG_BATCH_DECLARE(2)
DG_BATCH_DECLARE(3)
#undef DG_BATCH_DECLARE

#ifdef DG_BATCH_K
template <int K, bool LIM>
static cudaError_t launch_b2(const BatchArgs& b, unsigned g, unsigned bl, size_t sm, cudaStream_t s) {
  batch2d_kernel<K, EQ_EULER, BASIS_Q, PrecF32M, LIM><<<g, bl, sm, s>>>(b);
  return cudaGetLastError();
}
template <int K, bool LIM>
static cudaError_t smem_b2(size_t bytes) {
  return cudaFuncSetAttribute(batch2d_kernel<K, EQ_EULER, BASIS_Q, PrecF32M, LIM>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
template <int K, bool LIM>
static int occ_b2(unsigned block, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch2d_kernel<K, EQ_EULER, BASIS_Q, PrecF32M, LIM>,
                                                    (int)block, smem) != cudaSuccess)
    return 0;
  return n;
}
template <int K, bool LIM>
static BatchLauncher make_b2_impl() {
  return {&launch_b2<K, LIM>, &smem_b2<K, LIM>, Stage2D<K, EQ_EULER, BASIS_Q, PrecF32M, false, LIM>::warp_bytes(),
          &occ_b2<K, LIM>};
}
template <int K, bool LIM>
static PersistLauncher make_p2_impl() {
  return {(const void*)&persist2d_kernel<K, LIM>, Stage2D<K, EQ_EULER, BASIS_Q, PrecF32M, false, LIM, true>::warp_bytes()};
}
template <>
BatchLauncher make_b2<DG_BATCH_K, false>() {
  return make_b2_impl<DG_BATCH_K, false>();
}
template <>
BatchLauncher make_b2<DG_BATCH_K, true>() {
  return make_b2_impl<DG_BATCH_K, true>();
}
template <>
PersistLauncher make_p2<DG_BATCH_K, false>() {
  return make_p2_impl<DG_BATCH_K, false>();
}
template <>
PersistLauncher make_p2<DG_BATCH_K, true>() {
  return make_p2_impl<DG_BATCH_K, true>();
}
#else  // the main unit: 1D kernels and the selection tables
template <int K>
static cudaError_t launch_b1(const BatchArgs& b, unsigned g, unsigned bl, size_t sm, cudaStream_t s) {
  batch1d_kernel<K, EQ_EULER, PrecF32M><<<g, bl, sm, s>>>(b);
  return cudaGetLastError();
}
static cudaError_t smem_none(size_t) { return cudaSuccess; }

// lim: the 2D instantiation with the limiter code (classes of solves with the positivity limiter)
static BatchLauncher batch_launcher(int dim, int K, bool lim) {
  if (dim == 2) {
    switch (K) {
      case 1: return lim ? make_b2<1, true>() : make_b2<1, false>();
      case 2: return lim ? make_b2<2, true>() : make_b2<2, false>();
      case 3: return lim ? make_b2<3, true>() : make_b2<3, false>();
    }
  } else {
    switch (K) {
      case 1: return {&launch_b1<1>, &smem_none, 0, nullptr};
      case 2: return {&launch_b1<2>, &smem_none, 0, nullptr};
      case 3: return {&launch_b1<3>, &smem_none, 0, nullptr};
    }
  }
  return {nullptr, nullptr, 0, nullptr};
}

static PersistLauncher persist_launcher(int dim, int K, bool lim) {
  if (dim == 2) {
    switch (K) {
      case 1: return lim ? make_p2<1, true>() : make_p2<1, false>();
      case 2: return lim ? make_p2<2, true>() : make_p2<2, false>();
      case 3: return lim ? make_p2<3, true>() : make_p2<3, false>();
    }
  } else {
    switch (K) {
      case 1: return {(const void*)&persist1d_kernel<1>, 0};
      case 2: return {(const void*)&persist1d_kernel<2>, 0};
      case 3: return {(const void*)&persist1d_kernel<3>, 0};
    }
  }
  return {nullptr, 0};
}

// Polls of a persistent-kernel wait before it gives up (about a second at 256 ns a poll; a wait
// that is not broken lasts at most one stage of its instance, milliseconds)
constexpr unsigned PERSIST_POLL_LIMIT = 1u << 22;

#endif  // DG_BATCH_K

}  // namespace dgk

#ifndef DG_BATCH_K
using namespace dgk;

static dg_status batch_run(dg_solver* const* solvers, int n, long long steps, bool persistent) {
  if (!solvers || n < 1 || steps < 0) return DG_ERR_ARG;
  if (persistent && steps > (1LL << 30)) return DG_ERR_ARG;   // the stage counters are 32-bit
  int dev0 = -1;
  for (int i = 0; i < n; ++i) {
    const dg_solver* s = solvers[i];
    if (!s) return DG_ERR_ARG;
    if (s->eq != DG_EQ_EULER || s->prec != PREC_F32M || (s->dim == 2 && s->basis != DG_BASIS_Q) || s->hybrid ||
        s->geom.oedg)
      return DG_ERR_UNSUPPORTED;
  }
  if (cudaGetDevice(&dev0) != cudaSuccess) return DG_ERR_CUDA;
  for (int i = 0; i < n; ++i)
    if (solver_pull_control(solvers[i]) != DG_OK) return DG_ERR_CUDA;   // also orders prior work
  if (steps == 0) return DG_OK;

  // classes: 1D degree K -> K - 1; 2D degree K without / with the positivity limiter -> 2 + K,
  // 5 + K (the 2D kernel instantiation a solve runs alone)
  constexpr int NCLS = 9;
  std::vector<BatchInst> host;
  host.reserve(n);
  int cls_begin[NCLS], cls_count[NCLS], cls_wpb[NCLS];
  long long cls_items[NCLS];
  for (int c = 0; c < NCLS; ++c) {
    cls_begin[c] = (int)host.size();
    cls_items[c] = 0;
    cls_wpb[c] = 4;
    const int dim = c < 3 ? 1 : 2, K = c % 3 + 1, lim = c >= 6 ? 1 : 0;
    for (int i = 0; i < n; ++i) {
      const dg_solver* s = solvers[i];
      if (s->dim != dim || s->k != K || (dim == 2 && s->positivity != lim)) continue;
      BatchInst I;
      memset(&I, 0, sizeof(I));
      for (int b = 0; b < 3; ++b) I.buf[b] = s->buf[b];
      I.sc = s->sc;
      I.ncell = s->geom.ncell;
      I.item0 = cls_items[c];
      I.nx = s->mesh.nx;
      I.ny = s->dim == 2 ? s->mesh.ny : 1;
      I.bcx = s->mesh.bc[0];
      I.bcy = s->dim == 2 ? s->mesh.bc[2] : 0;
      I.H = s->dim == 2 ? s->H : 1;
      I.nstrips = s->dim == 2 ? s->nstrips : s->nwarps1d;
      I.nchunks = s->dim == 2 ? s->nchunks : 1;
      I.filter_on = s->filter_on;
      I.positivity = s->positivity;
      I.hx = s->geom.hx;
      I.hy = s->geom.hy;
      I.gamma = s->gamma;
      I.ax = s->ax;
      I.ay = s->ay;
      I.cfl = s->cfl;
      if (s->dim == 2) {
        Stage2DArgs t{};
        t.hx = s->geom.hx;
        t.hy = s->geom.hy;
        t.gamma = s->gamma;
        t.ax = s->ax;
        t.ay = s->ay;
        t.filter_on = s->filter_on;
        stage2d_consts(t);
        I.cf = t.cf;
        I.cd = t.cd;
      }
      {
        Stage1DArgs t{};
        t.h = s->geom.hx;
        stage1d_consts(t);
        I.inv_h_d = t.inv_h_d;
        I.scl_d = t.scl_d;
        I.inv_h_f = t.inv_h_f;
        I.scl_f = t.scl_f;
        for (int m = 0; m < 4; ++m) {
          I.wpow_d[m] = t.wpow_d[m];
          I.wpow_f[m] = t.wpow_f[m];
        }
      }
      cls_items[c] += (long long)I.nstrips * I.nchunks;
      host.push_back(I);
    }
    cls_count[c] = (int)host.size() - cls_begin[c];
    cls_wpb[c] = 4;
  }

  dg_status status = DG_OK;
  cudaStream_t main = solvers[0]->stream;
  BatchInst* dinst = nullptr;
  cudaStream_t side[NCLS] = {};
  cudaEvent_t fork = nullptr, join[NCLS] = {};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaMalloc(&dinst, sizeof(BatchInst) * host.size());
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dinst, host.data(), sizeof(BatchInst) * host.size(), cudaMemcpyHostToDevice, main);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  for (int c = 0; c < NCLS && e == cudaSuccess; ++c) {
    e = cudaStreamCreateWithFlags(&side[c], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[c], cudaEventDisableTiming);
  }
  // 2D classes: the block size with the most resident warps per SM (the row slots of 4, 2, 8 or 1
  // warps within 200 KB of shared memory) and one wave of resident blocks, whose warps then take
  // contiguous item ranges (measured on GB300, 512 uneven instances: 5.9e10 DOF-stage/s against
  // 4.6e10 with the instances' own 4-warp blocks and 4 blocks per SM). 1D classes: 4 blocks of 4
  // warps per SM.
  BatchLauncher BL[NCLS];
  long long cls_cap[NCLS];
  int nsm = 152;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev0) != cudaSuccess || nsm <= 0) nsm = 152;
  for (int c = 0; c < NCLS && e == cudaSuccess; ++c) {
    BL[c] = batch_launcher(c < 3 ? 1 : 2, c % 3 + 1, c >= 6);
    cls_cap[c] = (long long)nsm * 4;
    if (c >= 3 && cls_count[c] > 0) {
      int maxw = (int)((200 * 1024) / BL[c].warp_bytes);
      if (maxw > 8) maxw = 8;
      int best = -1, bw = 1, bb = 1;
      for (int cand : {4, 2, 8, 1}) {
        if (cand > maxw) continue;
        if (BL[c].set_smem(BL[c].warp_bytes * cand) != cudaSuccess) continue;
        const int bps = BL[c].blocks_per_sm(32u * cand, BL[c].warp_bytes * cand);
        if (bps * cand > best) {
          best = bps * cand;
          bw = cand;
          bb = bps;
        }
      }
      cls_wpb[c] = bw;
      cls_cap[c] = (long long)nsm * (bb > 0 ? bb : 1);
    }
    if (cls_count[c] > 0 && BL[c].set_smem) e = BL[c].set_smem(BL[c].warp_bytes * cls_wpb[c]);
  }
  unsigned char* pscr = nullptr;
  bool timed_out = false;
  if (!persistent && e == cudaSuccess) e = cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal);
  if (!persistent && e == cudaSuccess) {
    cudaError_t ce = cudaSuccess;
    const unsigned nb = (unsigned)((host.size() + 127) / 128);
    batch_begin_kernel<<<nb, 128, 0, main>>>(dinst, (int)host.size());
    ce = cudaGetLastError();
    for (int stage = 0; stage < 3 && ce == cudaSuccess; ++stage) {
      ce = cudaEventRecord(fork, main);
      for (int c = 0; c < NCLS && ce == cudaSuccess; ++c) {
        if (cls_count[c] == 0) continue;
        BatchArgs b;
        b.inst = dinst + cls_begin[c];
        b.ninst = cls_count[c];
        b.nitems = cls_items[c];
        b.stage = stage;
        {
          const double c0 = stage == 0 ? 0.0 : (stage == 1 ? 0.75 : 1.0 / 3.0);
          b.c0_hi = (float)c0;
          b.c0_lo = (float)(c0 - (double)b.c0_hi);
        }
        const int wpb = cls_wpb[c];
        long long blocks = (cls_items[c] + wpb - 1) / wpb;
        if (blocks > cls_cap[c]) blocks = cls_cap[c];   // warps then take contiguous item ranges
        ce = cudaStreamWaitEvent(side[c], fork, 0);
        if (ce == cudaSuccess)
          ce = BL[c].launch(b, (unsigned)blocks, 32u * wpb, BL[c].warp_bytes * wpb, side[c]);
        if (ce == cudaSuccess) ce = cudaEventRecord(join[c], side[c]);
      }
      for (int c = 0; c < NCLS && ce == cudaSuccess; ++c)
        if (cls_count[c] > 0) ce = cudaStreamWaitEvent(main, join[c], 0);
    }
    if (ce == cudaSuccess) {
      batch_end_kernel<<<nb, 128, 0, main>>>(dinst, (int)host.size());
      ce = cudaGetLastError();
    }
    e = cudaStreamEndCapture(main, &graph);
    if (ce != cudaSuccess) e = ce;
  }
  if (!persistent) {
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    for (long long i = 0; i < steps && e == cudaSuccess; ++i) e = cudaGraphLaunch(exec, main);
  } else if (e == cudaSuccess) {
    // persistent path: the begin kernel sets the first step's dt, then one cooperative launch per
    // class (classes in parallel) runs all the steps; scratch: the instances' barrier states, the
    // classes' queue counters and the status word
    const size_t ctl_bytes = sizeof(PersistCtl) * host.size();
    const size_t scr = ctl_bytes + sizeof(unsigned long long) * NCLS + 16;
    e = cudaMalloc(&pscr, scr);
    if (e == cudaSuccess) e = cudaMemsetAsync(pscr, 0, scr, main);
    PersistCtl* dctl = (PersistCtl*)pscr;
    unsigned long long* dq = (unsigned long long*)(pscr + ctl_bytes);
    unsigned* dstatus = (unsigned*)(dq + NCLS);
    if (e == cudaSuccess) {
      batch_begin_kernel<<<(unsigned)((host.size() + 127) / 128), 128, 0, main>>>(dinst, (int)host.size());
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(fork, main);
    for (int c = 0; c < NCLS && e == cudaSuccess; ++c) {
      if (cls_count[c] == 0) continue;
      const PersistLauncher PL = persist_launcher(c < 3 ? 1 : 2, c % 3 + 1, c >= 6);
      const int wpb = c < 3 ? 4 : cls_wpb[c];
      const unsigned block = 32u * wpb;
      const size_t smem = PL.warp_bytes * wpb;
      e = cudaFuncSetAttribute(PL.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      int bps = 0;
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, PL.fn, (int)block, smem);
      if (e != cudaSuccess) break;
      if (bps < 1) {
        e = cudaErrorInvalidConfiguration;
        break;
      }
      // all blocks resident (cooperative launch); no more warps than one stage of the class has items
      long long grid = (long long)bps * nsm;
      const long long need = (cls_items[c] + wpb - 1) / wpb;
      if (grid > need) grid = need;
      PersistArgs P;
      P.inst = dinst + cls_begin[c];
      P.ctl = dctl + cls_begin[c];
      P.ninst = cls_count[c];
      P.nitems = cls_items[c];
      P.total = cls_items[c] * 3 * steps;
      P.steps = steps;
      P.queue = dq + c;
      P.status = dstatus;
      P.poll_limit = PERSIST_POLL_LIMIT;
      void* args[] = {&P};
      e = cudaStreamWaitEvent(side[c], fork, 0);
      if (e == cudaSuccess) e = cudaLaunchCooperativeKernel(PL.fn, dim3((unsigned)grid), dim3(block), args, smem, side[c]);
      if (e == cudaSuccess) e = cudaEventRecord(join[c], side[c]);
    }
    for (int c = 0; c < NCLS && e == cudaSuccess; ++c)
      if (cls_count[c] > 0) e = cudaStreamWaitEvent(main, join[c], 0);
    unsigned hstatus = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hstatus, dstatus, sizeof(unsigned), cudaMemcpyDeviceToHost, main);
    if (e == cudaSuccess) e = cudaStreamSynchronize(main);
    timed_out = e == cudaSuccess && (hstatus & PERSIST_TIMEOUT) != 0;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(main);
  if (e != cudaSuccess) status = DG_ERR_CUDA;
  else if (timed_out) status = DG_ERR_TIMEOUT;
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  for (int c = 0; c < NCLS; ++c) {
    if (side[c]) cudaStreamDestroy(side[c]);
    if (join[c]) cudaEventDestroy(join[c]);
  }
  if (fork) cudaEventDestroy(fork);
  if (dinst) cudaFree(dinst);
  if (pscr) cudaFree(pscr);
  if (status != DG_OK) return status;
  int present = 0;
  for (int c = 0; c < NCLS; ++c) present += cls_count[c] > 0;
  // the graph's kernel nodes once per step; the persistent path's begin kernel and class launches
  solvers[0]->launches += persistent ? 1 + present : steps * (2 + 3LL * present);
  for (int i = 0; i < n; ++i) {
    dg_solver* s = solvers[i];
    if (solver_pull_control(s) != DG_OK) return DG_ERR_CUDA;
    if (s->h_sc->err) status = DG_ERR_NONPHYSICAL;
  }
  return status;
}

extern "C" dg_status dg_batch_run(dg_solver* const* solvers, int n, long long steps) {
  return batch_run(solvers, n, steps, false);
}

extern "C" dg_status dg_batch_run_persistent(dg_solver* const* solvers, int n, long long steps) {
  return batch_run(solvers, n, steps, true);
}

// One warp waits on a barrier state that nothing releases (phase 1 of an instance with no items).
__global__ void wait_timeout_probe_kernel(PersistCtl* ctl, unsigned* status, unsigned poll_limit) {
  persist_wait(ctl, 1, status, poll_limit);
}

extern "C" int dg_probe_wait_timeout(unsigned poll_limit, unsigned* status, double* ms) {
  if (!status || !ms || poll_limit > (1u << 24)) return -1;
  unsigned char* d = nullptr;
  if (cudaMalloc(&d, 64) != cudaSuccess) return -2;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, 64, st);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    wait_timeout_probe_kernel<<<1, 32, 0, st>>>((PersistCtl*)d, (unsigned*)(d + 32), poll_limit);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(status, d + 32, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float f = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&f, e0, e1);
  *ms = f;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(d);
  return e == cudaSuccess ? 0 : -6;
}
#endif  // !DG_BATCH_K
