// dg_noalloc.cu — dg_step_noalloc: one FP64 SSP-RK3 step with the jump filter that allocates no
// device memory.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they want a step — code that
// runs while a stream is being captured into a CUDA graph or inside a framework that owns every
// byte of device memory through a pre-planned arena, and latency-critical loops that must not pay
// for (or implicitly synchronise on) an allocation. They pass the input and output states; the
// two intermediate stage states and the step-control scalars live in one file-scope device array.
//
// The array: NOALLOC_SCRATCH_BYTES (32 MiB + 256 B) of static device memory, reserved on every GPU
// that loads this library until the process exits. Host code cannot use the array's name as a
// device address, so the first call on each device (with that device current) sets the device up
// once: it checks that the device is an sm_103 GPU, copies the Gauss rules that the initial
// CFL-rate kernel reads into the device's constant memory, and looks the array's address up with
// cudaGetSymbolAddress, caching it; make that first call outside any stream capture. The cached
// address belongs to the device's context of that moment: after a cudaDeviceReset in the same
// process it is stale, so no further call may be made on that device. All calls share the array
// and it keeps the last call's contents: each call clears the scalars it needs, and two calls whose
// kernels overlap on the GPU (different streams, no ordering) race on the array and give undefined
// results.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "../../include/dg.h"
#include "dg_internal.h"
#include "stage1d.cuh"

using namespace dgk;

namespace {

constexpr size_t NOALLOC_STATE_BYTES = (size_t)32 << 20;       // two stage states together
constexpr size_t NOALLOC_SCRATCH_BYTES = NOALLOC_STATE_BYTES + 256;  // + the scalars
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

void* g_scratch_addr[MAX_DEVICES];  // device address of g_noalloc_scratch, per device

__global__ void noalloc_reset(DevScalars* sc) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    sc->t = 0.0;
    sc->T_end = INFINITY;
    sc->dt = 0.0;
    sc->rate_bits[0] = 0ull;
    sc->rate_bits[1] = 0ull;
    sc->step = 0;
    sc->max_step = 1;
    sc->done = 0u;
    sc->err = 0u;
    sc->blocks_done = 0u;
    sc->is_last = 0u;
  }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" dg_status dg_step_noalloc(const dg_mesh* m, int k, int eq, const dg_filter_params* p,
                                     const double* u_in, double* u_out, double* dt_taken,
                                     void* cuda_stream) {
  const dg_status vs = validate_config(m, k, eq, p);   // the checks dg_create makes
  if (vs != DG_OK) return vs;
  if (!u_in || !u_out || u_in == u_out) return DG_ERR_ARG;
  if (p->precision != DG_PREC_FP64 || p->hybrid) return DG_ERR_UNSUPPORTED;
  if (p->enabled && p->filter_kind == DG_FILTER_OEDG) return DG_ERR_UNSUPPORTED;   // needs scratch of its own
  AuxGeom g;
  fill_geom(g, m, k, eq, p);
  const int dim = m->dim;
  const int basis = g.basis;
  const long long ncell = g.ncell;
  const size_t sbytes = align256(state_bytes(g));
  if (2 * sbytes > NOALLOC_STATE_BYTES) return DG_ERR_BUDGET;   // mesh too large for the array

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return DG_ERR_CUDA;
  if (!g_scratch_addr[dev]) {
    // once per device: an sm_103 GPU, the Gauss rules in constant memory, the array's address
    char why[128];
    if (check_device(why, sizeof(why)) != DG_OK) return DG_ERR_CUDA;
    if (aux_init_tables() != cudaSuccess) return DG_ERR_CUDA;
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return DG_ERR_CUDA;
    g_scratch_addr[dev] = ptr;
  }
  char* base = (char*)g_scratch_addr[dev];
  DevScalars* sc = (DevScalars*)(base + NOALLOC_STATE_BYTES);
  void* b1 = base;
  void* b2 = base + sbytes;
  cudaStream_t st = (cudaStream_t)cuda_stream;

  noalloc_reset<<<1, 32, 0, st>>>(sc);
  if (cudaGetLastError() != cudaSuccess) return DG_ERR_CUDA;
  if (launch_rate(g, u_in, sc, 0, st) != cudaSuccess) return DG_ERR_CUDA;

  static const double C0[3] = {0.0, 0.75, 1.0 / 3.0};
  static const double C1[3] = {1.0, 0.25, 2.0 / 3.0};
  const void* srcs[3] = {u_in, b1, b2};
  void* dsts[3] = {b1, b2, u_out};
  if (dim == 1) {
    StageLauncher L = stage1d_launcher(k, eq, PREC_F64);
    if (!L.launch) return DG_ERR_UNSUPPORTED;
    const int nwarps = (m->nx + STRIP_OUT - 1) / STRIP_OUT;
    for (int s = 0; s < 3; ++s) {
      Stage1DArgs a;
      a.uin = srcs[s];
      a.un = u_in;
      a.uout = dsts[s];
      a.nx = m->nx;
      a.ncell = ncell;
      a.h = g.hx;
      a.bc = m->bc[0];
      a.c0 = C0[s];
      a.c1 = C1[s];
      a.stage = s;
      a.filter_on = p->enabled ? FILT_JUMP + p->filter_kind : FILT_OFF;
      a.gamma = p->gamma;
      a.ax = p->adv_speed[0];
      a.cfl = p->cfl;
      a.nwarps = nwarps;
      a.positivity = (p->positivity && eq == DG_EQ_EULER) ? 1 : 0;
      a.hybrid = 0;
      a.hyb = HybridOut{};
      a.sc = sc;
      stage1d_consts(a);
      if (L.launch(&a, (unsigned)((nwarps + 3) / 4), 128, 256, st) != cudaSuccess) return DG_ERR_CUDA;
    }
  } else {
    StageLauncher L = stage2d_f64_launcher(k, eq, basis);
    if (!L.launch) return DG_ERR_UNSUPPORTED;
    const int nstrips = (m->nx + STRIP_OUT - 1) / STRIP_OUT;
    int wpb = (int)((200 * 1024 - 256) / L.slot_bytes_per_warp);
    if (wpb > 8) wpb = 8;
    if (wpb < 1) return DG_ERR_UNSUPPORTED;
    wpb = default_block_warps(L, wpb);
    const size_t smem = 256 + L.slot_bytes_per_warp * wpb;
    if (L.set_smem(smem) != cudaSuccess) return DG_ERR_CUDA;
    int H = default_chunk_rows(L, nstrips, m->ny, wpb, 32u * wpb, smem);
    if (H > m->ny) H = m->ny;
    const int nchunks = (m->ny + H - 1) / H;
    const long long nw = (long long)nstrips * nchunks;
    for (int s = 0; s < 3; ++s) {
      Stage2DArgs a;
      a.uin = srcs[s];
      a.un = u_in;
      a.uout = dsts[s];
      a.nx = m->nx;
      a.ny = m->ny;
      a.ncell = ncell;
      a.hx = g.hx;
      a.hy = g.hy;
      a.bcx = m->bc[0];
      a.bcy = m->bc[2];
      a.c0 = C0[s];
      a.c1 = C1[s];
      a.stage = s;
      a.filter_on = p->enabled ? FILT_JUMP + p->filter_kind : FILT_OFF;
      a.gamma = p->gamma;
      a.ax = p->adv_speed[0];
      a.ay = p->adv_speed[1];
      a.cfl = p->cfl;
      a.H = H;
      a.nstrips = nstrips;
      a.nchunks = nchunks;
      a.positivity = (p->positivity && eq == DG_EQ_EULER) ? 1 : 0;
      a.hybrid = 0;
      a.hyb = HybridOut{};
      a.sc = sc;
      stage2d_consts(a);
      if (L.launch(&a, (unsigned)((nw + wpb - 1) / wpb), 32 * wpb, smem, st) != cudaSuccess) return DG_ERR_CUDA;
    }
  }
  if (dt_taken) {
    DevScalars h;
    if (cudaMemcpyAsync(&h, sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, st) != cudaSuccess) return DG_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return DG_ERR_CUDA;
    if (h.err) return DG_ERR_NONPHYSICAL;
    *dt_taken = h.dt;
  }
  return DG_OK;
}
