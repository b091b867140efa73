// dg_api.cu — the C ABI (include/dg.h): solver handle, device memory, stage launches, CUDA-graph
// replay of step pairs, device-side step control and state conversion.
//
// Buffers: three state buffers B0, B1, B2. A step starting from B[p] (p = step parity) runs
//   stage 0: B[p] -> B[1-p];  stage 1: (B[1-p], B[p]) -> B2;  stage 2: (B2, B[p]) -> B[1-p]
// so the new state lands in B[1-p] and the input is only read: a failing step leaves the last good
// state where it was. Two consecutive steps form a fixed launch sequence (6 kernels) that is
// captured once into a CUDA graph and replayed; dt, t and the stop condition live on the device.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "../../include/dg.h"
#include "dg_internal.h"
#include "solver.h"
#include "stage1d.cuh"

using namespace dgk;

static thread_local char g_last_err[256] = "";

static dg_status cuda_fail(cudaError_t e, const char* where) {
  snprintf(g_last_err, sizeof(g_last_err), "%s: %s", where, cudaGetErrorString(e));
  return DG_ERR_CUDA;
}
#define CK(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)



extern "C" const char* dg_status_string(int s) {
  switch (s) {
    case DG_OK: return "ok";
    case DG_ERR_ARG: return "invalid argument";
    case DG_ERR_OOM: return "out of device memory";
    case DG_ERR_BUDGET: return "workspace or budget too small";
    case DG_ERR_NONPHYSICAL: return "non-physical or non-finite cell average";
    case DG_ERR_TIMEOUT: return "step limit reached before the target time";
    case DG_ERR_CUDA: return "CUDA error";
    case DG_ERR_STATE: return "call not valid in the current solver state";
    case DG_ERR_UNSUPPORTED: return "configuration not supported by the compiled kernels";
  }
  return "unknown status";
}

extern "C" const char* dg_last_error(void) { return g_last_err; }

extern "C" dg_status dg_params_default(dg_filter_params* p) {
  if (!p) return DG_ERR_ARG;
  memset(p, 0, sizeof(*p));
  p->enabled = 1;
  p->cfl = 0.1;
  p->gamma = 1.4;
  p->adv_speed[0] = 1.0;
  p->adv_speed[1] = 0.0;
  p->basis = DG_BASIS_Q;
  p->nq = 0;
  p->precision = DG_PREC_FP64;
  return DG_OK;
}

static int nvars_of(int dim, int eq) { return eq == DG_EQ_EULER ? (dim == 1 ? 3 : 4) : 1; }
static int nmodes_of(int dim, int k, int basis) {
  if (dim == 1) return k + 1;
  return basis == DG_BASIS_P ? (k + 1) * (k + 2) / 2 : (k + 1) * (k + 1);
}

dg_status dgk::validate_config(const dg_mesh* m, int k, int eq, const dg_filter_params* p) {
  if (!m || !p) return DG_ERR_ARG;
  if (m->dim != 1 && m->dim != 2) return DG_ERR_ARG;
  if (m->nx < 1 || (m->dim == 2 && m->ny < 1)) return DG_ERR_ARG;
  if (!(m->x1 > m->x0) || (m->dim == 2 && !(m->y1 > m->y0))) return DG_ERR_ARG;
  for (int i = 0; i < 2 * m->dim; ++i)
    if (m->bc[i] != DG_BC_PERIODIC && m->bc[i] != DG_BC_OUTFLOW) return DG_ERR_ARG;
  if ((m->bc[0] == DG_BC_PERIODIC) != (m->bc[1] == DG_BC_PERIODIC)) return DG_ERR_ARG;
  if (m->dim == 2 && (m->bc[2] == DG_BC_PERIODIC) != (m->bc[3] == DG_BC_PERIODIC)) return DG_ERR_ARG;
  if (m->bc[0] != m->bc[1] || (m->dim == 2 && m->bc[2] != m->bc[3])) return DG_ERR_UNSUPPORTED;
  if (eq < DG_EQ_ADVECTION || eq > DG_EQ_EULER) return DG_ERR_ARG;
  if (k < 1 || k > 3) return DG_ERR_UNSUPPORTED;
  if (p->nq != 0 && p->nq != k + 1) return DG_ERR_UNSUPPORTED;
  if (p->basis != DG_BASIS_Q && p->basis != DG_BASIS_P) return DG_ERR_ARG;
  if (p->precision != DG_PREC_FP64 && p->precision != DG_PREC_FP32_MIXED) return DG_ERR_ARG;
  if (!(p->cfl > 0.0) || !(p->gamma > 1.0)) return DG_ERR_ARG;
  if ((long long)m->nx * (m->dim == 2 ? m->ny : 1) > (1LL << 31)) return DG_ERR_UNSUPPORTED;
  if (p->hybrid && (!p->enabled || p->positivity)) return DG_ERR_UNSUPPORTED;
  if (p->filter_kind < DG_FILTER_JUMP || p->filter_kind > DG_FILTER_OEDG) return DG_ERR_ARG;
  if (p->hybrid && p->filter_kind != DG_FILTER_JUMP) return DG_ERR_UNSUPPORTED;
  // OEDG form: Burgers and Euler, without the positivity limiter (its coefficient needs the whole
  // stage solution, so the damping runs in a kernel of its own after the stage kernel)
  if (p->enabled && p->filter_kind == DG_FILTER_OEDG && (p->positivity || eq == DG_EQ_ADVECTION))
    return DG_ERR_UNSUPPORTED;
  return DG_OK;
}

dg_status dgk::check_device(char* why, size_t why_len) {
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) {
    snprintf(why, why_len, "cudaGetDevice: %s", cudaGetErrorString(ce));
    return DG_ERR_CUDA;
  }
  int major = 0, minor = 0;
  ce = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (ce != cudaSuccess) {
    snprintf(why, why_len, "cudaDeviceGetAttribute: %s", cudaGetErrorString(ce));
    return DG_ERR_CUDA;
  }
  if (major * 10 + minor != 103) {
    snprintf(why, why_len, "device %d is sm_%d%d; this library is built for sm_103a", dev, major, minor);
    return DG_ERR_CUDA;
  }
  return DG_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

void dgk::fill_geom(AuxGeom& g, const dg_mesh* m, int k, int eq, const dg_filter_params* p) {
  memset(&g, 0, sizeof(g));
  g.dim = m->dim;
  g.nx = m->nx;
  g.ny = m->dim == 2 ? m->ny : 1;
  g.k = k;
  g.eq = eq;
  g.basis = m->dim == 2 ? p->basis : DG_BASIS_Q;
  g.prec = p->precision == DG_PREC_FP64 ? PREC_F64 : PREC_F32M;
  g.nv = nvars_of(m->dim, eq);
  g.nm = nmodes_of(m->dim, k, g.basis);
  g.ncell = (long long)g.nx * g.ny;
  g.x0 = m->x0;
  g.y0 = m->dim == 2 ? m->y0 : 0.0;
  g.hx = (m->x1 - m->x0) / m->nx;
  g.hy = m->dim == 2 ? (m->y1 - m->y0) / m->ny : 1.0;
  g.gamma = p->gamma;
  g.ax = p->adv_speed[0];
  g.ay = p->adv_speed[1];
  g.pp = (p->positivity && eq == DG_EQ_EULER) ? 1 : 0;
  g.hyb = p->hybrid ? 1 : 0;
  g.oedg = (p->enabled && p->filter_kind == DG_FILTER_OEDG) ? 1 : 0;
  int idx = 0;
  if (m->dim == 1) {
    for (int l = 0; l <= k; ++l) { g.mp[l] = l; g.mq[l] = 0; }
  } else {
    for (int q = 0; q <= k; ++q)
      for (int pp = 0; pp <= k; ++pp) {
        if (g.basis == DG_BASIS_P && pp + q > k) continue;
        g.mp[idx] = pp;
        g.mq[idx] = q;
        ++idx;
      }
  }
}

// Layout of the single device allocation.
struct Layout {
  size_t off_buf[3], off_canon, off_part, off_mass, off_sc, off_hy_eta, off_hy_fac, off_hy_list, off_hy_sc,
      off_oe_A, off_oe_sc, total;
};
static Layout layout_of(const AuxGeom& g) {
  Layout L;
  size_t sb = align256(state_bytes(g)), o = 0;
  for (int i = 0; i < 3; ++i) { L.off_buf[i] = o; o += sb; }
  L.off_canon = o;
  if (g.prec != PREC_F64) o += align256(sizeof(double) * (size_t)g.nv * g.nm * g.ncell);
  L.off_part = o;
  o += align256(sizeof(double) * MASS_BLOCKS * 4);
  L.off_mass = o;
  o += 256;
  L.off_sc = o;
  o += align256(sizeof(DevScalars));
  L.off_hy_eta = L.off_hy_fac = L.off_hy_list = L.off_hy_sc = 0;
  if (g.hyb) {
    const size_t ts = g.prec == PREC_F64 ? sizeof(double) : sizeof(float);
    L.off_hy_eta = o;
    o += align256(ts * (size_t)g.ncell);
    L.off_hy_fac = o;
    o += align256(ts * (size_t)hybrid_lmax(g) * g.ncell);
    L.off_hy_list = o;
    o += align256(sizeof(int) * (size_t)g.ncell);
    L.off_hy_sc = o;
    o += align256(sizeof(HybridScalars));
  }
  L.off_oe_A = L.off_oe_sc = 0;
  if (g.oedg) {
    const size_t ts = g.prec == PREC_F64 ? sizeof(double) : sizeof(float);
    L.off_oe_A = o;
    o += align256(ts * (size_t)g.nv * hybrid_lmax(g) * g.ncell);
    L.off_oe_sc = o;
    o += align256(sizeof(OedgScalars));
  }
  L.total = o;
  return L;
}

extern "C" dg_status dg_workspace_size(const dg_mesh* mesh, int degree, int equation,
                                       const dg_filter_params* params, size_t* bytes) {
  dg_status st = validate_config(mesh, degree, equation, params);
  if (st != DG_OK) return st;
  if (!bytes) return DG_ERR_ARG;
  AuxGeom g;
  fill_geom(g, mesh, degree, equation, params);
  *bytes = layout_of(g).total;
  return DG_OK;
}

// One warp per (strip, chunk) item, so a 2D stage launch runs in waves of the resident warps. A
// warp sweeps H + 4 rows (two halo rows on each side): pick the H that minimises waves x (H + 4),
// never below 8 rows (the halo would dominate).
int dgk::default_chunk_rows(const StageLauncher& L, int nstrips, int ny, int wpb, unsigned block, size_t smem) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
    nsm = 152;
  int bps = L.blocks_per_sm ? L.blocks_per_sm(block, smem) : 0;
  if (bps <= 0) bps = 1;
  const long long W = (long long)nsm * bps * wpb;
  long long best = -1;
  int H = 8;
  for (int w = 1; w <= 16; ++w) {
    long long nch = w * W / nstrips;
    if (nch < 1) nch = 1;
    if (nch > ny) nch = ny;
    int h = (int)((ny + nch - 1) / nch);
    if (h < 8) h = 8;
    const long long items = (long long)nstrips * ((ny + h - 1) / h);
    const long long cost = ((items + W - 1) / W) * (h + 4);
    if (best < 0 || cost < best) {
      best = cost;
      H = h;
    }
  }
  return H;
}

// Warps per block when the caller gives none: of 4, 2, 8 and 1 warps (within max_wpb, the row-slot
// limit), the block with the most resident warps per SM; ties keep the earlier candidate.
int dgk::default_block_warps(const StageLauncher& L, int max_wpb) {
  int best = -1, wpb = max_wpb < 4 ? max_wpb : 4;
  for (int c : {4, 2, 8, 1}) {
    if (c > max_wpb) continue;
    const size_t smem = 256 + L.slot_bytes_per_warp * c;
    if (L.set_smem(smem) != cudaSuccess) continue;
    const int bps = L.blocks_per_sm ? L.blocks_per_sm(32u * c, smem) : 0;
    if (bps * c > best) {
      best = bps * c;
      wpb = c;
    }
  }
  return wpb;
}

static dg_status setup_launch(dg_solver* s, int tile_rows, int tile_warps) {
  if (s->dim == 1) {
    s->L = stage1d_launcher(s->k, s->eq, s->prec, s->geom.oedg != 0);
    if (!s->L.launch) return DG_ERR_UNSUPPORTED;
    s->nwarps1d = (s->mesh.nx + STRIP_OUT - 1) / STRIP_OUT;
    s->block = 128;
    // at most 8 blocks of 4 warps per SM (64 registers a thread); warps loop over strips
    long long g1 = (s->nwarps1d + 3) / 4;
    s->grid = (unsigned)(g1 < 152LL * 8 ? g1 : 152LL * 8);
    s->smem = 256;
    return DG_OK;
  }
  // the FP32 form of a solve without the positivity and hybrid limiters runs the kernel compiled
  // without their code (a smaller loop body)
  const bool lean = s->prec == PREC_F32M && !s->positivity && !s->hybrid;
  s->L = s->geom.oedg ? stage2d_oedg_launcher(s->k, s->eq, s->basis, s->prec)
                      : (s->prec == PREC_F64 ? stage2d_f64_launcher(s->k, s->eq, s->basis)
                                             : (lean ? stage2d_f32_lean_launcher(s->k, s->eq, s->basis)
                                                     : stage2d_f32_launcher(s->k, s->eq, s->basis)));
  if (!s->L.launch) return DG_ERR_UNSUPPORTED;
  const int nx = s->mesh.nx, ny = s->mesh.ny;
  s->nstrips = (nx + STRIP_OUT - 1) / STRIP_OUT;
  // warps per block: the caller's, else the block size with the most resident warps; at most the
  // row slots that fit in 200 KB of shared memory
  size_t per_warp = s->L.slot_bytes_per_warp;
  int wpb = (int)((200 * 1024 - 256) / per_warp);
  if (wpb > 8) wpb = 8;
  if (wpb < 1) return DG_ERR_UNSUPPORTED;
  if (tile_warps > 0) {
    if (tile_warps < wpb) wpb = tile_warps;
  } else {
    wpb = default_block_warps(s->L, wpb);
  }
  s->warps_per_block = wpb;
  s->block = 32 * wpb;
  s->smem = 256 + per_warp * wpb;
  CK(s->L.set_smem(s->smem));
  int H = tile_rows > 0 ? tile_rows : default_chunk_rows(s->L, s->nstrips, ny, wpb, s->block, s->smem);
  if (H > ny) H = ny;
  s->H = H;
  s->nchunks = (ny + H - 1) / H;
  long long nw = (long long)s->nstrips * s->nchunks;
  s->grid = (unsigned)((nw + wpb - 1) / wpb);
  return DG_OK;
}

extern "C" dg_status dg_create(const dg_mesh* mesh, int degree, int equation, int flux,
                               const dg_filter_params* params, void* cuda_stream, dg_solver** out) {
  if (!out) return DG_ERR_ARG;
  *out = nullptr;
  dg_status st = validate_config(mesh, degree, equation, params);
  if (st != DG_OK) return st;
  if (flux != DG_FLUX_LLF) return DG_ERR_UNSUPPORTED;
  st = check_device(g_last_err, sizeof(g_last_err));
  if (st != DG_OK) return st;
  cudaError_t ce;
  CK(aux_init_tables());

  dg_solver* s = new (std::nothrow) dg_solver();
  if (!s) return DG_ERR_OOM;
  s->mesh = *mesh;
  if (mesh->dim == 1) { s->mesh.ny = 1; s->mesh.y0 = 0.0; s->mesh.y1 = 1.0; }
  s->k = degree;
  s->eq = equation;
  s->dim = mesh->dim;
  s->basis = mesh->dim == 2 ? params->basis : DG_BASIS_Q;
  s->prec = params->precision == DG_PREC_FP64 ? PREC_F64 : PREC_F32M;
  s->filter_on = params->enabled ? FILT_JUMP + params->filter_kind : FILT_OFF;
  s->positivity = (params->positivity && equation == DG_EQ_EULER) ? 1 : 0;
  s->hybrid = params->hybrid ? 1 : 0;
  s->cfl = params->cfl;
  s->gamma = params->gamma;
  s->ax = params->adv_speed[0];
  s->ay = params->adv_speed[1];
  s->stream = (cudaStream_t)cuda_stream;
  if (!s->stream) {
    // the legacy default stream cannot be captured into a graph: use a private stream instead
    ce = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (ce != cudaSuccess) {
      delete s;
      return cuda_fail(ce, "cudaStreamCreate");
    }
    s->own_stream = true;
  }
  fill_geom(s->geom, mesh, degree, equation, params);
  s->ndof = (size_t)s->geom.nv * s->geom.nm * s->geom.ncell;
  s->sbytes = state_bytes(s->geom);

  st = setup_launch(s, params->tile_rows, params->tile_warps);
  if (st != DG_OK) { dg_destroy(s); return st; }

  Layout Lo = layout_of(s->geom);
  if (params->workspace) {
    if (params->workspace_bytes < Lo.total || ((size_t)params->workspace & 255)) {
      dg_destroy(s);
      return DG_ERR_BUDGET;
    }
    s->mem = params->workspace;
    s->own_mem = false;
  } else {
    ce = cudaMalloc(&s->mem, Lo.total);
    if (ce != cudaSuccess) {
      cudaGetLastError();
      s->mem = nullptr;
      dg_destroy(s);
      snprintf(g_last_err, sizeof(g_last_err), "cudaMalloc(%zu): %s", Lo.total, cudaGetErrorString(ce));
      return DG_ERR_OOM;
    }
    s->own_mem = true;
  }
  s->mem_bytes = Lo.total;
  char* base = (char*)s->mem;
  for (int i = 0; i < 3; ++i) s->buf[i] = base + Lo.off_buf[i];
  s->canon = s->prec == PREC_F64 ? nullptr : (double*)(base + Lo.off_canon);
  s->partials = (double*)(base + Lo.off_part);
  s->dmass = (double*)(base + Lo.off_mass);
  s->sc = (DevScalars*)(base + Lo.off_sc);
  s->hy = HybridOut{};
  if (s->hybrid) {
    s->hy.eta = base + Lo.off_hy_eta;
    s->hy.fac = base + Lo.off_hy_fac;
    s->hy.list = (int*)(base + Lo.off_hy_list);
    s->hy.sc = (HybridScalars*)(base + Lo.off_hy_sc);
  }
  s->oe = OedgOut{};
  if (s->geom.oedg) {
    s->oe.A = base + Lo.off_oe_A;
    s->oe.sc = (OedgScalars*)(base + Lo.off_oe_sc);       // zeroed below: empty sums, max and min
  }
  ce = cudaMallocHost(&s->h_sc, sizeof(DevScalars));
  if (ce != cudaSuccess) {
    s->h_sc = nullptr;
    dg_destroy(s);
    return cuda_fail(ce, "cudaMallocHost");
  }
  memset(s->h_sc, 0, sizeof(DevScalars));
  s->h_sc->T_end = INFINITY;
  s->h_sc->max_step = 1LL << 62;
  ce = cudaMemsetAsync(s->mem, 0, Lo.total, s->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(s->sc, s->h_sc, sizeof(DevScalars), cudaMemcpyHostToDevice, s->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  if (ce != cudaSuccess) {
    dg_destroy(s);
    return cuda_fail(ce, "initialise");
  }
  *out = s;
  return DG_OK;
}

extern "C" dg_status dg_destroy(dg_solver* s) {
  if (!s) return DG_OK;
  if (s->pair_ready) cudaGraphExecDestroy(s->pair_exec);
  cudaStreamSynchronize(s->stream);
  if (s->own_mem && s->mem) cudaFree(s->mem);
  if (s->h_sc) cudaFreeHost(s->h_sc);
  if (s->own_stream) cudaStreamDestroy(s->stream);
  delete s;
  return DG_OK;
}

extern "C" dg_status dg_state_size(const dg_solver* s, size_t* n) {
  if (!s || !n) return DG_ERR_ARG;
  *n = s->ndof;
  return DG_OK;
}

extern "C" dg_status dg_dims(const dg_solver* s, int* nvars, int* nmodes, long long* ncells) {
  if (!s) return DG_ERR_ARG;
  if (nvars) *nvars = s->geom.nv;
  if (nmodes) *nmodes = s->geom.nm;
  if (ncells) *ncells = s->geom.ncell;
  return DG_OK;
}

extern "C" dg_status dg_kernel_launches(const dg_solver* s, long long* launches) {
  if (!s || !launches) return DG_ERR_ARG;
  *launches = s->launches;
  return DG_OK;
}

// Reset the device step control to (t, step 0, no error) and compute the CFL rate of the state in
// B0, all on the stream.
static dg_status reset_control(dg_solver* s, double t) {
  memset(s->h_sc, 0, sizeof(DevScalars));
  s->h_sc->t = t;
  s->h_sc->T_end = INFINITY;
  s->h_sc->max_step = 1LL << 62;
  CK(cudaMemcpyAsync(s->sc, s->h_sc, sizeof(DevScalars), cudaMemcpyHostToDevice, s->stream));
  CK(launch_rate(s->geom, s->buf[0], s->sc, 0, s->stream));
  s->launches += 1;
  s->h_step = 0;
  return DG_OK;
}

// Copy a canonical FP64 state (device pointer) into B0.
static dg_status load_canonical_device(dg_solver* s, const double* dsrc) {
  if (s->prec == PREC_F64) {
    if (dsrc != (const double*)s->buf[0])
      CK(cudaMemcpyAsync(s->buf[0], dsrc, sizeof(double) * s->ndof, cudaMemcpyDeviceToDevice, s->stream));
  } else {
    CK(launch_to_storage(s->geom, dsrc, s->buf[0], s->stream));
    s->launches += 1;
  }
  return DG_OK;
}

extern "C" dg_status dg_set_initial(dg_solver* s, int ic, const double* prm, int nprm, int nq_init) {
  if (!s || (nprm > 0 && !prm) || nprm < 0 || nprm > 20) return DG_ERR_ARG;
  const int need[] = {4, 7, 5, 18, 4};
  if (ic < 0 || ic > 4 || nprm < need[ic]) return DG_ERR_ARG;
  if ((ic == DG_IC_RIEMANN1D || ic == DG_IC_ENTROPY1D) && (s->dim != 1 || s->eq != DG_EQ_EULER)) return DG_ERR_ARG;
  if ((ic == DG_IC_QUADRANT2D || ic == DG_IC_VORTEX2D) && (s->dim != 2 || s->eq != DG_EQ_EULER)) return DG_ERR_ARG;
  if (ic == DG_IC_SINE && s->eq == DG_EQ_EULER) return DG_ERR_ARG;
  int nq = nq_init > 0 ? nq_init : s->k + 3;
  if (nq > 8) return DG_ERR_UNSUPPORTED;
  double* target = s->prec == PREC_F64 ? (double*)s->buf[0] : s->canon;
  CK(launch_project(s->geom, ic, prm, nprm, nq, target, s->stream));
  s->launches += 1;
  dg_status st = load_canonical_device(s, target);
  if (st != DG_OK) return st;
  st = reset_control(s, 0.0);
  if (st != DG_OK) return st;
  CK(cudaStreamSynchronize(s->stream));
  return DG_OK;
}

extern "C" dg_status dg_write_state_device(dg_solver* s, const double* src, size_t n, double t) {
  if (!s || !src || n != s->ndof) return DG_ERR_ARG;
  dg_status st = load_canonical_device(s, src);
  if (st != DG_OK) return st;
  st = reset_control(s, t);
  if (st != DG_OK) return st;
  CK(cudaStreamSynchronize(s->stream));
  return DG_OK;
}

extern "C" dg_status dg_write_state(dg_solver* s, const double* host, size_t n, double t) {
  if (!s || !host || n != s->ndof) return DG_ERR_ARG;
  double* dst = s->prec == PREC_F64 ? (double*)s->buf[0] : s->canon;
  CK(cudaMemcpyAsync(dst, host, sizeof(double) * n, cudaMemcpyHostToDevice, s->stream));
  dg_status st = load_canonical_device(s, dst);
  if (st != DG_OK) return st;
  st = reset_control(s, t);
  if (st != DG_OK) return st;
  CK(cudaStreamSynchronize(s->stream));
  return DG_OK;
}

// Read the device control block (synchronising) and update the host's step record.
static dg_status pull_control(dg_solver* s) {
  CK(cudaMemcpyAsync(s->h_sc, s->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  s->h_step = s->h_sc->step;
  return DG_OK;
}

namespace dgk {
dg_status solver_pull_control(dg_solver* s) { return pull_control(s); }
}  // namespace dgk

static const void* current_state(const dg_solver* s) { return s->buf[s->h_step & 1]; }

extern "C" dg_status dg_read_state_device(const dg_solver* cs, double* dst, size_t n, double* t) {
  dg_solver* s = const_cast<dg_solver*>(cs);   // the solve is unchanged (as dg_read_state)
  if (!s || !dst || n != s->ndof) return DG_ERR_ARG;
  dg_status st = pull_control(s);
  if (st != DG_OK) return st;
  if (s->prec == PREC_F64) {
    CK(cudaMemcpyAsync(dst, current_state(s), sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream));
  } else {
    CK(launch_from_storage(s->geom, current_state(s), dst, s->stream));
    s->launches += 1;
  }
  CK(cudaStreamSynchronize(s->stream));
  if (t) *t = s->h_sc->t;
  return DG_OK;
}

// Reading leaves the solve unchanged; it refreshes the host mirror of the device scalars and uses
// the conversion buffer, which is why the handle is cast to non-const here.
extern "C" dg_status dg_read_state(const dg_solver* cs, double* host, size_t n, double* t) {
  dg_solver* s = const_cast<dg_solver*>(cs);
  if (!s || !host || n != s->ndof) return DG_ERR_ARG;
  dg_status st = pull_control(s);
  if (st != DG_OK) return st;
  if (s->prec == PREC_F64) {
    CK(cudaMemcpyAsync(host, current_state(s), sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
  } else {
    CK(launch_from_storage(s->geom, current_state(s), s->canon, s->stream));
    s->launches += 1;
    CK(cudaMemcpyAsync(host, s->canon, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
  }
  CK(cudaStreamSynchronize(s->stream));
  if (t) *t = s->h_sc->t;
  return DG_OK;
}

// Launch the three stages of one step starting from buffer parity p.
static const double SO_C0[3] = {0.0, 0.75, 1.0 / 3.0};
static const double SO_C1[3] = {1.0, 0.25, 2.0 / 3.0};

static cudaError_t launch_step(dg_solver* s, int p) {
  void* in = s->buf[p];
  void* nx = s->buf[1 - p];
  void* tmp = s->buf[2];
  const void* srcs[3] = {in, nx, tmp};
  void* dsts[3] = {nx, tmp, nx};
  for (int st = 0; st < 3; ++st) {
    cudaError_t e;
    if (s->dim == 1) {
      Stage1DArgs a;
      a.uin = srcs[st];
      a.un = in;
      a.uout = dsts[st];
      a.nx = s->mesh.nx;
      a.ncell = s->geom.ncell;
      a.h = s->geom.hx;
      a.bc = s->mesh.bc[0];
      a.c0 = SO_C0[st];
      a.c1 = SO_C1[st];
      a.stage = st;
      a.filter_on = s->filter_on;
      a.gamma = s->gamma;
      a.ax = s->ax;
      a.cfl = s->cfl;
      a.nwarps = s->nwarps1d;
      a.positivity = s->positivity;
      a.hybrid = s->hybrid;
      a.hyb = s->hy;
      a.oe = s->oe;
      a.sc = s->sc;
      stage1d_consts(a);
      e = s->L.launch(&a, s->grid, s->block, s->smem, s->stream);
    } else {
      Stage2DArgs a;
      a.uin = srcs[st];
      a.un = in;
      a.uout = dsts[st];
      a.nx = s->mesh.nx;
      a.ny = s->mesh.ny;
      a.ncell = s->geom.ncell;
      a.hx = s->geom.hx;
      a.hy = s->geom.hy;
      a.bcx = s->mesh.bc[0];
      a.bcy = s->mesh.bc[2];
      a.c0 = SO_C0[st];
      a.c1 = SO_C1[st];
      a.stage = st;
      a.filter_on = s->filter_on;
      a.gamma = s->gamma;
      a.ax = s->ax;
      a.ay = s->ay;
      a.cfl = s->cfl;
      a.H = s->H;
      a.nstrips = s->nstrips;
      a.nchunks = s->nchunks;
      a.positivity = s->positivity;
      a.hybrid = s->hybrid;
      a.hyb = s->hy;
      a.oe = s->oe;
      a.sc = s->sc;
      stage2d_consts(a);
      e = s->L.launch(&a, s->grid, s->block, s->smem, s->stream);
    }
    if (e != cudaSuccess) return e;
    s->launches += 1;
    if (s->hybrid) {
      // Algorithm 1: blend the troubled cells once max eta of this stage is known
      e = launch_hybrid_blend(s->geom, dsts[st], s->hy, s->stream);
      if (e != cudaSuccess) return e;
      s->launches += 1;
    }
    if (s->geom.oedg) {
      // OEDG: the damping once the stage's normalisers ||u_v - avg u_v||_inf are known
      e = launch_oedg_filter(s->geom, dsts[st], s->oe, s->sc, s->stream);
      if (e != cudaSuccess) return e;
      s->launches += 1;
    }
  }
  return cudaSuccess;
}

static dg_status ensure_pair_graph(dg_solver* s) {
  if (s->pair_ready) return DG_OK;
  cudaGraph_t g;
  const long long saved = s->launches;
  CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e1 = launch_step(s, 0);
  cudaError_t e2 = e1 == cudaSuccess ? launch_step(s, 1) : e1;
  cudaError_t e3 = cudaStreamEndCapture(s->stream, &g);
  s->pair_launches = s->launches - saved;
  s->launches = saved;
  if (e2 != cudaSuccess) return cuda_fail(e2, "capture step pair");
  if (e3 != cudaSuccess) return cuda_fail(e3, "cudaStreamEndCapture");
  cudaError_t e4 = cudaGraphInstantiate(&s->pair_exec, g, 0);
  cudaGraphDestroy(g);
  if (e4 != cudaSuccess) return cuda_fail(e4, "cudaGraphInstantiate");
  s->pair_ready = true;
  return DG_OK;
}

// Set the device stop condition (stop at T, or after nsteps more steps) without touching t, step
// or the rate.
static dg_status set_target(dg_solver* s, double T, long long nsteps) {
  dg_status st = pull_control(s);
  if (st != DG_OK) return st;
  if (s->h_sc->err) return DG_ERR_NONPHYSICAL;
  const long long max_step = s->h_sc->step + nsteps;
  s->h_sc->T_end = T;
  s->h_sc->max_step = max_step;
  s->h_sc->done = (s->h_sc->t >= T || s->h_sc->step >= max_step) ? 1u : 0u;
  CK(cudaMemcpyAsync(s->sc, s->h_sc, sizeof(DevScalars), cudaMemcpyHostToDevice, s->stream));
  return DG_OK;
}

// Enqueue n steps assuming the host step record is exact (no early stop expected).
static dg_status enqueue_steps(dg_solver* s, long long n) {
  dg_status st = ensure_pair_graph(s);
  if (st != DG_OK) return st;
  long long left = n;
  if (left > 0 && (s->h_step & 1)) {
    CK(launch_step(s, 1));
    s->h_step += 1;
    --left;
  }
  while (left >= 2) {
    CK(cudaGraphLaunch(s->pair_exec, s->stream));
    s->launches += s->pair_launches;
    s->h_step += 2;
    left -= 2;
  }
  if (left == 1) {
    CK(launch_step(s, 0));
    s->h_step += 1;
  }
  return DG_OK;
}

extern "C" dg_status dg_step(dg_solver* s, double* dt_taken) {
  if (!s) return DG_ERR_ARG;
  dg_status st = set_target(s, INFINITY, 1);
  if (st != DG_OK) return st;
  CK(launch_step(s, (int)(s->h_step & 1)));
  st = pull_control(s);
  if (st != DG_OK) return st;
  if (s->h_sc->err) return DG_ERR_NONPHYSICAL;
  if (dt_taken) *dt_taken = s->h_sc->dt;
  return DG_OK;
}

extern "C" dg_status dg_set_target(dg_solver* s, double T_end, long long max_steps) {
  if (!s || max_steps < 0 || !(T_end == T_end)) return DG_ERR_ARG;
  return set_target(s, T_end, max_steps);
}

extern "C" dg_status dg_advance_steps(dg_solver* s, long long nsteps) {
  if (!s || nsteps < 0) return DG_ERR_ARG;
  dg_status st = set_target(s, INFINITY, nsteps);
  if (st != DG_OK) return st;
  return enqueue_steps(s, nsteps);
}

extern "C" dg_status dg_sync(dg_solver* s, double* t, long long* steps) {
  if (!s) return DG_ERR_ARG;
  dg_status st = pull_control(s);
  if (st != DG_OK) return st;
  if (t) *t = s->h_sc->t;
  if (steps) *steps = s->h_sc->step;
  if (s->h_sc->err) return DG_ERR_NONPHYSICAL;
  return DG_OK;
}

extern "C" dg_status dg_advance_to(dg_solver* s, double T, long long max_steps, long long* steps_taken) {
  if (!s || max_steps < 0 || !(T == T)) return DG_ERR_ARG;
  dg_status st = pull_control(s);
  if (st != DG_OK) return st;
  const long long step0 = s->h_sc->step;
  st = set_target(s, T, max_steps);
  if (st != DG_OK) return st;
  long long chunk = 8;
  for (;;) {
    if (s->h_sc->done || s->h_sc->err) break;
    long long room = step0 + max_steps - s->h_step;
    long long n = chunk < room ? chunk : room;
    if (n <= 0) break;
    // steps past T are no-ops on the device; the parity record is refreshed by pull_control
    st = enqueue_steps(s, n);
    if (st != DG_OK) return st;
    st = pull_control(s);
    if (st != DG_OK) return st;
    if (chunk < 4096) chunk *= 2;
  }
  if (steps_taken) *steps_taken = s->h_sc->step - step0;
  if (s->h_sc->err) return DG_ERR_NONPHYSICAL;
  if (s->h_sc->t < T) return DG_ERR_TIMEOUT;
  return DG_OK;
}

extern "C" dg_status dg_mass(dg_solver* s, double* mass) {
  if (!s || !mass) return DG_ERR_ARG;
  dg_status st = pull_control(s);
  if (st != DG_OK) return st;
  CK(launch_mass(s->geom, current_state(s), s->partials, s->dmass, s->stream));
  s->launches += 2;
  CK(cudaMemcpyAsync(mass, s->dmass, sizeof(double) * s->geom.nv, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return DG_OK;
}
