// dg_internal.h — host-side pieces shared by the C-ABI implementation and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/dg.h"
#include "dg_device.cuh"

namespace dgk {

enum { PREC_F64 = 0, PREC_F32M = 1 };

// Type-erased launcher of one stage-kernel instantiation.
struct StageLauncher {
  // launch(args, grid, block, dynamic smem bytes, stream)
  cudaError_t (*launch)(const void* args, unsigned grid, unsigned block, size_t smem, cudaStream_t s);
  cudaError_t (*set_smem)(size_t bytes);  // raise the dynamic shared-memory limit
  size_t slot_bytes_per_warp;             // 2D: per-warp row slots; 1D: 0
  // resident blocks per SM for a block size and dynamic shared memory (2D; 0 if unknown)
  int (*blocks_per_sm)(unsigned block, size_t smem);
};

// Rows per chunk of the 2D stage kernel when the caller gives none: the fewest waves of resident
// warps times the rows a warp sweeps (H + 4 halo rows). Queries the current device.
int default_chunk_rows(const StageLauncher& L, int nstrips, int ny, int wpb, unsigned block, size_t smem);
// Warps per block of the 2D stage kernel when the caller gives none: the most resident warps per SM
// (4, 2, 8 or 1 warps, at most max_wpb). Changes the kernel's dynamic shared-memory limit.
int default_block_warps(const StageLauncher& L, int max_wpb);

// Instantiation tables (one per kernel file). Return {nullptr} if the combination is not compiled.
StageLauncher stage1d_launcher(int K, int EQ, int PREC, bool oedg = false);
StageLauncher stage2d_f64_launcher(int K, int EQ, int BASIS);
StageLauncher stage2d_f32_launcher(int K, int EQ, int BASIS);
StageLauncher stage2d_oedg_launcher(int K, int EQ, int BASIS, int PREC);  // OEDG form: Burgers, Euler
StageLauncher stage2d_f32_lean_launcher(int K, int EQ, int BASIS);         // FP32 form, no limiter code

// Geometry and physics of one solver, as the auxiliary kernels see it.
struct AuxGeom {
  int dim, nx, ny, k, nv, nm, basis, eq, prec;
  long long ncell;
  double x0, y0, hx, hy, gamma, ax, ay;
  int mp[16], mq[16];  // (p, q) of each mode
  int pp;              // Euler with the positivity limiter: the CFL rate also takes the limiter's points
  int hyb;             // hybrid limiter (Algorithm 1) scratch in the workspace
  int oedg;            // OEDG damping: jump sums and reductions in the workspace, filter kernel per stage
};

cudaError_t aux_init_tables();  // copy Gauss rules to constant memory of the current device

// Argument checks of dg_create (mesh, degree, equation, parameters); DG_OK or the status to return.
dg_status validate_config(const dg_mesh* m, int k, int eq, const dg_filter_params* p);
// Geometry and physics of a validated configuration, as the auxiliary kernels see it.
void fill_geom(AuxGeom& g, const dg_mesh* m, int k, int eq, const dg_filter_params* p);
// DG_OK if the current device is an sm_103 GPU; otherwise DG_ERR_CUDA with the reason in *why.
dg_status check_device(char* why, size_t why_len);
cudaError_t launch_project(const AuxGeom& g, int ic, const double* prm, int nprm, int nq,
                           double* canon_out, cudaStream_t s);
cudaError_t launch_rate(const AuxGeom& g, const void* state, DevScalars* sc, int slot, cudaStream_t s);
cudaError_t launch_to_storage(const AuxGeom& g, const double* canon, void* state, cudaStream_t s);
cudaError_t launch_from_storage(const AuxGeom& g, const void* state, double* canon, cudaStream_t s);
cudaError_t launch_mass(const AuxGeom& g, const void* state, double* partials, double* out, cudaStream_t s);
size_t state_bytes(const AuxGeom& g);
// Hybrid limiter: rescale the higher modes of the listed troubled cells of `state` by
// omega + (1 - omega) exp(-sigma^l dt), then clear the stage's scalars.
cudaError_t launch_hybrid_blend(const AuxGeom& g, void* state, const HybridOut& h, cudaStream_t s);
int hybrid_lmax(const AuxGeom& g);   // highest total degree l of a mode
// OEDG: sigma^l = max_v A_v(l) / (2 (2k-1) ||u_v - avg u_v||_inf), the modes of `state` rescaled by
// exp(-sigma^l dt) (dt of the step in progress), then the reductions cleared for the next stage.
cudaError_t launch_oedg_filter(const AuxGeom& g, void* state, const OedgOut& o, const DevScalars* sc,
                               cudaStream_t s);
constexpr int MASS_BLOCKS = 256;

}  // namespace dgk
