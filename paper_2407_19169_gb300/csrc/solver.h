// solver.h — the solver handle behind the opaque dg_solver of include/dg.h (library-internal).
#pragma once
#include <cuda_runtime.h>

#include "../../include/dg.h"
#include "dg_internal.h"

struct dg_solver {
  dg_mesh mesh;
  int k, eq, dim, basis, prec, filter_on, H, warps_per_block, positivity, hybrid;
  double cfl, gamma, ax, ay;
  dgk::AuxGeom geom;
  size_t ndof, sbytes;
  cudaStream_t stream;
  bool own_stream;
  bool own_mem;
  void* mem;
  size_t mem_bytes;
  void* buf[3];
  double* canon;        // FP64 conversion scratch (FP32 form only)
  double* partials;     // mass partial sums
  double* dmass;        // mass result
  dgk::DevScalars* sc;
  dgk::HybridOut hy;    // hybrid limiter scratch (null pointers when off)
  dgk::OedgOut oe;      // OEDG damping scratch (null pointers when off)
  dgk::DevScalars* h_sc;  // pinned mirror
  long long h_step;     // host's record of the device step count (buffer parity)
  dgk::StageLauncher L;
  unsigned grid, block;
  size_t smem;
  int nstrips, nchunks, nwarps1d;
  cudaGraphExec_t pair_exec;
  bool pair_ready;
  long long pair_launches;  // kernel nodes in the step-pair graph
  long long launches;
};

namespace dgk {
// Device control block of a solver as last read by the host (synchronises the solver's stream).
dg_status solver_pull_control(dg_solver* s);
}  // namespace dgk
