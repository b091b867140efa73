// stage2d_oedg.cu — instantiations of the fused 2D stage kernel in its OEDG form (DG_FILTER_OEDG:
// u~ stored unfiltered with the jump sums and reductions of the OEDG coefficient): degrees 1..3,
// Burgers / Euler, Q^k and P^k bases, FP64 and the FP32 form. A unit of its own, so that it compiles
// in parallel with the jump-filter instantiations.
#include "dg_internal.h"
#include "stage2d.cuh"

namespace dgk {

template <int K, int EQ, int B, class PR>
static cudaError_t launch2o(const void* args, unsigned grid, unsigned block, size_t smem, cudaStream_t s) {
  stage2d_kernel<K, EQ, B, PR, true><<<grid, block, smem, s>>>(*(const Stage2DArgs*)args);
  return cudaGetLastError();
}
template <int K, int EQ, int B, class PR>
static cudaError_t smem2o(size_t bytes) {
  return cudaFuncSetAttribute(stage2d_kernel<K, EQ, B, PR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes);
}
template <int K, int EQ, int B, class PR>
static int occ2o(unsigned block, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage2d_kernel<K, EQ, B, PR, true>, (int)block, smem) !=
      cudaSuccess)
    return 0;
  return n;
}
template <int K, int EQ, int B, class PR>
static StageLauncher make2o() {
  return StageLauncher{&launch2o<K, EQ, B, PR>, &smem2o<K, EQ, B, PR>,
                       Stage2D<K, EQ, B, PR, true>::slot_bytes_per_warp(), &occ2o<K, EQ, B, PR>};
}

template <int K, int B, class PR>
static StageLauncher pick_eq(int EQ) {
  switch (EQ) {
    case EQ_BURG: return make2o<K, EQ_BURG, B, PR>();
    case EQ_EULER: return make2o<K, EQ_EULER, B, PR>();
  }
  return StageLauncher{nullptr, nullptr, 0};
}

template <int B, class PR>
static StageLauncher pick_k(int K, int EQ) {
  switch (K) {
    case 1: return pick_eq<1, B, PR>(EQ);
    case 2: return pick_eq<2, B, PR>(EQ);
    case 3: return pick_eq<3, B, PR>(EQ);
  }
  return StageLauncher{nullptr, nullptr, 0};
}

template <class PR>
static StageLauncher pick_b(int K, int EQ, int BASIS) {
  return BASIS == BASIS_Q ? pick_k<BASIS_Q, PR>(K, EQ) : pick_k<BASIS_P, PR>(K, EQ);
}

StageLauncher stage2d_oedg_launcher(int K, int EQ, int BASIS, int PREC) {
  return PREC == PREC_F64 ? pick_b<PrecF64>(K, EQ, BASIS) : pick_b<PrecF32M>(K, EQ, BASIS);
}

}  // namespace dgk
