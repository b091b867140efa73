// stage2d_f32.cu — instantiations of the fused 2D stage kernel (PrecF32M): degrees 1..3,
// advection / Burgers / Euler, tensor-product (Q^k) and total-degree (P^k) bases.
#include "dg_internal.h"
#include "stage2d.cuh"

namespace dgk {

template <int K, int EQ, int B>
static cudaError_t launch2d(const void* args, unsigned grid, unsigned block, size_t smem, cudaStream_t s) {
  stage2d_kernel<K, EQ, B, PrecF32M><<<grid, block, smem, s>>>(*(const Stage2DArgs*)args);
  return cudaGetLastError();
}
template <int K, int EQ, int B>
static cudaError_t smem2d(size_t bytes) {
  return cudaFuncSetAttribute(stage2d_kernel<K, EQ, B, PrecF32M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes);
}
template <int K, int EQ, int B>
static int occ2d(unsigned block, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage2d_kernel<K, EQ, B, PrecF32M>, (int)block, smem) !=
      cudaSuccess)
    return 0;
  return n;
}
template <int K, int EQ, int B>
static StageLauncher make2d() {
  return StageLauncher{&launch2d<K, EQ, B>, &smem2d<K, EQ, B>,
                       Stage2D<K, EQ, B, PrecF32M>::slot_bytes_per_warp(), &occ2d<K, EQ, B>};
}

template <int K, int B>
static StageLauncher pick_eq(int EQ) {
  switch (EQ) {
    case EQ_ADV: return make2d<K, EQ_ADV, B>();
    case EQ_BURG: return make2d<K, EQ_BURG, B>();
    case EQ_EULER: return make2d<K, EQ_EULER, B>();
  }
  return StageLauncher{nullptr, nullptr, 0};
}

template <int B>
static StageLauncher pick_k(int K, int EQ) {
  switch (K) {
    case 1: return pick_eq<1, B>(EQ);
    case 2: return pick_eq<2, B>(EQ);
    case 3: return pick_eq<3, B>(EQ);
  }
  return StageLauncher{nullptr, nullptr, 0};
}

StageLauncher stage2d_f32_launcher(int K, int EQ, int BASIS) {
  return BASIS == BASIS_Q ? pick_k<BASIS_Q>(K, EQ) : pick_k<BASIS_P>(K, EQ);
}

}  // namespace dgk
