// stage1d.cu — instantiations of the fused 1D stage kernel: degrees 1..3, advection / Burgers /
// Euler, FP64 and the FP32 form.
#include "dg_internal.h"
#include "stage1d.cuh"

namespace dgk {

template <int K, int EQ, class PR, bool OE>
static cudaError_t launch1d(const void* args, unsigned grid, unsigned block, size_t smem, cudaStream_t s) {
  stage1d_kernel<K, EQ, PR, OE><<<grid, block, smem, s>>>(*(const Stage1DArgs*)args);
  return cudaGetLastError();
}
template <int K, int EQ, class PR, bool OE>
static cudaError_t smem1d(size_t bytes) {
  return cudaFuncSetAttribute(stage1d_kernel<K, EQ, PR, OE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes);
}
template <int K, int EQ, class PR, bool OE>
static StageLauncher make1d() {
  return StageLauncher{&launch1d<K, EQ, PR, OE>, &smem1d<K, EQ, PR, OE>, 0};
}

// the OEDG form (OE) for Burgers and Euler only
template <int K, class PR, bool OE>
static StageLauncher pick_eq(int EQ) {
  switch (EQ) {
    case EQ_ADV:
      if constexpr (!OE) return make1d<K, EQ_ADV, PR, false>();
      break;
    case EQ_BURG: return make1d<K, EQ_BURG, PR, OE>();
    case EQ_EULER: return make1d<K, EQ_EULER, PR, OE>();
  }
  return StageLauncher{nullptr, nullptr, 0};
}

template <class PR, bool OE>
static StageLauncher pick_k(int K, int EQ) {
  switch (K) {
    case 1: return pick_eq<1, PR, OE>(EQ);
    case 2: return pick_eq<2, PR, OE>(EQ);
    case 3: return pick_eq<3, PR, OE>(EQ);
  }
  return StageLauncher{nullptr, nullptr, 0};
}

StageLauncher stage1d_launcher(int K, int EQ, int PREC, bool oedg) {
  if (oedg) return PREC == PREC_F64 ? pick_k<PrecF64, true>(K, EQ) : pick_k<PrecF32M, true>(K, EQ);
  return PREC == PREC_F64 ? pick_k<PrecF64, false>(K, EQ) : pick_k<PrecF32M, false>(K, EQ);
}

}  // namespace dgk
