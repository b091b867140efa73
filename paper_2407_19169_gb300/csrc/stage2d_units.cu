// stage2d_units.cu — instantiations of the fused 2D stage kernel and their launch tables.
//
// The build compiles this file once per (form, degree), with -DS2_FORM=f -DS2_K=k, and once with
// -DS2_DISPATCH for the tables that select among them, so that the slow instantiations (FP64 and
// degree 3, with every loop of the stage unrolled at compile time) compile in parallel.
// Forms: 0 FP64; 1 FP32 form; 2 FP32 form without the positivity and hybrid limiter code (a smaller
// loop body for the solves that use neither); 3 OEDG damping, FP64; 4 OEDG damping, FP32 form.
// Each (form, degree) holds the advection, Burgers and Euler instantiations (OEDG: Burgers, Euler)
// on the Q^k and P^k bases.
#include "dg_internal.h"
#include "stage2d.cuh"

namespace dgk {

template <int FORM>
struct Form2D;
template <>
struct Form2D<0> {
  using PR = PrecF64;
  static constexpr bool OE = false, LIM = true;
};
template <>
struct Form2D<1> {
  using PR = PrecF32M;
  static constexpr bool OE = false, LIM = true;
};
template <>
struct Form2D<2> {
  using PR = PrecF32M;
  static constexpr bool OE = false, LIM = false;
};
template <>
struct Form2D<3> {
  using PR = PrecF64;
  static constexpr bool OE = true, LIM = true;
};
template <>
struct Form2D<4> {
  using PR = PrecF32M;
  static constexpr bool OE = true, LIM = true;
};

// The launch table of one (degree, form): {nullptr} for an equation or basis it does not hold.
template <int K, int FORM>
StageLauncher stage2d_table(int EQ, int BASIS);

#define S2_DECLARE(K)                                   \
  template <>                                           \
  StageLauncher stage2d_table<K, 0>(int EQ, int BASIS); \
  template <>                                           \
  StageLauncher stage2d_table<K, 1>(int EQ, int BASIS); \
  template <>                                           \
  StageLauncher stage2d_table<K, 2>(int EQ, int BASIS); \
  template <>                                           \
  StageLauncher stage2d_table<K, 3>(int EQ, int BASIS); \
  template <>                                           \
  StageLauncher stage2d_table<K, 4>(int EQ, int BASIS);
S2_DECLARE(1)
S2_DECLARE(2)
S2_DECLARE(3)
#undef S2_DECLARE

#if defined(S2_FORM) && defined(S2_K)

template <int K, int EQ, int B, int FORM>
static cudaError_t launch2(const void* args, unsigned grid, unsigned block, size_t smem, cudaStream_t s) {
  using F = Form2D<FORM>;
  stage2d_kernel<K, EQ, B, typename F::PR, F::OE, F::LIM><<<grid, block, smem, s>>>(*(const Stage2DArgs*)args);
  return cudaGetLastError();
}
template <int K, int EQ, int B, int FORM>
static cudaError_t smem2(size_t bytes) {
  using F = Form2D<FORM>;
  return cudaFuncSetAttribute(stage2d_kernel<K, EQ, B, typename F::PR, F::OE, F::LIM>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
template <int K, int EQ, int B, int FORM>
static int occ2(unsigned block, size_t smem) {
  using F = Form2D<FORM>;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage2d_kernel<K, EQ, B, typename F::PR, F::OE, F::LIM>,
                                                    (int)block, smem) != cudaSuccess)
    return 0;
  return n;
}
template <int K, int EQ, int B, int FORM>
static StageLauncher make2() {
  using F = Form2D<FORM>;
  return StageLauncher{&launch2<K, EQ, B, FORM>, &smem2<K, EQ, B, FORM>,
                       Stage2D<K, EQ, B, typename F::PR, F::OE, F::LIM>::slot_bytes_per_warp(),
                       &occ2<K, EQ, B, FORM>};
}
template <int K, int B, int FORM>
static StageLauncher pick_eq(int EQ) {
  constexpr bool oedg = Form2D<FORM>::OE;
  switch (EQ) {
    case EQ_ADV:
      if constexpr (!oedg) return make2<K, EQ_ADV, B, FORM>();
      break;
    case EQ_BURG: return make2<K, EQ_BURG, B, FORM>();
    case EQ_EULER: return make2<K, EQ_EULER, B, FORM>();
  }
  return StageLauncher{nullptr, nullptr, 0, nullptr};
}

template <>
StageLauncher stage2d_table<S2_K, S2_FORM>(int EQ, int BASIS) {
  return BASIS == BASIS_Q ? pick_eq<S2_K, BASIS_Q, S2_FORM>(EQ) : pick_eq<S2_K, BASIS_P, S2_FORM>(EQ);
}

#endif  // S2_FORM && S2_K

#ifdef S2_DISPATCH

template <int FORM>
static StageLauncher by_degree(int K, int EQ, int BASIS) {
  switch (K) {
    case 1: return stage2d_table<1, FORM>(EQ, BASIS);
    case 2: return stage2d_table<2, FORM>(EQ, BASIS);
    case 3: return stage2d_table<3, FORM>(EQ, BASIS);
  }
  return StageLauncher{nullptr, nullptr, 0, nullptr};
}

StageLauncher stage2d_f64_launcher(int K, int EQ, int BASIS) { return by_degree<0>(K, EQ, BASIS); }
StageLauncher stage2d_f32_launcher(int K, int EQ, int BASIS) { return by_degree<1>(K, EQ, BASIS); }
StageLauncher stage2d_f32_lean_launcher(int K, int EQ, int BASIS) { return by_degree<2>(K, EQ, BASIS); }
StageLauncher stage2d_oedg_launcher(int K, int EQ, int BASIS, int PREC) {
  return PREC == PREC_F64 ? by_degree<3>(K, EQ, BASIS) : by_degree<4>(K, EQ, BASIS);
}

#endif  // S2_DISPATCH

}  // namespace dgk
