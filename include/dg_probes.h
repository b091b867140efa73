/*
 * dg_probes.h — measurement probes of the GB300 stage kernels' design decisions. They are not part
 * of the paper's method (the paper has no counterpart); they time small synthetic kernels with CUDA
 * events on a private stream of the current device and change no device setting. Return 0 on
 * success, -1 for a bad argument, -2 if device memory could not be allocated, -6 on a CUDA error.
 */
#ifndef DG_PROBES_H
#define DG_PROBES_H
#ifndef DG_API
#define DG_API __attribute__((visibility("default")))
#endif
#ifdef __cplusplus
extern "C" {
#endif

/* Fused multiply-add throughput of the device in TFLOP/s (2 flops per FMA): kind 0 = FP32 FFMA,
 * 1 = the two-lane FP32 FFMA2, 2 = FP64 DFMA. 8 blocks of 256 threads per SM, each thread 8
 * independent chains of iters x 16 FMAs; three timed launches after one warm-up launch. */
DG_API int dg_probe_fma(int kind, int iters, double* tflops);

/* The modal -> volume-point transform of 2D Q2 (9 Legendre modes -> 9 Gauss points per cell, 4
 * variables) on ncell synthetic cells (averages near 1, higher modes a few per cent), timed over reps
 * launches: variant 0 = CUDA cores (sum-factorised FP32 FMAs, one thread per cell, as the stage
 * kernels), 1 = tensor cores via mma.sync m16n8k8 TF32 (one pass), 2 = the same with the 3xTF32
 * split. *ms_per_launch: mean launch time; *rel_l1: relative L1 of the result against an FP64
 * evaluation of the same transform. */
DG_API int dg_probe_transform(int variant, long long ncell, int reps, double* ms_per_launch, double* rel_l1);

/* The bounded wait of dg_batch_run_persistent's kernels, on a counter that nothing releases: one warp
 * polls it poll_limit (at most 2^24) times, 256 ns apart, and gives up. *status: the status word the kernel left
 * (1 = the wait gave up, as it must); *ms: the launch's duration. Shows that a wait which can never be
 * satisfied ends, reports, and leaves the context usable. */
DG_API int dg_probe_wait_timeout(unsigned poll_limit, unsigned* status, double* ms);

#ifdef __cplusplus
}
#endif
#endif /* DG_PROBES_H */
