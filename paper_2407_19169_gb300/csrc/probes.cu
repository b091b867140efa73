// probes.cu — measurement probes behind the design decisions of the stage kernels (not part of the
// method): the FP32 / packed-FP32 / FP64 fused multiply-add throughput of the device, and an A/B of
// the modal -> quadrature-point transform of the 2D Q2 stage (9 modes -> 9 volume Gauss points per
// cell and variable) on the CUDA cores (sum-factorised FMAs, the stage kernels' way) against the
// tensor cores through mma.sync m16n8k8 with TF32 operands (one pass, and the 3xTF32 split
// a_hi b_hi + a_hi b_lo + a_lo b_hi that restores FP32 accuracy). Timed with CUDA events on a
// private stream; nothing here changes a device setting.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/dg_probes.h"

namespace {

// ---- FMA throughput -----------------------------------------------------------------------
// 8 independent chains per thread, 16 unrolled steps per iteration; x -> x a + b stays bounded
// (a < 1), so no value overflows or becomes subnormal.
template <class T>
__global__ void fma_kernel(T* sink, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = T(threadIdx.x + j) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == T(-12345.0)) sink[threadIdx.x] = s;   // never true; keeps the chains live
}

// the two-lane FP32 instruction (one FFMA2 = two FMAs)
__global__ void ffma2_kernel(float* sink, int iters, float a, float b) {
  float2 x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = make_float2((threadIdx.x + j) * 1e-3f, (threadIdx.x + 2 * j) * 1e-3f);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = __ffma2_rn(x[j], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j].x + x[j].y;
  if (s == -12345.f) sink[threadIdx.x] = s;
}

// ---- the Q2 modal -> volume-point transform ---------------------------------------------------
// u[(v * 9 + m) * n + c] modes (m = p + 3 q), f[(v * 9 + i) * n + c] values at the volume Gauss
// points i = a + 3 b, (x_a, x_b) of the 3-point rule: f = sum_m u_m P_p(x_a) P_q(x_b).
struct Tab9 {
  float t[81];    // t[m * 9 + i]
  double td[81];
  float p3[3];    // P_0..P_2 at x_0 (the end nodes +-x_0 by parity)
  float p2m;      // P_2 at the middle node 0
};

__device__ __forceinline__ uint32_t hash32(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return (uint32_t)x;
}

// smooth-like data: averages near 1, higher modes a few per cent
__global__ void fill_kernel(float* u, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 36 * n; i += (long long)gridDim.x * blockDim.x) {
    const int m = (int)((i / n) % 9);
    const float r = (hash32((uint64_t)i * 0x9E3779B97F4A7C15ull) >> 8) * (1.0f / 16777216.0f) - 0.5f;
    u[i] = m == 0 ? 1.0f + 0.5f * r : 0.04f * r;
  }
}

// FP64 reference (dense sums in double)
__global__ void ref_kernel(const float* u, double* f, long long n, const Tab9 tb) {
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
    for (int v = 0; v < 4; ++v)
      for (int i = 0; i < 9; ++i) {
        double s = 0.0;
        for (int m = 0; m < 9; ++m) s += (double)u[(v * 9 + m) * n + c] * tb.td[m * 9 + i];
        f[(v * 9 + i) * n + c] = s;
      }
}

// CUDA cores: one thread per cell, sum factorisation in both directions (P_l of the 3-point rule:
// values at -x_0, 0, +x_0 from the even / odd parts), as the stage kernels do.
__global__ void fma_transform_kernel(const float* __restrict__ u, float* __restrict__ f, long long n, const Tab9 tb) {
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float w[9];
#pragma unroll
      for (int m = 0; m < 9; ++m) w[m] = __ldg(u + (v * 9 + m) * n + c);
      // collapse p at the three x nodes: C[a][q]
      float C[3][3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float e = fmaf(w[2 + 3 * q], tb.p3[2], w[3 * q]), o = w[1 + 3 * q] * tb.p3[1];
        C[0][q] = e + o;
        C[2][q] = e - o;
        C[1][q] = fmaf(w[2 + 3 * q], tb.p2m, w[3 * q]);
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float e = fmaf(C[a][2], tb.p3[2], C[a][0]), o = C[a][1] * tb.p3[1];
        f[(v * 9 + a + 0) * n + c] = e + o;
        f[(v * 9 + a + 6) * n + c] = e - o;
        f[(v * 9 + a + 3) * n + c] = fmaf(C[a][2], tb.p2m, C[a][0]);
      }
    }
  }
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Tensor cores: a warp takes 16 cells per tile; D[cell][point] = U[cell][mode] T[mode][point] as
// (16 x 16) x (16 x 16) with the modes and points padded from 9 to 16: 2 k-steps x 2 n-tiles of
// m16n8k8 per variable (SPLIT: x3 for the hi/lo products). Fragments (g = lane / 4, t = lane % 4):
// A a0 = U[g][t], a1 = U[g+8][t], a2 = U[g][t+4], a3 = U[g+8][t+4]; B b0 = T[t][g], b1 = T[t+4][g];
// D d0 = D[g][2t], d1 = D[g][2t+1], d2 = D[g+8][2t], d3 = D[g+8][2t+1].
template <bool SPLIT>
__global__ void mma_transform_kernel(const float* __restrict__ u, float* __restrict__ f, long long n, const Tab9 tb) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // B fragments of the padded table, hi and lo parts, for k-step kt and n-tile nt
  uint32_t bh[2][2][2], bl[2][2][2];
#pragma unroll
  for (int kt = 0; kt < 2; ++kt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = 8 * kt + t + 4 * h, i = 8 * nt + g;
        const float x = (m < 9 && i < 9) ? tb.t[m * 9 + i] : 0.f;
        bh[kt][nt][h] = to_tf32(x);
        bl[kt][nt][h] = to_tf32(x - __uint_as_float(bh[kt][nt][h]));
      }
  const long long tiles = (n + 15) / 16;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long tile = warp; tile < tiles; tile += nwarps) {
    const long long c0 = tile * 16 + g, c1 = c0 + 8;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float d[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
      for (int kt = 0; kt < 2; ++kt) {
        float av[4];
        const int m0 = 8 * kt + t, m1 = m0 + 4;
        av[0] = (m0 < 9 && c0 < n) ? __ldg(u + (v * 9 + m0) * n + c0) : 0.f;
        av[1] = (m0 < 9 && c1 < n) ? __ldg(u + (v * 9 + m0) * n + c1) : 0.f;
        av[2] = (m1 < 9 && c0 < n) ? __ldg(u + (v * 9 + m1) * n + c0) : 0.f;
        av[3] = (m1 < 9 && c1 < n) ? __ldg(u + (v * 9 + m1) * n + c1) : 0.f;
        uint32_t ah[4], al[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          ah[j] = to_tf32(av[j]);
          al[j] = to_tf32(av[j] - __uint_as_float(ah[j]));
        }
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const uint32_t bhh[2] = {bh[kt][nt][0], bh[kt][nt][1]};
          mma_tf32(d[nt], ah, bhh);
          if constexpr (SPLIT) {
            const uint32_t bll[2] = {bl[kt][nt][0], bl[kt][nt][1]};
            mma_tf32(d[nt], ah, bll);
            mma_tf32(d[nt], al, bhh);
          }
        }
      }
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int i0 = 8 * nt + 2 * t, i1 = i0 + 1;
        if (i0 < 9) {
          if (c0 < n) f[(v * 9 + i0) * n + c0] = d[nt][0];
          if (c1 < n) f[(v * 9 + i0) * n + c1] = d[nt][2];
        }
        if (i1 < 9) {
          if (c0 < n) f[(v * 9 + i1) * n + c0] = d[nt][1];
          if (c1 < n) f[(v * 9 + i1) * n + c1] = d[nt][3];
        }
      }
    }
  }
}

// relative L1 of a float result against the FP64 reference: partial sums per block
__global__ void err_kernel(const float* f, const double* r, long long total, double* acc) {
  __shared__ double sn[256], sd[256];
  double num = 0.0, den = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    num += fabs((double)f[i] - r[i]);
    den += fabs(r[i]);
  }
  sn[threadIdx.x] = num;
  sd[threadIdx.x] = den;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sn[threadIdx.x] += sn[threadIdx.x + o];
      sd[threadIdx.x] += sd[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(acc, sn[0]);
    atomicAdd(acc + 1, sd[0]);
  }
}

Tab9 make_table() {
  const double x0 = sqrt(0.6);
  const double xs[3] = {-x0, 0.0, x0};
  auto P = [](int l, double x) { return l == 0 ? 1.0 : (l == 1 ? x : 1.5 * x * x - 0.5); };
  Tab9 tb;
  for (int m = 0; m < 9; ++m)
    for (int i = 0; i < 9; ++i) {
      const double v = P(m % 3, xs[i % 3]) * P(m / 3, xs[i / 3]);
      tb.td[m * 9 + i] = v;
      tb.t[m * 9 + i] = (float)v;
    }
  // node order -x0, 0, +x0: C[0] at -x0 = e - o with o = P_1(x0) ... the kernel writes e + o to
  // index 0, so take P_1 at -x0 (negative) for the odd part
  tb.p3[0] = 1.0f;
  tb.p3[1] = (float)(-x0);
  tb.p3[2] = (float)(1.5 * 0.6 - 0.5);
  tb.p2m = -0.5f;
  return tb;
}

}  // namespace

extern "C" int dg_probe_fma(int kind, int iters, double* tflops) {
  if (!tflops || iters < 1 || kind < 0 || kind > 2) return -1;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return -6;
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return -6;
  void* sink = nullptr;
  if (cudaMalloc(&sink, 1024 * sizeof(double)) != cudaSuccess) {
    cudaStreamDestroy(st);
    return -2;
  }
  const unsigned blocks = 8u * (unsigned)nsm, threads = 256;
  auto launch = [&]() {
    if (kind == 0) fma_kernel<float><<<blocks, threads, 0, st>>>((float*)sink, iters, 0.9999f, 1e-4f);
    else if (kind == 1) ffma2_kernel<<<blocks, threads, 0, st>>>((float*)sink, iters, 0.9999f, 1e-4f);
    else fma_kernel<double><<<blocks, threads, 0, st>>>((double*)sink, iters, 0.9999, 1e-4);
  };
  launch();  // warm-up
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  for (int r = 0; r < 3; ++r) launch();
  cudaEventRecord(e1, st);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  const double fmas = 3.0 * blocks * threads * (double)iters * 16.0 * 8.0 * (kind == 1 ? 2.0 : 1.0);
  *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  cudaStreamDestroy(st);
  return (err == cudaSuccess && cudaGetLastError() == cudaSuccess) ? 0 : -6;
}

extern "C" int dg_probe_transform(int variant, long long ncell, int reps, double* ms_per_launch, double* rel_l1) {
  if (!ms_per_launch || !rel_l1 || variant < 0 || variant > 2 || ncell < 16 || reps < 1) return -1;
  const size_t nu = 36 * (size_t)ncell;
  float *u = nullptr, *f = nullptr;
  double *r = nullptr, *acc = nullptr;
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return -6;
  int status = 0;
  if (cudaMalloc(&u, nu * sizeof(float)) != cudaSuccess || cudaMalloc(&f, nu * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&r, nu * sizeof(double)) != cudaSuccess || cudaMalloc(&acc, 2 * sizeof(double)) != cudaSuccess) {
    status = -2;
  } else {
    const Tab9 tb = make_table();
    fill_kernel<<<1216, 256, 0, st>>>(u, ncell);
    ref_kernel<<<1216, 256, 0, st>>>(u, r, ncell, tb);
    auto launch = [&]() {
      if (variant == 0) fma_transform_kernel<<<1216, 256, 0, st>>>(u, f, ncell, tb);
      else if (variant == 1) mma_transform_kernel<false><<<1216, 256, 0, st>>>(u, f, ncell, tb);
      else mma_transform_kernel<true><<<1216, 256, 0, st>>>(u, f, ncell, tb);
    };
    launch();  // warm-up
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    for (int i = 0; i < reps; ++i) launch();
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    *ms_per_launch = ms / reps;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaMemsetAsync(acc, 0, 2 * sizeof(double), st);
    err_kernel<<<1216, 256, 0, st>>>(f, r, (long long)nu, acc);
    double h[2] = {0.0, 0.0};
    cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) status = -6;
    *rel_l1 = h[1] > 0.0 ? h[0] / h[1] : 0.0;
  }
  cudaFree(u);
  cudaFree(f);
  cudaFree(r);
  cudaFree(acc);
  cudaStreamDestroy(st);
  return status;
}
