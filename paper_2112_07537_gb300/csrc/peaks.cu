// peaks.cu -- compute-throughput probes of the current device: the
// compute-roofline denominators (FP32 / FP64 fused multiply-add and division
// rates) next to the measured copy bandwidth.  Each probe runs CH independent
// dependency chains per thread over a grid of 8 CTAs per SM, so the pipe,
// not latency, bounds it; results land in a static device sink (no
// allocation) that the host never reads.
#include <cstdio>
#include <type_traits>

#include "mr_internal.cuh"

namespace {

__device__ double mr_peak_sink[64];

constexpr int CH = 8;  // independent chains per thread

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T a, T b, int slot) {
  T x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = T(threadIdx.x + 1 + c) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  if (s == T(-1.2345)) mr_peak_sink[slot] = (double)s;  // keeps the chains live
}

// kind 0: FP32 __fdividef, 1: FP32 IEEE division, 2: FP64 division
template <int KIND>
__global__ void __launch_bounds__(256) k_div_chains(int iters, double a_, double b_, int slot) {
  using T = typename std::conditional<KIND == 2, double, float>::type;
  const T a = T(a_), b = T(b_);
  T x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = T(threadIdx.x + 1 + c) * T(1e-3) + T(1);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      if constexpr (KIND == 0) x[c] = __fdividef(a, x[c]) + b;
      else x[c] = a / x[c] + b;
    }
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  if (s == T(-1.2345)) mr_peak_sink[slot] = (double)s;
}

// seconds of one launch (best of reps, after one warm-up launch)
template <typename F>
static int time_launch(F launch, int reps, double *sec) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return 1;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return 1;
  }
  launch();
  double best = 1e30;
  int bad = 0;
  for (int r = 0; r < reps && !bad; ++r) {
    cudaEventRecord(e0, 0);
    launch();
    cudaEventRecord(e1, 0);
    bad |= cudaEventSynchronize(e1) != cudaSuccess;
    float ms = 0.f;
    bad |= cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess;
    if (ms > 0.f && ms * 1e-3 < best) best = ms * 1e-3;
  }
  bad |= cudaGetLastError() != cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *sec = best;
  return bad;
}

}  // namespace

extern "C" int mr_device_peaks(double *out) {
  using namespace mr;
  if (!out) return MR_ERR_INVALID;
  int dev = 0, sms = 0;
  if (check_cuda(cudaGetDevice(&dev), "cudaGetDevice") ||
      check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count"))
    return MR_ERR_CUDA;
  const int blocks = sms * 8, threads = 256;
  const double nthr = (double)blocks * threads;
  double t;
  // FP32 and FP64 fused multiply-add: 2 flops per FMA
  const int i32 = 2048, i64 = 128, d32 = 512, d64 = 64;
  if (time_launch([&] { k_fma_chains<float><<<blocks, threads>>>(i32, 0.999f, 1e-6f, 0); }, 5, &t)) goto fail;
  out[0] = 2.0 * CH * i32 * nthr / t / 1e12;
  if (time_launch([&] { k_fma_chains<double><<<blocks, threads>>>(i64, 0.999, 1e-6, 1); }, 3, &t)) goto fail;
  out[1] = 2.0 * CH * i64 * nthr / t / 1e12;
  // divisions per second (each chain step is one division and one add)
  if (time_launch([&] { k_div_chains<0><<<blocks, threads>>>(d32, 1.5, 0.5, 2); }, 5, &t)) goto fail;
  out[2] = (double)CH * d32 * nthr / t / 1e9;
  if (time_launch([&] { k_div_chains<1><<<blocks, threads>>>(d32, 1.5, 0.5, 3); }, 5, &t)) goto fail;
  out[3] = (double)CH * d32 * nthr / t / 1e9;
  if (time_launch([&] { k_div_chains<2><<<blocks, threads>>>(d64, 1.5, 0.5, 4); }, 3, &t)) goto fail;
  out[4] = (double)CH * d64 * nthr / t / 1e9;
  return MR_OK;
fail:
  check_cuda(cudaGetLastError(), "mr_device_peaks");
  return MR_ERR_CUDA;
}
