// mm_measure_peak: short microbenchmarks of the throughputs the map kernels'
// rooflines are measured against (the paper has no counterpart; these give
// the denominators of the achieved fractions the benchmark reports).
//
//   FP32 FMA : every thread runs 8 independent fmaf chains (2 flops each);
//   FP64 FMA : the same chains in double;
//   L2 RED   : every thread adds 1 to scattered u64 words of a 32 MiB array
//              (L2-resident on GB300) with atomicAdd whose result is unused
//              (a reduction, as the map's fixed-point accumulation issues);
//              "rows": a warp's 32 lanes add to 32 consecutive words.
//
// Each kind: one warm-up launch, then the best of three launches timed with
// CUDA events on `stream`.
#include <algorithm>
#include <cstdint>
#include <cstdio>

#include "mm.h"
#include "mm_kernels.h"

namespace {

constexpr int kChains = 8;

template <class T>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T b, T c, T *sink) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) a[k] = (T)(threadIdx.x + k);
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int u = 0; u < 16; u++) {
#pragma unroll
      for (int k = 0; k < kChains; k++) a[k] = fma(a[k], b, c);
    }
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += a[k];
  if (s == (T)-1.2345) sink[0] = s;  // keeps the chains live; never true
}

__global__ void __launch_bounds__(256) k_red_u64(unsigned long long *a, uint32_t mask,
                                                 int iters) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x = t * 0x9E3779B9u + 0x7F4A7C15u;
  for (int it = 0; it < iters; it++) {
    // xorshift32: a different scattered word per thread and step
    x ^= x << 13;
    x ^= x >> 17;
    x ^= x << 5;
    atomicAdd(a + (x & mask), 1ull);
  }
}

// each warp adds 1 to 32 consecutive words (8 sectors of one 256-byte
// span) at a scattered, warp-uniform position: the pattern of a pixel row's
// partially covered pixels dealt across a warp's lanes
__global__ void __launch_bounds__(256) k_red_u64_rows(unsigned long long *a, uint32_t mask,
                                                      int iters) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x = (t >> 5) * 0x9E3779B9u + 0x7F4A7C15u;
  for (int it = 0; it < iters; it++) {
    x ^= x << 13;
    x ^= x >> 17;
    x ^= x << 5;
    atomicAdd(a + (((x << 5) + (t & 31u)) & mask), 1ull);
  }
}

mm_status fail(mm_status s, const char *what, cudaError_t e) {
  char buf[256];
  snprintf(buf, sizeof buf, "mm_measure_peak: %s: %s", what, cudaGetErrorString(e));
  mm::set_last_error(buf);
  return s;
}

}  // namespace

extern "C" mm_status mm_measure_peak(int32_t kind, double *value, double *ms_out,
                                     void *stream) {
  if (!value) {
    mm::set_last_error("mm_measure_peak: value is NULL");
    return MM_EINVAL;
  }
  if (kind < MM_PEAK_FP32_FMA || kind > MM_PEAK_L2_RED_U64_ROWS) {
    mm::set_last_error("mm_measure_peak: unknown kind");
    return MM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(MM_ECUDA, "device query", e);
  sms = std::max(sms, 1);
  void *buf = nullptr;
  const size_t words = size_t(1) << 22;  // 32 MiB of u64
  const bool l2 = kind == MM_PEAK_L2_RED_U64 || kind == MM_PEAK_L2_RED_U64_ROWS;
  e = cudaMalloc(&buf, l2 ? words * 8 : 64);
  if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? MM_ENOMEM : MM_ECUDA,
                                    "cudaMalloc", e);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  mm_status status = MM_OK;
  double work = 0.0, best_ms = 1e300;
  do {
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
      status = fail(MM_ECUDA, "cudaEventCreate", e);
      break;
    }
    const int blocks = sms * 8, threads = 256;
    int iters = 0;
    if (kind == MM_PEAK_FP32_FMA) {
      iters = 4096;
      work = 2.0 * kChains * 16.0 * iters * (double)blocks * threads;
    } else if (kind == MM_PEAK_FP64_FMA) {
      iters = 128;
      work = 2.0 * kChains * 16.0 * iters * (double)blocks * threads;
    } else {
      iters = 2048;
      work = (double)iters * blocks * threads;
      if ((e = cudaMemsetAsync(buf, 0, words * 8, st)) != cudaSuccess) {
        status = fail(MM_ECUDA, "cudaMemsetAsync", e);
        break;
      }
    }
    for (int rep = 0; rep < 4 && status == MM_OK; rep++) {
      if ((e = cudaEventRecord(e0, st)) != cudaSuccess) {
        status = fail(MM_ECUDA, "cudaEventRecord", e);
        break;
      }
      if (kind == MM_PEAK_FP32_FMA)
        k_fma_chains<float><<<blocks, threads, 0, st>>>(iters, 0.999999f, 1e-6f, (float *)buf);
      else if (kind == MM_PEAK_FP64_FMA)
        k_fma_chains<double><<<blocks, threads, 0, st>>>(iters, 0.999999, 1e-6, (double *)buf);
      else if (kind == MM_PEAK_L2_RED_U64)
        k_red_u64<<<blocks, threads, 0, st>>>((unsigned long long *)buf, (uint32_t)(words - 1),
                                              iters);
      else
        k_red_u64_rows<<<blocks, threads, 0, st>>>((unsigned long long *)buf,
                                                   (uint32_t)(words - 1), iters);
      if ((e = cudaGetLastError()) != cudaSuccess ||
          (e = cudaEventRecord(e1, st)) != cudaSuccess ||
          (e = cudaEventSynchronize(e1)) != cudaSuccess) {
        status = fail(MM_ECUDA, "probe launch", e);
        break;
      }
      float t = 0.f;
      if ((e = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) {
        status = fail(MM_ECUDA, "cudaEventElapsedTime", e);
        break;
      }
      if (rep > 0) best_ms = std::min(best_ms, (double)t);  // rep 0 warms up
    }
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  if (status != MM_OK) return status;
  // TFLOP/s for the FMA kinds, G reductions/s for the L2 kind
  *value = l2 ? work / (best_ms * 1e-3) / 1e9 : work / (best_ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = best_ms;
  return MM_OK;
}
