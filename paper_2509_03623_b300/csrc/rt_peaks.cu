// Pipe-rate probe: sustained issue rates of the FP32 and MUFU operations the march is built
// from, per SM and second, measured on the device the library runs on. These are the
// denominators of the march's ALU rooflines.
//
// One launch runs exactly one wave: blocks_per_sm x SMs blocks of 256 threads, every thread
// advancing 8 independent chains of one operation `iters` times (so the pipe, not the
// dependency latency, binds). The rate is the results of one SM's blocks over the CUDA-event
// time of the launch (a few milliseconds, so the launch overhead is below 1e-3 of it). Each
// block also reads the cycle counter (clock64) around its loop; on B300 that counter does not
// run at the SM clock (about 1.27 GHz against a 2.03 GHz SM clock), so it is reported only as
// the counter's rate, and rates per SM clock are formed by the caller from a sampled SM clock.
// Operation of a step (chain value x):
//   FFMA   x = x * 0.9999 + 1e-4               (one FFMA)
//   FFMA2  (x, y) = (x, y) * 0.9999 + 1e-4     (one packed two-lane FFMA2: 2 FMAs)
//   EX2    x = ex2.approx(-x)                  (converges to 0.64)
//   RSQ    x = rsqrt.approx(x)                 (converges to 1)
//   LG2    x = lg2.approx(x) + 2               (converges to 4; one FADD beside each MUFU)
//   RCP    x = rcp.approx(x) + 0.5             (converges to 1.28; one FADD beside each MUFU)
//   SQRT   x = sqrt.approx(x)                  (converges to 1)
//   TANH   x = tanh.approx.f32(x)
//   TANH2  (x, y) = tanh.approx.f16x2(x, y)    (2 half-precision results per instruction)
#include <cuda_fp16.h>

#include <algorithm>
#include <vector>

#include "rt_internal.cuh"

namespace rtb {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;

template <int OP>
__device__ __forceinline__ float peak_step(float x) {
  float y;
  if (OP == RT_PEAK_FFMA) {
    y = fmaf(x, 0.9999f, 1e-4f);
  } else if (OP == RT_PEAK_EX2) {
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
  } else if (OP == RT_PEAK_RSQ) {
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  } else if (OP == RT_PEAK_LG2) {
    asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    y += 2.0f;
  } else if (OP == RT_PEAK_RCP) {
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    y += 0.5f;
  } else if (OP == RT_PEAK_SQRT) {
    asm volatile("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  } else {  // RT_PEAK_TANH
    asm volatile("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  }
  return y;
}

template <int OP>
__global__ void __launch_bounds__(kPeakThreads)
    peak_kernel(int iters, float *__restrict__ sink, long long *__restrict__ cycles) {
  const float seed = 1.0f + 1e-3f * (float)(threadIdx.x & 31);
  float out = 0.0f;
  long long t0, t1;
  if (OP == RT_PEAK_FFMA2) {
    float2 a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; j++) a[j] = make_float2(seed + j, seed - j);
    const float2 m = make_float2(0.9999f, 0.9999f), c = make_float2(1e-4f, 1e-4f);
    __syncthreads();
    t0 = clock64();
    for (int i = 0; i < iters; i++) {
#pragma unroll
      for (int j = 0; j < kChains; j++) a[j] = __ffma2_rn(a[j], m, c);
    }
    __syncthreads();
    t1 = clock64();
#pragma unroll
    for (int j = 0; j < kChains; j++) out += a[j].x + a[j].y;
  } else if (OP == RT_PEAK_TANH2) {
    unsigned a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; j++) {
      const __half2 h = __floats2half2_rn(0.5f + 0.01f * j, 0.25f + 0.01f * j);
      a[j] = *reinterpret_cast<const unsigned *>(&h);
    }
    __syncthreads();
    t0 = clock64();
    for (int i = 0; i < iters; i++) {
#pragma unroll
      for (int j = 0; j < kChains; j++)
        asm volatile("tanh.approx.f16x2 %0, %1;" : "=r"(a[j]) : "r"(a[j]));
    }
    __syncthreads();
    t1 = clock64();
#pragma unroll
    for (int j = 0; j < kChains; j++) {
      const __half2 h = *reinterpret_cast<const __half2 *>(&a[j]);
      out += __low2float(h) + __high2float(h);
    }
  } else {
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; j++) a[j] = seed + 0.1f * j;
    __syncthreads();
    t0 = clock64();
    for (int i = 0; i < iters; i++) {
#pragma unroll
      for (int j = 0; j < kChains; j++) a[j] = peak_step<OP>(a[j]);
    }
    __syncthreads();
    t1 = clock64();
#pragma unroll
    for (int j = 0; j < kChains; j++) out += a[j];
  }
  if (out == 12345.678f) sink[blockIdx.x] = out;  // keeps the chains alive, never true
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// Lane results per instruction of an operation (packed forms give two).
static int lanes_per_op(int op) { return (op == RT_PEAK_FFMA2 || op == RT_PEAK_TANH2) ? 2 : 1; }

template <int OP>
static int run_peak(int iters, int nsm, double *per_s_sm, double *ms, double *counter_mhz,
                    cudaStream_t stream) {
  int bps = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, peak_kernel<OP>,
                                                                kPeakThreads, 0);
  if (e != cudaSuccess || bps < 1)
    return set_error(RT_ECUDA, "peak occupancy: %s", cudaGetErrorString(e));
  const int blocks = bps * nsm;
  // one wave, sized for the device's SMs; freed before returning (this probe allocates)
  float *sink = nullptr;
  long long *cyc = nullptr;
  e = cudaMallocAsync((void **)&sink, blocks * sizeof(float), stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&cyc, blocks * sizeof(long long), stream);
  if (e != cudaSuccess) {
    if (sink) cudaFreeAsync(sink, stream);
    return set_error(RT_ENOMEM, "peak buffers: %s", cudaGetErrorString(e));
  }
  cudaEvent_t ev0, ev1;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  peak_kernel<OP><<<blocks, kPeakThreads, 0, stream>>>(iters / 8 + 1, sink, cyc);  // warm-up
  cudaEventRecord(ev0, stream);
  peak_kernel<OP><<<blocks, kPeakThreads, 0, stream>>>(iters, sink, cyc);
  cudaEventRecord(ev1, stream);
  std::vector<long long> h(blocks);
  e = cudaMemcpyAsync(h.data(), cyc, blocks * sizeof(long long), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  cudaFreeAsync(sink, stream);
  cudaFreeAsync(cyc, stream);
  if (e != cudaSuccess) return set_error(RT_ECUDA, "peak run: %s", cudaGetErrorString(e));
  std::nth_element(h.begin(), h.begin() + blocks / 2, h.end());
  const double cycles = (double)h[blocks / 2];
  const double ops_per_sm = (double)bps * kPeakThreads * kChains * iters * lanes_per_op(OP);
  *per_s_sm = ops_per_sm / (t * 1e-3);
  *ms = t;
  *counter_mhz = cycles / (t * 1e3);  // cycle-counter ticks of the wave / its wall time
  return RT_OK;
}

}  // namespace rtb

extern "C" int rt_pipe_peak(int op, int iters, double *per_s_sm, double *ms, double *counter_mhz,
                            void *stream) {
  using namespace rtb;
  if (!per_s_sm || !ms || !counter_mhz) return set_error(RT_EINVAL, "null output pointer");
  if (iters < 16 || iters > (1 << 24)) return set_error(RT_EINVAL, "iters %d out of range", iters);
  if (op < RT_PEAK_FFMA || op > RT_PEAK_TANH2) return set_error(RT_EINVAL, "unknown operation %d", op);
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return set_error(RT_ECUDA, "device query: %s", cudaGetErrorString(e));
  const cudaStream_t s = (cudaStream_t)stream;
  int rc;
  switch (op) {
    case RT_PEAK_FFMA: rc = run_peak<RT_PEAK_FFMA>(iters, nsm, per_s_sm, ms, counter_mhz, s); break;
    case RT_PEAK_FFMA2: rc = run_peak<RT_PEAK_FFMA2>(iters, nsm, per_s_sm, ms, counter_mhz, s); break;
    case RT_PEAK_EX2: rc = run_peak<RT_PEAK_EX2>(iters, nsm, per_s_sm, ms, counter_mhz, s); break;
    case RT_PEAK_RSQ: rc = run_peak<RT_PEAK_RSQ>(iters, nsm, per_s_sm, ms, counter_mhz, s); break;
    case RT_PEAK_LG2: rc = run_peak<RT_PEAK_LG2>(iters, nsm, per_s_sm, ms, counter_mhz, s); break;
    case RT_PEAK_RCP: rc = run_peak<RT_PEAK_RCP>(iters, nsm, per_s_sm, ms, counter_mhz, s); break;
    case RT_PEAK_SQRT: rc = run_peak<RT_PEAK_SQRT>(iters, nsm, per_s_sm, ms, counter_mhz, s); break;
    case RT_PEAK_TANH: rc = run_peak<RT_PEAK_TANH>(iters, nsm, per_s_sm, ms, counter_mhz, s); break;
    case RT_PEAK_TANH2: rc = run_peak<RT_PEAK_TANH2>(iters, nsm, per_s_sm, ms, counter_mhz, s); break;
    default: return set_error(RT_EINVAL, "unknown operation %d", op);
  }
  if (rc == RT_OK) clear_error();
  return rc;
}
