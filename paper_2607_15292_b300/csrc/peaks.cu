// Measured throughput of the execution units the kernels of this library
// are bound by (roofline denominators; the paper has no counterpart):
// FP32 and FP64 fused multiply-adds, the special-function unit (ex2), and
// the fifth-generation tensor core in kind::tf32 (operands in shared
// memory, FP32 accumulation in tensor memory) at the two shapes the
// tensor-core apply uses (M = 128, N = 128) and the widest one (N = 256).
// Each kernel runs enough independent work on every SM to keep the unit
// busy; the rate is work / CUDA-event time of the launch, after a warm-up
// launch.  The SM clock during the runs is measured from clock64() against
// the global nanosecond timer.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "tc.cuh"
#include "tma.cuh"

namespace gcq {

namespace {

constexpr int kChains = 8;   // independent dependency chains per thread

__global__ void k_peak_ffma(float* out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3f + c;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678f) out[0] = s;   // keeps the chains alive
}

__global__ void k_peak_dfma(double* out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3 + c;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678) out[0] = s;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__global__ void k_peak_mufu(float* out, int iters) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = -1e-3f * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = ex2_approx(x[c]) - 1.5f;   // stays in (-1.5, -0.5]
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678f) out[0] = s;
}

// one CTA per SM: thread 0 issues `iters` MMAs (M = 128, N, K = 8) on
// operands resident in shared memory, one commit at the end
template <int N>
__global__ void __launch_bounds__(128, 1) k_peak_tf32(int iters, int* err, long long* cycles) {
  constexpr int KD = 16;   // two K steps resident (static shared memory stays under 48 KB)
  __shared__ __align__(1024) unsigned char sa[128 * KD * 4];
  __shared__ __align__(1024) unsigned char sb[N * KD * 4];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int q = tid; q < 128 * KD; q += blockDim.x) reinterpret_cast<float*>(sa)[q] = 1.0f / 1024.0f;
  for (int q = tid; q < N * KD; q += blockDim.x) reinterpret_cast<float*>(sb)[q] = 1.0f / 1024.0f;
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  constexpr uint32_t cols = N <= 128 ? 128 : 256;
  if (warp == 0) tc::tmem_alloc(&slot, cols);
  fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = slot;
  const long long t0 = clock64();
  if (tid == 0) {
    constexpr uint32_t sbo = tc::sbo_bytes(KD);
    for (int i = 0; i < iters; ++i) {
      const int ks = i & 1;
      tc::mma_tf32(tmem, tc::sdesc(tc::smem_addr(sa) + ks * 256, tc::kLBO, sbo),
                   tc::sdesc(tc::smem_addr(sb) + ks * 256, tc::kLBO, sbo), tc::idesc_tf32(128, N), i > 0);
    }
    tc::commit(&bar);
  }
  // the MMA stream of `iters` steps takes well under the bounded wait
  const bool ok = mbar_wait(&bar, 0);
  if (tid == 0) {
    if (!ok) atomicExch(err, 1);
    atomicMax(cycles, clock64() - t0);
  }
  tc::fence_after_sync();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, cols);
}

// SM clock: cycles of clock64() per nanosecond of %globaltimer over a busy loop
__global__ void k_clock_rate(double* mhz, int spins) {
  uint64_t g0, g1;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g0));
  const long long c0 = clock64();
  float x = 1.0f;
  for (int i = 0; i < spins; ++i) x = fmaf(x, 0.999999f, 1e-7f);
  const long long c1 = clock64();
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g1));
  if (threadIdx.x == 0) mhz[blockIdx.x] = (double)(c1 - c0) / (double)(g1 - g0) * 1e3 + (x == 7.f ? 1.0 : 0.0);
}

template <typename F>
static cudaError_t time_ms(F launch, float* ms) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  launch();   // warm-up
  cudaEventRecord(e0);
  launch();
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace

}  // namespace gcq

extern "C" bem_status bem_measure_peaks(int32_t device, double* out) {
  using namespace gcq;
  if (!out || device < 0) return BEM_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return BEM_ERR_CUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  void* scratch = nullptr;
  int* err = nullptr;
  long long* cyc = nullptr;
  if (cudaMalloc(&scratch, 1 << 16) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&cyc, sizeof(long long)) != cudaSuccess) {
    cudaFree(scratch);
    cudaFree(err);
    return BEM_ERR_OOM;
  }
  cudaMemset(err, 0, sizeof(int));
  bem_status s = BEM_OK;
  float ms = 0.f;
  const int blocks = sms * 8, threads = 256, it_f = 1 << 14, it_d = 1 << 10, it_m = 1 << 12;
  cudaError_t e = time_ms([&] { k_peak_ffma<<<blocks, threads>>>((float*)scratch, it_f, 0.9999f, 1e-4f); }, &ms);
  out[0] = 2.0 * kChains * (double)it_f * blocks * threads / (ms * 1e-3) / 1e12;   // FP32 TFLOP/s
  if (e == cudaSuccess)
    e = time_ms([&] { k_peak_dfma<<<blocks, threads>>>((double*)scratch, it_d, 0.9999, 1e-4); }, &ms);
  out[1] = 2.0 * kChains * (double)it_d * blocks * threads / (ms * 1e-3) / 1e12;   // FP64 TFLOP/s
  if (e == cudaSuccess) e = time_ms([&] { k_peak_mufu<<<blocks, threads>>>((float*)scratch, it_m); }, &ms);
  out[2] = (double)kChains * it_m * blocks * threads / (ms * 1e-3) / 1e12;         // ex2 Tops/s
  const int it_t = 1 << 14;
  if (e == cudaSuccess) e = time_ms([&] { k_peak_tf32<128><<<sms, 128>>>(it_t, err, cyc); }, &ms);
  out[3] = 2.0 * 128 * 128 * 8 * (double)it_t * sms / (ms * 1e-3) / 1e12;          // TF32 TFLOP/s, N = 128
  if (e == cudaSuccess) e = time_ms([&] { k_peak_tf32<256><<<sms, 128>>>(it_t, err, cyc); }, &ms);
  out[4] = 2.0 * 128 * 256 * 8 * (double)it_t * sms / (ms * 1e-3) / 1e12;          // TF32 TFLOP/s, N = 256
  if (e == cudaSuccess) {
    k_clock_rate<<<sms, 32>>>((double*)scratch, 1 << 20);
    double mhz[1024];
    e = cudaMemcpy(mhz, scratch, sizeof(double) * sms, cudaMemcpyDeviceToHost);
    double sum = 0.0;
    for (int i = 0; i < sms; ++i) sum += mhz[i];
    out[5] = sms ? sum / sms : 0.0;                                                   // SM MHz
  }
  out[6] = sms;
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
  count_launches(11);
  if (e != cudaSuccess || herr) s = BEM_ERR_CUDA;
  cudaFree(scratch);
  cudaFree(err);
  cudaFree(cyc);
  return s;
}
