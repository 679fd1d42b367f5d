// misc.cu -- the step epilogue and the stateless device primitives of libshaken.
#include <cstdint>

#include "shaken_internal.cuh"

namespace shk {

// One block per context.  After the two half steps of step t: if tracking, the
// energy of sigma_t (sums collected during the step) updates the per-replica
// best and the optional series, and the sums are cleared; then t += 1.
// H = -(Jc E) - 2 lamc M - 2 LS (Eq. (ham1); on the lattice Eq. (HGibbs)).
__global__ void __launch_bounds__(256) epilogue_kernel(CtxDev* const* __restrict__ ctxs, int n) {
  if (blockIdx.x >= (unsigned)n) return;
  CtxDev* cd = ctxs[blockIdx.x];
  const uint32_t t = cd->step;
  if (t >= cd->t_end) return;
  if (cd->tracking) {
    for (uint32_t r = threadIdx.x; r < cd->R; r += blockDim.x) {
      double* s = cd->step_sums + (size_t)r * kNumSums;
      const double H = -(cd->Jc * s[kSumE]) - 2.0 * cd->lamc * s[kSumM] - 2.0 * s[kSumLS];
      if (H < cd->best[r]) {
        cd->best[r] = H;
        cd->best_step[r] = (long long)t;
      }
      if (cd->record && t - cd->series_t0 < cd->series_cap) {
        const size_t k = (size_t)(t - cd->series_t0) * cd->R + r;
        if (cd->series_m) cd->series_m[k] = s[kSumM] * cd->inv_n;
        if (cd->series_H) cd->series_H[k] = H;
      }
#pragma unroll
      for (int q = 0; q < kNumSums; ++q) s[q] = 0.0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) cd->step = t + 1u;
}

__global__ void philox_kernel(uint32_t key0, uint32_t key1, const uint4* __restrict__ ctr,
                              uint4* __restrict__ out, int64_t n) {
  const PhKey K = ph_key(key0, key1);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 c = ctr[i];
    out[i] = ph_call(K, c.x, c.y, c.z, c.w);
  }
}

__global__ void threshold_kernel(const double* __restrict__ h, const double* __restrict__ beta,
                                 unsigned long long* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = threshold_T(h[i], beta[i]);
}

cudaError_t launch_epilogue(CtxDev* const* ctxs, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  epilogue_kernel<<<n, 256, 0, st>>>(ctxs, n);
  return cudaGetLastError();
}

cudaError_t launch_philox(uint64_t seed, const uint32_t* ctr, uint32_t* out, int64_t n,
                          cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  philox_kernel<<<grid, 256, 0, st>>>((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32),
                                      reinterpret_cast<const uint4*>(ctr),
                                      reinterpret_cast<uint4*>(out), n);
  return cudaGetLastError();
}

cudaError_t launch_threshold(const double* h, const double* beta, uint64_t* out, int64_t n,
                             cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  threshold_kernel<<<grid, 256, 0, st>>>(h, beta, reinterpret_cast<unsigned long long*>(out), n);
  return cudaGetLastError();
}

}  // namespace shk

// ---------------------------------------------------------------------------- microbenchmarks
namespace shk {

// Register-only Philox: each thread chains `iters` calls (the output feeds the
// next counter) and xors the results into one word, so nothing is elided.
__global__ void __launch_bounds__(256) mb_philox_kernel(uint32_t iters, uint32_t* sink) {
  const PhKey K = ph_key(0x1234u + threadIdx.x, 0x9876u ^ blockIdx.x);
  uint4 c = make_uint4(threadIdx.x, blockIdx.x, 7u, 9u);
  uint32_t acc = 0u;
  for (uint32_t i = 0; i < iters; ++i) {
    c = ph_call(K, c.x, c.y, c.z + i, c.w);
    acc ^= c.x ^ c.y ^ c.z ^ c.w;
  }
  if (acc == 0x5eedu) sink[0] = acc;  // practically never taken
}

// 8 independent dependency chains of 3-input logic ops (LOP3) per thread.
__global__ void __launch_bounds__(256) mb_lop3_kernel(uint32_t iters, uint32_t* sink) {
  uint32_t a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * (k + 3) + blockIdx.x;
  const uint32_t m = blockIdx.x | 0x01010101u, n = threadIdx.x ^ 0x5a5a5a5au;
  for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (a[k] ^ m) & (a[k] | n);
  }
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) acc ^= a[k];
  if (acc == 0x5eedu) sink[0] = acc;
}

// 8 independent chains of 32-bit integer multiply-adds.
__global__ void __launch_bounds__(256) mb_imad_kernel(uint32_t iters, uint32_t* sink) {
  uint32_t a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * (k + 3) + blockIdx.x;
  const uint32_t m = blockIdx.x * 2u + 0x9E3779B9u, n = threadIdx.x + 17u;
  for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = a[k] * m + n;
  }
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) acc ^= a[k];
  if (acc == 0x5eedu) sink[0] = acc;
}

cudaError_t run_microbench(int kind, double* rate, double* ms_out) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = sms * 8, block = 256;
  uint32_t* sink = nullptr;
  cudaError_t e = cudaMalloc(&sink, 16);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const uint32_t iters = kind == 0 ? 4096u : 65536u;
  auto launch = [&]() {
    if (kind == 0)
      mb_philox_kernel<<<grid, block>>>(iters, sink);
    else if (kind == 1)
      mb_lop3_kernel<<<grid, block>>>(iters, sink);
    else
      mb_imad_kernel<<<grid, block>>>(iters, sink);
  };
  launch();  // warm-up
  cudaEventRecord(e0);
  for (int r = 0; r < 5; ++r) launch();
  cudaEventRecord(e1);
  e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  const double work = 5.0 * grid * block * (double)iters * (kind == 0 ? 1.0 : 8.0);
  *rate = ms > 0.0f ? work / (ms * 1e-3) : 0.0;
  if (ms_out) *ms_out = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  return e;
}

}  // namespace shk
