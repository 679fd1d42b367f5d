// misc.cu -- the step epilogue and the stateless device primitives of libshaken.
#include <cstdint>

#include "shaken_internal.cuh"

namespace shk {

// One block per context.  After the two half steps of step t: if tracking, the
// energy of sigma_t (sums collected during the step) updates the per-replica
// best and the optional series, and the sums are cleared; then t += 1.
// H = -(Jc E) - 2 lamc M - 2 LS (Eq. (ham1); on the lattice Eq. (HGibbs)).
__global__ void __launch_bounds__(256) epilogue_kernel(CtxDev* const* __restrict__ ctxs, int n) {
  pdl_enter();
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

// Batched copies between the members' device arrays and one packed buffer, so
// that a batch moves its states and observables to or from the host in one
// transfer each.  Grid: x strides over a member's words, y = member.
__global__ void __launch_bounds__(256) pack_states_kernel(const MemberDev* __restrict__ m,
                                                          uint32_t* __restrict__ dst) {
  const MemberDev M = m[blockIdx.y];
  uint32_t* d = dst + M.state_off;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < M.state_words;
       i += (size_t)gridDim.x * blockDim.x)
    d[i] = M.A[i];
}

__global__ void __launch_bounds__(256) unpack_states_kernel(const MemberDev* __restrict__ m,
                                                            const uint32_t* __restrict__ src) {
  const MemberDev M = m[blockIdx.y];
  const uint32_t* s = src + M.state_off;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < M.state_words;
       i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t v = s[i];
    M.A[i] = v;
    M.B[i] = v;
  }
}

__global__ void __launch_bounds__(256) pack_obs_kernel(const MemberDev* __restrict__ m,
                                                       double* __restrict__ dst) {
  const MemberDev M = m[blockIdx.y];
  double* d = dst + M.obs_off;
  const uint32_t ns = M.R * (uint32_t)kNumSums;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ns + 2u * M.R;
       i += gridDim.x * blockDim.x) {
    double v;
    if (i < ns)
      v = M.obs[i];
    else if (i < ns + M.R)
      v = M.best[i - ns];
    else
      v = __longlong_as_double(M.best_step[i - ns - M.R]);
    d[i] = v;
  }
}

// Every member's observables sums set to zero (before the observables kernels add
// into them): one launch for the whole batch.
__global__ void __launch_bounds__(256) zero_obs_kernel(const MemberDev* __restrict__ m) {
  const MemberDev M = m[blockIdx.y];
  const uint32_t ns = M.R * (uint32_t)kNumSums;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += gridDim.x * blockDim.x)
    M.obs[i] = 0.0;
}

__global__ void __launch_bounds__(256) unpack_best_kernel(const MemberDev* __restrict__ m,
                                                          const double* __restrict__ src) {
  const MemberDev M = m[blockIdx.y];
  const double* s = src + M.obs_off + (size_t)M.R * kNumSums;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < M.R;
       i += gridDim.x * blockDim.x) {
    M.best[i] = s[i];
    M.best_step[i] = __double_as_longlong(s[M.R + i]);
  }
}

// what: 0 pack states, 1 unpack states, 2 pack observables, 3 unpack best energies,
// 4 zero the observables sums (buf unused)
cudaError_t launch_member_copy(int what, const MemberDev* m, int n, void* buf,
                               unsigned long long max_words, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (n > 65535) return cudaErrorInvalidConfiguration;  // one grid row per member
  unsigned long long bx = (max_words + 255ull) / 256ull;
  if (bx < 1ull) bx = 1ull;
  if (bx > 64ull) bx = 64ull;
  const dim3 grid((unsigned)bx, (unsigned)n);
  if (what == 0)
    pack_states_kernel<<<grid, 256, 0, st>>>(m, static_cast<uint32_t*>(buf));
  else if (what == 1)
    unpack_states_kernel<<<grid, 256, 0, st>>>(m, static_cast<const uint32_t*>(buf));
  else if (what == 2)
    pack_obs_kernel<<<grid, 256, 0, st>>>(m, static_cast<double*>(buf));
  else if (what == 3)
    unpack_best_kernel<<<grid, 256, 0, st>>>(m, static_cast<const double*>(buf));
  else
    zero_obs_kernel<<<grid, 256, 0, st>>>(m);
  return cudaGetLastError();
}

cudaError_t launch_epilogue(CtxDev* const* ctxs, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  return launch_dependent(epilogue_kernel, dim3(n), dim3(256), 0, st, ctxs, n);
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
    for (int k = 0; k < 8; ++k)  // one three-input logic instruction: (a ^ m) & (a | n)
      asm volatile("lop3.b32 %0, %1, %2, %3, 0x38;" : "=r"(a[k]) : "r"(a[k]), "r"(m), "r"(n));
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

// 4 chains of LOP3 interleaved with 4 chains of IMAD: if the logic and the
// multiply-add pipes overlapped, this would run at the sum of the two rates.
__global__ void __launch_bounds__(256) mb_mix_kernel(uint32_t iters, uint32_t* sink) {
  uint32_t a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * (k + 3) + blockIdx.x;
  const uint32_t m = blockIdx.x | 0x01010101u, n = threadIdx.x ^ 0x5a5a5a5au;
  for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      asm volatile("lop3.b32 %0, %1, %2, %3, 0x38;" : "=r"(a[k]) : "r"(a[k]), "r"(m), "r"(n));
      a[k + 4] = a[k + 4] * m + n;
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) acc ^= a[k];
  if (acc == 0x5eedu) sink[0] = acc;
}

// 8 chains of 32 x 32 -> 64-bit multiply-adds (the Philox multiply).
__global__ void __launch_bounds__(256) mb_imad_wide_kernel(uint32_t iters, uint32_t* sink) {
  unsigned long long p[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) p[k] = threadIdx.x * (k + 3) + blockIdx.x;
  const uint32_t m = blockIdx.x * 2u + 0xD2511F53u;
  for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t a = (uint32_t)(p[k] >> 32);
      asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(p[k]) : "r"(a), "r"(m));
    }
  }
  unsigned long long acc = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) acc ^= p[k];
  if (acc == 0x5eedull) sink[0] = (uint32_t)acc;
}

// 8 chains of 32 x 32 -> 64-bit products without an addend (the form of the
// Philox multiply): both halves of each product feed the next one.
__global__ void __launch_bounds__(256) mb_mul_wide_kernel(uint32_t iters, uint32_t* sink) {
  uint32_t a[8], b[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    a[k] = threadIdx.x * (k + 3) + blockIdx.x;
    b[k] = 0xD2511F53u + k;
  }
  for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      unsigned long long p;
      asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a[k]), "r"(b[k]));
      a[k] = (uint32_t)p;
      b[k] = (uint32_t)(p >> 32);
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) acc ^= a[k] ^ b[k];
  if (acc == 0x5eedu) sink[0] = acc;
}

// 4 chains of 64-bit products interleaved with 4 chains of LOP3.
__global__ void __launch_bounds__(256) mb_mix_wide_kernel(uint32_t iters, uint32_t* sink) {
  uint32_t a[4], b[4], c[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    a[k] = threadIdx.x * (k + 3) + blockIdx.x;
    b[k] = 0xD2511F53u + k;
    c[k] = threadIdx.x ^ (k * 0x01234567u);
  }
  const uint32_t m = blockIdx.x | 0x01010101u, n = threadIdx.x ^ 0x5a5a5a5au;
  for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      unsigned long long p;
      asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a[k]), "r"(b[k]));
      a[k] = (uint32_t)p;
      b[k] = (uint32_t)(p >> 32);
      asm volatile("lop3.b32 %0, %1, %2, %3, 0x38;" : "=r"(c[k]) : "r"(c[k]), "r"(m), "r"(n));
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) acc ^= a[k] ^ b[k] ^ c[k];
  if (acc == 0x5eedu) sink[0] = acc;
}

// Philox-4x32-10 with each 32 x 32 -> 64-bit product split into a high and a
// low 32-bit multiply (same values as ph_call), chained like mb_philox_kernel.
__device__ __forceinline__ uint4 ph_call_split(const PhKey& K, uint32_t c0, uint32_t c1,
                                               uint32_t c2, uint32_t c3) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t h0, l0, h1, l1;
    asm volatile("mul.hi.u32 %0, %1, %2;" : "=r"(h0) : "r"(c0), "n"(kPhM0));
    asm volatile("mul.lo.u32 %0, %1, %2;" : "=r"(l0) : "r"(c0), "n"(kPhM0));
    asm volatile("mul.hi.u32 %0, %1, %2;" : "=r"(h1) : "r"(c2), "n"(kPhM1));
    asm volatile("mul.lo.u32 %0, %1, %2;" : "=r"(l1) : "r"(c2), "n"(kPhM1));
    const uint32_t n0 = h1 ^ c1 ^ K.k0[r];
    const uint32_t n2 = h0 ^ c3 ^ K.k1[r];
    c1 = l1;
    c3 = l0;
    c0 = n0;
    c2 = n2;
  }
  return make_uint4(c0, c1, c2, c3);
}

__global__ void __launch_bounds__(256) mb_philox_split_kernel(uint32_t iters, uint32_t* sink) {
  const PhKey K = ph_key(0x1234u + threadIdx.x, 0x9876u ^ blockIdx.x);
  uint4 c = make_uint4(threadIdx.x, blockIdx.x, 7u, 9u);
  uint32_t acc = 0u;
  for (uint32_t i = 0; i < iters; ++i) {
    c = ph_call_split(K, c.x, c.y, c.z + i, c.w);
    acc ^= c.x ^ c.y ^ c.z ^ c.w;
  }
  if (acc == 0x5eedu) sink[0] = acc;
}

cudaError_t run_microbench(int kind, double* rate, double* ms_out) {
  if (kind < 0 || kind > 7) return cudaErrorInvalidValue;
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
  const uint32_t iters = (kind == 0 || kind == 7) ? 4096u : 65536u;
  auto launch = [&]() {
    if (kind == 0)
      mb_philox_kernel<<<grid, block>>>(iters, sink);
    else if (kind == 1)
      mb_lop3_kernel<<<grid, block>>>(iters, sink);
    else if (kind == 2)
      mb_imad_kernel<<<grid, block>>>(iters, sink);
    else if (kind == 3)
      mb_mix_kernel<<<grid, block>>>(iters, sink);
    else if (kind == 4)
      mb_imad_wide_kernel<<<grid, block>>>(iters, sink);
    else if (kind == 5)
      mb_mul_wide_kernel<<<grid, block>>>(iters, sink);
    else if (kind == 6)
      mb_mix_wide_kernel<<<grid, block>>>(iters, sink);
    else
      mb_philox_split_kernel<<<grid, block>>>(iters, sink);
  };
  launch();  // warm-up
  cudaEventRecord(e0);
  for (int r = 0; r < 5; ++r) launch();
  cudaEventRecord(e1);
  e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  const double work = 5.0 * grid * block * (double)iters * ((kind == 0 || kind == 7) ? 1.0 : 8.0);
  *rate = ms > 0.0f ? work / (ms * 1e-3) : 0.0;
  if (ms_out) *ms_out = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  return e;
}

}  // namespace shk
