// noalloc.cu -- observables of a caller-held lattice state without any allocation.
//
// Some callers cannot call cudaMalloc: code that owns all device memory through
// its own pool or caching allocator and must keep every byte accounted for
// there, and loops that cannot afford the device-wide synchronisation a
// cudaMalloc / cudaFree may imply.  shaken_lattice_observables_noalloc serves
// them: the caller passes the spin buffers it already holds and a host array
// for the result; the reduction scratch lives in the file-scope device arrays
// below, which every GPU that loads the library holds until the process exits.
//
// The arrays are shared by all calls on a device and keep the last call's
// contents: each call clears the sums it accumulates into before its kernel
// runs.  Calls that overlap on the GPU (different streams, or different host
// threads) race on the arrays; callers must serialise them.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <mutex>

#include "../../include/shaken.h"
#include "shaken_internal.cuh"

void shaken_internal_set_error(const char* msg);  // runtime.cu (last-error slot)

namespace shk {

constexpr int kNoAllocMaxReplicas = 4096;

// sums[r][8] for up to 4096 replicas (256 KiB) and the finished observables (224 KiB)
static __device__ __align__(256) double g_noalloc_sums[kNoAllocMaxReplicas * kNumSums];
static __device__ __align__(256) shaken_obs g_noalloc_obs[kNoAllocMaxReplicas];

struct NoAllocPtrs {
  double* sums = nullptr;
  shaken_obs* obs = nullptr;
  bool ready = false;
};

constexpr int kMaxDevices = 64;
static NoAllocPtrs g_ptrs[kMaxDevices];
static std::mutex g_ptrs_mu;

// Device addresses of the scratch arrays for the current device, looked up once
// per device (with that device current) on its first call.
static cudaError_t noalloc_ptrs(NoAllocPtrs* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_ptrs_mu);
  NoAllocPtrs& p = g_ptrs[dev];
  if (!p.ready) {
    void* s = nullptr;
    void* o = nullptr;
    e = cudaGetSymbolAddress(&s, g_noalloc_sums);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress(&o, g_noalloc_obs);
    if (e != cudaSuccess) return e;
    p.sums = static_cast<double*>(s);
    p.obs = static_cast<shaken_obs*>(o);
    p.ready = true;
  }
  *out = p;
  return cudaSuccess;
}

__device__ __forceinline__ uint32_t nb_bits4(uint32_t w) {
  const uint32_t pos = (~w >> 7) & 0x01010101u;
  return ((pos * 0x00204081u) >> 21) & 0xFu;
}
__device__ __forceinline__ uint32_t nb_bits32(const uint8_t* p) {
  const uint4 a = reinterpret_cast<const uint4*>(p)[0];
  const uint4 b = reinterpret_cast<const uint4*>(p)[1];
  return nb_bits4(a.x) | (nb_bits4(a.y) << 4) | (nb_bits4(a.z) << 8) | (nb_bits4(a.w) << 12) |
         (nb_bits4(b.x) << 16) | (nb_bits4(b.y) << 20) | (nb_bits4(b.z) << 24) |
         (nb_bits4(b.w) << 28);
}

// Lane word w of one replica / group: own bits and the neighbour bits a sum needs.
// dir 0: down and left neighbours, dir 1: up and right.
template <int ENC>
__device__ __forceinline__ void na_words(const void* buf, uint32_t L, uint32_t w, int dir,
                                         uint32_t& S, uint32_t& V, uint32_t& H) {
  const uint32_t wpr = ENC == SHAKEN_MULTISPIN ? L : L / 32u;
  const uint32_t i = w / wpr, c = w - i * wpr;
  const uint32_t iv = dir == 0 ? (i == 0u ? L - 1u : i - 1u) : (i + 1u == L ? 0u : i + 1u);
  if (ENC == SHAKEN_INT8) {
    const uint8_t* A = static_cast<const uint8_t*>(buf);
    S = nb_bits32(A + (size_t)i * L + 32u * c);
    V = nb_bits32(A + (size_t)iv * L + 32u * c);
    const uint32_t jn = dir == 0 ? (c == 0u ? L - 1u : 32u * c - 1u)
                                 : (32u * c + 32u == L ? 0u : 32u * c + 32u);
    const uint32_t nb = (A[(size_t)i * L + jn] >> 7) ^ 1u;
    H = dir == 0 ? ((S << 1) | nb) : ((S >> 1) | (nb << 31));
  } else if (ENC == SHAKEN_PACKED) {
    const uint32_t* A = static_cast<const uint32_t*>(buf);
    S = A[(size_t)i * wpr + c];
    V = A[(size_t)iv * wpr + c];
    if (dir == 0)
      H = (S << 1) | (A[(size_t)i * wpr + (c == 0u ? wpr - 1u : c - 1u)] >> 31);
    else
      H = (S >> 1) | (A[(size_t)i * wpr + (c + 1u == wpr ? 0u : c + 1u)] << 31);
  } else {
    const uint32_t* A = static_cast<const uint32_t*>(buf);
    S = A[w];
    V = A[(size_t)iv * L + c];
    H = A[(size_t)i * L + (dir == 0 ? (c == 0u ? L - 1u : c - 1u) : (c + 1u == L ? 0u : c + 1u))];
  }
}

// blockIdx.y = replica (INT8 / PACKED) or group (MULTISPIN); each thread adds the
// sums of its lane words to the scratch sums of the replica(s) it covers.
// INT8 / PACKED lane words hold 32 sites of one replica (popcounts); MULTISPIN
// lane words hold one site of 32 replicas (lane k -> replica 32 g + k).
template <int ENC>
__global__ void __launch_bounds__(256) noalloc_sums_kernel(const void* __restrict__ A,
                                                           const void* __restrict__ B,
                                                           uint32_t L, double* __restrict__ sums) {
  const uint32_t nwords = ENC == SHAKEN_MULTISPIN ? L * L : L * (L / 32u);
  const size_t job_bytes = ENC == SHAKEN_INT8 ? (size_t)L * L : (size_t)nwords * 4u;
  const uint32_t job = blockIdx.y;
  const void* a = static_cast<const uint8_t*>(A) + job_bytes * job;
  const void* b = static_cast<const uint8_t*>(B) + job_bytes * job;
  if (ENC != SHAKEN_MULTISPIN) {
    long long v[6] = {0, 0, 0, 0, 0, 0};
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nwords;
         w += gridDim.x * blockDim.x) {
      uint32_t S, V, H, S2, U2, R2;
      na_words<ENC>(a, L, w, 0, S, V, H);
      na_words<ENC>(b, L, w, 1, S2, U2, R2);
      const int dv = __popc(S ^ V), dh = __popc(S ^ H);
      v[0] += 2 * __popc(S) - 32;
      v[1] += 64 - 2 * dv - 2 * dh;
      v[2] += 64 - 2 * __popc(S ^ U2) - 2 * __popc(S ^ R2);
      v[3] += 32 - 2 * __popc(S ^ S2);
      v[4] += 2 * __popc(S2) - 32;
      v[5] += dv + dh;
    }
    const int slot[6] = {kSumM, kSumE, kSumP1, kSumP2, kSumM2, kSumCut};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      long long x = v[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) == 0 && x != 0)
        atomicAdd(&sums[(size_t)job * kNumSums + slot[q]], (double)x);
    }
  } else {
    // warps walk 32 consecutive sites; lane k accumulates replica 32 g + k
    const int lane = threadIdx.x & 31;
    long long v[6] = {0, 0, 0, 0, 0, 0};
    const uint32_t warps = gridDim.x * (blockDim.x / 32u);
    const uint32_t wid = blockIdx.x * (blockDim.x / 32u) + (threadIdx.x >> 5);
    for (uint32_t base = wid * 32u; base < nwords; base += warps * 32u) {
      const uint32_t w = base + lane;
      const bool act = w < nwords;
      uint32_t S = 0, V = 0, H = 0, S2 = 0, U2 = 0, R2 = 0;
      if (act) {
        na_words<ENC>(a, L, w, 0, S, V, H);
        na_words<ENC>(b, L, w, 1, S2, U2, R2);
      }
      const uint32_t m = act ? 0xffffffffu : 0u;
      const int nact = __popc(__ballot_sync(0xffffffffu, act));
      for (int k = 0; k < 32; ++k) {
        const int c0 = __popc(__ballot_sync(0xffffffffu, (S & m) >> k & 1u));
        const int c1 = __popc(__ballot_sync(0xffffffffu, (~(S ^ V) & m) >> k & 1u)) +
                       __popc(__ballot_sync(0xffffffffu, (~(S ^ H) & m) >> k & 1u));
        const int c2 = __popc(__ballot_sync(0xffffffffu, (~(S ^ U2) & m) >> k & 1u)) +
                       __popc(__ballot_sync(0xffffffffu, (~(S ^ R2) & m) >> k & 1u));
        const int c3 = __popc(__ballot_sync(0xffffffffu, (~(S ^ S2) & m) >> k & 1u));
        const int c4 = __popc(__ballot_sync(0xffffffffu, (S2 & m) >> k & 1u));
        if (lane == k) {
          v[0] += 2 * c0 - nact;
          v[1] += 2 * c1 - 2 * nact;
          v[2] += 2 * c2 - 2 * nact;
          v[3] += 2 * c3 - nact;
          v[4] += 2 * c4 - nact;
          v[5] += 2 * nact - c1;
        }
      }
    }
    const int slot[6] = {kSumM, kSumE, kSumP1, kSumP2, kSumM2, kSumCut};
    double* dst = sums + ((size_t)job * 32u + lane) * kNumSums;
#pragma unroll
    for (int q = 0; q < 6; ++q)
      if (v[q] != 0) atomicAdd(&dst[slot[q]], (double)v[q]);
  }
}

// Observables from the sums (same formulas as shaken_observables: Eq. (HGibbs)
// for the energy, Eq. (ham2) for the pair energy).
__global__ void noalloc_finish_kernel(const double* __restrict__ sums, int R, double N, double J,
                                      double q, double lam, shaken_obs* __restrict__ out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const double* s = sums + (size_t)r * kNumSums;
  shaken_obs o;
  o.magnetization = s[kSumM] / N;
  o.energy = -(J * s[kSumE]) - 2.0 * lam * s[kSumM];
  o.pair_energy = -(J * s[kSumP1] + q * s[kSumP2] + lam * (s[kSumM] + s[kSumM2]));
  o.best_energy = o.energy;
  o.best_step = -1;
  o.cut_edges = (int64_t)llrint(s[kSumCut]);
  o.cut_weight = -J * s[kSumCut];
  out[r] = o;
}

}  // namespace shk

extern "C" shaken_status shaken_lattice_observables_noalloc(
    const void* sigma_dev, const void* sigma_prime_dev, int32_t encoding, int64_t L,
    int32_t replicas, double J, double q, double lambda_const, shaken_obs* out_host,
    void* cuda_stream) {
  using namespace shk;
  auto bad = [](const char* m) {
    shaken_internal_set_error(m);
    return SHAKEN_E_INVAL;
  };
  auto cuda_fail = [](const char* what, cudaError_t e) {
    const std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    shaken_internal_set_error(m.c_str());
    return SHAKEN_E_CUDA;
  };
  if (!sigma_dev || !sigma_prime_dev || !out_host) return bad("NULL argument");
  if ((reinterpret_cast<uintptr_t>(sigma_dev) | reinterpret_cast<uintptr_t>(sigma_prime_dev)) & 15u)
    return bad("spin buffers must be 16-byte aligned");
  if (encoding < SHAKEN_INT8 || encoding > SHAKEN_MULTISPIN) return bad("bad encoding");
  if (L < 32 || L > 32768 || L % 32 != 0)
    return bad("L must be a multiple of 32 in [32, 32768]");
  if (replicas < 1 || replicas > kNoAllocMaxReplicas)
    return bad("replicas must be in [1, 4096]: the allocation-free scratch holds 4096 replicas");
  if (encoding == SHAKEN_MULTISPIN && replicas % 32 != 0)
    return bad("MULTISPIN needs replicas % 32 == 0");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  NoAllocPtrs p;
  if (noalloc_ptrs(&p) != cudaSuccess) {
    shaken_internal_set_error("cudaGetSymbolAddress of the scratch array failed");
    return SHAKEN_E_CUDA;
  }
  cudaError_t e = cudaMemsetAsync(p.sums, 0, sizeof(double) * kNumSums * (size_t)replicas, st);
  if (e != cudaSuccess) return cuda_fail("clearing the scratch sums", e);
  const uint32_t Lu = (uint32_t)L;
  const int jobs = encoding == SHAKEN_MULTISPIN ? replicas / 32 : replicas;
  const uint32_t nwords = encoding == SHAKEN_MULTISPIN ? Lu * Lu : Lu * (Lu / 32u);
  const dim3 grid((nwords + 255u) / 256u < 1024u ? (nwords + 255u) / 256u : 1024u, jobs);
  if (encoding == SHAKEN_INT8)
    noalloc_sums_kernel<SHAKEN_INT8><<<grid, 256, 0, st>>>(sigma_dev, sigma_prime_dev, Lu, p.sums);
  else if (encoding == SHAKEN_PACKED)
    noalloc_sums_kernel<SHAKEN_PACKED><<<grid, 256, 0, st>>>(sigma_dev, sigma_prime_dev, Lu,
                                                             p.sums);
  else
    noalloc_sums_kernel<SHAKEN_MULTISPIN><<<grid, 256, 0, st>>>(sigma_dev, sigma_prime_dev, Lu,
                                                                p.sums);
  noalloc_finish_kernel<<<(replicas + 127) / 128, 128, 0, st>>>(
      p.sums, replicas, (double)L * (double)L, J, q, lambda_const, p.obs);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail("observables launch", e);
  e = cudaMemcpyAsync(out_host, p.obs, sizeof(shaken_obs) * (size_t)replicas,
                      cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail("copy of the observables to the host", e);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail("stream synchronisation", e);
  return SHAKEN_OK;
}
