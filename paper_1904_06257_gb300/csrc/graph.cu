// graph.cu -- half-step kernel of the shaken dynamics on an arbitrary graph
// G = (V, E) (Sec. 2 of arXiv:1904.06257), multispin over replicas, and the
// graph observables.
//
// Half step 0 (P^{1->2}): h_x = sum_{y : (y -> x) in E^o} J_xy s_y + q s_x + lambda_x,
// half step 1 (P^{2->1}): h_x = sum_{y : (x -> y) in E^o} J_xy s'_y + q s'_x + lambda_x
// (the fields below Eq. (ham21)); tau_x = +1 with probability e^{beta h} / 2cosh(beta h).
//
// Layout: spins uint32 [R/32][n], bit k of word x of group g = replica 32g+k.
// In-CSR (sources of edges into x) for half 0, out-CSR (heads of edges out of
// x) for half 1; with integer couplings the sign of J is bit 31 of the column.
// One thread owns one (vertex, group) word and its 32 lanes.
//
// Draws: lane k of word (x, g) uses u_k = W_k, the k-th of the 32 words
// Philox(key, (x, g, t, half + 2(k>>2)))[k & 3].
//
// Decision, integer couplings (exact): tau_k = +1 iff u_k < T(h_k, beta_k)
// with T = floor(2^32 / (1 + e^{-2 beta h})) in fp64 and h = (s + q sigma) +
// lambda_x.  The fp32 probability p~ decides directly whenever u_k / 2^32 lies
// outside p~ +- eps, eps = 2^-20 (2 + beta B) + 2^-23 (B = |s| + |q| + |lambda| + 1)
// bounds |p~ - p| (fp32 rounding of h, beta, the exp argument, __expf and the
// reciprocal) with a factor >= 4 to spare; otherwise T is computed in fp64.
// Real couplings (fp32 sums): tau_k = +1 iff u_k / 2^32 < p~ (statistical parity).
#include <cstdint>

#include "shaken_internal.cuh"

namespace shk {

__device__ __forceinline__ float prob_f32(float h, float beta) {
  const float e = __expf(-2.0f * beta * h);
  return __frcp_rn(1.0f + e);
}

// Exact decision for integer couplings (see header).
__device__ __forceinline__ bool decide_int(uint32_t u, int s, int sigma, float qf, double q,
                                           float lam, float betaf, double beta, bool exact_always) {
  const float hf = __fadd_rn(__fadd_rn((float)s, sigma > 0 ? qf : -qf), lam);
  const float pf = prob_f32(hf, betaf);
  const float B = fabsf((float)s) + fabsf(qf) + fabsf(lam) + 1.0f;
  const float eps = 9.5367431640625e-07f * (2.0f + betaf * B) + 1.1920928955078125e-07f;
  const float uf = __uint2float_rn(u) * 2.3283064365386963e-10f;
  if (!exact_always) {
    if (uf + eps < pf) return true;
    if (uf - eps > pf) return false;
  }
  const double h = field_h(1.0, s, q, sigma, (double)lam);
  return (unsigned long long)u < threshold_T(h, beta);
}

template <bool INTEGER>
__global__ void __launch_bounds__(kTile) graph_half_kernel(const GraphJob* __restrict__ jobs,
                                                           const Tile* __restrict__ tiles,
                                                           int n_tiles, uint32_t half,
                                                           int exact_always) {
  for (int ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
    const Tile tl = tiles[ti];
    const GraphJob& J = jobs[tl.job];
    const CtxDev* cd = J.cd;
    const uint32_t t = cd->step;
    if (t >= cd->t_end) continue;
    const uint32_t x = tl.w0 + threadIdx.x;
    if (x >= J.n) continue;
    const uint32_t* src = half == 0u ? J.A : J.B;
    uint32_t* dst = half == 0u ? J.B : J.A;
    const int32_t* ptr = half == 0u ? J.in_ptr : J.out_ptr;
    const uint32_t* col = half == 0u ? J.in_col : J.out_col;
    const float* Jr = half == 0u ? J.in_J : J.out_J;
    const int32_t p0 = ptr[x], p1 = ptr[x + 1];
    const int d = p1 - p0;
    const uint32_t S = src[x];
    const uint32_t F = J.frozen != nullptr ? J.frozen[x] : 0u;
    const float lam = J.lambda != nullptr ? J.lambda[x] : J.lambda_c;
    const float qf = (float)J.q;
    bool anneal = J.beta_sched != nullptr && cd->anneal_len != 0u;
    double beta_a = 0.0;
    if (anneal) {
      uint32_t k = t - cd->anneal_t0;
      if (k >= cd->anneal_len) k = cd->anneal_len - 1u;
      beta_a = J.beta_sched[k];
    }
    const PhKey K = ph_key(J.key0, J.key1);
    uint32_t res = F;
    if (INTEGER) {
      // bit-sliced count of +1 contributions J_xy s_y over the neighbours
      uint32_t P[6] = {0u, 0u, 0u, 0u, 0u, 0u};
      if (d <= 63) {
        for (int e = p0; e < p1; ++e) {
          const uint32_t cv = col[e];
          uint32_t carry = src[cv & 0x7fffffffu] ^ (0u - (cv >> 31));
#pragma unroll
          for (int b = 0; b < 6; ++b) {
            const uint32_t tmp = P[b] & carry;
            P[b] ^= carry;
            carry = tmp;
          }
        }
      }
      uint4 w = make_uint4(0, 0, 0, 0);
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        if ((k & 3) == 0) w = ph_call(K, x, J.b, t, half + 2u * (uint32_t)(k >> 2));
        const uint32_t u = (k & 3) == 0 ? w.x : (k & 3) == 1 ? w.y : (k & 3) == 2 ? w.z : w.w;
        int cnt;
        if (d <= 63) {
          cnt = 0;
#pragma unroll
          for (int b = 0; b < 6; ++b) cnt |= (int)((P[b] >> k) & 1u) << b;
        } else {
          cnt = 0;
          for (int e = p0; e < p1; ++e) {
            const uint32_t cv = col[e];
            cnt += (int)(((src[cv & 0x7fffffffu] ^ (0u - (cv >> 31))) >> k) & 1u);
          }
        }
        const int s = 2 * cnt - d;
        const int sigma = ((S >> k) & 1u) ? 1 : -1;
        const double beta = anneal ? beta_a : J.beta_lane[k];
        const bool plus = decide_int(u, s, sigma, qf, J.q, lam, (float)beta, beta,
                                     exact_always != 0);
        res |= (uint32_t)plus << k;
      }
    } else {
      float h[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) h[k] = 0.0f;
      for (int e = p0; e < p1; ++e) {
        const uint32_t y = col[e] & 0x7fffffffu;
        const float Jv = Jr[e];
        const uint32_t wy = src[y];
#pragma unroll
        for (int k = 0; k < 32; ++k) h[k] += ((wy >> k) & 1u) ? Jv : -Jv;
      }
      uint4 w = make_uint4(0, 0, 0, 0);
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        if ((k & 3) == 0) w = ph_call(K, x, J.b, t, half + 2u * (uint32_t)(k >> 2));
        const uint32_t u = (k & 3) == 0 ? w.x : (k & 3) == 1 ? w.y : (k & 3) == 2 ? w.z : w.w;
        const float hk = __fadd_rn(__fadd_rn(h[k], ((S >> k) & 1u) ? qf : -qf), lam);
        const double beta = anneal ? beta_a : J.beta_lane[k];
        const float pf = prob_f32(hk, (float)beta);
        const float uf = __uint2float_rn(u) * 2.3283064365386963e-10f;
        res |= (uint32_t)(uf < pf) << k;
      }
    }
    dst[x] = res;
  }
}

// Fields h_x (float) of the next half step as the update kernel computes them.
__global__ void __launch_bounds__(kTile) graph_fields_kernel(const GraphJob* __restrict__ jobs,
                                                             const Tile* __restrict__ tiles,
                                                             int n_tiles, uint32_t half,
                                                             float* __restrict__ out) {
  for (int ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
    const Tile tl = tiles[ti];
    const GraphJob& J = jobs[tl.job];
    const uint32_t x = tl.w0 + threadIdx.x;
    if (x >= J.n) continue;
    const uint32_t* src = half == 0u ? J.A : J.B;
    const int32_t* ptr = half == 0u ? J.in_ptr : J.out_ptr;
    const uint32_t* col = half == 0u ? J.in_col : J.out_col;
    const float* Jr = half == 0u ? J.in_J : J.out_J;
    const uint32_t S = src[x];
    const float lam = J.lambda != nullptr ? J.lambda[x] : J.lambda_c;
    const float qf = (float)J.q;
    for (int k = 0; k < 32; ++k) {
      float hk;
      if (J.integer) {
        int s = 0;
        for (int e = ptr[x]; e < ptr[x + 1]; ++e) {
          const uint32_t cv = col[e];
          s += (((src[cv & 0x7fffffffu] ^ (0u - (cv >> 31))) >> k) & 1u) ? 1 : -1;
        }
        hk = __fadd_rn(__fadd_rn((float)s, ((S >> k) & 1u) ? qf : -qf), lam);
      } else {
        float a = 0.0f;
        for (int e = ptr[x]; e < ptr[x + 1]; ++e) {
          const float Jv = Jr[e];
          a += ((src[col[e] & 0x7fffffffu] >> k) & 1u) ? Jv : -Jv;
        }
        hk = __fadd_rn(__fadd_rn(a, ((S >> k) & 1u) ? qf : -qf), lam);
      }
      out[(size_t)(J.rep0 + k) * J.n + x] = hk;
    }
  }
}

// Initial spins: lane k = +1 iff u_k < 2^31 (draw of step 0xFFFFFFFF, half 0).
__global__ void __launch_bounds__(kTile) graph_init_kernel(const GraphJob* __restrict__ jobs,
                                                           const Tile* __restrict__ tiles,
                                                           int n_tiles, int kind) {
  for (int ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
    const Tile tl = tiles[ti];
    const GraphJob& J = jobs[tl.job];
    const uint32_t x = tl.w0 + threadIdx.x;
    if (x >= J.n) continue;
    uint32_t s = 0u;
    if (kind == 1) {
      s = 0xffffffffu;
    } else if (kind == 2) {
      s = 0u;
    } else {
      const PhKey K = ph_key(J.key0, J.key1);
      uint4 w = make_uint4(0, 0, 0, 0);
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        if ((k & 3) == 0) w = ph_call(K, x, J.b, kInitStep, 2u * (uint32_t)(k >> 2));
        const uint32_t u = (k & 3) == 0 ? w.x : (k & 3) == 1 ? w.y : (k & 3) == 2 ? w.z : w.w;
        s |= (uint32_t)(u < 0x80000000u) << k;
      }
    }
    if (J.frozen != nullptr) s |= J.frozen[x];
    J.A[x] = s;
    J.B[x] = s;
  }
}

// Observables: each warp walks 32 vertices of its tile; lane k accumulates the
// sums of replica 32g+k, then the block combines its warps and adds once.
__global__ void __launch_bounds__(kTile) graph_obs_kernel(const GraphJob* __restrict__ jobs,
                                                          const Tile* __restrict__ tiles,
                                                          int n_tiles, int which, int full) {
  __shared__ double red[kTile / 32][32][kNumSums];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
    const Tile tl = tiles[ti];
    const GraphJob& J = jobs[tl.job];
    double acc[kNumSums];
#pragma unroll
    for (int q = 0; q < kNumSums; ++q) acc[q] = 0.0;
    long long im = 0, iE = 0, iP1 = 0, iP2 = 0, icut = 0;
    const uint32_t xb = tl.w0 + 32u * warp;
    for (uint32_t xi = 0; xi < 32u; ++xi) {
      const uint32_t x = xb + xi;
      if (x >= J.n) break;
      const int sx = ((J.A[x] >> lane) & 1u) ? 1 : -1;
      const float lam = J.lambda != nullptr ? J.lambda[x] : J.lambda_c;
      im += sx;
      acc[kSumLS] += (double)(lam * (float)sx);
      float eacc = 0.0f;
      for (int e = J.in_ptr[x]; e < J.in_ptr[x + 1]; ++e) {
        const uint32_t cv = J.in_col[e];
        const int sy = ((J.A[cv & 0x7fffffffu] >> lane) & 1u) ? 1 : -1;
        icut += (sx != sy);
        if (J.integer) {
          iE += (cv >> 31) ? -sx * sy : sx * sy;
        } else {
          eacc += J.in_J[e] * (float)(sx * sy);
        }
      }
      acc[kSumE] += (double)eacc;
      if (full) {
        const int s2 = ((J.B[x] >> lane) & 1u) ? 1 : -1;
        iP2 += sx * s2;
        acc[kSumLS2] += (double)(lam * (float)s2);
        float pacc = 0.0f;
        for (int e = J.out_ptr[x]; e < J.out_ptr[x + 1]; ++e) {
          const uint32_t cv = J.out_col[e];
          const int sy = ((J.B[cv & 0x7fffffffu] >> lane) & 1u) ? 1 : -1;
          if (J.integer) {
            iP1 += (cv >> 31) ? -sx * sy : sx * sy;
          } else {
            pacc += J.out_J[e] * (float)(sx * sy);
          }
        }
        acc[kSumP1] += (double)pacc;
      }
    }
    acc[kSumM] = (double)im;
    acc[kSumE] += (double)iE;
    acc[kSumP1] += (double)iP1;
    acc[kSumP2] = (double)iP2;
    acc[kSumCut] = (double)icut;
#pragma unroll
    for (int q = 0; q < kNumSums; ++q) red[warp][lane][q] = acc[q];
    __syncthreads();
    if (threadIdx.x < 32) {
      double* dst = (which ? J.obs : J.sums) + (size_t)threadIdx.x * kNumSums;
#pragma unroll
      for (int q = 0; q < kNumSums; ++q) {
        if (q == kSumM2) continue;
        if (!full && (q == kSumP1 || q == kSumP2 || q == kSumLS2)) continue;
        double s = 0.0;
        for (int wv = 0; wv < kTile / 32; ++wv) s += red[wv][threadIdx.x][q];
        if (s != 0.0) atomicAdd(dst + q, s);
      }
    }
    __syncthreads();
  }
}

static int grid_for(int n_tiles, int per_sm) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int g = sms * per_sm;
  return n_tiles < g ? (n_tiles > 0 ? n_tiles : 1) : g;
}

cudaError_t launch_graph_half(bool integer, const GraphJob* jobs, const Tile* tiles, int n_tiles,
                              uint32_t half, int exact_always, int blocks_per_sm, cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  const int grid = grid_for(n_tiles, blocks_per_sm);
  if (integer)
    graph_half_kernel<true><<<grid, kTile, 0, st>>>(jobs, tiles, n_tiles, half, exact_always);
  else
    graph_half_kernel<false><<<grid, kTile, 0, st>>>(jobs, tiles, n_tiles, half, exact_always);
  return cudaGetLastError();
}

cudaError_t launch_graph_init(const GraphJob* jobs, const Tile* tiles, int n_tiles, int kind,
                              cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  graph_init_kernel<<<grid_for(n_tiles, 8), kTile, 0, st>>>(jobs, tiles, n_tiles, kind);
  return cudaGetLastError();
}

cudaError_t launch_graph_obs(const GraphJob* jobs, const Tile* tiles, int n_tiles, int which,
                             int full, cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  graph_obs_kernel<<<grid_for(n_tiles, 4), kTile, 0, st>>>(jobs, tiles, n_tiles, which, full);
  return cudaGetLastError();
}

cudaError_t launch_graph_fields(const GraphJob* jobs, const Tile* tiles, int n_tiles, uint32_t half,
                                float* out, cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  graph_fields_kernel<<<grid_for(n_tiles, 8), kTile, 0, st>>>(jobs, tiles, n_tiles, half, out);
  return cudaGetLastError();
}

}  // namespace shk
