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
// lambda_x.  An fp32 evaluation of u (1 + e^{-2 beta h}) / 2^32 decides directly
// when it is farther than its error bound from 1 (see decide_int); otherwise T is
// computed in fp64.
// Real couplings (fp32 sums): tau_k = +1 iff u_k (1 + e~) / 2^32 < 1 (statistical parity).
#include <cstdint>

#include "shaken_internal.cuh"

namespace shk {

// 2^x (PTX ex2.approx: relative error below 2^-22 over the range used here).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Exact decision for integer couplings (see the header): +1 iff u < T(h, beta).
// With e~ = 2^(kb h~), kb = -2 beta log2(e), the condition u < 2^32 / (1 + e) is
// tested as t1 = (u + 1) 2^-32 (1 + e~) < 1 - eps (certainly +1) or
// t0 = u 2^-32 (1 + e~) > 1 + eps (certainly -1); eps = 2^-18 + 2^-18 beta B with
// B >= |s| + |q| + |lambda| + 1 is at least three times the fp32 error of t
// (rounding of h~, kb h~, ex2, the two products); in between, T is computed in fp64.
// The fp64 threshold test, out of line: it is reached with probability about
// 2^-17 (1 + beta B) per update, so it should not bloat the hot loop.
__device__ __noinline__ bool decide_exact(uint32_t u, int s, int sigma, double q, float lam,
                                          double beta) {
  const double h = field_h(1.0, s, q, sigma, (double)lam);
  return (unsigned long long)u < threshold_T(h, beta);
}

__device__ __forceinline__ bool decide_int(uint32_t u, int s, int sigma, float qf, double q,
                                           float lam, float kb, float eps, double beta,
                                           bool exact_always) {
  const float hf = __fadd_rn(__fadd_rn((float)s, sigma > 0 ? qf : -qf), lam);
  const float onep = 1.0f + ex2_approx(kb * hf);
  const float uf = __uint2float_rn(u) * 2.3283064365386963e-10f;
  if (!exact_always) {
    if ((uf + 2.3283064365386963e-10f) * onep < 1.0f - eps) return true;
    if (uf * onep > 1.0f + eps) return false;
  }
  return decide_exact(u, s, sigma, q, lam, beta);
}

// Number of neighbours y with J_xy s_y = +1 on lane k (slow path, one lane).
__device__ __noinline__ int lane_count(const uint32_t* __restrict__ src,
                                       const uint32_t* __restrict__ col, int p0, int p1, int k) {
  int cnt = 0;
  for (int e = p0; e < p1; ++e) {
    const uint32_t cv = col[e];
    cnt += (int)(((src[cv & 0x7fffffffu] ^ (0u - (cv >> 31))) >> k) & 1u);
  }
  return cnt;
}

// u_k of lane k of word (x, b) (slow path, one lane).
__device__ __noinline__ uint32_t lane_draw(uint32_t key0, uint32_t key1, uint32_t x, uint32_t b,
                                           uint32_t t, uint32_t typ, int k) {
  const uint4 w = ph_call(ph_key(key0, key1), x, b, t, typ + 2u * (uint32_t)(k >> 2));
  const int i = k & 3;
  return i == 0 ? w.x : i == 1 ? w.y : i == 2 ? w.z : w.w;
}

struct GraphShared;

// Fast decisions of the 32 lanes of a word (integer couplings, byte counters C):
// lane k = 8 c2 + m takes byte c2 of C[m] as its count and u_k from call k >> 2.
// With e~ = 2^(kb h~) the lane is +1 if (u + 1)(1 + e~) < 2^32 (1 - eps) and -1 if
// u (1 + e~) > 2^32 (1 + eps); otherwise its bit is set in `und` for the fp64 test.
// eps = 2^-18 + 2^-18 beta B, B = d + |q| + |lambda| + 1, is at least five times the
// fp32 error of the compared products (h~: three roundings of magnitude <= B;
// kb h~ -- with one beta on all lanes kb (2 cnt) + kb base, kb base rounded once,
// in one fused multiply-add, the same bound; ex2.approx, relative error 2^-22;
// 1 + e~; u to float; the product).
template <bool UNI>
__device__ __forceinline__ void int_lanes(const uint32_t (&C)[8], uint32_t S, const PhKey& K,
                                          uint32_t x, uint32_t b, uint32_t t, uint32_t typ,
                                          float bp, float bm, float a0, float B,
                                          const GraphShared& sh, bool fuse, float (*acc)[32],
                                          int lane, uint32_t& res, uint32_t& und);

struct GraphShared {
  float kb[32];   // -2 beta_k log2(e) per lane (anneal: the step's beta on every lane)
  float epc[32];  // 2^-18 beta_k per lane
  double beta[32];
  PhShared ph;    // Philox rounds shared by every call of the job at this step
  int uni;        // every lane has the same beta
  float acc[kTile / 32][32][32];  // [warp][replica lane k][thread lane]: tracking sums
  float red[kTile / 32][32];
};

template <bool UNI>
__device__ __forceinline__ void int_lanes(const uint32_t (&C)[8], uint32_t S, const PhKey& K,
                                          uint32_t x, uint32_t b, uint32_t t, uint32_t typ,
                                          float bp, float bm, float a0, float B,
                                          const GraphShared& sh, bool fuse, float (*acc)[32],
                                          int lane, uint32_t& res, uint32_t& und) {
  const float two32 = 4294967296.0f;
  float kb2 = 0.0f, kbp = 0.0f, kbm = 0.0f, lo0 = 0.0f, hi0 = 0.0f;
  if (UNI) {  // one beta: the exponent kb (2 cnt + base) is one fused multiply-add
    const float kb0 = sh.kb[0];
    kb2 = 2.0f * kb0;
    kbp = kb0 * bp;
    kbm = kb0 * bm;
    const float eps = 3.814697265625e-06f + sh.epc[0] * B;
    lo0 = two32 * (1.0f - eps);
    hi0 = two32 * (1.0f + eps);
  }
#pragma unroll 1
  for (uint32_t c2 = 0; c2 < 4u; ++c2) {
    const uint4 w0 = ph_call_shared(K, sh.ph, x, typ + 4u * c2);       // call 2 c2
    const uint4 w1 = ph_call_shared(K, sh.ph, x, typ + 4u * c2 + 2u);  // call 2 c2 + 1
    const uint32_t uw[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
    const uint32_t selb = 0x7540u + c2;  // byte c2 of C[m] under the exponent byte 0x4B
    const uint32_t s8 = S >> (8u * c2);  // sigma bits of lanes 8 c2 .. 8 c2 + 7
    uint32_t r8 = 0u, u8 = 0u;           // their decisions and undecided flags
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int k = 8 * (int)c2 + m;
      // count as a float: 2^23 + cnt exactly, minus 2^23
      const float cf = __fsub_rn(__int_as_float((int)__byte_perm(C[m], 0x4B000000u, selb)),
                                 8388608.0f);
      const bool up = (s8 >> m) & 1u;
      float x, lo = lo0, hi = hi0;
      if (UNI) {
        x = __fmaf_rn(kb2, cf, up ? kbp : kbm);
      } else {
        const float hf = __fmaf_rn(2.0f, cf, up ? bp : bm);
        x = sh.kb[k] * hf;
        const float eps = 3.814697265625e-06f + sh.epc[k] * B;
        lo = two32 * (1.0f - eps);
        hi = two32 * (1.0f + eps);
      }
      const float onep = 1.0f + ex2_approx(x);
      const float uf = __uint2float_rn(uw[m]);
      const bool plus = __fmaf_rn(uf, onep, onep) < lo;
      const bool minus = uf * onep > hi;
      r8 |= (uint32_t)plus << m;
      u8 |= (uint32_t)(!plus && !minus) << m;
      if (fuse) {
        const float a = __fmaf_rn(2.0f, cf, a0);
        acc[k][lane] += up ? a : -a;
      }
    }
    res |= r8 << (8u * c2);
    und |= u8 << (8u * c2);
  }
}

// One thread owns one (vertex, group) word.  Each block walks a contiguous range
// of tiles (one job per tile).  With tracking on, half 0 also accumulates per
// replica sum_x sigma_x (s_x + 2 lambda_x), i.e. -H(sigma_t) (Eq. (ham1)), reduced
// when the block leaves a job.
template <bool INTEGER>
__global__ void __launch_bounds__(kTile, 3) graph_half_kernel(const GraphJob* __restrict__ jobs,
                                                           const Tile* __restrict__ tiles,
                                                           int n_tiles, uint32_t half,
                                                           int exact_always) {
  __shared__ GraphShared sh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tb = (int)(((long long)blockIdx.x * n_tiles) / gridDim.x);
  const int te = (int)(((long long)(blockIdx.x + 1) * n_tiles) / gridDim.x);
  int cur_job = -1;
  bool fuse = false, skip = false;
  uint32_t t = 0, typ = 0;
  double* fuse_dst = nullptr;
  float(*acc)[32] = sh.acc[warp];  // acc[k][lane]: this thread's sum for replica lane k
#pragma unroll
  for (int k = 0; k < 32; ++k) acc[k][lane] = 0.0f;

  auto flush = [&]() {
    // block totals per replica lane -> step sums of the job's 32 replicas
    __syncthreads();
    {
      const int k = threadIdx.x & 31, w = threadIdx.x >> 5;  // row (w, k) of the accumulators
      float v = 0.0f;
#pragma unroll 8
      for (int l = 0; l < 32; ++l) v += sh.acc[w][k][(l + k) & 31];
      sh.red[w][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      float tot = 0.0f;
#pragma unroll
      for (int w = 0; w < kTile / 32; ++w) tot += sh.red[w][threadIdx.x];
      if (tot != 0.0f) atomicAdd(fuse_dst + (size_t)threadIdx.x * kNumSums + kSumE, (double)tot);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 32; ++k) acc[k][lane] = 0.0f;
  };

  for (int ti = tb; ti < te; ++ti) {
    const Tile tl = tiles[ti];
    const GraphJob& J = jobs[tl.job];
    if ((int)tl.job != cur_job) {
      if (fuse) flush();
      __syncthreads();  // shared per-job constants are about to change
      const CtxDev* cd = J.cd;
      t = cd->step;
      typ = half ^ cd->order;
      skip = t >= cd->t_end;
      fuse = !skip && half == 0u && cd->tracking && !cd->record && J.sums != nullptr;
      fuse_dst = J.sums;
      if (threadIdx.x < 32) {
        double beta;
        if (J.beta_sched != nullptr && cd->anneal_len != 0u) {
          uint32_t k = t - cd->anneal_t0;
          if (k >= cd->anneal_len) k = cd->anneal_len - 1u;
          beta = J.beta_sched[k];
        } else {
          beta = J.beta_lane[threadIdx.x];
        }
        sh.beta[threadIdx.x] = beta;
        sh.kb[threadIdx.x] = (float)(-2.0 * beta * 1.4426950408889634);
        sh.epc[threadIdx.x] = (float)beta * 3.814697265625e-06f;
        const double b0 = __shfl_sync(0xffffffffu, beta, 0);
        const bool same = __all_sync(0xffffffffu, beta == b0);
        if (threadIdx.x == 0) {
          sh.uni = same ? 1 : 0;
          sh.ph = ph_shared(ph_key(J.key0, J.key1), J.b, t);
        }
      }
      __syncthreads();
      cur_job = (int)tl.job;
    }
    if (skip) continue;
    const uint32_t x = tl.w0 + threadIdx.x;
    if (x >= J.n) continue;
    // `half` is the position in the step (buffers); typ the update type (neighbours, draws)
    const uint32_t* src = half == 0u ? J.A : J.B;
    uint32_t* dst = half == 0u ? J.B : J.A;
    const int32_t* ptr = typ == 0u ? J.in_ptr : J.out_ptr;
    const uint32_t* col = typ == 0u ? J.in_col : J.out_col;
    const float* Jr = typ == 0u ? J.in_J : J.out_J;
    const int32_t p0 = ptr[x], p1 = ptr[x + 1];
    const int d = p1 - p0;
    const uint32_t S = src[x];
    const uint32_t F = J.frozen != nullptr ? J.frozen[x] : 0u;
    const float lam = J.lambda != nullptr ? J.lambda[x] : J.lambda_c;
    const float qf = (float)J.q;
    const PhKey K = ph_key(J.key0, J.key1);
    uint32_t res = F;
    if (INTEGER) {
      const float B = (float)d + fabsf(qf) + fabsf(lam) + 1.0f;
      if (d <= 255) {
        // byte counters: byte i of C[m] = number of neighbours with J_xy s_y = +1 on
        // lane m + 8 i (at most d <= 255, so bytes never carry into each other)
        uint32_t C[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) C[m] = 0u;
        for (int e = p0; e < p1; ++e) {
          const uint32_t cv = __ldg(col + e);
          const uint32_t w = __ldg(src + (cv & 0x7fffffffu)) ^ (0u - (cv >> 31));
#pragma unroll
          for (int m = 0; m < 8; ++m) C[m] += (w >> m) & 0x01010101u;
        }
        // h = 2 cnt + (lambda - d +- q): one rounding in the fused multiply-add
        const float lmd = __fadd_rn(lam, -(float)d);
        const float bp = __fadd_rn(lmd, qf), bm = __fadd_rn(lmd, -qf);
        const float a0 = __fadd_rn(2.0f * lam, -(float)d);  // sigma (s + 2 lambda) = sigma (2 cnt + a0)
        uint32_t und = 0u;
        if (sh.uni)
          int_lanes<true>(C, S, K, x, J.b, t, typ, bp, bm, a0, B, sh, fuse, acc, lane, res, und);
        else
          int_lanes<false>(C, S, K, x, J.b, t, typ, bp, bm, a0, B, sh, fuse, acc, lane, res, und);
        while (und != 0u) {  // lanes inside the error bound of the fast test: fp64 threshold
          const int k = __ffs(und) - 1;
          und &= und - 1u;
          const int cnt = lane_count(src, col, p0, p1, k);
          const uint32_t u = lane_draw(J.key0, J.key1, x, J.b, t, typ, k);
          const int sigma = ((S >> k) & 1u) ? 1 : -1;
          res |= (uint32_t)decide_exact(u, 2 * cnt - d, sigma, J.q, lam, sh.beta[k]) << k;
        }
      } else {
#pragma unroll 1
        for (int k = 0; k < 32; ++k) {  // very high degree: one lane at a time
          const int cnt = lane_count(src, col, p0, p1, k);
          const uint32_t u = lane_draw(J.key0, J.key1, x, J.b, t, typ, k);
          const int s = 2 * cnt - d;
          const int sigma = ((S >> k) & 1u) ? 1 : -1;
          const float eps = 3.814697265625e-06f + sh.epc[k] * B;
          res |= (uint32_t)decide_int(u, s, sigma, qf, J.q, lam, sh.kb[k], eps, sh.beta[k],
                                      exact_always != 0) << k;
          if (fuse) {
            const float a = (float)s + 2.0f * lam;
            acc[k][lane] += sigma > 0 ? a : -a;
          }
        }
      }
      if (exact_always) {  // debugging aid: every lane through the fp64 threshold
        res = F;
#pragma unroll 1
        for (int k = 0; k < 32; ++k) {
          const int cnt = lane_count(src, col, p0, p1, k);
          const uint32_t u = lane_draw(J.key0, J.key1, x, J.b, t, typ, k);
          const int sigma = ((S >> k) & 1u) ? 1 : -1;
          res |= (uint32_t)decide_exact(u, 2 * cnt - d, sigma, J.q, lam, sh.beta[k]) << k;
        }
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
        if ((k & 3) == 0) w = ph_call_shared(K, sh.ph, x, typ + 2u * (uint32_t)(k >> 2));
        const uint32_t u = (k & 3) == 0 ? w.x : (k & 3) == 1 ? w.y : (k & 3) == 2 ? w.z : w.w;
        const bool up = (S >> k) & 1u;
        const float hk = __fadd_rn(__fadd_rn(h[k], up ? qf : -qf), lam);
        const float onep = 1.0f + ex2_approx(sh.kb[k] * hk);
        const float uf = __uint2float_rn(u) * 2.3283064365386963e-10f;
        res |= (uint32_t)(uf * onep < 1.0f) << k;
        if (fuse) {
          const float a = h[k] + 2.0f * lam;
          acc[k][lane] += up ? a : -a;
        }
      }
    }
    dst[x] = res;
  }
  if (fuse) flush();
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
  pdl_enter();
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
  (void)blocks_per_sm;
  if (n_tiles <= 0) return cudaSuccess;
  static int occ[2] = {0, 0};
  const int i = integer ? 1 : 0;
  if (occ[i] == 0) {
    int o = 1;
    if (integer)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, graph_half_kernel<true>, kTile, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, graph_half_kernel<false>, kTile, 0);
    occ[i] = o > 0 ? o : 1;
  }
  const int grid = grid_for(n_tiles, occ[i]);
  // a plain launch: with dependent launches the graph anneals ran 1-7% slower (the
  // blocks of a graph half step finish unevenly, and the next kernel's early blocks
  // then hold resources without work)
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
  return launch_dependent(graph_obs_kernel, dim3(grid_for(n_tiles, 4)), dim3(kTile), 0, st, jobs,
                          tiles, n_tiles, which, full);
}

cudaError_t launch_graph_fields(const GraphJob* jobs, const Tile* tiles, int n_tiles, uint32_t half,
                                float* out, cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  graph_fields_kernel<<<grid_for(n_tiles, 8), kTile, 0, st>>>(jobs, tiles, n_tiles, half, out);
  return cudaGetLastError();
}

}  // namespace shk
