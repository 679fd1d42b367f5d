// graph.cu -- half-step kernels of the shaken dynamics on an arbitrary graph
// G = (V, E) (Sec. 2 of arXiv:1904.06257), multispin over replicas, and the
// graph observables.
//
// Half step 0 (P^{1->2}): h_x = sum_{y : (y -> x) in E^o} J_xy s_y + q s_x + lambda_x,
// half step 1 (P^{2->1}): h_x = sum_{y : (x -> y) in E^o} J_xy s'_y + q s'_x + lambda_x
// (the fields below Eq. (ham21)); tau_x = +1 with probability e^{beta h} / 2cosh(beta h).
//
// Layout: spins uint32 [n][G], word x * G + g = vertex x of replicas 32 g .. 32 g + 31
// (bit k = replica 32 g + k).  In-CSR (sources of edges into x) for half 0, out-CSR
// (heads of edges out of x) for half 1; with integer couplings the sign of J is bit
// 31 of the column.  One thread owns one (vertex, group) word and its 32 lanes; the
// group words of a vertex are owned by adjacent threads, so they share the column
// loads and the neighbours' words arrive in common sectors.
//
// Integer couplings (exact).  Draws by bit planes: plane j of word (x, g) is
// W_j = Philox(key, (x, g, t, half + 2(j>>2)))[j & 3], and lane k's draw has bit 31-j
// equal to bit k of W_j.  Lane k is +1 iff u_k < T = floor(2^32 / (1 + e^{-2 beta h})).
// With one beta on every lane of a job (anneals), the threshold depends on the lane
// only through its class (a, sigma): a = number of in-neighbours with J s = +1, so
// h = (2a - d) + q sigma + lambda_x.  The threads of a vertex compute the top byte of
// T for each class of the vertex once (fp32 with a proven error bound; a class whose
// top byte the bound does not fix is marked), the lanes pick theirs by byte permutes,
// a bit transpose turns the 32 bytes into 8 threshold planes, and planes 0..7 (two
// Philox calls) decide every lane whose draw differs from its threshold in the top
// byte.  The rest (about 2^-8 of the lanes) is decided one lane at a time: more
// planes against the fp32 bounds on T, and T in fp64 where even they do not decide.
// Real couplings (fp32 sums): direct draws u_k = W_k and tau_k = +1 iff
// u_k (1 + e~) / 2^32 < 1 (statistical parity).
// Vertices of degree above 255 are left to graph_hub_kernel: their edge lists are cut
// into chunks of 2048 edges, one warp per (chunk, group) combines its lanes' counts or
// fields by a butterfly of shuffles, and the warp finishing a word's last chunk adds
// the chunk sums in chunk order and decides the word.  A job's tiles are listed so
// that the high-degree end of the visiting order spreads over the blocks.
#include <cstdint>

#include "shaken_internal.cuh"

namespace shk {

constexpr int kTableDeg = 31;  // per-vertex class tables for degree <= 31
// byte counters for degree <= kHubDeg (shaken_internal.cuh); above: graph_hub_kernel

// 2^x (PTX ex2.approx: relative error below 2^-22 over the range used here).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Bounds lo <= T <= hi on T = floor(2^32 / (1 + 2^x)), x = kb h, kb = -2 beta log2(e),
// from the fp32 field hf.  hf carries at most four roundings of magnitude <= B
// (B = d + |q| + |lambda| + 1), so kb hf is within |kb| B 2^-22 of kb h; with the
// rounding of kb hf, ex2.approx (2^-22), 1 + e, the reciprocal and the product, T~ is
// within min(T~, 2^32 - T~) eps + 2^8 of 2^32 p, eps = 2^-21 (2 + |x| + |kb| B)
// bounding twice the relative error; the margin 1024 also covers the floor.
__device__ __forceinline__ void t_bounds(float hf, float kb, float kbB, float& lo, float& hi) {
  const float x = kb * hf;
  const float e = ex2_approx(x);
  const float T = 4294967296.0f * rcp_approx(1.0f + e);
  const float m = fminf(T, 4294967296.0f - T);
  const float eps = 4.76837158203125e-07f * (2.0f + fabsf(x) + kbB);
  const float D = fmaf(m, eps, 1024.0f);
  lo = fmaxf(T - D, 0.0f);
  hi = fminf(T + D, 4294967296.0f);
}

// A field of exactly 0 gives T = 2^31 exactly (p = 1/2), on a byte boundary where the
// fp32 bounds cannot fix the top byte: with integer couplings and lambda = 0 (or q
// canceling lambda) it is a whole class of lanes.  When the fp32 field is 0, the fp64
// field (the rounding order of the threshold's definition) decides whether T is
// exactly 2^31.
__device__ __noinline__ bool field_is_zero(int s, int sig, double q, float lam) {
  return field_h(1.0, s, q, sig ? 1 : -1, (double)lam) == 0.0;
}

// Top byte of a value in [0, 2^32] (2^32, i.e. T that always accepts, maps to 255: a
// lane whose draw has top byte 255 is then left to the per-lane decision).
__device__ __forceinline__ uint32_t top_byte(float v) {
  const uint32_t b = __float2uint_rz(v * 5.9604644775390625e-08f);
  return b > 255u ? 255u : b;
}

// Bit transpose: R[m] byte i = threshold byte of lane m + 8 i  ->  P[j] bit k = bit 7 - j
// of the byte of lane k (plane j, most significant first).  Two 4 x 4 byte transposes
// gather the 8 x 8 bit blocks of lanes 8 i .. 8 i + 7, a three-stage delta swap
// transposes each block, two more byte transposes scatter the rows into planes.
__device__ __forceinline__ void t44(uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d) {
  const uint32_t t0 = __byte_perm(a, b, 0x5140), t1 = __byte_perm(a, b, 0x7362);
  const uint32_t t2 = __byte_perm(c, d, 0x5140), t3 = __byte_perm(c, d, 0x7362);
  a = __byte_perm(t0, t2, 0x5410);
  b = __byte_perm(t0, t2, 0x7632);
  c = __byte_perm(t1, t3, 0x5410);
  d = __byte_perm(t1, t3, 0x7632);
}

__device__ __forceinline__ void t88(uint32_t& lo, uint32_t& hi) {
  uint32_t t;
  t = (lo ^ (lo >> 7)) & 0x00AA00AAu;
  lo ^= t ^ (t << 7);
  t = (hi ^ (hi >> 7)) & 0x00AA00AAu;
  hi ^= t ^ (t << 7);
  t = (lo ^ (lo >> 14)) & 0x0000CCCCu;
  lo ^= t ^ (t << 14);
  t = (hi ^ (hi >> 14)) & 0x0000CCCCu;
  hi ^= t ^ (t << 14);
  t = (lo ^ __funnelshift_r(lo, hi, 28)) & 0xF0F0F0F0u;
  lo ^= t ^ (t << 28);
  hi ^= t >> 4;
}

__device__ __forceinline__ void bytes_to_planes(uint32_t (&R)[8], uint32_t (&P)[8]) {
  t44(R[0], R[1], R[2], R[3]);
  t44(R[4], R[5], R[6], R[7]);
  t88(R[0], R[4]);
  t88(R[1], R[5]);
  t88(R[2], R[6]);
  t88(R[3], R[7]);
  t44(R[0], R[1], R[2], R[3]);
  t44(R[4], R[5], R[6], R[7]);
#pragma unroll
  for (int j = 0; j < 8; ++j) P[j] = R[7 - j];
}

// Threshold bytes of lanes m + 8 i (byte i) from the class table of their vertex:
// Tm / Tp hold the top bytes for sigma = -1 / +1 and a = 0 .. 8 NW - 1 (4 per word);
// cnt holds the lanes' counts a (bytes), sbits their sigma bits (bit 8 i).  Byte
// permutes pick 8 entries at a time by the low three bits of a, byte masks the rest.
template <int NW>
__device__ __forceinline__ uint32_t lookup_bytes(const uint32_t (&Tm)[8], const uint32_t (&Tp)[8],
                                                 uint32_t cnt, uint32_t sbits) {
  const uint32_t x7 = cnt & 0x07070707u;
  const uint32_t sel = __byte_perm(x7 | (x7 >> 4), 0u, 0x0020);
  uint32_t vm = __byte_perm(Tm[0], Tm[1], sel), vp = __byte_perm(Tp[0], Tp[1], sel);
  if (NW >= 2) {
    const uint32_t m8 = ((cnt >> 3) & 0x01010101u) * 0xFFu;
    vm = (__byte_perm(Tm[2], Tm[3], sel) & m8) | (vm & ~m8);
    vp = (__byte_perm(Tp[2], Tp[3], sel) & m8) | (vp & ~m8);
    if (NW == 4) {
      const uint32_t m16 = ((cnt >> 4) & 0x01010101u) * 0xFFu;
      const uint32_t hm = (__byte_perm(Tm[6], Tm[7], sel) & m8) | (__byte_perm(Tm[4], Tm[5], sel) & ~m8);
      const uint32_t hp = (__byte_perm(Tp[6], Tp[7], sel) & m8) | (__byte_perm(Tp[4], Tp[5], sel) & ~m8);
      vm = (hm & m16) | (vm & ~m16);
      vp = (hp & m16) | (vp & ~m16);
    }
  }
  const uint32_t ms = sbits * 0xFFu;
  return (vp & ms) | (vm & ~ms);
}

// The same for collapsed classes (q = 1): one table T over a' = a + sigma, cnt holding
// a' in bytes.
template <int NW>
__device__ __forceinline__ uint32_t lookup_bytes_c(const uint32_t (&T)[8], uint32_t cnt) {
  const uint32_t x7 = cnt & 0x07070707u;
  const uint32_t sel = __byte_perm(x7 | (x7 >> 4), 0u, 0x0020);
  uint32_t v = __byte_perm(T[0], T[1], sel);
  if (NW >= 2) {
    const uint32_t m8 = ((cnt >> 3) & 0x01010101u) * 0xFFu;
    v = (__byte_perm(T[2], T[3], sel) & m8) | (v & ~m8);
    if (NW == 4) {
      const uint32_t m16 = ((cnt >> 4) & 0x01010101u) * 0xFFu;
      const uint32_t h = (__byte_perm(T[6], T[7], sel) & m8) | (__byte_perm(T[4], T[5], sel) & ~m8);
      v = (h & m16) | (v & ~m16);
    }
  }
  return v;
}

// Bits k of eight plane words, most significant first.
__device__ __forceinline__ uint32_t lane_byte(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3,
                                              uint32_t w4, uint32_t w5, uint32_t w6, uint32_t w7,
                                              int k) {
  return (((w0 >> k) & 1u) << 7) | (((w1 >> k) & 1u) << 6) | (((w2 >> k) & 1u) << 5) |
         (((w3 >> k) & 1u) << 4) | (((w4 >> k) & 1u) << 3) | (((w5 >> k) & 1u) << 2) |
         (((w6 >> k) & 1u) << 1) | ((w7 >> k) & 1u);
}

// Decision of one lane left undecided by the head (its draw's top byte u8 equals the
// threshold's, or its class's top byte was not certain): planes 8..15 and then 16..31
// against the fp32 bounds on T, and T in fp64 where the bounds do not decide
// (force_exact: straight to fp64).  Out of line: reached by about 2^-8 of the lanes.
__device__ __noinline__ bool decide_lane(uint32_t key0, uint32_t key1, uint32_t x, uint32_t g,
                                         uint32_t t, uint32_t typ, int k, uint32_t u8, int a,
                                         int d, int sig, float bp, float bm, double q, float lam,
                                         float kb, float kbB, double beta, bool force_exact) {
  float lo = 0.0f, hi = 4294967296.0f;
  if (!force_exact) {
    const float hf = fmaf(2.0f, (float)a, sig ? bp : bm);
    t_bounds(hf, kb, kbB, lo, hi);
    if (hf == 0.0f && field_is_zero(2 * a - d, sig, q, lam)) lo = hi = 2147483648.0f;  // T = 2^31
    if ((float)(u8 + 1u) * 16777216.0f <= lo) return true;  // u < (u8 + 1) 2^24 <= T
    if ((float)u8 * 16777216.0f >= hi) return false;        // u >= u8 2^24 >= T
  }
  const PhKey K = ph_key(key0, key1);
  const uint4 c2 = ph_call(K, x, g, t, typ + 4u), c3 = ph_call(K, x, g, t, typ + 6u);
  const uint32_t u16 = (u8 << 8) | lane_byte(c2.x, c2.y, c2.z, c2.w, c3.x, c3.y, c3.z, c3.w, k);
  if (!force_exact) {
    if ((float)(u16 + 1u) * 65536.0f <= lo) return true;
    if ((float)u16 * 65536.0f >= hi) return false;
  }
  const uint4 c4 = ph_call(K, x, g, t, typ + 8u), c5 = ph_call(K, x, g, t, typ + 10u);
  const uint4 c6 = ph_call(K, x, g, t, typ + 12u), c7 = ph_call(K, x, g, t, typ + 14u);
  const uint32_t u = (u16 << 16) |
                     (lane_byte(c4.x, c4.y, c4.z, c4.w, c5.x, c5.y, c5.z, c5.w, k) << 8) |
                     lane_byte(c6.x, c6.y, c6.z, c6.w, c7.x, c7.y, c7.z, c7.w, k);
  if (!force_exact) {
    if ((double)u < (double)lo) return true;
    if ((double)u >= (double)hi) return false;
  }
  const double h = field_h(1.0, 2 * a - d, q, sig ? 1 : -1, (double)lam);
  return (unsigned long long)u < threshold_T(h, beta);
}

// Threshold bytes of lanes m, m + 8, m + 16, m + 24 one lane at a time (per-lane betas,
// or a degree above the class tables): .x = bytes (byte i for lane m + 8 i), .y = the
// lanes whose top byte is not certain (bit k).
__device__ __noinline__ uint2 lane_bytes(uint32_t cnt, uint32_t S, int m, float bp, float bm,
                                         float B, const double* __restrict__ beta_lane,
                                         float kb_uni, bool uni, int d, double q, float lam) {
  float kbl[4];
  if (uni) {  // (kept out of the lane loop: an fp64 product per lane is slow here)
#pragma unroll
    for (int i = 0; i < 4; ++i) kbl[i] = kb_uni;
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) kbl[i] = (float)(-2.0 * beta_lane[m + 8 * i] * 1.4426950408889634);
  }
  uint32_t r = 0u, am = 0u;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = m + 8 * i;
    const int a = (int)((cnt >> (8 * i)) & 0xFFu);
    const int sig = (int)((S >> k) & 1u);
    const float hf = fmaf(2.0f, (float)a, sig ? bp : bm);
    float lo, hi;
    t_bounds(hf, kbl[i], fabsf(kbl[i]) * B, lo, hi);
    uint32_t bl = top_byte(lo), bh = top_byte(hi);
    if (hf == 0.0f && field_is_zero(2 * a - d, sig, q, lam)) bl = bh = 0x80u;  // T = 2^31
    r |= bh << (8 * i);
    am |= (uint32_t)(bl != bh) << k;
  }
  return make_uint2(r, am);
}

// Real couplings: the decisions of the 32 lanes from their fp32 fields h[k] (direct
// draws u_k = W_k of calls k >> 2); UNI: one beta on every lane (no per-lane fp64).
template <bool UNI>
__device__ __forceinline__ uint32_t real_lanes(const float (&h)[32], uint32_t S, float qf,
                                               float lam, float kbu,
                                               const double* __restrict__ beta_g,
                                               const PhKey& K, const PhShared& ph, uint32_t x,
                                               uint32_t typ, bool fuse, float (*acc)[32],
                                               int lane) {
  uint32_t res = 0u;
  uint4 w = make_uint4(0, 0, 0, 0);
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if ((k & 3) == 0) w = ph_call_shared(K, ph, x, typ + 2u * (uint32_t)(k >> 2));
    const uint32_t u = (k & 3) == 0 ? w.x : (k & 3) == 1 ? w.y : (k & 3) == 2 ? w.z : w.w;
    const bool up = (S >> k) & 1u;
    const float kb = UNI ? kbu : (float)(-2.0 * beta_g[k] * 1.4426950408889634);
    const float hk = __fadd_rn(__fadd_rn(h[k], up ? qf : -qf), lam);
    const float onep = 1.0f + ex2_approx(kb * hk);
    const float uf = __uint2float_rn(u) * 2.3283064365386963e-10f;
    res |= (uint32_t)(uf * onep < 1.0f) << k;
    if (fuse) {
      const float a = h[k] + 2.0f * lam;
      acc[k][lane] += up ? a : -a;
    }
  }
  return res;
}

// Per-replica partial values v[0..31] of the 32 lanes of a warp -> lane k holds the
// sum over the warp of v[k] in v[0] (each level halves the values a lane keeps).
template <typename V>
__device__ __forceinline__ V warp_transpose_sum(V (&v)[32], int lane) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const V send = up ? v[i] : v[i + s];
      const V keep = up ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  return v[0];
}

// Sum over the chunk's edges [e0, e1) of word (., g), lane l taking edges e0 + l,
// e0 + l + 32, ...; returns lane k's value for replica k: the number of neighbours
// with J_xy s_y = +1 (integer couplings; byte counters, at most kHubChunk / 32 = 64
// edges per lane) or the float sum of J_xy s_y (real couplings, as its bits).
template <bool INTEGER>
__device__ __forceinline__ uint32_t hub_chunk_sum(const uint32_t* src, const uint32_t* col,
                                                  const float* Jr, uint32_t e0, uint32_t e1,
                                                  uint32_t G, uint32_t g, int lane) {
  if (INTEGER) {
    uint32_t C[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) C[m] = 0u;
    for (uint32_t e = e0 + (uint32_t)lane; e < e1; e += 32u) {
      const uint32_t cv = __ldg(col + e);
      const uint32_t w = __ldg(src + (size_t)(cv & 0x7fffffffu) * G + g) ^ (0u - (cv >> 31));
#pragma unroll
      for (int m = 0; m < 8; ++m) C[m] += (w >> m) & 0x01010101u;
    }
    uint32_t v[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = (C[k & 7] >> (8 * (k >> 3))) & 0xFFu;
    return warp_transpose_sum(v, lane);
  }
  float v[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = 0.0f;
  for (uint32_t e = e0 + (uint32_t)lane; e < e1; e += 32u) {
    const uint32_t y = __ldg(col + e) & 0x7fffffffu;
    const float Jv = __ldg(Jr + e);
    const uint32_t wy = __ldg(src + (size_t)y * G + g);
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] += ((wy >> k) & 1u) ? Jv : -Jv;
  }
  return __float_as_uint(warp_transpose_sum(v, lane));
}

// Words of the vertices of degree above kHubDeg in the half step's direction, one
// warp per (chunk of kHubChunk edges, group): the warp sums its chunk into a partial
// row, and the warp that finishes a word's last chunk adds the rows in chunk order
// (the same sum whichever warp comes last), resets the word's counter and decides
// the 32 replicas, lane k replica k (integer: T in fp64 and the plane-assembled
// draw; real: the fp32 test of the direct draw).  Runs after the half-step kernel,
// which leaves these words alone.
template <bool INTEGER>
__global__ void __launch_bounds__(kTile) graph_hub_kernel(const GraphJob* __restrict__ jobs,
                                                          const HubItem* __restrict__ items,
                                                          const uint32_t* __restrict__ unit_item,
                                                          int n_units, uint32_t half,
                                                          uint32_t* __restrict__ partial,
                                                          uint32_t* __restrict__ done) {
  const int lane = threadIdx.x & 31;
  const int u = blockIdx.x * (kTile / 32) + (threadIdx.x >> 5);
  if (u >= n_units) return;  // the whole warp
  const HubItem it = items[unit_item[u]];
  const GraphJob& J = jobs[it.job];
  const CtxDev* cd = J.cd;
  const uint32_t t = cd->step;
  if (t >= cd->t_end) return;
  const uint32_t typ = half ^ cd->order;
  if (it.dir != typ) return;  // the other direction's vertices
  const uint32_t go = (uint32_t)u - it.ubase, g = J.g0 + go, G = J.G;
  const uint32_t* src = half == 0u ? J.A : J.B;
  uint32_t* dst = half == 0u ? J.B : J.A;
  const uint32_t* col = typ == 0u ? J.in_col : J.out_col;
  const float* Jr = typ == 0u ? J.in_J : J.out_J;
  const uint32_t v = hub_chunk_sum<INTEGER>(src, col, Jr, it.e0, it.e1, G, g, lane);
  uint32_t* rows = partial + (size_t)(it.pbase + go * it.nchunks) * 32u;
  rows[it.chunk * 32u + (uint32_t)lane] = v;
  __threadfence();
  __syncwarp();
  uint32_t last = 0u;
  if (lane == 0) last = atomicAdd(done + it.dbase + go, 1u) == it.nchunks - 1u ? 1u : 0u;
  if (__shfl_sync(0xffffffffu, last, 0) == 0u) return;
  __threadfence();
  if (lane == 0) done[it.dbase + go] = 0u;  // ready for the next half step
  const uint32_t x = it.x;
  const int32_t* ptr = typ == 0u ? J.in_ptr : J.out_ptr;
  const int d = ptr[x + 1] - ptr[x];
  const uint32_t S = src[(size_t)x * G + g];
  const uint32_t F = J.frozen != nullptr ? J.frozen[x] : 0u;
  const float lam = J.lambda != nullptr ? J.lambda[x] : J.lambda_c;
  double beta;
  if (J.beta_sched != nullptr && cd->anneal_len != 0u) {
    uint32_t k = t - cd->anneal_t0;
    if (k >= cd->anneal_len) k = cd->anneal_len - 1u;
    beta = J.beta_sched[k];
  } else {
    beta = J.beta_lane[32u * g + (uint32_t)lane];
  }
  const bool fuse = half == 0u && cd->tracking && !cd->record && J.sums != nullptr;
  const int sig = (int)((S >> lane) & 1u);
  const PhKey K = ph_key(J.key0, J.key1);
  bool tau;
  float contrib;
  if (INTEGER) {
    int a = 0;
    for (uint32_t c = 0; c < it.nchunks; ++c) a += (int)__ldcg(rows + c * 32u + (uint32_t)lane);
    // planes: lane c < 8 makes call c, then lane k gathers bit k of each plane
    const uint4 w = ph_call(K, x, g, t, typ + 2u * (uint32_t)(lane & 7));
    uint32_t uu = 0u;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const uint32_t c = (j & 3) == 0 ? w.x : (j & 3) == 1 ? w.y : (j & 3) == 2 ? w.z : w.w;
      uu |= ((__shfl_sync(0xffffffffu, c, j >> 2) >> lane) & 1u) << (31 - j);
    }
    const double h = field_h(1.0, 2 * a - d, J.q, sig ? 1 : -1, (double)lam);
    tau = (unsigned long long)uu < threshold_T(h, beta);
    contrib = (float)(2 * a - d) + 2.0f * lam;
  } else {
    float hs = 0.0f;
    for (uint32_t c = 0; c < it.nchunks; ++c)
      hs += __uint_as_float(__ldcg(rows + c * 32u + (uint32_t)lane));
    const uint4 w = ph_call(K, x, g, t, typ + 2u * (uint32_t)(lane >> 2));
    const uint32_t uu = (lane & 3) == 0 ? w.x : (lane & 3) == 1 ? w.y : (lane & 3) == 2 ? w.z : w.w;
    const float qf = (float)J.q;
    const float hk = __fadd_rn(__fadd_rn(hs, sig ? qf : -qf), lam);
    const float onep = 1.0f + ex2_approx((float)(-2.0 * beta * 1.4426950408889634) * hk);
    tau = __uint2float_rn(uu) * 2.3283064365386963e-10f * onep < 1.0f;
    contrib = hs + 2.0f * lam;
  }
  const uint32_t res = __ballot_sync(0xffffffffu, tau) | F;
  if (fuse) {  // -H(sigma_t) share of replica (g, lane): sigma (field sum + 2 lambda)
    const float c = sig ? contrib : -contrib;
    if (c != 0.0f)
      atomicAdd(J.sums + (size_t)(32u * g + (uint32_t)lane) * kNumSums + kSumE, (double)c);
  }
  if (lane == 0) dst[(size_t)x * G + g] = res;
}

// A lane left undecided by the head of its word, waiting in its warp's queue.
struct Pend {
  uint32_t x, g;
  uint32_t info;  // lane k (bits 0..4) | sigma (5) | top byte of u (6..13) | fp64 only (14)
  uint32_t pad;
};

constexpr int kQueue = 64;  // queue entries per warp

struct RoundArgs {
  const uint32_t* src;  // the half step's input configuration
  uint32_t t, typ;
  bool uni;
  double beta_u;
};

struct GraphShared {
  __align__(16) uint32_t tb[kTile][16];  // per vertex slot: top bytes of T by class (byte
                                         // a + 32 sigma), read as 16-byte vectors
  GraphJob J;       // the current job's descriptor
  RoundArgs ra;     // the current job's step: input, t, update type, beta
  uint32_t* dst;    // the half step's output configuration
  float kb_u;       // -2 beta_u log2(e)
  uint32_t skip, fuse;
  unsigned long long amb[kTile];  // per vertex slot: classes whose top byte is not certain
  Pend q[kTile / 32][kQueue];
  uint32_t wp[kTile][8];  // planes 0..7 of a word with lanes waiting to be queued
  float acc[kTile / 32][32][32];  // tracking sums [warp][replica lane k][thread lane]
};

// One round of queued lanes: lane i decides entry i (i < cnt) and sets its bit in the
// stored word if it is +1.  The words were stored by their owners before the round.
__device__ __forceinline__ void queue_round(const GraphJob& J, const Pend* q, int cnt,
                                            uint32_t* dst, const RoundArgs& A, int lane) {
  __syncwarp();
  if (lane < cnt) {
    const Pend e = q[lane];
    const int k = (int)(e.info & 31u);
    const int sig = (int)((e.info >> 5) & 1u);
    const uint32_t u8 = (e.info >> 6) & 0xFFu;
    const int32_t* ptr = A.typ == 0u ? J.in_ptr : J.out_ptr;
    const uint32_t* col = A.typ == 0u ? J.in_col : J.out_col;
    const int p0 = __ldg(ptr + e.x), d = __ldg(ptr + e.x + 1) - p0;
    int a = 0;  // neighbours with J_xy s_y = +1 on lane k
    for (int i = p0; i < p0 + d; ++i) {
      const uint32_t cv = __ldg(col + i);
      a += (int)(((__ldg(A.src + (size_t)(cv & 0x7fffffffu) * J.G + e.g) ^ (0u - (cv >> 31))) >>
                  k) & 1u);
    }
    const float lam = J.lambda != nullptr ? __ldg(J.lambda + e.x) : J.lambda_c;
    const float qf = (float)J.q;
    const float lmd = __fadd_rn(lam, -(float)d);
    const float bp = __fadd_rn(lmd, qf), bm = __fadd_rn(lmd, -qf);
    const float B = (float)d + fabsf(qf) + fabsf(lam) + 1.0f;
    const double beta = A.uni ? A.beta_u : J.beta_lane[32u * e.g + (uint32_t)k];
    const float kb = (float)(-2.0 * beta * 1.4426950408889634);
    if (decide_lane(J.key0, J.key1, e.x, e.g, A.t, A.typ, k, u8, a, d, sig, bp, bm, J.q, lam,
                    kb, fabsf(kb) * B, beta, ((e.info >> 14) & 1u) != 0u))
      atomicOr(dst + (size_t)e.x * J.G + e.g, 1u << k);
  }
  __syncwarp();
}

// One thread owns one (vertex, group) word.  Each block walks a contiguous range of
// tiles (one job per tile, kTile / Gp vertices of the half step's degree order x Gp
// threads).  Lanes the head leaves undecided wait in a per-warp queue and are decided
// 32 at a time.  With tracking on, half 0 also accumulates per replica
// sum_x sigma_x (s_x + 2 lambda_x), i.e. -H(sigma_t) (Eq. (ham1)), reduced when the
// block leaves a job.
template <bool INTEGER>
__global__ void __launch_bounds__(kTile, 3) graph_half_kernel(const GraphJob* __restrict__ jobs,
                                                           const Tile* __restrict__ tiles,
                                                           int n_tiles, uint32_t half,
                                                           int exact_always) {
  __shared__ GraphShared sh;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tb = (int)(((long long)blockIdx.x * n_tiles) / gridDim.x);
  const int te = (int)(((long long)(blockIdx.x + 1) * n_tiles) / gridDim.x);
  const GraphJob& J = sh.J;
  int cur_job = -1;
  int qn = 0;  // entries in this warp's queue (the same in every lane)
  Pend* q = sh.q[warp];
  float(*acc)[32] = sh.acc[warp];  // acc[k][lane]: this thread's sum for replica lane k
#pragma unroll
  for (int k = 0; k < 32; ++k) acc[k][lane] = 0.0f;

  auto flush = [&]() {
    // per replica (group offset go', lane k): the sum over the threads of group go'
    __syncthreads();
    const uint32_t Gj = J.Gj, Gp = J.Gp;
    for (uint32_t o = (uint32_t)tid; o < 32u * Gj; o += kTile) {
      const uint32_t gg = o >> 5, k = o & 31u;
      float v = 0.0f;
      for (uint32_t s = gg; s < (uint32_t)kTile; s += Gp) v += sh.acc[s >> 5][k][s & 31u];
      if (v != 0.0f)
        atomicAdd(J.sums + (size_t)(32u * (J.g0 + gg) + k) * kNumSums + kSumE, (double)v);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 32; ++k) acc[k][lane] = 0.0f;
  };

  for (int ti = tb; ti < te; ++ti) {
    const Tile tl = tiles[ti];
    if ((int)tl.job != cur_job) {
      if (cur_job >= 0) {
        if (qn > 0) queue_round(J, q, qn, sh.dst, sh.ra, lane);  // the old job's entries
        qn = 0;
        if (sh.fuse) flush();
      }
      __syncthreads();  // shared per-job values are about to change
      if (tid < (int)(sizeof(GraphJob) / 4))
        reinterpret_cast<uint32_t*>(&sh.J)[tid] =
            reinterpret_cast<const uint32_t*>(jobs + tl.job)[tid];
      __syncthreads();
      const CtxDev* cd = J.cd;
      const uint32_t t = cd->step;
      // one beta on every replica of the job at this step?
      const bool anneal = J.beta_sched != nullptr && cd->anneal_len != 0u;
      double b0;
      if (anneal) {
        uint32_t k = t - cd->anneal_t0;
        if (k >= cd->anneal_len) k = cd->anneal_len - 1u;
        b0 = J.beta_sched[k];
      } else {
        b0 = J.beta_lane[32u * J.g0];
      }
      bool same = true;
      if (!anneal)
        for (uint32_t r = (uint32_t)tid; r < 32u * J.Gj; r += kTile)
          same = same && J.beta_lane[32u * J.g0 + r] == b0;
      const int uni = __syncthreads_and(same ? 1 : 0);
      if (tid == 0) {
        const bool skip = t >= cd->t_end;
        sh.skip = skip ? 1u : 0u;
        sh.fuse = (!skip && half == 0u && cd->tracking && !cd->record && J.sums != nullptr) ? 1u
                                                                                           : 0u;
        sh.ra.src = half == 0u ? J.A : J.B;
        sh.dst = half == 0u ? J.B : J.A;
        sh.ra.t = t;
        sh.ra.typ = half ^ cd->order;
        sh.ra.uni = uni != 0;
        sh.ra.beta_u = b0;
        sh.kb_u = (float)(-2.0 * b0 * 1.4426950408889634);
      }
      __syncthreads();
      cur_job = (int)tl.job;
    }
    if (sh.skip) continue;
    const uint32_t Gj = J.Gj, Gp = J.Gp;
    const uint32_t go = (uint32_t)tid & (Gp - 1u), g = J.g0 + go;
    const uint32_t t = sh.ra.t, typ = sh.ra.typ;
    const bool uni = sh.ra.uni, fuse = sh.fuse != 0u;
    const uint32_t vx = (uint32_t)tid / Gp;
    const uint32_t slot = tl.w0 + vx;
    const bool valid = go < Gj && slot < J.n;
    // `half` is the position in the step (buffers); typ the update type (neighbours, draws)
    const uint32_t* src = sh.ra.src;
    uint32_t* dst = sh.dst;
    const int32_t* ptr = typ == 0u ? J.in_ptr : J.out_ptr;
    const uint32_t* col = typ == 0u ? J.in_col : J.out_col;
    uint32_t x = 0;
    int32_t p0 = 0;
    int d = 0;
    float lam = 0.0f;
    if (valid) {  // one 16-byte read: the vertex, its edge range and lambda_x
      const uint4 vi = __ldg((typ == 0u ? J.in_visit : J.out_visit) + slot);
      x = vi.x;
      p0 = (int32_t)vi.y;
      d = (int)vi.z;
      lam = __uint_as_float(vi.w);
    }
    const float qf = (float)J.q;
    const float lmd = __fadd_rn(lam, -(float)d);
    const float bp = __fadd_rn(lmd, qf), bm = __fadd_rn(lmd, -qf);  // h = 2a + (lambda - d +- q)
    const float B = (float)d + fabsf(qf) + fabsf(lam) + 1.0f;
    // class tables when they cost no more than per-lane thresholds: at most 32 classes
    // per thread of the vertex (2 (d + 1) <= 32 Gj).  With q = 1 the classes collapse
    // exactly: h(a, +1) = (2a - d + 1) + lambda = h(a + 1, -1), so one table over
    // a' = a + sigma in 0 .. d + 1 serves both (d <= 30)
    const bool collapse = J.q == 1.0;
    const bool table = INTEGER && uni && valid &&
                       (collapse ? d <= kTableDeg - 1 : (d <= kTableDeg && (uint32_t)(d + 1) <= 16u * Gj));
    const float kbu = sh.kb_u;  // in registers: the loops below store to shared memory
    const uint32_t G = J.G;
    const double* beta_g = J.beta_lane + 32u * g;
    unsigned long long vamb = 0ull;  // classes of this vertex whose top byte is not certain
    if (INTEGER && uni) {
      // class tables: the Gj threads of a vertex share its 2 (d + 1) classes (one warp
      // when Gp <= 32, else the block); byte a + 32 sigma
      unsigned long long mine = 0ull;
      if (table) {
        const float kb = kbu, kbB = fabsf(kb) * B;
        uint8_t* tbytes = reinterpret_cast<uint8_t*>(sh.tb[vx]);
        const uint32_t ncls = collapse ? (uint32_t)(d + 2) : 2u * (uint32_t)(d + 1);
        for (uint32_t i = go; i < ncls; i += Gj) {
          // collapsed: class a' = i with the sigma = -1 form; else (a, sigma) = (i/2, i%2)
          const uint32_t a = collapse ? i : i >> 1, s2 = collapse ? 0u : (i & 1u);
          const float hf = fmaf(2.0f, (float)a, s2 ? bp : bm);
          float lo, hi;
          t_bounds(hf, kb, kbB, lo, hi);
          uint32_t bl = top_byte(lo), bh = top_byte(hi);
          if (hf == 0.0f && field_is_zero(2 * (int)a - d, (int)s2, J.q, lam)) bl = bh = 0x80u;
          tbytes[a + 32u * s2] = (uint8_t)bh;
          mine |= (unsigned long long)(bl != bh) << (a + 32u * s2);
        }
      }
      if (Gp <= 32u) {
        for (uint32_t s2 = 1u; s2 < Gp; s2 <<= 1) mine |= __shfl_xor_sync(0xffffffffu, mine, s2);
        vamb = mine;
        __syncwarp();
      } else {
        if (go == 0u) sh.amb[vx] = 0ull;
        __syncthreads();
        if (mine != 0ull) atomicOr(&sh.amb[vx], mine);
        __syncthreads();
        vamb = sh.amb[vx];
      }
    }
    uint32_t res = 0u;
    const bool hub = valid && (uint32_t)d > kHubDeg;  // left to graph_hub_kernel
    // table entries the warp's lanes need: a < 8, < 16 or < 32 (warp-wide choice)
    // (collapsed: a' = a + sigma <= d + 1)
    const int dn = collapse ? d + 1 : d;
    const uint32_t nw = __reduce_max_sync(0xffffffffu, table ? (dn <= 7 ? 1u : dn <= 15 ? 2u : 4u) : 0u);
    uint32_t und = 0u;  // lanes left to the queue
    uint32_t S = 0u;
    if (valid && !hub) {
      S = __ldg(src + (size_t)x * G + g);
      const uint32_t F = J.frozen != nullptr ? __ldg(J.frozen + x) : 0u;
      if (INTEGER) {
        // byte counters: byte i of C[m] = number of neighbours with J_xy s_y = +1 on
        // lane m + 8 i (at most d <= 255, so bytes never carry into each other)
        uint32_t C[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) C[m] = 0u;
        for (int e = p0; e < p0 + d; ++e) {
          const uint32_t cv = __ldg(col + e);
          const uint32_t w = __ldg(src + (size_t)(cv & 0x7fffffffu) * G + g) ^ (0u - (cv >> 31));
#pragma unroll
          for (int m = 0; m < 8; ++m) C[m] += (w >> m) & 0x01010101u;
        }
        if (fuse) {  // sigma (s + 2 lambda) with s = 2a - d
          const float a0 = __fadd_rn(2.0f * lam, -(float)d);
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            const float cf = __fsub_rn(
                __int_as_float((int)__byte_perm(C[k & 7], 0x4B000000u, 0x7540u + (k >> 3))),
                8388608.0f);
            const float v = __fmaf_rn(2.0f, cf, a0);
            acc[k][lane] += ((S >> k) & 1u) ? v : -v;
          }
        }
        // threshold bytes R[m] (byte i: lane m + 8 i) and lanes of uncertain top byte
        uint32_t R[8], amb = 0u;
        if (table) {
          if (vamb != 0ull) {  // rare: lanes of the uncertain classes
#pragma unroll 1
            for (int k = 0; k < 32; ++k) {
              const uint32_t a = (C[k & 7] >> (8 * (k >> 3))) & 0xFFu, sk = (S >> k) & 1u;
              const uint32_t c = collapse ? a + sk : a + 32u * sk;
              amb |= (uint32_t)((vamb >> c) & 1ull) << k;
            }
          }
          uint32_t Tm[8], Tp[8];
          const uint4* tv = reinterpret_cast<const uint4*>(sh.tb[vx]);
          const uint4 m0 = tv[0], p0v = tv[2];
          Tm[0] = m0.x; Tm[1] = m0.y; Tm[2] = m0.z; Tm[3] = m0.w;
          Tp[0] = p0v.x; Tp[1] = p0v.y; Tp[2] = p0v.z; Tp[3] = p0v.w;
          if (nw == 4u) {
            const uint4 m1 = tv[1], p1v = tv[3];
            Tm[4] = m1.x; Tm[5] = m1.y; Tm[6] = m1.z; Tm[7] = m1.w;
            Tp[4] = p1v.x; Tp[5] = p1v.y; Tp[6] = p1v.z; Tp[7] = p1v.w;
          } else {
#pragma unroll
            for (int i = 4; i < 8; ++i) Tm[i] = Tp[i] = 0u;
          }
          if (collapse) {  // one table over a' = a + sigma (bytes: no carries, a' <= 31)
            if (nw == 1u) {
#pragma unroll
              for (int m = 0; m < 8; ++m) R[m] = lookup_bytes_c<1>(Tm, C[m] + ((S >> m) & 0x01010101u));
            } else if (nw == 2u) {
#pragma unroll
              for (int m = 0; m < 8; ++m) R[m] = lookup_bytes_c<2>(Tm, C[m] + ((S >> m) & 0x01010101u));
            } else {
#pragma unroll
              for (int m = 0; m < 8; ++m) R[m] = lookup_bytes_c<4>(Tm, C[m] + ((S >> m) & 0x01010101u));
            }
          } else if (nw == 1u) {
#pragma unroll
            for (int m = 0; m < 8; ++m) R[m] = lookup_bytes<1>(Tm, Tp, C[m], (S >> m) & 0x01010101u);
          } else if (nw == 2u) {
#pragma unroll
            for (int m = 0; m < 8; ++m) R[m] = lookup_bytes<2>(Tm, Tp, C[m], (S >> m) & 0x01010101u);
          } else {
#pragma unroll
            for (int m = 0; m < 8; ++m) R[m] = lookup_bytes<4>(Tm, Tp, C[m], (S >> m) & 0x01010101u);
          }
        } else {
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            const uint2 rb = lane_bytes(C[m], S, m, bp, bm, B, beta_g, kbu, uni, d, J.q, lam);
            R[m] = rb.x;
            amb |= rb.y;
          }
        }
        uint32_t P[8];
        bytes_to_planes(R, P);
        const PhKey K = ph_key(J.key0, J.key1);
        const PhShared ph = ph_shared(K, g, t);
        const uint4 w0 = ph_call_shared(K, ph, x, typ);
        const uint4 w1 = ph_call_shared(K, ph, x, typ + 2u);
        const uint32_t W[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
        und = exact_always ? 0u : ~(F | amb);
        uint32_t r = 0u;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          r |= und & ~W[j] & P[j];   // draw bit 0, threshold bit 1: u < T
          und &= ~(W[j] ^ P[j]);     // equal bits: not decided yet
        }
        // debugging aid (exact_always): every lane through the fp64 threshold
        und = exact_always ? ~F : (und | (amb & ~F));
        res = r | F;
        if (und != 0u) {
#pragma unroll
          for (int j = 0; j < 8; ++j) sh.wp[tid][j] = W[j];
        }
      } else {
        const PhKey K = ph_key(J.key0, J.key1);
        const PhShared ph = ph_shared(K, g, t);
        const float* Jr = typ == 0u ? J.in_J : J.out_J;
        float h[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) h[k] = 0.0f;
        for (int e = p0; e < p0 + d; ++e) {
          const uint32_t y = __ldg(col + e) & 0x7fffffffu;
          const float Jv = __ldg(Jr + e);
          const uint32_t wy = __ldg(src + (size_t)y * G + g);
#pragma unroll
          for (int k = 0; k < 32; ++k) h[k] += ((wy >> k) & 1u) ? Jv : -Jv;
        }
        if (uni)
          res = real_lanes<true>(h, S, qf, lam, kbu, beta_g, K, ph, x, typ, fuse, acc, lane);
        else
          res = real_lanes<false>(h, S, qf, lam, kbu, beta_g, K, ph, x, typ, fuse, acc, lane);
        res |= F;
      }
    }
    if (valid && !hub) dst[(size_t)x * G + g] = res;
    if (INTEGER) {
      // undecided lanes into the warp's queue (every lane of the warp takes part); a full
      // queue is decided 32 at a time, after the words are stored
      while (__any_sync(0xffffffffu, und != 0u)) {
        const bool has = und != 0u;
        const int k = has ? __ffs(und) - 1 : 0;
        const unsigned ball = __ballot_sync(0xffffffffu, has);
        if (has) {
          und &= und - 1u;
          const uint32_t* w = sh.wp[tid];
          const uint32_t u8 = lane_byte(w[0], w[1], w[2], w[3], w[4], w[5], w[6], w[7], k);
          q[qn + __popc(ball & ((1u << lane) - 1u))] =
              Pend{x, g, (uint32_t)k | (((S >> k) & 1u) << 5) | (u8 << 6) |
                             (exact_always ? (1u << 14) : 0u), 0u};
        }
        qn += __popc(ball);
        if (qn >= 32) {
          queue_round(J, q, 32, dst, sh.ra, lane);
          qn -= 32;
          if (lane < qn) q[lane] = q[32 + lane];
          __syncwarp();
        }
      }
    }
  }
  if (cur_job >= 0) {
    if (qn > 0) queue_round(J, q, qn, sh.dst, sh.ra, lane);
    if (sh.fuse) flush();
  }
}

// ------------------------------------------------------------------ per-group kernels
// Jobs of one group each (Gj = 1); tiles of kTile vertices.

// Fields h_x (float) of the next half step, summed in edge order (a diagnostic).
__global__ void __launch_bounds__(kTile) graph_fields_kernel(const GraphJob* __restrict__ jobs,
                                                             const Tile* __restrict__ tiles,
                                                             int n_tiles, uint32_t half,
                                                             float* __restrict__ out) {
  for (int ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
    const Tile tl = tiles[ti];
    const GraphJob& J = jobs[tl.job];
    const uint32_t x = tl.w0 + threadIdx.x;
    if (x >= J.n) continue;
    const uint32_t G = J.G, g = J.g0;
    const uint32_t* src = half == 0u ? J.A : J.B;
    const int32_t* ptr = half == 0u ? J.in_ptr : J.out_ptr;
    const uint32_t* col = half == 0u ? J.in_col : J.out_col;
    const float* Jr = half == 0u ? J.in_J : J.out_J;
    const uint32_t S = src[(size_t)x * G + g];
    const float lam = J.lambda != nullptr ? J.lambda[x] : J.lambda_c;
    const float qf = (float)J.q;
    for (int k = 0; k < 32; ++k) {
      float hk;
      if (J.integer) {
        int s = 0;
        for (int e = ptr[x]; e < ptr[x + 1]; ++e) {
          const uint32_t cv = col[e];
          s += (((src[(size_t)(cv & 0x7fffffffu) * G + g] ^ (0u - (cv >> 31))) >> k) & 1u) ? 1
                                                                                           : -1;
        }
        hk = __fadd_rn(__fadd_rn((float)s, ((S >> k) & 1u) ? qf : -qf), lam);
      } else {
        float a = 0.0f;
        for (int e = ptr[x]; e < ptr[x + 1]; ++e) {
          const float Jv = Jr[e];
          a += ((src[(size_t)(col[e] & 0x7fffffffu) * G + g] >> k) & 1u) ? Jv : -Jv;
        }
        hk = __fadd_rn(__fadd_rn(a, ((S >> k) & 1u) ? qf : -qf), lam);
      }
      out[(size_t)(32u * g + (uint32_t)k) * J.n + x] = hk;
    }
  }
}

// Initial spins: lane k = +1 iff u_k < 2^31 with the direct draw u_k = W_k of step
// 0xFFFFFFFF, half 0.
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
        if ((k & 3) == 0) w = ph_call(K, x, J.g0, kInitStep, 2u * (uint32_t)(k >> 2));
        const uint32_t u = (k & 3) == 0 ? w.x : (k & 3) == 1 ? w.y : (k & 3) == 2 ? w.z : w.w;
        s |= (uint32_t)(u < 0x80000000u) << k;
      }
    }
    if (J.frozen != nullptr) s |= J.frozen[x];
    J.A[(size_t)x * J.G + J.g0] = s;
    J.B[(size_t)x * J.G + J.g0] = s;
  }
}

// Adds one bit per lane (x) to the bit-sliced counter p (planes 0 .. B - 1).
__device__ __forceinline__ void bs_add(uint32_t (&p)[8], uint32_t x, int B) {
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    if (b < B) {
      const uint32_t c = p[b] & x;
      p[b] ^= x;
      x = c;
    }
  }
}

// Sums over the CSR edges (x -> y) of the warp's 32 vertices (thread t: vertex x of
// lane t), for lane k's replica: esum = sum of J_xy s_x s_y with s_y from Y, and (if
// want_cut) cut = the number of those edges with s_x != s_y.  Integer couplings: per
// thread, bit-sliced counters of the agreeing products (chunks of 255 edges), whose
// planes are transposed across the warp; real couplings: per-replica float sums,
// transposed once.  A thread's edges are read four at a time, the loads of the four
// independent of one another.
template <bool INTEGER>
__device__ __forceinline__ void obs_edges(const int32_t* ptr, const uint32_t* col,
                                          const float* Jr, const uint32_t* Y, uint32_t x,
                                          bool act, uint32_t S, uint32_t G, uint32_t g,
                                          bool want_cut, int lane, double& esum, double& cut) {
  const int e0 = act ? ptr[x] : 0;
  const int d = act ? ptr[x + 1] - e0 : 0;
  const int dmax = __reduce_max_sync(0xffffffffu, d);
  const int dsum = __reduce_add_sync(0xffffffffu, d);
  long long cj = 0, ca = 0;
  float fv[INTEGER ? 1 : 32];
#pragma unroll
  for (int k = 0; k < (INTEGER ? 1 : 32); ++k) fv[k] = 0.0f;
  for (int base = 0; base < dmax; base += 252) {
    const int B = 32 - __clz(min(dmax - base, 255));  // planes for counts up to the chunk
    uint32_t pj[8], pa[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) pj[b] = pa[b] = 0u;
    const int hi = min(d, base + 252);
    for (int e = base; e < hi; e += 4) {
      uint32_t cv[4], w[4];
      float Jv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) cv[i] = e + i < hi ? __ldg(col + e0 + e + i) : 0u;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        w[i] = e + i < hi ? __ldg(Y + (size_t)(cv[i] & 0x7fffffffu) * G + g) : 0u;
        if (!INTEGER) Jv[i] = e + i < hi ? __ldg(Jr + e0 + e + i) : 0.0f;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (e + i < hi) {
          const uint32_t agree = ~(S ^ w[i]);
          if constexpr (INTEGER) {
            bs_add(pj, agree ^ (0u - (cv[i] >> 31)), B);
          } else {
#pragma unroll
            for (int k = 0; k < 32; ++k) fv[k] += ((agree >> k) & 1u) ? Jv[i] : -Jv[i];
          }
          if (want_cut) bs_add(pa, agree, B);
        }
      }
    }
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      if (b < B) {
        if (INTEGER) cj += (long long)warp_column_count(pj[b], lane) << b;
        if (want_cut) ca += (long long)warp_column_count(pa[b], lane) << b;
      }
    }
  }
  if constexpr (INTEGER)
    esum = (double)(2 * cj - dsum);
  else
    esum = (double)warp_transpose_sum(fv, lane);
  cut = want_cut ? (double)(dsum - ca) : 0.0;
}

// Observables of one group (per-group jobs, Gj = 1): thread t of a tile takes vertex
// w0 + t; the sums over the warp's 32 vertices reach lane k (replica 32 g + k) by bit
// transposes of the sigma words and of bit-sliced edge counters (integer sums) or by
// transposing butterflies (float sums), and the block adds its warps once per tile.
template <bool INTEGER>
__global__ void __launch_bounds__(kTile) graph_obs_kernel(const GraphJob* __restrict__ jobs,
                                                          const Tile* __restrict__ tiles,
                                                          int n_tiles, int which, int full) {
  __shared__ double red[kTile / 32][32][kNumSums];
  pdl_enter();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
    const Tile tl = tiles[ti];
    const GraphJob& J = jobs[tl.job];
    const uint32_t G = J.G, g = J.g0;
    const uint32_t x = tl.w0 + (uint32_t)threadIdx.x;
    const bool act = x < J.n;
    const uint32_t am = act ? 0xffffffffu : 0u;
    const uint32_t S = act ? J.A[(size_t)x * G + g] : 0u;
    const uint32_t S2 = (act && full) ? J.B[(size_t)x * G + g] : 0u;
    const float lam = act ? (J.lambda != nullptr ? J.lambda[x] : J.lambda_c) : 0.0f;
    const int nact = __popc(__ballot_sync(0xffffffffu, act));
    double acc[kNumSums];
#pragma unroll
    for (int q = 0; q < kNumSums; ++q) acc[q] = 0.0;
    acc[kSumM] = (double)(2 * warp_column_count(S & am, lane) - nact);
    {
      float v[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = ((S >> k) & 1u) ? lam : -lam;
      acc[kSumLS] = (double)warp_transpose_sum(v, lane);
    }
    obs_edges<INTEGER>(J.in_ptr, J.in_col, J.in_J, J.A, x, act, S, G, g, true, lane,
                       acc[kSumE], acc[kSumCut]);
    if (full) {
      acc[kSumP2] = (double)(2 * warp_column_count(~(S ^ S2) & am, lane) - nact);
      float v[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = ((S2 >> k) & 1u) ? lam : -lam;
      acc[kSumLS2] = (double)warp_transpose_sum(v, lane);
      double unused;
      obs_edges<INTEGER>(J.out_ptr, J.out_col, J.out_J, J.B, x, act, S, G, g, false, lane,
                         acc[kSumP1], unused);
    }
#pragma unroll
    for (int q = 0; q < kNumSums; ++q) red[warp][lane][q] = acc[q];
    __syncthreads();
    if (threadIdx.x < 32) {
      double* dst = (which ? J.obs : J.sums) + (size_t)(32u * g + threadIdx.x) * kNumSums;
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

cudaError_t launch_graph_hub(bool integer, const GraphJob* jobs, const HubItem* items,
                             const uint32_t* unit_item, int n_units, uint32_t half,
                             uint32_t* partial, uint32_t* done, cudaStream_t st) {
  if (n_units <= 0) return cudaSuccess;
  constexpr int per = kTile / 32;
  const int grid = (n_units + per - 1) / per;
  if (integer)
    graph_hub_kernel<true><<<grid, kTile, 0, st>>>(jobs, items, unit_item, n_units, half, partial,
                                                   done);
  else
    graph_hub_kernel<false><<<grid, kTile, 0, st>>>(jobs, items, unit_item, n_units, half,
                                                    partial, done);
  return cudaGetLastError();
}

cudaError_t launch_graph_init(const GraphJob* jobs, const Tile* tiles, int n_tiles, int kind,
                              cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  graph_init_kernel<<<grid_for(n_tiles, 8), kTile, 0, st>>>(jobs, tiles, n_tiles, kind);
  return cudaGetLastError();
}

cudaError_t launch_graph_obs(bool integer, const GraphJob* jobs, const Tile* tiles, int n_tiles,
                             int which, int full, cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  const dim3 grid(grid_for(n_tiles, 4));
  if (integer)
    return launch_dependent(graph_obs_kernel<true>, grid, dim3(kTile), 0, st, jobs, tiles,
                            n_tiles, which, full);
  return launch_dependent(graph_obs_kernel<false>, grid, dim3(kTile), 0, st, jobs, tiles,
                          n_tiles, which, full);
}

cudaError_t launch_graph_fields(const GraphJob* jobs, const Tile* tiles, int n_tiles, uint32_t half,
                                float* out, cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  graph_fields_kernel<<<grid_for(n_tiles, 8), kTile, 0, st>>>(jobs, tiles, n_tiles, half, out);
  return cudaGetLastError();
}

}  // namespace shk
