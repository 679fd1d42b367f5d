// lattice.cu -- half-step kernels of the shaken dynamics on the L x L torus
// (Sec. 3 of arXiv:1904.06257) for three spin encodings, the threshold-table
// builder and the lattice observables.
//
// Half step 0 is P^dl: tau_x from h^dl_x = J (s_down + s_left) + q s_x + lambda
// (Eq. (hdl)); half step 1 is P^ur with h^ur_x = J (s_up + s_right) + q s_x +
// lambda (Eq. (hur)).  Every site of a half step is resampled at once from the
// other buffer (the parallel product form below Eq. (pasymm)).
//
// Work unit: a lane word = 32 decisions sharing Philox counter words (a, b):
//   INT8 / PACKED: 32 consecutive sites (i, 32c .. 32c+31) of one replica,
//                  a = i*L/32 + c, b = replica;
//   MULTISPIN:     one site x of 32 replicas (bit k = replica 32g+k), a = x, b = g.
// Decision: u_k < T(c_k, beta_k) where u_k's bit (31-j) is bit k of the plane
// word W_j = Philox(key, (a, b, t, half + 2(j>>2)))[j & 3].  The comparison is
// done for all 32 lanes at once, most significant plane first, and stops when
// every lane differs from its threshold in some plane already seen (later
// planes cannot change the result; the draws are counter-based, so planes never
// generated are simply never needed).  Per plane the lane's threshold bit is
// OR_c (class_mask_c & tm[j][c]).
#include <cstdint>

#include "shaken_internal.cuh"

namespace shk {

// --------------------------------------------------------------------------- tables
// One block per table, one warp per field class c (6 classes): lane k computes
// T(h_c, beta_k) in fp64 and the warp ballots its bit planes.
__global__ void __launch_bounds__(256) build_lattice_tables_kernel(
    const double* __restrict__ beta_lanes, int ntab, double J, double q, double lam,
    LatTable* __restrict__ out) {
  __shared__ unsigned long long Ts[8][32];
  __shared__ uint32_t sat_any[8];
  const int tab = blockIdx.x;
  if (tab >= ntab) return;
  const int lane = threadIdx.x & 31;
  const int c = threadIdx.x >> 5;  // 0..7
  LatTable* T = out + tab;
  if (c >= 6) {
    T->tm[lane][c] = 0u;
    if (lane == 0) {
      T->satp[c] = 0u;
      T->satm[c] = 0u;
      sat_any[c] = 0u;
    }
  } else {
    const int n = c >> 1, s = c & 1;
    const double beta = beta_lanes[(size_t)tab * 32 + lane];
    const double h = field_h(J, 2 * n - 2, q, 2 * s - 1, lam);
    const unsigned long long Tv = threshold_T(h, beta);
    Ts[c][lane] = Tv;
    const bool satp = Tv == 4294967296ULL;
    const bool satm = Tv == 0ULL;
    const unsigned sp = __ballot_sync(0xffffffffu, satp);
    const unsigned sm = __ballot_sync(0xffffffffu, satm);
    if (lane == 0) {
      T->satp[c] = sp;
      T->satm[c] = sm;
      sat_any[c] = sp | sm;
    }
    const uint32_t t32 = (satp || satm) ? 0u : (uint32_t)Tv;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const unsigned m = __ballot_sync(0xffffffffu, (t32 >> (31 - j)) & 1u);
      if (lane == 0) T->tm[j][c] = m;
    }
  }
  __syncthreads();
  if (c == 0) {
    // thresholds depending on n + s only: (0,1) == (1,0) and (1,1) == (2,0) on every lane
    const bool same = Ts[1][lane] == Ts[2][lane] && Ts[3][lane] == Ts[4][lane];
    const bool coll = __all_sync(0xffffffffu, same);
    if (lane == 0) {
      T->collapsed = coll ? 1u : 0u;
      uint32_t a = 0u;
      for (int k = 0; k < 6; ++k) a |= sat_any[k];
      T->anysat = a != 0u ? 1u : 0u;
      T->pad = 0u;
    }
  }
  __syncthreads();
  // planes by c = n + s: class 2n + s with (n, s) = (0,0), (0,1), (1,1), (2,1)
  if (threadIdx.x < 128) {
    const int j = threadIdx.x >> 2, cc = threadIdx.x & 3;
    const int cls = cc == 0 ? 0 : cc == 1 ? 1 : cc == 2 ? 3 : 5;
    T->tmc[j][cc] = T->tm[j][cls];
  }
  __syncthreads();
  // mirror test on the eight planes the head compares (lane j checks plane j)
  if (threadIdx.x < 32) {
    bool ok = true;
    if (lane < 8)
      ok = (T->tmc[lane][0] ^ T->tmc[lane][3]) == 0xffffffffu &&
           (T->tmc[lane][1] ^ T->tmc[lane][2]) == 0xffffffffu;
    ok = __all_sync(0xffffffffu, ok);
    if (lane == 0) T->mirror = (ok && T->collapsed != 0u && T->anysat == 0u) ? 1u : 0u;
  }
}

// --------------------------------------------------------------------------- decision core
// Field classes of a lane word.  S = sigma_x bits, V / H = the two in-neighbour
// bits (vertical / horizontal); x = V ^ H marks one +1 neighbour (n = 1), and
// where V == H the class is n = 0 (V = 0) or n = 2 (V = 1).
struct LaneWord {
  uint32_t S, V, X, U, res;  // U = lanes still undecided
};

// One plane of a threshold table, read from shared memory once and applied to
// every lane word of the thread.
struct PlaneRow {
  uint4 lo;  // classes 0..3 (collapsed: c = 0..3)
  uint2 hi;  // classes 4, 5 (unused when collapsed)
};

template <bool COLL>
__device__ __forceinline__ PlaneRow plane_row(const LatTable& tab, int j) {
  PlaneRow r;
  if (COLL) {
    r.lo = *reinterpret_cast<const uint4*>(&tab.tmc[j][0]);
    r.hi = make_uint2(0u, 0u);
  } else {
    r.lo = *reinterpret_cast<const uint4*>(&tab.tm[j][0]);
    r.hi = *reinterpret_cast<const uint2*>(&tab.tm[j][4]);
  }
  return r;
}

// Threshold bit of plane j for every lane: first select by sigma within each
// n-class, then by n: 5 three-input selects.
// Collapsed tables (thresholds by c = n + s): with c0 = parity and c1 =
// majority of (V, H, S), c = c0 + 2 c1 and the plane bit is 3 selects; there
// L.V holds c1 and L.X holds c0.
template <bool COLL>
__device__ __forceinline__ uint32_t plane_bits(const LaneWord& L, const PlaneRow& r) {
  if (COLL) {
    const uint32_t lo = (L.X & r.lo.y) | (~L.X & r.lo.x);  // c1 = 0
    const uint32_t hi = (L.X & r.lo.w) | (~L.X & r.lo.z);  // c1 = 1
    return (L.V & hi) | (~L.V & lo);
  }
  const uint32_t b0 = (L.S & r.lo.y) | (~L.S & r.lo.x);  // n = 0
  const uint32_t b1 = (L.S & r.lo.w) | (~L.S & r.lo.z);  // n = 1
  const uint32_t b2 = (L.S & r.hi.y) | (~L.S & r.hi.x);  // n = 2
  const uint32_t m = (L.V & b2) | (~L.V & b0);           // V == H
  return (L.X & b1) | (~L.X & m);
}

// MSB-first comparison of u_k with T_k over the four planes of one Philox call.
template <bool COLL>
__device__ __forceinline__ void apply_call(LaneWord& L, const uint4 w, const LatTable& tab,
                                           uint32_t call) {
  const uint32_t Wj[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t P = plane_bits<COLL>(L, plane_row<COLL>(tab, 4 * call + i));
    const uint32_t diff = (Wj[i] ^ P) & L.U;  // first plane where u and T differ
    L.res |= diff & P;                        // T has the 1 there: u < T
    L.U &= ~diff;
  }
}

// Initial classification: frozen lanes and saturated thresholds (T = 0 or 2^32)
// are decided before any draw.  For collapsed tables V and X are replaced by
// the majority and the parity of (V, H, S).
template <bool COLL>
__device__ __forceinline__ LaneWord classify(uint32_t S, uint32_t V, uint32_t H, uint32_t F,
                                             const LatTable& tab) {
  LaneWord L;
  L.S = S;
  L.V = V;
  L.X = V ^ H;
  uint32_t dec = F, res = F;
  if (tab.anysat) {
    const uint32_t n2 = V & H, n0 = ~(V | H), n1 = L.X;
    const uint32_t M[6] = {n0 & ~S, n0 & S, n1 & ~S, n1 & S, n2 & ~S, n2 & S};
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      dec |= M[c] & (tab.satp[c] | tab.satm[c]);
      res |= M[c] & tab.satp[c];
    }
  }
  if (COLL) {
    L.V = (V & H) | (S & (V | H));  // majority
    L.X = V ^ H ^ S;                // parity
  }
  L.U = ~dec;
  L.res = res;
  return L;
}

// Calls 0, 1 and 2 (planes 31..20) of a lane word, made unconditionally (the
// resident small-lattice kernel, where a half step is a dependent chain and the
// warp needs call 2 for some word about 98% of the time anyway): the three
// Philox calls are independent and overlap.  A lane is decided by its first
// differing plane, as call by call; after the twelve planes a lane is undecided
// with probability 2^-12.
template <bool COLL>
__device__ __forceinline__ void decide_head3(LaneWord& L, const LatTable& tab, const PhKey& K,
                                             const PhShared& P, uint32_t a, uint32_t half,
                                             uint32_t& calls) {
  const uint4 w0 = ph_call_shared(K, P, a, half);
  const uint4 w1 = ph_call_shared(K, P, a, half + 2u);
  const uint4 w2 = ph_call_shared(K, P, a, half + 4u);
  calls += 3;
  // the top twelve bits of u and T compared as a subtraction, least significant
  // plane first (borrow lt, equality eq): two short independent chains
  uint32_t lt = 0u, eq = 0xffffffffu;
#pragma unroll
  for (int j = 11; j >= 0; --j) {
    const uint4 Wc = j >= 8 ? w2 : j >= 4 ? w1 : w0;
    const int i = j & 3;
    const uint32_t w = i == 0 ? Wc.x : i == 1 ? Wc.y : i == 2 ? Wc.z : Wc.w;
    const uint32_t Pj = plane_bits<COLL>(L, plane_row<COLL>(tab, j));
    lt = (~w & Pj) | (~w & lt) | (Pj & lt);
    eq &= ~(w ^ Pj);
  }
  L.res |= L.U & ~eq & lt;
  L.U &= eq;
}

// Planes 31..24 (calls 0 and 1) of the thread's WPT lane words, plane-major:
// every table row is read once for all the words, and the WPT Philox calls of
// a group are independent of one another.  The top eight bits of u_k and T_k
// are compared as an eight-bit subtraction, least significant plane first:
// the borrow lt <- maj(~w, P, lt) ends as [u_top < T_top] and eq as
// [u_top == T_top].  Lanes with equal top bits stay undecided for planes 23..0
// (the warp queue of the tiled kernel, or decide_tail); the others are decided
// exactly as by the first differing plane.
// Four planes of one call (planes 4c+3 .. 4c, least significant first) for
// the WPT words: one step of the borrow chain per plane.
template <bool COLL, int WPT>
__device__ __forceinline__ void head_planes(const LaneWord (&Lw)[WPT], const LatTable& tab,
                                            int call, const uint4 (&W)[WPT], uint32_t (&lt)[WPT],
                                            uint32_t (&eq)[WPT]) {
#pragma unroll
  for (int i = 3; i >= 0; --i) {
    const PlaneRow r = plane_row<COLL>(tab, 4 * call + i);
#pragma unroll
    for (int k = 0; k < WPT; ++k) {
      const uint32_t w = i == 0 ? W[k].x : i == 1 ? W[k].y : i == 2 ? W[k].z : W[k].w;
      const uint32_t P = plane_bits<COLL>(Lw[k], r);
      lt[k] = (~w & P) | (~w & lt[k]) | (P & lt[k]);
      eq[k] &= ~(w ^ P);
    }
  }
}

// The same four planes for mirror tables: with c1 = majority (L.V) and c0 =
// parity (L.X), the class c = c0 + 2 c1 has field h > 0 exactly when c1 = 1, and
// |h| is the larger value when c0 == c1.  The plane is the T(|h|) plane picked by
// sel = ~(c0 ^ c1) from the rows of c = 2 and c = 3, complemented on the lanes
// with h < 0: two logic operations instead of three selects.
template <int WPT>
__device__ __forceinline__ void head_planes_mirror(const LaneWord (&Lw)[WPT],
                                                   const uint32_t (&sel)[WPT],
                                                   const LatTable& tab, int call,
                                                   const uint4 (&W)[WPT], uint32_t (&lt)[WPT],
                                                   uint32_t (&eq)[WPT]) {
#pragma unroll
  for (int i = 3; i >= 0; --i) {
    const uint2 r = *reinterpret_cast<const uint2*>(&tab.tmc[4 * call + i][2]);
#pragma unroll
    for (int k = 0; k < WPT; ++k) {
      const uint32_t w = i == 0 ? W[k].x : i == 1 ? W[k].y : i == 2 ? W[k].z : W[k].w;
      const uint32_t Q = (sel[k] & r.y) | (~sel[k] & r.x);
      const uint32_t P = ~(Q ^ Lw[k].V);
      lt[k] = (~w & P) | (~w & lt[k]) | (P & lt[k]);
      eq[k] &= ~(w ^ P);
    }
  }
}

template <int WPT>
__device__ __forceinline__ void head_finish(LaneWord (&Lw)[WPT], const uint32_t (&lt)[WPT],
                                            const uint32_t (&eq)[WPT]) {
#pragma unroll
  for (int k = 0; k < WPT; ++k) {
    Lw[k].res |= Lw[k].U & ~eq[k] & lt[k];
    Lw[k].U &= eq[k];
  }
}

// MIR: the table is a mirror table (collapsed, `mirror` set).
template <bool COLL, int WPT, bool MIR = false>
__device__ __forceinline__ void decide_head_words(LaneWord (&Lw)[WPT], const LatTable& tab,
                                                  const PhKey& K, const PhShared& P,
                                                  const uint32_t (&a)[WPT], uint32_t half) {
  uint32_t lt[WPT], eq[WPT], sel[WPT];
#pragma unroll
  for (int k = 0; k < WPT; ++k) {
    lt[k] = 0u;
    eq[k] = 0xffffffffu;
    sel[k] = MIR ? ~(Lw[k].X ^ Lw[k].V) : 0u;
  }
#pragma unroll
  for (int call = 1; call >= 0; --call) {
    uint4 W[WPT];
#pragma unroll
    for (int k = 0; k < WPT; ++k) W[k] = ph_call_shared(K, P, a[k], half + 2u * (uint32_t)call);
    if (MIR)
      head_planes_mirror<WPT>(Lw, sel, tab, call, W, lt, eq);
    else
      head_planes<COLL, WPT>(Lw, tab, call, W, lt, eq);
  }
  head_finish<WPT>(Lw, lt, eq);
}

// Calls first..7 while some lane is undecided (one word at a time: the resident
// small-lattice kernel).
template <bool COLL>
__device__ __forceinline__ void decide_tail(LaneWord& L, const LatTable& tab, const PhKey& K,
                                            const PhShared& P, uint32_t a, uint32_t half,
                                            uint32_t first, uint32_t& calls) {
#pragma unroll 1
  for (uint32_t call = first; call < 8 && L.U != 0u; ++call) {
    const uint4 w = ph_call_shared(K, P, a, half + 2u * call);
    ++calls;
    apply_call<COLL>(L, w, tab, call);
  }
}

// --------------------------------------------------------------------------- int8 <-> bits
// +1 = 0x01, -1 = 0xFF: the sign bit of a byte is clear for +1.
// Eight bytes (w0: sites 0..3, w1: sites 4..7, memory order) -> bits 24..31 of the
// result (bit 24 + j = site j is +1): the clear sign bits go to bits 0, 8, 16, 24
// (w0) and 4, 12, 20, 28 (w1), and one multiply by 2^24 + 2^17 + 2^10 + 2^3 moves
// byte k of w0 to bit 24 + k and byte k of w1 to bit 28 + k; every other partial
// product lands below bit 24 at a distinct position or above bit 31, so nothing
// carries into the top byte.
__device__ __forceinline__ uint32_t bits8_top(uint32_t w0, uint32_t w1) {
  const uint32_t m = ((~w0 >> 7) & 0x01010101u) | ((~w1 >> 3) & 0x10101010u);
  return m * 0x01020408u;
}
// 32 bytes (sites 0..15 in a, 16..31 in b) -> 32 bits, bit j = site j is +1.
__device__ __forceinline__ uint32_t bits32(uint4 a, uint4 b) {
  const uint32_t lo = __byte_perm(bits8_top(a.x, a.y), bits8_top(a.z, a.w), 0x0073u);
  const uint32_t hi = __byte_perm(bits8_top(b.x, b.y), bits8_top(b.z, b.w), 0x0073u);
  return __byte_perm(lo, hi, 0x5410u);
}
// 4 bits -> 4 bytes of +1/-1: bit k -> byte k (0 or 1), then 0xFF - 0xFE t per byte
// (no byte borrows from its neighbour)
__device__ __forceinline__ uint32_t bytes4(uint32_t b) {
  const uint32_t t = ((b & 0xFu) * 0x00204081u) & 0x01010101u;
  return 0xFFFFFFFFu - 0xFEu * t;
}
__device__ __forceinline__ uint4 bytes16(uint32_t b) {
  return make_uint4(bytes4(b), bytes4(b >> 4), bytes4(b >> 8), bytes4(b >> 12));
}

// --------------------------------------------------------------------------- reductions
template <int NV>
__device__ __forceinline__ void block_sum_atomic(double (&v)[NV], double* dst, double* smem) {
  // smem: at least (blockDim/32) * NV doubles
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) smem[warp * NV + k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += smem[w * NV + threadIdx.x];
    if (s != 0.0) atomicAdd(dst + threadIdx.x, s);
  }
  __syncthreads();
}

// Integer block sums added to fp64 totals (one atomic per value and block).
template <int NV>
__device__ __forceinline__ void block_sum_atomic_int(int (&v)[NV], double* dst, int* smem) {
  // smem: at least (blockDim/32) * NV ints
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = __reduce_add_sync(0xffffffffu, v[k]);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) smem[warp * NV + k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    long long s = 0;
    for (int w = 0; w < nw; ++w) s += smem[w * NV + threadIdx.x];
    if (s != 0) atomicAdd(dst + threadIdx.x, (double)s);
  }
  __syncthreads();
}

// --------------------------------------------------------------------------- half step
enum { kEncInt8 = 0, kEncPacked = 1, kEncMultispin = 2 };

// Lane-word coordinates: row i and word column c of lane word w.
__device__ __forceinline__ void word_rc(const LatJob& J, uint32_t w, uint32_t& i, uint32_t& c) {
  if (J.wpr_shift != 0xffffffffu) {
    i = w >> J.wpr_shift;
    c = w & (J.wpr - 1u);
  } else {
    i = w / J.wpr;
    c = w - i * J.wpr;
  }
}

// Loads the three lane words a decision needs from buffer src: S (own), V (the
// vertical in-neighbour row: i-1 for half 0, i+1 for half 1) and H (the
// horizontal in-neighbour: j-1 for half 0, j+1 for half 1).
// NC: buf is a global buffer not written during the launch (read through the
// non-coherent cache); otherwise a plain load (shared memory).
template <bool NC, typename T>
__device__ __forceinline__ T ld_ro(const T* p) {
  if (NC) return __ldg(p);
  return *p;
}

template <int ENC, bool NC = true>
__device__ __forceinline__ void load_lane_words(const LatJob& J, const void* buf, uint32_t w,
                                                uint32_t half, uint32_t& S, uint32_t& V,
                                                uint32_t& H) {
  const uint32_t L = J.L, wpr = J.wpr;
  if (ENC != kEncInt8 && J.wpr_shift != 0xffffffffu) {
    // power-of-two rows (then L * wpr is one too): the neighbour words by masks --
    // the vertical one wpr words away modulo the lattice, the horizontal one the
    // next word of the same row, cyclically
    const uint32_t* A = static_cast<const uint32_t*>(buf);
    const uint32_t rowmask = wpr - 1u, allmask = J.nwords - 1u;
    const uint32_t dv = half == 0u ? 0u - wpr : wpr;
    const uint32_t dh = half == 0u ? 0xffffffffu : 1u;
    S = ld_ro<NC>(A + w);
    V = ld_ro<NC>(A + ((w + dv) & allmask));
    const uint32_t hn = ld_ro<NC>(A + ((w & ~rowmask) | ((w + dh) & rowmask)));
    if (ENC == kEncPacked)
      H = half == 0u ? ((S << 1) | (hn >> 31)) : ((S >> 1) | (hn << 31));
    else
      H = hn;
    return;
  }
  uint32_t i, c;
  word_rc(J, w, i, c);
  const uint32_t iv = half == 0u ? (i == 0u ? L - 1u : i - 1u) : (i + 1u == L ? 0u : i + 1u);
  if (ENC == kEncInt8) {
    const uint8_t* A = static_cast<const uint8_t*>(buf);
    const uint4* own = reinterpret_cast<const uint4*>(A + (size_t)i * L + 32u * c);
    const uint4* ver = reinterpret_cast<const uint4*>(A + (size_t)iv * L + 32u * c);
    const uint4 o0 = ld_ro<NC>(own), o1 = ld_ro<NC>(own + 1), v0 = ld_ro<NC>(ver),
                v1 = ld_ro<NC>(ver + 1);
    const uint32_t jn = half == 0u ? (c == 0u ? L - 1u : 32u * c - 1u)
                                   : (32u * c + 32u == L ? 0u : 32u * c + 32u);
    const uint32_t nb = (ld_ro<NC>(A + (size_t)i * L + jn) >> 7) ^ 1u;  // 1 if +1
    S = bits32(o0, o1);
    V = bits32(v0, v1);
    H = half == 0u ? ((S << 1) | nb) : ((S >> 1) | (nb << 31));
  } else if (ENC == kEncPacked) {
    const uint32_t* A = static_cast<const uint32_t*>(buf);
    S = ld_ro<NC>(A + (size_t)i * wpr + c);
    V = ld_ro<NC>(A + (size_t)iv * wpr + c);
    if (half == 0u) {
      const uint32_t cl = c == 0u ? wpr - 1u : c - 1u;
      H = (S << 1) | (ld_ro<NC>(A + (size_t)i * wpr + cl) >> 31);
    } else {
      const uint32_t cr = c + 1u == wpr ? 0u : c + 1u;
      H = (S >> 1) | (ld_ro<NC>(A + (size_t)i * wpr + cr) << 31);
    }
  } else {
    const uint32_t* A = static_cast<const uint32_t*>(buf);
    const uint32_t jn = half == 0u ? (c == 0u ? L - 1u : c - 1u) : (c + 1u == L ? 0u : c + 1u);
    S = ld_ro<NC>(A + w);
    V = ld_ro<NC>(A + (size_t)iv * L + c);
    H = ld_ro<NC>(A + (size_t)i * L + jn);
  }
}

// Per-job state shared by the block: the job descriptor, its threshold table
// for this step and the step counter.  Staged only when the job changes (the
// step counter and the table of a job are fixed for the whole launch).
struct TileShared {
  LatJob job;
  LatTable tab;
  PhShared ph;  // Philox rounds shared by every call of the job at this step
  uint32_t t;
  uint32_t skip;
  uint32_t fuse;
  uint32_t typ;
  const LatTable* tab_src;
};

// A lane word with undecided lanes, parked in its warp's queue as one 16-byte
// entry: (w, U, res, call), `call` the next Philox call it needs (2..7: planes
// 4 call .. 4 call + 3).  The class bits are recomputed from the state when the
// word's round comes (the source buffer does not change during the half step),
// so parking a word is a single 16-byte store.
using Pending = uint4;



template <int ENC>
__device__ __forceinline__ void store_word(const LatJob& J, void* dstbuf, uint32_t w,
                                           uint32_t tau) {
  if (ENC == kEncInt8) {
    uint32_t i, c;
    word_rc(J, w, i, c);
    uint4* dst =
        reinterpret_cast<uint4*>(static_cast<uint8_t*>(dstbuf) + (size_t)i * J.L + 32u * c);
    dst[0] = bytes16(tau);
    dst[1] = bytes16(tau >> 16);
  } else {
    static_cast<uint32_t*>(dstbuf)[w] = tau;
  }
}

// One round of the warp's queue: the top n = min(qn, 32) entries each make their
// next call and compare its four planes; finished words are stored, the others
// go back on the queue.  qn is warp-uniform.
template <int ENC, bool COLL>
__device__ __forceinline__ void tail_round(const LatJob& J, const TileShared& sh,
                                           Pending* __restrict__ q, uint32_t& qn,
                                           const PhKey& K, uint32_t typ, const void* srcbuf,
                                           void* dstbuf, uint32_t& calls) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint32_t n = qn < 32u ? qn : 32u;
  const uint32_t base = qn - n;
  const bool act = (uint32_t)lane < n;
  Pending e = make_uint4(0u, 0u, 0u, 0u);  // (w, U, res, call)
  if (act) e = q[base + lane];
  __syncwarp();
  bool still = false;
  if (act) {
    const uint4 w = ph_call_shared(K, sh.ph, e.x, typ + 2u * e.w);
    uint32_t S, V, H;
    load_lane_words<ENC>(J, srcbuf, e.x, typ, S, V, H);
    LaneWord L;
    L.S = S;
    L.V = COLL ? ((V & H) | (S & (V | H))) : V;  // as classify: majority / in-neighbour
    L.X = COLL ? (V ^ H ^ S) : (V ^ H);          // parity / one +1 neighbour
    L.U = e.y;
    L.res = e.z;
    ++calls;
    apply_call<COLL>(L, w, sh.tab, e.w);
    if (L.U == 0u || e.w == 7u) {
      store_word<ENC>(J, dstbuf, e.x, L.res);  // after plane 0 of call 7: u == T, tau = -1
    } else {
      still = true;
      e.y = L.U;
      e.z = L.res;
      e.w += 1u;
    }
  }
  const uint32_t sm = __ballot_sync(0xffffffffu, still);
  if (still) q[base + __popc(sm & lt_mask)] = e;
  qn = base + (uint32_t)__popc(sm);
  __syncwarp();
}

// Every queued word of the warp to the end (before the staged job changes).
template <int ENC>
__device__ __forceinline__ void tail_drain(const LatJob& J, const TileShared& sh,
                                           Pending* __restrict__ q, uint32_t& qn,
                                           const PhKey& K, uint32_t typ, const void* srcbuf,
                                           void* dstbuf, uint32_t& calls) {
  if (sh.tab.collapsed) {
    while (qn != 0u) tail_round<ENC, true>(J, sh, q, qn, K, typ, srcbuf, dstbuf, calls);
  } else {
    while (qn != 0u) tail_round<ENC, false>(J, sh, q, qn, K, typ, srcbuf, dstbuf, calls);
  }
}

// After the head: words with undecided lanes go to the warp's queue, the others
// are stored; the queue runs a round (one more call for each of 32 words, planes
// 23..0 four at a time) whenever it holds 32 words.  With sh.fuse the sums of
// sigma_t over the words are accumulated as well.
template <int ENC, int WPT, bool COLL, bool FULL>
__device__ __forceinline__ void tile_commit(const LatJob& J, const TileShared& sh,
                                            Pending* __restrict__ q, uint32_t& qn,
                                            const PhKey& K, const uint32_t (&a)[WPT],
                                            uint32_t half, const uint32_t (&S)[WPT],
                                            const uint32_t (&V)[WPT], const uint32_t (&H)[WPT],
                                            const LaneWord (&Lws)[WPT], const void* srcbuf,
                                            void* dstbuf, int (&acc)[3], uint32_t& calls) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int k = 0; k < WPT; ++k) {
    const uint32_t w = a[k];
    const bool act = FULL || w < J.nwords;
    const LaneWord& Lw = Lws[k];
    const bool pend = act && Lw.U != 0u;
    const uint32_t pm = __ballot_sync(0xffffffffu, pend);
    if (pend) {
      q[qn + __popc(pm & lt_mask)] = make_uint4(w, Lw.U, Lw.res, 2u);
    } else if (act) {
      store_word<ENC>(J, dstbuf, w, Lw.res);
    }
    qn += __popc(pm);
    if (ENC != kEncMultispin && sh.fuse && act) {
      // sums of sigma_t over the lane word: M, E (in-edges down and left), cut
      const int dv = __popc(S[k] ^ V[k]), dh = __popc(S[k] ^ H[k]);
      acc[0] += 2 * __popc(S[k]) - 32;
      acc[1] += 64 - 2 * dv - 2 * dh;
      acc[2] += dv + dh;
    }
  }
  __syncwarp();
  // words of this and earlier tiles wait until a full warp of them can go on
  while (qn >= 32u) tail_round<ENC, COLL>(J, sh, q, qn, K, half, srcbuf, dstbuf, calls);
}

// Decisions of one tile: planes 31..24 of each of the thread's WPT lane words;
// words with undecided lanes go to the warp's queue, which runs whenever it holds
// a full warp of them (one call per word and round; words still undecided go
// back).  The queue carries over to the block's next tile of the same job and is
// drained when the job changes.  FULL: every word of the tile exists.
template <int ENC, int WPT, bool COLL, bool FULL, bool MIR>
__device__ __forceinline__ void tile_decide(const LatJob& J, const TileShared& sh,
                                            Pending* __restrict__ q, uint32_t& qn,
                                            const PhKey& K, uint32_t w0,
                                            uint32_t half, const uint32_t (&S)[WPT],
                                            const uint32_t (&V)[WPT], const uint32_t (&H)[WPT],
                                            const uint32_t (&F)[WPT], const void* srcbuf,
                                            void* dstbuf, int (&acc)[3], uint32_t& calls) {
  LaneWord Lws[WPT];
  uint32_t a[WPT];
#pragma unroll
  for (int k = 0; k < WPT; ++k) {
    a[k] = w0 + threadIdx.x + k * kTile;
    Lws[k] = classify<COLL>(S[k], V[k], H[k], F[k], sh.tab);
    if (!FULL && a[k] >= J.nwords) Lws[k].U = 0u;
  }
  decide_head_words<COLL, WPT, MIR>(Lws, sh.tab, K, sh.ph, a, half);
  calls += 2u * WPT;
  tile_commit<ENC, WPT, COLL, FULL>(J, sh, q, qn, K, a, half, S, V, H, Lws, srcbuf, dstbuf, acc,
                                    calls);
}

// Each block walks a contiguous range of tiles (kLatTile lane words each; a
// tile never spans two jobs).  Per tile every thread loads the words of its
// kWordsPerThread lane words (all loads in flight together) and runs planes
// 31..24 of each; words with lanes still undecided are parked in the warp's
// queue, which makes the rare later calls only in full rounds of 32 words, so
// the warp pays for them once per 32 such words instead of once per word position.
template <int ENC, int WPT>
__global__ void __launch_bounds__(kTile, kLatMinBlocks) lattice_half_kernel(const LatJob* __restrict__ jobs,
                                                                const Tile* __restrict__ tiles,
                                                                int n_tiles, uint32_t half,
                                                                unsigned long long* rng_calls) {
  __shared__ TileShared sh;
  __shared__ Pending queue[kTile / 32][32 * WPT + 32];  // a tile's words + fewer than 32 left
  __shared__ double red[(kTile / 32) * 3];
  pdl_enter();
  uint32_t calls = 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // balanced contiguous split: block b walks tiles [b n / G, (b+1) n / G)
  const int tb = (int)(((long long)blockIdx.x * n_tiles) / gridDim.x);
  const int te = (int)(((long long)(blockIdx.x + 1) * n_tiles) / gridDim.x);
  int cur_job = -1;
  PhKey K = ph_key(0u, 0u);  // the job's key schedule, rebuilt on job change only
  uint32_t qn = 0;           // warp-uniform length of this warp's queue
  for (int ti = tb; ti < te; ++ti) {
    const Tile tl = tiles[ti];
    if ((int)tl.job != cur_job) {
      if (qn != 0u)  // finish the previous job's queued words while its state is staged
        tail_drain<ENC>(sh.job, sh, queue[warp], qn, K, sh.typ,
                        half == 0u ? sh.job.A : sh.job.B, half == 0u ? sh.job.B : sh.job.A,
                        calls);
      __syncthreads();  // every warp is done with the previous job's staged state
      constexpr int nw = sizeof(LatJob) / 4;
      if (threadIdx.x < nw)
        reinterpret_cast<uint32_t*>(&sh.job)[threadIdx.x] =
            reinterpret_cast<const uint32_t*>(jobs + tl.job)[threadIdx.x];
      __syncthreads();
      if (threadIdx.x == 0) {
        const CtxDev* cd = sh.job.cd;
        const uint32_t t = cd->step;
        sh.t = t;
        sh.skip = t >= cd->t_end;
        sh.fuse = (ENC != kEncMultispin) && half == 0u && sh.job.sums != nullptr && cd->tracking;
        sh.typ = half ^ cd->order;  // update type: 0 = dl / 1->2, 1 = ur / 2->1
        sh.ph = ph_shared(ph_key(sh.job.key0, sh.job.key1), sh.job.b, t);
        const LatTable* src = sh.job.table;
        if (sh.job.anneal_tables != nullptr && cd->anneal_len != 0u) {
          uint32_t k = t - cd->anneal_t0;
          if (k >= cd->anneal_len) k = cd->anneal_len - 1u;
          src = sh.job.anneal_tables + k;
        }
        sh.tab_src = src;
      }
      __syncthreads();
      if (!sh.skip) {
        const uint32_t* g = reinterpret_cast<const uint32_t*>(sh.tab_src);
        uint32_t* d = reinterpret_cast<uint32_t*>(&sh.tab);
        for (int k = threadIdx.x; k < (int)(sizeof(LatTable) / 4); k += kTile) d[k] = g[k];
      }
      __syncthreads();
      cur_job = (int)tl.job;
      K = ph_key(sh.job.key0, sh.job.key1);
    }
    if (sh.skip) continue;
    const LatJob& J = sh.job;
    const uint32_t typ = sh.typ;
    const void* src = half == 0u ? J.A : J.B;  // `half` is the position in the step
    void* dstbuf = half == 0u ? J.B : J.A;
    uint32_t S[WPT], V[WPT], H[WPT], F[WPT];
#pragma unroll
    for (int k = 0; k < WPT; ++k) {
      const uint32_t w = tl.w0 + threadIdx.x + k * kTile;
      S[k] = V[k] = H[k] = 0u;
      F[k] = 0u;
      if (w < J.nwords) {
        load_lane_words<ENC>(J, src, w, typ, S[k], V[k], H[k]);
        if (J.frozen != nullptr) F[k] = __ldg(J.frozen + w);
      }
    }
    int acc[3] = {0, 0, 0};  // tracking sums of this tile (|sum| <= 64 per word)
    const bool full_tile = tl.w0 + kTile * WPT <= J.nwords;
    if (sh.tab.mirror) {
      if (full_tile)
        tile_decide<ENC, WPT, true, true, true>(J, sh, queue[warp], qn, K, tl.w0, typ, S, V, H,
                                                F, src, dstbuf, acc, calls);
      else
        tile_decide<ENC, WPT, true, false, true>(J, sh, queue[warp], qn, K, tl.w0, typ, S, V, H,
                                                 F, src, dstbuf, acc, calls);
    } else if (sh.tab.collapsed) {
      if (full_tile)
        tile_decide<ENC, WPT, true, true, false>(J, sh, queue[warp], qn, K, tl.w0, typ, S, V, H,
                                                 F, src, dstbuf, acc, calls);
      else
        tile_decide<ENC, WPT, true, false, false>(J, sh, queue[warp], qn, K, tl.w0, typ, S, V,
                                                  H, F, src, dstbuf, acc, calls);
    } else {
      if (full_tile)
        tile_decide<ENC, WPT, false, true, false>(J, sh, queue[warp], qn, K, tl.w0, typ, S, V,
                                                  H, F, src, dstbuf, acc, calls);
      else
        tile_decide<ENC, WPT, false, false, false>(J, sh, queue[warp], qn, K, tl.w0, typ, S, V,
                                                   H, F, src, dstbuf, acc, calls);
    }
    if (sh.fuse) {
      int* redi = reinterpret_cast<int*>(red);
      int v2[2] = {acc[0], acc[1]};
      block_sum_atomic_int<2>(v2, J.sums + kSumM, redi);
      int v1[1] = {acc[2]};
      block_sum_atomic_int<1>(v1, J.sums + kSumCut, redi);
    }
  }
  if (qn != 0u)
    tail_drain<ENC>(sh.job, sh, queue[warp], qn, K, sh.typ, half == 0u ? sh.job.A : sh.job.B,
                    half == 0u ? sh.job.B : sh.job.A, calls);
  if (rng_calls != nullptr) {
    const uint32_t wsum = __reduce_add_sync(0xffffffffu, calls);
    if (lane == 0 && wsum) atomicAdd(rng_calls, (unsigned long long)wsum);
  }
}

// --------------------------------------------------------------------------- init
// sigma = +1 iff u < 2^31 with u the draw of step 0xFFFFFFFF, half 0: bit 31 of u
// is bit k of the first plane word W_0, so sigma_k = +1 iff that bit is 0.
// kind: 0 random, 1 plus, 2 minus.  Frozen lanes +1.  Writes A and B.
template <int ENC>
__global__ void __launch_bounds__(kTile) lattice_init_kernel(const LatJob* __restrict__ jobs,
                                                             const Tile* __restrict__ tiles,
                                                             int n_tiles, int kind, int wpt) {
  for (int ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
    const Tile tl = tiles[ti];
    const LatJob& J = jobs[tl.job];
    for (int k = 0; k < wpt; ++k) {
      const uint32_t w = tl.w0 + threadIdx.x + k * kTile;
      if (w >= J.nwords) break;
      uint32_t s;
      if (kind == 1) {
        s = 0xffffffffu;
      } else if (kind == 2) {
        s = 0u;
      } else {
        const PhKey K = ph_key(J.key0, J.key1);
        const uint4 W = ph_call(K, w, J.b, kInitStep, 0u);
        s = ~W.x;
      }
      if (J.frozen != nullptr) s |= J.frozen[w];
      if (ENC == kEncInt8) {
        uint32_t i, c;
        word_rc(J, w, i, c);
        const size_t off = (size_t)i * J.L + 32u * c;
        uint4* a = reinterpret_cast<uint4*>(static_cast<uint8_t*>(J.A) + off);
        uint4* b = reinterpret_cast<uint4*>(static_cast<uint8_t*>(J.B) + off);
        a[0] = b[0] = bytes16(s);
        a[1] = b[1] = bytes16(s >> 16);
      } else {
        static_cast<uint32_t*>(J.A)[w] = s;
        static_cast<uint32_t*>(J.B)[w] = s;
      }
    }
  }
}

// --------------------------------------------------------------------------- observables
// INT8 / PACKED: per lane word, integer sums of sigma (A) and sigma' (B):
//   M, E = in-edge product sum (down, left), P1 = sum sigma_x (sigma'_up + sigma'_right),
//   P2 = sum sigma_x sigma'_x, M2 = sum sigma', cut.
template <int ENC>
__global__ void __launch_bounds__(kTile) lattice_obs_single_kernel(
    const LatJob* __restrict__ jobs, const Tile* __restrict__ tiles, int n_tiles, int which,
    int full, int wpt) {
  __shared__ double red[(kTile / 32) * 3];
  pdl_enter();
  for (int ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
    const Tile tl = tiles[ti];
    const LatJob& J = jobs[tl.job];
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int k = 0; k < wpt; ++k) {
      const uint32_t w = tl.w0 + threadIdx.x + k * kTile;
      if (w >= J.nwords) break;
      uint32_t S, V, H;
      load_lane_words<ENC>(J, J.A, w, 0u, S, V, H);
      const int dv = __popc(S ^ V), dh = __popc(S ^ H);
      v[0] += (double)(2 * __popc(S) - 32);
      v[1] += (double)(64 - 2 * dv - 2 * dh);
      v[5] += (double)(dv + dh);
      if (full) {
        uint32_t S2, U2, R2;
        load_lane_words<ENC>(J, J.B, w, 1u, S2, U2, R2);  // sigma', its up and right bits
        v[2] += (double)(64 - 2 * __popc(S ^ U2) - 2 * __popc(S ^ R2));
        v[3] += (double)(32 - 2 * __popc(S ^ S2));
        v[4] += (double)(2 * __popc(S2) - 32);
      }
    }
    double* dst = which ? J.obs : J.sums;
    double a[2] = {v[0], v[1]};
    block_sum_atomic<2>(a, dst + kSumM, red);
    double b3[3] = {v[2], v[3], v[4]};
    block_sum_atomic<3>(b3, dst + kSumP1, red);
    double c1[1] = {v[5]};
    block_sum_atomic<1>(c1, dst + kSumCut, red);
  }
}

// MULTISPIN: per-lane (= per replica) sums.  Each warp covers 32 consecutive sites at
// a time; for every mask the warp's 32 words are transposed so that lane k counts
// replica k's bits (warp_column_count).
__global__ void __launch_bounds__(kTile) lattice_obs_multispin_kernel(
    const LatJob* __restrict__ jobs, const Tile* __restrict__ tiles, int n_tiles, int which,
    int full, int wpt) {
  __shared__ int red[kTile / 32][32][6];
  pdl_enter();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
    const Tile tl = tiles[ti];
    const LatJob& J = jobs[tl.job];
    int cnt[6] = {0, 0, 0, 0, 0, 0};
    for (int sub = 0; sub < wpt; ++sub) {
      const uint32_t w = tl.w0 + threadIdx.x + sub * kTile;
      const bool act = w < J.nwords;
      uint32_t S = 0, V = 0, H = 0, S2 = 0, U2 = 0, R2 = 0;
      if (act) {
        load_lane_words<kEncMultispin>(J, J.A, w, 0u, S, V, H);
        if (full) load_lane_words<kEncMultispin>(J, J.B, w, 1u, S2, U2, R2);
      }
      const uint32_t act_m = act ? 0xffffffffu : 0u;
      const int nact = __popc(__ballot_sync(0xffffffffu, act));
      const int c0 = warp_column_count(S & act_m, lane);
      const int c1 = warp_column_count(~(S ^ V) & act_m, lane) +
                     warp_column_count(~(S ^ H) & act_m, lane);
      cnt[0] += 2 * c0 - nact;      // sum sigma
      cnt[1] += 2 * c1 - 2 * nact;  // in-edge products
      cnt[5] += 2 * nact - c1;      // cut = disagreements
      if (full) {
        const int c2 = warp_column_count(~(S ^ U2) & act_m, lane) +
                       warp_column_count(~(S ^ R2) & act_m, lane);
        cnt[2] += 2 * c2 - 2 * nact;                                  // P1
        cnt[3] += 2 * warp_column_count(~(S ^ S2) & act_m, lane) - nact;  // P2
        cnt[4] += 2 * warp_column_count(S2 & act_m, lane) - nact;         // M2
      }
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) red[warp][lane][q] = cnt[q];
    __syncthreads();
    if (threadIdx.x < 32) {
      int tot[6] = {0, 0, 0, 0, 0, 0};
      for (int wv = 0; wv < kTile / 32; ++wv)
#pragma unroll
        for (int q = 0; q < 6; ++q) tot[q] += red[wv][threadIdx.x][q];
      double* dst = (which ? J.obs : J.sums) + (size_t)threadIdx.x * kNumSums;
      if (tot[0]) atomicAdd(dst + kSumM, (double)tot[0]);
      if (tot[1]) atomicAdd(dst + kSumE, (double)tot[1]);
      if (full) {
        if (tot[2]) atomicAdd(dst + kSumP1, (double)tot[2]);
        if (tot[3]) atomicAdd(dst + kSumP2, (double)tot[3]);
        if (tot[4]) atomicAdd(dst + kSumM2, (double)tot[4]);
      }
      if (tot[5]) atomicAdd(dst + kSumCut, (double)tot[5]);
    }
    __syncthreads();
  }
}

// --------------------------------------------------------------------------- resident runs
// Small lattices: one block owns one job (an int8/packed replica or a multispin
// group) for a whole run of n steps.  The state lives in shared memory as bit
// lane words (the packed layout for INT8/PACKED, the multispin layout
// otherwise) between a barrier per half step; the draws, thresholds and
// decisions are the ones of lattice_half_kernel, so the trajectory is the same.
// With tracking (INT8/PACKED only) the block also evaluates H(sigma_t) each step
// and updates the best energy and the per-step series itself.
template <int ENC>
__device__ __forceinline__ uint32_t resident_load(const LatJob& J, uint32_t w) {
  if (ENC == kEncInt8) {
    uint32_t i, c;
    word_rc(J, w, i, c);
    const uint4* p = reinterpret_cast<const uint4*>(static_cast<const uint8_t*>(J.A) +
                                                    (size_t)i * J.L + 32u * c);
    return bits32(p[0], p[1]);
  }
  return static_cast<const uint32_t*>(J.A)[w];
}

template <int ENC>
__device__ __forceinline__ void resident_store(const LatJob& J, void* buf, uint32_t w,
                                               uint32_t bits) {
  if (ENC == kEncInt8) {
    uint32_t i, c;
    word_rc(J, w, i, c);
    uint4* p = reinterpret_cast<uint4*>(static_cast<uint8_t*>(buf) + (size_t)i * J.L + 32u * c);
    p[0] = bytes16(bits);
    p[1] = bytes16(bits >> 16);
  } else {
    static_cast<uint32_t*>(buf)[w] = bits;
  }
}

template <int ENC>
__global__ void __launch_bounds__(kTile) lattice_resident_kernel(const LatJob* __restrict__ jobs,
                                                                 uint32_t t0, uint32_t n_steps) {
  constexpr int SENC = ENC == kEncMultispin ? kEncMultispin : kEncPacked;  // smem layout
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ LatTable stab;
  __shared__ int red[kTile / 32][3];
  const LatJob J = jobs[blockIdx.x];  // by value: the fields stay in registers
  const uint32_t nw = J.nwords;
  uint32_t* sA = smem;
  uint32_t* sB = smem + nw;
  const CtxDev* cd = J.cd;
  const uint32_t anneal_t0 = cd->anneal_t0, anneal_len = cd->anneal_len;
  const bool track = ENC != kEncMultispin && cd->tracking && J.sums != nullptr;
  const uint32_t order = cd->order;
  const bool record = track && cd->record;
  // the context's constants for the per-step tracking, read once (nothing else
  // touches this context while the run is resident); the best energy in a register
  const uint32_t r = J.rep0;
  const double Jc = cd->Jc, lamc = cd->lamc, inv_n = cd->inv_n;
  const uint32_t series_t0 = cd->series_t0, series_cap = cd->series_cap, Rn = cd->R;
  double* const best_p = cd->best;
  long long* const best_step_p = cd->best_step;
  double* const series_m = cd->series_m;
  double* const series_H = cd->series_H;
  double best = track && threadIdx.x == 0 ? best_p[r] : 0.0;
  for (uint32_t w = threadIdx.x; w < nw; w += blockDim.x) sA[w] = resident_load<ENC>(J, w);
  const PhKey K = ph_key(J.key0, J.key1);
  const LatTable* staged = nullptr;
  uint32_t calls = 0;
  for (uint32_t st = 0; st < n_steps; ++st) {
    const uint32_t t = t0 + st;
    const LatTable* src = J.table;
    if (J.anneal_tables != nullptr && anneal_len != 0u) {
      uint32_t k = t - anneal_t0;
      if (k >= anneal_len) k = anneal_len - 1u;
      src = J.anneal_tables + k;
    }
    if (src != staged) {
      __syncthreads();
      const uint32_t* g = reinterpret_cast<const uint32_t*>(src);
      uint32_t* d = reinterpret_cast<uint32_t*>(&stab);
      for (int k = threadIdx.x; k < (int)(sizeof(LatTable) / 4); k += blockDim.x) d[k] = g[k];
      staged = src;
    }
    __syncthreads();  // sA complete (previous half step or the load), table staged
    const PhShared P = ph_shared(K, J.b, t);
    int acc[3] = {0, 0, 0};  // integer sums (at most 32 x 4096 sites per block)
    for (uint32_t pos = 0; pos < 2; ++pos) {
      const uint32_t half = pos ^ order;  // update type of this position
      const uint32_t* in = pos == 0u ? sA : sB;
      uint32_t* out = pos == 0u ? sB : sA;
      if (track && pos == 1u && threadIdx.x == 0) {
        // block totals of sigma_t's sums (written before the barrier that ended
        // position 0) -> best energy and series (Eq. (HGibbs)), off the barriers
        int Mi = 0, Ei = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
          Mi += red[w][0];
          Ei += red[w][1];
        }
        const double M = (double)Mi, E = (double)Ei;
        const double Hs = -(Jc * E) - 2.0 * lamc * M;
        if (Hs < best) {
          best = Hs;
          best_p[r] = Hs;
          best_step_p[r] = (long long)t;
        }
        if (record && t - series_t0 < series_cap) {
          const size_t k = (size_t)(t - series_t0) * Rn + r;
          if (series_m) series_m[k] = M * inv_n;
          if (series_H) series_H[k] = Hs;
        }
      }
      for (uint32_t w = threadIdx.x; w < nw; w += blockDim.x) {
        uint32_t S, V, H;
        load_lane_words<SENC, false>(J, in, w, half, S, V, H);
        const uint32_t F = J.frozen != nullptr ? J.frozen[w] : 0u;
        LaneWord Lw;
        if (stab.collapsed) {
          Lw = classify<true>(S, V, H, F, stab);
          decide_head3<true>(Lw, stab, K, P, w, half, calls);
          decide_tail<true>(Lw, stab, K, P, w, half, 3u, calls);
        } else {
          Lw = classify<false>(S, V, H, F, stab);
          decide_head3<false>(Lw, stab, K, P, w, half, calls);
          decide_tail<false>(Lw, stab, K, P, w, half, 3u, calls);
        }
        out[w] = Lw.res;
        if (track && pos == 0u) {
          const int dv = __popc(S ^ V), dh = __popc(S ^ H);
          acc[0] += 2 * __popc(S) - 32;
          acc[1] += 64 - 2 * dv - 2 * dh;
          acc[2] += dv + dh;
        }
      }
      if (track && pos == 0u) {  // warp totals of sigma_t's sums
#pragma unroll
        for (int q = 0; q < 2; ++q) acc[q] = __reduce_add_sync(0xffffffffu, acc[q]);
        if ((threadIdx.x & 31) == 0)
          for (int q = 0; q < 2; ++q) red[threadIdx.x >> 5][q] = acc[q];
      }
      __syncthreads();
    }
  }
  __syncthreads();
  for (uint32_t w = threadIdx.x; w < nw; w += blockDim.x) {
    resident_store<ENC>(J, J.A, w, sA[w]);
    resident_store<ENC>(J, J.B, w, sB[w]);
  }
  (void)calls;
}

// --------------------------------------------------------------------------- banded runs
// Mid-size single lattices (INT8/PACKED, one replica, more lane words than one
// block holds): a cooperative grid keeps the lattice in shared memory, in the
// packed layout, as bands of rows for a whole run of n steps.  Block b owns rows
// [b L / G, (b+1) L / G) and also holds the row above and the row below its band
// (halo rows; the lattice wraps).  A half step of type dl reads the row above each
// row, one of type ur the row below, so between two half steps one row crosses each
// band boundary, in one direction: in every half step a block first decides the
// own row its neighbour will read next and publishes it word by word to a global
// exchange area (two sets by half-step parity), then decides its other rows, then
// takes the one halo row it needs next from the neighbour on that side.  One grid
// barrier at the end of the run decides whether it is committed.
// The draws, thresholds and decisions are those of lattice_half_kernel (head of
// four words per thread, eight planes, a per-warp queue for the words still
// undecided), so the trajectory is the same.

constexpr uint64_t kBandWaitNs = 1000000000ull;  // a barrier wait gives up after 1 s (%globaltimer)
constexpr uint32_t kBandPollLimit = 1u << 26;      // and after this many polls in any case
constexpr int kBandMinBlocks = 2;  // blocks per SM: 126 registers, no spills (3: spills, slower)

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier of a cooperative launch in two phases, so a block can compute
// between announcing its rows and needing its neighbours'.  band_arrive: after a
// block barrier thread 0 fences (the fence orders the writes of every thread of
// the block that the barrier ordered before it) and counts the block in; the last
// block resets the count and advances the generation.
// band_wait: thread 0 polls the generation until a deadline of kBandWaitNs on the
// global timer (and at most kBandPollLimit polls); a wait that runs out, or that
// sees another block's error, sets the error flag and then settles the run's
// outcome with one compare-and-swap on `commit`: 0 -> 2 (aborted) unless the last
// barrier has already been passed by every block and the run committed (1), in
// which case this block still writes its band back.  Returns 0 to go on, 1 to
// return without writing, 2 to write back (only possible at the last barrier).
__device__ __forceinline__ void band_arrive(BandSync* bs, uint32_t gen) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&bs->count, 1u) == gridDim.x - 1u) {
      atomicExch(&bs->count, 0u);
      __threadfence();
      atomicExch(&bs->gen, gen + 1u);
    }
  }
}

__device__ __forceinline__ uint32_t band_wait(BandSync* bs, uint32_t& gen, uint32_t* s_flag,
                                              bool last) {
  if (threadIdx.x == 0) {
    const uint64_t limit = (last && bs->hurry == blockIdx.x) ? 0ull : kBandWaitNs;
    const uint64_t t0 = global_ns();
    uint32_t polls = 0, f = 0u;
    while (atomicAdd(&bs->gen, 0u) == gen) {
      if (atomicAdd(&bs->err, 0u) != 0u || global_ns() - t0 > limit || ++polls > kBandPollLimit) {
        atomicExch(&bs->err, 1u);
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    if (atomicAdd(&bs->err, 0u) != 0u) f = atomicCAS(&bs->commit, 0u, 2u) == 1u ? 2u : 1u;
    *s_flag = f;
  }
  gen += 1u;
  __syncthreads();
  return *s_flag;
}

// Neighbour exchange between half steps: every published row word is one 64-bit
// store of (half-step count << 32 | word), the count being the number of half
// steps of the launch done (1, 2, ...; the area is zeroed before each launch).
// A reader polls each halo word until its count is the one it needs: the word and
// its count are read together (single-copy atomic), so no fence or flag orders the
// exchange.  Two sets by half-step parity: a block overwrites the set of half step
// h at h + 2 only after it has read its neighbours' rows of h + 1, which they wrote
// after reading those of h.  A count other than the expected one is never taken;
// a wait gives up on the same deadline and error flag as the grid barrier.
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// The word of half step `count` at p; false when the wait gave up (error flag set,
// run aborted unless already committed, which cannot happen before the last barrier).
__device__ __forceinline__ bool band_fetch(const uint64_t* p, uint32_t count, BandSync* bs,
                                           uint32_t& v) {
  uint64_t x = ld_relaxed_u64(p);
  if ((uint32_t)(x >> 32) != count) {
    const uint64_t t0 = global_ns();
    uint32_t polls = 0;
    do {
      // the error flag by a plain load every 16 polls: many threads poll at once
      if (((++polls & 15u) == 0u && *reinterpret_cast<volatile const uint32_t*>(&bs->err) != 0u) ||
          global_ns() - t0 > kBandWaitNs || polls > kBandPollLimit) {
        atomicExch(&bs->err, 1u);
        atomicCAS(&bs->commit, 0u, 2u);
        return false;
      }
      __nanosleep(32);
      x = ld_relaxed_u64(p);
    } while ((uint32_t)(x >> 32) != count);
  }
  v = (uint32_t)x;
  return true;
}

// S, V, H of local word l (column c) of a band buffer (packed rows of wpr words;
// local rows 0 and nr + 1 are the halo rows, l lies in an own row).
__device__ __forceinline__ void band_words(const uint32_t* buf, uint32_t l, uint32_t c,
                                           uint32_t wpr, uint32_t typ, uint32_t& S, uint32_t& V,
                                           uint32_t& H) {
  S = buf[l];
  const uint32_t rowbase = l - c;
  if (typ == 0u) {  // dl: row i-1, column j-1
    V = buf[l - wpr];
    H = (S << 1) | (buf[rowbase + (c == 0u ? wpr - 1u : c - 1u)] >> 31);
  } else {          // ur: row i+1, column j+1
    V = buf[l + wpr];
    H = (S >> 1) | (buf[rowbase + (c + 1u == wpr ? 0u : c + 1u)] << 31);
  }
}

// One round of a warp's queue of band words still undecided after eight planes
// (entries (global word, undecided lanes, results, next call), as in the tiled
// kernel): the top min(qn, 32) entries each make their next call; finished words
// are written to out, the others go back on the queue.
template <bool COLL>
__device__ __forceinline__ void band_round(const LatTable& tab, const uint32_t* in, uint32_t* out,
                                           Pending* __restrict__ q, uint32_t& qn,
                                           uint32_t w_first, uint32_t wpr, bool pow2,
                                           uint32_t typ, const PhKey& K, const PhShared& P,
                                           uint32_t& calls) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint32_t n = qn < 32u ? qn : 32u;
  const uint32_t base = qn - n;
  const bool act = (uint32_t)lane < n;
  Pending e = make_uint4(0u, 0u, 0u, 0u);
  if (act) e = q[base + lane];
  __syncwarp();
  bool still = false;
  if (act) {
    const uint4 w = ph_call_shared(K, P, e.x, typ + 2u * e.w);
    const uint32_t o = e.x - w_first;
    const uint32_t loc = wpr + o, c = pow2 ? (o & (wpr - 1u)) : o % wpr;
    uint32_t S, V, H;
    band_words(in, loc, c, wpr, typ, S, V, H);
    LaneWord L;
    L.S = S;
    L.V = COLL ? ((V & H) | (S & (V | H))) : V;
    L.X = COLL ? (V ^ H ^ S) : (V ^ H);
    L.U = e.y;
    L.res = e.z;
    ++calls;
    apply_call<COLL>(L, w, tab, e.w);
    if (L.U == 0u || e.w == 7u) {
      out[loc] = L.res;
    } else {
      still = true;
      e.y = L.U;
      e.z = L.res;
      e.w += 1u;
    }
  }
  const uint32_t sm = __ballot_sync(0xffffffffu, still);
  if (still) q[base + __popc(sm & lt_mask)] = e;
  qn = base + (uint32_t)__popc(sm);
  __syncwarp();
}

// One pass over W x kTile own words of the band starting at own word o0: planes
// 31..24 of every word; words with undecided lanes go to the warp's queue, which
// runs a round whenever it holds 32 of them.
// Own words are addressed through an index: word idx of a range is own word
// idx + (idx < s1 ? o0 : idx < s2 ? o1 : o2), so the first own row, the last own
// row and a run of interior rows can be one range.
struct BandRange {
  uint32_t n, s1, s2, o0, o1, o2;
};

template <bool COLL, bool MIR, int W>
__device__ __forceinline__ void band_pass(const LatJob& J, const LatTable& tab,
                                          const uint32_t* in, uint32_t* out, uint32_t i0,
                                          const BandRange& R, uint32_t w_first, uint32_t wpr,
                                          bool pow2, uint32_t typ, const PhKey& K,
                                          const PhShared& P, Pending* __restrict__ q,
                                          uint32_t& qn, uint32_t& calls) {
  LaneWord Lw[W];
  uint32_t a[W];
  bool act[W];
#pragma unroll
  for (int k = 0; k < W; ++k) {
    const uint32_t idx = i0 + threadIdx.x + (uint32_t)k * kTile;
    act[k] = idx < R.n;
    const uint32_t oo = act[k] ? idx + (idx < R.s1 ? R.o0 : idx < R.s2 ? R.o1 : R.o2) : 0u;
    const uint32_t c = pow2 ? (oo & (wpr - 1u)) : oo % wpr;
    a[k] = w_first + oo;  // global lane word: the Philox counter and the frozen mask
    uint32_t S, V, H;
    band_words(in, wpr + oo, c, wpr, typ, S, V, H);  // own rows start at local row 1
    const uint32_t F = (J.frozen != nullptr && act[k]) ? J.frozen[a[k]] : 0u;
    Lw[k] = classify<COLL>(S, V, H, F, tab);
    if (!act[k]) Lw[k].U = 0u;
  }
  decide_head_words<COLL, W, MIR>(Lw, tab, K, P, a, typ);
  calls += 2u * W;
  const int lane = threadIdx.x & 31;
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    const bool pend = act[k] && Lw[k].U != 0u;
    const uint32_t pm = __ballot_sync(0xffffffffu, pend);
    if (pend)
      q[qn + __popc(pm & lt_mask)] = make_uint4(a[k], Lw[k].U, Lw[k].res, 2u);
    else if (act[k])
      out[a[k] - w_first + wpr] = Lw[k].res;
    qn += __popc(pm);
  }
  __syncwarp();
  while (qn >= 32u) band_round<COLL>(tab, in, out, q, qn, w_first, wpr, pow2, typ, K, P, calls);
}

// Every word of a range of own words decided (the queue drained at the end).
template <bool COLL, bool MIR>
__device__ __forceinline__ void band_range(const LatJob& J, const LatTable& tab,
                                           const uint32_t* in, uint32_t* out, const BandRange& R,
                                           uint32_t w_first, uint32_t wpr, uint32_t typ,
                                           const PhKey& K, const PhShared& P,
                                           Pending* __restrict__ q, uint32_t& calls) {
  const bool pow2 = J.wpr_shift != 0xffffffffu;
  uint32_t qn = 0, i0 = 0;
  for (; i0 + (uint32_t)kLatTile <= R.n; i0 += kLatTile)
    band_pass<COLL, MIR, kWordsPerThread>(J, tab, in, out, i0, R, w_first, wpr, pow2, typ, K, P,
                                          q, qn, calls);
  // the rest in one pass of as many words per thread as it needs
  const uint32_t rest = R.n - i0;
  if (rest > 3u * kTile)
    band_pass<COLL, MIR, 4>(J, tab, in, out, i0, R, w_first, wpr, pow2, typ, K, P, q, qn, calls);
  else if (rest > 2u * kTile)
    band_pass<COLL, MIR, 3>(J, tab, in, out, i0, R, w_first, wpr, pow2, typ, K, P, q, qn, calls);
  else if (rest > (uint32_t)kTile)
    band_pass<COLL, MIR, 2>(J, tab, in, out, i0, R, w_first, wpr, pow2, typ, K, P, q, qn, calls);
  else if (rest > 0u)
    band_pass<COLL, MIR, 1>(J, tab, in, out, i0, R, w_first, wpr, pow2, typ, K, P, q, qn, calls);
  while (qn != 0u) band_round<COLL>(tab, in, out, q, qn, w_first, wpr, pow2, typ, K, P, calls);
}

// band_range with the table's decision form.
__device__ __forceinline__ void band_decide(const LatJob& J, const LatTable& tab,
                                            const uint32_t* in, uint32_t* out,
                                            const BandRange& R, uint32_t w_first, uint32_t wpr,
                                            uint32_t typ, const PhKey& K, const PhShared& P,
                                            Pending* __restrict__ q, uint32_t& calls) {
  if (R.n == 0u) return;
  if (tab.mirror)
    band_range<true, true>(J, tab, in, out, R, w_first, wpr, typ, K, P, q, calls);
  else if (tab.collapsed)
    band_range<true, false>(J, tab, in, out, R, w_first, wpr, typ, K, P, q, calls);
  else
    band_range<false, false>(J, tab, in, out, R, w_first, wpr, typ, K, P, q, calls);
}

// The own row `orow` that a neighbour reads in the next half step: one word per
// thread, decided by three unconditional calls (twelve planes) and the rare later
// ones, without the warp queue, and published word by word (no block barrier).
// Word c goes to thread blockDim - 1 - c: the passes over the other rows give
// their extra words to the first threads.
template <bool COLL>
__device__ __forceinline__ void band_edge(const LatJob& J, const LatTable& tab,
                                          const uint32_t* in, uint32_t* out, uint32_t orow,
                                          uint32_t w_first, uint32_t wpr, uint32_t typ,
                                          const PhKey& K, const PhShared& P, uint64_t* pub,
                                          uint64_t tag, uint32_t& calls) {
  for (uint32_t c = blockDim.x - 1u - threadIdx.x; c < wpr; c += blockDim.x) {
    const uint32_t oo = orow * wpr + c, a = w_first + oo;
    uint32_t S, V, H;
    band_words(in, wpr + oo, c, wpr, typ, S, V, H);
    const uint32_t F = J.frozen != nullptr ? J.frozen[a] : 0u;
    LaneWord L = classify<COLL>(S, V, H, F, tab);
    decide_head3<COLL>(L, tab, K, P, a, typ, calls);
    if (L.U != 0u) decide_tail<COLL>(L, tab, K, P, a, typ, 3u, calls);
    out[wpr + oo] = L.res;
    st_relaxed_u64(pub + c, tag | L.res);
  }
}

// xch: exchange area, [2 parities][G blocks][wpr words] of (count << 32 | word),
// zeroed before the launch.
template <int ENC>
__global__ void __launch_bounds__(kTile, kBandMinBlocks) lattice_band_kernel(
    const LatJob* __restrict__ jobs, uint64_t* __restrict__ xch, BandSync* __restrict__ bs,
    uint32_t t0, uint32_t n_steps) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ LatTable stab;
  __shared__ LatJob sJ;  // the job descriptor, read from shared memory
  __shared__ uint32_t s_flag;
  __shared__ Pending queue[kTile / 32][32 * kWordsPerThread + 32];
  if (threadIdx.x < sizeof(LatJob) / 4)
    reinterpret_cast<uint32_t*>(&sJ)[threadIdx.x] =
        reinterpret_cast<const uint32_t*>(jobs)[threadIdx.x];
  __syncthreads();
  const LatJob& J = sJ;
  const uint32_t L = J.L, wpr = J.wpr, G = gridDim.x, b = blockIdx.x;
  const uint32_t r0 = (uint32_t)(((uint64_t)b * L) / G);
  const uint32_t r1 = (uint32_t)(((uint64_t)(b + 1u) * L) / G);
  const uint32_t nr = r1 - r0, n_own = nr * wpr, n_loc = n_own + 2u * wpr;
  uint32_t* buf[2] = {smem, smem + n_loc};  // sigma (A), sigma' (B)
  const uint32_t order = J.cd->order;
  uint32_t gen = 0;
  bool write_back = false;  // the run was committed while this block was giving up
  if (threadIdx.x == 0) gen = atomicAdd(&bs->gen, 0u);
  // sigma's rows r0 - 1 .. r1 (wrapping) and the table
  for (uint32_t l = threadIdx.x; l < n_loc; l += blockDim.x) {
    const uint32_t rl = l / wpr, c = l - rl * wpr;
    const uint32_t g = (r0 + L + rl - 1u) % L;
    buf[0][l] = resident_load<ENC>(J, g * wpr + c);
  }
  {
    const uint32_t* g = reinterpret_cast<const uint32_t*>(J.table);
    uint32_t* d = reinterpret_cast<uint32_t*>(&stab);
    for (int k = threadIdx.x; k < (int)(sizeof(LatTable) / 4); k += blockDim.x) d[k] = g[k];
  }
  const PhKey K = ph_key(J.key0, J.key1);
  const uint32_t w_first = r0 * wpr;
  Pending* q = queue[threadIdx.x >> 5];
  uint32_t calls = 0;
  __syncthreads();
  for (uint32_t st = 0; st < n_steps; ++st) {
    const PhShared P = ph_shared(K, J.b, t0 + st);
    for (uint32_t pos = 0; pos < 2u; ++pos) {
      const uint32_t typ = pos ^ order;  // update type of this position
      const uint32_t* in = buf[pos];
      uint32_t* out = buf[pos ^ 1u];
      // In the next half step (type typ ^ 1) a band reads one neighbouring row: the
      // one above it (type 0, dl) or below it (type 1, ur).  So this block publishes
      // one own row -- its last row for the block below, or its first row for the
      // block above -- first, then decides its other rows, then fetches the one halo
      // row it needs next, published by the neighbour on that side.
      const uint32_t nxt = typ ^ 1u;
      const uint32_t prow = nxt == 0u ? nr - 1u : 0u;
      const uint32_t count = 2u * st + pos + 1u;  // half steps of this launch done
      const uint64_t tag = (uint64_t)count << 32;
      if (stab.collapsed)
        band_edge<true>(J, stab, in, out, prow, w_first, wpr, typ, K, P,
                        xch + ((size_t)pos * G + b) * wpr, tag, calls);
      else
        band_edge<false>(J, stab, in, out, prow, w_first, wpr, typ, K, P,
                         xch + ((size_t)pos * G + b) * wpr, tag, calls);
      const BandRange R = {n_own - wpr, 0xffffffffu, 0xffffffffu, prow == 0u ? wpr : 0u, 0u,
                           0u};
      band_decide(J, stab, in, out, R, w_first, wpr, typ, K, P, q, calls);
      const uint32_t nbr = nxt == 0u ? (b + G - 1u) % G : (b + 1u) % G;
      const uint64_t* src = xch + ((size_t)pos * G + nbr) * wpr;
      uint32_t* halo = out + (nxt == 0u ? 0u : (nr + 1u) * wpr);
      bool ok = true;
      for (uint32_t c = threadIdx.x; c < wpr && ok; c += blockDim.x) {
        uint32_t v = 0u;
        ok = band_fetch(src + c, count, bs, v);
        halo[c] = v;
      }
      if (__syncthreads_or(!ok)) return;  // the run is aborted: nothing is written
    }
  }
  // one grid barrier for the whole chunk: every block has finished its last half step
  band_arrive(bs, gen);
  const uint32_t w = band_wait(bs, gen, &s_flag, true);
  if (w == 1u) return;
  write_back = w == 2u;
  if (!write_back) {
    // every block passed the last barrier: commit (0 -> 1) unless a block that gave
    // up has already aborted the run (2); the chunk is written back only if committed
    if (threadIdx.x == 0) s_flag = atomicCAS(&bs->commit, 0u, 1u) == 2u ? 1u : 0u;
    __syncthreads();
    if (s_flag != 0u) return;
  }
  for (uint32_t o = threadIdx.x; o < n_own; o += blockDim.x) {
    resident_store<ENC>(J, J.A, w_first + o, buf[0][wpr + o]);
    resident_store<ENC>(J, J.B, w_first + o, buf[1][wpr + o]);
  }
  (void)calls;
}

// --------------------------------------------------------------------------- launchers
static int grid_for(int n_tiles, int per_sm) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int g = sms * per_sm;
  return n_tiles < g ? (n_tiles > 0 ? n_tiles : 1) : g;
}

cudaError_t launch_build_lattice_tables(const double* beta_lanes, int ntab, double J, double q,
                                        double lam, LatTable* out, cudaStream_t st) {
  if (ntab <= 0) return cudaSuccess;
  build_lattice_tables_kernel<<<ntab, 256, 0, st>>>(beta_lanes, ntab, J, q, lam, out);
  return cudaGetLastError();
}

template <int ENC, int WPT>
static cudaError_t launch_half_t(const LatJob* jobs, const Tile* tiles, int n_tiles, uint32_t half,
                                 unsigned long long* rng_calls, int bps, cudaStream_t st) {
  // one wave: every block resident, each walking a contiguous range of tiles;
  // bps > 0 asks for fewer blocks per SM than fit (longer tile ranges per block)
  static int occ = 0;
  if (occ == 0) {
    int o = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, lattice_half_kernel<ENC, WPT>, kTile, 0);
    occ = o > 0 ? o : 1;
  }
  const int grid = grid_for(n_tiles, bps > 0 && bps < occ ? bps : occ);
  return launch_dependent(lattice_half_kernel<ENC, WPT>, dim3(grid), dim3(kTile), 0, st, jobs,
                          tiles, n_tiles, half, rng_calls);
}

int lattice_resident_blocks() {
  int o = 1, dev = 0, sms = 152;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, lattice_half_kernel<kEncMultispin, kWordsPerThread>,
                                                kTile, 0);
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (o > 0 ? o : 1) * sms;
}

cudaError_t launch_lattice_half(int enc, int wpt, const LatJob* jobs, const Tile* tiles,
                                int n_tiles, uint32_t half, unsigned long long* rng_calls,
                                cudaStream_t st, int bps) {
  if (n_tiles <= 0) return cudaSuccess;
  if (wpt == kWordsPerThread) {
    if (enc == kEncInt8)
      return launch_half_t<kEncInt8, kWordsPerThread>(jobs, tiles, n_tiles, half, rng_calls, bps,
                                                       st);
    if (enc == kEncPacked)
      return launch_half_t<kEncPacked, kWordsPerThread>(jobs, tiles, n_tiles, half, rng_calls,
                                                         bps, st);
    return launch_half_t<kEncMultispin, kWordsPerThread>(jobs, tiles, n_tiles, half, rng_calls,
                                                         bps, st);
  }
  if (enc == kEncInt8)
    return launch_half_t<kEncInt8, 1>(jobs, tiles, n_tiles, half, rng_calls, bps, st);
  if (enc == kEncPacked)
    return launch_half_t<kEncPacked, 1>(jobs, tiles, n_tiles, half, rng_calls, bps, st);
  return launch_half_t<kEncMultispin, 1>(jobs, tiles, n_tiles, half, rng_calls, bps, st);
}

int lattice_blocks_per_sm(int wpt) {
  int o = 1;
  if (wpt == kWordsPerThread)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &o, lattice_half_kernel<kEncMultispin, kWordsPerThread>, kTile, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, lattice_half_kernel<kEncMultispin, 1>,
                                                  kTile, 0);
  return o > 0 ? o : 1;
}

cudaError_t launch_lattice_init(int enc, int wpt, const LatJob* jobs, const Tile* tiles,
                                int n_tiles, int kind, cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  const int grid = grid_for(n_tiles, 8);
  switch (enc) {
    case kEncInt8:
      lattice_init_kernel<kEncInt8><<<grid, kTile, 0, st>>>(jobs, tiles, n_tiles, kind, wpt);
      break;
    case kEncPacked:
      lattice_init_kernel<kEncPacked><<<grid, kTile, 0, st>>>(jobs, tiles, n_tiles, kind, wpt);
      break;
    default:
      lattice_init_kernel<kEncMultispin><<<grid, kTile, 0, st>>>(jobs, tiles, n_tiles, kind,
                                                                  wpt);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_lattice_obs(int enc, int wpt, const LatJob* jobs, const Tile* tiles,
                               int n_tiles, int which, int full, cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  const int grid = grid_for(n_tiles, 8);
  switch (enc) {
    case kEncInt8:
      return launch_dependent(lattice_obs_single_kernel<kEncInt8>, dim3(grid), dim3(kTile), 0,
                              st, jobs, tiles, n_tiles, which, full, wpt);
    case kEncPacked:
      return launch_dependent(lattice_obs_single_kernel<kEncPacked>, dim3(grid), dim3(kTile), 0,
                              st, jobs, tiles, n_tiles, which, full, wpt);
    default:
      return launch_dependent(lattice_obs_multispin_kernel, dim3(grid), dim3(kTile), 0, st, jobs,
                              tiles, n_tiles, which, full, wpt);
  }
}

}  // namespace shk

namespace shk {
// Grid and shared memory of the banded kernel for an L x L lattice of wpr words
// per row: as many co-resident blocks as fit (at most L, one row each at least).
// Returns false when the lattice does not fit that way.
bool lattice_band_shape(int enc, uint32_t L, uint32_t wpr, int* grid, size_t* smem) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int max_smem = 0;
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  int G = sms * kBandMinBlocks;
  for (int it = 0; it < 8; ++it) {
    if (G > (int)L) G = (int)L;
    const uint32_t rows = (L + (uint32_t)G - 1u) / (uint32_t)G + 2u;
    const size_t bytes = (size_t)2 * rows * wpr * sizeof(uint32_t);
    if (bytes > (size_t)max_smem - sizeof(LatTable) - 64) return false;
    const void* k = enc == kEncInt8 ? (const void*)lattice_band_kernel<kEncInt8>
                                    : (const void*)lattice_band_kernel<kEncPacked>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    int o = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, kTile, bytes);
    cudaGetLastError();
    if (o <= 0) return false;
    if (o * sms >= G) {
      *grid = G;
      *smem = bytes;
      return true;
    }
    G = o * sms;
  }
  return false;
}

// n steps of the one job in `jobs` by the banded kernel (cooperative launch; the
// grid and shared memory from lattice_band_shape; bs zeroed by the caller).
cudaError_t launch_lattice_band(int enc, const LatJob* jobs, int grid, size_t smem,
                                uint64_t* xch, BandSync* bs, uint32_t t0, uint32_t n_steps,
                                cudaStream_t st) {
  if (n_steps == 0) return cudaSuccess;
  void* args[] = {(void*)&jobs, (void*)&xch, (void*)&bs, (void*)&t0, (void*)&n_steps};
  const void* k = enc == kEncInt8 ? (const void*)lattice_band_kernel<kEncInt8>
                                  : (const void*)lattice_band_kernel<kEncPacked>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kTile), args, smem, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// Run n steps of every job in `jobs` (one block each) inside one launch.
cudaError_t launch_lattice_resident(int enc, const LatJob* jobs, int n_jobs, uint32_t nwords,
                                    uint32_t t0, uint32_t n_steps, cudaStream_t st) {
  if (n_jobs <= 0 || n_steps == 0) return cudaSuccess;
  const size_t bytes = (size_t)2 * nwords * sizeof(uint32_t);
  int threads = (int)(nwords < (uint32_t)kTile ? nwords : (uint32_t)kTile);
  threads = (threads + 31) / 32 * 32;
  cudaError_t e = cudaSuccess;
  if (enc == kEncInt8) {
    e = cudaFuncSetAttribute(lattice_resident_kernel<kEncInt8>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
      lattice_resident_kernel<kEncInt8><<<n_jobs, threads, bytes, st>>>(jobs, t0, n_steps);
  } else if (enc == kEncPacked) {
    e = cudaFuncSetAttribute(lattice_resident_kernel<kEncPacked>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
      lattice_resident_kernel<kEncPacked><<<n_jobs, threads, bytes, st>>>(jobs, t0, n_steps);
  } else {
    e = cudaFuncSetAttribute(lattice_resident_kernel<kEncMultispin>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
      lattice_resident_kernel<kEncMultispin><<<n_jobs, threads, bytes, st>>>(jobs, t0, n_steps);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}
}  // namespace shk
