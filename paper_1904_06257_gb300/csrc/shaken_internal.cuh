// shaken_internal.cuh -- device math and launch descriptors shared by the
// kernels and the host runtime of libshaken (sm_103a).
//
// Device math (one definition of the random stream and of the heat-bath
// decision, used by every kernel):
//   * Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): multipliers
//     0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 / 0xBB67AE85,
//     key = (seed low, seed high), counter = (a, b, t, half + 2c).
//   * exp_sd: Cody & Waite reduction x = k ln2 + r with ln2 split in a 29-bit
//     head and a tail, Taylor polynomial of e^r to degree 13 (Horner with
//     fused multiply-add), scaling by 2^k; |x| >= 64 clamps (the threshold is
//     already exactly 0 or 2^32 there).  Every operation is an explicitly
//     rounded intrinsic so the result does not depend on contraction.
//   * threshold T(h, beta) = floor(2^32 p), p = 1 / (1 + exp_sd(-2 beta h)):
//     the heat-bath probability e^{beta h} / (2 cosh(beta h)) of tau_x = +1
//     (Sec. 2, laws of P^{1->2} and P^{2->1}; Sec. 3, P^dl and P^ur), and
//     tau_x = +1 iff u < T for the 32-bit draw u.
//   * field h = (Jc * s + q * sigma) + lambda, s the integer neighbour sum.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace shk {

constexpr uint32_t kPhM0 = 0xD2511F53u;
constexpr uint32_t kPhM1 = 0xCD9E8D57u;
constexpr uint32_t kPhW0 = 0x9E3779B9u;
constexpr uint32_t kPhW1 = 0xBB67AE85u;
constexpr uint32_t kInitStep = 0xFFFFFFFFu;  // step index of the initial draw

constexpr int kTile = 256;  // threads per block; graph tiles hold kTile vertices

// ---------------------------------------------------------------- dependent launches
// The kernels of a step (half steps, observables, epilogue) are launched with
// programmatic stream serialization: a kernel may be scheduled while its
// predecessor on the stream drains, and it waits for that predecessor's completion
// and memory (griddepcontrol.wait) before it touches global memory.  Each such
// kernel also lets its own successor be scheduled as soon as all its blocks run.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... P, typename... A>
cudaError_t launch_dependent(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem,
                             cudaStream_t st, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}
constexpr int kWordsPerThread = 4;                   // lattice lane words per thread and tile
constexpr int kLatTile = kTile * kWordsPerThread;    // lattice lane words per tile
constexpr int kLatMinBlocks = 3;                     // resident blocks per SM of the half-step kernel

// ---------------------------------------------------------------- Philox-4x32-10
struct PhKey {
  uint32_t k0[10];
  uint32_t k1[10];
};

__device__ __forceinline__ PhKey ph_key(uint32_t key0, uint32_t key1) {
  PhKey K;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    K.k0[r] = key0 + (uint32_t)r * kPhW0;
    K.k1[r] = key1 + (uint32_t)r * kPhW1;
  }
  return K;
}

__device__ __forceinline__ uint4 ph_call(const PhKey& K, uint32_t c0, uint32_t c1, uint32_t c2,
                                         uint32_t c3) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = (unsigned long long)kPhM0 * c0;
    const unsigned long long p1 = (unsigned long long)kPhM1 * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ K.k0[r];
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ K.k1[r];
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
  return make_uint4(c0, c1, c2, c3);
}

// Calls whose counters share (b, t): round 0 multiplies only words 0 and 2 of the
// counter, so after it word 0 = hi(M1 t) ^ b ^ k0[0] and word 1 = lo(M1 t) do not
// depend on (a, c3), and round 1's first product M0 * word0 does not either.
// ph_call_shared(K, P, a, c3) == ph_call(K, a, b, t, c3) with P = ph_shared(K, b, t).
struct PhShared {
  uint32_t u0, u1;    // counter words 0 and 1 after round 0
  uint32_t h01, l01;  // high and low halves of M0 * u0 (round 1)
};

__device__ __forceinline__ PhShared ph_shared(const PhKey& K, uint32_t b, uint32_t t) {
  PhShared P;
  const unsigned long long p1 = (unsigned long long)kPhM1 * t;
  P.u0 = (uint32_t)(p1 >> 32) ^ b ^ K.k0[0];
  P.u1 = (uint32_t)p1;
  const unsigned long long q = (unsigned long long)kPhM0 * P.u0;
  P.h01 = (uint32_t)(q >> 32);
  P.l01 = (uint32_t)q;
  return P;
}

__device__ __forceinline__ uint4 ph_call_shared(const PhKey& K, const PhShared& P, uint32_t a,
                                                uint32_t c3) {
  // round 0: only M0 * a depends on the lane word
  const unsigned long long p0 = (unsigned long long)kPhM0 * a;
  const uint32_t c2r0 = (uint32_t)(p0 >> 32) ^ c3 ^ K.k1[0];
  const uint32_t c3r0 = (uint32_t)p0;
  // round 1: M0 * u0 is shared
  const unsigned long long p1 = (unsigned long long)kPhM1 * c2r0;
  uint32_t c0 = (uint32_t)(p1 >> 32) ^ P.u1 ^ K.k0[1];
  uint32_t c1 = (uint32_t)p1;
  uint32_t c2 = P.h01 ^ c3r0 ^ K.k1[1];
  uint32_t c3v = P.l01;
#pragma unroll
  for (int r = 2; r < 10; ++r) {
    const unsigned long long q0 = (unsigned long long)kPhM0 * c0;
    const unsigned long long q1 = (unsigned long long)kPhM1 * c2;
    const uint32_t n0 = (uint32_t)(q1 >> 32) ^ c1 ^ K.k0[r];
    const uint32_t n2 = (uint32_t)(q0 >> 32) ^ c3v ^ K.k1[r];
    c1 = (uint32_t)q1;
    c3v = (uint32_t)q0;
    c0 = n0;
    c2 = n2;
  }
  return make_uint4(c0, c1, c2, c3v);
}

// ---------------------------------------------------------------- exp and threshold
__device__ __forceinline__ double exp_sd(double x) {
  if (x <= -64.0) return 0.0;
  if (x >= 64.0) return __longlong_as_double(0x7ff0000000000000LL);
  const double inv_ln2 = 0x1.71547652b82fep+0;
  const double ln2_hi = 0x1.62e42ff000000p-1;
  const double ln2_lo = -0x1.718432a1b0e26p-35;
  const double k = rint(__dmul_rn(x, inv_ln2));
  const double r = __dsub_rn(__dsub_rn(x, __dmul_rn(k, ln2_hi)), __dmul_rn(k, ln2_lo));
  // Taylor coefficients 1/n!, n = 13 .. 0 (correctly rounded)
  double p = 0x1.6124613a86d09p-33;
  p = __fma_rn(p, r, 0x1.1eed8eff8d898p-29);
  p = __fma_rn(p, r, 0x1.ae64567f544e4p-26);
  p = __fma_rn(p, r, 0x1.27e4fb7789f5cp-22);
  p = __fma_rn(p, r, 0x1.71de3a556c734p-19);
  p = __fma_rn(p, r, 0x1.a01a01a01a01ap-16);
  p = __fma_rn(p, r, 0x1.a01a01a01a01ap-13);
  p = __fma_rn(p, r, 0x1.6c16c16c16c17p-10);
  p = __fma_rn(p, r, 0x1.1111111111111p-7);
  p = __fma_rn(p, r, 0x1.5555555555555p-5);
  p = __fma_rn(p, r, 0x1.5555555555555p-3);
  p = __fma_rn(p, r, 0x1.0000000000000p-1);
  p = __fma_rn(p, r, 1.0);
  p = __fma_rn(p, r, 1.0);
  const long long ki = (long long)k;  // |k| <= 93: 2^k is a normal double
  return __dmul_rn(p, __longlong_as_double((ki + 1023LL) << 52));
}

// T = floor(2^32 / (1 + e^{-2 beta h})) in [0, 2^32].
__device__ __forceinline__ unsigned long long threshold_T(double h, double beta) {
  const double y = __dmul_rn(beta, h);
  const double e = exp_sd(-2.0 * y);
  const double p = __ddiv_rn(1.0, __dadd_rn(1.0, e));
  return (unsigned long long)floor(__dmul_rn(p, 4294967296.0));
}

__device__ __forceinline__ double field_h(double Jc, int s, double q, int sigma, double lam) {
  return __dadd_rn(__dadd_rn(__dmul_rn(Jc, (double)s), __dmul_rn(q, (double)sigma)), lam);
}

// ---------------------------------------------------------------- lattice tables
// Per beta-set (one int8/packed replica, or one 32-replica multispin group) the
// threshold of each field class c = 2 n + s (n = number of +1 in-neighbours,
// s = 1 if sigma_x = +1) as bit planes over the 32 lanes of a lane word:
//   tm[j][c]  bit k set iff T(c, beta_k) < 2^32, T(c, beta_k) > 0 and bit (31-j)
//             of T(c, beta_k) is 1 (planes most significant first);
//   satp[c]   lanes with T == 2^32 (always +1), satm[c] lanes with T == 0.
// When the thresholds of every lane depend on n + s only (classes (0,1) and
// (1,0) equal, (1,1) and (2,0) equal -- the case J = q), tmc[j][c] holds the
// planes by c = n + s in 0..3 and `collapsed` is set; `anysat` marks tables
// with at least one saturated lane.  `mirror` (collapsed, no saturated lane):
// on planes 0..7 the fields -h take the complemented planes of +h on every lane,
// tmc[j][0] == ~tmc[j][3] and tmc[j][1] == ~tmc[j][2] (T(-h) = 2^32 - T(h) up to
// rounding, which reaches the top eight bits only when the low 24 bits of T
// are within a few units of a multiple of 2^24).
struct __align__(16) LatTable {
  uint32_t tm[32][8];
  uint32_t tmc[32][4];
  uint32_t satp[8];
  uint32_t satm[8];
  uint32_t collapsed;
  uint32_t anysat;
  uint32_t mirror;
  uint32_t pad;
};

// ---------------------------------------------------------------- descriptors
// Device-resident state of one context, read by every kernel of a step and
// advanced by the step epilogue.
struct CtxDev {
  uint32_t step;        // current step t
  uint32_t t_end;       // kernels skip this context once step >= t_end
  uint32_t anneal_t0;   // first step of the running anneal (table / schedule index base)
  uint32_t anneal_len;  // schedule length (0 = no anneal)
  uint32_t tracking;    // evaluate H(sigma_t) each step
  uint32_t record;      // write the per-step series
  uint32_t series_t0;
  uint32_t series_cap;
  uint32_t R;
  uint32_t kind;        // 0 lattice, 1 graph
  uint32_t order;       // 0: P^{1->2} then P^{2->1} (dl then ur); 1: reversed (Sec. 3, P^{sh'})
  uint32_t pad0;
  double Jc;            // energy: H = -Jc E - 2 lamc M - 2 LS
  double lamc;
  double inv_n;
  double* step_sums;    // [R][8] sums of sigma_t for tracking (zeroed by the epilogue)
  double* best;         // [R]
  long long* best_step; // [R]
  double* series_m;     // [cap][R] or null
  double* series_H;     // [cap][R] or null
};

// Grid barrier of the banded lattice kernel: arrival count, generation, and an
// error flag set by a block whose wait ran out (the launch then stops early and
// the host reports a timeout).
struct BandSync {
  unsigned int count;   // blocks arrived at the current barrier
  unsigned int gen;     // barrier generation
  unsigned int err;     // a block gave up a wait
  unsigned int commit;  // 0 undecided, 1 every block finished (write back), 2 aborted
  unsigned int hurry;   // diagnostics: block that gives up its last wait at once (~0u: none)
  unsigned int pad[3];
};

// One member of a batch for the batched state and observables copies: its state
// buffers and observables arrays and where they sit in the packed buffers.  The
// packed observables of a member are [R][kNumSums] sums, then R best energies,
// then R best steps (as the bits of a double).
struct MemberDev {
  uint32_t* A;                   // sigma
  uint32_t* B;                   // sigma'
  double* obs;                   // [R][kNumSums] observables sums
  double* best;                  // [R]
  long long* best_step;          // [R]
  unsigned long long state_off;  // first 32-bit word of its state in the packed states
  unsigned long long obs_off;    // first double of its records in the packed observables
  unsigned long long state_words;  // state size in 32-bit words
  uint32_t R;
  uint32_t pad;
};

// Sum slots of a replica (all integer valued except the real-J graph sums).
enum : int {
  kSumM = 0,   // sum sigma
  kSumE = 1,   // sum over E^o of (J) sigma_tail sigma_head (lattice: unweighted)
  kSumLS = 2,  // graph: sum lambda_x sigma_x
  kSumP1 = 3,  // sum over E^o of (J) sigma_tail sigma'_head
  kSumP2 = 4,  // sum sigma_x sigma'_x
  kSumM2 = 5,  // lattice: sum sigma'
  kSumLS2 = 6, // graph: sum lambda_x sigma'_x
  kSumCut = 7, // edges with sigma_x != sigma_y
  kNumSums = 8
};

// One lattice lane-word job: an int8/packed replica or a multispin group.
struct LatJob {
  void* A;                       // sigma buffer of this replica / group
  void* B;                       // sigma' buffer
  const uint32_t* frozen;        // frozen lane masks per lane word, or null
  const LatTable* table;         // static table of this job
  const LatTable* anneal_tables; // per-step tables (index step - anneal_t0) or null
  CtxDev* cd;
  double* sums;                  // step sums of this job's replicas (tracking), [1 or 32][8]
  double* obs;                   // on-demand observable sums of this job's replicas
  uint32_t L;
  uint32_t wpr;                  // lane words per row (L/32 or L)
  uint32_t nwords;
  uint32_t b;                    // counter word b: replica (int8/packed) or group (multispin)
  uint32_t key0, key1;
  uint32_t rep0;                 // first replica index of the job within its context
  uint32_t wpr_shift;            // log2(wpr) when wpr is a power of two, else 0xffffffff
};

// One graph job: the groups [g0, g0 + Gj) of a graph context (Gj <= kTile).  The
// context's spins are uint32 [n][G]: word x * G + g holds vertex x of replicas
// 32 g .. 32 g + 31 (bit k = replica 32 g + k), so the group words of a vertex
// are adjacent.  A half-step tile holds kTile / Gp consecutive entries of the
// vertex order of its half step (in_perm or out_perm: vertices by increasing
// degree), each with Gp threads (Gp = Gj rounded up to a power of two), thread
// g - g0 of a vertex owning word (x, g); per-group jobs (Gj = 1) serve the init,
// observables and field kernels with tiles of kTile vertices in index order.
struct GraphJob {
  uint32_t* A;             // sigma, [n][G]
  uint32_t* B;             // sigma', [n][G]
  const int32_t* in_ptr;   // in-CSR (sources y of (y -> x) in E^o)
  const uint32_t* in_col;  // bit 31: J < 0 (integer couplings)
  const float* in_J;       // real couplings (null for integer)
  const int32_t* out_ptr;  // out-CSR (heads y of (x -> y))
  const uint32_t* out_col;
  const float* out_J;
  const uint4* in_visit;   // half-step order h^{1->2} (vertices by increasing in-degree):
                           // (x, first in-edge, in-degree, lambda_x bits) per slot
  const uint4* out_visit;  // the same for h^{2->1} (out-edges, out-degree)
  const float* lambda;     // [n] or null (lambda_c)
  const uint32_t* frozen;  // [n] lane masks or null
  const double* beta_lane; // [R] betas of the context
  const double* beta_sched;// anneal schedule (index step - anneal_t0) or null
  CtxDev* cd;
  double* sums;            // [R][8] step sums of the context's replicas (tracking)
  double* obs;             // [R][8] on-demand observable sums
  double q;
  float lambda_c;
  uint32_t n;
  uint32_t G;              // groups of the context (words per vertex)
  uint32_t g0;             // first group of this job
  uint32_t Gj;             // groups of this job
  uint32_t Gp;             // threads per vertex in half-step tiles (power of two >= Gj)
  uint32_t key0, key1;
  uint32_t integer;
};

// Column counts of the warp's 32 words: lane k gets the number of lanes whose word
// has bit k set.  Five butterfly exchanges transpose the 32 x 32 bit block (at the
// exchange of distance j, the lanes with bit j clear take the partner's low-column
// half into their high columns and the others the reverse), so lane k then holds
// column k, and a popcount finishes.
__device__ __forceinline__ int warp_column_count(uint32_t x, int lane) {
  const uint32_t Hm[5] = {0xFFFF0000u, 0xFF00FF00u, 0xF0F0F0F0u, 0xCCCCCCCCu, 0xAAAAAAAAu};
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int j = 16 >> i;
    const uint32_t p = __shfl_xor_sync(0xffffffffu, x, j);
    const bool hi = (lane & j) != 0;
    const uint32_t t = hi ? (p >> j) : (p << j);
    const uint32_t M = hi ? ~Hm[i] : Hm[i];
    x = (x & ~M) | (t & M);
  }
  return __popc(x);
}

struct Tile {
  uint32_t job;
  uint32_t w0;
};

// Vertices of degree above kHubDeg in a half step's direction are not decided by the
// half-step kernel: their edge lists are cut into chunks of kHubChunk edges, one warp
// per (chunk, group) sums the chunk's 32 per-replica fields, and the warp that
// finishes a vertex word last adds the chunk sums in chunk order and decides it.
constexpr uint32_t kHubDeg = 255;
constexpr uint32_t kHubChunk = 2048;

struct HubItem {
  uint32_t job;      // half-step job (index in the family's jobs)
  uint32_t x;        // the vertex
  uint32_t e0, e1;   // the chunk's edges [e0, e1) in the direction's CSR
  uint32_t chunk;    // index of the chunk among the vertex's
  uint32_t nchunks;  // chunks of the vertex
  uint32_t pbase;    // partial rows of the vertex: pbase + go * nchunks + chunk (32 words each)
  uint32_t dbase;    // finished-chunk counters of the vertex: dbase + go
  uint32_t dir;      // 0: in-edges (update type 0), 1: out-edges (type 1)
  uint32_t ubase;    // its warps (units) ubase + go for the job's groups go < Gj
};

}  // namespace shk
