// runtime.cu -- host runtime of libshaken: the C ABI declared in include/shaken.h.
//
// A context owns one problem (lattice or graph), its double-buffered device
// state, the threshold tables, the oriented in/out CSR of a graph (Sec. 2:
// E^o from an orientation rule; in-neighbours feed h^{1->2}, out-neighbours
// h^{2->1}) and a launch plan.  A plan holds the device job and tile lists of
// a set of contexts (one context alone, or the members of a batch); one step
// of a plan is
//   [tracking sums of multispin / graph members] -> half 0 (one launch per
//   encoding family) -> half 1 -> epilogue (best energy, series, t += 1).
// The step counter of each context lives on the device (CtxDev), so a chunk
// of steps can be captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/shaken.h"
#include "shaken_internal.cuh"

namespace shk {
cudaError_t launch_build_lattice_tables(const double*, int, double, double, double, LatTable*,
                                        cudaStream_t);
int lattice_blocks_per_sm(int);
cudaError_t launch_lattice_half(int, int, const LatJob*, const Tile*, int, uint32_t,
                                unsigned long long*, cudaStream_t, int);
int lattice_resident_blocks();
cudaError_t run_microbench(int, double*, double*);
cudaError_t launch_lattice_init(int, int, const LatJob*, const Tile*, int, int, cudaStream_t);
cudaError_t launch_lattice_obs(int, int, const LatJob*, const Tile*, int, int, int, cudaStream_t);
cudaError_t launch_graph_half(bool, const GraphJob*, const Tile*, int, uint32_t, int, int,
                              cudaStream_t);
cudaError_t launch_graph_hub(bool, const GraphJob*, const HubItem*, const uint32_t*, int, uint32_t,
                             uint32_t*, uint32_t*, cudaStream_t);
cudaError_t launch_graph_init(const GraphJob*, const Tile*, int, int, cudaStream_t);
cudaError_t launch_graph_obs(bool, const GraphJob*, const Tile*, int, int, int, cudaStream_t);
cudaError_t launch_graph_fields(const GraphJob*, const Tile*, int, uint32_t, float*,
                                cudaStream_t);
cudaError_t launch_epilogue(CtxDev* const*, int, cudaStream_t);
cudaError_t launch_member_copy(int, const shk::MemberDev*, int, void*, unsigned long long,
                               cudaStream_t);
bool lattice_band_shape(int, uint32_t, uint32_t, int*, size_t*);
cudaError_t launch_lattice_band(int, const LatJob*, int, size_t, uint64_t*, BandSync*, uint32_t,
                                uint32_t, cudaStream_t);
cudaError_t launch_lattice_resident(int, const LatJob*, int, uint32_t, uint32_t, uint32_t,
                                    cudaStream_t);
cudaError_t launch_philox(uint64_t, const uint32_t*, uint32_t*, int64_t, cudaStream_t);
cudaError_t launch_threshold(const double*, const double*, uint64_t*, int64_t, cudaStream_t);
}  // namespace shk

using shk::CtxDev;
using shk::GraphJob;
using shk::HubItem;
using shk::LatJob;
using shk::LatTable;
using shk::Tile;
using shk::kNumSums;
using shk::kTile;

// ============================================================================ errors
static thread_local std::string g_last_error;

static shaken_status fail(shaken_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

void shaken_internal_set_error(const char* msg) { g_last_error = msg; }

#define CU(call)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      cudaGetLastError();                                                           \
      return fail(e_ == cudaErrorMemoryAllocation ? SHAKEN_E_NOMEM : SHAKEN_E_CUDA, \
                  std::string(#call) + ": " + cudaGetErrorString(e_));              \
    }                                                                               \
  } while (0)

#define TRY(expr)                   \
  do {                              \
    shaken_status s_ = (expr);      \
    if (s_ != SHAKEN_OK) return s_; \
  } while (0)

// ============================================================================ device memory
struct DevMem {
  void* p = nullptr;
  size_t bytes = 0;
  DevMem() = default;
  DevMem(const DevMem&) = delete;
  DevMem& operator=(const DevMem&) = delete;
  ~DevMem() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  shaken_status alloc(size_t n) {
    release();
    if (n == 0) n = 16;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      return fail(SHAKEN_E_NOMEM,
                  "cudaMalloc(" + std::to_string(n) + "): " + cudaGetErrorString(e));
    }
    bytes = n;
    return SHAKEN_OK;
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

static shaken_status upload(DevMem& d, const void* src, size_t n, cudaStream_t st) {
  if (d.p == nullptr || d.bytes < n) TRY(d.alloc(n));
  if (n) CU(cudaMemcpyAsync(d.p, src, n, cudaMemcpyHostToDevice, st));
  return SHAKEN_OK;
}

// ============================================================================ plan
struct Family {
  int kind = 0;  // 0 lattice, 1 graph
  int enc = 0;   // lattice encoding; graph: 1 integer couplings, 0 real
  int wpt = 1;   // lattice: lane words per thread per tile (tile = 256 wpt words)
  int bps = 0;   // lattice: resident blocks per SM of the half step (0: as many as fit)
  DevMem jobs, tiles;  // graph: multi-group jobs and (vertex, group) pair tiles (half steps)
  int n_tiles = 0;
  DevMem ojobs, otiles;  // graph: one job per group and vertex tiles (init, observables)
  int n_otiles = 0;
  // graph: chunks of the edge lists of vertices of degree above kHubDeg, one warp per
  // (chunk, group) unit; partial rows and finished-chunk counters of their words
  DevMem hub_items, hub_units, hub_partial, hub_done;
  int n_hub_units = 0;
};

struct Plan {
  std::vector<shaken_ctx*> members;
  std::vector<std::unique_ptr<Family>> fams;
  DevMem ctxlist;
  int n_ctx = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int graph_steps = 0;
  uint64_t graph_launches = 0;
  bool dirty = true;
  bool autotune = true;  // pick the lattice tile shape by timing trial launches
  int pinned[3][2] = {{0, 0}, {0, 0}, {0, 0}};  // per lattice encoding: (wpt, bps) set by the caller
  int blocks_per_sm = 8;
  int timing = 0;           // bracket the half-step launches of every timing-th step (0: off)
  uint64_t steps_issued = 0;  // non-graph steps launched (for the timing stride)
  unsigned long long* rng_counter = nullptr;  // device counter of Philox calls (lattice), or null
  std::vector<cudaEvent_t> ev_free;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
  double timed_ms = 0.0;
  uint64_t timed_n = 0;
  // batched state / observables copies (built on first use, dropped with the plan)
  bool mtab_valid = false;
  DevMem mtab;                 // MemberDev per member
  size_t state_words = 0;      // packed states, 32-bit words
  size_t obs_doubles = 0;      // packed observables, doubles
  unsigned long long max_state_words = 0, max_obs = 0;
  DevMem stage_state, stage_obs;
  ~Plan() {
    drop_graph();
    for (auto& pr : ev_pending) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    for (cudaEvent_t e : ev_free) cudaEventDestroy(e);
  }
  cudaEvent_t get_event() {
    if (!ev_free.empty()) {
      cudaEvent_t e = ev_free.back();
      ev_free.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void collect() {
    for (auto& pr : ev_pending) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) {
        timed_ms += ms;
        timed_n++;
      }
      ev_free.push_back(pr.first);
      ev_free.push_back(pr.second);
    }
    ev_pending.clear();
  }
  void drop_graph() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    gexec = nullptr;
    graph = nullptr;
    graph_steps = 0;
  }
  void invalidate() {
    dirty = true;
    mtab_valid = false;
    drop_graph();
  }
};

// ============================================================================ context
struct shaken_ctx {
  int kind = 0, enc = 0;
  int64_t L = 0, n = 0, m = 0;
  int R = 0;
  double J = 0, q = 0, lam_c = 0;
  bool has_lambda = false, integer = false;
  std::vector<float> lambda;
  std::vector<uint8_t> frozen;  // [n], empty = none
  std::vector<double> beta;     // [R]
  double sumJ = 0.0;            // sum of couplings over E (cut weight)
  uint64_t seed = 0;
  cudaStream_t stream = nullptr;
  DevMem A, B;
  size_t spin_bytes = 0;
  DevMem frozen_lanes;
  DevMem tables, beta_lanes;
  DevMem anneal_tables, anneal_sched, anneal_lanes;
  DevMem cd;
  DevMem step_sums, obs_sums, best, best_step;
  DevMem series_m, series_H;
  DevMem in_ptr, in_col, in_J, out_ptr, out_col, out_J, lam_dev;
  DevMem in_visit, out_visit;  // half-step visiting order: (x, first edge, degree, lambda_x)
  std::vector<uint32_t> hubs[2];  // graph: (x, first edge, end edge) of the vertices of degree
                                  // above kHubDeg, in-CSR [0] and out-CSR [1]
  DevMem band_xch, band_sync;  // banded runs: row exchange area and grid barrier
  bool band_stall = false;     // diagnostics: the next banded run's barrier never completes
  int band_hurry = -1;         // diagnostics: block that gives up the next run's last wait at once
  CtxDev hcd{};
  uint64_t host_step = 0;
  bool tracking = false;
  shaken_batch* owner = nullptr;
  Plan solo;
  std::atomic<uint64_t> launches{0};
  int exact_always = 0;

  int64_t sites() const { return kind == SHAKEN_LATTICE ? L * L : n; }
};

struct shaken_batch {
  cudaStream_t stream = nullptr;
  Plan plan;
  std::atomic<uint64_t> launches{0};
};

static cudaStream_t ctx_stream(const shaken_ctx* c) {
  return c->owner ? c->owner->stream : c->stream;
}

static void add_tiles(std::vector<Tile>& tiles, uint32_t job, uint64_t count, uint32_t size) {
  for (uint64_t w = 0; w < count; w += size) tiles.push_back(Tile{job, (uint32_t)w});
}

// Graph half-step tiles of one job, vertices in degree order: the tiles are listed in
// the order k -> (k * s) mod N with s coprime to N near N (sqrt 5 - 1) / 2, so the
// heavy tiles (the highest degrees, at the end of the order) spread evenly over the
// contiguous tile ranges the blocks take instead of all falling to the last blocks.
static void add_graph_tiles(std::vector<Tile>& tiles, uint32_t job, uint64_t count,
                            uint32_t size) {
  const uint64_t N = (count + size - 1) / size;
  if (N == 0) return;
  uint64_t st = (uint64_t)((double)N * 0.6180339887498949);
  if (st == 0) st = 1;
  auto gcd = [](uint64_t a, uint64_t b) {
    while (b != 0) {
      const uint64_t t = a % b;
      a = b;
      b = t;
    }
    return a;
  };
  while (gcd(st, N) != 1) ++st;
  uint64_t pos = 0;
  for (uint64_t k = 0; k < N; ++k, pos = (pos + st) % N)
    tiles.push_back(Tile{job, (uint32_t)(pos * size)});
}

static void lattice_tiles(const std::vector<LatJob>& jobs, uint32_t size,
                          std::vector<Tile>& out) {
  out.clear();
  for (size_t j = 0; j < jobs.size(); ++j) add_tiles(out, (uint32_t)j, jobs[j].nwords, size);
}

// ============================================================================ autotuner
// Launch shape of the lattice half-step kernel per encoding family: tiles of
// kTile lane words (one per thread) or kLatTile (kWordsPerThread per thread).
// The choice is made by timing: each candidate runs the position-0 half step of
// the family on a copy of its job table without step sums (no fused tracking)
// and without the Philox counter.  Such a launch only writes sigma', with the
// values the real position-0 half step of the same step writes (the draws are
// counter-based), so the trials leave no trace in any trajectory.  Results are
// cached per (encoding, bit length of the lane-word count, bit length of the
// job count).  Families smaller than one resident wave of kLatTile tiles take
// one lane word per thread without trials.
namespace {
struct TuneKey {
  int enc, lw, lj;
  bool operator<(const TuneKey& o) const {
    if (enc != o.enc) return enc < o.enc;
    if (lw != o.lw) return lw < o.lw;
    return lj < o.lj;
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune;  // -> (words per thread, blocks per SM)
std::atomic<uint64_t> g_tune_trials{0};

int bit_length(uint64_t x) {
  int b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};
}  // namespace

// Mean device time (ms) of one position-0 half-step launch with tiles of kTile * wpt
// lane words and bps blocks per SM: 3 timed launches after one warm-up.
static shaken_status trial_lattice(int enc, int wpt, int bps, const DevMem& jobs_dev,
                                   const std::vector<LatJob>& jobs, cudaStream_t st, float* ms) {
  std::vector<Tile> tiles;
  lattice_tiles(jobs, (uint32_t)(kTile * wpt), tiles);
  DevMem td;
  TRY(upload(td, tiles.data(), tiles.size() * sizeof(Tile), st));
  EventPair ev;
  CU(cudaEventCreate(&ev.a));
  CU(cudaEventCreate(&ev.b));
  const int nt = (int)tiles.size();
  CU(shk::launch_lattice_half(enc, wpt, jobs_dev.as<LatJob>(), td.as<Tile>(), nt, 0u, nullptr, st,
                              bps));
  CU(cudaEventRecord(ev.a, st));
  for (int r = 0; r < 3; ++r)
    CU(shk::launch_lattice_half(enc, wpt, jobs_dev.as<LatJob>(), td.as<Tile>(), nt, 0u, nullptr,
                                st, bps));
  CU(cudaEventRecord(ev.b, st));
  CU(cudaEventSynchronize(ev.b));
  float t = 0.0f;
  CU(cudaEventElapsedTime(&t, ev.a, ev.b));
  *ms = t / 3.0f;
  return SHAKEN_OK;
}

// Launch shape of a lattice family: lane words per thread (1 or kWordsPerThread) and
// resident blocks per SM of the half step (every block that fits, or one fewer, so
// that each block walks a longer range of tiles).  A shape is {wpt, bps}, bps = 0
// meaning as many as fit.
struct LatShape {
  int wpt = 1, bps = 0;
};

static shaken_status choose_lattice_shape(const Plan& P, int enc, const std::vector<LatJob>& jobs,
                                          cudaStream_t st, LatShape* out) {
  if (P.pinned[enc][0] != 0) {  // a shape pinned by the caller
    out->wpt = P.pinned[enc][0];
    out->bps = P.pinned[enc][1];
    return SHAKEN_OK;
  }
  uint64_t words = 0;
  for (const LatJob& J : jobs) words += J.nwords;
  const uint64_t wave = (uint64_t)shk::lattice_resident_blocks();
  const uint64_t big_tiles = words / (uint64_t)shk::kLatTile;
  *out = LatShape{};
  if (big_tiles < wave) return SHAKEN_OK;  // not one wave of large tiles: one word per thread
  if (!P.autotune) {  // fixed rule: large tiles once the family fills 8 waves
    out->wpt = big_tiles >= 8 * wave ? shk::kWordsPerThread : 1;
    return SHAKEN_OK;
  }
  const TuneKey key{enc, bit_length(words), bit_length(jobs.size())};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      out->wpt = it->second.first;
      out->bps = it->second.second;
      return SHAKEN_OK;
    }
  }
  std::vector<LatJob> trial(jobs);
  for (LatJob& J : trial) J.sums = nullptr;
  DevMem jd;
  TRY(upload(jd, trial.data(), trial.size() * sizeof(LatJob), st));
  float best = 0.0f;
  bool first = true;
  for (int wpt : {1, shk::kWordsPerThread}) {
    const int occ = shk::lattice_blocks_per_sm(wpt);
    for (int bps : {0, occ - 1}) {
      if (bps < 0 || (bps == occ - 1 && occ <= 1)) continue;
      float ms = 0.0f;
      TRY(trial_lattice(enc, wpt, bps, jd, trial, st, &ms));
      if (first || ms < best) {
        best = ms;
        out->wpt = wpt;
        out->bps = bps;
        first = false;
      }
    }
  }
  g_tune_trials.fetch_add(1);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = {out->wpt, out->bps};
  return SHAKEN_OK;
}

static shaken_status build_plan(Plan& P, cudaStream_t st) {
  P.fams.clear();
  P.drop_graph();
  std::vector<std::vector<LatJob>> ljobs(3);
  std::vector<std::vector<GraphJob>> gjobs(2);  // 0 integer, 1 real: half-step jobs
  std::vector<std::vector<GraphJob>> ojobs(2);  // per-group jobs
  std::vector<std::vector<Tile>> otiles(2);
  std::vector<std::vector<Tile>> tiles(5);
  std::vector<std::vector<HubItem>> hitems(2);    // per graph family: hub chunks
  std::vector<std::vector<uint32_t>> hunits(2);   // unit -> item
  std::vector<uint32_t> hrows(2, 0u), hdone(2, 0u);
  std::vector<CtxDev*> cds;
  for (shaken_ctx* c : P.members) {
    CtxDev* cdp = c->cd.as<CtxDev>();
    cds.push_back(cdp);
    const uint32_t key0 = (uint32_t)(c->seed & 0xffffffffu), key1 = (uint32_t)(c->seed >> 32);
    if (c->kind == SHAKEN_LATTICE) {
      const int e = c->enc;
      const bool multi = e == SHAKEN_MULTISPIN;
      const int njobs = multi ? c->R / 32 : c->R;
      const uint32_t L = (uint32_t)c->L;
      const uint32_t wpr = multi ? L : L / 32u;
      const uint32_t nwords = L * wpr;
      const size_t job_bytes = c->spin_bytes / (size_t)njobs;
      for (int j = 0; j < njobs; ++j) {
        LatJob J{};
        J.A = c->A.as<uint8_t>() + job_bytes * j;
        J.B = c->B.as<uint8_t>() + job_bytes * j;
        J.frozen = c->frozen_lanes.p ? c->frozen_lanes.as<uint32_t>() : nullptr;
        J.table = c->tables.as<LatTable>() + j;
        J.anneal_tables = c->anneal_tables.p ? c->anneal_tables.as<LatTable>() : nullptr;
        J.cd = cdp;
        const int rep0 = multi ? 32 * j : j;
        J.sums = c->step_sums.as<double>() + (size_t)rep0 * kNumSums;
        J.obs = c->obs_sums.as<double>() + (size_t)rep0 * kNumSums;
        J.L = L;
        J.wpr = wpr;
        J.nwords = nwords;
        J.b = (uint32_t)j;
        J.key0 = key0;
        J.key1 = key1;
        J.rep0 = (uint32_t)rep0;
        J.wpr_shift = 0xffffffffu;
        for (uint32_t sh = 0; sh < 32; ++sh)
          if ((1u << sh) == wpr) J.wpr_shift = sh;
        ljobs[e].push_back(J);
      }
    } else {
      const int fi = c->integer ? 0 : 1;
      const uint32_t ng = (uint32_t)(c->R / 32);
      GraphJob J{};
      J.A = c->A.as<uint32_t>();
      J.B = c->B.as<uint32_t>();
      J.in_ptr = c->in_ptr.as<int32_t>();
      J.in_col = c->in_col.as<uint32_t>();
      J.in_J = c->integer ? nullptr : c->in_J.as<float>();
      J.out_ptr = c->out_ptr.as<int32_t>();
      J.out_col = c->out_col.as<uint32_t>();
      J.out_J = c->integer ? nullptr : c->out_J.as<float>();
      J.in_visit = c->in_visit.as<uint4>();
      J.out_visit = c->out_visit.as<uint4>();
      J.lambda = c->has_lambda ? c->lam_dev.as<float>() : nullptr;
      J.frozen = c->frozen_lanes.p ? c->frozen_lanes.as<uint32_t>() : nullptr;
      J.beta_lane = c->beta_lanes.as<double>();
      J.beta_sched = c->anneal_sched.p ? c->anneal_sched.as<double>() : nullptr;
      J.cd = cdp;
      J.sums = c->step_sums.as<double>();
      J.obs = c->obs_sums.as<double>();
      J.q = c->q;
      J.lambda_c = (float)c->lam_c;
      J.n = (uint32_t)c->n;
      J.G = ng;
      J.key0 = key0;
      J.key1 = key1;
      J.integer = c->integer ? 1u : 0u;
      // half steps: jobs of at most kTile groups; a vertex takes Gp threads (Gj rounded
      // up to a power of two) and a tile kTile / Gp vertices
      for (uint32_t g0 = 0; g0 < ng; g0 += (uint32_t)kTile) {
        GraphJob H = J;
        H.g0 = g0;
        H.Gj = std::min<uint32_t>((uint32_t)kTile, ng - g0);
        H.Gp = 1;
        while (H.Gp < H.Gj) H.Gp <<= 1;
        add_graph_tiles(tiles[3 + fi], (uint32_t)gjobs[fi].size(), (uint64_t)c->n,
                        (uint32_t)kTile / H.Gp);
        for (uint32_t dir = 0; dir < 2; ++dir) {
          const std::vector<uint32_t>& hv = c->hubs[dir];
          for (size_t k = 0; k + 2 < hv.size(); k += 3) {
            const uint32_t e0 = hv[k + 1], e1 = hv[k + 2];
            const uint32_t nch = (e1 - e0 + shk::kHubChunk - 1u) / shk::kHubChunk;
            for (uint32_t ch = 0; ch < nch; ++ch) {
              HubItem it{};
              it.job = (uint32_t)gjobs[fi].size();
              it.x = hv[k];
              it.e0 = e0 + ch * shk::kHubChunk;
              it.e1 = std::min(e1, it.e0 + shk::kHubChunk);
              it.chunk = ch;
              it.nchunks = nch;
              it.pbase = hrows[fi];
              it.dbase = hdone[fi];
              it.dir = dir;
              it.ubase = (uint32_t)hunits[fi].size();
              for (uint32_t go = 0; go < H.Gj; ++go)
                hunits[fi].push_back((uint32_t)hitems[fi].size());
              hitems[fi].push_back(it);
            }
            hrows[fi] += nch * H.Gj;
            hdone[fi] += H.Gj;
          }
        }
        gjobs[fi].push_back(H);
      }
      // init, observables, fields: one job per group, tiles of kTile vertices
      for (uint32_t g = 0; g < ng; ++g) {
        GraphJob O = J;
        O.g0 = g;
        O.Gj = 1;
        add_tiles(otiles[fi], (uint32_t)ojobs[fi].size(), (uint64_t)c->n, (uint32_t)kTile);
        ojobs[fi].push_back(O);
      }
    }
  }
  LatShape lat_shape[3];
  for (int e = 0; e < 3; ++e) {
    if (ljobs[e].empty()) continue;
    TRY(choose_lattice_shape(P, e, ljobs[e], st, &lat_shape[e]));
    lattice_tiles(ljobs[e], (uint32_t)(kTile * lat_shape[e].wpt), tiles[e]);
  }
  for (int e = 0; e < 3; ++e) {
    if (ljobs[e].empty()) continue;
    auto F = std::make_unique<Family>();
    F->kind = 0;
    F->enc = e;
    F->wpt = lat_shape[e].wpt;
    F->bps = lat_shape[e].bps;
    TRY(upload(F->jobs, ljobs[e].data(), ljobs[e].size() * sizeof(LatJob), st));
    TRY(upload(F->tiles, tiles[e].data(), tiles[e].size() * sizeof(Tile), st));
    F->n_tiles = (int)tiles[e].size();
    P.fams.push_back(std::move(F));
  }
  for (int fi = 0; fi < 2; ++fi) {
    if (gjobs[fi].empty()) continue;
    auto F = std::make_unique<Family>();
    F->kind = 1;
    F->enc = fi == 0 ? 1 : 0;
    TRY(upload(F->jobs, gjobs[fi].data(), gjobs[fi].size() * sizeof(GraphJob), st));
    TRY(upload(F->tiles, tiles[3 + fi].data(), tiles[3 + fi].size() * sizeof(Tile), st));
    F->n_tiles = (int)tiles[3 + fi].size();
    TRY(upload(F->ojobs, ojobs[fi].data(), ojobs[fi].size() * sizeof(GraphJob), st));
    TRY(upload(F->otiles, otiles[fi].data(), otiles[fi].size() * sizeof(Tile), st));
    F->n_otiles = (int)otiles[fi].size();
    if (!hunits[fi].empty()) {
      TRY(upload(F->hub_items, hitems[fi].data(), hitems[fi].size() * sizeof(HubItem), st));
      TRY(upload(F->hub_units, hunits[fi].data(), hunits[fi].size() * 4, st));
      TRY(F->hub_partial.alloc((size_t)hrows[fi] * 32u * 4u));
      TRY(F->hub_done.alloc((size_t)hdone[fi] * 4u));
      CU(cudaMemsetAsync(F->hub_done.p, 0, (size_t)hdone[fi] * 4u, st));
      F->n_hub_units = (int)hunits[fi].size();
    }
    P.fams.push_back(std::move(F));
  }
  TRY(upload(P.ctxlist, cds.data(), cds.size() * sizeof(CtxDev*), st));
  P.n_ctx = (int)cds.size();
  P.dirty = false;
  return SHAKEN_OK;
}

static shaken_status plan_step_launch(Plan& P, cudaStream_t st, uint64_t* nl,
                                      bool capturing = false) {
  uint64_t count = 0;
  const bool timed = P.timing > 0 && !capturing && P.steps_issued % (uint64_t)P.timing == 0;
  if (!capturing) ++P.steps_issued;
  bool obs_needed = false;
  int ex = 0;
  for (shaken_ctx* c : P.members) {
    // multispin lattices track with the observables kernel; graphs fuse tracking
    // into half 0 unless a per-step series (which also needs M) is recorded
    if (c->hcd.tracking && c->kind == SHAKEN_LATTICE && c->enc == SHAKEN_MULTISPIN)
      obs_needed = true;
    if (c->hcd.tracking && c->kind == SHAKEN_GRAPH && c->hcd.record) obs_needed = true;
    ex |= c->exact_always;
  }
  if (obs_needed) {
    for (auto& F : P.fams) {
      if (F->kind == 0 && F->enc == SHAKEN_MULTISPIN) {
        CU(shk::launch_lattice_obs(F->enc, F->wpt, F->jobs.as<LatJob>(), F->tiles.as<Tile>(),
                                   F->n_tiles, 0, 0, st));
        ++count;
      } else if (F->kind == 1) {
        CU(shk::launch_graph_obs(F->enc != 0, F->ojobs.as<GraphJob>(), F->otiles.as<Tile>(),
                                 F->n_otiles, 0, 0, st));
        ++count;
      }
    }
  }
  for (uint32_t half = 0; half < 2; ++half) {
    for (auto& F : P.fams) {
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (timed) {
        e0 = P.get_event();
        e1 = P.get_event();
        CU(cudaEventRecord(e0, st));
      }
      if (F->kind == 0)
        CU(shk::launch_lattice_half(F->enc, F->wpt, F->jobs.as<LatJob>(), F->tiles.as<Tile>(),
                                    F->n_tiles, half, P.rng_counter, st, F->bps));
      else
        CU(shk::launch_graph_half(F->enc != 0, F->jobs.as<GraphJob>(), F->tiles.as<Tile>(),
                                  F->n_tiles, half, ex, P.blocks_per_sm, st));
      ++count;
      if (F->kind == 1 && F->n_hub_units > 0) {
        CU(shk::launch_graph_hub(F->enc != 0, F->jobs.as<GraphJob>(), F->hub_items.as<HubItem>(),
                                 F->hub_units.as<uint32_t>(), F->n_hub_units, half,
                                 F->hub_partial.as<uint32_t>(), F->hub_done.as<uint32_t>(), st));
        ++count;
      }
      if (timed) {
        CU(cudaEventRecord(e1, st));
        P.ev_pending.emplace_back(e0, e1);
      }
    }
  }
  CU(shk::launch_epilogue(P.ctxlist.as<CtxDev*>(), P.n_ctx, st));
  ++count;
  *nl += count;
  return SHAKEN_OK;
}

static constexpr int kGraphChunk = 32;

static shaken_status plan_run(Plan& P, cudaStream_t st, uint64_t n_steps, bool use_graph,
                              uint64_t* nl) {
  if (P.dirty) TRY(build_plan(P, st));
  uint64_t done = 0;
  if (use_graph && n_steps >= (uint64_t)kGraphChunk) {
    if (!P.gexec) {
      cudaStream_t cap = nullptr;
      CU(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) {
        cudaStreamDestroy(cap);
        cudaGetLastError();
        return fail(SHAKEN_E_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
      }
      uint64_t cnt = 0;
      shaken_status s = SHAKEN_OK;
      for (int k = 0; k < kGraphChunk && s == SHAKEN_OK; ++k)
        s = plan_step_launch(P, cap, &cnt, true);
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(cap, &g);
      cudaStreamDestroy(cap);
      if (s != SHAKEN_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
      }
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SHAKEN_E_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
      }
      e = cudaGraphInstantiate(&P.gexec, g, 0);
      if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(SHAKEN_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
      }
      P.graph = g;
      P.graph_steps = kGraphChunk;
      P.graph_launches = cnt;
    }
    while (n_steps - done >= (uint64_t)P.graph_steps) {
      CU(cudaGraphLaunch(P.gexec, st));
      *nl += P.graph_launches;
      done += (uint64_t)P.graph_steps;
    }
  }
  for (; done < n_steps; ++done) TRY(plan_step_launch(P, st, nl));
  return SHAKEN_OK;
}

// ============================================================================ helpers
static shaken_status push_cd(shaken_ctx* c) {
  c->hcd.step = (uint32_t)c->host_step;
  CU(cudaMemcpyAsync(c->cd.p, &c->hcd, sizeof(CtxDev), cudaMemcpyHostToDevice, ctx_stream(c)));
  CU(cudaStreamSynchronize(ctx_stream(c)));
  return SHAKEN_OK;
}

static bool is_finite_d(double x) { return std::isfinite(x); }

static shaken_status build_tables_for_betas(shaken_ctx* c, const std::vector<double>& lanes,
                                            DevMem& dst_tables, DevMem& dst_lanes, int ntab,
                                            cudaStream_t st) {
  TRY(upload(dst_lanes, lanes.data(), lanes.size() * sizeof(double), st));
  if (dst_tables.p == nullptr || dst_tables.bytes < (size_t)ntab * sizeof(LatTable))
    TRY(dst_tables.alloc((size_t)ntab * sizeof(LatTable)));
  CU(shk::launch_build_lattice_tables(dst_lanes.as<double>(), ntab, c->J, c->q, c->lam_c,
                                      dst_tables.as<LatTable>(), st));
  c->launches++;
  return SHAKEN_OK;
}

// Expand per-replica betas to the lanes of each table (lattice).
static std::vector<double> lattice_table_lanes(const shaken_ctx* c) {
  std::vector<double> lanes;
  if (c->enc == SHAKEN_MULTISPIN) {
    lanes.assign(c->beta.begin(), c->beta.end());
  } else {
    lanes.resize((size_t)c->R * 32);
    for (int r = 0; r < c->R; ++r)
      for (int k = 0; k < 32; ++k) lanes[(size_t)r * 32 + k] = c->beta[r];
  }
  return lanes;
}

static int lattice_ntab(const shaken_ctx* c) {
  return c->enc == SHAKEN_MULTISPIN ? c->R / 32 : c->R;
}

// host spins [R][n] int8 <-> device encoding
static void encode_spins(const shaken_ctx* c, const int8_t* in, std::vector<uint8_t>& out) {
  const int64_t N = c->sites();
  out.assign(c->spin_bytes, 0);
  if (c->kind == SHAKEN_LATTICE && c->enc == SHAKEN_INT8) {
    std::memcpy(out.data(), in, (size_t)c->R * N);
    return;
  }
  uint32_t* w = reinterpret_cast<uint32_t*>(out.data());
  if (c->kind == SHAKEN_LATTICE && c->enc == SHAKEN_PACKED) {
    const int64_t words = N / 32;
    for (int r = 0; r < c->R; ++r)
      for (int64_t x = 0; x < N; ++x)
        if (in[(size_t)r * N + x] > 0) w[(size_t)r * words + (x >> 5)] |= 1u << (x & 31);
    return;
  }
  const int G = c->R / 32;
  const bool vmajor = c->kind == SHAKEN_GRAPH;  // graphs: [n][G]; lattices: [G][L][L]
  for (int r = 0; r < c->R; ++r) {
    const int g = r >> 5, k = r & 31;
    for (int64_t x = 0; x < N; ++x)
      if (in[(size_t)r * N + x] > 0) w[vmajor ? (size_t)x * G + g : (size_t)g * N + x] |= 1u << k;
  }
}

static void decode_spins(const shaken_ctx* c, const std::vector<uint8_t>& in, int8_t* out) {
  const int64_t N = c->sites();
  if (c->kind == SHAKEN_LATTICE && c->enc == SHAKEN_INT8) {
    std::memcpy(out, in.data(), (size_t)c->R * N);
    return;
  }
  const uint32_t* w = reinterpret_cast<const uint32_t*>(in.data());
  if (c->kind == SHAKEN_LATTICE && c->enc == SHAKEN_PACKED) {
    const int64_t words = N / 32;
    for (int r = 0; r < c->R; ++r)
      for (int64_t x = 0; x < N; ++x)
        out[(size_t)r * N + x] = (w[(size_t)r * words + (x >> 5)] >> (x & 31)) & 1u ? 1 : -1;
    return;
  }
  const int G = c->R / 32;
  const bool vmajor = c->kind == SHAKEN_GRAPH;
  for (int r = 0; r < c->R; ++r) {
    const int g = r >> 5, k = r & 31;
    for (int64_t x = 0; x < N; ++x)
      out[(size_t)r * N + x] =
          (w[vmajor ? (size_t)x * G + g : (size_t)g * N + x] >> k) & 1u ? 1 : -1;
  }
}

static shaken_status validate(const shaken_problem* p) {
  if (!p) return fail(SHAKEN_E_INVAL, "problem is NULL");
  if (!(p->q > 0.0) || !is_finite_d(p->q)) return fail(SHAKEN_E_INVAL, "q must be finite and > 0");
  if (p->replicas < 1) return fail(SHAKEN_E_INVAL, "replicas must be >= 1");
  if (!p->beta) return fail(SHAKEN_E_INVAL, "beta is NULL");
  for (int r = 0; r < p->replicas; ++r)
    if (!is_finite_d(p->beta[r]) || p->beta[r] < 0.0)
      return fail(SHAKEN_E_INVAL, "beta must be finite and >= 0");
  if (!is_finite_d(p->lambda_const)) return fail(SHAKEN_E_INVAL, "lambda_const not finite");
  if (p->init < 0 || p->init > 3) return fail(SHAKEN_E_INVAL, "bad init kind");
  if (p->init == SHAKEN_INIT_GIVEN && !p->init_spins)
    return fail(SHAKEN_E_INVAL, "init_spins is NULL");
  if (p->kind == SHAKEN_LATTICE) {
    if (p->L < 32 || p->L > 32768 || p->L % 32 != 0)
      return fail(SHAKEN_E_INVAL, "lattice L must be a multiple of 32 in [32, 32768]");
    if (p->encoding < 0 || p->encoding > 2) return fail(SHAKEN_E_INVAL, "bad encoding");
    if (p->encoding == SHAKEN_MULTISPIN && p->replicas % 32 != 0)
      return fail(SHAKEN_E_INVAL, "MULTISPIN needs replicas % 32 == 0");
    if (!is_finite_d(p->J)) return fail(SHAKEN_E_INVAL, "J not finite");
    if (p->boundary != 0 && p->boundary != 1) return fail(SHAKEN_E_INVAL, "bad boundary");
  } else if (p->kind == SHAKEN_GRAPH) {
    if (p->encoding != SHAKEN_MULTISPIN)
      return fail(SHAKEN_E_INVAL, "graphs use the MULTISPIN encoding");
    if (p->replicas % 32 != 0) return fail(SHAKEN_E_INVAL, "graphs need replicas % 32 == 0");
    if (p->n < 1 || p->n >= (int64_t)1 << 31) return fail(SHAKEN_E_INVAL, "graph n out of range");
    if (p->m < 0 || p->m >= (int64_t)1 << 31) return fail(SHAKEN_E_INVAL, "graph m out of range");
    if (p->m > 0 && (!p->u || !p->v || !p->J_edge))
      return fail(SHAKEN_E_INVAL, "graph edge arrays are NULL");
    if (p->orientation != SHAKEN_ORIENT_MIN_MAX && p->orientation != SHAKEN_ORIENT_GIVEN)
      return fail(SHAKEN_E_INVAL, "bad orientation");
    for (int64_t e = 0; e < p->m; ++e) {
      if (p->u[e] < 0 || p->u[e] >= p->n || p->v[e] < 0 || p->v[e] >= p->n)
        return fail(SHAKEN_E_INVAL, "edge endpoint out of range at edge " + std::to_string(e));
      if (p->u[e] == p->v[e]) return fail(SHAKEN_E_INVAL, "self-loop at edge " + std::to_string(e));
      if (!std::isfinite(p->J_edge[e])) return fail(SHAKEN_E_INVAL, "J_edge not finite");
      if (p->J_is_integer && p->J_edge[e] != 1.0f && p->J_edge[e] != -1.0f)
        return fail(SHAKEN_E_INVAL, "J_is_integer but J_edge is not +-1");
    }
  } else {
    return fail(SHAKEN_E_INVAL, "bad kind");
  }
  const int64_t N = p->kind == SHAKEN_LATTICE ? p->L * p->L : p->n;
  if (p->lambda)
    for (int64_t x = 0; x < N; ++x)
      if (!std::isfinite(p->lambda[x])) return fail(SHAKEN_E_INVAL, "lambda not finite");
  if (p->init == SHAKEN_INIT_GIVEN) {
    for (int64_t i = 0; i < (int64_t)p->replicas * N; ++i) {
      const int8_t s = p->init_spins[i];
      if (s != 1 && s != -1) return fail(SHAKEN_E_INVAL, "init_spins must be +1/-1");
    }
  }
  return SHAKEN_OK;
}

// Host-side preparation of a context (no CUDA call): orientation and CSR of a
// graph, frozen lane masks, initial spins.  Kept separate from the device
// set-up so that the server can prepare jobs on the submitting thread.
struct HostPrep {
  std::vector<int32_t> iptr, optr;
  std::vector<uint32_t> ivisit, ovisit;  // per slot of the degree order: x, first edge,
                                         // degree, lambda_x bits (in- / out-CSR)
  std::vector<uint32_t> hubs[2];       // (x, first edge, end edge) above kHubDeg: in, out
  std::vector<uint32_t> icol, ocol;
  std::vector<float> iJ, oJ;
  std::vector<uint32_t> frozen_lanes;
  std::vector<int8_t> init_spins;
  int init_kind = 0;
};

static void build_graph_host(shaken_ctx* c, const shaken_problem* p, HostPrep& hp) {
  const int64_t n = p->n, m = p->m;
  std::vector<int32_t> tail(m), head(m);
  for (int64_t e = 0; e < m; ++e) {
    if (p->orientation == SHAKEN_ORIENT_MIN_MAX) {
      tail[e] = std::min(p->u[e], p->v[e]);
      head[e] = std::max(p->u[e], p->v[e]);
    } else {
      tail[e] = p->u[e];
      head[e] = p->v[e];
    }
  }
  // in-CSR keyed by head (sources tail), out-CSR keyed by tail (heads); entries in edge order
  auto csr = [&](const std::vector<int32_t>& key, const std::vector<int32_t>& other,
                 std::vector<int32_t>& ptr, std::vector<uint32_t>& col, std::vector<float>& Jv) {
    ptr.assign(n + 1, 0);
    for (int64_t e = 0; e < m; ++e) ptr[key[e] + 1]++;
    for (int64_t x = 0; x < n; ++x) ptr[x + 1] += ptr[x];
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    col.assign(m, 0);
    if (!c->integer) Jv.assign(m, 0.0f);
    for (int64_t e = 0; e < m; ++e) {
      const int32_t pos = fill[key[e]]++;
      uint32_t cv = (uint32_t)other[e];
      if (c->integer && p->J_edge[e] < 0.0f) cv |= 0x80000000u;
      col[pos] = cv;
      if (!c->integer) Jv[pos] = p->J_edge[e];
    }
  };
  csr(head, tail, hp.iptr, hp.icol, hp.iJ);
  csr(tail, head, hp.optr, hp.ocol, hp.oJ);
  // visiting order of each half step: vertices by increasing degree (counting sort,
  // stable), so a warp's words have nearly equal edge loops and take the same path
  auto by_degree = [&](const std::vector<int32_t>& ptr, std::vector<uint32_t>& visit) {
    int32_t dmax = 0;
    for (int64_t x = 0; x < n; ++x) dmax = std::max(dmax, ptr[x + 1] - ptr[x]);
    std::vector<int64_t> start((size_t)dmax + 2, 0);
    for (int64_t x = 0; x < n; ++x) start[(size_t)(ptr[x + 1] - ptr[x]) + 1]++;
    for (size_t k = 1; k < start.size(); ++k) start[k] += start[k - 1];
    visit.assign((size_t)n * 4, 0u);
    for (int64_t x = 0; x < n; ++x) {
      const size_t sl = (size_t)start[(size_t)(ptr[x + 1] - ptr[x])]++;
      const float lam = p->lambda != nullptr ? p->lambda[x] : p->lambda_const;
      uint32_t lb;
      std::memcpy(&lb, &lam, 4);
      visit[4 * sl] = (uint32_t)x;
      visit[4 * sl + 1] = (uint32_t)ptr[x];
      visit[4 * sl + 2] = (uint32_t)(ptr[x + 1] - ptr[x]);
      visit[4 * sl + 3] = lb;
    }
  };
  by_degree(hp.iptr, hp.ivisit);
  by_degree(hp.optr, hp.ovisit);
  auto hubs = [&](const std::vector<int32_t>& ptr, std::vector<uint32_t>& out) {
    out.clear();
    for (int64_t x = 0; x < n; ++x)
      if ((uint32_t)(ptr[x + 1] - ptr[x]) > shk::kHubDeg) {
        out.push_back((uint32_t)x);
        out.push_back((uint32_t)ptr[x]);
        out.push_back((uint32_t)ptr[x + 1]);
      }
  };
  hubs(hp.iptr, hp.hubs[0]);
  hubs(hp.optr, hp.hubs[1]);
  c->sumJ = 0.0;
  for (int64_t e = 0; e < m; ++e) c->sumJ += (double)p->J_edge[e];
}

static shaken_status upload_graph(shaken_ctx* c, const HostPrep& hp, cudaStream_t st) {
  c->hubs[0] = hp.hubs[0];
  c->hubs[1] = hp.hubs[1];
  TRY(upload(c->in_ptr, hp.iptr.data(), hp.iptr.size() * 4, st));
  TRY(upload(c->in_visit, hp.ivisit.data(), hp.ivisit.size() * 4, st));
  TRY(upload(c->out_visit, hp.ovisit.data(), hp.ovisit.size() * 4, st));
  TRY(upload(c->out_ptr, hp.optr.data(), hp.optr.size() * 4, st));
  TRY(upload(c->in_col, hp.icol.data(), hp.icol.size() * 4, st));
  TRY(upload(c->out_col, hp.ocol.data(), hp.ocol.size() * 4, st));
  if (!c->integer) {
    TRY(upload(c->in_J, hp.iJ.data(), hp.iJ.size() * 4, st));
    TRY(upload(c->out_J, hp.oJ.data(), hp.oJ.size() * 4, st));
  }
  return SHAKEN_OK;
}

static shaken_status ctx_init_spins(shaken_ctx* c, int kind, const int8_t* given) {
  cudaStream_t st = ctx_stream(c);
  if (kind == SHAKEN_INIT_GIVEN) {
    std::vector<uint8_t> enc;
    encode_spins(c, given, enc);
    CU(cudaMemcpyAsync(c->A.p, enc.data(), enc.size(), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(c->B.p, enc.data(), enc.size(), cudaMemcpyHostToDevice, st));
    CU(cudaStreamSynchronize(st));
    return SHAKEN_OK;
  }
  if (c->solo.dirty) TRY(build_plan(c->solo, st));
  for (auto& F : c->solo.fams) {
    if (F->kind == 0)
      CU(shk::launch_lattice_init(F->enc, F->wpt, F->jobs.as<LatJob>(), F->tiles.as<Tile>(),
                                  F->n_tiles, kind, st));
    else
      CU(shk::launch_graph_init(F->ojobs.as<GraphJob>(), F->otiles.as<Tile>(), F->n_otiles, kind,
                                st));
    c->launches++;
  }
  return SHAKEN_OK;
}

static shaken_status reset_best(shaken_ctx* c) {
  std::vector<double> b(c->R, INFINITY);
  std::vector<long long> bs(c->R, -1);
  cudaStream_t st = ctx_stream(c);
  CU(cudaMemcpyAsync(c->best.p, b.data(), b.size() * 8, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(c->best_step.p, bs.data(), bs.size() * 8, cudaMemcpyHostToDevice, st));
  CU(cudaStreamSynchronize(st));
  return SHAKEN_OK;
}

// ============================================================================ C ABI: contexts
extern "C" {

}  // extern "C"

// Validates the problem and fills the context's host fields and the host-side
// preparation (no CUDA call).
static shaken_status prepare_ctx(const shaken_problem* p, uint64_t seed, void* cuda_stream,
                                 std::unique_ptr<shaken_ctx>& out, HostPrep& hp) {
  TRY(validate(p));
  std::unique_ptr<shaken_ctx> c(new shaken_ctx());
  c->kind = p->kind;
  c->enc = p->encoding;
  c->L = p->L;
  c->n = p->kind == SHAKEN_LATTICE ? p->L * p->L : p->n;
  c->m = p->kind == SHAKEN_LATTICE ? 2 * c->n : p->m;
  c->R = p->replicas;
  c->J = p->J;
  c->q = p->q;
  c->lam_c = p->lambda_const;
  c->seed = seed;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->integer = p->kind == SHAKEN_GRAPH && p->J_is_integer;
  c->beta.assign(p->beta, p->beta + p->replicas);
  const int64_t N = c->sites();
  if (p->lambda) {
    if (p->kind == SHAKEN_LATTICE)
      return fail(SHAKEN_E_INVAL, "lattices take a constant lambda (lambda_const)");
    c->has_lambda = true;
    c->lambda.assign(p->lambda, p->lambda + N);
  }
  if (p->frozen_mask || (p->kind == SHAKEN_LATTICE && p->boundary == 1)) {
    c->frozen.assign(N, 0);
    if (p->frozen_mask) {
      for (int64_t x = 0; x < N; ++x) c->frozen[x] = p->frozen_mask[x] ? 1 : 0;
    } else {
      for (int64_t j = 0; j < c->L; ++j) c->frozen[j] = 1;
      for (int64_t i = 0; i < c->L; ++i) c->frozen[i * c->L] = 1;
    }
    if (p->init == SHAKEN_INIT_GIVEN)
      for (int r = 0; r < c->R; ++r)
        for (int64_t x = 0; x < N; ++x)
          if (c->frozen[x] && p->init_spins[(size_t)r * N + x] != 1)
            return fail(SHAKEN_E_INVAL, "frozen sites must be +1 in init_spins");
    if (c->kind == SHAKEN_LATTICE && c->enc != SHAKEN_MULTISPIN) {
      hp.frozen_lanes.assign(N / 32, 0u);
      for (int64_t x = 0; x < N; ++x)
        if (c->frozen[x]) hp.frozen_lanes[x >> 5] |= 1u << (x & 31);
    } else {
      hp.frozen_lanes.assign(N, 0u);
      for (int64_t x = 0; x < N; ++x) hp.frozen_lanes[x] = c->frozen[x] ? 0xffffffffu : 0u;
    }
  }
  if (c->kind == SHAKEN_LATTICE) {
    if (c->enc == SHAKEN_INT8)
      c->spin_bytes = (size_t)c->R * N;
    else if (c->enc == SHAKEN_PACKED)
      c->spin_bytes = (size_t)c->R * N / 8;
    else
      c->spin_bytes = (size_t)(c->R / 32) * N * 4;
  } else {
    c->spin_bytes = (size_t)(c->R / 32) * N * 4;
    build_graph_host(c.get(), p, hp);
  }
  hp.init_kind = p->init;
  if (p->init == SHAKEN_INIT_GIVEN) hp.init_spins.assign(p->init_spins, p->init_spins + (size_t)c->R * N);
  out = std::move(c);
  return SHAKEN_OK;
}

// Device set-up of a prepared context: allocations, uploads, tables, initial spins.
static shaken_status setup_ctx(shaken_ctx* c, const HostPrep& hp) {
  cudaStream_t st = ctx_stream(c);
  const int64_t N = c->sites();
  TRY(c->A.alloc(c->spin_bytes));
  TRY(c->B.alloc(c->spin_bytes));
  if (!hp.frozen_lanes.empty())
    TRY(upload(c->frozen_lanes, hp.frozen_lanes.data(), hp.frozen_lanes.size() * 4, st));
  if (c->kind == SHAKEN_GRAPH) {
    TRY(upload_graph(c, hp, st));
    if (c->has_lambda) TRY(upload(c->lam_dev, c->lambda.data(), c->lambda.size() * 4, st));
    TRY(upload(c->beta_lanes, c->beta.data(), c->beta.size() * 8, st));
  } else {
    const std::vector<double> lanes = lattice_table_lanes(c);
    TRY(build_tables_for_betas(c, lanes, c->tables, c->beta_lanes, lattice_ntab(c), st));
  }
  CU(cudaStreamSynchronize(st));  // host sources of the uploads may go away after this
  const size_t sums_bytes = (size_t)c->R * kNumSums * sizeof(double);
  TRY(c->step_sums.alloc(sums_bytes));
  TRY(c->obs_sums.alloc(sums_bytes));
  CU(cudaMemsetAsync(c->step_sums.p, 0, sums_bytes, st));
  TRY(c->best.alloc((size_t)c->R * 8));
  TRY(c->best_step.alloc((size_t)c->R * 8));
  TRY(c->cd.alloc(sizeof(CtxDev)));
  CtxDev& h = c->hcd;
  std::memset(&h, 0, sizeof(h));
  h.step = 0;
  h.t_end = 0xFFFFFFFEu;
  h.R = (uint32_t)c->R;
  h.kind = (uint32_t)c->kind;
  h.Jc = c->kind == SHAKEN_LATTICE ? c->J : 1.0;
  h.lamc = c->kind == SHAKEN_LATTICE ? c->lam_c : 0.0;
  h.inv_n = 1.0 / (double)N;
  h.step_sums = c->step_sums.as<double>();
  h.best = c->best.as<double>();
  h.best_step = c->best_step.as<long long>();
  TRY(push_cd(c));
  TRY(reset_best(c));
  c->solo.members = {c};
  c->solo.dirty = true;
  TRY(ctx_init_spins(c, hp.init_kind, hp.init_spins.empty() ? nullptr : hp.init_spins.data()));
  CU(cudaStreamSynchronize(st));
  return SHAKEN_OK;
}

extern "C" {

shaken_status shaken_init(shaken_ctx** out, const shaken_problem* p, uint64_t seed,
                          void* cuda_stream) {
  if (!out) return fail(SHAKEN_E_INVAL, "out is NULL");
  *out = nullptr;
  std::unique_ptr<shaken_ctx> c;
  HostPrep hp;
  TRY(prepare_ctx(p, seed, cuda_stream, c, hp));
  TRY(setup_ctx(c.get(), hp));
  *out = c.release();
  return SHAKEN_OK;
}

void shaken_free(shaken_ctx* ctx) {
  if (!ctx) return;
  if (ctx->owner) shaken_batch_remove(ctx->owner, ctx);
  cudaStreamSynchronize(ctx->stream);
  delete ctx;
}

static shaken_status check_steps(shaken_ctx* c, uint64_t n) {
  if (c->host_step + n >= 0xFFFFFFFEull)
    return fail(SHAKEN_E_INVAL, "step counter would reach 2^32 - 2");
  return SHAKEN_OK;
}

// Small lattices run whole chunks of steps inside one launch, one block per
// replica (or multispin group), the state in shared memory.
static bool resident_eligible(const shaken_ctx* c, uint64_t n_steps) {
  if (c->kind != SHAKEN_LATTICE || c->owner || n_steps < 4) return false;
  const uint64_t words = c->enc == SHAKEN_MULTISPIN ? (uint64_t)c->L * c->L
                                                    : (uint64_t)c->L * c->L / 32;
  if (words > 4096) return false;
  if (c->enc == SHAKEN_MULTISPIN && (c->hcd.tracking || c->hcd.record)) return false;
  return true;
}

static shaken_status run_resident(shaken_ctx* c, uint64_t n_steps) {
  cudaStream_t st = c->stream;
  if (c->solo.dirty) TRY(build_plan(c->solo, st));
  const Family& F = *c->solo.fams[0];
  const int n_jobs = c->enc == SHAKEN_MULTISPIN ? c->R / 32 : c->R;
  const uint32_t words = c->enc == SHAKEN_MULTISPIN ? (uint32_t)(c->L * c->L)
                                                    : (uint32_t)(c->L * c->L / 32);
  uint64_t done = 0;
  while (done < n_steps) {
    const uint64_t chunk = std::min<uint64_t>(n_steps - done, 1u << 16);
    CU(shk::launch_lattice_resident(F.enc, F.jobs.as<LatJob>(), n_jobs, words,
                                    (uint32_t)(c->host_step + done), (uint32_t)chunk, st));
    c->launches++;
    done += chunk;
  }
  c->host_step += n_steps;
  return push_cd(c);  // the device step counter follows the host's
}

// Mid-size single lattices (INT8/PACKED, one replica, beyond the resident size)
// run whole chunks of steps in one cooperative launch that keeps the lattice in
// shared memory as row bands.  Not for tracking, recording or annealing runs.
static bool band_eligible(const shaken_ctx* c, uint64_t n_steps, int* grid, size_t* smem) {
  if (c->kind != SHAKEN_LATTICE || c->owner || n_steps < 8 || c->R != 1) return false;
  if (c->enc != SHAKEN_INT8 && c->enc != SHAKEN_PACKED) return false;
  if (c->hcd.tracking || c->hcd.record || c->hcd.anneal_len != 0) return false;
  if ((uint64_t)c->L * c->L / 32 <= 4096) return false;
  const int enc = c->enc == SHAKEN_INT8 ? 0 : 1;
  return shk::lattice_band_shape(enc, (uint32_t)c->L, (uint32_t)(c->L / 32), grid, smem);
}

static shaken_status run_band(shaken_ctx* c, uint64_t n_steps, int grid, size_t smem) {
  cudaStream_t st = c->stream;
  if (c->solo.dirty) TRY(build_plan(c->solo, st));
  const Family& F = *c->solo.fams[0];
  const uint32_t wpr = (uint32_t)(c->L / 32);
  // exchange rows [2 parities][grid][wpr] of (half-step count << 32 | word)
  const size_t xbytes = (size_t)2 * grid * wpr * sizeof(uint64_t);
  if (c->band_xch.p == nullptr || c->band_xch.bytes < xbytes) TRY(c->band_xch.alloc(xbytes));
  if (c->band_sync.p == nullptr) TRY(c->band_sync.alloc(sizeof(shk::BandSync)));
  uint64_t done = 0;
  while (done < n_steps) {
    const uint64_t chunk = std::min<uint64_t>(n_steps - done, 1u << 16);
    shk::BandSync h0{};
    h0.hurry = c->band_hurry >= 0 ? (unsigned)c->band_hurry : ~0u;
    if (c->band_stall) h0.count = (unsigned)grid;  // no block is ever the last to arrive
    c->band_stall = false;
    c->band_hurry = -1;
    CU(cudaMemcpyAsync(c->band_sync.p, &h0, sizeof(h0), cudaMemcpyHostToDevice, st));
    CU(cudaMemsetAsync(c->band_xch.p, 0, xbytes, st));  // no count is valid yet
    CU(shk::launch_lattice_band(F.enc, F.jobs.as<LatJob>(), grid, smem,
                                c->band_xch.as<uint64_t>(), c->band_sync.as<shk::BandSync>(),
                                (uint32_t)c->host_step, (uint32_t)chunk, st));
    c->launches++;
    shk::BandSync h{};
    CU(cudaMemcpyAsync(&h, c->band_sync.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (h.commit != 1u) {
      // the run was aborted before any block wrote the chunk back: the state is the
      // one before the chunk, and the step counter says so
      TRY(push_cd(c));
      return fail(SHAKEN_E_TIMEOUT,
                  "banded run: a grid barrier wait ran out; the chunk was not applied");
    }
    c->host_step += chunk;
    done += chunk;
  }
  return push_cd(c);  // the device step counter follows the host's
}

static shaken_status solo_run(shaken_ctx* ctx, uint64_t n_steps) {
  if (resident_eligible(ctx, n_steps)) return run_resident(ctx, n_steps);
  int grid = 0;
  size_t smem = 0;
  if (band_eligible(ctx, n_steps, &grid, &smem)) return run_band(ctx, n_steps, grid, smem);
  uint64_t nl = 0;
  shaken_status s = plan_run(ctx->solo, ctx->stream, n_steps, n_steps >= 64, &nl);
  ctx->launches += nl;
  if (s != SHAKEN_OK) return s;
  ctx->host_step += n_steps;
  return SHAKEN_OK;
}

shaken_status shaken_step(shaken_ctx* ctx, uint64_t n_steps) {
  if (!ctx) return fail(SHAKEN_E_INVAL, "ctx is NULL");
  if (ctx->owner) return fail(SHAKEN_E_STATE, "context belongs to a batch");
  TRY(check_steps(ctx, n_steps));
  return solo_run(ctx, n_steps);
}

shaken_status shaken_set_order(shaken_ctx* ctx, int reversed) {
  if (!ctx) return fail(SHAKEN_E_INVAL, "ctx is NULL");
  if (reversed != 0 && reversed != 1) return fail(SHAKEN_E_INVAL, "order must be 0 or 1");
  ctx->hcd.order = (uint32_t)reversed;
  ctx->solo.invalidate();
  if (ctx->owner) ctx->owner->plan.invalidate();
  return push_cd(ctx);
}

shaken_status shaken_set_tracking(shaken_ctx* ctx, int enable) {
  if (!ctx) return fail(SHAKEN_E_INVAL, "ctx is NULL");
  ctx->tracking = enable != 0;
  ctx->hcd.tracking = ctx->tracking ? 1u : 0u;
  ctx->solo.invalidate();
  if (ctx->owner) ctx->owner->plan.invalidate();
  return push_cd(ctx);
}

// Prepare an anneal of n steps from the current step (tables / schedule on the
// device, tracking on).  Used by shaken_anneal and by the server.
static shaken_status begin_anneal(shaken_ctx* c, const double* sched, uint64_t n) {
  if (!sched) return fail(SHAKEN_E_INVAL, "beta_schedule is NULL");
  for (uint64_t k = 0; k < n; ++k)
    if (!std::isfinite(sched[k]) || sched[k] < 0.0)
      return fail(SHAKEN_E_INVAL, "beta_schedule must be finite and >= 0");
  cudaStream_t st = ctx_stream(c);
  if (c->kind == SHAKEN_LATTICE) {
    std::vector<double> lanes((size_t)n * 32);
    for (uint64_t k = 0; k < n; ++k)
      for (int l = 0; l < 32; ++l) lanes[k * 32 + l] = sched[k];
    TRY(build_tables_for_betas(c, lanes, c->anneal_tables, c->anneal_lanes, (int)n, st));
  } else {
    TRY(upload(c->anneal_sched, sched, n * sizeof(double), st));
  }
  CU(cudaStreamSynchronize(st));
  c->hcd.anneal_t0 = (uint32_t)c->host_step;
  c->hcd.anneal_len = (uint32_t)n;
  c->hcd.tracking = 1u;
  c->solo.invalidate();
  if (c->owner) c->owner->plan.invalidate();
  return push_cd(c);
}

static shaken_status end_anneal(shaken_ctx* c) {
  c->hcd.anneal_len = 0u;
  c->hcd.tracking = c->tracking ? 1u : 0u;
  c->solo.invalidate();
  if (c->owner) c->owner->plan.invalidate();
  return push_cd(c);
}

shaken_status shaken_anneal(shaken_ctx* ctx, const double* beta_schedule, uint64_t n_steps) {
  if (!ctx) return fail(SHAKEN_E_INVAL, "ctx is NULL");
  if (ctx->owner) return fail(SHAKEN_E_STATE, "context belongs to a batch");
  if (n_steps == 0) return SHAKEN_OK;
  TRY(check_steps(ctx, n_steps));
  TRY(begin_anneal(ctx, beta_schedule, n_steps));
  TRY(solo_run(ctx, n_steps));
  return end_anneal(ctx);
}

shaken_status shaken_step_record(shaken_ctx* ctx, uint64_t n_steps, double* mag, double* energy) {
  if (!ctx) return fail(SHAKEN_E_INVAL, "ctx is NULL");
  if (ctx->owner) return fail(SHAKEN_E_STATE, "context belongs to a batch");
  TRY(check_steps(ctx, n_steps));
  if (n_steps == 0) return SHAKEN_OK;
  const size_t bytes = (size_t)n_steps * ctx->R * sizeof(double);
  TRY(ctx->series_m.alloc(bytes));
  TRY(ctx->series_H.alloc(bytes));
  ctx->hcd.record = 1u;
  ctx->hcd.series_t0 = (uint32_t)ctx->host_step;
  ctx->hcd.series_cap = (uint32_t)n_steps;
  ctx->hcd.series_m = ctx->series_m.as<double>();
  ctx->hcd.series_H = ctx->series_H.as<double>();
  ctx->hcd.tracking = 1u;
  ctx->solo.invalidate();
  TRY(push_cd(ctx));
  TRY(solo_run(ctx, n_steps));
  if (mag) CU(cudaMemcpyAsync(mag, ctx->series_m.p, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  if (energy)
    CU(cudaMemcpyAsync(energy, ctx->series_H.p, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  ctx->hcd.record = 0u;
  ctx->hcd.series_m = nullptr;
  ctx->hcd.series_H = nullptr;
  ctx->hcd.tracking = ctx->tracking ? 1u : 0u;
  ctx->solo.invalidate();
  TRY(push_cd(ctx));
  ctx->series_m.release();
  ctx->series_H.release();
  return SHAKEN_OK;
}

// Observables in two parts: the device sums of a context's replicas are
// cleared and, after the observables launches, copied to host buffers (obs_copy,
// or one packed copy for a whole batch); after a synchronisation obs_values turns
// them into shaken_obs records and lowers the best energies where the current
// energy is below them (the caller writes those back to the device).
struct ObsHost {
  std::vector<double> sums, best;
  std::vector<long long> bstep;
};

static shaken_status obs_copy(shaken_ctx* c, ObsHost& h, cudaStream_t st) {
  const int R = c->R;
  h.sums.assign((size_t)R * kNumSums, 0.0);
  h.best.assign(R, 0.0);
  h.bstep.assign(R, 0);
  CU(cudaMemcpyAsync(h.sums.data(), c->obs_sums.p, h.sums.size() * 8, cudaMemcpyDeviceToHost,
                     st));
  CU(cudaMemcpyAsync(h.best.data(), c->best.p, h.best.size() * 8, cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(h.bstep.data(), c->best_step.p, h.bstep.size() * 8,
                     cudaMemcpyDeviceToHost, st));
  return SHAKEN_OK;
}

static shaken_status obs_values(shaken_ctx* c, ObsHost& h, shaken_obs* out, bool* changed) {
  const int R = c->R;
  const double N = (double)c->sites();
  for (int r = 0; r < R; ++r) {
    const double* s = &h.sums[(size_t)r * kNumSums];
    shaken_obs& o = out[r];
    o.magnetization = s[shk::kSumM] / N;
    o.cut_edges = (int64_t)llround(s[shk::kSumCut]);
    if (c->kind == SHAKEN_LATTICE) {
      const double J = c->J, lam = c->lam_c, q = c->q;
      o.energy = -(J * s[shk::kSumE]) - 2.0 * lam * s[shk::kSumM];
      o.pair_energy = -(J * s[shk::kSumP1] + q * s[shk::kSumP2] +
                        lam * (s[shk::kSumM] + s[shk::kSumM2]));
      o.cut_weight = -J * s[shk::kSumCut];
    } else {
      o.energy = -s[shk::kSumE] - 2.0 * s[shk::kSumLS];
      o.pair_energy = -(s[shk::kSumP1] + c->q * s[shk::kSumP2] + s[shk::kSumLS] +
                        s[shk::kSumLS2]);
      o.cut_weight = 0.5 * (s[shk::kSumE] - c->sumJ);
    }
    if (o.energy < h.best[r]) {
      h.best[r] = o.energy;
      h.bstep[r] = (long long)c->host_step;
      *changed = true;
    }
    o.best_energy = h.best[r];
    o.best_step = h.bstep[r];
  }
  return SHAKEN_OK;
}

static shaken_status obs_launch(Plan& P, cudaStream_t st, uint64_t* launches) {
  for (auto& F : P.fams) {
    if (F->kind == 0)
      CU(shk::launch_lattice_obs(F->enc, F->wpt, F->jobs.as<LatJob>(), F->tiles.as<Tile>(),
                                 F->n_tiles, 1, 1, st));
    else
      CU(shk::launch_graph_obs(F->enc != 0, F->ojobs.as<GraphJob>(), F->otiles.as<Tile>(),
                               F->n_otiles, 1, 1, st));
    ++*launches;
  }
  return SHAKEN_OK;
}

shaken_status shaken_observables(shaken_ctx* ctx, shaken_obs* out) {
  if (!ctx || !out) return fail(SHAKEN_E_INVAL, "NULL argument");
  cudaStream_t st = ctx_stream(ctx);
  if (ctx->solo.dirty) TRY(build_plan(ctx->solo, st));
  CU(cudaMemsetAsync(ctx->obs_sums.p, 0, ctx->obs_sums.bytes, st));
  uint64_t nl = 0;
  TRY(obs_launch(ctx->solo, st, &nl));
  ctx->launches += nl;
  ObsHost h;
  TRY(obs_copy(ctx, h, st));
  CU(cudaStreamSynchronize(st));
  bool changed = false;
  TRY(obs_values(ctx, h, out, &changed));
  if (changed) {
    CU(cudaMemcpyAsync(ctx->best.p, h.best.data(), h.best.size() * 8, cudaMemcpyHostToDevice,
                       st));
    CU(cudaMemcpyAsync(ctx->best_step.p, h.bstep.data(), h.bstep.size() * 8,
                       cudaMemcpyHostToDevice, st));
    CU(cudaStreamSynchronize(st));
  }
  return SHAKEN_OK;
}

// The member table of a batch plan for the packed copies.
static shaken_status member_table(Plan& P, cudaStream_t st) {
  if (P.mtab_valid) return SHAKEN_OK;
  if (P.members.size() > 65535)
    return fail(SHAKEN_E_INVAL, "batched copies take at most 65535 members");
  std::vector<shk::MemberDev> m;
  size_t so = 0, oo = 0;
  P.max_state_words = P.max_obs = 0;
  for (shaken_ctx* c : P.members) {
    shk::MemberDev d{};
    d.A = static_cast<uint32_t*>(c->A.p);
    d.B = static_cast<uint32_t*>(c->B.p);
    d.obs = c->obs_sums.as<double>();
    d.best = c->best.as<double>();
    d.best_step = c->best_step.as<long long>();
    d.state_off = so;
    d.obs_off = oo;
    d.state_words = c->spin_bytes / 4;
    d.R = (uint32_t)c->R;
    so += d.state_words;
    oo += (size_t)c->R * (kNumSums + 2);
    P.max_state_words = std::max(P.max_state_words, d.state_words);
    P.max_obs = std::max(P.max_obs, (unsigned long long)c->R * (kNumSums + 2));
    m.push_back(d);
  }
  TRY(upload(P.mtab, m.data(), m.size() * sizeof(shk::MemberDev), st));
  P.state_words = so;
  P.obs_doubles = oo;
  P.mtab_valid = true;
  return SHAKEN_OK;
}

static shaken_status stage(DevMem& d, size_t bytes) {
  if (d.p == nullptr || d.bytes < bytes) TRY(d.alloc(bytes));
  return SHAKEN_OK;
}

shaken_status shaken_batch_observables(shaken_batch* b, shaken_obs* out) {
  if (!b || !out) return fail(SHAKEN_E_INVAL, "NULL argument");
  Plan& P = b->plan;
  if (P.members.empty()) return SHAKEN_OK;
  cudaStream_t st = b->stream;
  if (P.dirty) TRY(build_plan(P, st));
  TRY(member_table(P, st));
  TRY(stage(P.stage_obs, P.obs_doubles * sizeof(double)));
  // every member's sums zeroed by one launch (not one memset per member)
  CU(shk::launch_member_copy(4, P.mtab.as<shk::MemberDev>(), (int)P.members.size(), nullptr,
                             P.max_obs, st));
  uint64_t nl = 1;
  TRY(obs_launch(P, st, &nl));
  const int n = (int)P.members.size();
  CU(shk::launch_member_copy(2, P.mtab.as<shk::MemberDev>(), n, P.stage_obs.p, P.max_obs, st));
  b->launches += nl + 1;
  std::vector<double> packed(P.obs_doubles);
  CU(cudaMemcpyAsync(packed.data(), P.stage_obs.p, packed.size() * sizeof(double),
                     cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  // members' records from the packed buffer; best energies updated in place
  bool any = false;
  size_t off = 0, oo = 0;
  for (shaken_ctx* c : P.members) {
    const size_t R = (size_t)c->R, ns = R * kNumSums;
    ObsHost h;
    h.sums.assign(packed.begin() + oo, packed.begin() + oo + ns);
    h.best.assign(packed.begin() + oo + ns, packed.begin() + oo + ns + R);
    h.bstep.resize(R);
    std::memcpy(h.bstep.data(), packed.data() + oo + ns + R, R * sizeof(long long));
    bool changed = false;
    TRY(obs_values(c, h, out + off, &changed));
    if (changed) {
      std::copy(h.best.begin(), h.best.end(), packed.begin() + oo + ns);
      std::memcpy(packed.data() + oo + ns + R, h.bstep.data(), R * sizeof(long long));
      any = true;
    }
    off += R;
    oo += R * (kNumSums + 2);
  }
  if (any) {
    CU(cudaMemcpyAsync(P.stage_obs.p, packed.data(), packed.size() * sizeof(double),
                       cudaMemcpyHostToDevice, st));
    CU(shk::launch_member_copy(3, P.mtab.as<shk::MemberDev>(), n, P.stage_obs.p, P.max_obs,
                               st));
    b->launches += 1;
    CU(cudaStreamSynchronize(st));
  }
  return SHAKEN_OK;
}

shaken_status shaken_batch_state_bytes(shaken_batch* b, size_t* bytes) {
  if (!b || !bytes) return fail(SHAKEN_E_INVAL, "NULL argument");
  size_t n = 0;
  for (shaken_ctx* c : b->plan.members) n += c->spin_bytes;
  *bytes = n;
  return SHAKEN_OK;
}

shaken_status shaken_batch_set_states_raw(shaken_batch* b, const void* host, size_t bytes) {
  if (!b || !host) return fail(SHAKEN_E_INVAL, "NULL argument");
  Plan& P = b->plan;
  if (P.members.empty()) return SHAKEN_OK;
  cudaStream_t st = b->stream;
  TRY(member_table(P, st));
  if (bytes != P.state_words * 4) return fail(SHAKEN_E_INVAL, "state size mismatch");
  TRY(stage(P.stage_state, bytes));
  CU(cudaMemcpyAsync(P.stage_state.p, host, bytes, cudaMemcpyHostToDevice, st));
  CU(shk::launch_member_copy(1, P.mtab.as<shk::MemberDev>(), (int)P.members.size(),
                             P.stage_state.p, P.max_state_words, st));
  b->launches += 1;
  return SHAKEN_OK;
}

shaken_status shaken_batch_get_states_raw_async(shaken_batch* b, void* host, size_t bytes) {
  if (!b || !host) return fail(SHAKEN_E_INVAL, "NULL argument");
  Plan& P = b->plan;
  if (P.members.empty()) return SHAKEN_OK;
  cudaStream_t st = b->stream;
  TRY(member_table(P, st));
  if (bytes != P.state_words * 4) return fail(SHAKEN_E_INVAL, "state size mismatch");
  TRY(stage(P.stage_state, bytes));
  CU(shk::launch_member_copy(0, P.mtab.as<shk::MemberDev>(), (int)P.members.size(),
                             P.stage_state.p, P.max_state_words, st));
  b->launches += 1;
  CU(cudaMemcpyAsync(host, P.stage_state.p, bytes, cudaMemcpyDeviceToHost, st));
  return SHAKEN_OK;
}

shaken_status shaken_get_spins(shaken_ctx* ctx, int8_t* out) {
  if (!ctx || !out) return fail(SHAKEN_E_INVAL, "NULL argument");
  std::vector<uint8_t> buf(ctx->spin_bytes);
  cudaStream_t st = ctx_stream(ctx);
  CU(cudaMemcpyAsync(buf.data(), ctx->A.p, buf.size(), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  decode_spins(ctx, buf, out);
  return SHAKEN_OK;
}

shaken_status shaken_get_spins_prime(shaken_ctx* ctx, int8_t* out) {
  if (!ctx || !out) return fail(SHAKEN_E_INVAL, "NULL argument");
  std::vector<uint8_t> buf(ctx->spin_bytes);
  cudaStream_t st = ctx_stream(ctx);
  CU(cudaMemcpyAsync(buf.data(), ctx->B.p, buf.size(), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  decode_spins(ctx, buf, out);
  return SHAKEN_OK;
}

shaken_status shaken_set_spins(shaken_ctx* ctx, const int8_t* in) {
  if (!ctx || !in) return fail(SHAKEN_E_INVAL, "NULL argument");
  const int64_t N = ctx->sites();
  for (int64_t i = 0; i < (int64_t)ctx->R * N; ++i) {
    if (in[i] != 1 && in[i] != -1) return fail(SHAKEN_E_INVAL, "spins must be +1/-1");
    if (!ctx->frozen.empty() && ctx->frozen[i % N] && in[i] != 1)
      return fail(SHAKEN_E_INVAL, "frozen sites must be +1");
  }
  return ctx_init_spins(ctx, SHAKEN_INIT_GIVEN, in);
}

shaken_status shaken_state_bytes(shaken_ctx* ctx, size_t* bytes) {
  if (!ctx || !bytes) return fail(SHAKEN_E_INVAL, "NULL argument");
  *bytes = ctx->spin_bytes;
  return SHAKEN_OK;
}

shaken_status shaken_set_state_raw(shaken_ctx* ctx, const void* host_words, size_t bytes) {
  if (!ctx || !host_words) return fail(SHAKEN_E_INVAL, "NULL argument");
  if (bytes != ctx->spin_bytes) return fail(SHAKEN_E_INVAL, "state size mismatch");
  cudaStream_t st = ctx_stream(ctx);
  CU(cudaMemcpyAsync(ctx->A.p, host_words, bytes, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(ctx->B.p, ctx->A.p, bytes, cudaMemcpyDeviceToDevice, st));
  return SHAKEN_OK;
}

shaken_status shaken_get_state_raw(shaken_ctx* ctx, void* host_words, size_t bytes) {
  if (!ctx || !host_words) return fail(SHAKEN_E_INVAL, "NULL argument");
  if (bytes != ctx->spin_bytes) return fail(SHAKEN_E_INVAL, "state size mismatch");
  cudaStream_t st = ctx_stream(ctx);
  CU(cudaMemcpyAsync(host_words, ctx->A.p, bytes, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  return SHAKEN_OK;
}

shaken_status shaken_get_state_raw_async(shaken_ctx* ctx, void* host_words, size_t bytes) {
  if (!ctx || !host_words) return fail(SHAKEN_E_INVAL, "NULL argument");
  if (bytes != ctx->spin_bytes) return fail(SHAKEN_E_INVAL, "state size mismatch");
  CU(cudaMemcpyAsync(host_words, ctx->A.p, bytes, cudaMemcpyDeviceToHost, ctx_stream(ctx)));
  return SHAKEN_OK;
}

shaken_status shaken_get_step(shaken_ctx* ctx, uint64_t* t) {
  if (!ctx || !t) return fail(SHAKEN_E_INVAL, "NULL argument");
  *t = ctx->host_step;
  return SHAKEN_OK;
}

struct CkptHeader {
  char magic[8];
  uint32_t version, kind, enc, R;
  int64_t n;
  uint64_t step;
  uint64_t spin_bytes;
  uint32_t tracking, pad;
};

shaken_status shaken_save(shaken_ctx* ctx, void* buf, size_t* len) {
  if (!ctx || !len) return fail(SHAKEN_E_INVAL, "NULL argument");
  const size_t need = sizeof(CkptHeader) + 2 * ctx->spin_bytes + (size_t)ctx->R * 16;
  if (!buf) {
    *len = need;
    return SHAKEN_OK;
  }
  if (*len < need) return fail(SHAKEN_E_INVAL, "checkpoint buffer too small");
  CkptHeader h{};
  std::memcpy(h.magic, "SHAKEN01", 8);
  h.version = 1;
  h.kind = (uint32_t)ctx->kind;
  h.enc = (uint32_t)ctx->enc;
  h.R = (uint32_t)ctx->R;
  h.n = ctx->sites();
  h.step = ctx->host_step;
  h.spin_bytes = ctx->spin_bytes;
  h.tracking = ctx->tracking ? 1u : 0u;
  uint8_t* b = static_cast<uint8_t*>(buf);
  std::memcpy(b, &h, sizeof(h));
  cudaStream_t st = ctx_stream(ctx);
  uint8_t* p = b + sizeof(h);
  CU(cudaMemcpyAsync(p, ctx->A.p, ctx->spin_bytes, cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(p + ctx->spin_bytes, ctx->B.p, ctx->spin_bytes, cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(p + 2 * ctx->spin_bytes, ctx->best.p, (size_t)ctx->R * 8,
                     cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(p + 2 * ctx->spin_bytes + (size_t)ctx->R * 8, ctx->best_step.p,
                     (size_t)ctx->R * 8, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  *len = need;
  return SHAKEN_OK;
}

shaken_status shaken_load(shaken_ctx* ctx, const void* buf, size_t len) {
  if (!ctx || !buf) return fail(SHAKEN_E_INVAL, "NULL argument");
  if (len < sizeof(CkptHeader)) return fail(SHAKEN_E_INVAL, "checkpoint too short");
  CkptHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (std::memcmp(h.magic, "SHAKEN01", 8) != 0 || h.version != 1)
    return fail(SHAKEN_E_INVAL, "not a checkpoint");
  if (h.kind != (uint32_t)ctx->kind || h.enc != (uint32_t)ctx->enc || h.R != (uint32_t)ctx->R ||
      h.n != ctx->sites() || h.spin_bytes != ctx->spin_bytes)
    return fail(SHAKEN_E_INVAL, "checkpoint does not match this context");
  const size_t need = sizeof(CkptHeader) + 2 * ctx->spin_bytes + (size_t)ctx->R * 16;
  if (len < need) return fail(SHAKEN_E_INVAL, "checkpoint truncated");
  const uint8_t* p = static_cast<const uint8_t*>(buf) + sizeof(h);
  cudaStream_t st = ctx_stream(ctx);
  CU(cudaMemcpyAsync(ctx->A.p, p, ctx->spin_bytes, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(ctx->B.p, p + ctx->spin_bytes, ctx->spin_bytes, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(ctx->best.p, p + 2 * ctx->spin_bytes, (size_t)ctx->R * 8,
                     cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(ctx->best_step.p, p + 2 * ctx->spin_bytes + (size_t)ctx->R * 8,
                     (size_t)ctx->R * 8, cudaMemcpyHostToDevice, st));
  CU(cudaStreamSynchronize(st));
  ctx->host_step = h.step;
  ctx->tracking = h.tracking != 0;
  ctx->hcd.tracking = h.tracking;
  ctx->hcd.anneal_len = 0;
  ctx->solo.invalidate();
  return push_cd(ctx);
}

shaken_status shaken_debug_fields(shaken_ctx* ctx, int half, float* out) {
  if (!ctx || !out || (half != 0 && half != 1)) return fail(SHAKEN_E_INVAL, "bad argument");
  if (ctx->kind != SHAKEN_GRAPH) return fail(SHAKEN_E_STATE, "field dump is for graphs");
  cudaStream_t st = ctx_stream(ctx);
  if (ctx->solo.dirty) TRY(build_plan(ctx->solo, st));
  DevMem d;
  const size_t bytes = (size_t)ctx->R * ctx->n * sizeof(float);
  TRY(d.alloc(bytes));
  for (auto& F : ctx->solo.fams) {
    CU(shk::launch_graph_fields(F->ojobs.as<GraphJob>(), F->otiles.as<Tile>(), F->n_otiles,
                                (uint32_t)half, d.as<float>(), st));
    ctx->launches++;
  }
  CU(cudaMemcpyAsync(out, d.p, bytes, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  return SHAKEN_OK;
}

shaken_status shaken_launch_count(shaken_ctx* ctx, uint64_t* count) {
  if (!ctx || !count) return fail(SHAKEN_E_INVAL, "NULL argument");
  *count = ctx->launches.load();
  return SHAKEN_OK;
}

shaken_status shaken_sync(shaken_ctx* ctx) {
  if (!ctx) return fail(SHAKEN_E_INVAL, "ctx is NULL");
  CU(cudaStreamSynchronize(ctx_stream(ctx)));
  return SHAKEN_OK;
}

// Diagnostics: force the fp64 path of the integer graph decision (not in the header).
shaken_status shaken_debug_exact_always(shaken_ctx* ctx, int on) {
  if (!ctx) return fail(SHAKEN_E_INVAL, "ctx is NULL");
  ctx->exact_always = on ? 1 : 0;
  return SHAKEN_OK;
}

shaken_status shaken_debug_band_hurry(shaken_ctx* ctx, int block) {
  if (!ctx || block < 0) return fail(SHAKEN_E_INVAL, "bad argument");
  ctx->band_hurry = block;
  return SHAKEN_OK;
}

shaken_status shaken_debug_band_stall(shaken_ctx* ctx) {
  if (!ctx) return fail(SHAKEN_E_INVAL, "ctx is NULL");
  ctx->band_stall = true;
  return SHAKEN_OK;
}

// ============================================================================ C ABI: batches
shaken_status shaken_batch_create(shaken_batch** out, void* cuda_stream) {
  if (!out) return fail(SHAKEN_E_INVAL, "out is NULL");
  shaken_batch* b = new shaken_batch();
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  *out = b;
  return SHAKEN_OK;
}

shaken_status shaken_batch_add(shaken_batch* b, shaken_ctx* ctx) {
  if (!b || !ctx) return fail(SHAKEN_E_INVAL, "NULL argument");
  if (ctx->owner) return fail(SHAKEN_E_STATE, "context already belongs to a batch");
  CU(cudaStreamSynchronize(ctx->stream));
  ctx->owner = b;
  b->plan.members.push_back(ctx);
  b->plan.invalidate();
  return SHAKEN_OK;
}

shaken_status shaken_batch_remove(shaken_batch* b, shaken_ctx* ctx) {
  if (!b || !ctx) return fail(SHAKEN_E_INVAL, "NULL argument");
  if (ctx->owner != b) return fail(SHAKEN_E_STATE, "context is not a member");
  CU(cudaStreamSynchronize(b->stream));
  auto& M = b->plan.members;
  M.erase(std::remove(M.begin(), M.end(), ctx), M.end());
  ctx->owner = nullptr;
  b->plan.invalidate();
  return SHAKEN_OK;
}

shaken_status shaken_batch_step(shaken_batch* b, uint64_t n_steps, int use_graph) {
  if (!b) return fail(SHAKEN_E_INVAL, "batch is NULL");
  if (b->plan.members.empty() || n_steps == 0) return SHAKEN_OK;
  for (shaken_ctx* c : b->plan.members) TRY(check_steps(c, n_steps));
  uint64_t nl = 0;
  shaken_status s = plan_run(b->plan, b->stream, n_steps, use_graph != 0, &nl);
  b->launches += nl;
  if (s != SHAKEN_OK) return s;
  for (shaken_ctx* c : b->plan.members) c->host_step += n_steps;
  return SHAKEN_OK;
}

shaken_status shaken_batch_sync(shaken_batch* b) {
  if (!b) return fail(SHAKEN_E_INVAL, "batch is NULL");
  CU(cudaStreamSynchronize(b->stream));
  return SHAKEN_OK;
}

void shaken_batch_free(shaken_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (shaken_ctx* c : b->plan.members) c->owner = nullptr;
  delete b;
}

shaken_status shaken_batch_set_autotune(shaken_batch* b, int on) {
  if (!b) return fail(SHAKEN_E_INVAL, "NULL batch");
  b->plan.autotune = on != 0;
  b->plan.invalidate();
  return SHAKEN_OK;
}

shaken_status shaken_batch_set_lattice_shape(shaken_batch* b, int encoding, int words_per_thread,
                                             int blocks_per_sm) {
  if (!b || encoding < 0 || encoding > 2) return fail(SHAKEN_E_INVAL, "bad batch or encoding");
  if (words_per_thread == 0) {  // back to the tuner
    b->plan.pinned[encoding][0] = b->plan.pinned[encoding][1] = 0;
  } else {
    if (words_per_thread != 1 && words_per_thread != shk::kWordsPerThread)
      return fail(SHAKEN_E_INVAL, "words per thread must be 1 or 4");
    const int occ = shk::lattice_blocks_per_sm(words_per_thread);
    if (blocks_per_sm < 1 || blocks_per_sm > occ)
      return fail(SHAKEN_E_INVAL, "blocks per SM must be in [1, " + std::to_string(occ) + "]");
    b->plan.pinned[encoding][0] = words_per_thread;
    b->plan.pinned[encoding][1] = blocks_per_sm == occ ? 0 : blocks_per_sm;
  }
  b->plan.invalidate();
  return SHAKEN_OK;
}

shaken_status shaken_set_autotune(shaken_ctx* ctx, int on) {
  if (!ctx) return fail(SHAKEN_E_INVAL, "NULL context");
  ctx->solo.autotune = on != 0;
  ctx->solo.invalidate();
  return SHAKEN_OK;
}

static shaken_status plan_lattice_wpt(Plan& P, cudaStream_t st, int enc, int* wpt) {
  if (!wpt || enc < 0 || enc > 2) return fail(SHAKEN_E_INVAL, "bad encoding or NULL output");
  if (P.dirty) TRY(build_plan(P, st));
  *wpt = 0;
  for (auto& F : P.fams)
    if (F->kind == 0 && F->enc == enc) *wpt = F->wpt;
  return SHAKEN_OK;
}

shaken_status shaken_batch_lattice_wpt(shaken_batch* b, int encoding, int* words_per_thread) {
  if (!b) return fail(SHAKEN_E_INVAL, "NULL batch");
  return plan_lattice_wpt(b->plan, b->stream, encoding, words_per_thread);
}

shaken_status shaken_lattice_wpt(shaken_ctx* ctx, int* words_per_thread) {
  if (!ctx) return fail(SHAKEN_E_INVAL, "NULL context");
  if (ctx->kind != SHAKEN_LATTICE) return fail(SHAKEN_E_INVAL, "not a lattice context");
  if (ctx->owner) return fail(SHAKEN_E_STATE, "context belongs to a batch");
  return plan_lattice_wpt(ctx->solo, ctx->stream, ctx->enc, words_per_thread);
}

static shaken_status plan_lattice_shape(Plan& P, cudaStream_t st, int enc, int* wpt, int* bps) {
  if (!wpt || !bps || enc < 0 || enc > 2) return fail(SHAKEN_E_INVAL, "bad encoding or NULL output");
  if (P.dirty) TRY(build_plan(P, st));
  *wpt = 0;
  *bps = 0;
  for (auto& F : P.fams)
    if (F->kind == 0 && F->enc == enc) {
      *wpt = F->wpt;
      *bps = F->bps > 0 ? F->bps : shk::lattice_blocks_per_sm(F->wpt);
    }
  return SHAKEN_OK;
}

shaken_status shaken_batch_lattice_shape(shaken_batch* b, int encoding, int* words_per_thread,
                                         int* blocks_per_sm) {
  if (!b) return fail(SHAKEN_E_INVAL, "NULL batch");
  return plan_lattice_shape(b->plan, b->stream, encoding, words_per_thread, blocks_per_sm);
}

shaken_status shaken_autotune_stats(uint64_t* trials, uint64_t* cached) {
  if (!trials || !cached) return fail(SHAKEN_E_INVAL, "NULL argument");
  *trials = g_tune_trials.load();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  *cached = (uint64_t)g_tune.size();
  return SHAKEN_OK;
}

shaken_status shaken_autotune_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
  return SHAKEN_OK;
}

shaken_status shaken_batch_set_timing(shaken_batch* b, int on) {
  if (!b) return fail(SHAKEN_E_INVAL, "batch is NULL");
  CU(cudaStreamSynchronize(b->stream));
  b->plan.collect();
  if (on < 0) return fail(SHAKEN_E_INVAL, "timing stride must be >= 0");
  b->plan.timing = on;
  b->plan.steps_issued = 0;
  b->plan.timed_ms = 0.0;
  b->plan.timed_n = 0;
  return SHAKEN_OK;
}

shaken_status shaken_batch_kernel_time(shaken_batch* b, double* ms, uint64_t* launches) {
  if (!b) return fail(SHAKEN_E_INVAL, "batch is NULL");
  CU(cudaStreamSynchronize(b->stream));
  b->plan.collect();
  if (ms) *ms = b->plan.timed_ms;
  if (launches) *launches = b->plan.timed_n;
  return SHAKEN_OK;
}

shaken_status shaken_batch_set_rng_counter(shaken_batch* b, uint64_t* device_counter) {
  if (!b) return fail(SHAKEN_E_INVAL, "batch is NULL");
  CU(cudaStreamSynchronize(b->stream));
  b->plan.rng_counter = reinterpret_cast<unsigned long long*>(device_counter);
  b->plan.drop_graph();
  return SHAKEN_OK;
}

shaken_status shaken_microbench(int kind, double* rate, double* ms) {
  if (!rate) return fail(SHAKEN_E_INVAL, "rate is NULL");
  if (kind < 0 || kind > 7) return fail(SHAKEN_E_INVAL, "unknown microbenchmark kind");
  CU(shk::run_microbench(kind, rate, ms));
  return SHAKEN_OK;
}

shaken_status shaken_batch_launch_count(shaken_batch* b, uint64_t* count) {
  if (!b || !count) return fail(SHAKEN_E_INVAL, "NULL argument");
  *count = b->launches.load();
  return SHAKEN_OK;
}

// ============================================================================ C ABI: primitives
shaken_status shaken_philox_device(uint64_t seed, const uint32_t* ctr, uint32_t* out, int64_t n,
                                   void* cuda_stream) {
  if (n < 0 || (n > 0 && (!ctr || !out))) return fail(SHAKEN_E_INVAL, "bad argument");
  CU(shk::launch_philox(seed, ctr, out, n, static_cast<cudaStream_t>(cuda_stream)));
  return SHAKEN_OK;
}

shaken_status shaken_threshold_device(const double* h, const double* beta, uint64_t* out,
                                      int64_t n, void* cuda_stream) {
  if (n < 0 || (n > 0 && (!h || !beta || !out))) return fail(SHAKEN_E_INVAL, "bad argument");
  CU(shk::launch_threshold(h, beta, out, n, static_cast<cudaStream_t>(cuda_stream)));
  return SHAKEN_OK;
}

const char* shaken_strerror(shaken_status s) {
  switch (s) {
    case SHAKEN_OK: return "ok";
    case SHAKEN_E_INVAL: return "invalid argument";
    case SHAKEN_E_NOMEM: return "out of memory";
    case SHAKEN_E_CUDA: return "CUDA error";
    case SHAKEN_E_TIMEOUT: return "timeout";
    case SHAKEN_E_STATE: return "invalid state";
    case SHAKEN_E_BUDGET: return "over device-memory budget";
  }
  return "unknown status";
}

const char* shaken_last_error(void) { return g_last_error.c_str(); }

const char* shaken_version(void) { return "libshaken 0.1 (sm_103a)"; }

}  // extern "C"

// ============================================================================ server
// Continuous batching of annealing jobs.  A worker thread owns every device
// call of the server: it admits queued jobs while their device state fits the
// budget and the running set's work per step (site updates, 2 n R per job) stays
// under a cap, steps all running jobs together in chunks of chunk_steps (each
// job stops exactly at its own last step: the kernels skip a context once its
// step reaches t_end), and retires finished jobs.  The cap bounds the work in
// flight, so under overload the queue grows while jobs keep completing at the
// GPU's rate instead of every admitted job slowing down together.  Admission
// order: arrival order, first fit (a job that does not fit is passed over by
// later ones that do, at most kServerMaxSkips times, then the queue waits for
// it), or shortest total work first.
struct ServerJob {
  int64_t id = 0;
  std::unique_ptr<shaken_ctx> prepared;  // host-prepared context (device set-up in the worker)
  HostPrep hp;
  std::vector<double> sched;
  uint64_t seed = 0, n_steps = 0;
  size_t bytes = 0;
  double step_work = 0.0;  // site updates per full step: 2 n R
  int skips = 0;           // times a later job was admitted before this one
  int state = 0;  // 0 queued, 1 running, 2 done, 3 failed
  std::vector<uint8_t> final_state;  // raw sigma at retirement (keep_states)
  shaken_ctx* ctx = nullptr;
  double t_submit = 0, t_admit = 0, t_done = 0;
  std::vector<shaken_obs> result;
  std::string error;
};

static constexpr int kServerMaxSkips = 8;

struct shaken_server {
  size_t budget = 0, used = 0;
  double work_cap = 3e8;    // site updates per step of the running set
  double work = 0.0;        // of the running jobs
  int order = 0;            // 0 arrival order (first fit, aging), 1 shortest total work first
  bool keep_states = false;
  uint32_t chunk = 64;
  cudaStream_t stream = nullptr;
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::deque<int64_t> queue;
  std::map<int64_t, std::unique_ptr<ServerJob>> jobs;
  std::vector<ServerJob*> running;
  shaken_batch batch;
  int64_t next_id = 0;
  int64_t n_done = 0;
  double updates = 0.0;
  bool stop = false;
  std::thread worker;
  std::chrono::steady_clock::time_point t0;
  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

static size_t job_bytes(const shaken_problem* p) {
  const int64_t N = p->kind == SHAKEN_LATTICE ? p->L * p->L : p->n;
  size_t b = 2 * (size_t)(p->replicas / 32) * N * 4;  // A, B
  if (p->kind == SHAKEN_GRAPH) {
    b += 2 * (size_t)(N + 1) * 4 + 2 * (size_t)p->m * 4;  // CSR
    b += 2 * (size_t)N * 16;                                // visiting orders
    if (!p->J_is_integer) b += 2 * (size_t)p->m * 4;
    if (p->lambda) b += (size_t)N * 4;
    if (p->frozen_mask) b += (size_t)N * 4;
  }
  b += (size_t)p->replicas * (2 * kNumSums * 8 + 16 + 8);
  return b + 4096;
}

// Next queued job to admit (an iterator into s->queue), or end() if none fits now.
static std::deque<int64_t>::iterator server_pick(shaken_server* s) {
  auto fits = [&](const ServerJob* j) {
    if (s->running.empty()) return true;  // a job larger than the caps runs alone
    return s->used + j->bytes <= s->budget && s->work + j->step_work <= s->work_cap;
  };
  auto& Q = s->queue;
  if (s->order == 1) {  // shortest total work first
    auto best = Q.end();
    double bw = 0.0;
    for (auto it = Q.begin(); it != Q.end(); ++it) {
      const ServerJob* j = s->jobs[*it].get();
      const double w = j->step_work * (double)j->n_steps;
      if (fits(j) && (best == Q.end() || w < bw)) {
        best = it;
        bw = w;
      }
    }
    return best;
  }
  for (auto it = Q.begin(); it != Q.end(); ++it) {  // arrival order, first fit
    const ServerJob* j = s->jobs[*it].get();
    if (fits(j)) return it;
    if (j->skips >= kServerMaxSkips) return Q.end();  // the queue waits for this job
  }
  return Q.end();
}

static void server_loop(shaken_server* s) {
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    // admit
    while (!s->queue.empty()) {
      auto it = server_pick(s);
      if (it == s->queue.end()) break;
      for (auto jt = s->queue.begin(); jt != it; ++jt) s->jobs[*jt]->skips++;
      ServerJob* j = s->jobs[*it].get();
      s->queue.erase(it);
      lk.unlock();
      shaken_ctx* c = j->prepared.release();
      c->stream = s->stream;
      shaken_status st = setup_ctx(c, j->hp);
      j->hp = HostPrep();  // host copies are on the device now
      if (st == SHAKEN_OK) {
        c->owner = &s->batch;
        st = begin_anneal(c, j->sched.data(), j->n_steps);
        c->hcd.t_end = (uint32_t)j->n_steps;
        if (st == SHAKEN_OK) st = push_cd(c);
      }
      lk.lock();
      if (st != SHAKEN_OK) {
        j->state = 3;
        j->error = g_last_error;
        if (c) {
          c->owner = nullptr;
          shaken_free(c);
        }
        s->n_done++;
        s->done_cv.notify_all();
        continue;
      }
      j->ctx = c;
      j->state = 1;
      j->t_admit = s->now();
      s->used += j->bytes;
      s->work += j->step_work;
      s->running.push_back(j);
      s->batch.plan.members.push_back(c);
      s->batch.plan.invalidate();
    }
    if (s->stop) break;  // freeing the server cancels queued and running jobs
    if (s->running.empty()) {
      s->cv.wait_for(lk, std::chrono::milliseconds(2));
      if (s->stop && s->queue.empty()) break;
      continue;
    }
    // step every running job one chunk
    uint64_t chunk = s->chunk;
    lk.unlock();
    uint64_t nl = 0;
    shaken_status st = plan_run(s->batch.plan, s->stream, chunk, true, &nl);
    if (st == SHAKEN_OK) {
      cudaError_t e = cudaStreamSynchronize(s->stream);
      if (e != cudaSuccess) st = fail(SHAKEN_E_CUDA, cudaGetErrorString(e));
    }
    lk.lock();
    s->batch.launches += nl;
    std::vector<ServerJob*> still;
    for (ServerJob* j : s->running) {
      shaken_ctx* c = j->ctx;
      const uint64_t before = c->host_step;
      c->host_step = std::min<uint64_t>(c->host_step + chunk, j->n_steps);
      s->updates += 2.0 * (double)(c->host_step - before) * (double)c->R * (double)c->sites();
      if (st != SHAKEN_OK || c->host_step >= j->n_steps) {
        j->result.resize(c->R);
        const bool keep = s->keep_states;
        lk.unlock();
        shaken_status so = st == SHAKEN_OK ? shaken_observables(c, j->result.data()) : st;
        if (so == SHAKEN_OK && keep) {
          j->final_state.resize(c->spin_bytes);
          so = shaken_get_state_raw(c, j->final_state.data(), c->spin_bytes);
        }
        lk.lock();
        j->state = so == SHAKEN_OK ? 2 : 3;
        if (so != SHAKEN_OK) j->error = g_last_error;
        j->t_done = s->now();
        auto& M = s->batch.plan.members;
        M.erase(std::remove(M.begin(), M.end(), c), M.end());
        s->batch.plan.invalidate();
        c->owner = nullptr;
        shaken_free(c);
        j->ctx = nullptr;
        s->used -= j->bytes;
        s->work -= j->step_work;
        s->n_done++;
        s->done_cv.notify_all();
      } else {
        still.push_back(j);
      }
    }
    s->running.swap(still);
  }
}

extern "C" {

shaken_status shaken_server_create(shaken_server** out, size_t hbm_budget_bytes,
                                   uint32_t chunk_steps, void* cuda_stream) {
  if (!out || hbm_budget_bytes == 0 || chunk_steps == 0)
    return fail(SHAKEN_E_INVAL, "bad argument");
  shaken_server* s = new shaken_server();
  s->budget = hbm_budget_bytes;
  s->chunk = chunk_steps;
  s->stream = static_cast<cudaStream_t>(cuda_stream);
  s->batch.stream = s->stream;
  s->t0 = std::chrono::steady_clock::now();
  s->worker = std::thread(server_loop, s);
  *out = s;
  return SHAKEN_OK;
}

shaken_status shaken_server_submit(shaken_server* s, const shaken_problem* p, uint64_t seed,
                                   const double* beta_schedule, uint64_t n_steps,
                                   int64_t* job_id) {
  if (!s || !p || !beta_schedule || !job_id || n_steps == 0)
    return fail(SHAKEN_E_INVAL, "bad argument");
  if (n_steps >= 0xFFFFFFFEull) return fail(SHAKEN_E_INVAL, "too many steps");
  for (uint64_t k = 0; k < n_steps; ++k)
    if (!std::isfinite(beta_schedule[k]) || beta_schedule[k] < 0.0)
      return fail(SHAKEN_E_INVAL, "beta_schedule must be finite and >= 0");
  auto j = std::make_unique<ServerJob>();
  // validation, orientation and CSR on the submitting thread
  TRY(prepare_ctx(p, seed, s->stream, j->prepared, j->hp));
  j->sched.assign(beta_schedule, beta_schedule + n_steps);
  j->seed = seed;
  j->n_steps = n_steps;
  j->bytes = job_bytes(p);
  j->step_work = 2.0 * (double)j->prepared->R * (double)j->prepared->sites();
  if (j->bytes > s->budget) return fail(SHAKEN_E_BUDGET, "job exceeds the device-memory budget");
  std::lock_guard<std::mutex> lk(s->mu);
  j->id = s->next_id++;
  j->t_submit = s->now();
  *job_id = j->id;
  s->queue.push_back(j->id);
  s->jobs[j->id] = std::move(j);
  s->cv.notify_all();
  return SHAKEN_OK;
}

shaken_status shaken_server_set_policy(shaken_server* s, double max_step_updates, int order,
                                       int keep_states) {
  if (!s || !(max_step_updates > 0.0) || (order != 0 && order != 1))
    return fail(SHAKEN_E_INVAL, "bad argument");
  std::lock_guard<std::mutex> lk(s->mu);
  s->work_cap = max_step_updates;
  s->order = order;
  s->keep_states = keep_states != 0;
  s->cv.notify_all();
  return SHAKEN_OK;
}

shaken_status shaken_server_queue(shaken_server* s, int64_t* queued, int64_t* running) {
  if (!s) return fail(SHAKEN_E_INVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (queued) *queued = (int64_t)s->queue.size();
  if (running) *running = (int64_t)s->running.size();
  return SHAKEN_OK;
}

shaken_status shaken_server_result_state(shaken_server* s, int64_t job_id, void* host_words,
                                         size_t bytes) {
  if (!s || !host_words) return fail(SHAKEN_E_INVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return fail(SHAKEN_E_INVAL, "unknown job");
  ServerJob* j = it->second.get();
  if (j->state != 2) return fail(SHAKEN_E_STATE, "job not finished");
  if (j->final_state.empty()) return fail(SHAKEN_E_STATE, "final states are not kept");
  if (bytes != j->final_state.size()) return fail(SHAKEN_E_INVAL, "state size mismatch");
  std::memcpy(host_words, j->final_state.data(), bytes);
  return SHAKEN_OK;
}

shaken_status shaken_server_poll(shaken_server* s, int64_t job_id, int* state) {
  if (!s || !state) return fail(SHAKEN_E_INVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return fail(SHAKEN_E_INVAL, "unknown job");
  *state = it->second->state;
  return SHAKEN_OK;
}

shaken_status shaken_server_result(shaken_server* s, int64_t job_id, shaken_obs* out,
                                   double* t_admit, double* t_done) {
  if (!s) return fail(SHAKEN_E_INVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return fail(SHAKEN_E_INVAL, "unknown job");
  ServerJob* j = it->second.get();
  if (j->state == 3) return fail(SHAKEN_E_CUDA, "job failed: " + j->error);
  if (j->state != 2) return fail(SHAKEN_E_STATE, "job not finished");
  if (out) std::copy(j->result.begin(), j->result.end(), out);
  if (t_admit) *t_admit = j->t_admit;
  if (t_done) *t_done = j->t_done;
  return SHAKEN_OK;
}

shaken_status shaken_server_drain(shaken_server* s, double timeout_s) {
  if (!s) return fail(SHAKEN_E_INVAL, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::microseconds((int64_t)(timeout_s * 1e6));
  while (s->n_done < (int64_t)s->jobs.size()) {
    if (s->done_cv.wait_until(lk, deadline) == std::cv_status::timeout &&
        s->n_done < (int64_t)s->jobs.size())
      return fail(SHAKEN_E_TIMEOUT, "server drain timed out");
  }
  return SHAKEN_OK;
}

shaken_status shaken_server_stats(shaken_server* s, double* site_updates, uint64_t* launches,
                                  int64_t* jobs_done) {
  if (!s) return fail(SHAKEN_E_INVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (site_updates) *site_updates = s->updates;
  if (launches) *launches = s->batch.launches.load();
  if (jobs_done) *jobs_done = s->n_done;
  return SHAKEN_OK;
}

void shaken_server_free(shaken_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->queue.clear();
    for (auto& kv : s->jobs)
      if (kv.second->state == 0) kv.second->state = 3;
    s->cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  for (ServerJob* j : s->running) {
    if (j->ctx) {
      j->ctx->owner = nullptr;
      shaken_free(j->ctx);
    }
  }
  delete s;
}

}  // extern "C"
