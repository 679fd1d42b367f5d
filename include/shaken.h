/*
 * shaken.h -- C ABI of libshaken, a GB300 (sm_103a) implementation of the
 * per-half-step parallel update of the shaken dynamics of
 *   Apollonio, D'Autilia, Scoppola, Scoppola, Troiani,
 *   "Shaken dynamics: an easy way to parallel Markov Chain Monte Carlo",
 *   arXiv:1904.06257.
 *
 * Conventions (every entry point):
 *   - Returns a shaken_status; nothing throws across the ABI.  On error the
 *     context is left as it was before the call unless stated otherwise, and
 *     shaken_last_error() returns a one-line description (thread-local).
 *   - All pointers in shaken_problem and all result arrays are HOST memory,
 *     owned by the caller.  shaken_init deep-copies every input; nothing the
 *     caller passes is referenced after a call returns.
 *   - Device memory is allocated and owned by the library (cudaMalloc) and is
 *     released by shaken_free / shaken_batch_free / shaken_server_free.
 *   - A context is used by one host thread at a time; distinct contexts are
 *     independent.  Work is issued on the CUDA stream given at creation
 *     (borrowed, never destroyed; NULL = the legacy default stream).  Calls
 *     that return host data synchronise that stream.
 *   - Spins are +1 / -1.  Lattice site x = (i, j), i = row, index i*L + j.
 *   - "Step" means one full shaken step P^sh = P^{1->2} then P^{2->1}
 *     (Sec. 2; on the lattice P^dl then P^ur, Sec. 3).
 */
#ifndef SHAKEN_H
#define SHAKEN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct shaken_ctx shaken_ctx;
typedef struct shaken_batch shaken_batch;
typedef struct shaken_server shaken_server;

typedef enum {
  SHAKEN_OK = 0,
  SHAKEN_E_INVAL = -1,   /* invalid argument or problem (message in shaken_last_error) */
  SHAKEN_E_NOMEM = -2,   /* device or host allocation failed */
  SHAKEN_E_CUDA = -3,    /* a CUDA runtime call failed */
  SHAKEN_E_TIMEOUT = -4, /* a bounded wait gave up */
  SHAKEN_E_STATE = -5,   /* call not valid in the current state */
  SHAKEN_E_BUDGET = -6   /* request exceeds the server's device-memory budget */
} shaken_status;

enum { SHAKEN_LATTICE = 0, SHAKEN_GRAPH = 1 };

/* Spin encodings.
 *   INT8      lattice only: int8 [R][L][L] (+1/-1 bytes).
 *   PACKED    lattice only: uint32 [R][L][L/32], bit k of word (i, w) = site (i, 32w+k).
 *   MULTISPIN lattice: uint32 [R/32][L][L] (group g's lattice, then group g+1's);
 *             graph: uint32 [n][R/32] (the group words of a vertex adjacent); bit k
 *             of the word of group g = replica 32g+k.
 * INT8 and PACKED give bit-identical trajectories (same random stream). */
enum { SHAKEN_INT8 = 0, SHAKEN_PACKED = 1, SHAKEN_MULTISPIN = 2 };

enum { SHAKEN_INIT_RANDOM = 0, SHAKEN_INIT_PLUS = 1, SHAKEN_INIT_MINUS = 2, SHAKEN_INIT_GIVEN = 3 };

/* Orientation E^o of an undirected graph (Sec. 2, construction of the doubling
 * graph from an arbitrary orientation): MIN_MAX orients {u,v} from the smaller
 * to the larger index; GIVEN keeps (u[e] -> v[e]).  Feeding the lattice edges
 * (x -> x_up), (x -> x_right) with GIVEN reproduces the lattice fields. */
enum { SHAKEN_ORIENT_MIN_MAX = 0, SHAKEN_ORIENT_GIVEN = 2 };

/* Problem statement (Sec. 2: G = (V, E), J, lambda, q > 0, beta; Sec. 3: the
 * L x L torus with J constant and a frozen set B where sigma = +1).
 * H(sigma) = -sum_{e} J_e s_x s_y - 2 sum_x lambda_x s_x   (Eq. (ham1)). */
typedef struct {
  int32_t kind;           /* SHAKEN_LATTICE or SHAKEN_GRAPH */
  int32_t encoding;       /* lattice: INT8 / PACKED / MULTISPIN; graph: MULTISPIN */
  int64_t L;              /* lattice side; L % 32 == 0, 32 <= L <= 65536 */
  int32_t boundary;       /* lattice: 0 periodic torus, 1 frozen set (mask, or if the mask
                             is NULL the default B = row 0 and column 0) */
  const uint8_t* frozen_mask; /* optional [n] (n = L*L or graph n): nonzero = frozen at +1 */
  int64_t n;              /* graph: vertices, 1 <= n < 2^31 */
  int64_t m;              /* graph: undirected edges {u[e], v[e]}, u != v */
  const int32_t* u;
  const int32_t* v;
  const float* J_edge;    /* graph: coupling per edge */
  int32_t J_is_integer;   /* graph: 1 if every J_edge is +1 or -1 (exact integer path) */
  int32_t orientation;    /* graph: SHAKEN_ORIENT_* */
  double J;               /* lattice: coupling */
  const float* lambda;    /* optional per-vertex field [n]; NULL -> lambda_const */
  double lambda_const;
  double q;               /* self-interaction, q > 0 (Sec. 2) */
  int32_t replicas;       /* R >= 1; MULTISPIN needs R % 32 == 0 */
  const double* beta;     /* [R] inverse temperature per replica, >= 0 */
  int32_t init;           /* SHAKEN_INIT_* */
  const int8_t* init_spins; /* INIT_GIVEN: [R][n] of +1/-1 */
} shaken_problem;

/* Observables of one replica.  sigma = current configuration (after the last
 * full step), sigma' = the configuration of the last half step (before any
 * step: sigma' = sigma).
 *   magnetization = (1/|V|) sum_x sigma_x
 *   energy        = H(sigma), Eq. (ham1) (lattice: Eq. (HGibbs), field 2 lambda)
 *   pair_energy   = H(sigma, sigma'), Eq. (ham21) -- the doubled Hamiltonian
 *                   of Def. 2.2 on the pair (sigma^(1), sigma^(2)) = (sigma, sigma')
 *   best_energy   = min of H over the full-step configurations evaluated so far
 *                   (every step while tracking is on, and at every observables
 *                   call), best_step its step index (the lower bound of Thm 6.1
 *                   is min pair_energy + q|V|)
 *   cut_edges     = #{ {x,y} in E : sigma_x != sigma_y }
 *   cut_weight    = sum over those edges of -J_e  (max-cut <-> min H at lambda = 0) */
typedef struct {
  double magnetization;
  double energy;
  double pair_energy;
  double best_energy;
  int64_t best_step;
  int64_t cut_edges;
  double cut_weight;
} shaken_obs;

/* Create a context: validates and deep-copies the problem, builds the oriented
 * in/out CSR of a graph (Sec. 2), the heat-bath threshold tables, allocates the
 * double-buffered device spin state and initialises it (random: sigma = +1 iff
 * the draw of step 0xFFFFFFFF, half 0 is < 2^31; frozen sites +1).
 * seed keys the Philox-4x32-10 stream: key = (seed low word, seed high word).
 * Errors: E_INVAL (bad sizes, q <= 0, NaN/inf inputs, L or R not allowed by the
 * encoding, self-loops, vertex ids out of range), E_NOMEM, E_CUDA.
 * On error *out is set to NULL. */
shaken_status shaken_init(shaken_ctx** out, const shaken_problem* p, uint64_t seed,
                          void* cuda_stream);

/* Release all device and host memory of the context (NULL is a no-op). */
void shaken_free(shaken_ctx* ctx);

/* Run n full steps (Sec. 2: P^sh = P^{1->2} P^{2->1}; Sec. 3: P^dl then P^ur).
 * In each half step every non-frozen spin is resampled at once from the other
 * buffer: tau_x = +1 with probability e^{beta h_x} / (2 cosh(beta h_x)), decided
 * exactly as u < floor(2^32 / (1 + e^{-2 beta h})) with u the replica's 32-bit
 * Philox draw for (seed, replica, step, half, site).  Asynchronous on the
 * context's stream, except whole-run paths that synchronise at the end of the
 * call: small lattices (<= 4096 lane words per replica, n >= 4) run in one
 * launch per 65536 steps with the state in shared memory; one mid-size
 * INT8/PACKED lattice (one replica, n >= 8, no tracking or anneal) runs in one
 * cooperative launch per 65536 steps holding row bands in shared memory
 * (neighbouring bands pass one boundary row per half step), and returns
 * E_TIMEOUT if a wait for a neighbour's row or at the final grid barrier ran
 * out (the chunk is then not applied: sigma, sigma' and the step counter stay
 * as before it).  Every path
 * gives the same trajectory.  E_STATE if the context is owned by a batch. */
shaken_status shaken_step(shaken_ctx* ctx, uint64_t n_steps);

/* Annealing (the optimisation use of Sec. 6 / Thm 6.1): n_steps full steps,
 * step k using beta_schedule[k] (host, n_steps values, >= 0) for every
 * replica; best-energy tracking is on for these steps.  After the call the
 * per-replica beta reverts to the one given at init. */
shaken_status shaken_anneal(shaken_ctx* ctx, const double* beta_schedule, uint64_t n_steps);

/* Order of the two half steps within a step: 0 (default) P^{1->2} then P^{2->1}
 * (on the lattice P^dl then P^ur, Sec. 3); 1 the reversed chain P^{sh'} = P^ur then
 * P^dl (Sec. 3, end), i.e. out-neighbour fields first.  The draw of an update is
 * keyed by its type (dl / 1->2 = half 0, ur / 2->1 = half 1), not by its position.
 * observables' pair energy stays H(sigma, sigma') of Eq. (ham21) with sigma' the
 * configuration after the first half step of the last step. */
shaken_status shaken_set_order(shaken_ctx* ctx, int reversed);

/* Turn per-step best-energy tracking on (1) or off (0) for shaken_step.
 * Tracking evaluates H(sigma_t) of every full-step configuration; on INT8 and
 * PACKED lattices it is fused into the first half step. */
shaken_status shaken_set_tracking(shaken_ctx* ctx, int enable);

/* Run n steps and record, for each step k, the magnetization and energy of the
 * configuration at the START of that step (sigma_{t0+k}).  mag and energy are
 * host arrays [n_steps][R]; either may be NULL.  Synchronises. */
shaken_status shaken_step_record(shaken_ctx* ctx, uint64_t n_steps, double* mag, double* energy);

/* Observables of every replica into out[R] (host).  Synchronises. */
shaken_status shaken_observables(shaken_ctx* ctx, shaken_obs* out);

/* Copy the current configuration sigma to host out[R][n] as int8 +1/-1.
 * Synchronises. */
shaken_status shaken_get_spins(shaken_ctx* ctx, int8_t* out);

/* Copy sigma' -- the configuration after the first half step of the last full
 * step (Sec. 2: sigma^(2) of the pair (sigma^(1), sigma^(2)) the half steps
 * alternate; before any step sigma' = sigma) -- to host out[R][n] as int8
 * +1/-1.  With the default order sigma' = P^{1->2} applied to the previous
 * sigma; reversed order (shaken_set_order): P^{2->1}.  Synchronises. */
shaken_status shaken_get_spins_prime(shaken_ctx* ctx, int8_t* out);

/* Replace sigma (and sigma') by host in[R][n] (+1/-1; frozen sites must be
 * +1, else E_INVAL).  Does not change the step counter. */
shaken_status shaken_set_spins(shaken_ctx* ctx, const int8_t* in);

/* Raw device-encoded state (the layout of the context's encoding, see the
 * enum above): bytes must equal shaken_state_bytes().  Sets or reads sigma
 * (set also copies it into sigma').  No conversion on the host: this is the
 * fast path for callers that keep packed states. */
shaken_status shaken_state_bytes(shaken_ctx* ctx, size_t* bytes);
shaken_status shaken_set_state_raw(shaken_ctx* ctx, const void* host_words, size_t bytes);
shaken_status shaken_get_state_raw(shaken_ctx* ctx, void* host_words, size_t bytes);
/* As shaken_get_state_raw, without waiting: the copy of sigma is enqueued on the
 * context's stream (the batch's stream for a member) and host_words (pinned
 * memory for a truly asynchronous copy) holds it after the next shaken_sync,
 * shaken_batch_sync or other synchronising call on that stream.  The caller
 * keeps host_words alive until then. */
shaken_status shaken_get_state_raw_async(shaken_ctx* ctx, void* host_words, size_t bytes);

/* Current step counter t (number of full steps taken since init or load). */
shaken_status shaken_get_step(shaken_ctx* ctx, uint64_t* t);

/* Checkpoint: state = (sigma, sigma', step, best energies, tracking flag).
 * With buf == NULL, *len receives the size needed.  Because the random stream
 * is counter-based, resuming from a checkpoint reproduces the uninterrupted
 * run bit for bit.  shaken_load needs a context created from the same problem. */
shaken_status shaken_save(shaken_ctx* ctx, void* buf, size_t* len);
shaken_status shaken_load(shaken_ctx* ctx, const void* buf, size_t len);

/* Local fields h_x of the next half step (half 0: h^{1->2} from sigma; half 1:
 * h^{2->1} from sigma') as computed by the update kernels, into host
 * out[R][n] (float).  A diagnostic for field parity.  Synchronises. */
shaken_status shaken_debug_fields(shaken_ctx* ctx, int half, float* out);

/* Diagnostics: with on != 0 the integer-coupling graph path decides every
 * lane with the fp64 threshold instead of the fp32 fast path (same results,
 * slower); used to test the fast path's error margin. */
shaken_status shaken_debug_exact_always(shaken_ctx* ctx, int on);

/* Diagnostics for the failure path of banded runs (one mid-size INT8/PACKED
 * lattice, chunks of >= 8 steps without tracking, held in shared memory by a
 * cooperative grid: neighbouring blocks pass one boundary row per half step and
 * all blocks meet at one grid barrier at the end of the chunk): the next banded
 * chunk starts with that barrier's arrival count preset so that no block is ever
 * the last to arrive.  Every block's wait then runs out after its bounded spin
 * (one second on the GPU's global timer), the blocks return without writing the
 * chunk back, and the stepping call returns SHAKEN_E_TIMEOUT with sigma, sigma'
 * and the step counter as before the chunk; the context stays usable.
 * The outcome of a banded chunk is settled by one atomic decision: either every
 * block passed the last barrier and the chunk is written back whole (the call
 * succeeds), or a block gave up first and no block writes anything back. */
shaken_status shaken_debug_band_stall(shaken_ctx* ctx);

/* Diagnostics for the same failure path: in the next banded chunk, block `block`
 * (0 <= block < grid; no effect if larger) gives up its wait at the last barrier
 * at once instead of after one second.  Depending on whether the other blocks had
 * all arrived, the call then either succeeds with the chunk applied or returns
 * SHAKEN_E_TIMEOUT with the state as before the chunk -- never a mixture. */
shaken_status shaken_debug_band_hurry(shaken_ctx* ctx, int block);

/* Number of kernel launches this context has issued (all kinds). */
shaken_status shaken_launch_count(shaken_ctx* ctx, uint64_t* count);

/* Wait for all work of the context's stream. */
shaken_status shaken_sync(shaken_ctx* ctx);

/* ------------------------------------------------------------------------ */
/* Batching: contexts of any kinds and sizes stepped together, one launch per */
/* half step and encoding family covering every member (uneven sizes are cut  */
/* into fixed tiles), optionally replayed from a captured CUDA graph.  Each   */
/* member's trajectory is bit-identical to stepping it alone.                 */
/* ------------------------------------------------------------------------ */

/* Create an empty batch issuing on cuda_stream. */
shaken_status shaken_batch_create(shaken_batch** out, void* cuda_stream);
/* Add a context (it must not belong to another batch).  The context's own
 * stream is no longer used while it is a member. */
shaken_status shaken_batch_add(shaken_batch* b, shaken_ctx* ctx);
/* Remove a member; waits for the batch's stream first. */
shaken_status shaken_batch_remove(shaken_batch* b, shaken_ctx* ctx);
/* Step every member n full steps.  With use_graph != 0 the launches of a
 * chunk of steps are captured once into a CUDA graph and replayed. */
shaken_status shaken_batch_step(shaken_batch* b, uint64_t n_steps, int use_graph);
shaken_status shaken_batch_sync(shaken_batch* b);
/* Observables of every member's replicas, as shaken_observables computes them,
 * into host out[sum of the members' R], members in the order they were added
 * (replica r of the k-th member at out[R_0 + ... + R_{k-1} + r]).  One
 * observables launch per encoding family covers all members; synchronises once
 * (so it also completes earlier asynchronous copies on the batch's stream). */
shaken_status shaken_batch_observables(shaken_batch* b, shaken_obs* out);
/* Raw states of all members in one transfer each way: the members' raw states
 * (shaken_state_bytes each, the layout of shaken_get_state_raw) concatenated in
 * member order; state_bytes gives the total.  set copies host -> device in one
 * copy and spreads it over the members' sigma and sigma' (a kernel), without
 * waiting; get gathers the members' sigma (a kernel) and copies it to host in one
 * copy, without waiting: host holds it after the next synchronising call on the
 * batch's stream (pinned memory for asynchronous copies; keep host alive and
 * unchanged until then).  bytes must equal the total, else E_INVAL. */
shaken_status shaken_batch_state_bytes(shaken_batch* b, size_t* bytes);
shaken_status shaken_batch_set_states_raw(shaken_batch* b, const void* host, size_t bytes);
shaken_status shaken_batch_get_states_raw_async(shaken_batch* b, void* host, size_t bytes);
/* Kernel timing: set_timing(b, n) with n > 0 brackets the half-step launches of
 * every n-th non-graph batch step (counted from this call; n = 1: every step)
 * by CUDA events on the batch stream, n = 0 switches timing off, n < 0 is
 * E_INVAL (the events cost device time themselves, so a stride keeps the
 * timed run close to an untimed one).  kernel_time syncs the stream and returns
 * the summed device time (ms) and the number of timed half-step launches since
 * timing was set; launch_count is the total number of kernels the batch has
 * launched. */
shaken_status shaken_batch_set_timing(shaken_batch* b, int on);
shaken_status shaken_batch_kernel_time(shaken_batch* b, double* ms, uint64_t* launches);
shaken_status shaken_batch_launch_count(shaken_batch* b, uint64_t* count);
/* RNG accounting: with a DEVICE counter set (non-NULL), every lattice
 * half-step launch of the batch adds to it the number of Philox-4x32-10 calls
 * it made (the bit-plane decision stops drawing once all 32 lanes of a word
 * are decided).  NULL switches counting off. */
shaken_status shaken_batch_set_rng_counter(shaken_batch* b, uint64_t* device_counter);

/* Autotuner of the lattice launch shape.  For every lattice encoding family of
 * a plan (a batch, or a context stepped on its own) the half-step kernel runs
 * with tiles of 256 lane words (one per thread) or 1024 (four per thread), and
 * with as many resident blocks per SM as fit or one fewer (each block then walks
 * a longer range of tiles).  With autotuning on (the default) a family of at
 * least one resident wave of 1024-word tiles is timed once in each of the four
 * shapes -- trial launches of the first half step that rewrite sigma' with the
 * values the real step writes, so no trajectory changes -- and the fastest shape
 * is cached per (encoding, bit length of the lane-word count, bit length of the
 * job count).  Off: a
 * fixed rule (four words per thread once the family fills eight waves).
 * Trajectories are bit-identical under every shape.
 * lattice_wpt returns the words per thread the plan uses for an encoding
 * (SHAKEN_INT8 / SHAKEN_PACKED / SHAKEN_MULTISPIN), 0 if the plan has no such
 * family; it builds the plan (and may run the trials) if needed.  A context
 * that belongs to a batch: SHAKEN_E_STATE.  autotune_stats: number of tuning
 * searches run and of cached results in this process; autotune_clear empties
 * the cache. */
shaken_status shaken_batch_set_autotune(shaken_batch* b, int on);
shaken_status shaken_set_autotune(shaken_ctx* ctx, int on);
shaken_status shaken_batch_lattice_wpt(shaken_batch* b, int encoding, int* words_per_thread);
shaken_status shaken_lattice_wpt(shaken_ctx* ctx, int* words_per_thread);
/* The full shape a batch plan uses for an encoding: lane words per thread and
 * resident blocks per SM of its half-step kernel (0, 0 if it has no such family). */
shaken_status shaken_batch_lattice_shape(shaken_batch* b, int encoding, int* words_per_thread,
                                         int* blocks_per_sm);
/* Pin the launch shape of a batch's family of an encoding (words per thread 1 or 4,
 * blocks per SM from 1 to as many as fit), overriding the tuner; words_per_thread
 * = 0 returns the family to the tuner.  Trajectories are the same in every shape.
 * E_INVAL for other values. */
shaken_status shaken_batch_set_lattice_shape(shaken_batch* b, int encoding, int words_per_thread,
                                             int blocks_per_sm);
shaken_status shaken_autotune_stats(uint64_t* trials, uint64_t* cached);
shaken_status shaken_autotune_clear(void);

/* Device microbenchmarks on the current GPU (all SMs, register-only work):
 * kind 0 = Philox-4x32-10 calls per second, 1 = 32-bit LOP3 per second,
 * 2 = 32-bit IMAD per second, 3 = LOP3 and IMAD interleaved (operations per
 * second, both kinds counted), 4 = 32 x 32 -> 64-bit multiply-adds per second,
 * 5 = 32 x 32 -> 64-bit products per second, 6 = products and LOP3
 * interleaved (operations per second, both kinds counted), 7 = Philox-4x32-10
 * calls per second with each product as separate high and low multiplies.
 * *rate receives the rate, *ms (optional) the timed duration.  Unknown kind:
 * SHAKEN_E_INVAL. */
shaken_status shaken_microbench(int kind, double* rate, double* ms);
void shaken_batch_free(shaken_batch* b);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of annealing jobs (Sec. 6: combinatorial      */
/* optimisation on arbitrary graphs).  A worker thread admits queued jobs     */
/* while their device state fits the memory budget, steps all admitted jobs  */
/* together in chunks, and retires finished jobs, freeing their memory for   */
/* the next ones.  Results are the same as running each job alone.            */
/* ------------------------------------------------------------------------ */

/* Create a server with a device-memory budget (bytes) for job state and a
 * chunk length (steps per batched launch sequence between admissions). */
shaken_status shaken_server_create(shaken_server** out, size_t hbm_budget_bytes,
                                   uint32_t chunk_steps, void* cuda_stream);
/* Queue an annealing job (copied).  beta_schedule[n_steps] (host).  Returns its
 * id.  E_BUDGET if the job alone exceeds the budget. */
shaken_status shaken_server_submit(shaken_server* s, const shaken_problem* p, uint64_t seed,
                                   const double* beta_schedule, uint64_t n_steps,
                                   int64_t* job_id);
/* Admission policy (no counterpart in the paper; serving is this library's own
 * use of the anneal).  Besides the memory budget, a queued job is admitted only
 * while the running jobs' work per full step -- the sum of 2 n R site updates --
 * stays at or below max_step_updates (default 3e8, about a millisecond of GPU work per
 * step); a job larger than the cap
 * runs when nothing else does.  Bounding the work in flight keeps the GPU's rate
 * on the running jobs, so under overload jobs keep completing while the queue
 * grows.  order 0 (default): arrival order, first fit -- a job that does not fit
 * is passed over by later jobs that do, at most 8 times, then admission waits for
 * it; order 1: shortest total work (2 n R steps) first.  keep_states != 0: the
 * final raw state of every finished job is kept on the host for
 * shaken_server_result_state.  E_INVAL for max_step_updates <= 0 or another order.
 * Takes effect at the next admission. */
shaken_status shaken_server_set_policy(shaken_server* s, double max_step_updates, int order,
                                       int keep_states);
/* *state: 0 queued, 1 running, 2 done. */
shaken_status shaken_server_poll(shaken_server* s, int64_t job_id, int* state);
/* Jobs waiting for admission and jobs running now (either may be NULL). */
shaken_status shaken_server_queue(shaken_server* s, int64_t* queued, int64_t* running);
/* Final raw state (sigma in the job's encoding, as shaken_get_state_raw) of a
 * finished job into host_words; bytes must equal its shaken_state_bytes.
 * E_STATE if the job is not finished or states are not kept (set_policy). */
shaken_status shaken_server_result_state(shaken_server* s, int64_t job_id, void* host_words,
                                         size_t bytes);
/* Observables of a finished job into out[R]; also its admission and completion
 * times (seconds since server creation, host steady clock) if non-NULL. */
shaken_status shaken_server_result(shaken_server* s, int64_t job_id, shaken_obs* out,
                                   double* t_admit, double* t_done);
/* Block until every submitted job is done or timeout_s elapses (E_TIMEOUT). */
shaken_status shaken_server_drain(shaken_server* s, double timeout_s);
/* Aggregate counters: site updates done, kernel launches, jobs done. */
shaken_status shaken_server_stats(shaken_server* s, double* site_updates, uint64_t* launches,
                                  int64_t* jobs_done);
/* Stop the worker after its current chunk, cancel queued and running jobs and
 * release their device memory. */
void shaken_server_free(shaken_server* s);

/* ------------------------------------------------------------------------ */
/* Stateless primitives (diagnostics and tests).                              */
/* ------------------------------------------------------------------------ */

/* Philox-4x32-10 (Salmon et al., SC'11) on the device for n counters:
 * out[4i..4i+3] = Philox(key, ctr[4i..4i+3]); ctr and out are DEVICE pointers. */
shaken_status shaken_philox_device(uint64_t seed, const uint32_t* ctr, uint32_t* out, int64_t n,
                                   void* cuda_stream);

/* Heat-bath thresholds T = floor(2^32 / (1 + e^{-2 beta h})) computed by the
 * device code path for n (h, beta) pairs; h, beta, out are DEVICE pointers. */
shaken_status shaken_threshold_device(const double* h, const double* beta, uint64_t* out,
                                      int64_t n, void* cuda_stream);

/* Observables of a lattice state held by the caller, computed without any
 * device or host allocation.  The paper has no counterpart: this exists for
 * callers that cannot call cudaMalloc -- code that manages all device memory
 * through its own pool or caching allocator, or that must avoid the
 * synchronisation an allocation may imply in the middle of its work.
 *   sigma_dev, sigma_prime_dev: DEVICE pointers, 16-byte aligned, in the layout
 *     of `encoding` (see the enum above; INT8 [R][L][L], PACKED [R][L][L/32]
 *     uint32, MULTISPIN [R/32][L][L] uint32), owned by the caller, only read.
 *   out_host: HOST array [replicas] receiving magnetization, energy, pair
 *     energy, cut_edges and cut_weight as shaken_observables computes them;
 *     best_energy = energy and best_step = -1 (no history here).
 * The reduction scratch is a fixed device array inside the library (for at
 * most 4096 replicas, about 0.5 MiB, held by every GPU that loads the library
 * until the process exits).  More replicas return SHAKEN_E_INVAL.  The first
 * call on each device looks up that array's device address; make that first
 * call before any stream capture.  Every call clears the scratch it uses, but
 * all calls share it: calls that overlap on the GPU race and must be
 * serialised by the caller.  Synchronises cuda_stream before returning. */
shaken_status shaken_lattice_observables_noalloc(const void* sigma_dev,
                                                 const void* sigma_prime_dev, int32_t encoding,
                                                 int64_t L, int32_t replicas, double J, double q,
                                                 double lambda_const, shaken_obs* out_host,
                                                 void* cuda_stream);

const char* shaken_strerror(shaken_status s);
const char* shaken_last_error(void);
const char* shaken_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SHAKEN_H */
