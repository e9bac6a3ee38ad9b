/*
 * moda.h -- C ABI of the GB300 multi-objective Digital Annealer (MDA) for
 * the bi-objective quadratic assignment problem (bQAP).
 *
 * Method: Ayodele, Allmendinger, Lopez-Ibanez, Parizy, "Multi-objective QUBO
 * Solver: Bi-objective Quadratic Assignment Problem", arXiv 2205.13399.
 *   - Sec. 2.3, Eq. bf / mqap: the two penalised energies
 *       E_k(x) = c_k(x) + alpha_k g(x),
 *       c_k(x) = sum_{i,j,u,v} h^k_ij d_uv x_iu x_jv (Eq. cqap),
 *       g(x)   = sum_i (1 - sum_u x_iu)^2 + sum_u (1 - sum_i x_iu)^2 (Eq. gqap),
 *     over the n*n-bit two-way one-hot encoding (Sec. 2.2): bit i*n + u is
 *     set when facility i sits at location u.
 *   - Sec. 3.2, Eq. vermap / wvermaa and Sec. 3.3: alpha_k = w_k / 2 with
 *     w_k the largest change of c_k one flip can make.
 *   - Sec. 3.3, Alg. 3: the MDA loop (cooling, Delta E of every bit by
 *     Eq. cale, parallel trial by Eq. pacceptms or pacceptml, one accepted
 *     flip picked uniformly, archive update by Alg. 4 or Alg. 5, otherwise a
 *     jump to a random archive member); the alternative escape raises an
 *     energy offset by beta as the single-objective DA does (Alg. 1,
 *     Eq. paccepts).
 *
 * Every replica is an independent run of Alg. 3 with its own random stream:
 * Philox4x32-10 keyed by the seed, counter (bit group, iteration, replica
 * index, purpose).  The acceptance variate of bit p at iteration t is the
 * top 16 bits of word p mod 4 of counter (p / 4, t, replica, 0); a bit with
 * penalty a >= 0 (strict: sum_k max(0, dE_k); lenient: min_k max(0, dE_k);
 * dE_k reduced by the offset when that escape is used) is accepted iff
 * (double)a <= delta_t * (-ln((idx + 0.5) / 65536)) in IEEE double.  Runs
 * are bit-exact and independent of how replicas are placed on the device.
 *
 * Conventions for every call:
 *   - Status codes, never exceptions; on error no output is written and
 *     moda_last_error() returns a message (thread-local).
 *   - Host pointers are read during the call only; the library copies what
 *     it keeps.  Handles are owned by the library and freed by their
 *     destroy call.
 *   - Device work runs on the CUDA device that is current on the calling
 *     thread when the instance is created; later calls switch to it.
 *   - Flows and distances are non-negative int16; distances symmetric with
 *     a zero diagonal (MODA_EINVAL otherwise).  n in [2, 128].
 */
#ifndef MODA_H_
#define MODA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MODA_OK = 0,
  MODA_EINVAL = 1,       /* bad argument */
  MODA_ENOMEM = 2,       /* host or device allocation failed */
  MODA_EOVERFLOW = 3,    /* a local field could leave int32 (see below) */
  MODA_EUNSUPPORTED = 4, /* size or mode this build does not handle */
  MODA_ECUDA = 5,        /* CUDA runtime error, or a device-side check */
  MODA_ETIMEOUT = 6,     /* moda_wait ran out of time; the run continues */
  MODA_EBUSY = 7         /* the run is still executing */
} moda_status;

typedef struct moda_instance_s *moda_instance;
typedef struct moda_run_s *moda_run;
typedef struct moda_server_s *moda_server;
typedef struct moda_qubo_s *moda_qubo;
typedef struct moda_qrun_s *moda_qrun;

/* Sec. 3.3: strict = product of the per-objective probabilities
 * (Eq. pacceptms); lenient = their maximum (Eq. pacceptml). */
typedef enum { MODA_STRICT = 0, MODA_LENIENT = 1 } moda_accept;
/* Sec. 3.3: explorative (Alg. 4) or exploitative (Alg. 5) update. */
typedef enum { MODA_EXPLORE = 0, MODA_EXPLOIT = 1 } moda_archive;
/* Escape when no flip is accepted: jump to a random archive member
 * (Alg. 3), or raise the energy offset by beta (Alg. 1, Eq. paccepts). */
typedef enum { MODA_ESC_ARCHIVE = 0, MODA_ESC_OFFSET = 1 } moda_escape;

/* Penalty weights.  kind 0: w_k = (max_i sum_j Fs^k_ij) * (max_u sum_v d_uv)
 * with Fs^k = F^k + F^k^T, which is Eq. vermap on the symmetric form of
 * the cost QUBO when flows and distances are non-negative; kind 1: the
 * given w1, w2 (>= 0).  alpha_k = w_k / 2; g is always even, so every
 * energy is an exact integer. */
typedef struct {
  int32_t kind;
  int64_t w1, w2;
} moda_penalty;

/* Parameters of one anneal (Table 1 of the paper gives delta0 = 1e9,
 * deltaf = 1e4, xi = 1e-3, s = m, I_max = 0.25 m^2, beta = delta0 / I_max). */
typedef struct {
  int32_t replicas;      /* independent runs, >= 1 */
  int32_t replica_base;  /* replica index of the first run (RNG counter) */
  int64_t I_max;         /* iterations, 0 <= I_max < 2^32 */
  double delta0;         /* initial temperature, > 0 */
  double deltaf;         /* final temperature, > 0 */
  double xi;             /* decay, 0 < xi < 1 */
  int64_t beta;          /* offset increase (MODA_ESC_OFFSET), >= 0 */
  int32_t archive_size;  /* s, 0 means m = n*n; 1 <= s <= m */
  int32_t accept;        /* moda_accept */
  int32_t archive;       /* moda_archive */
  int32_t escape;        /* moda_escape */
  uint64_t seed;         /* Philox key */
  int32_t block_threads; /* 0: pick automatically; else a multiple of 32 */
  int32_t trace;         /* 1: record (E1, E2, event) of every iteration */
  int32_t field_cache;   /* jumps to the archive reload the member's local
                            fields from a per-slot device copy instead of
                            rebuilding them: 0 auto (when it fits in 60 % of
                            free device memory), 1 on (MODA_EUNSUPPORTED if it
                            does not fit), 2 off.  Results are identical. */
  int32_t prefetch;      /* field-cache prefetch distance: 0 auto, k in 1..4
                            (block engine; 1..15 for the warp engine, see
                            `engine`) copies a jump's target k - 1
                            iterations ahead (MODA_EUNSUPPORTED if it does
                            not fit). */
  int32_t normalize;     /* 1: QUBO normalisation of Sec. 4.2 -- each
                            objective's largest cost-QUBO coefficient set to
                            2^23 -- applied where it acts: the acceptance
                            test sees s_k Delta E_k, s_k = 2^23 / (max Fs^k_ij
                            * max d_uv), in IEEE double (the offset in the
                            same units); archives and energies stay the
                            unscaled integers, dominance being unchanged by
                            a positive scale per objective.  0: off. */
  int32_t snapshot_every; /* K > 0: after every iteration t with t % K == 0
                            the kernel copies each replica's archive to the
                            run (I_max / K snapshots, for the hypervolume
                            trace of Fig. mdasl; moda_read_snapshot);
                            0: none.  Not with moda_anneal_noalloc. */
  int32_t fast_forward;  /* 1: stop iterating once the rest of the run is
                            settled, with results identical to running every
                            iteration (archive escape only; not with
                            normalize or snapshot_every).  A trial at an
                            archive member in which no bit had an acceptance
                            penalty a <= hi_t marks that member as unable to
                            accept: hi_t never rises, so no later trial
                            there accepts either (until the slot is
                            rewritten).  Once every member is so marked and
                            the state about to be tried is a member, every
                            remaining iteration is a jump, and the run
                            lands on the final iteration's draw.  The
                            counters, trace and final state are those of the
                            full run; stats[6] counts the iterations not
                            executed.  0: every iteration runs (default). */
  int32_t engine;        /* which kernel runs the replicas; results are
                            identical:
                            1 block: one thread block per replica (all
                              options; lowest latency per iteration);
                            2 warp: one warp per replica, replicas of many
                              runs pulled from one device work list (the
                              archive escape only, without normalize,
                              snapshot_every or fast_forward;
                              MODA_EUNSUPPORTED otherwise).  Its field cache
                              holds the records of the first cache_slots
                              archive slots per resident team (field_cache
                              = 1: all s slots; 2: none); a jump to a slot
                              without records rebuilds its fields.  prefetch k in 1..15 copies
                              a jump's target k - 1 iterations ahead (0:
                              auto: up to 14 iterations, as shared memory
                              allows).  A team of G warps (1 to
                              8) runs each replica: automatically the
                              largest G that keeps every replica resident
                              at once, else 1; block_threads = 32 G
                              prescribes it.
                              While a replica only jumps, the trials of up
                              to prefetch iterations run together on the
                              members the earlier ones jump to (every bit of
                              every iteration is still tested; the first
                              iteration that accepts a bit flips and later
                              trials are discarded).
                            0 auto: warp when the options allow it and
                              block_threads is 0, else block. */
  int32_t cache_slots;   /* warp engine, field_cache = 0: archive slots with
                            field-cache records per team; 0: min(s, 1024),
                            k > 0: min(s, k), fewer where the launch's caches
                            would not fit the memory budget.  A jump to a
                            slot beyond it rebuilds the member's fields (as
                            slow as hundreds of jumps), so the cache should
                            cover the archive sizes runs reach.  Results are
                            identical for every value. */
} moda_params;

/* One archive member as returned by moda_read_archive. */
typedef struct {
  int64_t E1, E2;     /* penalised energies (Eq. mqap) */
  int64_t c1, c2;     /* QAP costs c_k = E_k - alpha_k g */
  int64_t g;          /* constraint value (0 iff a permutation) */
  int32_t feasible;   /* g == 0 */
  int32_t replica;    /* run index within the anneal (0-based) */
  int32_t slot;       /* archive slot within that run */
  int32_t pad;
} moda_point;

/* Build an instance from host flow matrices F1, F2 and distances D, each
 * n x n row-major int16 (Sec. 2.3: h_kij and d_uv).  Copies them to the
 * current device.  MODA_EOVERFLOW when (max_i sum_j Fs^k_ij) *
 * (max_u sum_v d_uv) >= 2^31 for either objective, the bound of the int32
 * local fields.  pen == NULL selects kind 0. */
moda_status moda_create_instance(int32_t n, const int16_t *F1,
                                 const int16_t *F2, const int16_t *D,
                                 const moda_penalty *pen, moda_instance *out);
/* Frees the instance's host and device memory, stream-ordered and without
 * synchronising the device.  Destroy an instance only after every run that
 * uses it has been destroyed (moda_destroy_run waits for its run) or has
 * finished. */
void moda_destroy_instance(moda_instance inst);
/* n and the penalty weights w1, w2 of an instance (any pointer may be
 * NULL). */
moda_status moda_instance_info(moda_instance inst, int32_t *n, int64_t *w1,
                               int64_t *w2);

/* Enqueue params->replicas independent runs of Alg. 3 on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream) and return at once.
 * The run owns its device buffers until moda_destroy_run. */
moda_status moda_anneal(moda_instance inst, const moda_params *params,
                        void *cuda_stream, moda_run *out);

/* Many anneals in one launch.  The paper solves each instance by a run of
 * Alg. 3 (Sec. 4 runs its instances one after another); nothing in a run
 * depends on another, so this call enqueues `count` of them -- request i is
 * exactly moda_anneal(insts[i], &params[i]) -- as one CUDA graph launch on
 * `cuda_stream` whose runs share no dependency, so the GPU runs the thread
 * blocks of many instances side by side instead of one small grid at a
 * time.  All instances live on one device.  outs[i] receives run i (owned
 * by the caller, moda_destroy_run); each has its own device buffers and
 * gives the same results as the plain call.  On failure nothing is
 * enqueued, no run is returned and the message names the request. */
moda_status moda_anneal_batch(const moda_instance *insts, const moda_params *params,
                              int32_t count, void *cuda_stream, moda_run *outs);

/* Wait for a run: MODA_OK when it finished, MODA_ETIMEOUT when timeout_ms
 * (>= 0; < 0 waits forever) passed first, MODA_ECUDA on a device error. */
moda_status moda_wait(moda_run run, int64_t timeout_ms);

/* Raw per-run results of a finished run, replica r (0-based), or all
 * replicas at once when r == -1 (arrays then hold `replicas` blocks):
 *   count    [1]        archive size |A|
 *   E        [s][2]     archive energies (E1, E2) in slot order
 *   bits     [s][W]     archive states, W = ceil(m / 32) words, bit p in
 *                       word p / 32 at position p % 32
 *   x        [W]        state after the last iteration
 *   E_final  [2]        its energies
 *   stats    [8]        accepted flips, jumps to the archive, escapes with an
 *                       empty archive, offset raises; then, for profiling,
 *                       jumps served by a prefetched field-cache record,
 *                       jumps that read the record directly, iterations
 *                       settled without being executed (params.fast_forward),
 *                       and jumps that rebuilt the fields of a slot without
 *                       records (warp engine; 0 in the block engine)
 * Any pointer may be NULL.  MODA_EBUSY while the run executes. */
moda_status moda_read_replica(moda_run run, int32_t r, int32_t *count,
                              int64_t *E, uint32_t *bits, uint32_t *x,
                              int64_t *E_final, int64_t *stats);

/* (E1, E2, event) of every iteration of replica r when params.trace was
 * set: event >= 0 is the flipped bit, -1 - slot a jump to that archive slot,
 * INT64_MIN an iteration without a flip or a jump.  trace holds I_max * 3
 * values. */
moda_status moda_read_trace(moda_run run, int32_t r, int64_t *trace);

/* The non-dominated members of replica r's archive (r >= 0), or of the
 * union of all replicas (r == -1), Sec. 3.3 "return all non-dominated
 * solutions from archive A" and Sec. 4.2 (merging runs).  Among equal
 * energy vectors the lowest (replica, slot) is kept.  Points are sorted by
 * E1.  Writes min(cap, total) points and sets *count to the total.  perms,
 * if not NULL, receives n bytes per written point: the location of each
 * facility, or 0xFF for an infeasible point. */
moda_status moda_read_archive(moda_run run, int32_t r, moda_point *pts,
                              int32_t cap, int32_t *count, uint8_t *perms);

/* As moda_read_archive, for the archive as it stood after iteration
 * (snap + 1) * params.snapshot_every (0 <= snap < I_max / snapshot_every). */
moda_status moda_read_snapshot(moda_run run, int32_t snap, int32_t r, moda_point *pts,
                               int32_t cap, int32_t *count, uint8_t *perms);

/* Device time of the anneal kernel of a finished run, in milliseconds
 * (CUDA events on the run's stream). */
moda_status moda_run_elapsed_ms(moda_run run, float *ms);

void moda_destroy_run(moda_run run);

/* ---- SB-DA (Sec. 3.2, Alg. 2), the paper's scalarisation baseline -----
 *
 * moda_scalarize builds the single-objective instance of weight gamma =
 * gamma_num / gamma_den, scaled by gamma_den so that it stays integral:
 * flows gamma_num Fs^1 + (gamma_den - gamma_num) Fs^2 (Alg. 2, cost line)
 * with the penalty weight of Eq. vermap taken on that cost (Alg. 2, alpha
 * line; the instance's w1, w2 are w and 0) and a second objective of zero.
 * MODA_EOVERFLOW when a scaled field could exceed int32.
 *
 * Alg. 1 (DA) on it is moda_anneal with escape = MODA_ESC_OFFSET,
 * archive_size = 1 and delta0, deltaf and beta multiplied by gamma_den:
 * with the second objective zero the acceptance penalty is
 * max(0, Delta E - E_offset), and the explorative archive of one slot
 * keeps the lowest-energy state reached by a flip (the earliest on ties),
 * which is DA's "best solution found" (the initial state if no flip is
 * ever accepted).
 *
 * moda_sbda_front merges finished runs of one source instance, one run per
 * weight: each replica's best state, if it is a permutation, with its QAP
 * costs (c1, c2) on the source instance, then the non-dominated points
 * (Alg. 2, last line), among equal cost vectors the lowest (run, replica).
 * Points come sorted by c1, with E = c, replica = replica and slot = run
 * index; perms as in moda_read_archive.  MODA_EBUSY if a run has not
 * finished. */
moda_status moda_scalarize(moda_instance src, int32_t gamma_num, int32_t gamma_den,
                           moda_instance *out);
moda_status moda_sbda_front(moda_instance src, const moda_run *runs, int32_t count,
                            moda_point *pts, int32_t cap, int32_t *total, uint8_t *perms);

/* ---- Explicit QUBOs with K objectives ---------------------------------
 *
 * Alg. 3 on objectives given as explicit QUBO matrices instead of the
 * bi-objective QAP: E_k(x) = x^T Q_k x with Q_k upper triangular (Sec. 2.2's
 * convention; entries below the diagonal are ignored), Delta E from the
 * stored P_k = Q_k + Q_k^T with P_pp = Q_pp (Eq. cale), and K-dimensional
 * dominance in the archive updates (Alg. 4 / Alg. 5).  Any constraint
 * penalty is part of the caller's Q_k.  Draws, acceptance (strict: the sum
 * of max(0, Delta E_k - E_offset) over the objectives; lenient: their
 * minimum), selection, archive and escape follow moda_anneal.
 *
 * moda_qubo_create copies K (1..3) matrices of m x m int32 (m <= 4096,
 * row-major, [K][m][m]) to the current device; MODA_EOVERFLOW when an
 * entry of Q + Q^T leaves int32.  moda_qubo_anneal enqueues params->replicas
 * runs on cuda_stream (params.normalize, params.snapshot_every and
 * params.fast_forward must be 0; params.field_cache == 2 turns the archive Delta E records off, jumps
 * then rebuild Delta E).  moda_qrun_read copies, for all replicas, any
 * non-NULL of: archive sizes [R], energies [R][s][K], states [R][s][W]
 * (W = ceil(m / 32), bit p in word p / 32), final states [R][W] and
 * energies [R][K], counters [R][4] (flips, jumps, empty escapes, offset
 * raises) and the trace [R][I_max][K + 1] (energies, event as in
 * moda_read_trace) of a run made with params.trace. */
moda_status moda_qubo_create(int32_t K, int32_t m, const int32_t *Q, moda_qubo *out);
void moda_qubo_destroy(moda_qubo q);
moda_status moda_qubo_anneal(moda_qubo q, const moda_params *params, void *cuda_stream,
                             moda_qrun *out);
moda_status moda_qrun_wait(moda_qrun run);
moda_status moda_qrun_read(moda_qrun run, int32_t *count, int64_t *E, uint32_t *bits,
                           uint32_t *x, int64_t *E_final, int64_t *stats, int64_t *trace);
moda_status moda_qrun_elapsed_ms(moda_qrun run, float *ms);
void moda_qrun_destroy(moda_qrun run);

/* Autotuner of the launch layout: for the block engine, times short trials
 * of every block shape the kernel has (bits per thread and threads per
 * block) and, when the escape jumps to the archive, of field-cache
 * prefetch distances 1 and 2 besides the automatic choice, on `inst` with
 * `params` (trial_iters iterations at the cold end of the schedule, delta =
 * deltaf, on at most one replica per SM); for the warp engine, prefetch
 * distances 0, 2, 6, 10 and 14 on the request's own replicas.  Writes into
 * *best a copy of *params with the fastest block_threads and prefetch; *best_ms (if not NULL) receives the
 * winning trial's time.  Results of a run do not depend on these two
 * fields, so tuning never changes what an anneal computes.  Blocks the
 * calling thread while the trials run on cuda_stream. */
moda_status moda_autotune(moda_instance inst, const moda_params *params, int32_t trial_iters,
                          void *cuda_stream, moda_params *best, float *best_ms);

/* ---- Serving ---------------------------------------------------------
 *
 * A queue of anneal requests served as they arrive (not in the paper:
 * serving many bi-objective QAP solves on one GPU).  A native thread of the
 * server admits waiting requests in arrival order while the device buffers
 * of the runs in flight (the bytes moda_anneal would allocate for each) fit
 * `hbm_budget`, and launches each admitted request at once on a stream of
 * its own (or on `cuda_stream` if not NULL, which orders them), so new
 * requests join the ones already running instead of waiting for a batch.
 * A request whose buffers with the field cache do not fit runs without it
 * (identical results) once nothing else is running, if that fits; it fails
 * with MODA_ENOMEM when it cannot fit even then.  A request whose device
 * allocation fails while other runs hold memory waits for them.  Each request's results equal those of moda_anneal on
 * the same instance and params.
 *
 *   hbm_budget  bytes for the buffers of runs in flight; 0 = the free
 *               device memory at creation less max(1/8 of it, 1 GiB)
 *   ticket      identifies a request; moda_server_poll sets *done to the
 *               finished run (then owned by the caller; its buffers count
 *               against the budget until moda_destroy_run) or to NULL while
 *               it waits or runs; a failed request returns its error once.
 *   instances   must outlive their requests.
 *   destroy     cancels requests not yet started (their poll would fail),
 *               waits for those running and frees finished runs nobody
 *               polled. */
moda_status moda_server_create(size_t hbm_budget, void *cuda_stream, moda_server *out);
moda_status moda_server_submit(moda_server srv, moda_instance inst,
                               const moda_params *params, int64_t *ticket);
moda_status moda_server_poll(moda_server srv, int64_t ticket, moda_run *done);
/* Queue state: requests waiting, requests running, bytes of their buffers
 * and the budget (any pointer may be NULL). */
moda_status moda_server_info(moda_server srv, int64_t *pending, int64_t *running,
                             size_t *bytes_in_use, size_t *budget);
void moda_server_destroy(moda_server srv);

/* Thread-local message of the last failed call on this thread. */
const char *moda_last_error(void);

/* ---- Annealing without device allocation ------------------------------
 *
 * The paper has no counterpart: this entry point serves callers that must
 * not allocate device memory when they anneal -- a serving process that
 * gives all of its device memory to its own pool, or code whose device
 * memory belongs to a host framework's allocator -- so cudaMalloc (and any
 * routine that allocates, torch's included) is off limits to them.
 *
 * moda_anneal_noalloc runs the same kernel as moda_anneal on the same
 * inputs and gives the same results, but allocates nothing: the instance
 * comes from host arrays (as in moda_create_instance), the results go to
 * device buffers the caller owns (below), and the kernel's scratch (the
 * field cache of moda_params.field_cache) plus the instance matrices, the
 * cooling schedule and the -ln(u) table live in fixed-size device arrays of
 * the library, held by every GPU that loads it until the process exits.
 *
 *   Limits (MODA_EUNSUPPORTED beyond them): n <= 128; with the archive
 *   escape, replicas * s * r * ceil8(n^2) bytes <= 64 MiB (s = archive
 *   size; r = 8 when every |Delta E_k| of the instance stays below 2^31,
 *   i.e. B_k + w_k (2n + 1) < 2^31 with B_k the bound of moda_create_instance,
 *   else 16); the offset escape uses no scratch; at most 65,536 schedule
 *   entries before delta reaches delta_f; params.trace = 0.
 *   params.field_cache and params.prefetch are ignored (the cache is used
 *   whenever the escape jumps to the archive).
 *   Shared state: all calls share the library's arrays; two calls whose
 *   device work overlaps (other streams or host threads) race and give
 *   wrong results.  Serialise them, e.g. on one stream.
 *   Set-up: the first call on a device (the device current on the calling
 *   thread) looks up the arrays' device addresses and uploads the table.
 *   Capture: no call may be made while cuda_stream is being captured into
 *   a CUDA graph (MODA_EUNSUPPORTED): each call stages its instance and
 *   schedule in host arrays that the next call overwrites.
 *   Asynchrony: returns once the work is enqueued on cuda_stream; the
 *   outputs are ready when that stream reaches this point.  The error word
 *   is set to 0 by the call and to a nonzero code by a device-side failure:
 *   1 when a bounded wait for a field-cache copy gave up, 2 when a kernel
 *   variant was launched for a run it does not fit (an internal error).
 */
typedef struct {
  int64_t *arch_E;      /* [replicas][s][2] archive energies */
  uint32_t *arch_bits;  /* [replicas][s][W] archive states, W = ceil(n^2 / 32),
                           plus 32 spare bytes at the end */
  int32_t *arch_count;  /* [replicas] archive sizes */
  uint32_t *x_final;    /* [replicas][W] final states */
  int64_t *E_final;     /* [replicas][2] their energies */
  int64_t *stats;       /* [replicas][8] counters as in moda_read_replica */
  int32_t *error;       /* [1] device status word */
} moda_device_outputs;

moda_status moda_anneal_noalloc(int32_t n, const int16_t *F1,
                                const int16_t *F2, const int16_t *D,
                                const moda_penalty *pen,
                                const moda_params *params,
                                const moda_device_outputs *out,
                                void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* MODA_H_ */
