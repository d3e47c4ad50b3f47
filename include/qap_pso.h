/*
 * qap_pso.h -- C-ABI of the GB300 multi-swarm PSO for the Quadratic Assignment
 * Problem (Szwed & Chmiel, "Multi-swarm PSO algorithm for the Quadratic
 * Assignment Problem: a massive parallel implementation on the OpenCL
 * platform", arXiv 1504.05158).
 *
 * Problem (section 2.1, Eq. 1 and Eq. 2): facilities 0..n-1 with flows F[i][j],
 * locations 0..n-1 with distances D[k][l]; an assignment p places facility i at
 * location p[i] and costs f(p) = sum_i sum_j F[i][j] * D[p[i]][p[j]].
 *
 * One PSO iteration (section 3.1 and 3.2) updates every particle of every swarm:
 *   velocity  V(t+1) = S_v(c1 V(t) + c2 r2 (P^L - X(t)) + c3 r3 (P^G - X(t)))   (Eq. 4)
 *   position  X(t+1) = S_x(X(t) + V(t))                                        (Eq. 5)
 *             with S_x = SecondTarget (Algorithm 1; depth 0 = GlobalMax),
 *   then the goal function, a best-improvement swap local search, the local
 *   best P^L, the swarm bests P^G and the migration between swarms (Algorithm 2,
 *   or a ring). Every random draw is Philox4x32-10 keyed by the seed and
 *   counted by (particle in swarm, swarm, iteration, purpose).
 *
 * Conventions for every function:
 *   - return a status code (QAP_OK = 0 or one of QAP_ERR_*); never abort;
 *   - output arguments are left untouched when the status is not QAP_OK;
 *   - matrices are row-major n x n int32; permutations are int32 arrays of n
 *     entries, 0-based, facility -> location;
 *   - pointers are host pointers unless the comment says "device";
 *   - handles own the device memory they allocate; the caller keeps ownership of
 *     every buffer it passes in;
 *   - a state is used by one host thread at a time; its work is queued on its
 *     CUDA stream; functions that return results to the host synchronise that
 *     stream.
 */
#ifndef QAP_PSO_H
#define QAP_PSO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define QAP_OK 0
#define QAP_ERR_INVALID_ARG 1 /* a size, pointer or parameter is out of range */
#define QAP_ERR_OOM 2         /* device memory could not be allocated */
#define QAP_ERR_CUDA 3        /* a CUDA call or kernel failed */
#define QAP_ERR_TIMEOUT 4     /* a bounded device wait gave up */
#define QAP_ERR_OVERFLOW 5    /* the instance's values could overflow the exact integer path */
#define QAP_ERR_UNSUPPORTED 6 /* a valid request this build does not implement */

/* Human-readable name of a status code (static string). */
const char* qap_status_string(int status);

/* ------------------------------------------------------------- instances */
typedef struct qap_instance* qap_instance_t;

/* Copies F and D (host, row-major n x n int32, entries >= 0 as section 2.1
 * requires) to the device. n in [2, 256]. Records whether both matrices are
 * symmetric with a zero diagonal (the case the GPU local search implements) and
 * the value bounds that select the exact integer arithmetic. Errors:
 * QAP_ERR_INVALID_ARG for n out of range, NULL pointers or negative entries;
 * QAP_ERR_OOM / QAP_ERR_CUDA on device failures. */
int qap_create_instance(int32_t n, const int32_t* F, const int32_t* D, qap_instance_t* out);
void qap_destroy_instance(qap_instance_t inst);

typedef struct {
    int32_t n;
    int32_t symmetric_zero_diag; /* 1 if F and D are both symmetric with zero diagonal */
    int32_t max_f, max_d;        /* largest entries */
    int32_t exact_int32;         /* 1 if n * max_f * max_d < 2^27 (all swap values fit int32) */
    int32_t exact_int64;         /* 1 if (n^2 + 8 n + 4) * max_f * max_d < 2^62: every cost and
                                    swap value fits int64, so the instance can be solved */
} qap_instance_info_t;
int qap_instance_info(qap_instance_t inst, qap_instance_info_t* out);

/* ------------------------------------------------------------ parameters */
enum { PSO_SV_RAW = 0, PSO_SV_NORM = 1 };              /* S_v, section 3.1 */
enum { PSO_SX_ALG1 = 0, PSO_SX_TOPD = 1 };             /* which elements SecondTarget ignores */
enum { PSO_TIE_RANDOM = 0, PSO_TIE_FIRST = 1 };        /* choice inside the set M of Algorithm 1 */
enum { PSO_MIG_NONE = 0, PSO_MIG_RANK = 1, PSO_MIG_RING = 2 };
enum { PSO_V_FP32 = 0, PSO_V_BF16 = 1 };               /* storage of V; arithmetic is fp32 */
enum { PSO_SXK_SECOND_TARGET = 0, PSO_SXK_PICK_COLUMN = 1 }; /* the S_x procedure (section 3.1) */

typedef struct {
    int32_t swarms;         /* m >= 1 */
    int32_t swarm_size;     /* particles per swarm >= 1 */
    float c1, c2, c3;       /* inertia, self recognition, social factor (Eq. 4) */
    int32_t sv_kind;        /* PSO_SV_RAW: clamp to [-v_max, v_max]; PSO_SV_NORM: clamp then
                               divide each column by its L1 norm (section 3.1) */
    float v_max;            /* > 0 */
    int32_t sx_rule;        /* PSO_SX_ALG1: Algorithm 1 as printed (all elements of X(t) equal
                               to 1 ignored in the first `depth` steps); PSO_SX_TOPD: only the
                               `depth` largest of them (the reading that reproduces Eq. 6) */
    int32_t depth;          /* SecondTarget depth, 0 <= depth < n; 0 = GlobalMax */
    int32_t tie_rule;       /* PSO_TIE_RANDOM (Algorithm 1) or PSO_TIE_FIRST */
    int32_t pos_uses_new_v; /* 0: Eq. 5 literal, X(t) + V(t); 1: X(t) + V(t+1) */
    int32_t ls_max_moves;   /* swap local search: < 0 none, 0 until no improving swap, > 0 cap */
    int32_t ls_at_init;     /* 1: also run the local search on the initial particles */
    int32_t mig_kind;       /* PSO_MIG_* (section 3.2) */
    int32_t mig_depth;      /* Algorithm 2's d, 0 <= 2 d < m */
    int32_t mig_period;     /* migrate after every mig_period-th iteration (>= 1) */
    int32_t ring_if_better; /* ring: replace P^G of swarm k+1 only if strictly better */
    int32_t v_storage;      /* PSO_V_FP32 or PSO_V_BF16 (round to nearest even) */
    int32_t sx_kind;        /* PSO_SXK_SECOND_TARGET (Algorithm 1; GlobalMax at depth 0) or
                               PSO_SXK_PICK_COLUMN: the columns in a random order (Philox
                               Fisher-Yates, tag 7), each taking its largest element over the
                               free rows; depth and sx_rule do not apply */
} pso_params_t;

/* Fills the defaults: m = 1, 32 particles, c1 = 0.8, c2 = c3 = 0.5 (the esc32
 * setting of section 4.1), Norm, v_max = 1, Algorithm 1 with depth 2, random
 * ties, Eq. 5 literal, local search to a local optimum, no migration, fp32. */
void pso_params_default(pso_params_t* p);

/* ----------------------------------------------------------------- state */
typedef struct pso_state* pso_state_t;

/* Allocates the population on the device and initialises it (random particles,
 * section 3.3): X(0) by a Fisher-Yates shuffle and V(0) uniform in
 * [-v_max, v_max), both from Philox; cost, P^L = X(0), P^G and the global best.
 * `stream` is a cudaStream_t (NULL = a new stream owned by the state). The state
 * keeps a pointer to `inst`, which must outlive it. Every instance whose costs
 * fit int64 (qap_instance_info_t.exact_int64) is solved exactly: the search kernel
 * is chosen by the instance (tensor-core set-up for small entries, int32 or int64
 * SIMT arithmetic otherwise, the general O(n) swap formula for asymmetric
 * instances with large entries). Errors: QAP_ERR_INVALID_ARG (bad parameters),
 * QAP_ERR_UNSUPPORTED (n above the velocity kernels' shared-memory limit),
 * QAP_ERR_OVERFLOW (a cost or swap value could leave int64), QAP_ERR_OOM,
 * QAP_ERR_CUDA. */
int pso_init(qap_instance_t inst, const pso_params_t* params, uint64_t seed, void* stream,
             pso_state_t* out);

/* Queues `iterations` (>= 0) full iterations on the state's stream and returns
 * without waiting: each is the iteration of section 3.1 and 3.2 (Eq. 4, Eq. 5 with
 * SecondTarget of Algorithm 1, the goal function of Eq. 1, the swap local search,
 * P^L, P^G, the global best, migration by Algorithm 2 or the ring) for every
 * particle. Iterations are replayed from a captured CUDA graph. A failure inside a
 * kernel (a bounded wait that gave up) is reported by the next pso_best. */
int pso_step(pso_state_t st, int32_t iterations);

/* Like pso_step, but launches each kernel of every iteration directly (no graph)
 * with CUDA events around it on the state's stream, then synchronises. Adds into
 * ms_out[0..4] the device milliseconds of (0) the particle update (velocity, Eq. 4,
 * and position, Eq. 5 with S_x: one kernel), (1) goal function + local search,
 * (2) bests + migration, summed over the iterations, (3) the sum of each
 * iteration's span from its first kernel's start to its last kernel's end, and
 * (4) nothing (0; the velocity has no kernel of its own).
 * If flush_buf (device, flush_bytes long) is not NULL it is overwritten before every
 * iteration, outside the timed spans, to evict the L2 cache. For measurement. */
int pso_step_timed(pso_state_t st, int32_t iterations, void* flush_buf, size_t flush_bytes,
                   float* ms_out);

/* Device bytes pso_init would allocate for a population of this instance size and
 * these parameters (for admission against a memory budget). */
int pso_footprint(int32_t n, const pso_params_t* params, size_t* bytes);

/* *done = 1 when every operation queued on the state's stream has finished, else
 * 0 (never waits). */
int pso_poll(pso_state_t st, int32_t* done);

/* Best solution found so far (synchronises): its cost (Eq. 1), its permutation (n
 * entries, may be NULL) and the number of completed iterations when it was found
 * (0 = during initialisation). The paper keeps this best on the host (section 3.3);
 * here it lives on the device and is read back in one copy together with the
 * kernels' error counter. Errors: QAP_ERR_TIMEOUT when any kernel of this state
 * gave up a bounded wait or skipped an inconsistent access (the results may then
 * be incomplete; outputs are left untouched), QAP_ERR_CUDA. */
int pso_best(pso_state_t st, int64_t* cost, int32_t* perm, int32_t* iter_found);

typedef struct {
    uint32_t size;          /* caller sets sizeof(pso_stats_t) */
    int32_t iteration;      /* completed iterations */
    int64_t best_cost;      /* global best ever */
    int64_t min, p5, p25, p50, p75, max; /* current costs, nearest-rank percentiles
                                            (section 4.2) */
    double mean;            /* the exact integer sum of the current costs (summed on the
                               device in 128 bits) divided by their count on the host */
    int64_t particle_iterations; /* counters since pso_init */
    int64_t ls_moves, ls_rounds;
    int64_t delta_full;     /* swap values formed from a fresh O(n^3) set-up (first round) */
    int64_t delta_incr;     /* swap values formed after an O(n^2) rank-1 update */
    int64_t sx_ties;        /* S_x steps whose set M had more than one element */
    int64_t errors;         /* internal consistency failures detected by the kernels (0) */
} pso_stats_t;

/* Population statistics of the current costs plus counters (synchronises). */
int pso_stats(pso_state_t st, pso_stats_t* out);

/* The same statistics over the particles of one swarm (0 <= swarm < m): the
 * percentile ranks the paper plots for its most successful swarms (section 4.2);
 * the counters are those of the whole population. Synchronous. */
int pso_stats_swarm(pso_state_t st, int32_t swarm, pso_stats_t* out);

/* Distribution of the current costs (the probability mass function of section 4.2,
 * up to the factor 1 / particles) of one swarm, or of every particle (swarm = -1):
 * counts (host, bins + 2 int64) receives [0] the costs below lo, [1 + b] those with
 * floor((cost - lo) bins / (hi - lo)) = b, [bins + 1] those at or above hi.
 * 1 <= bins <= 2^20, lo < hi. Synchronous. Errors: QAP_ERR_INVALID_ARG. */
int pso_cost_histogram(pso_state_t st, int32_t swarm, int64_t lo, int64_t hi, int32_t bins, int64_t* counts);

/* Per-iteration statistics recorded on the device (section 4.2: the percentile
 * ranks of Figs. 4 and 5, the probability mass function of Figs. 6 and 7). After
 * pso_trace_start, every iteration of pso_step appends one record to a ring of
 * `capacity` records in device memory (the captured iterations are re-captured with
 * one more kernel); the host reads them with one copy. A record is `len` =
 * 9 + 8 m + bins + 2 int64 words:
 *   [0]              completed iterations t after the iteration recorded;
 *   [1 .. 8]         the population's current costs: min, p5, p25, p50, p75, max
 *                    (nearest rank, as pso_stats) and their exact sum as a 128-bit
 *                    two's-complement integer (low word, then high word);
 *   [9 + 8k .. +8]   the same eight words for swarm k, 0 <= k < m;
 *   [9 + 8m ..]      the histogram of pso_cost_histogram over every particle: below
 *                    lo, bins equal-width bins of [lo, hi), at or above hi.
 * Allocates the ring (capacity * len * 8 bytes); synchronises the state's stream.
 * Batch members and swarms larger than 16384 particles are not traced
 * (QAP_ERR_UNSUPPORTED). pso_step_timed does not record. Errors:
 * QAP_ERR_INVALID_ARG (capacity < 1, bins outside [1, 2^20], hi <= lo), QAP_ERR_OOM. */
int pso_trace_start(pso_state_t st, int32_t capacity, int64_t lo, int64_t hi, int32_t bins);
/* Words per record of the running trace. */
int pso_trace_record_len(pso_state_t st, int32_t* len);
/* Copies the most recent min(recorded, capacity, max_records) records, oldest first,
 * into `records` (host, max_records * len int64); *count receives how many.
 * Synchronises. */
int pso_trace_read(pso_state_t st, int64_t* records, int32_t max_records, int32_t* count);
/* Stops recording and frees the ring (synchronises). */
int pso_trace_stop(pso_state_t st);

void pso_destroy(pso_state_t st);

/* ------------------------------------------------ parts of a run (one per process) */
/* A run of M swarms may be split by whole swarms over several processes (one GPU
 * each): swarms are independent within an iteration (section 3.2) and meet only in
 * the migration step, which moves one permutation per swarm. pso_init_part
 * allocates the part holding swarms [first_swarm, first_swarm + params->swarms) of
 * the run: every random draw uses the swarm's index in the whole run, so each
 * particle evolves exactly as in the unsplit run. The part does no migration
 * (params->mig_kind is ignored); the caller migrates between the parts with the
 * calls below (the exchange: the swarm-best costs of every part, then one
 * permutation per migrating swarm). Errors as pso_init. */
int pso_init_part(qap_instance_t inst, const pso_params_t* params, uint64_t seed, int32_t first_swarm,
                  void* stream, pso_state_t* out);
/* The swarm bests P^G of the state's m swarms: costs (host, m int64) and, if perms is
 * not NULL, the permutations (host, m x n int32). Synchronises. */
int pso_swarm_bests(pso_state_t st, int64_t* costs, int32_t* perms);
/* Replaces swarm `swarm`'s best P^G by (cost, perm) (a migrated solution, accepted
 * even if worse, section 3.2). perm: host, n int32. Synchronises (after the queued
 * work). Errors: QAP_ERR_INVALID_ARG (swarm out of range, perm not a permutation). */
int pso_set_swarm_best(pso_state_t st, int32_t swarm, int64_t cost, const int32_t* perm);
/* The current position and cost of particle `index` (swarm-major: swarm * swarm_size
 * + particle in swarm, within the state). Synchronises. */
int pso_particle(pso_state_t st, int32_t index, int64_t* cost, int32_t* perm);
/* The counter-based generator every draw of an iteration uses (Philox4x32-10,
 * Salmon et al., SC'11): key = (seed low 32 bits, seed high 32 bits), counter = (c0,
 * c1, c2, tag << 24 | block), tag < 256, block < 2^24. out4: host, 4 uint32. Host
 * code; for callers that reproduce a draw (the migration picks of a split run:
 * tag 4, counter (k, 0, t)). */
int qap_philox(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t tag, uint32_t block,
               uint32_t* out4);

/* ------------------------------------------------ state export / import */
/* Host copies of the whole state, e.g. for checkpoints and for comparing one
 * iteration with an independent implementation. Sizes: P = swarms * swarm_size.
 * V is exported as fp32 values (exact for bf16 storage). */
typedef struct {
    float* V;        /* P * n * n, row = location, column = facility */
    int32_t* X;      /* P * n current positions */
    int32_t* X_sx;   /* P * n S_x results of the last iteration, before local search */
    int32_t* PL;     /* P * n */
    int64_t* costL;  /* P */
    int64_t* cost;   /* P */
    int32_t* moves;  /* P local-search moves of the last iteration */
    int32_t* PG;     /* swarms * n */
    int64_t* costG;  /* swarms */
    int32_t* best;   /* n */
    int64_t best_cost;
    int32_t best_iter;
    int32_t t;       /* completed iterations */
} pso_host_state_t;

/* Copies the device state into caller-owned host buffers (synchronises). */
int pso_export_state(pso_state_t st, pso_host_state_t* out);
/* Overwrites the device state from host buffers (V values are rounded to the
 * storage format; X_sx and moves are ignored). Every V value must be finite and
 * every X, PL, PG and best row a permutation, else QAP_ERR_INVALID_ARG with the
 * state untouched. Synchronises. */
int pso_import_state(pso_state_t st, const pso_host_state_t* in);

/* ---------------------------------------------------------------- batches */
/* Many independent populations advanced together, e.g. many QAP instances of
 * different n (the multi-swarm method of section 3 applied to each). Every phase
 * of an iteration runs as one kernel launch over all members (the local search
 * as one launch per kernel kind present: tensor-core set-up for n <= 128 with small
 * entries, SIMT set-up otherwise); iterations are replayed from a captured CUDA
 * graph. Results of every member are identical to running it alone. */
typedef struct pso_batch* pso_batch_t;

/* insts, params, seeds: `count` entries each; every member must use the same
 * v_storage. stream as in pso_init (shared by all members). autotune != 0 times
 * candidate launch shapes on the batch's own data (cached per process by shape),
 * then re-initialises every member from its seed, so tuning never changes
 * results. Errors as pso_init for any member. */
int pso_batch_create(int32_t count, const qap_instance_t* insts, const pso_params_t* params,
                     const uint64_t* seeds, void* stream, int32_t autotune, pso_batch_t* out);
/* Queues `iterations` iterations of every member (asynchronous). */
int pso_batch_step(pso_batch_t b, int32_t iterations);
/* As pso_step_timed, over the whole batch (ms_out[1] covers every search launch). */
int pso_batch_step_timed(pso_batch_t b, int32_t iterations, void* flush_buf, size_t flush_bytes,
                         float* ms_out);
int pso_batch_size(pso_batch_t b, int32_t* count);
/* Borrowed handle of member `index` for pso_best, pso_stats, pso_export_state and
 * pso_import_state; it stays owned by the batch (never pso_destroy it). */
int pso_batch_member(pso_batch_t b, int32_t index, pso_state_t* out);
void pso_batch_destroy(pso_batch_t b);

/* ------------------------------------------------ single-kernel entry points */
/* Goal function (Eq. 1) of `count` permutations (host, count x n int32) on the
 * device; out: count int64. Any instance whose costs fit int64 (else
 * QAP_ERR_OVERFLOW). */
int qap_eval_costs(qap_instance_t inst, const int32_t* perms, int32_t count, int64_t* out);

/* Best-improvement swap local search (the search of every iteration) on `count`
 * permutations (host, count x n int32, improved in place), max_moves as
 * pso_params_t.ls_max_moves (>= 0). The paper defines no local search (section 4.2
 * only says that PSO searches a local neighbourhood); this one is the swap
 * neighbourhood {p o (r s)} searched best-improvement: the smallest swap value,
 * the lowest pair (r, s) in r-major order on ties, applied while negative, until
 * no swap improves or max_moves moves were made. Outputs (host, count entries
 * each, any may be NULL): final costs, moves, rounds (neighbourhood evaluations).
 * Any instance whose costs fit int64; errors: QAP_ERR_OVERFLOW otherwise. */
int qap_local_search(qap_instance_t inst, int32_t* perms, int32_t count, int32_t max_moves,
                     int64_t* costs, int32_t* moves, int32_t* rounds);

/* The goal function (max_moves < 0; perms are left unchanged and costs must not
 * be NULL) or the local search above (max_moves >= 0), on the search kernel named
 * by `kernel` instead of the automatic choice, so that the kernels can be compared
 * with each other:
 *   QAP_SEARCH_AUTO    the kernel pso_step uses for this instance;
 *   QAP_SEARCH_TENSOR  the tensor-core set-up (symmetric with zero diagonal: entries
 *                      <= 2048, n max_f max_d < 2^24, n <= 128, or n <= 160 with
 *                      entries <= 255; general: entries <= 2048, 2 n max_f max_d < 2^24,
 *                      n <= 128);
 *   QAP_SEARCH_SIMT    int32 SIMT set-up (symmetric, n max_f max_d < 2^27, D <= 65535);
 *   QAP_SEARCH_INT64   int64 arithmetic (the int64 SIMT set-up for symmetric
 *                      instances that fit it, else the direct kernel);
 *   QAP_SEARCH_DIRECT  every swap value from the general O(n) formula, int64.
 * kernel_ms (host, may be NULL) receives the device time of the kernel launch
 * (CUDA events around it). Errors: QAP_ERR_UNSUPPORTED when the named kernel is not
 * exact for the instance or does not serve its n; QAP_ERR_OVERFLOW,
 * QAP_ERR_INVALID_ARG as above. */
enum { QAP_SEARCH_AUTO = 0, QAP_SEARCH_TENSOR = 1, QAP_SEARCH_SIMT = 2, QAP_SEARCH_INT64 = 3,
       QAP_SEARCH_DIRECT = 4 };
int qap_search_with(qap_instance_t inst, int32_t kernel, int32_t* perms, int32_t count, int32_t max_moves,
                    int64_t* costs, int32_t* moves, int32_t* rounds, float* kernel_ms);

/* Swap values of one permutation: out[idx(r, s)] = f(p o (r s)) - f(p) for every
 * pair r < s, in r-major order (idx = r n - r (r + 1) / 2 + s - r - 1), by the
 * general O(n) formula (any instance; int64 arithmetic). perm: host, n int32 (a
 * permutation, facility -> location); out: host, n (n - 1) / 2 int64. Synchronous.
 * Errors: QAP_ERR_INVALID_ARG (NULL pointer, not a permutation), QAP_ERR_OOM,
 * QAP_ERR_CUDA. */
int qap_delta_table(qap_instance_t inst, const int32_t* perm, int64_t* out);

/* Position discretisation alone (S_x = SecondTarget, Algorithm 1 of section 3.1)
 * of `count` matrices: Y (host, count x n x n fp32, row = location, column =
 * facility) and Z (host, count x n int32 permutations, facility -> location; the
 * ones of X(t)). The sx_kind, depth, sx_rule and tie_rule of `params` apply (its other
 * fields are ignored); random ties draw from the same Philox stream as an
 * iteration of particle particle[i] of swarm swarm[i] at iteration t (host arrays
 * of count int32). out_perm: host, count x n int32. This is the S_x of pso_step
 * with Y = X(t) + V formed by the caller, so the kernel compares exactly the given
 * fp32 values. 2 <= n <= the device limit of the fp32 velocity kernel.
 * Synchronous. Errors: QAP_ERR_INVALID_ARG (bad sizes, parameters, negative swarm
 * or particle indices, Z not a permutation, non-finite Y), QAP_ERR_UNSUPPORTED
 * (n too large), QAP_ERR_OOM, QAP_ERR_CUDA, QAP_ERR_TIMEOUT (a bounded wait gave
 * up). */
int pso_discretize(const float* Y, const int32_t* Z, int32_t n, int32_t count, const pso_params_t* params,
                   uint64_t seed, const int32_t* swarm, const int32_t* particle, int32_t t,
                   int32_t* out_perm);

/* ------------------------------------------------------------ measurement */
/* Integer throughput of the current GPU, measured: every SM busy with independent
 * chains of 32-bit multiply-adds (*mad_ops_per_s, each counted as two operations)
 * and of adds (*add_ops_per_s, one operation each), best of three timed runs of a
 * few milliseconds on `stream` (cudaStream_t, NULL = legacy default stream;
 * synchronises it). The denominator of the roofline of the integer-bound search
 * kernels; the paper has no counterpart. Errors: QAP_ERR_INVALID_ARG,
 * QAP_ERR_OOM, QAP_ERR_CUDA. */
int qap_int32_peak(void* stream, double* mad_ops_per_s, double* add_ops_per_s);

/* ------------------------------------------------ allocation-free statistics */
/* The same statistics as pso_stats (min, 5/25/50/75 % nearest-rank percentiles,
 * max, mean), computed from `count` costs that the caller already holds in device
 * memory, without allocating anything. This is for callers that cannot allocate
 * device memory: for instance a serving loop that admits work against a fixed
 * device-memory budget and must not see memory appear behind its back, or code
 * that must not call cudaMalloc/cudaFree because those calls can synchronize the
 * whole device. The paper has no counterpart; it exists for such callers.
 *
 * costs: device pointer, count int64 values, 1 <= count <= QAP_NOALLOC_MAX_COUNT
 * (larger counts fail with QAP_ERR_INVALID_ARG). stream: cudaStream_t (NULL =
 * legacy default stream). out6 and mean: host pointers receiving
 * {min, p5, p25, p50, p75, max} and the mean; the call synchronizes `stream`.
 *
 * Scratch: one fixed device array inside this library (QAP_NOALLOC_MAX_COUNT
 * int64 sort slots plus 8 result slots, 512 KiB + 64 B), held by every GPU that
 * loads the library until the process exits (placed when the driver loads the
 * library's device code on that device; with CUDA's lazy module loading, at the
 * first call there). Each call rewrites every slot it
 * reads, so nothing from an earlier call leaks into a result. All calls share
 * the one array: calls whose work overlaps on the GPU (other streams, other host
 * threads) race and must be serialized by the caller. The first call on a device
 * looks up the array's device address once (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture. */
#define QAP_NOALLOC_MAX_COUNT 65536
int qap_cost_stats_noalloc(const int64_t* costs, int32_t count, void* stream, int64_t* out6,
                           double* mean);

#ifdef __cplusplus
}
#endif
#endif
