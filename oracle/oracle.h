/*
 * Plain CPU oracle for one iteration of the multi-swarm PSO for the Quadratic
 * Assignment Problem (Szwed & Chmiel, arXiv 1504.05158).
 *
 * TEST INFRASTRUCTURE ONLY. This code exists to check the CUDA path; it is
 * never part of it. Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it. It shares no source, header, table or
 * helper with the CUDA library and includes nothing from it.
 *
 * Style: every function is the plain definition or the algorithm's steps in
 * the paper's order, without blocking, fusion or incremental tricks. Doubles
 * (fp64) for all floating-point arithmetic, except where a floating-point value
 * decides an integer (S_x comparisons), which is done on the fp32 values that
 * the storage format of the velocity defines.
 *
 * Conventions (paper section 2.1 and 3.1): a permutation p maps facility j to
 * location p[j]; the permutation matrix has X[i][j] = 1 iff p[j] = i (row =
 * location, column = facility). Matrices are row-major int32 n x n; costs are
 * int64.
 *
 * Parity status: every function below is pinned by a test in tests/ against
 * something other than itself (brute force, closed forms, the paper's worked
 * example, a library Philox); see the test files named in each comment.
 */
#ifndef QAP_ORACLE_H
#define QAP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- counter-based RNG: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ---- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* key = (seed low 32, seed high 32); counter = (c0, c1, c2, tag << 24 | block). */
void orc_draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t tag,
              uint32_t block, uint32_t out[4]);
double orc_u01(uint32_t u);                  /* (u >> 8) * 2^-24, in [0, 1) */
uint32_t orc_below(uint32_t u, uint32_t k);  /* floor(u * k / 2^32), in [0, k) */

enum { ORC_TAG_R = 0, ORC_TAG_TIE = 1, ORC_TAG_INIT_X = 2, ORC_TAG_INIT_V = 3, ORC_TAG_MIG = 4,
       ORC_TAG_COLUMNS = 7 };

/* ---- QAP goal function and swap neighbourhood (section 2.1) ---- */
int64_t orc_cost(int n, const int32_t* F, const int32_t* D, const int32_t* p);
int64_t orc_cost_eq1(int n, const int32_t* F, const int32_t* D, const int32_t* p);
int64_t orc_delta(int n, const int32_t* F, const int32_t* D, const int32_t* p, int r, int s);
/* Best-improvement swap local search. max_moves: 0 = until no improving swap,
 * > 0 = at most that many moves. Returns the number of moves; *rounds = number
 * of full neighbourhood evaluations; trace (may be NULL) receives (r, s) per move. */
int orc_local_search(int n, const int32_t* F, const int32_t* D, int32_t* p, int max_moves,
                     int64_t* cost, int64_t* rounds, int32_t* trace, int trace_cap);
int64_t orc_brute_force(int n, const int32_t* F, const int32_t* D, int32_t* best_p);

/* ---- PSO parameters (Table 1 columns plus the readings of the silent points) ---- */
typedef struct {
    int32_t swarms, swarm_size;
    double c1, c2, c3;
    int32_t sv_kind;        /* 0 = Raw clamp, 1 = Norm (clamp + column L1 normalisation) */
    double v_max;
    int32_t depth;          /* SecondTarget depth d (0 = GlobalMax) */
    int32_t sx_rule;        /* 0 = Algorithm 1 literal, 1 = top-d reading of Eq. 6 */
    int32_t tie_rule;       /* 0 = random element of M, 1 = first element of M */
    int32_t pos_uses_new_v; /* 0 = Eq. 5 literal X + V(t), 1 = X + V(t+1) */
    int32_t ls_max_moves;   /* < 0 none, 0 to local optimum, > 0 cap */
    int32_t ls_at_init;
    int32_t mig_kind;       /* 0 none, 1 rank (Algorithm 2), 2 ring */
    int32_t mig_depth;      /* d of Algorithm 2 */
    int32_t mig_period;
    int32_t ring_if_better;
    int32_t v_storage;      /* 0 = fp32, 1 = bf16 (round to nearest even) */
    int32_t sx_kind;        /* 0 = SecondTarget (GlobalMax at depth 0), 1 = PickColumn */
} orc_params;

typedef struct {
    double* V;          /* P x n x n, values exactly representable in the storage format */
    int32_t* X;         /* P x n current positions */
    int32_t* PL;        /* P x n local bests */
    int64_t* costL;     /* P */
    int64_t* cost;      /* P current costs */
    int32_t* PG;        /* m x n swarm bests */
    int64_t* costG;     /* m */
    int32_t* best_p;    /* n, global best ever */
    int64_t* best_cost; /* 1 */
    int32_t* best_iter; /* 1, number of completed iterations when found */
    int32_t* t;         /* 1, completed iterations */
    int64_t* counters;  /* ORC_NCOUNTERS */
    int32_t* moves;     /* P, LS moves of the last iteration (may be NULL) */
} orc_state;

enum { ORC_C_PIT = 0, ORC_C_MOVES, ORC_C_ROUNDS, ORC_C_DELTA_FULL, ORC_C_DELTA_INCR,
       ORC_C_TIES, ORC_NCOUNTERS };

double orc_round_storage(double x, int v_storage);
double orc_round_bf16(double x);

/* Eq. 4 for one particle: W = S_v(c1 V + c2 r2 (P^L - X) + c3 r3 (P^G - X)), rounded
 * to the storage format. r2, r3 are inputs. Vout may alias nothing. */
void orc_velocity(const orc_params* q, int n, const double* V, const int32_t* x,
                  const int32_t* pl, const int32_t* pg, double r2, double r3, double* Vout);

/* S_x (SecondTarget, Algorithm 1 and the worked example of Eq. 6) on fp32 Y
 * with previous solution z. Tie draws come from Philox tag 1 at (c0,c1,c2).
 * Returns the number of steps where M had more than one element. */
int orc_second_target(const orc_params* q, int n, const float* Y, const int32_t* z,
                      uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, int32_t* out_p,
                      int32_t* order /* n x 2 picks (r, c) in order, may be NULL */);
/* PickColumn(Y) (section 3.1): the columns in a random order (a Fisher-Yates
 * shuffle, Philox tag 7, counter (c0, c1, c2)); each takes the largest element of
 * its column over the rows still free. Returns the number of columns whose maximum
 * was shared by several rows. order (may be NULL) receives the picks (r, c). */
int orc_pick_column(const orc_params* q, int n, const float* Y, uint64_t seed, uint32_t c0, uint32_t c1,
                    uint32_t c2, int32_t* out_p, int32_t* order);

/* One particle's whole iteration (Eq. 4, Eq. 5, S_x, cost, local search), given
 * its state at the start of iteration t. V_new receives V(t+1). p_sx receives the
 * S_x result, p_out the position after local search. */
void orc_particle_iteration(const orc_params* q, int n, const int32_t* F, const int32_t* D,
                            uint64_t seed, int t, int swarm, int pis, const double* V,
                            const int32_t* x, const int32_t* pl, const int32_t* pg,
                            double* V_new, int32_t* p_sx, int32_t* p_out, int64_t* cost_out,
                            int32_t* moves, int64_t* rounds, int32_t* ties);

void orc_init(const orc_params* q, int n, const int32_t* F, const int32_t* D, uint64_t seed,
              orc_state* s);
void orc_step(const orc_params* q, int n, const int32_t* F, const int32_t* D, uint64_t seed,
              orc_state* s);
/* The end-of-iteration bookkeeping alone (swarm bests, global best, migration) for
 * iteration t, given the post-local-search positions and costs of every particle. */
void orc_bests_and_migration(const orc_params* q, int n, uint64_t seed, int t, orc_state* s);

/* Nearest-rank percentiles of P costs: out = {min, p5, p25, p50, p75, max}; *mean =
 * the exact integer sum / P (quotient + remainder / P). */
/* Histogram of costs: counts[0] below lo, counts[1 + b] for b = floor((cost - lo) bins /
 * (hi - lo)), counts[bins + 1] at or above hi (the PMF of section 4.2 times P). */
void orc_histogram(const int64_t* cost, int P, int64_t lo, int64_t hi, int bins, int64_t* counts);
void orc_stats(const int64_t* cost, int P, int64_t out[6], double* mean);

#ifdef __cplusplus
}
#endif
#endif
