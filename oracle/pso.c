/*
 * Multi-swarm PSO iteration for the QAP: velocity (Eq. 4 with S_v), position
 * (Eq. 5 with the S_x procedure SecondTarget, Algorithm 1), goal function,
 * swap local search, local/swarm/global bests and migration (Algorithm 2 and a
 * ring variant), initialisation and population statistics.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h). Plain loops in the paper's order.
 */
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

/* ---------------------------------------------------------------- storage */

/* Round to bfloat16 (8 significant bits, fp32 exponent range), ties to even. */
double orc_round_bf16(double x) {
    if (x == 0.0 || !isfinite(x)) return x;
    if (fabs(x) < (double)FLT_MIN) {
        /* subnormal range: fixed quantum 2^-133 */
        return rint(ldexp(x, 133)) * ldexp(1.0, -133);
    }
    int e;
    double m = frexp(x, &e); /* x = m * 2^e, 0.5 <= |m| < 1 */
    return ldexp(rint(m * 256.0), e - 8);
}

double orc_round_storage(double x, int v_storage) {
    if (v_storage == 1) return orc_round_bf16(x);
    return (double)(float)x;
}

/* --------------------------------------------------------------- velocity */

/* Eq. 4: V(t+1) = S_v(c1 V(t) + c2 r2 (P^L - X) + c3 r3 (P^G - X)), with the
 * permutation matrices X[i][j] = 1 iff x[j] = i (section 3.1). S_v "Raw" clamps
 * every element to [-v_max, v_max]; "Norm" additionally divides each column j by
 * n_j = sum_i |v_ij| (a column whose n_j is 0 stays 0). The result is rounded
 * once to the storage format. */
void orc_velocity(const orc_params* q, int n, const double* V, const int32_t* x,
                  const int32_t* pl, const int32_t* pg, double r2, double r3, double* Vout) {
    const double a = q->c2 * r2;
    const double b = q->c3 * r3;
    double* W = (double*)malloc(sizeof(double) * n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double X = (x[j] == i) ? 1.0 : 0.0;
            double L = (pl[j] == i) ? 1.0 : 0.0;
            double G = (pg[j] == i) ? 1.0 : 0.0;
            double w = q->c1 * V[i * n + j] + a * (L - X) + b * (G - X);
            if (w > q->v_max) w = q->v_max;
            if (w < -q->v_max) w = -q->v_max;
            W[i * n + j] = w;
        }
    if (q->sv_kind == 1) {
        for (int j = 0; j < n; ++j) {
            double nj = 0.0;
            for (int i = 0; i < n; ++i) nj += fabs(W[i * n + j]);
            if (nj > 0.0)
                for (int i = 0; i < n; ++i) W[i * n + j] = W[i * n + j] / nj;
        }
    }
    for (int e = 0; e < n * n; ++e) Vout[e] = orc_round_storage(W[e], q->v_storage);
    free(W);
}

/* ------------------------------------------------------------------- S_x */

/* PickColumn(Y), section 3.1: "picks a column c, selects a maximum element x_rc,
 * replaces it by 1 and clears other elements in r and c", until every column is
 * assigned. The paper leaves the order of the columns open; here it is a
 * Fisher-Yates shuffle of 0..n-1 (i = n-1 .. 1, j uniform in [0, i], draw q = n-1-i
 * is word q mod 4 of block q/4 of tag 7 with counter (particle, swarm, t)), and the
 * k-th column of the shuffled order is taken at step k. A maximum shared by several
 * free rows is resolved like a tie of Algorithm 1: the rows in ascending order,
 * element floor(u m / 2^32) with u = word (step mod 4) of block step/4 of tag 1
 * (tie_rule 0), or the first (tie_rule 1). Comparisons on the fp32 values of Y. */
int orc_pick_column(const orc_params* q, int n, const float* Y, uint64_t seed, uint32_t c0, uint32_t c1,
                    uint32_t c2, int32_t* out_p, int32_t* order) {
    int32_t* cols = (int32_t*)malloc(sizeof(int32_t) * n);
    unsigned char* free_r = (unsigned char*)malloc(n);
    int32_t* rows = (int32_t*)malloc(sizeof(int32_t) * n);
    for (int c = 0; c < n; ++c) cols[c] = c;
    uint32_t w[4] = {0, 0, 0, 0};
    for (int i = n - 1; i >= 1; --i) {
        const int d = n - 1 - i;
        if (d % 4 == 0) orc_draw(seed, c0, c1, c2, ORC_TAG_COLUMNS, (uint32_t)(d / 4), w);
        const int j = (int)orc_below(w[d % 4], (uint32_t)(i + 1));
        const int32_t tmp = cols[i];
        cols[i] = cols[j];
        cols[j] = tmp;
    }
    memset(free_r, 1, n);
    int ties = 0;
    for (int step = 0; step < n; ++step) {
        const int c = cols[step];
        float best = 0.0f;
        int m = 0;
        for (int r = 0; r < n; ++r) {
            if (!free_r[r]) continue;
            const float y = Y[r * n + c];
            if (m == 0 || y > best) {
                best = y;
                m = 0;
            }
            if (y == best) rows[m++] = r;
        }
        int k = 0;
        if (m > 1) {
            ++ties;
            if (q->tie_rule == 0) {
                orc_draw(seed, c0, c1, c2, ORC_TAG_TIE, (uint32_t)(step / 4), w);
                k = (int)orc_below(w[step % 4], (uint32_t)m);
            }
        }
        const int r = rows[k];
        out_p[c] = r;
        free_r[r] = 0;
        if (order) {
            order[2 * step] = r;
            order[2 * step + 1] = c;
        }
    }
    free(cols);
    free(free_r);
    free(rows);
    return ties;
}

/* SecondTarget(Y, Z, depth), Algorithm 1: n greedy steps; each step takes the set
 * M of the largest remaining elements (rows and columns already used are gone),
 * picks one (r, c) of M, assigns facility c to location r and deletes row r and
 * column c. In the first `depth` steps some elements equal to 1 in Z = X(t) are
 * ignored:
 *   sx_rule 0 (Algorithm 1 as printed): all of them;
 *   sx_rule 1 (the reading that reproduces all three pictures of Eq. 6): only the
 *     `depth` of them with the largest Y value (lower column first on ties).
 * depth = 0 is GlobalMax. M is ordered column-major (column c, then row r); with
 * tie_rule 0 the k-th element is taken, k = floor(u |M| / 2^32), u = word
 * (step mod 4) of Philox block step/4 of tag 1; with tie_rule 1 the first.
 * All comparisons are on the fp32 values of Y. */
int orc_second_target(const orc_params* q, int n, const float* Y, const int32_t* z,
                      uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, int32_t* out_p,
                      int32_t* order) {
    unsigned char* alive_r = (unsigned char*)malloc(n);
    unsigned char* alive_c = (unsigned char*)malloc(n);
    unsigned char* excl = (unsigned char*)calloc((size_t)n * n, 1);
    memset(alive_r, 1, n);
    memset(alive_c, 1, n);
    if (q->depth > 0) {
        if (q->sx_rule == 0) {
            for (int c = 0; c < n; ++c) excl[z[c] * n + c] = 1;
        } else {
            unsigned char* chosen = (unsigned char*)calloc(n, 1);
            for (int k = 0; k < q->depth && k < n; ++k) {
                int bc = -1;
                for (int c = 0; c < n; ++c) {
                    if (chosen[c]) continue;
                    if (bc < 0 || Y[z[c] * n + c] > Y[z[bc] * n + bc]) bc = c;
                }
                chosen[bc] = 1;
                excl[z[bc] * n + bc] = 1;
            }
            free(chosen);
        }
    }
    int ties = 0;
    for (int step = 0; step < n; ++step) {
        const int use_excl = step < q->depth;
        int have = 0;
        float best = 0.0f;
        for (int c = 0; c < n; ++c) {
            if (!alive_c[c]) continue;
            for (int r = 0; r < n; ++r) {
                if (!alive_r[r]) continue;
                if (use_excl && excl[r * n + c]) continue;
                float v = Y[r * n + c];
                if (!have || v > best) { best = v; have = 1; }
            }
        }
        int count = 0;
        for (int c = 0; c < n; ++c) {
            if (!alive_c[c]) continue;
            for (int r = 0; r < n; ++r) {
                if (!alive_r[r]) continue;
                if (use_excl && excl[r * n + c]) continue;
                if (Y[r * n + c] == best) ++count;
            }
        }
        uint32_t k = 0;
        if (count > 1) {
            ++ties;
            if (q->tie_rule == 0) {
                uint32_t w[4];
                orc_draw(seed, c0, c1, c2, ORC_TAG_TIE, (uint32_t)(step / 4), w);
                k = orc_below(w[step % 4], (uint32_t)count);
            }
        }
        int pr = -1, pc = -1;
        uint32_t seen = 0;
        for (int c = 0; c < n && pr < 0; ++c) {
            if (!alive_c[c]) continue;
            for (int r = 0; r < n; ++r) {
                if (!alive_r[r]) continue;
                if (use_excl && excl[r * n + c]) continue;
                if (Y[r * n + c] == best) {
                    if (seen == k) { pr = r; pc = c; break; }
                    ++seen;
                }
            }
        }
        out_p[pc] = pr;
        alive_r[pr] = 0;
        alive_c[pc] = 0;
        if (order) { order[2 * step] = pr; order[2 * step + 1] = pc; }
    }
    free(alive_r);
    free(alive_c);
    free(excl);
    return ties;
}

/* ------------------------------------------------------- one particle step */

void orc_particle_iteration(const orc_params* q, int n, const int32_t* F, const int32_t* D,
                            uint64_t seed, int t, int swarm, int pis, const double* V,
                            const int32_t* x, const int32_t* pl, const int32_t* pg,
                            double* V_new, int32_t* p_sx, int32_t* p_out, int64_t* cost_out,
                            int32_t* moves, int64_t* rounds, int32_t* ties) {
    /* r2, r3 drawn per particle and iteration (section 3.1, after Eq. 5) */
    uint32_t w[4];
    orc_draw(seed, (uint32_t)pis, (uint32_t)swarm, (uint32_t)t, ORC_TAG_R, 0, w);
    const double r2 = orc_u01(w[0]);
    const double r3 = orc_u01(w[1]);
    orc_velocity(q, n, V, x, pl, pg, r2, r3, V_new);

    /* Eq. 5: X(t+1) = S_x(X(t) + V(t)); the sum is formed in fp32 */
    const double* Vsrc = q->pos_uses_new_v ? V_new : V;
    float* Y = (float*)malloc(sizeof(float) * n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            float xv = (x[j] == i) ? 1.0f : 0.0f;
            float vv = (float)Vsrc[i * n + j];
            Y[i * n + j] = vv + xv;
        }
    int nt = q->sx_kind == 1
                 ? orc_pick_column(q, n, Y, seed, (uint32_t)pis, (uint32_t)swarm, (uint32_t)t, p_sx, NULL)
                 : orc_second_target(q, n, Y, x, seed, (uint32_t)pis, (uint32_t)swarm, (uint32_t)t, p_sx, NULL);
    free(Y);
    memcpy(p_out, p_sx, sizeof(int32_t) * n);
    int mv = 0;
    int64_t rd = 0, c;
    if (q->ls_max_moves >= 0) {
        mv = orc_local_search(n, F, D, p_out, q->ls_max_moves, &c, &rd, NULL, 0);
    } else {
        c = orc_cost(n, F, D, p_out);
    }
    *cost_out = c;
    if (moves) *moves = mv;
    if (rounds) *rounds = rd;
    if (ties) *ties = nt;
}

/* ------------------------------------------------------- bests, migration */

static void copy_perm(int32_t* dst, const int32_t* src, int n) {
    memcpy(dst, src, sizeof(int32_t) * n);
}

/* Swarm bests P^G[k] (replaced only by a strictly better particle; the lowest
 * particle index wins ties), the global best ever, then migration. */
void orc_bests_and_migration(const orc_params* q, int n, uint64_t seed, int t, orc_state* s) {
    const int m = q->swarms, ss = q->swarm_size, P = m * ss;
    for (int k = 0; k < m; ++k) {
        int bi = k * ss;
        for (int j = 1; j < ss; ++j)
            if (s->cost[k * ss + j] < s->cost[bi]) bi = k * ss + j;
        if (s->cost[bi] < s->costG[k]) {
            s->costG[k] = s->cost[bi];
            copy_perm(s->PG + (size_t)k * n, s->X + (size_t)bi * n, n);
        }
    }
    int gi = 0;
    for (int i = 1; i < P; ++i)
        if (s->cost[i] < s->cost[gi]) gi = i;
    if (s->cost[gi] < *s->best_cost) {
        *s->best_cost = s->cost[gi];
        copy_perm(s->best_p, s->X + (size_t)gi * n, n);
        *s->best_iter = t + 1;
    }
    const int period = q->mig_period > 0 ? q->mig_period : 1;
    if ((t + 1) % period != 0) return;
    if (q->mig_kind == 1 && q->mig_depth > 0) {
        /* Algorithm 2: order swarms by their P^G value (best first, lower index on
         * ties); for k < d the k-th worst swarm receives a randomly chosen current
         * solution of the k-th best swarm, accepted even if it is worse. */
        int* ord = (int*)malloc(sizeof(int) * m);
        for (int k = 0; k < m; ++k) ord[k] = k;
        for (int a = 0; a < m; ++a)
            for (int b = a + 1; b < m; ++b) {
                int ia = ord[a], ib = ord[b];
                if (s->costG[ib] < s->costG[ia] || (s->costG[ib] == s->costG[ia] && ib < ia)) {
                    ord[a] = ib; ord[b] = ia;
                }
            }
        for (int k = 0; k < q->mig_depth; ++k) {
            const int donor = ord[k], target = ord[m - 1 - k];
            uint32_t w[4];
            orc_draw(seed, (uint32_t)k, 0u, (uint32_t)t, ORC_TAG_MIG, 0, w);
            const int j = (int)orc_below(w[0], (uint32_t)ss);
            const int src = donor * ss + j;
            copy_perm(s->PG + (size_t)target * n, s->X + (size_t)src * n, n);
            s->costG[target] = s->cost[src];
        }
        free(ord);
    } else if (q->mig_kind == 2) {
        /* ring: swarm k's best goes to swarm k+1 (mod m), all from a snapshot */
        int32_t* snap = (int32_t*)malloc(sizeof(int32_t) * (size_t)m * n);
        int64_t* snapc = (int64_t*)malloc(sizeof(int64_t) * m);
        memcpy(snap, s->PG, sizeof(int32_t) * (size_t)m * n);
        memcpy(snapc, s->costG, sizeof(int64_t) * m);
        for (int k = 0; k < m; ++k) {
            const int dst = (k + 1) % m;
            if (q->ring_if_better && !(snapc[k] < snapc[dst])) continue;
            copy_perm(s->PG + (size_t)dst * n, snap + (size_t)k * n, n);
            s->costG[dst] = snapc[k];
        }
        free(snap);
        free(snapc);
    }
}

/* ------------------------------------------------------------------ init */

/* Random particles (section 3.3: generated at start): X(0) by Fisher-Yates with
 * Philox tag 2 (for i = n-1 .. 1: j = below(u, i + 1), swap), V(0) uniform in
 * [-v_max, v_max) with Philox tag 3 (element e = i n + j uses word e mod 4 of block
 * e / 4), formed in fp32 as v_max (2u - 1), then rounded to the storage format. */
void orc_init(const orc_params* q, int n, const int32_t* F, const int32_t* D, uint64_t seed,
              orc_state* s) {
    const int m = q->swarms, ss = q->swarm_size, P = m * ss;
    for (int k = 0; k < m; ++k)
        for (int pis = 0; pis < ss; ++pis) {
            const int idx = k * ss + pis;
            int32_t* p = s->X + (size_t)idx * n;
            for (int i = 0; i < n; ++i) p[i] = i;
            for (int i = n - 1; i >= 1; --i) {
                const int qd = n - 1 - i;
                uint32_t w[4];
                orc_draw(seed, (uint32_t)pis, (uint32_t)k, 0u, ORC_TAG_INIT_X, (uint32_t)(qd / 4), w);
                const int j = (int)orc_below(w[qd % 4], (uint32_t)(i + 1));
                int32_t tmp = p[i]; p[i] = p[j]; p[j] = tmp;
            }
            double* V = s->V + (size_t)idx * n * n;
            const float vmax = (float)q->v_max;
            for (int e = 0; e < n * n; ++e) {
                uint32_t w[4];
                orc_draw(seed, (uint32_t)pis, (uint32_t)k, 0u, ORC_TAG_INIT_V, (uint32_t)(e / 4), w);
                const float u = (float)orc_u01(w[e % 4]);
                const float v = vmax * (2.0f * u - 1.0f);
                V[e] = orc_round_storage((double)v, q->v_storage);
            }
            int64_t c;
            if (q->ls_at_init && q->ls_max_moves >= 0) {
                int64_t rd;
                orc_local_search(n, F, D, p, q->ls_max_moves, &c, &rd, NULL, 0);
            } else {
                c = orc_cost(n, F, D, p);
            }
            s->cost[idx] = c;
            s->costL[idx] = c;
            copy_perm(s->PL + (size_t)idx * n, p, n);
            if (s->moves) s->moves[idx] = 0;
        }
    for (int k = 0; k < m; ++k) s->costG[k] = INT64_MAX;
    *s->best_cost = INT64_MAX;
    /* the same bookkeeping as after an iteration, with no migration */
    orc_params q0 = *q;
    q0.mig_kind = 0;
    orc_bests_and_migration(&q0, n, seed, -1, s);
    *s->t = 0;
    for (int c = 0; c < ORC_NCOUNTERS; ++c) s->counters[c] = 0;
    (void)P;
}

/* ------------------------------------------------------------------ step */

void orc_step(const orc_params* q, int n, const int32_t* F, const int32_t* D, uint64_t seed,
              orc_state* s) {
    const int m = q->swarms, ss = q->swarm_size;
    const int t = *s->t;
    const int64_t npairs = (int64_t)n * (n - 1) / 2;
    double* Vn = (double*)malloc(sizeof(double) * n * n);
    int32_t* psx = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* pout = (int32_t*)malloc(sizeof(int32_t) * n);
    for (int k = 0; k < m; ++k)
        for (int pis = 0; pis < ss; ++pis) {
            const int idx = k * ss + pis;
            double* V = s->V + (size_t)idx * n * n;
            int32_t* x = s->X + (size_t)idx * n;
            int32_t mv, nt;
            int64_t rd, c;
            orc_particle_iteration(q, n, F, D, seed, t, k, pis, V, x, s->PL + (size_t)idx * n,
                                   s->PG + (size_t)k * n, Vn, psx, pout, &c, &mv, &rd, &nt);
            memcpy(V, Vn, sizeof(double) * n * n);
            copy_perm(x, pout, n);
            s->cost[idx] = c;
            if (c < s->costL[idx]) {
                s->costL[idx] = c;
                copy_perm(s->PL + (size_t)idx * n, x, n);
            }
            if (s->moves) s->moves[idx] = mv;
            s->counters[ORC_C_PIT] += 1;
            s->counters[ORC_C_MOVES] += mv;
            s->counters[ORC_C_ROUNDS] += rd;
            if (rd > 0) {
                s->counters[ORC_C_DELTA_FULL] += npairs;
                s->counters[ORC_C_DELTA_INCR] += (rd - 1) * npairs;
            }
            s->counters[ORC_C_TIES] += nt;
        }
    free(Vn);
    free(psx);
    free(pout);
    orc_bests_and_migration(q, n, seed, t, s);
    *s->t = t + 1;
}

/* ----------------------------------------------------------------- stats */

static int cmp_i64(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

/* Percentile ranks of the goal values of a population (section 4.2): nearest
 * rank, P_q = sorted[ceil(q N) - 1]. */
void orc_histogram(const int64_t* cost, int P, int64_t lo, int64_t hi, int bins, int64_t* counts) {
    for (int b = 0; b < bins + 2; ++b) counts[b] = 0;
    for (int i = 0; i < P; ++i) {
        if (cost[i] < lo) {
            counts[0] += 1;
        } else if (cost[i] >= hi) {
            counts[bins + 1] += 1;
        } else {
            /* the bin whose half-open interval [lo + b w, lo + (b + 1) w), w = (hi - lo) / bins,
               holds the cost, found by scanning the bins in order */
            for (int b = 0; b < bins; ++b) {
                /* cost < lo + (b + 1)(hi - lo) / bins  <=>  (cost - lo) bins < (b + 1)(hi - lo) */
                if ((__int128)(cost[i] - lo) * bins < (__int128)(b + 1) * (hi - lo)) {
                    counts[1 + b] += 1;
                    break;
                }
            }
        }
    }
}

void orc_stats(const int64_t* cost, int P, int64_t out[6], double* mean) {
    int64_t* v = (int64_t*)malloc(sizeof(int64_t) * P);
    memcpy(v, cost, sizeof(int64_t) * P);
    qsort(v, P, sizeof(int64_t), cmp_i64);
    static const int pct[4] = {5, 25, 50, 75};
    out[0] = v[0];
    for (int i = 0; i < 4; ++i) {
        int64_t rank = ((int64_t)pct[i] * P + 99) / 100; /* ceil(pct P / 100) */
        out[1 + i] = v[rank - 1];
    }
    out[5] = v[P - 1];
    /* mean: the exact integer sum of the costs divided by P, as the quotient plus
       remainder / P (the sum in 128 bits cannot overflow) */
    __int128 sum = 0;
    for (int i = 0; i < P; ++i) sum += v[i];
    const __int128 quo = sum / P, rem = sum % P;
    *mean = (double)(int64_t)quo + (double)(int64_t)rem / (double)P;
    free(v);
}
