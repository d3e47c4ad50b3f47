/*
 * QAP goal function, swap-move values, best-improvement local search and
 * brute force. TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

/* Goal function of section 2.1 in permutation form: the assignment p places
 * facility i at location p[i]; cost = sum_i sum_j f_ij d_{p(i) p(j)}. */
int64_t orc_cost(int n, const int32_t* F, const int32_t* D, const int32_t* p) {
    int64_t total = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            total += (int64_t)F[i * n + j] * (int64_t)D[p[i] * n + p[j]];
    return total;
}

/* Eq. 1 written out literally: the quadruple sum over f_ij d_kl x_ki x_lj with
 * the permutation matrix x_ki = 1 iff k = p(i) (Eq. 2). O(n^4); tests only. */
int64_t orc_cost_eq1(int n, const int32_t* F, const int32_t* D, const int32_t* p) {
    int64_t total = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k)
                for (int l = 0; l < n; ++l) {
                    int x_ki = (p[i] == k);
                    int x_lj = (p[j] == l);
                    total += (int64_t)F[i * n + j] * (int64_t)D[k * n + l] * x_ki * x_lj;
                }
    return total;
}

/* Change of the goal function when facilities r and s exchange locations,
 * p' = p o (r s). The paper names no local search; this is the classical O(n)
 * swap-move value for general (asymmetric, nonzero-diagonal) F and D used in
 * Taillard's robust tabu search for the QAP (1991/1995): every term of the
 * double sum whose row or column index is r or s changes, the others do not. */
int64_t orc_delta(int n, const int32_t* F, const int32_t* D, const int32_t* p, int r, int s) {
    const int pr = p[r], ps = p[s];
    int64_t d = 0;
    /* i, j both in {r, s} */
    d += (int64_t)(F[r * n + r] - F[s * n + s]) * (int64_t)(D[ps * n + ps] - D[pr * n + pr]);
    d += (int64_t)(F[r * n + s] - F[s * n + r]) * (int64_t)(D[ps * n + pr] - D[pr * n + ps]);
    /* exactly one of i, j in {r, s} */
    for (int k = 0; k < n; ++k) {
        if (k == r || k == s) continue;
        const int pk = p[k];
        d += (int64_t)(F[k * n + r] - F[k * n + s]) * (int64_t)(D[pk * n + ps] - D[pk * n + pr]);
        d += (int64_t)(F[r * n + k] - F[s * n + k]) * (int64_t)(D[ps * n + pk] - D[pr * n + pk]);
    }
    return d;
}

/* Best-improvement local search in the swap neighbourhood N(p) = {p o (r s)}.
 * Each round evaluates every pair r < s from scratch in r-major order, keeps the
 * smallest value (the first such pair on ties), and applies it only if it is
 * negative. Terminates because the integer cost strictly decreases. */
int orc_local_search(int n, const int32_t* F, const int32_t* D, int32_t* p, int max_moves,
                     int64_t* cost, int64_t* rounds, int32_t* trace, int trace_cap) {
    int moves = 0;
    int64_t nrounds = 0;
    int64_t c = orc_cost(n, F, D, p);
    for (;;) {
        if (max_moves > 0 && moves >= max_moves) break;
        int64_t best = 0;
        int br = -1, bs = -1;
        for (int r = 0; r < n; ++r)
            for (int s = r + 1; s < n; ++s) {
                int64_t d = orc_delta(n, F, D, p, r, s);
                if (br < 0 || d < best) { best = d; br = r; bs = s; }
            }
        ++nrounds;
        if (br < 0 || best >= 0) break;
        int32_t tmp = p[br]; p[br] = p[bs]; p[bs] = tmp;
        c += best;
        if (trace && moves < trace_cap) { trace[2 * moves] = br; trace[2 * moves + 1] = bs; }
        ++moves;
    }
    if (cost) *cost = c;
    if (rounds) *rounds = nrounds;
    return moves;
}

/* Exhaustive search over all n! assignments (lexicographic order); returns the
 * optimum and the lexicographically first optimal permutation. */
int64_t orc_brute_force(int n, const int32_t* F, const int32_t* D, int32_t* best_p) {
    int32_t p[16];
    if (n < 1 || n > 12) return -1;
    for (int i = 0; i < n; ++i) p[i] = i;
    int64_t best = orc_cost(n, F, D, p);
    memcpy(best_p, p, sizeof(int32_t) * n);
    for (;;) {
        /* next permutation in lexicographic order */
        int i = n - 2;
        while (i >= 0 && p[i] >= p[i + 1]) --i;
        if (i < 0) break;
        int j = n - 1;
        while (p[j] <= p[i]) --j;
        int32_t t = p[i]; p[i] = p[j]; p[j] = t;
        for (int a = i + 1, b = n - 1; a < b; ++a, --b) { t = p[a]; p[a] = p[b]; p[b] = t; }
        int64_t c = orc_cost(n, F, D, p);
        if (c < best) { best = c; memcpy(best_p, p, sizeof(int32_t) * n); }
    }
    return best;
}
