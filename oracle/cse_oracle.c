/*
 * cse_oracle.c -- CPU oracle of the parallel heuristic CSE search.
 *
 * TEST INFRASTRUCTURE ONLY (see cse_oracle.h).  Plain C11, written for a
 * reader checking it against the paper, not for speed:
 *   - an expression set is a dense ternary coefficient matrix coef[r][v]
 *     (the alpha_ij of Section 3.2.1), one row per expression, one column per
 *     variable x_v (0-based; fresh variable t is column n_x + t);
 *   - every step recounts all canonical pairs from the rows (Algorithm 1,
 *     Analysis) with a sort, instead of updating counts incrementally;
 *   - Greedy-Intersections scores every candidate against every other one,
 *     the O(m^2) loop the paper describes (Section 3.4.2).
 *
 * Readings taken where the paper is silent or leaves a choice:
 *   R1 canonical pair (i, j, s): i < j, s = alpha_i * alpha_j, i.e. the
 *      coefficient of x_i normalised to +1 (Section 3.3.1).  Canonical ORDER
 *      is ascending key ((j << 10 | i) << 1) | (s < 0): by the larger index
 *      first, then the smaller, '+' before '-'.
 *   R2 random numbers: Philox4x32-10 keyed by the 64-bit seed; counter
 *      (process, step t, matrix<<24 | purpose<<20 | extra_hi, extra_lo).
 *      Purposes: RUN (drawn at a run start; lane 0 strategy, lane 1 alpha,
 *      lane 2 beta, lane 3 share coin), SHAREK (lane 0: prefix length),
 *      STEP (drawn per step when the strategy needs it; lane 0 mix, lane 1
 *      gr coin, lane 2 ga, lane 3 wr) and GI (coins, R9).
 *   R3 g and gi break ties by the lowest canonical key.
 *   R4 ga: index (u * n_ties) >> 32 among the ties in canonical order.
 *   R5 wr: x = (u * T) >> 32 with T = sum(c - 1); the first candidate whose
 *      running sum of (c - 1) exceeds x.
 *   R6 gr: ga when u < 3 * 2^30 (p = 0.75), else wr, separate draws.
 *   R7 mix: per step, (u * 15) >> 32 in [0,8) gi, [8,12) ga, [12,14) gr,
 *      [14,15) wr (weights 8/4/2/1 of Section 3.4.3).
 *   R7b gp (Greedy-Potential, Section 2.2 and the weights of Section 3.5.1):
 *      the potential N_p of a candidate is the number of signed pairs that
 *      occur at least twice after a trial substitution of p -- only pairs with
 *      the fresh variable can be new; score (c_p - 1) 2^16 + a N_p with the
 *      run's alpha = a / 2^16 (R8); argmax, lowest key on ties.
 *   R8 alpha = a / 2^16 with a = (u * 32769) >> 32 in [0, 32768];
 *      beta = b / 2^16 with b = 32768 + ((u * 32769) >> 32) in [32768, 65536];
 *      both drawn at the start of every run.  gi score
 *      S_p = (c_p - 1) * 2^32 + a * (2^16 * D_p + b * X_p)  (= H * 2^32).
 *   R9 gi coins: for candidate p = (i, j, s) let A_v be the list of all
 *      candidates that contain x_v, in canonical order.  A candidate q != p
 *      containing x_i (slot 0) takes the bit at its position x in A_i of the
 *      64-bit word (lane 0 | lane 1 << 32); a candidate containing x_j but
 *      not x_i (slot 1) takes the bit at its position x in A_j of the word
 *      (lane 2 | lane 3 << 32); both words come from the draw with purpose
 *      GI, extra_hi = x >> 6 (bit x & 63), extra_lo = key(p).  Positions
 *      count every member of A_v, p and its sign twin included, so each
 *      intersecting q gets its own bit.  Coin 1: q survives with weight beta.
 *   R9b shared coins (option ORACLE_GI_SHARED_COINS; the paper gives only the
 *      marginals): every candidate q gets one coin per step, the same for
 *      every p that intersects it: bit q & 31 of word (q >> 5) & 3 of the draw
 *      with purpose GIS (4), extra_hi = q >> 7, extra_lo = 0.  The score is
 *      the same sum over intersecting q; the op count per step is 40 per
 *      128 candidates + 18 per candidate + 2 per column.
 *   R10 the step clock: every process performs one step per t.  A step
 *      first (re)starts the run if t == 0 or the previous run ended, then
 *      makes one substitution if a pair with c > 1 exists and a free column
 *      is left; after the substitution the run ends if no such pair remains
 *      or the columns are used up.  A fresh run with nothing to substitute
 *      ends at once (its step makes no substitution).
 *   R11 run start: close the old run into the process best (strictly lower
 *      cost replaces); strategy = g for process 0's first run, else drawn
 *      from the weights (u * sum) >> 32 against cumulative weights in the
 *      order gi, ga, gr, wr, mix, g, gp; if a snapshot exists and
 *      u < floor(permille * 2^32 / 1000), L = snapshot length, K = floor(3L/4),
 *      and if K >= 1 the first k = 1 + ((u' * K) >> 32) substitutions of the
 *      snapshot are replayed (Section 3.5.2).  Replays are not steps.
 *   R12 sharing boundary after step t when (t + 1) % interval == 0: each
 *      process folds its current run into its best (strictly lower cost),
 *      then per matrix the lowest (best cost, process) replaces the snapshot
 *      if its cost is strictly lower.  Runs started in the next round read
 *      that snapshot.
 *   R13 end of budget: every process folds its current run; the result per
 *      matrix is the lowest (best cost, process).
 *   R15 method op count (a second, engine-independent count of the work the
 *      method itself must do per step): a rewrite costs 6 per 64-bit word of
 *      a column (W64 = ceil(rows / 64)) plus the nnz of every rewritten row
 *      before the rewrite (the pair counts it changes); every selection scans
 *      the m candidates (m); Greedy-Intersections adds 2 per intersect term
 *      (one coin bit and one conditional add), with shared coins 4 per
 *      candidate instead (its weight into two per-variable sums, plain and
 *      coin-selected); Greedy-Potential adds per candidate a trial rewrite:
 *      6 W64 plus the nnz of the candidate's rows.
 *   R16 random flips (Section 3.5.3).  The move is the flip of the flip graph
 *      the paper cites: two rank-one terms l != m whose factor X agrees up to
 *      a sign, X_m = sigma X_l, with Y, Z the other two factors, become
 *        Y_l <- Y_l + sigma Y_m,   Z_m <- Z_m - Z_l,
 *      which keeps sum_l U_l (x) V_l (x) W_l, hence every Brent equation.  A
 *      ternary flip is one whose new Y_l and Z_m stay in {-1, 0, 1} and are
 *      not zero (the rank is kept).  Variant 0 of an iteration is the input;
 *      variant v >= 1 applies F = 1 + ((u * max_flips) >> 32) flips, u lane 0
 *      of the draw (process v, step = iteration, purpose FLIP, extra 0);
 *      attempt a = 0, 1, ... (at most 32 F) draws lane 0..3 of (process v,
 *      step = iteration, purpose FLIP, extra_lo = a + 1): l = (u0 r) >> 32,
 *      m = (u1 (r - 1)) >> 32 (+1 if >= l), X = (u2 3) >> 32 (U, V, W), and
 *      u3 & 1 picks (Y, Z) = (X+1, X+2) or (X+2, X+1) mod 3; an attempt that
 *      is not a ternary flip changes nothing.
 *   R14 iteration mode (Sections 3.5.2 and 4: the paper's own schedule).
 *      Iteration tau: every process performs one whole run, from its start
 *      (strategy, alpha, beta, share coin and prefix replay as in R11) until
 *      it ends; its steps carry the clock values t = tau * cap, tau * cap + 1,
 *      ... (a run has fewer than cap steps, so every draw keeps its own
 *      counter).  After the iteration every process folds, and the snapshot
 *      takes the lowest (best cost, process) if strictly lower.  The search
 *      stops after max_iterations iterations, or earlier when the sum over
 *      the matrices of the best cost has not decreased for `patience`
 *      consecutive iterations (the paper: unchanged for 10; patience 0 never
 *      stops early).  The first iteration always counts as an improvement.
 */
#include "cse_oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define KEY(i, j, neg) (((((uint32_t)(j)) << 10 | (uint32_t)(i)) << 1) | (uint32_t)(neg))
#define KEY_I(k) (((k) >> 1) & 0x3FFu)
#define KEY_J(k) (((k) >> 11) & 0x3FFu)
#define KEY_NEG(k) ((k) & 1u)
#define ENTRY(i, j, neg) ((int32_t)((uint32_t)(i) | ((uint32_t)(j) << 10) | ((uint32_t)(neg) << 20)))
#define ENT_I(e) ((int32_t)((uint32_t)(e) & 0x3FFu))
#define ENT_J(e) ((int32_t)(((uint32_t)(e) >> 10) & 0x3FFu))
#define ENT_NEG(e) ((int32_t)(((uint32_t)(e) >> 20) & 1u))

enum { PU_RUN = 0, PU_SHAREK = 1, PU_STEP = 2, PU_GI = 3, PU_GIS = 4, PU_FLIP = 5 };

/* ------------------------------------------------------------------ */
/* Philox4x32-10, from the definition in Salmon et al., SC'11:          */
/* round: (hi0,lo0) = M0*c0, (hi1,lo1) = M1*c2,                         */
/*        c' = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0);                 */
/* the key is bumped by the Weyl constants between rounds.              */
/* ------------------------------------------------------------------ */
void oracle_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void oracle_philox_n(const uint32_t* ctr, const uint32_t key[2], int64_t n, uint32_t* out) {
    for (int64_t q = 0; q < n; q++) oracle_philox(ctr + 4 * q, key, out + 4 * q);
}

static void draw4(uint64_t seed, int32_t proc, int64_t t, int32_t mat, int32_t purpose,
                  uint32_t extra_hi, uint32_t extra_lo, uint32_t out[4]) {
    uint32_t ctr[4] = {(uint32_t)proc, (uint32_t)t,
                       ((uint32_t)mat & 0xFFu) << 24 | ((uint32_t)purpose & 0xFu) << 20 |
                           (extra_hi & 0xFFFFFu),
                       extra_lo};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    oracle_philox(ctr, key, out);
}

static uint32_t draw(uint64_t seed, int32_t proc, int64_t t, int32_t mat, int32_t purpose) {
    uint32_t o[4];
    draw4(seed, proc, t, mat, purpose, 0, 0, o);
    return o[0];
}

/* (u * n) >> 32: an integer in [0, n) for a 32-bit draw u. */
static uint32_t scale(uint32_t u, uint64_t n) { return (uint32_t)(((uint64_t)u * n) >> 32); }

/* FNV-1a over 32-bit words (test digest only). */
static uint64_t fnv(uint64_t h, uint32_t w) {
    h ^= w;
    return h * 0x100000001B3ull;
}
#define FNV0 0xCBF29CE484222325ull

/* ------------------------------------------------------------------ */
/* Definitions of Section 3.2.1                                        */
/* ------------------------------------------------------------------ */
static int64_t naive_rows(const int8_t* coef, int32_t rows, int32_t ncols, int32_t stride) {
    int64_t s = 0;
    for (int32_t r = 0; r < rows; r++) {
        int32_t nnz = 0;
        for (int32_t v = 0; v < ncols; v++) nnz += coef[(int64_t)r * stride + v] != 0;
        s += nnz - 1;
    }
    return s;
}

int64_t oracle_naive(const int8_t* mat, int32_t rows, int32_t cols) {
    return naive_rows(mat, rows, cols, cols);
}

static int cmp_u32(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
}

/* Analysis step of Algorithm 1: every pair of nonzeros of every row gives one
 * occurrence of its canonical pair; equal keys are counted after a sort.
 * Candidates (c >= min_c) come out in canonical (ascending key) order. */
static int32_t count_pairs(const int8_t* coef, int32_t rows, int32_t ncols, int32_t stride,
                           int32_t min_c, uint32_t* scratch, int32_t* nzbuf, uint32_t* keys,
                           int32_t* cnt, int32_t max_out) {
    int64_t n = 0;
    for (int32_t r = 0; r < rows; r++) {
        const int8_t* row = coef + (int64_t)r * stride;
        int32_t nz = 0;
        for (int32_t v = 0; v < ncols; v++)
            if (row[v]) nzbuf[nz++] = v;
        for (int32_t x = 0; x < nz; x++)
            for (int32_t y = x + 1; y < nz; y++) {
                int32_t i = nzbuf[x], j = nzbuf[y];
                scratch[n++] = KEY(i, j, row[i] * row[j] < 0);
            }
    }
    qsort(scratch, (size_t)n, sizeof(uint32_t), cmp_u32);
    int32_t m = 0;
    for (int64_t a = 0; a < n;) {
        int64_t b = a;
        while (b < n && scratch[b] == scratch[a]) b++;
        if (b - a >= min_c) {
            if (m < max_out) {
                keys[m] = scratch[a];
                cnt[m] = (int32_t)(b - a);
            }
            m++;
        }
        a = b;
    }
    return m;
}

static int64_t max_pair_occurrences(const int8_t* coef, int32_t rows, int32_t ncols, int32_t stride) {
    int64_t s = 0;
    for (int32_t r = 0; r < rows; r++) {
        int64_t nnz = 0;
        for (int32_t v = 0; v < ncols; v++) nnz += coef[(int64_t)r * stride + v] != 0;
        s += nnz * (nnz - 1) / 2;
    }
    return s;
}

int32_t oracle_pairs(const int8_t* mat, int32_t rows, int32_t cols, int32_t min_c,
                     uint32_t* keys, int32_t* counts, int32_t max_out) {
    int64_t occ = max_pair_occurrences(mat, rows, cols, cols);
    uint32_t* scratch = (uint32_t*)malloc((size_t)(occ + 1) * sizeof(uint32_t));
    int32_t* nz = (int32_t*)malloc((size_t)(cols + 1) * sizeof(int32_t));
    int32_t m = count_pairs(mat, rows, cols, cols, min_c, scratch, nz, keys, counts, max_out);
    free(scratch);
    free(nz);
    return m;
}

/* Substitution (Section 3.2.1, Algorithm 1): fresh x_k = x_i + s x_j.  In
 * every row where x_i and x_j occur as (x_i + s x_j) or -(x_i + s x_j), both
 * coefficients become 0 and alpha_k becomes +1 or -1.  Returns c, the number
 * of rows rewritten. */
static int32_t substitute(int8_t* coef, int32_t rows, int32_t stride, int32_t k, int32_t i,
                          int32_t j, int32_t neg) {
    int32_t s = neg ? -1 : 1, c = 0;
    for (int32_t r = 0; r < rows; r++) {
        int8_t* row = coef + (int64_t)r * stride;
        if (row[i] != 0 && row[j] == s * row[i]) {
            row[k] = row[i];
            row[i] = 0;
            row[j] = 0;
            c++;
        }
    }
    return c;
}

int64_t oracle_apply(const int8_t* mat, int32_t rows, int32_t cols, const int32_t* list,
                     int32_t n, int8_t* out) {
    int32_t stride = cols + n;
    memset(out, 0, (size_t)rows * (size_t)stride);
    for (int32_t r = 0; r < rows; r++)
        for (int32_t v = 0; v < cols; v++) out[(int64_t)r * stride + v] = mat[(int64_t)r * cols + v];
    for (int32_t t = 0; t < n; t++) {
        int32_t i = ENT_I(list[t]), j = ENT_J(list[t]);
        if (!(i < j && j < cols + t)) return -1;
        substitute(out, rows, stride, cols + t, i, j, ENT_NEG(list[t]));
    }
    return n + naive_rows(out, rows, stride, stride);
}

/* ------------------------------------------------------------------ */
/* Selection strategies (Section 3.4)                                  */
/* ------------------------------------------------------------------ */
static int32_t sel_g(const int32_t* cnt, int32_t m) {
    int32_t best = 0;
    for (int32_t t = 1; t < m; t++)
        if (cnt[t] > cnt[best]) best = t;
    return best;
}

static int32_t sel_ga(const int32_t* cnt, int32_t m, uint32_t u) {
    int32_t cmax = 0, ties = 0;
    for (int32_t t = 0; t < m; t++)
        if (cnt[t] > cmax) cmax = cnt[t];
    for (int32_t t = 0; t < m; t++) ties += cnt[t] == cmax;
    uint32_t want = scale(u, (uint64_t)ties);
    for (int32_t t = 0; t < m; t++)
        if (cnt[t] == cmax) {
            if (want == 0) return t;
            want--;
        }
    return -1;
}

static int32_t sel_wr(const int32_t* cnt, int32_t m, uint32_t u) {
    uint64_t total = 0;
    for (int32_t t = 0; t < m; t++) total += (uint64_t)(cnt[t] - 1);
    uint64_t x = scale(u, total), acc = 0;
    for (int32_t t = 0; t < m; t++) {
        acc += (uint64_t)(cnt[t] - 1);
        if (acc > x) return t;
    }
    return -1;
}

static int32_t sel_gr(const int32_t* cnt, int32_t m, uint32_t coin, uint32_t u_ga, uint32_t u_wr) {
    return coin < 0xC0000000u ? sel_ga(cnt, m, u_ga) : sel_wr(cnt, m, u_wr);
}

int32_t oracle_select_basic(int32_t kind, const int32_t* counts, int32_t m, const uint32_t* u) {
    if (m <= 0) return -1;
    switch (kind) {
        case OR_G: return sel_g(counts, m);
        case OR_GA: return sel_ga(counts, m, u[0]);
        case OR_WR: return sel_wr(counts, m, u[0]);
        case OR_GR: return sel_gr(counts, m, u[0], u[1], u[1]);
        default: return -1;
    }
}

/* Coin source for Greedy-Intersections. */
typedef struct {
    /* Philox mode */
    uint64_t seed;
    int32_t proc, mat;
    int64_t t;
    const uint32_t* keys;
    uint32_t block[4];
    int32_t block_idx, block_p;
    int64_t philox_calls;
    /* explicit mode */
    const uint8_t* bits;
    int32_t m;
    /* shared mode (R9b): one coin per candidate q per step, seen by every p */
    int32_t shared, ncols;
    /* if not NULL: record[p * m + q] = every coin drawn (test output) */
    uint8_t* record;
} coin_src;

static int coin_draw(coin_src* cs, int32_t p, int32_t q, int32_t slot, int32_t rho);

static int coin_at(coin_src* cs, int32_t p, int32_t q, int32_t slot, int32_t rho) {
    int c = coin_draw(cs, p, q, slot, rho);
    if (cs->record) cs->record[(int64_t)p * cs->m + q] = (uint8_t)c;
    return c;
}

static int coin_draw(coin_src* cs, int32_t p, int32_t q, int32_t slot, int32_t rho) {
    if (cs->bits) return cs->bits[(int64_t)p * cs->m + q] != 0;
    if (cs->shared) {
        uint32_t o[4];
        draw4(cs->seed, cs->proc, cs->t, cs->mat, PU_GIS, (uint32_t)q >> 7, 0, o);
        return (int)((o[(q >> 5) & 3] >> (q & 31)) & 1u);
    }
    int32_t blk = rho >> 6;
    if (cs->block_p != p || cs->block_idx != blk) {
        draw4(cs->seed, cs->proc, cs->t, cs->mat, PU_GI, (uint32_t)blk, cs->keys[p], cs->block);
        cs->block_p = p;
        cs->block_idx = blk;
    }
    uint64_t w = slot == 0 ? ((uint64_t)cs->block[0] | (uint64_t)cs->block[1] << 32)
                           : ((uint64_t)cs->block[2] | (uint64_t)cs->block[3] << 32);
    return (int)((w >> (rho & 63)) & 1u);
}

/* Greedy-Intersections (Section 3.4.2):
 *   H(s_p) = (c_p - 1) + alpha * sum_{q != p} I(s_p, s_q),
 *   I = c_q - 1 for q disjoint from p; 0 or beta (c_q - 1), each with
 *   probability 1/2, for q sharing a variable with p.
 * In integers: S_p = (c_p-1) 2^32 + a (2^16 D_p + b X_p), with D_p the sum over
 * disjoint q and X_p the sum over intersecting q whose coin is 1.  Pairs with
 * c = 1 contribute 0, so only candidates enter the sums.  Returns the argmax
 * (lowest key on ties).  *ops_out receives the algorithmic op count. */
static int32_t sel_gi(const uint32_t* keys, const int32_t* cnt, int32_t m, uint32_t a, uint32_t b,
                      coin_src* cs, int64_t* score, int64_t* ops_out, int64_t* mops_out) {
    int64_t total = 0;
    for (int32_t q = 0; q < m; q++) total += cnt[q] - 1;
    int32_t best = -1;
    int64_t best_s = 0, ops = 0, terms = 0;
    for (int32_t p = 0; p < m; p++) {
        uint32_t i = KEY_I(keys[p]), j = KEY_J(keys[p]);
        int64_t wp = cnt[p] - 1, inter = 0, x = 0;
        int32_t pos0 = 0, pos1 = 0, n_inter = 0; /* positions in A_i and A_j */
        for (int32_t q = 0; q < m; q++) {
            uint32_t qi = KEY_I(keys[q]), qj = KEY_J(keys[q]);
            int hold_i = qi == i || qj == i, hold_j = qi == j || qj == j;
            int coin = -1;
            if (hold_i) {
                if (q != p) coin = coin_at(cs, p, q, 0, pos0);
                pos0++;
                if (hold_j) pos1++; /* p or its sign twin: a place in A_j, no slot-1 coin */
            } else if (hold_j) {
                coin = coin_at(cs, p, q, 1, pos1);
                pos1++;
            }
            if (coin < 0) continue;
            n_inter++;
            inter += cnt[q] - 1;
            if (coin) x += cnt[q] - 1;
        }
        int64_t d = total - wp - inter;
        int64_t s = (wp << 32) + (int64_t)a * ((d << 16) + (int64_t)b * x);
        if (score) score[p] = s;
        if (best < 0 || s > best_s) {
            best = p;
            best_s = s;
        }
        int32_t b0 = (pos0 + 63) >> 6, b1 = (pos1 + 63) >> 6;
        ops += 3 * (int64_t)n_inter + 8 + (n_inter ? 40 * (int64_t)(b0 > b1 ? b0 : b1) : 0);
        terms += n_inter;
    }
    /* shared coins: 40 per Philox block of 128 candidates, 18 per candidate
     * (its two per-variable sums and its score), 2 per column */
    if (cs->shared) ops = 40 * (int64_t)((m + 127) / 128) + 18 * (int64_t)m + 2 * (int64_t)cs->ncols;
    if (ops_out) *ops_out = ops;
    /* R15: the scan of m, then 2 per intersect term (shared coins: 4 per candidate) */
    if (mops_out) *mops_out = (int64_t)m + (cs->shared ? 4 * (int64_t)m : 2 * terms);
    return best;
}

int32_t oracle_gi_philox_coins(const uint32_t* keys, const int32_t* counts, int32_t m, uint64_t seed,
                               int32_t proc, int64_t t, int32_t mat, int32_t shared, uint8_t* coins) {
    coin_src cs;
    memset(&cs, 0, sizeof cs);
    cs.seed = seed;
    cs.proc = proc;
    cs.mat = mat;
    cs.t = t;
    cs.keys = keys;
    cs.block_p = -1;
    cs.shared = shared != 0;
    cs.m = m;
    cs.record = coins;
    if (m <= 0) return -1;
    memset(coins, 255, (size_t)m * (size_t)m);
    return sel_gi(keys, counts, m, 1, 32768, &cs, NULL, NULL, NULL);
}

int32_t oracle_gi_scores_coins(const uint32_t* keys, const int32_t* counts, int32_t m,
                               uint32_t a, uint32_t b, const uint8_t* coin_bits, int64_t* score) {
    coin_src cs;
    memset(&cs, 0, sizeof cs);
    cs.bits = coin_bits;
    cs.m = m;
    if (m <= 0) return -1;
    return sel_gi(keys, counts, m, a, b, &cs, score, NULL, NULL);
}

/* Greedy-Potential: a trial substitution of every candidate on a copy of
 * the expressions, then a recount of the pairs that contain the fresh
 * variable x_k (the only pairs whose count can grow). */
static int32_t gp_potential(const int8_t* coef, int32_t rows, int32_t ncols, int32_t stride, uint32_t key,
                            int8_t* trial, uint32_t* scratch, int32_t* live_out) {
    memcpy(trial, coef, (size_t)rows * (size_t)stride);
    const int32_t k = ncols;
    substitute(trial, rows, stride, k, (int32_t)KEY_I(key), (int32_t)KEY_J(key), (int32_t)KEY_NEG(key));
    int64_t n = 0;
    for (int32_t r = 0; r < rows; r++) {
        const int8_t* row = trial + (int64_t)r * stride;
        if (!row[k]) continue;
        for (int32_t u = 0; u < k; u++)
            if (row[u]) scratch[n++] = KEY(u, k, row[u] * row[k] < 0);
    }
    qsort(scratch, (size_t)n, sizeof(uint32_t), cmp_u32);
    int32_t pot = 0;
    for (int64_t a = 0; a < n;) {
        int64_t b = a;
        while (b < n && scratch[b] == scratch[a]) b++;
        pot += (b - a) >= 2;
        a = b;
    }
    if (live_out) {
        int32_t live = 0;
        for (int32_t u = 0; u < k; u++) {
            int32_t any = 0;
            for (int32_t r = 0; r < rows && !any; r++) any = trial[(int64_t)r * stride + u] != 0;
            live += any;
        }
        *live_out = live;
    }
    return pot;
}

/* Greedy-Potential selection: score (c - 1) 2^16 + a N for every candidate,
 * N its potential and a the run's alpha in units of 2^-16; argmax, lowest key
 * on ties.  *ops grows by the algorithmic op count (5 per word of a column per
 * live column of the trial system, plus 8, per candidate). */
static int64_t rows_nnz_of_pair(const int8_t* coef, int32_t rows, int32_t ncols, int32_t stride, int32_t i,
                                int32_t j, int32_t neg);

static int32_t gp_select(const int8_t* coef, int32_t rows, int32_t ncols, int32_t stride, const uint32_t* keys,
                         const int32_t* cnt, int32_t m, int32_t a, int32_t w32, int8_t* trial, uint32_t* scratch,
                         int64_t* ops, int64_t* mops) {
    int32_t best = -1;
    int64_t best_s = 0;
    for (int32_t p = 0; p < m; p++) {
        int32_t live = 0;
        int32_t pot = gp_potential(coef, rows, ncols, stride, keys[p], trial, scratch, &live);
        int64_t sc = ((int64_t)(cnt[p] - 1) << 16) + (int64_t)a * pot;
        if (best < 0 || sc > best_s) {
            best = p;
            best_s = sc;
        }
        if (ops) *ops += 5 * (int64_t)w32 * live + 8;
        /* R15: a trial rewrite, 6 per 64-bit word plus the nnz of the candidate's rows */
        if (mops)
            *mops += 6 * (int64_t)((rows + 63) / 64) +
                     rows_nnz_of_pair(coef, rows, ncols, stride, (int32_t)KEY_I(keys[p]), (int32_t)KEY_J(keys[p]),
                                      (int32_t)KEY_NEG(keys[p]));
    }
    if (mops) *mops += m;
    return best;
}

int32_t oracle_gp_select(const int8_t* mat, int32_t rows, int32_t cols, int32_t a) {
    const int32_t stride = cols + 1;
    int8_t* coef = (int8_t*)calloc((size_t)rows * (size_t)stride, 1);
    int8_t* trial = (int8_t*)calloc((size_t)rows * (size_t)stride, 1);
    for (int32_t r = 0; r < rows; r++)
        for (int32_t v = 0; v < cols; v++) coef[(int64_t)r * stride + v] = mat[(int64_t)r * cols + v];
    int64_t occ = max_pair_occurrences(mat, rows, cols, cols);
    uint32_t* scratch = (uint32_t*)malloc((size_t)(occ + (int64_t)rows * stride + 1) * 4);
    uint32_t* keys = (uint32_t*)malloc((size_t)(occ + 1) * 4);
    int32_t* cnt = (int32_t*)malloc((size_t)(occ + 1) * 4);
    int32_t* nz = (int32_t*)malloc((size_t)(cols + 1) * 4);
    int32_t m = count_pairs(coef, rows, cols, stride, 2, scratch, nz, keys, cnt, (int32_t)occ + 1);
    int32_t sel = m > 0 ? gp_select(coef, rows, cols, stride, keys, cnt, m, a, 1, trial, scratch, NULL, NULL) : -1;
    free(coef);
    free(trial);
    free(scratch);
    free(keys);
    free(cnt);
    free(nz);
    return sel;
}

int32_t oracle_gp_potentials(const int8_t* mat, int32_t rows, int32_t cols, int32_t* pot, int32_t max_out) {
    const int32_t stride = cols + 1;
    int8_t* coef = (int8_t*)calloc((size_t)rows * (size_t)stride, 1);
    int8_t* trial = (int8_t*)calloc((size_t)rows * (size_t)stride, 1);
    for (int32_t r = 0; r < rows; r++)
        for (int32_t v = 0; v < cols; v++) coef[(int64_t)r * stride + v] = mat[(int64_t)r * cols + v];
    int64_t occ = max_pair_occurrences(mat, rows, cols, cols);
    uint32_t* scratch = (uint32_t*)malloc((size_t)(occ + (int64_t)rows * stride + 1) * 4);
    uint32_t* keys = (uint32_t*)malloc((size_t)(occ + 1) * 4);
    int32_t* cnt = (int32_t*)malloc((size_t)(occ + 1) * 4);
    int32_t nz[1024];
    int32_t m = count_pairs(coef, rows, cols, stride, 2, scratch, nz, keys, cnt, (int32_t)occ + 1);
    for (int32_t p = 0; p < m && p < max_out; p++)
        pot[p] = gp_potential(coef, rows, cols, stride, keys[p], trial, scratch, NULL);
    free(coef);
    free(trial);
    free(scratch);
    free(keys);
    free(cnt);
    return m;
}

/* Brent equations (Section 3.1): for every entry a_ij of A, b_jk of B and
 * c_ik of C, sum over the r products of u_ij v_j'k w_i'k' must be 1 exactly
 * when j = j', i = i' and k = k', and 0 otherwise.  U, V, W are r x (m n),
 * r x (n p), r x (m p), entries in row-major order.  Returns the number of
 * (a, b, c) index triples whose sum is wrong. */
/* ------------------------------------------------------------------ */
/* Random flips (Section 3.5.3, R16)                                   */
/* ------------------------------------------------------------------ */
int32_t oracle_flip_apply(int32_t r, int32_t len_u, int32_t len_v, int32_t len_w, int8_t* U, int8_t* V, int8_t* W,
                          int32_t l, int32_t m, int32_t x, int32_t side) {
    int8_t* f[3] = {U, V, W};
    const int32_t len[3] = {len_u, len_v, len_w};
    if (l < 0 || m < 0 || l >= r || m >= r || l == m || x < 0 || x > 2) return 0;
    const int32_t y = (x + 1 + side) % 3, z = (x + 2 - side) % 3;
    const int8_t* xl = f[x] + (int64_t)l * len[x];
    const int8_t* xm = f[x] + (int64_t)m * len[x];
    int same = 1, opp = 1, nz = 0;
    for (int32_t i = 0; i < len[x]; i++) {
        same &= xm[i] == xl[i];
        opp &= xm[i] == -xl[i];
        nz |= xl[i] != 0;
    }
    if (!nz || !(same || opp)) return 0;
    const int sigma = same ? 1 : -1;
    int8_t* yl = f[y] + (int64_t)l * len[y];
    const int8_t* ym = f[y] + (int64_t)m * len[y];
    int8_t* zm = f[z] + (int64_t)m * len[z];
    const int8_t* zl = f[z] + (int64_t)l * len[z];
    int ynz = 0, znz = 0;
    for (int32_t i = 0; i < len[y]; i++) {
        int v = yl[i] + sigma * ym[i];
        if (v < -1 || v > 1) return 0;
        ynz |= v != 0;
    }
    for (int32_t i = 0; i < len[z]; i++) {
        int v = zm[i] - zl[i];
        if (v < -1 || v > 1) return 0;
        znz |= v != 0;
    }
    if (!ynz || !znz) return 0;
    for (int32_t i = 0; i < len[y]; i++) yl[i] = (int8_t)(yl[i] + sigma * ym[i]);
    for (int32_t i = 0; i < len[z]; i++) zm[i] = (int8_t)(zm[i] - zl[i]);
    return 1;
}

int32_t oracle_flip_variant(int32_t mm, int32_t nn, int32_t pp, int32_t r, const int8_t* U, const int8_t* V,
                            const int8_t* W, uint64_t seed, int32_t iteration, int32_t variant, int32_t max_flips,
                            int8_t* oU, int8_t* oV, int8_t* oW) {
    const int32_t lu = mm * nn, lv = nn * pp, lw = mm * pp;
    memcpy(oU, U, (size_t)r * lu);
    memcpy(oV, V, (size_t)r * lv);
    memcpy(oW, W, (size_t)r * lw);
    if (variant == 0 || r < 2 || max_flips < 1) return 0;
    const int32_t want = 1 + (int32_t)scale(draw(seed, variant, iteration, 0, PU_FLIP), (uint64_t)max_flips);
    int32_t done = 0;
    for (int32_t a = 0; a < 32 * want && done < want; a++) {
        uint32_t d[4];
        draw4(seed, variant, iteration, 0, PU_FLIP, 0, (uint32_t)(a + 1), d);
        int32_t l = (int32_t)scale(d[0], (uint64_t)r);
        int32_t m = (int32_t)scale(d[1], (uint64_t)(r - 1));
        if (m >= l) m++;
        const int32_t x = (int32_t)scale(d[2], 3);
        done += oracle_flip_apply(r, lu, lv, lw, oU, oV, oW, l, m, x, (int32_t)(d[3] & 1u));
    }
    return done;
}

int64_t oracle_brent_violations(int32_t m, int32_t n, int32_t p, int32_t r, const int8_t* U, const int8_t* V,
                                const int8_t* W) {
    int64_t bad = 0;
    for (int32_t i = 0; i < m; i++)
        for (int32_t j = 0; j < n; j++)
            for (int32_t j2 = 0; j2 < n; j2++)
                for (int32_t k = 0; k < p; k++)
                    for (int32_t i2 = 0; i2 < m; i2++)
                        for (int32_t k2 = 0; k2 < p; k2++) {
                            int64_t sum = 0;
                            for (int32_t l = 0; l < r; l++)
                                sum += (int64_t)U[(int64_t)l * m * n + i * n + j] *
                                       V[(int64_t)l * n * p + j2 * p + k] * W[(int64_t)l * m * p + i2 * p + k2];
                            int64_t want = (j == j2 && i == i2 && k == k2) ? 1 : 0;
                            bad += sum != want;
                        }
    return bad;
}

/* ------------------------------------------------------------------ */
/* Brute force over Algorithm 1 sequences (tiny matrices, test pin)     */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t rows, cap;
    uint64_t* hkeys;
    int64_t* hval;
    uint8_t* hused;
    int64_t hsize, hcount;
    int overflow;
} bf_ctx;

static uint64_t state_hash(const int8_t* coef, int32_t rows, int32_t ncols, int32_t stride) {
    uint64_t h = fnv(FNV0, (uint32_t)ncols);
    for (int32_t r = 0; r < rows; r++)
        for (int32_t v = 0; v < ncols; v++) h = fnv(h, (uint32_t)(coef[(int64_t)r * stride + v] + 1));
    return h;
}

static int64_t bf_rec(bf_ctx* bc, int8_t* coef, int32_t ncols, int32_t nf) {
    int32_t rows = bc->rows, stride = bc->cap;
    uint64_t h = state_hash(coef, rows, ncols, stride);
    int64_t slot = (int64_t)(h % (uint64_t)bc->hsize);
    while (bc->hused[slot]) {
        if (bc->hkeys[slot] == h) return bc->hval[slot] + nf;
        slot = (slot + 1) % bc->hsize;
    }
    int64_t occ = max_pair_occurrences(coef, rows, ncols, stride);
    uint32_t* scratch = (uint32_t*)malloc((size_t)(occ + 1) * 4);
    uint32_t* keys = (uint32_t*)malloc((size_t)(occ + 1) * 4);
    int32_t* cnt = (int32_t*)malloc((size_t)(occ + 1) * 4);
    int32_t nz[1024];
    int32_t m = count_pairs(coef, rows, ncols, stride, 2, scratch, nz, keys, cnt, (int32_t)occ + 1);
    /* remaining cost measured from this state: fresh additions still to be
     * made plus the final naive count */
    int64_t best;
    if (m == 0 || ncols >= stride) {
        best = naive_rows(coef, rows, ncols, stride);
    } else {
        best = -1;
        int8_t* next = (int8_t*)malloc((size_t)rows * (size_t)stride);
        for (int32_t p = 0; p < m; p++) {
            memcpy(next, coef, (size_t)rows * (size_t)stride);
            substitute(next, rows, stride, ncols, (int32_t)KEY_I(keys[p]), (int32_t)KEY_J(keys[p]),
                       (int32_t)KEY_NEG(keys[p]));
            int64_t v = bf_rec(bc, next, ncols + 1, 0) + 1;
            if (best < 0 || v < best) best = v;
        }
        free(next);
    }
    free(scratch);
    free(keys);
    free(cnt);
    if (bc->hcount * 2 >= bc->hsize) {
        bc->overflow = 1;
    } else {
        slot = (int64_t)(h % (uint64_t)bc->hsize);
        while (bc->hused[slot]) slot = (slot + 1) % bc->hsize;
        bc->hused[slot] = 1;
        bc->hkeys[slot] = h;
        bc->hval[slot] = best;
        bc->hcount++;
    }
    return best + nf;
}

int64_t oracle_bruteforce(const int8_t* mat, int32_t rows, int32_t cols, int32_t cap) {
    if (rows <= 0 || cols <= 0 || cap <= cols || cap > 1024) return -1;
    bf_ctx bc;
    memset(&bc, 0, sizeof bc);
    bc.rows = rows;
    bc.cap = cap;
    bc.hsize = 1 << 22;
    bc.hkeys = (uint64_t*)calloc((size_t)bc.hsize, 8);
    bc.hval = (int64_t*)calloc((size_t)bc.hsize, 8);
    bc.hused = (uint8_t*)calloc((size_t)bc.hsize, 1);
    int8_t* coef = (int8_t*)calloc((size_t)rows * (size_t)cap, 1);
    for (int32_t r = 0; r < rows; r++)
        for (int32_t v = 0; v < cols; v++) coef[(int64_t)r * cap + v] = mat[(int64_t)r * cols + v];
    int64_t v = bf_rec(&bc, coef, cols, 0);
    free(coef);
    free(bc.hkeys);
    free(bc.hval);
    free(bc.hused);
    return bc.overflow ? -1 : v;
}

/* ------------------------------------------------------------------ */
/* The parallel search (Sections 3.3 and 3.5)                          */
/* ------------------------------------------------------------------ */
typedef struct {
    int8_t* coef;      /* rows x cap: current expressions                */
    int32_t ncols;     /* n_x + n_f                                      */
    int32_t* run;      /* current run's substitution list F              */
    int32_t nf;
    int32_t strategy, a, b;
    int32_t ended;     /* run has ended; the next step starts a new one  */
    uint32_t* keys;    /* current candidates (c >= 2), canonical order   */
    int32_t* cnt;
    int32_t m;
    int64_t best_cost;
    int32_t best_len;
    int32_t best_strategy; /* strategy of the run that gave the best record, -1 = none */
    int32_t* best;
    int32_t runs;
    uint64_t traj;
    int64_t ops, substeps;
    int64_t mops;      /* R15 method op count                            */
} proc_t;

typedef struct {
    const int8_t* orig;
    int32_t rows, cols, w32;
    int64_t naive, max_occ;
    int64_t snap_cost;
    int32_t snap_len;
    int32_t* snap;
    proc_t* procs;
} mat_t;

typedef struct {
    int32_t n_mats, n_proc, interval, permille, cap;
    int32_t gi_shared;  /* R9b */
    uint64_t seed;
    uint32_t w[OR_NSTRAT];
    uint64_t wsum;
    mat_t* mats;
    const int32_t* subset;
    int32_t n_sub;
} search_t;

typedef struct {
    uint32_t* scratch;
    int32_t* nz;
    int8_t* trial;  /* Greedy-Potential trial copy of the expressions */
} work_t;

static int64_t run_cost(const search_t* S, const mat_t* M, const proc_t* P) {
    return P->nf + naive_rows(P->coef, M->rows, P->ncols, S->cap);
}

static void recount(const search_t* S, const mat_t* M, proc_t* P, work_t* wk) {
    P->m = count_pairs(P->coef, M->rows, P->ncols, S->cap, 2, wk->scratch, wk->nz, P->keys, P->cnt,
                       (int32_t)M->max_occ + 1);
}

/* Sum over the rows holding the pair (x_i + s x_j), s = -1 if neg, of the
 * row's number of nonzeros (R15). */
static int64_t rows_nnz_of_pair(const int8_t* coef, int32_t rows, int32_t ncols, int32_t stride, int32_t i,
                                int32_t j, int32_t neg) {
    int32_t s = neg ? -1 : 1;
    int64_t n = 0;
    for (int32_t r = 0; r < rows; r++) {
        const int8_t* row = coef + (int64_t)r * stride;
        if (row[i] == 0 || row[j] != s * row[i]) continue;
        for (int32_t v = 0; v < ncols; v++) n += row[v] != 0;
    }
    return n;
}

/* Candidates whose count a substitution of (i, j) can change: those that
 * contain x_i or x_j (counted for the algorithmic op total). */
static int64_t touching(const proc_t* P, int32_t i, int32_t j) {
    int64_t n = 0;
    for (int32_t q = 0; q < P->m; q++) {
        int32_t qi = (int32_t)KEY_I(P->keys[q]), qj = (int32_t)KEY_J(P->keys[q]);
        n += (qi == i || qj == i || qi == j || qj == j);
    }
    return n;
}

static int32_t live_columns_below(const search_t* S, const mat_t* M, const proc_t* P, int32_t k) {
    int32_t n = 0;
    for (int32_t v = 0; v < k; v++) {
        int32_t any = 0;
        for (int32_t r = 0; r < M->rows && !any; r++) any = P->coef[(int64_t)r * S->cap + v] != 0;
        n += any;
    }
    return n;
}

/* One substitution of canonical pair key into process P; the candidate list
 * is recounted afterwards.  Algorithmic ops: the rewrite (10 per 32-bit word
 * of a column) plus 5 per word for every pair count that can change: the
 * candidates containing x_i or x_j, and x_k against every live column. */
static int32_t do_subst(const search_t* S, const mat_t* M, proc_t* P, work_t* wk, uint32_t key) {
    int32_t i = (int32_t)KEY_I(key), j = (int32_t)KEY_J(key), neg = (int32_t)KEY_NEG(key);
    int64_t nij = touching(P, i, j);
    /* R15: 6 per 64-bit word of a column, plus the nnz of the rewritten rows */
    P->mops += 6 * (int64_t)((M->rows + 63) / 64) + rows_nnz_of_pair(P->coef, M->rows, P->ncols, S->cap, i, j, neg);
    int32_t k = P->ncols;
    int32_t c = substitute(P->coef, M->rows, S->cap, k, i, j, neg);
    P->ncols++;
    P->run[P->nf++] = ENTRY(i, j, neg);
    int64_t nu = live_columns_below(S, M, P, k);
    P->ops += 10 * (int64_t)M->w32 + 5 * (int64_t)M->w32 * (nij + nu);
    recount(S, M, P, wk);
    return c;
}

static void fold(const search_t* S, const mat_t* M, proc_t* P) {
    int64_t c = run_cost(S, M, P);
    if (c < P->best_cost) {
        P->best_cost = c;
        P->best_len = P->nf;
        P->best_strategy = P->strategy;
        memcpy(P->best, P->run, (size_t)P->nf * sizeof(int32_t));
    }
}

/* R8: a run's alpha and beta in units of 2^-16, from its draws. */
int32_t oracle_alpha(uint32_t u) { return (int32_t)scale(u, 32769); }
int32_t oracle_beta(uint32_t u) { return 32768 + (int32_t)scale(u, 32769); }

static void start_run(const search_t* S, int32_t mi, int32_t pi, int64_t t, work_t* wk) {
    mat_t* M = &S->mats[mi];
    proc_t* P = &M->procs[pi];
    if (t > 0) fold(S, M, P);
    P->runs++;
    uint32_t run[4];
    draw4(S->seed, pi, t, mi, PU_RUN, 0, 0, run);
    if (pi == 0 && t == 0) {
        P->strategy = OR_G;
    } else {
        uint32_t x = scale(run[0], S->wsum);
        uint64_t acc = 0;
        P->strategy = -1;
        for (int32_t s = 0; s < OR_NSTRAT; s++) {
            acc += S->w[s];
            if (x < acc) {
                P->strategy = s;
                break;
            }
        }
    }
    P->a = oracle_alpha(run[1]);
    P->b = oracle_beta(run[2]);
    /* fresh copy of the original expressions */
    memset(P->coef, 0, (size_t)M->rows * (size_t)S->cap);
    for (int32_t r = 0; r < M->rows; r++)
        for (int32_t v = 0; v < M->cols; v++)
            P->coef[(int64_t)r * S->cap + v] = M->orig[(int64_t)r * M->cols + v];
    P->ncols = M->cols;
    P->nf = 0;
    recount(S, M, P, wk);
    int32_t k = 0;
    if (M->snap_cost < INT64_MAX) {
        uint64_t thr = ((uint64_t)S->permille << 32) / 1000u;
        if ((uint64_t)run[3] < thr) {
            int32_t big_k = (3 * M->snap_len) / 4;
            if (big_k >= 1) k = 1 + (int32_t)scale(draw(S->seed, pi, t, mi, PU_SHAREK), (uint64_t)big_k);
        }
    }
    for (int32_t e = 0; e < k; e++) {
        int32_t ent = M->snap[e];
        do_subst(S, M, P, wk, KEY(ENT_I(ent), ENT_J(ent), ENT_NEG(ent)));
    }
    P->ended = 0;
    P->traj = fnv(P->traj, (uint32_t)t);
    P->traj = fnv(P->traj, 0xA0000000u | (uint32_t)P->strategy << 12 | (uint32_t)k);
}

int32_t oracle_mix_strategy(uint32_t u) {
    uint32_t r = scale(u, 15);
    return r < 8 ? OR_GI : r < 12 ? OR_GA : r < 14 ? OR_GR : OR_WR;
}

static int32_t choose(const search_t* S, int32_t mi, int32_t pi, int64_t t, proc_t* P, work_t* wk) {
    int32_t strat = P->strategy;
    uint32_t d[4] = {0, 0, 0, 0};
    if (strat != OR_G && strat != OR_GI && strat != OR_GP) draw4(S->seed, pi, t, mi, PU_STEP, 0, 0, d);
    if (strat == OR_MIX) strat = oracle_mix_strategy(d[0]);
    switch (strat) {
        case OR_G: P->ops += 2 * (int64_t)P->m; P->mops += P->m; return sel_g(P->cnt, P->m);
        case OR_GA: P->ops += 2 * (int64_t)P->m; P->mops += P->m; return sel_ga(P->cnt, P->m, d[2]);
        case OR_WR: P->ops += 2 * (int64_t)P->m; P->mops += P->m; return sel_wr(P->cnt, P->m, d[3]);
        case OR_GR: P->ops += 2 * (int64_t)P->m; P->mops += P->m; return sel_gr(P->cnt, P->m, d[1], d[2], d[3]);
        case OR_GI: {
            coin_src cs;
            memset(&cs, 0, sizeof cs);
            cs.seed = S->seed;
            cs.proc = pi;
            cs.mat = mi;
            cs.t = t;
            cs.keys = P->keys;
            cs.block_p = -1;
            cs.shared = S->gi_shared;
            cs.ncols = P->ncols;
            int64_t ops = 0, mops = 0;
            int32_t sel = sel_gi(P->keys, P->cnt, P->m, (uint32_t)P->a, (uint32_t)P->b, &cs, NULL, &ops, &mops);
            P->ops += ops;
            P->mops += mops;
            return sel;
        }
        case OR_GP: {
            const mat_t* M = &S->mats[mi];
            return gp_select(P->coef, M->rows, P->ncols, S->cap, P->keys, P->cnt, P->m, P->a, M->w32, wk->trial,
                             wk->scratch, &P->ops, &P->mops);
        }
        default: return -1;
    }
}

static void step(const search_t* S, int32_t mi, int32_t pi, int64_t t, work_t* wk) {
    mat_t* M = &S->mats[mi];
    proc_t* P = &M->procs[pi];
    if (t == 0 || P->ended) start_run(S, mi, pi, t, wk);
    if (P->m == 0 || P->ncols >= S->cap) {
        P->ended = 1;
        return;
    }
    int32_t sel = choose(S, mi, pi, t, P, wk);
    uint32_t key = P->keys[sel];
    do_subst(S, M, P, wk, key);
    P->substeps++;
    P->traj = fnv(P->traj, (uint32_t)t);
    P->traj = fnv(P->traj, (uint32_t)P->run[P->nf - 1]);
    if (P->m == 0 || P->ncols >= S->cap) P->ended = 1;
}

typedef struct {
    const search_t* S;
    int64_t t0, t1;
    int64_t u0, u1; /* unit range: unit = mi * n_sub + subset index */
    int32_t whole_run; /* iteration mode: one whole run per process, from step t0 */
    int64_t steps;     /* steps executed by this job (iteration mode) */
    work_t wk;
} job_t;

static void* run_job(void* arg) {
    job_t* J = (job_t*)arg;
    const search_t* S = J->S;
    for (int64_t u = J->u0; u < J->u1; u++) {
        int32_t mi = (int32_t)(u / S->n_sub);
        int32_t pi = S->subset[u % S->n_sub];
        if (J->whole_run) {
            /* one iteration of Section 3.5.2: the run goes on until it ends */
            int64_t t = J->t0;
            do {
                step(S, mi, pi, t, &J->wk);
                t++;
            } while (!S->mats[mi].procs[pi].ended);
            J->steps += t - J->t0;
        } else {
            for (int64_t t = J->t0; t < J->t1; t++) step(S, mi, pi, t, &J->wk);
        }
    }
    return NULL;
}

static int valid_matrix(const int8_t* m, int32_t rows, int32_t cols) {
    for (int32_t r = 0; r < rows; r++) {
        int32_t nnz = 0;
        for (int32_t v = 0; v < cols; v++) {
            int8_t x = m[(int64_t)r * cols + v];
            if (x < -1 || x > 1) return 0;
            nnz += x != 0;
        }
        if (nnz == 0) return 0;
    }
    return 1;
}

/* The search in either mode.  interval >= 1: the step clock (R10-R13),
 * budget = steps.  interval == 0: iteration mode (R14), budget = maximum
 * iterations, patience as stated there.  stats (may be NULL): [0] rounds
 * run (steps rounded up to intervals, or iterations), [1] process-steps. */
static int search_impl(int32_t n_mats, const int8_t* const* mats, const int32_t* rows,
                       const int32_t* cols, const uint32_t* weights7, int32_t n_proc, uint64_t seed,
                       int64_t budget, int32_t interval, int32_t patience, int32_t permille, int32_t cap,
                       uint32_t flags, int32_t n_threads, const int32_t* proc_subset, int32_t n_subset,
                       int64_t* out_cost, int32_t* out_len, int32_t* out_list, oracle_digest* dig,
                       int64_t* stats, int32_t* curve, uint64_t* snap_hash, int32_t curve_cap) {
    if (flags & ~(uint32_t)ORACLE_GI_SHARED_COINS) return -1;
    if (n_mats < 1 || n_mats > 256 || n_proc < 1 || budget < 0 || interval < 0 || patience < 0 ||
        permille < 0 || permille > 1000 || cap < 2 || cap > 1024)
        return -1;
    if (interval == 0 && (proc_subset || budget > INT32_MAX / cap)) return -1;
    search_t S;
    memset(&S, 0, sizeof S);
    S.n_mats = n_mats;
    S.n_proc = n_proc;
    S.interval = interval;
    S.permille = permille;
    S.cap = cap;
    S.seed = seed;
    S.gi_shared = (flags & ORACLE_GI_SHARED_COINS) != 0;
    for (int32_t s = 0; s < OR_NSTRAT; s++) {
        S.w[s] = weights7[s];
        S.wsum += weights7[s];
    }
    if (S.wsum == 0 || S.wsum > 0xFFFFFFFFull) return -1;
    for (int32_t mi = 0; mi < n_mats; mi++)
        if (rows[mi] < 1 || rows[mi] > 256 || cols[mi] < 1 || cols[mi] >= cap ||
            !valid_matrix(mats[mi], rows[mi], cols[mi]))
            return -1;
    int32_t* all = NULL;
    if (proc_subset) {
        for (int32_t s = 0; s < n_subset; s++)
            if (proc_subset[s] < 0 || proc_subset[s] >= n_proc) return -1;
        S.subset = proc_subset;
        S.n_sub = n_subset;
    } else {
        all = (int32_t*)malloc((size_t)n_proc * sizeof(int32_t));
        for (int32_t p = 0; p < n_proc; p++) all[p] = p;
        S.subset = all;
        S.n_sub = n_proc;
    }
    if (n_threads < 1) n_threads = 1;

    S.mats = (mat_t*)calloc((size_t)n_mats, sizeof(mat_t));
    int64_t max_occ_all = 0;
    int32_t max_cols = 0, max_rows = 0;
    for (int32_t mi = 0; mi < n_mats; mi++) {
        mat_t* M = &S.mats[mi];
        M->orig = mats[mi];
        M->rows = rows[mi];
        M->cols = cols[mi];
        M->w32 = (rows[mi] + 31) / 32;
        M->naive = oracle_naive(mats[mi], rows[mi], cols[mi]);
        M->max_occ = max_pair_occurrences(mats[mi], rows[mi], cols[mi], cols[mi]);
        if (M->max_occ > max_occ_all) max_occ_all = M->max_occ;
        if (cols[mi] > max_cols) max_cols = cols[mi];
        if (rows[mi] > max_rows) max_rows = rows[mi];
        M->snap_cost = INT64_MAX;
        M->snap = (int32_t*)calloc((size_t)cap, sizeof(int32_t));
        M->procs = (proc_t*)calloc((size_t)n_proc, sizeof(proc_t));
        for (int32_t s = 0; s < S.n_sub; s++) {
            proc_t* P = &M->procs[S.subset[s]];
            P->coef = (int8_t*)calloc((size_t)M->rows * (size_t)cap, 1);
            P->run = (int32_t*)calloc((size_t)cap, sizeof(int32_t));
            P->best = (int32_t*)calloc((size_t)cap, sizeof(int32_t));
            P->keys = (uint32_t*)calloc((size_t)M->max_occ + 1, sizeof(uint32_t));
            P->cnt = (int32_t*)calloc((size_t)M->max_occ + 1, sizeof(int32_t));
            P->best_cost = M->naive;
            P->best_len = 0;
            P->best_strategy = -1;
            P->traj = FNV0;
        }
    }

    int64_t units = (int64_t)n_mats * S.n_sub;
    if (n_threads > units) n_threads = (int32_t)(units > 0 ? units : 1);
    job_t* jobs = (job_t*)calloc((size_t)n_threads, sizeof(job_t));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int32_t k = 0; k < n_threads; k++) {
        jobs[k].S = &S;
        jobs[k].wk.scratch = (uint32_t*)malloc((size_t)(max_occ_all + (int64_t)max_rows * cap + 1) * sizeof(uint32_t));
        jobs[k].wk.nz = (int32_t*)malloc((size_t)(cap + 1) * sizeof(int32_t));
        jobs[k].wk.trial = (int8_t*)malloc((size_t)max_rows * (size_t)cap);
        jobs[k].u0 = units * k / n_threads;
        jobs[k].u1 = units * (k + 1) / n_threads;
    }

    int64_t rounds = 0, psteps = 0;
    int64_t best_total = INT64_MAX;
    int32_t stale = 0;
    const int64_t n_rounds = interval > 0 ? (budget + interval - 1) / interval : budget;
    for (int64_t rd = 0; rd < n_rounds; rd++) {
        int64_t t0 = interval > 0 ? rd * interval : rd * cap;
        int64_t t1 = interval > 0 ? (t0 + interval < budget ? t0 + interval : budget) : t0;
        for (int32_t k = 0; k < n_threads; k++) {
            jobs[k].t0 = t0;
            jobs[k].t1 = t1;
            jobs[k].whole_run = interval == 0;
        }
        if (n_threads == 1) {
            run_job(&jobs[0]);
        } else {
            for (int32_t k = 0; k < n_threads; k++) pthread_create(&th[k], NULL, run_job, &jobs[k]);
            for (int32_t k = 0; k < n_threads; k++) pthread_join(th[k], NULL);
        }
        rounds++;
        if (interval > 0) psteps += (t1 - t0) * n_mats * S.n_sub;
        /* sharing boundary (or end of budget): fold, then publish */
        int64_t total = 0;
        for (int32_t mi = 0; mi < n_mats; mi++) {
            mat_t* M = &S.mats[mi];
            int32_t win = -1;
            for (int32_t s = 0; s < S.n_sub; s++) {
                int32_t p = S.subset[s];
                fold(&S, M, &M->procs[p]);
            }
            for (int32_t p = 0; p < n_proc; p++) {
                if (!M->procs[p].coef) continue;
                if (win < 0 || M->procs[p].best_cost < M->procs[win].best_cost) win = p;
            }
            int boundary = interval > 0 ? (t1 % interval == 0) : 1;
            if (boundary && win >= 0 && M->procs[win].best_cost < M->snap_cost) {
                M->snap_cost = M->procs[win].best_cost;
                M->snap_len = M->procs[win].best_len;
                memcpy(M->snap, M->procs[win].best, (size_t)M->snap_len * sizeof(int32_t));
            }
            if (win >= 0) total += M->procs[win].best_cost;
            /* the shared list in force after this round (FNV-1a; 0 = none) */
            if (snap_hash && rd < curve_cap) {
                uint64_t h = 0;
                if (M->snap_cost < INT64_MAX) {
                    h = FNV0;
                    for (int32_t e = 0; e < M->snap_len; e++) h = fnv(h, (uint32_t)M->snap[e]);
                }
                snap_hash[(int64_t)mi * curve_cap + rd] = h;
            }
            /* the best-Cost curve: the lowest best record after each round */
            if (curve && win >= 0 && rd < curve_cap) curve[(int64_t)mi * curve_cap + rd] = (int32_t)M->procs[win].best_cost;
        }
        if (interval == 0) {
            /* R14: convergence when the scheme's best total has not improved
             * for `patience` consecutive iterations */
            if (total < best_total) {
                best_total = total;
                stale = 0;
            } else {
                stale++;
            }
            if (patience > 0 && stale >= patience) break;
        }
    }
    for (int32_t k = 0; k < n_threads; k++) psteps += jobs[k].steps;
    if (stats) {
        stats[0] = rounds;
        stats[1] = psteps;
    }
    /* budget == 0: results are the inputs */

    for (int32_t mi = 0; mi < n_mats; mi++) {
        mat_t* M = &S.mats[mi];
        int32_t win = -1;
        for (int32_t p = 0; p < n_proc; p++) {
            proc_t* P = &M->procs[p];
            if (!P->coef) continue;
            if (win < 0 || P->best_cost < M->procs[win].best_cost) win = p;
            if (dig) {
                oracle_digest* d = &dig[(int64_t)mi * n_proc + p];
                d->best_cost = P->best_cost;
                d->best_len = P->best_len;
                d->runs = P->runs;
                uint64_t h = FNV0;
                for (int32_t e = 0; e < P->best_len; e++) h = fnv(h, (uint32_t)P->best[e]);
                d->best_hash = h;
                d->traj_hash = P->traj;
                d->ops = P->ops;
                d->method_ops = P->mops;
                d->substeps = P->substeps;
                d->best_strategy = P->best_strategy;
                d->pad = 0;
            }
        }
        if (out_cost) out_cost[mi] = M->procs[win].best_cost;
        if (out_len) out_len[mi] = M->procs[win].best_len;
        if (out_list) {
            memset(out_list + (int64_t)mi * cap, 0, (size_t)cap * sizeof(int32_t));
            memcpy(out_list + (int64_t)mi * cap, M->procs[win].best,
                   (size_t)M->procs[win].best_len * sizeof(int32_t));
        }
    }

    for (int32_t k = 0; k < n_threads; k++) {
        free(jobs[k].wk.scratch);
        free(jobs[k].wk.nz);
        free(jobs[k].wk.trial);
    }
    free(jobs);
    free(th);
    for (int32_t mi = 0; mi < n_mats; mi++) {
        mat_t* M = &S.mats[mi];
        for (int32_t p = 0; p < n_proc; p++) {
            proc_t* P = &M->procs[p];
            free(P->coef);
            free(P->run);
            free(P->best);
            free(P->keys);
            free(P->cnt);
        }
        free(M->procs);
        free(M->snap);
    }
    free(S.mats);
    free(all);
    return 0;
}

int oracle_search(int32_t n_mats, const int8_t* const* mats, const int32_t* rows,
                  const int32_t* cols, const uint32_t* weights7, int32_t n_proc, uint64_t seed,
                  int64_t budget, int32_t interval, int32_t permille, int32_t cap,
                  int32_t n_threads, const int32_t* proc_subset, int32_t n_subset,
                  int64_t* out_cost, int32_t* out_len, int32_t* out_list, oracle_digest* dig) {
    if (interval < 1) return -1;
    return search_impl(n_mats, mats, rows, cols, weights7, n_proc, seed, budget, interval, 0, permille, cap, 0,
                       n_threads, proc_subset, n_subset, out_cost, out_len, out_list, dig, NULL, NULL, NULL, 0);
}

int oracle_search_flags(int32_t n_mats, const int8_t* const* mats, const int32_t* rows,
                        const int32_t* cols, const uint32_t* weights7, int32_t n_proc, uint64_t seed,
                        int64_t budget, int32_t interval, int32_t permille, int32_t cap, uint32_t flags,
                        int32_t n_threads, const int32_t* proc_subset, int32_t n_subset,
                        int64_t* out_cost, int32_t* out_len, int32_t* out_list, oracle_digest* dig,
                        int32_t* curve, int32_t curve_cap) {
    if (interval < 1) return -1;
    return search_impl(n_mats, mats, rows, cols, weights7, n_proc, seed, budget, interval, 0, permille, cap,
                       flags, n_threads, proc_subset, n_subset, out_cost, out_len, out_list, dig, NULL, curve,
                       NULL, curve_cap);
}

int oracle_search_snapshots(int32_t n_mats, const int8_t* const* mats, const int32_t* rows,
                            const int32_t* cols, const uint32_t* weights7, int32_t n_proc, uint64_t seed,
                            int64_t budget, int32_t interval, int32_t permille, int32_t cap, int32_t n_threads,
                            int64_t* out_cost, int32_t* curve, uint64_t* snap_hash, int32_t curve_cap) {
    if (interval < 1) return -1;
    return search_impl(n_mats, mats, rows, cols, weights7, n_proc, seed, budget, interval, 0, permille, cap, 0,
                       n_threads, NULL, 0, out_cost, NULL, NULL, NULL, NULL, curve, snap_hash, curve_cap);
}

int oracle_search_iterations(int32_t n_mats, const int8_t* const* mats, const int32_t* rows,
                             const int32_t* cols, const uint32_t* weights7, int32_t n_proc, uint64_t seed,
                             int64_t max_iterations, int32_t patience, int32_t permille, int32_t cap,
                             uint32_t flags, int32_t n_threads, int64_t* out_cost, int32_t* out_len,
                             int32_t* out_list, oracle_digest* dig, int64_t* stats, int32_t* curve,
                             int32_t curve_cap) {
    return search_impl(n_mats, mats, rows, cols, weights7, n_proc, seed, max_iterations, 0, patience, permille,
                       cap, flags, n_threads, NULL, 0, out_cost, out_len, out_list, dig, stats, curve, NULL,
                       curve_cap);
}
