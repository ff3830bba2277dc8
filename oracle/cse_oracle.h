/*
 * cse_oracle.h -- CPU oracle of the parallel heuristic CSE search.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-purpose C
 * restatement of the method of "Parallel Heuristic Exploration for Additive
 * Complexity Reduction in Fast Matrix Multiplication" (Perminov), used to
 * check the CUDA library.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may call it; the library never does.  It
 * shares no code, header or table with the CUDA path.
 *
 * Readings of points the paper leaves open (random generator, canonical
 * order, tie breaks, fixed-point alpha/beta, sharing clock) are stated next to
 * the code that takes them in cse_oracle.c.
 */
#ifndef CSE_ORACLE_H
#define CSE_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Search flag: Greedy-Intersections with one coin per candidate per step,
 * shared by every candidate it intersects (R9b in cse_oracle.c). */
#define ORACLE_GI_SHARED_COINS 1u

/* Strategy indices (Section 3.4); weights are given in this order. */
enum { OR_GI = 0, OR_GA = 1, OR_GR = 2, OR_WR = 3, OR_MIX = 4, OR_G = 5, OR_GP = 6, OR_NSTRAT = 7 };

/* Per-process summary used by the parity tests. */
typedef struct {
    int64_t best_cost;   /* Cost(E) of the process's best record            */
    int32_t best_len;    /* substitutions in that record                    */
    int32_t runs;        /* runs started                                    */
    uint64_t best_hash;  /* FNV-1a over the 32-bit entries of the record    */
    uint64_t traj_hash;  /* FNV-1a over the trajectory events               */
    int64_t ops;         /* algorithmic integer-op count of the trajectory  */
    int64_t substeps;    /* steps that made a substitution                  */
    int32_t best_strategy; /* strategy of the run of the best record (-1: none) */
    int32_t pad;
    int64_t method_ops;  /* the method's own op count (R15 in cse_oracle.c)  */
} oracle_digest;

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void oracle_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* The same for n counters ctr[4q..4q+3] under one key, into out[4q..4q+3]. */
void oracle_philox_n(const uint32_t* ctr, const uint32_t key[2], int64_t n, uint32_t* out);

/* A_naive(E) = sum over rows of (nnz - 1)  (Section 3.2.1). */
int64_t oracle_naive(const int8_t* mat, int32_t rows, int32_t cols);

/* Canonical pair frequencies of a matrix (Algorithm 1, Analysis).
 * Writes up to max_out candidates (c >= min_c) in canonical order:
 * keys[t] = ((j << 10 | i) << 1) | (s < 0) with i < j, counts[t] = c.
 * Returns the number of candidates (may exceed max_out). */
int32_t oracle_pairs(const int8_t* mat, int32_t rows, int32_t cols, int32_t min_c,
                     uint32_t* keys, int32_t* counts, int32_t max_out);

/* Applies a substitution list (entries i | j<<10 | (s<0)<<20) to a matrix.
 * out has rows x (cols + n) entries.  Returns Cost = n + A_naive(E_final), or
 * -1 if an entry is not a valid pair of existing variables. */
int64_t oracle_apply(const int8_t* mat, int32_t rows, int32_t cols, const int32_t* list,
                     int32_t n, int8_t* out);

/* Basic selection strategies on an explicit candidate list (canonical order)
 * with explicit 32-bit draws: kind in {OR_G, OR_GA, OR_WR, OR_GR}; u[] holds
 * the draws the strategy reads (ga: u[0]; wr: u[0]; gr: u[0] coin, u[1] ga or
 * wr draw).  Returns the selected index. */
int32_t oracle_select_basic(int32_t kind, const int32_t* counts, int32_t m, const uint32_t* u);

/* The strategy a Mixed step runs (Section 3.4, reading R7): r = (u * 15) >> 32
 * of the step's draw u; r in [0,8) gi, [8,12) ga, [12,14) gr, 14 wr. */
int32_t oracle_mix_strategy(uint32_t u);

/* A run's alpha and beta in units of 2^-16 from its draws (Section 3.4.2,
 * reading R8): a = (u * 32769) >> 32 in [0, 32768], so alpha in [0, 0.5];
 * b = 32768 + ((u * 32769) >> 32) in [32768, 65536], so beta in [0.5, 1]. */
int32_t oracle_alpha(uint32_t u);
int32_t oracle_beta(uint32_t u);

/* Greedy-Intersections scores (Section 3.4.2) with explicit coins:
 * coin_bits[p*m + q] is the coin of candidate q as seen from candidate p.
 * Writes score[p] = H(s_p) * 2^32 in exact integers and returns argmax. */
int32_t oracle_gi_scores_coins(const uint32_t* keys, const int32_t* counts, int32_t m,
                               uint32_t a, uint32_t b, const uint8_t* coin_bits, int64_t* score);

/* The Greedy-Intersections coins a process draws at step t for a candidate
 * list (reading R9: Philox, independent per scored candidate p and
 * intersecting candidate q; shared != 0: R9b, one coin per q and step):
 * coins[p * m + q] = the coin of q in p's score, 255 where p draws none
 * (q = p or q disjoint from p).  Returns the argmax of the scores. */
int32_t oracle_gi_philox_coins(const uint32_t* keys, const int32_t* counts, int32_t m, uint64_t seed,
                               int32_t proc, int64_t t, int32_t mat, int32_t shared, uint8_t* coins);

/* Greedy-Potential potential of every candidate (c >= 2, canonical order) of
 * a matrix: N_p = number of signed pairs that occur at least twice after a
 * trial substitution of p, all of which contain the fresh variable.  Writes
 * up to max_out values; returns the number of candidates. */
int32_t oracle_gp_potentials(const int8_t* mat, int32_t rows, int32_t cols, int32_t* pot, int32_t max_out);

/* The candidate (index in canonical order) Greedy-Potential picks on a
 * matrix for alpha = a / 2^16: the highest (c - 1) 2^16 + a N, lowest key on
 * ties; -1 when no pair repeats. */
int32_t oracle_gp_select(const int8_t* mat, int32_t rows, int32_t cols, int32_t a);

/* Brent equations of a scheme (m,n,p:r) (Section 3.1): U is r x (m n), V is
 * r x (n p), W is r x (m p), row-major, matrix entries in row-major order.
 * Returns the number of index triples (a_ij, b_j'k, c_i'k') whose sum over the
 * products differs from [j = j'][i = i'][k = k']; 0 for a valid scheme. */
int64_t oracle_brent_violations(int32_t m, int32_t n, int32_t p, int32_t r, const int8_t* U, const int8_t* V,
                                const int8_t* W);

/* One flip of the flip graph (Section 3.5.3, R16 in cse_oracle.c) on a scheme
 * of rank r with factor rows of len_u, len_v, len_w entries: if factor x
 * (0 U, 1 V, 2 W) of terms l != m agrees up to a sign sigma, (Y, Z) = the
 * other two factors in the order (x+1, x+2) (side 0) or (x+2, x+1) (side 1),
 * Y_l += sigma Y_m and Z_m -= Z_l, provided both stay ternary and nonzero.
 * Modifies U, V, W in place; returns 1 if the flip was applied, else 0. */
int32_t oracle_flip_apply(int32_t r, int32_t len_u, int32_t len_v, int32_t len_w, int8_t* U, int8_t* V, int8_t* W,
                          int32_t l, int32_t m, int32_t x, int32_t side);

/* Variant `variant` of flip iteration `iteration` of the scheme (m,n,p:r)
 * (R16): oU/oV/oW receive the input with F random ternary flips applied
 * (variant 0: the input).  Returns the number of flips applied. */
int32_t oracle_flip_variant(int32_t m, int32_t n, int32_t p, int32_t r, const int8_t* U, const int8_t* V,
                            const int8_t* W, uint64_t seed, int32_t iteration, int32_t variant, int32_t max_flips,
                            int8_t* oU, int8_t* oV, int8_t* oW);

/* Exhaustive minimum of Cost over all sequences of Algorithm 1 on a tiny
 * matrix (rows * cols small).  Returns the optimum, or -1 on overflow. */
int64_t oracle_bruteforce(const int8_t* mat, int32_t rows, int32_t cols, int32_t cap);

/* The full search (Sections 3.3-3.5, Algorithm 1) over n_mats expression sets.
 * weights7: gi, ga, gr, wr, mix, g, gp.  Outputs per matrix: best cost, length,
 * list (cap entries per matrix).  dig: n_mats * n_proc digests or NULL.
 * proc_subset: if non-NULL, only these processes are simulated (exact only
 * while no snapshot is published, i.e. budget <= interval).
 * Returns 0, or a negative error code for invalid arguments. */
int oracle_search(int32_t n_mats, const int8_t* const* mats, const int32_t* rows,
                  const int32_t* cols, const uint32_t* weights7, int32_t n_proc, uint64_t seed,
                  int64_t budget, int32_t interval, int32_t permille, int32_t cap,
                  int32_t n_threads, const int32_t* proc_subset, int32_t n_subset,
                  int64_t* out_cost, int32_t* out_len, int32_t* out_list, oracle_digest* dig);

/* The search in iteration mode (Sections 3.5.2 and 4; R14 in cse_oracle.c):
 * every process performs one whole run per iteration, sharing happens between
 * iterations, and the search ends after max_iterations iterations or when the
 * total best cost has not improved for `patience` consecutive iterations
 * (0: never early).  stats (or NULL): [0] iterations run, [1] process-steps. */
int oracle_search_iterations(int32_t n_mats, const int8_t* const* mats, const int32_t* rows,
                             const int32_t* cols, const uint32_t* weights7, int32_t n_proc, uint64_t seed,
                             int64_t max_iterations, int32_t patience, int32_t permille, int32_t cap,
                             uint32_t flags, int32_t n_threads, int64_t* out_cost, int32_t* out_len,
                             int32_t* out_list, oracle_digest* dig, int64_t* stats, int32_t* curve,
                             int32_t curve_cap);

/* oracle_search with search flags (ORACLE_GI_SHARED_COINS) and, if curve is
 * not NULL, the best-Cost curve: curve[mi * curve_cap + r] = the lowest best
 * record of matrix mi after round r (r < curve_cap).  The same curve is an
 * optional output of oracle_search_iterations (one round per iteration). */
int oracle_search_flags(int32_t n_mats, const int8_t* const* mats, const int32_t* rows,
                        const int32_t* cols, const uint32_t* weights7, int32_t n_proc, uint64_t seed,
                        int64_t budget, int32_t interval, int32_t permille, int32_t cap, uint32_t flags,
                        int32_t n_threads, const int32_t* proc_subset, int32_t n_subset,
                        int64_t* out_cost, int32_t* out_len, int32_t* out_list, oracle_digest* dig,
                        int32_t* curve, int32_t curve_cap);

/* The step-clock search with its best-Cost curve and, per matrix and round,
 * snap_hash[mi * curve_cap + r] = FNV-1a of the shared list in force after
 * round r (0 while none is published), for r < curve_cap. */
int oracle_search_snapshots(int32_t n_mats, const int8_t* const* mats, const int32_t* rows,
                            const int32_t* cols, const uint32_t* weights7, int32_t n_proc, uint64_t seed,
                            int64_t budget, int32_t interval, int32_t permille, int32_t cap, int32_t n_threads,
                            int64_t* out_cost, int32_t* curve, uint64_t* snap_hash, int32_t curve_cap);

#ifdef __cplusplus
}
#endif
#endif
