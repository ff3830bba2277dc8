// Step engine of the parallel heuristic CSE search on sm_103a: the device
// code of the round kernel, included by the two translation units that
// instantiate its variants (cse_kernels.cu: independent coins per pair;
// cse_kernels_gs.cu: shared coins).
//
// One warp runs one process (Section 3.5.1).  Its expression set lives in
// shared memory as column bitsets: column v holds W 32-bit words of "rows
// with alpha_rv = +1" and W words of "rows with alpha_rv = -1" (uint2 x / y).
// Pair frequencies (Algorithm 1, Analysis) are AND + popc over those words:
// for columns a, b with rows-present masks A = Pa|Na, B = Pb|Nb,
//   c(a,b,-) = popc((Pa ^ Pb) & A & B),  c(a,b,+) = popc(A & B) - c(a,b,-).
// The candidate set (canonical pairs with c >= 2) is kept as a list sorted by
// key = hi << 11 | lo << 1 | (s < 0), i.e. by the larger index first.  A
// substitution x_k = x_i + s x_j only changes pairs that contain x_i, x_j or
// the new x_k, and x_k is the largest index so far, so after each step the
// list is updated in place: candidates containing x_i or x_j are recounted
// (a stable compaction drops those that fell below 2) and the pairs (u, k)
// are appended in order.  No step recounts the whole matrix.
//
// Every random draw is Philox4x32-10 (Salmon et al., SC'11) with key = seed
// and counter (process, t, matrix << 24 | purpose << 20 | extra_hi,
// extra_lo); all lanes of a warp evaluate the same draw, so no shuffles are
// needed to share it.

#pragma once

#include <algorithm>
#include <climits>
#include <cstdint>
#include <map>
#include <mutex>
#include <utility>

#include "cse_internal.h"

namespace cse {

#define FULL_MASK 0xFFFFFFFFu

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Philox4x32-10: round (hi0,lo0) = M0*c0, (hi1,lo1) = M1*c2,
// c' = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); key += Weyl constants.
__device__ __forceinline__ void philox(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                       uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
}

__device__ __forceinline__ uint32_t scale32(uint32_t u, uint32_t n) {
    return (uint32_t)(((uint64_t)u * n) >> 32);
}

__device__ __forceinline__ uint64_t fnv(uint64_t h, uint32_t w) { return (h ^ w) * 0x100000001B3ull; }

__device__ __forceinline__ int key_lo(uint32_t e) { return (int)((e >> 1) & 1023u); }
__device__ __forceinline__ int key_hi(uint32_t e) { return (int)((e >> 11) & 1023u); }
__device__ __forceinline__ int cand_c(uint32_t e) { return (int)(e >> 21); }
__device__ __forceinline__ uint32_t make_cand(int lo, int hi, int neg, int c) {
    return ((uint32_t)hi << 11) | ((uint32_t)lo << 1) | (uint32_t)neg | ((uint32_t)c << 21);
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL_MASK, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// The warp's argmax of Greedy-Intersections scores, lowest candidate index
// on ties: each lane holds its best (score, index), index -1 for none.  Every
// score is at least 2^32 (its immediate-gain term), so "none" maps to 0 and
// three 32-bit warp reductions (high word, low word, index) replace a 64-bit
// butterfly.
__device__ __forceinline__ int warp_argmax_score(long long best_s, int best_q) {
    const unsigned long long us = best_q >= 0 ? (unsigned long long)best_s : 0ull;
    const uint32_t hi = (uint32_t)(us >> 32), lo = (uint32_t)us;
    const uint32_t mhi = __reduce_max_sync(FULL_MASK, hi);
    const uint32_t mlo = __reduce_max_sync(FULL_MASK, hi == mhi ? lo : 0u);
    return (int)__reduce_min_sync(FULL_MASK, (hi == mhi && lo == mlo && best_q >= 0) ? (uint32_t)best_q : 0xFFFFFFFFu);
}

// 8 x 8 bit transpose (Hacker's Delight, section 7-3: three rounds of
// masked swaps): byte i of x is the weight of position i; byte k of the
// result holds bit k of the eight weights, position i at bit i.
__device__ __forceinline__ unsigned long long transpose8x8(unsigned long long x) {
    unsigned long long t;
    t = (x ^ (x >> 7)) & 0x00AA00AA00AA00AAull;
    x = x ^ t ^ (t << 7);
    t = (x ^ (x >> 14)) & 0x0000CCCC0000CCCCull;
    x = x ^ t ^ (t << 14);
    t = (x ^ (x >> 28)) & 0x00000000F0F0F0F0ull;
    x = x ^ t ^ (t << 28);
    return x;
}

// 4 x 4 byte transpose with byte permutes: out[k] = byte k of a, b, c, d.
__device__ __forceinline__ void transpose4x4_bytes(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t out[4]) {
    const uint32_t t0 = __byte_perm(a, b, 0x5140), t1 = __byte_perm(a, b, 0x7362);
    const uint32_t t2 = __byte_perm(c, d, 0x5140), t3 = __byte_perm(c, d, 0x7362);
    out[0] = __byte_perm(t0, t2, 0x5410);
    out[1] = __byte_perm(t0, t2, 0x7632);
    out[2] = __byte_perm(t1, t3, 0x5410);
    out[3] = __byte_perm(t1, t3, 0x7632);
}

// Coin-weighted weight sum over one 64-position block of some A_v,
// sum_k 2^k popc(plane_k & R).  The block's planes are stored in pairs (an
// even count per block, 16-byte aligned, the padding plane zero) so that each
// pair is one 16-byte load; B <= 8 (weights c - 1 <= 255) and the loop is
// unrolled to that bound with a warp-uniform test, so all its loads issue
// together.
__device__ __forceinline__ uint32_t plane_block_sum(const unsigned long long* P, unsigned long long R, int B) {
    const ulonglong2* P2 = reinterpret_cast<const ulonglong2*>(P);
    uint32_t x = 0;
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
        if (k < B) {
            const ulonglong2 v = P2[k >> 1];
            x += (uint32_t)(__popcll(v.x & R) + (__popcll(v.y & R) << 1)) << k;
        }
    }
    return x;
}

__device__ __forceinline__ long long warp_sum64(long long v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// The per-process engine.
// ---------------------------------------------------------------------------

// Out-of-line Philox for the per-run and per-step draws: one copy of the code
// instead of one per call site keeps the kernel small in the instruction cache.
static __device__ __noinline__ uint4 philox_call(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                          uint32_t k1) {
    philox(c0, c1, c2, c3, k0, k1);
    return make_uint4(c0, c1, c2, c3);
}

// Greedy-Potential (Section 2.2): N_p counts the signed pairs that occur at
// least twice after a trial substitution of candidate p = (x_i + s x_j).  Only
// pairs with the fresh x_k can be new, and x_i, x_j share no row with x_k
// afterwards, so N_p = #{(u, s') : u != i, j, c(u, k, s') >= 2}.  Score
// S_p = (c_p - 1) 2^16 + a N_p; argmax, lowest key on ties.  One candidate
// per lane: its trial column x_k stays in registers and every column u is a
// broadcast read of shared memory.  Adds the trial ops (5 W per live column
// of the trial system, plus 8, per candidate) to *ops_total, and the method
// ops (the scan of m, and per candidate a trial rewrite: 6 per 64-bit word
// plus the nnz of its rows, which is the sum over every column u of the
// rows u shares with the trial column) to *mops_total.  Kept out of line
// with plain values, not the engine: measured on the (3,3,3:23) search, the
// step engine runs 7% faster than with this function inlined.
template <int W>
__device__ __noinline__ int gp_select(const uint2* P, const uint32_t* C, int ncols, int m, uint32_t a, int lane,
                                      int wn, unsigned long long* ops_total, unsigned long long* mops_total) {
    int nlive = 0;
    for (int base = 0; base < ncols; base += 32) {
        const int u = base + lane;
        uint32_t sup = 0;
        if (u < ncols) {
#pragma unroll
            for (int w = 0; w < W; w++) sup |= P[u * W + w].x | P[u * W + w].y;
        }
        nlive += __popc(__ballot_sync(FULL_MASK, sup != 0));
    }
    uint32_t best_s = 0;
    int best_q = INT_MAX;
    unsigned ops = 0, mops = 0;
    for (int base = 0; base < m; base += 32) {
        const int p = base + lane;
        if (p < m) {
            const uint32_t e = C[p];
            const int i = key_lo(e), j = key_hi(e), c = cand_c(e);
            uint32_t kp[W], kn[W];
            int nni = 0, nnj = 0;
#pragma unroll
            for (int w = 0; w < W; w++) {
                const uint2 A = P[i * W + w], B = P[j * W + w];
                kp[w] = (e & 1u) ? (A.x & B.y) : (A.x & B.x);
                kn[w] = (e & 1u) ? (A.y & B.x) : (A.y & B.y);
                nni += __popc(A.x | A.y);
                nnj += __popc(B.x | B.y);
            }
            int N = 0, rnnz = 0;
#pragma unroll 2
            for (int u = 0; u < ncols; u++) {
                int both = 0, ng = 0;
#pragma unroll
                for (int w = 0; w < W; w++) {
                    const uint2 U = P[u * W + w];
                    const uint32_t bt = (U.x | U.y) & (kp[w] | kn[w]);
                    both += __popc(bt);
                    ng += __popc((U.x ^ kp[w]) & bt);
                }
                const int hit = (both - ng >= 2) + (ng >= 2);
                N += (u == i || u == j) ? 0 : hit;
                rnnz += both;
            }
            const uint32_t sc = ((uint32_t)(c - 1) << 16) + a * (uint32_t)N;
            if (best_q == INT_MAX || sc > best_s) {
                best_s = sc;
                best_q = p;
            }
            const int live = nlive - (nni == c) - (nnj == c);
            ops += 5u * (unsigned)wn * (unsigned)live + 8u;  // the matrix's own words (wn <= W)
            mops += 6u * (unsigned)((wn + 1) >> 1) + (unsigned)rnnz;
        }
    }
    const uint32_t top = __reduce_max_sync(FULL_MASK, best_q == INT_MAX ? 0u : best_s);
    const int q = (int)__reduce_min_sync(FULL_MASK, (best_q != INT_MAX && best_s == top) ? (uint32_t)best_q
                                                                                          : 0xFFFFFFFFu);
    ops = __reduce_add_sync(FULL_MASK, ops);
    mops = __reduce_add_sync(FULL_MASK, mops);
    if (lane == 0) {
        *ops_total += ops;
        *mops_total += mops + (unsigned)m;
    }
    __syncwarp();
    return q;
}

// Coin word of the 32 candidates [base, base + 32) under shared coins:
// word (base >> 5) & 3 of the purpose-GIS draw for block base >> 7.
__device__ __forceinline__ uint32_t shared_coin_word(uint32_t proc, uint32_t t, uint32_t c2s, uint64_t seed,
                                                     int base) {
    const uint4 r = philox_call(proc, t, c2s | ((uint32_t)base >> 7), 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
    const int wi = (base >> 5) & 3;
    return wi == 0 ? r.x : wi == 1 ? r.y : wi == 2 ? r.z : r.w;
}

// Greedy-Intersections with shared coins (CSE_FLAG_GI_SHARED_COINS): the
// score of the engine's sel_gi, but candidate q has one coin per step for
// every p.  Then the sums over the candidates intersecting p = (i, j) follow
// from per-variable sums: X_p = X_i + X_j - 2 coin_p w_p - coin_t w_t, t the
// sign twin, and likewise for the plain sums G.  O(m + ncols) per step.  G
// and XS are ncols-entry scratch arrays (the engine lends its adjacency
// arrays); adds the step's algorithmic ops to *tally.
__device__ __forceinline__ int gi_shared_select(const uint32_t* C, uint32_t* G, uint32_t* XS, int ncols, int m,
                                                int lane, uint32_t proc, uint32_t t, uint32_t c2s, uint64_t seed,
                                                long long a, long long b, unsigned long long* tally,
                                                unsigned long long* mtally) {
    for (int v = lane; v < ncols; v += 32) {
        G[v] = 0;
        XS[v] = 0;
    }
    __syncwarp();
    int part = 0;
    for (int base = 0; base < m; base += 32) {
        const uint32_t word = shared_coin_word(proc, t, c2s, seed, base);
        const int q = base + lane;
        if (q < m) {
            const uint32_t e = C[q];
            const uint32_t w = (uint32_t)(cand_c(e) - 1);
            const int hi = key_hi(e), lo = key_lo(e);
            part += (int)w;
            atomicAdd(G + hi, w);
            atomicAdd(G + lo, w);
            if ((word >> lane) & 1u) {
                atomicAdd(XS + hi, w);
                atomicAdd(XS + lo, w);
            }
        }
    }
    __syncwarp();
    const int T = __reduce_add_sync(FULL_MASK, part);
    long long best_s = LLONG_MIN;
    int best_q = -1;
    for (int base = 0; base < m; base += 32) {
        const uint32_t word = shared_coin_word(proc, t, c2s, seed, base);
        const int p = base + lane;
        if (p < m) {
            const uint32_t e = C[p];
            const int i = key_lo(e), j = key_hi(e), wp = cand_c(e) - 1;
            const uint32_t key = e & 0x1FFFFFu;
            int sib = -1, wsib = 0, csib = 0;
            {
                const int nb_ = (e & 1u) ? p - 1 : p + 1;
                const uint32_t en = (nb_ >= 0 && nb_ < m) ? C[nb_] : 0u;
                if (nb_ >= 0 && nb_ < m && (en & 0x1FFFFFu) == (key ^ 1u)) {
                    sib = nb_;
                    wsib = cand_c(en) - 1;
                }
            }
            if (sib >= 0) {
                const uint32_t sw = (sib >> 5) == (p >> 5) ? word : shared_coin_word(proc, t, c2s, seed, sib & ~31);
                csib = (int)((sw >> (sib & 31)) & 1u);
            }
            const int cp = (int)((word >> lane) & 1u);
            const int inter = (int)G[i] + (int)G[j] - 2 * wp - wsib;
            const long long X = (long long)XS[i] + (long long)XS[j] - 2LL * cp * wp - (long long)csib * wsib;
            const int D = T - wp - inter;
            const long long sc = ((long long)wp << 32) + a * (((long long)D << 16) + b * X);
            if (sc > best_s) {
                best_s = sc;
                best_q = p;
            }
        }
    }
    best_q = warp_argmax_score(best_s, best_q);
    if (lane == 0) {
        *tally += 40u * (unsigned)((m + 127) >> 7) + 18u * (unsigned)m + 2u * (unsigned)ncols;
        *mtally += 5u * (unsigned)m;  // method ops: the scan, and 4 per candidate
    }
    __syncwarp();
    return best_q;
}

// The engine variant with shared coins (GS) reaches both rarely taken
// selections through this one out-of-line call site.  kind 0:
// Greedy-Potential, 1: shared-coin Greedy-Intersections.
template <int W>
__device__ __noinline__ int rare_select(int kind, const uint2* P, const uint32_t* C, uint32_t* G, uint32_t* XS,
                                        int ncols, int m, int lane, uint32_t proc, uint32_t t, uint32_t c2s,
                                        uint64_t seed, long long a, long long b, int wn, unsigned long long* tally,
                                        unsigned long long* mtally) {
    if (kind == 0) return gp_select<W>(P, C, ncols, m, (uint32_t)a, lane, wn, tally, mtally);
    return gi_shared_select(C, G, XS, ncols, m, lane, proc, t, c2s, seed, a, b, tally, mtally);
}

// Per-process values touched a few times per step at most.  They live in
// the warp's shared memory (written by lane 0) rather than in 32 register
// copies: the step engine is register-bound.
struct Cold {
    unsigned long long traj;   // trajectory hash (CSE_FLAG_TRACE)
    unsigned long long ops;    // algorithmic-op total before this round
    unsigned long long mops;   // method-op total before this round
    unsigned long long t_rare; // algorithmic ops of this round's gp and shared-coin gi steps
    unsigned long long t_mrare; // method ops of this round's gp and shared-coin gi steps
    int runs, substeps, best_cost, best_len, trace, overflow, sub_before;
    int strat, a, b;           // the current run's strategy, alpha, beta
    int best_strat;            // strategy of the run that gave the best record (-1: none)
    // algorithmic-op tallies of the round: substitutions, pair counts that
    // can change, candidates scanned by g/ga/wr/gr; Greedy-Intersections
    // terms, Philox blocks and scored candidates
    unsigned t_sub, t_pairs, t_scan, t_gi_terms, t_gi_blocks, t_gi_cands;
    unsigned t_nnz;            // method ops: nnz of the rewritten rows before their rewrites
};

template <int W, bool GM, bool GS>
struct Engine {
    unsigned char* sm;   // this warp's shared memory
    const WarpLayout* L;
    // context
    const DevMat* M;
    const DevSearch* S;
    int proc, lane, cap, mmax;
    uint32_t gproc;  // the global process index (draws, round keys)
    // warp-uniform state
    int ncols, nf, m, cost, ended;

    __device__ __forceinline__ uint2* pn() const { return reinterpret_cast<uint2*>(sm + L->off_pn); }
    __device__ __forceinline__ uint32_t* cand() const { return reinterpret_cast<uint32_t*>(sm + L->off_cand); }
    __device__ __forceinline__ int32_t* F() const { return reinterpret_cast<int32_t*>(sm + L->off_f); }
    __device__ __forceinline__ uint8_t* aw() const { return sm + L->off_aw; }
    __device__ __forceinline__ uint16_t* poslo() const { return reinterpret_cast<uint16_t*>(sm + L->off_poslo); }
    __device__ __forceinline__ uint16_t* hs() const { return reinterpret_cast<uint16_t*>(sm + L->off_hs); }
    __device__ __forceinline__ uint16_t* he() const { return reinterpret_cast<uint16_t*>(sm + L->off_he); }
    __device__ __forceinline__ uint16_t* vbase() const { return reinterpret_cast<uint16_t*>(sm + L->off_base); }
    __device__ __forceinline__ uint16_t* lc() const { return reinterpret_cast<uint16_t*>(sm + L->off_lc); }
    // HBM path only: per-variable plane base and weight sum, and the planes
    __device__ __forceinline__ uint16_t* pbase() const { return reinterpret_cast<uint16_t*>(sm + L->off_pb); }
    __device__ __forceinline__ uint32_t* gsum() const { return reinterpret_cast<uint32_t*>(sm + L->off_g); }
    __device__ __forceinline__ unsigned long long* planes() const {
        return reinterpret_cast<unsigned long long*>(sm + L->off_pln);
    }
    __device__ __forceinline__ Cold* cold() const { return reinterpret_cast<Cold*>(sm + L->off_cold); }
    __device__ __forceinline__ VarRec* rec() const { return reinterpret_cast<VarRec*>(sm + L->off_rec); }
    __device__ __forceinline__ uint16_t* bvar() const { return reinterpret_cast<uint16_t*>(sm + L->off_bv); }

    __device__ __forceinline__ uint32_t c2(uint32_t purpose, uint32_t extra_hi) const {
        return ((uint32_t)M->mat_index & 0xFFu) << 24 | (purpose & 0xFu) << 20 | (extra_hi & 0xFFFFFu);
    }
    __device__ __forceinline__ uint4 draw(int t, uint32_t purpose) const {
        return philox_call(gproc, (uint32_t)t, c2(purpose, 0), 0u, (uint32_t)S->seed, (uint32_t)(S->seed >> 32));
    }

    // c(a, b, s) for columns a < b
    __device__ __forceinline__ void counts(int a_, int b_, int& cp, int& cm) const {
        const uint2* P = pn();
        int both = 0, ng = 0;
#pragma unroll
        for (int w = 0; w < W; w++) {
            const uint2 A = P[a_ * W + w], B = P[b_ * W + w];
            const uint32_t bt = (A.x | A.y) & (B.x | B.y);
            both += __popc(bt);
            ng += __popc((A.x ^ B.x) & bt);
        }
        cm = ng;
        cp = both - ng;
    }

    // Substitution of (x_i + s x_j), i < j, by the fresh x_k, k = ncols
    // (Section 3.2.1, Algorithm 1), with the candidate list update.
    __device__ void subst(int i, int j, int neg) {
        const uint32_t lt = lanemask_lt();
        uint2* P = pn();
        uint32_t* C = cand();
        const int k = ncols;
        int cpart = 0;
        if (lane < W) {
            uint2 A = P[i * W + lane], B = P[j * W + lane];
            uint32_t rp, rn;
            if (!neg) {  // rows with +x_i +x_j  /  -x_i -x_j
                rp = A.x & B.x;
                rn = A.y & B.y;
                B.x &= ~rp;
                B.y &= ~rn;
            } else {     // rows with +x_i -x_j  /  -x_i +x_j
                rp = A.x & B.y;
                rn = A.y & B.x;
                B.x &= ~rn;
                B.y &= ~rp;
            }
            A.x &= ~rp;
            A.y &= ~rn;
            P[i * W + lane] = A;
            P[j * W + lane] = B;
            P[k * W + lane] = make_uint2(rp, rn);
            cpart = __popc(rp) + __popc(rn);
        }
        const int c = W == 1 ? __shfl_sync(FULL_MASK, cpart, 0) : __reduce_add_sync(FULL_MASK, cpart);
        __syncwarp();
        // recount the candidates containing x_i or x_j; stable in-place compaction
        int newm = 0, nij = 0;
        uint32_t e_nx = lane < m ? C[lane] : 0u;  // the next chunk, one iteration ahead
        for (int base = 0; base < m; base += 32) {
            const int q = base + lane;
            uint32_t e = e_nx;
            e_nx = q + 32 < m ? C[q + 32] : 0u;
            bool keep = false, touch = false;
            if (q < m) {
                const int lo = key_lo(e), hi = key_hi(e);
                touch = lo == i || lo == j || hi == i || hi == j;
                keep = true;
                if (touch) {
                    int cp, cm;
                    counts(lo, hi, cp, cm);
                    const int cc = (e & 1u) ? cm : cp;
                    keep = cc >= 2;
                    e = (e & 0x1FFFFFu) | ((uint32_t)cc << 21);
                }
            }
            const uint32_t kb = __ballot_sync(FULL_MASK, keep);
            nij += __popc(__ballot_sync(FULL_MASK, touch));
            __syncwarp();
            if (keep) C[newm + __popc(kb & lt)] = e;
            newm += __popc(kb);
        }
        // the new pairs (u, k): x_k has the largest index, so they sort last.
        // rb sums, over the columns u, the rewritten rows u still holds: with
        // 2 c for x_i and x_j it is the nnz of the rewritten rows before the
        // rewrite (the method op count)
        int nu = 0, rb = 0;
        for (int base = 0; base < k; base += 32) {
            const int u = base + lane;
            int cp = 0, cm = 0;
            bool live = false;
            if (u < k) {
                uint32_t sup = 0;
                int both = 0, ng = 0;
#pragma unroll
                for (int w = 0; w < W; w++) {
                    const uint2 A = P[u * W + w], K = P[k * W + w];
                    sup |= A.x | A.y;
                    const uint32_t bt = (A.x | A.y) & (K.x | K.y);
                    both += __popc(bt);
                    ng += __popc((A.x ^ K.x) & bt);
                }
                live = sup != 0;
                cm = ng;
                cp = both - ng;
                rb += both;
            }
            nu += __popc(__ballot_sync(FULL_MASK, live));
            const bool ep = cp >= 2, em = cm >= 2;
            const uint32_t bp = __ballot_sync(FULL_MASK, ep), bm = __ballot_sync(FULL_MASK, em);
            int pos = newm + __popc(bp & lt) + __popc(bm & lt);
            if (ep) {
                if (pos < mmax) C[pos] = make_cand(u, k, 0, cp);
                pos++;
            }
            if (em && pos < mmax) C[pos] = make_cand(u, k, 1, cm);
            newm += __popc(bp) + __popc(bm);
        }
        if (newm > mmax) {
            if (lane == 0) cold()->overflow = 1;
            newm = mmax;
        }
        if (lane == 0) F()[nf] = (int32_t)((uint32_t)i | (uint32_t)j << 10 | (uint32_t)neg << 20);
        nf++;
        ncols++;
        cost -= c - 1;
        m = newm;
        rb = __reduce_add_sync(FULL_MASK, rb);
        if (lane == 0) {
            Cold* cd = cold();
            cd->t_sub++;
            cd->t_pairs += (unsigned)(nij + nu);
            cd->t_nnz += (unsigned)(rb + 2 * c);
        }
        __syncwarp();
    }

    // Closes the current run into the process's best record (strictly lower
    // cost replaces).
    __device__ void fold() {
        Cold* cd = cold();
        if (cost < cd->best_cost) {
            int32_t* dst = M->best_list + (size_t)proc * cap;
            const int32_t* f = F();
            for (int x = lane; x < nf; x += 32) dst[x] = f[x];
            __syncwarp();
            if (lane == 0) {
                cd->best_cost = cost;
                cd->best_len = nf;
                cd->best_strat = cd->strat;
            }
        }
        __syncwarp();
    }

    // Run start at step t (Section 3.5.1-3.5.2): strategy, alpha, beta, fresh
    // copy of the input.  Returns how many substitutions of the snapshot to
    // replay (Section 3.5.2); the caller replays them.
    __device__ int start_run(int t) {
        if (t > 0) fold();
        if (lane == 0) cold()->runs++;
        const uint4 R = draw(t, PU_RUN);
        int strat = ST_G;
        if (!(gproc == 0 && t == 0)) {
            const uint32_t x = scale32(R.x, S->wsum);
            uint32_t acc = 0;
            for (int s = 0; s < ST_N; s++) {
                acc += S->w[s];
                if (x < acc) {
                    strat = s;
                    break;
                }
            }
        }
        if (lane == 0) {
            Cold* cd = cold();
            cd->strat = strat;
            cd->a = (int)scale32(R.y, 32769u);
            cd->b = 32768 + (int)scale32(R.z, 32769u);
        }
        const int nx = M->nx;
        uint2* P = pn();
        uint32_t* C = cand();
        for (int x = lane; x < nx * W; x += 32) P[x] = M->pn0[x];
        const int m0 = M->meta0[1];
        for (int x = lane; x < m0; x += 32) C[x] = M->cand0[x];
        m = m0 < mmax ? m0 : mmax;
        ncols = nx;
        nf = 0;
        cost = M->meta0[0];
        int k = 0;
        if (M->snap_meta[0] != INT_MAX && (uint64_t)R.w < S->share_thr) {
            const int K = (3 * M->snap_meta[1]) / 4;
            if (K >= 1) k = 1 + (int)scale32(draw(t, PU_SHAREK).x, (uint32_t)K);
        }
        ended = 0;
        if (lane == 0) {
            Cold* cd = cold();
            if (cd->trace) cd->traj = fnv(fnv(cd->traj, (uint32_t)t), 0xA0000000u | (uint32_t)cd->strat << 12 | (uint32_t)k);
        }
        __syncwarp();
        return k;
    }

    // Greedy: highest c, lowest key.
    __device__ int sel_g() const {
        const uint32_t* C = cand();
        uint32_t best = 0;
        for (int q = lane; q < m; q += 32) {
            const uint32_t v = (uint32_t)cand_c(C[q]) << 16 | (uint32_t)(0xFFFF - q);
            best = best > v ? best : v;
        }
        best = __reduce_max_sync(FULL_MASK, best);
        return 0xFFFF - (int)(best & 0xFFFFu);
    }

    // Greedy-Alternative: uniform among the max-c ties, (u * n_ties) >> 32-th in order.
    __device__ int sel_ga(uint32_t u) const {
        const uint32_t lt = lanemask_lt();
        const uint32_t* C = cand();
        int lmax = 0, lcnt = 0;
        for (int q = lane; q < m; q += 32) {
            const int c = cand_c(C[q]);
            if (c > lmax) {
                lmax = c;
                lcnt = 1;
            } else if (c == lmax) {
                lcnt++;
            }
        }
        const int cmax = (int)__reduce_max_sync(FULL_MASK, (uint32_t)lmax);
        const int nt = __reduce_add_sync(FULL_MASK, lmax == cmax ? lcnt : 0);
        uint32_t want = scale32(u, (uint32_t)nt);
        for (int base = 0; base < m; base += 32) {
            const int q = base + lane;
            const bool tie = q < m && cand_c(C[q]) == cmax;
            const uint32_t bt = __ballot_sync(FULL_MASK, tie);
            const uint32_t n = (uint32_t)__popc(bt);
            if (want < n) {
                const uint32_t hit = __ballot_sync(FULL_MASK, tie && (uint32_t)__popc(bt & lt) == want);
                return base + __ffs(hit) - 1;
            }
            want -= n;
        }
        return 0;
    }

    // Weighted-Random: first candidate whose running sum of (c - 1) exceeds
    // (u * T) >> 32, T = sum (c - 1).
    __device__ int sel_wr(uint32_t u) const {
        const uint32_t* C = cand();
        int part = 0;
        for (int q = lane; q < m; q += 32) part += cand_c(C[q]) - 1;
        const uint32_t total = (uint32_t)__reduce_add_sync(FULL_MASK, part);
        const uint32_t x = scale32(u, total);
        uint32_t acc = 0;
        for (int base = 0; base < m; base += 32) {
            const int q = base + lane;
            const int w = q < m ? cand_c(C[q]) - 1 : 0;
            const int incl = warp_incl_scan(w, lane);
            const uint32_t hit = __ballot_sync(FULL_MASK, q < m && acc + (uint32_t)incl > x);
            if (hit) return base + __ffs(hit) - 1;
            acc += (uint32_t)__shfl_sync(FULL_MASK, incl, 31);
        }
        return m - 1;
    }

    // Greedy-Intersections (Section 3.4.2), exact integer score
    // S_p = (c_p - 1) 2^32 + a (2^16 D_p + b X_p); argmax, lowest key on ties.
    // For every variable v the weights (c - 1) of the candidates holding x_v
    // are gathered, in canonical order, into A_v = aw[base[v] ..): first the
    // hi-block of v (contiguous in the sorted list), then the candidates whose
    // lower index is v (a stable scatter).  A candidate's coin in a slot is the
    // Philox bit at its position in A_v, so each lane scores its candidate with
    // two straight loops over byte arrays.
    __device__ int sel_gi(int t) {
        const uint32_t lt = lanemask_lt();
        const uint32_t* C = cand();
        uint16_t* HS = hs();
        uint16_t* HE = he();
        uint16_t* VB = vbase();
        uint16_t* LC = lc();
        uint8_t* AW = aw();
        uint16_t* PL = poslo();
        int part = 0;
        for (int v = lane; v < ncols; v += 32) {
            HS[v] = 0;
            HE[v] = 0;
            LC[v] = 0;
        }
        __syncwarp();
        for (int base = 0; base < m; base += 32) {
            const int q = base + lane;
            const bool valid = q < m;
            const uint32_t act = __ballot_sync(FULL_MASK, valid);
            // the neighbours' hi from the adjacent lanes; only the chunk's
            // edge lanes read the list
            const uint32_t eq = valid ? C[q] : 0u;
            int hprev = __shfl_up_sync(FULL_MASK, key_hi(eq), 1);
            int hnext = __shfl_down_sync(FULL_MASK, key_hi(eq), 1);
            if (valid) {
                const uint32_t e = eq;
                const int hi = key_hi(e), lo = key_lo(e);
                part += cand_c(e) - 1;
                if (lane == 0) hprev = q > 0 ? key_hi(C[q - 1]) : -1;
                if (lane == 31 || q == m - 1) hnext = q + 1 < m ? key_hi(C[q + 1]) : -1;
                if (hprev != hi) HS[hi] = (uint16_t)q;
                if (hnext != hi) HE[hi] = (uint16_t)(q + 1);
                const uint32_t peers = __match_any_sync(act, lo);
                if ((peers & lt) == 0) LC[lo] = (uint16_t)(LC[lo] + __popc(peers));
            }
            __syncwarp();
        }
        const int T = __reduce_add_sync(FULL_MASK, part);
        int run = 0;
        for (int base = 0; base < ncols; base += 32) {
            const int v = base + lane;
            const int deg = v < ncols ? (HE[v] - HS[v]) + LC[v] : 0;
            const int incl = warp_incl_scan(deg, lane);
            if (v < ncols) {
                VB[v] = (uint16_t)(run + incl - deg);
                LC[v] = 0;
            }
            run += __shfl_sync(FULL_MASK, incl, 31);
        }
        __syncwarp();
        for (int base = 0; base < m; base += 32) {
            const int q = base + lane;
            const bool valid = q < m;
            const uint32_t act = __ballot_sync(FULL_MASK, valid);
            uint32_t peers = 0;
            int lo = 0;
            if (valid) {
                const uint32_t e = C[q];
                const int hi = key_hi(e);
                lo = key_lo(e);
                const uint8_t w = (uint8_t)(cand_c(e) - 1);
                AW[VB[hi] + (q - HS[hi])] = w;
                peers = __match_any_sync(act, lo);
                const int pos = VB[lo] + (HE[lo] - HS[lo]) + LC[lo] + __popc(peers & lt);
                AW[pos] = w;
                PL[q] = (uint16_t)pos;
            }
            __syncwarp();
            if (valid && (peers & lt) == 0) LC[lo] = (uint16_t)(LC[lo] + __popc(peers));
            __syncwarp();
        }
        // scoring: one candidate p per lane
        const uint32_t k0 = (uint32_t)S->seed, k1 = (uint32_t)(S->seed >> 32);
        const uint32_t c2g = c2(PU_GI, 0);
        const long long a = cold()->a, b = cold()->b;
        long long best_s = LLONG_MIN;
        int best_q = -1;
        unsigned gi_terms = 0, gi_blocks = 0;
        for (int base = 0; base < m; base += 32) {
            const int p = base + lane;
            if (p < m) {
                const uint32_t e = C[p];
                const int i = key_lo(e), j = key_hi(e), wp = cand_c(e) - 1;
                const uint32_t key = e & 0x1FFFFFu;
                const int b0 = VB[i], n0 = (HE[i] - HS[i]) + LC[i];
                const int b1 = VB[j], n1 = (HE[j] - HS[j]) + LC[j];
                const int lp0 = PL[p] - b0;     // p's place in A_i
                const int lp1 = p - HS[j];      // p's place in A_j
                // the sign twin (i, j, -s), if a candidate: the neighbour on the
                // side its sign sorts to, read once
                int sib = -1, wsib = 0;
                {
                    const int nb_ = (e & 1u) ? p - 1 : p + 1;
                    const uint32_t en = (nb_ >= 0 && nb_ < m) ? C[nb_] : 0u;
                    if (nb_ >= 0 && nb_ < m && (en & 0x1FFFFFu) == (key ^ 1u)) {
                        sib = nb_;
                        wsib = cand_c(en) - 1;
                    }
                }
                const int ls1 = sib - HS[j];
                const int nint = (n0 - 1) + (n1 - 1 - (sib >= 0 ? 1 : 0));
                int inter = 0, X = 0, nb = 0;
                if (nint > 0) {
                    const int nb0 = (n0 + 63) >> 6, nb1 = (n1 + 63) >> 6;
                    nb = nb0 > nb1 ? nb0 : nb1;
                    for (int blk = 0; blk < nb; blk++) {
                        uint32_t r0 = gproc, r1 = (uint32_t)t, r2 = c2g | (uint32_t)blk, r3 = key;
                        philox(r0, r1, r2, r3, k0, k1);
                        const int x0 = blk << 6;
                        // slot 0: A_i, then take p itself out
                        {
                            const int x1 = min(n0, x0 + 64);
#pragma unroll 4
                            for (int x = x0; x < x1; x++) {
                                const int w = AW[b0 + x];
                                const uint32_t word = (x & 32) ? r1 : r0;
                                inter += w;
                                X += ((word >> (x & 31)) & 1u) ? w : 0;
                            }
                            if (lp0 >= x0 && lp0 < x1) {
                                const uint32_t word = (lp0 & 32) ? r1 : r0;
                                inter -= wp;
                                X -= ((word >> (lp0 & 31)) & 1u) ? wp : 0;
                            }
                        }
                        // slot 1: A_j, then take out p and its twin (they hold x_i)
                        {
                            const int x1 = min(n1, x0 + 64);
#pragma unroll 4
                            for (int x = x0; x < x1; x++) {
                                const int w = AW[b1 + x];
                                const uint32_t word = (x & 32) ? r3 : r2;
                                inter += w;
                                X += ((word >> (x & 31)) & 1u) ? w : 0;
                            }
                            if (lp1 >= x0 && lp1 < x1) {
                                const uint32_t word = (lp1 & 32) ? r3 : r2;
                                inter -= wp;
                                X -= ((word >> (lp1 & 31)) & 1u) ? wp : 0;
                            }
                            if (sib >= 0 && ls1 >= x0 && ls1 < x1) {
                                const uint32_t word = (ls1 & 32) ? r3 : r2;
                                inter -= wsib;
                                X -= ((word >> (ls1 & 31)) & 1u) ? wsib : 0;
                            }
                        }
                    }
                }
                const int D = T - wp - inter;
                const long long sc = ((long long)wp << 32) +
                                     a * (((long long)D << 16) + b * (long long)X);
                if (sc > best_s) {
                    best_s = sc;
                    best_q = p;
                }
                gi_terms += nint;
                gi_blocks += nb;
            }
        }
        best_q = warp_argmax_score(best_s, best_q);
        gi_terms = __reduce_add_sync(FULL_MASK, gi_terms);
        gi_blocks = __reduce_add_sync(FULL_MASK, gi_blocks);
        if (lane == 0) {
            Cold* cd = cold();
            cd->t_gi_terms += gi_terms;
            cd->t_gi_blocks += gi_blocks;
            cd->t_gi_cands += (unsigned)m;
        }
        return best_q;
    }

    // Greedy-Intersections for large matrices (HBM path): the same exact
    // integer score as sel_gi, with the coin-weighted sums taken over
    // bit-planes instead of byte loops.  For every variable v and every 64
    // positions of A_v, plane k is the 64-bit mask of the positions whose
    // weight has bit k set; then sum coin(x) w(x) over a block is
    // sum_k 2^k popc(plane_k & coins), and the plain sums are G[v].  The lists
    // of these matrices hold hundreds of candidates, so this replaces
    // O(|A_i| + |A_j|) byte steps per candidate by O(B (|A_i| + |A_j|) / 64)
    // popcounts, B = bits of the largest weight.  The planes are built
    // without atomics: the placement pass writes each position's weight byte,
    // then one lane per 64-position block transposes its 64 bytes into the
    // block's planes and adds their sum to G[v] (one atomic per block: plane
    // bits set by atomics per candidate and bit, most of a chunk's lanes on
    // the same words, took about half of the whole search's time).
    __device__ int sel_gi_planes(int t) {
        const uint32_t lt = lanemask_lt();
        const uint32_t* C = cand();
        VarRec* R = rec();
        uint16_t* PL = poslo();
        uint16_t* BV = bvar();
        uint8_t* AW = aw();
        unsigned long long* PLN = planes();
        int part = 0, wmax = 1;
        for (int v = lane; v < ncols; v += 32) *reinterpret_cast<uint4*>(R + v) = make_uint4(0u, 0u, 0u, 0u);
        __syncwarp();
        // Every pass over the list below reads the next chunk's entries one
        // iteration ahead (the list lives in HBM: a chunk's work then waits
        // on one fewer round trip); a chunk's neighbours come from the
        // adjacent lanes, the previous chunk's last entry and the prefetch.
        uint32_t e_nx = lane < m ? C[lane] : 0u;
        int hi_last = -1;  // hi of the previous chunk's last entry
        for (int base = 0; base < m; base += 32) {
            const int q = base + lane;
            const bool valid = q < m;
            const uint32_t act = __ballot_sync(FULL_MASK, valid);
            const uint32_t e = e_nx;
            e_nx = q + 32 < m ? C[q + 32] : 0u;
            const int hi = key_hi(e), lo = key_lo(e);
            int hprev = __shfl_up_sync(FULL_MASK, hi, 1);
            int hnext = __shfl_down_sync(FULL_MASK, hi, 1);
            const int hfirst_nx = __shfl_sync(FULL_MASK, key_hi(e_nx), 0);
            if (lane == 0) hprev = hi_last;
            if (lane == 31) hnext = hfirst_nx;
            if (valid) {
                part += cand_c(e) - 1;
                wmax = max(wmax, cand_c(e) - 1);
                if (hprev != hi) R[hi].hs = (uint16_t)q;
                if (q == m - 1 || hnext != hi) R[hi].he = (uint16_t)(q + 1);
                const uint32_t peers = __match_any_sync(act, lo);
                if ((peers & lt) == 0) R[lo].lc = (uint16_t)(R[lo].lc + __popc(peers));
            }
            hi_last = __shfl_sync(FULL_MASK, hi, 31);
            __syncwarp();
        }
        const int T = __reduce_add_sync(FULL_MASK, part);
        const int B = 32 - __clz((int)__reduce_max_sync(FULL_MASK, (uint32_t)wmax));
        // positions (low 16 bits) and 64-position blocks (high 16 bits) of A_v
        uint32_t run = 0;
        for (int base = 0; base < ncols; base += 32) {
            const int v = base + lane;
            VarRec r{};
            if (v < ncols) r = R[v];
            const int deg = v < ncols ? (r.he - r.hs) + r.lc : 0;
            const uint32_t packed = (uint32_t)deg | (uint32_t)((deg + 63) >> 6) << 16;
            const uint32_t incl = (uint32_t)warp_incl_scan((int)packed, lane);
            if (v < ncols) {
                const uint32_t ex = run + incl - packed;
                r.vb = (uint16_t)(ex & 0xFFFFu);
                r.pb = (uint16_t)(ex >> 16);
                r.lct = r.lc;  // the lo count, kept for the scoring
                r.lc = 0;       // the running lo rank of the placement pass
                R[v] = r;
                for (int x = 0; x < (int)(packed >> 16); x++) BV[r.pb + x] = (uint16_t)v;
            }
            run += (uint32_t)__shfl_sync(FULL_MASK, (int)incl, 31);
        }
        const int nblocks = (int)(run >> 16);
        const int BP = (B + 1) & ~1;  // planes stored per block: B rounded up to even (the padding plane zero)
        e_nx = lane < m ? C[lane] : 0u;
        for (int base = 0; base < m; base += 32) {
            const int q = base + lane;
            const bool valid = q < m;
            const uint32_t act = __ballot_sync(FULL_MASK, valid);
            const uint32_t e = e_nx;
            e_nx = q + 32 < m ? C[q + 32] : 0u;
            uint32_t peers = 0;
            int lo = 0;
            if (valid) {
                const int hi = key_hi(e);
                lo = key_lo(e);
                const uint32_t w = (uint32_t)(cand_c(e) - 1);
                peers = __match_any_sync(act, lo);
                const VarRec rh = R[hi], rl = R[lo];
                const int xh = q - rh.hs;
                const int xl = (rl.he - rl.hs) + rl.lc + __popc(peers & lt);
                PL[q] = (uint16_t)(rl.vb + xl);
                AW[rh.vb + xh] = (uint8_t)w;
                AW[rl.vb + xl] = (uint8_t)w;
            }
            __syncwarp();
            if (valid && (peers & lt) == 0) R[lo].lc = (uint16_t)(R[lo].lc + __popc(peers));
            __syncwarp();
        }
        // the planes, one lane per block: its 64 weight bytes (read 8 bytes at
        // a time from the 8-byte boundary below the block's first position,
        // bytes past the variable's list masked off), eight 8 x 8 bit
        // transposes and a 4 x 4 byte transpose per 4 x 32 bits give planes
        // 0..7; the first BP are stored, and the block's weight sum goes to G
        for (int gb = lane; gb < nblocks; gb += 32) {
            const int v = BV[gb];
            const VarRec r = R[v];
            const int deg = (r.he - r.hs) + r.lct;
            const int bl = gb - r.pb;
            const int x0 = r.vb + 64 * bl, n = min(64, deg - 64 * bl);
            const unsigned long long* src = reinterpret_cast<const unsigned long long*>(AW + (x0 & ~7));
            const int sh = (x0 & 7) * 8;
            unsigned long long u = src[0], T[8];
            uint32_t gs = 0;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const unsigned long long nx = src[j + 1];
                unsigned long long x = sh ? (u >> sh) | (nx << (64 - sh)) : u;
                u = nx;
                const int valid = n - 8 * j;
                if (valid < 8) x = valid <= 0 ? 0ull : x & ((1ull << (8 * valid)) - 1ull);
                gs = __dp4a((uint32_t)x, 0x01010101u, gs);
                gs = __dp4a((uint32_t)(x >> 32), 0x01010101u, gs);
                T[j] = transpose8x8(x);
            }
            uint32_t lo4[4], hi4[4];  // planes 0..3: low and high 32 positions
            transpose4x4_bytes((uint32_t)T[0], (uint32_t)T[1], (uint32_t)T[2], (uint32_t)T[3], lo4);
            transpose4x4_bytes((uint32_t)T[4], (uint32_t)T[5], (uint32_t)T[6], (uint32_t)T[7], hi4);
            unsigned long long* dst = PLN + (size_t)gb * BP;
            for (int k = 0; k < BP && k < 4; k++) dst[k] = (unsigned long long)hi4[k] << 32 | lo4[k];
            if (BP > 4) {  // planes 4..7
                transpose4x4_bytes((uint32_t)(T[0] >> 32), (uint32_t)(T[1] >> 32), (uint32_t)(T[2] >> 32),
                                   (uint32_t)(T[3] >> 32), lo4);
                transpose4x4_bytes((uint32_t)(T[4] >> 32), (uint32_t)(T[5] >> 32), (uint32_t)(T[6] >> 32),
                                   (uint32_t)(T[7] >> 32), hi4);
                for (int k = 4; k < BP; k++) dst[k] = (unsigned long long)hi4[k - 4] << 32 | lo4[k - 4];
            }
            atomicAdd(&R[v].g, gs);
        }
        __threadfence_block();
        __syncwarp();
        // scoring: one candidate p per lane
        const uint32_t k0 = (uint32_t)S->seed, k1 = (uint32_t)(S->seed >> 32);
        const uint32_t c2g = c2(PU_GI, 0);
        const long long a = cold()->a, b = cold()->b;
        long long best_s = LLONG_MIN;
        int best_q = -1;
        unsigned gi_terms = 0, gi_blocks = 0;
        e_nx = lane < m ? C[lane] : 0u;
        int pl_nx = lane < m ? PL[lane] : 0;
        uint32_t e_last = 0;  // the previous chunk's last entry
        for (int base = 0; base < m; base += 32) {
            const int p = base + lane;
            const uint32_t e = e_nx;
            const int plp = pl_nx;
            e_nx = p + 32 < m ? C[p + 32] : 0u;
            pl_nx = p + 32 < m ? PL[p + 32] : 0;
            // the neighbours p - 1 and p + 1, for the sign twin
            uint32_t e_up = __shfl_up_sync(FULL_MASK, e, 1);
            uint32_t e_dn = __shfl_down_sync(FULL_MASK, e, 1);
            const uint32_t e_first_nx = __shfl_sync(FULL_MASK, e_nx, 0);
            if (lane == 0) e_up = e_last;
            if (lane == 31) e_dn = e_first_nx;
            e_last = __shfl_sync(FULL_MASK, e, 31);
            if (p < m) {
                const int i = key_lo(e), j = key_hi(e), wp = cand_c(e) - 1;
                const uint32_t key = e & 0x1FFFFFu;
                const VarRec ri = R[i], rj = R[j];
                // the first coin block does not depend on the records: drawn
                // while their loads are in flight
                uint32_t f0 = gproc, f1 = (uint32_t)t, f2 = c2g, f3 = key;
                philox(f0, f1, f2, f3, k0, k1);
                const int n0 = (ri.he - ri.hs) + ri.lct;
                const int n1 = (rj.he - rj.hs) + rj.lct;
                const int lp0 = plp - ri.vb;  // p's place in A_i
                const int lp1 = p - rj.hs;    // p's place in A_j
                // the sign twin (i, j, -s), if a candidate: the neighbour on the
                // side its sign sorts to
                int sib = -1, wsib = 0;
                {
                    const int nb_ = (e & 1u) ? p - 1 : p + 1;
                    const uint32_t en = (e & 1u) ? e_up : e_dn;
                    if (nb_ >= 0 && nb_ < m && (en & 0x1FFFFFu) == (key ^ 1u)) {
                        sib = nb_;
                        wsib = cand_c(en) - 1;
                    }
                }
                const int ls1 = sib - rj.hs;
                const int nint = (n0 - 1) + (n1 - 1 - (sib >= 0 ? 1 : 0));
                int X = 0, inter = 0, nb = 0;
                if (nint > 0) {
                    const int nb0 = (n0 + 63) >> 6, nb1 = (n1 + 63) >> 6;
                    nb = nb0 > nb1 ? nb0 : nb1;
                    const unsigned long long* P0 = PLN + (size_t)ri.pb * BP;
                    const unsigned long long* P1 = PLN + (size_t)rj.pb * BP;
                    for (int blk = 0; blk < nb; blk++) {
                        uint32_t r0 = f0, r1 = f1, r2 = f2, r3 = f3;
                        if (blk > 0) {
                            r0 = gproc, r1 = (uint32_t)t, r2 = c2g | (uint32_t)blk, r3 = key;
                            philox(r0, r1, r2, r3, k0, k1);
                        }
                        const unsigned long long R0 = (unsigned long long)r1 << 32 | r0;
                        const unsigned long long R1 = (unsigned long long)r3 << 32 | r2;
                        if (blk < nb0) {
                            X += (int)plane_block_sum(P0 + blk * BP, R0, B);
                            if ((lp0 >> 6) == blk && ((R0 >> (lp0 & 63)) & 1ull)) X -= wp;
                        }
                        if (blk < nb1) {
                            X += (int)plane_block_sum(P1 + blk * BP, R1, B);
                            if ((lp1 >> 6) == blk && ((R1 >> (lp1 & 63)) & 1ull)) X -= wp;
                            if (sib >= 0 && (ls1 >> 6) == blk && ((R1 >> (ls1 & 63)) & 1ull)) X -= wsib;
                        }
                    }
                    inter = (int)ri.g + (int)rj.g - 2 * wp - wsib;
                }
                const int D = T - wp - inter;
                const long long sc = ((long long)wp << 32) + a * (((long long)D << 16) + b * (long long)X);
                if (sc > best_s) {
                    best_s = sc;
                    best_q = p;
                }
                gi_terms += nint;
                gi_blocks += nb;
            }
        }
        best_q = warp_argmax_score(best_s, best_q);
        gi_terms = __reduce_add_sync(FULL_MASK, gi_terms);
        gi_blocks = __reduce_add_sync(FULL_MASK, gi_blocks);
        if (lane == 0) {
            Cold* cd = cold();
            cd->t_gi_terms += gi_terms;
            cd->t_gi_blocks += gi_blocks;
            cd->t_gi_cands += (unsigned)m;
        }
        return best_q;
    }

    // Greedy-Potential (kind 0) and shared-coin Greedy-Intersections (kind 1).
    __device__ int sel_rare(int kind, int t) {
        return rare_select<W>(kind, pn(), cand(), reinterpret_cast<uint32_t*>(hs()),
                              reinterpret_cast<uint32_t*>(vbase()), ncols, m, lane, gproc, (uint32_t)t,
                              c2(PU_GIS, 0), S->seed, cold()->a, cold()->b, M->wn, &cold()->t_rare,
                              &cold()->t_mrare);
    }

    __device__ int choose(int t) {
        int s = cold()->strat;
        uint4 d = make_uint4(0, 0, 0, 0);
        if (s != ST_G && s != ST_GI && s != ST_GP) d = draw(t, PU_STEP);
        if (s == ST_MIX) {
            const uint32_t r = scale32(d.x, 15u);
            s = r < 8 ? ST_GI : r < 12 ? ST_GA : r < 14 ? ST_GR : ST_WR;
        }
        if (s == ST_GR) s = d.y < 0xC0000000u ? ST_GA : ST_WR;
        if (s == ST_GI) {
            if constexpr (GS) return sel_rare(1, t);
            if constexpr (GM)
                return sel_gi_planes(t);
            else
                return sel_gi(t);
        }
        if (s == ST_GP) {
            if constexpr (GS)
                return sel_rare(0, t);
            else
                return gp_select<W>(pn(), cand(), ncols, m, (uint32_t)cold()->a, lane, M->wn, &cold()->t_rare,
                                    &cold()->t_mrare);
        }
        if (lane == 0) cold()->t_scan += (unsigned)m;
        if (s == ST_GA) return sel_ga(d.z);
        if (s == ST_WR) return sel_wr(d.w);
        return sel_g();
    }

    // One step of the step clock (one Algorithm 1 iteration).  A run start
    // first replays its shared prefix; replays and the step's own
    // substitution go through the one call site of subst().
    __device__ void step(int t) {
        int replay = 0;
        if (t == 0 || ended) replay = start_run(t);
        for (int e = 0;; e++) {
            int i, j, neg;
            if (e < replay) {
                const uint32_t ent = (uint32_t)M->snap[e];
                i = (int)(ent & 1023u);
                j = (int)((ent >> 10) & 1023u);
                neg = (int)((ent >> 20) & 1u);
            } else {
                if (m == 0 || ncols >= cap) {
                    ended = 1;
                    return;
                }
                const int sel = choose(t);
                const uint32_t ce = cand()[sel];
                __syncwarp();
                i = key_lo(ce);
                j = key_hi(ce);
                neg = (int)(ce & 1u);
            }
            subst(i, j, neg);
            if (e >= replay) break;
        }
        if (lane == 0) {
            Cold* cd = cold();
            cd->substeps++;
            if (cd->trace) cd->traj = fnv(fnv(cd->traj, (uint32_t)t), (uint32_t)F()[nf - 1]);
        }
        if (m == 0 || ncols >= cap) ended = 1;
    }
};

#ifndef CSE_MIN_BLOCKS
#define CSE_MIN_BLOCKS 8  // CTAs of 4 warps per SM the register budget must allow
#endif

// GM = false: the process's working arrays live in this warp's slice of
// shared memory and are loaded from / stored to its HBM state region at the
// round boundaries.  GM = true (matrices whose arrays are too large to share
// an SM between enough warps): the arrays stay in the state region itself and
// the engine works on them through the L1/L2 caches.
template <int W, bool GM, bool GS>
__device__ __forceinline__ void run_unit(const DevMat* __restrict__ mats, int n_mats,
                                         const DevSearch* __restrict__ searches, const WarpLayout& L,
                                         unsigned char* smem, int warp, int lane, int unit) {
    int mi = 0, mhi = n_mats - 1;  // the last matrix whose first unit is <= unit
    while (mi < mhi) {
        const int mid = (mi + mhi + 1) >> 1;
        if (mats[mid].unit_base <= unit) mi = mid; else mhi = mid - 1;
    }
    const DevMat* M = &mats[mi];
    const DevSearch* S = &searches[M->search];
    // step clock: this round runs steps [t0, t1).  Iteration mode: one whole
    // run per process, from step t0 = iteration * cap until the run ends.
    const int clk = *S->clock;
    if (clk >= S->budget || (S->interval == 0 && S->conv[1])) return;
    const int t0 = S->interval == 0 ? clk * M->cap : clk;

    uint32_t* st = M->state + (size_t)(unit - M->unit_base) * M->state_words;
    Engine<W, GM, GS> E;
    E.sm = GM ? reinterpret_cast<unsigned char*>(st + H_WORDS) : smem + (size_t)warp * L.per_warp;
    E.L = GM ? &M->gml : &L;
    E.M = M;
    E.S = S;
    E.proc = unit - M->unit_base;
    E.gproc = (uint32_t)(E.proc + M->proc_offset);
    E.lane = lane;
    E.cap = M->cap;
    E.mmax = M->mmax;
    Cold* cd = E.cold();
    if (t0 == 0) {
        E.ncols = M->nx;
        E.nf = 0;
        E.m = 0;
        E.cost = M->meta0[0];
        E.ended = 1;
        if (lane == 0) {
            cd->ops = 0;
            cd->mops = 0;
            cd->strat = ST_G;
            cd->a = 0;
            cd->b = 0;
            cd->runs = 0;
            cd->substeps = 0;
            cd->best_cost = M->meta0[0];
            cd->best_len = 0;
            cd->best_strat = -1;
            cd->traj = kFnv0;
        }
    } else {
        E.ncols = (int)st[H_NCOLS];
        E.nf = (int)st[H_NF];
        E.m = (int)st[H_M];
        E.cost = (int)st[H_COST];
        E.ended = (int)st[H_ENDED];
        if (lane == 0) {
            cd->ops = (uint64_t)st[H_OPS_LO] | (uint64_t)st[H_OPS_HI] << 32;
            cd->mops = (uint64_t)st[H_MOPS_LO] | (uint64_t)st[H_MOPS_HI] << 32;
            cd->strat = (int)st[H_STRAT];
            cd->a = (int)st[H_A];
            cd->b = (int)st[H_B];
            cd->runs = (int)st[H_RUNS];
            cd->substeps = (int)st[H_SUBSTEPS];
            cd->best_cost = (int)st[H_BEST_COST];
            cd->best_len = (int)st[H_BEST_LEN];
            cd->best_strat = (int)st[H_BEST_STRAT];
            cd->traj = (uint64_t)st[H_TRAJ_LO] | (uint64_t)st[H_TRAJ_HI] << 32;
        }
    }
    if (lane == 0) {
        cd->trace = S->trace;
        cd->overflow = 0;
        cd->t_sub = cd->t_pairs = cd->t_scan = 0;
        cd->t_gi_terms = cd->t_gi_blocks = cd->t_gi_cands = 0;
        cd->t_rare = 0;
        cd->t_mrare = 0;
        cd->t_nnz = 0;
    }
    if (t0 > 0 && !GM) {
        const uint2* spn = reinterpret_cast<const uint2*>(st + H_WORDS);
        uint2* P = E.pn();
        for (int x = lane; x < E.ncols * W; x += 32) P[x] = spn[x];
        const uint32_t* sc = st + H_WORDS + 2 * M->cap * W;
        uint32_t* C = E.cand();
        for (int x = lane; x < E.m; x += 32) C[x] = sc[x];
        const int32_t* sf = reinterpret_cast<const int32_t*>(sc + M->mmax);
        int32_t* F = E.F();
        for (int x = lane; x < E.nf; x += 32) F[x] = sf[x];
    }
    if (lane == 0) cd->sub_before = cd->substeps;
    __syncwarp();

    // Iteration mode: the run goes on until it ends; it makes at most
    // cap - nx substitutions plus the step that ends it, so it ends before
    // t0 + cap, the next iteration's first step (the bound is never reached).
    // One call site of step() keeps a single copy of the engine in the code.
    const bool iter = S->interval == 0;
    const int t1 = iter ? t0 + M->cap : min(t0 + S->interval, S->budget);
    int t = t0;
    while (t < t1) {
        E.step(t);
        t++;
        if (iter && E.ended) break;
    }
    E.fold();

    if (lane == 0) {
        // algorithmic ops of the round: 10 W per rewrite, 5 W per pair count
        // that can change, 2 per candidate scanned, and per gi candidate 3 per
        // intersecting term + 8 + 40 per Philox block; the gp trials
        const long long dops = 10LL * M->wn * cd->t_sub + 5LL * M->wn * cd->t_pairs + 2LL * cd->t_scan +
                               3LL * cd->t_gi_terms + 40LL * cd->t_gi_blocks + 8LL * cd->t_gi_cands +
                               (long long)cd->t_rare;
        const unsigned long long ops = cd->ops + (unsigned long long)dops;
        // method ops of the round: 6 per 64-bit word and the nnz of the
        // rewritten rows per rewrite, m per selection, 2 per gi intersect
        // term; the gp trials and shared-coin gi
        const long long dmops = 6LL * ((M->wn + 1) >> 1) * cd->t_sub + (long long)cd->t_nnz + cd->t_scan +
                                (long long)cd->t_gi_cands + 2LL * cd->t_gi_terms + (long long)cd->t_mrare;
        const unsigned long long mops = cd->mops + (unsigned long long)dmops;
        uint32_t* st = M->state + (size_t)E.proc * M->state_words;
        atomicMin(M->round_min, (unsigned long long)(uint32_t)cd->best_cost << 32 | E.gproc);
        atomicAdd(&M->counters[0], (unsigned long long)dops);
        atomicAdd(&M->counters[3], (unsigned long long)dmops);
        if (GM) atomicAdd(&M->counters[5], 1ull);  // process-rounds run on the HBM warp engine
        atomicAdd(&M->counters[1], (unsigned long long)(cd->substeps - cd->sub_before));
        if (S->interval == 0) atomicAdd(&M->counters[2], (unsigned long long)(t - t0));
        if (cd->overflow) atomicExch(S->status, 1);
        st[H_NCOLS] = (uint32_t)E.ncols;
        st[H_NF] = (uint32_t)E.nf;
        st[H_M] = (uint32_t)E.m;
        st[H_COST] = (uint32_t)E.cost;
        st[H_STRAT] = (uint32_t)cd->strat;
        st[H_A] = (uint32_t)cd->a;
        st[H_B] = (uint32_t)cd->b;
        st[H_ENDED] = (uint32_t)E.ended;
        st[H_RUNS] = (uint32_t)cd->runs;
        st[H_SUBSTEPS] = (uint32_t)cd->substeps;
        st[H_BEST_COST] = (uint32_t)cd->best_cost;
        st[H_BEST_LEN] = (uint32_t)cd->best_len;
        st[H_TRAJ_LO] = (uint32_t)cd->traj;
        st[H_TRAJ_HI] = (uint32_t)(cd->traj >> 32);
        st[H_OPS_LO] = (uint32_t)ops;
        st[H_OPS_HI] = (uint32_t)(ops >> 32);
        st[H_BEST_STRAT] = (uint32_t)cd->best_strat;
        st[H_MOPS_LO] = (uint32_t)mops;
        st[H_MOPS_HI] = (uint32_t)(mops >> 32);
    }
    if (!GM) {  // the next round, or a checkpoint, reads the state back
        uint2* spn = reinterpret_cast<uint2*>(st + H_WORDS);
        const uint2* P = E.pn();
        for (int x = lane; x < E.ncols * W; x += 32) spn[x] = P[x];
        uint32_t* sc = st + H_WORDS + 2 * M->cap * W;
        const uint32_t* C = E.cand();
        for (int x = lane; x < E.m; x += 32) sc[x] = C[x];
        int32_t* sf = reinterpret_cast<int32_t*>(sc + M->mmax);
        const int32_t* F = E.F();
        for (int x = lane; x < E.nf; x += 32) sf[x] = F[x];
    }
}

// One launch = one round of every process of a class of matrices.  The grid
// holds as many CTAs as fit on the GPU at once, and every warp takes the next
// process from the launch's work counter until none is left: a warp whose
// process finished early starts another at once instead of idling until its
// CTA's last warp is done.  The share kernel resets the counter for the next
// round.  With unit_list, the launch runs the units unit_list[0 ..
// *unit_count) instead of 0 .. total_units (the processes the process-per-CTA
// engine handed back this round).
template <int W, bool GM, bool GS>
__global__ void __launch_bounds__(128, CSE_MIN_BLOCKS) round_kernel(const DevMat* __restrict__ mats, int n_mats,
                                                       const DevSearch* __restrict__ searches,
                                                       int total_units, int* __restrict__ work,
                                                       const __grid_constant__ WarpLayout L,
                                                       const int* __restrict__ unit_list,
                                                       const int* __restrict__ unit_count) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_units = unit_list ? *unit_count : total_units;
    for (;;) {
        int unit = 0;
        if (lane == 0) unit = atomicAdd(work, 1);
        unit = __shfl_sync(FULL_MASK, unit, 0);
        if (unit >= n_units) return;
        if (unit_list) unit = unit_list[unit];
        run_unit<W, GM, GS>(mats, n_mats, searches, L, smem, warp, lane, unit);
        __syncwarp();
    }
}


// Raises a kernel's maximum dynamic shared memory on the current device to
// `bytes`, never lowering it: the attribute is global to the process, and a
// launch on another thread (the server's worker, another search) may rely on
// a larger value set earlier.
inline cudaError_t raise_max_dynamic_smem(const void* fn, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> set_to;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    auto it = set_to.find({fn, dev});
    if (it != set_to.end() && it->second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) set_to[{fn, dev}] = bytes;
    return e;
}

// Launchers of the round kernels of one engine variant (GS: shared coins).
template <int W, bool GM, bool GS>
static cudaError_t launch_round_w(const DevMat* mats, int n_mats, const DevSearch* searches, int total_units,
                                  int* work, const WarpLayout& L, int ppc, cudaStream_t stream, bool prepare_only,
                                  const int* unit_list = nullptr, const int* unit_count = nullptr) {
    const size_t smem = GM ? 0 : (size_t)L.per_warp * ppc;
    if (prepare_only) {
        if (GM) {  // the HBM path uses no shared memory: give the SM's unified cache to L1
            cudaError_t e = cudaFuncSetAttribute(round_kernel<W, GM, GS>,
                                                 cudaFuncAttributePreferredSharedMemoryCarveout, 0);
            if (e != cudaSuccess) return e;
        }
        return raise_max_dynamic_smem((const void*)round_kernel<W, GM, GS>, (int)smem);
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, round_kernel<W, GM, GS>, 32 * ppc, smem);
    if (e != cudaSuccess) return e;
    const long long need = (total_units + ppc - 1) / ppc;
    const int grid = (int)std::max(1LL, std::min(need, (long long)std::max(sms, 1) * std::max(per_sm, 1)));
    round_kernel<W, GM, GS><<<grid, 32 * ppc, smem, stream>>>(mats, n_mats, searches, total_units, work, L,
                                                              unit_list, unit_count);
    return cudaGetLastError();
}

template <bool GM, bool GS>
static cudaError_t launch_round_gm(int W, const DevMat* mats, int n_mats, const DevSearch* searches,
                                   int total_units, int* work, const WarpLayout& L, int ppc, cudaStream_t stream,
                                   bool prep) {
    switch (W) {
        case 1: return launch_round_w<1, GM, GS>(mats, n_mats, searches, total_units, work, L, ppc, stream, prep);
        case 2: return launch_round_w<2, GM, GS>(mats, n_mats, searches, total_units, work, L, ppc, stream, prep);
        case 3: return launch_round_w<3, GM, GS>(mats, n_mats, searches, total_units, work, L, ppc, stream, prep);
        case 4: return launch_round_w<4, GM, GS>(mats, n_mats, searches, total_units, work, L, ppc, stream, prep);
        case 5: return launch_round_w<5, GM, GS>(mats, n_mats, searches, total_units, work, L, ppc, stream, prep);
        case 6: return launch_round_w<6, GM, GS>(mats, n_mats, searches, total_units, work, L, ppc, stream, prep);
        case 7: return launch_round_w<7, GM, GS>(mats, n_mats, searches, total_units, work, L, ppc, stream, prep);
        case 8: return launch_round_w<8, GM, GS>(mats, n_mats, searches, total_units, work, L, ppc, stream, prep);
        default: return cudaErrorInvalidValue;
    }
}

template <bool GS>
static cudaError_t launch_round_variant(int W, bool gm, const DevMat* mats, int n_mats, const DevSearch* searches,
                                        int total_units, int* work, const WarpLayout& L, int ppc,
                                        cudaStream_t stream, bool prep) {
    return gm ? launch_round_gm<true, GS>(W, mats, n_mats, searches, total_units, work, L, ppc, stream, prep)
              : launch_round_gm<false, GS>(W, mats, n_mats, searches, total_units, work, L, ppc, stream, prep);
}

}  // namespace cse
