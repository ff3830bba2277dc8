// Process-per-CTA step engine for large expression sets (the (6,6,6:153)
// shape and the large served formats): the same Algorithm 1 steps, draws and
// integer scores as the one-warp-per-process engine (cse_engine.cuh), bit for
// bit, with one CTA of kCtaThreads threads per process and the process's
// working arrays in the CTA's shared memory instead of its HBM state region.
//
// Why: a large process has thousands of candidates, so every phase of a step
// is hundreds of 32-lane chunks; one warp per process keeps tens of such
// processes per SM, whose working sets (tens of KB each) live in L2, and the
// engine waits on L2.  Here two processes share an SM and each phase is
// spread over 16 warps whose loads hit shared memory.
//
// Layout of a process in shared memory: columns P[cap][W] (uint2: +rows,
// -rows), the candidate list C (sorted by key = hi << 11 | lo << 1 | neg),
// the current run's list F, and the Greedy-Intersections adjacency: for every
// variable v its list A_v (first the candidates whose larger index is v, a
// contiguous block of C, then those whose smaller index is v, in list order),
// A_v's weight bytes AW, and its bit-planes: plane k of 64 positions of A_v is
// the mask of the positions whose weight (c - 1) has bit k set.  The planes
// are packed with warp ballots from AW, without atomics.
//
// Order-dependent passes (compaction, lo-list ranks, the k-th tie, the
// weighted pick) split the list into one contiguous segment per warp; each
// warp walks its segment in list order and a prefix over the warps joins the
// segments.
//
// Capacities: the list holds ms <= kCtaListMax entries and the planes pln_cap
// words.  A process that would outgrow either (or whose list starts longer)
// stops, its state region untouched since the round started, and is listed
// for the warp engine, which redoes its whole round from that state (every
// draw is keyed by (seed, process, step), so the redo is the same round).

#pragma once

#include "cse_engine.cuh"

namespace cse {

// Block-wide scratch for reductions and broadcasts (sized for the widest CTA).
struct CtaShared {
    int bc[8];                     // broadcast slots
    int ws[kCtaWarps * 4];         // per-warp partial sums
    unsigned int wr[kCtaWarps * 3];  // per-warp argmax partials
};

// NW warps per process (a CTA of 32 NW threads).
template <int W, int NW>
struct CtaEngine {
    static constexpr int NT = 32 * NW;
    unsigned char* sm;
    const CtaLayout* L;
    const DevMat* M;
    const DevSearch* S;
    int proc, tid, lane, warp, cap, ms;
    uint32_t gproc;  // the global process index (draws, round keys)
    // block-uniform state (every thread holds the same values)
    int ncols, nf, m, cost, ended, abandon;

    __device__ __forceinline__ uint2* pn() const { return reinterpret_cast<uint2*>(sm + L->off_pn); }
    __device__ __forceinline__ uint32_t* cand() const { return reinterpret_cast<uint32_t*>(sm + L->off_cand); }
    __device__ __forceinline__ uint16_t* pl() const { return reinterpret_cast<uint16_t*>(sm + L->off_pl); }
    __device__ __forceinline__ uint8_t* aw() const { return sm + L->off_aw; }
    __device__ __forceinline__ uint16_t* hs() const { return reinterpret_cast<uint16_t*>(sm + L->off_hs); }
    __device__ __forceinline__ uint16_t* he() const { return reinterpret_cast<uint16_t*>(sm + L->off_he); }
    __device__ __forceinline__ uint16_t* vb() const { return reinterpret_cast<uint16_t*>(sm + L->off_vb); }
    __device__ __forceinline__ uint16_t* pb() const { return reinterpret_cast<uint16_t*>(sm + L->off_pb); }
    __device__ __forceinline__ uint16_t* lct() const { return reinterpret_cast<uint16_t*>(sm + L->off_lct); }
    __device__ __forceinline__ uint32_t* gsum() const { return reinterpret_cast<uint32_t*>(sm + L->off_g); }
    __device__ __forceinline__ uint16_t* lcw() const { return reinterpret_cast<uint16_t*>(sm + L->off_lcw); }
    __device__ __forceinline__ int32_t* F() const { return reinterpret_cast<int32_t*>(sm + L->off_f); }
    __device__ __forceinline__ unsigned long long* planes() const {
        return reinterpret_cast<unsigned long long*>(sm + L->off_pln);
    }
    __device__ __forceinline__ Cold* cold() const { return reinterpret_cast<Cold*>(sm + L->off_cold); }
    __device__ __forceinline__ CtaShared* sh() const { return reinterpret_cast<CtaShared*>(sm + L->off_sh); }

    __device__ __forceinline__ uint32_t c2(uint32_t purpose, uint32_t extra_hi) const {
        return ((uint32_t)M->mat_index & 0xFFu) << 24 | (purpose & 0xFu) << 20 | (extra_hi & 0xFFFFFu);
    }
    __device__ __forceinline__ uint4 draw(int t, uint32_t purpose) const {
        return philox_call(gproc, (uint32_t)t, c2(purpose, 0), 0u, (uint32_t)S->seed, (uint32_t)(S->seed >> 32));
    }

    // ---- block-wide helpers (each ends with every thread holding the result)
    __device__ __forceinline__ int4 bsum4(int a, int b, int c, int d) {
        a = __reduce_add_sync(FULL_MASK, a);
        b = __reduce_add_sync(FULL_MASK, b);
        c = __reduce_add_sync(FULL_MASK, c);
        d = __reduce_add_sync(FULL_MASK, d);
        int* ws = sh()->ws;
        if (lane == 0) {
            ws[4 * warp] = a;
            ws[4 * warp + 1] = b;
            ws[4 * warp + 2] = c;
            ws[4 * warp + 3] = d;
        }
        __syncthreads();
        int4 r = make_int4(0, 0, 0, 0);
#pragma unroll
        for (int w = 0; w < NW; w++) {
            r.x += ws[4 * w];
            r.y += ws[4 * w + 1];
            r.z += ws[4 * w + 2];
            r.w += ws[4 * w + 3];
        }
        __syncthreads();
        return r;
    }
    __device__ __forceinline__ uint32_t bmax(uint32_t v) {
        v = __reduce_max_sync(FULL_MASK, v);
        int* ws = sh()->ws;
        if (lane == 0) ws[warp] = (int)v;
        __syncthreads();
        uint32_t r = 0;
#pragma unroll
        for (int w = 0; w < NW; w++) r = max(r, (uint32_t)ws[w]);
        __syncthreads();
        return r;
    }
    // Exclusive prefix over the warps of a per-warp value (lane-uniform);
    // *total gets the sum over all warps.
    __device__ __forceinline__ int wprefix(int v, int* total) {
        int* ws = sh()->ws;
        if (lane == 0) ws[warp] = v;
        __syncthreads();
        int pre = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < NW; w++) {
            const int x = ws[w];
            pre += w < warp ? x : 0;
            tot += x;
        }
        __syncthreads();
        *total = tot;
        return pre;
    }
    // The block's argmax of (score >= 2^32, index): lowest index on ties;
    // best_q < 0 for none.
    __device__ __forceinline__ int bargmax(long long best_s, int best_q) {
        const unsigned long long us = best_q >= 0 ? (unsigned long long)best_s : 0ull;
        const uint32_t hi = (uint32_t)(us >> 32), lo = (uint32_t)us;
        const uint32_t mhi = __reduce_max_sync(FULL_MASK, hi);
        const uint32_t mlo = __reduce_max_sync(FULL_MASK, hi == mhi ? lo : 0u);
        const uint32_t mq =
            __reduce_min_sync(FULL_MASK, (hi == mhi && lo == mlo && best_q >= 0) ? (uint32_t)best_q : 0xFFFFFFFFu);
        unsigned int* wr = sh()->wr;
        if (lane == 0) {
            wr[3 * warp] = mhi;
            wr[3 * warp + 1] = mlo;
            wr[3 * warp + 2] = mq;
        }
        __syncthreads();
        uint32_t bh = 0, bl = 0, bq = 0xFFFFFFFFu;
#pragma unroll
        for (int w = 0; w < NW; w++) {
            const uint32_t h = wr[3 * w], l = wr[3 * w + 1], q = wr[3 * w + 2];
            if (q == 0xFFFFFFFFu) continue;
            if (h > bh || (h == bh && l > bl) || (h == bh && l == bl && q < bq)) {
                bh = h;
                bl = l;
                bq = q;
            }
        }
        __syncthreads();
        return (int)bq;
    }
    // This warp's segment of the list: [*b, *e), segments of a multiple of 32.
    __device__ __forceinline__ void segment(int* b, int* e) const {
        const int s = ((m + 32 * NW - 1) / (32 * NW)) * 32;
        *b = warp * s;
        *e = min(m, *b + s);
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

    // Substitution of (x_i + s x_j), i < j, by x_k, k = ncols (Section 3.2.1,
    // Algorithm 1), with the candidate list update: recount the candidates
    // holding x_i or x_j (stable compaction), then append the pairs (u, k).
    __device__ void subst(int i, int j, int neg) {
        const uint32_t lt = lanemask_lt();
        uint2* P = pn();
        uint32_t* C = cand();
        const int k = ncols;
        if (tid < W) {
            uint2 A = P[i * W + tid], B = P[j * W + tid];
            uint32_t rp, rn;
            if (!neg) {
                rp = A.x & B.x;
                rn = A.y & B.y;
                B.x &= ~rp;
                B.y &= ~rn;
            } else {
                rp = A.x & B.y;
                rn = A.y & B.x;
                B.x &= ~rn;
                B.y &= ~rp;
            }
            A.x &= ~rp;
            A.y &= ~rn;
            P[i * W + tid] = A;
            P[j * W + tid] = B;
            P[k * W + tid] = make_uint2(rp, rn);
        }
        if (warp == 0) {
            int cpart = 0;
            if (lane < W) {
                const uint2 K = P[k * W + lane];
                cpart = __popc(K.x) + __popc(K.y);
            }
            cpart = __reduce_add_sync(FULL_MASK, cpart);
            if (lane == 0) sh()->bc[0] = cpart;
        }
        __syncthreads();
        const int c = sh()->bc[0];
        // recount and compaction: this warp's segment is held in registers,
        // so every warp has read its entries before any warp writes
        int sb, se;
        segment(&sb, &se);
        uint32_t ev[kCtaSeg];  // 32 kCtaSeg NW >= ms entries: the whole segment
        int kept = 0, nij = 0;
#pragma unroll
        for (int x = 0; x < kCtaSeg; x++) {
            const int q = sb + 32 * x + lane;
            uint32_t e = 0;
            if (q < se) {
                e = C[q];
                const int lo = key_lo(e), hi = key_hi(e);
                if (lo == i || lo == j || hi == i || hi == j) {
                    int cp, cm;
                    counts(lo, hi, cp, cm);
                    e = (e & 0x1FFFFFu) | ((uint32_t)((e & 1u) ? cm : cp) << 21);
                    nij++;
                }
            }
            ev[x] = e;
            kept += cand_c(e) >= 2;
        }
        kept = __reduce_add_sync(FULL_MASK, kept);
        nij = __reduce_add_sync(FULL_MASK, nij);
        int newm = 0;
        int pos = wprefix(kept, &newm);
#pragma unroll
        for (int x = 0; x < kCtaSeg; x++) {
            const bool keep = cand_c(ev[x]) >= 2;
            const uint32_t kb = __ballot_sync(FULL_MASK, keep);
            if (keep) C[pos + __popc(kb & lt)] = ev[x];
            pos += __popc(kb);
        }
        // the new pairs (u, k), u < k, NT columns at a time
        int added = 0, nu = 0, rb = 0;
        int* ws = sh()->ws;
        int nij_all = 0;
        for (int ubase = 0; ubase < k; ubase += NT) {
            int cp = 0, cm = 0, both = 0;
            bool live = false;
            const int u = ubase + tid;
            if (u < k) {
                uint32_t sup = 0;
                int ng = 0;
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
            }
            const int ep = cp >= 2, em = cm >= 2;
            const int cnt = ep + em;
            const int incl = warp_incl_scan(cnt, lane);
            const int wtot = __shfl_sync(FULL_MASK, incl, 31);
            const int wlive = __popc(__ballot_sync(FULL_MASK, live));
            const int wboth = __reduce_add_sync(FULL_MASK, both);
            if (lane == 0) {
                ws[4 * warp] = wtot;
                ws[4 * warp + 1] = wlive;
                ws[4 * warp + 2] = wboth;
                ws[4 * warp + 3] = ubase == 0 ? nij : 0;  // this warp's recounted candidates
            }
            __syncthreads();  // also orders the compaction's writes before the appends
            int off = 0, chunk = 0;
#pragma unroll
            for (int w = 0; w < NW; w++) {
                const int x = ws[4 * w];
                off += w < warp ? x : 0;
                chunk += x;
                nu += ws[4 * w + 1];
                rb += ws[4 * w + 2];
                nij_all += ws[4 * w + 3];
            }
            __syncthreads();  // the partials are read before the next chunk writes them
            if (newm + added + chunk > ms) {  // the list would outgrow its shared-memory capacity
                abandon = 1;
                return;
            }
            int p = newm + added + off + incl - cnt;
            if (ep) C[p++] = make_cand(u, k, 0, cp);
            if (em) C[p] = make_cand(u, k, 1, cm);
            added += chunk;
        }
        nij = nij_all;
        if (tid == 0) {
            F()[nf] = (int32_t)((uint32_t)i | (uint32_t)j << 10 | (uint32_t)neg << 20);
            Cold* cd = cold();
            cd->t_sub++;
            cd->t_pairs += (unsigned)(nij + nu);
            cd->t_nnz += (unsigned)(rb + 2 * c);
        }
        nf++;
        ncols++;
        cost -= c - 1;
        m = newm + added;
        __syncthreads();
    }

    // Closes the current run into the process's best record (strictly lower
    // cost replaces).
    __device__ void fold() {
        Cold* cd = cold();
        const int bc = cd->best_cost;
        __syncthreads();
        if (cost < bc) {
            int32_t* dst = M->best_list + (size_t)proc * cap;
            const int32_t* f = F();
            for (int x = tid; x < nf; x += NT) dst[x] = f[x];
            if (tid == 0) {
                cd->best_cost = cost;
                cd->best_len = nf;
                cd->best_strat = cd->strat;
            }
        }
        __syncthreads();
    }

    // Run start at step t (Sections 3.5.1-3.5.2); returns the prefix length
    // of the snapshot to replay.
    __device__ int start_run(int t) {
        if (t > 0) fold();
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
        if (tid == 0) {
            Cold* cd = cold();
            cd->runs++;
            cd->strat = strat;
            cd->a = (int)scale32(R.y, 32769u);
            cd->b = 32768 + (int)scale32(R.z, 32769u);
        }
        const int nx = M->nx;
        const int m0 = M->meta0[1];
        if (m0 > ms) {
            abandon = 1;
            __syncthreads();
            return 0;
        }
        uint2* P = pn();
        uint32_t* C = cand();
        for (int x = tid; x < nx * W; x += NT) P[x] = M->pn0[x];
        for (int x = tid; x < m0; x += NT) C[x] = M->cand0[x];
        m = m0;
        ncols = nx;
        nf = 0;
        cost = M->meta0[0];
        int k = 0;
        if (M->snap_meta[0] != INT_MAX && (uint64_t)R.w < S->share_thr) {
            const int K = (3 * M->snap_meta[1]) / 4;
            if (K >= 1) k = 1 + (int)scale32(draw(t, PU_SHAREK).x, (uint32_t)K);
        }
        ended = 0;
        if (tid == 0) {
            Cold* cd = cold();
            if (cd->trace) cd->traj = fnv(fnv(cd->traj, (uint32_t)t), 0xA0000000u | (uint32_t)strat << 12 | (uint32_t)k);
        }
        __syncthreads();
        return k;
    }

    // Greedy: highest c, lowest key.
    __device__ int sel_g() {
        const uint32_t* C = cand();
        uint32_t best = 0;
        for (int q = tid; q < m; q += NT) {
            const uint32_t v = (uint32_t)cand_c(C[q]) << 16 | (uint32_t)(0xFFFF - q);
            best = best > v ? best : v;
        }
        best = bmax(best);
        return 0xFFFF - (int)(best & 0xFFFFu);
    }

    // Greedy-Alternative: the (u * n_ties) >> 32-th of the max-c ties in order.
    __device__ int sel_ga(uint32_t u) {
        const uint32_t lt = lanemask_lt();
        const uint32_t* C = cand();
        uint32_t lmax = 0;
        for (int q = tid; q < m; q += NT) lmax = max(lmax, (uint32_t)cand_c(C[q]));
        const int cmax = (int)bmax(lmax);
        int sb, se;
        segment(&sb, &se);
        int cnt = 0;
        for (int base = sb; base < se; base += 32) {
            const int q = base + lane;
            cnt += __popc(__ballot_sync(FULL_MASK, q < se && cand_c(C[q]) == cmax));
        }
        int nt = 0;
        const int pre = wprefix(cnt, &nt);
        const uint32_t want = scale32(u, (uint32_t)nt);
        if ((uint32_t)pre <= want && want < (uint32_t)(pre + cnt)) {
            uint32_t w = want - (uint32_t)pre;
            for (int base = sb; base < se; base += 32) {
                const int q = base + lane;
                const bool tie = q < se && cand_c(C[q]) == cmax;
                const uint32_t bt = __ballot_sync(FULL_MASK, tie);
                const uint32_t n = (uint32_t)__popc(bt);
                if (w < n) {
                    const uint32_t hit = __ballot_sync(FULL_MASK, tie && (uint32_t)__popc(bt & lt) == w);
                    if (lane == 0) sh()->bc[1] = base + __ffs(hit) - 1;
                    break;
                }
                w -= n;
            }
        }
        __syncthreads();
        const int r = sh()->bc[1];
        __syncthreads();
        return r;
    }

    // Weighted-Random: the first candidate whose running sum of (c - 1)
    // exceeds (u * T) >> 32, T = sum (c - 1).
    __device__ int sel_wr(uint32_t u) {
        const uint32_t* C = cand();
        int sb, se;
        segment(&sb, &se);
        int part = 0;
        for (int q = sb + lane; q < se; q += 32) part += cand_c(C[q]) - 1;
        part = __reduce_add_sync(FULL_MASK, part);
        int total = 0;
        const int pre = wprefix(part, &total);
        const uint32_t x = scale32(u, (uint32_t)total);
        if ((uint32_t)pre <= x && x < (uint32_t)(pre + part)) {
            uint32_t acc = (uint32_t)pre;
            for (int base = sb; base < se; base += 32) {
                const int q = base + lane;
                const int w = q < se ? cand_c(C[q]) - 1 : 0;
                const int incl = warp_incl_scan(w, lane);
                const uint32_t hit = __ballot_sync(FULL_MASK, q < se && acc + (uint32_t)incl > x);
                if (hit) {
                    if (lane == 0) sh()->bc[2] = base + __ffs(hit) - 1;
                    break;
                }
                acc += (uint32_t)__shfl_sync(FULL_MASK, incl, 31);
            }
        }
        __syncthreads();
        const int r = sh()->bc[2];
        __syncthreads();
        return r;
    }

    // Greedy-Intersections (Section 3.4.2): S_p = (c_p - 1) 2^32 + a (2^16
    // D_p + b X_p); the coin-weighted sums X_p over bit-planes of the lists
    // A_i, A_j; argmax, lowest key on ties.
    __device__ int sel_gi(int t) {
        const uint32_t lt = lanemask_lt();
        const uint32_t* C = cand();
        uint16_t* HS = hs();
        uint16_t* HE = he();
        uint16_t* VB = vb();
        uint16_t* PB = pb();
        uint16_t* LCT = lct();
        uint16_t* LCW = lcw() + warp * cap;  // this warp's lo counts, then lo bases
        uint32_t* G = gsum();
        uint16_t* PL = pl();
        uint8_t* AW = aw();
        unsigned long long* PLN = planes();
        for (int v = tid; v < ncols; v += NT) {
            HS[v] = 0;
            HE[v] = 0;
        }
        for (int v = lane; v < ncols; v += 32) LCW[v] = 0;  // each warp its own row
        __syncthreads();
        int sb, se;
        segment(&sb, &se);
        int part = 0;
        uint32_t wmax = 1;
        for (int base = sb; base < se; base += 32) {
            const int q = base + lane;
            const bool valid = q < se;
            const uint32_t act = __ballot_sync(FULL_MASK, valid);
            if (valid) {
                const uint32_t e = C[q];
                const int hi = key_hi(e), lo = key_lo(e);
                part += cand_c(e) - 1;
                wmax = max(wmax, (uint32_t)(cand_c(e) - 1));
                if (q == 0 || key_hi(C[q - 1]) != hi) HS[hi] = (uint16_t)q;
                if (q == m - 1 || key_hi(C[q + 1]) != hi) HE[hi] = (uint16_t)(q + 1);
                const uint32_t peers = __match_any_sync(act, lo);
                if ((peers & lt) == 0) LCW[lo] = (uint16_t)(LCW[lo] + __popc(peers));
            }
            __syncwarp();
        }
        const int T = bsum4(part, 0, 0, 0).x;
        const int B = 32 - __clz((int)bmax(wmax));
        // per variable: lo totals, each warp's lo base, degree; positions and
        // 64-position blocks of A_v by a block-wide exclusive scan, NT
        // variables at a time
        uint32_t carry = 0;
        for (int vbase = 0; vbase < ncols; vbase += NT) {
            uint32_t packed = 0;
            const int v = vbase + tid;
            if (v < ncols) {
                int run = 0;
#pragma unroll
                for (int w = 0; w < NW; w++) {
                    uint16_t* cw = lcw() + w * cap + v;
                    const int x = *cw;
                    *cw = (uint16_t)run;
                    run += x;
                }
                LCT[v] = (uint16_t)run;
                const int deg = (HE[v] - HS[v]) + run;
                packed = (uint32_t)deg | (uint32_t)((deg + 63) >> 6) << 16;
            }
            const uint32_t incl = (uint32_t)warp_incl_scan((int)packed, lane);
            int tot = 0;
            const int wpre = wprefix((int)__shfl_sync(FULL_MASK, incl, 31), &tot);
            if (v < ncols) {
                const uint32_t ex = carry + (uint32_t)wpre + incl - packed;
                VB[v] = (uint16_t)(ex & 0xFFFFu);
                PB[v] = (uint16_t)(ex >> 16);
            }
            carry += (uint32_t)tot;
        }
        const int nblk = (int)(carry >> 16);
        const int BP = (B + 1) & ~1;  // planes per block: B rounded up to even
        if (nblk * BP > L->pln_cap) {
            abandon = 1;
            __syncthreads();
            return 0;
        }
        __syncthreads();
        // positions in A_v and the weight bytes, in list order per segment
        for (int base = sb; base < se; base += 32) {
            const int q = base + lane;
            const bool valid = q < se;
            const uint32_t act = __ballot_sync(FULL_MASK, valid);
            uint32_t peers = 0;
            int lo = 0;
            if (valid) {
                const uint32_t e = C[q];
                const int hi = key_hi(e);
                lo = key_lo(e);
                const uint8_t w = (uint8_t)(cand_c(e) - 1);
                peers = __match_any_sync(act, lo);
                const int xl = (HE[lo] - HS[lo]) + LCW[lo] + __popc(peers & lt);
                PL[q] = (uint16_t)(VB[lo] + xl);
                AW[VB[hi] + (q - HS[hi])] = w;
                AW[VB[lo] + xl] = w;
            }
            __syncwarp();
            if (valid && (peers & lt) == 0) LCW[lo] = (uint16_t)(LCW[lo] + __popc(peers));
            __syncwarp();
        }
        __syncthreads();
        // bit-planes and weight sums: one variable per warp at a time
        for (int vv = warp; vv < ncols; vv += NW) {
            const int deg = (HE[vv] - HS[vv]) + LCT[vv];
            const int base = VB[vv];
            unsigned long long* dst = PLN + (size_t)PB[vv] * BP;
            int gs = 0;
            for (int x0 = 0; x0 < deg; x0 += 64) {
                const int w0 = x0 + lane < deg ? AW[base + x0 + lane] : 0;
                const int w1 = x0 + 32 + lane < deg ? AW[base + x0 + 32 + lane] : 0;
                gs += w0 + w1;
                for (int kk = 0; kk < BP; kk++) {  // plane B of an odd B is the zero padding
                    const uint32_t lo32 = __ballot_sync(FULL_MASK, (w0 >> kk) & 1);
                    const uint32_t hi32 = __ballot_sync(FULL_MASK, (w1 >> kk) & 1);
                    if (lane == kk) dst[kk] = (unsigned long long)hi32 << 32 | lo32;
                }
                dst += BP;
            }
            gs = __reduce_add_sync(FULL_MASK, gs);
            if (lane == 0) G[vv] = (uint32_t)gs;
        }
        __syncthreads();
        // scoring: candidates strided over the threads
        const uint32_t k0 = (uint32_t)S->seed, k1 = (uint32_t)(S->seed >> 32);
        const uint32_t c2g = c2(PU_GI, 0);
        const long long a = cold()->a, b = cold()->b;
        long long best_s = LLONG_MIN;
        int best_q = -1;
        unsigned gi_terms = 0, gi_blocks = 0;
        for (int p = tid; p < m; p += NT) {
            const uint32_t e = C[p];
            const int i = key_lo(e), j = key_hi(e), wp = cand_c(e) - 1;
            const uint32_t key = e & 0x1FFFFFu;
            const int n0 = (HE[i] - HS[i]) + LCT[i];
            const int n1 = (HE[j] - HS[j]) + LCT[j];
            const int lp0 = PL[p] - VB[i];  // p's place in A_i
            const int lp1 = p - HS[j];      // p's place in A_j
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
            int X = 0, inter = 0, nb = 0;
            if (nint > 0) {
                const int nb0 = (n0 + 63) >> 6, nb1 = (n1 + 63) >> 6;
                nb = nb0 > nb1 ? nb0 : nb1;
                const unsigned long long* P0 = PLN + (size_t)PB[i] * BP;
                const unsigned long long* P1 = PLN + (size_t)PB[j] * BP;
                for (int blk = 0; blk < nb; blk++) {
                    uint32_t r0 = gproc, r1 = (uint32_t)t, r2 = c2g | (uint32_t)blk, r3 = key;
                    philox(r0, r1, r2, r3, k0, k1);
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
                inter = (int)G[i] + (int)G[j] - 2 * wp - wsib;
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
        gi_terms = __reduce_add_sync(FULL_MASK, gi_terms);
        gi_blocks = __reduce_add_sync(FULL_MASK, gi_blocks);
        if (lane == 0) {
            Cold* cd = cold();
            atomicAdd(&cd->t_gi_terms, gi_terms);
            atomicAdd(&cd->t_gi_blocks, gi_blocks);
        }
        if (tid == 0) cold()->t_gi_cands += (unsigned)m;
        return bargmax(best_s, best_q);
    }

    // Greedy-Potential (Section 2.2): as gp_select of the warp engine, one
    // candidate per thread.
    __device__ int sel_gp() {
        const uint2* P = pn();
        const uint32_t* C = cand();
        const uint32_t a = (uint32_t)cold()->a;
        int lv = 0;
        for (int u = tid; u < ncols; u += NT) {
            uint32_t sup = 0;
#pragma unroll
            for (int w = 0; w < W; w++) sup |= P[u * W + w].x | P[u * W + w].y;
            lv += sup != 0;
        }
        const int nlive = bsum4(lv, 0, 0, 0).x;
        uint32_t best_s = 0;
        int best_q = -1;
        unsigned ops = 0, mops = 0;
        for (int p = tid; p < m; p += NT) {
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
            if (best_q < 0 || sc > best_s) {
                best_s = sc;
                best_q = p;
            }
            const int live = nlive - (nni == c) - (nnj == c);
            ops += 5u * (unsigned)M->wn * (unsigned)live + 8u;  // the matrix's own words
            mops += 6u * (unsigned)((M->wn + 1) >> 1) + (unsigned)rnnz;
        }
        ops = __reduce_add_sync(FULL_MASK, ops);
        mops = __reduce_add_sync(FULL_MASK, mops);
        if (lane == 0) {
            atomicAdd(&cold()->t_rare, (unsigned long long)ops);
            atomicAdd(&cold()->t_mrare, (unsigned long long)mops);
        }
        if (tid == 0) atomicAdd(&cold()->t_mrare, (unsigned long long)m);
        // scores fit 32 bits: put them in the high word of a 64-bit key
        // (adding 2^32 so that a valid score is never 0)
        return bargmax(best_q >= 0 ? (long long)(((unsigned long long)best_s + 1ull) << 32) : 0, best_q);
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
        if (s == ST_GI) return sel_gi(t);
        if (s == ST_GP) return sel_gp();
        if (tid == 0) cold()->t_scan += (unsigned)m;
        if (s == ST_GA) return sel_ga(d.z);
        if (s == ST_WR) return sel_wr(d.w);
        return sel_g();
    }

    // One step of the step clock (one Algorithm 1 iteration).
    __device__ void step(int t) {
        int replay = 0;
        if (t == 0 || ended) {
            replay = start_run(t);
            if (abandon) return;
        }
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
                if (abandon) return;
                const uint32_t ce = cand()[sel];
                __syncthreads();
                i = key_lo(ce);
                j = key_hi(ce);
                neg = (int)(ce & 1u);
            }
            subst(i, j, neg);
            if (abandon) return;
            if (e >= replay) break;
        }
        if (tid == 0) {
            Cold* cd = cold();
            cd->substeps++;
            if (cd->trace) cd->traj = fnv(fnv(cd->traj, (uint32_t)t), (uint32_t)F()[nf - 1]);
        }
        if (m == 0 || ncols >= cap) ended = 1;
    }
};

// One round of one process on a CTA; returns false if the process must be
// redone by the warp engine (nothing of its state region was written).
template <int W, int NW>
__device__ bool cta_run_unit(const DevMat* __restrict__ mats, int n_mats, const DevSearch* __restrict__ searches,
                             const CtaLayout& L, unsigned char* smem, int unit) {
    constexpr int NT = 32 * NW;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int mi = 0, mhi = n_mats - 1;  // the last matrix whose first unit is <= unit
    while (mi < mhi) {
        const int mid = (mi + mhi + 1) >> 1;
        if (mats[mid].unit_base <= unit) mi = mid; else mhi = mid - 1;
    }
    const DevMat* M = &mats[mi];
    const DevSearch* S = &searches[M->search];
    const int clk = *S->clock;
    if (clk >= S->budget || (S->interval == 0 && S->conv[1])) return true;
    const int t0 = S->interval == 0 ? clk * M->cap : clk;

    uint32_t* st = M->state + (size_t)(unit - M->unit_base) * M->state_words;
    unsigned char* gst = reinterpret_cast<unsigned char*>(st + H_WORDS);  // the HBM engine's arrays
    CtaEngine<W, NW> E;
    E.sm = smem;
    E.L = &L;
    E.M = M;
    E.S = S;
    E.proc = unit - M->unit_base;
    E.gproc = (uint32_t)(E.proc + M->proc_offset);
    E.tid = tid;
    E.lane = lane;
    E.warp = warp;
    E.cap = M->cap;
    E.ms = min(L.ms, M->mmax);
    E.abandon = 0;
    Cold* cd = E.cold();
    if (t0 == 0) {
        E.ncols = M->nx;
        E.nf = 0;
        E.m = 0;
        E.cost = M->meta0[0];
        E.ended = 1;
    } else {
        E.ncols = (int)st[H_NCOLS];
        E.nf = (int)st[H_NF];
        E.m = (int)st[H_M];
        E.cost = (int)st[H_COST];
        E.ended = (int)st[H_ENDED];
    }
    if (tid == 0) {
        if (t0 == 0) {
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
        } else {
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
        cd->trace = S->trace;
        cd->overflow = 0;
        cd->t_sub = cd->t_pairs = cd->t_scan = 0;
        cd->t_gi_terms = cd->t_gi_blocks = cd->t_gi_cands = 0;
        cd->t_rare = 0;
        cd->t_mrare = 0;
        cd->t_nnz = 0;
        cd->sub_before = cd->substeps;
    }
    // a list too long for shared memory, or (at a round start that is not a
    // run start) one short enough that one warp serves it better: the warp
    // engine takes the round
    if (E.m > E.ms || (t0 > 0 && !E.ended && E.m < L.min_m)) return false;
    if (t0 > 0) {  // the process's arrays, from the HBM engine's layout of its state region
        const uint2* spn = reinterpret_cast<const uint2*>(gst + M->gml.off_pn);
        uint2* P = E.pn();
        for (int x = tid; x < E.ncols * W; x += NT) P[x] = spn[x];
        const uint32_t* sc = reinterpret_cast<const uint32_t*>(gst + M->gml.off_cand);
        uint32_t* C = E.cand();
        for (int x = tid; x < E.m; x += NT) C[x] = sc[x];
        const int32_t* sf = reinterpret_cast<const int32_t*>(gst + M->gml.off_f);
        int32_t* F = E.F();
        for (int x = tid; x < E.nf; x += NT) F[x] = sf[x];
    }
    __syncthreads();

    const bool iter = S->interval == 0;
    const int t1 = iter ? t0 + M->cap : min(t0 + S->interval, S->budget);
    int t = t0;
    while (t < t1) {
        E.step(t);
        if (E.abandon) return false;
        t++;
        if (iter && E.ended) break;
    }
    E.fold();

    if (tid == 0) {
        const long long dops = 10LL * M->wn * cd->t_sub + 5LL * M->wn * cd->t_pairs + 2LL * cd->t_scan +
                               3LL * cd->t_gi_terms + 40LL * cd->t_gi_blocks + 8LL * cd->t_gi_cands +
                               (long long)cd->t_rare;
        const unsigned long long ops = cd->ops + (unsigned long long)dops;
        const long long dmops = 6LL * ((M->wn + 1) >> 1) * cd->t_sub + (long long)cd->t_nnz + cd->t_scan +
                                (long long)cd->t_gi_cands + 2LL * cd->t_gi_terms + (long long)cd->t_mrare;
        const unsigned long long mops = cd->mops + (unsigned long long)dmops;
        atomicMin(M->round_min, (unsigned long long)(uint32_t)cd->best_cost << 32 | E.gproc);
        atomicAdd(&M->counters[0], (unsigned long long)dops);
        atomicAdd(&M->counters[1], (unsigned long long)(cd->substeps - cd->sub_before));
        atomicAdd(&M->counters[3], (unsigned long long)dmops);
        atomicAdd(&M->counters[4], 1ull);  // process-rounds run on this engine
        if (iter) atomicAdd(&M->counters[2], (unsigned long long)(t - t0));
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
    {
        uint2* spn = reinterpret_cast<uint2*>(gst + M->gml.off_pn);
        const uint2* P = E.pn();
        for (int x = tid; x < E.ncols * W; x += NT) spn[x] = P[x];
        uint32_t* sc = reinterpret_cast<uint32_t*>(gst + M->gml.off_cand);
        const uint32_t* C = E.cand();
        for (int x = tid; x < E.m; x += NT) sc[x] = C[x];
        int32_t* sf = reinterpret_cast<int32_t*>(gst + M->gml.off_f);
        const int32_t* F = E.F();
        for (int x = tid; x < E.nf; x += NT) sf[x] = F[x];
    }
    return true;
}

// One launch = one round of every process of a class of large matrices, one
// process per CTA at a time (persistent grid, work counter work3[0]);
// processes that outgrow the shared-memory capacities are appended to
// redo_list (count work3[2]) for the warp engine's launch that follows.
template <int W, int NW>
__global__ void __launch_bounds__(32 * NW, 1024 / (32 * NW)) cta_round_kernel(const DevMat* __restrict__ mats, int n_mats,
                                                                  const DevSearch* __restrict__ searches,
                                                                  int total_units, int* __restrict__ work3,
                                                                  int* __restrict__ redo_list,
                                                                  const __grid_constant__ CtaLayout L) {
    extern __shared__ __align__(16) unsigned char smem[];
    CtaShared* sh = reinterpret_cast<CtaShared*>(smem + L.off_sh);
    for (;;) {
        if (threadIdx.x == 0) sh->bc[7] = atomicAdd(&work3[0], 1);
        __syncthreads();
        const int unit = sh->bc[7];
        __syncthreads();
        if (unit >= total_units) return;
        const bool done = cta_run_unit<W, NW>(mats, n_mats, searches, L, smem, unit);
        if (!done && threadIdx.x == 0) redo_list[atomicAdd(&work3[2], 1)] = unit;
        __syncthreads();
    }
}

}  // namespace cse
