// Kernels of the parallel heuristic CSE search on sm_103a other than the step
// engine (cse_engine.cuh): ingest, the sharing boundary, the Brent check, and
// the host-side launchers; this unit instantiates the engine with independent
// coins per pair.

#include "cse_engine.cuh"

namespace cse {

// ---------------------------------------------------------------------------
// Ingest: int8 rows -> column bitsets; initial candidate list.
// One warp per matrix.
// ---------------------------------------------------------------------------
__global__ void ingest_kernel(const int8_t* __restrict__ raw, int rows, int nx, int W,
                              uint2* __restrict__ pn0, uint32_t* __restrict__ cand0,
                              int32_t* __restrict__ meta0, int mmax) {
    const int lane = threadIdx.x & 31;
    // columns
    for (int x = lane; x < nx * W; x += 32) {
        const int v = x / W, w = x % W;
        uint32_t p = 0, n = 0;
        for (int b = 0; b < 32; b++) {
            const int r = w * 32 + b;
            if (r >= rows) break;
            const int8_t a = raw[(size_t)r * nx + v];
            p |= (uint32_t)(a == 1) << b;
            n |= (uint32_t)(a == -1) << b;
        }
        pn0[x] = make_uint2(p, n);
    }
    // naive additions: sum over rows of (nnz - 1)
    int part = 0;
    for (int r = lane; r < rows; r += 32) {
        int nnz = 0;
        for (int v = 0; v < nx; v++) nnz += raw[(size_t)r * nx + v] != 0;
        part += nnz - 1;
    }
    const int naive = __reduce_add_sync(FULL_MASK, part);
    __syncwarp();
    // all pairs (u, v), u < v, in canonical order: v ascending, then u, '+' first
    const uint32_t lt = lanemask_lt();
    int m = 0;
    for (int v = 1; v < nx; v++) {
        for (int base = 0; base < v; base += 32) {
            const int u = base + lane;
            int cp = 0, cm = 0;
            if (u < v) {
                for (int w = 0; w < W; w++) {
                    const uint2 A = pn0[u * W + w], B = pn0[v * W + w];
                    const uint32_t bt = (A.x | A.y) & (B.x | B.y);
                    const int ng = __popc((A.x ^ B.x) & bt);
                    cm += ng;
                    cp += __popc(bt) - ng;
                }
            }
            const bool ep = cp >= 2, em = cm >= 2;
            const uint32_t bp = __ballot_sync(FULL_MASK, ep), bm = __ballot_sync(FULL_MASK, em);
            int pos = m + __popc(bp & lt) + __popc(bm & lt);
            if (ep && pos < mmax) cand0[pos] = make_cand(u, v, 0, cp);
            if (ep) pos++;
            if (em && pos < mmax) cand0[pos] = make_cand(u, v, 1, cm);
            m += __popc(bp) + __popc(bm);
        }
    }
    if (lane == 0) {
        meta0[0] = naive;
        meta0[1] = m;
    }
}

// Sharing boundary (Section 3.5.2) and result publication.  One CTA per
// search, one warp per matrix.  In iteration mode every round is a boundary,
// followed by the convergence test on the sum of the matrices' best costs
// (Section 4: unchanged for `patience` iterations ends the search).
__device__ void share_one(const DevMat* __restrict__ mats, const DevSearch* __restrict__ S);

__global__ void share_kernel(const DevMat* __restrict__ mats, const DevSearch* __restrict__ searches,
                             int* __restrict__ work, int n_work) {
    // the round kernels' work counters, for the next round
    if (blockIdx.x == 0 && (int)threadIdx.x < n_work) work[threadIdx.x] = 0;
    share_one(mats, &searches[blockIdx.x]);
}

// The sharing boundary of one search, by the threads of one CTA (one warp
// per matrix at a time).
__device__ void share_one(const DevMat* __restrict__ mats, const DevSearch* __restrict__ S) {
    const bool iter_mode = S->interval == 0;
    const int c0 = *S->clock;
    if (c0 >= S->budget || (iter_mode && S->conv[1])) return;
    const int c1 = iter_mode ? c0 + 1 : min(c0 + S->interval, S->budget);
    const bool boundary = iter_mode || c1 % S->interval == 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __shared__ int s_total, s_final;
    if (threadIdx.x == 0) s_total = 0;
    __syncthreads();
    for (int k = warp; k < S->n_mats; k += nw) {
        const DevMat* M = &mats[S->mat_pos[k]];
        const unsigned long long key = *M->round_min;
        if (key == ~0ull) continue;  // no process reported (cannot happen while the search runs)
        const int cost = (int)(key >> 32), win = (int)(key & 0xFFFFFFFFu) - M->proc_offset;
        const bool local = win >= 0 && win < M->n_proc;  // else another rank's (a shard)
        if (boundary && cost < M->snap_meta[0]) {
            const int len = local ? (int)M->state[(size_t)win * M->state_words + H_BEST_LEN] : *M->ext_len;
            const int32_t* src = local ? M->best_list + (size_t)win * M->cap : M->ext_list;
            for (int x = lane; x < len; x += 32) M->snap[x] = src[x];
            __syncwarp();
            if (lane == 0) {
                M->snap_meta[0] = cost;
                M->snap_meta[1] = len;
            }
        }
        if (lane == 0) {
            atomicAdd(&s_total, cost);
            // the best-Cost curve: one point per round (per iteration)
            const int r = iter_mode ? c0 : c0 / S->interval;
            if (r < kCurvePoints) M->curve[r] = cost;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bool fin = c1 == S->budget;
        if (iter_mode) {
            int32_t* cv = S->conv;
            if (s_total < cv[2]) {
                cv[2] = s_total;
                cv[0] = 0;
            } else {
                cv[0]++;
            }
            // converged: set only by the patience rule, so that a search
            // that merely used up its iterations can be resumed
            if (S->patience > 0 && cv[0] >= S->patience) {
                fin = true;
                cv[1] = 1;
            }
            cv[3] = c1;
        }
        s_final = fin ? 1 : 0;
    }
    __syncthreads();
    for (int k = warp; k < S->n_mats; k += nw) {
        const DevMat* M = &mats[S->mat_pos[k]];
        const unsigned long long key = *M->round_min;
        if (key == ~0ull) continue;
        if (s_final) {
            const int cost = (int)(key >> 32), win = (int)(key & 0xFFFFFFFFu) - M->proc_offset;
            const bool local = win >= 0 && win < M->n_proc;
            const int len = local ? (int)M->state[(size_t)win * M->state_words + H_BEST_LEN] : *M->ext_len;
            const int32_t* src = local ? M->best_list + (size_t)win * M->cap : M->ext_list;
            for (int x = lane; x < len; x += 32) M->result[x] = src[x];
            if (lane == 0) {
                M->result_meta[0] = cost;
                M->result_meta[1] = len;
            }
        }
        __syncwarp();
        if (lane == 0) *M->round_min = ~0ull;
    }
    __syncthreads();
    if (threadIdx.x == 0) *S->clock = c1;
}

// A bounded grid barrier for a cooperative launch (every CTA co-resident):
// the last CTA to arrive resets the count and bumps the generation; the
// others poll the generation at most max_spin times (a short sleep between
// polls).  A CTA that gives up, or that sees another one's time-out, writes
// 1 to *status and returns false; so does every later barrier, so that no
// CTA waits on one that has left.
__device__ bool grid_barrier(unsigned* bar, unsigned long long max_spin, int* status) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned* gen = bar + 1;
        volatile int* st = status;
        const unsigned g = *gen;
        __threadfence();
        if (*st != 0) {
            ok = 0;
        } else if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned long long n = 0;
            while (*gen == g) {
                if (*st != 0 || ++n > max_spin) {
                    atomicExch(status, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// A whole batch (Section 3.5: every search's rounds and sharing boundaries)
// in one persistent cooperative launch, for batches whose matrices all run
// on the shared-memory engine with at most 2 words per column: per round,
// every warp takes processes from the round's work counter (work[round]),
// dispatching on the matrix's word width; then a grid barrier, the sharing
// boundary of every search (CTA b takes searches b, b + grid, ...), and
// another barrier.  Each search keeps its own clock, so the results are
// those of the searches run alone.
__global__ void __launch_bounds__(128, CSE_MIN_BLOCKS)
    batch_kernel(const DevMat* __restrict__ mats, int n_mats, const DevSearch* __restrict__ searches,
                 int n_searches, int total_units, int rounds, int* __restrict__ work, unsigned* __restrict__ bar,
                 int* __restrict__ status, unsigned long long max_spin, const __grid_constant__ WarpLayout L) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int rd = 0; rd < rounds; rd++) {
        for (;;) {
            int unit = 0;
            if (lane == 0) unit = atomicAdd(&work[rd], 1);
            unit = __shfl_sync(FULL_MASK, unit, 0);
            if (unit >= total_units) break;
            int mi = 0;
            while (mi + 1 < n_mats && mats[mi + 1].unit_base <= unit) mi++;
            if (mats[mi].W == 1)
                run_unit<1, false, false>(mats, n_mats, searches, L, smem, warp, lane, unit);
            else
                run_unit<2, false, false>(mats, n_mats, searches, L, smem, warp, lane, unit);
            __syncwarp();
        }
        if (!grid_barrier(bar, max_spin, status)) return;
        for (int sidx = blockIdx.x; sidx < n_searches; sidx += gridDim.x) share_one(mats, &searches[sidx]);
        if (!grid_barrier(bar, max_spin, status)) return;
    }
}

cudaError_t launch_batch_persistent(const DevMat* mats, int n_mats, const DevSearch* searches, int n_searches,
                                    int total_units, int rounds, int* work, unsigned* bar, int* status,
                                    unsigned long long max_spin, const WarpLayout& L, int ppc, cudaStream_t stream,
                                    bool prepare_only) {
    const size_t smem = (size_t)L.per_warp * ppc;
    if (prepare_only) return raise_max_dynamic_smem((const void*)batch_kernel, (int)smem);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, 32 * ppc, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(sms * per_sm));
    cfg.blockDim = dim3((unsigned)(32 * ppc));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_kernel, mats, n_mats, searches, n_searches, total_units, rounds, work, bar,
                              status, max_spin, L);
}

// Brent equations (Section 3.1) of a scheme (m,n,p:r): one thread per index
// triple (a_ij, b_j'k, c_i'k'), grid-stride; counts the triples whose sum
// over the r products differs from [j = j'][i = i'][k = k'].  Consecutive
// threads take consecutive c, so the W reads coalesce and U, V broadcast.
__global__ void brent_kernel(const int8_t* __restrict__ U, const int8_t* __restrict__ V,
                             const int8_t* __restrict__ W, int m, int n, int p, int r, long long total,
                             unsigned long long* __restrict__ bad) {
    const int mn = m * n, np = n * p, mp = m * p;
    unsigned long long cnt = 0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t % mp);
        const long long ab = t / mp;
        const int b = (int)(ab % np), a = (int)(ab / np);
        int sum = 0;
        for (int l = 0; l < r; l++)
            sum += (int)U[(size_t)l * mn + a] * (int)V[(size_t)l * np + b] * (int)W[(size_t)l * mp + c];
        const int i = a / n, j = a % n, j2 = b / p, k = b % p, i2 = c / p, k2 = c % p;
        const int want = (j == j2 && i == i2 && k == k2) ? 1 : 0;
        cnt += sum != want;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(FULL_MASK, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(bad, cnt);
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------
static int align16(int x) { return (x + 15) & ~15; }

WarpLayout make_layout(int W, int cap, int mmax, bool planes) {
    WarpLayout L{};
    int o = 0;
    L.off_cold = o;
    o = align16(o + (int)sizeof(Cold));
    L.off_pn = o;
    o = align16(o + cap * W * 8);
    L.off_cand = o;
    o = align16(o + mmax * 4);
    L.off_f = o;
    o = align16(o + cap * 4);
    L.off_aw = o;
    o = align16(o + (planes ? 0 : 2 * mmax));
    L.off_poslo = o;
    o = align16(o + mmax * 2);
    L.off_hs = o;
    o = align16(o + cap * 2);
    L.off_he = o;
    o = align16(o + cap * 2);
    L.off_base = o;
    o = align16(o + cap * 2);
    L.off_lc = o;
    o = align16(o + cap * 2);
    if (planes) {
        // sum over v of ceil(|A_v| / 64) <= (2 mmax + 63 cap) / 64; 8 planes
        // cover any weight c - 1 <= 255
        const int max_blocks = (2 * mmax + 63 * cap) / 64 + 1;
        L.off_pb = o;
        o = align16(o + cap * 2);
        L.off_g = o;
        o = align16(o + cap * 4);
        L.off_pln = o;
        o = align16(o + max_blocks * 8 * 8);
        L.off_rec = o;
        o = align16(o + cap * (int)sizeof(VarRec));
    }
    L.per_warp = o;
    return L;
}

int state_words(int W, int cap, int mmax) {
    const int w = H_WORDS + 2 * cap * W + mmax + cap;
    return (w + 3) & ~3;
}

int state_words_gm(const WarpLayout& L) { return H_WORDS + ((L.per_warp / 4 + 3) & ~3); }

cudaError_t launch_ingest(const int8_t* raw, int rows, int nx, int W, uint2* pn0, uint32_t* cand0,
                          int32_t* meta0, int mmax, cudaStream_t stream) {
    ingest_kernel<<<1, 32, 0, stream>>>(raw, rows, nx, W, pn0, cand0, meta0, mmax);
    return cudaGetLastError();
}

cudaError_t launch_round(int W, bool gm, bool gs, const DevMat* mats, int n_mats, const DevSearch* searches,
                         int total_units, int* work, const WarpLayout& L, int ppc, cudaStream_t stream) {
    return gs ? launch_round_gs(W, gm, mats, n_mats, searches, total_units, work, L, ppc, stream, false)
              : launch_round_variant<false>(W, gm, mats, n_mats, searches, total_units, work, L, ppc, stream, false);
}

cudaError_t launch_round_list(int W, const DevMat* mats, int n_mats, const DevSearch* searches, int max_units,
                              const int* unit_list, const int* unit_count, int* work, int ppc, cudaStream_t stream) {
    const WarpLayout none{};
    switch (W) {
#define CSE_LIST_CASE(w)                                                                                       \
    case w:                                                                                                    \
        return launch_round_w<w, true, false>(mats, n_mats, searches, max_units, work, none, ppc, stream, false, \
                                              unit_list, unit_count);
        CSE_LIST_CASE(1)
        CSE_LIST_CASE(2)
        CSE_LIST_CASE(3)
        CSE_LIST_CASE(4)
        CSE_LIST_CASE(5)
        CSE_LIST_CASE(6)
        CSE_LIST_CASE(7)
        CSE_LIST_CASE(8)
#undef CSE_LIST_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_round(int W, bool gm, bool gs, const WarpLayout& L, int ppc) {
    return gs ? launch_round_gs(W, gm, nullptr, 0, nullptr, 0, nullptr, L, ppc, nullptr, true)
              : launch_round_variant<false>(W, gm, nullptr, 0, nullptr, 0, nullptr, L, ppc, nullptr, true);
}

cudaError_t launch_share(const DevMat* mats, const DevSearch* searches, int n_searches, int* work, int n_work,
                         cudaStream_t stream) {
    if (n_work > 128) return cudaErrorInvalidValue;
    share_kernel<<<n_searches, 128, 0, stream>>>(mats, searches, work, n_work);
    return cudaGetLastError();
}

cudaError_t launch_brent(const int8_t* U, const int8_t* V, const int8_t* W, int m, int n, int p, int r,
                         unsigned long long* bad, cudaStream_t stream) {
    const long long total = (long long)m * n * n * p * m * p;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (total + 255) / 256;
    const int grid = (int)std::max(1LL, std::min(want, (long long)std::max(sms, 1) * 8));
    brent_kernel<<<grid, 256, 0, stream>>>(U, V, W, m, n, p, r, total, bad);
    return cudaGetLastError();
}

int max_smem_per_block() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    return v;
}

}  // namespace cse
