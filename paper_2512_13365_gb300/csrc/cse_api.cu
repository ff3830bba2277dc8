// C ABI of the GB300 CSE library (include/cse.h): validation, device buffers,
// launch sequencing.  The method's arithmetic runs in cse_kernels.cu.

#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "cse.h"
#include "cse_internal.h"

using namespace cse;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define CUDA_TRY(x)                                                                    \
    do {                                                                               \
        cudaError_t e_ = (x);                                                          \
        if (e_ != cudaSuccess)                                                         \
            return fail(CSE_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Bump allocator over one device block.
struct Carve {
    size_t off = 0;
    size_t take(size_t bytes) {
        size_t o = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return o;
    }
};

uint64_t fnv(uint64_t h, uint32_t w) { return (h ^ w) * 0x100000001B3ull; }

void set_pool_threshold_once() {
    static bool done = false;
    if (done) return;
    done = true;
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
}

}  // namespace

struct cse_scheme {
    int n_mats = 0;
    int rows[CSE_MAX_MATS], cols[CSE_MAX_MATS], W[CSE_MAX_MATS], mmax[CSE_MAX_MATS];
    int8_t* d_raw[CSE_MAX_MATS];
    uint2* d_pn0[CSE_MAX_MATS];
    uint32_t* d_cand0[CSE_MAX_MATS];
    int32_t* d_meta0[CSE_MAX_MATS];
    void* d_block = nullptr;
};

// One launch: the device allocation, events and (optionally) the CUDA graph
// shared by the results of the searches it ran.
struct Batch {
    int refs = 0;
    int rounds = 0;
    cudaStream_t stream = nullptr;
    void* d_block = nullptr;
    std::vector<DevMat> hmats;       // device order
    std::vector<DevSearch> hsearch;
    cudaEvent_t ev_begin = nullptr, ev_end = nullptr;
    std::vector<cudaEvent_t> ev_round;   // begin/end of the round kernels of each round
    std::vector<cudaEvent_t> ev_fork;    // fork/join events of concurrent groups
    std::vector<cudaStream_t> aux;       // streams of concurrent groups
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap_stream = nullptr;   // stream the graph is captured on
    int launches_per_round = 0;

    void release() {
        if (ev_end) cudaEventSynchronize(ev_end);
        if (d_block) cudaFreeAsync(d_block, stream);
        for (auto ev : ev_round) cudaEventDestroy(ev);
        for (auto ev : ev_fork) cudaEventDestroy(ev);
        for (auto st : aux) cudaStreamDestroy(st);
        if (ev_begin) cudaEventDestroy(ev_begin);
        if (ev_end) cudaEventDestroy(ev_end);
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
};

struct cse_result {
    Batch* batch = nullptr;
    int search = 0;                   // index of the search in its batch
    int n_mats = 0, n_proc = 0, cap = 0;
    int64_t budget = 0;
    std::vector<int> pos_of_mat;      // matrix index -> position in batch->hmats
};

extern "C" {

const char* cse_last_error(void) { return g_err.c_str(); }

void cse_opts_default(cse_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->share_interval = 32;
    o->share_permille = 400;
    o->col_cap = 128;
}

int cse_scheme_load(const int8_t* const* mats, const int32_t* rows, const int32_t* cols,
                    int32_t n_mats, cse_scheme** out) {
    if (!out) return fail(CSE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!mats || !rows || !cols) return fail(CSE_EINVAL, "NULL input array");
    if (n_mats < 1 || n_mats > CSE_MAX_MATS) return fail(CSE_EINVAL, "n_mats must be in [1, 16]");
    cse_scheme* s = new (std::nothrow) cse_scheme();
    if (!s) return fail(CSE_ENOMEM, "host allocation");
    s->n_mats = n_mats;
    Carve cv;
    size_t off_raw[CSE_MAX_MATS], off_pn[CSE_MAX_MATS], off_cand[CSE_MAX_MATS], off_meta[CSE_MAX_MATS];
    for (int k = 0; k < n_mats; k++) {
        const int R = rows[k], C = cols[k];
        if (!mats[k] || R < 1 || R > CSE_MAX_ROWS || C < 1 || C >= CSE_MAX_COLS) {
            delete s;
            return fail(CSE_EINVAL, "matrix " + std::to_string(k) + ": need 1 <= rows <= 256, 1 <= cols < 512");
        }
        long long occ = 0;
        for (int r = 0; r < R; r++) {
            int nnz = 0;
            for (int v = 0; v < C; v++) {
                const int8_t a = mats[k][(size_t)r * C + v];
                if (a < -1 || a > 1) {
                    delete s;
                    return fail(CSE_EINVAL, "matrix " + std::to_string(k) + ": entry not in {-1,0,1}");
                }
                nnz += a != 0;
            }
            if (nnz == 0) {
                delete s;
                return fail(CSE_EINVAL, "matrix " + std::to_string(k) + ": row " + std::to_string(r) +
                                            " has no nonzero (A_naive would count -1)");
            }
            occ += (long long)nnz * (nnz - 1) / 2;
        }
        s->rows[k] = R;
        s->cols[k] = C;
        s->W[k] = (R + 31) / 32;
        // candidates have c >= 2 and row nnz never grows, so m <= occ / 2
        s->mmax[k] = (int)std::max(1LL, std::min(occ / 2, 32767LL));
        off_raw[k] = cv.take((size_t)R * C);
        off_pn[k] = cv.take((size_t)C * s->W[k] * sizeof(uint2));
        off_cand[k] = cv.take((size_t)s->mmax[k] * 4);
        off_meta[k] = cv.take(16);
    }
    if (cudaMalloc(&s->d_block, cv.off) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return fail(CSE_ECUDA, "cudaMalloc of the scheme failed (no CUDA device?)");
    }
    char* b = (char*)s->d_block;
    for (int k = 0; k < n_mats; k++) {
        s->d_raw[k] = (int8_t*)(b + off_raw[k]);
        s->d_pn0[k] = (uint2*)(b + off_pn[k]);
        s->d_cand0[k] = (uint32_t*)(b + off_cand[k]);
        s->d_meta0[k] = (int32_t*)(b + off_meta[k]);
        cudaError_t e = cudaMemcpy(s->d_raw[k], mats[k], (size_t)s->rows[k] * s->cols[k], cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = launch_ingest(s->d_raw[k], s->rows[k], s->cols[k], s->W[k], s->d_pn0[k], s->d_cand0[k],
                              s->d_meta0[k], s->mmax[k], 0);
        if (e != cudaSuccess) {
            cudaFree(s->d_block);
            delete s;
            return fail(CSE_ECUDA, std::string("scheme upload: ") + cudaGetErrorString(e));
        }
    }
    cudaError_t e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) {
        cudaFree(s->d_block);
        delete s;
        return fail(CSE_ECUDA, std::string("scheme ingest: ") + cudaGetErrorString(e));
    }
    *out = s;
    return CSE_OK;
}

int cse_scheme_load_uvw(int32_t m, int32_t n, int32_t p, int32_t r, const int8_t* U, const int8_t* V,
                        const int8_t* W, cse_scheme** out) {
    if (m < 1 || n < 1 || p < 1 || r < 1 || !U || !V || !W) return fail(CSE_EINVAL, "bad scheme dimensions");
    std::vector<int8_t> wt((size_t)m * p * r);
    for (int l = 0; l < r; l++)
        for (int c = 0; c < m * p; c++) wt[(size_t)c * r + l] = W[(size_t)l * m * p + c];
    const int8_t* mats[3] = {U, V, wt.data()};
    const int32_t rows[3] = {r, r, m * p};
    const int32_t cols[3] = {m * n, n * p, r};
    return cse_scheme_load(mats, rows, cols, 3, out);
}

int cse_scheme_shape(const cse_scheme* s, int32_t mat, int32_t* rows, int32_t* cols) {
    if (!s || mat < 0 || mat >= s->n_mats) return fail(CSE_EINVAL, "bad scheme or matrix index");
    if (rows) *rows = s->rows[mat];
    if (cols) *cols = s->cols[mat];
    return CSE_OK;
}

void cse_scheme_free(cse_scheme* s) {
    if (!s) return;
    if (s->d_block) cudaFree(s->d_block);  // cudaFree waits for work using it
    delete s;
}

static int check_mix(const cse_strategy_mix* mix, uint64_t* wsum_out) {
    if (!mix) return fail(CSE_EINVAL, "NULL strategy mix");
    if (mix->w_gp != 0) return fail(CSE_EINVAL, "Greedy-Potential (w_gp) is not implemented; set it to 0");
    const uint64_t wsum = (uint64_t)mix->w_gi + mix->w_ga + mix->w_gr + mix->w_wr + mix->w_mix + mix->w_g;
    if (wsum == 0 || wsum > 0xFFFFFFFFull) return fail(CSE_EINVAL, "strategy weights: sum must be in [1, 2^32)");
    *wsum_out = wsum;
    return CSE_OK;
}

// Builds and enqueues n independent searches as one launch sequence: per
// round, one round kernel per class of equal words-per-column (and memory
// path), then one share kernel over all searches.  Each search keeps its own
// step clock, so its result does not depend on the others.
static int run_batch(int n, const cse_scheme* const* schemes, const cse_strategy_mix* mixes,
                     const int32_t* n_procs, const uint64_t* seeds, const int64_t* budgets,
                     const cse_opts* opts_in, void* cuda_stream, cse_result** outs) {
    if (!outs) return fail(CSE_EINVAL, "out is NULL");
    if (n < 1 || !schemes || !mixes || !n_procs || !seeds || !budgets)
        return fail(CSE_EINVAL, "n_searches must be >= 1 with non-NULL arrays");
    for (int i = 0; i < n; i++) outs[i] = nullptr;
    cse_opts opts;
    if (opts_in)
        opts = *opts_in;
    else
        cse_opts_default(&opts);
    if (opts.share_interval < 1) return fail(CSE_EINVAL, "share_interval must be >= 1");
    if (opts.share_permille > 1000) return fail(CSE_EINVAL, "share_permille must be <= 1000");
    if (opts.patience_rounds != 0 || (opts.flags & ~(uint32_t)CSE_FLAG_GRAPH) != 0)
        return fail(CSE_EINVAL, "reserved option fields must be 0");
    const int cap = (int)opts.col_cap;
    if (cap > CSE_MAX_COLS) return fail(CSE_EINVAL, "col_cap must be <= 512");
    const int ppc_req = (int)opts.procs_per_cta;
    if (ppc_req < 0 || ppc_req > 4) return fail(CSE_EINVAL, "procs_per_cta must be in [0, 4]");
    std::vector<uint64_t> wsums(n);
    int64_t max_budget = 0, total_mats = 0;
    for (int i = 0; i < n; i++) {
        const cse_scheme* s = schemes[i];
        if (!s) return fail(CSE_EINVAL, "NULL scheme");
        int rc = check_mix(&mixes[i], &wsums[i]);
        if (rc) return rc;
        if (n_procs[i] < 1 || n_procs[i] > (1 << 20)) return fail(CSE_EINVAL, "n_processes must be in [1, 2^20]");
        if (budgets[i] < 0 || budgets[i] >= INT32_MAX) return fail(CSE_EINVAL, "step_budget must be in [0, 2^31)");
        for (int k = 0; k < s->n_mats; k++)
            if (s->cols[k] >= cap) return fail(CSE_EINVAL, "col_cap must exceed every matrix's column count");
        max_budget = std::max(max_budget, budgets[i]);
        total_mats += s->n_mats;
    }
    const int smem_max = max_smem_per_block();
    if (smem_max <= 0) return fail(CSE_ECUDA, "no CUDA device");
    set_pool_threshold_once();
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    const bool use_graph = (opts.flags & CSE_FLAG_GRAPH) != 0;

    // every matrix of every search, ordered by words per column
    struct Ref { int search, mat, W, mmax, n_proc; };
    std::vector<Ref> refs;
    for (int i = 0; i < n; i++)
        for (int k = 0; k < schemes[i]->n_mats; k++)
            refs.push_back({i, k, schemes[i]->W[k], schemes[i]->mmax[k], n_procs[i]});
    std::stable_sort(refs.begin(), refs.end(), [](const Ref& x, const Ref& y) { return x.W < y.W; });
    const int nm = (int)refs.size();

    // launch groups: equal W, one round kernel launch each; a group whose
    // per-process arrays are too large for a shared-memory slice runs on HBM
    struct Group { int W, begin, count, units, mmax; bool gm; WarpLayout L; int ppc; };
    std::vector<Group> groups;
    std::vector<int> group_of(nm);
    for (int q = 0; q < nm; q++) {
        if (groups.empty() || groups.back().W != refs[q].W) groups.push_back({refs[q].W, q, 0, 0, 0, false, {}, 0});
        Group& g = groups.back();
        g.count++;
        g.units += refs[q].n_proc;
        g.mmax = std::max(g.mmax, refs[q].mmax);
        group_of[q] = (int)groups.size() - 1;
    }
    for (Group& g : groups) {
        g.L = make_layout(g.W, cap, g.mmax);
        g.gm = g.L.per_warp > kSmemPerWarpLimit;
        g.ppc = ppc_req ? ppc_req : 4;
        if (!g.gm)
            while (g.ppc > 1 && (long long)g.L.per_warp * g.ppc > smem_max) g.ppc--;
        cudaError_t e = prepare_round(g.W, g.gm, g.L, g.ppc);
        if (e != cudaSuccess) return fail(CSE_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
    }

    Carve cv;
    struct Offs { size_t state, best, snap, snapm, rmin, res, resm, cnt; int sw; };
    std::vector<Offs> of(nm);
    for (int q = 0; q < nm; q++) {
        const Ref& rf = refs[q];
        const Group& g = groups[group_of[q]];
        Offs& o = of[q];
        o.sw = g.gm ? state_words_gm(g.L) : state_words(rf.W, cap, rf.mmax);
        o.state = cv.take((size_t)rf.n_proc * o.sw * 4);
        o.best = cv.take((size_t)rf.n_proc * cap * 4);
        o.snap = cv.take((size_t)cap * 4);
        o.snapm = cv.take(8);
        o.rmin = cv.take(8);
        o.res = cv.take((size_t)cap * 4);
        o.resm = cv.take(8);
        o.cnt = cv.take(16);
    }
    const size_t off_clock = cv.take(4 * (size_t)n), off_status = cv.take(4 * (size_t)n);
    const size_t off_pos = cv.take(4 * (size_t)nm);
    const size_t off_mats = cv.take(sizeof(DevMat) * nm), off_search = cv.take(sizeof(DevSearch) * n);

    Batch* B = new (std::nothrow) Batch();
    if (!B) return fail(CSE_ENOMEM, "host allocation");
    B->stream = stream;
    B->rounds = 0;
    for (int i = 0; i < n; i++)
        B->rounds = std::max(B->rounds, (int)((budgets[i] + opts.share_interval - 1) / opts.share_interval));
    cudaError_t e = cudaMallocAsync(&B->d_block, cv.off, stream);
    if (e != cudaSuccess) {
        B->d_block = nullptr;
        delete B;
        return fail(e == cudaErrorMemoryAllocation ? CSE_ENOMEM : CSE_ECUDA,
                    std::string("device allocation: ") + cudaGetErrorString(e));
    }
    char* b = (char*)B->d_block;
    auto bail = [&](cudaError_t err, const char* what) {
        cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
        if (B->cap_stream && cudaStreamIsCapturing(B->cap_stream, &cst) == cudaSuccess &&
            cst != cudaStreamCaptureStatusNone) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(B->cap_stream, &g);
            if (g) cudaGraphDestroy(g);
        }
        B->ev_end = nullptr;
        B->release();
        delete B;
        return fail(CSE_ECUDA, std::string(what) + ": " + cudaGetErrorString(err));
    };

    // per-search parameters; positions of each search's matrices
    std::vector<int32_t> pos((size_t)nm);
    std::vector<int> first_pos(n, 0), count(n, 0);
    {
        std::vector<std::vector<int>> by_search(n);
        for (int q = 0; q < nm; q++) by_search[refs[q].search].push_back(q);
        int o = 0;
        for (int i = 0; i < n; i++) {
            first_pos[i] = o;
            count[i] = (int)by_search[i].size();
            for (int q : by_search[i]) pos[o++] = q;
        }
    }
    B->hsearch.resize(n);
    for (int i = 0; i < n; i++) {
        DevSearch& S = B->hsearch[i];
        const cse_strategy_mix* mix = &mixes[i];
        S.seed = seeds[i];
        S.w[ST_GI] = mix->w_gi;
        S.w[ST_GA] = mix->w_ga;
        S.w[ST_GR] = mix->w_gr;
        S.w[ST_WR] = mix->w_wr;
        S.w[ST_MIX] = mix->w_mix;
        S.w[ST_G] = mix->w_g;
        S.wsum = (uint32_t)wsums[i];
        S.budget = (int32_t)budgets[i];
        S.interval = (int32_t)opts.share_interval;
        S.share_thr = ((uint64_t)opts.share_permille << 32) / 1000u;
        S.clock = (int32_t*)(b + off_clock) + i;
        S.status = (int32_t*)(b + off_status) + i;
        S.mat_pos = (const int32_t*)(b + off_pos) + first_pos[i];
        S.n_mats = count[i];
    }
    B->hmats.resize(nm);
    for (int q = 0; q < nm; q++) {
        const Ref& rf = refs[q];
        const cse_scheme* s = schemes[rf.search];
        const int k = rf.mat;
        const Group& g = groups[group_of[q]];
        DevMat& M = B->hmats[q];
        M.pn0 = s->d_pn0[k];
        M.cand0 = s->d_cand0[k];
        M.meta0 = s->d_meta0[k];
        M.rows = s->rows[k];
        M.nx = s->cols[k];
        M.W = s->W[k];
        M.cap = cap;
        M.mmax = s->mmax[k];
        M.mat_index = k;
        M.n_proc = rf.n_proc;
        M.search = rf.search;
        M.unit_base = 0;
        M.state_words = of[q].sw;
        M.state = (uint32_t*)(b + of[q].state);
        M.best_list = (int32_t*)(b + of[q].best);
        M.snap = (int32_t*)(b + of[q].snap);
        M.snap_meta = (int32_t*)(b + of[q].snapm);
        M.round_min = (unsigned long long*)(b + of[q].rmin);
        M.result = (int32_t*)(b + of[q].res);
        M.result_meta = (int32_t*)(b + of[q].resm);
        M.counters = (unsigned long long*)(b + of[q].cnt);
        (void)g;
    }
    for (const Group& g : groups) {  // unit_base is relative to the group's launch
        int u = 0;
        for (int q = g.begin; q < g.begin + g.count; q++) {
            B->hmats[q].unit_base = u;
            u += refs[q].n_proc;
        }
    }
    DevMat* d_mats = (DevMat*)(b + off_mats);
    DevSearch* d_search = (DevSearch*)(b + off_search);
    e = cudaMemcpyAsync(d_mats, B->hmats.data(), sizeof(DevMat) * nm, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_search, B->hsearch.data(), sizeof(DevSearch) * n, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + off_pos, pos.data(), 4 * (size_t)nm, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return bail(e, "parameter upload");
    if ((e = cudaEventCreate(&B->ev_begin)) != cudaSuccess) return bail(e, "event");
    if ((e = cudaEventCreate(&B->ev_end)) != cudaSuccess) return bail(e, "event");
    B->ev_round.resize(2 * (size_t)B->rounds);
    for (auto& ev : B->ev_round)
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return bail(e, "event");
    const bool concurrent = use_graph && groups.size() > 1;
    if (concurrent) {
        B->aux.resize(groups.size());
        B->ev_fork.resize(groups.size() + 1);
        for (auto& st : B->aux)
            if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return bail(e, "stream");
        for (auto& ev : B->ev_fork)
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return bail(e, "event");
    }
    B->launches_per_round = (int)groups.size() + 1;

    // With CSE_FLAG_GRAPH the sequence is captured on a private stream (the
    // caller's may be the legacy default stream, which cannot be captured)
    // and the instantiated graph is launched once on the caller's stream.
    cudaStream_t ls = stream;
    if (use_graph) {
        if ((e = cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return bail(e, "stream");
        ls = B->cap_stream;
        if ((e = cudaStreamBeginCapture(ls, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return bail(e, "stream capture");
    }
    // timing events: inside a capture they must be external record nodes
    auto rec = [&](cudaEvent_t ev) {
        return use_graph ? cudaEventRecordWithFlags(ev, ls, cudaEventRecordExternal) : cudaEventRecord(ev, ls);
    };
    rec(B->ev_begin);
    if ((e = launch_init(d_mats, nm, d_search, n, ls)) != cudaSuccess) return bail(e, "init");
    for (int rd = 0; rd < B->rounds; rd++) {
        rec(B->ev_round[2 * rd]);
        if (concurrent) {  // the groups of a round are independent: parallel graph branches
            cudaEventRecord(B->ev_fork[0], ls);
            for (size_t gi = 0; gi < groups.size(); gi++) {
                const Group& g = groups[gi];
                cudaStreamWaitEvent(B->aux[gi], B->ev_fork[0], 0);
                e = launch_round(g.W, g.gm, d_mats + g.begin, g.count, d_search, g.units, g.L, g.ppc, B->aux[gi]);
                if (e != cudaSuccess) return bail(e, "round kernel");
                cudaEventRecord(B->ev_fork[gi + 1], B->aux[gi]);
                cudaStreamWaitEvent(ls, B->ev_fork[gi + 1], 0);
            }
        } else {
            for (const Group& g : groups) {
                e = launch_round(g.W, g.gm, d_mats + g.begin, g.count, d_search, g.units, g.L, g.ppc, ls);
                if (e != cudaSuccess) return bail(e, "round kernel");
            }
        }
        rec(B->ev_round[2 * rd + 1]);
        if ((e = launch_share(d_mats, d_search, n, ls)) != cudaSuccess) return bail(e, "share kernel");
    }
    if ((e = rec(B->ev_end)) != cudaSuccess) return bail(e, "event record");
    if (use_graph) {
        if ((e = cudaStreamEndCapture(ls, &B->graph)) != cudaSuccess) return bail(e, "end capture");
        if ((e = cudaGraphInstantiate(&B->gexec, B->graph, 0)) != cudaSuccess) return bail(e, "graph instantiate");
        if ((e = cudaGraphLaunch(B->gexec, stream)) != cudaSuccess) return bail(e, "graph launch");
    }

    for (int i = 0; i < n; i++) {
        cse_result* r = new (std::nothrow) cse_result();
        if (!r) {
            for (int j = 0; j < i; j++) {
                delete outs[j];
                outs[j] = nullptr;
            }
            B->release();
            delete B;
            return fail(CSE_ENOMEM, "host allocation");
        }
        r->batch = B;
        r->search = i;
        r->n_mats = schemes[i]->n_mats;
        r->n_proc = n_procs[i];
        r->cap = cap;
        r->budget = budgets[i];
        r->pos_of_mat.assign(r->n_mats, 0);
        for (int q = 0; q < nm; q++)
            if (refs[q].search == i) r->pos_of_mat[refs[q].mat] = q;
        B->refs++;
        outs[i] = r;
    }
    return CSE_OK;
}

int cse_search(const cse_scheme* s, const cse_strategy_mix* mix, int32_t n_proc, uint64_t seed,
               int64_t budget, const cse_opts* opts, void* cuda_stream, cse_result** out) {
    if (!out) return fail(CSE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!s || !mix) return fail(CSE_EINVAL, "NULL scheme or strategy mix");
    return run_batch(1, &s, mix, &n_proc, &seed, &budget, opts, cuda_stream, out);
}

int cse_search_batch(int32_t n_searches, const cse_scheme* const* schemes, const cse_strategy_mix* mixes,
                     const int32_t* n_processes, const uint64_t* seeds, const int64_t* step_budgets,
                     const cse_opts* opts, void* cuda_stream, cse_result** outs) {
    return run_batch(n_searches, schemes, mixes, n_processes, seeds, step_budgets, opts, cuda_stream, outs);
}

static int wait_result(const cse_result* r) {
    if (!r) return fail(CSE_EINVAL, "NULL result");
    CUDA_TRY(cudaEventSynchronize(r->batch->ev_end));
    int32_t status = 0;
    CUDA_TRY(cudaMemcpy(&status, r->batch->hsearch[r->search].status, 4, cudaMemcpyDeviceToHost));
    if (status != 0) return fail(CSE_ESTATE, "device consistency check failed (candidate list overflow)");
    return CSE_OK;
}

int cse_result_fetch(const cse_result* r, int32_t mat, int32_t* subst, int32_t cap_entries, int32_t* n_subst,
                     int64_t* additions, int64_t* total_additions) {
    int rc = wait_result(r);
    if (rc) return rc;
    if (mat < 0 || mat >= r->n_mats) return fail(CSE_EINVAL, "matrix index out of range");
    int64_t total = 0;
    int32_t meta[2] = {0, 0};
    for (int k = 0; k < r->n_mats; k++) {
        const DevMat& M = r->batch->hmats[r->pos_of_mat[k]];
        int32_t mk[2];
        CUDA_TRY(cudaMemcpy(mk, M.result_meta, 8, cudaMemcpyDeviceToHost));
        total += mk[0];
        if (k == mat) std::memcpy(meta, mk, 8);
    }
    const DevMat& M = r->batch->hmats[r->pos_of_mat[mat]];
    if (subst && cap_entries > 0) {
        const int n = std::min(cap_entries, meta[1]);
        if (n > 0) CUDA_TRY(cudaMemcpy(subst, M.result, (size_t)n * 4, cudaMemcpyDeviceToHost));
    }
    if (n_subst) *n_subst = meta[1];
    if (additions) *additions = meta[0];
    if (total_additions) *total_additions = total;
    return CSE_OK;
}

int cse_result_procs(const cse_result* r, int32_t mat, cse_proc_record* out) {
    int rc = wait_result(r);
    if (rc) return rc;
    if (mat < 0 || mat >= r->n_mats || !out) return fail(CSE_EINVAL, "bad matrix index or output");
    const DevMat& M = r->batch->hmats[r->pos_of_mat[mat]];
    if (r->budget == 0) {  // no step ran: every record is the input itself
        int32_t meta[2];
        CUDA_TRY(cudaMemcpy(meta, M.result_meta, 8, cudaMemcpyDeviceToHost));
        for (int p = 0; p < r->n_proc; p++) {
            out[p].best_cost = meta[0];
            out[p].best_len = 0;
            out[p].runs = 0;
            out[p].best_hash = kFnv0;
            out[p].traj_hash = kFnv0;
            out[p].ops = 0;
            out[p].substeps = 0;
        }
        return CSE_OK;
    }
    std::vector<uint32_t> hdr((size_t)r->n_proc * H_WORDS);
    CUDA_TRY(cudaMemcpy2D(hdr.data(), H_WORDS * 4, M.state, (size_t)M.state_words * 4, H_WORDS * 4, r->n_proc,
                          cudaMemcpyDeviceToHost));
    std::vector<int32_t> lists((size_t)r->n_proc * r->cap);
    CUDA_TRY(cudaMemcpy(lists.data(), M.best_list, lists.size() * 4, cudaMemcpyDeviceToHost));
    for (int p = 0; p < r->n_proc; p++) {
        const uint32_t* h = &hdr[(size_t)p * H_WORDS];
        cse_proc_record& o = out[p];
        o.best_cost = (int32_t)h[H_BEST_COST];
        o.best_len = (int32_t)h[H_BEST_LEN];
        o.runs = (int32_t)h[H_RUNS];
        uint64_t hh = kFnv0;
        for (int x = 0; x < o.best_len; x++) hh = fnv(hh, (uint32_t)lists[(size_t)p * r->cap + x]);
        o.best_hash = hh;
        o.traj_hash = (uint64_t)h[H_TRAJ_LO] | (uint64_t)h[H_TRAJ_HI] << 32;
        o.ops = (int64_t)((uint64_t)h[H_OPS_LO] | (uint64_t)h[H_OPS_HI] << 32);
        o.substeps = (int32_t)h[H_SUBSTEPS];
    }
    return CSE_OK;
}

int cse_result_counters(const cse_result* r, int64_t* process_steps, int64_t* substeps, int64_t* alg_ops) {
    int rc = wait_result(r);
    if (rc) return rc;
    uint64_t ops = 0, sub = 0;
    for (int k = 0; k < r->n_mats; k++) {
        const DevMat& M = r->batch->hmats[r->pos_of_mat[k]];
        unsigned long long c[2];
        CUDA_TRY(cudaMemcpy(c, M.counters, 16, cudaMemcpyDeviceToHost));
        ops += c[0];
        sub += c[1];
    }
    if (process_steps) *process_steps = (int64_t)r->n_mats * r->n_proc * r->budget;
    if (substeps) *substeps = (int64_t)sub;
    if (alg_ops) *alg_ops = (int64_t)ops;
    return CSE_OK;
}

int cse_result_timing(const cse_result* r, float* round_ms, float* total_ms, int32_t* n_rounds) {
    int rc = wait_result(r);
    if (rc) return rc;
    const Batch* B = r->batch;
    float sum = 0.f, tot = 0.f;
    for (int rd = 0; rd < B->rounds; rd++) {
        float x = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&x, B->ev_round[2 * rd], B->ev_round[2 * rd + 1]));
        sum += x;
    }
    CUDA_TRY(cudaEventElapsedTime(&tot, B->ev_begin, B->ev_end));
    if (round_ms) *round_ms = sum;
    if (total_ms) *total_ms = tot;
    if (n_rounds) *n_rounds = B->rounds;
    return CSE_OK;
}

int cse_result_launches(const cse_result* r, int32_t* kernels, int32_t* searches_in_launch) {
    if (!r) return fail(CSE_EINVAL, "NULL result");
    const Batch* B = r->batch;
    if (kernels) *kernels = 1 + B->rounds * B->launches_per_round;
    if (searches_in_launch) *searches_in_launch = (int32_t)B->hsearch.size();
    return CSE_OK;
}

void cse_result_free(cse_result* r) {
    if (!r) return;
    Batch* B = r->batch;
    delete r;
    if (B && --B->refs == 0) {
        B->release();
        delete B;
    }
}

}  // extern "C"
