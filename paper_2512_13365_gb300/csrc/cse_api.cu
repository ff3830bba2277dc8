// C ABI of the GB300 CSE library (include/cse.h): validation, device buffers,
// launch sequencing.  The method's arithmetic runs in cse_kernels.cu.

#include <algorithm>
#include <climits>
#include <cstdio>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

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

// NVTX range over a host-side span (enqueueing a search, a served round, a
// result fetch), for timeline tools; free when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

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

// Iteration mode: rounds enqueued between two reads of the convergence state.
constexpr int kIterationChunk = 4;

// Keeps freed search memory in the current device's default pool (no
// release threshold), once per device; callers may be on any thread.
void set_pool_threshold_once() {
    static std::mutex mu;
    static std::set<int> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lk(mu);
    if (!done.insert(dev).second) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
}

// Launch-parameter cache filled by cse_autotune: processes per CTA for a
// class of matrices (words per column, memory path, column cap, bucket of the
// candidate bound).  Launch parameters never change results.
struct ClassKey {
    int W, gm, cap, mbucket;
    bool operator<(const ClassKey& o) const {
        if (W != o.W) return W < o.W;
        if (gm != o.gm) return gm < o.gm;
        if (cap != o.cap) return cap < o.cap;
        return mbucket < o.mbucket;
    }
};
std::mutex g_tune_mu;
constexpr size_t kServerMaxPending = 1 << 16;
constexpr int64_t kServerWaves = 64;  // default cap on active processes, in waves of resident warps
std::map<ClassKey, int> g_tuned_ppc;
// kernel words per column chosen by cse_autotune for a class (keyed by the
// matrices' own words per column)
std::map<ClassKey, int> g_tuned_words;

int mbucket(int mmax) {
    int b = 1;
    while (b < mmax) b <<= 1;
    return b;
}

// The next power of two of a word count: the wider kernel a matrix may run on.
int widen_words(int W) {
    int w = 1;
    while (w < W) w <<= 1;
    return w;
}

// How search_plan picks a matrix's kernel words per column.
enum WordsPolicy { kWordsDefault = 0, kWordsNatural = 1, kWordsWide = 2 };

// Trial-run controls used by the tuner.
struct Trial {
    int force_ppc = 0;                     // processes per CTA for every class
    int words = kWordsNatural;             // kernel words of every matrix
    std::vector<float>* group_ms = nullptr;   // out: round-kernel time per class
    std::vector<ClassKey>* keys = nullptr;    // out: class keys, same order
};

}  // namespace

int cse::set_error(int code, const std::string& msg) { return fail(code, msg); }

// ---------------------------------------------------------------------------
// One search on the device: its own allocation (process states, best lists,
// snapshot, round minimum, result, counters, clock, status) and the host
// copies of the per-matrix and per-search kernel parameters.
// ---------------------------------------------------------------------------
struct SearchDev {
    void* d_block = nullptr;
    cudaStream_t stream = nullptr;
    int n_mats = 0, n_proc = 0, cap = 0, rounds = 0, rounds_done = 0;
    int64_t budget = 0;
    size_t bytes = 0;
    std::vector<DevMat> mats;   // matrix k at index k
    std::vector<char> gm;       // matrix k runs on its HBM state region
    DevSearch search{};
    int rows[CSE_MAX_MATS], cols[CSE_MAX_MATS];
    int words[CSE_MAX_MATS];    // kernel words per column of matrix k (>= its own)
    // the parameters it was created with (checkpoints record them)
    cse_strategy_mix mix{};
    cse_opts opts{};
    uint64_t seed = 0;
    uint64_t input_hash = 0;  // the scheme's (a checkpoint records it)
};

// A checkpoint: this header, then the search's device block byte for byte.
struct CkptHeader {
    uint64_t magic;
    uint32_t version, interval, permille, cap, patience, flags;
    int32_t n_mats, n_proc;
    int32_t rows[CSE_MAX_MATS], cols[CSE_MAX_MATS];
    uint64_t seed;
    cse_strategy_mix mix;
    int64_t done;     // steps (iterations in iteration mode) already run
    uint64_t bytes;   // size of the device block that follows
    uint64_t input_hash;  // the scheme's cse_scheme::input_hash
    int32_t words[CSE_MAX_MATS];  // kernel words per column (the state layout)
};
constexpr uint64_t kCkptMagic = 0x3154504B43455343ull;  // "CSECKPT1" as little-endian bytes
constexpr uint32_t kCkptVersion = 3;

// Resume of one search from a checkpoint (run_batch).
struct Resume {
    const CkptHeader* hdr;
    const void* block;
};

// Kernel parameters of one launch over a set of searches: matrices grouped
// into classes of equal words per column and memory path (one round kernel
// launch per class), then the share kernel over all searches.
struct LaunchSet {
    struct Group {
        int W, begin, count, units, mmax, cap;
        bool gm;
        WarpLayout L;
        int ppc;
        ClassKey key;
        bool cta = false;        // large matrices on the process-per-CTA engine
        CtaLayout CL{};
        int* redo_list = nullptr;  // processes it hands back to the warp engine
    };
    std::vector<DevMat> mats;
    std::vector<DevSearch> searches;
    std::vector<int32_t> pos;
    std::vector<Group> groups;
    void* d_params = nullptr;
    DevMat* d_mats = nullptr;
    DevSearch* d_searches = nullptr;
    int* d_work = nullptr;  // three work counters per group (round kernel launches; see launch_round_cta)
    bool gs = false;  // the searches use shared Greedy-Intersections coins
};

// One static launch (cse_search / cse_search_batch): events, the parameter
// block, and (optionally) the CUDA graph shared by the results it produced.
struct Batch {
    int refs = 0;
    int rounds = 0;
    cudaStream_t stream = nullptr;
    LaunchSet ls;
    cudaEvent_t ev_begin = nullptr, ev_end = nullptr;
    std::vector<cudaEvent_t> ev_round;   // begin/end of the round kernels of each round
    std::vector<cudaEvent_t> ev_fork;    // fork/join events of concurrent groups
    std::vector<cudaEvent_t> ev_group;   // trial runs: begin/end of every class launch
    std::vector<cudaStream_t> aux;       // streams of concurrent groups
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap_stream = nullptr;   // stream the graph is captured on
    // CSE_FLAG_PERSISTENT: one cooperative kernel; its block holds the
    // per-round work counters, the barrier words, the barrier status and the
    // matrices in one unit space
    bool persistent = false;
    void* d_pers = nullptr;
    int* pers_status = nullptr;

    void release() {
        if (ev_end) cudaEventSynchronize(ev_end);
        if (ls.d_params) cudaFreeAsync(ls.d_params, stream);
        for (auto ev : ev_round) cudaEventDestroy(ev);
        for (auto ev : ev_fork) cudaEventDestroy(ev);
        for (auto ev : ev_group) cudaEventDestroy(ev);
        for (auto st : aux) cudaStreamDestroy(st);
        if (ev_begin) cudaEventDestroy(ev_begin);
        if (ev_end) cudaEventDestroy(ev_end);
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (d_pers) cudaFreeAsync(d_pers, stream);
    }
};

// A shard of a search split across ranks: its rounds are enqueued one at a
// time (cse_shard_round), and each sharing boundary is completed with the
// minima and winner lists of all shards (cse_shard_share).
struct ShardState {
    int rounds_done = 0;
    bool in_round = false;  // a round ran and its boundary is not completed yet
    int32_t total = 0, offset = 0;
};

struct cse_result {
    SearchDev* sd = nullptr;     // owned
    Batch* batch = nullptr;      // shared (static launches), or NULL (served)
    double latency_ms = 0.0;     // served requests: submit to completion
    ShardState* shard = nullptr; // owned; a shard of a search split across ranks
};

static void search_free(SearchDev* sd) {
    if (!sd) return;
    if (sd->d_block) cudaFreeAsync(sd->d_block, sd->stream);
    delete sd;
}

static int check_mix(const cse_strategy_mix* mix, uint64_t* wsum_out) {
    if (!mix) return fail(CSE_EINVAL, "NULL strategy mix");
    const uint64_t wsum = (uint64_t)mix->w_gi + mix->w_ga + mix->w_gr + mix->w_wr + mix->w_mix + mix->w_g + mix->w_gp;
    if (wsum == 0 || wsum > 0xFFFFFFFFull) return fail(CSE_EINVAL, "strategy weights: sum must be in [1, 2^32)");
    *wsum_out = wsum;
    return CSE_OK;
}

static int check_opts(const cse_opts* opts_in, cse_opts* opts) {
    if (opts_in)
        *opts = *opts_in;
    else
        cse_opts_default(opts);
    if (opts->share_permille > 1000) return fail(CSE_EINVAL, "share_permille must be <= 1000");
    if ((opts->flags & ~(uint32_t)(CSE_FLAG_GRAPH | CSE_FLAG_TRACE | CSE_FLAG_GI_SHARED_COINS |
                                   CSE_FLAG_WARP_ENGINE | CSE_FLAG_PERSISTENT | CSE_FLAG_WIDE_WORDS |
                                   CSE_FLAG_CTA_ENGINE)) != 0)
        return fail(CSE_EINVAL, "reserved option fields must be 0");
    if (opts->share_interval != 0 && opts->patience_rounds != 0)
        return fail(CSE_EINVAL, "patience_rounds applies to iteration mode (share_interval = 0) only");
    if (opts->share_interval == 0 && (opts->flags & CSE_FLAG_GRAPH))
        return fail(CSE_EINVAL, "iteration mode (share_interval = 0) cannot be captured in a graph: "
                                "its length depends on convergence");
    if (opts->col_cap > CSE_MAX_COLS) return fail(CSE_EINVAL, "col_cap must be <= 512");
    if (opts->procs_per_cta > 4) return fail(CSE_EINVAL, "procs_per_cta must be in [0, 4]");
    return CSE_OK;
}

// Validates one search and computes its layout and device footprint.
// Offsets of a search's device block: kOffsPerMat per matrix, then the
// search's clock, status and convergence state.
constexpr int kOffsPerMat = 11;

// Kernel words per column of matrix k: forced (a resumed checkpoint's), the
// matrix's own, the next power of two (CSE_FLAG_WIDE_WORDS or a wide trial),
// or the width cse_autotune cached for its class.  A wider shared-memory
// slice that would no longer fit its memory path keeps the matrix's own.
static int kernel_words(const cse_scheme* s, int k, bool gm, int cap, const cse_opts& opts, int policy,
                        const int32_t* forced) {
    const int own = s->W[k];
    if (forced) return forced[k];
    int w = own;
    if (policy == kWordsWide || (policy == kWordsDefault && (opts.flags & CSE_FLAG_WIDE_WORDS))) {
        w = widen_words(own);
    } else if (policy == kWordsDefault) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned_words.find(ClassKey{own, gm ? 1 : 0, cap, 0});
        if (it != g_tuned_words.end()) w = it->second;
    }
    if (w != own && !gm && make_layout(w, cap, s->mmax[k]).per_warp > kSmemPerWarpLimit) w = own;
    return w;
}

static int search_plan(const cse_scheme* s, const cse_strategy_mix* mix, int n_proc, int64_t budget,
                       const cse_opts& opts, SearchDev* sd, uint64_t* wsum, std::vector<size_t>* offs,
                       int words_policy = kWordsDefault, const int32_t* forced_words = nullptr) {
    if (!s) return fail(CSE_EINVAL, "NULL scheme");
    int rc = check_mix(mix, wsum);
    if (rc) return rc;
    if (n_proc < 1 || n_proc > (1 << 20)) return fail(CSE_EINVAL, "n_processes must be in [1, 2^20]");
    if (budget < 0 || budget >= INT32_MAX) return fail(CSE_EINVAL, "step_budget must be in [0, 2^31)");
    const int cap = (int)opts.col_cap;
    if (opts.share_interval == 0 && cap > 0 && budget > INT32_MAX / cap - 1)
        return fail(CSE_EINVAL, "iteration mode: max iterations x col_cap must stay below 2^31");
    for (int k = 0; k < s->n_mats; k++)
        if (s->cols[k] >= cap) return fail(CSE_EINVAL, "col_cap must exceed every matrix's column count");
    sd->n_mats = s->n_mats;
    sd->n_proc = n_proc;
    sd->cap = cap;
    sd->budget = budget;
    sd->rounds = opts.share_interval ? (int)((budget + opts.share_interval - 1) / opts.share_interval)
                                     : (int)budget;  // iteration mode: at most `budget` iterations
    sd->mats.assign(s->n_mats, DevMat{});
    sd->gm.assign(s->n_mats, 0);
    Carve cv;
    offs->clear();
    for (int k = 0; k < s->n_mats; k++) {
        sd->rows[k] = s->rows[k];
        sd->cols[k] = s->cols[k];
        const bool gm = make_layout(s->W[k], cap, s->mmax[k]).per_warp > kSmemPerWarpLimit;
        const int Wk = kernel_words(s, k, gm, cap, opts, words_policy, forced_words);
        if (Wk < s->W[k] || Wk > 8) return fail(CSE_EINVAL, "kernel words per column must be in [W, 8]");
        sd->gm[k] = gm;
        sd->words[k] = Wk;
        DevMat& M = sd->mats[k];
        M.gml = make_layout(Wk, cap, s->mmax[k], gm);
        M.state_words = gm ? state_words_gm(M.gml) : state_words(Wk, cap, s->mmax[k]);
        offs->push_back(cv.take((size_t)n_proc * M.state_words * 4));   // state
        offs->push_back(cv.take((size_t)n_proc * cap * 4));             // best lists
        offs->push_back(cv.take((size_t)cap * 4));                      // snapshot
        offs->push_back(cv.take(8));                                    // snapshot meta
        offs->push_back(cv.take(8));                                    // round minimum
        offs->push_back(cv.take((size_t)cap * 4));                      // result
        offs->push_back(cv.take(8));                                    // result meta
        offs->push_back(cv.take(64));                                   // counters
        offs->push_back(cv.take((size_t)kCurvePoints * 4));             // best-Cost curve
        offs->push_back(cv.take((size_t)(cap + 1) * 4));                // a shard's external winner list
        offs->push_back(cv.take(Wk != s->W[k] ? (size_t)s->cols[k] * Wk * 8 : 0));  // columns at Wk words
    }
    offs->push_back(cv.take(4));   // clock
    offs->push_back(cv.take(4));   // status
    offs->push_back(cv.take(16));  // convergence state (iteration mode)
    sd->bytes = cv.off;
    return CSE_OK;
}

// Allocates and initialises one search on `stream` (stream-ordered).
static int search_create(const cse_scheme* s, const cse_strategy_mix* mix, int n_proc, uint64_t seed,
                         int64_t budget, const cse_opts& opts, cudaStream_t stream, SearchDev** out,
                         int words_policy = kWordsDefault, const int32_t* forced_words = nullptr) {
    *out = nullptr;
    SearchDev* sd = new (std::nothrow) SearchDev();
    if (!sd) return fail(CSE_ENOMEM, "host allocation");
    uint64_t wsum = 0;
    std::vector<size_t> of;
    int rc = search_plan(s, mix, n_proc, budget, opts, sd, &wsum, &of, words_policy, forced_words);
    if (rc) {
        delete sd;
        return rc;
    }
    sd->stream = stream;
    sd->mix = *mix;
    sd->opts = opts;
    sd->seed = seed;
    sd->input_hash = s->input_hash;
    set_pool_threshold_once();
    cudaError_t e = cudaMallocAsync(&sd->d_block, sd->bytes, stream);
    if (e != cudaSuccess) {
        sd->d_block = nullptr;
        delete sd;
        return fail(e == cudaErrorMemoryAllocation ? CSE_ENOMEM : CSE_ECUDA,
                    std::string("device allocation: ") + cudaGetErrorString(e));
    }
    char* b = (char*)sd->d_block;
    DevSearch& S = sd->search;
    S.seed = seed;
    S.w[ST_GI] = mix->w_gi;
    S.w[ST_GA] = mix->w_ga;
    S.w[ST_GR] = mix->w_gr;
    S.w[ST_WR] = mix->w_wr;
    S.w[ST_MIX] = mix->w_mix;
    S.w[ST_G] = mix->w_g;
    S.w[ST_GP] = mix->w_gp;
    S.wsum = (uint32_t)wsum;
    S.budget = (int32_t)budget;
    S.interval = (int32_t)opts.share_interval;
    S.patience = (int32_t)opts.patience_rounds;
    S.share_thr = ((uint64_t)opts.share_permille << 32) / 1000u;
    S.clock = (int32_t*)(b + of[kOffsPerMat * s->n_mats]);
    S.status = (int32_t*)(b + of[kOffsPerMat * s->n_mats + 1]);
    S.conv = (int32_t*)(b + of[kOffsPerMat * s->n_mats + 2]);
    S.n_mats = s->n_mats;
    S.trace = (opts.flags & CSE_FLAG_TRACE) ? 1 : 0;
    S.gi_shared = (opts.flags & CSE_FLAG_GI_SHARED_COINS) ? 1 : 0;
    static const int32_t snap_init[2] = {INT_MAX, 0};
    for (int k = 0; k < s->n_mats; k++) {
        DevMat& M = sd->mats[k];
        const size_t* o = &of[kOffsPerMat * k];
        M.pn0 = s->d_pn0[k];
        M.cand0 = s->d_cand0[k];
        M.meta0 = s->d_meta0[k];
        M.rows = s->rows[k];
        M.nx = s->cols[k];
        M.W = sd->words[k];
        M.wn = s->W[k];
        M.cap = sd->cap;
        M.mmax = s->mmax[k];
        M.mat_index = k;
        M.n_proc = n_proc;
        M.state = (uint32_t*)(b + o[0]);
        M.best_list = (int32_t*)(b + o[1]);
        M.snap = (int32_t*)(b + o[2]);
        M.snap_meta = (int32_t*)(b + o[3]);
        M.round_min = (unsigned long long*)(b + o[4]);
        M.result = (int32_t*)(b + o[5]);
        M.result_meta = (int32_t*)(b + o[6]);
        M.counters = (unsigned long long*)(b + o[7]);
        M.curve = (int32_t*)(b + o[8]);
        M.proc_offset = 0;
        M.ext_list = (const int32_t*)(b + o[9]);
        M.ext_len = (const int32_t*)(b + o[9]) + sd->cap;
        if (M.W != M.wn) {  // a wider kernel: the columns again at M.W words, the extra row bits zero
            uint2* wide = (uint2*)(b + o[10]);
            M.pn0 = wide;
            if (e == cudaSuccess) e = cudaMemsetAsync(wide, 0, (size_t)M.nx * M.W * 8, stream);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(wide, (size_t)M.W * 8, s->d_pn0[k], (size_t)M.wn * 8, (size_t)M.wn * 8, M.nx,
                                      cudaMemcpyDeviceToDevice, stream);
        }
        // initial values: no round minimum, no snapshot, result = the input
        if (e == cudaSuccess) e = cudaMemsetAsync(M.round_min, 0xFF, 8, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(M.snap_meta, snap_init, 8, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(M.result_meta, M.meta0, 4, cudaMemcpyDeviceToDevice, stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(M.result_meta + 1, 0, 4, stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(M.counters, 0, 64, stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(M.curve, 0xFF, (size_t)kCurvePoints * 4, stream);
    }
    static const int32_t conv_init[4] = {0, 0, INT_MAX, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(S.conv, conv_init, 16, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(S.clock, 0, 4, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(S.status, 0, 4, stream);
    if (e != cudaSuccess) {
        search_free(sd);
        return fail(CSE_ECUDA, std::string("search init: ") + cudaGetErrorString(e));
    }
    *out = sd;
    return CSE_OK;
}

// Builds the launch parameters of a set of searches and uploads them.
static int build_launch(const std::vector<SearchDev*>& act, int ppc_req, const Trial* trial, cudaStream_t stream,
                        LaunchSet* ls) {
    const int smem_max = max_smem_per_block();
    if (smem_max <= 0) return fail(CSE_ECUDA, "no CUDA device");
    struct Ref { int search, mat, W, gm; };
    std::vector<Ref> refs;
    for (int i = 0; i < (int)act.size(); i++)
        for (int k = 0; k < act[i]->n_mats; k++)
            refs.push_back({i, k, act[i]->mats[k].W, act[i]->gm[k] ? 1 : 0});
    std::stable_sort(refs.begin(), refs.end(), [](const Ref& x, const Ref& y) {
        return x.W != y.W ? x.W < y.W : x.gm < y.gm;
    });
    const int nm = (int)refs.size(), n = (int)act.size();
    ls->gs = n > 0 && act[0]->search.gi_shared != 0;
    for (int i = 1; i < n; i++)
        if ((act[i]->search.gi_shared != 0) != ls->gs) return fail(CSE_EINVAL, "searches of one launch differ in coin mode");
    ls->mats.resize(nm);
    ls->groups.clear();
    for (int q = 0; q < nm; q++) {
        const SearchDev* sd = act[refs[q].search];
        ls->mats[q] = sd->mats[refs[q].mat];
        ls->mats[q].search = refs[q].search;
        if (ls->groups.empty() || ls->groups.back().W != refs[q].W || ls->groups.back().gm != (refs[q].gm != 0))
            ls->groups.push_back({refs[q].W, q, 0, 0, 0, 0, refs[q].gm != 0, {}, 0, {}, false, {}, nullptr});
        LaunchSet::Group& g = ls->groups.back();
        ls->mats[q].unit_base = g.units;
        g.count++;
        g.units += ls->mats[q].n_proc;
        g.mmax = std::max(g.mmax, ls->mats[q].mmax);
        g.cap = std::max(g.cap, ls->mats[q].cap);
    }
    for (auto& g : ls->groups) {
        g.L = g.gm ? WarpLayout{} : make_layout(g.W, g.cap, g.mmax);
        g.key = ClassKey{g.W, g.gm ? 1 : 0, g.cap, mbucket(g.mmax)};
        // measured defaults: 2 processes per CTA on the shared-memory path
        // ((3,3,3:23) shape), 4 on the HBM path ((6,6,6:153) shape), whose
        // kernels take the largest L1 carve-out and so fit 8 CTAs per SM
        g.ppc = ppc_req ? ppc_req : (g.gm ? 4 : 2);
        if (trial && trial->force_ppc) {
            g.ppc = trial->force_ppc;
        } else if (!ppc_req) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tuned_ppc.find(g.key);
            if (it != g_tuned_ppc.end()) g.ppc = it->second;
        }
        if (!g.gm)
            while (g.ppc > 1 && (long long)g.L.per_warp * g.ppc > smem_max) g.ppc--;
        if (!g.gm && g.L.per_warp > smem_max) return fail(CSE_ENOMEM, "process slice exceeds shared memory");
        const uint32_t fl = act[0]->opts.flags;
        if (g.gm && !ls->gs && (fl & CSE_FLAG_CTA_ENGINE) && !(fl & CSE_FLAG_WARP_ENGINE)) {
            g.CL = make_cta_layout(g.W, g.cap, g.mmax, (int)act[0]->opts.cta_list_cap,
                                   (int)act[0]->opts.cta_min_list, smem_max);
            g.cta = g.CL.bytes > 0;
        }
        cudaError_t e = g.cta ? prepare_round_cta(g.W, g.CL, g.ppc) : prepare_round(g.W, g.gm, ls->gs, g.L, g.ppc);
        if (e != cudaSuccess) return fail(CSE_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
        if (trial && trial->keys) trial->keys->push_back(g.key);
    }
    // positions of each search's matrices
    ls->pos.assign(nm, 0);
    std::vector<int> first(n, 0), cnt(n, 0);
    for (int q = 0; q < nm; q++) cnt[refs[q].search]++;
    for (int i = 1; i < n; i++) first[i] = first[i - 1] + cnt[i - 1];
    std::vector<int> fill(first);
    for (int q = 0; q < nm; q++) ls->pos[fill[refs[q].search]++] = q;
    Carve cv;
    const size_t om = cv.take(sizeof(DevMat) * nm), os = cv.take(sizeof(DevSearch) * n), op = cv.take(4 * (size_t)nm);
    const size_t ow = cv.take(3 * 4 * ls->groups.size());
    std::vector<size_t> oredo(ls->groups.size(), 0);
    for (size_t gi = 0; gi < ls->groups.size(); gi++)
        if (ls->groups[gi].cta) oredo[gi] = cv.take(4 * (size_t)ls->groups[gi].units);
    cudaError_t e = cudaMallocAsync(&ls->d_params, cv.off, stream);
    if (e != cudaSuccess) {
        ls->d_params = nullptr;
        return fail(CSE_ENOMEM, std::string("parameter block: ") + cudaGetErrorString(e));
    }
    char* b = (char*)ls->d_params;
    ls->d_mats = (DevMat*)(b + om);
    ls->d_searches = (DevSearch*)(b + os);
    ls->d_work = (int*)(b + ow);
    for (size_t gi = 0; gi < ls->groups.size(); gi++)
        if (ls->groups[gi].cta) ls->groups[gi].redo_list = (int*)(b + oredo[gi]);
    ls->searches.resize(n);
    for (int i = 0; i < n; i++) {
        ls->searches[i] = act[i]->search;
        ls->searches[i].mat_pos = (const int32_t*)(b + op) + first[i];
    }
    e = cudaMemcpyAsync(ls->d_mats, ls->mats.data(), sizeof(DevMat) * nm, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ls->d_searches, ls->searches.data(), sizeof(DevSearch) * n, cudaMemcpyHostToDevice,
                            stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + op, ls->pos.data(), 4 * (size_t)nm, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ls->d_work, 0, 3 * 4 * ls->groups.size(), stream);
    if (e != cudaSuccess) return fail(CSE_ECUDA, std::string("parameter upload: ") + cudaGetErrorString(e));
    return CSE_OK;
}

// Enqueues one round: the class launches (in parallel branches when aux
// streams are given) and the share kernel.
static cudaError_t enqueue_round(const LaunchSet& ls, cudaStream_t st, const std::vector<cudaStream_t>* aux,
                                 const std::vector<cudaEvent_t>* fork, cudaEvent_t* group_ev) {
    cudaError_t e = cudaSuccess;
    const size_t ng = ls.groups.size();
    if (aux && ng > 1) {
        cudaEventRecord((*fork)[0], st);
        for (size_t gi = 0; gi < ng; gi++) {
            const auto& g = ls.groups[gi];
            cudaStreamWaitEvent((*aux)[gi], (*fork)[0], 0);
            e = g.cta ? launch_round_cta(g.W, ls.d_mats + g.begin, g.count, ls.d_searches, g.units,
                                         ls.d_work + 3 * gi, g.redo_list, g.CL, g.ppc, (*aux)[gi])
                      : launch_round(g.W, g.gm, ls.gs, ls.d_mats + g.begin, g.count, ls.d_searches, g.units,
                                     ls.d_work + 3 * gi, g.L, g.ppc, (*aux)[gi]);
            if (e != cudaSuccess) return e;
            cudaEventRecord((*fork)[gi + 1], (*aux)[gi]);
            cudaStreamWaitEvent(st, (*fork)[gi + 1], 0);
        }
    } else {
        for (size_t gi = 0; gi < ng; gi++) {
            const auto& g = ls.groups[gi];
            if (group_ev) cudaEventRecord(group_ev[2 * gi], st);
            e = g.cta ? launch_round_cta(g.W, ls.d_mats + g.begin, g.count, ls.d_searches, g.units,
                                         ls.d_work + 3 * gi, g.redo_list, g.CL, g.ppc, st)
                      : launch_round(g.W, g.gm, ls.gs, ls.d_mats + g.begin, g.count, ls.d_searches, g.units,
                                     ls.d_work + 3 * gi, g.L, g.ppc, st);
            if (e != cudaSuccess) return e;
            if (group_ev) cudaEventRecord(group_ev[2 * gi + 1], st);
        }
    }
    return launch_share(ls.d_mats, ls.d_searches, (int)ls.searches.size(), ls.d_work, 3 * (int)ng, st);
}

// Builds and enqueues n independent searches as one static launch sequence.
// Each search keeps its own step clock, so its result does not depend on
// the others.
static int run_batch(int n, const cse_scheme* const* schemes, const cse_strategy_mix* mixes,
                     const int32_t* n_procs, const uint64_t* seeds, const int64_t* budgets,
                     const cse_opts* opts_in, void* cuda_stream, cse_result** outs,
                     const Trial* trial = nullptr, const Resume* resume = nullptr) {
    NvtxRange nvtx(trial ? "cse_trial" : resume ? "cse_search_resume" : n > 1 ? "cse_search_batch" : "cse_search");
    if (!outs) return fail(CSE_EINVAL, "out is NULL");
    if (n < 1 || !schemes || !mixes || !n_procs || !seeds || !budgets)
        return fail(CSE_EINVAL, "n_searches must be >= 1 with non-NULL arrays");
    for (int i = 0; i < n; i++) outs[i] = nullptr;
    cse_opts opts;
    int rc = check_opts(opts_in, &opts);
    if (rc) return rc;
    const bool iter_mode = opts.share_interval == 0;
    if (iter_mode && trial) return fail(CSE_EINVAL, "launch tuning runs in step-clock mode (share_interval >= 1)");
    const int words_policy = trial ? trial->words : kWordsDefault;
    // forced kernel words per column: a resume keeps the checkpoint's state
    // layout; the persistent batch kernel holds one engine, of 2 words, so
    // its matrices of 1 word run on the 2-word kernel
    std::vector<std::vector<int32_t>> forced(n);
    for (int i = 0; i < n; i++) {
        if (resume) {
            forced[i].assign(resume->hdr->words, resume->hdr->words + CSE_MAX_MATS);
        } else if (opts.flags & CSE_FLAG_PERSISTENT) {
            if (!schemes[i]) return fail(CSE_EINVAL, "NULL scheme");
            for (int k = 0; k < schemes[i]->n_mats; k++) forced[i].push_back(std::max(2, schemes[i]->W[k]));
        }
    }
    auto forced_of = [&](int i) { return forced[i].empty() ? nullptr : forced[i].data(); };
    for (int i = 0; i < n; i++) {  // validate everything before allocating
        SearchDev tmp;
        uint64_t w;
        std::vector<size_t> of;
        rc = search_plan(schemes[i], &mixes[i], n_procs[i], budgets[i], opts, &tmp, &w, &of, words_policy,
                         forced_of(i));
        if (rc) return rc;
    }
    if (max_smem_per_block() <= 0) return fail(CSE_ECUDA, "no CUDA device");
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    const bool use_graph = (opts.flags & CSE_FLAG_GRAPH) != 0 && !trial;
    std::vector<SearchDev*> sds(n, nullptr);
    auto drop = [&]() {
        for (auto* sd : sds) search_free(sd);
    };
    for (int i = 0; i < n; i++) {
        rc = search_create(schemes[i], &mixes[i], n_procs[i], seeds[i], budgets[i], opts, stream, &sds[i],
                           words_policy, forced_of(i));
        if (rc) {
            drop();
            return rc;
        }
    }
    if (resume) {  // one search: its device block comes from the checkpoint
        SearchDev* sd = sds[0];
        if (resume->hdr->bytes != sd->bytes) {
            drop();
            return fail(CSE_EINVAL, "checkpoint does not match this scheme and these options");
        }
        cudaError_t e = cudaMemcpyAsync(sd->d_block, resume->block, sd->bytes, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) {
            drop();
            return fail(CSE_ECUDA, std::string("checkpoint upload: ") + cudaGetErrorString(e));
        }
        const int64_t more = sd->budget - resume->hdr->done;
        sd->rounds = iter_mode ? (int)more : (int)((more + opts.share_interval - 1) / opts.share_interval);
    }
    Batch* B = new (std::nothrow) Batch();
    if (!B) {
        drop();
        return fail(CSE_ENOMEM, "host allocation");
    }
    B->stream = stream;
    for (int i = 0; i < n; i++) {
        outs[i] = new (std::nothrow) cse_result();
        if (!outs[i]) {
            for (int j = 0; j < i; j++) {
                delete outs[j];
                outs[j] = nullptr;
            }
            delete B;
            drop();
            return fail(CSE_ENOMEM, "host allocation");
        }
    }
    for (auto* sd : sds) B->rounds = std::max(B->rounds, sd->rounds);
    rc = build_launch(sds, (int)opts.procs_per_cta, trial, stream, &B->ls);
    cudaError_t e = cudaSuccess;
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
        drop();
        for (int j = 0; j < n; j++) {
            delete outs[j];
            outs[j] = nullptr;
        }
        return err == cudaSuccess ? rc : fail(CSE_ECUDA, std::string(what) + ": " + cudaGetErrorString(err));
    };
    if (rc) return bail(cudaSuccess, "");
    const size_t ng = B->ls.groups.size();
    // CSE_FLAG_PERSISTENT: every matrix in one unit space, one cooperative
    // kernel over all rounds
    B->persistent = (opts.flags & CSE_FLAG_PERSISTENT) != 0;
    WarpLayout pL{};
    DevMat* p_mats = nullptr;
    int p_units = 0, p_ppc = 2;
    int* p_work = nullptr;
    unsigned* p_bar = nullptr;
    if (B->persistent) {
        if (iter_mode || trial || B->ls.gs) {
            rc = fail(CSE_EINVAL, "CSE_FLAG_PERSISTENT runs the step clock, without shared coins");
            return bail(cudaSuccess, "");
        }
        int pcap = 0, pmmax = 0;
        for (const auto& g : B->ls.groups) {
            if (g.gm || g.W > 2) {
                rc = fail(CSE_EINVAL, "CSE_FLAG_PERSISTENT needs every matrix on the shared-memory engine with at "
                                      "most 64 rows");
                return bail(cudaSuccess, "");
            }
            pcap = std::max(pcap, g.cap);
            pmmax = std::max(pmmax, g.mmax);
        }
        pL = make_layout(2, pcap, pmmax);  // every matrix runs on the 2-word kernel
        p_ppc = opts.procs_per_cta ? (int)opts.procs_per_cta : 2;
        while (p_ppc > 1 && (long long)pL.per_warp * p_ppc > max_smem_per_block()) p_ppc--;
        if ((long long)pL.per_warp * p_ppc > max_smem_per_block()) {
            rc = fail(CSE_ENOMEM, "process slice exceeds shared memory");
            return bail(cudaSuccess, "");
        }
        std::vector<DevMat> pm(B->ls.mats);
        for (auto& M : pm) {
            M.unit_base = p_units;
            p_units += M.n_proc;
        }
        Carve pc;
        const size_t o_m = pc.take(sizeof(DevMat) * pm.size()), o_w = pc.take(4 * (size_t)B->rounds);
        const size_t o_b = pc.take(8), o_s = pc.take(4);
        if ((e = cudaMallocAsync(&B->d_pers, pc.off, stream)) != cudaSuccess) {
            B->d_pers = nullptr;
            return bail(e, "persistent launch block");
        }
        char* pb = (char*)B->d_pers;
        p_mats = (DevMat*)(pb + o_m);
        p_work = (int*)(pb + o_w);
        p_bar = (unsigned*)(pb + o_b);
        B->pers_status = (int*)(pb + o_s);
        if ((e = cudaMemcpyAsync(p_mats, pm.data(), sizeof(DevMat) * pm.size(), cudaMemcpyHostToDevice, stream)) !=
            cudaSuccess)
            return bail(e, "persistent launch block");
        if ((e = launch_batch_persistent(nullptr, 0, nullptr, 0, 0, 0, nullptr, nullptr, nullptr, 0, pL, p_ppc,
                                         nullptr, true)) != cudaSuccess)
            return bail(e, "kernel attributes");
    }
    if ((e = cudaEventCreate(&B->ev_begin)) != cudaSuccess) return bail(e, "event");
    if ((e = cudaEventCreate(&B->ev_end)) != cudaSuccess) return bail(e, "event");
    B->ev_round.resize(iter_mode ? 0 : 2 * (size_t)B->rounds);  // iteration mode: created per round
    for (auto& ev : B->ev_round)
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return bail(e, "event");
    if (trial) {
        B->ev_group.resize(2 * ng * (size_t)B->rounds);
        for (auto& ev : B->ev_group)
            if ((e = cudaEventCreate(&ev)) != cudaSuccess) return bail(e, "event");
    }
    const bool concurrent = use_graph && ng > 1 && !B->persistent;
    if (concurrent) {
        B->aux.resize(ng);
        B->ev_fork.resize(ng + 1);
        for (auto& st : B->aux)
            if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return bail(e, "stream");
        for (auto& ev : B->ev_fork)
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return bail(e, "event");
    }
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
    if (B->persistent) {
        // the per-round work counters, the barrier and its status start at 0
        e = cudaMemsetAsync((char*)p_work, 0, (size_t)((char*)B->pers_status + 4 - (char*)p_work), ls);
        if (e == cudaSuccess) rec(B->ev_round[0]);
        if (e == cudaSuccess)
            e = launch_batch_persistent(p_mats, (int)B->ls.mats.size(), B->ls.d_searches, (int)B->ls.searches.size(),
                                        p_units, B->rounds, p_work, p_bar, B->pers_status,
                                        opts.max_spin ? opts.max_spin : (1ull << 26), pL, p_ppc, ls, false);
        if (e == cudaSuccess) rec(B->ev_round[1]);
        if (e != cudaSuccess) return bail(e, "persistent batch launch");
    } else if (iter_mode) {
        // Iteration mode (Section 3.5.2, stopping rule of Section 4): rounds
        // are enqueued in chunks; between chunks the host reads every
        // search's convergence state and stops once all have finished.
        // Rounds of a finished search return at once on the device.
        std::vector<int32_t> conv(4 * (size_t)n, 0);
        int rd = 0;
        while (rd < B->rounds) {
            const int end = std::min(B->rounds, rd + kIterationChunk);
            for (; rd < end; rd++) {
                cudaEvent_t a = nullptr, z = nullptr;
                if ((e = cudaEventCreate(&a)) != cudaSuccess) return bail(e, "event");
                B->ev_round.push_back(a);
                if ((e = cudaEventCreate(&z)) != cudaSuccess) return bail(e, "event");
                B->ev_round.push_back(z);
                rec(a);
                e = enqueue_round(B->ls, ls, nullptr, nullptr, nullptr);
                if (e != cudaSuccess) return bail(e, "round launch");
                rec(z);
            }
            for (int i = 0; i < n && e == cudaSuccess; i++)
                e = cudaMemcpyAsync(&conv[4 * (size_t)i], sds[i]->search.conv, 16, cudaMemcpyDeviceToHost, ls);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ls);
            if (e != cudaSuccess) return bail(e, "convergence read");
            bool all = true;
            for (int i = 0; i < n; i++) all = all && (conv[4 * (size_t)i + 1] != 0 || conv[4 * (size_t)i + 3] >= sds[i]->budget);
            if (all) break;
        }
        B->rounds = rd;
    } else {
        for (int rd = 0; rd < B->rounds; rd++) {
            rec(B->ev_round[2 * rd]);
            e = enqueue_round(B->ls, ls, concurrent ? &B->aux : nullptr, concurrent ? &B->ev_fork : nullptr,
                              trial ? &B->ev_group[2 * ng * rd] : nullptr);
            if (e != cudaSuccess) return bail(e, "round launch");
            rec(B->ev_round[2 * rd + 1]);
        }
    }
    if ((e = rec(B->ev_end)) != cudaSuccess) return bail(e, "event record");
    if (use_graph) {
        if ((e = cudaStreamEndCapture(ls, &B->graph)) != cudaSuccess) return bail(e, "end capture");
        if ((e = cudaGraphInstantiate(&B->gexec, B->graph, 0)) != cudaSuccess) return bail(e, "graph instantiate");
        if ((e = cudaGraphLaunch(B->gexec, stream)) != cudaSuccess) return bail(e, "graph launch");
    }
    for (int i = 0; i < n; i++) {
        outs[i]->sd = sds[i];
        outs[i]->batch = B;
        B->refs++;
    }
    return CSE_OK;
}

// Per-class round-kernel time of a finished trial batch.
static int trial_times(const cse_result* r, std::vector<float>* ms) {
    const Batch* B = r->batch;
    const size_t ng = B->ls.groups.size();
    CUDA_TRY(cudaEventSynchronize(B->ev_end));
    ms->assign(ng, 0.f);
    for (int rd = 0; rd < B->rounds; rd++)
        for (size_t gi = 0; gi < ng; gi++) {
            float x = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&x, B->ev_group[2 * (rd * ng + gi)], B->ev_group[2 * (rd * ng + gi) + 1]));
            (*ms)[gi] += x;
        }
    return CSE_OK;
}

// ---------------------------------------------------------------------------
// Serving: a worker thread runs rounds over the searches admitted so far;
// new requests join at a round boundary when their device footprint fits.
// ---------------------------------------------------------------------------
struct Request {
    uint64_t ticket = 0;
    const cse_scheme* scheme = nullptr;
    cse_strategy_mix mix{};
    int n_proc = 0;
    uint64_t seed = 0;
    int64_t budget = 0;
    size_t bytes = 0;
    int64_t units = 0;
    uint64_t smem = 0;  // shared-memory footprint of its process pools
    std::chrono::steady_clock::time_point t_submit;
    SearchDev* sd = nullptr;
    cse_result* res = nullptr;
    int status = CSE_OK;
    std::string error;
    bool done = false;
    bool cancel = false;  // leave at the next round boundary
};

struct cse_server {
    cse_opts opts{};
    uint64_t hbm_budget = 0;
    int64_t max_units = 0;     // cap on the processes (all matrices) of active searches
    int64_t active_units = 0;
    uint64_t smem_budget = 0;  // cap on the shared-memory footprint of active searches
    uint64_t used_smem = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> pending;
    std::vector<Request*> active;
    std::map<uint64_t, Request*> by_ticket;
    bool stop = false;
    uint64_t next_ticket = 1;
    uint64_t used_bytes = 0;
    // statistics
    std::vector<double> latencies_ms;
    int64_t steps_done = 0;
    std::chrono::steady_clock::time_point t_first, t_last;
    bool any = false;
    int rounds_run = 0, max_active = 0;
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
    NvtxRange nvtx("cse_scheme_load");
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
    cudaError_t ea = cudaMalloc(&s->d_block, cv.off);
    if (ea == cudaErrorMemoryAllocation) {
        // the searches' stream-ordered pool keeps what it freed (its release
        // threshold is unbounded): hand that back to the device and try again
        cudaGetLastError();
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            cudaDeviceSynchronize();
            cudaMemPoolTrimTo(pool, 0);
        }
        ea = cudaMalloc(&s->d_block, cv.off);
    }
    if (ea != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return fail(ea == cudaErrorMemoryAllocation ? CSE_ENOMEM : CSE_ECUDA,
                    std::string("device allocation of the scheme: ") + cudaGetErrorString(ea));
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
    // The candidate arrays hold mmax entries and positions within a
    // variable's list are 16-bit: a matrix whose initial list is longer than
    // mmax cannot be searched.  (mmax bounds every later list, since no row
    // grows, except where it was clipped to 32767.)
    for (int k = 0; k < n_mats; k++) {
        int32_t meta[2] = {0, 0};
        e = cudaMemcpy(meta, s->d_meta0[k], sizeof meta, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            cudaFree(s->d_block);
            delete s;
            return fail(CSE_ECUDA, std::string("scheme ingest: ") + cudaGetErrorString(e));
        }
        if (meta[1] > s->mmax[k]) {
            const int mm = s->mmax[k];
            cudaFree(s->d_block);
            delete s;
            return fail(CSE_EINVAL, "matrix " + std::to_string(k) + ": " + std::to_string(meta[1]) +
                                        " initial repeated pairs, more than the " + std::to_string(mm) +
                                        " a candidate list holds");
        }
    }
    uint64_t ih = 0xCBF29CE484222325ull;
    for (int k = 0; k < n_mats; k++) {
        ih = fnv(fnv(ih, (uint32_t)s->rows[k]), (uint32_t)s->cols[k]);
        for (size_t x = 0; x < (size_t)s->rows[k] * s->cols[k]; x++) ih = fnv(ih, (uint32_t)(uint8_t)mats[k][x]);
    }
    s->input_hash = ih;
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

int cse_brent_check(int32_t m, int32_t n, int32_t p, int32_t r, const int8_t* U, const int8_t* V, const int8_t* W,
                    int64_t* violations) {
    if (m < 1 || n < 1 || p < 1 || r < 1 || !U || !V || !W || !violations)
        return fail(CSE_EINVAL, "bad scheme dimensions or NULL argument");
    if ((int64_t)m * n > 4096 || (int64_t)n * p > 4096 || (int64_t)m * p > 4096 || r > 65536)
        return fail(CSE_EINVAL, "scheme too large for the Brent check (m n, n p, m p <= 4096, r <= 65536)");
    const size_t su = (size_t)r * m * n, sv = (size_t)r * n * p, sw = (size_t)r * m * p;
    char* d = nullptr;
    CUDA_TRY(cudaMalloc(&d, su + sv + sw + 16));
    int8_t* dU = (int8_t*)d + 16;
    int8_t* dV = dU + su;
    int8_t* dW = dV + sv;
    unsigned long long* dbad = (unsigned long long*)d;
    unsigned long long bad = 0;
    cudaError_t e = cudaMemset(dbad, 0, 8);
    if (e == cudaSuccess) e = cudaMemcpy(dU, U, su, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dV, V, sv, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dW, W, sw, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_brent(dU, dV, dW, m, n, p, r, dbad, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(&bad, dbad, 8, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(CSE_ECUDA, std::string("Brent check: ") + cudaGetErrorString(e));
    *violations = (int64_t)bad;
    return CSE_OK;
}

int cse_philox(uint64_t seed, const uint32_t* counters, int64_t n, uint32_t* out) {
    if (n < 0 || n > (int64_t(1) << 24)) return fail(CSE_EINVAL, "n out of range [0, 2^24]");
    if (n > 0 && (!counters || !out)) return fail(CSE_EINVAL, "NULL counters or out");
    if (n == 0) return CSE_OK;
    const size_t bytes = (size_t)n * 16;
    char* d = nullptr;
    CUDA_TRY(cudaMalloc(&d, 2 * bytes));
    uint32_t* dc = reinterpret_cast<uint32_t*>(d);
    uint32_t* dout = reinterpret_cast<uint32_t*>(d + bytes);
    cudaError_t e = cudaMemcpy(dc, counters, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_philox(dc, n, seed, dout, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, bytes, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(CSE_ECUDA, std::string("Philox: ") + cudaGetErrorString(e));
    return CSE_OK;
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



int cse_search(const cse_scheme* s, const cse_strategy_mix* mix, int32_t n_proc, uint64_t seed,
               int64_t budget, const cse_opts* opts, void* cuda_stream, cse_result** out) {
    if (!out) return fail(CSE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!s || !mix) return fail(CSE_EINVAL, "NULL scheme or strategy mix");
    return run_batch(1, &s, mix, &n_proc, &seed, &budget, opts, cuda_stream, out);
}

static int wait_result(const cse_result* r);

int cse_checkpoint_size(const cse_result* r, size_t* bytes) {
    if (!r || !r->sd || !bytes) return fail(CSE_EINVAL, "NULL result or output");
    *bytes = sizeof(CkptHeader) + r->sd->bytes;
    return CSE_OK;
}

int cse_checkpoint_save(const cse_result* r, void* host_buf, size_t bytes) {
    NvtxRange nvtx("cse_checkpoint_save");
    if (!r || !r->sd || !host_buf) return fail(CSE_EINVAL, "NULL result or buffer");
    const SearchDev* sd = r->sd;
    if (bytes < sizeof(CkptHeader) + sd->bytes) return fail(CSE_EINVAL, "checkpoint buffer too small");
    const uint32_t iv = sd->opts.share_interval;
    if (iv != 0 && sd->budget % iv != 0)
        return fail(CSE_EINVAL, "a checkpoint needs a step budget that is a multiple of share_interval");
    int rc = wait_result(r);
    if (rc) return rc;
    CkptHeader h{};
    h.magic = kCkptMagic;
    h.version = kCkptVersion;
    h.interval = iv;
    h.permille = sd->opts.share_permille;
    h.cap = sd->opts.col_cap;
    h.patience = sd->opts.patience_rounds;
    h.flags = sd->opts.flags & (CSE_FLAG_GI_SHARED_COINS | CSE_FLAG_TRACE);
    h.n_mats = sd->n_mats;
    h.n_proc = sd->n_proc;
    for (int k = 0; k < sd->n_mats; k++) {
        h.rows[k] = sd->rows[k];
        h.cols[k] = sd->cols[k];
        h.words[k] = sd->words[k];
    }
    h.seed = sd->seed;
    h.mix = sd->mix;
    h.done = sd->budget;
    h.bytes = sd->bytes;
    h.input_hash = sd->input_hash;
    std::memcpy(host_buf, &h, sizeof h);
    CUDA_TRY(cudaMemcpy((char*)host_buf + sizeof h, sd->d_block, sd->bytes, cudaMemcpyDeviceToHost));
    return CSE_OK;
}

int cse_search_resume(const cse_scheme* s, const void* ckpt, size_t bytes, int64_t more_steps,
                      const cse_opts* launch_opts, void* cuda_stream, cse_result** out) {
    if (!out) return fail(CSE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!s || !ckpt || bytes < sizeof(CkptHeader)) return fail(CSE_EINVAL, "NULL scheme or short checkpoint");
    CkptHeader h;
    std::memcpy(&h, ckpt, sizeof h);
    if (h.magic != kCkptMagic || h.version != kCkptVersion) return fail(CSE_EINVAL, "not a checkpoint of this library");
    if (bytes < sizeof h + h.bytes) return fail(CSE_EINVAL, "truncated checkpoint");
    if (more_steps < 0 || h.done < 0 || h.done + more_steps >= INT32_MAX) return fail(CSE_EINVAL, "bad step count");
    if (h.n_mats != s->n_mats) return fail(CSE_EINVAL, "checkpoint of another scheme");
    for (int k = 0; k < s->n_mats; k++)
        if (h.rows[k] != s->rows[k] || h.cols[k] != s->cols[k]) return fail(CSE_EINVAL, "checkpoint of another scheme");
    if (h.input_hash != s->input_hash)
        return fail(CSE_EINVAL, "checkpoint of another scheme: the matrices differ from those it was taken on");
    cse_opts opts;
    cse_opts_default(&opts);
    if (launch_opts) opts = *launch_opts;  // the launch fields (procs_per_cta) come from the caller
    opts.share_interval = h.interval;
    opts.share_permille = h.permille;
    opts.col_cap = h.cap;
    opts.patience_rounds = h.patience;
    // the coin mode changes results and the trace flag the trajectory record:
    // both are the checkpoint's
    opts.flags = (opts.flags & ~(uint32_t)(CSE_FLAG_GI_SHARED_COINS | CSE_FLAG_GRAPH | CSE_FLAG_TRACE)) | h.flags;
    const int64_t total = h.done + more_steps;
    const int32_t n_proc = h.n_proc;
    const uint64_t seed = h.seed;
    Resume res{&h, (const char*)ckpt + sizeof h};
    return run_batch(1, &s, &h.mix, &n_proc, &seed, &total, &opts, cuda_stream, out, nullptr, &res);
}

int cse_search_batch(int32_t n_searches, const cse_scheme* const* schemes, const cse_strategy_mix* mixes,
                     const int32_t* n_processes, const uint64_t* seeds, const int64_t* step_budgets,
                     const cse_opts* opts, void* cuda_stream, cse_result** outs) {
    return run_batch(n_searches, schemes, mixes, n_processes, seeds, step_budgets, opts, cuda_stream, outs);
}

int cse_autotune(int32_t n_searches, const cse_scheme* const* schemes, const cse_strategy_mix* mixes,
                 const int32_t* n_processes, const uint64_t* seeds, const int64_t* step_budgets,
                 const cse_opts* opts, int32_t trial_steps, void* cuda_stream, cse_tune_entry* entries,
                 int32_t max_entries, int32_t* n_entries) {
    if (n_searches < 1 || n_searches > 4096 || !step_budgets || !schemes) return fail(CSE_EINVAL, "bad n_searches");
    if (trial_steps < 1) return fail(CSE_EINVAL, "trial_steps must be >= 1");
    std::vector<int64_t> tb(n_searches);
    for (int i = 0; i < n_searches; i++) tb[i] = std::min<int64_t>(step_budgets[i], trial_steps);
    std::vector<cse_result*> outs(n_searches);
    // trial rounds with 1..4 processes per CTA, at each matrix's own words and,
    // if some matrix's words are not a power of two, at the wider kernel
    bool any_wide = false;
    for (int i = 0; i < n_searches; i++)
        for (int k = 0; schemes[i] && k < schemes[i]->n_mats; k++) any_wide |= widen_words(schemes[i]->W[k]) != schemes[i]->W[k];
    std::vector<std::vector<float>> ms[2] = {std::vector<std::vector<float>>(4), std::vector<std::vector<float>>(4)};
    std::vector<ClassKey> keys[2];
    for (int pol = 0; pol < (any_wide ? 2 : 1); pol++) {
        for (int ppc = 1; ppc <= 4; ppc++) {
            for (int rep = 0; rep < 2; rep++) {  // the first run warms up
                Trial tr;
                tr.force_ppc = ppc;
                tr.words = pol == 0 ? kWordsNatural : kWordsWide;
                std::vector<ClassKey> k;
                tr.keys = &k;
                int rc = run_batch(n_searches, schemes, mixes, n_processes, seeds, tb.data(), opts, cuda_stream,
                                   outs.data(), &tr);
                if (rc) return rc;
                rc = trial_times(outs[0], &ms[pol][ppc - 1]);
                for (auto* r : outs) cse_result_free(r);
                if (rc) return rc;
                keys[pol] = k;
            }
        }
    }
    auto best_ppc = [&](int pol, size_t gi) {
        int best = 1;
        for (int ppc = 2; ppc <= 4; ppc++)
            if (ms[pol][ppc - 1][gi] < ms[pol][best - 1][gi]) best = ppc;
        return best;
    };
    std::lock_guard<std::mutex> lk(g_tune_mu);
    std::vector<int> chosen_words(keys[0].size()), chosen_ppc(keys[0].size());
    std::vector<int> wide_of(keys[0].size(), -1);  // the wide trial's group holding class gi
    for (size_t gi = 0; gi < keys[0].size(); gi++) {
        chosen_words[gi] = keys[0][gi].W;
        chosen_ppc[gi] = best_ppc(0, gi);
        g_tuned_ppc[keys[0][gi]] = chosen_ppc[gi];
    }
    // a wider kernel is kept for the classes it absorbs when its round kernels
    // take less time than theirs, each class at its best processes per CTA
    for (size_t wj = 0; wj < keys[1].size(); wj++) {
        const ClassKey& K = keys[1][wj];
        float t_own = 0.f;
        bool widened = false;
        std::vector<size_t> members;
        for (size_t gi = 0; gi < keys[0].size(); gi++) {
            const ClassKey& k = keys[0][gi];
            if (k.gm != K.gm || k.cap != K.cap || (k.W != K.W && widen_words(k.W) != K.W)) continue;
            members.push_back(gi);
            widened |= k.W < K.W;
            t_own += ms[0][chosen_ppc[gi] - 1][gi];
        }
        if (!widened) continue;
        const int wppc = best_ppc(1, wj);
        const bool take = ms[1][wppc - 1][wj] < t_own;
        for (size_t gi : members) {
            wide_of[gi] = (int)wj;
            const ClassKey own{keys[0][gi].W, keys[0][gi].gm, keys[0][gi].cap, 0};
            if (keys[0][gi].W == K.W) continue;
            if (take) {
                g_tuned_words[own] = K.W;
                chosen_words[gi] = K.W;
                chosen_ppc[gi] = wppc;
            } else {
                g_tuned_words.erase(own);
            }
        }
        if (take) g_tuned_ppc[K] = wppc;
    }
    int32_t ne = 0;
    for (size_t gi = 0; gi < keys[0].size(); gi++) {
        if (entries && ne < max_entries) {
            cse_tune_entry& en = entries[ne];
            en.words_per_column = keys[0][gi].W;
            en.hbm_path = keys[0][gi].gm;
            en.candidate_bound = keys[0][gi].mbucket;
            en.procs_per_cta = chosen_ppc[gi];
            en.kernel_words = chosen_words[gi];
            for (int ppc = 1; ppc <= 4; ppc++) {
                en.trial_ms[ppc - 1] = ms[0][ppc - 1][gi];
                en.trial_ms_wide[ppc - 1] = wide_of[gi] >= 0 && keys[0][gi].W != keys[1][wide_of[gi]].W
                                                ? ms[1][ppc - 1][wide_of[gi]]
                                                : -1.f;
            }
        }
        ne++;
    }
    if (n_entries) *n_entries = ne;
    return CSE_OK;
}

int cse_tune_interval(int32_t n_searches, const cse_scheme* const* schemes, const cse_strategy_mix* mixes,
                      const int32_t* n_processes, const uint64_t* seeds, const int64_t* step_budgets,
                      const cse_opts* opts_in, const uint32_t* candidates, int32_t n_candidates,
                      int32_t trial_steps, void* cuda_stream, uint32_t* best_interval, int64_t* best_total) {
    if (!candidates || n_candidates < 1 || trial_steps < 1 || !step_budgets || n_searches < 1)
        return fail(CSE_EINVAL, "bad interval candidates or trial size");
    for (int c = 0; c < n_candidates; c++)
        if (candidates[c] < 1) return fail(CSE_EINVAL, "interval candidates must be >= 1");
    cse_opts opts;
    int rc = check_opts(opts_in, &opts);
    if (rc) return rc;
    std::vector<int64_t> tb(n_searches);
    for (int i = 0; i < n_searches; i++) tb[i] = std::min<int64_t>(step_budgets[i], trial_steps);
    std::vector<cse_result*> outs(n_searches);
    int64_t best = INT64_MAX;
    uint32_t besti = candidates[0];
    for (int c = 0; c < n_candidates; c++) {
        opts.share_interval = candidates[c];
        rc = run_batch(n_searches, schemes, mixes, n_processes, seeds, tb.data(), &opts, cuda_stream, outs.data());
        if (rc) return rc;
        int64_t total = 0;
        for (auto* r : outs) {
            int64_t t = 0;
            if (rc == CSE_OK) rc = cse_result_fetch(r, 0, nullptr, 0, nullptr, nullptr, &t);
            total += t;
        }
        for (auto* r : outs) cse_result_free(r);
        if (rc) return rc;
        if (total < best) {
            best = total;
            besti = candidates[c];
        }
    }
    if (best_interval) *best_interval = besti;
    if (best_total) *best_total = best;
    return CSE_OK;
}

static int wait_result(const cse_result* r) {
    if (!r || !r->sd) return fail(CSE_EINVAL, "NULL result");
    if (r->batch) CUDA_TRY(cudaEventSynchronize(r->batch->ev_end));
    if (r->batch && r->batch->pers_status) {
        int32_t ps = 0;
        CUDA_TRY(cudaMemcpy(&ps, r->batch->pers_status, 4, cudaMemcpyDeviceToHost));
        if (ps != 0) return fail(CSE_ETIMEOUT, "a grid barrier of the persistent batch kernel gave up (max_spin)");
    }
    int32_t status = 0;
    CUDA_TRY(cudaMemcpy(&status, r->sd->search.status, 4, cudaMemcpyDeviceToHost));
    if (status != 0) return fail(CSE_ESTATE, "device consistency check failed (candidate list overflow)");
    return CSE_OK;
}

int cse_result_fetch(const cse_result* r, int32_t mat, int32_t* subst, int32_t cap_entries, int32_t* n_subst,
                     int64_t* additions, int64_t* total_additions) {
    NvtxRange nvtx("cse_result_fetch");
    int rc = wait_result(r);
    if (rc) return rc;
    const SearchDev* sd = r->sd;
    if (mat < 0 || mat >= sd->n_mats) return fail(CSE_EINVAL, "matrix index out of range");
    int64_t total = 0;
    int32_t meta[2] = {0, 0};
    for (int k = 0; k < sd->n_mats; k++) {
        int32_t mk[2];
        CUDA_TRY(cudaMemcpy(mk, sd->mats[k].result_meta, 8, cudaMemcpyDeviceToHost));
        total += mk[0];
        if (k == mat) std::memcpy(meta, mk, 8);
    }
    if (subst && cap_entries > 0) {
        const int nn = std::min(cap_entries, meta[1]);
        if (nn > 0) CUDA_TRY(cudaMemcpy(subst, sd->mats[mat].result, (size_t)nn * 4, cudaMemcpyDeviceToHost));
    }
    if (n_subst) *n_subst = meta[1];
    if (additions) *additions = meta[0];
    if (total_additions) *total_additions = total;
    return CSE_OK;
}

int cse_result_procs(const cse_result* r, int32_t mat, cse_proc_record* out) {
    int rc = wait_result(r);
    if (rc) return rc;
    const SearchDev* sd = r->sd;
    if (mat < 0 || mat >= sd->n_mats || !out) return fail(CSE_EINVAL, "bad matrix index or output");
    const DevMat& M = sd->mats[mat];
    if (sd->budget == 0) {  // no step ran: every record is the input itself
        int32_t meta[2];
        CUDA_TRY(cudaMemcpy(meta, M.result_meta, 8, cudaMemcpyDeviceToHost));
        for (int p = 0; p < sd->n_proc; p++) {
            out[p].best_cost = meta[0];
            out[p].best_len = 0;
            out[p].runs = 0;
            out[p].best_hash = kFnv0;
            out[p].traj_hash = kFnv0;
            out[p].ops = 0;
            out[p].substeps = 0;
            out[p].best_strategy = -1;
            out[p].pad = 0;
            out[p].method_ops = 0;
        }
        return CSE_OK;
    }
    std::vector<uint32_t> hdr((size_t)sd->n_proc * H_WORDS);
    CUDA_TRY(cudaMemcpy2D(hdr.data(), H_WORDS * 4, M.state, (size_t)M.state_words * 4, H_WORDS * 4, sd->n_proc,
                          cudaMemcpyDeviceToHost));
    std::vector<int32_t> lists((size_t)sd->n_proc * sd->cap);
    CUDA_TRY(cudaMemcpy(lists.data(), M.best_list, lists.size() * 4, cudaMemcpyDeviceToHost));
    for (int p = 0; p < sd->n_proc; p++) {
        const uint32_t* h = &hdr[(size_t)p * H_WORDS];
        cse_proc_record& o = out[p];
        o.best_cost = (int32_t)h[H_BEST_COST];
        o.best_len = (int32_t)h[H_BEST_LEN];
        o.runs = (int32_t)h[H_RUNS];
        uint64_t hh = kFnv0;
        for (int x = 0; x < o.best_len; x++) hh = fnv(hh, (uint32_t)lists[(size_t)p * sd->cap + x]);
        o.best_hash = hh;
        o.traj_hash = (uint64_t)h[H_TRAJ_LO] | (uint64_t)h[H_TRAJ_HI] << 32;
        o.ops = (int64_t)((uint64_t)h[H_OPS_LO] | (uint64_t)h[H_OPS_HI] << 32);
        o.substeps = (int32_t)h[H_SUBSTEPS];
        o.best_strategy = (int32_t)h[H_BEST_STRAT];
        o.pad = 0;
        o.method_ops = (int64_t)((uint64_t)h[H_MOPS_LO] | (uint64_t)h[H_MOPS_HI] << 32);
    }
    return CSE_OK;
}

int cse_result_curve(const cse_result* r, int32_t mat, int32_t* costs, int32_t max_points, int32_t* n_points) {
    int rc = wait_result(r);
    if (rc) return rc;
    const SearchDev* sd = r->sd;
    if (mat < 0 || mat >= sd->n_mats) return fail(CSE_EINVAL, "matrix index out of range");
    int32_t rounds = 0;
    if (sd->search.interval == 0) {
        int32_t conv[4];
        CUDA_TRY(cudaMemcpy(conv, sd->search.conv, 16, cudaMemcpyDeviceToHost));
        rounds = conv[3];
    } else {
        rounds = (int32_t)((sd->budget + sd->search.interval - 1) / sd->search.interval);
    }
    rounds = std::min(rounds, (int32_t)kCurvePoints);
    if (n_points) *n_points = rounds;
    const int32_t n = std::min(rounds, max_points);
    if (costs && n > 0) CUDA_TRY(cudaMemcpy(costs, sd->mats[mat].curve, (size_t)n * 4, cudaMemcpyDeviceToHost));
    return CSE_OK;
}

int cse_result_counters(const cse_result* r, int64_t* process_steps, int64_t* substeps, int64_t* alg_ops) {
    int rc = wait_result(r);
    if (rc) return rc;
    const SearchDev* sd = r->sd;
    uint64_t ops = 0, sub = 0, steps = 0;
    for (int k = 0; k < sd->n_mats; k++) {
        unsigned long long c[3];
        CUDA_TRY(cudaMemcpy(c, sd->mats[k].counters, 24, cudaMemcpyDeviceToHost));
        ops += c[0];
        sub += c[1];
        steps += c[2];
    }
    if (process_steps)  // iteration mode: counted on the device (runs differ in length)
        *process_steps = sd->search.interval == 0 ? (int64_t)steps : (int64_t)sd->n_mats * sd->n_proc * sd->budget;
    if (substeps) *substeps = (int64_t)sub;
    if (alg_ops) *alg_ops = (int64_t)ops;
    return CSE_OK;
}

int cse_result_engine_rounds(const cse_result* r, int64_t* cta_rounds, int64_t* warp_rounds) {
    int rc = wait_result(r);
    if (rc) return rc;
    const SearchDev* sd = r->sd;
    uint64_t a = 0, b = 0;
    for (int k = 0; k < sd->n_mats; k++) {
        unsigned long long c[6];
        CUDA_TRY(cudaMemcpy(c, sd->mats[k].counters, 48, cudaMemcpyDeviceToHost));
        a += c[4];
        b += c[5];
    }
    if (cta_rounds) *cta_rounds = (int64_t)a;
    if (warp_rounds) *warp_rounds = (int64_t)b;
    return CSE_OK;
}

int cse_result_method_ops(const cse_result* r, int64_t* method_ops) {
    int rc = wait_result(r);
    if (rc) return rc;
    if (!method_ops) return fail(CSE_EINVAL, "method_ops is NULL");
    const SearchDev* sd = r->sd;
    uint64_t mops = 0;
    for (int k = 0; k < sd->n_mats; k++) {
        unsigned long long c[4];
        CUDA_TRY(cudaMemcpy(c, sd->mats[k].counters, 32, cudaMemcpyDeviceToHost));
        mops += c[3];
    }
    *method_ops = (int64_t)mops;
    return CSE_OK;
}

int cse_result_timing(const cse_result* r, float* round_ms, float* total_ms, int32_t* n_rounds) {
    int rc = wait_result(r);
    if (rc) return rc;
    const Batch* B = r->batch;
    if (!B) {  // a served request: time from submission to completion
        if (round_ms) *round_ms = (float)r->latency_ms;
        if (total_ms) *total_ms = (float)r->latency_ms;
        if (n_rounds) *n_rounds = r->sd->rounds;
        return CSE_OK;
    }
    float sum = 0.f, tot = 0.f;
    for (int rd = 0; rd < (B->persistent ? 1 : B->rounds); rd++) {  // persistent: one launch, all rounds
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

int cse_result_iterations(const cse_result* r, int32_t* iterations, int32_t* converged, int64_t* best_total) {
    int rc = wait_result(r);
    if (rc) return rc;
    const SearchDev* sd = r->sd;
    if (sd->search.interval != 0) return fail(CSE_EINVAL, "not an iteration-mode search (share_interval = 0)");
    int32_t conv[4];
    CUDA_TRY(cudaMemcpy(conv, sd->search.conv, 16, cudaMemcpyDeviceToHost));
    if (iterations) *iterations = conv[3];
    if (converged) *converged = conv[1] != 0 && conv[3] < sd->budget ? 1 : 0;
    if (best_total) *best_total = conv[2] == INT_MAX ? -1 : conv[2];
    return CSE_OK;
}

int cse_result_hybrid(const cse_result* const* results, int32_t n_results, int32_t* best_result,
                      int64_t* total_additions) {
    if (!results || n_results < 1 || !best_result) return fail(CSE_EINVAL, "no results or NULL output");
    const SearchDev* s0 = results[0] ? results[0]->sd : nullptr;
    if (!s0) return fail(CSE_EINVAL, "NULL result");
    for (int i = 1; i < n_results; i++) {
        const SearchDev* si = results[i] ? results[i]->sd : nullptr;
        if (!si || si->n_mats != s0->n_mats) return fail(CSE_EINVAL, "results of different schemes");
        for (int k = 0; k < s0->n_mats; k++)
            if (si->rows[k] != s0->rows[k] || si->cols[k] != s0->cols[k])
                return fail(CSE_EINVAL, "results of different schemes");
    }
    std::vector<int64_t> best(s0->n_mats, INT64_MAX);
    for (int i = 0; i < n_results; i++) {
        int rc = wait_result(results[i]);
        if (rc) return rc;
        for (int k = 0; k < s0->n_mats; k++) {
            int32_t meta[2];
            CUDA_TRY(cudaMemcpy(meta, results[i]->sd->mats[k].result_meta, 8, cudaMemcpyDeviceToHost));
            if (meta[0] < best[k]) {  // strictly lower: the first result wins ties
                best[k] = meta[0];
                best_result[k] = i;
            }
        }
    }
    int64_t t = 0;
    for (int64_t b : best) t += b;
    if (total_additions) *total_additions = t;
    return CSE_OK;
}

int cse_search_shard(const cse_scheme* s, const cse_strategy_mix* mix, int32_t n_processes, int32_t proc_begin,
                     int32_t proc_count, uint64_t seed, int64_t step_budget, const cse_opts* opts_in, void* cuda_stream,
                     cse_result** out) {
    NvtxRange nvtx("cse_search_shard");
    if (!out) return fail(CSE_EINVAL, "out is NULL");
    *out = nullptr;
    cse_opts opts;
    int rc = check_opts(opts_in, &opts);
    if (rc) return rc;
    if (opts.share_interval == 0) return fail(CSE_EINVAL, "a shard runs the step clock (share_interval >= 1)");
    if (opts.flags & CSE_FLAG_GRAPH) return fail(CSE_EINVAL, "a shard's rounds are enqueued one at a time: no graph");
    if (n_processes < 1 || n_processes > (1 << 20) || proc_begin < 0 || proc_count < 1 ||
        (int64_t)proc_begin + proc_count > n_processes)
        return fail(CSE_EINVAL, "need 0 <= proc_begin < proc_begin + proc_count <= n_processes <= 2^20");
    if (max_smem_per_block() <= 0) return fail(CSE_ECUDA, "no CUDA device");
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    SearchDev* sd = nullptr;
    rc = search_create(s, mix, proc_count, seed, step_budget, opts, stream, &sd);
    if (rc) return rc;
    for (auto& M : sd->mats) M.proc_offset = proc_begin;
    Batch* B = new (std::nothrow) Batch();
    cse_result* r = new (std::nothrow) cse_result();
    ShardState* sh = new (std::nothrow) ShardState();
    auto bail = [&](int code, const std::string& msg) {
        if (B) {
            B->ev_end = nullptr;
            B->release();
        }
        delete B;
        delete r;
        delete sh;
        search_free(sd);
        return fail(code, msg);
    };
    if (!B || !r || !sh) return bail(CSE_ENOMEM, "host allocation");
    B->stream = stream;
    rc = build_launch({sd}, (int)opts.procs_per_cta, nullptr, stream, &B->ls);
    if (rc) return bail(rc, cse_last_error());
    cudaError_t e = cudaEventCreate(&B->ev_begin);
    if (e == cudaSuccess) e = cudaEventCreate(&B->ev_end);
    B->ev_round.assign(2 * (size_t)sd->rounds, nullptr);
    for (auto& ev : B->ev_round)
        if (e == cudaSuccess) e = cudaEventCreate(&ev);
    if (e == cudaSuccess) e = cudaEventRecord(B->ev_begin, stream);
    if (e != cudaSuccess) return bail(CSE_ECUDA, std::string("shard events: ") + cudaGetErrorString(e));
    B->refs = 1;
    sh->total = n_processes;
    sh->offset = proc_begin;
    r->sd = sd;
    r->batch = B;
    r->shard = sh;
    *out = r;
    return CSE_OK;
}

int cse_shard_round(cse_result* r, uint64_t* round_keys, int32_t* rounds_left) {
    if (!r || !r->shard || !r->batch || !round_keys || !rounds_left) return fail(CSE_EINVAL, "not a shard, or NULL output");
    ShardState* sh = r->shard;
    SearchDev* sd = r->sd;
    Batch* B = r->batch;
    if (sh->in_round) return fail(CSE_EINVAL, "the previous round's boundary is not completed (cse_shard_share)");
    if (sh->rounds_done >= sd->rounds) {
        *rounds_left = 0;
        return CSE_OK;
    }
    const LaunchSet& ls = B->ls;
    cudaStream_t st = B->stream;
    cudaEventRecord(B->ev_round[2 * sh->rounds_done], st);
    for (size_t gi = 0; gi < ls.groups.size(); gi++) {
        const auto& g = ls.groups[gi];
        cudaError_t e = g.cta ? launch_round_cta(g.W, ls.d_mats + g.begin, g.count, ls.d_searches, g.units,
                                                 ls.d_work + 3 * gi, g.redo_list, g.CL, g.ppc, st)
                              : launch_round(g.W, g.gm, ls.gs, ls.d_mats + g.begin, g.count, ls.d_searches, g.units,
                                             ls.d_work + 3 * gi, g.L, g.ppc, st);
        if (e != cudaSuccess) return fail(CSE_ECUDA, std::string("round launch: ") + cudaGetErrorString(e));
    }
    cudaEventRecord(B->ev_round[2 * sh->rounds_done + 1], st);
    for (int k = 0; k < sd->n_mats; k++)
        CUDA_TRY(cudaMemcpyAsync(&round_keys[k], sd->mats[k].round_min, 8, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    int32_t status = 0;
    CUDA_TRY(cudaMemcpy(&status, sd->search.status, 4, cudaMemcpyDeviceToHost));
    if (status != 0) return fail(CSE_ESTATE, "device consistency check failed (candidate list overflow)");
    sh->in_round = true;
    *rounds_left = sd->rounds - sh->rounds_done;
    return CSE_OK;
}

int cse_shard_best_list(const cse_result* r, int32_t mat, uint64_t round_key, int32_t* list, int32_t* len) {
    if (!r || !r->shard || !list || !len) return fail(CSE_EINVAL, "not a shard, or NULL output");
    const SearchDev* sd = r->sd;
    if (mat < 0 || mat >= sd->n_mats) return fail(CSE_EINVAL, "matrix index out of range");
    const int win = (int)(round_key & 0xFFFFFFFFu) - r->shard->offset;
    if (win < 0 || win >= sd->n_proc) return fail(CSE_EINVAL, "the key's process is not in this shard");
    const DevMat& M = sd->mats[mat];
    int32_t n = 0;
    CUDA_TRY(cudaMemcpy(&n, M.state + (size_t)win * M.state_words + H_BEST_LEN, 4, cudaMemcpyDeviceToHost));
    if (n < 0 || n > sd->cap) return fail(CSE_ESTATE, "corrupt best-list length");
    if (n > 0) CUDA_TRY(cudaMemcpy(list, M.best_list + (size_t)win * sd->cap, (size_t)n * 4, cudaMemcpyDeviceToHost));
    *len = n;
    return CSE_OK;
}

int cse_shard_share(cse_result* r, const uint64_t* keys, const int32_t* lists, const int32_t* lens) {
    if (!r || !r->shard || !keys) return fail(CSE_EINVAL, "not a shard, or NULL keys");
    ShardState* sh = r->shard;
    SearchDev* sd = r->sd;
    Batch* B = r->batch;
    if (!sh->in_round) return fail(CSE_EINVAL, "no round to complete (cse_shard_round first)");
    cudaStream_t st = B->stream;
    for (int k = 0; k < sd->n_mats; k++) {
        const DevMat& M = sd->mats[k];
        const int win = (int)(keys[k] & 0xFFFFFFFFu) - sh->offset;
        const bool local = win >= 0 && win < sd->n_proc;
        if (keys[k] != ~0ull && (keys[k] & 0xFFFFFFFFu) >= (uint64_t)sh->total)
            return fail(CSE_EINVAL, "a key names a process outside the search");
        if (!local && keys[k] != ~0ull) {
            if (!lists || !lens || lens[k] < 0 || lens[k] > sd->cap)
                return fail(CSE_EINVAL, "another shard's winner needs its list and length");
            CUDA_TRY(cudaMemcpyAsync((void*)M.ext_list, lists + (size_t)k * sd->cap, (size_t)lens[k] * 4,
                                     cudaMemcpyHostToDevice, st));
            CUDA_TRY(cudaMemcpyAsync((void*)M.ext_len, &lens[k], 4, cudaMemcpyHostToDevice, st));
        }
        CUDA_TRY(cudaMemcpyAsync(M.round_min, &keys[k], 8, cudaMemcpyHostToDevice, st));
    }
    cudaError_t e = launch_share(B->ls.d_mats, B->ls.d_searches, 1, B->ls.d_work, 3 * (int)B->ls.groups.size(), st);
    if (e != cudaSuccess) return fail(CSE_ECUDA, std::string("share launch: ") + cudaGetErrorString(e));
    sh->rounds_done++;
    sh->in_round = false;
    B->rounds = sh->rounds_done;
    if (sh->rounds_done == sd->rounds) CUDA_TRY(cudaEventRecord(B->ev_end, st));
    CUDA_TRY(cudaStreamSynchronize(st));  // the caller's key and list buffers may be reused on return
    return CSE_OK;
}

int cse_result_launches(const cse_result* r, int32_t* kernels, int32_t* searches_in_launch) {
    if (!r || !r->sd) return fail(CSE_EINVAL, "NULL result");
    const Batch* B = r->batch;
    int per_round = 1;  // the share kernel, then per class one launch (two on the process-per-CTA engine)
    if (B)
        for (const auto& g : B->ls.groups) per_round += g.cta ? 2 : 1;
    if (kernels) *kernels = B ? (B->persistent ? 1 : B->rounds * per_round) : 0;
    if (searches_in_launch) *searches_in_launch = B ? (int32_t)B->ls.searches.size() : 0;
    return CSE_OK;
}

void cse_result_free(cse_result* r) {
    if (!r) return;
    Batch* B = r->batch;
    if (B && r->shard) {
        cudaStreamSynchronize(B->stream);  // a shard records its end event only after its last boundary
    } else if (B) {
        cudaEventSynchronize(B->ev_end);
    }
    search_free(r->sd);
    delete r->shard;
    delete r;
    if (B && --B->refs == 0) {
        B->release();
        delete B;
    }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// server worker
// ---------------------------------------------------------------------------
static void server_finish(cse_server* sv, Request* q) {
    const auto now = std::chrono::steady_clock::now();
    if (q->status == CSE_OK) {
        q->res = new (std::nothrow) cse_result();
        if (!q->res) {
            q->status = CSE_ENOMEM;
            q->error = "host allocation";
        } else {
            q->sd->stream = nullptr;  // freed later on the default stream: its kernels are done
            q->res->sd = q->sd;
            q->res->latency_ms = std::chrono::duration<double, std::milli>(now - q->t_submit).count();
            q->sd = nullptr;
            sv->latencies_ms.push_back(q->res->latency_ms);
            sv->steps_done += (int64_t)q->res->sd->n_mats * q->res->sd->n_proc * q->res->sd->budget;
            sv->t_last = now;
        }
    }
    if (q->sd) {
        search_free(q->sd);
        q->sd = nullptr;
    }
    q->done = true;
}

static void server_loop(cse_server* sv) {
    cudaSetDevice(sv->device);
    LaunchSet ls;
    bool dirty = true;
    while (true) {
        std::vector<Request*> admitted;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_work.wait(lk, [&] { return sv->stop || !sv->pending.empty() || !sv->active.empty(); });
            if (sv->stop) break;
            // FIFO admission by device footprint, at a round boundary; a
            // request that does not fit waits, unless nothing else would run
            while (!sv->pending.empty()) {
                Request* q = sv->pending.front();
                const bool others = !sv->active.empty() || !admitted.empty();
                if (others && (sv->used_bytes + q->bytes > sv->hbm_budget ||
                                            sv->active_units + q->units > sv->max_units ||
                                            sv->used_smem + q->smem > sv->smem_budget))
                    break;
                sv->pending.pop_front();
                sv->used_bytes += q->bytes;
                sv->active_units += q->units;
                sv->used_smem += q->smem;
                admitted.push_back(q);
            }
        }
        std::vector<Request*> finished;
        for (Request* q : admitted) {
            const int rc = search_create(q->scheme, &q->mix, q->n_proc, q->seed, q->budget, sv->opts, sv->stream, &q->sd);
            if (rc) {
                q->status = rc;
                q->error = g_err;
                finished.push_back(q);
            } else if (q->sd->rounds == 0) {
                finished.push_back(q);
            } else {
                std::lock_guard<std::mutex> lk(sv->mu);
                sv->active.push_back(q);
                dirty = true;
            }
        }
        std::vector<Request*> act;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            act = sv->active;
        }
        int err = CSE_OK;
        std::string msg;
        if (!act.empty()) {
            if (dirty) {
                if (ls.d_params) cudaFreeAsync(ls.d_params, sv->stream);
                ls = LaunchSet();
                std::vector<SearchDev*> sds;
                for (Request* q : act) sds.push_back(q->sd);
                err = build_launch(sds, (int)sv->opts.procs_per_cta, nullptr, sv->stream, &ls);
                if (err) msg = g_err;
                dirty = false;
            }
            if (err == CSE_OK) {
                NvtxRange nvtx("cse_server_round");
                cudaError_t e = enqueue_round(ls, sv->stream, nullptr, nullptr, nullptr);
                if (e == cudaSuccess) e = cudaStreamSynchronize(sv->stream);
                if (e != cudaSuccess) {
                    err = CSE_ECUDA;
                    msg = std::string("round: ") + cudaGetErrorString(e);
                }
            }
        }
        std::lock_guard<std::mutex> lk(sv->mu);
        if (!act.empty()) {
            sv->rounds_run++;
            sv->max_active = std::max(sv->max_active, (int)act.size());
        }
        for (Request* q : act) {
            if (err) {
                q->status = err;
                q->error = msg;
            } else if (q->cancel) {
                q->status = CSE_ECANCELED;
                q->error = "cancelled";
            } else if (++q->sd->rounds_done < q->sd->rounds) {
                continue;
            }
            finished.push_back(q);
            sv->active.erase(std::find(sv->active.begin(), sv->active.end(), q));
            dirty = true;
        }
        for (Request* q : finished) {
            sv->active_units -= q->units;
            sv->used_smem -= q->smem;
            server_finish(sv, q);
            // a finished search's device block stays with its result (and in
            // the budget) until the client waits for it
            if (!q->res) sv->used_bytes -= q->bytes;
        }
        if (!finished.empty()) sv->cv_done.notify_all();
    }
    if (ls.d_params) cudaFreeAsync(ls.d_params, sv->stream);
    cudaStreamSynchronize(sv->stream);
}

extern "C" {

int cse_server_create(const cse_opts* opts_in, uint64_t hbm_budget_bytes, int64_t max_active_processes,
                      cse_server** out) {
    if (!out) return fail(CSE_EINVAL, "out is NULL");
    *out = nullptr;
    cse_opts opts;
    int rc = check_opts(opts_in, &opts);
    if (rc) return rc;
    opts.flags &= CSE_FLAG_TRACE | CSE_FLAG_GI_SHARED_COINS;
    if (opts.share_interval == 0)
        return fail(CSE_EINVAL, "the server admits requests at round boundaries of the step clock: share_interval >= 1");
    if (max_smem_per_block() <= 0) return fail(CSE_ECUDA, "no CUDA device");
    cse_server* sv = new (std::nothrow) cse_server();
    if (!sv) return fail(CSE_ENOMEM, "host allocation");
    sv->opts = opts;
    cudaGetDevice(&sv->device);
    if (hbm_budget_bytes) {
        sv->hbm_budget = hbm_budget_bytes;
    } else {  // default: 85% of the device memory free at creation
        size_t free_b = 0, total_b = 0;
        sv->hbm_budget = cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && free_b > 0
                             ? (uint64_t)(free_b / 20 * 17)
                             : UINT64_MAX;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, sv->device);
    // a wave: one process per resident warp (32 per SM).  The process cap
    // (default kServerWaves waves) also sets the shared-memory cap: as many
    // waves of the GPU's shared memory.
    const int64_t wave = (int64_t)32 * std::max(sms, 1);
    sv->max_units = max_active_processes > 0 ? max_active_processes : (int64_t)kServerWaves * wave;
    const int64_t waves = std::max<int64_t>(1, (sv->max_units + wave - 1) / wave);
    int smem_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, sv->device);
    sv->smem_budget = (uint64_t)waves * (uint64_t)std::max(sms, 1) * (uint64_t)std::max(smem_sm, 1);
    cudaError_t e = cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete sv;
        return fail(CSE_ECUDA, std::string("stream: ") + cudaGetErrorString(e));
    }
    sv->worker = std::thread(server_loop, sv);
    *out = sv;
    return CSE_OK;
}

int cse_server_submit(cse_server* sv, const cse_scheme* s, const cse_strategy_mix* mix, int32_t n_proc,
                      uint64_t seed, int64_t step_budget, uint64_t* ticket) {
    if (!sv || !ticket) return fail(CSE_EINVAL, "NULL server or ticket");
    SearchDev tmp;
    uint64_t w;
    std::vector<size_t> of;
    int rc = search_plan(s, mix, n_proc, step_budget, sv->opts, &tmp, &w, &of);
    if (rc) return rc;
    Request* q = new (std::nothrow) Request();
    if (!q) return fail(CSE_ENOMEM, "host allocation");
    q->scheme = s;
    q->mix = *mix;
    q->n_proc = n_proc;
    q->seed = seed;
    q->budget = step_budget;
    q->bytes = tmp.bytes;
    q->units = (int64_t)tmp.n_mats * tmp.n_proc;
    for (int k = 0; k < tmp.n_mats; k++)  // a slice per process of every shared-memory matrix
        if (!tmp.gm[k]) q->smem += (uint64_t)tmp.mats[k].gml.per_warp * (uint64_t)n_proc;
    q->t_submit = std::chrono::steady_clock::now();
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) {
        delete q;
        return fail(CSE_EBUSY, "server is stopping");
    }
    if (sv->pending.size() >= kServerMaxPending) {
        delete q;
        return fail(CSE_EBUSY, "server queue is full");
    }
    q->ticket = sv->next_ticket++;
    if (!sv->any) {
        sv->any = true;
        sv->t_first = q->t_submit;
    }
    sv->pending.push_back(q);
    sv->by_ticket[q->ticket] = q;
    *ticket = q->ticket;
    sv->cv_work.notify_one();
    return CSE_OK;
}

int cse_server_cancel(cse_server* sv, uint64_t ticket) {
    if (!sv) return fail(CSE_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->by_ticket.find(ticket);
    if (it == sv->by_ticket.end()) return fail(CSE_EINVAL, "unknown ticket");
    Request* q = it->second;
    if (q->done) return fail(CSE_EINVAL, "the request has already finished");
    auto pos = std::find(sv->pending.begin(), sv->pending.end(), q);
    if (pos != sv->pending.end()) {  // still queued: nothing on the device yet
        sv->pending.erase(pos);
        q->status = CSE_ECANCELED;
        q->error = "cancelled";
        q->done = true;
        sv->cv_done.notify_all();
    } else {
        q->cancel = true;  // running: the worker retires it at the next round boundary
        sv->cv_work.notify_one();
    }
    return CSE_OK;
}

int cse_server_wait(cse_server* sv, uint64_t ticket, int64_t timeout_us, cse_result** out) {
    if (!sv || !out) return fail(CSE_EINVAL, "NULL server or output");
    *out = nullptr;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->by_ticket.find(ticket);
    if (it == sv->by_ticket.end()) return fail(CSE_EINVAL, "unknown ticket");
    Request* q = it->second;
    auto ready = [&] { return q->done; };
    if (timeout_us < 0) {
        sv->cv_done.wait(lk, ready);
    } else if (!sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
        return fail(CSE_ETIMEOUT, "request not finished within the timeout");
    }
    sv->by_ticket.erase(it);
    const int st = q->status;
    const std::string err = q->error;
    *out = q->res;
    if (q->res) sv->used_bytes -= q->bytes;  // the result, and its device memory, are the caller's now
    delete q;
    if (st != CSE_OK) return fail(st, err);
    return CSE_OK;
}

int cse_server_stats(cse_server* sv, double* p50_ms, double* p99_ms, double* steps_per_s, int32_t* completed) {
    if (!sv) return fail(CSE_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(sv->mu);
    std::vector<double> v = sv->latencies_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) -> double {
        if (v.empty()) return 0.0;
        size_t i = (size_t)std::ceil(p * (double)v.size()) - 1;
        return v[std::min(i, v.size() - 1)];
    };
    if (p50_ms) *p50_ms = pct(0.50);
    if (p99_ms) *p99_ms = pct(0.99);
    if (steps_per_s) {
        const double s = sv->any ? std::chrono::duration<double>(sv->t_last - sv->t_first).count() : 0.0;
        *steps_per_s = s > 0 ? (double)sv->steps_done / s : 0.0;
    }
    if (completed) *completed = (int32_t)v.size();
    return CSE_OK;
}

int cse_server_peak(cse_server* sv, int32_t* max_active_searches, int32_t* rounds) {
    if (!sv) return fail(CSE_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (max_active_searches) *max_active_searches = sv->max_active;
    if (rounds) *rounds = sv->rounds_run;
    return CSE_OK;
}

void cse_server_free(cse_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    for (Request* q : sv->active) search_free(q->sd);
    for (auto& kv : sv->by_ticket) {
        Request* q = kv.second;
        if (q->res) cse_result_free(q->res);
        else if (q->sd && std::find(sv->active.begin(), sv->active.end(), q) == sv->active.end()) search_free(q->sd);
        delete q;
    }
    cudaStreamDestroy(sv->stream);
    delete sv;
}

}  // extern "C"
