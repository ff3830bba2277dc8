// cse_search_static: a search that allocates no device memory.
//
// Who needs it: code that must not call cudaMalloc or a caching allocator at
// the moment it runs a search -- for example a host that has handed all
// device memory to another framework's pool, a real-time loop where an
// allocation could block on a device-wide synchronisation, or a plugin that
// is only given device pointers by its host application.  Such a caller
// loads the scheme beforehand (cse_scheme_load) and passes device buffers
// for the results; every other byte the search needs (process states, best
// lists, sharing snapshots, launch parameters) comes from one file-scope
// device array of CSE_STATIC_SCRATCH_BYTES, which every GPU that loads this
// library holds until the process exits.
//
// The kernels are the same round and share kernels as cse_search; only the
// scratch comes from the static array.

#include <algorithm>
#include <climits>
#include <mutex>
#include <string>
#include <vector>

#include "cse.h"
#include "cse_internal.h"

using namespace cse;

namespace {

// The scratch.  Its host-side name is only a stand-in for the symbol: the
// device address comes from cudaGetSymbolAddress, per device.
__device__ __align__(256) unsigned char g_static_scratch[CSE_STATIC_SCRATCH_BYTES];

std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
unsigned char* g_static_ptr[kMaxDevices] = {};

size_t take(size_t& off, size_t bytes) {
    const size_t o = off;
    off = (off + bytes + 255) & ~(size_t)255;
    return o;
}

// Device address of the scratch on the current device (looked up once per
// device, with that device current).
int scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(CSE_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_error(CSE_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return set_error(CSE_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_static_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_static_ptr[dev];
    return CSE_OK;
}

}  // namespace

extern "C" int cse_search_static(const cse_scheme* s, const cse_strategy_mix* mix, int32_t n_proc, uint64_t seed,
                                 int64_t budget, const cse_opts* opts_in, void* cuda_stream, int32_t* d_lists,
                                 int32_t* d_meta) {
    // ---- arguments (the same rules as cse_search)
    if (!s || !mix || !d_lists || !d_meta) return set_error(CSE_EINVAL, "NULL scheme, mix or output buffer");
    cse_opts opts;
    if (opts_in)
        opts = *opts_in;
    else
        cse_opts_default(&opts);
    if (opts.share_interval < 1 || opts.share_permille > 1000 || opts.patience_rounds != 0 ||
        (opts.flags & ~(uint32_t)(CSE_FLAG_TRACE | CSE_FLAG_GI_SHARED_COINS)) != 0 || opts.col_cap > CSE_MAX_COLS ||
        opts.procs_per_cta > 4)
        return set_error(CSE_EINVAL, "invalid options (this entry point runs the step clock only: share_interval >= 1, "
                                     "patience_rounds 0, and takes no CSE_FLAG_GRAPH)");
    const uint64_t wsum = (uint64_t)mix->w_gi + mix->w_ga + mix->w_gr + mix->w_wr + mix->w_mix + mix->w_g + mix->w_gp;
    if (wsum == 0 || wsum > 0xFFFFFFFFull) return set_error(CSE_EINVAL, "strategy weights: sum must be in [1, 2^32)");
    if (n_proc < 1 || n_proc > (1 << 20)) return set_error(CSE_EINVAL, "n_processes must be in [1, 2^20]");
    if (budget < 0 || budget >= INT32_MAX) return set_error(CSE_EINVAL, "step_budget must be in [0, 2^31)");
    const int cap = (int)opts.col_cap, nm = s->n_mats;
    for (int k = 0; k < nm; k++)
        if (s->cols[k] >= cap) return set_error(CSE_EINVAL, "col_cap must exceed every matrix's column count");
    const int smem_max = max_smem_per_block();
    if (smem_max <= 0) return set_error(CSE_ECUDA, "no CUDA device");

    // ---- the carve-up of the scratch, checked against its size
    std::vector<DevMat> mats(nm);
    std::vector<char> gm(nm);
    std::vector<size_t> o_state(nm), o_best(nm), o_snap(nm), o_snapm(nm), o_rmin(nm), o_cnt(nm), o_curve(nm);
    size_t off = 0;
    for (int k = 0; k < nm; k++) {
        const WarpLayout own = make_layout(s->W[k], cap, s->mmax[k]);
        gm[k] = own.per_warp > kSmemPerWarpLimit;
        mats[k].gml = gm[k] ? make_layout(s->W[k], cap, s->mmax[k], true) : own;
        mats[k].state_words = gm[k] ? state_words_gm(mats[k].gml) : state_words(s->W[k], cap, s->mmax[k]);
        o_state[k] = take(off, (size_t)n_proc * mats[k].state_words * 4);
        o_best[k] = take(off, (size_t)n_proc * cap * 4);
        o_snap[k] = take(off, (size_t)cap * 4);
        o_snapm[k] = take(off, 8);
        o_rmin[k] = take(off, 8);
        o_cnt[k] = take(off, 64);
        o_curve[k] = take(off, (size_t)kCurvePoints * 4);
    }
    const size_t o_clock = take(off, 4), o_status = take(off, 4);
    const size_t o_mats = take(off, sizeof(DevMat) * nm), o_search = take(off, sizeof(DevSearch));
    const size_t o_pos = take(off, 4 * (size_t)nm);
    const size_t o_work = take(off, 4 * (size_t)nm);  // one round-kernel work counter per group (<= nm groups)
    if (off > (size_t)CSE_STATIC_SCRATCH_BYTES)
        return set_error(CSE_ENOMEM, "this search needs " + std::to_string(off) +
                                         " bytes of scratch; the static scratch holds " +
                                         std::to_string((size_t)CSE_STATIC_SCRATCH_BYTES) +
                                         " (use fewer processes or a smaller col_cap)");
    unsigned char* b = nullptr;
    int rc = scratch_address(&b);
    if (rc) return rc;
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    // ---- parameters: the matrices in launch order (classes of equal W and path)
    std::vector<int> order(nm);
    for (int k = 0; k < nm; k++) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return s->W[x] != s->W[y] ? s->W[x] < s->W[y] : gm[x] < gm[y];
    });
    DevSearch S{};
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
    S.share_thr = ((uint64_t)opts.share_permille << 32) / 1000u;
    S.clock = (int32_t*)(b + o_clock);
    S.status = (int32_t*)(b + o_status);
    S.mat_pos = (const int32_t*)(b + o_pos);
    S.n_mats = nm;
    S.trace = (opts.flags & CSE_FLAG_TRACE) ? 1 : 0;
    S.gi_shared = (opts.flags & CSE_FLAG_GI_SHARED_COINS) ? 1 : 0;
    struct Group { int W, begin, count, units, mmax; bool gm; WarpLayout L; int ppc; };
    std::vector<Group> groups;
    std::vector<DevMat> dm(nm);
    std::vector<int32_t> pos(nm);
    for (int q = 0; q < nm; q++) {
        const int k = order[q];
        DevMat& M = dm[q];
        M = mats[k];
        M.pn0 = s->d_pn0[k];
        M.cand0 = s->d_cand0[k];
        M.meta0 = s->d_meta0[k];
        M.rows = s->rows[k];
        M.nx = s->cols[k];
        M.W = s->W[k];
        M.wn = s->W[k];
        M.cap = cap;
        M.mmax = s->mmax[k];
        M.mat_index = k;
        M.n_proc = n_proc;
        M.search = 0;
        M.state = (uint32_t*)(b + o_state[k]);
        M.best_list = (int32_t*)(b + o_best[k]);
        M.snap = (int32_t*)(b + o_snap[k]);
        M.snap_meta = (int32_t*)(b + o_snapm[k]);
        M.round_min = (unsigned long long*)(b + o_rmin[k]);
        M.result = d_lists + (size_t)k * cap;  // results go straight to the caller's buffers
        M.result_meta = d_meta + 2 * (size_t)k;
        M.counters = (unsigned long long*)(b + o_cnt[k]);
        M.curve = (int32_t*)(b + o_curve[k]);
        pos[q] = q;
        if (groups.empty() || groups.back().W != M.W || groups.back().gm != (gm[k] != 0))
            groups.push_back({M.W, q, 0, 0, 0, gm[k] != 0, {}, 0});
        Group& g = groups.back();
        M.unit_base = g.units;
        g.count++;
        g.units += n_proc;
        g.mmax = std::max(g.mmax, M.mmax);
    }
    for (Group& g : groups) {
        g.L = g.gm ? WarpLayout{} : make_layout(g.W, cap, g.mmax);
        g.ppc = opts.procs_per_cta ? (int)opts.procs_per_cta : (g.gm ? 4 : 2);  // as cse_search
        if (!g.gm)
            while (g.ppc > 1 && (long long)g.L.per_warp * g.ppc > smem_max) g.ppc--;
        cudaError_t e = prepare_round(g.W, g.gm, S.gi_shared != 0, g.L, g.ppc);
        if (e != cudaSuccess) return set_error(CSE_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
    }

    // ---- initial values (the scratch keeps the previous call's contents)
    static const int32_t snap_init[2] = {INT_MAX, 0};
    DevMat* d_mats = (DevMat*)(b + o_mats);
    DevSearch* d_search = (DevSearch*)(b + o_search);
    cudaError_t e = cudaMemcpyAsync(d_mats, dm.data(), sizeof(DevMat) * nm, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_search, &S, sizeof(DevSearch), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_pos, pos.data(), 4 * (size_t)nm, cudaMemcpyHostToDevice, stream);
    for (int k = 0; k < nm && e == cudaSuccess; k++) {
        e = cudaMemsetAsync(b + o_rmin[k], 0xFF, 8, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_snapm[k], snap_init, 8, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_meta + 2 * k, s->d_meta0[k], 4, cudaMemcpyDeviceToDevice, stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_meta + 2 * k + 1, 0, 4, stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(b + o_cnt[k], 0, 64, stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(b + o_curve[k], 0xFF, (size_t)kCurvePoints * 4, stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(b + o_clock, 0, 4, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b + o_status, 0, 4, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b + o_work, 0, 4 * (size_t)nm, stream);
    if (e != cudaSuccess) return set_error(CSE_ECUDA, std::string("scratch set-up: ") + cudaGetErrorString(e));

    // ---- the rounds
    const int rounds = (int)((budget + opts.share_interval - 1) / opts.share_interval);
    for (int rd = 0; rd < rounds && e == cudaSuccess; rd++) {
        int* work = (int*)(b + o_work);
        for (size_t gi = 0; gi < groups.size(); gi++) {
            const Group& g = groups[gi];
            e = launch_round(g.W, g.gm, S.gi_shared != 0, d_mats + g.begin, g.count, d_search, g.units, work + gi,
                             g.L, g.ppc, stream);
            if (e != cudaSuccess) break;
        }
        if (e == cudaSuccess) e = launch_share(d_mats, d_search, 1, work, (int)groups.size(), stream);
    }
    if (e != cudaSuccess) return set_error(CSE_ECUDA, std::string("launch: ") + cudaGetErrorString(e));

    // ---- wait, then read the device-side consistency word
    int32_t status = 0;
    e = cudaMemcpyAsync(&status, b + o_status, 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return set_error(CSE_ECUDA, std::string("search: ") + cudaGetErrorString(e));
    if (status != 0) return set_error(CSE_ESTATE, "device consistency check failed (candidate list overflow)");
    return CSE_OK;
}
