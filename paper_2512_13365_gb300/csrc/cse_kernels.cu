// Kernels of the parallel heuristic CSE search on sm_103a other than the step
// engine (cse_engine.cuh): ingest, the sharing boundary, the Brent check, and
// the host-side launchers; this unit instantiates the engine with independent
// coins per pair.

#include "cse_engine.cuh"
#include "cse_share.cuh"

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
__global__ void share_kernel(const DevMat* __restrict__ mats, const DevSearch* __restrict__ searches,
                             int* __restrict__ work, int n_work) {
    // the round kernels' work counters, for the next round
    if (blockIdx.x == 0 && (int)threadIdx.x < n_work) work[threadIdx.x] = 0;
    share_one(mats, &searches[blockIdx.x]);
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
    // the weight bytes of every position (the HBM path reads them 8 bytes at
    // a time from an 8-byte boundary, up to 72 bytes past a block's start)
    o = align16(o + 2 * mmax + (planes ? 80 : 0));
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
        L.off_bv = o;
        o = align16(o + max_blocks * 2);
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
