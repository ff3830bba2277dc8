// Instantiations and launchers of the process-per-CTA engine (cse_cta.cuh)
// for large matrices: one round kernel per word width, then the warp engine
// over the processes it handed back.

#include "cse_cta.cuh"

namespace cse {

static int align16_cta(int x) { return (x + 15) & ~15; }

static CtaLayout cta_layout_for(int W, int cap, int ms, int pln, int nw) {
    CtaLayout L{};
    int o = 0;
    L.off_cold = o;
    o = align16_cta(o + (int)sizeof(Cold));
    L.off_sh = o;
    o = align16_cta(o + (int)sizeof(CtaShared));
    L.off_pn = o;
    o = align16_cta(o + cap * W * 8);
    L.off_cand = o;
    o = align16_cta(o + ms * 4);
    L.off_pl = o;
    o = align16_cta(o + ms * 2);
    L.off_aw = o;
    o = align16_cta(o + 2 * ms);
    L.off_hs = o;
    o = align16_cta(o + cap * 2);
    L.off_he = o;
    o = align16_cta(o + cap * 2);
    L.off_vb = o;
    o = align16_cta(o + cap * 2);
    L.off_pb = o;
    o = align16_cta(o + cap * 2);
    L.off_lct = o;
    o = align16_cta(o + cap * 2);
    L.off_g = o;
    o = align16_cta(o + cap * 4);
    L.off_lcw = o;
    o = align16_cta(o + nw * cap * 2);
    L.off_f = o;
    o = align16_cta(o + cap * 4);
    L.off_pln = o;
    o = align16_cta(o + pln * 8);
    L.ms = ms;
    L.pln_cap = pln;
    L.bytes = o;
    L.nw = nw;
    return L;
}

// The list capacity is the largest (up to 32 kCtaSeg nw, in steps of 512)
// that leaves the planes room for a typical step: about 2 ms / 64 + cap / 2
// blocks of 6 planes.  16 warps: two CTAs per SM (the register file's
// limit); 8 warps: four CTAs per SM if a useful layout fits, else three.
CtaLayout make_cta_layout(int W, int cap, int mmax, int list_cap, int min_list, int smem_per_block, int nw) {
    int dev = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
        return CtaLayout{};
    if (W < 1 || W > kMaxW || (nw != 8 && nw != 16)) return CtaLayout{};
    const int ms_max = 32 * kCtaSeg * nw;
    for (int ctas = nw == 16 ? 2 : 4; ctas >= 2; ctas--) {
        const int budget = std::min(smem_per_block, per_sm / ctas - 1024);
        int ms = std::min(mmax, ms_max);
        if (list_cap > 0) ms = std::min(ms, list_cap);
        const bool fixed = list_cap > 0;
        for (;;) {
            const CtaLayout base = cta_layout_for(W, cap, ms, 0, nw);
            const int pln = (budget - base.bytes) / 8;
            const int want = (2 * ms / 64 + cap / 2) * 6;
            if (pln >= want || (fixed && pln >= 64)) {
                const int most = ((2 * ms + 63 * cap) / 64 + 1) * 8;  // no step needs more
                CtaLayout L = cta_layout_for(W, cap, ms, std::min(pln, most), nw);
                L.min_m = min_list > 0 ? min_list : kCtaMinList;
                return L;
            }
            if (ms <= 1024) break;
            ms = std::max(1024, ms - 512);
        }
    }
    return CtaLayout{};
}

template <int W, int NW>
static cudaError_t launch_cta_wn(const DevMat* mats, int n_mats, const DevSearch* searches, int total_units,
                                 int* work3, int* redo_list, const CtaLayout& CL, int redo_ppc, cudaStream_t stream,
                                 bool prepare_only) {
    if (prepare_only) {
        cudaError_t e = raise_max_dynamic_smem((const void*)cta_round_kernel<W, NW>, CL.bytes);
        if (e != cudaSuccess) return e;
        return prepare_round(W, true, false, WarpLayout{}, redo_ppc);
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cta_round_kernel<W, NW>, 32 * NW, CL.bytes);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::max(1LL, std::min((long long)total_units, (long long)std::max(sms, 1) * std::max(per_sm, 1)));
    cta_round_kernel<W, NW><<<grid, 32 * NW, CL.bytes, stream>>>(mats, n_mats, searches, total_units, work3,
                                                                 redo_list, CL);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_round_list(W, mats, n_mats, searches, total_units, redo_list, work3 + 2, work3 + 1, redo_ppc,
                             stream);
}

template <int W>
static cudaError_t launch_cta_w(const DevMat* mats, int n_mats, const DevSearch* searches, int total_units,
                                int* work3, int* redo_list, const CtaLayout& CL, int redo_ppc, cudaStream_t stream,
                                bool prepare_only) {
    // the layouts of this build are 16 warps wide (make_cta_layout's default)
    if (CL.nw != kCtaWarps) return cudaErrorInvalidValue;
    return launch_cta_wn<W, kCtaWarps>(mats, n_mats, searches, total_units, work3, redo_list, CL, redo_ppc, stream,
                                       prepare_only);
}

static cudaError_t launch_cta(int W, const DevMat* mats, int n_mats, const DevSearch* searches, int total_units,
                              int* work3, int* redo_list, const CtaLayout& CL, int redo_ppc, cudaStream_t stream,
                              bool prep) {
    switch (W) {
        case 1: return launch_cta_w<1>(mats, n_mats, searches, total_units, work3, redo_list, CL, redo_ppc, stream, prep);
        case 2: return launch_cta_w<2>(mats, n_mats, searches, total_units, work3, redo_list, CL, redo_ppc, stream, prep);
        case 3: return launch_cta_w<3>(mats, n_mats, searches, total_units, work3, redo_list, CL, redo_ppc, stream, prep);
        case 4: return launch_cta_w<4>(mats, n_mats, searches, total_units, work3, redo_list, CL, redo_ppc, stream, prep);
        case 5: return launch_cta_w<5>(mats, n_mats, searches, total_units, work3, redo_list, CL, redo_ppc, stream, prep);
        case 6: return launch_cta_w<6>(mats, n_mats, searches, total_units, work3, redo_list, CL, redo_ppc, stream, prep);
        case 7: return launch_cta_w<7>(mats, n_mats, searches, total_units, work3, redo_list, CL, redo_ppc, stream, prep);
        case 8: return launch_cta_w<8>(mats, n_mats, searches, total_units, work3, redo_list, CL, redo_ppc, stream, prep);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_round_cta(int W, const DevMat* mats, int n_mats, const DevSearch* searches, int total_units,
                             int* work3, int* redo_list, const CtaLayout& CL, int redo_ppc, cudaStream_t stream) {
    return launch_cta(W, mats, n_mats, searches, total_units, work3, redo_list, CL, redo_ppc, stream, false);
}

cudaError_t prepare_round_cta(int W, const CtaLayout& CL, int redo_ppc) {
    return launch_cta(W, nullptr, 0, nullptr, 0, nullptr, nullptr, CL, redo_ppc, nullptr, true);
}

}  // namespace cse
