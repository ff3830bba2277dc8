// The persistent batch kernel (CSE_FLAG_PERSISTENT): every round and sharing
// boundary of every search of a batch in one cooperative launch.

#include "cse_engine.cuh"
#include "cse_share.cuh"

namespace cse {

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
// on the shared-memory engine with at most 2 words per column, every one on
// the 2-word engine (the host gives matrices of 1 word the 2-word kernel
// width: one engine keeps the register allocation of the round kernel, where
// two inlined engines spilled about three times as much): per round, every
// warp takes processes from the round's work counter (work[round]); then a
// grid barrier, the sharing boundary of every search (CTA b takes searches
// b, b + grid, ...), and another barrier.  Each search keeps its own clock,
// so the results are those of the searches run alone.
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

}  // namespace cse
