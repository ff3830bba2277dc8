// The sharing boundary (Section 3.5.2) of one search, shared by the share
// kernel (cse_kernels.cu) and the persistent batch kernel (cse_batch.cu).

#pragma once

#include "cse_engine.cuh"

namespace cse {

// The sharing boundary of one search, by the threads of one CTA (one warp
// per matrix at a time).
static __device__ __forceinline__ void share_one(const DevMat* __restrict__ mats, const DevSearch* __restrict__ S) {
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

}  // namespace cse
