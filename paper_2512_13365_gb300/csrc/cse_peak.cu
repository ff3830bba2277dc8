// Integer-pipe microbenchmarks (cse_int_peak): the measured peaks behind the
// roofline of the step engine, which is integer bitset work (AND, popcount,
// add, compare) and not a dense contraction.
//
// Every thread runs kChains independent dependency chains of one instruction
// mix, written as inline PTX so that the compiler keeps each instruction, for
// `iters` iterations.  The grid holds blocks_per_sm blocks of 128 threads per
// SM, all resident at once, so every SM is busy for the whole launch; each
// block records its own clock64() span, and ops per clock per SM = ops of the
// launch / (SMs x mean block span).
//
//   kind 0  LOP3 (3-input XOR) + IADD3: 2 lane-ops per chain step
//   kind 1  AND + POPC + IADD (the pair-count core): 3 lane-ops per step,
//           of which one POPC
//   kind 2  IMAD (32-bit multiply-add, the Philox round's low product)
//   kind 3  IMAD.HI (32-bit multiply-high, the Philox round's high product)
//   kind 4  LOP3 alone (3-input XOR)
//   kind 5  IADD3 alone (3-input add; two PTX adds that the compiler fuses)

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "cse.h"
#include "cse_internal.h"

namespace cse {

constexpr int kChains = 8;
constexpr int kPeakThreads = 128;

template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) int_peak_kernel(uint32_t seed, long long iters,
                                                                 uint32_t* __restrict__ sink,
                                                                 long long* __restrict__ span) {
    uint32_t x[kChains], y[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) {
        x[c] = seed * (threadIdx.x + 1u) + (uint32_t)c * 0x9E3779B9u;
        y[c] = (seed ^ blockIdx.x) + (uint32_t)c * 0x7F4A7C15u;
    }
    const uint32_t k1 = seed | 1u, k2 = seed * 3u + 7u;
    __syncthreads();
    const long long t0 = clock64();
    for (long long it = 0; it < iters; it++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) {
            if (KIND == 0) {
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[c]) : "r"(y[c]), "r"(k1));
                asm volatile("add.u32 %0, %0, %1;" : "+r"(y[c]) : "r"(x[c]));
            } else if (KIND == 1) {
                uint32_t t, p;
                asm volatile("and.b32 %0, %1, %2;" : "=r"(t) : "r"(x[c]), "r"(y[c]));
                asm volatile("popc.b32 %0, %1;" : "=r"(p) : "r"(t));
                asm volatile("add.u32 %0, %0, %1;" : "+r"(x[c]) : "r"(p));
            } else if (KIND == 2) {
                asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(k1), "r"(y[c]));
            } else if (KIND == 3) {
                asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(x[c]) : "r"(k2));
            } else if (KIND == 4) {
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[c]) : "r"(y[c]), "r"(k1));
            } else {  // one 3-input add (the compiler fuses the two adds into one IADD3)
                uint32_t t;
                asm volatile("add.u32 %0, %1, %2;" : "=r"(t) : "r"(x[c]), "r"(k1));
                asm volatile("add.u32 %0, %1, %2;" : "=r"(x[c]) : "r"(t), "r"(y[c]));
            }
        }
    }
    const long long t1 = clock64();
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; c++) acc ^= x[c] ^ y[c];
    if (acc == 0x12345678u) sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;  // keeps the work alive
    __syncthreads();
    if (threadIdx.x == 0) span[blockIdx.x] = t1 - t0;
}

// Lane-ops per chain step of each kind.
// Lane-ops are counted as instructions: kind 5's two adds run as one IADD3.
static const int kOpsPerStep[6] = {2, 3, 1, 1, 1, 1};

}  // namespace cse

using namespace cse;

extern "C" int cse_int_peak(int32_t kind, int64_t iters, void* cuda_stream, double* ops_per_clk_per_sm,
                            double* lane_ops_per_s, double* seconds) {
    if (kind < 0 || kind > 5) return set_error(CSE_EINVAL, "kind must be 0..5");
    if (iters < 1 || iters > (int64_t)1 << 40) return set_error(CSE_EINVAL, "iters must be in [1, 2^40]");
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms <= 0) return set_error(CSE_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    const void* fn = kind == 0   ? (const void*)int_peak_kernel<0>
                     : kind == 1 ? (const void*)int_peak_kernel<1>
                     : kind == 2 ? (const void*)int_peak_kernel<2>
                     : kind == 3 ? (const void*)int_peak_kernel<3>
                     : kind == 4 ? (const void*)int_peak_kernel<4>
                                 : (const void*)int_peak_kernel<5>;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPeakThreads, 0);
    if (e != cudaSuccess || per_sm <= 0) return set_error(CSE_ECUDA, "occupancy query failed");
    per_sm = per_sm > 8 ? 8 : per_sm;  // 32 warps per SM: enough to fill every scheduler
    const int grid = sms * per_sm;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    void* buf = nullptr;
    const size_t sink_bytes = (size_t)grid * kPeakThreads * 4, span_bytes = (size_t)grid * 8;
    e = cudaMalloc(&buf, sink_bytes + span_bytes);
    if (e != cudaSuccess) return set_error(CSE_ENOMEM, std::string("peak buffers: ") + cudaGetErrorString(e));
    uint32_t* sink = (uint32_t*)buf;
    long long* span = (long long*)((char*)buf + sink_bytes);
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
    switch (kind) {
        case 0: int_peak_kernel<0><<<grid, kPeakThreads, 0, st>>>(0x2545F491u, iters, sink, span); break;
        case 1: int_peak_kernel<1><<<grid, kPeakThreads, 0, st>>>(0x2545F491u, iters, sink, span); break;
        case 2: int_peak_kernel<2><<<grid, kPeakThreads, 0, st>>>(0x2545F491u, iters, sink, span); break;
        case 3: int_peak_kernel<3><<<grid, kPeakThreads, 0, st>>>(0x2545F491u, iters, sink, span); break;
        case 4: int_peak_kernel<4><<<grid, kPeakThreads, 0, st>>>(0x2545F491u, iters, sink, span); break;
        default: int_peak_kernel<5><<<grid, kPeakThreads, 0, st>>>(0x2545F491u, iters, sink, span); break;
    }
    e = cudaGetLastError();
    cudaEventRecord(b, st);
    std::vector<long long> h(grid);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), span, span_bytes, cudaMemcpyDeviceToHost);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(buf);
    if (e != cudaSuccess) return set_error(CSE_ECUDA, std::string("peak kernel: ") + cudaGetErrorString(e));
    double mean = 0.0;
    for (long long v : h) mean += (double)v;
    mean /= (double)grid;
    const double ops = (double)grid * kPeakThreads * (double)iters * kChains * kOpsPerStep[kind];
    if (ops_per_clk_per_sm) *ops_per_clk_per_sm = mean > 0 ? ops / ((double)sms * mean) : 0.0;
    if (lane_ops_per_s) *lane_ops_per_s = ms > 0 ? ops / (ms * 1e-3) : 0.0;
    if (seconds) *seconds = ms * 1e-3;
    return CSE_OK;
}
