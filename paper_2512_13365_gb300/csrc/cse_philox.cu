// The device Philox4x32-10 exposed for verification (cse_philox): the round
// function every draw of the step engine goes through (cse_engine.cuh),
// applied to a caller's counters.

#include <algorithm>

#include "cse_engine.cuh"

namespace cse {

__global__ void philox_kernel(const uint4* __restrict__ ctr, long long n, uint32_t k0, uint32_t k1,
                              uint4* __restrict__ out) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        uint4 c = ctr[q];
        philox(c.x, c.y, c.z, c.w, k0, k1);
        out[q] = c;
    }
}

cudaError_t launch_philox(const uint32_t* ctr, long long n, uint64_t seed, uint32_t* out, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (n + 255) / 256;
    const int grid = (int)std::max(1LL, std::min(want, (long long)std::max(sms, 1) * 8));
    philox_kernel<<<grid, 256, 0, stream>>>(reinterpret_cast<const uint4*>(ctr), n, (uint32_t)seed,
                                            (uint32_t)(seed >> 32), reinterpret_cast<uint4*>(out));
    return cudaGetLastError();
}

}  // namespace cse
