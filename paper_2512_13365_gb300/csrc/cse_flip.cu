// Random-flip mode (Section 3.5.3): M variants of a scheme, each the input
// with a random number of ternary flips, regenerated every iteration and
// searched side by side.
//
// The flip is the move of the flip graph the paper cites: terms l != m whose
// factor X agrees up to a sign (X_m = sigma X_l), Y and Z the other two
// factors, become Y_l + sigma Y_m and Z_m - Z_l; the sum over the terms of
// U_l (x) V_l (x) W_l, and with it every Brent equation (Section 3.1), is
// unchanged.  Only ternary flips are taken (the new Y_l and Z_m stay in
// {-1, 0, 1}) that keep both terms nonzero (the rank).
//
// Draws (Philox4x32-10, key = seed): variant v >= 1 of iteration `it`
// applies F = 1 + ((u * max_flips) >> 32) flips, u lane 0 of counter
// (v, it, FLIP << 20, 0); attempt a (at most 32 F, stopping at F flips)
// reads counter (v, it, FLIP << 20, a + 1): l = (u0 r) >> 32, m = (u1 (r-1))
// >> 32 (+1 if >= l), X = (u2 3) >> 32, (Y, Z) = (X+1, X+2) if u3 is even
// else (X+2, X+1), mod 3; an attempt that is not a ternary flip changes
// nothing.  Variant 0 is the input.

#include <string>

#include "cse_engine.cuh"

namespace cse {

constexpr uint32_t kPurposeFlip = 5;

// One warp per variant: copy the input into the variant's slot, then the
// flips, one after the other (each may use the previous one's result).
__global__ void flip_kernel(const int8_t* __restrict__ U, const int8_t* __restrict__ V,
                            const int8_t* __restrict__ W, int r, int lu, int lv, int lw, uint64_t seed,
                            int iteration, int max_flips, int8_t* __restrict__ oU, int8_t* __restrict__ oV,
                            int8_t* __restrict__ oW, int* __restrict__ flips) {
    const int v = blockIdx.x, lane = threadIdx.x;
    int8_t* f[3] = {oU + (size_t)v * r * lu, oV + (size_t)v * r * lv, oW + (size_t)v * r * lw};
    const int8_t* in[3] = {U, V, W};
    const int len[3] = {lu, lv, lw};
    for (int k = 0; k < 3; k++)
        for (int x = lane; x < r * len[k]; x += 32) f[k][x] = in[k][x];
    __syncwarp();
    if (v == 0 || r < 2 || max_flips < 1) {
        if (lane == 0) flips[v] = 0;
        return;
    }
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32), c2 = kPurposeFlip << 20;
    const int want = 1 + (int)scale32(philox_call((uint32_t)v, (uint32_t)iteration, c2, 0u, k0, k1).x,
                                      (uint32_t)max_flips);
    int done = 0;
    for (int a = 0; a < 32 * want && done < want; a++) {
        const uint4 d = philox_call((uint32_t)v, (uint32_t)iteration, c2, (uint32_t)(a + 1), k0, k1);
        const int l = (int)scale32(d.x, (uint32_t)r);
        int m = (int)scale32(d.y, (uint32_t)(r - 1));
        if (m >= l) m++;
        const int x = (int)scale32(d.z, 3u), side = (int)(d.w & 1u);
        const int y = (x + 1 + side) % 3, z = (x + 2 - side) % 3;
        // X_m = sigma X_l, X_l nonzero
        bool same = true, opp = true, nz = false;
        for (int i = lane; i < len[x]; i += 32) {
            const int a_ = f[x][(size_t)l * len[x] + i], b_ = f[x][(size_t)m * len[x] + i];
            same &= b_ == a_;
            opp &= b_ == -a_;
            nz |= a_ != 0;
        }
        same = __all_sync(FULL_MASK, same);
        opp = __all_sync(FULL_MASK, opp);
        nz = __any_sync(FULL_MASK, nz);
        if (!nz || !(same || opp)) continue;
        const int sigma = same ? 1 : -1;
        // the new Y_l and Z_m must be ternary and nonzero
        bool ok = true, ynz = false, znz = false;
        for (int i = lane; i < len[y]; i += 32) {
            const int t = f[y][(size_t)l * len[y] + i] + sigma * f[y][(size_t)m * len[y] + i];
            ok &= t >= -1 && t <= 1;
            ynz |= t != 0;
        }
        for (int i = lane; i < len[z]; i += 32) {
            const int t = f[z][(size_t)m * len[z] + i] - f[z][(size_t)l * len[z] + i];
            ok &= t >= -1 && t <= 1;
            znz |= t != 0;
        }
        ok = __all_sync(FULL_MASK, ok) && __any_sync(FULL_MASK, ynz) && __any_sync(FULL_MASK, znz);
        if (!ok) continue;
        for (int i = lane; i < len[y]; i += 32)
            f[y][(size_t)l * len[y] + i] = (int8_t)(f[y][(size_t)l * len[y] + i] + sigma * f[y][(size_t)m * len[y] + i]);
        for (int i = lane; i < len[z]; i += 32)
            f[z][(size_t)m * len[z] + i] = (int8_t)(f[z][(size_t)m * len[z] + i] - f[z][(size_t)l * len[z] + i]);
        __syncwarp();
        done++;
    }
    if (lane == 0) flips[v] = done;
}

}  // namespace cse

using namespace cse;

extern "C" int cse_flip_variants(int32_t m, int32_t n, int32_t p, int32_t r, const int8_t* U, const int8_t* V,
                                 const int8_t* W, int32_t n_variants, uint64_t seed, int32_t iteration,
                                 int32_t max_flips, int8_t* out_U, int8_t* out_V, int8_t* out_W, int32_t* flips,
                                 int64_t* brent_violations) {
    if (m < 1 || n < 1 || p < 1 || r < 1 || !U || !V || !W || !out_U || !out_V || !out_W || !flips)
        return set_error(CSE_EINVAL, "bad scheme dimensions or NULL argument");
    if (n_variants < 1 || n_variants > 4096 || iteration < 0 || max_flips < 0 || max_flips > (1 << 20))
        return set_error(CSE_EINVAL, "need 1 <= n_variants <= 4096, iteration >= 0, 0 <= max_flips <= 2^20");
    if ((int64_t)m * n > 4096 || (int64_t)n * p > 4096 || (int64_t)m * p > 4096 || r > 65536)
        return set_error(CSE_EINVAL, "scheme too large (m n, n p, m p <= 4096, r <= 65536)");
    for (int k = 0; k < 3; k++) {
        const int8_t* a = k == 0 ? U : k == 1 ? V : W;
        const int64_t len = (int64_t)r * (k == 0 ? m * n : k == 1 ? n * p : m * p);
        for (int64_t x = 0; x < len; x++)
            if (a[x] < -1 || a[x] > 1) return set_error(CSE_EINVAL, "entry not in {-1, 0, 1}");
    }
    const size_t lu = (size_t)m * n, lv = (size_t)n * p, lw = (size_t)m * p;
    const size_t one = (size_t)r * (lu + lv + lw), nv = (size_t)n_variants;
    const size_t bytes = ((one + 255) & ~(size_t)255) * (nv + 1) + nv * 4 + nv * 8 + 256;
    char* d = nullptr;
    cudaError_t e = cudaMalloc(&d, bytes);
    if (e != cudaSuccess) return set_error(CSE_ENOMEM, std::string("flip buffers: ") + cudaGetErrorString(e));
    const size_t stride = (one + 255) & ~(size_t)255;
    int8_t* dU = (int8_t*)d;
    int8_t* dV = dU + (size_t)r * lu;
    int8_t* dW = dV + (size_t)r * lv;
    int8_t* vU = (int8_t*)d + stride;
    int8_t* vV = vU + nv * r * lu;
    int8_t* vW = vV + nv * r * lv;
    int* dflips = (int*)((char*)d + stride * (nv + 1));
    unsigned long long* dbad = (unsigned long long*)((char*)dflips + ((nv * 4 + 7) & ~(size_t)7));
    e = cudaMemcpy(dU, U, (size_t)r * lu, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dV, V, (size_t)r * lv, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dW, W, (size_t)r * lw, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(dbad, 0, nv * 8);
    if (e == cudaSuccess) {
        flip_kernel<<<n_variants, 32>>>(dU, dV, dW, r, (int)lu, (int)lv, (int)lw, seed, iteration, max_flips, vU, vV,
                                        vW, dflips);
        e = cudaGetLastError();
    }
    // every variant's Brent equations, on the device
    for (int v = 0; v < n_variants && e == cudaSuccess; v++)
        e = launch_brent(vU + (size_t)v * r * lu, vV + (size_t)v * r * lv, vW + (size_t)v * r * lw, m, n, p, r,
                         dbad + v, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out_U, vU, nv * r * lu, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(out_V, vV, nv * r * lv, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(out_W, vW, nv * r * lw, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(flips, dflips, nv * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && brent_violations) e = cudaMemcpy(brent_violations, dbad, nv * 8, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return set_error(CSE_ECUDA, std::string("flip variants: ") + cudaGetErrorString(e));
    return CSE_OK;
}
