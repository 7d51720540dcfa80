// Shared helpers of the MMGaP kernels: dynamic shared-memory limits, the Philox4x32-10
// counter-based generator and the explicit IEEE round-to-nearest arithmetic.
#pragma once
#include <algorithm>
#include <atomic>
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"

namespace mmgap {

// Raise a kernel's dynamic shared-memory limit once per device: the largest
// size granted so far is remembered, so a launch that needs no more skips the
// driver call (it sits on the host between dependent launches otherwise).
template <auto Kernel>
cudaError_t ensure_dynamic_smem(size_t bytes) {
    static std::atomic<int> granted[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices)
        return cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if ((int)bytes <= granted[dev].load(std::memory_order_relaxed)) return cudaSuccess;
    e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    int cur = granted[dev].load(std::memory_order_relaxed);
    while ((int)bytes > cur && !granted[dev].compare_exchange_weak(cur, (int)bytes)) {
    }
    return cudaSuccess;
}

constexpr int kQBits = 14;

// ----------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64
// multiplies with the Weyl key schedule between rounds.
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
        const uint32_t lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += W0;
        k1 += W1;
    }
    return c;
}

// ------------------------------------------------------------ FP helpers
__device__ __forceinline__ float fmarn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float mulrn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float addrn(float a, float b) { return __fadd_rn(a, b); }

// exponent e of the smallest power of two 2^e >= mx (mx > 0 finite), else 0
__device__ __forceinline__ int sigma_exp_f(float mx) {
    if (!(mx > 0.0f) || isinf(mx)) return 0;
    int E;
    const float f = frexpf(mx, &E);
    return (f == 0.5f) ? E - 1 : E;
}
__device__ __forceinline__ int sigma_exp_d(double mx) {
    if (!(mx > 0.0) || isinf(mx)) return 0;
    int E;
    const double f = frexp(mx, &E);
    return (f == 0.5) ? E - 1 : E;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

}  // namespace mmgap
