// MMGaP hot-path kernels for sm_103a.
//
// Three stages (Sec. 3.2, Fig. 4: pre-processing, solver, post-processing):
//   build_detect_kernel  -- Gram + matched filter + MMSE guess + field +
//                           Q14 quantisation, one warp per resource element
//   cac_solve_kernel     -- CIM-CAC anneals (Eqs. 10-11) with the half-size
//                           coupling field of Fig. 5, one thread per anneal,
//                           warp shuffles for the arg-min, fused decode
//   vpp_* kernels        -- downlink VPP (Sec. 3.3) in FP64
//
// Every floating-point operation that decides an integer result is written
// with an explicit IEEE round-to-nearest intrinsic (__fmaf_rn, __fmul_rn,
// __fadd_rn, __fdiv_rn, __fsqrt_rn and their double forms) in a fixed order,
// so that guesses, quantised couplings, spins and symbols are reproducible
// bit for bit by a sequential CPU implementation of the same order.  The
// translation units are compiled with -fmad=false as a second guard.
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

// =========================================================================
// Builder: one warp per problem (resource element).
// =========================================================================
constexpr int kBuildWarps = 4;

template <int NT>
__host__ __device__ constexpr int build_smem_floats(int n_r) {
    // Hs [n_r][NT] c, Gc [NT][NT] c, L [NT][NT] c, y [n_r] c, z [n_r] c, m [NT] c, g [2NT],
    // flag + pivot scratch (perm [NT], d [NT])
    return 2 * n_r * NT + 4 * NT * NT + 4 * n_r + 4 * NT + 4 + 2 * NT;
}

// Where one problem's build writes its results (global or shared memory).
struct BuildOut {
    int16_t* Aq;        // [n][n]
    int16_t* hq;        // [n]
    int8_t* g;          // [n]
    float* G32;         // [n][n] or nullptr
    float* h32;         // [n] or nullptr
    int32_t* sigma_exp; // or nullptr
};

// Build problem p of `a` with one warp; ws = build_smem_floats<NT>(n_r)
// floats of this warp's shared memory.
template <int NT>
__device__ __forceinline__ void build_problem_warp(const BuildArgs& a, int p, int lane, float* ws, const BuildOut& o) {
    constexpr int n = 2 * NT;
    const int n_r = a.n_r;
    float* Hs = ws;
    float* Gc = Hs + 2 * n_r * NT;
    float* Lc = Gc + 2 * NT * NT;
    float* yv = Lc + 2 * NT * NT;
    float* zv = yv + 2 * n_r;
    float* mv = zv + 2 * n_r;  // matched filter [NT] c
    float* gv = mv + 2 * NT;   // g as floats [2NT]
    int* flag = reinterpret_cast<int*>(gv + 2 * NT);
    int* perm = flag + 4;      // position -> user (SIC)
    float* dg = reinterpret_cast<float*>(perm + NT);  // current Schur diagonal per user (SIC)

    const int c = a.chan_index ? a.chan_index[p] : p;
    if (c < 0 || c >= a.n_chan) {  // bad channel index: flag it, emit an all-zero problem
        if (lane == 0) atomicOr(a.err, kErrChanIndex);
        if (o.Aq)
            for (int e = lane; e < n * n; e += 32) o.Aq[e] = 0;
        for (int e = lane; e < n; e += 32) {
            if (o.hq) o.hq[e] = 0;
            o.g[e] = 0;
        }
        __syncwarp();
        return;
    }
    const float* Hg = a.H + (size_t)c * 2 * n_r * NT;
    const float* yg = a.y + (size_t)p * 2 * n_r;
    for (int e = lane; e < 2 * n_r * NT; e += 32) Hs[e] = mulrn(a.kappa, Hg[e]);
    for (int e = lane; e < 2 * n_r; e += 32) yv[e] = yg[e];
    if (lane == 0) flag[0] = 0;
    __syncwarp();

    // Gram G_c = Hs^H Hs (upper triangle + Hermitian mirror) and m = Hs^H y.
    // With a precomputed (tensor-core) Gram only the matched filter is formed here.
    const float* Gpre = a.Gc_pre ? a.Gc_pre + (size_t)c * 2 * NT * NT : nullptr;
    if (Gpre)
        for (int e = lane; e < 2 * NT * NT; e += 32) Gc[e] = Gpre[e];
    for (int t = lane + (Gpre ? NT * NT : 0); t < NT * NT + NT; t += 32) {
        if (t < NT * NT) {
            const int i = t / NT, j = t % NT;
            if (i > j) continue;
            if (i == j) {
                float acc = 0.0f;
                for (int k = 0; k < n_r; ++k) {
                    const float ar = Hs[2 * (k * NT + i)], ai = Hs[2 * (k * NT + i) + 1];
                    acc = fmarn(ar, ar, acc);
                    acc = fmarn(ai, ai, acc);
                }
                Gc[2 * (i * NT + i)] = acc;
                Gc[2 * (i * NT + i) + 1] = 0.0f;
            } else {
                float re = 0.0f, im = 0.0f;
                for (int k = 0; k < n_r; ++k) {
                    const float ar = Hs[2 * (k * NT + i)], ai = Hs[2 * (k * NT + i) + 1];
                    const float br = Hs[2 * (k * NT + j)], bi = Hs[2 * (k * NT + j) + 1];
                    re = fmarn(ar, br, re);
                    re = fmarn(ai, bi, re);
                    im = fmarn(ar, bi, im);
                    im = fmarn(-ai, br, im);
                }
                Gc[2 * (i * NT + j)] = re;
                Gc[2 * (i * NT + j) + 1] = im;
                Gc[2 * (j * NT + i)] = re;
                Gc[2 * (j * NT + i) + 1] = -im;
            }
        } else {
            const int i = t - NT * NT;
            float re = 0.0f, im = 0.0f;
            for (int k = 0; k < n_r; ++k) {
                const float ar = Hs[2 * (k * NT + i)], ai = Hs[2 * (k * NT + i) + 1];
                const float br = yv[2 * k], bi = yv[2 * k + 1];
                re = fmarn(ar, br, re);
                re = fmarn(ai, bi, re);
                im = fmarn(ar, bi, im);
                im = fmarn(-ai, br, im);
            }
            mv[2 * i] = re;
            mv[2 * i + 1] = im;
        }
    }
    __syncwarp();

    const int side = 1 << (a.mod_bits >> 1);
    const float Lm = (float)(side - 1);
    auto slice = [&](float v) -> float {  // nearest alphabet point (ties upward)
        float xc = fmaxf(v, -Lm);
        xc = fminf(xc, Lm);
        return (float)(2 * (int)floorf(mulrn(xc, 0.5f)) + 1);
    };
    if (a.guess_mode == 2) {
        // externally supplied guess (a previous stage's solution)
        if (lane < NT) {
            gv[lane] = (float)a.g_in[(size_t)p * n + lane];
            gv[NT + lane] = (float)a.g_in[(size_t)p * n + NT + lane];
        }
        __syncwarp();
    } else {
        // Cholesky of B = G_c + rho I (rho = noise_var kappa^2), left-looking, one
        // column per step; lane j the pivot, lanes i > j the rest.  MMSE (Eq. 3)
        // factors in natural order; MMSE-SIC (Sec. 3.2.2) pivots on the smallest
        // current Schur diagonal (ties: first position), rows of L being positions.
        const bool sic = a.guess_mode == 1;
        const float rho = mulrn(a.noise_var[p], a.kappa2);
        if (lane < NT) {
            perm[lane] = lane;
            dg[lane] = addrn(Gc[2 * (lane * NT + lane)], rho);
        }
        __syncwarp();
        for (int j = 0; j < NT; ++j) {
            if (sic) {
                if (lane == 0) {
                    int best = j;
                    for (int i = j + 1; i < NT; ++i)
                        if (dg[perm[i]] < dg[perm[best]]) best = i;
                    flag[1] = best;
                    const int t = perm[j];
                    perm[j] = perm[best];
                    perm[best] = t;
                }
                __syncwarp();
                const int best = flag[1];
                if (lane < j && best != j) {  // swap the computed part of rows j and best
                    const float r0 = Lc[2 * (j * NT + lane)], r1 = Lc[2 * (j * NT + lane) + 1];
                    Lc[2 * (j * NT + lane)] = Lc[2 * (best * NT + lane)];
                    Lc[2 * (j * NT + lane) + 1] = Lc[2 * (best * NT + lane) + 1];
                    Lc[2 * (best * NT + lane)] = r0;
                    Lc[2 * (best * NT + lane) + 1] = r1;
                }
                __syncwarp();
            }
            const int u = sic ? perm[j] : j;
            if (lane == j) {
                float d;
                if (sic) {
                    d = dg[u];
                } else {
                    d = addrn(Gc[2 * (j * NT + j)], rho);
                    for (int k = 0; k < j; ++k) {
                        const float lr = Lc[2 * (j * NT + k)], li = Lc[2 * (j * NT + k) + 1];
                        d = fmarn(-lr, lr, d);
                        d = fmarn(-li, li, d);
                    }
                }
                const bool ok = (d > 0.0f) && !isinf(d);
                if (!ok) flag[0] = 1;
                Lc[2 * (j * NT + j)] = ok ? __fsqrt_rn(d) : 1.0f;
                Lc[2 * (j * NT + j) + 1] = 0.0f;
            }
            __syncwarp();
            const float ljj = Lc[2 * (j * NT + j)];
            if (lane > j && lane < NT) {
                const int i = lane;
                const int v = sic ? perm[i] : i;
                float re = Gc[2 * (v * NT + u)], im = Gc[2 * (v * NT + u) + 1];
                for (int k = 0; k < j; ++k) {
                    const float ar = Lc[2 * (i * NT + k)], ai = Lc[2 * (i * NT + k) + 1];
                    const float br = Lc[2 * (j * NT + k)], bi = Lc[2 * (j * NT + k) + 1];
                    re = fmarn(-ar, br, re);
                    re = fmarn(-ai, bi, re);
                    im = fmarn(-ai, br, im);
                    im = fmarn(ar, bi, im);
                }
                const float lr = __fdiv_rn(re, ljj), li = __fdiv_rn(im, ljj);
                Lc[2 * (i * NT + j)] = lr;
                Lc[2 * (i * NT + j) + 1] = li;
                if (sic) {
                    float dv = dg[v];
                    dv = fmarn(-lr, lr, dv);
                    dv = fmarn(-li, li, dv);
                    dg[v] = dv;
                }
            }
            __syncwarp();
        }
        const bool chol_failed = flag[0] != 0;

        // forward solve L w = P m (right-looking; per row the updates arrive in
        // ascending k, the same sequence as the left-looking sum)
        float accr = 0.0f, acci = 0.0f;
        if (lane < NT) {
            const int src = sic ? perm[lane] : lane;
            accr = mv[2 * src];
            acci = mv[2 * src + 1];
        }
        float wr = 0.0f, wi = 0.0f;
        for (int k = 0; k < NT; ++k) {
            if (lane == k) {
                const float lkk = Lc[2 * (k * NT + k)];
                wr = __fdiv_rn(accr, lkk);
                wi = __fdiv_rn(acci, lkk);
            }
            const float br = __shfl_sync(0xffffffffu, wr, k), bi = __shfl_sync(0xffffffffu, wi, k);
            if (lane > k && lane < NT) {
                const float ar = Lc[2 * (lane * NT + k)], ai = Lc[2 * (lane * NT + k) + 1];
                accr = fmarn(-ar, br, accr);
                accr = fmarn(ai, bi, accr);
                acci = fmarn(-ar, bi, acci);
                acci = fmarn(-ai, br, acci);
            }
        }
        // backward solve L^H x = w, k descending; SIC slices each x_k before
        // it is substituted (successive interference cancellation)
        accr = wr;
        acci = wi;
        float xr = 0.0f, xi = 0.0f;
        for (int k = NT - 1; k >= 0; --k) {
            if (lane == k) {
                const float lkk = Lc[2 * (k * NT + k)];
                xr = __fdiv_rn(accr, lkk);
                xi = __fdiv_rn(acci, lkk);
                if (sic) {
                    xr = slice(xr);
                    xi = slice(xi);
                }
            }
            const float br = __shfl_sync(0xffffffffu, xr, k), bi = __shfl_sync(0xffffffffu, xi, k);
            if (lane < k) {
                const float ar = Lc[2 * (k * NT + lane)], ai = Lc[2 * (k * NT + lane) + 1];
                accr = fmarn(-ar, br, accr);
                accr = fmarn(-ai, bi, accr);
                acci = fmarn(-ar, bi, acci);
                acci = fmarn(ai, br, acci);
            }
        }
        // hard decision to the nearest alphabet point (ties upward)
        if (lane < NT) {
            const int dst = sic ? perm[lane] : lane;
            gv[dst] = slice(chol_failed ? 0.0f : xr);
            gv[NT + dst] = slice(chol_failed ? 0.0f : xi);
        }
        __syncwarp();
    }

    // residual z = y - Hs g, field h_c = Hs^H z
    for (int k = lane; k < n_r; k += 32) {
        float re = yv[2 * k], im = yv[2 * k + 1];
        for (int j = 0; j < NT; ++j) {
            const float ar = Hs[2 * (k * NT + j)], ai = Hs[2 * (k * NT + j) + 1];
            const float br = gv[j], bi = gv[NT + j];
            re = fmarn(-ar, br, re);
            re = fmarn(ai, bi, re);
            im = fmarn(-ar, bi, im);
            im = fmarn(-ai, br, im);
        }
        zv[2 * k] = re;
        zv[2 * k + 1] = im;
    }
    __syncwarp();
    float hre = 0.0f, him = 0.0f;
    if (lane < NT) {
        for (int k = 0; k < n_r; ++k) {
            const float ar = Hs[2 * (k * NT + lane)], ai = Hs[2 * (k * NT + lane) + 1];
            const float br = zv[2 * k], bi = zv[2 * k + 1];
            hre = fmarn(ar, br, hre);
            hre = fmarn(ai, bi, hre);
            him = fmarn(ar, bi, him);
            him = fmarn(-ai, br, him);
        }
    }

    // power-of-two normaliser over the real-form couplings and field
    float mx = 0.0f;
    for (int e = lane; e < NT * NT; e += 32) mx = fmaxf(mx, fmaxf(fabsf(Gc[2 * e]), fabsf(Gc[2 * e + 1])));
    if (lane < NT) mx = fmaxf(mx, fmaxf(fabsf(hre), fabsf(him)));
    mx = warp_max(mx);
    const int se = sigma_exp_f(mx);
    const bool finite = isfinite(mx);
    const float s = ldexpf(1.0f, kQBits - se);

    if (o.Aq)  // (the direct mapping uses only the guess and the Gram / matched filter left in ws)
        for (int e = lane; e < n * n; e += 32) {
            const int i = e / n, j = e % n;
            const int ib = i % NT, jb = j % NT;
            const float re = Gc[2 * (ib * NT + jb)], im = Gc[2 * (ib * NT + jb) + 1];
            // G = [[Re G_c, -Im G_c], [Im G_c, Re G_c]]
            const float G = (i < NT) == (j < NT) ? re : (i < NT ? -im : im);
            o.Aq[e] = finite ? (int16_t)(int)rintf(mulrn(-G, s)) : (int16_t)0;
            if (o.G32) o.G32[e] = G;
        }
    if (lane < NT) {
        if (o.hq) {
            o.hq[lane] = finite ? (int16_t)(int)rintf(mulrn(hre, s)) : (int16_t)0;
            o.hq[NT + lane] = finite ? (int16_t)(int)rintf(mulrn(him, s)) : (int16_t)0;
        }
        o.g[lane] = (int8_t)(int)gv[lane];
        o.g[NT + lane] = (int8_t)(int)gv[NT + lane];
        if (o.h32) {
            o.h32[lane] = hre;
            o.h32[NT + lane] = him;
        }
    }
    if (lane == 0 && o.sigma_exp) *o.sigma_exp = se;
    __syncwarp();
}

template <int NT>
__global__ void __launch_bounds__(kBuildWarps * 32) build_detect_kernel(BuildArgs a) {
    extern __shared__ __align__(16) float smem[];
    constexpr int n = 2 * NT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * kBuildWarps + warp;
    if (p >= a.n_problems) return;  // warp-uniform; no block-wide barrier below
    BuildOut o;
    o.Aq = a.Aq + (size_t)p * n * n;
    o.hq = a.hq + (size_t)p * n;
    o.g = a.g + (size_t)p * n;
    o.G32 = a.G32 ? a.G32 + (size_t)p * n * n : nullptr;
    o.h32 = a.h32 ? a.h32 + (size_t)p * n : nullptr;
    o.sigma_exp = a.sigma_exp ? a.sigma_exp + p : nullptr;
    build_problem_warp<NT>(a, p, lane, smem + warp * build_smem_floats<NT>(a.n_r), o);
}

// =========================================================================
// CIM-CAC solver: one CTA per problem, one thread per anneal (runs = CTA
// size, a multiple of 32).  Each thread keeps its 2n+1 amplitudes x and
// error variables e in registers; the couplings sit in shared memory and
// are read as warp-uniform broadcasts.
// =========================================================================

// One forward-Euler step of Eqs. 10-11 for one spin with frozen field mu
// (mu already carries the factor eps dt):
//   x' = x (1 + dt (p-1) - dt x^2) + e mu,   e' = e (1 + dt zeta a - dt zeta x^2)
__device__ __forceinline__ void euler_spin(float& x, float& e, float mu, const EulerConsts& k) {
    const float q = mulrn(x, x);
    const float t = fmarn(k.cdt, q, k.c1);
    const float em = mulrn(e, mu);
    const float xn = fmarn(x, t, em);
    const float r = fmarn(k.cz, q, k.c2);
    e = mulrn(e, r);
    x = xn;
}

template <int NT>
struct SolveSmem {
    static constexpr int n = 2 * NT;
    float A[n * n];       // eps dt * A_q 2^-14
    float h[n];           // eps dt * h_q 2^-14
    float nd[n];          // -diag(A)
    int16_t Aq[n * n];    // integer copy for the exact energy
    int16_t hq[n];
    int8_t g[n];
    long long key[4];
    int ndiv[4];
};

// Coupling field refresh (Fig. 5): u = x1 + x2, m = A u, mu_a = b^T u.
template <int n>
__device__ __forceinline__ void coupling_mvm(const float* sA, const float* sh,
                                             const float (&x)[2 * n + 1], float (&m)[n], float& mua) {
    // The couplings are loop invariant; without this barrier (and without
    // __restrict__ on the shared-memory pointers, which would let the compiler
    // look through it) all n^2 loads are hoisted out of the time loop into
    // registers and spill.  Re-reading them as warp-uniform broadcasts costs
    // one LDS.128 per four FMAs.
    asm volatile("" ::: "memory");
#pragma unroll
    for (int i = 0; i < n; ++i) m[i] = 0.0f;
    mua = 0.0f;
#pragma unroll
    for (int j = 0; j < n; ++j) {
        const float u = addrn(x[j], x[n + j]);
        mua = fmarn(sh[j], u, mua);
        if constexpr (n % 4 == 0) {
            const float4* row = reinterpret_cast<const float4*>(sA + j * n);
#pragma unroll
            for (int i4 = 0; i4 < n / 4; ++i4) {
                const float4 a4 = row[i4];
                m[4 * i4 + 0] = fmarn(a4.x, u, m[4 * i4 + 0]);
                m[4 * i4 + 1] = fmarn(a4.y, u, m[4 * i4 + 1]);
                m[4 * i4 + 2] = fmarn(a4.z, u, m[4 * i4 + 2]);
                m[4 * i4 + 3] = fmarn(a4.w, u, m[4 * i4 + 3]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < n; ++i) m[i] = fmarn(sA[j * n + i], u, m[i]);
        }
    }
}

// L Euler steps of every spin with the field frozen at the refresh:
// c = m + b x_a, mu1 = c - diag(A) o x1, mu2 = c - diag(A) o x2.
// Spins are independent while the field is frozen, so each spin's L steps
// run back to back.
template <int n, int L>
__device__ __forceinline__ void frozen_steps(const float* sh, const float* snd,
                                             float (&x)[2 * n + 1], float (&e)[2 * n + 1], const float (&m)[n],
                                             float mua, const EulerConsts& k) {
    const float xa = x[2 * n];
#pragma unroll
    for (int i = 0; i < n; ++i) {
        const float c = fmarn(sh[i], xa, m[i]);
        const float mu1 = fmarn(snd[i], x[i], c);
        const float mu2 = fmarn(snd[i], x[n + i], c);
#pragma unroll
        for (int s = 0; s < L; ++s) {
            euler_spin(x[i], e[i], mu1, k);
            euler_spin(x[n + i], e[n + i], mu2, k);
        }
    }
#pragma unroll
    for (int s = 0; s < L; ++s) euler_spin(x[2 * n], e[2 * n], mua, k);
}

template <int n>
__device__ __forceinline__ void frozen_steps_rt(const float* sh, const float* snd,
                                                float (&x)[2 * n + 1], float (&e)[2 * n + 1], const float (&m)[n],
                                                float mua, int L, const EulerConsts& k) {
    const float xa = x[2 * n];
#pragma unroll
    for (int i = 0; i < n; ++i) {
        const float c = fmarn(sh[i], xa, m[i]);
        const float mu1 = fmarn(snd[i], x[i], c);
        const float mu2 = fmarn(snd[i], x[n + i], c);
#pragma unroll 1
        for (int s = 0; s < L; ++s) {
            euler_spin(x[i], e[i], mu1, k);
            euler_spin(x[n + i], e[n + i], mu2, k);
        }
    }
#pragma unroll 1
    for (int s = 0; s < L; ++s) euler_spin(x[2 * n], e[2 * n], mua, k);
}

// F > 0: compile-time refresh period; F == 0: runtime period a.f_mvm.
template <int NT, int F>
__global__ void __launch_bounds__(128) cac_solve_kernel(SolveArgs a) {
    constexpr int n = 2 * NT;
    constexpr int N = 2 * n + 1;
    __shared__ __align__(16) SolveSmem<NT> sm;
    const int p = blockIdx.x;
    const int run = threadIdx.x;
    const int R = blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const EulerConsts k = a.k;

    // stage the problem: Q14 codes -> exact floats -> one rounding by eps dt
    {
        const int16_t* Aq = a.Aq + (size_t)p * n * n;
        for (int e = run; e < n * n; e += R) {
            const int16_t v = Aq[e];
            sm.Aq[e] = v;
            sm.A[e] = mulrn(mulrn((float)v, 0x1p-14f), k.ce);
        }
        const int16_t* hq = a.hq + (size_t)p * n;
        for (int i = run; i < n; i += R) {
            const int16_t v = hq[i];
            sm.hq[i] = v;
            sm.h[i] = mulrn(mulrn((float)v, 0x1p-14f), k.ce);
            sm.g[i] = a.g ? a.g[(size_t)p * n + i] : (int8_t)0;
        }
    }
    __syncthreads();
    for (int i = run; i < n; i += R) sm.nd[i] = -sm.A[i * n + i];
    __syncthreads();

    // initial amplitudes from Philox: spin k uses word k%4 of counter
    // (k/4, run, problem_lo, problem_hi)
    float x[N], e[N];
    {
        const uint64_t pg = a.problem_offset + (uint64_t)p;
#pragma unroll
        for (int q4 = 0; q4 < (N + 3) / 4; ++q4) {
            const U4 w = philox4x32_10(U4{(uint32_t)q4, (uint32_t)run, (uint32_t)pg, (uint32_t)(pg >> 32)}, a.key0,
                                       a.key1);
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (4 * q4 + t < N) {
                    const int v = (int)(ws[t] >> 8) - 8388608;
                    x[4 * q4 + t] = mulrn((float)v, k.xs);
                    e[4 * q4 + t] = 1.0f;
                }
            }
        }
    }

    // anneal
    float m[n];
    float mua;
    const int S = a.steps;
    int t = 0;
    if constexpr (F > 0) {
#pragma unroll 1
        for (; t + F <= S; t += F) {
            coupling_mvm<n>(sm.A, sm.h, x, m, mua);
            frozen_steps<n, F>(sm.h, sm.nd, x, e, m, mua, k);
        }
    } else {
        const int f = a.f_mvm;
#pragma unroll 1
        for (; t + f <= S; t += f) {
            coupling_mvm<n>(sm.A, sm.h, x, m, mua);
            frozen_steps_rt<n>(sm.h, sm.nd, x, e, m, mua, f, k);
        }
    }
    if (t < S) {
        coupling_mvm<n>(sm.A, sm.h, x, m, mua);
        frozen_steps_rt<n>(sm.h, sm.nd, x, e, m, mua, S - t, k);
    }

    // spins -> offset d = s_a (s1 + s2) / 2, clipped to the alphabet
    bool valid = true;
#pragma unroll
    for (int q = 0; q < N; ++q) valid = valid && (fabsf(x[q]) <= k.x_max) && (e[q] > 0.0f);
    if (a.spins_out) {  // final sign of every spin (bit q: x_q >= 0) and a divergence flag (word 1, bit 63)
        uint64_t w0 = 0, w1 = 0;
#pragma unroll
        for (int q = 0; q < N; ++q) {
            const uint64_t bit = x[q] >= 0.0f ? 1ull : 0ull;
            if (q < 64) w0 |= bit << q;
            else w1 |= bit << (q - 64);
        }
        if (!valid) w1 |= 1ull << 63;
        a.spins_out[((size_t)p * R + run) * 2] = w0;
        a.spins_out[((size_t)p * R + run) * 2 + 1] = w1;
    }
    const int sa = x[2 * n] >= 0.0f ? 1 : -1;
    int d[n];
#pragma unroll
    for (int i = 0; i < n; ++i) {
        const int s1 = x[i] >= 0.0f ? 1 : -1, s2 = x[n + i] >= 0.0f ? 1 : -1;
        int di = sa * (s1 + s2) / 2;
        if (a.level_max > 0) {
            const int xv = (int)sm.g[i] + 2 * di;
            if (xv > a.level_max || xv < -a.level_max) di = 0;
        }
        d[i] = di;
    }
    // exact quantised energy E = -d^T A_q d - h_q^T d
    int E = 0;
#pragma unroll
    for (int i = 0; i < n; ++i) {
        int r = 0;
#pragma unroll
        for (int j = 0; j < n; ++j) r += (int)sm.Aq[i * n + j] * d[j];
        E -= d[i] * r;
        E -= (int)sm.hq[i] * d[i];
    }
    // MMSE fallback: a diverged anneal or one worse than the guess returns the guess
    const bool keep = valid && E <= 0;
    const int Ec = keep ? E : 0;
    long long key = (long long)Ec * 4294967296LL + (long long)run;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long other = __shfl_xor_sync(0xffffffffu, key, o);
        key = other < key ? other : key;
    }
    const unsigned divmask = __ballot_sync(0xffffffffu, !valid);
    if (lane == 0) {
        sm.key[warp] = key;
        sm.ndiv[warp] = __popc(divmask);
    }
    __syncthreads();
    long long best = sm.key[0];
    int ndiv = sm.ndiv[0];
    for (int w = 1; w < R / 32; ++w) {
        best = sm.key[w] < best ? sm.key[w] : best;
        ndiv += sm.ndiv[w];
    }
    const int best_run = (int)(best & 0xffffffffLL);
    if (run == best_run) {
        const int bestE = (int)((best - (long long)best_run) / 4294967296LL);
        if (a.d_out) {
            int8_t* dout = a.d_out + (size_t)p * n;
#pragma unroll
            for (int i = 0; i < n; ++i) dout[i] = keep ? (int8_t)d[i] : (int8_t)0;
        }
        if (a.E_out) a.E_out[p] = bestE;
        if (a.run_out) a.run_out[p] = best_run;
        if (a.ndiv_out) a.ndiv_out[p] = ndiv;
        if (a.x_out) {
#pragma unroll
            for (int i = 0; i < n; ++i) a.x_out[(size_t)p * n + i] = (int8_t)((int)sm.g[i] + 2 * (keep ? d[i] : 0));
        }
        if (a.sym_out) {
            // fused decode: lattice x = g + 2d -> symbol index
            const int side = 1 << (a.mod_bits >> 1), L = side - 1;
            uint8_t* so = a.sym_out + (size_t)p * NT;
#pragma unroll
            for (int i = 0; i < NT; ++i) {
                const int xr = (int)sm.g[i] + 2 * (keep ? d[i] : 0);
                const int xi = (int)sm.g[NT + i] + 2 * (keep ? d[NT + i] : 0);
                so[i] = (uint8_t)(((xr + L) / 2) * side + (xi + L) / 2);
            }
        }
    }
}

// =========================================================================
// Tuned CIM-CAC solver: TPA threads per anneal.  Thread q of an anneal owns
// rows [q NS, (q+1) NS) of both half-size blocks (NS = n / TPA) and keeps the
// auxiliary spin redundantly; at each field refresh the anneal's u = x1 + x2 is
// gathered with warp shuffles, then every thread forms its NS rows of m = A u
// in the same ascending-j FMA order as the one-thread form.  PACKED runs
// pairs of rows with the packed FP32 instructions (__ffma2_rn, __fmul2_rn,
// __fadd2_rn: two IEEE round-to-nearest operations each).  All variants
// produce bit-identical results; they differ in registers per thread
// (hence warps in flight to hide shared-memory latency) and instruction count.
// =========================================================================

__device__ __forceinline__ void euler_pair(float2& x, float2& e, float2 mu, float2 cdt, float2 c1, float2 cz,
                                           float2 c2) {
    const float2 q = __fmul2_rn(x, x);
    const float2 t = __ffma2_rn(cdt, q, c1);
    const float2 em = __fmul2_rn(e, mu);
    const float2 xn = __ffma2_rn(x, t, em);
    const float2 r = __ffma2_rn(cz, q, c2);
    e = __fmul2_rn(e, r);
    x = xn;
}

// Field refresh + L frozen Euler steps of one thread's rows (L == 0: runtime Lrt).
// PAIR (one thread per anneal, packed): lanes 2k and 2k+1 share the refresh
// of their two anneals -- each forms half the rows of m for both anneals
// (the partner's u_j arrives by shuffle), so each coupling loaded from shared
// memory feeds two fused multiply-adds; the halves are then swapped.  Every
// m_i is still the ascending-j FMA chain from 0, so results are unchanged.
template <int n, int NS, int TPA, bool PACKED, int L, bool PAIR = false>
__device__ __forceinline__ void tuned_block(const float* sA, const float* sh, const float* snd, float (&x1)[NS],
                                            float (&x2)[NS], float (&e1)[NS], float (&e2)[NS], float& xa, float& ea,
                                            int q, int lane, int Lrt, const EulerConsts& k) {
    asm volatile("" ::: "memory");  // keep the coupling loads inside the time loop
    const int row0 = q * NS;
    // u = x1 + x2 of this thread's rows, then of the whole anneal
    float uo[NS];
    if constexpr (PACKED) {
#pragma unroll
        for (int i = 0; i < NS; i += 2) {
            const float2 s2 = __fadd2_rn(make_float2(x1[i], x1[i + 1]), make_float2(x2[i], x2[i + 1]));
            uo[i] = s2.x;
            uo[i + 1] = s2.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < NS; ++i) uo[i] = addrn(x1[i], x2[i]);
    }
    float u[TPA == 1 ? 1 : n];
    if constexpr (TPA == 1) {
        // uo is the whole anneal's u; used directly below
    } else if constexpr (TPA == 2) {
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const float other = __shfl_xor_sync(0xffffffffu, uo[i], 1);
            u[i] = q == 0 ? uo[i] : other;
            u[NS + i] = q == 0 ? other : uo[i];
        }
    } else {
        const int base = lane & ~(TPA - 1);
#pragma unroll
        for (int qq = 0; qq < TPA; ++qq)
#pragma unroll
            for (int i = 0; i < NS; ++i) u[qq * NS + i] = __shfl_sync(0xffffffffu, uo[i], base | qq);
    }
    // m = A u for this thread's rows (ascending j), mu_a = b^T u
    float m[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) m[i] = 0.0f;
    float mua = 0.0f;
    if constexpr (PAIR) {
        static_assert(TPA == 1 && PACKED && n % 8 == 0, "paired refresh: one thread per anneal, packed");
        constexpr int H = n / 2;
        const int half = lane & 1;
        float mo[H], mp[H];  // this half's rows of m for this anneal and for the partner's
#pragma unroll
        for (int i = 0; i < H; ++i) mo[i] = mp[i] = 0.0f;
#pragma unroll
        for (int j = 0; j < n; ++j) {
            const float uj = uo[j];
            const float up = __shfl_xor_sync(0xffffffffu, uj, 1);
            mua = fmarn(sh[j], uj, mua);
            const float4* row = reinterpret_cast<const float4*>(sA + j * n + half * H);
            const float2 uu = make_float2(uj, uj), pp = make_float2(up, up);
#pragma unroll
            for (int i4 = 0; i4 < H / 4; ++i4) {
                const float4 a4 = row[i4];
                const float2 al = make_float2(a4.x, a4.y), ah = make_float2(a4.z, a4.w);
                float2 v = __ffma2_rn(al, uu, make_float2(mo[4 * i4], mo[4 * i4 + 1]));
                mo[4 * i4] = v.x;
                mo[4 * i4 + 1] = v.y;
                v = __ffma2_rn(ah, uu, make_float2(mo[4 * i4 + 2], mo[4 * i4 + 3]));
                mo[4 * i4 + 2] = v.x;
                mo[4 * i4 + 3] = v.y;
                v = __ffma2_rn(al, pp, make_float2(mp[4 * i4], mp[4 * i4 + 1]));
                mp[4 * i4] = v.x;
                mp[4 * i4 + 1] = v.y;
                v = __ffma2_rn(ah, pp, make_float2(mp[4 * i4 + 2], mp[4 * i4 + 3]));
                mp[4 * i4 + 2] = v.x;
                mp[4 * i4 + 3] = v.y;
            }
        }
        // swap: the partner formed this anneal's other half
#pragma unroll
        for (int i = 0; i < H; ++i) {  // (selects, not a runtime index: m stays in registers)
            const float other = __shfl_xor_sync(0xffffffffu, mp[i], 1);
            m[i] = half ? other : mo[i];
            m[H + i] = half ? mo[i] : other;
        }
    } else {
#pragma unroll
    for (int j = 0; j < n; ++j) {
        float uj;
        if constexpr (TPA == 1) uj = uo[j];
        else uj = u[j];
        mua = fmarn(sh[j], uj, mua);
        const float4* row = reinterpret_cast<const float4*>(sA + j * n + row0);
#pragma unroll
        for (int i4 = 0; i4 < NS / 4; ++i4) {
            const float4 a4 = row[i4];
            if constexpr (PACKED) {
                const float2 uu = make_float2(uj, uj);
                const float2 lo = __ffma2_rn(make_float2(a4.x, a4.y), uu, make_float2(m[4 * i4], m[4 * i4 + 1]));
                const float2 hi = __ffma2_rn(make_float2(a4.z, a4.w), uu, make_float2(m[4 * i4 + 2], m[4 * i4 + 3]));
                m[4 * i4] = lo.x;
                m[4 * i4 + 1] = lo.y;
                m[4 * i4 + 2] = hi.x;
                m[4 * i4 + 3] = hi.y;
            } else {
                m[4 * i4 + 0] = fmarn(a4.x, uj, m[4 * i4 + 0]);
                m[4 * i4 + 1] = fmarn(a4.y, uj, m[4 * i4 + 1]);
                m[4 * i4 + 2] = fmarn(a4.z, uj, m[4 * i4 + 2]);
                m[4 * i4 + 3] = fmarn(a4.w, uj, m[4 * i4 + 3]);
            }
        }
    }
    }
    // frozen field: c = m + b x_a, mu1 = c - diag(A) x1, mu2 = c - diag(A) x2
    if constexpr (PACKED) {
        const float2 xa2 = make_float2(xa, xa);
        const float2 cdt = make_float2(k.cdt, k.cdt), c1 = make_float2(k.c1, k.c1);
        const float2 cz = make_float2(k.cz, k.cz), c2 = make_float2(k.c2, k.c2);
#pragma unroll
        for (int i = 0; i < NS; i += 2) {
            const float2 hh = *reinterpret_cast<const float2*>(sh + row0 + i);
            const float2 nd = *reinterpret_cast<const float2*>(snd + row0 + i);
            const float2 c = __ffma2_rn(hh, xa2, make_float2(m[i], m[i + 1]));
            float2 X1 = make_float2(x1[i], x1[i + 1]), X2 = make_float2(x2[i], x2[i + 1]);
            float2 E1 = make_float2(e1[i], e1[i + 1]), E2 = make_float2(e2[i], e2[i + 1]);
            const float2 mu1 = __ffma2_rn(nd, X1, c);
            const float2 mu2 = __ffma2_rn(nd, X2, c);
            if constexpr (L > 0) {
#pragma unroll
                for (int s = 0; s < L; ++s) {
                    euler_pair(X1, E1, mu1, cdt, c1, cz, c2);
                    euler_pair(X2, E2, mu2, cdt, c1, cz, c2);
                }
            } else {
#pragma unroll 1
                for (int s = 0; s < Lrt; ++s) {
                    euler_pair(X1, E1, mu1, cdt, c1, cz, c2);
                    euler_pair(X2, E2, mu2, cdt, c1, cz, c2);
                }
            }
            x1[i] = X1.x; x1[i + 1] = X1.y; x2[i] = X2.x; x2[i + 1] = X2.y;
            e1[i] = E1.x; e1[i + 1] = E1.y; e2[i] = E2.x; e2[i + 1] = E2.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const float c = fmarn(sh[row0 + i], xa, m[i]);
            const float mu1 = fmarn(snd[row0 + i], x1[i], c);
            const float mu2 = fmarn(snd[row0 + i], x2[i], c);
            if constexpr (L > 0) {
#pragma unroll
                for (int s = 0; s < L; ++s) {
                    euler_spin(x1[i], e1[i], mu1, k);
                    euler_spin(x2[i], e2[i], mu2, k);
                }
            } else {
#pragma unroll 1
                for (int s = 0; s < Lrt; ++s) {
                    euler_spin(x1[i], e1[i], mu1, k);
                    euler_spin(x2[i], e2[i], mu2, k);
                }
            }
        }
    }
    if constexpr (L > 0) {
#pragma unroll
        for (int s = 0; s < L; ++s) euler_spin(xa, ea, mua, k);
    } else {
#pragma unroll 1
        for (int s = 0; s < Lrt; ++s) euler_spin(xa, ea, mua, k);
    }
}

// FP16 / BF16 packing and the warp MMA used by the tensor-core refresh and Gram.
__device__ __forceinline__ uint32_t pack16(float lo, float hi, int fp16) {
    uint32_t r;
    if (fp16) {
        asm("{ .reg .f16 l, h;\n cvt.rn.f16.f32 l, %1;\n cvt.rn.f16.f32 h, %2;\n mov.b32 %0, {l, h}; }"
            : "=r"(r) : "f"(lo), "f"(hi));
    } else {
        asm("cvt.rn.bf16x2.f32 %0, %2, %1;" : "=r"(r) : "f"(lo), "f"(hi));
    }
    return r;
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2], int fp16) {
    if (fp16) {
        asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                     "{%0,%1,%2,%3};"
                     : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                     : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    } else {
        asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                     "{%0,%1,%2,%3};"
                     : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                     : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
}

// -------------------------------------------------------------------------
// Tensor-core field refresh (a precision variant of the refresh above; its
// results are not bit-identical to the FP32 path's).  Per warp, the 32
// anneals' fields are one product M = A U (n x n by n x 32) on mma.sync
// m16n8k16 with FP16 operands and FP32 accumulation.  The Q14 couplings
// c 2^-14 are exact as an FP16 pair (hi + lo); u 2^5 is split the same way
// (22 bits), and M = Al Uh + Ah Ul + Ah Uh (the Al Ul term, ~2^-22, is
// dropped), so m matches the FP32 refresh to about 2^-21 of sum |A||u|.
// The scale 2^5 keeps |u| <= 2047 (every valid anneal: |x| <= x_max = 1000)
// below the FP16 maximum; a larger u overflows to inf and its anneal ends
// invalid.  U goes from registers to the MMA's B fragments through shared
// memory (each lane writes its anneal's row of U^T), and M back to each
// lane's registers the same way (rows of M^T; row strides padded so that
// every access is free of bank conflicts).  mu_a = b^T u stays FP32.
// -------------------------------------------------------------------------
template <int NT>
struct TcShape {
    static constexpr int n = 2 * NT;
    static constexpr int MT = n / 16;     // M tiles (rows i)
    static constexpr int KT = n / 16;     // K steps (columns j)
    static constexpr int UW = n / 2 + 4;  // 32-bit words per row of U^T (FP16 pairs), padded
    static constexpr int MW = n + 4;      // floats per row of M^T, padded
    // exchange buffer of a warp with AW anneals (32 / threads per anneal)
    static constexpr int warp_words(int AW) { return 2 * AW * UW > AW * MW ? 2 * AW * UW : AW * MW; }
    static constexpr int WARP_WORDS = warp_words(32);
    static constexpr int AF_WORDS = MT * KT * 2 * 4 * 32;  // A fragments, hi and lo
};

__device__ __forceinline__ uint32_t h2pack(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.f16x2.f32 %0, %2, %1;" : "=r"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 h2unpack(uint32_t v) {
    float2 f;
    asm("{ .reg .f16 l, h;\n mov.b32 {l, h}, %2;\n cvt.f32.f16 %0, l;\n cvt.f32.f16 %1, h; }"
        : "=f"(f.x), "=f"(f.y) : "r"(v));
    return f;
}

// A fragments of every (M tile, K step) in lane order: word
// ((mt KT + kk) 2 + hl) 4 + r) 32 + lane, hl = 0 hi, 1 lo.
template <int NT>
__device__ __forceinline__ void tc_stage_fragments(const int16_t* sAq, uint32_t* sAf, int tid, int T) {
    using S = TcShape<NT>;
    constexpr int n = S::n;
    for (int idx = tid; idx < S::MT * S::KT * 4 * 32; idx += T) {
        const int ln = idx & 31, r = (idx >> 5) & 3, tile = idx >> 7;
        const int mt = tile / S::KT, kk = tile % S::KT;
        const int g = ln >> 2, tg = ln & 3;
        const int row = mt * 16 + g + ((r & 1) ? 8 : 0);
        const int col = kk * 16 + 2 * tg + ((r & 2) ? 8 : 0);
        const float a0 = (float)sAq[row * n + col] * 0x1p-14f, a1 = (float)sAq[row * n + col + 1] * 0x1p-14f;
        const uint32_t hi = h2pack(a0, a1);
        const float2 hf = h2unpack(hi);
        const uint32_t lo = h2pack(a0 - hf.x, a1 - hf.y);  // exact: the codes have at most 15 bits
        sAf[((tile * 2 + 0) * 4 + r) * 32 + ln] = hi;
        sAf[((tile * 2 + 1) * 4 + r) * 32 + ln] = lo;
    }
}

// Tensor-core refresh + L frozen Euler steps (packed FP32).  TPA threads per
// anneal (1 or 2): the warp's 32 / TPA anneals are the N columns of the MMA;
// thread q of an anneal owns rows [q NS, (q+1) NS) (NS = n / TPA), writes
// them into its anneal's row of U^T, reads them back from M^T, and keeps the
// auxiliary spin redundantly (mu_a: this thread's part of b^T u plus the
// partner's, by shuffle; the same sum on both threads).
template <int NT, int L, int TPA = 1>
__device__ __forceinline__ void tc_block(const uint32_t* sAf, const float* sh, const float* snd, uint32_t* wsm,
                                         float (&x1)[2 * NT / TPA], float (&x2)[2 * NT / TPA],
                                         float (&e1)[2 * NT / TPA], float (&e2)[2 * NT / TPA], float& xa,
                                         float& ea, int lane, int Lrt, float mscale, const EulerConsts& k) {
    using S = TcShape<NT>;
    constexpr int n = S::n;
    constexpr int NS = n / TPA;      // rows per thread
    constexpr int AW = 32 / TPA;     // anneals per warp
    constexpr int NTL = AW / 8;      // N tiles
    static_assert(TPA == 1 || TPA == 2, "one or two threads per anneal");
    static_assert(NS % 8 == 0, "whole uint4 stores of U^T");
    asm volatile("" ::: "memory");
    const int q = lane % TPA, rl = lane / TPA, row0 = q * NS;
    uint32_t* sUh = wsm;
    uint32_t* sUl = wsm + AW * S::UW;
    float* sM = reinterpret_cast<float*>(wsm);
    // u = x1 + x2 and this thread's part of mu_a = b^T u (FP32, ascending j); FP16 split of 2^5 u into
    // this thread's half of row rl of U^T
    float mua = 0.0f;
#pragma unroll
    for (int w4 = 0; w4 < NS / 8; ++w4) {
        uint32_t hv[4], lv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int j = 8 * w4 + 2 * t;
            const float2 u2 = __fadd2_rn(make_float2(x1[j], x1[j + 1]), make_float2(x2[j], x2[j + 1]));
            mua = fmarn(sh[row0 + j], u2.x, mua);
            mua = fmarn(sh[row0 + j + 1], u2.y, mua);
            const float2 us = __fmul2_rn(u2, make_float2(32.0f, 32.0f));
            hv[t] = h2pack(us.x, us.y);
            const float2 hf = h2unpack(hv[t]);
            lv[t] = h2pack(__fsub_rn(us.x, hf.x), __fsub_rn(us.y, hf.y));
        }
        const int wo = rl * S::UW + row0 / 2 + 4 * w4;
        *reinterpret_cast<uint4*>(sUh + wo) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
        *reinterpret_cast<uint4*>(sUl + wo) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
    }
    if constexpr (TPA == 2) mua = addrn(mua, __shfl_xor_sync(0xffffffffu, mua, 1));
    __syncwarp();
    const int g = lane >> 2, tg = lane & 3;
    float acc[S::MT][NTL][4];
#pragma unroll
    for (int mt = 0; mt < S::MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NTL; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[mt][nt][c] = 0.0f;
#pragma unroll
    for (int kk = 0; kk < S::KT; ++kk) {
        uint32_t ah[S::MT][4], al[S::MT][4];
#pragma unroll
        for (int mt = 0; mt < S::MT; ++mt)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                ah[mt][r] = sAf[(((mt * S::KT + kk) * 2 + 0) * 4 + r) * 32 + lane];
                al[mt][r] = sAf[(((mt * S::KT + kk) * 2 + 1) * 4 + r) * 32 + lane];
            }
#pragma unroll
        for (int nt = 0; nt < NTL; ++nt) {
            const int row = (nt * 8 + g) * S::UW + kk * 8 + tg;
            const uint32_t bh[2] = {sUh[row], sUh[row + 4]};
            const uint32_t bl[2] = {sUl[row], sUl[row + 4]};
#pragma unroll
            for (int mt = 0; mt < S::MT; ++mt) {  // small terms first
                mma16816(acc[mt][nt], al[mt], bh, 1);
                mma16816(acc[mt][nt], ah[mt], bl, 1);
                mma16816(acc[mt][nt], ah[mt], bh, 1);
            }
        }
    }
    __syncwarp();  // every lane's B loads are done before M^T overwrites U^T
#pragma unroll
    for (int mt = 0; mt < S::MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NTL; ++nt) {
            const int r0 = nt * 8 + 2 * tg, i0 = mt * 16 + g;
            sM[r0 * S::MW + i0] = acc[mt][nt][0];
            sM[(r0 + 1) * S::MW + i0] = acc[mt][nt][1];
            sM[r0 * S::MW + i0 + 8] = acc[mt][nt][2];
            sM[(r0 + 1) * S::MW + i0 + 8] = acc[mt][nt][3];
        }
    __syncwarp();
    float m[NS];
#pragma unroll
    for (int i4 = 0; i4 < NS / 4; ++i4) {
        const float4 v = *reinterpret_cast<const float4*>(sM + rl * S::MW + row0 + 4 * i4);
        const float2 lo = __fmul2_rn(make_float2(v.x, v.y), make_float2(mscale, mscale));
        const float2 hi = __fmul2_rn(make_float2(v.z, v.w), make_float2(mscale, mscale));
        m[4 * i4] = lo.x;
        m[4 * i4 + 1] = lo.y;
        m[4 * i4 + 2] = hi.x;
        m[4 * i4 + 3] = hi.y;
    }
    __syncwarp();  // the next refresh rewrites this warp's buffer
    const float2 xa2 = make_float2(xa, xa);
    const float2 cdt = make_float2(k.cdt, k.cdt), c1 = make_float2(k.c1, k.c1);
    const float2 cz = make_float2(k.cz, k.cz), c2 = make_float2(k.c2, k.c2);
#pragma unroll
    for (int i = 0; i < NS; i += 2) {
        const float2 hh = *reinterpret_cast<const float2*>(sh + row0 + i);
        const float2 nd = *reinterpret_cast<const float2*>(snd + row0 + i);
        const float2 c = __ffma2_rn(hh, xa2, make_float2(m[i], m[i + 1]));
        float2 X1 = make_float2(x1[i], x1[i + 1]), X2 = make_float2(x2[i], x2[i + 1]);
        float2 E1 = make_float2(e1[i], e1[i + 1]), E2 = make_float2(e2[i], e2[i + 1]);
        const float2 mu1 = __ffma2_rn(nd, X1, c);
        const float2 mu2 = __ffma2_rn(nd, X2, c);
        if constexpr (L > 0) {
#pragma unroll
            for (int s = 0; s < L; ++s) {
                euler_pair(X1, E1, mu1, cdt, c1, cz, c2);
                euler_pair(X2, E2, mu2, cdt, c1, cz, c2);
            }
        } else {
#pragma unroll 1
            for (int s = 0; s < Lrt; ++s) {
                euler_pair(X1, E1, mu1, cdt, c1, cz, c2);
                euler_pair(X2, E2, mu2, cdt, c1, cz, c2);
            }
        }
        x1[i] = X1.x; x1[i + 1] = X1.y; x2[i] = X2.x; x2[i + 1] = X2.y;
        e1[i] = E1.x; e1[i + 1] = E1.y; e2[i] = E2.x; e2[i + 1] = E2.y;
    }
    if constexpr (L > 0) {
#pragma unroll
        for (int s = 0; s < L; ++s) euler_spin(xa, ea, mua, k);
    } else {
#pragma unroll 1
        for (int s = 0; s < Lrt; ++s) euler_spin(xa, ea, mua, k);
    }
}

template <int NT, int F, int TPA, bool PACKED, bool TC = false, bool PAIR = false>
__global__ void __launch_bounds__(128 * TPA) cac_solve_tuned_kernel(SolveArgs a) {
    constexpr int n = 2 * NT;
    constexpr int NS = n / TPA;
    static_assert(n % TPA == 0 && NS % 4 == 0, "rows per thread must be a multiple of 4");
    static_assert(F > 0, "compile-time refresh period");
    static_assert(!TC || (TPA <= 2 && PACKED && n % 16 == 0), "tensor-core refresh: 1 or 2 threads per anneal");
    __shared__ __align__(16) SolveSmem<NT> sm;
    __shared__ long long skey[4 * TPA];
    __shared__ int sdiv[4 * TPA];
    __shared__ __align__(16) uint32_t tc_af[TC ? TcShape<NT>::AF_WORDS : 1];
    extern __shared__ __align__(16) uint32_t tc_ws[];  // TC: TcShape<NT>::warp_words(32 / TPA) per warp (dynamic)
    const int p = blockIdx.x;
    const int tid = threadIdx.x, T = blockDim.x;
    const int q = tid % TPA, run = tid / TPA;
    const int lane = tid & 31, warp = tid >> 5;
    const int row0 = q * NS;
    const EulerConsts k = a.k;
    {
        const int16_t* Aq = a.Aq + (size_t)p * n * n;
        for (int e = tid; e < n * n; e += T) {
            const int16_t v = Aq[e];
            sm.Aq[e] = v;
            sm.A[e] = mulrn(mulrn((float)v, 0x1p-14f), k.ce);
        }
        const int16_t* hq = a.hq + (size_t)p * n;
        for (int i = tid; i < n; i += T) {
            const int16_t v = hq[i];
            sm.hq[i] = v;
            sm.h[i] = mulrn(mulrn((float)v, 0x1p-14f), k.ce);
            sm.g[i] = a.g ? a.g[(size_t)p * n + i] : (int8_t)0;
        }
    }
    __syncthreads();
    for (int i = tid; i < n; i += T) sm.nd[i] = -sm.A[i * n + i];
    if constexpr (TC) tc_stage_fragments<NT>(sm.Aq, tc_af, tid, T);
    __syncthreads();

    // Philox initial amplitudes of this thread's spins (k = row, n + row, 2n)
    float x1[NS], x2[NS], e1[NS], e2[NS], xa, ea = 1.0f;
    {
        const uint64_t pg = a.problem_offset + (uint64_t)p;
        const uint32_t c2 = (uint32_t)pg, c3 = (uint32_t)(pg >> 32);
#pragma unroll
        for (int b = 0; b < NS / 4; ++b) {
            const U4 w1 = philox4x32_10(U4{(uint32_t)((row0 >> 2) + b), (uint32_t)run, c2, c3}, a.key0, a.key1);
            const U4 w2 = philox4x32_10(U4{(uint32_t)(((n + row0) >> 2) + b), (uint32_t)run, c2, c3}, a.key0, a.key1);
            const uint32_t v1[4] = {w1.x, w1.y, w1.z, w1.w}, v2[4] = {w2.x, w2.y, w2.z, w2.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                x1[4 * b + t] = mulrn((float)((int)(v1[t] >> 8) - 8388608), k.xs);
                x2[4 * b + t] = mulrn((float)((int)(v2[t] >> 8) - 8388608), k.xs);
                e1[4 * b + t] = 1.0f;
                e2[4 * b + t] = 1.0f;
            }
        }
        const U4 wa = philox4x32_10(U4{(uint32_t)((2 * n) >> 2), (uint32_t)run, c2, c3}, a.key0, a.key1);
        xa = mulrn((float)((int)(wa.x >> 8) - 8388608), k.xs);  // 2n is a multiple of 4: word 0
    }

    const int S = a.steps;
    int t = 0;
    if constexpr (TC) {
        uint32_t* wsm = tc_ws + warp * TcShape<NT>::warp_words(32 / TPA);
        const float mscale = mulrn(k.ce, 0x1p-5f);  // eps dt, and the 2^5 of u
#pragma unroll 1
        for (; t + F <= S; t += F)
            tc_block<NT, F, TPA>(tc_af, sm.h, sm.nd, wsm, x1, x2, e1, e2, xa, ea, lane, F, mscale, k);
        if (t < S) tc_block<NT, 0, TPA>(tc_af, sm.h, sm.nd, wsm, x1, x2, e1, e2, xa, ea, lane, S - t, mscale, k);
    } else {
#pragma unroll 1
        for (; t + F <= S; t += F)
            tuned_block<n, NS, TPA, PACKED, F, PAIR>(sm.A, sm.h, sm.nd, x1, x2, e1, e2, xa, ea, q, lane, F, k);
        if (t < S)
            tuned_block<n, NS, TPA, PACKED, 0, PAIR>(sm.A, sm.h, sm.nd, x1, x2, e1, e2, xa, ea, q, lane, S - t, k);
    }

    // validity over the whole anneal
    bool valid = (fabsf(xa) <= k.x_max) && (ea > 0.0f);
#pragma unroll
    for (int i = 0; i < NS; ++i)
        valid = valid && (fabsf(x1[i]) <= k.x_max) && (e1[i] > 0.0f) && (fabsf(x2[i]) <= k.x_max) && (e2[i] > 0.0f);
#pragma unroll
    for (int o = 1; o < TPA; o <<= 1) valid = __shfl_xor_sync(0xffffffffu, (int)valid, o) && valid;
    // offsets of this thread's rows, then the whole anneal's (2-bit codes)
    const int sa = xa >= 0.0f ? 1 : -1;
    int dmine[NS];
    uint64_t code = 0;  // 2-bit two's-complement offset per row
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const int s1 = x1[i] >= 0.0f ? 1 : -1, s2 = x2[i] >= 0.0f ? 1 : -1;
        int di = sa * (s1 + s2) / 2;
        if (a.level_max > 0) {
            const int xv = (int)sm.g[row0 + i] + 2 * di;
            if (xv > a.level_max || xv < -a.level_max) di = 0;
        }
        dmine[i] = di;
        code |= (uint64_t)(di & 3) << (2 * i);
    }
    int d[n];
    {
        const int base = lane & ~(TPA - 1);
#pragma unroll
        for (int qq = 0; qq < TPA; ++qq) {
            const uint64_t c = TPA == 1 ? code : __shfl_sync(0xffffffffu, code, base | qq);
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                const int v = (int)((c >> (2 * i)) & 3u);
                d[qq * NS + i] = v == 3 ? -1 : v;
            }
        }
    }
    // exact quantised energy: this thread's rows, then summed over the anneal
    int E = 0;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        int r = 0;
#pragma unroll
        for (int j = 0; j < n; ++j) r += (int)sm.Aq[(row0 + i) * n + j] * d[j];
        E -= dmine[i] * r;
        E -= (int)sm.hq[row0 + i] * dmine[i];
    }
#pragma unroll
    for (int o = 1; o < TPA; o <<= 1) E += __shfl_xor_sync(0xffffffffu, E, o);
    const bool keep = valid && E <= 0;
    const int Ec = keep ? E : 0;
    long long key = (long long)Ec * 4294967296LL + (long long)run;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long other = __shfl_xor_sync(0xffffffffu, key, o);
        key = other < key ? other : key;
    }
    const unsigned divmask = __ballot_sync(0xffffffffu, !valid && q == 0);
    if (lane == 0) {
        skey[warp] = key;
        sdiv[warp] = __popc(divmask);
    }
    __syncthreads();
    long long best = skey[0];
    int ndiv = sdiv[0];
    for (int w = 1; w < T / 32; ++w) {
        best = skey[w] < best ? skey[w] : best;
        ndiv += sdiv[w];
    }
    const int best_run = (int)(best & 0xffffffffLL);
    if (run == best_run) {
        if (a.d_out) {
#pragma unroll
            for (int i = 0; i < NS; ++i) a.d_out[(size_t)p * n + row0 + i] = keep ? (int8_t)dmine[i] : (int8_t)0;
        }
        if (q == 0) {
            const int bestE = (int)((best - (long long)best_run) / 4294967296LL);
            if (a.E_out) a.E_out[p] = bestE;
            if (a.run_out) a.run_out[p] = best_run;
            if (a.ndiv_out) a.ndiv_out[p] = ndiv;
            if (a.x_out) {
#pragma unroll
                for (int i = 0; i < n; ++i)
                    a.x_out[(size_t)p * n + i] = (int8_t)((int)sm.g[i] + 2 * (keep ? d[i] : 0));
            }
            if (a.sym_out) {
                const int side = 1 << (a.mod_bits >> 1), L = side - 1;
                uint8_t* so = a.sym_out + (size_t)p * NT;
#pragma unroll
                for (int i = 0; i < NT; ++i) {
                    const int xr = (int)sm.g[i] + 2 * (keep ? d[i] : 0);
                    const int xi = (int)sm.g[NT + i] + 2 * (keep ? d[NT + i] : 0);
                    so[i] = (uint8_t)(((xr + L) / 2) * side + (xi + L) / 2);
                }
            }
        }
    }
}

// =========================================================================
// tcgen05 field refresh (solver shape 8; a precision variant like shape 5,
// the same FP16-split product, on the fifth-generation tensor cores).
// One CTA of 128 threads is the 128 rows of one UMMA tile: PP = 128 / runs
// problems of `runs` anneals, one thread per anneal.  At each refresh every
// thread writes its anneal's 2^5 u (u = x1 + x2, split into an FP16 pair) as
// one row of U^T in shared memory; one thread issues D = U^T C^T with C the
// PP problems' couplings c 2^-14 (an exact FP16 pair) stacked along N, so
// N = PP n and the cross-problem blocks of D are computed but never read --
// unless the tile's problems carry identical couplings (one channel), when
// one C serves all of them and N = n.
// D = Uh Cl + Ul Ch + Uh Ch accumulates in FP32 in tensor memory (TMEM); its
// row r is anneal r, and one tcgen05.ld hands each thread its own row -- the
// field m of its problem's n columns -- with no shared-memory round trip.
// Both operands are K-major without swizzle: core matrices of 8 rows x 16
// bytes, 128 B apart along K (LBO) and 16 n B apart per 8 rows (SBO).
// Every wait on the MMA's completion barrier is bounded (kUmmaWaitNs); on
// expiry the CTA stops annealing, reports its problems' guesses as if every
// anneal had diverged, sets bit 1 of the device error word, waits once more
// (bounded) for the MMA in flight and frees its TMEM.
// =========================================================================

constexpr unsigned long long kUmmaWaitNs = 200000000ull;  // 0.2 s; an MMA here takes microseconds

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, LBO, SBO (all >> 4),
// descriptor version 1, base offset 0, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D FP32, A and B FP16, both K-major, M = 128.
__host__ __device__ constexpr uint32_t umma_idesc_f16(int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         int accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void tc05_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc05_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of parity `parity` to complete; false if it has not
// within kUmmaWaitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity) {
    if (mbar_try_wait(mbar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(mbar, parity))
        if (global_ns() - t0 > kUmmaWaitNs) return false;
    return true;
}

// TMEM allocation and release (whole warp, converged).
__device__ __forceinline__ void tmem_alloc(uint32_t slot_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// This thread's TMEM lane, NC consecutive 32-bit columns from taddr, and the
// wait for the load in the same statement (the registers are not read before it).
__device__ __forceinline__ void tmem_ld_row(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_row(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        " tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory layout of one CTA (bytes), for PP problems of n = 2 NT spins.
template <int NT>
struct UmmaSmem {
    static constexpr int n = 2 * NT;
    static constexpr int SBO = 16 * n;              // bytes per 8-row group of a K-major FP16 plane
    static constexpr int U_PLANE = 128 * 2 * n;     // U^T: 128 rows x n FP16
    int pp;
    __host__ __device__ constexpr UmmaSmem(int pp_) : pp(pp_) {}
    __host__ __device__ constexpr int c_plane() const { return pp * n * 2 * n; }  // C: PP n rows x n FP16
    __host__ __device__ constexpr int off_uh() const { return 0; }
    __host__ __device__ constexpr int off_ul() const { return U_PLANE; }
    __host__ __device__ constexpr int off_ch() const { return 2 * U_PLANE; }
    __host__ __device__ constexpr int off_cl() const { return 2 * U_PLANE + c_plane(); }
    __host__ __device__ constexpr int off_aq() const { return 2 * U_PLANE + 2 * c_plane(); }   // int16 [PP][n][n]
    __host__ __device__ constexpr int off_hq() const { return off_aq() + pp * n * n * 2; }    // int16 [PP][n]
    __host__ __device__ constexpr int off_h() const { return off_hq() + pp * n * 2; }         // float [PP][n]
    __host__ __device__ constexpr int off_nd() const { return off_h() + pp * n * 4; }         // float [PP][n]
    __host__ __device__ constexpr int off_g() const { return off_nd() + pp * n * 4; }         // int8 [PP][n]
    __host__ __device__ constexpr int bytes() const { return off_g() + ((pp * n + 15) & ~15); }
};

// Refresh through the tensor cores + L frozen Euler steps (L == 0: runtime
// Lrt).  Returns false, without stepping, once any thread of the CTA has met
// an expired wait (the decision is CTA-uniform).
template <int NT, int L>
__device__ __forceinline__ bool umma_block(uint8_t* su_h, uint8_t* su_l, uint32_t a_h, uint32_t a_l, uint32_t c_h,
                                           uint32_t c_l, uint32_t idesc, uint32_t d_tmem, uint32_t my_cols,
                                           uint32_t mbar, uint32_t& phase, bool& failed, const float* sh,
                                           const float* snd, float (&x1)[2 * NT], float (&x2)[2 * NT],
                                           float (&e1)[2 * NT], float (&e2)[2 * NT], float& xa, float& ea, int tid,
                                           int Lrt, float mscale, const EulerConsts& k) {
    constexpr int n = 2 * NT;
    constexpr int SBO = UmmaSmem<NT>::SBO;
    asm volatile("" ::: "memory");
    // u = x1 + x2, mu_a = b^T u (FP32, ascending j), FP16 split of 2^5 u into row tid of U^T
    float mua = 0.0f;
    const int rowoff = (tid >> 3) * SBO + (tid & 7) * 16;
#pragma unroll
    for (int c = 0; c < n / 8; ++c) {
        uint32_t hv[4], lv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int j = 8 * c + 2 * t;
            const float2 u2 = __fadd2_rn(make_float2(x1[j], x1[j + 1]), make_float2(x2[j], x2[j + 1]));
            mua = fmarn(sh[j], u2.x, mua);
            mua = fmarn(sh[j + 1], u2.y, mua);
            const float2 us = __fmul2_rn(u2, make_float2(32.0f, 32.0f));
            hv[t] = h2pack(us.x, us.y);
            const float2 hf = h2unpack(hv[t]);
            lv[t] = h2pack(__fsub_rn(us.x, hf.x), __fsub_rn(us.y, hf.y));
        }
        *reinterpret_cast<uint4*>(su_h + rowoff + 128 * c) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
        *reinterpret_cast<uint4*>(su_l + rowoff + 128 * c) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
    }
    fence_async_smem();  // the generic-proxy rows become visible to the tensor cores
    tc05_fence_before();
    const int stop = __syncthreads_or(failed ? 1 : 0);
    tc05_fence_after();
    if (stop) return false;
    if (tid == 0) {
#pragma unroll
        for (int kk = 0; kk < n / 16; ++kk) {  // K steps of 16: two core matrices, 256 B
            const uint32_t o = 256u * kk;
            const uint64_t ah = umma_desc(a_h + o, 128, SBO), al = umma_desc(a_l + o, 128, SBO);
            const uint64_t ch = umma_desc(c_h + o, 128, SBO), cl = umma_desc(c_l + o, 128, SBO);
            umma_f16(d_tmem, ah, cl, idesc, kk > 0);  // small terms first
            umma_f16(d_tmem, al, ch, idesc, 1);
            umma_f16(d_tmem, ah, ch, idesc, 1);
        }
        umma_commit(mbar);
    }
    const bool ok = mbar_wait_bounded(mbar, phase);
    if (!ok) {
        failed = true;
        return true;  // the next barrier (or the caller's) stops the CTA
    }
    phase ^= 1u;
    tc05_fence_after();
    float m[n];
    tmem_ld_row(my_cols, m);
    const float2 xa2 = make_float2(xa, xa);
    const float2 ms2 = make_float2(mscale, mscale);
    const float2 cdt = make_float2(k.cdt, k.cdt), c1 = make_float2(k.c1, k.c1);
    const float2 cz = make_float2(k.cz, k.cz), c2 = make_float2(k.c2, k.c2);
#pragma unroll
    for (int i = 0; i < n; i += 2) {
        const float2 mm = __fmul2_rn(make_float2(m[i], m[i + 1]), ms2);
        const float2 hh = *reinterpret_cast<const float2*>(sh + i);
        const float2 nd = *reinterpret_cast<const float2*>(snd + i);
        const float2 c = __ffma2_rn(hh, xa2, mm);
        float2 X1 = make_float2(x1[i], x1[i + 1]), X2 = make_float2(x2[i], x2[i + 1]);
        float2 E1 = make_float2(e1[i], e1[i + 1]), E2 = make_float2(e2[i], e2[i + 1]);
        const float2 mu1 = __ffma2_rn(nd, X1, c);
        const float2 mu2 = __ffma2_rn(nd, X2, c);
        if constexpr (L > 0) {
#pragma unroll
            for (int s = 0; s < L; ++s) {
                euler_pair(X1, E1, mu1, cdt, c1, cz, c2);
                euler_pair(X2, E2, mu2, cdt, c1, cz, c2);
            }
        } else {
#pragma unroll 1
            for (int s = 0; s < Lrt; ++s) {
                euler_pair(X1, E1, mu1, cdt, c1, cz, c2);
                euler_pair(X2, E2, mu2, cdt, c1, cz, c2);
            }
        }
        x1[i] = X1.x; x1[i + 1] = X1.y; x2[i] = X2.x; x2[i + 1] = X2.y;
        e1[i] = E1.x; e1[i + 1] = E1.y; e2[i] = E2.x; e2[i + 1] = E2.y;
    }
    if constexpr (L > 0) {
#pragma unroll
        for (int s = 0; s < L; ++s) euler_spin(xa, ea, mua, k);
    } else {
#pragma unroll 1
        for (int s = 0; s < Lrt; ++s) euler_spin(xa, ea, mua, k);
    }
    return true;
}

// One CTA-tile of shape 8: the 128 / runs problems starting at T's base,
// annealed, selected and written.  Called by all 128 threads of the CTA with
// `usm` the CTA's dynamic shared memory (UmmaSmem<NT>(128 / runs).bytes()).
struct UmmaTile {
    const int16_t* Aq;      // couplings of the tile's first problem ([n][n] per problem)
    const int16_t* hq;      // fields ([n] per problem)
    const int8_t* g;        // guesses ([n] per problem) or nullptr (0)
    int n_live;             // problems of the tile that exist (the rest run on zeros)
    uint64_t problem0;      // Philox problem index of the first problem
    uint32_t key0, key1;
    int level_max;          // clip offsets to the alphabet (0: no clipping)
    int steps;
    EulerConsts k;
    int* err;               // device error word or nullptr
    // outputs for the tile's first problem (each may be nullptr)
    int8_t* d_out;          // [n] offsets (0 where the guess was kept)
    int32_t* E_out;
    int32_t* run_out;
    int32_t* ndiv_out;
    int8_t* x_out;          // [n] g + 2d
    int8_t* guess_out;      // [n] g
    uint8_t* sym_out;       // [n_t] decoded symbols
    int mod_bits;
};

template <int NT, int F>
__device__ __forceinline__ void umma_tile(const UmmaTile& a, int runs, uint8_t* usm) {
    constexpr int n = 2 * NT;
    static_assert(n % 16 == 0 && F > 0, "tcgen05 refresh: n a multiple of 16, compile-time refresh period");
    __shared__ __align__(8) uint64_t mbar_store;
    __shared__ uint32_t tmem_slot;
    __shared__ long long skey[4];
    __shared__ int sdiv[4];
    const int PP = 128 / runs;
    const UmmaSmem<NT> L(PP);
    const int N = PP * n;
    const uint32_t ncols = N < 32 ? 32u : (uint32_t)N;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int pl = tid / runs, run = tid % runs;
    const bool live = pl < a.n_live;
    const EulerConsts k = a.k;
    int16_t* sAq = reinterpret_cast<int16_t*>(usm + L.off_aq());
    int16_t* shq = reinterpret_cast<int16_t*>(usm + L.off_hq());
    float* sh = reinterpret_cast<float*>(usm + L.off_h());
    float* snd = reinterpret_cast<float*>(usm + L.off_nd());
    int8_t* sg = reinterpret_cast<int8_t*>(usm + L.off_g());
    // stage the PP problems (a missing tail problem is all zeros)
    for (int e = tid; e < PP * n * n; e += 128) sAq[e] = e / (n * n) < a.n_live ? a.Aq[e] : (int16_t)0;
    for (int e = tid; e < PP * n; e += 128) {
        const bool have = e / n < a.n_live;
        const int16_t v = have ? a.hq[e] : (int16_t)0;
        shq[e] = v;
        sh[e] = mulrn(mulrn((float)v, 0x1p-14f), k.ce);
        sg[e] = have && a.g ? a.g[e] : (int8_t)0;
    }
    if (warp == 0) tmem_alloc(smem_u32(&tmem_slot), ncols);
    const uint32_t mbar = smem_u32(&mbar_store);
    if (tid == 0) mbar_init(mbar, 1);
    __syncthreads();
    // couplings c 2^-14 as FP16 pairs (exact: at most 15 significant bits), -diag(A)
    for (int e = tid; e < PP * n * (n / 2); e += 128) {
        const int row = e / (n / 2), j = 2 * (e % (n / 2));  // row = q n + i
        const float a0 = (float)sAq[row * n + j] * 0x1p-14f, a1 = (float)sAq[row * n + j + 1] * 0x1p-14f;
        const uint32_t hi = h2pack(a0, a1);
        const float2 hf = h2unpack(hi);
        const uint32_t lo = h2pack(a0 - hf.x, a1 - hf.y);
        const int off = (row >> 3) * UmmaSmem<NT>::SBO + (j >> 3) * 128 + (row & 7) * 16 + (j & 7) * 2;
        *reinterpret_cast<uint32_t*>(usm + L.off_ch() + off) = hi;
        *reinterpret_cast<uint32_t*>(usm + L.off_cl() + off) = lo;
    }
    for (int e = tid; e < PP * n; e += 128) {
        const int q = e / n, i = e % n;
        snd[e] = -mulrn(mulrn((float)sAq[(q * n + i) * n + i], 0x1p-14f), k.ce);
    }
    // A tile whose problems carry bitwise-identical couplings (one channel, one
    // normaliser: the common case when a channel serves consecutive problems)
    // multiplies by one C: N = n instead of PP n, every warp reading columns 0..n-1.
    int differ = 0;
    for (int e = tid; e < (PP - 1) * n * n; e += 128) differ |= sAq[n * n + e] != sAq[e % (n * n)];
    tc05_fence_before();
    const bool shared_c = __syncthreads_or(differ) == 0;
    tc05_fence_after();
    const uint32_t tmem = tmem_slot;

    // Philox initial amplitudes (the same counters as every other shape)
    float x1[n], x2[n], e1[n], e2[n], xa, ea = 1.0f;
    {
        const uint64_t pg = a.problem0 + (uint64_t)pl;
        const uint32_t c2 = (uint32_t)pg, c3 = (uint32_t)(pg >> 32);
#pragma unroll
        for (int b = 0; b < n / 4; ++b) {
            const U4 w1 = philox4x32_10(U4{(uint32_t)b, (uint32_t)run, c2, c3}, a.key0, a.key1);
            const U4 w2 = philox4x32_10(U4{(uint32_t)((n >> 2) + b), (uint32_t)run, c2, c3}, a.key0, a.key1);
            const uint32_t v1[4] = {w1.x, w1.y, w1.z, w1.w}, v2[4] = {w2.x, w2.y, w2.z, w2.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                x1[4 * b + t] = mulrn((float)((int)(v1[t] >> 8) - 8388608), k.xs);
                x2[4 * b + t] = mulrn((float)((int)(v2[t] >> 8) - 8388608), k.xs);
                e1[4 * b + t] = 1.0f;
                e2[4 * b + t] = 1.0f;
            }
        }
        const U4 wa = philox4x32_10(U4{(uint32_t)((2 * n) >> 2), (uint32_t)run, c2, c3}, a.key0, a.key1);
        xa = mulrn((float)((int)(wa.x >> 8) - 8388608), k.xs);
    }

    uint8_t* su_h = usm + L.off_uh();
    uint8_t* su_l = usm + L.off_ul();
    const uint32_t a_h = smem_u32(su_h), a_l = smem_u32(su_l);
    const uint32_t c_h = smem_u32(usm + L.off_ch()), c_l = smem_u32(usm + L.off_cl());
    const uint32_t idesc = umma_idesc_f16(shared_c ? n : N);
    const uint32_t my_cols = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(shared_c ? 0 : pl * n);
    const float mscale = mulrn(k.ce, 0x1p-5f);  // eps dt, and the 2^5 of u
    const float* shp = sh + pl * n;
    const float* sndp = snd + pl * n;
    uint32_t phase = 0;
    bool failed = false;
    const int S = a.steps;
    int t = 0;
    bool go = true;
#pragma unroll 1
    for (; go && t + F <= S; t += F)
        go = umma_block<NT, F>(su_h, su_l, a_h, a_l, c_h, c_l, idesc, tmem, my_cols, mbar, phase, failed, shp, sndp,
                               x1, x2, e1, e2, xa, ea, tid, F, mscale, k);
    if (go && t < S)
        umma_block<NT, 0>(su_h, su_l, a_h, a_l, c_h, c_l, idesc, tmem, my_cols, mbar, phase, failed, shp, sndp, x1,
                          x2, e1, e2, xa, ea, tid, S - t, mscale, k);
    tc05_fence_before();
    const bool cta_failed = __syncthreads_or(failed ? 1 : 0) != 0;
    if (cta_failed) {
        // one more bounded wait for the MMA in flight, then report
        if (tid == 0) {
            mbar_wait_bounded(mbar, phase);
            if (a.err) atomicOr(a.err, 2);
        }
        __syncthreads();
    }
    if (warp == 0) {
        tc05_fence_after();
        tmem_dealloc(tmem, ncols);
    }

    bool valid = !cta_failed && (fabsf(xa) <= k.x_max) && (ea > 0.0f);
#pragma unroll
    for (int i = 0; i < n; ++i)
        valid = valid && (fabsf(x1[i]) <= k.x_max) && (e1[i] > 0.0f) && (fabsf(x2[i]) <= k.x_max) && (e2[i] > 0.0f);
    const int sa = xa >= 0.0f ? 1 : -1;
    const int8_t* g = sg + pl * n;
    int d[n];
#pragma unroll
    for (int i = 0; i < n; ++i) {
        const int s1 = x1[i] >= 0.0f ? 1 : -1, s2 = x2[i] >= 0.0f ? 1 : -1;
        int di = sa * (s1 + s2) / 2;
        if (a.level_max > 0) {
            const int xv = (int)g[i] + 2 * di;
            if (xv > a.level_max || xv < -a.level_max) di = 0;
        }
        d[i] = di;
    }
    // exact quantised energy of this anneal's offsets
    const int16_t* Aq = sAq + pl * n * n;
    const int16_t* hq = shq + pl * n;
    int E = 0;
#pragma unroll
    for (int i = 0; i < n; ++i) {
        int r = 0;
#pragma unroll
        for (int j = 0; j < n; ++j) r += (int)Aq[i * n + j] * d[j];
        E -= d[i] * r;
        E -= (int)hq[i] * d[i];
    }
    const bool keep = valid && E <= 0;
    const int Ec = keep ? E : 0;
    long long key = (long long)Ec * 4294967296LL + (long long)run;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long other = __shfl_xor_sync(0xffffffffu, key, o);
        key = other < key ? other : key;
    }
    const unsigned divmask = __ballot_sync(0xffffffffu, !valid);
    if (lane == 0) {
        skey[warp] = key;
        sdiv[warp] = __popc(divmask);
    }
    __syncthreads();
    const int wpp = runs / 32, w0 = pl * wpp;  // this problem's warps
    long long best = skey[w0];
    int ndiv = sdiv[w0];
    for (int w = 1; w < wpp; ++w) {
        best = skey[w0 + w] < best ? skey[w0 + w] : best;
        ndiv += sdiv[w0 + w];
    }
    const int best_run = (int)(best & 0xffffffffLL);
    if (live && run == best_run) {
        const int p = pl;  // within the tile
        if (a.d_out) {
#pragma unroll
            for (int i = 0; i < n; ++i) a.d_out[(size_t)p * n + i] = keep ? (int8_t)d[i] : (int8_t)0;
        }
        const int bestE = (int)((best - (long long)best_run) / 4294967296LL);
        if (a.E_out) a.E_out[p] = bestE;
        if (a.run_out) a.run_out[p] = best_run;
        if (a.ndiv_out) a.ndiv_out[p] = ndiv;
        if (a.x_out) {
#pragma unroll
            for (int i = 0; i < n; ++i) a.x_out[(size_t)p * n + i] = (int8_t)((int)g[i] + 2 * (keep ? d[i] : 0));
        }
        if (a.guess_out) {
#pragma unroll
            for (int i = 0; i < n; ++i) a.guess_out[(size_t)p * n + i] = g[i];
        }
        if (a.sym_out) {
            const int side = 1 << (a.mod_bits >> 1), Lv = side - 1;
            uint8_t* so = a.sym_out + (size_t)p * NT;
#pragma unroll
            for (int i = 0; i < NT; ++i) {
                const int xr = (int)g[i] + 2 * (keep ? d[i] : 0);
                const int xi = (int)g[NT + i] + 2 * (keep ? d[NT + i] : 0);
                so[i] = (uint8_t)(((xr + Lv) / 2) * side + (xi + Lv) / 2);
            }
        }
    }
}

template <int NT, int F>
__global__ void __launch_bounds__(128) cac_solve_umma_kernel(SolveArgs a, int runs) {
    constexpr int n = 2 * NT;
    extern __shared__ __align__(128) uint8_t usm[];
    const int PP = 128 / runs;
    const int base = blockIdx.x * PP;
    auto at = [&](auto* ptr, size_t per) { return ptr ? ptr + (size_t)base * per : ptr; };
    UmmaTile t;
    t.Aq = a.Aq + (size_t)base * n * n;
    t.hq = a.hq + (size_t)base * n;
    t.g = at(a.g, n);
    t.n_live = min(PP, a.n_problems - base);
    t.problem0 = a.problem_offset + (uint64_t)base;
    t.key0 = a.key0;
    t.key1 = a.key1;
    t.level_max = a.level_max;
    t.steps = a.steps;
    t.k = a.k;
    t.err = a.err;
    t.d_out = at(a.d_out, n);
    t.E_out = at(a.E_out, 1);
    t.run_out = at(a.run_out, 1);
    t.ndiv_out = at(a.ndiv_out, 1);
    t.x_out = at(a.x_out, n);
    t.guess_out = nullptr;
    t.sym_out = at(a.sym_out, NT);
    t.mod_bits = a.mod_bits;
    umma_tile<NT, F>(t, runs, usm);
}

// =========================================================================
// Batched launch of mixed-size uplink jobs, in two kernels replayed as one
// graph.  The builder runs one warp per problem over the whole batch (all
// jobs, all sizes) into batch scratch; the solver is persistent: warps pull
// problems from one atomic counter over a device job table (largest users
// first), stage the problem's Q14 couplings in shared memory and anneal it
// with 32 anneals on the warp's 32 lanes (one thread per anneal, packed
// FP32).  Results equal the per-job path bit for bit: the Philox counters use
// each problem's index within its own job.
// =========================================================================
struct BatchJob {
    BuildArgs b;            // inputs, n_r, mod_bits, n_problems, n_chan, kappa, err
    int nt;
    int kind;               // 0 detection (built by the batch builder); 1 VPP, built before the
                            // batch: no clipping (guess 0), offsets to offset_out, no symbols
    uint32_t key0, key1;
    long long first;        // batch index of the job's problem 0
    long long tile_first;   // tensor-core solver: index of the job's first 4-problem tile
    int16_t* Aq;            // scratch [P][n][n]
    int16_t* hq;            // scratch [P][n]
    int8_t* g;              // scratch [P][n]
    uint8_t* sym_out;
    int32_t* energy_out;
    int8_t* guess_out;
    int8_t* offset_out;
    int32_t* ndiv_out;
};

struct BatchHeader {
    int n_jobs;
    int pad;
    long long total;             // problems in the batch
    unsigned long long counter;  // next problem to hand out (reset before each run)
    long long tiles;             // 4-problem tiles of the tensor-core solver (no tile spans two jobs)
};

struct BatchArgs {
    const BatchJob* jobs;
    BatchHeader* head;
    int steps;
    EulerConsts k;
    int build_floats;       // builder shared memory per warp (floats)
};

template <int NTMAX>
__host__ __device__ constexpr size_t batch_solve_bytes() {
    return (sizeof(SolveSmem<NTMAX>) + 15) / 16 * 16;
}

__device__ __forceinline__ int batch_find_job(const BatchJob* jobs, int n_jobs, long long w) {
    int lo = 0, hi = n_jobs - 1;  // last job with first <= w
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].first <= w) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Builder over the whole batch: warp w of the grid builds problem w.
template <int NTMAX>
__global__ void __launch_bounds__(kBuildWarps * 32, 8) batch_build_kernel(BatchArgs A) {
    extern __shared__ __align__(16) float bws[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long total = A.head->total;
    const int n_jobs = A.head->n_jobs;
    float* ws = bws + warp * A.build_floats;
    for (long long w = (long long)blockIdx.x * kBuildWarps + warp; w < total;
         w += (long long)gridDim.x * kBuildWarps) {
        const BatchJob& J = A.jobs[batch_find_job(A.jobs, n_jobs, w)];
        if (J.kind != 0) continue;  // built before the batch
        const int p = (int)(w - J.first);
        const int n = 2 * J.nt;
        BuildOut o{J.Aq + (size_t)p * n * n, J.hq + (size_t)p * n, J.g + (size_t)p * n, nullptr, nullptr, nullptr};
        // a register copy of the job's arguments: read through the reference, every field would be
        // reloaded from global memory after each of the builder's global stores
        const BuildArgs b = J.b;
        if (J.nt == 16) {
            if constexpr (NTMAX >= 16) build_problem_warp<16>(b, p, lane, ws, o);
        } else if (J.nt == 8) {
            if constexpr (NTMAX >= 8) build_problem_warp<8>(b, p, lane, ws, o);
        } else {
            build_problem_warp<4>(b, p, lane, ws, o);
        }
    }
}

// Anneal one problem already built into sm (Aq, hq, g) with one warp.
template <int NT, int F>
__device__ __forceinline__ void batch_solve_warp(const BatchArgs& A, const BatchJob& J, int p, int lane,
                                                 SolveSmem<NT>& sm) {
    constexpr int n = 2 * NT;
    const EulerConsts k = A.k;
    for (int e = lane; e < n * n; e += 32) sm.A[e] = mulrn(mulrn((float)sm.Aq[e], 0x1p-14f), k.ce);
    for (int i = lane; i < n; i += 32) sm.h[i] = mulrn(mulrn((float)sm.hq[i], 0x1p-14f), k.ce);
    __syncwarp();
    for (int i = lane; i < n; i += 32) sm.nd[i] = -sm.A[i * n + i];
    __syncwarp();
    const int run = lane;
    float x1[n], x2[n], e1[n], e2[n], xa, ea = 1.0f;
    {
        const uint32_t c2 = (uint32_t)p, c3 = 0u;
#pragma unroll
        for (int b = 0; b < n / 4; ++b) {
            const U4 w1 = philox4x32_10(U4{(uint32_t)b, (uint32_t)run, c2, c3}, J.key0, J.key1);
            const U4 w2 = philox4x32_10(U4{(uint32_t)((n >> 2) + b), (uint32_t)run, c2, c3}, J.key0, J.key1);
            const uint32_t v1[4] = {w1.x, w1.y, w1.z, w1.w}, v2[4] = {w2.x, w2.y, w2.z, w2.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                x1[4 * b + t] = mulrn((float)((int)(v1[t] >> 8) - 8388608), k.xs);
                x2[4 * b + t] = mulrn((float)((int)(v2[t] >> 8) - 8388608), k.xs);
                e1[4 * b + t] = 1.0f;
                e2[4 * b + t] = 1.0f;
            }
        }
        const U4 wa = philox4x32_10(U4{(uint32_t)((2 * n) >> 2), (uint32_t)run, c2, c3}, J.key0, J.key1);
        xa = mulrn((float)((int)(wa.x >> 8) - 8388608), k.xs);
    }
    const int S = A.steps;
    int t = 0;
    {
        // 16 users: the paired refresh (faster there, same bits); fewer users: one anneal per lane
        constexpr bool kPair = NT == 16;
#pragma unroll 1
        for (; t + F <= S; t += F)
            tuned_block<n, n, 1, true, F, kPair>(sm.A, sm.h, sm.nd, x1, x2, e1, e2, xa, ea, 0, lane, F, k);
        if (t < S)
            tuned_block<n, n, 1, true, 0, kPair>(sm.A, sm.h, sm.nd, x1, x2, e1, e2, xa, ea, 0, lane, S - t, k);
    }

    bool valid = (fabsf(xa) <= k.x_max) && (ea > 0.0f);
#pragma unroll
    for (int i = 0; i < n; ++i)
        valid = valid && (fabsf(x1[i]) <= k.x_max) && (e1[i] > 0.0f) && (fabsf(x2[i]) <= k.x_max) && (e2[i] > 0.0f);
    const int level_max = J.kind == 0 ? (1 << (J.b.mod_bits >> 1)) - 1 : 0;  // 0: no clipping
    const int sa = xa >= 0.0f ? 1 : -1;
    int d[n];
#pragma unroll
    for (int i = 0; i < n; ++i) {
        const int s1 = x1[i] >= 0.0f ? 1 : -1, s2 = x2[i] >= 0.0f ? 1 : -1;
        int di = sa * (s1 + s2) / 2;
        const int xv = (int)sm.g[i] + 2 * di;
        if (level_max > 0 && (xv > level_max || xv < -level_max)) di = 0;
        d[i] = di;
    }
    int E = 0;
#pragma unroll
    for (int i = 0; i < n; ++i) {
        int r = 0;
#pragma unroll
        for (int j = 0; j < n; ++j) r += (int)sm.Aq[i * n + j] * d[j];
        E -= d[i] * r;
        E -= (int)sm.hq[i] * d[i];
    }
    const bool keep = valid && E <= 0;
    const int Ec = keep ? E : 0;
    long long key = (long long)Ec * 4294967296LL + (long long)run;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long other = __shfl_xor_sync(0xffffffffu, key, o);
        key = other < key ? other : key;
    }
    const int ndiv = __popc(__ballot_sync(0xffffffffu, !valid));
    const int best_run = (int)(key & 0xffffffffLL);
    if (run == best_run) {
        const int bestE = (int)((key - (long long)best_run) / 4294967296LL);
        if (J.energy_out) J.energy_out[p] = bestE;
        if (J.ndiv_out) J.ndiv_out[p] = ndiv;
        if (J.offset_out) {
#pragma unroll
            for (int i = 0; i < n; ++i) J.offset_out[(size_t)p * n + i] = keep ? (int8_t)d[i] : (int8_t)0;
        }
        if (J.guess_out) {
#pragma unroll
            for (int i = 0; i < n; ++i) J.guess_out[(size_t)p * n + i] = sm.g[i];
        }
        if (J.sym_out) {
            const int side = 1 << (J.b.mod_bits >> 1), L = side - 1;
            uint8_t* so = J.sym_out + (size_t)p * NT;
#pragma unroll
            for (int i = 0; i < NT; ++i) {
                const int xr = (int)sm.g[i] + 2 * (keep ? d[i] : 0);
                const int xi = (int)sm.g[NT + i] + 2 * (keep ? d[NT + i] : 0);
                so[i] = (uint8_t)(((xr + L) / 2) * side + (xi + L) / 2);
            }
        }
    }
    __syncwarp();  // the warp's shared memory is reused by its next problem
}

template <int NT, int F>
__device__ __forceinline__ void batch_solve_problem(const BatchArgs& A, const BatchJob& J, int p, int lane,
                                                    unsigned char* solve_mem) {
    constexpr int n = 2 * NT;
    SolveSmem<NT>& sm = *reinterpret_cast<SolveSmem<NT>*>(solve_mem);
    const int16_t* Aq = J.Aq + (size_t)p * n * n;
    for (int e = lane; e < n * n; e += 32) sm.Aq[e] = Aq[e];
    for (int i = lane; i < n; i += 32) {
        sm.hq[i] = J.hq[(size_t)p * n + i];
        sm.g[i] = J.g ? J.g[(size_t)p * n + i] : (int8_t)0;
    }
    __syncwarp();
    batch_solve_warp<NT, F>(A, J, p, lane, sm);
}

// Grid solver over the batch: one 32-thread CTA per problem (the hardware
// CTA scheduler balances sizes); CTAs past the staged total exit.
template <int NTMAX, int F>
__global__ void __launch_bounds__(32) batch_solve_grid_kernel(BatchArgs A) {
    __shared__ __align__(16) unsigned char ssm[batch_solve_bytes<NTMAX>()];
    const long long w = blockIdx.x;
    if (w >= A.head->total) return;
    const BatchJob& J = A.jobs[batch_find_job(A.jobs, A.head->n_jobs, w)];
    const int p = (int)(w - J.first);
    const int lane = threadIdx.x;
    if (J.nt == 16) {
        if constexpr (NTMAX >= 16) batch_solve_problem<16, F>(A, J, p, lane, ssm);
    } else if (J.nt == 8) {
        if constexpr (NTMAX >= 8) batch_solve_problem<8, F>(A, J, p, lane, ssm);
    } else {
        batch_solve_problem<4, F>(A, J, p, lane, ssm);
    }
}

// Persistent solver over the batch: one warp per problem, problems handed
// out by an atomic counter.
template <int NTMAX, int F>
__global__ void __launch_bounds__(128) batch_solve_kernel(BatchArgs A) {
    __shared__ __align__(16) unsigned char ssm[4 * batch_solve_bytes<NTMAX>()];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* mine = ssm + (size_t)warp * batch_solve_bytes<NTMAX>();
    const int n_jobs = A.head->n_jobs;
    const long long total = A.head->total;
    for (;;) {
        unsigned long long w = 0;
        if (lane == 0) w = atomicAdd(&A.head->counter, 1ULL);
        w = __shfl_sync(0xffffffffu, w, 0);
        if ((long long)w >= total) break;
        const BatchJob& J = A.jobs[batch_find_job(A.jobs, n_jobs, (long long)w)];
        const int p = (int)((long long)w - J.first);
        if (J.nt == 16) {
            if constexpr (NTMAX >= 16) batch_solve_problem<16, F>(A, J, p, lane, mine);
        } else if (J.nt == 8) {
            if constexpr (NTMAX >= 8) batch_solve_problem<8, F>(A, J, p, lane, mine);
        } else {
            batch_solve_problem<4, F>(A, J, p, lane, mine);
        }
    }
}

// Batched tensor-core solver (tcgen05, solver shape 8): one 128-thread CTA
// per tile of 4 consecutive problems of one job; 8- and 16-user tiles run
// umma_tile (the same tiles as mmgap_detect with shape 8, so the same bits),
// 4-user tiles one exact warp per problem.
template <int NTMAX>
__host__ __device__ constexpr size_t batch_umma_bytes() {
    constexpr size_t u = NTMAX >= 8 ? (size_t)UmmaSmem<NTMAX >= 16 ? 16 : 8>(4).bytes() : 0;
    constexpr size_t w = 4 * batch_solve_bytes<4>();
    return u > w ? u : w;
}

template <int NTMAX, int F>
__global__ void __launch_bounds__(128) batch_solve_umma_kernel(BatchArgs A) {
    extern __shared__ __align__(128) uint8_t usm[];
    const long long t = blockIdx.x;
    if (t >= A.head->tiles) return;
    int lo = 0, hi = A.head->n_jobs - 1;  // last job whose tiles start at or before t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (A.jobs[mid].tile_first <= t) lo = mid;
        else hi = mid - 1;
    }
    const BatchJob& J = A.jobs[lo];
    const int base = (int)(t - J.tile_first) * 4;
    const int live = min(4, J.b.n_problems - base);
    if (J.nt >= 8) {
        if constexpr (NTMAX >= 8) {
            const int nt = J.nt, n = 2 * nt;
            UmmaTile u;
            u.Aq = J.Aq + (size_t)base * n * n;
            u.hq = J.hq + (size_t)base * n;
            u.g = J.g ? J.g + (size_t)base * n : nullptr;
            u.n_live = live;
            u.problem0 = (uint64_t)base;
            u.key0 = J.key0;
            u.key1 = J.key1;
            u.level_max = J.kind == 0 ? (1 << (J.b.mod_bits >> 1)) - 1 : 0;
            u.steps = A.steps;
            u.k = A.k;
            u.err = J.b.err;
            u.d_out = J.offset_out ? J.offset_out + (size_t)base * n : nullptr;
            u.E_out = J.energy_out ? J.energy_out + base : nullptr;
            u.run_out = nullptr;
            u.ndiv_out = J.ndiv_out ? J.ndiv_out + base : nullptr;
            u.x_out = nullptr;
            u.guess_out = J.guess_out ? J.guess_out + (size_t)base * n : nullptr;
            u.sym_out = J.sym_out ? J.sym_out + (size_t)base * nt : nullptr;
            u.mod_bits = J.b.mod_bits;
            if (nt == 16) {
                if constexpr (NTMAX >= 16) umma_tile<16, F>(u, 32, usm);
            } else {
                umma_tile<8, F>(u, 32, usm);
            }
        }
    } else {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (warp < live) batch_solve_problem<4, F>(A, J, base + warp, lane, usm + warp * batch_solve_bytes<4>());
    }
}

// =========================================================================
// Precision variant of the Gram (pre-processing, Sec. 3.2): G_c = Hs^H Hs per
// channel with mma.sync m16n8k16 (BF16, FP16 or split BF16x3 operands, FP32
// accumulation).
// With A = [Re Hs^T | Im Hs^T] (n_t x 2 n_r):
//   Re G_c = A [Re Hs; Im Hs],   Im G_c = A [Im Hs; -Re Hs].
// One warp per channel; n_t <= 16 (rows padded to 16), 2 n_r padded to a
// multiple of 16.  Each element of Hs = kappa H is rounded once to FP32 and
// once to the 16-bit type.
// Direct (binary-weighted) mapping build: one warp per problem.  The delta
// builder leaves the guess (as floats), the complex Gram and the matched
// filter in the warp's shared memory; J and c are their exact power-of-two
// expansions:  J_ij = -(2^(b_i + b_j) G_(k_i k_j)) for i != j (0 on the
// diagonal), c_i = 2^(b_i) mf_(k_i), with spin i = k B + b (k: real-form
// dimension, b: bit).  Quantised with the same power-of-two normaliser rule.
template <int NT>
__global__ void __launch_bounds__(kBuildWarps * 32) build_direct_kernel(DirectBuildArgs a) {
    extern __shared__ __align__(16) float smem[];
    constexpr int n = 2 * NT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * kBuildWarps + warp;
    if (p >= a.b.n_problems) return;  // warp-uniform
    const int B = a.B, N = n * B;
    const int n_r = a.b.n_r;
    float* ws = smem + warp * build_smem_floats<NT>(n_r);
    BuildOut o{nullptr, nullptr, a.b.g + (size_t)p * n, nullptr, nullptr, nullptr};
    build_problem_warp<NT>(a.b, p, lane, ws, o);
    int16_t* Jq = a.Jq + (size_t)p * N * N;
    int16_t* cq = a.cq + (size_t)p * N;
    const int c = a.b.chan_index ? a.b.chan_index[p] : p;
    if (c < 0 || c >= a.b.n_chan) {  // flagged by the build: an all-zero problem
        for (int e = lane; e < N * N; e += 32) {
            Jq[e] = 0;
            if (a.J32) a.J32[(size_t)p * N * N + e] = 0.0f;
        }
        for (int i = lane; i < N; i += 32) {
            cq[i] = 0;
            if (a.c32) a.c32[(size_t)p * N + i] = 0.0f;
            if (a.s_ref) a.s_ref[(size_t)p * N + i] = 1;
        }
        if (lane == 0 && a.sigma_exp) a.sigma_exp[p] = 0;
        return;
    }
    const float* Gc = ws + 2 * n_r * NT;
    const float* mv = Gc + 4 * NT * NT + 4 * n_r;
    const float* gv = mv + 2 * NT;
    auto Gr = [&](int k, int kk) -> float {  // real form [[Re, -Im], [Im, Re]]
        const int kb = k % NT, kkb = kk % NT;
        const float re = Gc[2 * (kb * NT + kkb)], im = Gc[2 * (kb * NT + kkb) + 1];
        return (k < NT) == (kk < NT) ? re : (k < NT ? -im : im);
    };
    auto mf = [&](int k) -> float { return k < NT ? mv[2 * k] : mv[2 * (k - NT) + 1]; };
    float mx = 0.0f;
    for (int e = lane; e < N * N; e += 32) {
        const int i = e / N, j = e % N;
        if (i != j) mx = fmaxf(mx, fabsf(ldexpf(Gr(i / B, j / B), i % B + j % B)));
    }
    for (int i = lane; i < N; i += 32) mx = fmaxf(mx, fabsf(ldexpf(mf(i / B), i % B)));
    mx = warp_max(mx);
    const int se = sigma_exp_f(mx);
    const bool finite = isfinite(mx);
    const float sc = ldexpf(1.0f, kQBits - se);
    for (int e = lane; e < N * N; e += 32) {
        const int i = e / N, j = e % N;
        const float J = i == j ? 0.0f : -ldexpf(Gr(i / B, j / B), i % B + j % B);
        Jq[e] = finite ? (int16_t)(int)rintf(mulrn(J, sc)) : (int16_t)0;
        if (a.J32) a.J32[(size_t)p * N * N + e] = J;
    }
    for (int i = lane; i < N; i += 32) {
        const float cv = ldexpf(mf(i / B), i % B);
        cq[i] = finite ? (int16_t)(int)rintf(mulrn(cv, sc)) : (int16_t)0;
        if (a.c32) a.c32[(size_t)p * N + i] = cv;
    }
    if (a.s_ref)
        for (int i = lane; i < N; i += 32) {  // spins of the guess: bits of (g + 2^B - 1) / 2
            const int u = ((int)gv[i / B] + (1 << B) - 1) / 2;
            a.s_ref[(size_t)p * N + i] = ((u >> (i % B)) & 1) ? (int8_t)1 : (int8_t)-1;
        }
    if (lane == 0 && a.sigma_exp) a.sigma_exp[p] = se;
}

template <int NT>
cudaError_t launch_build_direct_impl(const DirectBuildArgs& a, cudaStream_t s) {
    if (a.b.n_problems <= 0) return cudaSuccess;
    const size_t smem = (size_t)kBuildWarps * build_smem_floats<NT>(a.b.n_r) * sizeof(float);
    cudaError_t err =
        ensure_dynamic_smem<build_direct_kernel<NT>>(smem);
    if (err != cudaSuccess) return err;
    const int blocks = (a.b.n_problems + kBuildWarps - 1) / kBuildWarps;
    build_direct_kernel<NT><<<blocks, kBuildWarps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

// =========================================================================
// General-coupling CIM-CAC solver (direct mapping; any Ising problem with an
// auxiliary spin).  One CTA per problem, TPA threads per anneal: thread q
// owns spins [q NS, (q+1) NS) and keeps the auxiliary spin redundantly.  At
// each refresh the anneal's amplitudes go through a shared-memory row
// (stride N + 1: the rows of a warp's anneals fall in distinct banks), then
// every thread forms its rows of m = J x in ascending j from 0 (the oracle's
// order; packed pairs of rows, each an IEEE fused multiply-add) and the
// whole mu_a = c^T x.  Selection: exact int32 energy, arg-min of
// (E, candidate) with the reference candidate first.
// =========================================================================
template <int N>
__host__ __device__ constexpr int general_tpa() { return N <= 32 ? 1 : (N <= 64 ? 2 : 4); }

// Row j of eps dt J is stored as TPA slices of NS columns, each followed by 4
// floats of padding (row stride N + 4 TPA): the TPA threads of an anneal read
// their slices of one row in the same instruction, and without the padding
// those slices would start 128 bytes apart, in the same banks.
template <int N>
__host__ __device__ constexpr int general_row_stride() { return N + 4 * general_tpa<N>(); }

template <int N, int NS, int L>
__device__ __forceinline__ void general_block(const float* Jmine, const float* cf, float* xrow, float (&x)[NS],
                                              float (&e)[NS], float& xa, float& ea, int row0, int Lrt,
                                              const EulerConsts& k) {
    constexpr int JS = general_row_stride<N>();
    asm volatile("" ::: "memory");
    __syncwarp();  // the anneal's threads finished reading the previous refresh's row
#pragma unroll
    for (int i = 0; i < NS; ++i) xrow[row0 + i] = x[i];
    __syncwarp();
    float m[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) m[i] = 0.0f;
    float mua = 0.0f;
#pragma unroll 4
    for (int j = 0; j < N; ++j) {
        const float xj = xrow[j];
        mua = fmarn(cf[j], xj, mua);
        const float4* row = reinterpret_cast<const float4*>(Jmine + j * JS);
        const float2 xx = make_float2(xj, xj);
#pragma unroll
        for (int i4 = 0; i4 < NS / 4; ++i4) {
            const float4 a4 = row[i4];
            const float2 lo = __ffma2_rn(make_float2(a4.x, a4.y), xx, make_float2(m[4 * i4], m[4 * i4 + 1]));
            const float2 hi = __ffma2_rn(make_float2(a4.z, a4.w), xx, make_float2(m[4 * i4 + 2], m[4 * i4 + 3]));
            m[4 * i4] = lo.x;
            m[4 * i4 + 1] = lo.y;
            m[4 * i4 + 2] = hi.x;
            m[4 * i4 + 3] = hi.y;
        }
    }
    const float2 xa2 = make_float2(xa, xa);
    const float2 cdt = make_float2(k.cdt, k.cdt), c1 = make_float2(k.c1, k.c1);
    const float2 cz = make_float2(k.cz, k.cz), c2 = make_float2(k.c2, k.c2);
#pragma unroll
    for (int i = 0; i < NS; i += 2) {
        const float2 cc = *reinterpret_cast<const float2*>(cf + row0 + i);
        const float2 mu = __ffma2_rn(cc, xa2, make_float2(m[i], m[i + 1]));
        float2 X = make_float2(x[i], x[i + 1]), E = make_float2(e[i], e[i + 1]);
        if constexpr (L > 0) {
#pragma unroll
            for (int s = 0; s < L; ++s) euler_pair(X, E, mu, cdt, c1, cz, c2);
        } else {
#pragma unroll 1
            for (int s = 0; s < Lrt; ++s) euler_pair(X, E, mu, cdt, c1, cz, c2);
        }
        x[i] = X.x;
        x[i + 1] = X.y;
        e[i] = E.x;
        e[i + 1] = E.y;
    }
    if constexpr (L > 0) {
#pragma unroll
        for (int s = 0; s < L; ++s) euler_spin(xa, ea, mua, k);
    } else {
#pragma unroll 1
        for (int s = 0; s < Lrt; ++s) euler_spin(xa, ea, mua, k);
    }
}


template <int N>
__host__ __device__ constexpr size_t general_smem_bytes(int runs) {
    return ((size_t)N * general_row_stride<N>() + N + (size_t)runs * (N + 1)) * sizeof(float);
}

template <int N, int F>
__global__ void __launch_bounds__(256) cac_general_kernel(GeneralArgs a) {
    constexpr int TPA = general_tpa<N>();
    constexpr int NS = N / TPA;
    static_assert(N % TPA == 0 && NS % 4 == 0 && NS <= 32, "rows per thread: a multiple of 4, at most 32");
    extern __shared__ __align__(16) float gsm[];
    constexpr int JS = general_row_stride<N>();
    float* Jf = gsm;         // [N][JS] eps dt J, rows in TPA padded slices
    float* cf = Jf + N * JS; // [N]   eps dt c
    float* Xr = cf + N;      // [runs][N + 1]
    __shared__ long long skey[8];
    __shared__ int sdiv[8];
    __shared__ int sEref;
    const int p = blockIdx.x;
    const int tid = threadIdx.x, T = blockDim.x;
    const int q = tid % TPA, run = tid / TPA;
    const int lane = tid & 31, warp = tid >> 5;
    const int row0 = q * NS;
    const EulerConsts k = a.k;
    const int16_t* Jq = a.Jq + (size_t)p * N * N;
    const int16_t* cq = a.cq + (size_t)p * N;
    const int8_t* sref = a.s_ref ? a.s_ref + (size_t)p * N : nullptr;
    for (int e = tid; e < N * N; e += T) {
        const int j = e / N, i = e % N;
        Jf[j * JS + (i / NS) * (NS + 4) + i % NS] = mulrn(mulrn((float)Jq[e], 0x1p-14f), k.ce);
    }
    for (int i = tid; i < N; i += T) cf[i] = mulrn(mulrn((float)cq[i], 0x1p-14f), k.ce);
    if (tid == 0) sEref = 0;
    __syncthreads();
    // energy of the reference candidate (+1 everywhere when there is none)
    {
        int part = 0;
        for (int i = tid; i < N; i += T) {
            const int si = sref ? (int)sref[i] : 1;
            int r = 0;
            for (int j = 0; j < N; ++j) r += (int)Jq[i * N + j] * (sref ? (int)sref[j] : 1);
            part -= si * r;
            part -= 2 * (int)cq[i] * si;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0 && part != 0) atomicAdd(&sEref, part);
    }

    float x[NS], e[NS], xa, ea = 1.0f;
    {
        const uint64_t pg = a.problem_offset + (uint64_t)p;
        const uint32_t c2 = (uint32_t)pg, c3 = (uint32_t)(pg >> 32);
#pragma unroll
        for (int b = 0; b < NS / 4; ++b) {
            const U4 w = philox4x32_10(U4{(uint32_t)((row0 >> 2) + b), (uint32_t)run, c2, c3}, a.key0, a.key1);
            const uint32_t v[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                x[4 * b + t] = mulrn((float)((int)(v[t] >> 8) - 8388608), k.xs);
                e[4 * b + t] = 1.0f;
            }
        }
        const U4 wa = philox4x32_10(U4{(uint32_t)(N >> 2), (uint32_t)run, c2, c3}, a.key0, a.key1);
        xa = mulrn((float)((int)(wa.x >> 8) - 8388608), k.xs);  // N is a multiple of 4: word 0
    }
    float* xrow = Xr + run * (N + 1);
    const int S = a.steps;
    int t = 0;
    const float* Jmine = Jf + q * (NS + 4);  // this thread's slice of every row
    if constexpr (F > 0) {
#pragma unroll 1
        for (; t + F <= S; t += F) general_block<N, NS, F>(Jmine, cf, xrow, x, e, xa, ea, row0, F, k);
    } else {
        const int f = a.f_mvm;
#pragma unroll 1
        for (; t + f <= S; t += f) general_block<N, NS, 0>(Jmine, cf, xrow, x, e, xa, ea, row0, f, k);
    }
    if (t < S) general_block<N, NS, 0>(Jmine, cf, xrow, x, e, xa, ea, row0, S - t, k);

    bool valid = (fabsf(xa) <= k.x_max) && (ea > 0.0f);
#pragma unroll
    for (int i = 0; i < NS; ++i) valid = valid && (fabsf(x[i]) <= k.x_max) && (e[i] > 0.0f);
#pragma unroll
    for (int o = 1; o < TPA; o <<= 1) valid = __shfl_xor_sync(0xffffffffu, (int)valid, o) && valid;
    const bool sa_pos = xa >= 0.0f;
    uint32_t bits = 0;  // bit i: spin row0 + i is +1 after the gauge s_i = sign(x_i) sign(x_a)
#pragma unroll
    for (int i = 0; i < NS; ++i) bits |= (uint32_t)((x[i] >= 0.0f) == sa_pos) << i;
    uint32_t wds[TPA];
    {
        const int base = lane & ~(TPA - 1);
#pragma unroll
        for (int qq = 0; qq < TPA; ++qq) wds[qq] = TPA == 1 ? bits : __shfl_sync(0xffffffffu, bits, base | qq);
    }
    auto spin = [&](int j) -> int { return ((wds[j / NS] >> (j % NS)) & 1u) ? 1 : -1; };
    int E = 0;
#pragma unroll 1
    for (int i = 0; i < NS; ++i) {
        const int gi = row0 + i;
        const int si = ((bits >> i) & 1u) ? 1 : -1;
        int r = 0;
        for (int j = 0; j < N; ++j) r += (int)__ldg(Jq + gi * N + j) * spin(j);
        E -= si * r;
        E -= 2 * (int)__ldg(cq + gi) * si;
    }
#pragma unroll
    for (int o = 1; o < TPA; o <<= 1) E += __shfl_xor_sync(0xffffffffu, E, o);
    long long key = valid ? (long long)E * 4294967296LL + (long long)(run + 1) : LLONG_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long other = __shfl_xor_sync(0xffffffffu, key, o);
        key = other < key ? other : key;
    }
    const unsigned divmask = __ballot_sync(0xffffffffu, !valid && q == 0);
    if (lane == 0) {
        skey[warp] = key;
        sdiv[warp] = __popc(divmask);
    }
    __syncthreads();
    const long long ref_key = sref ? (long long)sEref * 4294967296LL : LLONG_MAX - 1;
    long long best = ref_key;
    int ndiv = 0;
    for (int w = 0; w < T / 32; ++w) {
        best = skey[w] < best ? skey[w] : best;
        ndiv += sdiv[w];
    }
    const bool ref_wins = best == ref_key;
    const int best_run = ref_wins ? -1 : (int)(best & 0xffffffffLL) - 1;
    const bool writer = ref_wins ? tid == 0 : (run == best_run && q == 0);
    if (!writer) return;
    const int bestE = ref_wins ? sEref : (int)((best - (long long)(best_run + 1)) / 4294967296LL);
    auto out_spin = [&](int j) -> int { return ref_wins ? (sref ? (int)sref[j] : 1) : spin(j); };
    if (a.s_out)
        for (int j = 0; j < N; ++j) a.s_out[(size_t)p * N + j] = (int8_t)out_spin(j);
    if (a.E_out) a.E_out[p] = bestE;
    if (a.run_out) a.run_out[p] = best_run;
    if (a.ndiv_out) a.ndiv_out[p] = ndiv;
    if (a.mod_bits > 0) {
        const int B = a.mod_bits >> 1, side = 1 << B, Lm = side - 1;
        const int nt = N / (2 * B);
        for (int u = 0; u < nt; ++u) {
            int xr = 0, xi = 0;
            for (int b = 0; b < B; ++b) {
                xr += (1 << b) * out_spin(u * B + b);
                xi += (1 << b) * out_spin((nt + u) * B + b);
            }
            if (a.sym_out) a.sym_out[(size_t)p * nt + u] = (uint8_t)(((xr + Lm) / 2) * side + (xi + Lm) / 2);
            if (a.offset_out && a.g) {
                a.offset_out[(size_t)p * 2 * nt + u] = (int8_t)((xr - (int)a.g[(size_t)p * 2 * nt + u]) / 2);
                a.offset_out[(size_t)p * 2 * nt + nt + u] =
                    (int8_t)((xi - (int)a.g[(size_t)p * 2 * nt + nt + u]) / 2);
            }
        }
    }
}

template <int N>
cudaError_t launch_general_impl(const GeneralArgs& a, int runs, cudaStream_t s) {
    if (a.n_problems <= 0) return cudaSuccess;
    constexpr int TPA = general_tpa<N>();
    const int threads = runs * TPA;
    if (runs % 32 || threads > 256) return cudaErrorInvalidConfiguration;
    const size_t smem = general_smem_bytes<N>(runs);
    cudaError_t err;
    if (a.f_mvm == 2) {
        if ((err = ensure_dynamic_smem<cac_general_kernel<N, 2>>(smem)) != cudaSuccess)
            return err;
        cac_general_kernel<N, 2><<<a.n_problems, threads, smem, s>>>(a);
    } else if (a.f_mvm == 1) {
        if ((err = ensure_dynamic_smem<cac_general_kernel<N, 1>>(smem)) != cudaSuccess)
            return err;
        cac_general_kernel<N, 1><<<a.n_problems, threads, smem, s>>>(a);
    } else {
        if ((err = ensure_dynamic_smem<cac_general_kernel<N, 0>>(smem)) != cudaSuccess)
            return err;
        cac_general_kernel<N, 0><<<a.n_problems, threads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

// =========================================================================
template <int NT>
__global__ void __launch_bounds__(128) gram_tc_kernel(GramArgs a) {
    static_assert(NT <= 16, "one 16-row tile");
    extern __shared__ __align__(16) float gsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * 4 + warp;
    if (c >= a.n_chan) return;
    const int n_r = a.n_r;
    const int K = (2 * n_r + 15) / 16 * 16;
    float* Hs = gsm + (size_t)warp * 2 * kMaxNr * NT;  // [n_r][NT] complex
    const float* Hg = a.H + (size_t)c * 2 * n_r * NT;
    for (int e = lane; e < 2 * n_r * NT; e += 32) Hs[e] = mulrn(a.kappa, Hg[e]);
    __syncwarp();
    // element (k', col) of the stacked operands, zero outside the matrix
    auto At = [&](int row, int kk) -> float {  // A[row][kk] = [Re Hs^T | Im Hs^T]
        if (row >= NT || kk >= 2 * n_r) return 0.0f;
        return kk < n_r ? Hs[2 * (kk * NT + row)] : Hs[2 * ((kk - n_r) * NT + row) + 1];
    };
    auto Bre = [&](int kk, int col) -> float {  // [Re Hs; Im Hs]
        if (col >= NT || kk >= 2 * n_r) return 0.0f;
        return kk < n_r ? Hs[2 * (kk * NT + col)] : Hs[2 * ((kk - n_r) * NT + col) + 1];
    };
    auto Bim = [&](int kk, int col) -> float {  // [Im Hs; -Re Hs]
        if (col >= NT || kk >= 2 * n_r) return 0.0f;
        return kk < n_r ? Hs[2 * (kk * NT + col) + 1] : -Hs[2 * ((kk - n_r) * NT + col)];
    };
    const int gid = lane >> 2, tig = lane & 3;
    constexpr int NTILES = (NT + 7) / 8;
    float re[NTILES][4], im[NTILES][4];
#pragma unroll
    for (int t = 0; t < NTILES; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) re[t][q] = im[t][q] = 0.0f;
    // split operands (BF16x3): v = hi + lo with hi = bf16(v), lo = bf16(v - hi);
    // products hi*hi + hi*lo + lo*hi
    const int fp16 = a.fp16 == 1;
    const bool split = a.fp16 == 2;
    auto hi = [&](float v) -> float { return split ? __bfloat162float(__float2bfloat16_rn(v)) : v; };
    auto lo = [&](float v) -> float { return __fsub_rn(v, hi(v)); };
    for (int k0 = 0; k0 < K; k0 += 16) {
        const float av[8] = {At(gid, k0 + 2 * tig), At(gid, k0 + 2 * tig + 1), At(gid + 8, k0 + 2 * tig),
                             At(gid + 8, k0 + 2 * tig + 1), At(gid, k0 + 2 * tig + 8), At(gid, k0 + 2 * tig + 9),
                             At(gid + 8, k0 + 2 * tig + 8), At(gid + 8, k0 + 2 * tig + 9)};
        uint32_t fa[4], fal[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            fa[r] = pack16(hi(av[2 * r]), hi(av[2 * r + 1]), fp16);
            fal[r] = pack16(lo(av[2 * r]), lo(av[2 * r + 1]), fp16);
        }
#pragma unroll
        for (int t = 0; t < NTILES; ++t) {
            const int col = 8 * t + gid;
            const float rv[4] = {Bre(k0 + 2 * tig, col), Bre(k0 + 2 * tig + 1, col), Bre(k0 + 2 * tig + 8, col),
                                 Bre(k0 + 2 * tig + 9, col)};
            const float iv[4] = {Bim(k0 + 2 * tig, col), Bim(k0 + 2 * tig + 1, col), Bim(k0 + 2 * tig + 8, col),
                                 Bim(k0 + 2 * tig + 9, col)};
            uint32_t br[2], bi[2], brl[2], bil[2];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                br[r] = pack16(hi(rv[2 * r]), hi(rv[2 * r + 1]), fp16);
                bi[r] = pack16(hi(iv[2 * r]), hi(iv[2 * r + 1]), fp16);
                brl[r] = pack16(lo(rv[2 * r]), lo(rv[2 * r + 1]), fp16);
                bil[r] = pack16(lo(iv[2 * r]), lo(iv[2 * r + 1]), fp16);
            }
            if (split) {  // small terms first
                mma16816(re[t], fal, br, 0);
                mma16816(re[t], fa, brl, 0);
                mma16816(im[t], fal, bi, 0);
                mma16816(im[t], fa, bil, 0);
            }
            mma16816(re[t], fa, br, fp16);
            mma16816(im[t], fa, bi, fp16);
        }
    }
    // accumulator (row, col): [0] (gid, 2tig) [1] (gid, 2tig+1) [2] (gid+8, 2tig) [3] (gid+8, 2tig+1);
    // write the upper triangle and its Hermitian mirror
    float* G = a.Gc + (size_t)c * 2 * NT * NT;
#pragma unroll
    for (int t = 0; t < NTILES; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int row = gid + (q >= 2 ? 8 : 0), col = 8 * t + 2 * tig + (q & 1);
            if (row >= NT || col >= NT || row > col) continue;
            const float r = re[t][q], m = row == col ? 0.0f : im[t][q];
            G[2 * (row * NT + col)] = r;
            G[2 * (row * NT + col) + 1] = m;
            G[2 * (col * NT + row)] = r;
            G[2 * (col * NT + row) + 1] = -m;
        }
}

template <int NT>
cudaError_t launch_gram_tc_impl(const GramArgs& a, cudaStream_t s) {
    if (a.n_chan <= 0) return cudaSuccess;
    if constexpr (NT > 16) {
        return cudaErrorInvalidValue;
    } else {
        const size_t smem = (size_t)4 * 2 * kMaxNr * NT * sizeof(float);
        cudaError_t err =
            ensure_dynamic_smem<gram_tc_kernel<NT>>(smem);
        if (err != cudaSuccess) return err;
        gram_tc_kernel<NT><<<(a.n_chan + 3) / 4, 128, smem, s>>>(a);
        return cudaGetLastError();
    }
}

// =========================================================================
// MMGaP-E selection (Sec. 3.2.2: the overall best solution is the output):
// one warp per problem evaluates ||y - Hs x||^2 of every lattice candidate in
// FP32 (residual r_k = y_k - sum_j Hs_kj x_j with j ascending, lanes over k;
// then lane 0 sums k ascending) and keeps the first smallest.
// =========================================================================
template <int NT>
__global__ void __launch_bounds__(128) select_kernel(SelectArgs a) {
    extern __shared__ __align__(16) float ssel[];
    constexpr int n = 2 * NT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * 4 + warp;
    if (p >= a.n_problems) return;
    const int n_r = a.n_r;
    float* Hs = ssel + (size_t)warp * (2 * kMaxNr * NT + 2 * kMaxNr + 2 * kMaxNr);
    float* yv = Hs + 2 * kMaxNr * NT;
    float* rr = yv + 2 * kMaxNr;
    int c = a.chan_index ? a.chan_index[p] : p;
    if (c < 0 || c >= a.n_chan) c = 0;  // flagged by the build stage
    const float* Hg = a.H + (size_t)c * 2 * n_r * NT;
    for (int e = lane; e < 2 * n_r * NT; e += 32) Hs[e] = mulrn(a.kappa, Hg[e]);
    for (int e = lane; e < 2 * n_r; e += 32) yv[e] = a.y[(size_t)p * 2 * n_r + e];
    __syncwarp();
    float best_obj = 0.0f;
    int best = 0;
    for (int cand = 0; cand < a.n_cand; ++cand) {
        const int8_t* x = a.cand + ((size_t)cand * a.n_problems + p) * n;
        for (int k = lane; k < n_r; k += 32) {
            float re = yv[2 * k], im = yv[2 * k + 1];
            for (int j = 0; j < NT; ++j) {
                const float ar = Hs[2 * (k * NT + j)], ai = Hs[2 * (k * NT + j) + 1];
                const float br = (float)x[j], bi = (float)x[NT + j];
                re = fmarn(-ar, br, re);
                re = fmarn(ai, bi, re);
                im = fmarn(-ar, bi, im);
                im = fmarn(-ai, br, im);
            }
            rr[2 * k] = re;
            rr[2 * k + 1] = im;
        }
        __syncwarp();
        if (lane == 0) {
            float obj = 0.0f;
            for (int k = 0; k < n_r; ++k) {
                obj = fmarn(rr[2 * k], rr[2 * k], obj);
                obj = fmarn(rr[2 * k + 1], rr[2 * k + 1], obj);
            }
            if (cand == 0 || obj < best_obj) {
                best_obj = obj;
                best = cand;
            }
        }
        __syncwarp();
    }
    best = __shfl_sync(0xffffffffu, best, 0);
    const int8_t* x = a.cand + ((size_t)best * a.n_problems + p) * n;
    const int side = 1 << (a.mod_bits >> 1), L = side - 1;
    if (lane < NT) {
        const int xr = x[lane], xi = x[NT + lane];
        a.sym_out[(size_t)p * NT + lane] = (uint8_t)(((xr + L) / 2) * side + (xi + L) / 2);
    }
    if (lane == 0) {
        if (a.best_out) a.best_out[p] = best;
        if (a.obj_out) a.obj_out[p] = best_obj;
    }
}

template <int NT>
cudaError_t launch_select_impl(const SelectArgs& a, cudaStream_t s) {
    if (a.n_problems <= 0) return cudaSuccess;
    const size_t smem = (size_t)4 * (2 * kMaxNr * NT + 4 * kMaxNr) * sizeof(float);
    cudaError_t err = ensure_dynamic_smem<select_kernel<NT>>(smem);
    if (err != cudaSuccess) return err;
    select_kernel<NT><<<(a.n_problems + 3) / 4, 128, smem, s>>>(a);
    return cudaGetLastError();
}

// =========================================================================
// Downlink VPP (Sec. 3.3) in FP64.
// =========================================================================
constexpr int kVppMaxNt = 64;

// Q = (H H^H)^-1 per channel: one warp per channel.
template <int NU>
__global__ void __launch_bounds__(32) vpp_inverse_kernel(VppInvArgs a) {
    extern __shared__ __align__(16) double dsm[];
    const int c = blockIdx.x;
    if (a.only_failed && a.status[c] == 0) return;
    const int lane = threadIdx.x;
    const int n_t = a.n_t;
    double* Hd = dsm;                    // [NU][n_t] c
    double* K = Hd + 2 * NU * n_t;       // [NU][NU] c
    double* Lc = K + 2 * NU * NU;        // [NU][NU] c
    double* W = Lc + 2 * NU * NU;        // per column c: w [NU] c   ([NU][NU] c)
    double* Cc = W + 2 * NU * NU;        // per column c: col [NU] c ([NU][NU] c)
    __shared__ int fail;
    const float* Hg = a.H + (size_t)c * 2 * NU * n_t;
    for (int e = lane; e < 2 * NU * n_t; e += 32) Hd[e] = (double)Hg[e];
    if (lane == 0) fail = 0;
    __syncwarp();
    for (int t = lane; t < NU * NU; t += 32) {
        const int i = t / NU, j = t % NU;
        if (i > j) continue;
        if (i == j) {
            double acc = 0.0;
            for (int k = 0; k < n_t; ++k) {
                const double ar = Hd[2 * (i * n_t + k)], ai = Hd[2 * (i * n_t + k) + 1];
                acc = __fma_rn(ar, ar, acc);
                acc = __fma_rn(ai, ai, acc);
            }
            K[2 * (i * NU + i)] = acc;
            K[2 * (i * NU + i) + 1] = 0.0;
        } else {
            double re = 0.0, im = 0.0;
            for (int k = 0; k < n_t; ++k) {
                const double ar = Hd[2 * (i * n_t + k)], ai = Hd[2 * (i * n_t + k) + 1];
                const double br = Hd[2 * (j * n_t + k)], bi = Hd[2 * (j * n_t + k) + 1];
                re = __fma_rn(ar, br, re);
                re = __fma_rn(ai, bi, re);
                im = __fma_rn(ai, br, im);
                im = __fma_rn(-ar, bi, im);
            }
            K[2 * (i * NU + j)] = re;
            K[2 * (i * NU + j) + 1] = im;
            K[2 * (j * NU + i)] = re;
            K[2 * (j * NU + i) + 1] = -im;
        }
    }
    __syncwarp();
    for (int j = 0; j < NU; ++j) {
        if (lane == j) {
            double d = K[2 * (j * NU + j)];
            for (int k = 0; k < j; ++k) {
                const double lr = Lc[2 * (j * NU + k)], li = Lc[2 * (j * NU + k) + 1];
                d = __fma_rn(-lr, lr, d);
                d = __fma_rn(-li, li, d);
            }
            const bool ok = (d > 0.0) && !isinf(d);
            if (!ok) fail = 1;
            Lc[2 * (j * NU + j)] = ok ? __dsqrt_rn(d) : 1.0;
            Lc[2 * (j * NU + j) + 1] = 0.0;
        }
        __syncwarp();
        const double ljj = Lc[2 * (j * NU + j)];
        if (lane > j && lane < NU) {
            const int i = lane;
            double re = K[2 * (i * NU + j)], im = K[2 * (i * NU + j) + 1];
            for (int k = 0; k < j; ++k) {
                const double ar = Lc[2 * (i * NU + k)], ai = Lc[2 * (i * NU + k) + 1];
                const double br = Lc[2 * (j * NU + k)], bi = Lc[2 * (j * NU + k) + 1];
                re = __fma_rn(-ar, br, re);
                re = __fma_rn(-ai, bi, re);
                im = __fma_rn(-ai, br, im);
                im = __fma_rn(ar, bi, im);
            }
            Lc[2 * (i * NU + j)] = __ddiv_rn(re, ljj);
            Lc[2 * (i * NU + j) + 1] = __ddiv_rn(im, ljj);
        }
        __syncwarp();
    }
    // lane cc solves K q = e_cc (forward ascending, backward descending); element k of
    // column cc sits at [2 (k NU + cc)], so the lanes' accesses fall in distinct banks
    if (lane < NU) {
        const int cc = lane;
        double* w = W + 2 * cc;
        double* col = Cc + 2 * cc;
        for (int i = 0; i < NU; ++i) {
            double re = (i == cc) ? 1.0 : 0.0, im = 0.0;
            for (int k = 0; k < i; ++k) {
                const double ar = Lc[2 * (i * NU + k)], ai = Lc[2 * (i * NU + k) + 1];
                const double br = w[2 * NU * k], bi = w[2 * NU * k + 1];
                re = __fma_rn(-ar, br, re);
                re = __fma_rn(ai, bi, re);
                im = __fma_rn(-ar, bi, im);
                im = __fma_rn(-ai, br, im);
            }
            const double lii = Lc[2 * (i * NU + i)];
            w[2 * NU * i] = __ddiv_rn(re, lii);
            w[2 * NU * i + 1] = __ddiv_rn(im, lii);
        }
        for (int i = NU - 1; i >= 0; --i) {
            double re = w[2 * NU * i], im = w[2 * NU * i + 1];
            for (int k = NU - 1; k > i; --k) {
                const double ar = Lc[2 * (k * NU + i)], ai = Lc[2 * (k * NU + i) + 1];
                const double br = col[2 * NU * k], bi = col[2 * NU * k + 1];
                re = __fma_rn(-ar, br, re);
                re = __fma_rn(-ai, bi, re);
                im = __fma_rn(-ar, bi, im);
                im = __fma_rn(ai, br, im);
            }
            const double lii = Lc[2 * (i * NU + i)];
            col[2 * NU * i] = __ddiv_rn(re, lii);
            col[2 * NU * i + 1] = __ddiv_rn(im, lii);
        }
    }
    __syncwarp();
    double* Q = a.Q + (size_t)c * 2 * NU * NU;
    const bool failed = fail != 0;
    for (int t = lane; t < NU * NU; t += 32) {
        const int i = t / NU, j = t % NU;
        double re, im;
        if (i <= j) {
            re = Cc[2 * (NU * i + j)];
            im = (i == j) ? 0.0 : Cc[2 * (NU * i + j) + 1];
        } else {
            re = Cc[2 * (NU * j + i)];
            im = -Cc[2 * (NU * j + i) + 1];
        }
        Q[2 * t] = failed ? 0.0 : re;
        Q[2 * t + 1] = failed ? 0.0 : im;
    }
    if (lane == 0 && a.status) a.status[c] = failed ? 1 : 0;
}

// FP32 inverse with iterative refinement, the precision variant of the FP64
// inverse above.  K = H H^H is formed in double-FP32 (exact products by FMA,
// TwoSum accumulation) as Kh + Kl; Cholesky of Kh and the column solves in
// FP32 give X0.  X is then kept as a normalised double-FP32 pair (Xh, Xl)
// and refined: R = I - K X (double-FP32; the Kh Xh products exact, the
// Kh Xl + Kl Xh terms in FP32), X <- X + solve(R).  The work is O(n_u^3) FP32
// per step, where GB300 has ~64x the FP64 rate.  A channel that is not
// accepted when the steps stop (or whose FP32 Cholesky fails) gets status 2,
// and the FP64 kernel recomputes it (only_failed).  Q is Hermitian by construction (upper triangle mirrored).
struct DF { float hi, lo; };  // unevaluated sum hi + lo
__device__ __forceinline__ DF df_add(DF x, float p, float e) {  // (x.hi + x.lo) + (p + e), renormalised
    const float s = __fadd_rn(x.hi, p);
    const float bb = __fsub_rn(s, x.hi);
    const float t = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));  // TwoSum error
    const float u = __fadd_rn(__fadd_rn(t, x.lo), e);
    const float hi = __fadd_rn(s, u);
    return DF{hi, __fsub_rn(u, __fsub_rn(hi, s))};
}
// s + a b with the rounding errors of the product and of the sum added to e
// (one step of a compensated dot product, Ogita, Rump and Oishi's Dot2)
__device__ __forceinline__ void two_sum_prod(float& s, float& e, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float q = __fmaf_rn(a, b, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    e = __fadd_rn(e, __fadd_rn(__fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z)), q));
    s = t;
}
constexpr int kVppRefineMax = 16;

template <int NU>
__global__ void __launch_bounds__(32) vpp_inverse_ir_kernel(VppInvArgs a) {
    // LPC lanes per column of X: lane = col * LPC + part; part 0 runs the
    // triangular solves of its column, all LPC lanes share its residual rows.
    constexpr int LPC = NU > 16 ? 1 : NU > 8 ? 2 : NU > 4 ? 4 : NU > 2 ? 8 : NU > 1 ? 16 : 32;
    extern __shared__ __align__(16) float2 fsm2[];
    const int c = blockIdx.x;
    const int lane = threadIdx.x;
    const int n_t = a.n_t;
    const int cc = lane / LPC, part = lane % LPC;
    const bool active = cc < NU;
    // complex matrices, element (row i, column j) at [i * NU + j]; K's rows are
    // padded to KS = NU + 1 so that the two lanes of a column, reading rows i and
    // i + 1 in the residual, fall in different banks
    constexpr int KS = NU + 1;
    float2* Kh = fsm2;             // K = Kh + Kl, [NU][KS]
    float2* Kl = Kh + NU * KS;
    float2* Lc = Kl + NU * KS;     // FP32 Cholesky factor of Kh; diagonal holds 1 / L_ii
    float2* Hf = Lc + NU * NU;     // H [NU][n_t], until K is formed; then
    float2* Xh = Hf;               // X = Xh + Xl
    float2* Xl = Xh + NU * NU;
    float2* Rm = Xl + NU * NU;     // residual, then correction
    __shared__ int fail;
    const float2* Hg = reinterpret_cast<const float2*>(a.H) + (size_t)c * NU * n_t;
    for (int e = lane; e < NU * n_t; e += 32) Hf[e] = Hg[e];
    if (lane == 0) fail = 0;
    __syncwarp();
    for (int t = lane; t < NU * (NU + 1) / 2; t += 32) {  // upper triangle, row by row
        int i = 0, rem = t;
        while (rem >= NU - i) rem -= NU - i++;
        const int j = i + rem;
        float sr = 0.0f, er = 0.0f, si = 0.0f, ei = 0.0f;  // K_ij = sum_k H_ik conj(H_jk), compensated
        for (int k = 0; k < n_t; ++k) {
            const float2 hi = Hf[i * n_t + k], hj = Hf[j * n_t + k];
            two_sum_prod(sr, er, hi.x, hj.x);
            two_sum_prod(sr, er, hi.y, hj.y);
            if (i != j) {
                two_sum_prod(si, ei, hi.y, hj.x);
                two_sum_prod(si, ei, -hi.x, hj.y);
            }
        }
        const DF re = df_add(DF{sr, 0.0f}, er, 0.0f), im = df_add(DF{si, 0.0f}, ei, 0.0f);
        Kh[i * KS + j] = make_float2(re.hi, im.hi);
        Kl[i * KS + j] = make_float2(re.lo, im.lo);
        Kh[j * KS + i] = make_float2(re.hi, -im.hi);
        Kl[j * KS + i] = make_float2(re.lo, -im.lo);
    }
    __syncwarp();
    for (int j = 0; j < NU; ++j) {
        if (lane == j) {
            float d = Kh[j * KS + j].x;
            for (int k = 0; k < j; ++k) {
                const float2 l = Lc[j * NU + k];
                d = fmarn(-l.x, l.x, d);
                d = fmarn(-l.y, l.y, d);
            }
            const bool ok = (d > 0.0f) && !isinf(d);
            if (!ok) fail = 1;
            Lc[j * NU + j] = make_float2(ok ? __frcp_rn(__fsqrt_rn(d)) : 1.0f, 0.0f);
        }
        __syncwarp();
        const float rjj = Lc[j * NU + j].x;
        if (lane > j && lane < NU) {
            const int i = lane;
            float2 v = Kh[i * KS + j];
            for (int k = 0; k < j; ++k) {  // v -= L_ik conj(L_jk)
                const float2 x = Lc[i * NU + k], y = Lc[j * NU + k];
                v.x = fmarn(-x.x, y.x, v.x);
                v.x = fmarn(-x.y, y.y, v.x);
                v.y = fmarn(-x.y, y.x, v.y);
                v.y = fmarn(x.x, y.y, v.y);
            }
            Lc[i * NU + j] = make_float2(__fmul_rn(v.x, rjj), __fmul_rn(v.y, rjj));
        }
        __syncwarp();
    }
    // column `col` of M := Kh^-1 (column col of M), forward then backward substitution
    auto solve_col = [&](float2* M, int col) {
        for (int i = 0; i < NU; ++i) {
            float2 v = M[i * NU + col];
            for (int k = 0; k < i; ++k) {  // v -= L_ik w_k
                const float2 l = Lc[i * NU + k], w = M[k * NU + col];
                v.x = fmarn(-l.x, w.x, v.x);
                v.x = fmarn(l.y, w.y, v.x);
                v.y = fmarn(-l.x, w.y, v.y);
                v.y = fmarn(-l.y, w.x, v.y);
            }
            const float r = Lc[i * NU + i].x;
            M[i * NU + col] = make_float2(__fmul_rn(v.x, r), __fmul_rn(v.y, r));
        }
        for (int i = NU - 1; i >= 0; --i) {
            float2 v = M[i * NU + col];
            for (int k = NU - 1; k > i; --k) {  // v -= conj(L_ki) x_k
                const float2 l = Lc[k * NU + i], x = M[k * NU + col];
                v.x = fmarn(-l.x, x.x, v.x);
                v.x = fmarn(-l.y, x.y, v.x);
                v.y = fmarn(-l.x, x.y, v.y);
                v.y = fmarn(l.y, x.x, v.y);
            }
            const float r = Lc[i * NU + i].x;
            M[i * NU + col] = make_float2(__fmul_rn(v.x, r), __fmul_rn(v.y, r));
        }
    };
    float xmax = 0.0f;
    if (active) {
        for (int i = part; i < NU; i += LPC) {
            Xh[i * NU + cc] = make_float2(i == cc ? 1.0f : 0.0f, 0.0f);
            Xl[i * NU + cc] = make_float2(0.0f, 0.0f);
        }
    }
    __syncwarp();
    if (active && part == 0) solve_col(Xh, cc);
    __syncwarp();
    if (active)
        for (int i = part; i < NU; i += LPC) {
            const float2 x = Xh[i * NU + cc];
            xmax = fmaxf(xmax, fmaxf(fabsf(x.x), fabsf(x.y)));
        }
    for (int o = 16; o > 0; o >>= 1) xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
    // c_k = max|correction k|.  The error left after step k is about
    // c_k^2 / c_(k-1) (the observed contraction times c_k).  Stop when that
    // is below 2^-40 max|X| (from the first step only if c_1 <= 2^-24 max|X|),
    // or when the corrections stall (at the residual floor, or diverging).
    // Accept when c_k <= 2^-24 max|X|, or when the predicted error is.
    bool done = false, accepted = false;
    float cprev = xmax;
    for (int it = 0; it < a.refine && !done; ++it) {
        if (active) {
            for (int i = part; i < NU; i += LPC) {  // r_i = delta_i,cc - sum_j K_ij X_j,cc
                // compensated sums (TwoProd by FMA, TwoSum): s + e carries the Kh Xh part
                // exactly to about 2^-48; e also takes - (Kh Xl + Kl Xh) in FP32
                float sr = i == cc ? 1.0f : 0.0f, si = 0.0f, er = 0.0f, ei = 0.0f;
                for (int j = 0; j < NU; ++j) {
                    const float2 kh = Kh[i * KS + j], kl = Kl[i * KS + j];
                    const float2 xh = Xh[j * NU + cc], xl = Xl[j * NU + cc];
                    two_sum_prod(sr, er, -kh.x, xh.x);
                    two_sum_prod(sr, er, kh.y, xh.y);
                    two_sum_prod(si, ei, -kh.x, xh.y);
                    two_sum_prod(si, ei, -kh.y, xh.x);
                    er = fmarn(-kh.x, xl.x, fmarn(kh.y, xl.y, fmarn(-kl.x, xh.x, fmarn(kl.y, xh.y, er))));
                    ei = fmarn(-kh.x, xl.y, fmarn(-kh.y, xl.x, fmarn(-kl.x, xh.y, fmarn(-kl.y, xh.x, ei))));
                }
                Rm[i * NU + cc] = make_float2(__fadd_rn(sr, er), __fadd_rn(si, ei));
            }
        }
        __syncwarp();
        if (active && part == 0) solve_col(Rm, cc);
        __syncwarp();
        float cmax = 0.0f;
        if (active)
            for (int i = part; i < NU; i += LPC) {
                const float2 r = Rm[i * NU + cc], xh = Xh[i * NU + cc], xl = Xl[i * NU + cc];
                const DF nr = df_add(DF{xh.x, xl.x}, r.x, 0.0f);
                const DF ni = df_add(DF{xh.y, xl.y}, r.y, 0.0f);
                Xh[i * NU + cc] = make_float2(nr.hi, ni.hi);
                Xl[i * NU + cc] = make_float2(nr.lo, ni.lo);
                cmax = fmaxf(cmax, fmaxf(fabsf(r.x), fabsf(r.y)));
            }
        for (int o = 16; o > 0; o >>= 1) cmax = fmaxf(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
        const bool small = cmax <= xmax * 0x1p-24f;
        const bool stalled = !(cmax <= 0.5f * cprev);
        const float c2 = __fmul_rn(cmax, cmax);
        const bool tiny = (it > 0 || small) && c2 <= __fmul_rn(__fmul_rn(xmax, 0x1p-40f), cprev);
        accepted = small || (it > 0 && !stalled && c2 <= __fmul_rn(__fmul_rn(xmax, 0x1p-24f), cprev));
        done = tiny || stalled;
        cprev = cmax;
        __syncwarp();
    }
    __syncwarp();
    const bool failed = fail != 0 || !accepted || !(xmax <= 3.0e38f);
    double2* Q = reinterpret_cast<double2*>(a.Q) + (size_t)c * NU * NU;
    for (int t = lane; t < NU * NU; t += 32) {
        const int i = t / NU, j = t % NU;
        const int u = i <= j ? i * NU + j : j * NU + i;  // upper-triangle element
        const float2 xh = Xh[u], xl = Xl[u];
        const double re = (double)xh.x + (double)xl.x;
        const double im = i == j ? 0.0 : (i < j ? 1.0 : -1.0) * ((double)xh.y + (double)xl.y);
        Q[t] = failed ? make_double2(0.0, 0.0) : make_double2(re, im);
    }
    if (lane == 0 && a.status) a.status[c] = failed ? 2 : 0;
}

template <int NU>
cudaError_t launch_vpp_inverse_ir_impl(const VppInvArgs& a, cudaStream_t s) {
    if (a.n_chan <= 0) return cudaSuccess;
    if (a.refine < 1 || a.refine > kVppRefineMax) return cudaErrorInvalidValue;
    const size_t smem = (size_t)(2 * NU * (NU + 1) + NU * NU + std::max(NU * a.n_t, 3 * NU * NU)) * sizeof(float2);
    cudaError_t err =
        ensure_dynamic_smem<vpp_inverse_ir_kernel<NU>>(smem);
    if (err != cudaSuccess) return err;
    vpp_inverse_ir_kernel<NU><<<a.n_chan, 32, smem, s>>>(a);
    return cudaGetLastError();
}

// VPP delta-Ising build: G = (tau/2)^2 rr(Q), h = -(tau/2) rr(Q u), guess 0.
template <int NU>
__global__ void __launch_bounds__(128) vpp_build_kernel(VppBuildArgs a) {
    constexpr int n = 2 * NU;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * 4 + warp;
    if (p >= a.n_problems) return;
    const int c = a.chan_index ? a.chan_index[p] : p;
    if (c < 0 || c >= a.n_chan) {
        if (lane == 0) atomicOr(a.err, kErrChanIndex);
        for (int e = lane; e < n * n; e += 32) a.Aq[(size_t)p * n * n + e] = 0;
        for (int e = lane; e < n; e += 32) a.hq[(size_t)p * n + e] = 0;
        return;
    }
    const double* Q = a.Q + (size_t)c * 2 * NU * NU;
    const uint8_t* u = a.u_sym + (size_t)p * NU;
    const int side = 1 << (a.mod_bits >> 1), L = side - 1;
    const double half_tau = (double)side;  // tau / 2 = sqrt(M)
    const double s2 = half_tau * half_tau;
    double hre = 0.0, him = 0.0;
    if (lane < NU) {
        double re = 0.0, im = 0.0;
        for (int j = 0; j < NU; ++j) {
            const int sym = u[j];
            const double ur = (double)(2 * (sym / side) - L), ui = (double)(2 * (sym % side) - L);
            const double qr = Q[2 * (lane * NU + j)], qi = Q[2 * (lane * NU + j) + 1];
            re = __fma_rn(qr, ur, re);
            re = __fma_rn(-qi, ui, re);
            im = __fma_rn(qr, ui, im);
            im = __fma_rn(qi, ur, im);
        }
        hre = __dmul_rn(-half_tau, re);
        him = __dmul_rn(-half_tau, im);
    }
    double mx = 0.0;
    for (int e = lane; e < NU * NU; e += 32)
        mx = fmax(mx, fmax(fabs(__dmul_rn(Q[2 * e], s2)), fabs(__dmul_rn(Q[2 * e + 1], s2))));
    if (lane < NU) mx = fmax(mx, fmax(fabs(hre), fabs(him)));
    mx = warp_max(mx);
    const int se = sigma_exp_d(mx);
    const double s = ldexp(1.0, kQBits - se);
    int16_t* Aq = a.Aq + (size_t)p * n * n;
    for (int e = lane; e < n * n; e += 32) {
        const int i = e / n, j = e % n;
        const int ib = i % NU, jb = j % NU;
        const double re = __dmul_rn(Q[2 * (ib * NU + jb)], s2), im = __dmul_rn(Q[2 * (ib * NU + jb) + 1], s2);
        const double G = (i < NU) == (j < NU) ? re : (i < NU ? -im : im);
        Aq[e] = (int16_t)(int)rint(__dmul_rn(-G, s));
    }
    if (lane < NU) {
        int16_t* hq = a.hq + (size_t)p * n;
        hq[lane] = (int16_t)(int)rint(__dmul_rn(hre, s));
        hq[NU + lane] = (int16_t)(int)rint(__dmul_rn(him, s));
    }
}

// Precoder output: v = d, t = u + tau v, w = Q t, x = H^H w, power = t^H Q t.
template <int NU>
__global__ void __launch_bounds__(128) vpp_output_kernel(VppOutArgs a) {
    constexpr int n = 2 * NU;
    __shared__ double sw[4][2 * NU];
    __shared__ double st[4][2 * NU];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * 4 + warp;
    if (p >= a.n_problems) return;
    int c = a.chan_index ? a.chan_index[p] : p;
    if (c < 0 || c >= a.n_chan) {  // flagged by the build stage; keep the reads in bounds
        if (lane == 0) atomicOr(a.err, kErrChanIndex);
        c = 0;
    }
    const double* Q = a.Q + (size_t)c * 2 * NU * NU;
    const uint8_t* u = a.u_sym + (size_t)p * NU;
    const int8_t* d = a.d + (size_t)p * n;
    const int side = 1 << (a.mod_bits >> 1), L = side - 1, tau = 2 * side;
    if (lane < NU) {
        const int sym = u[lane];
        st[warp][2 * lane] = (double)(2 * (sym / side) - L + tau * (int)d[lane]);
        st[warp][2 * lane + 1] = (double)(2 * (sym % side) - L + tau * (int)d[NU + lane]);
        if (a.v_out) {
            a.v_out[(size_t)p * n + 2 * lane] = d[lane];
            a.v_out[(size_t)p * n + 2 * lane + 1] = d[NU + lane];
        }
    }
    __syncwarp();
    if (lane < NU) {
        double re = 0.0, im = 0.0;
        for (int j = 0; j < NU; ++j) {
            const double qr = Q[2 * (lane * NU + j)], qi = Q[2 * (lane * NU + j) + 1];
            const double tr = st[warp][2 * j], ti = st[warp][2 * j + 1];
            re = __fma_rn(qr, tr, re);
            re = __fma_rn(-qi, ti, re);
            im = __fma_rn(qr, ti, im);
            im = __fma_rn(qi, tr, im);
        }
        sw[warp][2 * lane] = re;
        sw[warp][2 * lane + 1] = im;
    }
    __syncwarp();
    const int n_t = a.n_t;
    if (a.x_out) {
        const float* Hg = a.H + (size_t)c * 2 * NU * n_t;
        for (int kk = lane; kk < n_t; kk += 32) {
            double re = 0.0, im = 0.0;
            for (int i = 0; i < NU; ++i) {
                const double ar = (double)Hg[2 * (i * n_t + kk)], ai = (double)Hg[2 * (i * n_t + kk) + 1];
                const double wr = sw[warp][2 * i], wi = sw[warp][2 * i + 1];
                re = __fma_rn(ar, wr, re);
                re = __fma_rn(ai, wi, re);
                im = __fma_rn(ar, wi, im);
                im = __fma_rn(-ai, wr, im);
            }
            a.x_out[(size_t)p * 2 * n_t + 2 * kk] = (float)re;
            a.x_out[(size_t)p * 2 * n_t + 2 * kk + 1] = (float)im;
        }
    }
    if (lane == 0 && a.power_out) {
        double pw = 0.0;
        for (int i = 0; i < NU; ++i) {
            pw = __fma_rn(st[warp][2 * i], sw[warp][2 * i], pw);
            pw = __fma_rn(st[warp][2 * i + 1], sw[warp][2 * i + 1], pw);
        }
        a.power_out[p] = (float)pw;
    }
}

// ------------------------------------------------------------- launchers
template <int NT>
cudaError_t launch_build_detect_impl(const BuildArgs& a, cudaStream_t s) {
    if (a.n_problems <= 0) return cudaSuccess;
    const size_t smem = (size_t)kBuildWarps * build_smem_floats<NT>(a.n_r) * sizeof(float);
    cudaError_t err = ensure_dynamic_smem<build_detect_kernel<NT>>(smem);
    if (err != cudaSuccess) return err;
    const int blocks = (a.n_problems + kBuildWarps - 1) / kBuildWarps;
    build_detect_kernel<NT><<<blocks, kBuildWarps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

// Tuned kernels exist for n_t in {4, 8, 16} and f_mvm in {1, 2}.
__host__ __device__ constexpr bool tuned_size(int NT) { return NT == 4 || NT == 8 || NT == 16; }

// Shape 8: CTAs of 128 anneals.  The CTAs resident on an SM share its 512
// TMEM columns, so shared memory is padded where needed to keep at most
// 512 / ncols of them on one SM (registers already allow fewer here).
template <int NT, int F>
cudaError_t launch_umma(const SolveArgs& a, int runs, cudaStream_t s) {
    const int pp = 128 / runs;
    const int N = pp * 2 * NT;
    const int ncols = N < 32 ? 32 : N;
    const int max_ctas = 512 / ncols;
    int dev = 0, smem_sm = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (err != cudaSuccess) return err;
    size_t smem = (size_t)UmmaSmem<NT>(pp).bytes();
    const size_t floor_bytes = (size_t)smem_sm / (size_t)(max_ctas + 1) + 1;  // (max_ctas + 1) CTAs no longer fit
    if (smem < floor_bytes) smem = (floor_bytes + 127) & ~(size_t)127;
    err = ensure_dynamic_smem<cac_solve_umma_kernel<NT, F>>(smem);
    if (err != cudaSuccess) return err;
    const int blocks = (a.n_problems + pp - 1) / pp;
    cac_solve_umma_kernel<NT, F><<<blocks, 128, smem, s>>>(a, runs);
    return cudaGetLastError();
}

template <int NT, int F>
cudaError_t launch_tuned(const SolveArgs& a, int runs, int variant, cudaStream_t s) {
    if constexpr (tuned_size(NT)) {
        switch (variant) {
        case kVariantTpa1: cac_solve_tuned_kernel<NT, F, 1, false><<<a.n_problems, runs, 0, s>>>(a); break;
        case kVariantTpa1Packed: cac_solve_tuned_kernel<NT, F, 1, true><<<a.n_problems, runs, 0, s>>>(a); break;
        case kVariantTpa2Packed: cac_solve_tuned_kernel<NT, F, 2, true><<<a.n_problems, 2 * runs, 0, s>>>(a); break;
        case kVariantTpa4Packed:  // (smaller sizes are resolved to shape 4 before launch)
            if constexpr (NT >= 8) cac_solve_tuned_kernel<NT, F, 4, true><<<a.n_problems, 4 * runs, 0, s>>>(a);
            else cac_solve_tuned_kernel<NT, F, 2, true><<<a.n_problems, 2 * runs, 0, s>>>(a);
            break;
        case kVariantTpa8Packed:
            if constexpr (NT >= 16) cac_solve_tuned_kernel<NT, F, 8, true><<<a.n_problems, 8 * runs, 0, s>>>(a);
            else cac_solve_tuned_kernel<NT, F, 2, true><<<a.n_problems, 2 * runs, 0, s>>>(a);
            break;
        case kVariantPairPacked:
            cac_solve_tuned_kernel<NT, F, 1, true, false, true><<<a.n_problems, runs, 0, s>>>(a);
            break;
        case kVariantUmma:
            if constexpr (NT % 8 == 0) {
                if (runs != 96) return launch_umma<NT, F>(a, runs, s);
            }
            [[fallthrough]];  // 96 anneals do not tile the 128 rows: shape 5
        case kVariantTensorCore:
            if constexpr (NT % 8 == 0) {
                cac_solve_tuned_kernel<NT, F, 1, true, true>
                    <<<a.n_problems, runs, (size_t)(runs / 32) * TcShape<NT>::warp_words(32) * 4, s>>>(a);
                break;
            }
            [[fallthrough]];
        case kVariantTensorCore2:
            if constexpr (NT % 8 == 0) {
                cac_solve_tuned_kernel<NT, F, 2, true, true>
                    <<<a.n_problems, 2 * runs, (size_t)(2 * runs / 32) * TcShape<NT>::warp_words(16) * 4, s>>>(a);
                break;
            }
            [[fallthrough]];
        default: cac_solve_kernel<NT, F><<<a.n_problems, runs, 0, s>>>(a); break;
        }
    } else {
        cac_solve_kernel<NT, F><<<a.n_problems, runs, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template <int NT>
cudaError_t launch_solve_impl(const SolveArgs& a, int runs, cudaStream_t s) {
    if (a.n_problems <= 0) return cudaSuccess;
    const int v = a.spins_out ? (int)kVariantPlain : resolve_variant(NT, a.f_mvm, a.variant, a.n_problems, a.n_sm);
    if (a.f_mvm == 2) return launch_tuned<NT, 2>(a, runs, v, s);
    if (a.f_mvm == 1) return launch_tuned<NT, 1>(a, runs, v, s);
    cac_solve_kernel<NT, 0><<<a.n_problems, runs, 0, s>>>(a);
    return cudaGetLastError();
}

template <int NT>
cudaError_t launch_vpp_inverse_impl(const VppInvArgs& a, cudaStream_t s) {
    if (a.n_chan <= 0) return cudaSuccess;
    const size_t smem = (size_t)(2 * NT * a.n_t + 8 * NT * NT) * sizeof(double);
    cudaError_t err = ensure_dynamic_smem<vpp_inverse_kernel<NT>>(smem);
    if (err != cudaSuccess) return err;
    vpp_inverse_kernel<NT><<<a.n_chan, 32, smem, s>>>(a);
    return cudaGetLastError();
}

template <int NT>
cudaError_t launch_vpp_build_impl(const VppBuildArgs& a, cudaStream_t s) {
    if (a.n_problems <= 0) return cudaSuccess;
    vpp_build_kernel<NT><<<(a.n_problems + 3) / 4, 128, 0, s>>>(a);
    return cudaGetLastError();
}

template <int NT>
cudaError_t launch_vpp_output_impl(const VppOutArgs& a, cudaStream_t s) {
    if (a.n_problems <= 0) return cudaSuccess;
    vpp_output_kernel<NT><<<(a.n_problems + 3) / 4, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mmgap

// Explicit instantiation of every launcher for one n_t.
#define MMGAP_INSTANTIATE(NT)                                                                                  \
    namespace mmgap {                                                                                          \
    template <> cudaError_t launch_build_detect<NT>(const BuildArgs& a, cudaStream_t s) {                      \
        return launch_build_detect_impl<NT>(a, s);                                                             \
    }                                                                                                          \
    template <> cudaError_t launch_solve<NT>(const SolveArgs& a, int runs, cudaStream_t s) {                   \
        return launch_solve_impl<NT>(a, runs, s);                                                              \
    }                                                                                                          \
    template <> cudaError_t launch_vpp_inverse<NT>(const VppInvArgs& a, cudaStream_t s) {                      \
        return launch_vpp_inverse_impl<NT>(a, s);                                                              \
    }                                                                                                          \
    template <> cudaError_t launch_vpp_build<NT>(const VppBuildArgs& a, cudaStream_t s) {                      \
        return launch_vpp_build_impl<NT>(a, s);                                                                \
    }                                                                                                          \
    template <> cudaError_t launch_vpp_output<NT>(const VppOutArgs& a, cudaStream_t s) {                       \
        return launch_vpp_output_impl<NT>(a, s);                                                               \
    }                                                                                                          \
    template <> cudaError_t launch_gram_tc<NT>(const GramArgs& a, cudaStream_t s) {                            \
        return launch_gram_tc_impl<NT>(a, s);                                                                  \
    }                                                                                                          \
    template <> cudaError_t launch_select<NT>(const SelectArgs& a, cudaStream_t s) {                           \
        return launch_select_impl<NT>(a, s);                                                                   \
    }                                                                                                          \
    template <> cudaError_t launch_vpp_inverse_ir<NT>(const VppInvArgs& a, cudaStream_t s) {                   \
        return launch_vpp_inverse_ir_impl<NT>(a, s);                                                           \
    }                                                                                                          \
    template <> cudaError_t launch_build_direct<NT>(const DirectBuildArgs& a, cudaStream_t s) {                \
        return launch_build_direct_impl<NT>(a, s);                                                             \
    }                                                                                                          \
    }
