// CIM-CAC solver (Eqs. 10-11, Sec. 3.2.1): the one-thread-per-anneal kernel, the
// bit-identical tuned launch shapes and the mma.sync tensor-core refresh (shapes 5, 7).
#pragma once
#include <cooperative_groups.h>

#include "common.cuh"

namespace mmgap {

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

// Early exit (SolveArgs::early_exit = K > 0; a budget lever, not in the
// paper, which anneals a fixed N_I steps): a problem's anneals advance
// together, and at every K-th field refresh, t = j K f_mvm with 0 < t < S,
// the signs [x >= 0] of all spins of all its anneals are compared with those
// at the previous check point.  If none changed, every anneal of the problem
// stops at t; its state there is final.  One CTA holds one problem, so the
// decision is one CTA-wide vote (__syncthreads_or), uniform across the CTA.
template <int M>
__device__ __forceinline__ uint32_t sign_word(const float* x) {
    static_assert(M <= 32, "one word per 32 spins");
    uint32_t w = 0;
#pragma unroll
    for (int i = 0; i < M; ++i) w |= (x[i] >= 0.0f ? 1u : 0u) << i;
    return w;
}

// Sign words of x[0..M) compared with prev (updated); true if any sign changed.
template <int M>
__device__ __forceinline__ bool signs_changed(const float (&x)[M], uint32_t (&prev)[(M + 31) / 32]) {
    bool changed = false;
#pragma unroll
    for (int b = 0; b < (M + 31) / 32; ++b) {
        constexpr int W = 32;
        uint32_t w = 0;
#pragma unroll
        for (int i = 0; i < W; ++i)
            if (W * b + i < M) w |= (x[W * b + i] >= 0.0f ? 1u : 0u) << i;
        changed = changed || w != prev[b];
        prev[b] = w;
    }
    return changed;
}

// steps_out of a launch without early exit: every problem took all S steps.
static __global__ void fill_steps_kernel(int32_t* out, int n, int S) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = S;
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
    if (a.early_exit > 0) {
        // refresh intervals one at a time, with the early-exit check before each K-th refresh
        const int K = a.early_exit;
        const int f = F > 0 ? F : a.f_mvm;
        uint32_t prev[(N + 31) / 32] = {};
        signs_changed<N>(x, prev);  // (records the initial signs)
        int c = K;
#pragma unroll 1
        for (; t < S; t += f) {
            if (t > 0 && --c == 0) {
                c = K;
                const bool changed = signs_changed<N>(x, prev);
                if (!__syncthreads_or(changed)) break;
            }
            coupling_mvm<n>(sm.A, sm.h, x, m, mua);
            frozen_steps_rt<n>(sm.h, sm.nd, x, e, m, mua, S - t < f ? S - t : f, k);
        }
        if (a.steps_out && run == 0) a.steps_out[p] = t < S ? t : S;
        t = S;  // (the tail below is part of the loop here)
    } else if constexpr (F > 0) {
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

    if (a.early_exit <= 0 && a.steps_out && run == 0) a.steps_out[p] = S;

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

// CL > 1 (latency: few problems): a cluster of CL CTAs per problem, each with
// R / CL of its anneals on its own SM.  The anneals keep their indices in the
// problem (Philox streams and arg-min key), so the results are the same bits;
// the arg-min and the divergence count are combined through distributed
// shared memory.
template <int NT, int F, int TPA, bool PACKED, bool TC = false, bool PAIR = false, bool EE = false, int CL = 1>
__global__ void __launch_bounds__(128 * TPA) cac_solve_tuned_kernel(SolveArgs a) {
    constexpr int n = 2 * NT;
    constexpr int NS = n / TPA;
    static_assert(n % TPA == 0 && NS % 4 == 0, "rows per thread must be a multiple of 4");
    static_assert(F > 0, "compile-time refresh period");
    static_assert(!TC || (TPA <= 2 && PACKED && n % 16 == 0), "tensor-core refresh: 1 or 2 threads per anneal");
    static_assert(!(TC && EE), "early exit runs on the bit-identical shapes");
    static_assert(CL == 1 || (!TC && !EE), "clusters: the exact shapes without early exit");
    __shared__ __align__(16) SolveSmem<NT> sm;
    __shared__ long long skey[4 * TPA];
    __shared__ int sdiv[4 * TPA];
    __shared__ __align__(16) uint32_t tc_af[TC ? TcShape<NT>::AF_WORDS : 1];
    extern __shared__ __align__(16) uint32_t tc_ws[];  // TC: TcShape<NT>::warp_words(32 / TPA) per warp (dynamic)
    const int p = blockIdx.x / CL;
    const int tid = threadIdx.x, T = blockDim.x;
    const int crank = CL > 1 ? (int)cooperative_groups::this_cluster().block_rank() : 0;
    const int q = tid % TPA, run = crank * (T / TPA) + tid / TPA;  // the anneal's index in the problem
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
    if constexpr (EE) {
        // refresh intervals one at a time, with the early-exit check before each K-th refresh
        // (this thread's spins: its rows of x1 and x2 and its copy of the auxiliary spin)
        const int K = a.early_exit;
        uint32_t p1 = sign_word<NS>(x1), p2 = sign_word<NS>(x2);
        bool pa = xa >= 0.0f;
        int c = K;
#pragma unroll 1
        for (; t < S; t += F) {
            if (t > 0 && --c == 0) {
                c = K;
                const uint32_t w1 = sign_word<NS>(x1), w2 = sign_word<NS>(x2);
                const bool wa = xa >= 0.0f;
                const bool changed = (w1 != p1) || (w2 != p2) || (wa != pa);
                p1 = w1;
                p2 = w2;
                pa = wa;
                if (!__syncthreads_or(changed)) break;
            }
            if (t + F <= S)
                tuned_block<n, NS, TPA, PACKED, F, PAIR>(sm.A, sm.h, sm.nd, x1, x2, e1, e2, xa, ea, q, lane, F, k);
            else
                tuned_block<n, NS, TPA, PACKED, 0, PAIR>(sm.A, sm.h, sm.nd, x1, x2, e1, e2, xa, ea, q, lane, S - t,
                                                          k);
        }
    } else if constexpr (TC) {
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
    if constexpr (CL > 1) {
        __shared__ long long ckey;
        __shared__ int cdiv;
        cooperative_groups::cluster_group cluster = cooperative_groups::this_cluster();
        if (tid == 0) {
            ckey = best;
            cdiv = ndiv;
        }
        cluster.sync();
        best = 0x7fffffffffffffffLL;
        ndiv = 0;
#pragma unroll
        for (int r = 0; r < CL; ++r) {
            const long long kr = *cluster.map_shared_rank(&ckey, (unsigned)r);
            best = kr < best ? kr : best;
            ndiv += *cluster.map_shared_rank(&cdiv, (unsigned)r);
        }
        cluster.sync();  // no CTA leaves while another still reads its shared memory
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
            if constexpr (EE) {  // (without early exit the launcher fills steps_out with S)
                if (a.steps_out) a.steps_out[p] = t < S ? t : S;
            }
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

}  // namespace mmgap
