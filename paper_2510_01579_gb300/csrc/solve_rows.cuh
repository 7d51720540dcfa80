// CIM-CAC solver for 32 users (n = 64, Eqs. 10-11, Fig. 5): row blocks of
// two anneals per thread.  Bit-identical to the one-thread-per-anneal kernel.
#pragma once
#include <cooperative_groups.h>

#include "solve.cuh"

namespace mmgap {

// =========================================================================
// Layout.  A CTA anneals one problem with R anneals (R a multiple of 32) on
// 4 R threads: each group of 32 anneals has four warps, and half-warp h of
// warp w owns the 8-row block rb = 2 w + h (rows [8 rb, 8 rb + 8)) of
// anneals a and a + 16 (a = lane % 16 within the group).  Per field-refresh
// column j a half-warp therefore issues one broadcast coupling address and
// every coupling value feeds four FMA lanes (two rows x two anneals), which
// halves the shared-memory wavefronts per FMA of a one-anneal-per-thread
// row split.  The anneals' u vectors go through double-buffered padded
// shared-memory rows published by a named barrier of the group's warps.
// Every m_i stays the ascending-j FMA chain from 0, so the results equal the
// one-thread-per-anneal kernel's (and the oracle's) bit for bit.
// =========================================================================
constexpr int kRowsNs = 8;  // rows per thread

// Frozen-field Euler steps of one anneal's 8 rows (packed pairs) and of its
// auxiliary spin: c = m + b x_a, mu1 = c - diag(A) x1, mu2 = c - diag(A) x2.
template <int L>
__device__ __forceinline__ void rows_frozen_steps(const float* sh, const float* snd, int row0,
                                                  const float (&m)[kRowsNs], float (&x1)[kRowsNs],
                                                  float (&x2)[kRowsNs], float (&e1)[kRowsNs], float (&e2)[kRowsNs],
                                                  float& xa, float& ea, float mua, int Lrt, const EulerConsts& k) {
    const float2 xa2 = make_float2(xa, xa);
    const float2 cdt = make_float2(k.cdt, k.cdt), c1 = make_float2(k.c1, k.c1);
    const float2 cz = make_float2(k.cz, k.cz), c2 = make_float2(k.c2, k.c2);
#pragma unroll
    for (int i = 0; i < kRowsNs; i += 2) {
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

// One field refresh + L frozen steps for the thread's two anneals.
// ua, ub: this buffer's u rows of the two anneals; bar: the group's barrier.
template <int n, int L>
__device__ __forceinline__ void rows_block(const float* sA, const float* sh, const float* snd, int row0,
                                           float (&x1)[2][kRowsNs], float (&x2)[2][kRowsNs],
                                           float (&e1)[2][kRowsNs], float (&e2)[2][kRowsNs], float (&xa)[2],
                                           float (&ea)[2], float* ua, float* ub, int bar, int Lrt,
                                           const EulerConsts& k) {
    asm volatile("" ::: "memory");  // keep the coupling loads inside the time loop
    // publish u = x1 + x2 of this thread's rows for both anneals
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        float uo[kRowsNs];
#pragma unroll
        for (int i = 0; i < kRowsNs; i += 2) {
            const float2 s2 = __fadd2_rn(make_float2(x1[t][i], x1[t][i + 1]), make_float2(x2[t][i], x2[t][i + 1]));
            uo[i] = s2.x;
            uo[i + 1] = s2.y;
        }
        float* dst = (t == 0 ? ua : ub) + row0;
        *reinterpret_cast<float4*>(dst) = make_float4(uo[0], uo[1], uo[2], uo[3]);
        *reinterpret_cast<float4*>(dst + 4) = make_float4(uo[4], uo[5], uo[6], uo[7]);
    }
    asm volatile("bar.sync %0, 128;" ::"r"(bar) : "memory");
    // m = A u for both anneals (ascending j), mu_a = b^T u
    float m0[kRowsNs], m1[kRowsNs];
#pragma unroll
    for (int i = 0; i < kRowsNs; ++i) m0[i] = m1[i] = 0.0f;
    float2 mua = make_float2(0.0f, 0.0f);
    float4 u4a = make_float4(0.0f, 0.0f, 0.0f, 0.0f), u4b = u4a, h4 = u4a;
#pragma unroll
    for (int j = 0; j < n; ++j) {
        const int jj = j & 3;
        if (jj == 0) {
            u4a = *reinterpret_cast<const float4*>(ua + j);
            u4b = *reinterpret_cast<const float4*>(ub + j);
            h4 = *reinterpret_cast<const float4*>(sh + j);
        }
        const float va = jj == 0 ? u4a.x : jj == 1 ? u4a.y : jj == 2 ? u4a.z : u4a.w;
        const float vb = jj == 0 ? u4b.x : jj == 1 ? u4b.y : jj == 2 ? u4b.z : u4b.w;
        const float hj = jj == 0 ? h4.x : jj == 1 ? h4.y : jj == 2 ? h4.z : h4.w;
        mua = __ffma2_rn(make_float2(hj, hj), make_float2(va, vb), mua);
        const float4* row = reinterpret_cast<const float4*>(sA + j * n + row0);
        const float2 uu = make_float2(va, va), vv = make_float2(vb, vb);
#pragma unroll
        for (int i4 = 0; i4 < kRowsNs / 4; ++i4) {
            const float4 a4 = row[i4];
            const float2 al = make_float2(a4.x, a4.y), ah = make_float2(a4.z, a4.w);
            float2 r = __ffma2_rn(al, uu, make_float2(m0[4 * i4], m0[4 * i4 + 1]));
            m0[4 * i4] = r.x;
            m0[4 * i4 + 1] = r.y;
            r = __ffma2_rn(ah, uu, make_float2(m0[4 * i4 + 2], m0[4 * i4 + 3]));
            m0[4 * i4 + 2] = r.x;
            m0[4 * i4 + 3] = r.y;
            r = __ffma2_rn(al, vv, make_float2(m1[4 * i4], m1[4 * i4 + 1]));
            m1[4 * i4] = r.x;
            m1[4 * i4 + 1] = r.y;
            r = __ffma2_rn(ah, vv, make_float2(m1[4 * i4 + 2], m1[4 * i4 + 3]));
            m1[4 * i4 + 2] = r.x;
            m1[4 * i4 + 3] = r.y;
        }
    }
    rows_frozen_steps<L>(sh, snd, row0, m0, x1[0], x2[0], e1[0], e2[0], xa[0], ea[0], mua.x, Lrt, k);
    rows_frozen_steps<L>(sh, snd, row0, m1, x1[1], x2[1], e1[1], e2[1], xa[1], ea[1], mua.y, Lrt, k);
}

// Dynamic shared memory of the row-block kernel: two u buffers of R rows of
// n + 4 floats (the exchange of validity, codes and energies reuses them).
__host__ __device__ constexpr size_t rows_dyn_bytes(int n, int runs) {
    return 2 * (size_t)runs * (size_t)(n + 4) * sizeof(float);
}

// CL > 1 (latency: few problems): a cluster of CL CTAs per problem, each
// with R / CL of its anneals on its own SM; the arg-min and the divergence
// count are combined through distributed shared memory.
template <int NT, int F, int CL = 1>
__global__ void __launch_bounds__(512) cac_solve_rows_kernel(SolveArgs a) {
    constexpr int n = 2 * NT;
    constexpr int NRB = n / kRowsNs;  // row blocks per anneal
    static_assert(n == 64, "two 8-row blocks per warp and four warps per 32 anneals: n = 64");
    static_assert(F >= 0, "refresh period: compile-time F > 0, or F = 0 for a.f_mvm at run time");
    __shared__ __align__(16) SolveSmem<NT> sm;
    __shared__ long long skey[16];
    __shared__ int sdiv[16];
    extern __shared__ __align__(16) uint32_t rows_ws[];
    const int p = blockIdx.x / CL;
    const int crank = CL > 1 ? (int)cooperative_groups::this_cluster().block_rank() : 0;
    const int tid = threadIdx.x, T = blockDim.x;
    const int R = T / 4;  // anneals of this CTA
    const int lane = tid & 31, warp = tid >> 5;
    const int grp = warp >> 2;                        // group of 32 anneals
    const int rb = 2 * (warp & 3) + (lane >> 4);     // row block
    const int row0 = rb * kRowsNs;
    const int run[2] = {grp * 32 + (lane & 15), grp * 32 + (lane & 15) + 16};  // this CTA's anneals
    const int grun[2] = {crank * R + run[0], crank * R + run[1]};              // the problem's anneal index
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
    __syncthreads();

    // Philox initial amplitudes (counter word of spin k = row, n + row, 2n; run; problem)
    float x1[2][kRowsNs], x2[2][kRowsNs], e1[2][kRowsNs], e2[2][kRowsNs], xa[2], ea[2] = {1.0f, 1.0f};
    {
        const uint64_t pg = a.problem_offset + (uint64_t)p;
        const uint32_t c2 = (uint32_t)pg, c3 = (uint32_t)(pg >> 32);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
#pragma unroll
            for (int b = 0; b < kRowsNs / 4; ++b) {
                const U4 w1 = philox4x32_10(U4{(uint32_t)((row0 >> 2) + b), (uint32_t)grun[t], c2, c3}, a.key0, a.key1);
                const U4 w2 =
                    philox4x32_10(U4{(uint32_t)(((n + row0) >> 2) + b), (uint32_t)grun[t], c2, c3}, a.key0, a.key1);
                const uint32_t v1[4] = {w1.x, w1.y, w1.z, w1.w}, v2[4] = {w2.x, w2.y, w2.z, w2.w};
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    x1[t][4 * b + s] = mulrn((float)((int)(v1[s] >> 8) - 8388608), k.xs);
                    x2[t][4 * b + s] = mulrn((float)((int)(v2[s] >> 8) - 8388608), k.xs);
                    e1[t][4 * b + s] = 1.0f;
                    e2[t][4 * b + s] = 1.0f;
                }
            }
            const U4 wa = philox4x32_10(U4{(uint32_t)((2 * n) >> 2), (uint32_t)grun[t], c2, c3}, a.key0, a.key1);
            xa[t] = mulrn((float)((int)(wa.x >> 8) - 8388608), k.xs);
        }
    }

    float* ubase = reinterpret_cast<float*>(rows_ws);
    const int ubuf = R * (n + 4);  // floats per buffer
    const int bar = 1 + grp;
    const int S = a.steps;
    const int f = F > 0 ? F : a.f_mvm;
    int t = 0, b = 0;
#pragma unroll 1
    for (; t + f <= S; t += f, b ^= 1)
        rows_block<n, F>(sm.A, sm.h, sm.nd, row0, x1, x2, e1, e2, xa, ea, ubase + b * ubuf + run[0] * (n + 4),
                         ubase + b * ubuf + run[1] * (n + 4), bar, f, k);
    if (t < S)
        rows_block<n, 0>(sm.A, sm.h, sm.nd, row0, x1, x2, e1, e2, xa, ea, ubase + b * ubuf + run[0] * (n + 4),
                         ubase + b * ubuf + run[1] * (n + 4), bar, S - t, k);
    __syncthreads();  // every read of the u rows is done: the buffers now hold the exchange

    // exchange: validity and 2-bit offset codes of each row block, then energies
    uint32_t* xv = rows_ws;            // [NRB][R]
    uint32_t* xc = rows_ws + NRB * R;  // [NRB][R], 8 two-bit codes
    int* xe = reinterpret_cast<int*>(rows_ws + 2 * NRB * R);
    int dmine[2][kRowsNs];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        bool valid = (fabsf(xa[s]) <= k.x_max) && (ea[s] > 0.0f);
#pragma unroll
        for (int i = 0; i < kRowsNs; ++i)
            valid = valid && (fabsf(x1[s][i]) <= k.x_max) && (e1[s][i] > 0.0f) && (fabsf(x2[s][i]) <= k.x_max) &&
                    (e2[s][i] > 0.0f);
        const int sa = xa[s] >= 0.0f ? 1 : -1;
        uint32_t code = 0;
#pragma unroll
        for (int i = 0; i < kRowsNs; ++i) {
            const int s1 = x1[s][i] >= 0.0f ? 1 : -1, s2 = x2[s][i] >= 0.0f ? 1 : -1;
            int di = sa * (s1 + s2) / 2;
            if (a.level_max > 0) {
                const int xv_ = (int)sm.g[row0 + i] + 2 * di;
                if (xv_ > a.level_max || xv_ < -a.level_max) di = 0;
            }
            dmine[s][i] = di;
            code |= (uint32_t)(di & 3) << (2 * i);
        }
        xv[rb * R + run[s]] = valid ? 1u : 0u;
        xc[rb * R + run[s]] = code;
    }
    __syncthreads();
    bool valid[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        valid[s] = true;
#pragma unroll
        for (int r = 0; r < NRB; ++r) valid[s] = valid[s] && xv[r * R + run[s]] != 0u;
        // exact quantised energy of this thread's rows: r_i = sum_j Aq_ij d_j, one column block at a time
        int acc[kRowsNs];
#pragma unroll
        for (int i = 0; i < kRowsNs; ++i) acc[i] = 0;
#pragma unroll 1
        for (int r = 0; r < NRB; ++r) {
            const uint32_t code = xc[r * R + run[s]];
#pragma unroll
            for (int c = 0; c < kRowsNs; ++c) {
                const int v = (int)((code >> (2 * c)) & 3u);
                const int dj = v == 3 ? -1 : v;
#pragma unroll
                for (int i = 0; i < kRowsNs; ++i) acc[i] += (int)sm.Aq[(row0 + i) * n + r * kRowsNs + c] * dj;
            }
        }
        int E = 0;
#pragma unroll
        for (int i = 0; i < kRowsNs; ++i) {
            E -= dmine[s][i] * acc[i];
            E -= (int)sm.hq[row0 + i] * dmine[s][i];
        }
        xe[rb * R + run[s]] = E;
    }
    __syncthreads();
    long long key = 0x7fffffffffffffffLL;
    bool keep[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        int E = 0;
#pragma unroll
        for (int r = 0; r < NRB; ++r) E += xe[r * R + run[s]];
        keep[s] = valid[s] && E <= 0;
        const long long ks = (long long)(keep[s] ? E : 0) * 4294967296LL + (long long)grun[s];
        key = ks < key ? ks : key;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long other = __shfl_xor_sync(0xffffffffu, key, o);
        key = other < key ? other : key;
    }
    // each anneal is counted once: by row block 0 (lanes 0-15 of the group's first warp)
    const unsigned d0 = __ballot_sync(0xffffffffu, !valid[0] && rb == 0);
    const unsigned d1 = __ballot_sync(0xffffffffu, !valid[1] && rb == 0);
    if (lane == 0) {
        skey[warp] = key;
        sdiv[warp] = __popc(d0) + __popc(d1);
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
    const int best_local = best_run - crank * R;  // (in the CTA that holds the winner)
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        if (grun[s] != best_run) continue;
        if (a.d_out) {
#pragma unroll
            for (int i = 0; i < kRowsNs; ++i)
                a.d_out[(size_t)p * n + row0 + i] = keep[s] ? (int8_t)dmine[s][i] : (int8_t)0;
        }
        if (rb == 0) {
            const int bestE = (int)((best - (long long)best_run) / 4294967296LL);
            if (a.E_out) a.E_out[p] = bestE;
            if (a.run_out) a.run_out[p] = best_run;
            if (a.ndiv_out) a.ndiv_out[p] = ndiv;
            auto dj = [&](int j) {  // the winning anneal's offset of row j (0 unless kept)
                const int v = (int)((xc[(j / kRowsNs) * R + best_local] >> (2 * (j % kRowsNs))) & 3u);
                return keep[s] ? (v == 3 ? -1 : v) : 0;
            };
            if (a.x_out) {
                for (int i = 0; i < n; ++i) a.x_out[(size_t)p * n + i] = (int8_t)((int)sm.g[i] + 2 * dj(i));
            }
            if (a.sym_out) {
                const int side = 1 << (a.mod_bits >> 1), L = side - 1;
                uint8_t* so = a.sym_out + (size_t)p * NT;
                for (int i = 0; i < NT; ++i) {
                    const int xr = (int)sm.g[i] + 2 * dj(i);
                    const int xi = (int)sm.g[NT + i] + 2 * dj(NT + i);
                    so[i] = (uint8_t)(((xr + L) / 2) * side + (xi + L) / 2);
                }
            }
        }
    }
}

}  // namespace mmgap
