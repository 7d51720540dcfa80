// Direct (binary-weighted) spin mapping: builder and the general-coupling solver.
#pragma once
#include "build.cuh"
#include "solve.cuh"

namespace mmgap {

// =========================================================================
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

}  // namespace mmgap
