// Batched launch of mixed-size jobs: builder over the job table, the grid solver
// and the tcgen05 tile solver.
#pragma once
#include "build.cuh"
#include "solve.cuh"
#include "umma.cuh"

namespace mmgap {

// =========================================================================
// Batched launch of mixed-size uplink jobs, in two kernels replayed as one
// graph.  The builder runs one warp per problem over the whole batch (all
// jobs, all sizes) into batch scratch; the solver runs one 32-thread CTA per
// problem over a device job table (largest users first), stages the problem's
// Q14 couplings in shared memory and anneals it with 32 anneals on the warp's
// 32 lanes (one thread per anneal, packed FP32).  Results equal the per-job
// path bit for bit: the Philox counters use each problem's index within its
// own job.
// =========================================================================
struct BatchJob {
    BuildArgs b;            // inputs, n_r, mod_bits, n_problems, n_chan, kappa, err
    int nt;
    int kind;               // 0 detection (built by the batch builder); 1 VPP, built before the
                            // batch: no clipping (guess 0), offsets to offset_out, no symbols
    uint32_t key0, key1;
    unsigned long long poff;  // the job's problem_offset (Philox counter of its problem 0)
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
    int32_t* steps_out;     // Euler steps each problem took, or nullptr
};

struct BatchHeader {
    int n_jobs;
    int pad;
    long long total;             // problems in the batch
    long long tiles;             // 4-problem tiles of the tensor-core solver (no tile spans two jobs)
};

struct BatchArgs {
    const BatchJob* jobs;
    // the staged header's counts, as kernel arguments (a graph replay updates them with the grids):
    // read from the constant bank, they add no dependent load ahead of each warp's job lookup
    int n_jobs;
    long long total;
    long long tiles;
    // the grid solver's size classes (16, 8 and 4 users, batch_class): the table holds each class's
    // jobs contiguously, class c's problems being [cls_first[c], cls_first[c] + cls_count[c])
    long long cls_first[3];
    long long cls_count[3];
    long long cls_tile_first[3];  // the tcgen05 solver's 4-problem tiles of each class, likewise
    long long cls_tiles[3];
    int steps;
    int early_exit;         // K > 0: the early-exit rule of the per-job solver (grid solver only)
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

// Builder over the whole batch: warp w of the grid builds problem w, as the
// per-job builder does.  The job's arguments are staged in shared memory and
// read from there: unlike a reference into the job table, they cannot alias the
// builder's global stores, and unlike a register copy they cost no registers
// (the per-job builder reads them from the kernel parameters).
template <int NTMAX>
__global__ void __launch_bounds__(kBuildWarps * 32) batch_build_kernel(BatchArgs A) {
    extern __shared__ __align__(16) float bws[];
    __shared__ __align__(16) BuildArgs sargs[kBuildWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long w = (long long)blockIdx.x * kBuildWarps + warp;
    if (w >= A.total) return;  // warp-uniform; no block-wide barrier below
    const BatchJob& J = A.jobs[batch_find_job(A.jobs, A.n_jobs, w)];
    if (J.kind != 0) return;  // built before the batch
    static_assert(sizeof(BuildArgs) % 4 == 0, "copied as words");
    const int* src = reinterpret_cast<const int*>(&J.b);
    int* dst = reinterpret_cast<int*>(&sargs[warp]);
    for (int i = lane; i < (int)(sizeof(BuildArgs) / 4); i += 32) dst[i] = src[i];
    __syncwarp();
    const BuildArgs& b = sargs[warp];
    const int p = (int)(w - J.first);
    const int nt = J.nt, n = 2 * nt;
    BuildOut o{J.Aq + (size_t)p * n * n, J.hq + (size_t)p * n, J.g + (size_t)p * n, nullptr, nullptr, nullptr};
    // the host rounds the stride to 4 floats; saying so lets the compiler vectorise the
    // builder's shared-memory accesses as in the per-job builder (there the stride is a
    // compile-time multiple of 4): with an unknown alignment every access is split into
    // 4-byte loads
    float* ws = bws + warp * (A.build_floats & ~3);
    if (nt == 16) {
        if constexpr (NTMAX >= 16) build_problem_warp<16>(b, p, lane, ws, o);
    } else if (nt == 8) {
        if constexpr (NTMAX >= 8) build_problem_warp<8>(b, p, lane, ws, o);
    } else {
        build_problem_warp<4>(b, p, lane, ws, o);
    }
}

// Anneal one problem already built into sm (Aq, hq, g) with one warp.
template <int NT, int F, bool EE = false>
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
        const unsigned long long pg = J.poff + (unsigned long long)p;
        const uint32_t c2 = (uint32_t)pg, c3 = (uint32_t)(pg >> 32);
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
    // 16 users: the paired refresh (faster there, same bits); fewer users: one anneal per lane
    constexpr bool kPair = NT == 16;
    if constexpr (EE) {
        // early exit, the per-job solver's rule: the problem is this warp, so one warp vote decides
        const int K = A.early_exit;
        uint32_t p1 = sign_word<n>(x1), p2 = sign_word<n>(x2);
        bool pa = xa >= 0.0f;
        int c = K;
#pragma unroll 1
        for (; t < S; t += F) {
            if (t > 0 && --c == 0) {
                c = K;
                const uint32_t w1 = sign_word<n>(x1), w2 = sign_word<n>(x2);
                const bool wa = xa >= 0.0f;
                const bool changed = (w1 != p1) || (w2 != p2) || (wa != pa);
                p1 = w1;
                p2 = w2;
                pa = wa;
                if (!__any_sync(0xffffffffu, changed)) break;
            }
            if (t + F <= S)
                tuned_block<n, n, 1, true, F, kPair>(sm.A, sm.h, sm.nd, x1, x2, e1, e2, xa, ea, 0, lane, F, k);
            else
                tuned_block<n, n, 1, true, 0, kPair>(sm.A, sm.h, sm.nd, x1, x2, e1, e2, xa, ea, 0, lane, S - t, k);
        }
    } else {
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
        if constexpr (EE) {  // (without early exit the runner fills steps_out with S)
            if (J.steps_out) J.steps_out[p] = t < S ? t : S;
        }
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

template <int NT, int F, bool EE = false>
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
    batch_solve_warp<NT, F, EE>(A, J, p, lane, sm);
}

// Per-channel MMSE factorisations of the staged detection jobs (chan_factor_warp)
// in three launches for all jobs: the jobs' channels are numbered one after
// another from chan_first, their problems from prob_first.
struct FactorJob {
    ChanFactorArgs a;
    int nt;
    long long chan_first;
    long long prob_first;
};

struct FactorBatch {
    const FactorJob* jobs;
    int n_jobs;
    long long n_chan;      // channels of all jobs
    long long n_problems;  // problems of all jobs
    int build_floats;      // shared memory per warp of the factor kernel (floats, a multiple of 4)
};

// Last job whose channels (CHAN) or problems start at or before v.
template <bool CHAN>
__device__ __forceinline__ int factor_find_job(const FactorJob* jobs, int n_jobs, long long v) {
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((CHAN ? jobs[mid].chan_first : jobs[mid].prob_first) <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Every channel's first-problem slot to a value above any problem index.
static __global__ void batch_factor_init_kernel(FactorBatch F) {
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < F.n_chan;
         g += (long long)gridDim.x * blockDim.x) {
        const FactorJob& J = F.jobs[factor_find_job<true>(F.jobs, F.n_jobs, g)];
        J.a.first[g - J.chan_first] = 0x7fffffff;
    }
}

// First problem of each channel of every job (atomic minimum over the job's problems).
static __global__ void batch_factor_first_kernel(FactorBatch F) {
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < F.n_problems;
         g += (long long)gridDim.x * blockDim.x) {
        const FactorJob& J = F.jobs[factor_find_job<false>(F.jobs, F.n_jobs, g)];
        const int p = (int)(g - J.prob_first);
        const int c = J.a.chan_index[p];
        if (c >= 0 && c < J.a.n_chan) atomicMin(J.a.first + c, p);
    }
}

// One warp per channel of every job.
template <int NTMAX>
__global__ void __launch_bounds__(kBuildWarps * 32) batch_factor_kernel(FactorBatch F) {
    extern __shared__ __align__(16) float fws[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long g = (long long)blockIdx.x * kBuildWarps + warp;
    if (g >= F.n_chan) return;  // warp-uniform
    const FactorJob& J = F.jobs[factor_find_job<true>(F.jobs, F.n_jobs, g)];
    const int c = (int)(g - J.chan_first);
    float* ws = fws + warp * (F.build_floats & ~3);  // (a multiple of 4: vectorised accesses)
    if (J.nt == 16) {
        if constexpr (NTMAX >= 16) chan_factor_warp<16>(J.a, c, lane, ws);
    } else if (J.nt == 8) {
        if constexpr (NTMAX >= 8) chan_factor_warp<8>(J.a, c, lane, ws);
    } else {
        chan_factor_warp<4>(J.a, c, lane, ws);
    }
}

// Size class of a table job's user count: 0 for 16 users, 1 for 8, 2 for 4.
__host__ __device__ constexpr int batch_class(int nt) { return nt == 16 ? 0 : (nt == 8 ? 1 : 2); }

// Grid solver of one size class: one 32-thread CTA per problem of the class's
// jobs.  Each class is its own kernel, with its own size's registers and
// shared memory (one kernel over all sizes ran every problem at the 16-user
// footprint); the classes' kernels are independent and may run concurrently.
// CTAs past the class's count exit.
template <int NT, int F, bool EE = false>
__global__ void __launch_bounds__(32) batch_solve_grid_kernel(BatchArgs A) {
    __shared__ __align__(16) unsigned char ssm[batch_solve_bytes<NT>()];
    constexpr int c = batch_class(NT);
    if ((long long)blockIdx.x >= A.cls_count[c]) return;
    const long long w = A.cls_first[c] + blockIdx.x;
    const BatchJob& J = A.jobs[batch_find_job(A.jobs, A.n_jobs, w)];
    batch_solve_problem<NT, F, EE>(A, J, (int)(w - J.first), threadIdx.x, ssm);
}

// Batched tensor-core solver (tcgen05, solver shape 8) of one size class: one
// 128-thread CTA per tile of 4 consecutive problems of one job of the class
// (the table holds each class's tiles contiguously: [cls_tile_first[c],
// cls_tile_first[c] + cls_tiles[c])).  8- and 16-user tiles run umma_tile (the
// same tiles as mmgap_detect with shape 8, so the same bits), 4-user tiles one
// exact warp per problem.  Each class is its own kernel, with its own size's
// registers and shared memory, and the classes may run concurrently.
template <int NT>
__host__ __device__ constexpr size_t batch_umma_bytes() {
    return NT >= 8 ? (size_t)UmmaSmem<NT >= 16 ? 16 : 8>(4).bytes() : 4 * batch_solve_bytes<4>();
}

template <int NT, int F>
__global__ void __launch_bounds__(128) batch_solve_umma_kernel(BatchArgs A) {
    extern __shared__ __align__(128) uint8_t usm[];
    constexpr int c = batch_class(NT);
    if ((long long)blockIdx.x >= A.cls_tiles[c]) return;
    const long long t = A.cls_tile_first[c] + blockIdx.x;
    int lo = 0, hi = A.n_jobs - 1;  // last job whose tiles start at or before t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (A.jobs[mid].tile_first <= t) lo = mid;
        else hi = mid - 1;
    }
    const BatchJob& J = A.jobs[lo];
    const int base = (int)(t - J.tile_first) * 4;
    const int live = min(4, J.b.n_problems - base);
    if constexpr (NT >= 8) {
        constexpr int n = 2 * NT;
        UmmaTile u;
        u.Aq = J.Aq + (size_t)base * n * n;
        u.hq = J.hq + (size_t)base * n;
        u.g = J.g ? J.g + (size_t)base * n : nullptr;
        u.n_live = live;
        u.problem0 = J.poff + (uint64_t)base;
        u.key0 = J.key0;
        u.key1 = J.key1;
        u.level_max = J.kind == 0 ? (1 << (J.b.mod_bits >> 1)) - 1 : 0;
        u.steps = A.steps;
        u.k = A.k;
        u.wait_ns = kDefaultDeviceWaitNs;
        u.err = J.b.err;
        u.d_out = J.offset_out ? J.offset_out + (size_t)base * n : nullptr;
        u.E_out = J.energy_out ? J.energy_out + base : nullptr;
        u.run_out = nullptr;
        u.ndiv_out = J.ndiv_out ? J.ndiv_out + base : nullptr;
        u.x_out = nullptr;
        u.guess_out = J.guess_out ? J.guess_out + (size_t)base * n : nullptr;
        u.sym_out = J.sym_out ? J.sym_out + (size_t)base * NT : nullptr;
        u.mod_bits = J.b.mod_bits;
        umma_tile<NT, F>(u, 32, usm);
    } else {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (warp < live) batch_solve_problem<4, F>(A, J, base + warp, lane, usm + warp * batch_solve_bytes<4>());
    }
}

}  // namespace mmgap
