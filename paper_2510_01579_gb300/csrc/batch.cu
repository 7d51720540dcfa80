// Batched launch of mixed-size uplink jobs (mmgap_batch_*).
//
// A batch is a fixed set of detection jobs (device inputs and outputs).  One
// run = job-table upload, one builder kernel over every problem of every job
// and one solver kernel with a CTA per problem across all jobs, largest
// problems first, so jobs of different sizes share the GPU instead of one pair
// of grids per job.  The run can be captured once into a CUDA graph and
// replayed.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mmgap.h"
#include "batch.h"
#include "kernels.cuh"

using namespace mmgap;

namespace mmgap {

namespace {

bool batch_nt(int nt) { return nt == 4 || nt == 8 || nt == 16; }

int build_floats_for(int nt, int n_r) {
    switch (nt) {
    case 16: return build_smem_floats<16>(n_r);
    case 8: return build_smem_floats<8>(n_r);
    default: return build_smem_floats<4>(n_r);
    }
}

// tcgen05 tiles of 4 problems (solver shape 8) of size class c (batch_class)
const void* umma_solve(int c, int f) {
    switch (c) {
    case 0: return f == 1 ? (const void*)batch_solve_umma_kernel<16, 1> : (const void*)batch_solve_umma_kernel<16, 2>;
    case 1: return f == 1 ? (const void*)batch_solve_umma_kernel<8, 1> : (const void*)batch_solve_umma_kernel<8, 2>;
    default: return f == 1 ? (const void*)batch_solve_umma_kernel<4, 1> : (const void*)batch_solve_umma_kernel<4, 2>;
    }
}

template <int NT>
const void* class_solve_nt(int f, bool ee) {
    if (ee)  // the early-exit rule of the per-job solver
        return f == 1 ? (const void*)batch_solve_grid_kernel<NT, 1, true> : (const void*)batch_solve_grid_kernel<NT, 2, true>;
    return f == 1 ? (const void*)batch_solve_grid_kernel<NT, 1> : (const void*)batch_solve_grid_kernel<NT, 2>;
}

// the grid solver of size class c (batch_class)
const void* class_solve(int c, int f, bool ee) {
    switch (c) {
    case 0: return class_solve_nt<16>(f, ee);
    case 1: return class_solve_nt<8>(f, ee);
    default: return class_solve_nt<4>(f, ee);
    }
}

const void* pick_factor(int ntmax) {
    switch (ntmax) {
    case 16: return (const void*)batch_factor_kernel<16>;
    case 8: return (const void*)batch_factor_kernel<8>;
    default: return (const void*)batch_factor_kernel<4>;
    }
}

const void* pick_build(int ntmax) {
    switch (ntmax) {
    case 16: return (const void*)batch_build_kernel<16>;
    case 8: return (const void*)batch_build_kernel<8>;
    default: return (const void*)batch_build_kernel<4>;
    }
}


// Constants of the Euler discretisation of Eqs. 10-11 (the helper every
// entry point uses, so the rounding is the same on every path).
EulerConsts batch_consts(const mmgap_params& P) {
    return euler_consts(P.dt, P.p, P.a, P.zeta, P.eps, P.sigma0, P.x_max);
}
constexpr size_t kScratchAlign = 256;
size_t salign(size_t v) { return (v + kScratchAlign - 1) / kScratchAlign * kScratchAlign; }

}  // namespace

const char* BatchRunner::check_params(const mmgap_params& P) {
    if (P.runs != 32) return "batched launch runs 32 anneals per problem (one warp)";
    if (P.f_mvm != 1 && P.f_mvm != 2) return "batched launch supports f_mvm 1 or 2";
    if (P.steps < 0 || P.steps > (1 << 20) || !(P.dt > 0.0f) || !(P.x_max > 0.0f)) return "bad solver parameters";
    if (P.early_exit < 0) return "early_exit must be >= 0";
    return nullptr;
}

const char* BatchRunner::check_early_exit(const mmgap_params& P, const mmgap_detect_job* jobs, int n_jobs,
                                          bool tensor_core) {
    if (P.early_exit <= 0) return nullptr;
    if (tensor_core) return "early exit runs on the exact solver, not the tcgen05 tiles";
    for (int i = 0; i < n_jobs; ++i)
        if (jobs[i].n_t == 32) return "early exit: up to 16 users (a 32-user job)";
    return nullptr;
}

const char* BatchRunner::check_job(const mmgap_detect_job& J) {
    if (!batch_nt(J.n_t) && J.n_t != 32) return "batched launch supports n_t 4, 8, 16, 32";
    if (J.n_r < 1 || J.n_r > kMaxNr) return "n_r out of [1, 64]";
    if (!(J.mod_bits == 2 || J.mod_bits == 4 || J.mod_bits == 6)) return "mod_bits must be 2, 4 or 6";
    if (J.n_problems < 0) return "n_problems < 0";
    if (J.n_problems > 0 && (!J.H || !J.y || !J.noise_var || !J.sym_out || J.n_chan < 1)) return "NULL input/output";
    if (J.n_problems > 0 && !J.chan_index && J.n_chan < J.n_problems) return "chan_index NULL needs n_chan >= n";
    if (J.gram_precision != 0) return "batched launch builds the Gram in FP32 (gram_precision 0)";
    if (J.mapping != MMGAP_MAPPING_DELTA) return "batched launch uses the delta mapping";
    return nullptr;
}

const char* BatchRunner::check_precode(const mmgap_precode_job& J) {
    if (!batch_nt(J.n_u)) return "batched launch supports n_u 4, 8, 16";
    if (J.n_t < J.n_u || J.n_t > kMaxNr) return "n_t out of [n_u, 64]";
    if (!(J.mod_bits == 2 || J.mod_bits == 4 || J.mod_bits == 6)) return "mod_bits must be 2, 4 or 6";
    if (J.n_problems < 0) return "n_problems < 0";
    if (J.inv_precision != MMGAP_INV_FP64 && J.inv_precision != MMGAP_INV_FP32_IR) return "bad inv_precision";
    if (J.n_problems > 0 && (!J.H || !J.u_sym || !J.v_out || J.n_chan < 1)) return "NULL input/output";
    if (J.n_problems > 0 && (uintptr_t)J.H % 8) return "H must be 8-byte aligned";
    if (J.n_problems > 0 && !J.chan_index && J.n_chan < J.n_problems) return "chan_index NULL needs n_chan >= n";
    return nullptr;
}

size_t BatchRunner::precode_scratch_bytes(const mmgap_precode_job& J) {
    const size_t n = 2 * (size_t)J.n_u, P = (size_t)J.n_problems;
    const size_t n_chan = J.chan_index ? (size_t)J.n_chan : P;
    return salign(P * n * n * 2) + salign(P * n * 2) + salign(P * n) +
           salign(n_chan * J.n_u * J.n_u * 16) + salign(n_chan * 4);
}

size_t BatchRunner::factor_bytes(int n_t, int n_chan) {
    const size_t nc = (size_t)std::max(0, n_chan);
    return 2 * salign(nc * 2 * n_t * n_t * sizeof(float)) + 3 * salign(nc * 4);
}

size_t BatchRunner::scratch_bytes(int n_t, int n_problems) {
    const size_t n = 2 * (size_t)n_t, P = (size_t)n_problems;
    return salign(P * n * n * 2) + salign(P * n * 2) + salign(P * n);
}

cudaError_t BatchRunner::init(int device, int capacity_jobs, long long capacity_problems, size_t scratch, int max_n_r,
                              int ntmax, int* err_word, bool tensor_core) {
    device_ = device;
    ntmax = std::min(ntmax, 16);  // the table's kernels; 32-user jobs run their own launches
    tc_ = tensor_core && ntmax >= 8;
    capacity_ = capacity_jobs;
    capacity_problems_ = capacity_problems;
    ntmax_ = ntmax;
    err_word_ = err_word;
    build_floats_ = 0;
    for (int nt : {4, 8, 16})
        if (nt <= ntmax) build_floats_ = std::max(build_floats_, build_floats_for(nt, max_n_r));
    build_floats_ = (build_floats_ + 3) / 4 * 4;
    build_smem_ = (size_t)kBuildWarps * build_floats_ * 4;
    scratch_bytes_ = scratch;
    cudaError_t e;
    if ((e = cudaMalloc(&d_jobs_, sizeof(BatchJob) * (size_t)std::max(1, capacity_jobs))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&scratch_, std::max<size_t>(scratch, 256))) != cudaSuccess) return e;
    if ((e = cudaMallocHost(&h_jobs_, sizeof(BatchJob) * (size_t)std::max(1, capacity_jobs))) != cudaSuccess)
        return e;
    if ((e = cudaMallocHost(&h_head_, sizeof(BatchHeader))) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(pick_build(ntmax), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)build_smem_)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(pick_factor(ntmax), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)build_smem_)) != cudaSuccess)
        return e;
    if ((e = cudaMalloc(&d_fac_, sizeof(FactorJob) * (size_t)std::max(1, capacity_jobs))) != cudaSuccess) return e;
    if ((e = cudaMallocHost(&h_fac_, sizeof(FactorJob) * (size_t)std::max(1, capacity_jobs))) != cudaSuccess)
        return e;
    if (tc_) {
        // the tiles resident on an SM share its 512 TMEM columns (128 per 16-user tile, 64 per
        // 8-user tile): pad shared memory so that no more of them fit
        int smem_sm = 0;
        if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device)) != cudaSuccess)
            return e;
        for (int c = class_lo(); c < 3; ++c) {
            const int ncols = c == 0 ? 128 : (c == 1 ? 64 : 0);  // (4-user tiles take no tensor memory)
            size_t smem = c == 0 ? batch_umma_bytes<16>() : (c == 1 ? batch_umma_bytes<8>() : batch_umma_bytes<4>());
            if (ncols > 0) {
                const size_t floor_bytes = (size_t)smem_sm / (size_t)(512 / ncols + 1) + 1;
                if (smem < floor_bytes) smem = (floor_bytes + 127) & ~(size_t)127;
            }
            umma_smem_[c] = smem;
            for (int f : {1, 2})
                if ((e = cudaFuncSetAttribute(umma_solve(c, f), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem)) != cudaSuccess)
                    return e;
        }
    }
    for (int i = 0; i < 2; ++i)
        if ((e = cudaStreamCreateWithFlags(&side_[i], cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&join_[i], cudaEventDisableTiming)) != cudaSuccess)
            return e;
    return cudaEventCreateWithFlags(&fork_, cudaEventDisableTiming);
}

void BatchRunner::release() {
    if (cap_stream_) cudaStreamDestroy(cap_stream_);
    cap_stream_ = nullptr;
    for (int i = 0; i < 2; ++i) {
        if (side_[i]) cudaStreamDestroy(side_[i]);
        if (join_[i]) cudaEventDestroy(join_[i]);
        side_[i] = nullptr;
        join_[i] = nullptr;
    }
    if (fork_) cudaEventDestroy(fork_);
    fork_ = nullptr;
    if (exec_) cudaGraphExecDestroy(exec_);
    if (graph_) cudaGraphDestroy(graph_);
    if (d_jobs_) cudaFree(d_jobs_);
    if (d_fac_) cudaFree(d_fac_);
    if (h_fac_) cudaFreeHost(h_fac_);
    d_fac_ = h_fac_ = nullptr;
    if (scratch_) cudaFree(scratch_);
    scratch_ = nullptr;
    if (h_jobs_) cudaFreeHost(h_jobs_);
    if (h_head_) cudaFreeHost(h_head_);
    exec_ = nullptr;
    graph_ = nullptr;
    d_jobs_ = h_jobs_ = nullptr;
    h_head_ = nullptr;
}

int BatchRunner::stage(const mmgap_detect_job* jobs, const int* order, int n_jobs) {
    if (n_jobs > capacity_) return -1;
    std::vector<GroupJob> g((size_t)std::max(0, n_jobs));
    for (int i = 0; i < n_jobs; ++i) g[i].det = &jobs[i];
    return stage(g.data(), order, n_jobs);
}

int BatchRunner::stage(const GroupJob* jobs, const int* order, int n_jobs) {
    if (n_jobs > capacity_) return -1;
    pre_.clear();
    wide_.clear();
    // the table groups its jobs by size class (16, then 8, then 4 users; 32-user jobs stay outside
    // it), so that each class's problems are contiguous for the class's solver kernel; within a
    // class the given order holds
    std::vector<int> ord((size_t)std::max(0, n_jobs));
    for (int i = 0; i < n_jobs; ++i) ord[(size_t)i] = order ? order[i] : i;
    auto class_key = [&](int j) { return jobs[j].n_t() == 32 ? -1 : batch_class(jobs[j].n_t()); };
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return class_key(x) < class_key(y); });
    long long first = 0, tiles = 0;
    size_t off = 0;
    int n_table = 0;
    std::vector<int> slot((size_t)std::max(0, n_jobs));  // table index, or -1 - (index into wide_)
    for (int i = 0; i < n_jobs; ++i) {
        const GroupJob& G = jobs[ord[(size_t)i]];
        if (G.det && G.det->n_t == 32) {
            const mmgap_detect_job& J = *G.det;
            const size_t n = 64, P = (size_t)J.n_problems;
            if (off + scratch_bytes(32, J.n_problems) > scratch_bytes_) return -2;
            Wide W{};
            BuildArgs& b = W.b;
            b.H = J.H;
            b.chan_index = J.chan_index;
            b.y = J.y;
            b.noise_var = J.noise_var;
            b.n_r = J.n_r;
            b.mod_bits = J.mod_bits;
            b.n_problems = J.n_problems;
            b.n_chan = J.chan_index ? J.n_chan : J.n_problems;
            qam_kappa(J.mod_bits, &b.kappa, &b.kappa2);
            b.guess_mode = J.guess_in ? 2 : 0;
            b.g_in = J.guess_in;
            b.err = err_word_;
            b.Aq = (int16_t*)(scratch_ + off);
            b.hq = (int16_t*)(scratch_ + off + salign(P * n * n * 2));
            b.g = (int8_t*)(scratch_ + off + salign(P * n * n * 2) + salign(P * n * 2));
            off += scratch_bytes(32, J.n_problems);
            SolveArgs& a = W.a;
            a.err = err_word_;
            a.Aq = b.Aq;
            a.hq = b.hq;
            a.g = b.g;
            a.level_max = (1 << (J.mod_bits >> 1)) - 1;
            a.n_problems = J.n_problems;
            a.key0 = (uint32_t)J.seed;
            a.key1 = (uint32_t)(J.seed >> 32);
            a.problem_offset = J.problem_offset;
            a.d_out = J.offset_out;
            a.E_out = J.energy_out;
            a.ndiv_out = J.ndiv_out;
            a.steps_out = J.steps_out;
            a.sym_out = J.sym_out;
            a.mod_bits = J.mod_bits;
            W.guess_out = J.guess_out;
            slot[i] = -1 - (int)wide_.size();
            if (J.n_problems > 0) wide_.push_back(W);
            continue;
        }
        slot[i] = n_table;
        BatchJob& B = h_jobs_[n_table++];
        B = BatchJob{};
        B.first = first;
        B.tile_first = tiles;
        B.b.err = err_word_;
        if (G.det) {
            const mmgap_detect_job& J = *G.det;
            B.b.H = J.H;
            B.b.chan_index = J.chan_index;
            B.b.y = J.y;
            B.b.noise_var = J.noise_var;
            B.b.n_r = J.n_r;
            B.b.mod_bits = J.mod_bits;
            B.b.n_problems = J.n_problems;
            B.b.n_chan = J.chan_index ? J.n_chan : J.n_problems;
            qam_kappa(J.mod_bits, &B.b.kappa, &B.b.kappa2);
            B.b.guess_mode = J.guess_in ? 2 : 0;
            B.b.g_in = J.guess_in;
            B.nt = J.n_t;
            B.kind = 0;
            B.key0 = (uint32_t)J.seed;
            B.key1 = (uint32_t)(J.seed >> 32);
            B.poff = J.problem_offset;
            const size_t n = 2 * (size_t)J.n_t, P = (size_t)J.n_problems;
            if (off + scratch_bytes(J.n_t, J.n_problems) > scratch_bytes_) return -2;
            B.Aq = (int16_t*)(scratch_ + off);
            B.hq = (int16_t*)(scratch_ + off + salign(P * n * n * 2));
            B.g = (int8_t*)(scratch_ + off + salign(P * n * n * 2) + salign(P * n * 2));
            off += scratch_bytes(J.n_t, J.n_problems);
            B.sym_out = J.sym_out;
            B.energy_out = J.energy_out;
            B.guess_out = J.guess_out;
            B.offset_out = J.offset_out;
            B.ndiv_out = J.ndiv_out;
            B.steps_out = J.steps_out;
            first += J.n_problems;
            tiles += (J.n_problems + 3) / 4;
        } else {
            const mmgap_precode_job& J = *G.pre;
            const size_t n = 2 * (size_t)J.n_u, P = (size_t)J.n_problems;
            const size_t n_chan = J.chan_index ? (size_t)J.n_chan : P;
            if (off + precode_scratch_bytes(J) > scratch_bytes_) return -2;
            char* base = scratch_ + off;
            Precode R{};
            R.job = J;
            R.Aq = (int16_t*)base;
            R.hq = (int16_t*)(base + salign(P * n * n * 2));
            R.d = (int8_t*)((char*)R.hq + salign(P * n * 2));
            R.Q = (double*)((char*)R.d + salign(P * n));
            R.status = (int32_t*)((char*)R.Q + salign(n_chan * J.n_u * J.n_u * 16));
            off += precode_scratch_bytes(J);
            B.b.mod_bits = J.mod_bits;
            B.b.n_problems = J.n_problems;
            B.nt = J.n_u;
            B.kind = 1;
            B.key0 = (uint32_t)J.seed;
            B.key1 = (uint32_t)(J.seed >> 32);
            B.poff = 0;
            B.Aq = R.Aq;
            B.hq = R.hq;
            B.g = nullptr;
            B.offset_out = R.d;
            B.energy_out = J.energy_out;
            B.ndiv_out = J.ndiv_out;
            first += J.n_problems;
            tiles += (J.n_problems + 3) / 4;
            if (J.n_problems > 0) pre_.push_back(R);
        }
    }
    if (first > capacity_problems_) return -3;
    // second pass: per-channel factors for detection jobs whose channels serve
    // several problems, as far as the remaining scratch allows
    fac_.clear();
    for (int i = 0; i < n_jobs; ++i) {
        const GroupJob& G = jobs[ord[(size_t)i]];
        if (!G.det) continue;
        const mmgap_detect_job& J = *G.det;
        if (!J.chan_index || J.n_chan >= J.n_problems || J.n_problems == 0) continue;
        if (J.guess_in) continue;  // a caller-supplied guess needs no MMSE factor
        const size_t fb = factor_bytes(J.n_t, J.n_chan);
        if (off + fb > scratch_bytes_) continue;
        if (slot[i] < 0 && J.n_problems == 0) continue;  // (empty wide jobs are not staged)
        const size_t nc = (size_t)J.n_chan, lb = salign(nc * 2 * J.n_t * J.n_t * sizeof(float)), rb = salign(nc * 4);
        char* base = scratch_ + off;
        off += fb;
        BuildArgs& B = slot[i] >= 0 ? h_jobs_[slot[i]].b : wide_[(size_t)(-1 - slot[i])].b;
        Factor F{};
        F.n_t = J.n_t;
        ChanFactorArgs& f = F.args;
        f.H = J.H;
        f.chan_index = J.chan_index;
        f.noise_var = J.noise_var;
        f.n_r = J.n_r;
        f.n_problems = J.n_problems;
        f.n_chan = J.n_chan;
        f.kappa = B.kappa;
        f.kappa2 = B.kappa2;
        f.L_out = (float*)base;
        f.rho_out = (float*)(base + lb);
        f.chol_out = (int32_t*)(base + lb + rb);
        f.first = (int32_t*)(base + lb + 2 * rb);
        f.G_out = (float*)(base + lb + 3 * rb);
        B.Gc_pre = f.G_out;
        B.L_pre = f.L_out;
        B.rho_pre = f.rho_out;
        B.chol_pre = f.chol_out;
        fac_.push_back(F);
    }
    n_fac_ = 0;
    fac_chan_ = fac_prob_ = 0;
    for (const Factor& F : fac_) {
        if (F.n_t == 32) continue;  // (their own launches)
        FactorJob& Q = h_fac_[n_fac_++];
        Q.a = F.args;
        Q.nt = F.n_t;
        Q.chan_first = fac_chan_;
        Q.prob_first = fac_prob_;
        fac_chan_ += F.args.n_chan;
        fac_prob_ += F.args.n_problems;
    }
    h_head_->n_jobs = n_table;
    h_head_->pad = 0;
    for (int c = 0; c < 3; ++c) cls_first_[c] = cls_count_[c] = cls_tile_first_[c] = cls_tiles_[c] = 0;
    for (int j = 0; j < n_table; ++j) {
        const BatchJob& B = h_jobs_[j];
        const int c = batch_class(B.nt);
        if (cls_count_[c] == 0) cls_first_[c] = B.first;
        if (cls_tiles_[c] == 0) cls_tile_first_[c] = B.tile_first;
        cls_count_[c] += B.b.n_problems;
        cls_tiles_[c] += (B.b.n_problems + 3) / 4;
    }
    h_head_->total = first;
    h_head_->tiles = tiles;
    return 0;
}

namespace {

cudaError_t vpp_build_nu(int n_u, const VppBuildArgs& a, cudaStream_t s) {
    switch (n_u) {
    case 16: return launch_vpp_build<16>(a, s);
    case 8: return launch_vpp_build<8>(a, s);
    default: return launch_vpp_build<4>(a, s);
    }
}

cudaError_t vpp_output_nu(int n_u, const VppOutArgs& a, cudaStream_t s) {
    switch (n_u) {
    case 16: return launch_vpp_output<16>(a, s);
    case 8: return launch_vpp_output<8>(a, s);
    default: return launch_vpp_output<4>(a, s);
    }
}

}  // namespace

cudaError_t BatchRunner::wide_before(const mmgap_params& P, cudaStream_t s) {
    const EulerConsts k = batch_consts(P);
    for (Wide& W : wide_) {
        cudaError_t e = launch_build_detect<32>(W.b, s);
        if (e != cudaSuccess) return e;
        W.a.steps = P.steps;
        W.a.f_mvm = P.f_mvm;
        W.a.k = k;
        if ((e = launch_solve<32>(W.a, P.runs, s)) != cudaSuccess) return e;
        if (W.guess_out &&
            (e = cudaMemcpyAsync(W.guess_out, W.b.g, (size_t)W.b.n_problems * 64, cudaMemcpyDeviceToDevice, s)) !=
                cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

cudaError_t BatchRunner::factor_before(cudaStream_t s) {
    cudaError_t e;
    for (const Factor& F : fac_)
        if (F.n_t == 32 && (e = launch_chan_factor<32>(F.args, s)) != cudaSuccess) return e;
    if (n_fac_ == 0) return cudaSuccess;
    // every other job's channels in three launches (one launch per job and kernel left the GPU
    // idle between small jobs' launches)
    if ((e = cudaMemcpyAsync(d_fac_, h_fac_, sizeof(FactorJob) * (size_t)n_fac_, cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return e;
    FactorBatch F{d_fac_, n_fac_, fac_chan_, fac_prob_, build_floats_};
    auto blocks = [](long long n) { return (unsigned)std::min<long long>(std::max(1LL, (n + 255) / 256), 4096); };
    batch_factor_init_kernel<<<blocks(fac_chan_), 256, 0, s>>>(F);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    batch_factor_first_kernel<<<blocks(fac_prob_), 256, 0, s>>>(F);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    void* args[] = {&F};
    return cudaLaunchKernel(pick_factor(ntmax_), dim3((unsigned)((fac_chan_ + kBuildWarps - 1) / kBuildWarps)),
                            dim3(kBuildWarps * 32), args, build_smem_, s);
}

cudaError_t BatchRunner::precode_before(cudaStream_t s) {
    for (const Precode& R : pre_) {
        const mmgap_precode_job& J = R.job;
        const int n_chan = J.chan_index ? J.n_chan : J.n_problems;
        cudaError_t e = vpp_inverse_any(J.n_u, J.n_t, n_chan, J.H, J.inv_precision, R.Q, R.status, s);
        if (e != cudaSuccess) return e;
        VppBuildArgs b{};
        b.Q = R.Q;
        b.chan_index = J.chan_index;
        b.u_sym = J.u_sym;
        b.mod_bits = J.mod_bits;
        b.n_problems = J.n_problems;
        b.n_chan = n_chan;
        b.err = err_word_;
        b.Aq = R.Aq;
        b.hq = R.hq;
        if ((e = vpp_build_nu(J.n_u, b, s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t BatchRunner::precode_after(cudaStream_t s) {
    for (const Precode& R : pre_) {
        const mmgap_precode_job& J = R.job;
        VppOutArgs o{};
        o.H = J.H;
        o.Q = R.Q;
        o.chan_index = J.chan_index;
        o.u_sym = J.u_sym;
        o.d = R.d;
        o.n_t = J.n_t;
        o.mod_bits = J.mod_bits;
        o.n_problems = J.n_problems;
        o.n_chan = J.chan_index ? J.n_chan : J.n_problems;
        o.err = err_word_;
        o.v_out = J.v_out;
        o.x_out = J.x_out;
        o.power_out = J.power_out;
        cudaError_t e = vpp_output_nu(J.n_u, o, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

unsigned BatchRunner::build_grid() const {  // one warp per problem
    return (unsigned)((std::max(1LL, h_head_->total) + kBuildWarps - 1) / kBuildWarps);
}

const void* BatchRunner::solver_fn(int c, const mmgap_params& P) const {
    return tc_ ? umma_solve(c, P.f_mvm) : class_solve(c, P.f_mvm, P.early_exit > 0);
}

unsigned BatchRunner::solver_grid(int c) const {  // a CTA per problem, or per tile of 4 problems of one job
    return (unsigned)std::max(1LL, tc_ ? cls_tiles_[c] : cls_count_[c]);
}

int BatchRunner::class_lo() const { return batch_class(ntmax_); }

cudaError_t BatchRunner::enqueue(const mmgap_params& P, cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaMemcpyAsync(d_jobs_, h_jobs_, sizeof(BatchJob) * (size_t)std::max(1, capacity_),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return e;
    BatchArgs& a = args_;
    a = BatchArgs{};
    a.jobs = d_jobs_;
    a.n_jobs = h_head_->n_jobs;
    a.total = h_head_->total;
    a.tiles = h_head_->tiles;
    a.steps = P.steps;
    a.early_exit = P.early_exit;
    a.k = batch_consts(P);
    a.build_floats = build_floats_;
    for (int c = 0; c < 3; ++c) {
        a.cls_first[c] = cls_first_[c];
        a.cls_count[c] = cls_count_[c];
        a.cls_tile_first[c] = cls_tile_first_[c];
        a.cls_tiles[c] = cls_tiles_[c];
    }
    void* args[] = {&a};
    if ((e = cudaLaunchKernel(pick_build(ntmax_), dim3(build_grid()), dim3(kBuildWarps * 32), args, build_smem_,
                              s)) != cudaSuccess)
        return e;
    // one solver kernel per size class; with more than one class they are independent branches
    // (fork from s through an event, the other classes on the side streams, joined back into s)
    const int c0 = class_lo(), nside = 2 - c0;
    if (nside > 0) {
        if ((e = cudaEventRecord(fork_, s)) != cudaSuccess) return e;
        for (int i = 0; i < nside; ++i)
            if ((e = cudaStreamWaitEvent(side_[i], fork_, 0)) != cudaSuccess) return e;
    }
    for (int c = c0; c < 3; ++c) {
        cudaStream_t cs = c == c0 ? s : side_[c - c0 - 1];
        if ((e = cudaLaunchKernel(solver_fn(c, P), dim3(solver_grid(c)), dim3(solver_block()), args, solver_smem(c),
                                  cs)) != cudaSuccess)
            return e;
    }
    for (int i = 0; i < nside; ++i) {
        if ((e = cudaEventRecord(join_[i], side_[i])) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s, join_[i], 0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t BatchRunner::run(const mmgap_params& P, cudaStream_t s, bool use_graph) {
    cudaError_t e = factor_before(s);
    if (e != cudaSuccess) return e;
    e = precode_before(s);
    if (e != cudaSuccess) return e;
    if ((e = wide_before(P, s)) != cudaSuccess) return e;
    if (h_head_->n_jobs > 0 && (e = run_batch(P, s, use_graph)) != cudaSuccess) return e;
    if (P.early_exit <= 0) {  // every problem of the table's jobs took all the steps
        for (int j = 0; j < h_head_->n_jobs; ++j) {
            const BatchJob& B = h_jobs_[j];
            if (!B.steps_out || B.b.n_problems <= 0) continue;
            fill_steps_kernel<<<(B.b.n_problems + 255) / 256, 256, 0, s>>>(B.steps_out, B.b.n_problems, P.steps);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    return precode_after(s);
}

cudaError_t BatchRunner::run_batch(const mmgap_params& P, cudaStream_t s, bool use_graph) {
    if (!use_graph) return enqueue(P, s);
    cudaError_t e;
    if (exec_ && std::memcmp(&graph_params_, &P, sizeof P) != 0) {  // parameters are baked into the graph
        cudaGraphExecDestroy(exec_);
        cudaGraphDestroy(graph_);
        exec_ = nullptr;
        graph_ = nullptr;
    }
    if (!exec_) {
        // capture on the runner's own stream (the caller's may be the legacy
        // default stream, which cannot be captured); replay on the caller's
        if (!cap_stream_ && (e = cudaStreamCreateWithFlags(&cap_stream_, cudaStreamNonBlocking)) != cudaSuccess)
            return e;
        if ((e = cudaStreamBeginCapture(cap_stream_, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
        cudaError_t le = enqueue(P, cap_stream_);
        e = cudaStreamEndCapture(cap_stream_, &graph_);
        if (le != cudaSuccess) return le;
        if (e != cudaSuccess) return e;
        if ((e = cudaGraphInstantiate(&exec_, graph_, 0)) != cudaSuccess) return e;
        graph_params_ = P;
        // remember the kernel nodes so each replay can size their grids: the builder and one
        // solver per size class
        build_node_ = nullptr;
        for (cudaGraphNode_t& nd : solve_nodes_) nd = nullptr;
        size_t count = 0;
        if ((e = cudaGraphGetNodes(graph_, nullptr, &count)) != cudaSuccess) return e;
        std::vector<cudaGraphNode_t> nodes(count);
        if ((e = cudaGraphGetNodes(graph_, nodes.data(), &count)) != cudaSuccess) return e;
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
            cudaKernelNodeParams kp;
            if (cudaGraphKernelNodeGetParams(nd, &kp) != cudaSuccess) continue;
            if (kp.func == pick_build(ntmax_)) build_node_ = nd;
            else
                for (int c = class_lo(); c < 3; ++c)
                    if (kp.func == solver_fn(c, P)) solve_nodes_[c] = nd;
        }
        if (!build_node_) return cudaErrorInvalidValue;
        for (int c = class_lo(); c < 3; ++c)
            if (!solve_nodes_[c]) return cudaErrorInvalidValue;
    } else {
        // grids and counts follow the staged header; the other kernel arguments are unchanged
        args_.n_jobs = h_head_->n_jobs;
        args_.total = h_head_->total;
        args_.tiles = h_head_->tiles;
        for (int c = 0; c < 3; ++c) {
            args_.cls_first[c] = cls_first_[c];
            args_.cls_count[c] = cls_count_[c];
            args_.cls_tile_first[c] = cls_tile_first_[c];
            args_.cls_tiles[c] = cls_tiles_[c];
        }
        void* args[] = {&args_};
        cudaKernelNodeParams kb{};
        kb.func = (void*)pick_build(ntmax_);
        kb.gridDim = dim3(build_grid());
        kb.blockDim = dim3(kBuildWarps * 32);
        kb.sharedMemBytes = (unsigned)build_smem_;
        kb.kernelParams = args;
        if ((e = cudaGraphExecKernelNodeSetParams(exec_, build_node_, &kb)) != cudaSuccess) return e;
        cudaKernelNodeParams ks{};
        ks.kernelParams = args;
        for (int c = class_lo(); c < 3; ++c) {
            ks.func = (void*)solver_fn(c, P);
            ks.gridDim = dim3(solver_grid(c));
            ks.blockDim = dim3(solver_block());
            ks.sharedMemBytes = (unsigned)solver_smem(c);
            if ((e = cudaGraphExecKernelNodeSetParams(exec_, solve_nodes_[c], &ks)) != cudaSuccess) return e;
        }
    }
    return cudaGraphLaunch(exec_, s);
}

}  // namespace mmgap

struct mmgap_batch {
    mmgap::BatchRunner runner;
    mmgap_params params{};
    std::vector<mmgap_detect_job> jobs;
    int* err_word = nullptr;
    int device = 0;
};

extern "C" {

mmgap_status mmgap_batch_create(mmgap_batch** out, int device, const mmgap_params* params,
                                const mmgap_detect_job* jobs, int n_jobs, int flags) {
    if (!out) return MMGAP_EINVAL;
    *out = nullptr;
    if (!params || n_jobs < 1 || !jobs) return MMGAP_EINVAL;
    if (flags & ~MMGAP_BATCH_TENSOR_CORE) {
        fprintf(stderr, "mmgap_batch_create: unknown flags 0x%x\n", (unsigned)flags);
        return MMGAP_EINVAL;
    }
    if (const char* why = BatchRunner::check_early_exit(*params, jobs, n_jobs, (flags & MMGAP_BATCH_TENSOR_CORE) != 0)) {
        fprintf(stderr, "mmgap_batch_create: %s\n", why);
        return MMGAP_EUNSUPPORTED;
    }
    if (BatchRunner::check_params(*params)) {
        fprintf(stderr, "mmgap_batch_create: %s\n", BatchRunner::check_params(*params));
        return MMGAP_EUNSUPPORTED;
    }
    int ntmax = 4, max_n_r = 1;
    long long total = 0;
    size_t scratch = 0;
    for (int i = 0; i < n_jobs; ++i) {
        if (const char* why = BatchRunner::check_job(jobs[i])) {
            fprintf(stderr, "mmgap_batch_create: job %d: %s\n", i, why);
            return MMGAP_EUNSUPPORTED;
        }
        if (jobs[i].n_t != 32) {  // (32-user jobs run their own launches: not in the table's kernels)
            ntmax = std::max(ntmax, jobs[i].n_t);
            max_n_r = std::max(max_n_r, jobs[i].n_r);
            total += jobs[i].n_problems;
        }
        scratch += BatchRunner::scratch_bytes(jobs[i].n_t, jobs[i].n_problems);
        if (jobs[i].chan_index && jobs[i].n_chan < jobs[i].n_problems)
            scratch += BatchRunner::factor_bytes(jobs[i].n_t, jobs[i].n_chan);
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return MMGAP_EINVAL;
    auto* b = new (std::nothrow) mmgap_batch();
    if (!b) return MMGAP_ENOMEM;
    b->device = device;
    b->params = *params;
    b->jobs.assign(jobs, jobs + n_jobs);
    mmgap_status st = MMGAP_OK;
    if (cudaMalloc(&b->err_word, sizeof(int)) != cudaSuccess || cudaMemset(b->err_word, 0, sizeof(int)) != cudaSuccess)
        st = MMGAP_ENOMEM;
    if (st == MMGAP_OK && b->runner.init(device, n_jobs, total, scratch, max_n_r, ntmax, b->err_word,
                                         (flags & MMGAP_BATCH_TENSOR_CORE) != 0) != cudaSuccess)
        st = MMGAP_ENOMEM;
    if (st == MMGAP_OK) {
        // largest problems first, so the tail of the launch is made of small ones
        std::vector<int> order(n_jobs);
        for (int i = 0; i < n_jobs; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return jobs[x].n_t > jobs[y].n_t; });
        if (b->runner.stage(jobs, order.data(), n_jobs) != 0) st = MMGAP_EINVAL;
    }
    if (st != MMGAP_OK) {
        cudaGetLastError();
        b->runner.release();
        if (b->err_word) cudaFree(b->err_word);
        delete b;
        if (prev >= 0) cudaSetDevice(prev);
        return st;
    }
    if (prev >= 0) cudaSetDevice(prev);
    *out = b;
    return MMGAP_OK;
}

mmgap_status mmgap_batch_run(mmgap_batch* b, int use_graph, void* stream) {
    NvtxRange nvtx_range("mmgap_batch_run");
    if (!b) return MMGAP_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    cudaError_t e = b->runner.run(b->params, (cudaStream_t)stream, use_graph != 0);
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        fprintf(stderr, "mmgap_batch_run: %s\n", cudaGetErrorString(e));
        return MMGAP_ECUDA;
    }
    return MMGAP_OK;
}

mmgap_status mmgap_batch_destroy(mmgap_batch* b) {
    if (!b) return MMGAP_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    b->runner.release();
    cudaFree(b->err_word);
    delete b;
    if (prev >= 0) cudaSetDevice(prev);
    return MMGAP_OK;
}

}  // extern "C"
