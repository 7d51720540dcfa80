// Internal runner of the batched launch (shared by the batch objects and the
// serving loop).  Not part of the ABI.
#pragma once
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mmgap.h"
#include "kernels.cuh"

namespace mmgap {

// One job of a group: a detection job or a VPP precoding job (exactly one set).
struct GroupJob {
    const mmgap_detect_job* det = nullptr;
    const mmgap_precode_job* pre = nullptr;
    int n_t() const { return det ? det->n_t : pre->n_u; }
};

class BatchRunner {
  public:
    // Reasons a parameter set / job cannot use the batched launch (nullptr = ok).
    static const char* check_params(const mmgap_params& P);
    static const char* check_job(const mmgap_detect_job& J);
    static const char* check_precode(const mmgap_precode_job& J);
    // Early exit (params.early_exit > 0) needs the exact solver and jobs of at most 16 users.
    static const char* check_early_exit(const mmgap_params& P, const mmgap_detect_job* jobs, int n_jobs,
                                        bool tensor_core);

    // Scratch bytes (Q14 couplings, field, guess) of one job.
    static size_t scratch_bytes(int n_t, int n_problems);
    // Scratch bytes of the per-channel MMSE factors of a detection job whose
    // n_chan channels serve several problems each (optional: staged when the
    // scratch has room after every job's own scratch).
    static size_t factor_bytes(int n_t, int n_chan);
    // Scratch bytes of one precoding job: couplings, field, offsets, the
    // channel inverses and their flags.
    static size_t precode_scratch_bytes(const mmgap_precode_job& J);
    // Device job table for up to capacity_jobs jobs and capacity_problems
    // problems with n_r <= max_n_r and n_t <= ntmax (the table's kernels are
    // sized for min(ntmax, 16); 32-user jobs stay outside the table), `scratch`
    // bytes of coupling scratch; err_word receives out-of-range channel indices.
    // The solver runs one 32-thread CTA per problem, one kernel per size class
    // (the classes concurrently, on the runner's side streams); tensor_core: the
    // field refresh of 8- and 16-user problems as tcgen05 MMAs instead (solver
    // shape 8, a precision variant; 128-thread CTAs over 4-problem tiles).
    // Creates the side streams and events of the class launches.
    cudaError_t init(int device, int capacity_jobs, long long capacity_problems, size_t scratch, int max_n_r, int ntmax,
                     int* err_word, bool tensor_core = false);
    void release();
    // Fill the pinned host table with jobs[order[i]] (order may be NULL),
    // grouped by size class (16, 8, 4 users) with the given order kept within
    // each class, and the factor table of the jobs' per-channel factorisations;
    // returns 0, or < 0 if the jobs exceed the table, scratch or problem capacity.
    int stage(const mmgap_detect_job* jobs, const int* order, int n_jobs);
    int stage(const GroupJob* jobs, const int* order, int n_jobs);
    // Launch on s: the per-channel factorisations, each precoding job's
    // channel inverse and VPP build, each 32-user job's build and row-block
    // solve, then the batch of the other jobs (table upload, builder,
    // solver; or the graph of them), then each precoding job's output kernel.
    cudaError_t run(const mmgap_params& P, cudaStream_t s, bool use_graph);

  private:
    struct Precode {  // a staged precoding job and its scratch
        mmgap_precode_job job;
        int16_t* Aq;
        int16_t* hq;
        int8_t* d;
        double* Q;
        int32_t* status;
    };
    cudaError_t enqueue(const mmgap_params& P, cudaStream_t s);
    cudaError_t run_batch(const mmgap_params& P, cudaStream_t s, bool use_graph);
    cudaError_t precode_before(cudaStream_t s);
    // per-channel factorisation of the staged jobs: 32-user jobs one launch each, the others in
    // three launches over the factor table
    cudaError_t factor_before(cudaStream_t s);
    struct Factor {
        int n_t;
        ChanFactorArgs args;
    };
    std::vector<Factor> fac_;
    FactorJob* h_fac_ = nullptr;  // pinned factor table (jobs of up to 16 users)
    FactorJob* d_fac_ = nullptr;
    int n_fac_ = 0;
    long long fac_chan_ = 0, fac_prob_ = 0;  // channels and problems of the factor table
    cudaError_t precode_after(cudaStream_t s);
    std::vector<Precode> pre_;
    // 32-user detection jobs: outside the job table (the mixed-size kernels
    // stop at 16 users), with their own builder and row-block solver launches
    struct Wide {
        BuildArgs b;
        SolveArgs a;
        int8_t* guess_out;
    };
    std::vector<Wide> wide_;
    cudaError_t wide_before(const mmgap_params& P, cudaStream_t s);
    unsigned build_grid() const;
    int class_lo() const;  // the runner's first size class: batch_class(ntmax_)
    // size class c's solver: the grid kernel (CTA per problem) or the tcgen05 tiles
    const void* solver_fn(int c, const mmgap_params& P) const;
    unsigned solver_grid(int c) const;  // (at least 1 CTA)
    unsigned solver_block() const { return tc_ ? 128u : 32u; }
    size_t solver_smem(int c) const { return tc_ ? umma_smem_[c] : 0; }
    int device_ = 0, capacity_ = 0, ntmax_ = 16, build_floats_ = 0;
    bool tc_ = false;  // tcgen05 field refresh for 8 and 16 users (4-problem tiles)
    size_t umma_smem_[3] = {0, 0, 0};  // dynamic shared memory of each class's tcgen05 solver
    long long capacity_problems_ = 0;
    size_t build_smem_ = 0, scratch_bytes_ = 0;
    char* scratch_ = nullptr;
    int* err_word_ = nullptr;
    BatchJob* d_jobs_ = nullptr;
    BatchJob* h_jobs_ = nullptr;
    BatchHeader* h_head_ = nullptr;
    // the grid solver's size classes (batch_class): first problem and count of each in the table
    long long cls_first_[3] = {0, 0, 0}, cls_count_[3] = {0, 0, 0};
    long long cls_tile_first_[3] = {0, 0, 0}, cls_tiles_[3] = {0, 0, 0};  // the tcgen05 solver's tiles
    // side streams and events of the classes' concurrent solver launches (fork and join)
    cudaStream_t side_[2] = {nullptr, nullptr};
    cudaEvent_t fork_ = nullptr, join_[2] = {nullptr, nullptr};
    cudaStream_t cap_stream_ = nullptr;
    cudaGraph_t graph_ = nullptr;
    cudaGraphNode_t build_node_ = nullptr, solve_nodes_[3] = {nullptr, nullptr, nullptr};
    cudaGraphExec_t exec_ = nullptr;
    mmgap_params graph_params_{};
    BatchArgs args_{};
};

}  // namespace mmgap
