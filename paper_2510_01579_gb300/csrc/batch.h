// Internal runner of the batched persistent launch (shared by the batch
// objects and the serving loop).  Not part of the ABI.
#pragma once
#include <cstring>

#include <cuda_runtime.h>

#include "../../include/mmgap.h"
#include "kernels.cuh"

namespace mmgap {

class BatchRunner {
  public:
    // Reasons a parameter set / job cannot use the batched launch (nullptr = ok).
    static const char* check_params(const mmgap_params& P);
    static const char* check_job(const mmgap_detect_job& J);

    // Scratch bytes (Q14 couplings, field, guess) of one job.
    static size_t scratch_bytes(int n_t, int n_problems);
    // Device job table for up to capacity_jobs jobs and capacity_problems
    // problems with n_r <= max_n_r and n_t <= ntmax, `scratch` bytes of
    // coupling scratch; err_word receives out-of-range channel indices.
    // persistent: the solver runs warps that pull problems from an atomic
    // counter; otherwise one 32-thread CTA per problem.
    cudaError_t init(int device, int capacity_jobs, long long capacity_problems, size_t scratch, int max_n_r, int ntmax,
                     int* err_word, bool persistent);
    void release();
    // Fill the pinned host table with jobs[order[i]] (order may be NULL);
    // returns 0, or < 0 if the jobs exceed the table, scratch or problem capacity.
    int stage(const mmgap_detect_job* jobs, const int* order, int n_jobs);
    // Copy the staged table to the device and launch (or replay the graph of)
    // the persistent kernel on s.
    cudaError_t run(const mmgap_params& P, cudaStream_t s, bool use_graph);
    int grid() const { return grid_; }

  private:
    cudaError_t enqueue(const mmgap_params& P, cudaStream_t s);
    void grids(unsigned* build_grid, unsigned* solve_grid) const;
    int device_ = 0, capacity_ = 0, ntmax_ = 16, build_floats_ = 0, grid_ = 0, build_grid_max_ = 1;
    bool persistent_ = false;
    long long capacity_problems_ = 0;
    size_t build_smem_ = 0, scratch_bytes_ = 0;
    char* scratch_ = nullptr;
    int* err_word_ = nullptr;
    BatchJob* d_jobs_ = nullptr;
    BatchJob* h_jobs_ = nullptr;
    BatchHeader* d_head_ = nullptr;
    BatchHeader* h_head_ = nullptr;
    cudaStream_t cap_stream_ = nullptr;
    cudaGraph_t graph_ = nullptr;
    cudaGraphNode_t build_node_ = nullptr, solve_node_ = nullptr;
    cudaGraphExec_t exec_ = nullptr;
    mmgap_params graph_params_{};
    BatchArgs args_{};
};

}  // namespace mmgap
