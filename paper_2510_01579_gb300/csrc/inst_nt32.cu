// Launchers for 32 users: detection only (per-channel factor, build, solve).
#include "kernels.cuh"

namespace mmgap {
template <> cudaError_t launch_build_detect<32>(const BuildArgs& a, cudaStream_t s) {
    return launch_build_detect_impl<32>(a, s);
}
template <> cudaError_t launch_chan_factor<32>(const ChanFactorArgs& a, cudaStream_t s) {
    return launch_chan_factor_impl<32>(a, s);
}
template <> cudaError_t launch_solve<32>(const SolveArgs& a, int runs, cudaStream_t s) {
    return launch_solve_impl<32>(a, runs, s);
}
}  // namespace mmgap
