// General-coupling CIM-CAC solver instances (direct spin mapping).
#include "kernels.cuh"

namespace mmgap {

bool general_supported(int N) { return N == 8 || N == 16 || N == 24 || N == 32 || N == 48 || N == 64 || N == 96; }

cudaError_t launch_solve_general(int N, const GeneralArgs& a, int runs, cudaStream_t s) {
    switch (N) {
    case 8: return launch_general_impl<8>(a, runs, s);
    case 16: return launch_general_impl<16>(a, runs, s);
    case 24: return launch_general_impl<24>(a, runs, s);
    case 32: return launch_general_impl<32>(a, runs, s);
    case 48: return launch_general_impl<48>(a, runs, s);
    case 64: return launch_general_impl<64>(a, runs, s);
    case 96: return launch_general_impl<96>(a, runs, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace mmgap
