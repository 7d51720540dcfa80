// Kernel instantiations for n_t = 16 users (n = 32 half-size spins).
// One translation unit per size so the build compiles them in parallel.
#include "kernels.cuh"

MMGAP_INSTANTIATE(16)
