// Kernel instantiations for n_t = 1 users (n = 2 half-size spins).
// One translation unit per size so the build compiles them in parallel.
#include "kernels.cuh"

MMGAP_INSTANTIATE(1)
