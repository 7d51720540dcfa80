// Kernel instantiations for n_t = 2 users (n = 4 half-size spins).
// One translation unit per size so the build compiles them in parallel.
#include "kernels.cuh"

MMGAP_INSTANTIATE(2)
