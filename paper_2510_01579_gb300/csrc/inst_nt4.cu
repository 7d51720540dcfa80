// Kernel instantiations for n_t = 4 users (n = 8 half-size spins).
// One translation unit per size so the build compiles them in parallel.
#include "kernels.cuh"

MMGAP_INSTANTIATE(4)
