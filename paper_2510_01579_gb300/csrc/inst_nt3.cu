// Kernel instantiations for n_t = 3 users (n = 6 half-size spins).
// One translation unit per size so the build compiles them in parallel.
#include "kernels.cuh"

MMGAP_INSTANTIATE(3)
