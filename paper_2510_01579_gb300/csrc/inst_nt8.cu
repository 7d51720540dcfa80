// Kernel instantiations for n_t = 8 users (n = 16 half-size spins).
// One translation unit per size so the build compiles them in parallel.
#include "kernels.cuh"

MMGAP_INSTANTIATE(8)
