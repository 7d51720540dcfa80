// MMGaP hot-path kernels for sm_103a.
//
// Three stages (Sec. 3.2, Fig. 4: pre-processing, solver, post-processing):
//   build_detect_kernel  -- Gram + matched filter + MMSE guess + field +
//                           Q14 quantisation, one warp per resource element
//   cac_solve_kernel     -- CIM-CAC anneals (Eqs. 10-11) with the half-size
//                           coupling field of Fig. 5, one thread per anneal,
//                           warp shuffles for the arg-min, fused decode
//   vpp_* kernels        -- downlink VPP (Sec. 3.3) in FP64
//
// Every floating-point operation that decides an integer result is written
// with an explicit IEEE round-to-nearest intrinsic (__fmaf_rn, __fmul_rn,
// __fadd_rn, __fdiv_rn, __fsqrt_rn and their double forms) in a fixed order,
// so that guesses, quantised couplings, spins and symbols are reproducible
// bit for bit by a sequential CPU implementation of the same order.  The
// translation units are compiled with -fmad=false as a second guard.
//
// The kernels live in one header per stage, included here in dependency order:
//   common.cuh        Philox, IEEE helpers, dynamic shared-memory limits
//   build.cuh         builder (Gram, MMSE / SIC guess, field, Q14)
//   solve.cuh         CIM-CAC solver and its bit-identical launch shapes
//   solve_rows.cuh    CIM-CAC solver for 32 users (row blocks, two anneals per thread)
//   umma.cuh          tcgen05 field refresh (solver shape 8)
//   batch_kernels.cuh batched launch over a job table
//   direct.cuh        direct spin mapping: builder and general solver
//   gram_select.cuh   tensor-core Gram, MMGaP-E selection
//   vpp.cuh           downlink VPP
//   launch.cuh        host-side launchers
#pragma once
#include "launch.cuh"

// Explicit instantiation of every launcher for one n_t.
#define MMGAP_INSTANTIATE(NT)                                                                                  \
    namespace mmgap {                                                                                          \
    template <> cudaError_t launch_build_detect<NT>(const BuildArgs& a, cudaStream_t s) {                      \
        return launch_build_detect_impl<NT>(a, s);                                                             \
    }                                                                                                          \
    template <> cudaError_t launch_chan_factor<NT>(const ChanFactorArgs& a, cudaStream_t s) {                  \
        return launch_chan_factor_impl<NT>(a, s);                                                              \
    }                                                                                                          \
    template <> cudaError_t launch_solve<NT>(const SolveArgs& a, int runs, cudaStream_t s) {                   \
        return launch_solve_impl<NT>(a, runs, s);                                                              \
    }                                                                                                          \
    template <> cudaError_t launch_vpp_inverse<NT>(const VppInvArgs& a, cudaStream_t s) {                      \
        return launch_vpp_inverse_impl<NT>(a, s);                                                              \
    }                                                                                                          \
    template <> cudaError_t launch_vpp_build<NT>(const VppBuildArgs& a, cudaStream_t s) {                      \
        return launch_vpp_build_impl<NT>(a, s);                                                                \
    }                                                                                                          \
    template <> cudaError_t launch_vpp_output<NT>(const VppOutArgs& a, cudaStream_t s) {                       \
        return launch_vpp_output_impl<NT>(a, s);                                                               \
    }                                                                                                          \
    template <> cudaError_t launch_gram_tc<NT>(const GramArgs& a, cudaStream_t s) {                            \
        return launch_gram_tc_impl<NT>(a, s);                                                                  \
    }                                                                                                          \
    template <> cudaError_t launch_select<NT>(const SelectArgs& a, cudaStream_t s) {                           \
        return launch_select_impl<NT>(a, s);                                                                   \
    }                                                                                                          \
    template <> cudaError_t launch_vpp_inverse_ir<NT>(const VppInvArgs& a, cudaStream_t s) {                   \
        return launch_vpp_inverse_ir_impl<NT>(a, s);                                                           \
    }                                                                                                          \
    template <> cudaError_t launch_build_direct<NT>(const DirectBuildArgs& a, cudaStream_t s) {                \
        return launch_build_direct_impl<NT>(a, s);                                                             \
    }                                                                                                          \
    }
