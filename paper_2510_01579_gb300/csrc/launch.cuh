// Host-side launchers of every kernel (grid sizes, dynamic shared memory, shapes).
#pragma once
#include "build.cuh"
#include "solve.cuh"
#include "solve_rows.cuh"
#include "umma.cuh"
#include "batch_kernels.cuh"
#include "direct.cuh"
#include "gram_select.cuh"
#include "vpp.cuh"

namespace mmgap {

// ------------------------------------------------------------- launchers
template <int NT>
cudaError_t launch_build_detect_impl(const BuildArgs& a, cudaStream_t s) {
    if (a.n_problems <= 0) return cudaSuccess;
    const size_t smem = (size_t)kBuildWarps * build_smem_floats<NT>(a.n_r) * sizeof(float);
    cudaError_t err = ensure_dynamic_smem<build_detect_kernel<NT>>(smem);
    if (err != cudaSuccess) return err;
    const int blocks = (a.n_problems + kBuildWarps - 1) / kBuildWarps;
    build_detect_kernel<NT><<<blocks, kBuildWarps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

template <int NT>
cudaError_t launch_chan_factor_impl(const ChanFactorArgs& a, cudaStream_t s) {
    if (a.n_chan <= 0 || a.n_problems <= 0) return cudaSuccess;
    cudaError_t err = cudaMemsetAsync(a.first, 0x7f, (size_t)a.n_chan * sizeof(int32_t), s);  // > any index
    if (err != cudaSuccess) return err;
    chan_first_kernel<NT><<<(a.n_problems + 255) / 256, 256, 0, s>>>(a);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    const size_t smem = (size_t)kBuildWarps * build_smem_floats<NT>(a.n_r) * sizeof(float);
    if ((err = ensure_dynamic_smem<chan_factor_kernel<NT>>(smem)) != cudaSuccess) return err;
    chan_factor_kernel<NT><<<(a.n_chan + kBuildWarps - 1) / kBuildWarps, kBuildWarps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

// Latency: when few problems would leave SMs idle, each problem of a shape with
// TPA threads per anneal runs as a cluster of CL CTAs (4 or 2), each with
// runs / CL of its anneals on its own SM; the same bits (the anneals keep their
// indices in the problem).  Returns the cluster size to use, 1 for none.
template <int TPA>
int tuned_cluster_size(const SolveArgs& a, int runs) {
    if (a.n_sm <= 0 || a.n_problems <= 0) return 1;
    for (int cl : {4, 2})
        if (runs % cl == 0 && (runs / cl * TPA) % 32 == 0 && (long long)a.n_problems * cl <= a.n_sm) return cl;
    return 1;
}

template <int NT, int F, int TPA, int CL>
cudaError_t launch_tuned_cluster(const SolveArgs& a, int runs, cudaStream_t s) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(a.n_problems * CL));
    cfg.blockDim = dim3((unsigned)(runs / CL * TPA));
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cac_solve_tuned_kernel<NT, F, TPA, true, false, false, false, CL>, a);
}

// A TPA-threads-per-anneal shape, as a cluster per problem when few problems leave SMs idle.
template <int NT, int F, int TPA>
cudaError_t launch_tuned_latency(const SolveArgs& a, int runs, cudaStream_t s) {
    const int cl = tuned_cluster_size<TPA>(a, runs);
    if (cl == 4) return launch_tuned_cluster<NT, F, TPA, 4>(a, runs, s);
    if (cl == 2) return launch_tuned_cluster<NT, F, TPA, 2>(a, runs, s);
    cac_solve_tuned_kernel<NT, F, TPA, true><<<a.n_problems, TPA * runs, 0, s>>>(a);
    return cudaGetLastError();
}

// Tuned kernels exist for n_t in {4, 8, 16} and f_mvm in {1, 2}.
__host__ __device__ constexpr bool tuned_size(int NT) { return NT == 4 || NT == 8 || NT == 16; }

// Shape 8: CTAs of 128 anneals.  The CTAs resident on an SM share its 512
// TMEM columns, so shared memory is padded where needed to keep at most
// 512 / ncols of them on one SM (registers already allow fewer here).
template <int NT, int F>
cudaError_t launch_umma(const SolveArgs& a, int runs, cudaStream_t s) {
    const int pp = 128 / runs;
    const int N = pp * 2 * NT;
    const int ncols = N < 32 ? 32 : N;
    const int max_ctas = 512 / ncols;
    int dev = 0, smem_sm = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (err != cudaSuccess) return err;
    size_t smem = (size_t)UmmaSmem<NT>(pp).bytes();
    const size_t floor_bytes = (size_t)smem_sm / (size_t)(max_ctas + 1) + 1;  // (max_ctas + 1) CTAs no longer fit
    if (smem < floor_bytes) smem = (floor_bytes + 127) & ~(size_t)127;
    err = ensure_dynamic_smem<cac_solve_umma_kernel<NT, F>>(smem);
    if (err != cudaSuccess) return err;
    const int blocks = (a.n_problems + pp - 1) / pp;
    cac_solve_umma_kernel<NT, F><<<blocks, 128, smem, s>>>(a, runs);
    return cudaGetLastError();
}

// The bit-identical tuned shapes with early exit (SolveArgs::early_exit > 0).
template <int NT, int F>
cudaError_t launch_tuned_early_exit(const SolveArgs& a, int runs, int variant, cudaStream_t s) {
    switch (variant) {
    case kVariantTpa1: cac_solve_tuned_kernel<NT, F, 1, false, false, false, true><<<a.n_problems, runs, 0, s>>>(a); break;
    case kVariantTpa1Packed:
        cac_solve_tuned_kernel<NT, F, 1, true, false, false, true><<<a.n_problems, runs, 0, s>>>(a);
        break;
    case kVariantTpa2Packed:
        cac_solve_tuned_kernel<NT, F, 2, true, false, false, true><<<a.n_problems, 2 * runs, 0, s>>>(a);
        break;
    case kVariantTpa4Packed:
        if constexpr (NT >= 8) cac_solve_tuned_kernel<NT, F, 4, true, false, false, true><<<a.n_problems, 4 * runs, 0, s>>>(a);
        else cac_solve_tuned_kernel<NT, F, 2, true, false, false, true><<<a.n_problems, 2 * runs, 0, s>>>(a);
        break;
    case kVariantTpa8Packed:
        if constexpr (NT >= 16) cac_solve_tuned_kernel<NT, F, 8, true, false, false, true><<<a.n_problems, 8 * runs, 0, s>>>(a);
        else cac_solve_tuned_kernel<NT, F, 2, true, false, false, true><<<a.n_problems, 2 * runs, 0, s>>>(a);
        break;
    case kVariantPairPacked:
        cac_solve_tuned_kernel<NT, F, 1, true, false, true, true><<<a.n_problems, runs, 0, s>>>(a);
        break;
    case kVariantTensorCore:
    case kVariantTensorCore2:
    case kVariantUmma: return cudaErrorNotSupported;  // (the entry points refuse this combination first)
    default: cac_solve_kernel<NT, F><<<a.n_problems, runs, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

template <int NT, int F>
cudaError_t launch_tuned(const SolveArgs& a, int runs, int variant, cudaStream_t s) {
    if constexpr (tuned_size(NT)) {
        if (a.early_exit > 0) return launch_tuned_early_exit<NT, F>(a, runs, variant, s);
        if (a.steps_out && variant != kVariantPlain) {  // (the tuned kernels without early exit leave it)
            fill_steps_kernel<<<(a.n_problems + 255) / 256, 256, 0, s>>>(a.steps_out, a.n_problems, a.steps);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        switch (variant) {
        case kVariantTpa1: cac_solve_tuned_kernel<NT, F, 1, false><<<a.n_problems, runs, 0, s>>>(a); break;
        case kVariantTpa1Packed: cac_solve_tuned_kernel<NT, F, 1, true><<<a.n_problems, runs, 0, s>>>(a); break;
        case kVariantTpa2Packed: cac_solve_tuned_kernel<NT, F, 2, true><<<a.n_problems, 2 * runs, 0, s>>>(a); break;
        case kVariantTpa4Packed:  // (smaller sizes are resolved to shape 4 before launch)
            if constexpr (NT >= 8) return launch_tuned_latency<NT, F, 4>(a, runs, s);
            else cac_solve_tuned_kernel<NT, F, 2, true><<<a.n_problems, 2 * runs, 0, s>>>(a);
            break;
        case kVariantTpa8Packed:
            if constexpr (NT >= 16) return launch_tuned_latency<NT, F, 8>(a, runs, s);
            else cac_solve_tuned_kernel<NT, F, 2, true><<<a.n_problems, 2 * runs, 0, s>>>(a);
            break;
        case kVariantPairPacked:
            cac_solve_tuned_kernel<NT, F, 1, true, false, true><<<a.n_problems, runs, 0, s>>>(a);
            break;
        case kVariantUmma:
            if constexpr (NT % 8 == 0) {
                if (runs != 96) return launch_umma<NT, F>(a, runs, s);
            }
            [[fallthrough]];  // 96 anneals do not tile the 128 rows: shape 5
        case kVariantTensorCore:
            if constexpr (NT % 8 == 0) {
                cac_solve_tuned_kernel<NT, F, 1, true, true>
                    <<<a.n_problems, runs, (size_t)(runs / 32) * TcShape<NT>::warp_words(32) * 4, s>>>(a);
                break;
            }
            [[fallthrough]];
        case kVariantTensorCore2:
            if constexpr (NT % 8 == 0) {
                cac_solve_tuned_kernel<NT, F, 2, true, true>
                    <<<a.n_problems, 2 * runs, (size_t)(2 * runs / 32) * TcShape<NT>::warp_words(16) * 4, s>>>(a);
                break;
            }
            [[fallthrough]];
        default: cac_solve_kernel<NT, F><<<a.n_problems, runs, 0, s>>>(a); break;
        }
    } else {
        cac_solve_kernel<NT, F><<<a.n_problems, runs, 0, s>>>(a);
    }
    return cudaGetLastError();
}

// 32 users, few problems: a cluster of CL CTAs of 32 anneals per problem.
template <int F, int CL>
cudaError_t launch_rows_cluster(const SolveArgs& a, cudaStream_t s) {
    const size_t smem = rows_dyn_bytes(64, 32);
    cudaError_t err = ensure_dynamic_smem<cac_solve_rows_kernel<32, F, CL>>(smem);
    if (err != cudaSuccess) return err;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(a.n_problems * CL));
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cac_solve_rows_kernel<32, F, CL>, a);
}

template <int NT>
cudaError_t launch_solve_impl(const SolveArgs& a, int runs, cudaStream_t s) {
    if (a.n_problems <= 0) return cudaSuccess;
    if constexpr (NT == 32) {
        // 32 users (n = 64): the row-block kernel (two anneals x 8 rows per thread, four warps per 32
        // anneals); f_mvm 1 and 2 compiled in, others at run time; no spin dump (129 spins do not fit
        // the 128-bit state words, and the API refuses it)
        if (a.spins_out || a.early_exit || a.f_mvm < 1 || runs % 32 != 0) return cudaErrorInvalidValue;
        if (a.steps_out) {  // (every anneal takes all steps here)
            fill_steps_kernel<<<(a.n_problems + 255) / 256, 256, 0, s>>>(a.steps_out, a.n_problems, a.steps);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        // latency: when the problems' 32-anneal groups fit the SMs, each problem is a cluster of
        // runs / 32 CTAs (same results: anneal indices and the arg-min key are the problem's)
        const int cl = runs / 32;
        if (cl > 1 && (a.f_mvm == 1 || a.f_mvm == 2) && a.n_sm > 0 && (long long)a.n_problems * cl <= a.n_sm) {
            if (cl == 2) return a.f_mvm == 2 ? launch_rows_cluster<2, 2>(a, s) : launch_rows_cluster<1, 2>(a, s);
            if (cl == 3) return a.f_mvm == 2 ? launch_rows_cluster<2, 3>(a, s) : launch_rows_cluster<1, 3>(a, s);
            return a.f_mvm == 2 ? launch_rows_cluster<2, 4>(a, s) : launch_rows_cluster<1, 4>(a, s);
        }
        const size_t smem = rows_dyn_bytes(2 * NT, runs);
        cudaError_t err;
        if (a.f_mvm == 2) {
            if ((err = ensure_dynamic_smem<cac_solve_rows_kernel<32, 2>>(smem)) != cudaSuccess) return err;
            cac_solve_rows_kernel<32, 2><<<a.n_problems, 4 * runs, smem, s>>>(a);
        } else if (a.f_mvm == 1) {
            if ((err = ensure_dynamic_smem<cac_solve_rows_kernel<32, 1>>(smem)) != cudaSuccess) return err;
            cac_solve_rows_kernel<32, 1><<<a.n_problems, 4 * runs, smem, s>>>(a);
        } else {
            if ((err = ensure_dynamic_smem<cac_solve_rows_kernel<32, 0>>(smem)) != cudaSuccess) return err;
            cac_solve_rows_kernel<32, 0><<<a.n_problems, 4 * runs, smem, s>>>(a);
        }
        return cudaGetLastError();
    } else {
        const int v = a.spins_out ? (int)kVariantPlain : resolve_variant(NT, a.f_mvm, a.variant, a.n_problems, a.n_sm);
        if (a.f_mvm == 2) return launch_tuned<NT, 2>(a, runs, v, s);
        if (a.f_mvm == 1) return launch_tuned<NT, 1>(a, runs, v, s);
        cac_solve_kernel<NT, 0><<<a.n_problems, runs, 0, s>>>(a);
        return cudaGetLastError();
    }
}

template <int NT>
cudaError_t launch_vpp_inverse_impl(const VppInvArgs& a, cudaStream_t s) {
    if (a.n_chan <= 0) return cudaSuccess;
    const size_t smem = (size_t)(2 * NT * a.n_t + 8 * NT * NT) * sizeof(double);
    cudaError_t err = ensure_dynamic_smem<vpp_inverse_kernel<NT>>(smem);
    if (err != cudaSuccess) return err;
    vpp_inverse_kernel<NT><<<a.n_chan, 32, smem, s>>>(a);
    return cudaGetLastError();
}

template <int NT>
cudaError_t launch_vpp_build_impl(const VppBuildArgs& a, cudaStream_t s) {
    if (a.n_problems <= 0) return cudaSuccess;
    vpp_build_kernel<NT><<<(a.n_problems + 3) / 4, 128, 0, s>>>(a);
    return cudaGetLastError();
}

template <int NT>
cudaError_t launch_vpp_output_impl(const VppOutArgs& a, cudaStream_t s) {
    if (a.n_problems <= 0) return cudaSuccess;
    vpp_output_kernel<NT><<<(a.n_problems + 3) / 4, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mmgap
