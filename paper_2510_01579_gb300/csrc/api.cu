// C-ABI front end of the MMGaP hot path: argument checking, workspace
// chunking, size dispatch and per-stage timing.  All arithmetic of the path
// runs in the kernels of the csrc/*.cuh headers (listed in kernels.cuh).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mmgap.h"
#include "internal.h"
#include "kernels.cuh"

using namespace mmgap;

struct mmgap_ctx {
    int device = 0;
    char* ws = nullptr;         // device workspace
    size_t ws_bytes = 0;
    int* dev_err = nullptr;     // device error word
    std::string err;
    bool timing = false;
    std::vector<cudaEvent_t> events;  // 4 per chunk: start, built, solved, output
    int n_chunks = 0;
    int variant[33] = {};             // solver launch shape per n_t (0 = default)
    int n_sm = 0;                     // SMs of the device
    unsigned long long wait_ns = kDefaultDeviceWaitNs;  // limit of the bounded device waits
};

namespace mmgap {
__global__ void random_ising_kernel(int16_t* Aq, int16_t* hq, int n, int n_problems, uint32_t k0, uint32_t k1) {
    const long long total = (long long)n_problems * n * (n + 1);
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(idx / (n * (n + 1)));
        const int r = (int)(idx % (n * (n + 1)));
        const U4 w = philox4x32_10(U4{(uint32_t)r, (uint32_t)p, 0x7u, 0u}, k0, k1);
        const int16_t v = (int16_t)((int)(w.x % 32769u) - 16384);
        if (r < n * n) {
            const int i = r / n, j = r % n;
            if (i <= j) {
                Aq[(size_t)p * n * n + i * n + j] = v;
                Aq[(size_t)p * n * n + j * n + i] = v;
            }
        } else {
            hq[(size_t)p * n + (r - n * n)] = v;
        }
    }
}
cudaError_t launch_random_ising(int16_t* Aq, int16_t* hq, int n, int n_problems, uint64_t seed, cudaStream_t s) {
    random_ising_kernel<<<1024, 256, 0, s>>>(Aq, hq, n, n_problems, (uint32_t)seed, (uint32_t)(seed >> 32));
    return cudaGetLastError();
}
}  // namespace mmgap

// Constants of the Euler discretisation of Eqs. 10-11, each computed in
// double from the float parameters and rounded once to float.
EulerConsts mmgap::euler_consts(float dt_f, float p_f, float a_f, float zeta_f, float eps_f, float sigma0,
                                float x_max) {
    const double dt = dt_f, p = p_f, a = a_f, zeta = zeta_f, eps = eps_f;
    EulerConsts k;
    k.c1 = (float)(1.0 + dt * (p - 1.0));
    k.cdt = (float)(-dt);
    k.cz = (float)(-(dt * zeta));
    k.c2 = (float)(1.0 + (dt * zeta) * a);
    k.ce = (float)(eps * dt);
    k.xs = (float)((double)sigma0 * 0x1p-23);
    k.x_max = x_max;
    return k;
}

void mmgap::qam_kappa(int mod_bits, float* kappa, float* kappa2) {
    const double M = (double)(1 << mod_bits);
    *kappa = (float)(1.0 / std::sqrt(2.0 * (M - 1.0) / 3.0));
    *kappa2 = (float)(1.0 / (2.0 * (M - 1.0) / 3.0));
}

int mmgap::resolve_variant(int n_t, int f_mvm, int requested, int n_problems, int n_sm) {
    const bool tuned = (n_t == 4 || n_t == 8 || n_t == 16) && (f_mvm == 1 || f_mvm == 2);
    if (!tuned) return kVariantPlain;
    if (requested <= kVariantAuto || requested >= kVariantCount) {
        // Measured on GB300 (detect of P problems, 32 x 200 anneals): up to one problem per SM,
        // 8 (16 users) or 4 (8 users) threads per anneal are 1.5x faster than the throughput
        // shapes; up to two per SM, two threads per anneal; beyond that the throughput shapes.
        if (n_problems >= 0 && n_sm > 0 && n_t >= 8) {
            if (n_problems <= n_sm) return n_t == 16 ? kVariantTpa8Packed : kVariantTpa4Packed;
            if (n_problems <= 2 * n_sm) return kVariantTpa2Packed;
        }
        return n_t == 16 ? kVariantPairPacked : kVariantTpa1Packed;  // the measured fastest for large calls
    }
    if (variant_tensor_core(requested) && n_t == 4) return kVariantTpa1Packed;
    // more threads per anneal need at least 4 rows (one float4 of couplings) per thread
    if (requested == kVariantTpa8Packed && n_t < 16) return n_t == 8 ? kVariantTpa4Packed : kVariantTpa2Packed;
    if (requested == kVariantTpa4Packed && n_t < 8) return kVariantTpa2Packed;
    return requested;
}

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

mmgap_status fail(mmgap_ctx* ctx, mmgap_status st, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
mmgap_status fail(mmgap_ctx* ctx, mmgap_status st, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

mmgap_status cuda_fail(mmgap_ctx* ctx, cudaError_t e, const char* what) {
    return fail(ctx, MMGAP_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool nt_supported(int nt) { return nt == 1 || nt == 2 || nt == 3 || nt == 4 || nt == 8 || nt == 16; }

EulerConsts euler_consts(const mmgap_params& P) {
    return mmgap::euler_consts(P.dt, P.p, P.a, P.zeta, P.eps, P.sigma0, P.x_max);
}

mmgap_status check_params(mmgap_ctx* ctx, const mmgap_params* P) {
    if (!P) return fail(ctx, MMGAP_EINVAL, "params is NULL");
    if (!(P->runs == 32 || P->runs == 64 || P->runs == 96 || P->runs == 128))
        return fail(ctx, MMGAP_EUNSUPPORTED, "runs=%d: supported 32, 64, 96, 128", P->runs);
    if (P->steps < 0 || P->steps > (1 << 20)) return fail(ctx, MMGAP_EINVAL, "steps=%d out of [0, 2^20]", P->steps);
    if (P->f_mvm < 1 || P->f_mvm > 64) return fail(ctx, MMGAP_EINVAL, "f_mvm=%d out of [1, 64]", P->f_mvm);
    if (!(P->dt > 0.0f) || !std::isfinite(P->dt)) return fail(ctx, MMGAP_EINVAL, "dt must be positive and finite");
    if (!std::isfinite(P->p) || !std::isfinite(P->a) || !std::isfinite(P->zeta) || !std::isfinite(P->eps) ||
        !std::isfinite(P->sigma0) || !(P->x_max > 0.0f))
        return fail(ctx, MMGAP_EINVAL, "non-finite solver parameter or x_max <= 0");
    if (P->early_exit < 0) return fail(ctx, MMGAP_EINVAL, "early_exit=%d must be >= 0", P->early_exit);
    return MMGAP_OK;
}

// Early exit runs on the bit-identical solver shapes up to 16 users.
mmgap_status check_early_exit(mmgap_ctx* ctx, const mmgap_params* P, int n_t) {
    if (P->early_exit == 0) return MMGAP_OK;
    if (n_t > 16) return fail(ctx, MMGAP_EUNSUPPORTED, "early exit: up to 16 users");
    if (variant_tensor_core(resolve_variant(n_t, P->f_mvm, ctx->variant[n_t])))
        return fail(ctx, MMGAP_EUNSUPPORTED, "early exit runs on the bit-identical solver shapes, not 5, 7 or 8");
    return MMGAP_OK;
}

// Operations that also exist for 32 users (delta-mapping detection and the solver only).
template <template <int> class Op> struct Has32 { static constexpr bool value = false; };

template <template <int> class Op, class... Args>
cudaError_t dispatch_nt(int nt, Args&&... args) {
    switch (nt) {
    case 1: return Op<1>::run(args...);
    case 2: return Op<2>::run(args...);
    case 3: return Op<3>::run(args...);
    case 4: return Op<4>::run(args...);
    case 8: return Op<8>::run(args...);
    case 16: return Op<16>::run(args...);
    case 32:
        if constexpr (Has32<Op>::value) return Op<32>::run(args...);
        else return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

template <int NT> struct OpBuild { static cudaError_t run(const BuildArgs& a, cudaStream_t s) { return launch_build_detect<NT>(a, s); } };
template <int NT> struct OpFactor { static cudaError_t run(const ChanFactorArgs& a, cudaStream_t s) { return launch_chan_factor<NT>(a, s); } };
template <int NT> struct OpSolve { static cudaError_t run(const SolveArgs& a, int r, cudaStream_t s) { return launch_solve<NT>(a, r, s); } };
template <int NT> struct OpVppInv { static cudaError_t run(const VppInvArgs& a, cudaStream_t s) { return launch_vpp_inverse<NT>(a, s); } };
template <int NT> struct OpVppInvIr { static cudaError_t run(const VppInvArgs& a, cudaStream_t s) { return launch_vpp_inverse_ir<NT>(a, s); } };
template <int NT> struct OpVppBuild { static cudaError_t run(const VppBuildArgs& a, cudaStream_t s) { return launch_vpp_build<NT>(a, s); } };
template <int NT> struct OpVppOut { static cudaError_t run(const VppOutArgs& a, cudaStream_t s) { return launch_vpp_output<NT>(a, s); } };
template <int NT> struct OpGram { static cudaError_t run(const GramArgs& a, cudaStream_t s) { return launch_gram_tc<NT>(a, s); } };
template <int NT> struct OpSelect { static cudaError_t run(const SelectArgs& a, cudaStream_t s) { return launch_select<NT>(a, s); } };
template <> struct Has32<OpBuild> { static constexpr bool value = true; };
template <> struct Has32<OpFactor> { static constexpr bool value = true; };
template <> struct Has32<OpSolve> { static constexpr bool value = true; };


struct CurrentDevice {
    int prev = -1;
    explicit CurrentDevice(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~CurrentDevice() {
        int now = -1;
        cudaGetDevice(&now);
        if (prev >= 0 && now != prev) cudaSetDevice(prev);
    }
};

mmgap_status timing_begin(mmgap_ctx* ctx) {
    ctx->n_chunks = 0;
    return MMGAP_OK;
}

// Record stage event `stage` (0..3) of the current chunk.
mmgap_status timing_mark(mmgap_ctx* ctx, int stage, cudaStream_t s) {
    if (!ctx->timing) return MMGAP_OK;
    const size_t idx = (size_t)ctx->n_chunks * 4 + stage;
    while (ctx->events.size() <= idx) {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventCreate");
        ctx->events.push_back(ev);
    }
    cudaError_t e = cudaEventRecord(ctx->events[idx], s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventRecord");
    if (stage == 3) ctx->n_chunks++;
    return MMGAP_OK;
}

mmgap_status check_detect_job(mmgap_ctx* ctx, const mmgap_detect_job& j, bool need_sym) {
    if (!nt_supported(j.n_t) && j.n_t != 32)
        return fail(ctx, MMGAP_EUNSUPPORTED, "n_t=%d: supported 1, 2, 3, 4, 8, 16, 32", j.n_t);
    if (j.n_t == 32 && (j.mapping != MMGAP_MAPPING_DELTA || j.gram_precision != 0))
        return fail(ctx, MMGAP_EUNSUPPORTED, "n_t=32: delta mapping with the FP32 Gram only");
    if (j.n_r < 1 || j.n_r > kMaxNr) return fail(ctx, MMGAP_EUNSUPPORTED, "n_r=%d out of [1, %d]", j.n_r, kMaxNr);
    if (!(j.mod_bits == 2 || j.mod_bits == 4 || j.mod_bits == 6))
        return fail(ctx, MMGAP_EUNSUPPORTED, "mod_bits=%d: supported 2, 4, 6", j.mod_bits);
    if (j.n_problems < 0) return fail(ctx, MMGAP_EINVAL, "n_problems < 0");
    if (j.n_problems == 0) return MMGAP_OK;
    if (!j.H || !j.y || !j.noise_var || (need_sym && !j.sym_out))
        return fail(ctx, MMGAP_EINVAL, "NULL H, y, noise_var or sym_out");
    if (j.n_chan < 1) return fail(ctx, MMGAP_EINVAL, "n_chan < 1");
    if (!j.chan_index && j.n_chan < j.n_problems)
        return fail(ctx, MMGAP_EINVAL, "chan_index NULL needs n_chan >= n_problems");
    if (j.gram_precision < 0 || j.gram_precision > 3)
        return fail(ctx, MMGAP_EINVAL, "gram_precision=%d: 0 FP32, 1 BF16, 2 FP16, 3 BF16x3", j.gram_precision);
    if (j.mapping != MMGAP_MAPPING_DELTA && j.mapping != MMGAP_MAPPING_DIRECT)
        return fail(ctx, MMGAP_EINVAL, "mapping=%d: 0 delta, 1 direct", j.mapping);
    if (j.mapping == MMGAP_MAPPING_DIRECT) {
        if (j.guess_in) return fail(ctx, MMGAP_EUNSUPPORTED, "direct mapping: the guess is the MMSE guess");
        if (j.steps_out) return fail(ctx, MMGAP_EUNSUPPORTED, "direct mapping: no steps_out");
        if (!(j.n_t == 4 || j.n_t == 8 || j.n_t == 16))
            return fail(ctx, MMGAP_EUNSUPPORTED, "direct mapping: n_t=%d, supported 4, 8, 16", j.n_t);
        if (j.gram_precision != 0) return fail(ctx, MMGAP_EUNSUPPORTED, "direct mapping builds the Gram in FP32");
    }
    return MMGAP_OK;
}

int direct_spins(const mmgap_detect_job& j) { return 2 * j.n_t * (j.mod_bits / 2); }

// TPA of the general solver for N spins (as general_tpa<N>()).
int general_threads_per_anneal(int N) { return N <= 32 ? 1 : (N <= 64 ? 2 : 4); }

mmgap_status check_general_runs(mmgap_ctx* ctx, const mmgap_params* params, int N) {
    if (params->runs % 32 || params->runs * general_threads_per_anneal(N) > 256)
        return fail(ctx, MMGAP_EUNSUPPORTED, "general solver with N=%d: runs a multiple of 32, at most %d", N,
                    256 / general_threads_per_anneal(N));
    return MMGAP_OK;
}

cudaError_t dispatch_build_direct(int n_t, const DirectBuildArgs& a, cudaStream_t s) {
    switch (n_t) {
    case 16: return launch_build_direct<16>(a, s);
    case 8: return launch_build_direct<8>(a, s);
    case 4: return launch_build_direct<4>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

// BuildArgs of problems [p0, p0 + P) of a detection job.
BuildArgs job_build_args(mmgap_ctx* ctx, const mmgap_detect_job& J, long long p0, int P) {
    BuildArgs b{};
    b.H = J.chan_index ? J.H : J.H + (size_t)p0 * 2 * J.n_r * J.n_t;
    b.chan_index = J.chan_index ? J.chan_index + p0 : nullptr;
    b.y = J.y + (size_t)p0 * 2 * J.n_r;
    b.noise_var = J.noise_var + p0;
    b.n_r = J.n_r;
    b.mod_bits = J.mod_bits;
    b.n_problems = P;
    b.n_chan = J.chan_index ? J.n_chan : P;
    qam_kappa(J.mod_bits, &b.kappa, &b.kappa2);
    b.err = ctx->dev_err;
    return b;
}

// Direct-mapping detection of one job: per chunk, the direct build (J_q,
// c_q, guess, reference spins) into the workspace, then the general solver
// with the fused decode.
mmgap_status detect_direct_job(mmgap_ctx* ctx, const mmgap_params* params, const mmgap_detect_job& J,
                               const EulerConsts& k, cudaStream_t s) {
    const int N = direct_spins(J), n = 2 * J.n_t;
    mmgap_status st = check_general_runs(ctx, params, N);
    if (st != MMGAP_OK) return st;
    const size_t per = align_up((size_t)N * N * 2) + align_up((size_t)N * 2) + align_up((size_t)n) +
                       align_up((size_t)N);
    long long chunk = (long long)(ctx->ws_bytes / (per + 4 * kAlign));
    if (chunk < 1) return fail(ctx, MMGAP_ENOMEM, "workspace of %zu bytes holds no problem", ctx->ws_bytes);
    if (chunk > J.n_problems) chunk = J.n_problems;
    for (long long p0 = 0; p0 < J.n_problems; p0 += chunk) {
        const int P = (int)std::min<long long>(chunk, J.n_problems - p0);
        char* base = ctx->ws;
        int16_t* Jq = (int16_t*)base;
        int16_t* cq = (int16_t*)(base + align_up((size_t)P * N * N * 2));
        int8_t* g = (int8_t*)((char*)cq + align_up((size_t)P * N * 2));
        int8_t* sref = (int8_t*)((char*)g + align_up((size_t)P * n));
        if ((st = timing_mark(ctx, 0, s)) != MMGAP_OK) return st;
        DirectBuildArgs d{};
        d.b = job_build_args(ctx, J, p0, P);
        d.b.g = J.guess_out ? J.guess_out + (size_t)p0 * n : g;
        d.B = J.mod_bits / 2;
        d.Jq = Jq;
        d.cq = cq;
        d.s_ref = sref;
        cudaError_t e = dispatch_build_direct(J.n_t, d, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "build_direct launch");
        if ((st = timing_mark(ctx, 1, s)) != MMGAP_OK) return st;
        GeneralArgs a{};
        a.Jq = Jq;
        a.cq = cq;
        a.s_ref = sref;
        a.n_problems = P;
        a.steps = params->steps;
        a.f_mvm = params->f_mvm;
        a.key0 = (uint32_t)J.seed;
        a.key1 = (uint32_t)(J.seed >> 32);
        a.problem_offset = J.problem_offset + (uint64_t)p0;
        a.k = k;
        a.E_out = J.energy_out ? J.energy_out + p0 : nullptr;
        a.ndiv_out = J.ndiv_out ? J.ndiv_out + p0 : nullptr;
        a.mod_bits = J.mod_bits;
        a.sym_out = J.sym_out + (size_t)p0 * J.n_t;
        a.g = d.b.g;
        a.offset_out = J.offset_out ? J.offset_out + (size_t)p0 * n : nullptr;
        e = launch_solve_general(N, a, params->runs, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cac_general launch");
        if ((st = timing_mark(ctx, 2, s)) != MMGAP_OK) return st;
        if ((st = timing_mark(ctx, 3, s)) != MMGAP_OK) return st;
    }
    return MMGAP_OK;
}

// Tensor-core Gram of every channel of a job into the workspace head (for
// gram_precision 1/2); *gc_out = nullptr for the FP32 path.
mmgap_status job_gram(mmgap_ctx* ctx, const mmgap_detect_job& J, cudaStream_t s, float** gc_out, size_t* used) {
    *gc_out = nullptr;
    *used = 0;
    if (J.gram_precision == 0 || J.n_problems == 0) return MMGAP_OK;
    const int n_chan = J.chan_index ? J.n_chan : J.n_problems;
    const size_t bytes = align_up((size_t)n_chan * J.n_t * J.n_t * 8);
    if (bytes + 4 * kAlign >= ctx->ws_bytes) return fail(ctx, MMGAP_ENOMEM, "workspace too small for the Gram");
    GramArgs g{};
    g.H = J.H;
    g.n_r = J.n_r;
    g.n_chan = n_chan;
    float k2;
    qam_kappa(J.mod_bits, &g.kappa, &k2);
    g.fp16 = J.gram_precision == 2 ? 1 : (J.gram_precision == 3 ? 2 : 0);
    g.Gc = (float*)ctx->ws;
    cudaError_t e = dispatch_nt<OpGram>(J.n_t, g, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gram_tc launch");
    *gc_out = g.Gc;
    *used = bytes;
    return MMGAP_OK;
}

mmgap_status check_precode_job(mmgap_ctx* ctx, const mmgap_precode_job& j) {
    if (!nt_supported(j.n_u)) return fail(ctx, MMGAP_EUNSUPPORTED, "n_u=%d: supported 1, 2, 3, 4, 8, 16", j.n_u);
    if (j.n_t < j.n_u || j.n_t > kMaxNr)
        return fail(ctx, MMGAP_EUNSUPPORTED, "n_t=%d out of [n_u, %d]", j.n_t, kMaxNr);
    if (!(j.mod_bits == 2 || j.mod_bits == 4 || j.mod_bits == 6))
        return fail(ctx, MMGAP_EUNSUPPORTED, "mod_bits=%d: supported 2, 4, 6", j.mod_bits);
    if (j.n_problems < 0) return fail(ctx, MMGAP_EINVAL, "n_problems < 0");
    if (j.n_problems == 0) return MMGAP_OK;
    if (!j.H || !j.u_sym || !j.v_out) return fail(ctx, MMGAP_EINVAL, "NULL H, u_sym or v_out");
    if (j.n_chan < 1) return fail(ctx, MMGAP_EINVAL, "n_chan < 1");
    if (!j.chan_index && j.n_chan < j.n_problems)
        return fail(ctx, MMGAP_EINVAL, "chan_index NULL needs n_chan >= n_problems");
    if ((uintptr_t)j.H % 8) return fail(ctx, MMGAP_EINVAL, "H must be 8-byte aligned");
    if (j.inv_precision != MMGAP_INV_FP64 && j.inv_precision != MMGAP_INV_FP32_IR)
        return fail(ctx, MMGAP_EINVAL, "inv_precision=%d: 0 (FP64) or 1 (FP32 + refinement)", j.inv_precision);
    return MMGAP_OK;
}

}  // namespace

namespace mmgap {

cudaError_t vpp_inverse_any(int n_u, int n_t, int n_chan, const float* H, int inv_precision, double* Q,
                            int32_t* status, cudaStream_t s) {
    VppInvArgs vi{};
    vi.H = H;
    vi.n_t = n_t;
    vi.n_chan = n_chan;
    vi.Q = Q;
    vi.status = status;
    vi.refine = kVppRefineSteps;
    if (inv_precision == MMGAP_INV_FP64) return dispatch_nt<OpVppInv>(n_u, vi, s);
    cudaError_t e = dispatch_nt<OpVppInvIr>(n_u, vi, s);
    if (e != cudaSuccess) return e;
    vi.only_failed = 1;
    return dispatch_nt<OpVppInv>(n_u, vi, s);
}

}  // namespace mmgap

extern "C" {

mmgap_status mmgap_default_params(mmgap_params* p) {
    if (!p) return MMGAP_EINVAL;
    p->runs = 32;
    p->steps = 200;
    p->f_mvm = 2;
    p->dt = 0.02f;
    p->p = 1.2f;
    p->a = 1.0f;
    p->zeta = 3.0f;
    p->eps = 0.5f;
    p->sigma0 = 0.1f;
    p->x_max = 1000.0f;
    p->early_exit = 0;
    return MMGAP_OK;
}

mmgap_status mmgap_create(mmgap_ctx** out, int device, size_t workspace_bytes) {
    if (!out) return MMGAP_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return MMGAP_EINVAL;
    auto* ctx = new (std::nothrow) mmgap_ctx();
    if (!ctx) return MMGAP_ENOMEM;
    ctx->device = device;
    CurrentDevice cd(device);
    if (cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        ctx->n_sm = 0;  // unknown: the throughput shapes for every call
    }
    ctx->ws_bytes = workspace_bytes ? workspace_bytes : ((size_t)256 << 20);
    if (cudaMalloc(&ctx->ws, ctx->ws_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return MMGAP_ENOMEM;
    }
    if (cudaMalloc(&ctx->dev_err, 256) != cudaSuccess || cudaMemset(ctx->dev_err, 0, 256) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(ctx->ws);
        delete ctx;
        return MMGAP_ENOMEM;
    }
    *out = ctx;
    return MMGAP_OK;
}

mmgap_status mmgap_destroy(mmgap_ctx* ctx) {
    if (!ctx) return MMGAP_OK;
    CurrentDevice cd(ctx->device);
    cudaDeviceSynchronize();
    for (auto ev : ctx->events) cudaEventDestroy(ev);
    cudaFree(ctx->ws);
    cudaFree(ctx->dev_err);
    delete ctx;
    return MMGAP_OK;
}

const char* mmgap_last_error(const mmgap_ctx* ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

mmgap_status mmgap_set_timing(mmgap_ctx* ctx, int enable) {
    if (!ctx) return MMGAP_EINVAL;
    ctx->timing = enable != 0;
    return MMGAP_OK;
}

mmgap_status mmgap_stage_times(mmgap_ctx* ctx, float ms_out[4], int* n_chunks_out) {
    if (!ctx || !ms_out) return MMGAP_EINVAL;
    for (int i = 0; i < 4; ++i) ms_out[i] = 0.0f;
    if (n_chunks_out) *n_chunks_out = ctx->n_chunks;
    if (ctx->n_chunks == 0) return MMGAP_OK;
    CurrentDevice cd(ctx->device);
    const int last = ctx->n_chunks * 4 - 1;
    cudaError_t e = cudaEventSynchronize(ctx->events[last]);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventSynchronize");
    for (int c = 0; c < ctx->n_chunks; ++c) {
        for (int s = 0; s < 3; ++s) {
            float ms = 0.0f;
            e = cudaEventElapsedTime(&ms, ctx->events[c * 4 + s], ctx->events[c * 4 + s + 1]);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventElapsedTime");
            ms_out[s] += ms;
        }
    }
    float all = 0.0f;
    e = cudaEventElapsedTime(&all, ctx->events[0], ctx->events[last]);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventElapsedTime");
    ms_out[3] = all;
    return MMGAP_OK;
}

mmgap_status mmgap_device_errors(mmgap_ctx* ctx, int* flags_out, int clear) {
    if (!ctx || !flags_out) return MMGAP_EINVAL;
    CurrentDevice cd(ctx->device);
    cudaError_t e = cudaMemcpy(flags_out, ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reading the device error word");
    if (clear) {
        e = cudaMemset(ctx->dev_err, 0, sizeof(int));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "clearing the device error word");
    }
    return MMGAP_OK;
}

mmgap_status mmgap_build_detect(mmgap_ctx* ctx, const mmgap_detect_job* job, int16_t* A_q_out, int16_t* h_q_out,
                                int8_t* g_out, float* G_out, float* h_out, int32_t* sigma_exp_out, void* stream) {
    NvtxRange nvtx_range("mmgap_build_detect");
    if (!ctx) return MMGAP_EINVAL;
    if (!job) return fail(ctx, MMGAP_EINVAL, "job is NULL");
    mmgap_status st = check_detect_job(ctx, *job, false);
    if (st != MMGAP_OK) return st;
    if (job->n_problems == 0) return MMGAP_OK;
    if (!A_q_out || !h_q_out || !g_out) return fail(ctx, MMGAP_EINVAL, "NULL A_q_out, h_q_out or g_out");
    CurrentDevice cd(ctx->device);
    if (job->mapping == MMGAP_MAPPING_DIRECT) {
        DirectBuildArgs d{};
        d.b = job_build_args(ctx, *job, 0, job->n_problems);
        d.b.n_chan = job->n_chan;
        d.b.g = g_out;
        d.B = job->mod_bits / 2;
        d.Jq = A_q_out;
        d.cq = h_q_out;
        d.J32 = G_out;
        d.c32 = h_out;
        d.sigma_exp = sigma_exp_out;
        cudaError_t e = dispatch_build_direct(job->n_t, d, (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "build_direct launch");
        return MMGAP_OK;
    }
    BuildArgs a{};
    a.H = job->H;
    a.chan_index = job->chan_index;
    a.y = job->y;
    a.noise_var = job->noise_var;
    a.n_r = job->n_r;
    a.mod_bits = job->mod_bits;
    a.n_problems = job->n_problems;
    a.n_chan = job->n_chan;
    qam_kappa(job->mod_bits, &a.kappa, &a.kappa2);
    a.err = ctx->dev_err;
    a.guess_mode = job->guess_in ? 2 : 0;
    a.g_in = job->guess_in;
    a.Aq = A_q_out;
    a.hq = h_q_out;
    a.g = g_out;
    a.G32 = G_out;
    a.h32 = h_out;
    a.sigma_exp = sigma_exp_out;
    float* gc = nullptr;
    size_t used = 0;
    if ((st = job_gram(ctx, *job, (cudaStream_t)stream, &gc, &used)) != MMGAP_OK) return st;
    a.Gc_pre = gc;
    cudaError_t e = dispatch_nt<OpBuild>(job->n_t, a, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "build_detect launch");
    return MMGAP_OK;
}

mmgap_status mmgap_solve_ising(mmgap_ctx* ctx, const mmgap_params* params, int n, int n_problems, const int16_t* A_q,
                               const int16_t* h_q, const int8_t* g, int level_max, uint64_t seed, int8_t* d_out,
                               int32_t* E_out, int32_t* run_out, int32_t* ndiv_out, void* stream) {
    NvtxRange nvtx_range("mmgap_solve_ising");
    if (!ctx) return MMGAP_EINVAL;
    mmgap_status st = check_params(ctx, params);
    if (st != MMGAP_OK) return st;
    if (n < 2 || (n & 1) || (!nt_supported(n / 2) && n != 64))
        return fail(ctx, MMGAP_EUNSUPPORTED, "n=%d: supported 2, 4, 6, 8, 16, 32, 64", n);
    if (n_problems < 0) return fail(ctx, MMGAP_EINVAL, "n_problems < 0");
    if (n_problems == 0) return MMGAP_OK;
    if (!A_q || !h_q || !d_out) return fail(ctx, MMGAP_EINVAL, "NULL A_q, h_q or d_out");
    if (level_max < 0 || (level_max > 0 && !g)) return fail(ctx, MMGAP_EINVAL, "level_max needs g");
    if ((st = check_early_exit(ctx, params, n / 2)) != MMGAP_OK) return st;
    CurrentDevice cd(ctx->device);
    SolveArgs a{};
    a.err = ctx->dev_err;
    a.n_sm = ctx->n_sm;
    a.Aq = A_q;
    a.hq = h_q;
    a.g = g;
    a.level_max = level_max;
    a.n_problems = n_problems;
    a.steps = params->steps;
    a.f_mvm = params->f_mvm;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.problem_offset = 0;
    a.k = euler_consts(*params);
    a.d_out = d_out;
    a.E_out = E_out;
    a.run_out = run_out;
    a.ndiv_out = ndiv_out;
    a.early_exit = params->early_exit;
    a.wait_ns = ctx->wait_ns;
    a.variant = ctx->variant[n / 2];
    cudaError_t e = dispatch_nt<OpSolve>(n / 2, a, params->runs, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cac_solve launch");
    return MMGAP_OK;
}

mmgap_status mmgap_solve_general(mmgap_ctx* ctx, const mmgap_params* params, int N, int n_problems,
                                 const int16_t* J_q, const int16_t* c_q, const int8_t* s_ref, uint64_t seed,
                                 int8_t* s_out, int32_t* E_out, int32_t* run_out, int32_t* ndiv_out, void* stream) {
    NvtxRange nvtx_range("mmgap_solve_general");
    if (!ctx) return MMGAP_EINVAL;
    mmgap_status st = check_params(ctx, params);
    if (st != MMGAP_OK) return st;
    if (!general_supported(N)) return fail(ctx, MMGAP_EUNSUPPORTED, "N=%d: supported 8, 16, 24, 32, 48, 64, 96", N);
    if (params->early_exit) return fail(ctx, MMGAP_EUNSUPPORTED, "the general solver has no early exit");
    if ((st = check_general_runs(ctx, params, N)) != MMGAP_OK) return st;
    if (n_problems < 0) return fail(ctx, MMGAP_EINVAL, "n_problems < 0");
    if (n_problems == 0) return MMGAP_OK;
    if (!J_q || !c_q || !s_out) return fail(ctx, MMGAP_EINVAL, "NULL J_q, c_q or s_out");
    CurrentDevice cd(ctx->device);
    GeneralArgs a{};
    a.Jq = J_q;
    a.cq = c_q;
    a.s_ref = s_ref;
    a.n_problems = n_problems;
    a.steps = params->steps;
    a.f_mvm = params->f_mvm;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.k = euler_consts(*params);
    a.s_out = s_out;
    a.E_out = E_out;
    a.run_out = run_out;
    a.ndiv_out = ndiv_out;
    cudaError_t e = launch_solve_general(N, a, params->runs, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cac_general launch");
    return MMGAP_OK;
}

mmgap_status mmgap_detect(mmgap_ctx* ctx, const mmgap_params* params, const mmgap_detect_job* jobs, int n_jobs,
                          void* stream) {
    NvtxRange nvtx_range("mmgap_detect");
    if (!ctx) return MMGAP_EINVAL;
    mmgap_status st = check_params(ctx, params);
    if (st != MMGAP_OK) return st;
    if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return fail(ctx, MMGAP_EINVAL, "bad jobs array");
    for (int j = 0; j < n_jobs; ++j) {
        if ((st = check_detect_job(ctx, jobs[j], true)) != MMGAP_OK) return st;
        if (jobs[j].mapping == MMGAP_MAPPING_DIRECT && params->early_exit)
            return fail(ctx, MMGAP_EUNSUPPORTED, "the direct mapping has no early exit");
        if ((st = check_early_exit(ctx, params, jobs[j].n_t)) != MMGAP_OK) return st;
    }
    CurrentDevice cd(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const EulerConsts k = euler_consts(*params);
    timing_begin(ctx);
    for (int j = 0; j < n_jobs; ++j) {
        const mmgap_detect_job& J = jobs[j];
        if (J.n_problems == 0) continue;
        if (J.mapping == MMGAP_MAPPING_DIRECT) {
            if ((st = detect_direct_job(ctx, params, J, k, s)) != MMGAP_OK) return st;
            continue;
        }
        const int n = 2 * J.n_t;
        const size_t per = align_up((size_t)n * n * 2) + align_up((size_t)n * 2) + align_up((size_t)n);
        if ((st = timing_mark(ctx, 0, s)) != MMGAP_OK) return st;
        float* gc = nullptr;
        size_t gc_bytes = 0;
        if ((st = job_gram(ctx, J, s, &gc, &gc_bytes)) != MMGAP_OK) return st;
        // Channels that serve several problems (the symbols of a subcarrier, the
        // resource elements of a PRB) are factorised once: the builder of a
        // problem whose rho equals its channel's reads the factor instead of
        // repeating the column-sequential Cholesky (the same bits).  Skipped when
        // the workspace cannot hold the factors and one problem besides.
        size_t fac_bytes = 0;
        const float* L_pre = nullptr;
        const float* rho_pre = nullptr;
        const int32_t* chol_pre = nullptr;
        if (!gc && !J.guess_in && J.chan_index && J.n_chan < J.n_problems) {
            const size_t nc = (size_t)J.n_chan;
            const size_t lb = align_up(nc * 2 * J.n_t * J.n_t * sizeof(float)), rb = align_up(nc * 4);
            if (gc_bytes + 2 * lb + 3 * rb + per + 3 * kAlign <= ctx->ws_bytes) {
                char* fb = ctx->ws + gc_bytes;
                ChanFactorArgs f{};
                f.H = J.H;
                f.chan_index = J.chan_index;
                f.noise_var = J.noise_var;
                f.n_r = J.n_r;
                f.n_problems = J.n_problems;
                f.n_chan = J.n_chan;
                qam_kappa(J.mod_bits, &f.kappa, &f.kappa2);
                f.L_out = (float*)fb;
                f.rho_out = (float*)(fb + lb);
                f.chol_out = (int32_t*)(fb + lb + rb);
                f.first = (int32_t*)(fb + lb + 2 * rb);
                f.G_out = (float*)(fb + lb + 3 * rb);
                cudaError_t e = dispatch_nt<OpFactor>(J.n_t, f, s);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "chan_factor launch");
                L_pre = f.L_out;
                rho_pre = f.rho_out;
                chol_pre = f.chol_out;
                gc = f.G_out;  // each channel's Gram, made once (read by channel index, as the tensor-core Gram)
                fac_bytes = 2 * lb + 3 * rb;
            }
        }
        char* base = ctx->ws + gc_bytes + fac_bytes;
        const size_t avail = ctx->ws_bytes - gc_bytes - fac_bytes;
        // chunk so that three aligned regions of chunk size fit the workspace
        long long chunk = (long long)(avail / (per + 3 * kAlign));
        if (chunk < 1) return fail(ctx, MMGAP_ENOMEM, "workspace of %zu bytes holds no problem", ctx->ws_bytes);
        if (chunk > J.n_problems) chunk = J.n_problems;
        for (long long p0 = 0; p0 < J.n_problems; p0 += chunk) {
            const int P = (int)std::min<long long>(chunk, J.n_problems - p0);
            int16_t* Aq = (int16_t*)base;
            int16_t* hq = (int16_t*)(base + align_up((size_t)P * n * n * 2));
            int8_t* g = (int8_t*)((char*)hq + align_up((size_t)P * n * 2));
            if (p0 > 0 && (st = timing_mark(ctx, 0, s)) != MMGAP_OK) return st;
            BuildArgs b{};
            b.Gc_pre = gc ? (J.chan_index ? gc : gc + (size_t)p0 * 2 * J.n_t * J.n_t) : nullptr;
            b.L_pre = L_pre;
            b.rho_pre = rho_pre;
            b.chol_pre = chol_pre;
            b.H = J.chan_index ? J.H : J.H + (size_t)p0 * 2 * J.n_r * J.n_t;
            b.chan_index = J.chan_index ? J.chan_index + p0 : nullptr;
            b.y = J.y + (size_t)p0 * 2 * J.n_r;
            b.noise_var = J.noise_var + p0;
            b.n_r = J.n_r;
            b.mod_bits = J.mod_bits;
            b.n_problems = P;
            b.n_chan = J.chan_index ? J.n_chan : P;
            qam_kappa(J.mod_bits, &b.kappa, &b.kappa2);
            b.err = ctx->dev_err;
            b.guess_mode = J.guess_in ? 2 : 0;
            b.g_in = J.guess_in ? J.guess_in + (size_t)p0 * n : nullptr;
            b.Aq = Aq;
            b.hq = hq;
            b.g = g;
            cudaError_t e = dispatch_nt<OpBuild>(J.n_t, b, s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "build_detect launch");
            if ((st = timing_mark(ctx, 1, s)) != MMGAP_OK) return st;
            SolveArgs a{};
            a.err = ctx->dev_err;
            a.n_sm = ctx->n_sm;
            a.Aq = Aq;
            a.hq = hq;
            a.g = g;
            a.level_max = (1 << (J.mod_bits >> 1)) - 1;
            a.n_problems = P;
            a.steps = params->steps;
            a.f_mvm = params->f_mvm;
            a.key0 = (uint32_t)J.seed;
            a.key1 = (uint32_t)(J.seed >> 32);
            a.problem_offset = J.problem_offset + (uint64_t)p0;
            a.k = k;
            a.d_out = J.offset_out ? J.offset_out + (size_t)p0 * n : nullptr;
            a.E_out = J.energy_out ? J.energy_out + p0 : nullptr;
            a.run_out = nullptr;
            a.ndiv_out = J.ndiv_out ? J.ndiv_out + p0 : nullptr;
            a.sym_out = J.sym_out + (size_t)p0 * J.n_t;
            a.mod_bits = J.mod_bits;
            a.variant = ctx->variant[J.n_t];
            a.early_exit = params->early_exit;
            a.wait_ns = ctx->wait_ns;
            a.steps_out = J.steps_out ? J.steps_out + p0 : nullptr;
            e = dispatch_nt<OpSolve>(J.n_t, a, params->runs, s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cac_solve launch");
            if (J.guess_out) {
                e = cudaMemcpyAsync(J.guess_out + (size_t)p0 * n, g, (size_t)P * n, cudaMemcpyDeviceToDevice, s);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "guess copy");
            }
            if ((st = timing_mark(ctx, 2, s)) != MMGAP_OK) return st;
            if ((st = timing_mark(ctx, 3, s)) != MMGAP_OK) return st;
        }
    }
    return MMGAP_OK;
}

mmgap_status mmgap_precode(mmgap_ctx* ctx, const mmgap_params* params, const mmgap_precode_job* jobs, int n_jobs,
                           void* stream) {
    NvtxRange nvtx_range("mmgap_precode");
    if (!ctx) return MMGAP_EINVAL;
    mmgap_status st = check_params(ctx, params);
    if (st != MMGAP_OK) return st;
    if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return fail(ctx, MMGAP_EINVAL, "bad jobs array");
    for (int j = 0; j < n_jobs; ++j) {
        if ((st = check_precode_job(ctx, jobs[j])) != MMGAP_OK) return st;
        if ((st = check_early_exit(ctx, params, jobs[j].n_u)) != MMGAP_OK) return st;
    }
    CurrentDevice cd(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const EulerConsts k = euler_consts(*params);
    timing_begin(ctx);
    for (int j = 0; j < n_jobs; ++j) {
        const mmgap_precode_job& J = jobs[j];
        if (J.n_problems == 0) continue;
        const int n = 2 * J.n_u;
        // channels whose inverse this job needs
        const int n_chan = J.chan_index ? J.n_chan : J.n_problems;
        const size_t qbytes = align_up((size_t)n_chan * J.n_u * J.n_u * 16) + align_up((size_t)n_chan * 4);
        const size_t per = align_up((size_t)n * n * 2) + align_up((size_t)n * 2) + align_up((size_t)n);
        if (qbytes + per + 3 * kAlign > ctx->ws_bytes)
            return fail(ctx, MMGAP_ENOMEM, "workspace of %zu bytes too small for %d channel inverses", ctx->ws_bytes,
                        n_chan);
        long long chunk = (long long)((ctx->ws_bytes - qbytes) / (per + 3 * kAlign));
        if (chunk > J.n_problems) chunk = J.n_problems;
        double* Q = (double*)ctx->ws;
        int32_t* qstat = (int32_t*)(ctx->ws + align_up((size_t)n_chan * J.n_u * J.n_u * 16));
        char* base = ctx->ws + qbytes;
        if ((st = timing_mark(ctx, 0, s)) != MMGAP_OK) return st;
        cudaError_t e = vpp_inverse_any(J.n_u, J.n_t, n_chan, J.H, J.inv_precision, Q, qstat, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "vpp_inverse launch");
        for (long long p0 = 0; p0 < J.n_problems; p0 += chunk) {
            const int P = (int)std::min<long long>(chunk, J.n_problems - p0);
            int16_t* Aq = (int16_t*)base;
            int16_t* hq = (int16_t*)(base + align_up((size_t)P * n * n * 2));
            int8_t* d = (int8_t*)((char*)hq + align_up((size_t)P * n * 2));
            if (p0 > 0 && (st = timing_mark(ctx, 0, s)) != MMGAP_OK) return st;
            VppBuildArgs b{};
            b.Q = J.chan_index ? Q : Q + (size_t)p0 * 2 * J.n_u * J.n_u;
            b.chan_index = J.chan_index ? J.chan_index + p0 : nullptr;
            b.u_sym = J.u_sym + (size_t)p0 * J.n_u;
            b.mod_bits = J.mod_bits;
            b.n_problems = P;
            b.n_chan = J.chan_index ? n_chan : P;
            b.err = ctx->dev_err;
            b.Aq = Aq;
            b.hq = hq;
            e = dispatch_nt<OpVppBuild>(J.n_u, b, s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "vpp_build launch");
            if ((st = timing_mark(ctx, 1, s)) != MMGAP_OK) return st;
            SolveArgs a{};
            a.err = ctx->dev_err;
            a.n_sm = ctx->n_sm;
            a.Aq = Aq;
            a.hq = hq;
            a.g = nullptr;
            a.level_max = 0;
            a.n_problems = P;
            a.steps = params->steps;
            a.f_mvm = params->f_mvm;
            a.key0 = (uint32_t)J.seed;
            a.key1 = (uint32_t)(J.seed >> 32);
            a.problem_offset = (uint64_t)p0;
            a.k = k;
            a.d_out = d;
            a.E_out = J.energy_out ? J.energy_out + p0 : nullptr;
            a.ndiv_out = J.ndiv_out ? J.ndiv_out + p0 : nullptr;
            a.variant = ctx->variant[J.n_u];
            a.early_exit = params->early_exit;
            a.wait_ns = ctx->wait_ns;
            e = dispatch_nt<OpSolve>(J.n_u, a, params->runs, s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cac_solve launch");
            if ((st = timing_mark(ctx, 2, s)) != MMGAP_OK) return st;
            VppOutArgs o{};
            o.H = J.chan_index ? J.H : J.H + (size_t)p0 * 2 * J.n_u * J.n_t;
            o.Q = b.Q;
            o.chan_index = b.chan_index;
            o.u_sym = b.u_sym;
            o.d = d;
            o.n_t = J.n_t;
            o.mod_bits = J.mod_bits;
            o.n_problems = P;
            o.n_chan = b.n_chan;
            o.err = ctx->dev_err;
            o.v_out = J.v_out + (size_t)p0 * n;
            o.x_out = J.x_out ? J.x_out + (size_t)p0 * 2 * J.n_t : nullptr;
            o.power_out = J.power_out ? J.power_out + p0 : nullptr;
            e = dispatch_nt<OpVppOut>(J.n_u, o, s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "vpp_output launch");
            if ((st = timing_mark(ctx, 3, s)) != MMGAP_OK) return st;
        }
    }
    return MMGAP_OK;
}

mmgap_status mmgap_vpp_inverse(mmgap_ctx* ctx, int n_u, int n_t, int n_chan, const float* H, int inv_precision,
                               double* Q_out, int32_t* status_out, void* stream) {
    NvtxRange nvtx_range("mmgap_vpp_inverse");
    if (!ctx) return MMGAP_EINVAL;
    if (!nt_supported(n_u)) return fail(ctx, MMGAP_EUNSUPPORTED, "n_u=%d: supported 1, 2, 3, 4, 8, 16", n_u);
    if (n_t < n_u || n_t > kMaxNr) return fail(ctx, MMGAP_EUNSUPPORTED, "n_t=%d out of [n_u, %d]", n_t, kMaxNr);
    if (n_chan < 0) return fail(ctx, MMGAP_EINVAL, "n_chan < 0");
    if (inv_precision != MMGAP_INV_FP64 && inv_precision != MMGAP_INV_FP32_IR)
        return fail(ctx, MMGAP_EINVAL, "inv_precision=%d: 0 (FP64) or 1 (FP32 + refinement)", inv_precision);
    if (n_chan == 0) return MMGAP_OK;
    if (!H || !Q_out) return fail(ctx, MMGAP_EINVAL, "NULL H or Q_out");
    if ((uintptr_t)H % 8 || (uintptr_t)Q_out % 16)
        return fail(ctx, MMGAP_EINVAL, "H must be 8-byte and Q_out 16-byte aligned");
    int32_t* status = status_out;
    if (!status) {
        if ((size_t)n_chan * 4 > ctx->ws_bytes)
            return fail(ctx, MMGAP_ENOMEM, "workspace too small for %d channel flags", n_chan);
        status = (int32_t*)ctx->ws;
    }
    CurrentDevice cd(ctx->device);
    cudaError_t e = vpp_inverse_any(n_u, n_t, n_chan, H, inv_precision, Q_out, status, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "vpp_inverse launch");
    return MMGAP_OK;
}

mmgap_status mmgap_detect_e(mmgap_ctx* ctx, const mmgap_params* params, const mmgap_detect_job* job, int stages,
                            int32_t* best_out, float* obj_out, int8_t* cand_out, void* stream) {
    NvtxRange nvtx_range("mmgap_detect_e");
    if (!ctx) return MMGAP_EINVAL;
    mmgap_status st = check_params(ctx, params);
    if (st != MMGAP_OK) return st;
    if (!job) return fail(ctx, MMGAP_EINVAL, "job is NULL");
    if ((st = check_detect_job(ctx, *job, true)) != MMGAP_OK) return st;
    if (job->mapping != MMGAP_MAPPING_DELTA) return fail(ctx, MMGAP_EUNSUPPORTED, "MMGaP-E uses the delta mapping");
    if (job->n_t == 32) return fail(ctx, MMGAP_EUNSUPPORTED, "MMGaP-E: n_t up to 16");
    if (job->guess_in) return fail(ctx, MMGAP_EUNSUPPORTED, "MMGaP-E makes its own guesses (guess_in must be NULL)");
    if ((st = check_early_exit(ctx, params, job->n_t)) != MMGAP_OK) return st;
    if (stages < 1 || stages > 8) return fail(ctx, MMGAP_EINVAL, "stages=%d out of [1, 8]", stages);
    const mmgap_detect_job& J = *job;
    if (J.n_problems == 0) return MMGAP_OK;
    CurrentDevice cd(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int n = 2 * J.n_t, nc = 2 + 2 * stages;
    const EulerConsts k = euler_consts(*params);
    timing_begin(ctx);
    if ((st = timing_mark(ctx, 0, s)) != MMGAP_OK) return st;
    float* gc = nullptr;
    size_t gc_bytes = 0;
    if ((st = job_gram(ctx, J, s, &gc, &gc_bytes)) != MMGAP_OK) return st;
    char* base = ctx->ws + gc_bytes;
    const size_t avail = ctx->ws_bytes - gc_bytes;
    const size_t per = align_up((size_t)n * n * 2) + align_up((size_t)n * 2) + align_up((size_t)n) + (size_t)nc * n;
    long long chunk = (long long)(avail / (per + 5 * kAlign));
    if (chunk < 1) return fail(ctx, MMGAP_ENOMEM, "workspace of %zu bytes holds no problem", ctx->ws_bytes);
    if (chunk > J.n_problems) chunk = J.n_problems;
    float kappa, kappa2;
    qam_kappa(J.mod_bits, &kappa, &kappa2);
    for (long long p0 = 0; p0 < J.n_problems; p0 += chunk) {
        const int P = (int)std::min<long long>(chunk, J.n_problems - p0);
        int16_t* Aq = (int16_t*)base;
        int16_t* hq = (int16_t*)(base + align_up((size_t)P * n * n * 2));
        int8_t* gtmp = (int8_t*)((char*)hq + align_up((size_t)P * n * 2));
        int8_t* cand = (int8_t*)((char*)gtmp + align_up((size_t)P * n));
        auto C = [&](int c) { return cand + (size_t)c * P * n; };
        if (p0 > 0 && (st = timing_mark(ctx, 0, s)) != MMGAP_OK) return st;
        BuildArgs b{};
        b.H = J.chan_index ? J.H : J.H + (size_t)p0 * 2 * J.n_r * J.n_t;
        b.chan_index = J.chan_index ? J.chan_index + p0 : nullptr;
        b.y = J.y + (size_t)p0 * 2 * J.n_r;
        b.noise_var = J.noise_var + p0;
        b.n_r = J.n_r;
        b.mod_bits = J.mod_bits;
        b.n_problems = P;
        b.n_chan = J.chan_index ? J.n_chan : P;
        b.kappa = kappa;
        b.kappa2 = kappa2;
        b.err = ctx->dev_err;
        b.Aq = Aq;
        b.hq = hq;
        b.Gc_pre = gc ? (J.chan_index ? gc : gc + (size_t)p0 * 2 * J.n_t * J.n_t) : nullptr;
        SolveArgs a{};
        a.err = ctx->dev_err;
        a.n_sm = ctx->n_sm;
        a.Aq = Aq;
        a.hq = hq;
        a.level_max = (1 << (J.mod_bits >> 1)) - 1;
        a.n_problems = P;
        a.steps = params->steps;
        a.f_mvm = params->f_mvm;
        a.problem_offset = J.problem_offset + (uint64_t)p0;
        a.k = k;
        a.mod_bits = J.mod_bits;
        a.variant = ctx->variant[J.n_t];
        a.early_exit = params->early_exit;
        a.wait_ns = ctx->wait_ns;
        cudaError_t e = cudaSuccess;
        for (int stg = 1; stg <= stages && e == cudaSuccess; ++stg)
            for (int inst = 0; inst < 2 && e == cudaSuccess; ++inst) {
                // instance inst of stage stg: around the MMSE / SIC guess (stage 1) or
                // around its own previous solution
                if (stg == 1) {
                    b.guess_mode = inst;  // 0 MMSE, 1 MMSE-SIC
                    b.g_in = nullptr;
                    b.g = C(inst);
                } else {
                    b.guess_mode = 2;
                    b.g_in = C(2 + 2 * (stg - 2) + inst);
                    b.g = gtmp;
                }
                e = dispatch_nt<OpBuild>(J.n_t, b, s);
                if (e != cudaSuccess) break;
                const uint64_t seed = J.seed + (uint64_t)(2 * (stg - 1) + inst) * 0x9E3779B97F4A7C15ULL;
                a.key0 = (uint32_t)seed;
                a.key1 = (uint32_t)(seed >> 32);
                a.g = stg == 1 ? C(inst) : C(2 + 2 * (stg - 2) + inst);
                a.x_out = C(2 + 2 * (stg - 1) + inst);
                e = dispatch_nt<OpSolve>(J.n_t, a, params->runs, s);
            }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "MMGaP-E stage launch");
        if ((st = timing_mark(ctx, 1, s)) != MMGAP_OK) return st;
        if ((st = timing_mark(ctx, 2, s)) != MMGAP_OK) return st;
        SelectArgs sa{};
        sa.H = b.H;
        sa.chan_index = b.chan_index;
        sa.y = b.y;
        sa.n_r = J.n_r;
        sa.mod_bits = J.mod_bits;
        sa.n_problems = P;
        sa.n_chan = b.n_chan;
        sa.kappa = kappa;
        sa.cand = cand;
        sa.n_cand = nc;
        sa.sym_out = J.sym_out + (size_t)p0 * J.n_t;
        sa.best_out = best_out ? best_out + p0 : nullptr;
        sa.obj_out = obj_out ? obj_out + p0 : nullptr;
        e = dispatch_nt<OpSelect>(J.n_t, sa, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "select launch");
        if (cand_out)
            for (int c = 0; c < nc; ++c) {
                e = cudaMemcpyAsync(cand_out + ((size_t)c * J.n_problems + p0) * n, C(c), (size_t)P * n,
                                    cudaMemcpyDeviceToDevice, s);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "candidate copy");
            }
        if ((st = timing_mark(ctx, 3, s)) != MMGAP_OK) return st;
    }
    return MMGAP_OK;
}

mmgap_status mmgap_anneal_spins(mmgap_ctx* ctx, const mmgap_params* params, int n, int n_problems, const int16_t* A_q,
                                const int16_t* h_q, uint64_t seed, uint64_t* spins_out, void* stream) {
    NvtxRange nvtx_range("mmgap_anneal_spins");
    if (!ctx) return MMGAP_EINVAL;
    mmgap_status st = check_params(ctx, params);
    if (st != MMGAP_OK) return st;
    if (n < 2 || (n & 1) || !nt_supported(n / 2))
        return fail(ctx, MMGAP_EUNSUPPORTED, "n=%d: supported 2, 4, 6, 8, 16, 32", n);
    if (n_problems < 0) return fail(ctx, MMGAP_EINVAL, "n_problems < 0");
    if (params->early_exit) return fail(ctx, MMGAP_EUNSUPPORTED, "the integration study anneals all steps");
    if (n_problems == 0) return MMGAP_OK;
    if (!A_q || !h_q || !spins_out) return fail(ctx, MMGAP_EINVAL, "NULL A_q, h_q or spins_out");
    CurrentDevice cd(ctx->device);
    SolveArgs a{};
    a.err = ctx->dev_err;
    a.n_sm = ctx->n_sm;
    a.Aq = A_q;
    a.hq = h_q;
    a.n_problems = n_problems;
    a.steps = params->steps;
    a.f_mvm = params->f_mvm;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.k = euler_consts(*params);
    a.spins_out = spins_out;
    // the selection still runs; its outputs go to the workspace
    if (ctx->ws_bytes < (size_t)n_problems * (n + 16) + 4 * kAlign)
        return fail(ctx, MMGAP_ENOMEM, "workspace too small");
    a.d_out = (int8_t*)ctx->ws;
    cudaError_t e = dispatch_nt<OpSolve>(n / 2, a, params->runs, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cac_solve launch");
    return MMGAP_OK;
}

mmgap_status mmgap_set_solver_variant(mmgap_ctx* ctx, int n_t, int variant) {
    if (!ctx) return MMGAP_EINVAL;
    if (!nt_supported(n_t)) return fail(ctx, MMGAP_EUNSUPPORTED, "n_t=%d", n_t);
    if (variant < 0 || variant >= kVariantCount) return fail(ctx, MMGAP_EINVAL, "variant=%d", variant);
    if (variant_tensor_core(variant) && n_t != 8 && n_t != 16)
        return fail(ctx, MMGAP_EUNSUPPORTED, "tensor-core refresh needs n_t 8 or 16");
    ctx->variant[n_t] = variant;
    return MMGAP_OK;
}

mmgap_status mmgap_set_device_wait(mmgap_ctx* ctx, uint64_t limit_ns) {
    if (!ctx) return MMGAP_EINVAL;
    ctx->wait_ns = limit_ns;
    return MMGAP_OK;
}

mmgap_status mmgap_get_solver_variant(mmgap_ctx* ctx, int n_t, int f_mvm, int* variant_out) {
    if (!ctx || !variant_out) return MMGAP_EINVAL;
    if (!nt_supported(n_t)) return fail(ctx, MMGAP_EUNSUPPORTED, "n_t=%d", n_t);
    *variant_out = resolve_variant(n_t, f_mvm, ctx->variant[n_t]);
    return MMGAP_OK;
}

mmgap_status mmgap_autotune(mmgap_ctx* ctx, const mmgap_params* params, int n_t, int n_problems, int* variant_out,
                            float ms_out[16]) {
    NvtxRange nvtx_range("mmgap_autotune");
    if (!ctx) return MMGAP_EINVAL;
    mmgap_status st = check_params(ctx, params);
    if (st != MMGAP_OK) return st;
    if (!nt_supported(n_t)) return fail(ctx, MMGAP_EUNSUPPORTED, "n_t=%d", n_t);
    const int n = 2 * n_t;
    if (n_problems <= 0) n_problems = 8192;
    const size_t per = (size_t)n * n * 2 + (size_t)n * 2 + (size_t)n + 32;
    const size_t cap = ctx->ws_bytes > 4 * kAlign ? (ctx->ws_bytes - 4 * kAlign) / per : 0;
    if (cap < 1) return fail(ctx, MMGAP_ENOMEM, "workspace too small for autotuning");
    if ((size_t)n_problems > cap) n_problems = (int)cap;
    CurrentDevice cd(ctx->device);
    int16_t* Aq = (int16_t*)ctx->ws;
    int16_t* hq = (int16_t*)(ctx->ws + align_up((size_t)n_problems * n * n * 2));
    int8_t* d = (int8_t*)((char*)hq + align_up((size_t)n_problems * n * 2));
    int32_t* E = (int32_t*)((char*)d + align_up((size_t)n_problems * n));
    cudaStream_t s = nullptr;
    cudaError_t e = launch_random_ising(Aq, hq, n, n_problems, 0x5eedULL, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "random problems");
    SolveArgs a{};
    a.err = ctx->dev_err;
    a.n_sm = ctx->n_sm;
    a.Aq = Aq;
    a.hq = hq;
    a.n_problems = n_problems;
    a.steps = params->steps;
    a.f_mvm = params->f_mvm;
    a.key0 = 1;
    a.k = euler_consts(*params);
    a.early_exit = params->early_exit;
    a.d_out = d;
    a.E_out = E;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if ((e = cudaEventCreate(&t0)) != cudaSuccess || (e = cudaEventCreate(&t1)) != cudaSuccess) {
        if (t0) cudaEventDestroy(t0);
        return cuda_fail(ctx, e, "cudaEventCreate");
    }
    float best = 1e30f;
    int best_v = kVariantPlain;
    static_assert(kVariantCount <= 16, "mmgap_autotune reports 16 slots");
    if (ms_out)
        for (int v = 0; v < 16; ++v) ms_out[v] = -1.0f;
    for (int v = kVariantPlain; v < kVariantCount; ++v) {
        if (!variant_exact(v)) continue;                             // bit-identical shapes only
        if (resolve_variant(n_t, params->f_mvm, v) != v) continue;  // not compiled for this size
        a.variant = v;
        e = dispatch_nt<OpSolve>(n_t, a, params->runs, s);  // warm up
        float ms = 0.0f;
        for (int r = 0; r < 2 && e == cudaSuccess; ++r) {
            cudaEventRecord(t0, s);
            e = dispatch_nt<OpSolve>(n_t, a, params->runs, s);
            cudaEventRecord(t1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(t1);
            float m = 0.0f;
            cudaEventElapsedTime(&m, t0, t1);
            ms = r == 0 ? m : std::min(ms, m);
        }
        if (e != cudaSuccess) break;
        if (ms_out) ms_out[v] = ms;
        if (ms < best) {
            best = ms;
            best_v = v;
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune");
    ctx->variant[n_t] = best_v;
    if (variant_out) *variant_out = best_v;
    if (ms_out) ms_out[0] = best;
    return MMGAP_OK;
}

}  // extern "C"
