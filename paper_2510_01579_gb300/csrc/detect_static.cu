// Allocation-free uplink detection: mmgap_detect_static.
//
// Some callers cannot allocate device memory.  A real-time slot loop may not
// call cudaMalloc once it is running, because an allocation can synchronise
// the device and blow a 0.5 ms slot; a plug-in hosted by an application that
// owns every device allocation may not allocate at all.  This entry point
// serves them: it needs no context and takes its per-problem scratch (the
// quantised couplings, field and guess between the build and solve kernels)
// from a fixed array compiled into the library instead of from a workspace.
//
// The scratch is a file-scope __device__ array of kStaticScratchBytes, so
// every GPU that loads this library holds that much memory until the process
// exits (with lazy module loading, from the first call on that device).
// Host code only ever sees a host-side stand-in for the array's name; its
// device address is looked up with cudaGetSymbolAddress once per device (with
// that device current) and cached, together with the device's SM count.
#include <cstdio>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/mmgap.h"
#include "internal.h"

using namespace mmgap;

namespace {

constexpr size_t kStaticScratchBytes = (size_t)8 << 20;  // 8 MiB per device
constexpr size_t kAlign = 256;

static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct DeviceInfo {
    unsigned char* scratch = nullptr;  // device address of g_scratch on this device
    int n_sm = 0;                      // SMs, for the small-call launch shapes
};

std::mutex g_mu;
DeviceInfo g_info[kMaxDevices];

// Address of the static scratch and SM count of the current device `dev`
// (looked up on the first call on that device, with it current).
mmgap_status device_info(int dev, DeviceInfo* out) {
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceInfo& d = g_info[dev];
    if (!d.scratch) {
        void* s = nullptr;
        if (cudaGetSymbolAddress(&s, g_scratch) != cudaSuccess) {
            cudaGetLastError();
            return MMGAP_ECUDA;
        }
        int n_sm = 0;
        if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            n_sm = 0;  // unknown: the throughput shapes for every call
        }
        d.n_sm = n_sm;
        d.scratch = (unsigned char*)s;
    }
    *out = d;
    return MMGAP_OK;
}

// Same per-size launchers as the context path.
template <template <int> class Op, class... Args>
cudaError_t dispatch_nt(int nt, Args&&... args) {
    switch (nt) {
    case 1: return Op<1>::run(args...);
    case 2: return Op<2>::run(args...);
    case 3: return Op<3>::run(args...);
    case 4: return Op<4>::run(args...);
    case 8: return Op<8>::run(args...);
    case 16: return Op<16>::run(args...);
    case 32: return Op<32>::run(args...);  // (both operations exist for 32 users)
    default: return cudaErrorInvalidValue;
    }
}
template <int NT> struct OpBuild { static cudaError_t run(const BuildArgs& a, cudaStream_t s) { return launch_build_detect<NT>(a, s); } };
template <int NT> struct OpSolve { static cudaError_t run(const SolveArgs& a, int r, cudaStream_t s) { return launch_solve<NT>(a, r, s); } };

bool nt_ok(int nt) { return nt == 1 || nt == 2 || nt == 3 || nt == 4 || nt == 8 || nt == 16 || nt == 32; }

}  // namespace

extern "C" {

mmgap_status mmgap_detect_static(const mmgap_params* params, const mmgap_detect_job* job, void* stream) {
    NvtxRange nvtx_range("mmgap_detect_static");
    if (!params || !job) return MMGAP_EINVAL;
    const mmgap_params& P = *params;
    if (!(P.runs == 32 || P.runs == 64 || P.runs == 96 || P.runs == 128)) return MMGAP_EUNSUPPORTED;
    if (P.steps < 0 || P.steps > (1 << 20) || P.f_mvm < 1 || P.f_mvm > 64 || !(P.dt > 0.0f) || !(P.x_max > 0.0f) ||
        P.early_exit < 0)
        return MMGAP_EINVAL;
    const mmgap_detect_job& J = *job;
    if (!nt_ok(J.n_t) || J.n_r < 1 || J.n_r > kMaxNr || !(J.mod_bits == 2 || J.mod_bits == 4 || J.mod_bits == 6))
        return MMGAP_EUNSUPPORTED;
    if (J.n_problems < 0) return MMGAP_EINVAL;
    if (J.n_problems == 0) return MMGAP_OK;
    if (!J.H || !J.y || !J.noise_var || !J.sym_out || J.n_chan < 1) return MMGAP_EINVAL;
    if (!J.chan_index && J.n_chan < J.n_problems) return MMGAP_EINVAL;
    if (J.gram_precision != 0) return MMGAP_EUNSUPPORTED;  // the tensor-core Gram needs a workspace
    if (J.mapping != MMGAP_MAPPING_DELTA) return MMGAP_EUNSUPPORTED;  // the direct mapping has its own scratch layout
    if (P.early_exit > 0 && J.n_t == 32) return MMGAP_EUNSUPPORTED;     // early exit: up to 16 users

    // scratch this job needs: A_q, h_q and g in three 256-B-aligned regions
    const int n = 2 * J.n_t;
    const size_t need = align_up((size_t)J.n_problems * n * n * 2) + align_up((size_t)J.n_problems * n * 2) +
                        align_up((size_t)J.n_problems * n);
    if (need > kStaticScratchBytes) {
        fprintf(stderr,
                "mmgap_detect_static: %d problems of %d users need %zu bytes of scratch, more than the %zu-byte "
                "static array; split the job\n",
                J.n_problems, J.n_t, need, kStaticScratchBytes);
        return MMGAP_ENOMEM;
    }

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MMGAP_ECUDA;
    DeviceInfo info;
    mmgap_status st = device_info(dev, &info);
    if (st != MMGAP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;

    // Every region below is written in full by the build kernel before the
    // solver reads it, so nothing left by an earlier call is ever read.
    int16_t* Aq = (int16_t*)info.scratch;
    int16_t* hq = (int16_t*)(info.scratch + align_up((size_t)J.n_problems * n * n * 2));
    int8_t* g = (int8_t*)((unsigned char*)hq + align_up((size_t)J.n_problems * n * 2));

    BuildArgs b{};
    b.H = J.H;
    b.chan_index = J.chan_index;
    b.y = J.y;
    b.noise_var = J.noise_var;
    b.n_r = J.n_r;
    b.mod_bits = J.mod_bits;
    b.n_problems = J.n_problems;
    b.n_chan = J.chan_index ? J.n_chan : J.n_problems;
    qam_kappa(J.mod_bits, &b.kappa, &b.kappa2);
    b.err = nullptr;  // no error word: a bad channel index gives an all-zero problem, unreported
    b.guess_mode = J.guess_in ? 2 : 0;
    b.g_in = J.guess_in;
    b.Aq = Aq;
    b.hq = hq;
    b.g = g;
    if (dispatch_nt<OpBuild>(J.n_t, b, s) != cudaSuccess) return MMGAP_ECUDA;

    SolveArgs a{};
    a.Aq = Aq;
    a.hq = hq;
    a.g = g;
    a.level_max = (1 << (J.mod_bits >> 1)) - 1;
    a.n_problems = J.n_problems;
    a.steps = P.steps;
    a.f_mvm = P.f_mvm;
    a.key0 = (uint32_t)J.seed;
    a.key1 = (uint32_t)(J.seed >> 32);
    a.problem_offset = J.problem_offset;
    a.k = euler_consts(P.dt, P.p, P.a, P.zeta, P.eps, P.sigma0, P.x_max);
    a.n_sm = info.n_sm;
    a.early_exit = P.early_exit;
    a.steps_out = J.steps_out;
    a.d_out = J.offset_out;
    a.E_out = J.energy_out;
    a.ndiv_out = J.ndiv_out;
    a.sym_out = J.sym_out;
    a.mod_bits = J.mod_bits;
    if (dispatch_nt<OpSolve>(J.n_t, a, P.runs, s) != cudaSuccess) return MMGAP_ECUDA;
    if (J.guess_out &&
        cudaMemcpyAsync(J.guess_out, g, (size_t)J.n_problems * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return MMGAP_ECUDA;
    return MMGAP_OK;
}

}  // extern "C"
