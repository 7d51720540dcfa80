// Allocation-free uplink detection: mmgap_detect_static.
//
// Some callers cannot allocate device memory.  A real-time slot loop may not
// call cudaMalloc once it is running, because an allocation can synchronise
// the device and blow a 0.5 ms slot; a plug-in hosted by an application that
// owns every device allocation may not allocate at all; and code that records
// its work into a CUDA graph cannot have an allocation inside the recorded
// section.  This entry point serves them: it needs no context and takes its
// per-problem scratch (the quantised couplings, field and guess between the
// build and solve kernels) from a fixed array compiled into the library
// instead of from a workspace.
//
// The scratch is a file-scope __device__ array of kStaticScratchBytes, so
// every GPU that loads this library holds that much memory until the process
// exits.  Host code only ever sees a host-side stand-in for the array's name;
// its device address is looked up with cudaGetSymbolAddress once per device
// (with that device current) and cached.
#include <cmath>
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
static __device__ __align__(256) int g_scratch_err[1];

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct DevicePtrs {
    unsigned char* scratch = nullptr;
    int* err = nullptr;
};

std::mutex g_mu;
DevicePtrs g_ptrs[kMaxDevices];

// Device addresses of the static scratch on the current device (looked up on
// the first call on that device).
mmgap_status device_ptrs(int dev, DevicePtrs* out) {
    std::lock_guard<std::mutex> lock(g_mu);
    DevicePtrs& p = g_ptrs[dev];
    if (!p.scratch) {
        void* s = nullptr;
        void* e = nullptr;
        if (cudaGetSymbolAddress(&s, g_scratch) != cudaSuccess) return MMGAP_ECUDA;
        if (cudaGetSymbolAddress(&e, g_scratch_err) != cudaSuccess) return MMGAP_ECUDA;
        p.scratch = (unsigned char*)s;
        p.err = (int*)e;
    }
    *out = p;
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
    if (P.steps < 0 || P.steps > (1 << 20) || P.f_mvm < 1 || P.f_mvm > 64 || !(P.dt > 0.0f) || !(P.x_max > 0.0f))
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
    DevicePtrs ptr;
    mmgap_status st = device_ptrs(dev, &ptr);
    if (st != MMGAP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // the error word is OR-ed by the build kernel; it starts from zero on every call
    if (cudaMemsetAsync(ptr.err, 0, sizeof(int), s) != cudaSuccess) return MMGAP_ECUDA;

    int16_t* Aq = (int16_t*)ptr.scratch;
    int16_t* hq = (int16_t*)(ptr.scratch + align_up((size_t)J.n_problems * n * n * 2));
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
    {
        const double M = (double)(1 << J.mod_bits);
        b.kappa = (float)(1.0 / std::sqrt(2.0 * (M - 1.0) / 3.0));
        b.kappa2 = (float)(1.0 / (2.0 * (M - 1.0) / 3.0));
    }
    b.err = ptr.err;
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
    a.problem_offset = 0;
    {
        const double dt = P.dt, p = P.p, aa = P.a, zeta = P.zeta, eps = P.eps;
        a.k.c1 = (float)(1.0 + dt * (p - 1.0));
        a.k.cdt = (float)(-dt);
        a.k.cz = (float)(-(dt * zeta));
        a.k.c2 = (float)(1.0 + (dt * zeta) * aa);
        a.k.ce = (float)(eps * dt);
        a.k.xs = (float)((double)P.sigma0 * 0x1p-23);
        a.k.x_max = P.x_max;
    }
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
