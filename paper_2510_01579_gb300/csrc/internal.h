// Internal (C++) interface between the C-ABI front end (api.cu) and the
// per-size kernel translation units (inst_nt*.cu).  Not part of the ABI.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace mmgap {

// NVTX range over one library call (visible in Nsight timelines; a no-op
// without a tool attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};


// Derived constants of the Euler discretisation of Eqs. 10-11, each rounded
// once to FP32 from a double expression of the float parameters.
struct EulerConsts {
    float c1;   // 1 + dt (p - 1)
    float cdt;  // -dt
    float cz;   // -dt zeta
    float c2;   // 1 + dt zeta a
    float ce;   // eps dt, folded into the couplings
    float xs;   // sigma0 2^-23 (initial-amplitude scale)
    float x_max;
};

// Host-side derivation of the constants above, shared by every entry point so
// that all paths round them identically.
EulerConsts euler_consts(float dt, float p, float a, float zeta, float eps, float sigma0, float x_max);
// QAM normalisation kappa = 1/sqrt(2 (M-1)/3) and kappa^2, each rounded once to float.
void qam_kappa(int mod_bits, float* kappa, float* kappa2);

// Default limit of the bounded device-side waits (0.2 s; the awaited work takes microseconds).
constexpr unsigned long long kDefaultDeviceWaitNs = 200000000ull;

struct SolveArgs {
    const int16_t* Aq;   // [P][n][n]
    const int16_t* hq;   // [P][n]
    const int8_t* g;     // [P][n] or nullptr
    int level_max;
    int n_problems;
    int steps;
    int f_mvm;
    uint32_t key0, key1;       // Philox key (seed)
    uint64_t problem_offset;   // job-local index of problem 0 of this launch
    EulerConsts k;
    // outputs (solver boundary)
    int8_t* d_out;             // [P][n] or nullptr
    int32_t* E_out;
    int32_t* run_out;
    int32_t* ndiv_out;
    // fused uplink decode (detect): symbols of g + 2 d
    uint8_t* sym_out;          // [P][n_t] or nullptr
    int mod_bits;
    int variant;               // SolverVariant; 0 = the size's default
    int8_t* x_out;             // [P][n] selected lattice point g + 2d, or nullptr
    uint64_t* spins_out;       // [P][runs][2] final sign bits per anneal (plain kernel), or nullptr
    int* err;                  // device error word (bit 1: a tcgen05 wait expired), or nullptr
    int n_sm;                  // SMs of the device (0: unknown); picks latency shapes for small calls
    int early_exit;            // K > 0: stop a problem's anneals at the first K-th refresh with no sign change
    int32_t* steps_out;        // [P] Euler steps taken, or nullptr
    // limit of each bounded device wait (tcgen05 completion, shape 8); 0 = give up at once
    unsigned long long wait_ns = kDefaultDeviceWaitNs;
};

// Launch shapes of the solver.  All produce bit-identical results.
enum SolverVariant : int {
    kVariantAuto = 0,
    kVariantPlain = 1,       // one thread per anneal, scalar FP32 (the paper's design point)
    kVariantTpa1 = 2,        // tuned kernel, one thread per anneal
    kVariantTpa1Packed = 3,  // tuned kernel, one thread per anneal, packed FP32 pairs
    kVariantTpa2Packed = 4,  // tuned kernel, two threads per anneal, packed FP32 pairs
    kVariantTensorCore = 5,  // field refresh on tensor cores (FP16 split, FP32 accumulation): not bit-identical
    kVariantPairPacked = 6,  // tuned kernel, one thread per anneal, refresh shared by lane pairs
    kVariantTensorCore2 = 7, // field refresh on tensor cores, two threads per anneal: not bit-identical
    kVariantUmma = 8,        // field refresh by tcgen05 UMMA into tensor memory: not bit-identical
    kVariantTpa4Packed = 9,  // tuned kernel, four threads per anneal, packed FP32 pairs (n_t 8, 16)
    kVariantTpa8Packed = 10, // tuned kernel, eight threads per anneal, packed FP32 pairs (n_t 16)
    kVariantCount = 11
};

// Variant used for n_t users and refresh period f_mvm when `requested` is
// kVariantAuto or not compiled for that size.  With the call's problem count
// and the device's SM count known, kVariantAuto takes the latency shapes when
// the call leaves SMs idle.
int resolve_variant(int n_t, int f_mvm, int requested, int n_problems = -1, int n_sm = 0);
// Shapes whose results are bit-identical to the plain kernel's (the autotuner's candidates).
constexpr bool variant_exact(int v) {
    return v != kVariantTensorCore && v != kVariantTensorCore2 && v != kVariantUmma;
}
constexpr bool variant_tensor_core(int v) { return !variant_exact(v); }

struct BuildArgs {
    const float* H;            // complex [n_chan][n_r][n_t]
    const int32_t* chan_index; // [P] or nullptr (identity)
    const float* y;            // complex [P][n_r]
    const float* noise_var;    // [P]
    int n_r;
    int mod_bits;
    int n_problems;
    int n_chan;                // channels addressable through chan_index
    float kappa, kappa2;
    int* err;                  // device error word (bit 0: channel index out of range)
    const float* Gc_pre;       // optional precomputed Gram of kappa H per channel, complex [n_chan][n_t][n_t]
    // optional MMSE Cholesky factor of each channel (chan_factor_kernel), used by a problem whose
    // rho = noise_var kappa^2 equals the channel's: L complex [n_chan][n_t][n_t], rho, failed-pivot flag
    const float* L_pre;
    const float* rho_pre;
    const int32_t* chol_pre;
    int guess_mode;            // 0: MMSE, 1: MMSE-SIC (sorted Cholesky), 2: given g_in
    const int8_t* g_in;        // [P][n] lattice guesses for guess_mode 2
    // outputs
    int16_t* Aq;               // [P][n][n]
    int16_t* hq;               // [P][n]
    int8_t* g;                 // [P][n]
    float* G32;                // [P][n][n] or nullptr
    float* h32;                // [P][n] or nullptr
    int32_t* sigma_exp;        // [P] or nullptr
};

// Per-channel MMSE factorisation ahead of the builder: for every channel, the
// Cholesky factor of G_c + rho I with rho from the channel's first problem.
struct ChanFactorArgs {
    const float* H;            // complex [n_chan][n_r][n_t]
    const int32_t* chan_index; // [P]
    const float* noise_var;    // [P]
    int n_r, n_problems, n_chan;
    float kappa, kappa2;
    int32_t* first;            // scratch [n_chan]: first problem of each channel
    float* L_out;              // complex [n_chan][n_t][n_t]
    float* rho_out;            // [n_chan] (NaN for a channel no problem uses)
    int32_t* chol_out;         // [n_chan] 1 if a pivot failed
    float* G_out;              // complex [n_chan][n_t][n_t]: the Gram of kappa H (the builder's Gc_pre), or nullptr
};

// Direct (binary-weighted) spin mapping: the delta build's MMSE guess, Gram
// and matched filter (b.Aq / b.hq unused; b.g receives the guess), expanded by
// powers of two into J = -(T^T G T) (zero diagonal) and c = T^T Hs^T y over
// N = 2 n_t B spins, quantised like the delta form.
struct DirectBuildArgs {
    BuildArgs b;
    int B;                     // spins per real dimension, mod_bits / 2
    int16_t* Jq;               // [P][N][N]
    int16_t* cq;               // [P][N]
    int8_t* s_ref;             // [P][N] spins of the guess, or nullptr
    float* J32;                // [P][N][N] or nullptr
    float* c32;                // [P][N] or nullptr
    int32_t* sigma_exp;        // [P] or nullptr
};

// General Ising problem with an auxiliary spin (J symmetric, zero diagonal;
// c couples through the auxiliary spin), annealed by the same CIM-CAC steps.
struct GeneralArgs {
    const int16_t* Jq;         // [P][N][N]
    const int16_t* cq;         // [P][N]
    const int8_t* s_ref;       // [P][N] reference candidate (wins ties), or nullptr
    int n_problems;
    int steps;
    int f_mvm;
    uint32_t key0, key1;
    uint64_t problem_offset;
    EulerConsts k;
    int8_t* s_out;             // [P][N] or nullptr
    int32_t* E_out;            // [P] or nullptr
    int32_t* run_out;          // [P] or nullptr (-1: the reference)
    int32_t* ndiv_out;         // [P] or nullptr
    // detection decode of x = T s (B = mod_bits / 2 spins per dimension)
    int mod_bits;              // 0: no decode
    uint8_t* sym_out;          // [P][n_t] or nullptr
    const int8_t* g;           // [P][2 n_t] guess, for offset_out
    int8_t* offset_out;        // [P][2 n_t] (x - g) / 2, or nullptr
};

// Gram of kappa H per channel on tensor cores (BF16 or FP16 operands, FP32
// accumulation); Hermitian by construction (upper triangle mirrored).
struct GramArgs {
    const float* H;   // complex [n_chan][n_r][n_t]
    int n_r;
    int n_chan;
    float kappa;
    int fp16;         // 0: BF16 operands, 1: FP16 operands, 2: split BF16 (hi + lo, three products)
    float* Gc;        // complex [n_chan][n_t][n_t]
};

// Best of several lattice candidates per problem by the FP32 ML objective.
struct SelectArgs {
    const float* H;            // complex [n_chan][n_r][n_t]
    const int32_t* chan_index;
    const float* y;            // complex [P][n_r]
    int n_r, mod_bits, n_problems, n_chan;
    float kappa;
    const int8_t* cand;        // [n_cand][P][n]
    int n_cand;
    uint8_t* sym_out;          // [P][n_t]
    int32_t* best_out;         // [P] or nullptr
    float* obj_out;            // [P] or nullptr
};

struct VppInvArgs {
    const float* H;   // complex [n_chan][n_u][n_t]
    int n_t;
    int n_chan;
    double* Q;        // complex [n_chan][n_u][n_u]
    int32_t* status;  // [n_chan] 0 ok, 1 not positive definite, 2 FP32 refinement did not converge
    int refine;       // FP32 path: maximum refinement steps
    int only_failed;  // FP64 path: recompute only channels whose status is non-zero
};

struct VppBuildArgs {
    const double* Q;           // complex [n_chan][n_u][n_u]
    const int32_t* chan_index; // [P] or nullptr
    const uint8_t* u_sym;      // [P][n_u]
    int mod_bits;
    int n_problems;
    int n_chan;
    int* err;
    int16_t* Aq;
    int16_t* hq;
};

struct VppOutArgs {
    const float* H;            // complex [n_chan][n_u][n_t]
    const double* Q;
    const int32_t* chan_index;
    const uint8_t* u_sym;
    const int8_t* d;           // [P][n]
    int n_t;
    int mod_bits;
    int n_problems;
    int n_chan;
    int* err;
    int8_t* v_out;
    float* x_out;
    float* power_out;
};

// Launchers, one set per n_t (defined in inst_nt<N>.cu).  Return the launch
// error (cudaSuccess on success).
template <int NT> cudaError_t launch_build_detect(const BuildArgs& a, cudaStream_t s);
template <int NT> cudaError_t launch_chan_factor(const ChanFactorArgs& a, cudaStream_t s);
template <int NT> cudaError_t launch_solve(const SolveArgs& a, int runs, cudaStream_t s);
template <int NT> cudaError_t launch_vpp_inverse(const VppInvArgs& a, cudaStream_t s);
template <int NT> cudaError_t launch_vpp_inverse_ir(const VppInvArgs& a, cudaStream_t s);
template <int NT> cudaError_t launch_build_direct(const DirectBuildArgs& a, cudaStream_t s);
// N in {8, 16, 24, 32, 48, 64, 96} (defined in general.cu); runs a multiple of 32.
bool general_supported(int N);
cudaError_t launch_solve_general(int N, const GeneralArgs& a, int runs, cudaStream_t s);
template <int NT> cudaError_t launch_gram_tc(const GramArgs& a, cudaStream_t s);
template <int NT> cudaError_t launch_select(const SelectArgs& a, cudaStream_t s);
template <int NT> cudaError_t launch_vpp_build(const VppBuildArgs& a, cudaStream_t s);
template <int NT> cudaError_t launch_vpp_output(const VppOutArgs& a, cudaStream_t s);

// Q = (H H^H)^-1 for n_chan channels of n_u users (see mmgap_vpp_inverse):
// FP64, or FP32 with iterative refinement and FP64 for the channels it does
// not accept.  status: int32 [n_chan], required.  Defined in api.cu.
constexpr int kVppRefineSteps = 10;
cudaError_t vpp_inverse_any(int n_u, int n_t, int n_chan, const float* H, int inv_precision, double* Q,
                            int32_t* status, cudaStream_t s);

// Random symmetric Q14 problems (uniform codes in [-2^14, 2^14]) for the
// autotuner, drawn from Philox on the device (defined in api.cu).
cudaError_t launch_random_ising(int16_t* Aq, int16_t* hq, int n, int n_problems, uint64_t seed, cudaStream_t s);

constexpr int kMaxNr = 64;
constexpr int kMaxDevices = 64;  // devices whose per-kernel launch attributes are cached

// Bits of the device error word.
constexpr int kErrChanIndex = 1;
constexpr int kErrGuess = 4;  // a caller-supplied guess entry is not an alphabet point

}  // namespace mmgap
