/*
 * mmgap.h -- C ABI of the GB300 (sm_103a) MMGaP hot path.
 *
 * MMGaP (Singh & Jamieson, "Multi-User MIMO Detection and Precoding using
 * GPU-assisted Physics-inspired Computation") turns every subcarrier's
 * uplink ML detection problem (Sec. 2.1, Eq. 2) and every downlink
 * vector-perturbation precoding problem (Sec. 2.2 Eq. 8, Sec. 3.3 Eq. 13)
 * into a delta-Ising problem around a guess (Sec. 2.3 Eq. 9, Sec. 3.2.1,
 * Fig. 5), runs many CIM-CAC anneals on it (Eqs. 10-11, Sec. 3.2) and keeps
 * the lowest-energy candidate.  The paper's three kernels (pre-processing,
 * solver, post-processing; Sec. 3.2, Fig. 4) map to: a batched builder
 * (Gram, matched filter, MMSE guess, field, Q14 quantisation), the CIM-CAC
 * solver with the arg-min folded in, and a decoder.
 *
 * Conventions for every entry point:
 *   - Array arguments are DEVICE pointers owned by the caller, unless stated
 *     otherwise.  Complex arrays are interleaved float32 (re, im) pairs, row
 *     major.  Pointers must be 4-byte aligned (complex: 8-byte).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued asynchronously on it; the caller synchronises.
 *   - Argument errors are reported synchronously (MMGAP_EINVAL /
 *     MMGAP_EUNSUPPORTED / MMGAP_ENOMEM) before anything is launched.  A CUDA
 *     launch error returns MMGAP_ECUDA; asynchronous device faults surface on
 *     the caller's next synchronisation.  mmgap_last_error() describes the
 *     last failure.  No C++ exception crosses this boundary.
 *   - Determinism: results depend only on the inputs, the parameters, the job
 *     seed and the problem's index within its job, never on batch position,
 *     chunking or stream.  For identical inputs the integer outputs (guesses,
 *     quantised couplings, offsets, symbols, energies) equal the CPU oracle's
 *     bit for bit.
 *   - A context is not thread safe; use one context per host thread.
 */
#ifndef MMGAP_H
#define MMGAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mmgap_ctx mmgap_ctx;

typedef enum {
    MMGAP_OK = 0,
    MMGAP_EINVAL = 1,       /* bad argument (NULL pointer, size out of range) */
    MMGAP_ENOMEM = 2,       /* workspace too small for one problem / allocation failed */
    MMGAP_ECUDA = 3,        /* CUDA runtime error */
    MMGAP_ETIMEOUT = 4,     /* a bounded wait expired */
    MMGAP_EUNSUPPORTED = 5, /* size or option not compiled in */
    MMGAP_EBUSY = 6         /* resource in use */
} mmgap_status;

/*
 * Solver parameters.  dt, f_mvm: Appendix A (the paper uses dt = 0.02,
 * f_mvm = 2); p, a, zeta, eps: the free parameters of Eqs. 10-11 (the paper
 * prints no values); runs: N_a anneals per problem (Sec. 2.3, Sec. 3.2;
 * the paper uses 32, one warp); steps: N_I Euler steps per anneal.
 * sigma0: initial amplitudes are uniform in [-sigma0, sigma0) (Sec. 2.3:
 * random initialisation); x_max: an anneal whose final |x| exceeds x_max, is
 * not finite, or whose error variable left (0, inf) is counted as diverged
 * (Appendix A, P_diverge) and replaced by the guess.
 * Limits: runs in {32, 64, 96, 128}; steps in [0, 1<<20]; f_mvm in [1, 64];
 * dt > 0.
 * early_exit: 0 = every anneal runs all `steps` steps (the paper's fixed N_I).
 *   K > 0 = early exit, a budget lever with no counterpart in the paper: a
 *   problem's anneals advance together, and every K-th field refresh, at
 *   t = j K f_mvm (0 < t < steps), the signs [x >= 0] of all spins of all of
 *   its anneals are compared with their signs at t - K f_mvm; if none changed,
 *   all of the problem's anneals stop at t (their state there is final) and
 *   selection proceeds as usual.  Results stay bit-exact with the CPU oracle
 *   under the same rule.  Supported by mmgap_detect (delta mapping, up to 16
 *   users, the bit-identical solver shapes), mmgap_detect_e, mmgap_precode,
 *   mmgap_solve_ising (n <= 32), mmgap_detect_static, the batched launch and
 *   the server (without MMGAP_BATCH_TENSOR_CORE / tensor_core, up to 16
 *   users); the other calls and the tensor-core shapes 5, 7 and 8 return
 *   MMGAP_EUNSUPPORTED when K > 0.
 */
typedef struct {
    int32_t runs;
    int32_t steps;
    int32_t f_mvm;
    float dt, p, a, zeta, eps;
    float sigma0;
    float x_max;
    int32_t early_exit;
} mmgap_params;

/*
 * One uplink detection job: n_problems problems (resource elements) of the
 * same size (Sec. 3.2: inputs are H and y per problem, Fig. 4).
 *   n_t in {1, 2, 3, 4, 8, 16, 32} users, n_r in [1, 64] antennas; 32 users
 *   (the 32x32 high-connectivity case) only with the delta mapping and the
 *   FP32 Gram, and not in MMGaP-E,
 *   mod_bits in {2, 4, 6} (QPSK, 16-QAM, 64-QAM; symbol index q maps to the
 *   lattice point (2 (q / sqrt(M)) - L) + i (2 (q % sqrt(M)) - L),
 *   L = sqrt(M) - 1, scaled by 1/sqrt(2 (M - 1) / 3)).
 *   H:         complex [n_chan][n_r][n_t]
 *   chan_index: int32 [n_problems], channel of each problem; NULL = identity
 *              (then n_chan >= n_problems)
 *   y:         complex [n_problems][n_r]
 *   noise_var: float [n_problems], noise variance per receive antenna
 *              (rho of Eq. 3 with unit symbol energy)
 *   seed:      Philox4x32-10 key; problem k of the job draws from counter
 *              space (., run, problem_offset + k).
 *   problem_offset: index of the job's problem 0 in that counter space; 0 for
 *              a whole job.  A job cut into shards (contiguous PRB ranges of
 *              one slot on several GPUs, Sec. 3.2) gives each shard the index
 *              of its first problem, and the shards' results then equal the
 *              whole job's bit for bit.
 * Outputs (NULL = not wanted, except sym_out):
 *   sym_out:    uint8 [n_problems][n_t] detected QAM symbol indices
 *   energy_out: int32 [n_problems] selected quantised energy (<= 0; 0 = guess)
 *   guess_out:  int8 [n_problems][2 n_t] MMSE lattice guess (re block, im block)
 *   offset_out: int8 [n_problems][2 n_t] selected offset d in {-1, 0, 1}
 *   ndiv_out:   int32 [n_problems] diverged anneals
 *   steps_out:  int32 [n_problems] Euler steps the problem's anneals took
 *               (params->steps unless early exit stopped them)
 * guess_in: int8 [n_problems][2 n_t] (re block, im block) lattice guess that
 *   replaces the MMSE guess (Sec. 3.2: the guess is an input of the
 *   pre-processing); NULL = MMSE.  Each entry must be an alphabet point, odd
 *   with |g| <= sqrt(M) - 1; the builder sets bit 2 of the device error word
 *   for any other value (the problem is built around it as given).  Honoured
 *   by mmgap_detect, mmgap_build_detect, mmgap_detect_static, the batch and
 *   the server with the delta mapping; refused (MMGAP_EUNSUPPORTED) with the
 *   direct mapping and by mmgap_detect_e (which makes its own guesses).
 * gram_precision: 0 = FP32 Gram in the fixed operation order (bit-exact
 *   against the CPU oracle); 1 = BF16, 2 = FP16 and 3 = split BF16 (each
 *   operand as bf16 hi + bf16 lo, products hi*hi + hi*lo + lo*hi) on tensor
 *   cores with FP32 accumulation (a precision variant of the Sec. 3.2
 *   pre-processing: per element |dG_ij| <= (2u + u^2 + 2 n_r 2^-24)
 *   sum_k |Hs_ki| |Hs_kj|, u = 2^-8 for BF16, 2^-11 for FP16, 2^-15 for the
 *   split form; the matched filter, MMSE, field and quantisation stay FP32).
 *   Only mmgap_detect and mmgap_build_detect accept 1-3.
 * mapping: how a problem becomes an Ising problem.
 *   MMGAP_MAPPING_DELTA (0): the paper's delta form (Sec. 2.3, Sec. 3.2.1):
 *     2 n_t spin pairs plus an auxiliary spin around the MMSE guess.
 *   MMGAP_MAPPING_DIRECT (1): the binary-weighted form of earlier Ising
 *     detectors (no counterpart formula in the paper): each real dimension
 *     x = sum_b 2^b s_b over B = mod_bits / 2 spins, N = 2 n_t B spins plus an
 *     auxiliary one; J = -(T^T G T) with zero diagonal, c = T^T Hs^T y
 *     (G, Hs^T y: the FP32 Gram and matched filter of the delta build),
 *     quantised like the delta form; annealed by the same CIM-CAC steps with
 *     the full N x N field, scored by the exact energy -s^T Jq s - 2 cq^T s
 *     with the MMSE guess as the reference candidate (it wins ties).
 *     n_t in {4, 8, 16}, gram_precision 0, runs a multiple of 32 with
 *     runs <= 256 / TPA (TPA = 1 for N <= 32, 2 for N <= 64, 4 for N = 96).
 *     Outputs: sym_out; energy_out the selected candidate's energy;
 *     guess_out the MMSE guess; offset_out (x - g) / 2 per real dimension;
 *     ndiv_out.  Only mmgap_detect and mmgap_build_detect accept it.
 */
enum { MMGAP_MAPPING_DELTA = 0, MMGAP_MAPPING_DIRECT = 1 };
typedef struct {
    int32_t n_r, n_t, mod_bits;
    int32_t n_problems, n_chan;
    const int32_t* chan_index;
    const float* H;
    const float* y;
    const float* noise_var;
    uint64_t seed;
    uint8_t* sym_out;
    int32_t* energy_out;
    int8_t* guess_out;
    int8_t* offset_out;
    int32_t* ndiv_out;
    int32_t gram_precision;
    int32_t mapping;
    const int8_t* guess_in;
    int32_t* steps_out;
    uint64_t problem_offset;
} mmgap_detect_job;

/*
 * One downlink VPP job (Sec. 2.2, Sec. 3.3): n_u users, n_t antennas.
 *   n_u in {1, 2, 3, 4, 8, 16}, n_t in [n_u, 64], mod_bits in {2, 4, 6}.
 *   H:     complex [n_chan][n_u][n_t] (users' channels)
 *   chan_index: as above
 *   u_sym: uint8 [n_problems][n_u] intended QAM symbol indices
 *   seed:  as above
 * Outputs:
 *   v_out:      int8 [n_problems][n_u][2] Gaussian-integer perturbation
 *               (re, im), each in {-1, 0, 1}
 *   x_out:      complex [n_problems][n_t] transmit vector W (u + tau v),
 *               unnormalised (Eq. 6 scales it to power P); may be NULL
 *   power_out:  float [n_problems] ||W (u + tau v)||^2; may be NULL
 *   energy_out, ndiv_out: as for detection; may be NULL
 *   inv_precision: how Q = (H H^H)^-1 is computed, see mmgap_vpp_inverse:
 *               MMGAP_INV_FP64 (0) or MMGAP_INV_FP32_IR (1)
 * tau = 2 sqrt(M) in lattice units (2 (c_max + Delta / 2), Delta = 2).
 * W = H^H (H H^H)^-1 (Eq. 5) is formed through Q = (H H^H)^-1.
 */
typedef struct {
    int32_t n_u, n_t, mod_bits;
    int32_t n_problems, n_chan;
    int32_t inv_precision;
    const int32_t* chan_index;
    const float* H;
    const uint8_t* u_sym;
    uint64_t seed;
    int8_t* v_out;
    float* x_out;
    float* power_out;
    int32_t* energy_out;
    int32_t* ndiv_out;
} mmgap_precode_job;

/* Fill *p with the library defaults: runs 32, steps 200, f_mvm 2, dt 0.02,
 * p 1.2, a 1.0, zeta 3.0, eps 0.5, sigma0 0.1, x_max 1000, early_exit 0.
 * p/a/zeta/eps were chosen on the CPU oracle (the paper does not print them). */
mmgap_status mmgap_default_params(mmgap_params* p);

/* Create a context on CUDA device `device` owning `workspace_bytes` of device
 * memory (0 = 256 MiB) for per-problem Ising coefficients.  Jobs larger than
 * the workspace are processed in chunks.  *ctx = NULL on failure. */
mmgap_status mmgap_create(mmgap_ctx** ctx, int device, size_t workspace_bytes);

/* Destroy a context and free its workspace.  Synchronises the device first.
 * NULL is accepted. */
mmgap_status mmgap_destroy(mmgap_ctx* ctx);

/* Message describing the last error on this context ("" if none).  Owned by
 * the context; valid until the next call on it. */
const char* mmgap_last_error(const mmgap_ctx* ctx);

/* Uplink MIMO detection (Sec. 3.2): for each job, build the delta-Ising
 * problem of every resource element around its MMSE guess, run
 * params->runs anneals, keep the lowest-energy candidate (the guess if no
 * anneal is better) and decode it to symbols. */
mmgap_status mmgap_detect(mmgap_ctx* ctx, const mmgap_params* params, const mmgap_detect_job* jobs, int n_jobs,
                          void* stream);

/*
 * MMGaP-E (Sec. 3.2.2): multi-stage, multi-seed uplink detection.  For each
 * problem two delta-Ising instances are solved per stage: instance 0 around
 * the MMSE guess, instance 1 around an MMSE-SIC guess (the Cholesky of
 * H^H H + rho I pivoted on the smallest current Schur diagonal, back
 * substitution with each symbol sliced before it is cancelled); in each later
 * stage an instance is rebuilt around its own previous solution.  Stage s,
 * instance i anneals with Philox key seed + (2 (s - 1) + i) 0x9E3779B97F4A7C15.
 * The output is the candidate with the lowest FP32 ML objective ||y - Hs x||^2
 * (ties: first) among [MMSE guess, SIC guess, stage-1 solutions (instance 0,
 * 1), stage-2 solutions, ...].
 *   stages in [1, 8]; job outputs used: sym_out (required); other job
 *   outputs are ignored.
 *   best_out: int32 [P] index of the chosen candidate (may be NULL)
 *   obj_out:  float [P] its objective (may be NULL)
 *   cand_out: int8 [2 + 2 stages][P][2 n_t] every candidate (may be NULL)
 */
mmgap_status mmgap_detect_e(mmgap_ctx* ctx, const mmgap_params* params, const mmgap_detect_job* job, int stages,
                            int32_t* best_out, float* obj_out, int8_t* cand_out, void* stream);

/* Downlink vector-perturbation precoding (Sec. 3.3): the same solver on the
 * detection form y~ = W u, H_p = -tau W / 2, guess 0. */
mmgap_status mmgap_precode(mmgap_ctx* ctx, const mmgap_params* params, const mmgap_precode_job* jobs, int n_jobs,
                           void* stream);

/*
 * Solver boundary (Sec. 2.3, Sec. 3.2): anneal n_problems quantised
 * delta-Ising problems of half-size n (2n + 1 spins, n = 2 n_t,
 * n in {2, 4, 6, 8, 16, 32, 64}).
 *   A_q: int16 [n_problems][n][n] symmetric Q14 half-size block A = -G
 *        (Fig. 5(a): J = [[A~, A, b], [A, A~, b], [b^T, b^T, 0]])
 *   h_q: int16 [n_problems][n] Q14 auxiliary block b
 *   g:   int8 [n_problems][n] lattice guess, or NULL (then level_max must be 0)
 *   level_max: offsets d_i with |g_i + 2 d_i| > level_max are set to 0
 *              before scoring (0 = no clipping)
 *   seed: Philox key; problem k draws from counter space (., run, k).
 * Outputs: d_out int8 [n_problems][n] (required), E_out int32 [n_problems],
 * run_out int32 [n_problems] (index of the winning anneal), ndiv_out int32
 * [n_problems]; the last three may be NULL.
 */
mmgap_status mmgap_solve_ising(mmgap_ctx* ctx, const mmgap_params* params, int n, int n_problems,
                               const int16_t* A_q, const int16_t* h_q, const int8_t* g, int level_max, uint64_t seed,
                               int8_t* d_out, int32_t* E_out, int32_t* run_out, int32_t* ndiv_out, void* stream);

/*
 * Integration study boundary (Appendix A): anneal n_problems quantised
 * problems exactly as mmgap_solve_ising (no clipping, one-thread-per-anneal
 * kernel) and return every anneal's final state instead of the selection:
 * spins_out uint64 [n_problems][runs][2], word 0 bit q (q < 64) and word 1
 * bit q - 64 set iff x_q >= 0 at the end (spin order x1, x2, x_a), word 1
 * bit 63 set iff the anneal diverged.  P_diverge and P_error of the paper's
 * (dt, f_mvm) study follow from comparing these words across parameter sets
 * with equal N_I dt.  Uses the workspace for the discarded selection.
 * n in {2, 4, 6, 8, 16, 32}: n = 64 is refused with MMGAP_EUNSUPPORTED, since
 * its 129 spins do not fit the 127 state bits of the two words.
 */
mmgap_status mmgap_anneal_spins(mmgap_ctx* ctx, const mmgap_params* params, int n, int n_problems,
                                const int16_t* A_q, const int16_t* h_q, uint64_t seed, uint64_t* spins_out,
                                void* stream);

/*
 * Channel inverse of VPP (Sec. 2.2, Eq. 5): Q_c = (H_c H_c^H)^-1 for each of
 * n_chan channels H_c, complex [n_chan][n_u][n_t] (device), written to Q_out,
 * complex double [n_chan][n_u][n_u] (device, Hermitian).
 *   MMGAP_INV_FP64 (0): Cholesky and column solves in FP64.
 *   MMGAP_INV_FP32_IR (1): H H^H as an unevaluated double-FP32 sum, FP32
 *     Cholesky and solves, then up to 10 refinement steps X <- X + K^-1 (I - K X)
 *     with the residual as a compensated (double-FP32) sum, stopping when
 *     the remaining error (last correction squared over the one before) is
 *     predicted below 2^-40 max|X| or the corrections stall; a channel whose
 *     remaining error is not below 2^-24 max|X| is recomputed in FP64.  Accuracy per channel: max|Q - Q_exact| <= about
 *     (2^-44 kappa + 2^-28) max|Q| with kappa the condition number of H H^H.
 * H must be 8-byte and Q_out 16-byte aligned.
 * status_out (device int32 [n_chan]): 0, or 1 when H H^H is not positive
 * definite in FP64 (Q_c is then all zero); when NULL the flags go to the
 * context workspace.  n_u in {1, 2, 3, 4, 8, 16}, n_t in [n_u, 64].
 */
enum { MMGAP_INV_FP64 = 0, MMGAP_INV_FP32_IR = 1 };
mmgap_status mmgap_vpp_inverse(mmgap_ctx* ctx, int n_u, int n_t, int n_chan, const float* H, int inv_precision,
                               double* Q_out, int32_t* status_out, void* stream);

/*
 * Builder boundary (Sec. 3.2 pre-processing, Eq. 3, Fig. 5): the delta-Ising
 * coefficients of one detection job, without solving.
 * Outputs (device): A_q int16 [P][n][n], h_q int16 [P][n], g int8 [P][n]
 * (required); optional G_out float [P][n][n] and h_out float [P][n] (real-form
 * Gram and field in lattice units before quantisation), sigma_exp_out int32
 * [P] (normaliser 2^sigma_exp).  job->sym_out etc. are ignored.
 * With job->mapping == MMGAP_MAPPING_DIRECT the same pointers receive the
 * direct form: A_q = J_q [P][N][N], h_q = c_q [P][N], g = the MMSE guess
 * [P][2 n_t], G_out = J [P][N][N], h_out = c [P][N] (before quantisation).
 */
mmgap_status mmgap_build_detect(mmgap_ctx* ctx, const mmgap_detect_job* job, int16_t* A_q_out, int16_t* h_q_out,
                                int8_t* g_out, float* G_out, float* h_out, int32_t* sigma_exp_out, void* stream);

/*
 * General Ising boundary (the direct mapping's solver): P problems of N
 * spins plus an auxiliary spin, J_q int16 [P][N][N] (symmetric, zero
 * diagonal) and c_q int16 [P][N] (coupled through the auxiliary spin),
 * annealed with params->runs CIM-CAC anneals (Eqs. 10-11, couplings
 * J_q 2^-14, spin k of anneal r initialised from Philox word k mod 4 of
 * counter (k/4, r, problem), k = N the auxiliary spin).  Each anneal's
 * spins s_i = sign(x_i) sign(x_a) are scored by E(s) = -s^T J_q s - 2 c_q^T s
 * (exact int32); a diverged anneal is not a candidate.  s_ref int8 [P][N]
 * (may be NULL) is a reference candidate that wins ties; the result is the
 * lowest (E, candidate) (run -1 = the reference, or all +1 when there is no
 * reference and every anneal diverged).
 * N in {8, 16, 24, 32, 48, 64, 96}; runs as for the direct mapping.
 * Outputs (device): s_out int8 [P][N], E_out, run_out, ndiv_out int32 [P]
 * (each may be NULL except s_out).  Uses no workspace.
 */
mmgap_status mmgap_solve_general(mmgap_ctx* ctx, const mmgap_params* params, int N, int n_problems,
                                 const int16_t* J_q, const int16_t* c_q, const int8_t* s_ref, uint64_t seed,
                                 int8_t* s_out, int32_t* E_out, int32_t* run_out, int32_t* ndiv_out, void* stream);

/* Enable (1) or disable (0) per-stage CUDA-event timing of later detect /
 * precode calls on this context. */
mmgap_status mmgap_set_timing(mmgap_ctx* ctx, int enable);

/* Device time in ms of each stage of the last timed detect / precode call,
 * summed over its chunks: ms_out[0] build, [1] solve, [2] output
 * (precode only; 0 for detect), [3] whole call.  Synchronises on the call's
 * events.  *n_chunks_out (may be NULL) receives the number of chunks. */
mmgap_status mmgap_stage_times(mmgap_ctx* ctx, float ms_out[4], int* n_chunks_out);

/* Limit, in ns, of every bounded wait inside this context's kernels: the
 * waits of solver shape 8 for its tensor-core product (an MMA that takes
 * microseconds).  Default 200,000,000 (0.2 s).  0 makes each wait give up at
 * once unless the product is already complete.  A wait that gives up makes
 * the CTA return its problems' guesses with every anneal counted as diverged
 * and set bit 1 of the device error word; the CTA still waits (bounded, 0.2 s)
 * for its product in flight before it frees its tensor memory, so the
 * context stays usable.  Applies to later calls on the context. */
mmgap_status mmgap_set_device_wait(mmgap_ctx* ctx, uint64_t limit_ns);

/* Device-side error word of this context (bit 0: a channel index outside
 * [0, n_chan) was met; the problem was computed as all-zero couplings;
 * bit 1: a wait of solver shape 8 on its tensor-core product expired; the
 * problems of that CTA returned their guesses with every anneal counted as
 * diverged; bit 2: a caller-supplied guess (guess_in) held a value that is
 * not an alphabet point).
 * Synchronises the device; clears the word if `clear` is non-zero. */
mmgap_status mmgap_device_errors(mmgap_ctx* ctx, int* flags_out, int clear);

/*
 * Launch shape of the CIM-CAC solver for n_t users (no counterpart in the
 * paper, which runs one thread per anneal).  Shapes 0-4, 6, 9 and 10 give
 * bit-identical results; they differ only in speed:
 *   0 default for the size and the call: calls of at most one problem per
 *     SM run 10 (16 users) or 9 (8 users), of at most two per SM 4, larger
 *     calls 6 (16 users) or 3 (4 and 8 users; 4 users always), 1 elsewhere
 *   1 plain: one thread per anneal, scalar FP32 (the paper's design point)
 *   2 tuned kernel, one thread per anneal, scalar FP32
 *   3 tuned kernel, one thread per anneal, packed FP32 pairs
 *   4 tuned kernel, two threads per anneal (shuffle-gathered field), packed
 *   6 tuned kernel, one thread per anneal, packed, the field refresh shared
 *     by lane pairs (each coupling read once for two anneals)
 *   9 tuned kernel, four threads per anneal, packed (n_t 8 and 16; 4 runs 4)
 *  10 tuned kernel, eight threads per anneal, packed (n_t 16; 8 runs 9,
 *     4 runs 4) -- shapes for latency, when few problems leave SMs idle;
 *     with at most a quarter (half) as many problems as SMs, each problem
 *     runs as a cluster of 4 (2) CTAs with a quarter (half) of its anneals
 *     each (the same results)
 * Shapes 2-4, 6, 9 and 10 exist for n_t in {4, 8, 16} with f_mvm in {1, 2};
 * elsewhere 1 runs.  Shape 5 is a precision variant, not bit-identical: shape 3 with
 * the coupling field of a warp's 32 anneals computed on the tensor cores
 * (mma.sync m16n8k16, couplings and u split into FP16 pairs, FP32
 * accumulation; about 2^-21 of sum |A||u| from the FP32 field), for n_t in
 * {8, 16} (MMGAP_EUNSUPPORTED otherwise); shape 7 is the same refresh with
 * two threads per anneal (half the registers per thread; b^T u summed as two
 * halves, so not bit-identical to shape 5 either).  Shape 8 forms the same
 * FP16-split product with tcgen05 MMAs (Blackwell fifth-generation tensor
 * cores): CTAs of 128 anneals (128 / runs problems), the product's FP32
 * accumulator in tensor memory, read back by each anneal's thread; n_t in
 * {8, 16} (runs = 96 runs shape 5).  The autotuner never picks 5, 7 or 8.
 * The choice is per context and applies to detect, precode and solve_ising
 * calls.
 */
mmgap_status mmgap_set_solver_variant(mmgap_ctx* ctx, int n_t, int variant);

/* The shape a large call (more than two problems per SM) with n_t users and
 * refresh period f_mvm would run. */
mmgap_status mmgap_get_solver_variant(mmgap_ctx* ctx, int n_t, int f_mvm, int* variant_out);

/*
 * Autotuner: time every compiled bit-identical solver shape (1-4, 6, 9, 10) for
 * n_t users on n_problems random Q14 problems (0 = 8192; clamped to the
 * workspace) with *params, keep the fastest for this context and return it
 * in *variant_out.
 * ms_out (may be NULL, else 16 floats) receives [0] the best time and [v] the
 * time of shape v (-1 if not compiled or not bit-identical).  Synchronises the device; uses the workspace.
 */
mmgap_status mmgap_autotune(mmgap_ctx* ctx, const mmgap_params* params, int n_t, int n_problems, int* variant_out,
                            float ms_out[16]);

/*
 * Batched launch of mixed-size uplink jobs (no counterpart in the paper,
 * which launches one fixed-size grid per kernel).
 *
 * mmgap_batch_create validates the jobs (n_t in {4, 8, 16, 32}, n_r <= 64,
 * runs = 32, f_mvm in {1, 2}) and uploads a job table (largest users first).
 * 32-user jobs stay out of the table: each run launches their builder and
 * row-block solver (the kernels mmgap_detect uses for 32 users) ahead of the
 * table's kernels, outside the graph, always exact (MMGAP_BATCH_TENSOR_CORE
 * applies to the table's jobs).
 * A run is one builder kernel over every problem of every job (the Sec. 3.2
 * pre-processing, one warp per resource element) into batch-owned scratch,
 * then one solver kernel that anneals each problem with 32 anneals on the 32
 * lanes of a warp (solver and post-processing), one 32-thread CTA per problem
 * across all jobs (the hardware CTA scheduler balances the sizes).  Outputs
 * equal mmgap_detect's bit for bit.  A problem's Philox stream, and so its
 * result, depends only on its job's seed and problem_offset and its index in
 * its job.  flags: 0, or MMGAP_BATCH_TENSOR_CORE; other bits: MMGAP_EINVAL.
 * Job arrays are the caller's device memory and must stay valid for the life
 * of the batch; their contents may change between runs.  The batch owns a
 * small device table (allocated at create).
 * mmgap_batch_run enqueues the whole batch on `stream` as one kernel launch;
 * with use_graph != 0 the first run captures the launch into a CUDA graph (on
 * a private stream) and this and later runs launch the graph on `stream`.
 */
typedef struct mmgap_batch mmgap_batch;
#define MMGAP_BATCH_TENSOR_CORE 2 /* flags: tcgen05 field refresh for 8 and 16 users (solver shape 8: a
                                     precision variant, results as mmgap_detect with that shape; 128-thread
                                     CTAs over tiles of 4 problems of one job) */
mmgap_status mmgap_batch_create(mmgap_batch** batch, int device, const mmgap_params* params,
                                const mmgap_detect_job* jobs, int n_jobs, int flags);
mmgap_status mmgap_batch_run(mmgap_batch* batch, int use_graph, void* stream);
mmgap_status mmgap_batch_destroy(mmgap_batch* batch);

/*
 * Serving loop with continuous batching (no counterpart in the paper, which
 * times one batch; this is the slot-driven request path of a 5G receiver).
 *
 * Jobs are uplink detection jobs whose inputs are already on the device
 * (channel state can stay resident across slots) and whose outputs are the
 * caller's device memory; they must stay valid until the job completes.  A
 * dispatcher thread admits queued jobs in arrival order into launch groups:
 * a group goes to a free lane (a CUDA stream with its own job table and
 * coupling scratch of scratch_bytes / n_lanes) and takes jobs while they fit
 * that lane's scratch and limits (admission by memory).  Each group is one
 * batched launch (as mmgap_batch_run, replayed from a CUDA graph when
 * use_graph != 0); groups on different lanes overlap on the device, and jobs
 * that arrive while others run are admitted as soon as a lane frees up.
 * Precoding jobs (mmgap_server_submit_precode) share the groups: their
 * channel inverses and VPP builds run just before the group's batched launch,
 * their problems go through its solver, their outputs right after it.
 * Results equal mmgap_detect's / mmgap_precode's bit for bit, whatever the
 * grouping.
 * Latency = completion (host callback at the end of the group) - submission,
 * on the host's steady clock.  deadline_us > 0 counts jobs over it;
 * inject_delay_us > 0 delays every launch on the host (fault injection for
 * tests: a stalled dispatcher).  Limits as mmgap_batch_create (n_t in
 * {4, 8, 16, 32} up to max_n_t, n_r <= max_n_r, runs = 32, f_mvm in
 * {1, 2}); max_n_t in {4, 8, 16, 32}; precoding jobs up to 16 users.
 */
typedef struct mmgap_server mmgap_server;
typedef struct {
    int32_t n_lanes;                /* concurrent groups (streams), 1..16 */
    int32_t max_jobs_per_group;
    int64_t max_problems_per_group;
    size_t scratch_bytes;           /* device memory budget for coupling scratch, split across lanes */
    int32_t max_n_t, max_n_r;
    double deadline_us;
    double inject_delay_us;
    int32_t use_graph;
    int32_t tensor_core;            /* as MMGAP_BATCH_TENSOR_CORE (precision variant) */
} mmgap_server_config;
typedef struct {
    uint64_t ticket;
    int32_t status;                 /* MMGAP_OK when done */
    double submit_us, start_us, done_us;
} mmgap_job_info;
typedef struct {
    int64_t completed, problems, deadline_misses, groups, max_group_jobs, queued;
    double p50_us, p99_us, max_us, mean_us, span_us;  /* latency percentiles; span = first submit .. last done */
} mmgap_serve_stats;

mmgap_status mmgap_server_create(mmgap_server** server, int device, const mmgap_params* params,
                                 const mmgap_server_config* config);
/* Queue a job (non-blocking).  MMGAP_ENOMEM if it could never fit a lane. */
mmgap_status mmgap_server_submit(mmgap_server* server, const mmgap_detect_job* job, uint64_t* ticket);
/* Queue a downlink VPP precoding job (non-blocking): n_u in {4, 8, 16} up to
 * max_n_t, n_t (antennas) up to 64, either inv_precision.  Its results equal
 * mmgap_precode's for the same job.  MMGAP_ENOMEM if it could never fit a
 * lane (its scratch adds n_chan n_u^2 16 bytes of channel inverses). */
mmgap_status mmgap_server_submit_precode(mmgap_server* server, const mmgap_precode_job* job, uint64_t* ticket);
/* Wait for a job (timeout_us < 0: forever).  MMGAP_ETIMEOUT if not done in
 * time (the job stays queued or running; wait again).  On completion the
 * ticket is released and *info (may be NULL) gets its timestamps. */
mmgap_status mmgap_server_wait(mmgap_server* server, uint64_t ticket, int64_t timeout_us, mmgap_job_info* info);
/* Statistics of completed jobs since creation or the last reset. */
mmgap_status mmgap_server_stats(mmgap_server* server, mmgap_serve_stats* out, int reset);
/* Finish queued and running jobs, then stop and free the server. */
mmgap_status mmgap_server_destroy(mmgap_server* server);

/*
 * Uplink detection that allocates nothing (no counterpart in the paper; this
 * is a service to callers that cannot allocate device memory: a running
 * real-time slot loop, where cudaMalloc may synchronise the device and miss
 * the slot, or a plug-in inside an application that owns all device memory).
 *
 * Computes exactly what mmgap_detect computes for one job, without a
 * context: the scratch between the build and solve kernels comes from an
 * 8 MiB array compiled into the library (every GPU that loads the library
 * holds it until the process exits; with CUDA's lazy module loading the
 * memory is taken on the first call on each device).  Inputs and outputs are
 * the caller's device memory, as for mmgap_detect; the call runs on the
 * current device.  guess_in, steps_out and params->early_exit (up to 16 users)
 * are honoured as by mmgap_detect.
 *
 * Limit: the job must fit the array, i.e. align256(P n^2 2) + align256(P n 2)
 * + align256(P n) <= 8 MiB with n = 2 n_t (about 1,000 problems of 32 users, 3,900 of 16 users,
 * 14,900 of 8 users); a larger job returns MMGAP_ENOMEM (with a message on
 * stderr) and launches nothing.  Split it.
 * The first call on a device looks up the array's device address and the
 * device's SM count (with that device current); make that first call before
 * any stream capture.
 * Every call shares the one array, which keeps the last call's contents (each
 * call writes every byte it reads before reading it), so calls whose work
 * overlaps on the GPU (other streams, other host threads) race: serialise
 * them.  A channel index out of range gives an all-zero problem, as for
 * mmgap_detect, but is not reported (there is no error word).
 * Returns MMGAP_EINVAL / MMGAP_EUNSUPPORTED for bad arguments, MMGAP_ECUDA
 * for a CUDA error.
 */
mmgap_status mmgap_detect_static(const mmgap_params* params, const mmgap_detect_job* job, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MMGAP_H */
