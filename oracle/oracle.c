/*
 * CPU oracle for the MMGaP hot path (Singh & Jamieson, "MMGaP: Multi-User MIMO
 * Detection and Precoding using GPU-assisted Physics-inspired Computation").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product path (the
 * CUDA library and its Python binding) never calls it; the two share no code.
 *
 * Plain, slow, single-threaded C.  Two layers:
 *
 *   1. FP64 "truth": the plain definitions of the system model (Sec. 2.1,
 *      Eqs. 1-3), the delta-Ising mapping (Sec. 2.3 Eq. 9, Sec. 3.2.1), the
 *      exhaustive ML detector (Eq. 2), the brute-force Ising minimum and the
 *      downlink inverse (Sec. 2.2 Eq. 5).  These pin the layer below.
 *
 *   2. FP32 "mirror": the same method computed in the precision the GPU path
 *      computes in, with every floating-point operation (each fused
 *      multiply-add, multiply, add, divide, square root and rounding) taken in
 *      the plain sequential loop order written below.  Spins, lattice guesses
 *      and quantised couplings are integers decided by floating point; both
 *      sides take those decisions in the same precision and order, so the GPU
 *      path must reproduce this layer bit for bit.
 *
 * Compile with -ffp-contract=off (no implicit contraction of a*b+c) and without
 * -ffast-math; fmaf()/fma() are the only fused operations.
 *
 * The CIM-CAC trajectory (Eqs. 10-11 under the forward Euler reading) has no
 * worked example in the paper.  It is pinned by closed forms (eps = 0
 * decoupled dynamics), the dense-J identity of the half-size coupling field
 * (Fig. 5), an FP64 integration of Eqs. 10-11 over short anneals (error
 * bound) and statistical behaviour; beyond short horizons the FP32 trajectory
 * has no independent reference.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENUM 2 /* non-finite / not positive definite */

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC'11).  Counter-based: out = bijection_key(counter).    */
/* ------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { /* Weyl key schedule between rounds */
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------- */
/* Constellation (Sec. 2.1: x drawn from a square QAM alphabet Omega).        */
/* Lattice units: each real dimension takes {-L,...,-1,1,...,L}, L=sqrt(M)-1, */
/* physical symbol = kappa * lattice point with E|x|^2 = 1.                   */
/* ------------------------------------------------------------------------- */
int orc_qam_side(int mod_bits) { return 1 << (mod_bits / 2); } /* sqrt(M) */

int orc_qam_level_max(int mod_bits) { return orc_qam_side(mod_bits) - 1; }

double orc_qam_kappa(int mod_bits)
{
    double M = (double)(1 << mod_bits);
    return 1.0 / sqrt(2.0 * (M - 1.0) / 3.0);
}

/* ========================================================================= */
/* Layer 1: FP64 truth                                                       */
/* ========================================================================= */

/* Complex helpers on interleaved (re, im) doubles. */
typedef struct { double re, im; } cd;
static cd cd_ld(const double* p) { cd z = {p[0], p[1]}; return z; }
static cd cd_mul(cd a, cd b) { cd z = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; return z; }
static cd cd_cmul(cd a, cd b) /* conj(a) * b */ { cd z = {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re}; return z; }
static cd cd_add(cd a, cd b) { cd z = {a.re + b.re, a.im + b.im}; return z; }
static cd cd_sub(cd a, cd b) { cd z = {a.re - b.re, a.im - b.im}; return z; }
static cd cd_scale(cd a, double s) { cd z = {a.re * s, a.im * s}; return z; }

/* Hermitian positive-definite solve B x = b by Cholesky (FP64, plain). */
static int chol64(int n, cd* B /* n*n, overwritten by L */)
{
    for (int j = 0; j < n; ++j) {
        double d = B[j * n + j].re;
        for (int k = 0; k < j; ++k) d -= B[j * n + k].re * B[j * n + k].re + B[j * n + k].im * B[j * n + k].im;
        if (!(d > 0.0)) return ORC_ENUM;
        double ljj = sqrt(d);
        B[j * n + j].re = ljj;
        B[j * n + j].im = 0.0;
        for (int i = j + 1; i < n; ++i) {
            cd acc = B[i * n + j];
            for (int k = 0; k < j; ++k) acc = cd_sub(acc, cd_mul(B[i * n + k], (cd){B[j * n + k].re, -B[j * n + k].im}));
            B[i * n + j] = cd_scale(acc, 1.0 / ljj);
        }
    }
    return ORC_OK;
}

static void cholsolve64(int n, const cd* L, const cd* b, cd* x)
{
    cd* w = (cd*)malloc(sizeof(cd) * (size_t)n);
    for (int i = 0; i < n; ++i) {
        cd acc = b[i];
        for (int k = 0; k < i; ++k) acc = cd_sub(acc, cd_mul(L[i * n + k], w[k]));
        w[i] = cd_scale(acc, 1.0 / L[i * n + i].re);
    }
    for (int i = n - 1; i >= 0; --i) {
        cd acc = w[i];
        for (int k = i + 1; k < n; ++k) acc = cd_sub(acc, cd_cmul(L[k * n + i], x[k]));
        x[i] = cd_scale(acc, 1.0 / L[i * n + i].re);
    }
    free(w);
}

/*
 * Delta-Ising problem of one uplink detection problem, FP64 (Sec. 2.1 Eqs. 1-3,
 * Sec. 2.3 Eq. 9, Sec. 3.2.1).
 *
 *   Hs = kappa H (lattice units), G_c = Hs^H Hs, m = Hs^H y,
 *   x_mmse = (G_c + rho I)^-1 m with rho = noise_var * kappa^2 (Eq. 3 in
 *   lattice units: E|x_lat|^2 = 1/kappa^2), guess g = nearest odd lattice point
 *   of x_mmse per real dimension clipped to +-L (ties upward) unless g_in given,
 *   z = y - Hs g, h_c = Hs^H z,
 *   real form: G = [[Re G_c, -Im G_c], [Im G_c, Re G_c]], h = [Re h_c; Im h_c].
 *
 * The Ising coupling blocks of Fig. 5 are A = -G (the half-size matrix) and
 * b = h (the auxiliary-spin vector): ||y - Hs(g + s_a(s1+s2))||^2 equals
 * -s^T J s + ||z||^2 + 2 tr(G).
 *
 * H: [n_r][n_t] complex, y: [n_r] complex (interleaved re, im).
 * Outputs (any may be NULL): x_mmse [2 n_t] (re block then im block),
 * g [2 n_t], G [n*n], h [n], znorm2.
 */
int orc_build_detect64(int n_r, int n_t, int mod_bits, const double* H, const double* y, double noise_var,
                       const int* g_in, double* x_mmse_out, int* g_out, double* G_out, double* h_out,
                       double* znorm2_out)
{
    if (n_r < 1 || n_t < 1 || mod_bits < 2 || (mod_bits & 1)) return ORC_EINVAL;
    const int n = 2 * n_t;
    const int Lmax = orc_qam_level_max(mod_bits);
    const double kappa = orc_qam_kappa(mod_bits);
    cd* Hs = (cd*)malloc(sizeof(cd) * (size_t)(n_r * n_t));
    cd* Gc = (cd*)malloc(sizeof(cd) * (size_t)(n_t * n_t));
    cd* B = (cd*)malloc(sizeof(cd) * (size_t)(n_t * n_t));
    cd* m = (cd*)malloc(sizeof(cd) * (size_t)n_t);
    cd* xm = (cd*)malloc(sizeof(cd) * (size_t)n_t);
    cd* z = (cd*)malloc(sizeof(cd) * (size_t)n_r);
    cd* hc = (cd*)malloc(sizeof(cd) * (size_t)n_t);
    int* g = (int*)malloc(sizeof(int) * (size_t)n);
    int status = ORC_OK;

    for (int k = 0; k < n_r; ++k)
        for (int i = 0; i < n_t; ++i) Hs[k * n_t + i] = cd_scale(cd_ld(H + 2 * (k * n_t + i)), kappa);
    for (int i = 0; i < n_t; ++i)
        for (int j = 0; j < n_t; ++j) {
            cd acc = {0.0, 0.0};
            for (int k = 0; k < n_r; ++k) acc = cd_add(acc, cd_cmul(Hs[k * n_t + i], Hs[k * n_t + j]));
            Gc[i * n_t + j] = acc;
        }
    for (int i = 0; i < n_t; ++i) {
        cd acc = {0.0, 0.0};
        for (int k = 0; k < n_r; ++k) acc = cd_add(acc, cd_cmul(Hs[k * n_t + i], cd_ld(y + 2 * k)));
        m[i] = acc;
    }
    double rho = noise_var * kappa * kappa;
    memcpy(B, Gc, sizeof(cd) * (size_t)(n_t * n_t));
    for (int i = 0; i < n_t; ++i) B[i * n_t + i].re += rho;
    if (chol64(n_t, B) == ORC_OK) {
        cholsolve64(n_t, B, m, xm);
    } else {
        for (int i = 0; i < n_t; ++i) xm[i] = (cd){0.0, 0.0};
        status = ORC_ENUM;
    }
    for (int i = 0; i < n_t; ++i) {
        if (x_mmse_out) {
            x_mmse_out[i] = xm[i].re;
            x_mmse_out[n_t + i] = xm[i].im;
        }
        double v[2] = {xm[i].re, xm[i].im};
        for (int c = 0; c < 2; ++c) {
            int gi;
            if (g_in) {
                gi = g_in[c * n_t + i];
            } else {
                double xc = v[c];
                if (!(xc >= -Lmax)) xc = -Lmax; /* also maps NaN to -L */
                if (xc > Lmax) xc = Lmax;
                gi = 2 * (int)floor(xc / 2.0) + 1;
            }
            g[c * n_t + i] = gi;
        }
    }
    for (int k = 0; k < n_r; ++k) {
        cd acc = cd_ld(y + 2 * k);
        for (int j = 0; j < n_t; ++j) acc = cd_sub(acc, cd_mul(Hs[k * n_t + j], (cd){(double)g[j], (double)g[n_t + j]}));
        z[k] = acc;
    }
    double zn = 0.0;
    for (int k = 0; k < n_r; ++k) zn += z[k].re * z[k].re + z[k].im * z[k].im;
    for (int i = 0; i < n_t; ++i) {
        cd acc = {0.0, 0.0};
        for (int k = 0; k < n_r; ++k) acc = cd_add(acc, cd_cmul(Hs[k * n_t + i], z[k]));
        hc[i] = acc;
    }
    if (G_out)
        for (int i = 0; i < n_t; ++i)
            for (int j = 0; j < n_t; ++j) {
                cd v = Gc[i * n_t + j];
                G_out[i * n + j] = v.re;
                G_out[i * n + (n_t + j)] = -v.im;
                G_out[(n_t + i) * n + j] = v.im;
                G_out[(n_t + i) * n + (n_t + j)] = v.re;
            }
    if (h_out)
        for (int i = 0; i < n_t; ++i) {
            h_out[i] = hc[i].re;
            h_out[n_t + i] = hc[i].im;
        }
    if (g_out) memcpy(g_out, g, sizeof(int) * (size_t)n);
    if (znorm2_out) *znorm2_out = zn;
    free(Hs); free(Gc); free(B); free(m); free(xm); free(z); free(hc); free(g);
    return status;
}

/* Dense (2n+1)x(2n+1) Ising matrix J = [[A~, A, b], [A, A~, b], [b^T, b^T, 0]]
 * with A = -G, A~ = A with zero diagonal, b = h (Sec. 3.2.1, Fig. 5(a)). */
void orc_dense_J(int n, const double* G, const double* h, double* J)
{
    const int N = 2 * n + 1;
    memset(J, 0, sizeof(double) * (size_t)(N * N));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double a = -G[i * n + j];
            J[i * N + (n + j)] = a;
            J[(n + i) * N + j] = a;
            if (i != j) {
                J[i * N + j] = a;
                J[(n + i) * N + (n + j)] = a;
            }
        }
    for (int i = 0; i < n; ++i) {
        J[i * N + 2 * n] = h[i];
        J[(n + i) * N + 2 * n] = h[i];
        J[2 * n * N + i] = h[i];
        J[2 * n * N + n + i] = h[i];
    }
}

/* Ising energy -s^T J s (Eq. 9). */
double orc_ising_energy(int N, const double* J, const int8_t* s)
{
    double e = 0.0;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) e += (double)s[i] * J[i * N + j] * (double)s[j];
    return -e;
}

/* ||y - Hs x||^2 for a lattice vector x (re block then im block). */
double orc_ml_objective(int n_r, int n_t, int mod_bits, const double* H, const double* y, const int* x)
{
    const double kappa = orc_qam_kappa(mod_bits);
    double e = 0.0;
    for (int k = 0; k < n_r; ++k) {
        cd acc = cd_ld(y + 2 * k);
        for (int j = 0; j < n_t; ++j)
            acc = cd_sub(acc, cd_mul(cd_scale(cd_ld(H + 2 * (k * n_t + j)), kappa), (cd){(double)x[j], (double)x[n_t + j]}));
        e += acc.re * acc.re + acc.im * acc.im;
    }
    return e;
}

/* Exhaustive maximum-likelihood detection over Omega^{n_t} (Eq. 2).  Returns
 * the minimum objective; x_out gets the lattice minimiser (first in
 * enumeration order on ties).  Cost M^{n_t}: small cases only. */
double orc_ml_exhaustive(int n_r, int n_t, int mod_bits, const double* H, const double* y, int* x_out)
{
    if (n_r < 1 || n_t < 1 || n_t > 16) return NAN;
    const int side = orc_qam_side(mod_bits);
    const int M = side * side;
    const int n = 2 * n_t;
    int* idx = (int*)calloc((size_t)n_t, sizeof(int));
    int* x = (int*)malloc(sizeof(int) * (size_t)n);
    double best = INFINITY;
    for (;;) {
        for (int i = 0; i < n_t; ++i) {
            x[i] = 2 * (idx[i] / side) - (side - 1);
            x[n_t + i] = 2 * (idx[i] % side) - (side - 1);
        }
        double e = orc_ml_objective(n_r, n_t, mod_bits, H, y, x);
        if (e < best) {
            best = e;
            memcpy(x_out, x, sizeof(int) * (size_t)n);
        }
        int i = 0;
        while (i < n_t && ++idx[i] == M) idx[i++] = 0;
        if (i == n_t) break;
    }
    free(idx);
    free(x);
    return best;
}

/* Brute-force ground state of -s^T J s over all 2^N spin vectors (N <= 24).
 * If g/level_max are given, only states whose decoded lattice point
 * g + s_a (s1 + s2) stays inside +-level_max are admitted. */
double orc_ising_bruteforce(int n, const double* J, const int* g, int level_max, int8_t* s_out)
{
    const int N = 2 * n + 1;
    int8_t* s = (int8_t*)malloc((size_t)N);
    double best = INFINITY;
    for (uint64_t code = 0; code < ((uint64_t)1 << N); ++code) {
        for (int k = 0; k < N; ++k) s[k] = (code >> k & 1) ? 1 : -1;
        if (g && level_max > 0) {
            int ok = 1;
            for (int i = 0; i < n && ok; ++i) {
                int xv = g[i] + s[2 * n] * (s[i] + s[n + i]);
                if (xv > level_max || xv < -level_max) ok = 0;
            }
            if (!ok) continue;
        }
        double e = orc_ising_energy(N, J, s);
        if (e < best) {
            best = e;
            memcpy(s_out, s, (size_t)N);
        }
    }
    free(s);
    return best;
}

/* ========================================================================= */
/* Layer 2: FP32 mirror (the GPU path's arithmetic, in this exact order)      */
/* ========================================================================= */

/* float helpers: every rounding is explicit */
static float f_mul(float a, float b) { return a * b; }
static float f_add(float a, float b) { return a + b; }

/* kappa, kappa^2 as FP32, rounded once from FP64 */
static float qam_kappa_f(int mod_bits) { return (float)orc_qam_kappa(mod_bits); }
static float qam_kappa2_f(int mod_bits)
{
    double M = (double)(1 << mod_bits);
    return (float)(1.0 / (2.0 * (M - 1.0) / 3.0));
}

/* 2^k as float for k in [-126, 127] (exact) */
static float pow2f(int k) { return ldexpf(1.0f, k); }

/* Exponent e of the power-of-two normaliser sigma = 2^e >= mx (Sec. 3.2.1 keeps
 * J on a fixed scale; the paper gives no rule, so sigma is the smallest power
 * of two not below the largest |coupling|).  mx == 0 or non-finite -> 0. */
static int sigma_exp_f(float mx)
{
    if (!(mx > 0.0f) || isinf(mx)) return 0;
    int E;
    float f = frexpf(mx, &E);
    return (f == 0.5f) ? E - 1 : E;
}

static int sigma_exp_d(double mx)
{
    if (!(mx > 0.0) || isinf(mx)) return 0;
    int E;
    double f = frexp(mx, &E);
    return (f == 0.5) ? E - 1 : E;
}

#define QBITS 14

/*
 * FP32 delta-Ising build of one uplink problem, in the pinned order.
 *
 * Inputs: H [n_r][n_t] complex float, y [n_r] complex float, noise_var.
 * g_in: optional externally supplied guess (lattice, [2 n_t]); NULL = MMSE.
 * Outputs: g [2 n_t] (int), G32 [n*n], h32 [n] (FP32 real-form Gram and field,
 * before quantisation), sigma_exp, Aq [n*n] = rint(-G / 2^e * 2^14),
 * hq [n] = rint(h / 2^e * 2^14).
 * Returns ORC_ENUM if the Cholesky pivot is not positive (then x_mmse := 0).
 *
 * Operation order (each line is one IEEE FP32 rounding):
 *   Hs_ki     = kappa * H_ki                                   (re, im)
 *   G_c ii    = sum_k fma(a.re, a.re), fma(a.im, a.im)     from 0, k ascending
 *   G_c ij i<j: re = fma(a.re,b.re), fma(a.im,b.im);  im = fma(a.re,b.im), fma(-a.im,b.re)
 *               (a = Hs_ki, b = Hs_kj, k ascending, from 0); G_c ji = conj(G_c ij)
 *   m_i       = same pattern as G_c ij with b = y_k
 *   B_ii      = G_c ii + rho  (rho = noise_var * kappa^2)
 *   Cholesky  left-looking, k ascending; L_jj = sqrt(B_jj - sum |L_jk|^2),
 *             L_ij = (B_ij - sum L_ik conj(L_jk)) / L_jj  (two real divides)
 *   forward   w_i = (m_i - sum_{k<i} L_ik w_k) / L_ii, k ascending
 *   backward  x_i = (w_i - sum_{k>i} conj(L_ki) x_k) / L_ii, k DESCENDING
 *   guess     g = 2 floor(clip(x, -L, L) * 0.5) + 1
 *   z_k       = y_k - sum_j Hs_kj g_j, j ascending
 *   h_c,i     = sum_k conj(Hs_ki) z_k, k ascending
 */
int orc_build_detect32(int n_r, int n_t, int mod_bits, const float* H, const float* y, float noise_var,
                       const int* g_in, int* g_out, float* G32_out, float* h32_out, int* sigma_exp_out,
                       int16_t* Aq_out, int16_t* hq_out)
{
    if (n_r < 1 || n_t < 1 || mod_bits < 2 || (mod_bits & 1)) return ORC_EINVAL;
    const int n = 2 * n_t;
    const int Lmax = orc_qam_level_max(mod_bits);
    const float kappa = qam_kappa_f(mod_bits);
    const float rho = f_mul(noise_var, qam_kappa2_f(mod_bits));
    float* Hs = (float*)malloc(sizeof(float) * 2 * (size_t)(n_r * n_t));
    float* Gc = (float*)malloc(sizeof(float) * 2 * (size_t)(n_t * n_t));
    float* Lc = (float*)malloc(sizeof(float) * 2 * (size_t)(n_t * n_t));
    float* m = (float*)malloc(sizeof(float) * 2 * (size_t)n_t);
    float* w = (float*)malloc(sizeof(float) * 2 * (size_t)n_t);
    float* xm = (float*)malloc(sizeof(float) * 2 * (size_t)n_t);
    float* z = (float*)malloc(sizeof(float) * 2 * (size_t)n_r);
    float* hc = (float*)malloc(sizeof(float) * 2 * (size_t)n_t);
    int* g = (int*)malloc(sizeof(int) * (size_t)n);
    float* G = (float*)malloc(sizeof(float) * (size_t)(n * n));
    float* h = (float*)malloc(sizeof(float) * (size_t)n);
    int status = ORC_OK;

    for (int e = 0; e < 2 * n_r * n_t; ++e) Hs[e] = f_mul(kappa, H[e]);

    /* Gram, upper triangle then Hermitian mirror */
    for (int i = 0; i < n_t; ++i) {
        float acc = 0.0f;
        for (int k = 0; k < n_r; ++k) {
            const float* a = Hs + 2 * (k * n_t + i);
            acc = fmaf(a[0], a[0], acc);
            acc = fmaf(a[1], a[1], acc);
        }
        Gc[2 * (i * n_t + i)] = acc;
        Gc[2 * (i * n_t + i) + 1] = 0.0f;
        for (int j = i + 1; j < n_t; ++j) {
            float re = 0.0f, im = 0.0f;
            for (int k = 0; k < n_r; ++k) {
                const float* a = Hs + 2 * (k * n_t + i);
                const float* b = Hs + 2 * (k * n_t + j);
                re = fmaf(a[0], b[0], re);
                re = fmaf(a[1], b[1], re);
                im = fmaf(a[0], b[1], im);
                im = fmaf(-a[1], b[0], im);
            }
            Gc[2 * (i * n_t + j)] = re;
            Gc[2 * (i * n_t + j) + 1] = im;
            Gc[2 * (j * n_t + i)] = re;
            Gc[2 * (j * n_t + i) + 1] = -im;
        }
    }
    /* matched filter m = Hs^H y */
    for (int i = 0; i < n_t; ++i) {
        float re = 0.0f, im = 0.0f;
        for (int k = 0; k < n_r; ++k) {
            const float* a = Hs + 2 * (k * n_t + i);
            const float* b = y + 2 * k;
            re = fmaf(a[0], b[0], re);
            re = fmaf(a[1], b[1], re);
            im = fmaf(a[0], b[1], im);
            im = fmaf(-a[1], b[0], im);
        }
        m[2 * i] = re;
        m[2 * i + 1] = im;
    }

    if (g_in) {
        memcpy(g, g_in, sizeof(int) * (size_t)n);
    } else {
        /* MMSE (Eq. 3): Cholesky of G_c + rho I, left-looking */
        int ok = 1;
        for (int j = 0; j < n_t && ok; ++j) {
            float d = f_add(Gc[2 * (j * n_t + j)], rho);
            for (int k = 0; k < j; ++k) {
                const float* l = Lc + 2 * (j * n_t + k);
                d = fmaf(-l[0], l[0], d);
                d = fmaf(-l[1], l[1], d);
            }
            if (!(d > 0.0f) || isinf(d)) { ok = 0; break; }
            float ljj = sqrtf(d);
            Lc[2 * (j * n_t + j)] = ljj;
            Lc[2 * (j * n_t + j) + 1] = 0.0f;
            for (int i = j + 1; i < n_t; ++i) {
                float re = Gc[2 * (i * n_t + j)], im = Gc[2 * (i * n_t + j) + 1];
                for (int k = 0; k < j; ++k) {
                    const float* a = Lc + 2 * (i * n_t + k); /* L_ik */
                    const float* b = Lc + 2 * (j * n_t + k); /* L_jk, used conjugated */
                    re = fmaf(-a[0], b[0], re);
                    re = fmaf(-a[1], b[1], re);
                    im = fmaf(-a[1], b[0], im);
                    im = fmaf(a[0], b[1], im);
                }
                Lc[2 * (i * n_t + j)] = re / ljj;
                Lc[2 * (i * n_t + j) + 1] = im / ljj;
            }
        }
        if (ok) {
            for (int i = 0; i < n_t; ++i) {
                float re = m[2 * i], im = m[2 * i + 1];
                for (int k = 0; k < i; ++k) {
                    const float* a = Lc + 2 * (i * n_t + k);
                    const float* b = w + 2 * k;
                    re = fmaf(-a[0], b[0], re);
                    re = fmaf(a[1], b[1], re);
                    im = fmaf(-a[0], b[1], im);
                    im = fmaf(-a[1], b[0], im);
                }
                float lii = Lc[2 * (i * n_t + i)];
                w[2 * i] = re / lii;
                w[2 * i + 1] = im / lii;
            }
            for (int i = n_t - 1; i >= 0; --i) {
                float re = w[2 * i], im = w[2 * i + 1];
                for (int k = n_t - 1; k > i; --k) {
                    const float* a = Lc + 2 * (k * n_t + i); /* L_ki, used conjugated */
                    const float* b = xm + 2 * k;
                    re = fmaf(-a[0], b[0], re);
                    re = fmaf(-a[1], b[1], re);
                    im = fmaf(-a[0], b[1], im);
                    im = fmaf(a[1], b[0], im);
                }
                float lii = Lc[2 * (i * n_t + i)];
                xm[2 * i] = re / lii;
                xm[2 * i + 1] = im / lii;
            }
        } else {
            for (int i = 0; i < 2 * n_t; ++i) xm[i] = 0.0f;
            status = ORC_ENUM;
        }
        for (int i = 0; i < n_t; ++i)
            for (int c = 0; c < 2; ++c) {
                float xc = xm[2 * i + c];
                xc = fmaxf(xc, (float)-Lmax); /* fmaxf(NaN, -L) = -L */
                xc = fminf(xc, (float)Lmax);
                g[c * n_t + i] = 2 * (int)floorf(f_mul(xc, 0.5f)) + 1;
            }
    }

    /* residual z = y - Hs g and field h_c = Hs^H z */
    for (int k = 0; k < n_r; ++k) {
        float re = y[2 * k], im = y[2 * k + 1];
        for (int j = 0; j < n_t; ++j) {
            const float* a = Hs + 2 * (k * n_t + j);
            float bre = (float)g[j], bim = (float)g[n_t + j];
            re = fmaf(-a[0], bre, re);
            re = fmaf(a[1], bim, re);
            im = fmaf(-a[0], bim, im);
            im = fmaf(-a[1], bre, im);
        }
        z[2 * k] = re;
        z[2 * k + 1] = im;
    }
    for (int i = 0; i < n_t; ++i) {
        float re = 0.0f, im = 0.0f;
        for (int k = 0; k < n_r; ++k) {
            const float* a = Hs + 2 * (k * n_t + i);
            const float* b = z + 2 * k;
            re = fmaf(a[0], b[0], re);
            re = fmaf(a[1], b[1], re);
            im = fmaf(a[0], b[1], im);
            im = fmaf(-a[1], b[0], im);
        }
        hc[2 * i] = re;
        hc[2 * i + 1] = im;
    }

    /* real form */
    for (int i = 0; i < n_t; ++i)
        for (int j = 0; j < n_t; ++j) {
            float re = Gc[2 * (i * n_t + j)], im = Gc[2 * (i * n_t + j) + 1];
            G[i * n + j] = re;
            G[i * n + (n_t + j)] = -im;
            G[(n_t + i) * n + j] = im;
            G[(n_t + i) * n + (n_t + j)] = re;
        }
    for (int i = 0; i < n_t; ++i) {
        h[i] = hc[2 * i];
        h[n_t + i] = hc[2 * i + 1];
    }

    /* normalise by a power of two and quantise to Q14 */
    float mx = 0.0f;
    for (int e = 0; e < n * n; ++e) mx = fmaxf(mx, fabsf(G[e]));
    for (int i = 0; i < n; ++i) mx = fmaxf(mx, fabsf(h[i]));
    int se = sigma_exp_f(mx);
    int finite = isfinite(mx);
    float s = pow2f(QBITS - se);
    for (int e = 0; e < n * n; ++e) Aq_out[e] = finite ? (int16_t)rintf(f_mul(-G[e], s)) : 0;
    for (int i = 0; i < n; ++i) hq_out[i] = finite ? (int16_t)rintf(f_mul(h[i], s)) : 0;
    if (!finite) status = ORC_ENUM;

    if (g_out) memcpy(g_out, g, sizeof(int) * (size_t)n);
    if (G32_out) memcpy(G32_out, G, sizeof(float) * (size_t)(n * n));
    if (h32_out) memcpy(h32_out, h, sizeof(float) * (size_t)n);
    if (sigma_exp_out) *sigma_exp_out = se;
    free(Hs); free(Gc); free(Lc); free(m); free(w); free(xm); free(z); free(hc); free(g); free(G); free(h);
    return status;
}

/* Quantise an FP64 real-form (G, h) exactly as the FP32 layer does (same
 * normaliser rule, round half to even); used to compare codes. */
void orc_quantise64(int n, const double* G, const double* h, int* sigma_exp_out, int32_t* Aq_out, int32_t* hq_out)
{
    double mx = 0.0;
    for (int e = 0; e < n * n; ++e) mx = fmax(mx, fabs(G[e]));
    for (int i = 0; i < n; ++i) mx = fmax(mx, fabs(h[i]));
    int se = sigma_exp_d(mx);
    double s = ldexp(1.0, QBITS - se);
    for (int e = 0; e < n * n; ++e) Aq_out[e] = (int32_t)rint(-G[e] * s);
    for (int i = 0; i < n; ++i) hq_out[i] = (int32_t)rint(h[i] * s);
    *sigma_exp_out = se;
}

/* ------------------------------------------------------------------------- */
/* Quantised Ising energy of a lattice offset d in {-1,0,1}^n (Sec. 3.2,      */
/* post-processing selects the lowest ML energy).                             */
/*   E(d) = d^T G_q d - h_q^T d with G_q = -A_q                               */
/* equals (||z - 2 Hs d||^2 - ||z||^2) * 2^14 / (4 sigma) up to quantisation. */
/* Exact int32 arithmetic.                                                    */
/* ------------------------------------------------------------------------- */
int32_t orc_energy_q(int n, const int16_t* Aq, const int16_t* hq, const int8_t* d)
{
    int32_t e = 0;
    for (int i = 0; i < n; ++i) {
        if (!d[i]) continue;
        int32_t r = 0;
        for (int j = 0; j < n; ++j) r += (int32_t)Aq[i * n + j] * (int32_t)d[j];
        e -= (int32_t)d[i] * r;
        e -= (int32_t)hq[i] * (int32_t)d[i];
    }
    return e;
}

/* ------------------------------------------------------------------------- */
/* CIM-CAC solver (Sec. 2.3 Eqs. 10-11; Sec. 3.2.1 MVM decomposition and      */
/* f_mvm; Sec. 3.2 anneals, MMSE fallback and post-processing).               */
/* ------------------------------------------------------------------------- */
typedef struct {
    int runs;     /* anneals per problem, N_a */
    int steps;    /* Euler steps per anneal, N_I */
    int f_mvm;    /* coupling refresh period */
    float dt;     /* Euler step */
    float p, a, zeta, eps; /* CIM-CAC parameters of Eqs. 10-11 */
    float sigma0; /* initial amplitudes uniform in [-sigma0, sigma0) */
    float x_max;  /* divergence bound on |x| at the end of an anneal */
    int early_exit; /* K > 0: stop a problem's anneals at the first K-th refresh
                       point where no spin sign of any of them changed since the
                       previous one (anneal_early_exit); 0 = off */
} orc_params;

typedef struct {
    float c1;  /* 1 + dt (p - 1) */
    float cdt; /* -dt */
    float cz;  /* -dt zeta */
    float c2;  /* 1 + dt zeta a */
    float ce;  /* eps dt, folded into the couplings */
    float xs;  /* sigma0 * 2^-23 */
} orc_consts;

/* Discretisation constants, each rounded once from FP64. */
void orc_cac_consts(const orc_params* P, orc_consts* C)
{
    double dt = (double)P->dt, p = (double)P->p, a = (double)P->a, zeta = (double)P->zeta, eps = (double)P->eps;
    C->c1 = (float)(1.0 + dt * (p - 1.0));
    C->cdt = (float)(-dt);
    C->cz = (float)(-(dt * zeta));
    C->c2 = (float)(1.0 + (dt * zeta) * a);
    C->ce = (float)(eps * dt);
    C->xs = (float)((double)P->sigma0 * 0x1p-23);
}

/* Initial amplitude of spin k of run r of problem `problem`: Philox word
 * (k mod 4) of counter (k/4, r, problem_lo, problem_hi) under key (seed_lo,
 * seed_hi); x0 = ((w >> 8) - 2^23) * sigma0 2^-23, uniform in [-sigma0, sigma0). */
float orc_initial_x(uint64_t seed, uint64_t problem, int run, int k, float xs)
{
    uint32_t ctr[4] = {(uint32_t)(k / 4), (uint32_t)run, (uint32_t)problem, (uint32_t)(problem >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    int32_t v = (int32_t)(out[k % 4] >> 8) - 8388608;
    return f_mul((float)v, xs);
}

/* Coupling field mu = J x of the state (x1, x2, x_a) through the half-size
 * decomposition of Fig. 5:  u = x1 + x2,  m = A u  (one half-size MVM),
 * mu_a = b^T u (one dot product), c = m + b x_a (scaling),
 * mu1 = c - diag(A) o x1, mu2 = c - diag(A) o x2 (element-wise products).
 * Af: [n][n] FP32 couplings, hf: [n]; x, mu: [2n+1].  The solver passes the
 * couplings pre-multiplied by eps dt, so mu is already eps dt J x. */
void orc_coupling_field(int n, const float* Af, const float* hf, const float* x, float* mu)
{
    float* macc = (float*)malloc(sizeof(float) * (size_t)n);
    for (int i = 0; i < n; ++i) macc[i] = 0.0f;
    float mua = 0.0f;
    for (int j = 0; j < n; ++j) {
        float u = f_add(x[j], x[n + j]);
        mua = fmaf(hf[j], u, mua);
        for (int i = 0; i < n; ++i) macc[i] = fmaf(Af[j * n + i], u, macc[i]);
    }
    const float xa = x[2 * n];
    for (int i = 0; i < n; ++i) {
        float c = fmaf(hf[i], xa, macc[i]);
        float nd = -Af[i * n + i];
        mu[i] = fmaf(nd, x[i], c);
        mu[n + i] = fmaf(nd, x[n + i], c);
    }
    mu[2 * n] = mua;
    free(macc);
}

/* One forward-Euler step of Eqs. 10-11 for one spin with frozen field
 * mu = eps dt (J x)_i:
 *   x' = x (1 + dt(p-1) - dt x^2) + e mu
 *   e' = e (1 + dt zeta a - dt zeta x^2)                                    */
static void euler_spin(float* x, float* eh, float mu, const orc_consts* C)
{
    float q = f_mul(*x, *x);
    float t = fmaf(C->cdt, q, C->c1);
    float em = f_mul(*eh, mu);
    float xn = fmaf(*x, t, em);
    float r = fmaf(C->cz, q, C->c2);
    *eh = f_mul(*eh, r);
    *x = xn;
}

void orc_euler_spin(float* x, float* eh, float mu, const orc_consts* C) { euler_spin(x, eh, mu, C); }

/* One anneal: S Euler steps, field refreshed when t mod f_mvm == 0.
 * x, eh: [2n+1] in/out. */
void orc_anneal(int n, const float* Af, const float* hf, const orc_params* P, const orc_consts* C, float* x, float* eh)
{
    const int N = 2 * n + 1;
    float* mu = (float*)malloc(sizeof(float) * (size_t)N);
    for (int t = 0; t < P->steps; ++t) {
        if (t % P->f_mvm == 0) orc_coupling_field(n, Af, hf, x, mu);
        for (int k = 0; k < N; ++k) euler_spin(&x[k], &eh[k], mu[k], C);
    }
    free(mu);
}

/*
 * The R anneals of one problem with early exit (a budget lever; the paper
 * anneals every run for a fixed N_I steps, Appendix A).  The anneals advance
 * together, one refresh interval at a time, each exactly as orc_anneal
 * advances it.  Every K-th refresh point, t = j K f_mvm with 0 < t < S
 * (K = P->early_exit), is a check point: the spin signs s_k = [x_k >= 0] of
 * every anneal (all 2n+1 spins) are compared with their signs at the previous
 * check point t - K f_mvm (the initial state for the first).  If no sign of
 * any anneal changed, the anneals stop at t: their state at t is final and no
 * refresh is made there.
 * X, EH: [R][2n+1] in/out.  Returns the Euler steps taken (<= S).
 */
static int anneal_early_exit(int n, const float* Af, const float* hf, const orc_params* P, const orc_consts* C,
                             float* X, float* EH)
{
    const int N = 2 * n + 1, R = P->runs, S = P->steps, f = P->f_mvm, K = P->early_exit;
    unsigned char* sg = (unsigned char*)malloc((size_t)R * N);
    float* mu = (float*)malloc(sizeof(float) * (size_t)N);
    for (int i = 0; i < R * N; ++i) sg[i] = X[i] >= 0.0f;
    int taken = S;
    for (int t = 0; t < S; t += f) {
        if (t > 0 && (t / f) % K == 0) {
            int changed = 0;
            for (int i = 0; i < R * N; ++i) {
                const unsigned char s = X[i] >= 0.0f;
                if (s != sg[i]) changed = 1;
                sg[i] = s;
            }
            if (!changed) {
                taken = t;
                break;
            }
        }
        const int L = (S - t < f) ? S - t : f;
        for (int r = 0; r < R; ++r) {
            float* x = X + (size_t)r * N;
            float* eh = EH + (size_t)r * N;
            orc_coupling_field(n, Af, hf, x, mu);
            for (int s = 0; s < L; ++s)
                for (int k = 0; k < N; ++k) euler_spin(&x[k], &eh[k], mu[k], C);
        }
    }
    free(sg);
    free(mu);
    return taken;
}

/*
 * Solve one delta-Ising problem with R anneals and keep the best candidate.
 *
 * Aq [n][n], hq [n]: Q14 couplings (A = -G block, b = h).
 * g [n], level_max: lattice guess and clip bound; offsets that leave
 * [-level_max, level_max] are set to 0 before scoring.  level_max = 0: no clip.
 * Selection: each anneal's spins s = sign(x) (x >= 0 -> +1) give
 * d = s_a (s1 + s2) / 2; a diverged anneal (|x| > x_max, non-finite, or
 * e <= 0 anywhere) or one whose energy is larger than the guess's (E > 0)
 * returns the guess (d = 0, E = 0) instead (Sec. 3.2 solver kernel); the best
 * candidate is the lowest (E, run index) (Sec. 3.2 post-processing).
 *
 * With P->early_exit = K > 0 the anneals stop together as anneal_early_exit
 * states; selection is unchanged.
 *
 * Outputs: d_out [n], E_out, run_out, n_div_out; optional x_final [R][2n+1],
 * E_runs [R] (raw energy of each anneal's clipped offset, INT32_MAX if diverged),
 * steps_out (Euler steps the anneals took).
 */
int orc_cac_solve_steps(int n, const int16_t* Aq, const int16_t* hq, const int* g, int level_max,
                        const orc_params* P, uint64_t seed, uint64_t problem, int8_t* d_out, int32_t* E_out,
                        int32_t* run_out, int32_t* n_div_out, float* x_final, int32_t* E_runs, int32_t* steps_out)
{
    if (n < 1 || P->runs < 1 || P->steps < 0 || P->f_mvm < 1 || P->early_exit < 0) return ORC_EINVAL;
    const int N = 2 * n + 1;
    orc_consts C;
    orc_cac_consts(P, &C);
    float* Af = (float*)malloc(sizeof(float) * (size_t)(n * n));
    float* hf = (float*)malloc(sizeof(float) * (size_t)n);
    const float q = pow2f(-QBITS);
    /* J = J_q 2^-14 (exact), then one rounding by eps dt */
    for (int e = 0; e < n * n; ++e) Af[e] = f_mul(f_mul((float)Aq[e], q), C.ce);
    for (int i = 0; i < n; ++i) hf[i] = f_mul(f_mul((float)hq[i], q), C.ce);
    float* x = (float*)malloc(sizeof(float) * (size_t)N);
    float* eh = (float*)malloc(sizeof(float) * (size_t)N);
    int8_t* d = (int8_t*)malloc((size_t)n);
    int32_t bestE = 0;
    int bestRun = -1, ndiv = 0;
    memset(d_out, 0, (size_t)n);
    /* with early exit the anneals run together first; their final states are
       then scored one by one below */
    float* XE = NULL;
    float* EE = NULL;
    int taken = P->steps;
    if (P->early_exit > 0) {
        XE = (float*)malloc(sizeof(float) * (size_t)P->runs * N);
        EE = (float*)malloc(sizeof(float) * (size_t)P->runs * N);
        for (int r = 0; r < P->runs; ++r)
            for (int k = 0; k < N; ++k) {
                XE[(size_t)r * N + k] = orc_initial_x(seed, problem, r, k, C.xs);
                EE[(size_t)r * N + k] = 1.0f;
            }
        taken = anneal_early_exit(n, Af, hf, P, &C, XE, EE);
    }
    if (steps_out) *steps_out = taken;

    for (int r = 0; r < P->runs; ++r) {
        if (XE) {
            memcpy(x, XE + (size_t)r * N, sizeof(float) * (size_t)N);
            memcpy(eh, EE + (size_t)r * N, sizeof(float) * (size_t)N);
        } else {
            for (int k = 0; k < N; ++k) {
                x[k] = orc_initial_x(seed, problem, r, k, C.xs);
                eh[k] = 1.0f;
            }
            orc_anneal(n, Af, hf, P, &C, x, eh);
        }
        if (x_final) memcpy(x_final + (size_t)r * N, x, sizeof(float) * (size_t)N);
        int valid = 1;
        for (int k = 0; k < N; ++k)
            if (!(fabsf(x[k]) <= P->x_max) || !(eh[k] > 0.0f)) valid = 0;
        int sa = x[2 * n] >= 0.0f ? 1 : -1;
        for (int i = 0; i < n; ++i) {
            int s1 = x[i] >= 0.0f ? 1 : -1, s2 = x[n + i] >= 0.0f ? 1 : -1;
            int di = sa * (s1 + s2) / 2;
            if (level_max > 0) {
                int xv = g[i] + 2 * di;
                if (xv > level_max || xv < -level_max) di = 0;
            }
            d[i] = (int8_t)di;
        }
        int32_t E = valid ? orc_energy_q(n, Aq, hq, d) : INT32_MAX;
        if (E_runs) E_runs[r] = E;
        if (!valid) ndiv++;
        int32_t Ec = (valid && E <= 0) ? E : 0;
        if (bestRun < 0 || Ec < bestE) {
            bestE = Ec;
            bestRun = r;
            if (valid && E <= 0) memcpy(d_out, d, (size_t)n);
            else memset(d_out, 0, (size_t)n);
        }
    }
    *E_out = bestE;
    *run_out = bestRun;
    *n_div_out = ndiv;
    free(Af); free(hf); free(x); free(eh); free(d); free(XE); free(EE);
    return ORC_OK;
}

int orc_cac_solve(int n, const int16_t* Aq, const int16_t* hq, const int* g, int level_max, const orc_params* P,
                  uint64_t seed, uint64_t problem, int8_t* d_out, int32_t* E_out, int32_t* run_out,
                  int32_t* n_div_out, float* x_final, int32_t* E_runs)
{
    return orc_cac_solve_steps(n, Aq, hq, g, level_max, P, seed, problem, d_out, E_out, run_out, n_div_out, x_final,
                               E_runs, NULL);
}

/* Decoded uplink symbol of user i: lattice x = g + 2d per real dimension,
 * symbol index = ((x_re + L) / 2) * sqrt(M) + (x_im + L) / 2. */
void orc_decode_detect(int n_t, int mod_bits, const int* g, const int8_t* d, uint8_t* sym_out)
{
    const int side = orc_qam_side(mod_bits), L = side - 1;
    for (int i = 0; i < n_t; ++i) {
        int xr = g[i] + 2 * d[i], xi = g[n_t + i] + 2 * d[n_t + i];
        sym_out[i] = (uint8_t)(((xr + L) / 2) * side + (xi + L) / 2);
    }
}

/* ========================================================================= */
/* Downlink vector-perturbation precoding (Sec. 2.2 Eqs. 5, 8; Sec. 3.3       */
/* Eqs. 12-13), FP64 in the pinned order (the GPU path computes this layer in */
/* FP64 too).                                                                 */
/* ========================================================================= */

/* Q = (H H^H)^-1 for H [n_u][n_t] complex (FP64).  Pinned order:
 *   K_ii = sum_k fma(a.re,a.re), fma(a.im,a.im), a = H_ik, k ascending
 *   K_ij (i<j) = sum_k H_ik conj(H_jk): re = fma(a.re,b.re), fma(a.im,b.im),
 *                im = fma(a.im,b.re), fma(-a.re,b.im); K_ji = conj(K_ij)
 *   Cholesky as the FP32 layer; columns j of Q from the forward/backward
 *   solves of e_j, keep the upper triangle i <= j, Q_ji = conj(Q_ij),
 *   diagonal imaginary part 0.
 * Q: [n_u][n_u] complex. */
int orc_vpp_inverse64(int n_u, int n_t, const double* H, double* Q)
{
    if (n_u < 1 || n_t < 1) return ORC_EINVAL;
    double* K = (double*)malloc(sizeof(double) * 2 * (size_t)(n_u * n_u));
    double* L = (double*)calloc(2 * (size_t)(n_u * n_u), sizeof(double));
    double* w = (double*)malloc(sizeof(double) * 2 * (size_t)n_u);
    double* col = (double*)malloc(sizeof(double) * 2 * (size_t)n_u);
    int status = ORC_OK;
    for (int i = 0; i < n_u; ++i) {
        double acc = 0.0;
        for (int k = 0; k < n_t; ++k) {
            const double* a = H + 2 * (i * n_t + k);
            acc = fma(a[0], a[0], acc);
            acc = fma(a[1], a[1], acc);
        }
        K[2 * (i * n_u + i)] = acc;
        K[2 * (i * n_u + i) + 1] = 0.0;
        for (int j = i + 1; j < n_u; ++j) {
            double re = 0.0, im = 0.0;
            for (int k = 0; k < n_t; ++k) {
                const double* a = H + 2 * (i * n_t + k);
                const double* b = H + 2 * (j * n_t + k);
                re = fma(a[0], b[0], re);
                re = fma(a[1], b[1], re);
                im = fma(a[1], b[0], im);
                im = fma(-a[0], b[1], im);
            }
            K[2 * (i * n_u + j)] = re;
            K[2 * (i * n_u + j) + 1] = im;
            K[2 * (j * n_u + i)] = re;
            K[2 * (j * n_u + i) + 1] = -im;
        }
    }
    for (int j = 0; j < n_u && status == ORC_OK; ++j) {
        double d = K[2 * (j * n_u + j)];
        for (int k = 0; k < j; ++k) {
            const double* l = L + 2 * (j * n_u + k);
            d = fma(-l[0], l[0], d);
            d = fma(-l[1], l[1], d);
        }
        if (!(d > 0.0) || isinf(d)) { status = ORC_ENUM; break; }
        double ljj = sqrt(d);
        L[2 * (j * n_u + j)] = ljj;
        for (int i = j + 1; i < n_u; ++i) {
            double re = K[2 * (i * n_u + j)], im = K[2 * (i * n_u + j) + 1];
            for (int k = 0; k < j; ++k) {
                const double* a = L + 2 * (i * n_u + k);
                const double* b = L + 2 * (j * n_u + k);
                re = fma(-a[0], b[0], re);
                re = fma(-a[1], b[1], re);
                im = fma(-a[1], b[0], im);
                im = fma(a[0], b[1], im);
            }
            L[2 * (i * n_u + j)] = re / ljj;
            L[2 * (i * n_u + j) + 1] = im / ljj;
        }
    }
    if (status == ORC_OK) {
        for (int c = 0; c < n_u; ++c) {
            for (int i = 0; i < n_u; ++i) {
                double re = (i == c) ? 1.0 : 0.0, im = 0.0;
                for (int k = 0; k < i; ++k) {
                    const double* a = L + 2 * (i * n_u + k);
                    const double* b = w + 2 * k;
                    re = fma(-a[0], b[0], re);
                    re = fma(a[1], b[1], re);
                    im = fma(-a[0], b[1], im);
                    im = fma(-a[1], b[0], im);
                }
                double lii = L[2 * (i * n_u + i)];
                w[2 * i] = re / lii;
                w[2 * i + 1] = im / lii;
            }
            for (int i = n_u - 1; i >= 0; --i) {
                double re = w[2 * i], im = w[2 * i + 1];
                for (int k = n_u - 1; k > i; --k) {
                    const double* a = L + 2 * (k * n_u + i);
                    const double* b = col + 2 * k;
                    re = fma(-a[0], b[0], re);
                    re = fma(-a[1], b[1], re);
                    im = fma(-a[0], b[1], im);
                    im = fma(a[1], b[0], im);
                }
                double lii = L[2 * (i * n_u + i)];
                col[2 * i] = re / lii;
                col[2 * i + 1] = im / lii;
            }
            for (int i = 0; i <= c; ++i) {
                double re = col[2 * i], im = (i == c) ? 0.0 : col[2 * i + 1];
                Q[2 * (i * n_u + c)] = re;
                Q[2 * (i * n_u + c) + 1] = im;
                Q[2 * (c * n_u + i)] = re;
                Q[2 * (c * n_u + i) + 1] = -im;
            }
        }
    } else {
        memset(Q, 0, sizeof(double) * 2 * (size_t)(n_u * n_u));
    }
    free(K); free(L); free(w); free(col);
    return status;
}

/* Lattice point of a QAM symbol index (inverse of orc_decode_detect). */
static void sym_to_lattice(int mod_bits, int sym, int* re, int* im)
{
    const int side = orc_qam_side(mod_bits), L = side - 1;
    *re = 2 * (sym / side) - L;
    *im = 2 * (sym % side) - L;
}

/* tau = 2 (c_max + Delta/2) with c_max = L and lattice spacing Delta = 2,
 * i.e. tau = 2 sqrt(M) in lattice units. */
int orc_vpp_tau(int mod_bits) { return 2 * orc_qam_side(mod_bits); }

/*
 * Delta-Ising problem of one VPP problem (Sec. 3.3, Eqs. 12-13): detection with
 * y~ = W u, H_p = -tau W / 2, x = 2v, guess 0.  With Q = (H H^H)^-1 = W^H W:
 *   G = H_p^H H_p = (tau/2)^2 Q,  h = H_p^H y~ = -(tau/2) Q u.
 * FP64, pinned order: (Qu)_i = sum_j Q_ij u_j, j ascending
 * (re = fma(q.re,u.re), fma(-q.im,u.im); im = fma(q.re,u.im), fma(q.im,u.re)),
 * then exact power-of-two scalings by tau/2 = sqrt(M) and quantisation as
 * orc_quantise64.
 * Outputs: Q [n_u][n_u] complex (optional), G [n*n], h [n], sigma_exp, Aq, hq.
 */
int orc_build_precode(int n_u, int n_t, int mod_bits, const double* H, const uint8_t* u_sym, double* Q_out,
                      double* G_out, double* h_out, int* sigma_exp_out, int16_t* Aq_out, int16_t* hq_out)
{
    const int n = 2 * n_u;
    double* Q = (double*)malloc(sizeof(double) * 2 * (size_t)(n_u * n_u));
    double* G = (double*)malloc(sizeof(double) * (size_t)(n * n));
    double* h = (double*)malloc(sizeof(double) * (size_t)n);
    int32_t* A32 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n * n));
    int32_t* h32 = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int status = orc_vpp_inverse64(n_u, n_t, H, Q);
    const double half_tau = (double)orc_vpp_tau(mod_bits) / 2.0;
    const double s2 = half_tau * half_tau;
    for (int i = 0; i < n_u; ++i) {
        double re = 0.0, im = 0.0;
        for (int j = 0; j < n_u; ++j) {
            int ur, ui;
            sym_to_lattice(mod_bits, u_sym[j], &ur, &ui);
            const double* q = Q + 2 * (i * n_u + j);
            re = fma(q[0], (double)ur, re);
            re = fma(-q[1], (double)ui, re);
            im = fma(q[0], (double)ui, im);
            im = fma(q[1], (double)ur, im);
        }
        h[i] = -half_tau * re;
        h[n_u + i] = -half_tau * im;
    }
    for (int i = 0; i < n_u; ++i)
        for (int j = 0; j < n_u; ++j) {
            double re = Q[2 * (i * n_u + j)] * s2, im = Q[2 * (i * n_u + j) + 1] * s2;
            G[i * n + j] = re;
            G[i * n + (n_u + j)] = -im;
            G[(n_u + i) * n + j] = im;
            G[(n_u + i) * n + (n_u + j)] = re;
        }
    int se;
    orc_quantise64(n, G, h, &se, A32, h32);
    for (int e = 0; e < n * n; ++e) Aq_out[e] = (int16_t)A32[e];
    for (int i = 0; i < n; ++i) hq_out[i] = (int16_t)h32[i];
    if (sigma_exp_out) *sigma_exp_out = se;
    if (Q_out) memcpy(Q_out, Q, sizeof(double) * 2 * (size_t)(n_u * n_u));
    if (G_out) memcpy(G_out, G, sizeof(double) * (size_t)(n * n));
    if (h_out) memcpy(h_out, h, sizeof(double) * (size_t)n);
    free(Q); free(G); free(h); free(A32); free(h32);
    return status;
}

/*
 * Precoder output of one VPP problem: perturbation v = d_re + i d_im per user,
 * t = u + tau v, w = Q t, transmit vector x = H^H w = W (u + tau v)
 * (unnormalised; Eq. 6 scales it to power P) and its power
 * ||x||^2 = t^H Q t.  FP64, pinned order:
 *   w_i = sum_j Q_ij t_j  (j ascending; same fma pattern as Q u)
 *   x_k = sum_i conj(H_ik) w_i  (i ascending; re = fma(a.re,w.re), fma(a.im,w.im),
 *                                 im = fma(a.re,w.im), fma(-a.im,w.re))
 *   power = sum_i (fma(t.re, w.re), fma(t.im, w.im)), i ascending, from 0
 * Outputs: v [n_u][2] int8, x [n_t] complex float (rounded once), power (float).
 */
void orc_precode_output(int n_u, int n_t, int mod_bits, const double* H, const double* Q, const uint8_t* u_sym,
                        const int8_t* d, int8_t* v_out, float* x_out, float* power_out)
{
    const int tau = orc_vpp_tau(mod_bits);
    double* t = (double*)malloc(sizeof(double) * 2 * (size_t)n_u);
    double* w = (double*)malloc(sizeof(double) * 2 * (size_t)n_u);
    for (int i = 0; i < n_u; ++i) {
        int ur, ui;
        sym_to_lattice(mod_bits, u_sym[i], &ur, &ui);
        v_out[2 * i] = d[i];
        v_out[2 * i + 1] = d[n_u + i];
        t[2 * i] = (double)(ur + tau * d[i]);
        t[2 * i + 1] = (double)(ui + tau * d[n_u + i]);
    }
    for (int i = 0; i < n_u; ++i) {
        double re = 0.0, im = 0.0;
        for (int j = 0; j < n_u; ++j) {
            const double* q = Q + 2 * (i * n_u + j);
            re = fma(q[0], t[2 * j], re);
            re = fma(-q[1], t[2 * j + 1], re);
            im = fma(q[0], t[2 * j + 1], im);
            im = fma(q[1], t[2 * j], im);
        }
        w[2 * i] = re;
        w[2 * i + 1] = im;
    }
    for (int k = 0; k < n_t; ++k) {
        double re = 0.0, im = 0.0;
        for (int i = 0; i < n_u; ++i) {
            const double* a = H + 2 * (i * n_t + k);
            re = fma(a[0], w[2 * i], re);
            re = fma(a[1], w[2 * i + 1], re);
            im = fma(a[0], w[2 * i + 1], im);
            im = fma(-a[1], w[2 * i], im);
        }
        x_out[2 * k] = (float)re;
        x_out[2 * k + 1] = (float)im;
    }
    double pw = 0.0;
    for (int i = 0; i < n_u; ++i) {
        pw = fma(t[2 * i], w[2 * i], pw);
        pw = fma(t[2 * i + 1], w[2 * i + 1], pw);
    }
    *power_out = (float)pw;
    free(t);
    free(w);
}

/* ========================================================================= */
/* Batched drivers (loops over problems; used by tests and the CPU baseline)  */
/* ========================================================================= */

/*
 * Full uplink pipeline for a batch: FP32 build -> CAC solve -> decode.
 * H: [n_chan][n_r][n_t] complex float, chan_index: [P] (NULL = identity),
 * y: [P][n_r] complex float, noise_var: [P].  Problem p uses Philox counter
 * space (seed, p).  Outputs: sym [P][n_t], E [P], run [P], n_div [P],
 * optional g [P][n], d [P][n], steps [P] (Euler steps taken).
 */
int orc_detect_batch(int n_r, int n_t, int mod_bits, int P, const int32_t* chan_index, const float* H,
                     const float* y, const float* noise_var, const orc_params* prm, uint64_t seed, uint8_t* sym,
                     int32_t* E, int32_t* run, int32_t* n_div, int32_t* g_out, int8_t* d_out, int32_t* steps_out)
{
    const int n = 2 * n_t;
    int* g = (int*)malloc(sizeof(int) * (size_t)n);
    int16_t* Aq = (int16_t*)malloc(sizeof(int16_t) * (size_t)(n * n));
    int16_t* hq = (int16_t*)malloc(sizeof(int16_t) * (size_t)n);
    int8_t* d = (int8_t*)malloc((size_t)n);
    int status = ORC_OK;
    for (int p = 0; p < P; ++p) {
        int c = chan_index ? chan_index[p] : p;
        int se;
        orc_build_detect32(n_r, n_t, mod_bits, H + (size_t)c * 2 * n_r * n_t, y + (size_t)p * 2 * n_r,
                           noise_var[p], NULL, g, NULL, NULL, &se, Aq, hq);
        int st = orc_cac_solve_steps(n, Aq, hq, g, orc_qam_level_max(mod_bits), prm, seed, (uint64_t)p, d, &E[p],
                                     &run[p], &n_div[p], NULL, NULL, steps_out ? &steps_out[p] : NULL);
        if (st != ORC_OK) status = st;
        orc_decode_detect(n_t, mod_bits, g, d, sym + (size_t)p * n_t);
        if (g_out)
            for (int i = 0; i < n; ++i) g_out[(size_t)p * n + i] = g[i];
        if (d_out) memcpy(d_out + (size_t)p * n, d, (size_t)n);
    }
    free(g); free(Aq); free(hq); free(d);
    return status;
}

/* ========================================================================= */
/* MMGaP-E (Sec. 3.2.2): a second guess from MMSE-SIC and multi-stage        */
/* re-centring, FP32 mirror.                                                  */
/* ========================================================================= */

/* Nearest alphabet point of one real dimension (ties upward), as the guess. */
static int slice_f(float x, int Lmax)
{
    float xc = fmaxf(x, (float)-Lmax);
    xc = fminf(xc, (float)Lmax);
    return 2 * (int)floorf(f_mul(xc, 0.5f)) + 1;
}

/*
 * MMSE-SIC guess (the paper's second initial guess, Sec. 3.2.2), FP32.
 * Cholesky of B = G_c + rho I with sorted pivoting: at step j the remaining
 * user with the smallest current Schur diagonal d (ties: first position) is
 * factored next, so the users with the largest d are detected first.  The
 * forward solve gives w = L^-1 P m; successive interference cancellation is
 * then the back substitution x_j = (w_j - sum_{k>j} conj(L_kj) xhat_k) / L_jj
 * (k descending) with each x_j sliced to the alphabet before it is
 * substituted.  Same operation patterns as orc_build_detect32.
 * Outputs g [2 n_t] (re block, im block) and, optionally, perm [n_t]
 * (position -> user).  Returns ORC_ENUM if a pivot is not positive
 * (then the guess is the slice of 0 for every user).
 */
int orc_sic_guess32(int n_r, int n_t, int mod_bits, const float* H, const float* y, float noise_var, int* g_out,
                    int* perm_out)
{
    if (n_r < 1 || n_t < 1 || mod_bits < 2 || (mod_bits & 1)) return ORC_EINVAL;
    const int Lmax = orc_qam_level_max(mod_bits);
    const float kappa = qam_kappa_f(mod_bits);
    const float rho = f_mul(noise_var, qam_kappa2_f(mod_bits));
    float* Hs = (float*)malloc(sizeof(float) * 2 * (size_t)(n_r * n_t));
    float* Gc = (float*)malloc(sizeof(float) * 2 * (size_t)(n_t * n_t));
    float* Lc = (float*)calloc(2 * (size_t)(n_t * n_t), sizeof(float));
    float* m = (float*)malloc(sizeof(float) * 2 * (size_t)n_t);
    float* w = (float*)malloc(sizeof(float) * 2 * (size_t)n_t);
    float* xh = (float*)malloc(sizeof(float) * 2 * (size_t)n_t);
    float* d = (float*)malloc(sizeof(float) * (size_t)n_t);
    int* perm = (int*)malloc(sizeof(int) * (size_t)n_t);
    int status = ORC_OK;
    for (int e = 0; e < 2 * n_r * n_t; ++e) Hs[e] = f_mul(kappa, H[e]);
    for (int i = 0; i < n_t; ++i) {
        float acc = 0.0f;
        for (int k = 0; k < n_r; ++k) {
            const float* a = Hs + 2 * (k * n_t + i);
            acc = fmaf(a[0], a[0], acc);
            acc = fmaf(a[1], a[1], acc);
        }
        Gc[2 * (i * n_t + i)] = acc;
        Gc[2 * (i * n_t + i) + 1] = 0.0f;
        for (int j = i + 1; j < n_t; ++j) {
            float re = 0.0f, im = 0.0f;
            for (int k = 0; k < n_r; ++k) {
                const float* a = Hs + 2 * (k * n_t + i);
                const float* b = Hs + 2 * (k * n_t + j);
                re = fmaf(a[0], b[0], re);
                re = fmaf(a[1], b[1], re);
                im = fmaf(a[0], b[1], im);
                im = fmaf(-a[1], b[0], im);
            }
            Gc[2 * (i * n_t + j)] = re;
            Gc[2 * (i * n_t + j) + 1] = im;
            Gc[2 * (j * n_t + i)] = re;
            Gc[2 * (j * n_t + i) + 1] = -im;
        }
    }
    for (int i = 0; i < n_t; ++i) {
        float re = 0.0f, im = 0.0f;
        for (int k = 0; k < n_r; ++k) {
            const float* a = Hs + 2 * (k * n_t + i);
            const float* b = y + 2 * k;
            re = fmaf(a[0], b[0], re);
            re = fmaf(a[1], b[1], re);
            im = fmaf(a[0], b[1], im);
            im = fmaf(-a[1], b[0], im);
        }
        m[2 * i] = re;
        m[2 * i + 1] = im;
    }
    for (int i = 0; i < n_t; ++i) {
        perm[i] = i;
        d[i] = f_add(Gc[2 * (i * n_t + i)], rho);
    }
    int ok = 1;
    for (int j = 0; j < n_t && ok; ++j) {
        int best = j; /* position of the smallest current diagonal among j..n_t-1 */
        for (int i = j + 1; i < n_t; ++i)
            if (d[perm[i]] < d[perm[best]]) best = i;
        int t = perm[j];
        perm[j] = perm[best];
        perm[best] = t;
        /* rows of L are positions; swap the already computed columns k < j of rows j and best */
        for (int k = 0; k < j; ++k) {
            float r0 = Lc[2 * (j * n_t + k)], r1 = Lc[2 * (j * n_t + k) + 1];
            Lc[2 * (j * n_t + k)] = Lc[2 * (best * n_t + k)];
            Lc[2 * (j * n_t + k) + 1] = Lc[2 * (best * n_t + k) + 1];
            Lc[2 * (best * n_t + k)] = r0;
            Lc[2 * (best * n_t + k) + 1] = r1;
        }
        const int u = perm[j];
        float dj = d[u];
        if (!(dj > 0.0f) || isinf(dj)) { ok = 0; break; }
        float ljj = sqrtf(dj);
        Lc[2 * (j * n_t + j)] = ljj;
        Lc[2 * (j * n_t + j) + 1] = 0.0f;
        for (int i = j + 1; i < n_t; ++i) {
            const int v = perm[i];
            float re = Gc[2 * (v * n_t + u)], im = Gc[2 * (v * n_t + u) + 1];
            for (int k = 0; k < j; ++k) {
                const float* a = Lc + 2 * (i * n_t + k);
                const float* b = Lc + 2 * (j * n_t + k);
                re = fmaf(-a[0], b[0], re);
                re = fmaf(-a[1], b[1], re);
                im = fmaf(-a[1], b[0], im);
                im = fmaf(a[0], b[1], im);
            }
            float lr = re / ljj, li = im / ljj;
            Lc[2 * (i * n_t + j)] = lr;
            Lc[2 * (i * n_t + j) + 1] = li;
            d[v] = fmaf(-lr, lr, d[v]);
            d[v] = fmaf(-li, li, d[v]);
        }
    }
    if (ok) {
        for (int i = 0; i < n_t; ++i) {
            float re = m[2 * perm[i]], im = m[2 * perm[i] + 1];
            for (int k = 0; k < i; ++k) {
                const float* a = Lc + 2 * (i * n_t + k);
                const float* b = w + 2 * k;
                re = fmaf(-a[0], b[0], re);
                re = fmaf(a[1], b[1], re);
                im = fmaf(-a[0], b[1], im);
                im = fmaf(-a[1], b[0], im);
            }
            float lii = Lc[2 * (i * n_t + i)];
            w[2 * i] = re / lii;
            w[2 * i + 1] = im / lii;
        }
        for (int i = n_t - 1; i >= 0; --i) {
            float re = w[2 * i], im = w[2 * i + 1];
            for (int k = n_t - 1; k > i; --k) {
                const float* a = Lc + 2 * (k * n_t + i);
                const float* b = xh + 2 * k;
                re = fmaf(-a[0], b[0], re);
                re = fmaf(-a[1], b[1], re);
                im = fmaf(-a[0], b[1], im);
                im = fmaf(a[1], b[0], im);
            }
            float lii = Lc[2 * (i * n_t + i)];
            xh[2 * i] = (float)slice_f(re / lii, Lmax);
            xh[2 * i + 1] = (float)slice_f(im / lii, Lmax);
        }
        for (int i = 0; i < n_t; ++i) {
            g_out[perm[i]] = (int)xh[2 * i];
            g_out[n_t + perm[i]] = (int)xh[2 * i + 1];
        }
    } else {
        for (int i = 0; i < n_t; ++i) {
            g_out[i] = slice_f(0.0f, Lmax);
            g_out[n_t + i] = slice_f(0.0f, Lmax);
        }
        status = ORC_ENUM;
    }
    if (perm_out) memcpy(perm_out, perm, sizeof(int) * (size_t)n_t);
    free(Hs); free(Gc); free(Lc); free(m); free(w); free(xh); free(d); free(perm);
    return status;
}

/* ML objective ||y - Hs x||^2 of a lattice vector in FP32, pinned order:
 * r_k = y_k - sum_j Hs_kj x_j (j ascending, as the residual of the build),
 * then sum_k fma(r.re, r.re), fma(r.im, r.im) from 0, k ascending. */
float orc_ml_objective32(int n_r, int n_t, int mod_bits, const float* H, const float* y, const int* x)
{
    const float kappa = qam_kappa_f(mod_bits);
    float obj = 0.0f;
    for (int k = 0; k < n_r; ++k) {
        float re = y[2 * k], im = y[2 * k + 1];
        for (int j = 0; j < n_t; ++j) {
            float ar = f_mul(kappa, H[2 * (k * n_t + j)]), ai = f_mul(kappa, H[2 * (k * n_t + j) + 1]);
            float br = (float)x[j], bi = (float)x[n_t + j];
            re = fmaf(-ar, br, re);
            re = fmaf(ai, bi, re);
            im = fmaf(-ar, bi, im);
            im = fmaf(-ai, br, im);
        }
        obj = fmaf(re, re, obj);
        obj = fmaf(im, im, obj);
    }
    return obj;
}

/* Seed of instance `inst` (0: from the MMSE guess, 1: from the SIC guess) of
 * stage `stage` (1-based): seed + (2 (stage - 1) + inst) * 0x9E3779B97F4A7C15. */
uint64_t orc_stage_seed(uint64_t seed, int stage, int inst)
{
    return seed + (uint64_t)(2 * (stage - 1) + inst) * 0x9E3779B97F4A7C15ULL;
}

/*
 * MMGaP-E for one problem (Sec. 3.2.2): candidates in this order --
 * the MMSE guess, the SIC guess, then for each stage s = 1..stages the
 * solutions of instance 0 and instance 1; instance i of stage s is the
 * delta-Ising problem around instance i's previous candidate (stage 1: the
 * MMSE / SIC guess), annealed with orc_stage_seed(seed, s, i).  The output is
 * the candidate with the lowest FP32 ML objective (ties: first).
 * Outputs sym [n_t], best (candidate index), obj (its objective), and
 * optionally all candidates x_all [(2 + 2 stages)][2 n_t].
 */
int orc_detect_e(int n_r, int n_t, int mod_bits, const float* H, const float* y, float noise_var, int stages,
                 const orc_params* P, uint64_t seed, uint64_t problem, uint8_t* sym, int* best_out, float* obj_out,
                 int* x_all)
{
    const int n = 2 * n_t, nc = 2 + 2 * stages;
    const int Lm = orc_qam_level_max(mod_bits);
    int* X = (int*)malloc(sizeof(int) * (size_t)(nc * n));
    int16_t* Aq = (int16_t*)malloc(sizeof(int16_t) * (size_t)(n * n));
    int16_t* hq = (int16_t*)malloc(sizeof(int16_t) * (size_t)n);
    int* g = (int*)malloc(sizeof(int) * (size_t)n);
    int8_t* d = (int8_t*)malloc((size_t)n);
    int se;
    orc_build_detect32(n_r, n_t, mod_bits, H, y, noise_var, NULL, X, NULL, NULL, &se, Aq, hq);
    orc_sic_guess32(n_r, n_t, mod_bits, H, y, noise_var, X + n, NULL);
    for (int s = 1; s <= stages; ++s)
        for (int inst = 0; inst < 2; ++inst) {
            const int* prev = X + (size_t)(s == 1 ? inst : 2 + 2 * (s - 2) + inst) * n;
            orc_build_detect32(n_r, n_t, mod_bits, H, y, noise_var, prev, g, NULL, NULL, &se, Aq, hq);
            int32_t E, run, nd;
            orc_cac_solve(n, Aq, hq, g, Lm, P, orc_stage_seed(seed, s, inst), problem, d, &E, &run, &nd, NULL, NULL);
            int* out = X + (size_t)(2 + 2 * (s - 1) + inst) * n;
            for (int i = 0; i < n; ++i) out[i] = g[i] + 2 * d[i];
        }
    int best = 0;
    float bo = orc_ml_objective32(n_r, n_t, mod_bits, H, y, X);
    for (int c = 1; c < nc; ++c) {
        float o = orc_ml_objective32(n_r, n_t, mod_bits, H, y, X + (size_t)c * n);
        if (o < bo) { bo = o; best = c; }
    }
    int8_t* zero = (int8_t*)calloc((size_t)n, 1);
    orc_decode_detect(n_t, mod_bits, X + (size_t)best * n, zero, sym);
    if (best_out) *best_out = best;
    if (obj_out) *obj_out = bo;
    if (x_all) memcpy(x_all, X, sizeof(int) * (size_t)(nc * n));
    free(zero); free(X); free(Aq); free(hq); free(g); free(d);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Direct (binary-weighted) spin mapping.  The paper's method is the delta   */
/* form above (Sec. 2.3, Sec. 3.2.1); the direct form is the mapping of the  */
/* Ising-machine detectors it builds on, where each real dimension of the    */
/* lattice symbol is a binary-weighted sum of spins.  The paper gives no     */
/* formulas for it; the readings are:                                        */
/*   B = mod_bits / 2 spins per real dimension, x_k = sum_b 2^b s_(kB+b),    */
/*   i.e. x = T s with T = I_(2 n_t) (x) [1, 2, ..., 2^(B-1)]; real          */
/*   dimensions k in the real-form order (Re of users, then Im of users).   */
/*   ||y - Hs T s||^2 = s^T (T^T G T) s - 2 (T^T mf)^T s + ||y||^2 with     */
/*   G = Hs_r^T Hs_r and mf = Hs_r^T y_r (real forms), so with an auxiliary  */
/*   spin s_a the Ising form to maximise is s^T J s + 2 s_a c^T s with       */
/*   J = -(T^T G T) (diagonal set to 0: s_i^2 = 1) and c = T^T mf, and       */
/*   ||y - Hs T s||^2 = -s^T J s - 2 c^T s + ||y||^2 + tr(T^T G T).          */
/* N = 2 n_t B spins (16 for 8x8 QPSK, 64 for 16x16 16-QAM, 96 for 16x16     */
/* 64-QAM) plus the auxiliary one.                                          */
/* ------------------------------------------------------------------------- */

/* FP64 truth: J [N*N], c [N], and the constant ||y||^2 + tr(T^T G T). */
int orc_build_direct64(int n_r, int n_t, int mod_bits, const double* H, const double* y, double* J_out,
                       double* c_out, double* const_out)
{
    if (n_r < 1 || n_t < 1 || mod_bits < 2 || (mod_bits & 1)) return ORC_EINVAL;
    const int n = 2 * n_t, B = mod_bits / 2, N = n * B;
    const double kappa = orc_qam_kappa(mod_bits);
    /* real forms Hr [2 n_r][n], yr [2 n_r] */
    double* Hr = (double*)malloc(sizeof(double) * (size_t)(2 * n_r * n));
    double* yr = (double*)malloc(sizeof(double) * (size_t)(2 * n_r));
    for (int k = 0; k < n_r; ++k) {
        yr[k] = y[2 * k];
        yr[n_r + k] = y[2 * k + 1];
        for (int i = 0; i < n_t; ++i) {
            double re = kappa * H[2 * (k * n_t + i)], im = kappa * H[2 * (k * n_t + i) + 1];
            Hr[k * n + i] = re;
            Hr[k * n + n_t + i] = -im;
            Hr[(n_r + k) * n + i] = im;
            Hr[(n_r + k) * n + n_t + i] = re;
        }
    }
    double* G = (double*)calloc((size_t)(n * n), sizeof(double));
    double* mf = (double*)calloc((size_t)n, sizeof(double));
    for (int a = 0; a < n; ++a) {
        for (int b = 0; b < n; ++b)
            for (int r = 0; r < 2 * n_r; ++r) G[a * n + b] += Hr[r * n + a] * Hr[r * n + b];
        for (int r = 0; r < 2 * n_r; ++r) mf[a] += Hr[r * n + a] * yr[r];
    }
    double tr = 0.0, yy = 0.0;
    for (int i = 0; i < N; ++i) {
        const int ki = i / B, bi = i % B;
        for (int j = 0; j < N; ++j) {
            const int kj = j / B, bj = j % B;
            const double v = ldexp(G[ki * n + kj], bi + bj);
            if (i == j) tr += v;
            if (J_out) J_out[i * N + j] = i == j ? 0.0 : -v;
        }
        if (c_out) c_out[i] = ldexp(mf[ki], bi);
    }
    for (int r = 0; r < 2 * n_r; ++r) yy += yr[r] * yr[r];
    if (const_out) *const_out = yy + tr;
    free(Hr); free(yr); free(G); free(mf);
    return ORC_OK;
}

/* Lattice symbol x [2 n_t] of spins s [N] (x = T s). */
void orc_direct_lattice(int n_t, int mod_bits, const int8_t* s, int* x)
{
    const int B = mod_bits / 2;
    for (int k = 0; k < 2 * n_t; ++k) {
        int v = 0;
        for (int b = 0; b < B; ++b) v += (1 << b) * (int)s[k * B + b];
        x[k] = v;
    }
}

/* Spins of an alphabet point: s_b = 2 bit_b((x + 2^B - 1) / 2) - 1. */
void orc_direct_spins(int n_t, int mod_bits, const int* x, int8_t* s)
{
    const int B = mod_bits / 2;
    for (int k = 0; k < 2 * n_t; ++k) {
        const int u = (x[k] + (1 << B) - 1) / 2;
        for (int b = 0; b < B; ++b) s[k * B + b] = (int8_t)(((u >> b) & 1) ? 1 : -1);
    }
}

/* Exact quantised energy of spins s: E(s) = -s^T J_q s - 2 c_q^T s (int32),
 * lower is better; equals (||y - Hs T s||^2 - const) 2^14 / sigma up to
 * quantisation. */
int32_t orc_energy_direct(int N, const int16_t* Jq, const int16_t* cq, const int8_t* s)
{
    int32_t e = 0;
    for (int i = 0; i < N; ++i) {
        int32_t r = 0;
        for (int j = 0; j < N; ++j) r += (int32_t)Jq[i * N + j] * (int32_t)s[j];
        e -= (int32_t)s[i] * r;
        e -= 2 * (int32_t)cq[i] * (int32_t)s[i];
    }
    return e;
}

/*
 * FP32 direct build in the pinned order: the FP32 real-form Gram G32 and the
 * MMSE guess g are those of orc_build_detect32; the matched filter
 * mf = Hs^H y follows its pattern (k ascending, from 0); then
 *   J32_ij = -(2^(b_i + b_j) G32_(k_i k_j)) for i != j, 0 on the diagonal,
 *   c32_i  = 2^(b_i) mf_(k_i)
 * (exact scalings), sigma = 2^e the smallest power of two >= max(|J32|, |c32|),
 * Jq = rint(J32 2^(14-e)), cq = rint(c32 2^(14-e)) as int16.
 * Outputs: g [2 n_t], J32 [N*N], c32 [N] (may be NULL), sigma_exp, Jq, cq.
 */
int orc_build_direct32(int n_r, int n_t, int mod_bits, const float* H, const float* y, float noise_var, int* g_out,
                       float* J32_out, float* c32_out, int* sigma_exp_out, int16_t* Jq_out, int16_t* cq_out)
{
    if (n_r < 1 || n_t < 1 || mod_bits < 2 || (mod_bits & 1)) return ORC_EINVAL;
    const int n = 2 * n_t, B = mod_bits / 2, N = n * B;
    float* G = (float*)malloc(sizeof(float) * (size_t)(n * n));
    int16_t* Aq = (int16_t*)malloc(sizeof(int16_t) * (size_t)(n * n));
    int16_t* hq = (int16_t*)malloc(sizeof(int16_t) * (size_t)n);
    int se0;
    int status = orc_build_detect32(n_r, n_t, mod_bits, H, y, noise_var, NULL, g_out, G, NULL, &se0, Aq, hq);
    const float kappa = qam_kappa_f(mod_bits);
    float* mf = (float*)malloc(sizeof(float) * (size_t)n);
    for (int i = 0; i < n_t; ++i) {
        float re = 0.0f, im = 0.0f;
        for (int k = 0; k < n_r; ++k) {
            const float ar = f_mul(kappa, H[2 * (k * n_t + i)]), ai = f_mul(kappa, H[2 * (k * n_t + i) + 1]);
            const float br = y[2 * k], bi = y[2 * k + 1];
            re = fmaf(ar, br, re);
            re = fmaf(ai, bi, re);
            im = fmaf(ar, bi, im);
            im = fmaf(-ai, br, im);
        }
        mf[i] = re;
        mf[n_t + i] = im;
    }
    float* J = (float*)malloc(sizeof(float) * (size_t)(N * N));
    float* c = (float*)malloc(sizeof(float) * (size_t)N);
    float mx = 0.0f;
    for (int i = 0; i < N; ++i) {
        const int ki = i / B, bi = i % B;
        for (int j = 0; j < N; ++j) {
            const int kj = j / B, bj = j % B;
            J[i * N + j] = i == j ? 0.0f : -ldexpf(G[ki * n + kj], bi + bj);
            mx = fmaxf(mx, fabsf(J[i * N + j]));
        }
        c[i] = ldexpf(mf[ki], bi);
        mx = fmaxf(mx, fabsf(c[i]));
    }
    const int se = sigma_exp_f(mx);
    const int finite = isfinite(mx);
    const float s = pow2f(QBITS - se);
    for (int e = 0; e < N * N; ++e) Jq_out[e] = finite ? (int16_t)rintf(f_mul(J[e], s)) : 0;
    for (int i = 0; i < N; ++i) cq_out[i] = finite ? (int16_t)rintf(f_mul(c[i], s)) : 0;
    if (!finite) status = ORC_ENUM;
    if (J32_out) memcpy(J32_out, J, sizeof(float) * (size_t)(N * N));
    if (c32_out) memcpy(c32_out, c, sizeof(float) * (size_t)N);
    if (sigma_exp_out) *sigma_exp_out = se;
    free(G); free(Aq); free(hq); free(mf); free(J); free(c);
    return status;
}

/* Coupling field of a general Ising problem with an auxiliary spin:
 * m_i = sum_j J_ji x_j (j ascending, FMA chain from 0; J symmetric with zero
 * diagonal), mu_i = m_i + c_i x_a, mu_a = sum_j c_j x_j (j ascending).
 * Jf, cf carry eps dt.  x, mu: [N + 1] (x_a last). */
void orc_general_field(int N, const float* Jf, const float* cf, const float* x, float* mu)
{
    const float xa = x[N];
    float mua = 0.0f;
    for (int i = 0; i < N; ++i) {
        float m = 0.0f;
        for (int j = 0; j < N; ++j) m = fmaf(Jf[j * N + i], x[j], m);
        mu[i] = fmaf(cf[i], xa, m);
    }
    for (int j = 0; j < N; ++j) mua = fmaf(cf[j], x[j], mua);
    mu[N] = mua;
}

/*
 * Anneal a general Ising problem (Jq [N*N] symmetric, zero diagonal; cq [N],
 * coupled through the auxiliary spin) with R anneals of the same CIM-CAC
 * dynamics as orc_cac_solve (initial amplitudes: spin k of run r is Philox
 * word k mod 4 of counter (k/4, r, problem), k = N the auxiliary spin).
 * Each anneal's spins s_i = sign(x_i) sign(x_a) (x >= 0 -> +1) are scored by
 * the exact energy E(s); a diverged anneal is not a candidate.  The reference
 * spins s_ref (may be NULL) are candidate -1 and win ties.  The output is the
 * lowest (E, candidate index).
 * Outputs: s_out [N], E_out, run_out (-1: s_ref, or no valid candidate when
 * s_ref is NULL, then s = +1 and E = E(+1)), n_div_out; optional E_runs [R]
 * (INT32_MAX for diverged anneals) and x_final [R][N+1] (final amplitudes,
 * the auxiliary spin last).
 */
int orc_cac_solve_general(int N, const int16_t* Jq, const int16_t* cq, const int8_t* s_ref, const orc_params* P,
                          uint64_t seed, uint64_t problem, int8_t* s_out, int32_t* E_out, int32_t* run_out,
                          int32_t* n_div_out, int32_t* E_runs, float* x_final)
{
    if (N < 1 || P->runs < 1 || P->steps < 0 || P->f_mvm < 1) return ORC_EINVAL;
    orc_consts C;
    orc_cac_consts(P, &C);
    const float q = pow2f(-QBITS);
    float* Jf = (float*)malloc(sizeof(float) * (size_t)(N * N));
    float* cf = (float*)malloc(sizeof(float) * (size_t)N);
    for (int e = 0; e < N * N; ++e) Jf[e] = f_mul(f_mul((float)Jq[e], q), C.ce);
    for (int i = 0; i < N; ++i) cf[i] = f_mul(f_mul((float)cq[i], q), C.ce);
    float* x = (float*)malloc(sizeof(float) * (size_t)(N + 1));
    float* eh = (float*)malloc(sizeof(float) * (size_t)(N + 1));
    float* mu = (float*)malloc(sizeof(float) * (size_t)(N + 1));
    int8_t* s = (int8_t*)malloc((size_t)N);
    int32_t bestE;
    int bestRun = -1, ndiv = 0;
    if (s_ref) {
        memcpy(s_out, s_ref, (size_t)N);
    } else {
        memset(s_out, 1, (size_t)N);
    }
    bestE = orc_energy_direct(N, Jq, cq, s_out);
    int have = s_ref != NULL;
    for (int r = 0; r < P->runs; ++r) {
        for (int k = 0; k <= N; ++k) {
            x[k] = orc_initial_x(seed, problem, r, k, C.xs);
            eh[k] = 1.0f;
        }
        for (int t = 0; t < P->steps; ++t) {
            if (t % P->f_mvm == 0) orc_general_field(N, Jf, cf, x, mu);
            for (int k = 0; k <= N; ++k) euler_spin(&x[k], &eh[k], mu[k], &C);
        }
        if (x_final) memcpy(x_final + (size_t)r * (N + 1), x, sizeof(float) * (size_t)(N + 1));
        int valid = 1;
        for (int k = 0; k <= N; ++k)
            if (!(fabsf(x[k]) <= P->x_max) || !(eh[k] > 0.0f)) valid = 0;
        const int sa = x[N] >= 0.0f ? 1 : -1;
        for (int i = 0; i < N; ++i) s[i] = (int8_t)((x[i] >= 0.0f ? 1 : -1) * sa);
        const int32_t E = valid ? orc_energy_direct(N, Jq, cq, s) : INT32_MAX;
        if (E_runs) E_runs[r] = E;
        if (!valid) {
            ndiv++;
            continue;
        }
        if (!have || E < bestE) {
            bestE = E;
            bestRun = r;
            memcpy(s_out, s, (size_t)N);
            have = 1;
        }
    }
    *E_out = bestE;
    *run_out = bestRun;
    *n_div_out = ndiv;
    free(Jf); free(cf); free(x); free(eh); free(mu); free(s);
    return ORC_OK;
}

/*
 * Uplink detection of one problem with the direct mapping (FP32 mirror):
 * build (orc_build_direct32), anneal with the MMSE guess's spins as the
 * reference candidate, decode x = T s to symbol indices.
 * Outputs: sym [n_t], g (MMSE guess, [2 n_t]), s [N], E, run, n_div.
 */
int orc_detect_direct(int n_r, int n_t, int mod_bits, const float* H, const float* y, float noise_var,
                      const orc_params* P, uint64_t seed, uint64_t problem, uint8_t* sym, int* g, int8_t* s,
                      int32_t* E, int32_t* run, int32_t* n_div)
{
    const int n = 2 * n_t, N = n * (mod_bits / 2);
    int16_t* Jq = (int16_t*)malloc(sizeof(int16_t) * (size_t)(N * N));
    int16_t* cq = (int16_t*)malloc(sizeof(int16_t) * (size_t)N);
    int8_t* sref = (int8_t*)malloc((size_t)N);
    int* x = (int*)malloc(sizeof(int) * (size_t)n);
    int se;
    orc_build_direct32(n_r, n_t, mod_bits, H, y, noise_var, g, NULL, NULL, &se, Jq, cq);
    orc_direct_spins(n_t, mod_bits, g, sref);
    orc_cac_solve_general(N, Jq, cq, sref, P, seed, problem, s, E, run, n_div, NULL, NULL);
    orc_direct_lattice(n_t, mod_bits, s, x);
    int8_t* zero = (int8_t*)calloc((size_t)n, 1);
    orc_decode_detect(n_t, mod_bits, x, zero, sym);
    free(Jq); free(cq); free(sref); free(x); free(zero);
    return ORC_OK;
}
