// Builder: Gram, matched filter, MMSE (or SIC) guess, field and Q14 quantisation,
// one warp per problem (Sec. 3.2 pre-processing, Eqs. 3 and 9, Fig. 5).
#pragma once
#include "common.cuh"

namespace mmgap {

// =========================================================================
// Builder: one warp per problem (resource element).
// =========================================================================
constexpr int kBuildWarps = 4;

template <int NT>
__host__ __device__ constexpr int build_smem_floats(int n_r) {
    // Hs [n_r][NT] c, Gc [NT][NT] c, L [NT][NT] c, y [n_r] c, z [n_r] c, m [NT] c, g [2NT],
    // flag + pivot scratch (perm [NT], d [NT])
    return 2 * n_r * NT + 4 * NT * NT + 4 * n_r + 4 * NT + 4 + 2 * NT;
}

// Where one problem's build writes its results (global or shared memory).
struct BuildOut {
    int16_t* Aq;        // [n][n]
    int16_t* hq;        // [n]
    int8_t* g;          // [n]
    float* G32;         // [n][n] or nullptr
    float* h32;         // [n] or nullptr
    int32_t* sigma_exp; // or nullptr
};

// Tasks t in [t0, t1) of a warp: t < NT^2 the Gram element (i, j) = (t / NT,
// t % NT) of G_c = Hs^H Hs (upper triangle, mirrored), t >= NT^2 the matched
// filter m_i = (Hs^H y)_i, i = t - NT^2.  Each value's FMA order is fixed, so
// it does not depend on which lane (or which kernel) computes it.
template <int NT>
__device__ __forceinline__ void gram_mf_warp(const float* Hs, const float* yv, int n_r, float* Gc, float* mv, int t0,
                                             int t1, int lane) {
    for (int t = t0 + lane; t < t1; t += 32) {
        if (t < NT * NT) {
            const int i = t / NT, j = t % NT;
            if (i > j) continue;
            if (i == j) {
                float acc = 0.0f;
                for (int k = 0; k < n_r; ++k) {
                    const float ar = Hs[2 * (k * NT + i)], ai = Hs[2 * (k * NT + i) + 1];
                    acc = fmarn(ar, ar, acc);
                    acc = fmarn(ai, ai, acc);
                }
                Gc[2 * (i * NT + i)] = acc;
                Gc[2 * (i * NT + i) + 1] = 0.0f;
            } else {
                float re = 0.0f, im = 0.0f;
                for (int k = 0; k < n_r; ++k) {
                    const float ar = Hs[2 * (k * NT + i)], ai = Hs[2 * (k * NT + i) + 1];
                    const float br = Hs[2 * (k * NT + j)], bi = Hs[2 * (k * NT + j) + 1];
                    re = fmarn(ar, br, re);
                    re = fmarn(ai, bi, re);
                    im = fmarn(ar, bi, im);
                    im = fmarn(-ai, br, im);
                }
                Gc[2 * (i * NT + j)] = re;
                Gc[2 * (i * NT + j) + 1] = im;
                Gc[2 * (j * NT + i)] = re;
                Gc[2 * (j * NT + i) + 1] = -im;
            }
        } else {
            const int i = t - NT * NT;
            float re = 0.0f, im = 0.0f;
            for (int k = 0; k < n_r; ++k) {
                const float ar = Hs[2 * (k * NT + i)], ai = Hs[2 * (k * NT + i) + 1];
                const float br = yv[2 * k], bi = yv[2 * k + 1];
                re = fmarn(ar, br, re);
                re = fmarn(ai, bi, re);
                im = fmarn(ar, bi, im);
                im = fmarn(-ai, br, im);
            }
            mv[2 * i] = re;
            mv[2 * i + 1] = im;
        }
    }
}

// Cholesky of B = G_c + rho I (Eq. 3), left-looking, one column per step;
// lane j the pivot, lanes i > j the rest.  MMSE factors in natural order;
// MMSE-SIC (Sec. 3.2.2) pivots on the smallest current Schur diagonal (ties:
// first position), rows of L being positions (perm: position -> user).  L goes
// to Lc (lower triangle); flag[0] is set on a failed pivot (the pivot is then
// taken as 1).  Whole warp.
template <int NT>
__device__ __forceinline__ void cholesky_warp(const float* Gc, float rho, bool sic, float* Lc, int* flag, int* perm,
                                              float* dg, int lane) {
    if (lane < NT) {
        perm[lane] = lane;
        dg[lane] = addrn(Gc[2 * (lane * NT + lane)], rho);
    }
    __syncwarp();
    for (int j = 0; j < NT; ++j) {
        if (sic) {
            if (lane == 0) {
                int best = j;
                for (int i = j + 1; i < NT; ++i)
                    if (dg[perm[i]] < dg[perm[best]]) best = i;
                flag[1] = best;
                const int t = perm[j];
                perm[j] = perm[best];
                perm[best] = t;
            }
            __syncwarp();
            const int best = flag[1];
            if (lane < j && best != j) {  // swap the computed part of rows j and best
                const float r0 = Lc[2 * (j * NT + lane)], r1 = Lc[2 * (j * NT + lane) + 1];
                Lc[2 * (j * NT + lane)] = Lc[2 * (best * NT + lane)];
                Lc[2 * (j * NT + lane) + 1] = Lc[2 * (best * NT + lane) + 1];
                Lc[2 * (best * NT + lane)] = r0;
                Lc[2 * (best * NT + lane) + 1] = r1;
            }
            __syncwarp();
        }
        const int u = sic ? perm[j] : j;
        if (lane == j) {
            float d;
            if (sic) {
                d = dg[u];
            } else {
                d = addrn(Gc[2 * (j * NT + j)], rho);
                for (int k = 0; k < j; ++k) {
                    const float lr = Lc[2 * (j * NT + k)], li = Lc[2 * (j * NT + k) + 1];
                    d = fmarn(-lr, lr, d);
                    d = fmarn(-li, li, d);
                }
            }
            const bool ok = (d > 0.0f) && !isinf(d);
            if (!ok) flag[0] = 1;
            Lc[2 * (j * NT + j)] = ok ? __fsqrt_rn(d) : 1.0f;
            Lc[2 * (j * NT + j) + 1] = 0.0f;
        }
        __syncwarp();
        const float ljj = Lc[2 * (j * NT + j)];
        if (lane > j && lane < NT) {
            const int i = lane;
            const int v = sic ? perm[i] : i;
            float re = Gc[2 * (v * NT + u)], im = Gc[2 * (v * NT + u) + 1];
            for (int k = 0; k < j; ++k) {
                const float ar = Lc[2 * (i * NT + k)], ai = Lc[2 * (i * NT + k) + 1];
                const float br = Lc[2 * (j * NT + k)], bi = Lc[2 * (j * NT + k) + 1];
                re = fmarn(-ar, br, re);
                re = fmarn(-ai, bi, re);
                im = fmarn(-ai, br, im);
                im = fmarn(ar, bi, im);
            }
            const float lr = __fdiv_rn(re, ljj), li = __fdiv_rn(im, ljj);
            Lc[2 * (i * NT + j)] = lr;
            Lc[2 * (i * NT + j) + 1] = li;
            if (sic) {
                float dv = dg[v];
                dv = fmarn(-lr, lr, dv);
                dv = fmarn(-li, li, dv);
                dg[v] = dv;
            }
        }
        __syncwarp();
    }
}

// Build problem p of `a` with one warp; ws = build_smem_floats<NT>(n_r)
// floats of this warp's shared memory.
template <int NT>
__device__ __forceinline__ void build_problem_warp(const BuildArgs& a, int p, int lane, float* ws, const BuildOut& o) {
    constexpr int n = 2 * NT;
    const int n_r = a.n_r;
    float* Hs = ws;
    float* Gc = Hs + 2 * n_r * NT;
    float* Lc = Gc + 2 * NT * NT;
    float* yv = Lc + 2 * NT * NT;
    float* zv = yv + 2 * n_r;
    float* mv = zv + 2 * n_r;  // matched filter [NT] c
    float* gv = mv + 2 * NT;   // g as floats [2NT]
    int* flag = reinterpret_cast<int*>(gv + 2 * NT);
    int* perm = flag + 4;      // position -> user (SIC)
    float* dg = reinterpret_cast<float*>(perm + NT);  // current Schur diagonal per user (SIC)

    const int c = a.chan_index ? a.chan_index[p] : p;
    if (c < 0 || c >= a.n_chan) {  // bad channel index: flag it, emit an all-zero problem
        if (lane == 0 && a.err) atomicOr(a.err, kErrChanIndex);
        if (o.Aq)
            for (int e = lane; e < n * n; e += 32) o.Aq[e] = 0;
        for (int e = lane; e < n; e += 32) {
            if (o.hq) o.hq[e] = 0;
            o.g[e] = 0;
        }
        __syncwarp();
        return;
    }
    const float* Hg = a.H + (size_t)c * 2 * n_r * NT;
    const float* yg = a.y + (size_t)p * 2 * n_r;
    for (int e = lane; e < 2 * n_r * NT; e += 32) Hs[e] = mulrn(a.kappa, Hg[e]);
    for (int e = lane; e < 2 * n_r; e += 32) yv[e] = yg[e];
    if (lane == 0) flag[0] = 0;
    __syncwarp();

    // Gram G_c = Hs^H Hs (upper triangle + Hermitian mirror) and m = Hs^H y.
    // With a precomputed (tensor-core) Gram only the matched filter is formed here.
    const float* Gpre = a.Gc_pre ? a.Gc_pre + (size_t)c * 2 * NT * NT : nullptr;
    if (Gpre)
        for (int e = lane; e < 2 * NT * NT; e += 32) Gc[e] = Gpre[e];
    gram_mf_warp<NT>(Hs, yv, n_r, Gc, mv, Gpre ? NT * NT : 0, NT * NT + NT, lane);
    __syncwarp();

    const int side = 1 << (a.mod_bits >> 1);
    const float Lm = (float)(side - 1);
    auto slice = [&](float v) -> float {  // nearest alphabet point (ties upward)
        float xc = fmaxf(v, -Lm);
        xc = fminf(xc, Lm);
        return (float)(2 * (int)floorf(mulrn(xc, 0.5f)) + 1);
    };
    if (a.guess_mode == 2) {
        // externally supplied guess (a previous stage's solution, or the caller's); an entry that
        // is not an alphabet point (odd, |g| <= sqrt(M) - 1) is used as given and flagged
        bool bad = false;
        if (lane < NT) {
            const int gr = a.g_in[(size_t)p * n + lane], gi = a.g_in[(size_t)p * n + NT + lane];
            const int L = side - 1;
            bad = !(gr & 1) || !(gi & 1) || gr > L || gr < -L || gi > L || gi < -L;
            gv[lane] = (float)gr;
            gv[NT + lane] = (float)gi;
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0 && a.err) atomicOr(a.err, kErrGuess);
        __syncwarp();
    } else {
        // Cholesky of B = G_c + rho I, rho = noise_var kappa^2 (cholesky_warp)
        const bool sic = a.guess_mode == 1;
        const float rho = mulrn(a.noise_var[p], a.kappa2);
        if (!sic && a.L_pre && a.rho_pre[c] == rho) {
            // this channel's factor, made once by chan_factor_kernel with the same rho: the same bits
            const float* Lg = a.L_pre + (size_t)c * 2 * NT * NT;
            for (int e = lane; e < 2 * NT * NT; e += 32) Lc[e] = Lg[e];
            if (lane == 0) flag[0] = a.chol_pre[c];
            __syncwarp();
        } else {
            cholesky_warp<NT>(Gc, rho, sic, Lc, flag, perm, dg, lane);
        }
        const bool chol_failed = flag[0] != 0;

        // forward solve L w = P m (right-looking; per row the updates arrive in
        // ascending k, the same sequence as the left-looking sum)
        float accr = 0.0f, acci = 0.0f;
        if (lane < NT) {
            const int src = sic ? perm[lane] : lane;
            accr = mv[2 * src];
            acci = mv[2 * src + 1];
        }
        float wr = 0.0f, wi = 0.0f;
        for (int k = 0; k < NT; ++k) {
            if (lane == k) {
                const float lkk = Lc[2 * (k * NT + k)];
                wr = __fdiv_rn(accr, lkk);
                wi = __fdiv_rn(acci, lkk);
            }
            const float br = __shfl_sync(0xffffffffu, wr, k), bi = __shfl_sync(0xffffffffu, wi, k);
            if (lane > k && lane < NT) {
                const float ar = Lc[2 * (lane * NT + k)], ai = Lc[2 * (lane * NT + k) + 1];
                accr = fmarn(-ar, br, accr);
                accr = fmarn(ai, bi, accr);
                acci = fmarn(-ar, bi, acci);
                acci = fmarn(-ai, br, acci);
            }
        }
        // backward solve L^H x = w, k descending; SIC slices each x_k before
        // it is substituted (successive interference cancellation)
        accr = wr;
        acci = wi;
        float xr = 0.0f, xi = 0.0f;
        for (int k = NT - 1; k >= 0; --k) {
            if (lane == k) {
                const float lkk = Lc[2 * (k * NT + k)];
                xr = __fdiv_rn(accr, lkk);
                xi = __fdiv_rn(acci, lkk);
                if (sic) {
                    xr = slice(xr);
                    xi = slice(xi);
                }
            }
            const float br = __shfl_sync(0xffffffffu, xr, k), bi = __shfl_sync(0xffffffffu, xi, k);
            if (lane < k) {
                const float ar = Lc[2 * (k * NT + lane)], ai = Lc[2 * (k * NT + lane) + 1];
                accr = fmarn(-ar, br, accr);
                accr = fmarn(-ai, bi, accr);
                acci = fmarn(-ar, bi, acci);
                acci = fmarn(ai, br, acci);
            }
        }
        // hard decision to the nearest alphabet point (ties upward)
        if (lane < NT) {
            const int dst = sic ? perm[lane] : lane;
            gv[dst] = slice(chol_failed ? 0.0f : xr);
            gv[NT + dst] = slice(chol_failed ? 0.0f : xi);
        }
        __syncwarp();
    }

    // residual z = y - Hs g, field h_c = Hs^H z
    for (int k = lane; k < n_r; k += 32) {
        float re = yv[2 * k], im = yv[2 * k + 1];
        for (int j = 0; j < NT; ++j) {
            const float ar = Hs[2 * (k * NT + j)], ai = Hs[2 * (k * NT + j) + 1];
            const float br = gv[j], bi = gv[NT + j];
            re = fmarn(-ar, br, re);
            re = fmarn(ai, bi, re);
            im = fmarn(-ar, bi, im);
            im = fmarn(-ai, br, im);
        }
        zv[2 * k] = re;
        zv[2 * k + 1] = im;
    }
    __syncwarp();
    float hre = 0.0f, him = 0.0f;
    if (lane < NT) {
        for (int k = 0; k < n_r; ++k) {
            const float ar = Hs[2 * (k * NT + lane)], ai = Hs[2 * (k * NT + lane) + 1];
            const float br = zv[2 * k], bi = zv[2 * k + 1];
            hre = fmarn(ar, br, hre);
            hre = fmarn(ai, bi, hre);
            him = fmarn(ar, bi, him);
            him = fmarn(-ai, br, him);
        }
    }

    // power-of-two normaliser over the real-form couplings and field
    float mx = 0.0f;
    for (int e = lane; e < NT * NT; e += 32) mx = fmaxf(mx, fmaxf(fabsf(Gc[2 * e]), fabsf(Gc[2 * e + 1])));
    if (lane < NT) mx = fmaxf(mx, fmaxf(fabsf(hre), fabsf(him)));
    mx = warp_max(mx);
    const int se = sigma_exp_f(mx);
    const bool finite = isfinite(mx);
    const float s = ldexpf(1.0f, kQBits - se);

    if (o.Aq)  // (the direct mapping uses only the guess and the Gram / matched filter left in ws)
        for (int e = lane; e < n * n; e += 32) {
            const int i = e / n, j = e % n;
            const int ib = i % NT, jb = j % NT;
            const float re = Gc[2 * (ib * NT + jb)], im = Gc[2 * (ib * NT + jb) + 1];
            // G = [[Re G_c, -Im G_c], [Im G_c, Re G_c]]
            const float G = (i < NT) == (j < NT) ? re : (i < NT ? -im : im);
            o.Aq[e] = finite ? (int16_t)(int)rintf(mulrn(-G, s)) : (int16_t)0;
            if (o.G32) o.G32[e] = G;
        }
    if (lane < NT) {
        if (o.hq) {
            o.hq[lane] = finite ? (int16_t)(int)rintf(mulrn(hre, s)) : (int16_t)0;
            o.hq[NT + lane] = finite ? (int16_t)(int)rintf(mulrn(him, s)) : (int16_t)0;
        }
        o.g[lane] = (int8_t)(int)gv[lane];
        o.g[NT + lane] = (int8_t)(int)gv[NT + lane];
        if (o.h32) {
            o.h32[lane] = hre;
            o.h32[NT + lane] = him;
        }
    }
    if (lane == 0 && o.sigma_exp) *o.sigma_exp = se;
    __syncwarp();
}

template <int NT>
__global__ void __launch_bounds__(kBuildWarps * 32) build_detect_kernel(BuildArgs a) {
    extern __shared__ __align__(16) float smem[];
    constexpr int n = 2 * NT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * kBuildWarps + warp;
    if (p >= a.n_problems) return;  // warp-uniform; no block-wide barrier below
    BuildOut o;
    o.Aq = a.Aq + (size_t)p * n * n;
    o.hq = a.hq + (size_t)p * n;
    o.g = a.g + (size_t)p * n;
    o.G32 = a.G32 ? a.G32 + (size_t)p * n * n : nullptr;
    o.h32 = a.h32 ? a.h32 + (size_t)p * n : nullptr;
    o.sigma_exp = a.sigma_exp ? a.sigma_exp + p : nullptr;
    build_problem_warp<NT>(a, p, lane, smem + warp * build_smem_floats<NT>(a.n_r), o);
}

// First problem of each channel (atomic minimum over the problems).
template <int NT>
__global__ void chan_first_kernel(ChanFactorArgs a) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < a.n_problems; p += gridDim.x * blockDim.x) {
        const int c = a.chan_index[p];
        if (c >= 0 && c < a.n_chan) atomicMin(a.first + c, p);
    }
}

// Channel c of `a` with one warp: Hs = kappa H, the Gram and the MMSE Cholesky
// factor with rho of the channel's first problem -- the same functions and
// shared memory layout as build_problem_warp, so a problem with that rho finds
// the bits its own factorisation would give.  ws: build_smem_floats<NT>(n_r)
// floats of this warp's shared memory.
template <int NT>
__device__ __forceinline__ void chan_factor_warp(const ChanFactorArgs& a, int c, int lane, float* ws) {
    const int p0 = a.first[c];
    if (p0 < 0 || p0 >= a.n_problems) {
        if (lane == 0) a.rho_out[c] = __int_as_float(0x7fc00000);  // NaN: no problem compares equal
        return;
    }
    const int n_r = a.n_r;
    float* Hs = ws;
    float* Gc = Hs + 2 * n_r * NT;
    float* Lc = Gc + 2 * NT * NT;
    float* yv = Lc + 2 * NT * NT;
    float* zv = yv + 2 * n_r;
    float* mv = zv + 2 * n_r;
    float* gv = mv + 2 * NT;
    int* flag = reinterpret_cast<int*>(gv + 2 * NT);
    int* perm = flag + 4;
    float* dg = reinterpret_cast<float*>(perm + NT);
    const float* Hg = a.H + (size_t)c * 2 * n_r * NT;
    for (int e = lane; e < 2 * n_r * NT; e += 32) Hs[e] = mulrn(a.kappa, Hg[e]);
    if (lane == 0) flag[0] = 0;
    __syncwarp();
    gram_mf_warp<NT>(Hs, yv, n_r, Gc, mv, 0, NT * NT, lane);
    __syncwarp();
    if (a.G_out) {  // the channel's Gram, for every problem of the channel (the same function, the same bits)
        float* Gg = a.G_out + (size_t)c * 2 * NT * NT;
        for (int e = lane; e < 2 * NT * NT; e += 32) Gg[e] = Gc[e];
    }
    const float rho = mulrn(a.noise_var[p0], a.kappa2);
    cholesky_warp<NT>(Gc, rho, false, Lc, flag, perm, dg, lane);
    float* Lg = a.L_out + (size_t)c * 2 * NT * NT;
    for (int e = lane; e < 2 * NT * NT; e += 32) Lg[e] = Lc[e];
    if (lane == 0) {
        a.rho_out[c] = rho;
        a.chol_out[c] = flag[0];
    }
}

// One warp per channel (chan_factor_warp).
template <int NT>
__global__ void __launch_bounds__(kBuildWarps * 32) chan_factor_kernel(ChanFactorArgs a) {
    extern __shared__ __align__(16) float smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * kBuildWarps + warp;
    if (c >= a.n_chan) return;  // warp-uniform
    chan_factor_warp<NT>(a, c, lane, smem + warp * build_smem_floats<NT>(a.n_r));
}

}  // namespace mmgap
