// Tensor-core Gram precision variant and the MMGaP-E candidate selection.
#pragma once
#include "build.cuh"
#include "solve.cuh"

namespace mmgap {

// =========================================================================
// Precision variant of the Gram (pre-processing, Sec. 3.2): G_c = Hs^H Hs per
// channel with mma.sync m16n8k16 (BF16, FP16 or split BF16x3 operands, FP32
// accumulation).
// With A = [Re Hs^T | Im Hs^T] (n_t x 2 n_r):
//   Re G_c = A [Re Hs; Im Hs],   Im G_c = A [Im Hs; -Re Hs].
// One warp per channel; n_t <= 16 (rows padded to 16), 2 n_r padded to a
// multiple of 16.  Each element of Hs = kappa H is rounded once to FP32 and
// once to the 16-bit type.
// =========================================================================
template <int NT>
__global__ void __launch_bounds__(128) gram_tc_kernel(GramArgs a) {
    static_assert(NT <= 16, "one 16-row tile");
    extern __shared__ __align__(16) float gsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * 4 + warp;
    if (c >= a.n_chan) return;
    const int n_r = a.n_r;
    const int K = (2 * n_r + 15) / 16 * 16;
    float* Hs = gsm + (size_t)warp * 2 * kMaxNr * NT;  // [n_r][NT] complex
    const float* Hg = a.H + (size_t)c * 2 * n_r * NT;
    for (int e = lane; e < 2 * n_r * NT; e += 32) Hs[e] = mulrn(a.kappa, Hg[e]);
    __syncwarp();
    // element (k', col) of the stacked operands, zero outside the matrix
    auto At = [&](int row, int kk) -> float {  // A[row][kk] = [Re Hs^T | Im Hs^T]
        if (row >= NT || kk >= 2 * n_r) return 0.0f;
        return kk < n_r ? Hs[2 * (kk * NT + row)] : Hs[2 * ((kk - n_r) * NT + row) + 1];
    };
    auto Bre = [&](int kk, int col) -> float {  // [Re Hs; Im Hs]
        if (col >= NT || kk >= 2 * n_r) return 0.0f;
        return kk < n_r ? Hs[2 * (kk * NT + col)] : Hs[2 * ((kk - n_r) * NT + col) + 1];
    };
    auto Bim = [&](int kk, int col) -> float {  // [Im Hs; -Re Hs]
        if (col >= NT || kk >= 2 * n_r) return 0.0f;
        return kk < n_r ? Hs[2 * (kk * NT + col) + 1] : -Hs[2 * ((kk - n_r) * NT + col)];
    };
    const int gid = lane >> 2, tig = lane & 3;
    constexpr int NTILES = (NT + 7) / 8;
    float re[NTILES][4], im[NTILES][4];
#pragma unroll
    for (int t = 0; t < NTILES; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) re[t][q] = im[t][q] = 0.0f;
    // split operands (BF16x3): v = hi + lo with hi = bf16(v), lo = bf16(v - hi);
    // products hi*hi + hi*lo + lo*hi
    const int fp16 = a.fp16 == 1;
    const bool split = a.fp16 == 2;
    auto hi = [&](float v) -> float { return split ? __bfloat162float(__float2bfloat16_rn(v)) : v; };
    auto lo = [&](float v) -> float { return __fsub_rn(v, hi(v)); };
    for (int k0 = 0; k0 < K; k0 += 16) {
        const float av[8] = {At(gid, k0 + 2 * tig), At(gid, k0 + 2 * tig + 1), At(gid + 8, k0 + 2 * tig),
                             At(gid + 8, k0 + 2 * tig + 1), At(gid, k0 + 2 * tig + 8), At(gid, k0 + 2 * tig + 9),
                             At(gid + 8, k0 + 2 * tig + 8), At(gid + 8, k0 + 2 * tig + 9)};
        uint32_t fa[4], fal[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            fa[r] = pack16(hi(av[2 * r]), hi(av[2 * r + 1]), fp16);
            fal[r] = pack16(lo(av[2 * r]), lo(av[2 * r + 1]), fp16);
        }
#pragma unroll
        for (int t = 0; t < NTILES; ++t) {
            const int col = 8 * t + gid;
            const float rv[4] = {Bre(k0 + 2 * tig, col), Bre(k0 + 2 * tig + 1, col), Bre(k0 + 2 * tig + 8, col),
                                 Bre(k0 + 2 * tig + 9, col)};
            const float iv[4] = {Bim(k0 + 2 * tig, col), Bim(k0 + 2 * tig + 1, col), Bim(k0 + 2 * tig + 8, col),
                                 Bim(k0 + 2 * tig + 9, col)};
            uint32_t br[2], bi[2], brl[2], bil[2];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                br[r] = pack16(hi(rv[2 * r]), hi(rv[2 * r + 1]), fp16);
                bi[r] = pack16(hi(iv[2 * r]), hi(iv[2 * r + 1]), fp16);
                brl[r] = pack16(lo(rv[2 * r]), lo(rv[2 * r + 1]), fp16);
                bil[r] = pack16(lo(iv[2 * r]), lo(iv[2 * r + 1]), fp16);
            }
            if (split) {  // small terms first
                mma16816(re[t], fal, br, 0);
                mma16816(re[t], fa, brl, 0);
                mma16816(im[t], fal, bi, 0);
                mma16816(im[t], fa, bil, 0);
            }
            mma16816(re[t], fa, br, fp16);
            mma16816(im[t], fa, bi, fp16);
        }
    }
    // accumulator (row, col): [0] (gid, 2tig) [1] (gid, 2tig+1) [2] (gid+8, 2tig) [3] (gid+8, 2tig+1);
    // write the upper triangle and its Hermitian mirror
    float* G = a.Gc + (size_t)c * 2 * NT * NT;
#pragma unroll
    for (int t = 0; t < NTILES; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int row = gid + (q >= 2 ? 8 : 0), col = 8 * t + 2 * tig + (q & 1);
            if (row >= NT || col >= NT || row > col) continue;
            const float r = re[t][q], m = row == col ? 0.0f : im[t][q];
            G[2 * (row * NT + col)] = r;
            G[2 * (row * NT + col) + 1] = m;
            G[2 * (col * NT + row)] = r;
            G[2 * (col * NT + row) + 1] = -m;
        }
}

template <int NT>
cudaError_t launch_gram_tc_impl(const GramArgs& a, cudaStream_t s) {
    if (a.n_chan <= 0) return cudaSuccess;
    if constexpr (NT > 16) {
        return cudaErrorInvalidValue;
    } else {
        const size_t smem = (size_t)4 * 2 * kMaxNr * NT * sizeof(float);
        cudaError_t err =
            ensure_dynamic_smem<gram_tc_kernel<NT>>(smem);
        if (err != cudaSuccess) return err;
        gram_tc_kernel<NT><<<(a.n_chan + 3) / 4, 128, smem, s>>>(a);
        return cudaGetLastError();
    }
}

// =========================================================================
// MMGaP-E selection (Sec. 3.2.2: the overall best solution is the output):
// one warp per problem evaluates ||y - Hs x||^2 of every lattice candidate in
// FP32 (residual r_k = y_k - sum_j Hs_kj x_j with j ascending, lanes over k;
// then lane 0 sums k ascending) and keeps the first smallest.
// =========================================================================
template <int NT>
__global__ void __launch_bounds__(128) select_kernel(SelectArgs a) {
    extern __shared__ __align__(16) float ssel[];
    constexpr int n = 2 * NT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * 4 + warp;
    if (p >= a.n_problems) return;
    const int n_r = a.n_r;
    float* Hs = ssel + (size_t)warp * (2 * kMaxNr * NT + 2 * kMaxNr + 2 * kMaxNr);
    float* yv = Hs + 2 * kMaxNr * NT;
    float* rr = yv + 2 * kMaxNr;
    int c = a.chan_index ? a.chan_index[p] : p;
    if (c < 0 || c >= a.n_chan) c = 0;  // flagged by the build stage
    const float* Hg = a.H + (size_t)c * 2 * n_r * NT;
    for (int e = lane; e < 2 * n_r * NT; e += 32) Hs[e] = mulrn(a.kappa, Hg[e]);
    for (int e = lane; e < 2 * n_r; e += 32) yv[e] = a.y[(size_t)p * 2 * n_r + e];
    __syncwarp();
    float best_obj = 0.0f;
    int best = 0;
    for (int cand = 0; cand < a.n_cand; ++cand) {
        const int8_t* x = a.cand + ((size_t)cand * a.n_problems + p) * n;
        for (int k = lane; k < n_r; k += 32) {
            float re = yv[2 * k], im = yv[2 * k + 1];
            for (int j = 0; j < NT; ++j) {
                const float ar = Hs[2 * (k * NT + j)], ai = Hs[2 * (k * NT + j) + 1];
                const float br = (float)x[j], bi = (float)x[NT + j];
                re = fmarn(-ar, br, re);
                re = fmarn(ai, bi, re);
                im = fmarn(-ar, bi, im);
                im = fmarn(-ai, br, im);
            }
            rr[2 * k] = re;
            rr[2 * k + 1] = im;
        }
        __syncwarp();
        if (lane == 0) {
            float obj = 0.0f;
            for (int k = 0; k < n_r; ++k) {
                obj = fmarn(rr[2 * k], rr[2 * k], obj);
                obj = fmarn(rr[2 * k + 1], rr[2 * k + 1], obj);
            }
            if (cand == 0 || obj < best_obj) {
                best_obj = obj;
                best = cand;
            }
        }
        __syncwarp();
    }
    best = __shfl_sync(0xffffffffu, best, 0);
    const int8_t* x = a.cand + ((size_t)best * a.n_problems + p) * n;
    const int side = 1 << (a.mod_bits >> 1), L = side - 1;
    if (lane < NT) {
        const int xr = x[lane], xi = x[NT + lane];
        a.sym_out[(size_t)p * NT + lane] = (uint8_t)(((xr + L) / 2) * side + (xi + L) / 2);
    }
    if (lane == 0) {
        if (a.best_out) a.best_out[p] = best;
        if (a.obj_out) a.obj_out[p] = best_obj;
    }
}

template <int NT>
cudaError_t launch_select_impl(const SelectArgs& a, cudaStream_t s) {
    if (a.n_problems <= 0) return cudaSuccess;
    const size_t smem = (size_t)4 * (2 * kMaxNr * NT + 4 * kMaxNr) * sizeof(float);
    cudaError_t err = ensure_dynamic_smem<select_kernel<NT>>(smem);
    if (err != cudaSuccess) return err;
    select_kernel<NT><<<(a.n_problems + 3) / 4, 128, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mmgap
