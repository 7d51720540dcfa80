/*
 * A plain C client of the library's ABI (include/mmgap.h), with no Python in
 * the process: it reads one detection job from a binary file, copies it to the
 * device, runs mmgap_detect and mmgap_detect_static on it, and writes both
 * results back to a file for the test to compare with the CPU oracle.
 *
 * Input file (little-endian): int32 n_r, n_t, mod_bits, P, n_chan, steps;
 * uint64 seed; float H[n_chan][n_r][n_t][2]; float y[P][n_r][2];
 * float noise_var[P]; int32 chan_index[P].
 * Output file: uint8 sym[P][n_t] and int32 energy[P] from mmgap_detect, then
 * the same two arrays from mmgap_detect_static.
 * Exit status 0 on success; a failing call prints its status and message.
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "mmgap.h"

#define CHECK_CUDA(x)                                                              \
    do {                                                                           \
        cudaError_t e_ = (x);                                                      \
        if (e_ != cudaSuccess) {                                                   \
            fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));               \
            return 2;                                                              \
        }                                                                          \
    } while (0)

static int read_all(FILE* f, void* p, size_t n) { return fread(p, 1, n, f) == n ? 0 : -1; }

int main(int argc, char** argv) {
    if (argc != 3) {
        fprintf(stderr, "usage: %s job.bin out.bin\n", argv[0]);
        return 1;
    }
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 1;
    int32_t hdr[6];
    uint64_t seed;
    if (read_all(f, hdr, sizeof hdr) || read_all(f, &seed, sizeof seed)) return 1;
    const int n_r = hdr[0], n_t = hdr[1], mod_bits = hdr[2], P = hdr[3], n_chan = hdr[4], steps = hdr[5];
    const size_t hb = (size_t)n_chan * n_r * n_t * 2 * sizeof(float), yb = (size_t)P * n_r * 2 * sizeof(float);
    float* H = (float*)malloc(hb);
    float* y = (float*)malloc(yb);
    float* nv = (float*)malloc((size_t)P * sizeof(float));
    int32_t* ci = (int32_t*)malloc((size_t)P * sizeof(int32_t));
    if (!H || !y || !nv || !ci) return 1;
    if (read_all(f, H, hb) || read_all(f, y, yb) || read_all(f, nv, (size_t)P * 4) || read_all(f, ci, (size_t)P * 4))
        return 1;
    fclose(f);

    void *dH, *dy, *dnv, *dci, *dsym, *dE;
    CHECK_CUDA(cudaMalloc(&dH, hb));
    CHECK_CUDA(cudaMalloc(&dy, yb));
    CHECK_CUDA(cudaMalloc(&dnv, (size_t)P * 4));
    CHECK_CUDA(cudaMalloc(&dci, (size_t)P * 4));
    CHECK_CUDA(cudaMalloc(&dsym, (size_t)P * n_t));
    CHECK_CUDA(cudaMalloc(&dE, (size_t)P * 4));
    CHECK_CUDA(cudaMemcpy(dH, H, hb, cudaMemcpyHostToDevice));
    CHECK_CUDA(cudaMemcpy(dy, y, yb, cudaMemcpyHostToDevice));
    CHECK_CUDA(cudaMemcpy(dnv, nv, (size_t)P * 4, cudaMemcpyHostToDevice));
    CHECK_CUDA(cudaMemcpy(dci, ci, (size_t)P * 4, cudaMemcpyHostToDevice));

    mmgap_params prm;
    mmgap_default_params(&prm);
    prm.steps = steps;
    mmgap_detect_job job;
    memset(&job, 0, sizeof job);
    job.n_r = n_r;
    job.n_t = n_t;
    job.mod_bits = mod_bits;
    job.n_problems = P;
    job.n_chan = n_chan;
    job.chan_index = (const int32_t*)dci;
    job.H = (const float*)dH;
    job.y = (const float*)dy;
    job.noise_var = (const float*)dnv;
    job.seed = seed;
    job.sym_out = (uint8_t*)dsym;
    job.energy_out = (int32_t*)dE;

    uint8_t* sym = (uint8_t*)malloc((size_t)P * n_t);
    int32_t* E = (int32_t*)malloc((size_t)P * 4);
    FILE* o = fopen(argv[2], "wb");
    if (!sym || !E || !o) return 1;

    mmgap_ctx* ctx = NULL;
    mmgap_status st = mmgap_create(&ctx, 0, 0);
    if (st != MMGAP_OK) {
        fprintf(stderr, "mmgap_create: %d\n", (int)st);
        return 3;
    }
    st = mmgap_detect(ctx, &prm, &job, 1, NULL);
    if (st != MMGAP_OK) {
        fprintf(stderr, "mmgap_detect: %d %s\n", (int)st, mmgap_last_error(ctx));
        return 3;
    }
    CHECK_CUDA(cudaDeviceSynchronize());
    CHECK_CUDA(cudaMemcpy(sym, dsym, (size_t)P * n_t, cudaMemcpyDeviceToHost));
    CHECK_CUDA(cudaMemcpy(E, dE, (size_t)P * 4, cudaMemcpyDeviceToHost));
    fwrite(sym, 1, (size_t)P * n_t, o);
    fwrite(E, 4, (size_t)P, o);

    CHECK_CUDA(cudaMemset(dsym, 0xff, (size_t)P * n_t));
    st = mmgap_detect_static(&prm, &job, NULL);
    if (st != MMGAP_OK) {
        fprintf(stderr, "mmgap_detect_static: %d\n", (int)st);
        return 3;
    }
    CHECK_CUDA(cudaDeviceSynchronize());
    CHECK_CUDA(cudaMemcpy(sym, dsym, (size_t)P * n_t, cudaMemcpyDeviceToHost));
    CHECK_CUDA(cudaMemcpy(E, dE, (size_t)P * 4, cudaMemcpyDeviceToHost));
    fwrite(sym, 1, (size_t)P * n_t, o);
    fwrite(E, 4, (size_t)P, o);
    fclose(o);
    mmgap_destroy(ctx);
    return 0;
}
