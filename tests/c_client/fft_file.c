/* A plain C user of the library: no Python, no torch.  Reads `batch` arrays
 * of shape dims (interleaved re, im in the storage type) from a file, runs
 * one wsfft plan over them on the device and writes the result to another
 * file.  Used by the tests to check the C ABI from C.
 *
 *   fft_file IN OUT DTYPE DIRECTION BATCH D0 [D1 [D2]]
 *
 * DTYPE is a wsfft_dtype (0 complex64, 1 FP16 pairs, 2 BF16 pairs);
 * DIRECTION is -1 (forward) or 1 (inverse); exit status 0 on success, else
 * the step that failed is printed with the library's status string. */
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "wsfft.h"

static int fail_cuda(const char *what, cudaError_t e) {
    fprintf(stderr, "%s: %s\n", what, cudaGetErrorString(e));
    return 2;
}

static int fail_wsfft(const char *what, int st) {
    fprintf(stderr, "%s: %s\n", what, wsfft_status_string(st));
    return 3;
}

int main(int argc, char **argv) {
    if (argc < 7 || argc > 9) {
        fprintf(stderr, "usage: %s IN OUT DTYPE DIRECTION BATCH D0 [D1 [D2]]\n", argv[0]);
        return 1;
    }
    const int dtype = atoi(argv[3]);
    const int direction = atoi(argv[4]);
    const int64_t batch = atoll(argv[5]);
    const int rank = argc - 6;
    int64_t dims[3] = {1, 1, 1};
    int64_t elems = batch;
    for (int i = 0; i < rank; ++i) {
        dims[i] = atoll(argv[6 + i]);
        elems *= dims[i];
    }
    const size_t elem_bytes = dtype == WSFFT_C32 ? 8 : 4;
    const size_t bytes = (size_t)elems * elem_bytes;
    unsigned char *host = (unsigned char *)malloc(bytes);
    if (!host) return 1;
    FILE *f = fopen(argv[1], "rb");
    if (!f || fread(host, 1, bytes, f) != bytes) {
        fprintf(stderr, "cannot read %s\n", argv[1]);
        return 1;
    }
    fclose(f);

    void *d_in = NULL, *d_out = NULL;
    cudaError_t e = cudaMalloc(&d_in, bytes);
    if (e != cudaSuccess) return fail_cuda("cudaMalloc", e);
    e = cudaMalloc(&d_out, bytes);
    if (e != cudaSuccess) return fail_cuda("cudaMalloc", e);
    e = cudaMemcpy(d_in, host, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail_cuda("cudaMemcpy in", e);

    wsfft_plan plan = NULL;
    int st = wsfft_plan_create(&plan, dims, rank, dtype, direction, batch);
    if (st != WSFFT_SUCCESS) return fail_wsfft("wsfft_plan_create", st);
    st = wsfft_execute(plan, d_in, d_out, NULL);
    if (st != WSFFT_SUCCESS) return fail_wsfft("wsfft_execute", st);
    st = wsfft_plan_sync_status(plan, NULL);
    if (st != WSFFT_SUCCESS) return fail_wsfft("wsfft_plan_sync_status", st);
    st = wsfft_destroy(plan);
    if (st != WSFFT_SUCCESS) return fail_wsfft("wsfft_destroy", st);

    e = cudaMemcpy(host, d_out, bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail_cuda("cudaMemcpy out", e);
    cudaFree(d_in);
    cudaFree(d_out);
    f = fopen(argv[2], "wb");
    if (!f || fwrite(host, 1, bytes, f) != bytes) {
        fprintf(stderr, "cannot write %s\n", argv[2]);
        return 1;
    }
    fclose(f);
    free(host);
    return 0;
}
