// wsfft_transpose_outer: out[b][a][c] = in[a][b][c].
//
// The redistribution step of a transform whose array is split over several
// GPUs (Section 2.1: each processor holds a slab or pencils; Section 4.3:
// between supersteps the data is redistributed so that the next axis is
// local).  Before an all-to-all, each rank's slab [a = local rows][b =
// destination rank][c = the destination's share of a row] is regrouped by
// destination, [b][a][c], so that what goes to one rank is one contiguous
// run; after the all-to-all of the inverse the received [source][a][c]
// chunks are put back in row order the same way.  The last axis c is copied
// as a whole run, so the kernel moves 16-byte vectors whenever c's byte
// length and both pointers allow it: a plain HBM-bound copy (one read and
// one write of the array).
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/wsfft.h"

namespace wsfft {
namespace {

// V: vector type moved per access; c counted in vectors.  Block (x, y)
// copies chunk y (up to 1024 vectors; then y + gridDim.y, ...) of run
// x = a*B + b; its 256 threads
// take consecutive vectors, four each, so every warp access is a contiguous
// 512-byte run of both arrays (16-byte vectors) and four loads are in flight
// per thread.
constexpr int kChunk = 1024;

template <class V>
__global__ void __launch_bounds__(256) transpose_outer_kernel(const V *__restrict__ in, V *__restrict__ out,
                                                              int64_t A, int B, int64_t Cv) {
    const int64_t run = blockIdx.x;
    const int64_t a = run / B, b = run - a * B;
    const V *src = in + run * Cv;
    V *dst = out + (b * A + a) * Cv;
    // chunks of one run: blockIdx.y, then every gridDim.y-th (runs of more
    // than 65535 chunks)
    for (int64_t ch = blockIdx.y; ch * kChunk < Cv; ch += gridDim.y) {
        const int64_t c0 = ch * kChunk + threadIdx.x;
        V v[kChunk / 256];
#pragma unroll
        for (int k = 0; k < kChunk / 256; ++k)
            if (c0 + k * 256 < Cv) v[k] = src[c0 + k * 256];
#pragma unroll
        for (int k = 0; k < kChunk / 256; ++k)
            if (c0 + k * 256 < Cv) dst[c0 + k * 256] = v[k];
    }
}

template <class V>
cudaError_t launch_transpose(const void *in, void *out, int64_t A, int64_t B, int64_t Cv, cudaStream_t st) {
    const int64_t runs = A * B;
    int64_t chunks = (Cv + kChunk - 1) / kChunk;
    if (chunks > 65535) chunks = 65535;
    if (runs > 0x7fffffffLL || B > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    transpose_outer_kernel<V><<<dim3((unsigned)runs, (unsigned)chunks), 256, 0, st>>>(
        static_cast<const V *>(in), static_cast<V *>(out), A, (int)B, Cv);
    return cudaGetLastError();
}

}  // namespace
}  // namespace wsfft

extern "C" int wsfft_transpose_outer(const void *in, void *out, int64_t a, int64_t b, int64_t c, int dtype,
                                     wsfft_stream stream) {
    if (!in || !out || in == out || a < 1 || b < 1 || c < 1) return WSFFT_ERR_INVALID_ARG;
    if (dtype != WSFFT_C32 && dtype != WSFFT_C16F && dtype != WSFFT_C16BF) return WSFFT_ERR_INVALID_ARG;
    const int64_t eb = dtype == WSFFT_C32 ? 8 : 4;
    const int64_t bytes = a * b * c * eb;
    const char *pi = static_cast<const char *>(in);
    const char *po = static_cast<const char *>(out);
    if (pi < po + bytes && po < pi + bytes) return WSFFT_ERR_INVALID_ARG;  // overlapping
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t run = c * eb;  // bytes per (a, b) run
    const uintptr_t al = (uintptr_t)in | (uintptr_t)out;
    cudaError_t e;
    if (run % 16 == 0 && al % 16 == 0) e = wsfft::launch_transpose<uint4>(in, out, a, b, run / 16, st);
    else if (run % 8 == 0 && al % 8 == 0) e = wsfft::launch_transpose<uint2>(in, out, a, b, run / 8, st);
    else e = wsfft::launch_transpose<uint32_t>(in, out, a, b, run / 4, st);
    if (e == cudaErrorInvalidConfiguration) return WSFFT_ERR_UNSUPPORTED;
    return e == cudaSuccess ? WSFFT_SUCCESS : WSFFT_ERR_CUDA;
}
