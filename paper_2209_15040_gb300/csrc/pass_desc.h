// Per-launch arguments of a superstep kernel and the launcher entry points
// that the host plan code calls (one set per storage type).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <utility>

namespace wsfft {

// Dynamic shared memory above 48 KB must be enabled per kernel, and the
// setting belongs to the current device: launchers call this before every
// launch and it sets the attribute once per (kernel, device).
inline cudaError_t set_smem_attr(const void *kernel, int bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> set;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_pair(kernel, dev);
    if (set.count(key)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) set[key] = bytes;
    return e;
}

struct PassArgs {
    int64_t npencils;   // outer * inner pencils in this launch
    int64_t inner;      // element stride between consecutive pencil elements
    int log_inner;      // log2(inner)
    const float2 *tw;   // stage twiddle table of this (N, E) schedule
    float conj_in;      // +1, or -1 to conjugate every loaded value
    float sx, sy;       // store scale of re and im (sy = -sx conjugates)
    int64_t trans_rows; // contiguous transposed store: rows per transform
    const float2 *tw_hi;  // four-step twiddle w_L^m = tw_hi[m >> tw_shift] * tw_lo[m & (2^tw_shift - 1)]
    const float2 *tw_lo;
    int tw_shift;
    int tw_mask;        // four-step twiddle: L - 1
    int64_t tile0;      // strided launches: index of the first tile (set by the launcher)
    int *status;        // plan's device status word (kernels with bounded waits)
    uint64_t timeout_ns;  // bound of each wait
    int reverse;        // strided launches: 1 = blocks take the tiles from the last one down
};

// tile codes at or above this select the complex64 pencil-pair strided
// kernel with (code - PAIR_TILE) pencils per block
constexpr int PAIR_TILE = 1000;
// tile code of the tensor-core contiguous superstep (16-bit storage, N = 512)
constexpr int TC_TILE = 2000;
// its table (device, 16-byte aligned), in float2 units:
//   [0, 128)    B_hi of the DFT-16 in the K-major no-swizzle core-matrix byte order
//   [128, 256)  B_lo, same order
//   [256, 768)  w512^(k1*n2) at 256 + n2*16 + k1 (k1 in [0,16), n2 in [0,32))
constexpr int TC_TABLE_TW = 256;
constexpr int TC_TABLE_FLOAT2 = 768;
// tile codes at or above this select the split-form pencil-pair strided
// kernel (packed FP32x2 butterflies) with (code - SPLIT_TILE) pencils per block
constexpr int SPLIT_TILE = 3000;

enum PassKind {
    PASS_CONTIG = 0,     // one launch, contiguous axis
    PASS_STRIDED = 1,    // one launch, strided axis
    PASS_ENGINE_A = 2,   // pipelined engine: z and y of every slab
    PASS_ENGINE_B = 3,   // pipelined engine: x
    PASS_PERSIST_A = 4,  // persistent kernel: z and y of every slab
    PASS_WP_A = 5,       // warp-per-pencil persistent kernel: z and y of every slab
    PASS_WP_B = 6,       // warp-per-pencil strided superstep: x
    PASS_SLAB_A = 7,     // cluster-fused z and y of every n x n slab (slab_cluster.cuh)
};

// Launch one superstep.  variant: contiguous -> transposed store,
// strided -> four-step twiddle on store.  tile: 0 = the default tile shape
// for (N, E); otherwise pencils per block (P or W) of an extra instantiated
// shape.  Returns cudaErrorInvalidValue for a combination the library does
// not instantiate.
cudaError_t launch_pass_c32(int kind, int N, int E, int tile, bool variant, const void *in,
                            void *out, const PassArgs &a, cudaStream_t st);
cudaError_t launch_pass_c16f(int kind, int N, int E, int tile, bool variant, const void *in,
                             void *out, const PassArgs &a, cudaStream_t st);
cudaError_t launch_pass_c16bf(int kind, int N, int E, int tile, bool variant, const void *in,
                              void *out, const PassArgs &a, cudaStream_t st);

}  // namespace wsfft
