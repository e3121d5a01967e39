// Host-visible interface of the persistent engine (engine.cuh).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace wsfft {

struct EngArgs;

// Pencil lengths the engine is built for (cubes n^3 use it for both passes);
// each has tiles of 8192 elements: P = W = 8192 / n pencils, 16 values per
// thread, 512 consumer threads + one producer warp per block.
inline bool engine_supports(int n) { return n == 128 || n == 256 || n == 512 || n == 1024; }
// tiles per queue item of the persistent kernel (the 512 instantiation groups them)
#ifndef WSFFT_PERSIST_SUB
#define WSFFT_PERSIST_SUB 2
#endif
inline int persist_sub(int n) { return n == 512 ? WSFFT_PERSIST_SUB : 1; }
// shape of the persistent 512 kernel's tiles: 1 = contiguous tiles of 8
// pencils and strided tiles of 16 pencils with 32 values per thread; 0 =
// contiguous tiles of 16 pencils and strided tiles of 8 pencil pairs with 8
// values per pencil
#ifndef WSFFT_PERSIST512_E32
#define WSFFT_PERSIST512_E32 0
#endif
inline int persist512_tile_z() { return WSFFT_PERSIST512_E32 ? 8 : 16; }
inline int persist512_values_y() { return WSFFT_PERSIST512_E32 ? 32 : 8; }
inline int engine_tile_pencils(int n) { return 8192 / n; }

// Persistent one-ticket-per-block kernel (persist.cuh).  grid_per_sm != NULL:
// only report how many blocks fit on one SM.
cudaError_t launch_persist_c32(int n, const EngArgs &a, int s_mode, int *grid_per_sm, int grid,
                               cudaStream_t st);
cudaError_t launch_persist_c16f(int n, const EngArgs &a, int s_mode, int *grid_per_sm, int grid,
                                cudaStream_t st);
cudaError_t launch_persist_c16bf(int n, const EngArgs &a, int s_mode, int *grid_per_sm, int grid,
                                 cudaStream_t st);

// Warp-per-pencil kernels (warp_kernels.cuh): persistent pass A of an n^3
// cube (n in {128, 256, 512}), and a one-tile-per-block strided superstep.
struct WpStridedArgs {
    const void *in;
    void *out;
    int64_t inner;
    int log_inner;
    int64_t npencils;
    const float2 *tw;
    float ci, sx, sy;
};
inline bool wp_supports(int n) { return n == 128 || n == 256 || n == 512; }
// pencils per contiguous tile and per strided tile
inline int wp_tile_z(int n) { return 8 * (32 / (n / 16)); }
inline int wp_tile_y(int n) { return wp_tile_z(n) < 16 ? 16 : wp_tile_z(n); }
cudaError_t launch_wpp_c32(int n, const EngArgs &a, int *grid_per_sm, int grid, cudaStream_t st);
cudaError_t launch_wpp_c16f(int n, const EngArgs &a, int *grid_per_sm, int grid, cudaStream_t st);
cudaError_t launch_wpp_c16bf(int n, const EngArgs &a, int *grid_per_sm, int grid, cudaStream_t st);
cudaError_t launch_wps_c32(int n, const WpStridedArgs &b, cudaStream_t st);
cudaError_t launch_wps_c16f(int n, const WpStridedArgs &b, cudaStream_t st);
cudaError_t launch_wps_c16bf(int n, const WpStridedArgs &b, cudaStream_t st);

cudaError_t launch_engine_c32(int n, const EngArgs &a, int grid, cudaStream_t st);
cudaError_t launch_engine_c16f(int n, const EngArgs &a, int grid, cudaStream_t st);
cudaError_t launch_engine_c16bf(int n, const EngArgs &a, int grid, cudaStream_t st);

}  // namespace wsfft
