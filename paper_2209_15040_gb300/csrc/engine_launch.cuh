// Instantiation and launch of the persistent engine for one storage type
// (included by engine_c32.cu, engine_c16f.cu, engine_c16bf.cu).
#pragma once

#include "engine.cuh"
#include "persist.cuh"
#include "warp_kernels.cuh"
#include "engine_desc.h"

namespace wsfft {
namespace {

template <int NC, int EC, int P, int NS, int ES, int W, class S>
cudaError_t launch_eng(const EngArgs &a, int grid, cudaStream_t st) {
    using C = EngCfg<NC, EC, P, NS, ES, W, S>;
    auto kern = engine_kernel<NC, EC, P, NS, ES, W, S>;
    const cudaError_t attr = set_smem_attr(reinterpret_cast<const void *>(kern), C::SMEM);
    if (attr != cudaSuccess) return attr;
    if (grid <= 0) return cudaSuccess;
    kern<<<grid, C::THREADS, C::SMEM, st>>>(a);
    return cudaGetLastError();
}

#ifndef WSFFT_PERSIST_SUB
#define WSFFT_PERSIST_SUB 2
#endif
template <int NC, int EC, int P, int NS, int ES, int W, class S, int MODE, bool PAIRS>
cudaError_t launch_per_mode(const EngArgs &a, int *grid_per_sm, int grid, cudaStream_t st) {
    using C = PCfg<NC, EC, P, NS, ES, W, S, PAIRS>;
    auto kern = persist_kernel<NC, EC, P, NS, ES, W, S, MODE, PAIRS, (NC == 512 ? WSFFT_PERSIST_SUB : 1)>;
    const cudaError_t attr = set_smem_attr(reinterpret_cast<const void *>(kern), C::SMEM);
    if (attr != cudaSuccess) return attr;
    if (grid_per_sm) {
        int nb = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, C::THREADS, C::SMEM);
        if (e != cudaSuccess) return e;
        *grid_per_sm = nb;
        return cudaSuccess;
    }
    if (grid <= 0) return cudaSuccess;
    kern<<<grid, C::THREADS, C::SMEM, st>>>(a);
    return cudaGetLastError();
}

template <int NC, int EC, int P, int NS, int ES, int W, class S, bool PAIRS = false>
cudaError_t launch_per(const EngArgs &a, int s_mode, int *grid_per_sm, int grid, cudaStream_t st) {
    if (s_mode == 0) return launch_per_mode<NC, EC, P, NS, ES, W, S, 0, PAIRS>(a, grid_per_sm, grid, st);
    return launch_per_mode<NC, EC, P, NS, ES, W, S, 1, PAIRS>(a, grid_per_sm, grid, st);
}

template <int N, class S>
cudaError_t launch_wpp(const EngArgs &a, int *grid_per_sm, int grid, cudaStream_t st) {
    using C = WCfg<N, S>;
    auto kern = wp_persist_kernel<N, S>;
    const cudaError_t attr = set_smem_attr(reinterpret_cast<const void *>(kern), C::SMEM);
    if (attr != cudaSuccess) return attr;
    if (grid_per_sm) {
        int nb = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, C::THREADS, C::SMEM);
        if (e != cudaSuccess) return e;
        *grid_per_sm = nb;
        return cudaSuccess;
    }
    if (grid <= 0) return cudaSuccess;
    kern<<<grid, C::THREADS, C::SMEM, st>>>(a);
    return cudaGetLastError();
}

template <int N, class S>
cudaError_t launch_wps(const WpStridedArgs &b, cudaStream_t st) {
    using C = WCfg<N, S>;
    auto kern = wp_strided_kernel<N, S>;
    const cudaError_t attr = set_smem_attr(reinterpret_cast<const void *>(kern), C::SMEM);
    if (attr != cudaSuccess) return attr;
    if (b.inner % C::W != 0) return cudaErrorInvalidValue;
    const int64_t ntiles = b.npencils / C::W;
    if (ntiles <= 0) return cudaSuccess;
    if (ntiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)ntiles, C::THREADS, C::SMEM, st>>>(
        (const S *)b.in, (S *)b.out, b.inner, b.log_inner, ntiles, b.tw, b.ci, b.sx, b.sy);
    return cudaGetLastError();
}

}  // namespace

// Warp-per-pencil kernels (warp_kernels.cuh).
cudaError_t WSFFT_WPP_NAME(int n, const EngArgs &a, int *grid_per_sm, int grid, cudaStream_t st) {
    using S = WSFFT_STORE;
    switch (n) {
        case 128: return launch_wpp<128, S>(a, grid_per_sm, grid, st);
        case 256: return launch_wpp<256, S>(a, grid_per_sm, grid, st);
        case 512: return launch_wpp<512, S>(a, grid_per_sm, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t WSFFT_WPS_NAME(int n, const WpStridedArgs &b, cudaStream_t st) {
    using S = WSFFT_STORE;
    switch (n) {
        case 128: return launch_wps<128, S>(b, st);
        case 256: return launch_wps<256, S>(b, st);
        case 512: return launch_wps<512, S>(b, st);
        default: return cudaErrorInvalidValue;
    }
}

// Persistent kernel: grid_per_sm != NULL only queries resident blocks per SM.
cudaError_t WSFFT_PERSIST_NAME(int n, const EngArgs &a, int s_mode, int *grid_per_sm, int grid,
                               cudaStream_t st) {
    using S = WSFFT_STORE;
    switch (n) {
        case 128: return launch_per<128, 16, 64, 128, 16, 64, S>(a, s_mode, grid_per_sm, grid, st);
        case 256: return launch_per<256, 16, 32, 256, 16, 32, S>(a, s_mode, grid_per_sm, grid, st);
#if WSFFT_PERSIST512_E32
        case 512: return launch_per<512, 16, 8, 512, 32, 16, S>(a, s_mode, grid_per_sm, grid, st);
#else
        case 512: return launch_per<512, 16, 16, 512, 8, 16, S, true>(a, s_mode, grid_per_sm, grid, st);
#endif
        case 1024: return launch_per<1024, 16, 8, 1024, 16, 8, S>(a, s_mode, grid_per_sm, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t WSFFT_ENGINE_NAME(int n, const EngArgs &a, int grid, cudaStream_t st) {
    using S = WSFFT_STORE;
    switch (n) {
        case 128: return launch_eng<128, 16, 64, 128, 16, 64, S>(a, grid, st);
        case 256: return launch_eng<256, 16, 32, 256, 16, 32, S>(a, grid, st);
        case 512: return launch_eng<512, 16, 16, 512, 16, 16, S>(a, grid, st);
        case 1024: return launch_eng<1024, 16, 8, 1024, 16, 8, S>(a, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace wsfft
