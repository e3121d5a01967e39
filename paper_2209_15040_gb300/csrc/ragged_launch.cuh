// Launch of the ragged-batch kernel for one storage type (included by
// ragged_c32.cu, ragged_c16f.cu, ragged_c16bf.cu).
#pragma once

#include "ragged.cuh"
#include "ragged_desc.h"

namespace wsfft {

cudaError_t WSFFT_RAGGED_NAME(const RagArgs &a, int *grid_per_sm, int grid, cudaStream_t st) {
    using S = WSFFT_STORE;
    auto kern = ragged_kernel<S>;
    if (grid_per_sm) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(grid_per_sm, kern, RAG_THREADS, 0);
    if (grid <= 0) return cudaSuccess;
    kern<<<grid, RAG_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace wsfft
