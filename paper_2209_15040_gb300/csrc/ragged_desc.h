// Host-visible interface of the ragged-batch kernel (ragged.cuh).
#pragma once

#include <cuda_runtime.h>

namespace wsfft {

struct RagArgs;

// grid_per_sm != NULL: only report how many blocks fit on one SM.
cudaError_t launch_ragged_c32(const RagArgs &a, int *grid_per_sm, int grid, cudaStream_t st);
cudaError_t launch_ragged_c16f(const RagArgs &a, int *grid_per_sm, int grid, cudaStream_t st);
cudaError_t launch_ragged_c16bf(const RagArgs &a, int *grid_per_sm, int grid, cudaStream_t st);

}  // namespace wsfft
