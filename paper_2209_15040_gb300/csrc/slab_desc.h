// Launcher entry points of the cluster-fused pass A (slab_cluster.cuh), one
// per storage type.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace wsfft {

struct SlabArgs;

// Slab edges the fused pass A is built for, and its cluster size per edge.
inline bool slab_supports(int n) { return n == 256 || n == 512; }
inline int slab_cluster(int n) { return n == 512 ? 16 : 8; }
// values per thread of the z tiles (complex64 / 16-bit storage) and of the
// y tiles: the stage-twiddle tables the plan passes in SlabArgs
constexpr int slab_ez(bool half_storage) { return half_storage ? 8 : 16; }
constexpr int slab_ey() { return 16; }

// Launch the z and y supersteps of `nslabs` n x n slabs (slab u at element
// u*n*n of in and out; in == out allowed).  With max_clusters != nullptr
// nothing is launched: *max_clusters receives how many clusters of this
// kernel can be resident at once on the current device (0: cannot run).
// Returns cudaErrorInvalidValue for an edge that is not built.
cudaError_t launch_slab_c32(int n, const void *in, void *out, int64_t nslabs, const SlabArgs &a, bool pdl,
                            cudaStream_t st, int *max_clusters);
cudaError_t launch_slab_c16f(int n, const void *in, void *out, int64_t nslabs, const SlabArgs &a, bool pdl,
                             cudaStream_t st, int *max_clusters);
cudaError_t launch_slab_c16bf(int n, const void *in, void *out, int64_t nslabs, const SlabArgs &a, bool pdl,
                              cudaStream_t st, int *max_clusters);

}  // namespace wsfft
