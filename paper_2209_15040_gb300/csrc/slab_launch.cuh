// Launcher of the cluster-fused pass A for one storage type.  Included once
// per storage type by slab_c32.cu, slab_c16f.cu, slab_c16bf.cu (with
// WSFFT_STORE and WSFFT_SLAB_NAME defined).
#pragma once

#include <map>
#include <mutex>
#include <utility>

#include "slab_cluster.cuh"
#include "slab_desc.h"

namespace wsfft {
namespace {

// Clusters of more than 8 blocks need an opt-in per kernel; like the
// shared-memory size it is set once per (kernel, device).
inline cudaError_t set_cluster_attrs(const void *kernel, int smem, int cluster) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, bool> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_pair(kernel, dev);
    if (done.count(key)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess && cluster > 8) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) done[key] = true;
    return e;
}

template <int N, class S>
cudaError_t launch_slab_n(const void *in, void *out, int64_t nslabs, const SlabArgs &a, bool pdl, cudaStream_t st,
                          int *max_clusters) {
    constexpr int C = N == 512 ? 16 : 8;
    using Sh = SlabShape<N, C, S>;
    static_assert(Sh::EZ == slab_ez(Sh::kSplitZ) && Sh::EY == slab_ey(), "twiddle tables the plan builds");
    const bool plain = a.ci == 1.f && a.zsx == 1.f && a.zsy == 1.f;
    auto kern = plain ? slab_kernel<N, C, S, true> : slab_kernel<N, C, S, false>;
    cudaError_t e = set_cluster_attrs(reinterpret_cast<const void *>(slab_kernel<N, C, S, true>), Sh::SMEM, C);
    if (e == cudaSuccess)
        e = set_cluster_attrs(reinterpret_cast<const void *>(slab_kernel<N, C, S, false>), Sh::SMEM, C);
    if (e != cudaSuccess) return e;
    if (!max_clusters && nslabs <= 0) return cudaSuccess;
    if (nslabs * C > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((nslabs > 0 ? nslabs : 1) * C));
    cfg.blockDim = dim3(Sh::THREADS);
    cfg.dynamicSmemBytes = (size_t)Sh::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 2 : 1;
    if (max_clusters) {
        *max_clusters = 0;
        cfg.numAttrs = 1;
        return cudaOccupancyMaxActiveClusters(max_clusters, reinterpret_cast<const void *>(kern), &cfg);
    }
    return cudaLaunchKernelEx(&cfg, kern, (const S *)in, (S *)out, a);
}

}  // namespace

cudaError_t WSFFT_SLAB_NAME(int n, const void *in, void *out, int64_t nslabs, const SlabArgs &a, bool pdl,
                            cudaStream_t st, int *max_clusters) {
    using S = WSFFT_STORE;
    switch (n) {
        case 256: return launch_slab_n<256, S>(in, out, nslabs, a, pdl, st, max_clusters);
        case 512: return launch_slab_n<512, S>(in, out, nslabs, a, pdl, st, max_clusters);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace wsfft
