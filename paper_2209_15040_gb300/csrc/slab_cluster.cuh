// Fused pass A of a rank-3 transform whose two inner axes are equal (n x n
// slabs): the z and y supersteps of one slab in one thread-block cluster,
// so the array makes two trips through HBM (this pass, then the x
// superstep) instead of three.
//
// The paper runs the three supersteps with a redistribution between them
// (Section 4.2, 4.3).  Here the redistribution between z and y stays inside
// one slab, and that slab is handed from the z superstep to the y superstep
// through L2 within one cluster of C thread blocks:
//
//   block r of the cluster (slab u = cluster index):
//     z: rows [r*n/C, (r+1)*n/C) of the slab, whole contiguous pencils,
//        read from `in`, written to `out`;
//     cluster barrier (release / acquire at cluster scope: every z row of
//        the slab is written and visible to every block of the cluster);
//     y: columns [r*n/C, (r+1)*n/C) of the slab, split-form pencil pairs
//        read back from L2 (ld.global.cg) and written to `out` in place.
//
// The slab (2 MiB in complex64 at n = 512) is written once by the z tiles and
// read back before it leaves L2: only the clusters in flight hold a slab, so
// the L2 working set is (resident clusters) x (slab bytes).  Measured on this
// GPU with the same access pattern and no arithmetic: clusters of 16 blocks
// keep about 21 slabs in flight and move a pass A in 0.44 ms, clusters of 8
// or 4 blocks hold more slabs than L2 keeps and take 0.57 / 0.62 ms (two
// separate passes: 0.64 ms).  No block waits on another block's flag: the
// only synchronisation is the hardware cluster barrier, which every block of
// the cluster reaches after the same fixed number of tiles.
#pragma once

#include <type_traits>

#include "pass_kernels.cuh"

namespace wsfft {

struct SlabArgs {
    float ci;               // z: +1, or -1 to conjugate on load
    float zsx, zsy;         // z: store scale of re and im
    float ysx, ysy;         // y: store scale of re and im
    const float2 *tw_z;     // stage twiddles of the z pencils (N, SlabShape::EZ)
    const float2 *tw_y;     // stage twiddles of the y pencils (N, SlabShape::EY)
};

__device__ __forceinline__ unsigned cluster_rank_x() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_index_x() {
    unsigned r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
// Asynchronous bulk prefetch of `bytes` (a multiple of 16) at `p` into L2.
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// every thread of every block of the cluster: writes before the barrier
// (global and shared) are visible to reads after it
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Tile shapes: 256 threads, at most 85 registers each (three blocks per
// SM), 16 values per thread in both supersteps -- the fastest of the shapes
// measured at 512^3 complex64 (256 or 512 threads, 8 or 16 values per
// thread in y, two to four blocks per SM, clusters of 8 or 16):
//   z: complex64 one pencil per warp (warp-only exchanges), 16-bit storage
//      split-form pencil pairs with EZ = 8 (a pair per 64 threads);
//   y: split-form pencil pairs, YW adjacent pencils per tile.
template <int N, int C, class S>
struct SlabShape {
    static constexpr bool kSplitZ = !std::is_same<S, float2>::value;
    static constexpr int THREADS = 256;
    static constexpr int EZ = kSplitZ ? 8 : 16;
    static constexpr int TZ = N / EZ;                                          // threads per z pencil (pair)
    static constexpr int ZP = kSplitZ ? 2 * (THREADS / TZ) : THREADS / TZ;    // rows per z tile
    static constexpr int EY = 16;
    static constexpr int TY = N / EY;                                          // threads per y pencil pair
    static constexpr int YW = 2 * (THREADS / TY);                              // columns per y tile
    static constexpr int ROWS = N / C;                                         // rows and columns per block
    static constexpr int ZTILES = ROWS / ZP;
    static constexpr int YTILES = ROWS / YW;
    static constexpr int SMEM_Z = kSplitZ ? (ZP / 2) * contig_PS(N) * 16 : ZP * contig_PS(N) * 8;
    static constexpr int SMEM_Y = N * (YW / 2) * 16;
    static constexpr int SMEM = SMEM_Z > SMEM_Y ? SMEM_Z : SMEM_Y;
    static constexpr bool ZWARP = TZ <= 32;  // a z pencil (pair) within one warp: warp-only exchanges
    static_assert(ROWS % ZP == 0 && ROWS % YW == 0 && ZTILES >= 1 && YTILES >= 1, "tiles per block");
};

// One z tile: ZP whole rows of the slab from `row0`.  Out of line for the
// same reason as the y tile.
template <int N, int C, class S, bool PLAINZ>
__device__ __noinline__ void slab_z_tile(const S *__restrict__ slab_in, S *__restrict__ slab_out, int row0,
                                         const SlabArgs &a, float4 *sm) {
    using Sh = SlabShape<N, C, S>;
    constexpr int T = Sh::TZ;
    const int t = threadIdx.x % T, p = threadIdx.x / T;
    if constexpr (Sh::kSplitZ) {
        const int64_t q = (int64_t)(row0 + 2 * p) * N;
        ContigSplitAcc<S, PLAINZ, Sh::ZWARP> acc{slab_in + q, slab_out + q, sm + p * contig_PS(N), N,
                                                 a.ci, a.zsx, a.zsy, true, true};
        pencil_fft<N, Sh::EZ>(acc, t, a.tw_z);
    } else {
        const int64_t q = (int64_t)(row0 + p) * N;
        ContigAcc<S, OP_DEF, OP_DEF, PLAINZ, Sh::ZWARP> acc{slab_in + q, slab_out + q,
                                                            reinterpret_cast<float2 *>(sm) + p * contig_PS(N),
                                                            a.ci, {a.zsx, a.zsy}, true};
        pencil_fft<N, Sh::EZ>(acc, t, a.tw_z);
    }
}

// One y tile: YW adjacent columns of the slab at `col0`, rows N elements
// apart.  Kept out of line: inlined into the tile loop, the compiler held
// values of the next iteration live and spilled (110 registers for one tile,
// spills at the 128-register bound for two).
template <int N, int C, class S>
__device__ __noinline__ void slab_y_tile(S *__restrict__ slab, int col0, const SlabArgs &a, float4 *sm) {
    using Sh = SlabShape<N, C, S>;
    using PT = typename SplitPair<S>::T;
    constexpr int WP = Sh::YW / 2;
    const int wp = threadIdx.x % WP, t = threadIdx.x / WP;
    StridedSplitAcc<S, Sh::YW, false, OP_CG, OP_CS> acc;
    acc.in = reinterpret_cast<const PT *>(slab + col0 + 2 * wp);
    acc.out = reinterpret_cast<PT *>(slab + col0 + 2 * wp);
    acc.sm = sm;
    acc.stride = N / 2;
    acc.wp = wp;
    acc.ci = 1.f;
    acc.sx = a.ysx;
    acc.sy = a.ysy;
    acc.active = true;
    pencil_fft<N, Sh::EY>(acc, t, a.tw_y);
}

template <int N, int C, class S, bool PLAINZ>
__global__ void __launch_bounds__(256, 3)
    slab_kernel(const S *__restrict__ in, S *__restrict__ out, SlabArgs a) {
    using Sh = SlabShape<N, C, S>;
    extern __shared__ float4 slab_smem[];
    pdl_enter();
    const int tid = threadIdx.x;
    const int r = (int)cluster_rank_x();
    const int64_t base = (int64_t)cluster_index_x() * N * N;  // first element of the slab

    // This block's z rows are one contiguous run of ROWS*N elements: ask for
    // all of it at once (one bulk prefetch per row, from the first warp), so
    // the rows stream into L2 while the tiles compute and the later tiles'
    // loads hit L2 (measured 3% faster than without).
    if (tid < Sh::ROWS)
        prefetch_l2_bulk(in + base + (int64_t)(r * Sh::ROWS + tid) * N, (unsigned)(N * sizeof(S)));

    // z superstep: ZTILES tiles of ZP whole rows
#pragma unroll 1
    for (int zt = 0; zt < Sh::ZTILES; ++zt)
        slab_z_tile<N, C, S, PLAINZ>(in + base, out + base, r * Sh::ROWS + zt * Sh::ZP, a, slab_smem);

    cluster_barrier();

    // y superstep: YTILES tiles of YW adjacent columns
#pragma unroll 1
    for (int yt = 0; yt < Sh::YTILES; ++yt)
        slab_y_tile<N, C, S>(out + base, r * Sh::ROWS + yt * Sh::YW, a, slab_smem);
}

}  // namespace wsfft
