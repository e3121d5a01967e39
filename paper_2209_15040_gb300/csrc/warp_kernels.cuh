// Warp-per-pencil superstep kernels.
//
// With E = 16 values per thread, a pencil of N <= 512 elements fits in one
// warp (N/16 <= 32 lanes; for N < 512 a warp holds 512/N pencils).  Every
// exchange between radix stages then stays inside the warp: each warp owns a
// private, padded row of shared memory per pencil and synchronises with
// __syncwarp() only.  Thread blocks synchronise only where the whole tile
// has to be coherent:
//  * contiguous tiles (the superstep along the contiguous axis): none -- a
//    warp loads its pencils straight from global memory (consecutive lanes,
//    consecutive elements) and stores them straight back;
//  * strided tiles: the block stages N rows of W adjacent pencils (128-byte
//    rows at W = 16) into pencil-major shared memory, synchronises, lets each
//    warp transform its pencils, synchronises, and writes the rows back.
// This replaces the barrier per exchange of the one-tile-per-block kernels,
// which left the SM idle at each of 4-6 barriers per tile.
//
// Shared-memory index of element k of a pencil: k + k/16 in a row of
// N + N/16 + 1 elements.  Consecutive lanes reading k = t + 32r, and the
// Stockham writes k = 16t + r and (t/16)*256 + t%16 + 16r, each touch every
// bank pair exactly twice per warp; the row length (1 mod 16) keeps the
// row-wise staging stores conflict-free as well.
#pragma once

#include "engine.cuh"
#include "fft_core.cuh"

#ifndef WSFFT_WP_BATCH
#define WSFFT_WP_BATCH 16
#endif
#ifndef WSFFT_WP_MINB
#define WSFFT_WP_MINB 2
#endif

namespace wsfft {

__host__ __device__ constexpr int wp_row(int N) { return N + N / 16 + 1; }

// Accessor over one warp-private pencil row.  Z mode: first stage loads and
// last stage stores go to global memory.  Staged mode: both go to the row.
template <class S, int LOP, int SOP, bool STAGED>
struct WarpAcc {
    const S *gin;   // Z: pencil in global memory
    S *gout;
    float2 *row;    // pencil's shared-memory row
    float ci, sx, sy;
    __device__ __forceinline__ static int sidx(int k) { return k + (k >> 4); }
    __device__ __forceinline__ float2 gload(int k) const {
        float2 v;
        if constexpr (STAGED) v = row[sidx(k)];
        else v = Cvt<S>::template load<LOP>(gin + k);
        v.y *= ci;
        return v;
    }
    __device__ __forceinline__ void after_load() const {
        if constexpr (STAGED) __syncwarp();  // the row is rewritten by the first exchange
    }
    __device__ __forceinline__ void gstore(int k, float2 v) const {
        v = make_float2(v.x * sx, v.y * sy);
        if constexpr (STAGED) row[sidx(k)] = v;
        else Cvt<S>::template store<SOP>(gout + k, v);
    }
    __device__ __forceinline__ void sstore(int k, float2 v) const { row[sidx(k)] = v; }
    __device__ __forceinline__ float2 sload(int k) const { return row[sidx(k)]; }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
};

template <int N, class S>
struct WCfg {
    static_assert(N >= 32 && N <= 512, "one warp per pencil or less");
    static constexpr int E = 16;
    static constexpr int T = N / E;          // lanes per pencil
    static constexpr int G = 32 / T;         // pencils per warp
    static constexpr int WARPS = 8;
    static constexpr int THREADS = 32 * WARPS;
    static constexpr int PZ = WARPS * G;     // pencils per contiguous tile
    static constexpr int W = PZ < 16 ? 16 : PZ;  // pencils per strided tile
    static constexpr int ROUNDS = W / PZ;    // strided pencils per lane group
    static constexpr int ROW = wp_row(N);
    static constexpr int SMEM = W * ROW * 8;
};

// Contiguous tile: pencils q0 .. q0 + PZ - 1 (consecutive rows of N).
template <int N, class S, int LOP, int SOP>
__device__ __forceinline__ void wp_contig_tile(const S *in, S *out, int64_t q0, float2 *smem,
                                               const float2 *tw, float ci, float sx, float sy) {
    using C = WCfg<N, S>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / C::T, t = lane % C::T;
    const int p = warp * C::G + g;
    const int64_t off = (q0 + p) * N;
    WarpAcc<S, LOP, SOP, false> acc{in + off, out + off, smem + p * C::ROW, ci, sx, sy};
    pencil_fft<N, C::E>(acc, t, tw);
}

// Strided tile: W adjacent pencils starting at `base` (element offset of
// pencil 0, element 0), rows `stride` elements apart.  Must be called by the
// whole block.
template <int N, class S, int LOP, int SOP>
__device__ __forceinline__ void wp_strided_tile(const S *in, S *out, int64_t base, int64_t stride,
                                                float2 *smem, const float2 *tw, float ci, float sx,
                                                float sy) {
    using C = WCfg<N, S>;
    constexpr int W = C::W;
    constexpr int RPR = C::THREADS / W;  // rows per round of the staging loop
    constexpr int BATCH = WSFFT_WP_BATCH;  // loads in flight per thread
    const int tid = threadIdx.x;
    const int w = tid % W, r0 = tid / W;
    // stage: rows k (W consecutive elements each) -> pencil-major rows
#pragma unroll 1
    for (int k0 = 0; k0 < N; k0 += RPR * BATCH) {
        float2 v[BATCH];
#pragma unroll
        for (int j = 0; j < BATCH; ++j) {
            const int k = k0 + r0 + j * RPR;
            v[j] = k < N ? Cvt<S>::template load<LOP>(in + base + (int64_t)k * stride + w)
                         : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < BATCH; ++j) {
            const int k = k0 + r0 + j * RPR;
            if (k < N) smem[w * C::ROW + k + (k >> 4)] = v[j];
        }
    }
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5;
    const int g = lane / C::T, t = lane % C::T;
#pragma unroll 1
    for (int rd = 0; rd < C::ROUNDS; ++rd) {
        const int p = (rd * C::WARPS + warp) * C::G + g;
        WarpAcc<S, LOP, SOP, true> acc{nullptr, nullptr, smem + p * C::ROW, ci, sx, sy};
        pencil_fft<N, C::E>(acc, t, tw);
    }
    __syncthreads();
    // unstage: pencil-major rows -> rows of W consecutive elements
#pragma unroll 4
    for (int k = r0; k < N; k += RPR)
        Cvt<S>::template store<SOP>(out + base + (int64_t)k * stride + w, smem[w * C::ROW + k + (k >> 4)]);
}

// One strided tile per block (the superstep along the outer axis): the
// array viewed as [outer][N][inner], tiles of W consecutive inner indices.
template <int N, class S>
__global__ void __launch_bounds__(WCfg<N, S>::THREADS, WSFFT_WP_MINB)
    wp_strided_kernel(const S *__restrict__ in, S *__restrict__ out, int64_t inner, int log_inner,
                      int64_t ntiles, const float2 *__restrict__ tw, float ci, float sx, float sy) {
    using C = WCfg<N, S>;
    extern __shared__ float2 wp_smem[];
    const int64_t tile = blockIdx.x;
    if (tile >= ntiles) return;
    const int64_t q0 = tile * C::W;  // first pencil (inner is a multiple of W)
    const int64_t o = q0 >> log_inner, i = q0 & (inner - 1);
    const int64_t base = o * ((int64_t)N << log_inner) + i;
    wp_strided_tile<N, S, OP_CS, OP_CS>(in, out, base, inner, wp_smem, tw, ci, sx, sy);
}

// Persistent pass A of an n^3 transform: the tile queue of engine.cuh with
// contiguous tiles (z) that signal their slab and strided tiles (y) that wait
// for it (bounded).  Thread 0 keeps the queue two tiles ahead.
template <int N, class S>
__global__ void __launch_bounds__(WCfg<N, S>::THREADS, WSFFT_WP_MINB) wp_persist_kernel(EngArgs a) {
    using C = WCfg<N, S>;
    extern __shared__ float2 wp_smem[];
    __shared__ int4 s_item;
    const int tid = threadIdx.x;
    int4 next = make_int4(ITEM_END, 0, 0, 0);
    int after = 0;
    if (tid == 0) {
        const int t0 = (int)atomicAdd(&a.ctr[0], 1u);
        if (t0 < a.nitems) {
            const EngItem e = a.items[t0];
            next = make_int4(e.flags, e.unit, e.tile, 0);
        }
        after = (int)atomicAdd(&a.ctr[0], 1u);
    }
    for (;;) {
        if (tid == 0) {
            int4 it = next;
            next = make_int4(ITEM_END, 0, 0, 0);
            if (after < a.nitems) {
                const EngItem e = a.items[after];
                next = make_int4(e.flags, e.unit, e.tile, 0);
                after = (int)atomicAdd(&a.ctr[0], 1u);
            }
            if (it.x & ITEM_WAIT) {
                const uint32_t *dep = a.ctr + 1 + it.y;
                if (ld_acquire_u32(dep) < a.dep_target) {
                    const uint64_t dl = gtimer() + a.timeout_ns;
                    while (ld_acquire_u32(dep) < a.dep_target) {
                        if (gtimer() > dl) {
                            atomicExch(a.status, 1);
                            it.x = ITEM_SKIP;
                            break;
                        }
                        __nanosleep(100);
                    }
                }
                __threadfence();
            }
            s_item = it;
        }
        __syncthreads();
        const int4 it = s_item;
        if (it.x & ITEM_END) break;
        if (!(it.x & ITEM_SKIP)) {
            if (it.x & ITEM_STRIDED) {
                const int64_t base = (int64_t)it.y * a.unit_elems + (int64_t)it.z * C::W;
                wp_strided_tile<N, S, OP_CG, OP_CS>(reinterpret_cast<const S *>(a.s_src),
                                                    reinterpret_cast<S *>(a.s_dst), base, a.s_stride,
                                                    wp_smem, a.tw_s, a.s_ci, a.s_sx, a.s_sy);
            } else {
                const int64_t q0 = (int64_t)it.y * (a.unit_elems / N) + (int64_t)it.z * C::PZ;
                wp_contig_tile<N, S, OP_CS, OP_DEF>(reinterpret_cast<const S *>(a.c_src),
                                                    reinterpret_cast<S *>(a.c_dst), q0, wp_smem, a.tw_c,
                                                    a.c_ci, a.c_sx, a.c_sy);
            }
        }
        __syncthreads();  // tile done: shared rows and s_item free
        if ((it.x & ITEM_SIGNAL) && !(it.x & ITEM_SKIP) && tid == 0) {
            __threadfence();
            red_release_add_u32(a.ctr + 1 + it.y, 1u);
        }
    }
}

}  // namespace wsfft
