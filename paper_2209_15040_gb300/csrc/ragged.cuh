// Ragged batch: many independent 3D transforms of uneven shapes in one
// persistent launch.
//
// The paper maps one problem onto an n x n processor mesh and notes that
// several small problems could share the machine (Section 5.3 discussion of
// many 32^3 transforms; Section 4.4 for several pencils per processor).  Here
// every instance contributes three supersteps' worth of tiles to one queue:
//   z tiles (contiguous axis, P whole pencils), signal the instance's z counter
//   y tiles (middle axis, W adjacent pencils), wait for all z tiles, signal y
//   x tiles (outer axis, W adjacent pencils), wait for all y tiles.
// The queue interleaves instances (z of instance s, y of s-L, x of s-2L for
// a lag L the plan chooses, 1 by default), so an instance is usually still in
// L2 when its next superstep reads it, and a tile only ever waits for tiles
// with smaller tickets (deadlock-free with any number of resident blocks).
// Axis lengths 32..256 and their tile shape (one of two per length, chosen
// by the plan) are dispatched at run time inside the kernel; every tile kind
// uses the same 256 threads.
#pragma once

#include "engine.cuh"
#include "pass_kernels.cuh"

namespace wsfft {

struct RagInst {
    const void *in;
    void *out;
    int n[3];          // axis lengths, n[2] contiguous
    int log_n2, log_n12;
    int tiles[3];      // tiles of the z, y, x supersteps
    float scale[3];    // store scale of the z, y, x supersteps
    int pad;
};

struct RagItem {
    int flags;     // ITEM_* of engine.cuh; bits 8..9: superstep (0 z, 1 y, 2 x)
    int inst;
    int tile;
    int pad;
};

struct RagArgs {
    const RagItem *items;
    int nitems;
    const RagInst *inst;
    uint32_t *ctr;         // [0] tickets, [1 + 2*i] z done of instance i, [2 + 2*i] y done
    int *status;
    const float2 *tw[4][2];  // stage tables [log2(N) - 5][shape] for N = 32..256
    int esel;              // bit log2(N) - 5 set: axes of length N use their second shape
    float ci;              // +1, or -1: conjugate on the z load (inverse)
    float co;              // +1, or -1: conjugate on the x store (inverse)
    uint64_t timeout_ns;
};

constexpr int RAG_THREADS = 256;

// Two tile shapes per axis length N (values per thread E; a tile is 256
// threads, T = N/E per pencil, 256/T pencils): shape 0 is the default, shape
// 1 the alternative the autotuner may pick per length.
__host__ __device__ constexpr int rag_E(int N, int alt = 0) {
    return alt ? (N <= 64 ? 16 : 8) : (N <= 64 ? 8 : 16);
}
__host__ __device__ constexpr int rag_T(int N, int alt = 0) { return N / rag_E(N, alt); }
__host__ __device__ constexpr int rag_P(int N, int alt = 0) { return RAG_THREADS / rag_T(N, alt); }  // z pencils per tile
__host__ __device__ constexpr int rag_W(int N, int alt = 0) { return RAG_THREADS / rag_T(N, alt); }  // y/x pencils per tile
constexpr int RAG_SMEM = 5120;  // float2: the largest exchange buffer of any shape below
__host__ __device__ constexpr int rag_smem_elems() { return RAG_SMEM; }
__host__ __device__ constexpr bool rag_fits(int N, int alt) {
    return rag_P(N, alt) * contig_PS(N) <= RAG_SMEM && N * rag_W(N, alt) * 17 / 16 <= RAG_SMEM;
}
static_assert(rag_fits(32, 0) && rag_fits(64, 0) && rag_fits(128, 0) && rag_fits(256, 0) && rag_fits(32, 1) &&
                  rag_fits(64, 1) && rag_fits(128, 1) && rag_fits(256, 1),
              "exchange buffers fit");

template <int N, int ALT, class S>
__device__ __forceinline__ void rag_contig(const RagInst &I, int tile, const float2 *tw, float ci,
                                           float sc, float2 *smem) {
    constexpr int T = rag_T(N, ALT), P = rag_P(N, ALT);
    const int t = threadIdx.x % T, p = threadIdx.x / T;
    const int64_t npen = (int64_t)I.n[0] * I.n[1];
    const int64_t q = (int64_t)tile * P + p;
    ContigAcc<S, OP_DEF, OP_DEF, false, (T <= 32)> acc{reinterpret_cast<const S *>(I.in) + q * N,
                                     reinterpret_cast<S *>(I.out) + q * N, smem + p * contig_PS(N), ci,
                                     {sc, sc}, q < npen};
    pencil_fft<N, rag_E(N, ALT)>(acc, t, tw);
}

// strided superstep along axis d (1: y, inner n2; 2: x, inner n1*n2), read
// and written in `out` (L2-coherent loads: other blocks wrote it this launch)
template <int N, int ALT, class S>
__device__ __forceinline__ void rag_strided(const RagInst &I, int d, int tile, const float2 *tw,
                                            float sx, float sy, float2 *smem) {
    constexpr int T = rag_T(N, ALT), W = rag_W(N, ALT);
    const int w = threadIdx.x % W, t = threadIdx.x / W;
    const int log_inner = d == 1 ? I.log_n2 : I.log_n12;
    const int64_t inner = (int64_t)1 << log_inner;
    const int64_t npen = d == 1 ? (int64_t)I.n[0] * I.n[2] : (int64_t)I.n[1] * I.n[2];
    const int64_t q = (int64_t)tile * W + w;
    const int64_t o = q >> log_inner, i = q & (inner - 1);
    const int64_t base = o * ((int64_t)N << log_inner) + i;
    StridedAcc<S, false, OP_CG, OP_DEF, W> acc;
    acc.in = reinterpret_cast<const S *>(I.out) + base;
    acc.out = reinterpret_cast<S *>(I.out) + base;
    acc.sm = smem;
    acc.stride = inner;
    acc.w = w;
    acc.ci = 1.f;
    acc.epi = Epi{sx, sy};
    acc.active = q < npen;
    acc.twq = 0;
    acc.tw_hi = nullptr;
    acc.tw_lo = nullptr;
    acc.tw_shift = 0;
    acc.tw_mask = 0;
    (void)T;
    pencil_fft<N, rag_E(N, ALT)>(acc, t, tw);
}

template <int N, class S>
__device__ __forceinline__ void rag_tile_n(const RagArgs &a, const RagInst &I, int d, int tile, float2 *smem,
                                           const float2 *tw0, const float2 *tw1, int alt) {
    if (d == 0) {
        if (alt) rag_contig<N, 1, S>(I, tile, tw1, a.ci, I.scale[0], smem);
        else rag_contig<N, 0, S>(I, tile, tw0, a.ci, I.scale[0], smem);
    } else {
        const float sx = I.scale[d], sy = d == 2 ? a.co * I.scale[d] : I.scale[d];
        if (alt) rag_strided<N, 1, S>(I, d, tile, tw1, sx, sy, smem);
        else rag_strided<N, 0, S>(I, d, tile, tw0, sx, sy, smem);
    }
}

template <class S>
__device__ __forceinline__ void rag_tile(const RagArgs &a, const RagInst &I, int d, int tile,
                                         float2 *smem) {
    const int N = I.n[2 - d];
    // stage tables with constant indices (a run-time index into the
    // parameter array would copy it to local memory)
    switch (N) {
        case 32: rag_tile_n<32, S>(a, I, d, tile, smem, a.tw[0][0], a.tw[0][1], a.esel & 1); break;
        case 64: rag_tile_n<64, S>(a, I, d, tile, smem, a.tw[1][0], a.tw[1][1], a.esel & 2); break;
        case 128: rag_tile_n<128, S>(a, I, d, tile, smem, a.tw[2][0], a.tw[2][1], a.esel & 4); break;
        default: rag_tile_n<256, S>(a, I, d, tile, smem, a.tw[3][0], a.tw[3][1], a.esel & 8); break;
    }
}

template <class S>
__global__ void __launch_bounds__(RAG_THREADS, 4) ragged_kernel(RagArgs a) {
    __shared__ float2 smem[rag_smem_elems()];
    __shared__ int4 s_item;
    __shared__ RagInst s_inst;
    const int tid = threadIdx.x;
    // Thread 0 keeps the queue one tile ahead: the next ticket and its item
    // are fetched while the current tile is processed.
    // Tickets are still processed in increasing order per block, so the
    // smallest unfinished ticket is always some block's current tile and the
    // waits stay deadlock-free.
    int4 next = make_int4(ITEM_END, 0, 0, 0);
    int after = 0;
    auto fetch = [&](int ticket) {
        next = make_int4(ITEM_END, 0, 0, 0);
        if (ticket < a.nitems) {
            const RagItem e = a.items[ticket];
            next = make_int4(e.flags, e.inst, e.tile, 0);
            after = (int)atomicAdd(&a.ctr[0], 1u);
        }
    };
    if (tid == 0) fetch((int)atomicAdd(&a.ctr[0], 1u));
    for (;;) {
        if (tid == 0) {
            int4 it = next;
            fetch(after);
            if (it.x & ITEM_WAIT) {
                const int d = (it.x >> 8) & 3;  // wait for superstep d-1 of this instance
                const uint32_t *dep = a.ctr + 1 + 2 * it.y + (d - 1);
                const uint32_t target = (uint32_t)a.inst[it.y].tiles[d - 1];
                if (ld_acquire_u32(dep) < target) {
                    const uint64_t dl = gtimer() + a.timeout_ns;
                    while (ld_acquire_u32(dep) < target) {
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
            if (!(it.x & (ITEM_END | ITEM_SKIP))) s_inst = a.inst[it.y];
        }
        __syncthreads();
        const int4 it = s_item;
        if (it.x & ITEM_END) break;
        // the instance record is read in place (shared memory, indexed by the
        // superstep at run time; thread 0 rewrites it only after the barrier below)
        if (!(it.x & ITEM_SKIP)) rag_tile<S>(a, s_inst, (it.x >> 8) & 3, it.z, smem);
        __syncthreads();
        if ((it.x & ITEM_SIGNAL) && !(it.x & ITEM_SKIP) && tid == 0) {
            __threadfence();
            red_release_add_u32(a.ctr + 1 + 2 * it.y + ((it.x >> 8) & 3), 1u);
        }
    }
}

}  // namespace wsfft
