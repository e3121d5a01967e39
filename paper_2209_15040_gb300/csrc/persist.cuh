// Persistent superstep kernel with per-slab dependencies.
//
// The same tile queue as the pipelined engine (engine.cuh: EngItem, EngArgs),
// executed by several thread blocks per SM that each take one ticket at a
// time and load their tile straight into registers, as the one-tile-per-block
// kernels do.  Latency is hidden by the other resident blocks rather than by
// an in-block copy pipeline.
//
// Pass A of an n^3 transform puts, for every slab (fixed first index), the
// contiguous-axis tiles (z) in the queue a few slabs ahead of the same slab's
// strided tiles (y).  A y tile waits, with a bounded spin, until all z tiles
// of its slab have signalled; by then the slab (2 MiB at 512^3) is still in
// L2, so the array is read from and written to HBM once for both supersteps.
// Ticket order makes the waits deadlock-free: a tile only ever waits for
// tiles with smaller tickets, which running blocks already hold.
#pragma once

#include "engine.cuh"

namespace wsfft {

// PAIRS: strided tiles carry pencil pairs (StridedPairAcc, W/2 pairs)
template <int NC, int EC, int P, int NS, int ES, int W, class S, bool PAIRS = false>
struct PCfg {
    static constexpr int THREADS = P * (NC / EC);
    static_assert(THREADS == (PAIRS ? W / 2 : W) * (NS / ES), "both tile kinds need the same thread count");
    static constexpr int XC = P * contig_PS(NC);
    static constexpr int XS = PAIRS ? NS * W : NS * W + (NS * W) / 16;
    static constexpr int SMEM = (XC > XS ? XC : XS) * 8;
    static constexpr int TILE_C = P * NC;
};

// MODE 0 (pass A): contiguous and strided tiles; strided loads bypass L1
// (.cg: the data was written by other blocks in this launch) and their stores
// stream (.cs).  MODE 1 (pass B): strided tiles only, loads and stores stream.
// SUB: tiles per queue item (an item covers tiles tile*SUB .. tile*SUB+SUB-1),
// which spreads the per-item ticket, dependency and barrier cost.
template <int NC, int EC, int P, int NS, int ES, int W, class S, int MODE, bool PAIRS = false, int SUB = 1>
__global__ void __launch_bounds__(PCfg<NC, EC, P, NS, ES, W, S, PAIRS>::THREADS, 2)
    persist_kernel(EngArgs a) {
    using C = PCfg<NC, EC, P, NS, ES, W, S, PAIRS>;
    extern __shared__ float2 p_smem[];
    __shared__ int4 s_item;
    const int tid = threadIdx.x;
    // Thread 0 keeps the queue two tiles ahead: the ticket after next is
    // taken and the next item read while the current tile is processed, so
    // neither global round trip sits between two tiles.  Tickets are still
    // processed in increasing order per block, which keeps the waits
    // deadlock-free (the smallest unfinished ticket is always a block's
    // current tile, whose inputs are complete).
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
            // fetch the following item now; it is only used next iteration
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
                            // record the failure and drop this tile, but keep
                            // working through the queue so no held ticket is
                            // abandoned (waits never chain)
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
        const int4 it0 = s_item;
        if (it0.x & ITEM_END) break;
        if (it0.x & ITEM_SKIP) {
            __syncthreads();  // everyone has read s_item before thread 0 rewrites it
            continue;
        }
#pragma unroll 1
        for (int sub = 0; sub < SUB; ++sub) {
        if (sub > 0) __syncthreads();  // the exchange buffer is reused by the next tile
        int4 it = it0;
        it.z = it0.z * SUB + sub;
        if (it.x & ITEM_STRIDED) {
          if constexpr (PAIRS) {
            constexpr int WP = W / 2;
            using PT = typename Pair<S>::T;
            const int wp = tid % WP, t = tid / WP;
            const int64_t base = (int64_t)it.y * a.unit_elems + (int64_t)it.z * W + 2 * wp;
            StridedPairAcc<S, W, false, MODE == 0 ? OP_CG : OP_CS, OP_CS> acc;
            acc.in = reinterpret_cast<const PT *>(reinterpret_cast<const S *>(a.s_src) + base);
            acc.out = reinterpret_cast<PT *>(reinterpret_cast<S *>(a.s_dst) + base);
            acc.sm = reinterpret_cast<float4 *>(p_smem);
            acc.stride = a.s_stride / 2;
            acc.wp = wp;
            acc.ci = a.s_ci;
            acc.sx = a.s_sx;
            acc.sy = a.s_sy;
            acc.active = true;
            pencil_fft<NS, ES>(acc, t, a.tw_s);
          } else {
            const int w = tid % W, t = tid / W;
            const int64_t base = (int64_t)it.y * a.unit_elems + (int64_t)it.z * W + w;
            const Epi epi{a.s_sx, a.s_sy};
            if constexpr (MODE == 0) {
                StridedAcc<S, false, OP_CG, OP_CS, W> acc;
                acc.in = reinterpret_cast<const S *>(a.s_src) + base;
                acc.out = reinterpret_cast<S *>(a.s_dst) + base;
                acc.sm = p_smem;
                acc.stride = a.s_stride;
                acc.w = w;
                acc.ci = a.s_ci;
                acc.epi = epi;
                acc.active = true;
                pencil_fft<NS, ES>(acc, t, a.tw_s);
            } else {
                StridedAcc<S, false, OP_CS, OP_CS, W> acc;
                acc.in = reinterpret_cast<const S *>(a.s_src) + base;
                acc.out = reinterpret_cast<S *>(a.s_dst) + base;
                acc.sm = p_smem;
                acc.stride = a.s_stride;
                acc.w = w;
                acc.ci = a.s_ci;
                acc.epi = epi;
                acc.active = true;
                pencil_fft<NS, ES>(acc, t, a.tw_s);
            }
          }
        } else if constexpr (MODE == 0) {
            constexpr int T = NC / EC;
            const int t = tid % T, p = tid / T;
            const int64_t off = (int64_t)it.y * a.unit_elems + (int64_t)it.z * C::TILE_C + (int64_t)p * NC;
            ContigAcc<S, OP_CS, OP_DEF, false, (T <= 32)> acc{reinterpret_cast<const S *>(a.c_src) + off,
                                            reinterpret_cast<S *>(a.c_dst) + off,
                                            p_smem + p * contig_PS(NC),
                                            a.c_ci,
                                            {a.c_sx, a.c_sy},
                                            true};
            pencil_fft<NC, EC>(acc, t, a.tw_c);
        }
        }  // sub-tiles
        __syncthreads();  // item done: exchange buffer and s_item free
        if ((it0.x & ITEM_SIGNAL) && tid == 0) {
            __threadfence();
            red_release_add_u32(a.ctr + 1 + it0.y, 1u);
        }
    }
}

}  // namespace wsfft
