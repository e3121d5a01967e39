// Persistent superstep engine: one launch works through a queue of tiles.
//
// Each thread block is one producer warp plus CONS consumer threads.  The
// producer takes the next ticket from a global counter, waits (bounded) until
// the tile's inputs are complete, and streams the tile into a two-stage
// shared-memory ring with bulk asynchronous copies that complete on an
// mbarrier.  The consumers run the register FFT of `fft_core.cuh` on the tile
// in the ring, exchange through a separate shared buffer, and store the
// results straight from registers.  Loads of the next two tiles are in flight
// while a tile is computed, which the one-tile-per-block kernels could not do.
//
// Two kinds of tile share the kernel:
//  * contiguous tile: P pencils of length NC that are consecutive in memory
//    (the superstep along the contiguous axis);
//  * strided tile: W adjacent pencils of length NS, one row of W elements
//    per pencil element, rows `s_stride` elements apart (a superstep along a
//    strided axis; the paper's transpose, Section 4.3, becomes the choice of
//    rows).
// A contiguous tile may signal a per-unit counter when its stores are done
// and a strided tile may wait for a unit's counter to reach a target.  This
// is how the supersteps along the two inner axes of one slab (unit) of a 3D
// array run in a single launch: the strided tiles of a slab are queued a few
// slabs after its contiguous tiles, so the intermediate result is re-read
// while it is still in L2 and the array makes two trips through HBM instead
// of three (Section 4.2 runs the z, x and y supersteps with transposes in
// between; the order of axes is free, Section 1).
//
// Every wait is bounded by a deadline on %globaltimer; when one runs out the
// block records WSFFT_ERR_DEVICE_TIMEOUT in the plan's status word and stops
// taking tickets.
#pragma once

#include "fft_core.cuh"
#include "pass_kernels.cuh"

namespace wsfft {

// ---------------------------------------------------------------------------
// PTX wrappers (mbarrier, bulk async copy, cache policy, ordering)

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                          uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_normal() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u32(uint32_t *p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void consumer_bar(int nthreads) {
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}
// barrier over the consumers that also returns whether any of them passed v
__device__ __forceinline__ bool consumer_any(bool v, int nthreads) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\t"
        "setp.ne.u32 pi, %1, 0;\n\t"
        "bar.red.or.pred po, 1, %2, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(nthreads)
        : "memory");
    return r != 0;
}

// ---------------------------------------------------------------------------

enum : int {
    ITEM_STRIDED = 1,  // else contiguous
    ITEM_WAIT = 2,     // wait for ctr[1 + unit] >= dep_target before loading
    ITEM_SIGNAL = 4,   // add 1 to ctr[1 + unit] after the stores
    ITEM_END = 8,
    ITEM_SKIP = 16,    // (in a block only) the wait for this tile ran out
};

struct EngItem {
    int flags;
    int unit;
    int tile;
    int pad;
};

struct EngArgs {
    const EngItem *items;
    int nitems;
    uint32_t *ctr;          // [0] ticket counter, [1 + u] per-unit completion counters
    int *status;            // set to 1 when a wait runs out
    const void *c_src;      // contiguous tiles: source base
    void *c_dst;            //                   destination base
    const void *s_src;      // strided tiles
    void *s_dst;
    int64_t unit_elems;     // elements per unit
    int64_t s_stride;       // strided tiles: element stride between rows
    const float2 *tw_c, *tw_s;
    float c_ci, c_sx, c_sy;  // contiguous: load conjugation, store scale (re, im)
    float s_ci, s_sx, s_sy;
    uint32_t dep_target;
    int s_evict_first;      // strided loads stream (read once) rather than reuse
    uint64_t timeout_ns;
};

template <class S, int NC, int P, int CONS>
struct EngContigAcc {
    const S *ring;   // this pencil's row in the ring stage
    S *out;          // this pencil in global memory
    float2 *sm;      // this pencil's exchange row
    uint64_t *empty;
    float ci, sx, sy;
    __device__ __forceinline__ float2 gload(int k) const {
        float2 v = Cvt<S>::load(ring + k);
        v.y *= ci;
        return v;
    }
    __device__ __forceinline__ void after_load() const { mbar_arrive(empty); }
    __device__ __forceinline__ void gstore(int k, float2 v) const {
        Cvt<S>::store(out + k, make_float2(v.x * sx, v.y * sy));
    }
    __device__ __forceinline__ void sstore(int k, float2 v) const { sm[k + (k >> 4)] = v; }
    __device__ __forceinline__ float2 sload(int k) const { return sm[k + (k >> 4)]; }
    __device__ __forceinline__ void sync() const { consumer_bar(CONS); }
};

template <class S, int W, int CONS>
struct EngStridedAcc {
    const S *ring;   // ring stage base ([k][W] dense)
    S *out;          // this pencil's first element in global memory
    float2 *sm;      // exchange buffer base
    uint64_t *empty;
    int64_t stride;
    int w;
    float ci, sx, sy;
    __device__ __forceinline__ float2 gload(int k) const {
        float2 v = Cvt<S>::load(ring + k * W + w);
        v.y *= ci;
        return v;
    }
    __device__ __forceinline__ void after_load() const { mbar_arrive(empty); }
    __device__ __forceinline__ void gstore(int k, float2 v) const {
        Cvt<S>::store(out + (int64_t)k * stride, make_float2(v.x * sx, v.y * sy));
    }
    __device__ __forceinline__ int sidx(int k) const { return k * W + w + ((k * W) >> 4); }
    __device__ __forceinline__ void sstore(int k, float2 v) const { sm[sidx(k)] = v; }
    __device__ __forceinline__ float2 sload(int k) const { return sm[sidx(k)]; }
    __device__ __forceinline__ void sync() const { consumer_bar(CONS); }
};

template <int NC, int EC, int P, int NS, int ES, int W, class S>
struct EngCfg {
    static constexpr int CONS = P * (NC / EC);
    static_assert(CONS == W * (NS / ES), "both tile kinds need the same thread count");
    static_assert(CONS % 32 == 0, "whole warps");
    static constexpr int NSTAGE = 2;
    static constexpr int TILE_C = P * NC;
    static constexpr int TILE_S = NS * W;
    static constexpr int TILE = TILE_C > TILE_S ? TILE_C : TILE_S;  // elements
    static constexpr int TILE_BYTES = TILE * (int)sizeof(S);
    static constexpr int XC = P * contig_PS(NC);
    static constexpr int XS = NS * W + (NS * W) / 16;
    static constexpr int XELEMS = XC > XS ? XC : XS;
    static constexpr int RING_BYTES = NSTAGE * TILE_BYTES;
    static constexpr int SMEM = RING_BYTES + XELEMS * 8 + 2 * NSTAGE * 8 + NSTAGE * 16;
    static constexpr int THREADS = CONS + 32;
};

template <int NC, int EC, int P, int NS, int ES, int W, class S>
__global__ void __launch_bounds__(EngCfg<NC, EC, P, NS, ES, W, S>::THREADS, 1)
    engine_kernel(EngArgs a) {
    using C = EngCfg<NC, EC, P, NS, ES, W, S>;
    constexpr int CONS = C::CONS;
    constexpr int NSTAGE = C::NSTAGE;
    extern __shared__ __align__(128) unsigned char eng_smem[];
    S *ring = reinterpret_cast<S *>(eng_smem);
    float2 *xbuf = reinterpret_cast<float2 *>(eng_smem + C::RING_BYTES);
    uint64_t *full = reinterpret_cast<uint64_t *>(xbuf + C::XELEMS);
    uint64_t *empty = full + NSTAGE;
    int4 *slot = reinterpret_cast<int4 *>(empty + NSTAGE);

    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int i = 0; i < NSTAGE; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], CONS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (tid >= CONS) {
        // ------------------------------------------------------------- producer
        const int lane = tid - CONS;
        const uint64_t pol_first = policy_evict_first();
        const uint64_t pol_norm = policy_evict_normal();
        bool stop = false;
        for (int it = 0; !stop; ++it) {
            const int st = it % NSTAGE;
            int ticket = 0;
            if (lane == 0) ticket = (int)atomicAdd(&a.ctr[0], 1u);
            ticket = __shfl_sync(0xffffffffu, ticket, 0);
            EngItem item;
            if (ticket < a.nitems) {
                item = a.items[ticket];
            } else {
                item.flags = ITEM_END;
                item.unit = item.tile = item.pad = 0;
            }
            int fail = 0;
            // stage free?  (its previous tile has been read by every consumer)
            if (it >= NSTAGE && lane == 0) {
                const uint32_t par = ((it / NSTAGE) - 1) & 1;
                const uint64_t dl = gtimer() + a.timeout_ns;
                while (!mbar_try_wait(&empty[st], par)) {
                    if (gtimer() > dl) {
                        fail = 1;
                        break;
                    }
                }
            }
            // inputs complete?
            const uint32_t *dep = a.ctr + 1 + item.unit;
            if (!fail && (item.flags & ITEM_WAIT) && lane == 0) {
                if (ld_acquire_u32(dep) < a.dep_target) {
                    const uint64_t dl = gtimer() + a.timeout_ns;
                    while (ld_acquire_u32(dep) < a.dep_target) {
                        if (gtimer() > dl) {
                            fail = 1;
                            break;
                        }
                        __nanosleep(64);
                    }
                }
            }
            fail = __shfl_sync(0xffffffffu, fail, 0);
            if (!fail && (item.flags & ITEM_WAIT)) {
                // every lane that issues a copy of the tile acquires the
                // counter itself, then orders the copies (async proxy) after it
                (void)ld_acquire_u32(dep);
                fence_proxy_async_global();
            }
            if (fail) {
                if (lane == 0) atomicExch(a.status, 1);
                item.flags = ITEM_END;
            }
            if (item.flags & ITEM_END) {
                stop = true;
                if (lane == 0) {
                    // the consumers read a stage's slot before they release the
                    // stage, so the slot is free even after a failed wait
                    slot[st] = make_int4(ITEM_END, 0, 0, 0);
                    mbar_arrive(&full[st]);
                }
                break;
            }
            if (lane == 0) {
                slot[st] = make_int4(item.flags, item.unit, item.tile, 0);
                mbar_arrive_expect_tx(&full[st], (item.flags & ITEM_STRIDED)
                                                     ? C::TILE_S * (int)sizeof(S)
                                                     : C::TILE_C * (int)sizeof(S));
            }
            __syncwarp();
            S *dst = ring + (size_t)st * C::TILE;
            if (item.flags & ITEM_STRIDED) {
                const S *src = reinterpret_cast<const S *>(a.s_src) + (int64_t)item.unit * a.unit_elems +
                               (int64_t)item.tile * W;
                const uint64_t pol = a.s_evict_first ? pol_first : pol_norm;
                for (int r = lane; r < NS; r += 32)
                    bulk_load(dst + r * W, src + (int64_t)r * a.s_stride, W * (int)sizeof(S), &full[st], pol);
            } else {
                const S *src = reinterpret_cast<const S *>(a.c_src) + (int64_t)item.unit * a.unit_elems +
                               (int64_t)item.tile * C::TILE_C;
                for (int r = lane; r < P; r += 32)
                    bulk_load(dst + r * NC, src + (int64_t)r * NC, NC * (int)sizeof(S), &full[st], pol_first);
            }
        }
        return;
    }

    // ----------------------------------------------------------------- consumers
    for (int it = 0;; ++it) {
        const int st = it % NSTAGE;
        const uint32_t par = (it / NSTAGE) & 1;
        const uint64_t dl = gtimer() + 4 * a.timeout_ns;
        bool ok = true;
        while (!mbar_try_wait(&full[st], par)) {
            if (gtimer() > dl) {
                ok = false;
                break;
            }
        }
        // all consumers take the same decision, so their barriers stay matched
        if (consumer_any(!ok, CONS)) {
            if (tid == 0) atomicExch(a.status, 1);
            break;
        }
        const int4 item = slot[st];
        if (item.x & ITEM_END) break;
        const S *rs = ring + (size_t)st * C::TILE;
        if (item.x & ITEM_STRIDED) {
            constexpr int T = NS / ES;
            const int w = tid % W, t = tid / W;
            EngStridedAcc<S, W, CONS> acc;
            acc.ring = rs;
            acc.out = reinterpret_cast<S *>(a.s_dst) + (int64_t)item.y * a.unit_elems +
                      (int64_t)item.z * W + w;
            acc.sm = xbuf;
            acc.empty = &empty[st];
            acc.stride = a.s_stride;
            acc.w = w;
            acc.ci = a.s_ci;
            acc.sx = a.s_sx;
            acc.sy = a.s_sy;
            (void)T;
            pencil_fft<NS, ES>(acc, t, a.tw_s);
        } else {
            constexpr int T = NC / EC;
            const int t = tid % T, p = tid / T;
            EngContigAcc<S, NC, P, CONS> acc;
            acc.ring = rs + p * NC;
            acc.out = reinterpret_cast<S *>(a.c_dst) + (int64_t)item.y * a.unit_elems +
                      (int64_t)item.z * C::TILE_C + (int64_t)p * NC;
            acc.sm = xbuf + p * contig_PS(NC);
            acc.empty = &empty[st];
            acc.ci = a.c_ci;
            acc.sx = a.c_sx;
            acc.sy = a.c_sy;
            pencil_fft<NC, EC>(acc, t, a.tw_c);
        }
        if (item.x & ITEM_SIGNAL) {
            consumer_bar(CONS);
            if (tid == 0) {
                __threadfence();
                red_release_add_u32(a.ctr + 1 + item.y, 1u);
            }
        }
    }
}

}  // namespace wsfft
