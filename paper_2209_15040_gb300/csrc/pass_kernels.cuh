// Superstep kernels: one launch transforms every pencil along one axis.
//
// The array is viewed, for the axis being transformed, as [outer][N][inner]
// elements: `inner` is the product of the later axes (1 for the contiguous
// axis), `outer` the product of the earlier axes and the batch.  A pencil is
// one (outer, inner) pair (Section 2.1, pencil decomposition); the paper's
// processing element that owns a pencil becomes a group of T = N/E threads,
// and the redistribution between supersteps (Section 4.3) becomes the choice
// of which pencils a thread block gathers:
//
//  * contiguous axis (inner == 1): a block takes P whole pencils, each a
//    contiguous run of N elements; threads of a pencil are consecutive, so
//    each warp-wide load or store touches consecutive addresses.
//  * strided axis (inner > 1): a block takes W pencils that are adjacent in
//    memory (consecutive inner index).  Row k of the tile is W consecutive
//    elements, so the "transpose" of the paper is fused into loads and stores
//    that read whole 128-byte rows; the pencil index is the fastest thread
//    index, which keeps shared-memory exchanges free of bank conflicts.
#pragma once

#include <type_traits>

#include "fft_core.cuh"
#include "pass_desc.h"

namespace wsfft {

// Programmatic dependent launch: every block lets the next kernel in the
// stream start launching (its blocks take SM slots as this grid drains, and
// its launch latency overlaps this grid's tail), and waits until the
// previous kernel has completed and its writes are visible before touching
// memory.  Both are no-ops for a launch without the attribute.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Elements per thread for an axis of length N (the default variant).
__host__ __device__ constexpr int default_E(int N) {
    return N <= 16 ? N : (N <= 64 ? 8 : (N == 512 ? 8 : 16));
}
// pencils per block, contiguous axis
__host__ __device__ constexpr int contig_P(int N, int E, bool trans) {
    return trans ? ((N / E) >= 64 ? 1024 / (N / E) : (256 / (N / E) > 16 ? 256 / (N / E) : 16))
                 : ((N / E) >= 256 ? 1 : 256 / (N / E));
}
// pencils per block, strided axis
__host__ __device__ constexpr int strided_W(int N, int E) {
    return (N / E) >= 16 ? ((N / E) <= 64 ? 16 : 1024 / (N / E)) : 256 / (N / E);
}
// shared-memory row stride (complex elements) of one pencil, contiguous axis
__host__ __device__ constexpr int contig_PS(int N) { return N + N / 16 + 4; }

__host__ __device__ constexpr int contig_smem_elems(int N, int E, int P, bool trans) {
    return (N / E) == 1 && !trans
               ? P * (N + 1)  // one thread per pencil: staging tile for coalesced copies
               : (P * contig_PS(N) > (trans ? N * (P + 1) : 0) ? P * contig_PS(N) : N * (P + 1));
}
__host__ __device__ constexpr int strided_smem_elems(int N, int E, int W) {
    return (N / E) == 1 ? 0 : N * W + (N * W) / 16;
}

// Epilogue: optional four-step twiddle, then scale and conjugate.
struct Epi {
    float sx, sy;  // multiply re by sx, im by sy (sy = -sx conjugates)
};

// PLAIN: no conjugation on load and no scaling on store (the forward pass
// of the unscaled transform), which saves three multiplies per element.
// WARP: the pencil's threads all sit in one warp (at most 32 threads per
// pencil) and its exchange row is theirs alone, so the exchanges need only
// a warp barrier.
template <class S, int LOP = OP_DEF, int SOP = OP_DEF, bool PLAIN = false, bool WARP = false>
struct ContigAcc {
    const S *in;   // this pencil's first element
    S *out;        // this pencil's first element (unused when transposing)
    float2 *sm;    // this pencil's shared-memory row
    float ci;      // +1, or -1 to conjugate on load
    Epi epi;
    bool active;
    __device__ __forceinline__ float2 gload(int k) const {
        float2 v = active ? Cvt<S>::template load<LOP>(in + k) : make_float2(0.f, 0.f);
        if constexpr (!PLAIN) v.y *= ci;
        return v;
    }
    __device__ __forceinline__ void gstore(int k, float2 v) const {
        if constexpr (!PLAIN) v = make_float2(v.x * epi.sx, v.y * epi.sy);
        if (active) Cvt<S>::template store<SOP>(out + k, v);
    }
    // element k sits at k + k/16: one pad per 16 spreads the radix-16/8
    // Stockham patterns over all banks; unsigned keeps (t + 16m) >> 4 linear
    __device__ __forceinline__ static int sidx(int k) { return (int)((unsigned)k + ((unsigned)k >> 4)); }
    __device__ __forceinline__ void sstore(int k, float2 v) const { sm[sidx(k)] = v; }
    __device__ __forceinline__ float2 sload(int k) const { return sm[sidx(k)]; }
    __device__ __forceinline__ void sync() const {
        if constexpr (WARP) __syncwarp();
        else __syncthreads();
    }
    __device__ __forceinline__ void after_load() const {}
};

// One thread's pencil staged in a shared-memory row (first loads and last
// stores of the register FFT go to the row; no exchanges happen).
template <class S, bool PLAIN>
struct WarpStagedRow {
    float2 *row;
    float ci, sx, sy;
    __device__ __forceinline__ float2 gload(int k) const {
        float2 v = row[k];
        if constexpr (!PLAIN) v.y *= ci;
        return v;
    }
    __device__ __forceinline__ void gstore(int k, float2 v) const {
        if constexpr (!PLAIN) v = make_float2(v.x * sx, v.y * sy);
        row[k] = v;
    }
    __device__ __forceinline__ void sstore(int k, float2 v) const { row[k] = v; }
    __device__ __forceinline__ float2 sload(int k) const { return row[k]; }
    __device__ __forceinline__ void sync() const {}
    __device__ __forceinline__ void after_load() const {}
};

// Contiguous axis, transposed store for the four-step split of a long 1D
// axis: the result of pencil p (row k2 of transform b) element k goes to
// out[b*N + k*rows + k2], staged through shared memory so the global store
// is P consecutive elements per k.
template <class S>
struct ContigTransAcc : ContigAcc<S> {
    float2 *stage;  // [N][P+1] staging
    int p, P;
    __device__ __forceinline__ void gstore(int k, float2 v) const { stage[k * (P + 1) + p] = v; }
};

template <int N, int E, int P, class S, bool TRANS, bool PLAIN = false>
__global__ void __launch_bounds__(P *(N / E))
    contig_kernel(const S *__restrict__ in, S *__restrict__ out, PassArgs a) {
    extern __shared__ float2 smem[];
    // Pencils of up to 512 points stored in place let the next kernel start
    // launching only after their stores (measured, complex64: 512^3 step
    // 967.4 -> 964.9 us, 128^3 19.7 -> 19.2 us, 256^3 unchanged); the
    // transposing and 1024-point variants keep the early signal (with the
    // late one the 1D 2^20 four-step lost 0.5%, 1024^3 0.5%)
    constexpr bool late_signal = !TRANS && N <= 512;
    if constexpr (late_signal) {
        asm volatile("griddepcontrol.wait;" ::: "memory");
    } else {
        pdl_enter();
    }
    constexpr int T = N / E;
    const int t = threadIdx.x % T;
    const int p = threadIdx.x / T;
    const int64_t tile = blockIdx.x;
    const int64_t q = tile * P + p;
    const bool active = q < a.npencils;
    if constexpr (!TRANS && T == 1) {
        // One thread per pencil (N <= 16): a thread's own loads would be N*8
        // bytes apart across the warp, so the block copies its P*N-element
        // slab (contiguous in memory) through shared memory, row stride N+1.
        const int64_t base = tile * P * N;
        const int64_t avail = (a.npencils - tile * P) * N;  // elements present in this tile
        for (int e = threadIdx.x; e < P * N; e += P)
            if (e < avail) smem[(e / N) * (N + 1) + e % N] = Cvt<S>::load(in + base + e);
        __syncthreads();
        WarpStagedRow<S, PLAIN> acc{smem + p * (N + 1), a.conj_in, a.sx, a.sy};
        pencil_fft<N, E>(acc, t, a.tw);
        __syncthreads();
        for (int e = threadIdx.x; e < P * N; e += P)
            if (e < avail) Cvt<S>::store(out + base + e, smem[(e / N) * (N + 1) + e % N]);
    } else if constexpr (!TRANS) {
        ContigAcc<S, OP_DEF, OP_DEF, PLAIN, (T <= 32)> acc{in + q * N, out + q * N, smem + p * contig_PS(N),
                                                           a.conj_in, {a.sx, a.sy}, active};
        pencil_fft<N, E>(acc, t, a.tw);
    } else {
        ContigTransAcc<S> acc;
        acc.in = in + q * N;
        acc.out = nullptr;
        acc.sm = smem + p * contig_PS(N);
        acc.ci = a.conj_in;
        acc.epi = {a.sx, a.sy};
        acc.active = active;
        acc.stage = smem;
        acc.p = p;
        acc.P = P;
        pencil_fft<N, E>(acc, t, a.tw);
        __syncthreads();
        // rows per transform a.trans_rows is a multiple of P, so the tile's
        // rows belong to one transform
        const int64_t q0 = tile * P;
        const int64_t b = q0 / a.trans_rows;
        const int64_t row0 = q0 - b * a.trans_rows;
        S *ob = out + b * (int64_t)N * a.trans_rows + row0;
        for (int idx = threadIdx.x; idx < N * P; idx += P * T) {
            const int pp = idx % P, k = idx / P;
            if (q0 + pp < a.npencils) {
                const float2 v = smem[k * (P + 1) + pp];
                Cvt<S>::store(ob + (int64_t)k * a.trans_rows + pp,
                              make_float2(v.x * a.sx, v.y * a.sy));
            }
        }
    }
    if constexpr (late_signal) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <class S, bool TWID, int LOP, int SOP, int W, bool PLAIN = false>
struct StridedAcc {
    const S *in;   // this pencil's first element
    S *out;
    float2 *sm;    // tile base in shared memory
    int64_t stride;
    int w;
    float ci;
    Epi epi;
    bool active;
    int twq;        // four-step: inner index of this pencil
    const float2 *tw_hi, *tw_lo;  // four-step: w_L^m = tw_hi[m >> tw_shift] * tw_lo[m & low mask]
    int tw_shift;
    int tw_mask;    // four-step: L - 1 (L = length of the long transform)
    __device__ __forceinline__ float2 gload(int k) const {
        float2 v = active ? Cvt<S>::template load<LOP>(in + (int64_t)k * stride) : make_float2(0.f, 0.f);
        if constexpr (!PLAIN) v.y *= ci;
        return v;
    }
    __device__ __forceinline__ void gstore(int k, float2 v) const {
        if constexpr (TWID) {
            // w_L^(q*k), L = tw_mask + 1, from two tables of the host's
            // long-double roots: w_L^m = w_L^(m_hi << shift) * w_L^(m_lo)
            const int m = (twq * k) & tw_mask;
            v = cmul(v, cmul(__ldg(&tw_hi[m >> tw_shift]), __ldg(&tw_lo[m & ((1 << tw_shift) - 1)])));
        }
        if constexpr (!PLAIN) v = make_float2(v.x * epi.sx, v.y * epi.sy);
        if (active) Cvt<S>::template store<SOP>(out + (int64_t)k * stride, v);
    }
    // row k of W elements plus one pad per 16 elements; linear in k when W is
    // a multiple of 16, so every index is a per-thread base plus a constant
    __device__ __forceinline__ int sidx(int k) const {
        if constexpr (W % 16 == 0) return k * (W + W / 16) + w;
        else return k * W + w + ((k * W) >> 4);
    }
    __device__ __forceinline__ void sstore(int k, float2 v) const { sm[sidx(k)] = v; }
    __device__ __forceinline__ float2 sload(int k) const { return sm[sidx(k)]; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ void after_load() const {}
};

// Blocks of up to 512 threads are held to 1024 threads per SM worth of
// registers (two 512-thread blocks at 64 registers): measured faster at
// 512^3 than letting the compiler use more registers and fit one block.
// Blocks per SM the register budget is held to: 1024 threads per SM for up
// to 16 values per thread, 512 threads per SM for 32 (their radix-32 stages
// need about twice the registers).
__host__ __device__ constexpr int strided_min_blocks(int threads, int values) {
    return values >= 32 ? (threads <= 256 ? 512 / threads : 1) : (threads <= 512 ? 1024 / threads : 1);
}
template <int N, int E, int W, class S, bool TWID, bool PLAIN = false>
__global__ void __launch_bounds__(W *(N / E), strided_min_blocks(W *(N / E), E))
    strided_kernel(const S *__restrict__ in, S *__restrict__ out, PassArgs a) {
    extern __shared__ float2 smem[];
    pdl_enter();
    const int w = threadIdx.x % W;
    const int t = threadIdx.x / W;
    const int64_t blk = a.reverse ? (int64_t)gridDim.x - 1 - blockIdx.x : (int64_t)blockIdx.x;
    const int64_t q = (blk + a.tile0) * W + w;
    const int64_t o = q >> a.log_inner;
    const int64_t i = q & (a.inner - 1);
    const int64_t base = o * ((int64_t)N << a.log_inner) + i;
    StridedAcc<S, TWID, OP_DEF, OP_DEF, W, PLAIN> acc;
    acc.in = in + base;
    acc.out = out + base;
    acc.sm = smem;
    acc.stride = a.inner;
    acc.w = w;
    acc.ci = a.conj_in;
    acc.epi = {a.sx, a.sy};
    acc.active = q < a.npencils;
    acc.twq = (int)i;
    acc.tw_hi = a.tw_hi;
    acc.tw_lo = a.tw_lo;
    acc.tw_shift = a.tw_shift;
    acc.tw_mask = a.tw_mask;
    pencil_fft<N, E>(acc, t, a.tw);
}

// Pencil pairs: thread (wp, t) carries pencils 2wp and 2wp+1 of a strided
// tile as float4 values (re0, im0, re1, im1), so each global access moves
// two adjacent elements of a row at once (16 bytes in complex64, 8 in the
// half types), each shared access 16 bytes, and each twiddle serves both
// pencils.  W pencils = W/2 pairs per row.
template <class S>
struct Pair;
template <>
struct Pair<float2> {
    using T = float4;
    template <int OP = OP_DEF>
    __device__ __forceinline__ static float4 load(const T *p) { return ld_op<OP>(p); }
    template <int OP = OP_DEF>
    __device__ __forceinline__ static void store(T *p, float4 v) { st_op<OP>(p, v); }
};
template <>
struct Pair<__half2> {
    using T = uint2;
    template <int OP = OP_DEF>
    __device__ __forceinline__ static float4 load(const T *p) {
        const uint2 u = ld_op<OP>(p);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    template <int OP = OP_DEF>
    __device__ __forceinline__ static void store(T *p, float4 v) {
        const __half2 a = __float22half2_rn(make_float2(v.x, v.y));
        const __half2 b = __float22half2_rn(make_float2(v.z, v.w));
        uint2 u;
        u.x = *reinterpret_cast<const unsigned *>(&a);
        u.y = *reinterpret_cast<const unsigned *>(&b);
        st_op<OP>(p, u);
    }
};
template <>
struct Pair<__nv_bfloat162> {
    using T = uint2;
    template <int OP = OP_DEF>
    __device__ __forceinline__ static float4 load(const T *p) {
        const uint2 u = ld_op<OP>(p);
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    template <int OP = OP_DEF>
    __device__ __forceinline__ static void store(T *p, float4 v) {
        const __nv_bfloat162 a = __float22bfloat162_rn(make_float2(v.x, v.y));
        const __nv_bfloat162 b = __float22bfloat162_rn(make_float2(v.z, v.w));
        uint2 u;
        u.x = *reinterpret_cast<const unsigned *>(&a);
        u.y = *reinterpret_cast<const unsigned *>(&b);
        st_op<OP>(p, u);
    }
};

template <class S, int W, bool PLAIN, int LOP = OP_DEF, int SOP = OP_DEF>
struct StridedPairAcc {
    using value_type = float4;
    using PT = typename Pair<S>::T;
    const PT *in;       // this pair's element 0
    PT *out;
    float4 *sm;         // tile base, [k][W/2] float4
    int64_t stride;     // in pair units: element stride / 2
    int wp;
    float ci, sx, sy;
    bool active;
    __device__ __forceinline__ float4 gload(int k) const {
        float4 v = active ? Pair<S>::template load<LOP>(in + (int64_t)k * stride) : make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (!PLAIN) {
            v.y *= ci;
            v.w *= ci;
        }
        return v;
    }
    __device__ __forceinline__ void gstore(int k, float4 v) const {
        if constexpr (!PLAIN) v = make_float4(v.x * sx, v.y * sy, v.z * sx, v.w * sy);
        if (active) Pair<S>::template store<SOP>(out + (int64_t)k * stride, v);
    }
    // a row of W/2 float4 is 8*W bytes; rows of 128 bytes cover all banks,
    // so four rows per warp access are four wavefronts, the minimum
    __device__ __forceinline__ int sidx(int k) const { return k * (W / 2) + wp; }
    __device__ __forceinline__ void sstore(int k, float4 v) const { sm[sidx(k)] = v; }
    __device__ __forceinline__ float4 sload(int k) const { return sm[sidx(k)]; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ void after_load() const {}
};

// Split-form pencil pairs: the same tile and memory accesses as the pairs
// above, but each value is held as (re0, re1), (im0, im1) so that the
// butterflies run as packed FP32x2 instructions (cpair).  16-bit storage
// converts straight into that form (two byte permutes per element pair).
template <class S>
struct SplitPair;
template <>
struct SplitPair<float2> {
    using T = float4;
    template <int OP = OP_DEF>
    __device__ __forceinline__ static cpair load(const T *p) {
        const float4 v = ld_op<OP>(p);
        return {make_float2(v.x, v.z), make_float2(v.y, v.w)};
    }
    template <int OP = OP_DEF>
    __device__ __forceinline__ static void store(T *p, cpair v) {
        st_op<OP>(p, make_float4(v.re.x, v.im.x, v.re.y, v.im.y));
    }
};
template <>
struct SplitPair<__half2> {
    using T = uint2;
    template <int OP = OP_DEF>
    __device__ __forceinline__ static cpair load(const T *p) {
        const uint2 u = ld_op<OP>(p);
        const __half2 a = *reinterpret_cast<const __half2 *>(&u.x);  // (re0, im0)
        const __half2 b = *reinterpret_cast<const __half2 *>(&u.y);  // (re1, im1)
        return {__half22float2(__lows2half2(a, b)), __half22float2(__highs2half2(a, b))};
    }
    template <int OP = OP_DEF>
    __device__ __forceinline__ static void store(T *p, cpair v) {
        const __half2 r = __float22half2_rn(v.re), i = __float22half2_rn(v.im);
        const __half2 a = __lows2half2(r, i), b = __highs2half2(r, i);
        uint2 u;
        u.x = *reinterpret_cast<const unsigned *>(&a);
        u.y = *reinterpret_cast<const unsigned *>(&b);
        st_op<OP>(p, u);
    }
};
template <>
struct SplitPair<__nv_bfloat162> {
    using T = uint2;
    template <int OP = OP_DEF>
    __device__ __forceinline__ static cpair load(const T *p) {
        const uint2 u = ld_op<OP>(p);
        const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162 *>(&u.x);
        const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162 *>(&u.y);
        return {__bfloat1622float2(__lows2bfloat162(a, b)), __bfloat1622float2(__highs2bfloat162(a, b))};
    }
    template <int OP = OP_DEF>
    __device__ __forceinline__ static void store(T *p, cpair v) {
        const __nv_bfloat162 r = __float22bfloat162_rn(v.re), i = __float22bfloat162_rn(v.im);
        const __nv_bfloat162 a = __lows2bfloat162(r, i), b = __highs2bfloat162(r, i);
        uint2 u;
        u.x = *reinterpret_cast<const unsigned *>(&a);
        u.y = *reinterpret_cast<const unsigned *>(&b);
        st_op<OP>(p, u);
    }
};

template <class S, int W, bool PLAIN, int LOP = OP_DEF, int SOP = OP_DEF>
struct StridedSplitAcc {
    using value_type = cpair;
    using PT = typename SplitPair<S>::T;
    const PT *in;       // this pair's element 0
    PT *out;
    float4 *sm;         // tile base, [k][W/2] float4 (re0, re1, im0, im1)
    int64_t stride;     // in pair units: element stride / 2
    int wp;
    float ci, sx, sy;
    bool active;
    __device__ __forceinline__ cpair gload(int k) const {
        cpair v = active ? SplitPair<S>::template load<LOP>(in + (int64_t)k * stride)
                         : cpair{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        if constexpr (!PLAIN) v.im = __fmul2_rn(v.im, f2dup(ci));
        return v;
    }
    __device__ __forceinline__ void gstore(int k, cpair v) const {
        if constexpr (!PLAIN) {
            v.re = __fmul2_rn(v.re, f2dup(sx));
            v.im = __fmul2_rn(v.im, f2dup(sy));
        }
        if (active) SplitPair<S>::template store<SOP>(out + (int64_t)k * stride, v);
    }
    __device__ __forceinline__ int sidx(int k) const { return k * (W / 2) + wp; }
    __device__ __forceinline__ void sstore(int k, cpair v) const {
        sm[sidx(k)] = make_float4(v.re.x, v.re.y, v.im.x, v.im.y);
    }
    __device__ __forceinline__ cpair sload(int k) const {
        const float4 v = sm[sidx(k)];
        return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
    }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ void after_load() const {}
};

// Split form of two single elements (one of each pencil of a pair)
template <class S>
struct SplitCvt;
template <>
struct SplitCvt<float2> {
    __device__ __forceinline__ static float2 zero() { return make_float2(0.f, 0.f); }
    __device__ __forceinline__ static cpair join(float2 a, float2 b) {
        return {make_float2(a.x, b.x), make_float2(a.y, b.y)};
    }
    __device__ __forceinline__ static void split(cpair v, float2 &a, float2 &b) {
        a = make_float2(v.re.x, v.im.x);
        b = make_float2(v.re.y, v.im.y);
    }
};
template <>
struct SplitCvt<__half2> {
    __device__ __forceinline__ static __half2 zero() { return __float2half2_rn(0.f); }
    __device__ __forceinline__ static cpair join(__half2 a, __half2 b) {
        return {__half22float2(__lows2half2(a, b)), __half22float2(__highs2half2(a, b))};
    }
    __device__ __forceinline__ static void split(cpair v, __half2 &a, __half2 &b) {
        const __half2 r = __float22half2_rn(v.re), i = __float22half2_rn(v.im);
        a = __lows2half2(r, i);
        b = __highs2half2(r, i);
    }
};
template <>
struct SplitCvt<__nv_bfloat162> {
    __device__ __forceinline__ static __nv_bfloat162 zero() { return __float2bfloat162_rn(0.f); }
    __device__ __forceinline__ static cpair join(__nv_bfloat162 a, __nv_bfloat162 b) {
        return {__bfloat1622float2(__lows2bfloat162(a, b)), __bfloat1622float2(__highs2bfloat162(a, b))};
    }
    __device__ __forceinline__ static void split(cpair v, __nv_bfloat162 &a, __nv_bfloat162 &b) {
        const __nv_bfloat162 r = __float22bfloat162_rn(v.re), i = __float22bfloat162_rn(v.im);
        a = __lows2bfloat162(r, i);
        b = __highs2bfloat162(r, i);
    }
};

// Contiguous axis, split-form pencil pairs: the T = N/E threads of a pair
// carry element k of two neighbouring pencils (q, q+1) as one cpair.  Each
// global access is one pencil's element (so a warp still reads consecutive
// addresses of one pencil per instruction), each shared access 16 bytes.
template <class S, bool PLAIN, bool WARP>
struct ContigSplitAcc {
    using value_type = cpair;
    const S *in;   // pencil q's first element; pencil q+1 follows at +N
    S *out;
    float4 *sm;    // this pair's shared-memory row, float4 (re0, re1, im0, im1)
    int n;         // pencil length
    float ci, sx, sy;
    bool act0, act1;
    __device__ __forceinline__ cpair gload(int k) const {
        const S a = act0 ? in[k] : SplitCvt<S>::zero();
        const S b = act1 ? in[n + k] : SplitCvt<S>::zero();
        cpair v = SplitCvt<S>::join(a, b);
        if constexpr (!PLAIN) v.im = __fmul2_rn(v.im, f2dup(ci));
        return v;
    }
    __device__ __forceinline__ void gstore(int k, cpair v) const {
        if constexpr (!PLAIN) {
            v.re = __fmul2_rn(v.re, f2dup(sx));
            v.im = __fmul2_rn(v.im, f2dup(sy));
        }
        S a, b;
        SplitCvt<S>::split(v, a, b);
        if (act0) out[k] = a;
        if (act1) out[n + k] = b;
    }
    // same padding as the one-pencil rows: one pad per 16 elements
    __device__ __forceinline__ static int sidx(int k) { return (int)((unsigned)k + ((unsigned)k >> 4)); }
    __device__ __forceinline__ void sstore(int k, cpair v) const {
        sm[sidx(k)] = make_float4(v.re.x, v.re.y, v.im.x, v.im.y);
    }
    __device__ __forceinline__ cpair sload(int k) const {
        const float4 v = sm[sidx(k)];
        return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
    }
    __device__ __forceinline__ void sync() const {
        if constexpr (WARP) __syncwarp();
        else __syncthreads();
    }
    __device__ __forceinline__ void after_load() const {}
};

// P pencils per block as P/2 split-form pairs.  Unlike the other superstep
// kernels, a block lets the next kernel start launching only after its own
// stores: the next kernel's blocks, arriving while this kernel's last wave
// ran, slowed it (512^3 FP16 step 750 us with the early signal, 713 us with
// no programmatic dependent launch after this kernel at all, 711 us with
// the signal after the stores)
template <int N, int E, int P, class S, bool PLAIN>
__global__ void __launch_bounds__((P / 2) * (N / E))
    contig_split_kernel(const S *__restrict__ in, S *__restrict__ out, PassArgs a) {
    extern __shared__ float4 qsmem[];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    constexpr int T = N / E;
    const int t = threadIdx.x % T;
    const int pp = threadIdx.x / T;
    const int64_t q = (int64_t)blockIdx.x * P + 2 * pp;
    ContigSplitAcc<S, PLAIN, (T <= 32)> acc{in + q * N, out + q * N, qsmem + pp * contig_PS(N), N,
                                            a.conj_in, a.sx, a.sy, q < a.npencils, q + 1 < a.npencils};
    pencil_fft<N, E>(acc, t, a.tw);
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// SPLIT selects the split-form accessor (packed FP32x2 butterflies)
template <int N, int E, int W, class S, bool PLAIN = false, bool SPLIT = false>
__global__ void __launch_bounds__((W / 2) * (N / E), strided_min_blocks((W / 2) * (N / E), 2 * E))
    strided_pair_kernel(const S *__restrict__ in, S *__restrict__ out, PassArgs a) {
    extern __shared__ float4 psmem[];
    pdl_enter();
    using PT = typename Pair<S>::T;
    constexpr int WP = W / 2;
    const int wp = threadIdx.x % WP;
    const int t = threadIdx.x / WP;
    const int64_t blk = a.reverse ? (int64_t)gridDim.x - 1 - blockIdx.x : (int64_t)blockIdx.x;
    const int64_t q = (blk + a.tile0) * W + 2 * wp;  // first pencil of the pair
    const int64_t o = q >> a.log_inner;
    const int64_t i = q & (a.inner - 1);
    const int64_t base = o * ((int64_t)N << a.log_inner) + i;   // element offset (even)
    std::conditional_t<SPLIT, StridedSplitAcc<S, W, PLAIN>, StridedPairAcc<S, W, PLAIN>> acc;
    acc.in = reinterpret_cast<const PT *>(in + base);
    acc.out = reinterpret_cast<PT *>(out + base);
    acc.sm = psmem;
    acc.stride = a.inner / 2;
    acc.wp = wp;
    acc.ci = a.conj_in;
    acc.sx = a.sx;
    acc.sy = a.sy;
    acc.active = q < a.npencils;  // pencil counts are multiples of W here
    pencil_fft<N, E>(acc, t, a.tw);
}

}  // namespace wsfft
