// Instantiation and dispatch of the superstep kernels for one storage type.
// Included once per storage type by pass_c32.cu, pass_c16f.cu, pass_c16bf.cu
// (with WSFFT_STORE and WSFFT_LAUNCH_NAME defined) so the three compile in
// parallel.
#pragma once

#include <cudaTypedefs.h>

#include <algorithm>
#include <type_traits>

#include "pass_kernels.cuh"
#include "tc_contig.cuh"

namespace wsfft {
namespace {

template <class K>
cudaError_t set_smem(K kernel, int bytes) {
    return set_smem_attr(reinterpret_cast<const void *>(kernel), bytes);
}

inline bool plain_pass(const PassArgs &a) { return a.conj_in == 1.f && a.sx == 1.f && a.sy == 1.f; }

// Launch with programmatic stream serialization (see pdl_enter): the kernel
// may begin launching while the previous kernel in the stream drains.  Used
// for passes over at most 2 GiB: measured 0.7% faster per transform at 512^3
// and 5% at 256^3, but 14% slower at 1024^3 (8 GiB), so larger passes
// launch plainly.
inline bool pdl_pass(const PassArgs &a, int N, int elem_bytes) {
    return a.npencils * (int64_t)N * elem_bytes <= ((int64_t)2 << 30);
}
template <class... KArgs, class... Args>
cudaError_t launch_pdl(bool pdl, void (*kernel)(KArgs...), unsigned grid, unsigned block, int smem,
                       cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int N, int E, int P, class S, bool TRANS>
cudaError_t launch_contig(const void *in, void *out, const PassArgs &a, cudaStream_t st) {
    constexpr int T = N / E;
    constexpr int smem = contig_smem_elems(N, E, P, TRANS) * (int)sizeof(float2);
    const bool plain = !TRANS && plain_pass(a);
    auto kern = plain ? contig_kernel<N, E, P, S, TRANS, !TRANS> : contig_kernel<N, E, P, S, TRANS, false>;
    const cudaError_t attr0 = set_smem(contig_kernel<N, E, P, S, TRANS, false>, smem);
    const cudaError_t attr1 = set_smem(contig_kernel<N, E, P, S, TRANS, !TRANS>, smem);
    if (attr0 != cudaSuccess) return attr0;
    if (attr1 != cudaSuccess) return attr1;
    const int64_t blocks = (a.npencils + P - 1) / P;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    return launch_pdl(pdl_pass(a, N, sizeof(S)), kern, (unsigned)blocks, P * T, smem, st, (const S *)in, (S *)out,
                      a);
}

template <int N, int E, int P, class S>
cudaError_t launch_contig_split(const void *in, void *out, const PassArgs &a, cudaStream_t st) {
    static_assert(P % 2 == 0, "pairs");
    constexpr int smem = (P / 2) * contig_PS(N) * (int)sizeof(float4);
    const bool plain = plain_pass(a);
    auto kern = plain ? contig_split_kernel<N, E, P, S, true> : contig_split_kernel<N, E, P, S, false>;
    const cudaError_t attr0 = set_smem(contig_split_kernel<N, E, P, S, false>, smem);
    const cudaError_t attr1 = set_smem(contig_split_kernel<N, E, P, S, true>, smem);
    if (attr0 != cudaSuccess) return attr0;
    if (attr1 != cudaSuccess) return attr1;
    const int64_t blocks = (a.npencils + P - 1) / P;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    return launch_pdl(pdl_pass(a, N, sizeof(S)), kern, (unsigned)blocks, (P / 2) * (N / E), smem, st,
                      (const S *)in, (S *)out, a);
}

template <int N, int E, int W, class S, bool TWID>
cudaError_t launch_strided(const void *in, void *out, const PassArgs &a, cudaStream_t st) {
    constexpr int T = N / E;
    constexpr int smem = strided_smem_elems(N, E, W) * (int)sizeof(float2);
    // the general variant (conjugate on load, scale on store) even for plain
    // passes: measured faster than the multiply-free variant at 512^3
    const cudaError_t attr = set_smem(strided_kernel<N, E, W, S, TWID, false>, smem);
    if (attr != cudaSuccess) return attr;
    const int64_t blocks = (a.npencils + W - 1) / W;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    PassArgs b = a;
    b.tile0 = 0;
    return launch_pdl(pdl_pass(a, N, sizeof(S)), strided_kernel<N, E, W, S, TWID, false>, (unsigned)blocks, W * T,
                      smem, st, (const S *)in, (S *)out, b);
}

// Pencil-pair strided kernel: tile codes >= PAIR_TILE select it with
// W = tile - PAIR_TILE pencils per block.
template <int N, int E, int W, class S, bool SPLIT = false>
cudaError_t launch_strided_pair(const void *in, void *out, const PassArgs &a, cudaStream_t st) {
    constexpr int TH = (W / 2) * (N / E);
    constexpr int smem = N * (W / 2) * (int)sizeof(float4);
    const cudaError_t attr = set_smem(strided_pair_kernel<N, E, W, S, false, SPLIT>, smem);
    if (attr != cudaSuccess) return attr;
    if (a.npencils % W != 0 || a.inner % W != 0) return cudaErrorInvalidValue;
    const int64_t blocks = a.npencils / W;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    PassArgs b = a;
    b.tile0 = 0;
    // The general variant (conjugate on load, scale on store) is used even
    // for plain passes: at 512^3 it measured 8% faster than the variant
    // without those multiplies.
    return launch_pdl(pdl_pass(a, N, sizeof(S)), strided_pair_kernel<N, E, W, S, false, SPLIT>, (unsigned)blocks, TH, smem,
                      st, (const S *)in, (S *)out, b);
}

// default tile shape for (N, E)
template <int N, int E, class S>
cudaError_t launch_n(int kind, bool variant, const void *in, void *out, const PassArgs &a,
                     cudaStream_t st) {
    if (kind == PASS_CONTIG) {
        if (!variant) return launch_contig<N, E, contig_P(N, E, false), S, false>(in, out, a, st);
        if constexpr (N >= 64) return launch_contig<N, E, contig_P(N, E, true), S, true>(in, out, a, st);
    } else {
        if (!variant) return launch_strided<N, E, strided_W(N, E), S, false>(in, out, a, st);
        if constexpr (N >= 64) return launch_strided<N, E, strided_W(N, E), S, true>(in, out, a, st);
    }
    return cudaErrorInvalidValue;
}

// Extra (E, tile) shapes for the autotuner: plain (non-variant) passes only.
// tile = P for the contiguous axis, W for strided axes.
template <class S>
cudaError_t launch_extra(int kind, int N, int E, int tile, const void *in, void *out,
                         const PassArgs &a, cudaStream_t st) {
#define WSFFT_XC(n, e, t) \
    if (kind == PASS_CONTIG && N == n && E == e && tile == t) return launch_contig<n, e, t, S, false>(in, out, a, st);
#define WSFFT_XS(n, e, t) \
    if (kind == PASS_STRIDED && N == n && E == e && tile == t) return launch_strided<n, e, t, S, false>(in, out, a, st);
    WSFFT_XS(512, 16, 16)
    WSFFT_XS(512, 32, 16)
    WSFFT_XS(512, 32, 8)
    WSFFT_XS(512, 32, 32)
    WSFFT_XS(512, 8, 8)
    WSFFT_XS(512, 16, 8)
    WSFFT_XS(512, 16, 32)
    WSFFT_XS(256, 16, 32)
    WSFFT_XS(256, 8, 16)
    WSFFT_XS(1024, 16, 8)
    WSFFT_XS(1024, 32, 8)
    WSFFT_XS(1024, 32, 16)
    WSFFT_XC(1024, 32, 8)
    WSFFT_XC(512, 16, 8)
    WSFFT_XC(512, 32, 16)
    WSFFT_XC(512, 32, 8)
    WSFFT_XC(512, 32, 32)
    WSFFT_XC(512, 8, 8)
    WSFFT_XC(256, 8, 8)
    if (kind == PASS_CONTIG && tile >= SPLIT_TILE) {
        if (N == 512 && E == 16 && tile == SPLIT_TILE + 16) return launch_contig_split<512, 16, 16, S>(in, out, a, st);
        if (N == 512 && E == 16 && tile == SPLIT_TILE + 8) return launch_contig_split<512, 16, 8, S>(in, out, a, st);
        if (N == 512 && E == 8 && tile == SPLIT_TILE + 8) return launch_contig_split<512, 8, 8, S>(in, out, a, st);
        return cudaErrorInvalidValue;
    }
    if (kind == PASS_STRIDED && tile >= SPLIT_TILE) {
        if (N == 1024 && E == 16 && tile == SPLIT_TILE + 8)
            return launch_strided_pair<1024, 16, 8, S, true>(in, out, a, st);
        if (N == 512 && E == 16 && tile == SPLIT_TILE + 16)
            return launch_strided_pair<512, 16, 16, S, true>(in, out, a, st);
        if (N == 512 && E == 16 && tile == SPLIT_TILE + 32)
            return launch_strided_pair<512, 16, 32, S, true>(in, out, a, st);
        if (N == 512 && E == 8 && tile == SPLIT_TILE + 16)
            return launch_strided_pair<512, 8, 16, S, true>(in, out, a, st);
        if (N == 512 && E == 8 && tile == SPLIT_TILE + 32)
            return launch_strided_pair<512, 8, 32, S, true>(in, out, a, st);
        return cudaErrorInvalidValue;
    }
    if (kind == PASS_STRIDED && tile >= PAIR_TILE) {
        if (N == 512 && E == 8 && tile == PAIR_TILE + 16) return launch_strided_pair<512, 8, 16, S>(in, out, a, st);
        if (N == 512 && E == 8 && tile == PAIR_TILE + 32) return launch_strided_pair<512, 8, 32, S>(in, out, a, st);
        if (N == 512 && E == 8 && tile == PAIR_TILE + 8) return launch_strided_pair<512, 8, 8, S>(in, out, a, st);
        if (N == 512 && E == 16 && tile == PAIR_TILE + 16) return launch_strided_pair<512, 16, 16, S>(in, out, a, st);
        if (N == 512 && E == 16 && tile == PAIR_TILE + 32) return launch_strided_pair<512, 16, 32, S>(in, out, a, st);
        if (N == 256 && E == 8 && tile == PAIR_TILE + 16) return launch_strided_pair<256, 8, 16, S>(in, out, a, st);
    }
#undef WSFFT_XC
#undef WSFFT_XS
    return cudaErrorInvalidValue;
}

// Extra shapes of the variant passes (four-step twiddle on a strided store,
// transposed contiguous store).
template <class S>
cudaError_t launch_extra_variant(int kind, int N, int E, int tile, const void *in, void *out,
                                 const PassArgs &a, cudaStream_t st) {
    if (kind == PASS_STRIDED && N == 512 && E == 32 && tile == 16)
        return launch_strided<512, 32, 16, S, true>(in, out, a, st);
    if (kind == PASS_STRIDED && N == 1024 && E == 32 && tile == 8)
        return launch_strided<1024, 32, 8, S, true>(in, out, a, st);
    if (kind == PASS_STRIDED && N == 1024 && E == 32 && tile == 16)
        return launch_strided<1024, 32, 16, S, true>(in, out, a, st);
    if (kind == PASS_CONTIG && N == 1024 && E == 32 && tile == 8)
        return launch_contig<1024, 32, 8, S, true>(in, out, a, st);
    if (kind == PASS_CONTIG && N == 512 && E == 32 && tile == 16)
        return launch_contig<512, 32, 16, S, true>(in, out, a, st);
    return cudaErrorInvalidValue;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// dependency on the driver library)
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

// Tensor-core contiguous superstep (16-bit storage, N = 512).  The input is
// viewed as rows of 128 bytes (16 rows per pencil); the tensor map loads
// TC_P pencils per box with 128-byte swizzle.
template <class S>
cudaError_t launch_tc_contig(int N, const void *in, void *out, const PassArgs &a, cudaStream_t st) {
    if constexpr (std::is_same<S, float2>::value) {
        return cudaErrorInvalidValue;
    } else {
        if (N != 512) return cudaErrorInvalidValue;
        const cudaError_t attr = set_smem(tc_contig512_kernel<S>, TC_SMEM);
        if (attr != cudaSuccess) return attr;
        if (a.npencils <= 0) return cudaSuccess;
        const int64_t rows = a.npencils * 16;
        PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
        if (rows >= ((int64_t)1 << 31) || ((uintptr_t)in & 15) || !enc || !a.status)
            return launch_n<512, default_E(512), S>(PASS_CONTIG, false, in, out, a, st);
        // 128-byte swizzle: the MMA operand layout
        CUtensorMap map;
        const cuuint64_t dims[2] = {64, (cuuint64_t)rows};
        const cuuint64_t strides[1] = {128};
        const cuuint32_t box[2] = {64, (cuuint32_t)(TC_P * 16)};
        const cuuint32_t es[2] = {1, 1};
        if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void *>(in), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
        // persistent: one resident block per SM, tiles strided by the grid
        // (SM count and residency looked up once per device)
        constexpr int kMaxDev = 64;
        static int per_sm_dev[kMaxDev] = {}, sms_dev[kMaxDev] = {};
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return cudaErrorInvalidValue;
        if (per_sm_dev[dev] == 0) {
            int ps = 0, n = 0;
            if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, tc_contig512_kernel<S>, TC_THREADS, TC_SMEM) !=
                    cudaSuccess)
                return cudaErrorInvalidValue;
            sms_dev[dev] = n;
            per_sm_dev[dev] = ps > 1 ? 1 : (ps < 1 ? -1 : ps);  // one block holds all 512 tensor-memory columns
        }
        const int per_sm = per_sm_dev[dev], sms = sms_dev[dev];
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        const int64_t ntiles = (a.npencils + TC_P - 1) / TC_P;
        const int64_t blocks = std::min<int64_t>(ntiles, (int64_t)per_sm * sms);
        tc_contig512_kernel<S><<<(unsigned)blocks, TC_THREADS, TC_SMEM, st>>>(map, (S *)out, a);
        return cudaGetLastError();
    }
}

}  // namespace

cudaError_t WSFFT_LAUNCH_NAME(int kind, int N, int E, int tile, bool variant, const void *in,
                              void *out, const PassArgs &a, cudaStream_t st) {
    using S = WSFFT_STORE;
    if (tile == TC_TILE) {
        if (variant || kind != PASS_CONTIG) return cudaErrorInvalidValue;
        return launch_tc_contig<S>(N, in, out, a, st);
    }
    if (tile > 0) {
        if (variant) return launch_extra_variant<S>(kind, N, E, tile, in, out, a, st);
        return launch_extra<S>(kind, N, E, tile, in, out, a, st);
    }
#define WSFFT_CASE(n)                                                              \
    case n:                                                                        \
        if (E == default_E(n)) return launch_n<n, default_E(n), S>(kind, variant, in, out, a, st); \
        break;
    switch (N) {
        WSFFT_CASE(1)
        WSFFT_CASE(2)
        WSFFT_CASE(4)
        WSFFT_CASE(8)
        WSFFT_CASE(16)
        WSFFT_CASE(32)
        WSFFT_CASE(64)
        WSFFT_CASE(128)
        WSFFT_CASE(256)
        WSFFT_CASE(512)
        WSFFT_CASE(1024)
        WSFFT_CASE(2048)
        WSFFT_CASE(4096)
        default:
            break;
    }
#undef WSFFT_CASE
    return cudaErrorInvalidValue;
}

}  // namespace wsfft
