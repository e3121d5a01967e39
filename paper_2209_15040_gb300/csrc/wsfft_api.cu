// C ABI of the library (include/wsfft.h): plan construction, twiddle tables,
// pass schedule and launch sequencing.
//
// Schedule (Section 1: one superstep per axis, in any order; Section 4.2:
// the 3D sequence z, then the other axes):
//   rank 2/3: superstep along the contiguous axis (in -> out), then one
//             superstep per remaining axis, last axis first (out -> out,
//             each kernel reading and writing the same tile).
//   rank 1, n <= 4096: one contiguous superstep.
//   rank 1, n > 4096: the long axis is split as a 2D problem n = n1*n2
//             (Section 8 proposes decomposing large 1D transforms as a
//             higher-dimensional FFT): a strided superstep of length n2 with
//             the inter-step twiddles w_n^(j1*k2) applied on store (in ->
//             workspace), then a contiguous superstep of length n1 whose
//             store transposes into natural order (workspace -> out).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "../../include/wsfft.h"
#include "fft_core.cuh"
#include "host_roots.h"
#include "pass_desc.h"
#include "pass_kernels.cuh"
#include "engine.cuh"
#include "engine_desc.h"
#include "plan_internal.h"
#include "ragged.cuh"
#include "ragged_desc.h"
#include "slab_cluster.cuh"
#include "slab_desc.h"

namespace wsfft {

float2 host_root(int64_t m, int64_t n) {
    m %= n;
    if (m < 0) m += n;
    const int64_t o = (8 * m) / n;      // octant
    const int64_t rho = 8 * m - o * n;  // position inside the octant, [0, n)
    const long double q = 0.78539816339744830961566084581987572L;  // pi/4
    long double c, s;
    if ((o & 1) == 0) {
        const long double phi = q * (long double)rho / (long double)n;
        const long double cp = cosl(phi), sp = sinl(phi);
        switch (o) {
            case 0: c = cp; s = sp; break;
            case 2: c = -sp; s = cp; break;
            case 4: c = -cp; s = -sp; break;
            default: c = sp; s = -cp; break;  // 6
        }
    } else {
        const long double phi = q * (long double)(n - rho) / (long double)n;
        const long double cp = cosl(phi), sp = sinl(phi);
        switch (o) {
            case 1: c = sp; s = cp; break;
            case 3: c = -cp; s = sp; break;
            case 5: c = -sp; s = -cp; break;
            default: c = cp; s = -sp; break;  // 7
        }
    }
    return make_float2((float)c, (float)-s);
}

int fill_stage_table(float2 *dst, int cap, int N, int E) {
    const int size = sched_tw_size(N, E);
    if (size + 1 > cap) return -1;
    const int ns = sched_nstages(N, E);
    for (int s = 1; s < ns; ++s) {
        const int R = sched_radix(N, E, s), Ns = sched_ns_before(N, E, s);
        const int off = sched_tw_offset(N, E, s);
        for (int r = 1; r < R; ++r)
            for (int k = 0; k < Ns; ++k) dst[off + (r - 1) * Ns + k] = host_root((int64_t)r * k, (int64_t)Ns * R);
    }
    dst[size] = make_float2(0.f, 0.f);
    return size + 1;
}

}  // namespace wsfft

using namespace wsfft;

namespace {

bool is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

int ilog2(int64_t n) {
    int l = 0;
    while (((int64_t)1 << l) < n) ++l;
    return l;
}

int64_t elem_bytes(int dtype) { return dtype == WSFFT_C32 ? 8 : 4; }

std::vector<float2> stage_table(int N, int E) {
    std::vector<float2> t((size_t)sched_tw_size(N, E) + 1);
    fill_stage_table(t.data(), (int)t.size(), N, E);
    return t;
}

// Table of the tensor-core contiguous superstep at N = 512 (layout in
// tc_contig.cuh): the DFT-16 matrix B[n = 2*k1 + part][k = n1] = (Re, Im)
// w16^(n1*k1) as 16-bit high parts and 16-bit remainders in the K-major
// core-matrix byte order, then the inter-stage twiddles w512^(k1*n2).
std::vector<float2> tc_table_host(int dtype) {
    std::vector<float2> t(TC_TABLE_FLOAT2);
    uint16_t *hi = reinterpret_cast<uint16_t *>(t.data());
    uint16_t *lo = hi + 512;
    for (int n = 0; n < 32; ++n)
        for (int k = 0; k < 16; ++k) {
            const int k1 = n / 2, part = n % 2, n1 = k;
            const float2 w = host_root((int64_t)n1 * k1, 16);
            const float v = part ? w.y : w.x;
            uint16_t h, l;
            if (dtype == WSFFT_C16BF) {
                const __nv_bfloat16 hb = __float2bfloat16_rn(v);
                h = __bfloat16_as_ushort(hb);
                l = __bfloat16_as_ushort(__float2bfloat16_rn(v - __bfloat162float(hb)));
            } else {
                const __half hh = __float2half_rn(v);
                h = __half_as_ushort(hh);
                l = __half_as_ushort(__float2half_rn(v - __half2float(hh)));
            }
            const int off = (n / 8) * 256 + (k / 8) * 128 + (n % 8) * 16 + (k % 8) * 2;  // bytes
            hi[off / 2] = h;
            lo[off / 2] = l;
        }
    for (int n2 = 0; n2 < 32; ++n2)
        for (int k1 = 0; k1 < 16; ++k1) t[TC_TABLE_TW + n2 * 16 + k1] = host_root((int64_t)k1 * n2, 512);
    return t;
}

float axis_scale(int64_t n, int dir, int norm) {
    if (norm == WSFFT_NORM_PAPER) return dir == WSFFT_INVERSE ? (float)(1.0 / (double)n) : 1.f;
    if (norm == WSFFT_NORM_ORTHO) return (float)(1.0 / std::sqrt((double)n));
    if (norm == WSFFT_NORM_FORWARD) return dir == WSFFT_FORWARD ? (float)(1.0 / (double)n) : 1.f;
    return 1.f;
}

cudaError_t launch_engine(int dtype, int n, const EngArgs &a, int grid, cudaStream_t st) {
    switch (dtype) {
        case WSFFT_C32: return launch_engine_c32(n, a, grid, st);
        case WSFFT_C16F: return launch_engine_c16f(n, a, grid, st);
        default: return launch_engine_c16bf(n, a, grid, st);
    }
}

cudaError_t launch_persist(int dtype, int n, const EngArgs &a, int s_mode, int *per_sm, int grid,
                           cudaStream_t st) {
    switch (dtype) {
        case WSFFT_C32: return launch_persist_c32(n, a, s_mode, per_sm, grid, st);
        case WSFFT_C16F: return launch_persist_c16f(n, a, s_mode, per_sm, grid, st);
        default: return launch_persist_c16bf(n, a, s_mode, per_sm, grid, st);
    }
}

cudaError_t launch_wpp(int dtype, int n, const EngArgs &a, int *per_sm, int grid, cudaStream_t st) {
    switch (dtype) {
        case WSFFT_C32: return launch_wpp_c32(n, a, per_sm, grid, st);
        case WSFFT_C16F: return launch_wpp_c16f(n, a, per_sm, grid, st);
        default: return launch_wpp_c16bf(n, a, per_sm, grid, st);
    }
}

cudaError_t launch_wps(int dtype, int n, const WpStridedArgs &b, cudaStream_t st) {
    switch (dtype) {
        case WSFFT_C32: return launch_wps_c32(n, b, st);
        case WSFFT_C16F: return launch_wps_c16f(n, b, st);
        default: return launch_wps_c16bf(n, b, st);
    }
}

cudaError_t launch_slab(int dtype, int n, const void *in, void *out, int64_t nslabs, const SlabArgs &a, bool pdl,
                        cudaStream_t st, int *max_clusters) {
    switch (dtype) {
        case WSFFT_C32: return launch_slab_c32(n, in, out, nslabs, a, pdl, st, max_clusters);
        case WSFFT_C16F: return launch_slab_c16f(n, in, out, nslabs, a, pdl, st, max_clusters);
        default: return launch_slab_c16bf(n, in, out, nslabs, a, pdl, st, max_clusters);
    }
}

cudaError_t launch(int dtype, const PassSpec &p, const void *in, void *out, const PassArgs &a,
                   cudaStream_t st) {
    switch (dtype) {
        case WSFFT_C32: return launch_pass_c32(p.kind, p.N, p.E, p.tile, p.variant, in, out, a, st);
        case WSFFT_C16F: return launch_pass_c16f(p.kind, p.N, p.E, p.tile, p.variant, in, out, a, st);
        default: return launch_pass_c16bf(p.kind, p.N, p.E, p.tile, p.variant, in, out, a, st);
    }
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? WSFFT_SUCCESS : WSFFT_ERR_CUDA; }

// a pass-shape override the schedule builder may apply: a power-of-two count
// of values per thread within the pencil (the builder makes twiddle tables for
// it) and a non-negative tile code; whether a kernel of that shape exists is
// checked separately (Plan::overrides_launchable)
bool override_usable(int E, int tile, int N) {
    return E >= 1 && E <= 32 && E <= N && (E & (E - 1)) == 0 && tile >= 0;
}

// two buffers of `bytes` that share some bytes without being the same buffer
bool partial_overlap(const void *a, const void *b, size_t bytes) {
    const char *x = static_cast<const char *>(a), *y = static_cast<const char *>(b);
    return x != y && x < y + bytes && y < x + bytes;
}

}  // namespace

namespace wsfft {

const float2 *Plan::tc_table(int N) {
    if (N != 512 || dtype == WSFFT_C32) return nullptr;
    auto key = std::make_pair(N, TC_TILE);
    auto it = tables.find(key);
    if (it != tables.end()) return it->second;
    std::vector<float2> h = tc_table_host(dtype);
    float2 *d = nullptr;
    if (cudaMalloc(&d, h.size() * sizeof(float2)) != cudaSuccess) return nullptr;
    if (upload(d, h.data(), h.size() * sizeof(float2)) != WSFFT_SUCCESS) {
        cudaFree(d);
        return nullptr;
    }
    tables[key] = d;
    return d;
}

// Four-step inter-superstep twiddles w_L^m, m < L, as two tables: the high
// part w_L^(i << shift) for i < L >> shift, then the low part w_L^j for
// j < 2^shift (w_L^m is their product; both from host_root).
const float2 *Plan::fourstep_table(int64_t L, int shift) {
    auto it = fs_tables.find(L);
    if (it != fs_tables.end()) return it->second;
    const int64_t nh = L >> shift, nl = (int64_t)1 << shift;
    std::vector<float2> h((size_t)(nh + nl));
    for (int64_t i = 0; i < nh; ++i) h[(size_t)i] = host_root(i << shift, L);
    for (int64_t j = 0; j < nl; ++j) h[(size_t)(nh + j)] = host_root(j, L);
    float2 *d = nullptr;
    if (cudaMalloc(&d, h.size() * sizeof(float2)) != cudaSuccess) return nullptr;
    if (upload(d, h.data(), h.size() * sizeof(float2)) != WSFFT_SUCCESS) {
        cudaFree(d);
        return nullptr;
    }
    fs_tables[L] = d;
    return d;
}

const float2 *Plan::table(int N, int E) {
    auto key = std::make_pair(N, E);
    auto it = tables.find(key);
    if (it != tables.end()) return it->second;
    std::vector<float2> h = stage_table(N, E);
    float2 *d = nullptr;
    if (cudaMalloc(&d, h.size() * sizeof(float2)) != cudaSuccess) return nullptr;
    if (upload(d, h.data(), h.size() * sizeof(float2)) != WSFFT_SUCCESS) {
        cudaFree(d);
        return nullptr;
    }
    tables[key] = d;
    return d;
}

// Two-launch schedule of an n^3 cube on the persistent engine.
// Pass A: per slab (fixed first index), the contiguous superstep (z) then the
// strided superstep along the middle axis (y), queued `lag` slabs apart so
// the slab is still in L2 when it is read again.  Pass B: the superstep along
// the first axis (x).
int Plan::build_engine(int64_t n0, int64_t n, bool inv) {
    int grid = eng_grid;
    if (engine_mode == 1 || engine_mode == 3) {
        int per_sm = 0;
        EngArgs dummy{};
        cudaError_t e = engine_mode == 1 ? launch_persist(dtype, (int)n, dummy, 0, &per_sm, 0, 0)
                                         : launch_wpp(dtype, (int)n, dummy, &per_sm, 0, 0);
        if (e != cudaSuccess || per_sm < 1) return WSFFT_ERR_UNSUPPORTED;
        persist_grid = per_sm * sm_count;
        grid = persist_grid;
    }
    // pencils per contiguous tile (tp) and per strided tile (tq)
    int64_t tp, tq;
    if (engine_mode == 3) {
        tp = wp_tile_z((int)n);
        tq = wp_tile_y((int)n);
    } else if (engine_mode == 1 && n == 512) {
        tp = persist512_tile_z();  // contiguous tiles: one warp per pencil
        tq = 16;                   // strided tiles: 16 pencils
    } else {
        tp = engine_tile_pencils((int)n);
        tq = tp;
    }
    const int64_t sub = engine_mode == 1 ? persist_sub((int)n) : 1;  // tiles per queue item
    const int64_t zper = n / tp / sub, yper = n / tq / sub;  // queue items per slab of each kind
    const int64_t U = batch * n0;                     // slabs
    if (U * (zper + yper) > (int64_t)1 << 30) return WSFFT_ERR_UNSUPPORTED;
    const int64_t window = engine_mode == 2 ? 3 * (int64_t)grid : 2 * (int64_t)grid;  // tiles held
    int64_t lag = (window + zper + yper - 1) / (zper + yper) + 2;  // measured: deeper lags do not help
    if (lag > U) lag = U;
    std::vector<EngItem> items;
    items.reserve((size_t)(U * (zper + yper) + batch * n * n / tq));
    for (int64_t j = 0; j < U + lag; ++j) {
        if (j < U)
            for (int64_t t = 0; t < zper; ++t)
                items.push_back(EngItem{ITEM_SIGNAL, (int)j, (int)t, 0});
        if (j >= lag)
            for (int64_t t = 0; t < yper; ++t)
                items.push_back(EngItem{ITEM_STRIDED | ITEM_WAIT, (int)(j - lag), (int)t, 0});
    }
    if (withhold) items[0].flags &= ~ITEM_SIGNAL;
    const int na = (int)items.size();
    if (engine_mode == 2)  // pipelined engine: x tiles too (cubes only, n0 == n)
        for (int64_t b = 0; b < batch; ++b)
            for (int64_t t = 0; t < n * n / tq; ++t) items.push_back(EngItem{ITEM_STRIDED, (int)b, (int)t, 0});
    const int nb = (int)items.size() - na;
    if (d_items) cudaFree(d_items);
    d_items = nullptr;
    if (cudaMalloc(&d_items, items.size() * sizeof(EngItem)) != cudaSuccess) {
        d_items = nullptr;
        return WSFFT_ERR_ALLOC;
    }
    if (upload(d_items, items.data(), items.size() * sizeof(EngItem)) != WSFFT_SUCCESS) return WSFFT_ERR_CUDA;
    if (1 + U > ctr_cap) {
        if (d_ctr) cudaFree(d_ctr);
        d_ctr = nullptr;
        ctr_cap = 0;
        if (cudaMalloc(&d_ctr, (size_t)(1 + U) * sizeof(uint32_t)) != cudaSuccess) {
            d_ctr = nullptr;
            return WSFFT_ERR_ALLOC;
        }
        ctr_cap = 1 + U;
    }
    const float sc = axis_scale(n, dir, norm), sc0 = axis_scale(n0, dir, norm);
    PassSpec a{};
    a.kind = engine_mode == 1 ? PASS_PERSIST_A : engine_mode == 3 ? PASS_WP_A : PASS_ENGINE_A;
    a.N = (int)n;
    a.E = 16;
    a.tile = (int)tp;
    a.trans_rows = zper;  // completion target of a slab
    a.items = d_items;
    a.nitems = na;
    a.units = U;
    a.conj_in = inv;
    a.c_scale = sc;
    a.s_scale = sc;
    a.transform_elems = n0 * n * n;
    PassSpec b{};
    if (engine_mode == 3 && wp_supports((int)n0)) {
        b.kind = PASS_WP_B;
        b.N = (int)n0;
        b.E = 16;
        b.inner = n * n;
        b.npencils_per_batch = n * n;
        b.src = SRC_OUT;
        b.dst = DST_OUT;
    } else if (engine_mode == 2) {
        b.kind = PASS_ENGINE_B;
        b.N = (int)n;
        b.E = 16;
        b.items = (const EngItem *)d_items + na;
        b.nitems = nb;
        b.units = 0;
    } else {
        // x: one launch of the strided superstep kernel, with the shape of
        // the one-launch-per-superstep schedule at 512 (16 pencils per block:
        // 32 values per thread in complex64, split-form pencil pairs in the
        // 16-bit types)
        b.kind = PASS_STRIDED;
        b.N = (int)n0;
        b.E = n0 == 512 ? (dtype == WSFFT_C32 ? 32 : 16) : default_E((int)n0);
        b.tile = n0 == 512 ? (dtype == WSFFT_C32 ? 16 : SPLIT_TILE + 16) : 0;
        b.inner = n * n;
        b.npencils_per_batch = n * n;
        b.src = SRC_OUT;
        b.dst = DST_OUT;
    }
    b.conj_out = inv;
    b.scale = engine_mode == 2 ? sc : sc0;
    b.transform_elems = n0 * n * n;
    passes.push_back(a);
    passes.push_back(b);
    for (auto &kv : overrides) {
        if (kv.first < (int)passes.size() && passes[kv.first].kind == PASS_STRIDED &&
            override_usable(kv.second.first, kv.second.second, passes[kv.first].N)) {
            passes[kv.first].E = kv.second.first;
            passes[kv.first].tile = kv.second.second;
        }
    }
    for (auto &p : passes) {
        p.tw = table(p.N, p.E);
        if (!p.tw) return WSFFT_ERR_ALLOC;
    }
    if (engine_mode == 1 && n == 512) {
        // the persistent 512 kernel's strided tiles have their own values per thread
        passes[0].tw2 = table(512, persist512_values_y());
        if (!passes[0].tw2) return WSFFT_ERR_ALLOC;
    }
    return WSFFT_SUCCESS;
}

// Whether the cluster-fused pass A of slab edge n can be resident on this
// plan's device (asked once per edge).
bool Plan::slab_runs(int n) {
    if (!slab_supports(n)) return false;
    int &c = slab_checked[n == 512 ? 1 : 0];
    if (c == 0) {
        SlabArgs probe{};
        int clusters = 0;
        const cudaError_t e = launch_slab(dtype, n, nullptr, nullptr, 1, probe, false, 0, &clusters);
        cudaGetLastError();  // a refused query leaves no sticky error
        c = (e == cudaSuccess && clusters > 0) ? 1 : -1;
    }
    return c > 0;
}

// Two-trip schedule of an n0 x n x n transform with the cluster-fused pass A
// (slab_cluster.cuh): the z and y supersteps of each n x n slab in one
// thread-block cluster (in -> out), then the x superstep as one launch of the
// strided kernel (out, in place).
int Plan::build_slab(int64_t n0, int64_t n, bool inv) {
    PassSpec a{};
    a.kind = PASS_SLAB_A;
    a.N = (int)n;
    a.inner = 1;
    a.npencils_per_batch = n0 * n;  // z pencils per transform
    a.units = n0;                   // slabs per transform
    a.transform_elems = n0 * n * n;
    a.src = SRC_IN;
    a.dst = DST_OUT;
    a.conj_in = inv;
    PassSpec b{};
    b.kind = PASS_STRIDED;
    b.N = (int)n0;
    b.E = default_E((int)n0);
    b.tile = 0;
    if (n0 == 512) {
        // the shape of the x superstep in the one-launch-per-superstep
        // schedule: 32 values per thread in complex64, split-form pencil
        // pairs in the 16-bit types
        b.E = dtype == WSFFT_C32 ? 32 : 16;
        b.tile = dtype == WSFFT_C32 ? 16 : SPLIT_TILE + 16;
    } else if (n0 == 1024) {
        b.E = 32;
        b.tile = 16;
    }
    b.inner = n * n;
    b.npencils_per_batch = n * n;
    b.transform_elems = n0 * n * n;
    b.src = SRC_OUT;
    b.dst = DST_OUT;
    b.conj_out = inv;
    const float sc = axis_scale(n, dir, norm), sc0 = axis_scale(n0, dir, norm);
    if (dtype == WSFFT_C32 && norm != WSFFT_NORM_ORTHO) {
        // complex64 defers every superstep's scale to the last store
        a.c_scale = a.s_scale = 1.f;
        b.scale = (float)((double)sc * (double)sc * (double)sc0);
    } else {
        a.c_scale = a.s_scale = sc;
        b.scale = sc0;
    }
    passes.push_back(a);
    passes.push_back(b);
    for (auto &kv : overrides)
        if (kv.first == 1 && override_usable(kv.second.first, kv.second.second, passes[1].N)) {
            passes[1].E = kv.second.first;
            passes[1].tile = kv.second.second;
        }
    passes[0].E = slab_ez(dtype != WSFFT_C32);
    passes[0].tw = table((int)n, passes[0].E);
    passes[0].tw2 = table((int)n, slab_ey());
    passes[1].tw = table(passes[1].N, passes[1].E);
    if (!passes[0].tw || !passes[0].tw2 || !passes[1].tw) return WSFFT_ERR_ALLOC;
    return WSFFT_SUCCESS;
}

// (Re)build the pass list from shape, direction and normalisation.
int Plan::build_schedule() {
    passes.clear();
    std::vector<int64_t> d;
    for (int i = 0; i < rank; ++i)
        if (dims[i] > 1) d.push_back(dims[i]);
    if (d.empty()) d.push_back(1);
    const int r = (int)d.size();
    const bool inv = dir == WSFFT_INVERSE;
    work_elems = 0;
    chunk = batch;

    // kernel shapes of a one-launch contiguous or strided superstep
    auto tune = [&](PassSpec &p, int64_t inner) {
        if (p.kind == PASS_CONTIG && p.N == 512) {
            // measured fastest at 512^3: 16 values per thread (radices
            // 16, 16, 2), 8 pencils per block (32 values per thread
            // matched it forward but lost 30% with the conjugate on load
            // of the inverse); complex64 one pencil per warp (256-thread
            // blocks, at the copy bandwidth), the 16-bit types as
            // split-form pairs (one pair per warp, packed FP32x2
            // butterflies: 13% faster there, the same in complex64)
            p.E = 16;
            p.tile = dtype == WSFFT_C32 ? 8 : SPLIT_TILE + 8;
        }
        if (p.N == 1024) {
            // measured at 1024^3: 32 values per thread (radix 32 x 32, one
            // exchange); contiguous: one warp per pencil, 8 per block;
            // strided: 16 pencils per block at strides of 2^17 elements
            // and more (128-byte rows: narrower tiles lost 10-50% there),
            // below that split-form pencil pairs with 16 values per pencil
            // and 8 pencils per block (two blocks per SM: 0.404 vs 0.427 ms
            // for 32 values per thread on a 1 GiB array at stride 1024)
            p.E = 32;
            p.tile = 8;
            if (p.kind == PASS_STRIDED) {
                if (inner >= ((int64_t)1 << 17)) {
                    p.tile = 16;
                } else if (inner % 8 == 0) {
                    p.E = 16;
                    p.tile = SPLIT_TILE + 8;
                } else if (dtype != WSFFT_C32) {
                    p.E = 16;
                }
            }
        }
        if (p.kind == PASS_STRIDED && p.N == 512 && inner % 16 == 0) {
            // measured fastest at 512^3: split-form pencil pairs (packed
            // FP32x2 butterflies, two adjacent elements per access), 16
            // values per pencil, 16 pencils per block, except for complex64
            // at strides of 2^17 elements and more, where 32 values per
            // thread for one pencil (one shared-memory exchange) match them
            p.E = 16;
            p.tile = SPLIT_TILE + 16;
            if (dtype == WSFFT_C32 && inner >= ((int64_t)1 << 17)) {
                p.E = 32;
                p.tile = 16;
            }
        }
    };

    // cluster-fused pass A (the default): the two inner axes equal and built
    // for that edge, and the kernel resident on this device
    if (layout == WSFFT_LAYOUT_NATURAL && r == 3 && engine_mode == 4 && d[1] == d[2] && slab_runs((int)d[1]))
        return build_slab(d[0], d[1], inv);
    // fused schedules: the two inner axes equal (n x n slabs); the pipelined
    // engine also runs the outer axis, so it needs a cube
    if (layout == WSFFT_LAYOUT_NATURAL && r == 3 && engine_mode >= 1 && engine_mode <= 3 && d[1] == d[2] &&
        engine_supports((int)d[1]) &&
        (engine_mode != 2 || d[0] == d[1]) && (engine_mode != 3 || wp_supports((int)d[1])) &&
        eng_grid > 0) {
        return build_engine(d[0], d[1], inv);
    }
    if (axis_inner > 0) {
        // wsfft_plan_create_axis: one superstep along an axis of length
        // dims[0] whose consecutive elements are axis_inner apart; pencils
        // (b, i) for batch index b and i < axis_inner
        PassSpec p{};
        p.N = (int)dims[0];
        p.kind = axis_inner == 1 ? PASS_CONTIG : PASS_STRIDED;
        p.E = default_E(p.N);
        tune(p, axis_inner);
        p.inner = axis_inner;
        p.npencils_per_batch = axis_inner;
        p.transform_elems = dims[0] * axis_inner;
        p.src = SRC_IN;
        p.dst = DST_OUT;
        p.conj_in = inv;
        p.conj_out = inv;
        p.scale = axis_scale(dims[0], dir, norm);
        passes.push_back(p);
    } else if (layout == WSFFT_LAYOUT_WAFER) {
        // Spectral side in the wafer's own order [n2][n0][n1] (Section 4.2:
        // after z is transformed, x and z swap places, then x and y; with the
        // PEs numbered like the input, X[k0][k1][k2] ends at k2 * n0 * n1 +
        // k0 * n1 + k1).  Built from the transposing store (pencil (t, row)
        // element k to t*N*rows + k*rows + row), three trips as in natural
        // order:
        //   forward:  z with the transposed store, rows n0*n1 (in -> work):
        //             [n0][n1][n2] -> [n2][n0][n1]; y contiguous (work ->
        //             out); x strided with stride n1 (out, in place)
        //   inverse:  y with the transposed store, rows n2*n0 (in -> work):
        //             [n2][n0][n1] -> [n1][n2][n0]; x with the transposed
        //             store, rows n1*n2 (work -> out): -> [n0][n1][n2]; z
        //             contiguous (out, in place)
        const int64_t n0 = dims[0], n1 = dims[1], n2 = dims[2];
        const int64_t total = n0 * n1 * n2;
        const int64_t per = total * elem_bytes(dtype);
        chunk = std::max<int64_t>(1, std::min<int64_t>(batch, ((int64_t)4096 << 20) / per));
        work_elems = chunk * total;
        auto trans = [&](int64_t n, int64_t rows, int src, int dst) {
            PassSpec t{};
            t.kind = PASS_CONTIG;
            t.N = (int)n;
            t.E = default_E(t.N);
            if (t.N == 1024 && dtype == WSFFT_C32) {
                t.E = 32;  // as in the four-step: one warp per pencil, 8 per block
                t.tile = 8;
            } else if (t.N == 512) {
                t.E = 32;  // half a warp per pencil, 16 per block (as in the swapped layout)
                t.tile = 16;
            }
            t.variant = true;
            t.inner = 1;
            t.npencils_per_batch = rows;
            t.trans_rows = rows;
            t.src = src;
            t.dst = dst;
            t.scale = axis_scale(n, dir, norm);
            t.transform_elems = total;
            return t;
        };
        if (!inv) {
            passes.push_back(trans(n2, n0 * n1, SRC_IN, DST_WORK));
            PassSpec c{};
            c.kind = PASS_CONTIG;
            c.N = (int)n1;
            c.E = default_E(c.N);
            tune(c, 1);
            c.inner = 1;
            c.npencils_per_batch = n2 * n0;
            c.src = SRC_WORK;
            c.dst = DST_OUT;
            c.scale = axis_scale(n1, dir, norm);
            c.transform_elems = total;
            passes.push_back(c);
            PassSpec a{};
            a.kind = PASS_STRIDED;
            a.N = (int)n0;
            a.E = default_E(a.N);
            tune(a, n1);
            a.inner = n1;
            a.npencils_per_batch = n2 * n1;
            a.src = SRC_OUT;
            a.dst = DST_OUT;
            a.scale = axis_scale(n0, dir, norm);
            a.transform_elems = total;
            passes.push_back(a);
        } else {
            passes.push_back(trans(n1, n2 * n0, SRC_IN, DST_WORK));
            passes.push_back(trans(n0, n1 * n2, SRC_WORK, DST_OUT));
            PassSpec c{};
            c.kind = PASS_CONTIG;
            c.N = (int)n2;
            c.E = default_E(c.N);
            tune(c, 1);
            c.inner = 1;
            c.npencils_per_batch = n0 * n1;
            c.src = SRC_OUT;
            c.dst = DST_OUT;
            c.scale = axis_scale(n2, dir, norm);
            c.transform_elems = total;
            passes.push_back(c);
        }
        passes.front().conj_in = inv;
        passes.back().conj_out = inv;
        if (dtype == WSFFT_C32 && norm != WSFFT_NORM_ORTHO) {
            double total_scale = 1.0;
            for (auto &q : passes) {
                total_scale *= q.scale;
                q.scale = 1.f;
            }
            passes.back().scale = (float)total_scale;
        }
    } else if (layout == WSFFT_LAYOUT_SWAPPED) {
        // Spectral side with the last two axes swapped (the wafer's order,
        // Section 4.2).  The superstep along the last axis of the natural
        // side stores its pencils transposed (the four-step's staged store:
        // pencil (plane, row) element k to plane*N*rows + k*rows + row) into
        // the workspace, which turns the natural [a][b][c] into [a][c][b] or
        // back; the next axis is then contiguous on both sides of the swap,
        // and the first axis of a rank-3 array keeps its stride.
        //   forward:  c with the transposed store (in -> work), b contiguous
        //             (work -> out), a strided (out, in place)
        //   inverse:  b with the transposed store (in -> work), c contiguous
        //             (work -> out), a strided (out, in place)
        const int64_t A = rank == 3 ? dims[0] : 1, B = dims[rank - 2], C = dims[rank - 1];
        const int64_t total = A * B * C;
        const int64_t per = total * elem_bytes(dtype);
        chunk = std::max<int64_t>(1, std::min<int64_t>(batch, ((int64_t)4096 << 20) / per));
        work_elems = chunk * total;
        const int64_t n_t = inv ? B : C;  // axis of the transposing superstep
        const int64_t n_c = inv ? C : B;  // the other of the last two axes
        PassSpec t{};
        t.kind = PASS_CONTIG;
        t.N = (int)n_t;
        t.E = default_E(t.N);
        if (t.N == 1024 && dtype == WSFFT_C32) {
            t.E = 32;  // as in the four-step: one warp per pencil, 8 per block
            t.tile = 8;
        } else if (t.N == 512) {
            // 32 values per thread, 16 pencils per block: 0.33 against 0.39 ms
            // per GiB for the default 8 values x 16 pencils in complex64, 0.30
            // against 0.45 ms per 512 MiB in the 16-bit types (two resident
            // blocks of 256 threads against one of 1024)
            t.E = 32;
            t.tile = 16;
        }
        t.variant = true;
        t.inner = 1;
        t.npencils_per_batch = A * n_c;
        t.trans_rows = n_c;
        t.src = SRC_IN;
        t.dst = DST_WORK;
        t.conj_in = inv;
        t.scale = axis_scale(n_t, dir, norm);
        t.transform_elems = total;
        PassSpec c{};
        c.kind = PASS_CONTIG;
        c.N = (int)n_c;
        c.E = default_E(c.N);
        tune(c, 1);
        c.inner = 1;
        c.npencils_per_batch = A * n_t;
        c.src = SRC_WORK;
        c.dst = DST_OUT;
        c.scale = axis_scale(n_c, dir, norm);
        c.transform_elems = total;
        passes.push_back(t);
        passes.push_back(c);
        if (A > 1) {
            PassSpec a{};
            a.kind = PASS_STRIDED;
            a.N = (int)A;
            a.E = default_E(a.N);
            tune(a, B * C);
            a.inner = B * C;
            a.npencils_per_batch = B * C;
            a.src = SRC_OUT;
            a.dst = DST_OUT;
            a.scale = axis_scale(A, dir, norm);
            a.transform_elems = total;
            passes.push_back(a);
        }
        passes.back().conj_out = inv;
        if (dtype == WSFFT_C32 && norm != WSFFT_NORM_ORTHO) {
            double total_scale = 1.0;
            for (auto &q : passes) {
                total_scale *= q.scale;
                q.scale = 1.f;
            }
            passes.back().scale = (float)total_scale;
        }
    } else if (r == 1 && d[0] > 4096) {
        const int64_t n = d[0];
        const int lg = ilog2(n);
        // complex64 at n = 2^20 splits 2048 (contiguous) x 512 (strided)
        // rather than 1024 x 1024: the 512-point strided superstep with the
        // inter-step twiddle runs at 1.61 ms per 512 x 2^20 execute against
        // 2.11 ms for the 1024-point one, the 2048-point contiguous superstep
        // costs 1.97 against 1.81 ms (3.57 vs 3.91 ms per execute)
        const int lg1 = (lg == 20 && dtype == WSFFT_C32) ? 11 : (lg + 1) / 2;
        const int64_t n1 = (int64_t)1 << lg1;  // contiguous length
        const int64_t n2 = n / n1;             // strided length
        const float sc = axis_scale(n, dir, norm);
        // workspace holds `chunk` transforms (at most ~4 GiB: measured 5%
        // faster than 512 MiB chunks at 512 x 2^20, fewer launch tails;
        // chunks small enough to stay in L2 were slower still)
        const int64_t per = n * elem_bytes(dtype);
        chunk = std::max<int64_t>(1, std::min<int64_t>(batch, ((int64_t)4096 << 20) / per));
        work_elems = chunk * n;
        PassSpec a{};
        a.kind = PASS_STRIDED;
        a.N = (int)n2;
        a.E = default_E((int)n2);
        if ((n2 == 1024 || n2 == 512) && dtype == WSFFT_C32) {
            // measured fastest at n = 2^20: 32 values per thread, 16 pencils per block
            a.E = 32;
            a.tile = 16;
        }
        a.variant = true;
        a.inner = n1;
        a.npencils_per_batch = n1;
        a.src = SRC_IN;
        a.dst = DST_WORK;
        a.conj_in = inv;
        a.conj_out = false;
        a.scale = 1.f;
        a.twid_len = n;
        a.twid_shift = (lg + 1) / 2;
        a.transform_elems = n;
        PassSpec b{};
        b.kind = PASS_CONTIG;
        b.N = (int)n1;
        b.E = default_E((int)n1);
        if (n1 == 1024 && dtype == WSFFT_C32) {
            // one warp per pencil (32 values per thread), 8 pencils per block
            b.E = 32;
            b.tile = 8;
        } else if (n1 == 512) {
            // half a warp per pencil, 16 pencils per block (as in the swapped layout)
            b.E = 32;
            b.tile = 16;
        }
        b.variant = true;
        b.inner = 1;
        b.npencils_per_batch = n2;
        b.src = SRC_WORK;
        b.dst = DST_OUT;
        b.conj_in = false;
        b.conj_out = inv;
        b.scale = sc;
        b.trans_rows = n2;
        b.transform_elems = n;
        passes.push_back(a);
        passes.push_back(b);
    } else {
        int64_t total = 1;
        for (auto v : d) total *= v;
        for (int ax = r - 1; ax >= 0; --ax) {
            int64_t inner = 1;
            for (int e = ax + 1; e < r; ++e) inner *= d[e];
            PassSpec p{};
            p.kind = ax == r - 1 ? PASS_CONTIG : PASS_STRIDED;
            p.N = (int)d[ax];
            p.E = default_E(p.N);
            p.variant = false;
            tune(p, inner);
            p.inner = inner;
            p.npencils_per_batch = total / d[ax];
            p.src = ax == r - 1 ? SRC_IN : SRC_OUT;
            p.dst = DST_OUT;
            p.conj_in = inv && ax == r - 1;
            p.conj_out = inv && ax == 0;
            p.scale = axis_scale(d[ax], dir, norm);
            p.transform_elems = total;
            passes.push_back(p);
        }
        if (dtype == WSFFT_C32 && norm != WSFFT_NORM_ORTHO) {
            // complex64 has the range to defer every superstep's 1/n to the
            // last pass (one scaled store instead of one per pass); the
            // reduced-precision types keep the per-superstep scale
            double total_scale = 1.0;
            for (auto &p : passes) {
                total_scale *= p.scale;
                p.scale = 1.f;
            }
            passes.back().scale = (float)total_scale;
        }
    }
    for (auto &kv : overrides) {
        if (kv.first < (int)passes.size() &&
            (passes[kv.first].kind == PASS_CONTIG || passes[kv.first].kind == PASS_STRIDED) &&
            override_usable(kv.second.first, kv.second.second, passes[kv.first].N)) {
            passes[kv.first].E = kv.second.first;
            passes[kv.first].tile = kv.second.second;
        }
    }
    // A strided superstep right after a contiguous one (the y superstep after
    // z) takes its tiles from the last slab down: the contiguous pass wrote
    // the last slabs last, and the first blocks then find them in L2
    // (measured at 512^3: y 0.330 -> 0.323 ms, 973 -> 967 us per transform)
    for (size_t i = 0; i < passes.size(); ++i)
        passes[i].reverse = i > 0 && passes[i].kind == PASS_STRIDED && passes[i - 1].kind == PASS_CONTIG &&
                            !passes[i].variant && !passes[i - 1].variant;
    for (auto &p : passes) {
        if (p.N > 4096 || !is_pow2(p.N)) return WSFFT_ERR_INVALID_SIZE;
        p.tw = p.tile == TC_TILE ? tc_table(p.N) : table(p.N, p.E);
        if (p.twid_len) {
            p.tw2 = fourstep_table(p.twid_len, p.twid_shift);
            if (!p.tw2) return WSFFT_ERR_ALLOC;
        }
        if (!p.tw) return WSFFT_ERR_ALLOC;
    }
    if (work_elems > work_cap) {
        if (work) cudaFree(work);
        work = nullptr;
        work_cap = 0;
        if (cudaMalloc(&work, (size_t)(work_elems * elem_bytes(dtype))) != cudaSuccess) {
            work = nullptr;
            return WSFFT_ERR_ALLOC;
        }
        work_cap = work_elems;
    }
    return WSFFT_SUCCESS;
}

bool Plan::overrides_launchable() const {
    for (const auto &kv : overrides) {
        if (kv.first < 0 || kv.first >= (int)passes.size()) return false;
        const PassSpec &ps = passes[kv.first];
        if (ps.E != kv.second.first || ps.tile != kv.second.second) return false;  // not applied
        PassArgs a{};
        a.npencils = 0;  // an empty launch returns before running
        if (launch(dtype, ps, nullptr, nullptr, a, 0) == cudaErrorInvalidValue) return false;
    }
    return true;
}

int Plan::run(const void *in, void *out, cudaStream_t st) {
    const int64_t eb = elem_bytes(dtype);
    for (int64_t b0 = 0; b0 < batch; b0 += chunk) {
        const int64_t nb = std::min(chunk, batch - b0);
        for (const auto &p : passes) {
            if (p.kind == PASS_WP_B) {
                WpStridedArgs b{};
                b.in = out;
                b.out = out;
                b.inner = p.inner;
                b.log_inner = ilog2(p.inner);
                b.npencils = p.npencils_per_batch * batch;
                b.tw = p.tw;
                b.ci = 1.f;
                b.sx = p.scale;
                b.sy = p.conj_out ? -p.scale : p.scale;
                prof_begin(st);
                cudaError_t err = launch_wps(dtype, p.N, b, st);
                prof_end(st);
                if (err != cudaSuccess) return err == cudaErrorInvalidValue ? WSFFT_ERR_UNSUPPORTED : WSFFT_ERR_CUDA;
                continue;
            }
            if (p.kind == PASS_SLAB_A) {
                const int64_t off = b0 * p.transform_elems * eb;
                SlabArgs sa{};
                sa.ci = p.conj_in ? -1.f : 1.f;
                sa.zsx = sa.zsy = p.c_scale;
                sa.ysx = sa.ysy = p.s_scale;
                sa.tw_z = p.tw;
                sa.tw_y = p.tw2;
                const int64_t nslabs = p.units * nb;
                const bool pdl = nslabs * (int64_t)p.N * p.N * eb <= ((int64_t)2 << 30);
                prof_begin(st);
                cudaError_t e = launch_slab(dtype, p.N, (const char *)in + off, (char *)out + off, nslabs, sa, pdl,
                                            st, nullptr);
                prof_end(st);
                if (e != cudaSuccess) return e == cudaErrorInvalidValue ? WSFFT_ERR_UNSUPPORTED : WSFFT_ERR_CUDA;
                continue;
            }
            if (p.kind == PASS_ENGINE_A || p.kind == PASS_ENGINE_B || p.kind == PASS_PERSIST_A ||
                p.kind == PASS_WP_A) {
                EngArgs e{};
                e.items = (const EngItem *)p.items;
                e.nitems = p.nitems;
                e.ctr = d_ctr;
                e.status = d_status;
                e.tw_c = p.tw;
                e.tw_s = p.tw2 ? p.tw2 : p.tw;
                e.timeout_ns = (uint64_t)wait_timeout_ns;
                const int64_t n = p.N;
                if (p.kind == PASS_ENGINE_A || p.kind == PASS_PERSIST_A || p.kind == PASS_WP_A) {
                    e.c_src = in;
                    e.c_dst = out;
                    e.s_src = out;
                    e.s_dst = out;
                    e.unit_elems = n * n;
                    e.s_stride = n;
                    e.c_ci = p.conj_in ? -1.f : 1.f;
                    e.c_sx = e.c_sy = p.c_scale;
                    e.s_ci = 1.f;
                    e.s_sx = e.s_sy = p.s_scale;
                    e.dep_target = (uint32_t)p.trans_rows;
                    e.s_evict_first = 0;
                } else {
                    e.s_src = out;
                    e.s_dst = out;
                    e.unit_elems = n * n * n;
                    e.s_stride = n * n;
                    e.s_ci = 1.f;
                    e.s_sx = p.scale;
                    e.s_sy = p.conj_out ? -p.scale : p.scale;
                    e.s_evict_first = 1;
                }
                if (cudaMemsetAsync(d_ctr, 0, (size_t)(1 + p.units) * sizeof(uint32_t), st) != cudaSuccess)
                    return WSFFT_ERR_CUDA;
                prof_begin(st);
                cudaError_t err = p.kind == PASS_PERSIST_A
                                      ? launch_persist(dtype, p.N, e, 0, nullptr, persist_grid, st)
                                  : p.kind == PASS_WP_A ? launch_wpp(dtype, p.N, e, nullptr, persist_grid, st)
                                                        : launch_engine(dtype, p.N, e, eng_grid, st);
                prof_end(st);
                if (err != cudaSuccess) return err == cudaErrorInvalidValue ? WSFFT_ERR_UNSUPPORTED : WSFFT_ERR_CUDA;
                continue;
            }
            const int64_t off = b0 * p.transform_elems * eb;
            const char *src = p.src == SRC_IN ? (const char *)in + off
                              : p.src == SRC_OUT ? (const char *)out + off
                                                 : (const char *)work;
            char *dst = p.dst == DST_OUT ? (char *)out + off : (char *)work;
            const PassArgs a = pass_args(p, p.npencils_per_batch * nb);
            prof_begin(st);
            cudaError_t e = launch(dtype, p, src, dst, a, st);
            prof_end(st);
            if (e != cudaSuccess) return e == cudaErrorInvalidValue ? WSFFT_ERR_UNSUPPORTED : WSFFT_ERR_CUDA;
        }
    }
    return WSFFT_SUCCESS;
}

PassArgs Plan::pass_args(const PassSpec &p, int64_t npencils) const {
    PassArgs a{};
    a.npencils = npencils;
    a.inner = p.inner;
    a.log_inner = ilog2(p.inner);
    a.tw = p.tw;
    a.conj_in = p.conj_in ? -1.f : 1.f;
    a.sx = p.scale;
    a.sy = p.conj_out ? -p.scale : p.scale;
    a.trans_rows = p.trans_rows;
    a.tw_hi = p.twid_len ? p.tw2 : nullptr;
    a.tw_lo = p.twid_len ? p.tw2 + (p.twid_len >> p.twid_shift) : nullptr;
    a.tw_shift = p.twid_len ? p.twid_shift : 0;
    a.tw_mask = p.twid_len ? (int)(p.twid_len - 1) : 0;
    a.status = d_status;
    a.timeout_ns = (uint64_t)wait_timeout_ns;
    a.reverse = p.reverse ? 1 : 0;
    return a;
}

// Host buffers, rank 3 with one launch per superstep: the copies overlap the
// supersteps.  Slab chunks (along the first axis) are copied in on a second
// stream and the z superstep of each chunk (slab-local) runs as soon as the
// chunk has arrived; the x superstep, which needs every slab, runs over the
// whole array; then the y superstep (slab-local again) runs chunk by chunk
// and each finished chunk goes back to the host with one contiguous copy, on
// a third stream, while the next is transformed.  The supersteps are taken in
// the order z, x, y (the order of axes is free, Section 1).  The data crosses
// the host link once in each direction; the x superstep and one chunk's z
// and y are the only compute of a lone transform not hidden behind a copy,
// and in a batch the next transform's copies in share the time of the
// previous one's copies out (the two directions of the link).  (Chunking the
// x superstep instead would need strided 2D copies back, measured 17% slower
// than contiguous ones on this link.)
bool Plan::can_pipeline_host() const {
    if (ragged || rank != 3 || chunk != batch || passes.size() != 3 || dims[0] < 2) return false;
    if (passes[0].kind != PASS_CONTIG || passes[1].kind != PASS_STRIDED || passes[2].kind != PASS_STRIDED)
        return false;
    for (const auto &p : passes)
        if (p.variant || p.src == SRC_WORK || p.dst == DST_WORK) return false;
    return true;
}

int Plan::run_host_pipelined(const void *hin, void *hout, cudaStream_t st) {
    constexpr int K = 8;  // chunks per direction
    // streams and events are made on first use; a call that failed half-way
    // through making them leaves nothing half-made for the next one
    if (!copy_stream && cudaStreamCreateWithFlags(&copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
        copy_stream = nullptr;
        return WSFFT_ERR_CUDA;
    }
    if (!copy_out_stream && cudaStreamCreateWithFlags(&copy_out_stream, cudaStreamNonBlocking) != cudaSuccess) {
        copy_out_stream = nullptr;
        return WSFFT_ERR_CUDA;
    }
    if (pipe_ev.size() != 2 * K + 2) {
        std::vector<cudaEvent_t> evs(2 * K + 2, nullptr);
        for (auto &e : evs)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
                for (auto made : evs)
                    if (made) cudaEventDestroy(made);
                return WSFFT_ERR_CUDA;
            }
        pipe_ev.swap(evs);
    }
    const int64_t eb = elem_bytes(dtype);
    const int64_t n0 = dims[0], I = dims[1] * dims[2];
    const int kz = (int)std::min<int64_t>(K, n0);
    cudaEvent_t ev_start = pipe_ev[2 * K], ev_done = pipe_ev[2 * K + 1];
    char *dev = (char *)host_buf;
    auto ck = [](cudaError_t e) { return e == cudaSuccess; };
    // Both copy streams start after the work already on `st`.  Copies in run
    // on copy_stream and copies out on copy_out_stream, so with a batch the
    // next transform's chunks come in (one direction of the link) while the
    // previous one's go out (the other): the transforms own disjoint parts of
    // the device buffer and of the host buffers (also in place: transform b
    // reads and writes only its own host slice).
    if (!ck(cudaEventRecord(ev_start, st)) || !ck(cudaStreamWaitEvent(copy_stream, ev_start, 0)) ||
        !ck(cudaStreamWaitEvent(copy_out_stream, ev_start, 0)))
        return WSFFT_ERR_CUDA;
    for (int64_t b = 0; b < batch; ++b) {
        const char *hb = (const char *)hin + b * elems * eb;
        char *ho = (char *)hout + b * elems * eb;
        char *db = dev + b * elems * eb;
        auto run_pass = [&](const PassSpec &p, char *ptr, int64_t npencils) {
            const PassArgs a = pass_args(p, npencils);
            prof_begin(st);
            cudaError_t e = launch(dtype, p, ptr, ptr, a, st);
            prof_end(st);
            return e == cudaSuccess ? WSFFT_SUCCESS : e == cudaErrorInvalidValue ? WSFFT_ERR_UNSUPPORTED : WSFFT_ERR_CUDA;
        };
        // in: slab chunks, each followed by its z superstep
        for (int c = 0; c < kz; ++c) {
            const int64_t s0 = c * n0 / kz, s1 = (c + 1) * n0 / kz;
            const int64_t o = s0 * I * eb, bytes = (s1 - s0) * I * eb;
            if (!ck(cudaMemcpyAsync(db + o, hb + o, (size_t)bytes, cudaMemcpyHostToDevice, copy_stream)) ||
                !ck(cudaEventRecord(pipe_ev[c], copy_stream)) || !ck(cudaStreamWaitEvent(st, pipe_ev[c], 0)))
                return WSFFT_ERR_CUDA;
            const int rc = run_pass(passes[0], db + o, (s1 - s0) * dims[1]);
            if (rc != WSFFT_SUCCESS) return rc;
        }
        // the x superstep over the whole array; the inverse's conjugation of
        // the output moves to the y superstep, which now runs last
        PassSpec px = passes[2], py = passes[1];
        py.conj_out = px.conj_out;
        px.conj_out = false;
        int rc = run_pass(px, db, I);
        if (rc != WSFFT_SUCCESS) return rc;
        // out: the y superstep of each slab chunk, then its copy back
        for (int c = 0; c < kz; ++c) {
            const int64_t s0 = c * n0 / kz, s1 = (c + 1) * n0 / kz;
            const int64_t o = s0 * I * eb, bytes = (s1 - s0) * I * eb;
            rc = run_pass(py, db + o, (s1 - s0) * dims[2]);
            if (rc != WSFFT_SUCCESS) return rc;
            if (!ck(cudaEventRecord(pipe_ev[K + c], st)) ||
                !ck(cudaStreamWaitEvent(copy_out_stream, pipe_ev[K + c], 0)) ||
                !ck(cudaMemcpyAsync(ho + o, db + o, (size_t)bytes, cudaMemcpyDeviceToHost, copy_out_stream)))
                return WSFFT_ERR_CUDA;
        }
    }
    // `st` ends after the last copy out (every copy in was waited for by a
    // z superstep on `st`)
    if (!ck(cudaEventRecord(ev_done, copy_out_stream)) || !ck(cudaStreamWaitEvent(st, ev_done, 0)))
        return WSFFT_ERR_CUDA;
    return WSFFT_SUCCESS;
}

// (Re)build a ragged plan's instance records and tile queue for its current
// tile-shape selection and lag: tile counts per superstep follow the chosen
// shape of each axis length; the queue holds z tiles of instance s, y tiles
// of s - lag and x tiles of s - 2*lag, so every wait is on smaller tickets.
int Plan::rag_build() {
    const int count = rag_count;
    if (wait_own_work() != WSFFT_SUCCESS) return WSFFT_ERR_CUDA;  // no execute may still read the tables
    if (rag_uploaded && cudaEventSynchronize(rag_copied) != cudaSuccess) return WSFFT_ERR_CUDA;
    for (int k = 0; k < 4; ++k)
        for (int alt = 0; alt < 2; ++alt) {
            rag_tw[k][alt] = table(32 << k, rag_E(32 << k, alt));
            if (!rag_tw[k][alt]) return WSFFT_ERR_ALLOC;
        }
    auto alt_of = [&](int64_t N) { return (rag_esel >> (ilog2(N) - 5)) & 1; };
    std::vector<RagInst> inst((size_t)count);
    for (int i = 0; i < count; ++i) {
        RagInst &I = inst[i];
        memset(&I, 0, sizeof(I));
        for (int d = 0; d < 3; ++d) I.n[d] = (int)rag_dims[3 * (size_t)i + d];
        I.log_n2 = ilog2(I.n[2]);
        I.log_n12 = ilog2((int64_t)I.n[1] * I.n[2]);
        const int64_t n0 = I.n[0], n1 = I.n[1], n2 = I.n[2];
        const int64_t P = rag_P((int)n2, alt_of(n2)), W1 = rag_W((int)n1, alt_of(n1)), W0 = rag_W((int)n0, alt_of(n0));
        I.tiles[0] = (int)((n0 * n1 + P - 1) / P);
        I.tiles[1] = (int)((n0 * n2 + W1 - 1) / W1);
        I.tiles[2] = (int)((n1 * n2 + W0 - 1) / W0);
        // scales of the z, y, x supersteps
        I.scale[0] = axis_scale(n2, dir, norm);
        I.scale[1] = axis_scale(n1, dir, norm);
        I.scale[2] = axis_scale(n0, dir, norm);
    }
    const int L = rag_lag;
    std::vector<RagItem> items;
    for (int s = 0; s < count + 2 * L; ++s) {
        if (s < count)
            for (int t = 0; t < inst[s].tiles[0]; ++t) items.push_back(RagItem{ITEM_SIGNAL | (0 << 8), s, t, 0});
        if (s - L >= 0 && s - L < count)
            for (int t = 0; t < inst[s - L].tiles[1]; ++t)
                items.push_back(RagItem{ITEM_STRIDED | ITEM_WAIT | ITEM_SIGNAL | (1 << 8), s - L, t, 0});
        if (s - 2 * L >= 0 && s - 2 * L < count)
            for (int t = 0; t < inst[s - 2 * L].tiles[2]; ++t)
                items.push_back(RagItem{ITEM_STRIDED | ITEM_WAIT | (2 << 8), s - 2 * L, t, 0});
    }
    if (items.size() > (size_t)0x7fffffff) return WSFFT_ERR_UNSUPPORTED;
    const size_t ib = items.size() * sizeof(RagItem), nb = inst.size() * sizeof(RagInst);
    if (items.size() > (size_t)rag_items_cap) {
        if (rag_items) cudaFree(rag_items);
        rag_items = nullptr;
        rag_items_cap = 0;
        if (cudaMalloc(&rag_items, ib) != cudaSuccess) {
            rag_items = nullptr;
            return WSFFT_ERR_ALLOC;
        }
        rag_items_cap = (int64_t)items.size();
    }
    if (!rag_inst) {
        if (cudaMalloc(&rag_inst, nb) != cudaSuccess) {
            rag_inst = nullptr;
            return WSFFT_ERR_ALLOC;
        }
        if (cudaMallocHost(&rag_inst_host, nb) != cudaSuccess) {
            rag_inst_host = nullptr;
            return WSFFT_ERR_ALLOC;
        }
    } else {
        // keep the pointers of the last execute; the tile counts changed
        const RagInst *old = static_cast<const RagInst *>(rag_inst_host);
        for (int i = 0; i < count; ++i) {
            inst[i].in = old[i].in;
            inst[i].out = old[i].out;
        }
    }
    memcpy(rag_inst_host, inst.data(), nb);
    rag_uploaded = false;  // the next execute uploads the records again
    rag_nitems = (int)items.size();
    return upload(rag_items, items.data(), ib);
}

int Plan::upload(void *dst, const void *src, size_t bytes) {
    if (!setup_st && cudaStreamCreateWithFlags(&setup_st, cudaStreamNonBlocking) != cudaSuccess) {
        setup_st = nullptr;
        return WSFFT_ERR_CUDA;
    }
    if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, setup_st) != cudaSuccess) return WSFFT_ERR_CUDA;
    return cudaStreamSynchronize(setup_st) == cudaSuccess ? WSFFT_SUCCESS : WSFFT_ERR_CUDA;
}

int Plan::zero(void *dst, size_t bytes) {
    if (!setup_st && cudaStreamCreateWithFlags(&setup_st, cudaStreamNonBlocking) != cudaSuccess) {
        setup_st = nullptr;
        return WSFFT_ERR_CUDA;
    }
    if (cudaMemsetAsync(dst, 0, bytes, setup_st) != cudaSuccess) return WSFFT_ERR_CUDA;
    return cudaStreamSynchronize(setup_st) == cudaSuccess ? WSFFT_SUCCESS : WSFFT_ERR_CUDA;
}

void Plan::mark_done(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (cs != cudaStreamCaptureStatusNone) return;  // a graph's launches are the caller's to wait for
    auto it = done_ev.find(st);
    if (it == done_ev.end()) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return;
        it = done_ev.emplace(st, e).first;
    }
    cudaEventRecord(it->second, st);
}

int Plan::wait_own_work() {
    bool ok = true;
    for (auto &kv : done_ev) ok &= cudaEventSynchronize(kv.second) == cudaSuccess;
    if (copy_stream) ok &= cudaStreamSynchronize(copy_stream) == cudaSuccess;
    if (copy_out_stream) ok &= cudaStreamSynchronize(copy_out_stream) == cudaSuccess;
    if (setup_st) ok &= cudaStreamSynchronize(setup_st) == cudaSuccess;
    return ok ? WSFFT_SUCCESS : WSFFT_ERR_CUDA;
}

void Plan::prof_begin(cudaStream_t st) {
    if (prof_used < (int)prof_ev.size() / 2) cudaEventRecord(prof_ev[2 * prof_used], st);
}

void Plan::prof_end(cudaStream_t st) {
    if (prof_used < (int)prof_ev.size() / 2) {
        cudaEventRecord(prof_ev[2 * prof_used + 1], st);
        ++prof_used;
    }
}

Plan::~Plan() {
    for (auto e : prof_ev) cudaEventDestroy(e);
    if (rag_items) cudaFree(rag_items);
    if (rag_inst) cudaFree(rag_inst);
    if (rag_inst_host) cudaFreeHost(rag_inst_host);
    if (rag_copied) cudaEventDestroy(rag_copied);
    if (d_items) cudaFree(d_items);
    if (d_ctr) cudaFree(d_ctr);
    for (auto &kv : tables) cudaFree(kv.second);
    for (auto &kv : fs_tables) cudaFree(kv.second);
    if (work) cudaFree(work);
    if (host_buf) cudaFree(host_buf);
    for (auto e : pipe_ev)
        if (e) cudaEventDestroy(e);
    if (copy_stream) cudaStreamDestroy(copy_stream);
    if (copy_out_stream) cudaStreamDestroy(copy_out_stream);
    if (d_status) cudaFree(d_status);
    for (auto &kv : done_ev) cudaEventDestroy(kv.second);
    if (setup_st) cudaStreamDestroy(setup_st);
}

}  // namespace wsfft

extern "C" {

const char *wsfft_status_string(int s) {
    switch (s) {
        case WSFFT_SUCCESS: return "success";
        case WSFFT_ERR_INVALID_ARG: return "invalid argument";
        case WSFFT_ERR_INVALID_SIZE: return "invalid size (axes must be powers of two within range)";
        case WSFFT_ERR_UNSUPPORTED: return "unsupported configuration";
        case WSFFT_ERR_ALLOC: return "allocation failed";
        case WSFFT_ERR_CUDA: return "CUDA runtime error";
        case WSFFT_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
        default: return "unknown status";
    }
}

int wsfft_plan_create(wsfft_plan *plan, const int64_t *dims, int rank, int dtype, int direction,
                      int64_t batch) {
    if (!plan) return WSFFT_ERR_INVALID_ARG;
    *plan = nullptr;
    if (!dims || rank < 1 || rank > 3 || batch < 1) return WSFFT_ERR_INVALID_ARG;
    if (dtype != WSFFT_C32 && dtype != WSFFT_C16F && dtype != WSFFT_C16BF) return WSFFT_ERR_INVALID_ARG;
    if (direction != WSFFT_FORWARD && direction != WSFFT_INVERSE) return WSFFT_ERR_INVALID_ARG;
    for (int i = 0; i < rank; ++i) {
        if (!is_pow2(dims[i])) return WSFFT_ERR_INVALID_SIZE;
        if (rank > 1 && dims[i] > 4096) return WSFFT_ERR_INVALID_SIZE;
        if (rank == 1 && dims[i] > ((int64_t)1 << 24)) return WSFFT_ERR_INVALID_SIZE;
    }
    Plan *p = new (std::nothrow) Plan();
    if (!p) return WSFFT_ERR_ALLOC;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return WSFFT_ERR_CUDA;
    }
    p->rank = rank;
    for (int i = 0; i < rank; ++i) p->dims[i] = dims[i];
    cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
    p->eng_grid = p->sm_count;  // one engine block per SM (its shared memory fills the SM)
    p->dtype = dtype;
    p->dir = direction;
    p->batch = batch;
    p->norm = dtype == WSFFT_C32 ? WSFFT_NORM_PAPER : WSFFT_NORM_ORTHO;
    p->elems = 1;
    for (int i = 0; i < rank; ++i) p->elems *= dims[i];
    if (cudaMalloc(&p->d_status, sizeof(int)) != cudaSuccess) {
        p->d_status = nullptr;
        delete p;
        return WSFFT_ERR_ALLOC;
    }
    if (p->zero(p->d_status, sizeof(int)) != WSFFT_SUCCESS) {
        delete p;
        return WSFFT_ERR_CUDA;
    }
    int rc = p->build_schedule();
    if (rc != WSFFT_SUCCESS) {
        delete p;
        return rc;
    }
    autotune_apply_cached(*p);  // a remembered choice for this key, if any
    *plan = reinterpret_cast<wsfft_plan>(p);
    return WSFFT_SUCCESS;
}

int wsfft_plan_create_axis(wsfft_plan *plan, int64_t n, int64_t inner, int dtype, int direction, int64_t batch) {
    if (!plan) return WSFFT_ERR_INVALID_ARG;
    *plan = nullptr;
    if (batch < 1 || inner < 1) return WSFFT_ERR_INVALID_ARG;
    if (dtype != WSFFT_C32 && dtype != WSFFT_C16F && dtype != WSFFT_C16BF) return WSFFT_ERR_INVALID_ARG;
    if (direction != WSFFT_FORWARD && direction != WSFFT_INVERSE) return WSFFT_ERR_INVALID_ARG;
    if (!is_pow2(n) || n > 4096 || !is_pow2(inner) || inner > ((int64_t)1 << 40)) return WSFFT_ERR_INVALID_SIZE;
    Plan *p = new (std::nothrow) Plan();
    if (!p) return WSFFT_ERR_ALLOC;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return WSFFT_ERR_CUDA;
    }
    cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
    p->eng_grid = p->sm_count;
    p->rank = 1;
    p->dims[0] = n;
    p->axis_inner = inner;
    p->dtype = dtype;
    p->dir = direction;
    p->batch = batch;
    p->norm = dtype == WSFFT_C32 ? WSFFT_NORM_PAPER : WSFFT_NORM_ORTHO;
    p->elems = n * inner;
    if (cudaMalloc(&p->d_status, sizeof(int)) != cudaSuccess) {
        p->d_status = nullptr;
        delete p;
        return WSFFT_ERR_ALLOC;
    }
    int rc = p->zero(p->d_status, sizeof(int));
    if (rc == WSFFT_SUCCESS) rc = p->build_schedule();
    if (rc != WSFFT_SUCCESS) {
        delete p;
        return rc;
    }
    *plan = reinterpret_cast<wsfft_plan>(p);
    return WSFFT_SUCCESS;
}

int wsfft_plan_set_norm(wsfft_plan plan, int norm) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || norm < WSFFT_NORM_PAPER || norm > WSFFT_NORM_FORWARD) return WSFFT_ERR_INVALID_ARG;
    if (p->ragged) return WSFFT_ERR_UNSUPPORTED;
    p->norm = norm;
    return p->build_schedule();
}

int wsfft_plan_set_layout(wsfft_plan plan, int layout) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || (layout != WSFFT_LAYOUT_NATURAL && layout != WSFFT_LAYOUT_SWAPPED && layout != WSFFT_LAYOUT_WAFER))
        return WSFFT_ERR_INVALID_ARG;
    if (p->ragged || (p->axis_inner > 0 && layout != WSFFT_LAYOUT_NATURAL)) return WSFFT_ERR_UNSUPPORTED;
    if (layout == WSFFT_LAYOUT_WAFER) {
        // every axis passes through the transposing store in one direction
        // or the other: 64..4096 points each (its row counts, products of
        // two axes, are then multiples of its pencils per block)
        if (p->rank != 3) return WSFFT_ERR_UNSUPPORTED;
        for (int i = 0; i < 3; ++i)
            if (p->dims[i] < 64 || p->dims[i] > 4096) return WSFFT_ERR_UNSUPPORTED;
    }
    if (layout == WSFFT_LAYOUT_SWAPPED) {
        // the transposing store is built for pencils of 64..4096 points, and
        // its tiles need the row count to be a multiple of their pencils per
        // block (at most 32, so rows >= 64 suffice)
        if (p->rank < 2) return WSFFT_ERR_UNSUPPORTED;
        for (int i = p->rank - 2; i < p->rank; ++i)
            if (p->dims[i] < 64 || p->dims[i] > 4096) return WSFFT_ERR_UNSUPPORTED;
    }
    const int old_layout = p->layout;
    const auto old_over = p->overrides;
    p->layout = layout;
    p->overrides.clear();
    const int rc = p->build_schedule();
    if (rc != WSFFT_SUCCESS) {
        p->layout = old_layout;
        p->overrides = old_over;
        p->build_schedule();
    }
    return rc;
}

int wsfft_execute(wsfft_plan plan, const void *in, void *out, wsfft_stream stream) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || p->ragged || !in || !out) return WSFFT_ERR_INVALID_ARG;
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return WSFFT_ERR_INVALID_ARG;
    if (partial_overlap(in, out, (size_t)(p->batch * p->elems * elem_bytes(p->dtype)))) return WSFFT_ERR_INVALID_ARG;
    const int rc = p->run(in, out, (cudaStream_t)stream);
    p->mark_done((cudaStream_t)stream);
    return rc;
}

int wsfft_execute_host(wsfft_plan plan, const void *host_in, void *host_out, wsfft_stream stream) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || p->ragged || !host_in || !host_out) return WSFFT_ERR_INVALID_ARG;
    const size_t bytes = (size_t)(p->batch * p->elems * elem_bytes(p->dtype));
    if (partial_overlap(host_in, host_out, bytes)) return WSFFT_ERR_INVALID_ARG;
    if (!p->host_buf) {
        if (cudaMalloc(&p->host_buf, bytes) != cudaSuccess) {
            p->host_buf = nullptr;
            return WSFFT_ERR_ALLOC;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (p->can_pipeline_host()) {
        const int rc = p->run_host_pipelined(host_in, host_out, st);
        if (rc != WSFFT_SUCCESS) return rc;
        return cuda_status(cudaStreamSynchronize(st));
    }
    if (!p->passes.empty() && p->passes[0].kind == PASS_SLAB_A) {
        // The host pipeline overlaps the copies with the three one-launch
        // supersteps (the slab-local z and y hide behind the chunked
        // copies); the fused pass A would leave the copy back unoverlapped.
        // Use that schedule for this call, then restore the plan's own.
        const int mode = p->engine_mode;
        const auto over = p->overrides;
        p->engine_mode = 0;
        p->overrides.clear();
        int rc = p->build_schedule();
        const bool ok = rc == WSFFT_SUCCESS && p->can_pipeline_host();
        if (ok) rc = p->run_host_pipelined(host_in, host_out, st);
        p->engine_mode = mode;
        p->overrides = over;
        const int rc2 = p->build_schedule();
        if (ok) {
            if (rc != WSFFT_SUCCESS) return rc;
            if (rc2 != WSFFT_SUCCESS) return rc2;
            return cuda_status(cudaStreamSynchronize(st));
        }
        if (rc2 != WSFFT_SUCCESS) return rc2;
    }
    if (cudaMemcpyAsync(p->host_buf, host_in, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return WSFFT_ERR_CUDA;
    int rc = p->run(p->host_buf, p->host_buf, st);
    if (rc != WSFFT_SUCCESS) return rc;
    if (cudaMemcpyAsync(host_out, p->host_buf, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return WSFFT_ERR_CUDA;
    return cuda_status(cudaStreamSynchronize(st));
}

int wsfft_destroy(wsfft_plan plan) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p) return WSFFT_SUCCESS;
    int prev = -1;
    const int dev = p->device;
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
    const int rc = p->wait_own_work();  // this plan's executes only, not the whole device
    delete p;
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    return rc;
}

int wsfft_plan_set_pass_variant(wsfft_plan plan, int pass, int values_per_thread, int tile) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || pass < 0 || pass >= (int)p->passes.size() || values_per_thread < 0 || tile < 0)
        return WSFFT_ERR_INVALID_ARG;
    if (values_per_thread == 0 && tile == 0) {
        p->overrides.erase(pass);
        return p->build_schedule();
    }
    const PassSpec &ps = p->passes[pass];
    if (ps.kind != PASS_CONTIG && ps.kind != PASS_STRIDED) return WSFFT_ERR_UNSUPPORTED;
    // probe: is this shape instantiated?  (an empty launch returns before running)
    PassArgs a{};
    a.npencils = 0;
    PassSpec probe = ps;
    probe.E = values_per_thread;
    probe.tile = tile;
    if (launch(p->dtype, probe, nullptr, nullptr, a, 0) == cudaErrorInvalidValue)
        return WSFFT_ERR_UNSUPPORTED;
    p->overrides[pass] = std::make_pair(values_per_thread, tile);
    return p->build_schedule();
}

int wsfft_plan_set_engine(wsfft_plan plan, int mode) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || mode < 0 || mode > 4) return WSFFT_ERR_INVALID_ARG;
    if (p->ragged) return WSFFT_ERR_UNSUPPORTED;
    p->engine_mode = mode;
    return p->build_schedule();
}

int wsfft_plan_set_wait_test(wsfft_plan plan, int withhold, int64_t timeout_ns) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || timeout_ns <= 0) return WSFFT_ERR_INVALID_ARG;
    bool uses_engine = false;
    for (auto &ps : p->passes)
        uses_engine |= ps.kind == PASS_ENGINE_A || ps.kind == PASS_PERSIST_A || ps.kind == PASS_WP_A;
    if (!uses_engine) return WSFFT_ERR_UNSUPPORTED;
    p->withhold = withhold != 0;
    p->wait_timeout_ns = timeout_ns;
    return p->build_schedule();
}

int wsfft_plan_sync_status(wsfft_plan plan, wsfft_stream stream) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p) return WSFFT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    if (cudaMemcpyAsync(&h, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return WSFFT_ERR_CUDA;
    if (h != 0 && (cudaMemsetAsync(p->d_status, 0, sizeof(int), st) != cudaSuccess ||
                   cudaStreamSynchronize(st) != cudaSuccess))
        return WSFFT_ERR_CUDA;
    return h == 0 ? WSFFT_SUCCESS : WSFFT_ERR_DEVICE_TIMEOUT;
}

int wsfft_plan_passes(wsfft_plan plan, int *passes, int64_t *bytes) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p) return WSFFT_ERR_INVALID_ARG;
    const int np = p->ragged ? 3 : (int)p->passes.size();
    if (passes) *passes = np;
    if (bytes) *bytes = (int64_t)np * 2 * p->batch * p->elems * elem_bytes(p->dtype);
    return WSFFT_SUCCESS;
}

int wsfft_plan_profile(wsfft_plan plan, int capacity) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || capacity < 0) return WSFFT_ERR_INVALID_ARG;
    for (auto e : p->prof_ev) cudaEventDestroy(e);
    p->prof_ev.clear();
    p->prof_used = 0;
    for (int i = 0; i < 2 * capacity; ++i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return WSFFT_ERR_CUDA;
        p->prof_ev.push_back(e);
    }
    return WSFFT_SUCCESS;
}

int wsfft_plan_launch_times(wsfft_plan plan, float *ms, int capacity, int *count) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || capacity < 0) return WSFFT_ERR_INVALID_ARG;
    const int n = p->prof_used;
    if (n > 0 && cudaEventSynchronize(p->prof_ev[2 * n - 1]) != cudaSuccess) return WSFFT_ERR_CUDA;
    for (int i = 0; i < n && ms && i < capacity; ++i) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, p->prof_ev[2 * i], p->prof_ev[2 * i + 1]) != cudaSuccess)
            return WSFFT_ERR_CUDA;
        ms[i] = t;
    }
    if (count) *count = n;
    p->prof_used = 0;
    return WSFFT_SUCCESS;
}

int wsfft_plan_create_ragged(wsfft_plan *plan, int count, const int64_t *dims, int dtype,
                             int direction) {
    if (!plan) return WSFFT_ERR_INVALID_ARG;
    *plan = nullptr;
    if (!dims || count < 1 || count > (1 << 20)) return WSFFT_ERR_INVALID_ARG;
    if (dtype != WSFFT_C32 && dtype != WSFFT_C16F && dtype != WSFFT_C16BF) return WSFFT_ERR_INVALID_ARG;
    if (direction != WSFFT_FORWARD && direction != WSFFT_INVERSE) return WSFFT_ERR_INVALID_ARG;
    for (int i = 0; i < 3 * count; ++i)
        if (!is_pow2(dims[i]) || dims[i] < 32 || dims[i] > 256) return WSFFT_ERR_INVALID_SIZE;
    Plan *p = new (std::nothrow) Plan();
    if (!p) return WSFFT_ERR_ALLOC;
    p->ragged = true;
    p->rag_count = count;
    p->dtype = dtype;
    p->dir = direction;
    p->norm = dtype == WSFFT_C32 ? WSFFT_NORM_PAPER : WSFFT_NORM_ORTHO;
    p->batch = 1;
    auto fail = [&](int rc) {
        delete p;
        return rc;
    };
    if (cudaGetDevice(&p->device) != cudaSuccess) return fail(WSFFT_ERR_CUDA);
    cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
    if (cudaMalloc(&p->d_status, sizeof(int)) != cudaSuccess) {
        p->d_status = nullptr;
        return fail(WSFFT_ERR_ALLOC);
    }
    if (p->zero(p->d_status, sizeof(int)) != WSFFT_SUCCESS) return fail(WSFFT_ERR_CUDA);
    p->rag_dims.assign(dims, dims + 3 * (size_t)count);
    p->elems = 0;
    for (int i = 0; i < count; ++i) p->elems += dims[3 * i] * dims[3 * i + 1] * dims[3 * i + 2];
    {
        const int rc = p->rag_build();
        if (rc != WSFFT_SUCCESS) return fail(rc);
    }
    if (cudaMalloc(&p->d_ctr, (size_t)(1 + 2 * count) * sizeof(uint32_t)) != cudaSuccess) {
        p->d_ctr = nullptr;
        return fail(WSFFT_ERR_ALLOC);
    }
    p->ctr_cap = 1 + 2 * count;
    if (cudaEventCreateWithFlags(&p->rag_copied, cudaEventDisableTiming) != cudaSuccess) {
        p->rag_copied = nullptr;
        return fail(WSFFT_ERR_CUDA);
    }
    int per_sm = 0;
    RagArgs dummy{};
    cudaError_t e = dtype == WSFFT_C32 ? launch_ragged_c32(dummy, &per_sm, 0, 0)
                    : dtype == WSFFT_C16F ? launch_ragged_c16f(dummy, &per_sm, 0, 0)
                                          : launch_ragged_c16bf(dummy, &per_sm, 0, 0);
    if (e != cudaSuccess || per_sm < 1) return fail(WSFFT_ERR_CUDA);
    p->rag_grid = per_sm * p->sm_count;
    autotune_apply_cached(*p);  // a remembered tile-shape choice and lag for this shape set, if any
    *plan = reinterpret_cast<wsfft_plan>(p);
    return WSFFT_SUCCESS;
}

int wsfft_plan_set_ragged_variant(wsfft_plan plan, int shape_select, int lag) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || shape_select < 0 || shape_select > 15 || lag < 1 || lag > 64) return WSFFT_ERR_INVALID_ARG;
    if (!p->ragged) return WSFFT_ERR_UNSUPPORTED;
    const int old_sel = p->rag_esel, old_lag = p->rag_lag;
    p->rag_esel = shape_select;
    p->rag_lag = lag;
    const int rc = p->rag_build();
    if (rc != WSFFT_SUCCESS) {
        p->rag_esel = old_sel;
        p->rag_lag = old_lag;
        p->rag_build();
    }
    return rc;
}

int wsfft_execute_ragged(wsfft_plan plan, const void *const *in, void *const *out,
                         wsfft_stream stream) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || !p->ragged || !in || !out) return WSFFT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    RagInst *h = static_cast<RagInst *>(p->rag_inst_host);
    bool changed = !p->rag_uploaded;
    for (int i = 0; i < p->rag_count; ++i) {
        if (!in[i] || !out[i] || ((uintptr_t)in[i] & 15) || ((uintptr_t)out[i] & 15)) return WSFFT_ERR_INVALID_ARG;
        changed |= h[i].in != in[i] || h[i].out != out[i];
    }
    if (changed) {
        // the previous upload may still be reading the pinned table
        if (p->rag_uploaded && cudaEventSynchronize(p->rag_copied) != cudaSuccess) return WSFFT_ERR_CUDA;
        for (int i = 0; i < p->rag_count; ++i) {
            h[i].in = in[i];
            h[i].out = out[i];
        }
        if (cudaMemcpyAsync(p->rag_inst, h, sizeof(RagInst) * (size_t)p->rag_count, cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
            return WSFFT_ERR_CUDA;
        if (cudaEventRecord(p->rag_copied, st) != cudaSuccess) return WSFFT_ERR_CUDA;
        p->rag_uploaded = true;
    }
    if (cudaMemsetAsync(p->d_ctr, 0, sizeof(uint32_t) * (size_t)(1 + 2 * p->rag_count), st) != cudaSuccess)
        return WSFFT_ERR_CUDA;
    RagArgs a{};
    a.items = static_cast<const RagItem *>(p->rag_items);
    a.nitems = p->rag_nitems;
    a.inst = static_cast<const RagInst *>(p->rag_inst);
    a.ctr = p->d_ctr;
    a.status = p->d_status;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 2; ++j) a.tw[i][j] = p->rag_tw[i][j];
    a.esel = p->rag_esel;
    a.ci = p->dir == WSFFT_INVERSE ? -1.f : 1.f;
    a.co = a.ci;
    a.timeout_ns = (uint64_t)p->wait_timeout_ns;
    p->prof_begin(st);
    cudaError_t e = p->dtype == WSFFT_C32 ? launch_ragged_c32(a, nullptr, p->rag_grid, st)
                    : p->dtype == WSFFT_C16F ? launch_ragged_c16f(a, nullptr, p->rag_grid, st)
                                             : launch_ragged_c16bf(a, nullptr, p->rag_grid, st);
    p->prof_end(st);
    p->mark_done(st);
    return e == cudaSuccess ? WSFFT_SUCCESS : WSFFT_ERR_CUDA;
}


}  // extern "C"
