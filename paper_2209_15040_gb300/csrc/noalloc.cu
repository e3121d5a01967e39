// wsfft_execute_cube_noalloc: an n^3 complex64 transform that allocates no
// device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a CUDA
// graph being captured, code whose memory is handed out by another
// framework's allocator, or embedded callers that reserve all device memory
// up front.  For them this entry point runs the two-launch cube schedule of
// persist.cuh (the z and y supersteps of each slab chained through L2 in one
// persistent launch, then the x superstep) with its scratch memory -- the
// ticket counter and the per-slab completion counters -- in a file-scope
// static __device__ array, and its twiddle tables in another, instead of in
// plan-owned allocations.
//
// Limits: complex64 only, n in {128, 256, 512}, batch * n <= 4096 slabs.
// The counter array holds 1 + 4096 32-bit words (16 KiB) and the twiddle
// array 2048 complex values (16 KiB); every GPU that loads the library keeps
// both until the process exits.
//
// Sharing: every call on a device uses the same arrays, which keep the last
// call's contents; each call clears the counters it uses (cudaMemsetAsync on
// its stream) before its kernels run.  Calls that overlap on the GPU -- on
// two streams, or from two host threads -- race on the counters and must not
// be issued.
//
// Set-up: the first call on each device (with that device current) uploads
// the twiddle tables with cudaMemcpyToSymbol, looks up the arrays' device
// addresses with cudaGetSymbolAddress and queries the occupancy of the
// persistent kernel.  Make that first call before any stream capture.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/wsfft.h"
#include "fft_core.cuh"
#include "pass_desc.h"
#include "persist.cuh"

namespace wsfft {
namespace {

constexpr int kMaxSlabs = 4096;     // batch * n limit
constexpr int kTwElems = 2048;      // complex entries in the static twiddle array
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint32_t g_noalloc_ctr[1 + kMaxSlabs];
static __device__ __align__(256) float2 g_noalloc_tw[kTwElems];

// schedules used: persistent pass A per n, and the x superstep per n
struct CubeShape {
    int n;
    int ea;      // values per thread of pass A (both tile kinds)
    int tp;      // pencils per pass-A tile
    int eb;      // values per thread of the x superstep
    int tileb;   // pencils per block of the x superstep (0 = default shape)
};
constexpr CubeShape kShapes[3] = {{128, 16, 64, 16, 0}, {256, 16, 32, 16, 0}, {512, 8, 8, 16, 16}};

struct DevState {
    bool ready = false;
    int status = 0;
    uint32_t *ctr = nullptr;
    float2 *tw = nullptr;
    int tw_off[3][2] = {};   // [shape][pass A / pass B] offset in the twiddle array
    int grid[3] = {};
};

DevState g_dev[kMaxDevices];
std::mutex g_mu;

// exp(-2*pi*i*m/n), evaluated in long double on the angle folded into
// [0, pi/2] by quadrant, then rounded to float.
float2 root_ld(int64_t m, int64_t n) {
    m %= n;
    if (m < 0) m += n;
    const int64_t q = (4 * m) / n;
    const long double f = (long double)(4 * m - q * n) / (long double)n;  // [0, 1)
    const long double a = 1.57079632679489661923132169163975144L * f;
    const long double c = cosl(a), s = sinl(a);
    long double cr, sr;
    switch (q) {
        case 0: cr = c; sr = s; break;
        case 1: cr = -s; sr = c; break;
        case 2: cr = -c; sr = -s; break;
        default: cr = s; sr = -c; break;
    }
    return make_float2((float)cr, (float)-sr);
}

int fill_stage_table(float2 *dst, int cap, int N, int E) {
    const int size = sched_tw_size(N, E);
    if (size + 1 > cap) return -1;
    const int ns = sched_nstages(N, E);
    for (int s = 1; s < ns; ++s) {
        const int R = sched_radix(N, E, s), Ns = sched_ns_before(N, E, s);
        const int off = sched_tw_offset(N, E, s);
        for (int r = 1; r < R; ++r)
            for (int k = 0; k < Ns; ++k) dst[off + (r - 1) * Ns + k] = root_ld((int64_t)r * k, (int64_t)Ns * R);
    }
    dst[size] = make_float2(0.f, 0.f);
    return size + 1;
}

// Tile order of pass A (the same rule as the plan builder's): slab j's
// contiguous tiles, then the strided tiles of slab j - lag.  Decoded from
// the ticket, so no item table is needed.
__device__ __forceinline__ int4 decode_item(int t, int per, int U, int lag) {
    if (t < lag * per) return make_int4(ITEM_SIGNAL, t / per, t % per, 0);
    const int t2 = t - lag * per;
    const int mid = (U - lag) * 2 * per;
    if (t2 < mid) {
        const int j = lag + t2 / (2 * per), o = t2 % (2 * per);
        if (o < per) return make_int4(ITEM_SIGNAL, j, o, 0);
        return make_int4(ITEM_STRIDED | ITEM_WAIT, j - lag, o - per, 0);
    }
    const int t3 = t2 - mid;
    return make_int4(ITEM_STRIDED | ITEM_WAIT, U + t3 / per - lag, t3 % per, 0);
}

// Pass A of persist.cuh with the item decoded from the ticket.
template <int NC, int EC, int P, int NS, int ES, int W>
__global__ void __launch_bounds__(PCfg<NC, EC, P, NS, ES, W, float2>::THREADS, 2)
    noalloc_pass_a(EngArgs a, int per, int U, int lag) {
    using C = PCfg<NC, EC, P, NS, ES, W, float2>;
    extern __shared__ float2 na_smem[];
    __shared__ int4 s_item;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) {
            const int ticket = (int)atomicAdd(&a.ctr[0], 1u);
            int4 it = ticket < a.nitems ? decode_item(ticket, per, U, lag) : make_int4(ITEM_END, 0, 0, 0);
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
                const int w = tid % W, t = tid / W;
                const int64_t base = (int64_t)it.y * a.unit_elems + (int64_t)it.z * W + w;
                StridedAcc<float2, false, OP_CG, OP_CS, W> acc;
                acc.in = reinterpret_cast<const float2 *>(a.s_src) + base;
                acc.out = reinterpret_cast<float2 *>(a.s_dst) + base;
                acc.sm = na_smem;
                acc.stride = a.s_stride;
                acc.w = w;
                acc.ci = a.s_ci;
                acc.epi = Epi{a.s_sx, a.s_sy};
                acc.active = true;
                pencil_fft<NS, ES>(acc, t, a.tw_s);
            } else {
                constexpr int T = NC / EC;
                const int t = tid % T, p = tid / T;
                const int64_t off =
                    (int64_t)it.y * a.unit_elems + (int64_t)it.z * C::TILE_C + (int64_t)p * NC;
                ContigAcc<float2, OP_CS, OP_DEF> acc{reinterpret_cast<const float2 *>(a.c_src) + off,
                                                     reinterpret_cast<float2 *>(a.c_dst) + off,
                                                     na_smem + p * contig_PS(NC),
                                                     a.c_ci,
                                                     {a.c_sx, a.c_sy},
                                                     true};
                pencil_fft<NC, EC>(acc, t, a.tw_c);
            }
        }
        __syncthreads();
        if ((it.x & ITEM_SIGNAL) && !(it.x & ITEM_SKIP) && tid == 0) {
            __threadfence();
            red_release_add_u32(a.ctr + 1 + it.y, 1u);
        }
    }
}

template <int NC, int EC, int P>
cudaError_t setup_kernel(int sm_count, int *grid) {
    using C = PCfg<NC, EC, P, NC, EC, P, float2>;
    auto kern = noalloc_pass_a<NC, EC, P, NC, EC, P>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, C::THREADS, C::SMEM);
    if (e != cudaSuccess) return e;
    *grid = nb * sm_count;
    return nb > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

template <int NC, int EC, int P>
cudaError_t launch_a(const EngArgs &a, int per, int U, int lag, int grid, cudaStream_t st) {
    using C = PCfg<NC, EC, P, NC, EC, P, float2>;
    noalloc_pass_a<NC, EC, P, NC, EC, P><<<grid, C::THREADS, C::SMEM, st>>>(a, per, U, lag);
    return cudaGetLastError();
}

// Once per device, with that device current: tables, symbol addresses,
// occupancy.  Returns a wsfft_status.
int setup_device(int dev, DevState &d) {
    static float2 host_tw[kTwElems];  // static: set-up allocates nothing either
    int off = 0;
    for (int s = 0; s < 3; ++s) {
        for (int pass = 0; pass < 2; ++pass) {
            const int E = pass == 0 ? kShapes[s].ea : kShapes[s].eb;
            if (pass == 1 && kShapes[s].eb == kShapes[s].ea) {
                d.tw_off[s][1] = d.tw_off[s][0];
                continue;
            }
            const int used = fill_stage_table(host_tw + off, kTwElems - off, kShapes[s].n, E);
            if (used < 0) return WSFFT_ERR_UNSUPPORTED;
            d.tw_off[s][pass] = off;
            off += (used + 1) & ~1;  // keep 16-byte alignment
        }
    }
    if (cudaMemcpyToSymbol(g_noalloc_tw, host_tw, sizeof(float2) * off) != cudaSuccess) return WSFFT_ERR_CUDA;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_ctr) != cudaSuccess || !p) return WSFFT_ERR_CUDA;
    d.ctr = static_cast<uint32_t *>(p);
    p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_tw) != cudaSuccess || !p) return WSFFT_ERR_CUDA;
    d.tw = static_cast<float2 *>(p);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return WSFFT_ERR_CUDA;
    if (setup_kernel<128, 16, 64>(sms, &d.grid[0]) != cudaSuccess) return WSFFT_ERR_CUDA;
    if (setup_kernel<256, 16, 32>(sms, &d.grid[1]) != cudaSuccess) return WSFFT_ERR_CUDA;
    if (setup_kernel<512, 8, 8>(sms, &d.grid[2]) != cudaSuccess) return WSFFT_ERR_CUDA;
    d.ready = true;
    return WSFFT_SUCCESS;
}

// Status word the kernel's bounded waits write to if one ever runs out (the
// waits only depend on tiles of the same call, so this needs a faulty GPU).
static __device__ __align__(256) int g_noalloc_status;

}  // namespace
}  // namespace wsfft

using namespace wsfft;

extern "C" int wsfft_execute_cube_noalloc(const void *in, void *out, int64_t n, int64_t batch,
                                          int direction, wsfft_stream stream) {
    if (!in || !out || ((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return WSFFT_ERR_INVALID_ARG;
    if (direction != WSFFT_FORWARD && direction != WSFFT_INVERSE) return WSFFT_ERR_INVALID_ARG;
    int s = -1;
    for (int i = 0; i < 3; ++i)
        if (kShapes[i].n == n) s = i;
    if (s < 0 || batch < 1) return WSFFT_ERR_INVALID_SIZE;
    if (batch * n > kMaxSlabs) return WSFFT_ERR_INVALID_SIZE;  // counter array too small
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return WSFFT_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return WSFFT_ERR_UNSUPPORTED;
    DevState &d = g_dev[dev];
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!d.ready) {
            const int rc = setup_device(dev, d);
            if (rc != WSFFT_SUCCESS) return rc;
        }
    }
    int *status = nullptr;
    {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_status) != cudaSuccess || !p) return WSFFT_ERR_CUDA;
        status = static_cast<int *>(p);
    }
    cudaStream_t st = (cudaStream_t)stream;
    const CubeShape &cs = kShapes[s];
    const int per = (int)(n / cs.tp);
    const int U = (int)(batch * n);
    int lag = (2 * d.grid[s] + 2 * per - 1) / (2 * per) + 2;
    if (lag > U) lag = U;
    const bool inv = direction == WSFFT_INVERSE;
    const float sc = inv ? (float)(1.0 / (double)n) : 1.f;  // 1/n per superstep on the inverse

    // clear the counters this call uses: the array keeps the previous call's values
    if (cudaMemsetAsync(d.ctr, 0, sizeof(uint32_t) * (size_t)(1 + U), st) != cudaSuccess) return WSFFT_ERR_CUDA;

    EngArgs a{};
    a.items = nullptr;
    a.nitems = 2 * per * U;
    a.ctr = d.ctr;
    a.status = status;
    a.c_src = in;
    a.c_dst = out;
    a.s_src = out;
    a.s_dst = out;
    a.unit_elems = n * n;
    a.s_stride = n;
    a.tw_c = d.tw + d.tw_off[s][0];
    a.tw_s = a.tw_c;
    a.c_ci = inv ? -1.f : 1.f;
    a.c_sx = a.c_sy = sc;
    a.s_ci = 1.f;
    a.s_sx = a.s_sy = sc;
    a.dep_target = (uint32_t)per;
    a.timeout_ns = 1000000000ull;
    cudaError_t e;
    switch (n) {
        case 128: e = launch_a<128, 16, 64>(a, per, U, lag, d.grid[0], st); break;
        case 256: e = launch_a<256, 16, 32>(a, per, U, lag, d.grid[1], st); break;
        default: e = launch_a<512, 8, 8>(a, per, U, lag, d.grid[2], st); break;
    }
    if (e != cudaSuccess) return WSFFT_ERR_CUDA;

    // x superstep: the strided kernel, no scratch
    PassArgs b{};
    b.npencils = batch * n * n;
    b.inner = n * n;
    int li = 0;
    while (((int64_t)1 << li) < n * n) ++li;
    b.log_inner = li;
    b.tw = d.tw + d.tw_off[s][1];
    b.conj_in = 1.f;
    b.sx = sc;
    b.sy = inv ? -sc : sc;
    e = launch_pass_c32(PASS_STRIDED, (int)n, cs.eb, cs.tileb, false, out, out, b, st);
    return e == cudaSuccess ? WSFFT_SUCCESS : WSFFT_ERR_CUDA;
}
