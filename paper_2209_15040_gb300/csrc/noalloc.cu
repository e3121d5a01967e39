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
// Set-up: the first call on each device (with that device current) copies
// the twiddle tables into their array on the caller's stream and waits for
// that stream, looks up the arrays' device addresses with
// cudaGetSymbolAddress and queries the occupancy of the persistent kernel.
//
// Timeouts: pass A's waits are bounded (one second each); a wait that runs
// out sets a status word in a third static array and its tile is skipped, so
// that call's result is incomplete.  The call itself cannot see this (it
// does not wait for the GPU); wsfft_noalloc_sync_status reports and clears
// it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/wsfft.h"
#include "fft_core.cuh"
#include "host_roots.h"
#include "pass_desc.h"
#include "persist.cuh"

namespace wsfft {
namespace {

constexpr int kMaxSlabs = 4096;     // batch * n limit
constexpr int kTwElems = 2048;      // complex entries in the static twiddle array
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint32_t g_noalloc_ctr[1 + kMaxSlabs];
static __device__ __align__(256) float2 g_noalloc_tw[kTwElems];
// Status word of the bounded waits: set to 1 when a wait of pass A runs out
// (the tiles that wait skip their work, so the result of that call is
// incomplete).  Sticky until wsfft_noalloc_sync_status reads and clears it.
static __device__ __align__(256) int g_noalloc_status;

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
    uint32_t *ctr = nullptr;
    float2 *tw = nullptr;
    int *status = nullptr;
    int tw_off[3][2] = {};   // [shape][pass A / pass B] offset in the twiddle array
    int grid[3] = {};
};

DevState g_dev[kMaxDevices];
std::mutex g_mu;

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

// Once per device, with that device current: tables (copied on `st`, which
// is then synchronised), symbol addresses, occupancy.  Returns a
// wsfft_status.
int setup_device(int dev, DevState &d, cudaStream_t st) {
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
    if (cudaMemcpyToSymbolAsync(g_noalloc_tw, host_tw, sizeof(float2) * off, 0, cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return WSFFT_ERR_CUDA;
    // host code sees only host-side stand-ins for the arrays: their device
    // addresses come from the runtime, per device
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_ctr) != cudaSuccess || !p) return WSFFT_ERR_CUDA;
    d.ctr = static_cast<uint32_t *>(p);
    p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_tw) != cudaSuccess || !p) return WSFFT_ERR_CUDA;
    d.tw = static_cast<float2 *>(p);
    p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_status) != cudaSuccess || !p) return WSFFT_ERR_CUDA;
    d.status = static_cast<int *>(p);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return WSFFT_ERR_CUDA;
    if (setup_kernel<128, 16, 64>(sms, &d.grid[0]) != cudaSuccess) return WSFFT_ERR_CUDA;
    if (setup_kernel<256, 16, 32>(sms, &d.grid[1]) != cudaSuccess) return WSFFT_ERR_CUDA;
    if (setup_kernel<512, 8, 8>(sms, &d.grid[2]) != cudaSuccess) return WSFFT_ERR_CUDA;
    d.ready = true;
    return WSFFT_SUCCESS;
}

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
    {
        // in == out is the in-place form; any other shared bytes would be
        // read after another tile wrote them
        const char *a = static_cast<const char *>(in), *b = static_cast<const char *>(out);
        const size_t bytes = (size_t)(batch * n * n * n) * sizeof(float2);
        if (a != b && a < b + bytes && b < a + bytes) return WSFFT_ERR_INVALID_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return WSFFT_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return WSFFT_ERR_UNSUPPORTED;
    DevState &d = g_dev[dev];
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!d.ready) {
            const int rc = setup_device(dev, d, (cudaStream_t)stream);
            if (rc != WSFFT_SUCCESS) return rc;
        }
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
    a.status = d.status;
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

extern "C" int wsfft_noalloc_sync_status(wsfft_stream stream) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return WSFFT_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return WSFFT_ERR_UNSUPPORTED;
    int *status = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_dev[dev].ready) return WSFFT_SUCCESS;  // no call has run on this device
        status = g_dev[dev].status;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    if (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return WSFFT_ERR_CUDA;
    if (h != 0 && (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess))
        return WSFFT_ERR_CUDA;
    return h == 0 ? WSFFT_SUCCESS : WSFFT_ERR_DEVICE_TIMEOUT;
}
