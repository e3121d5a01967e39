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
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "../../include/wsfft.h"
#include "fft_core.cuh"
#include "pass_desc.h"
#include "pass_kernels.cuh"
#include "plan_internal.h"

using namespace wsfft;

namespace {

bool is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

int ilog2(int64_t n) {
    int l = 0;
    while (((int64_t)1 << l) < n) ++l;
    return l;
}

int64_t elem_bytes(int dtype) { return dtype == WSFFT_C32 ? 8 : 4; }

// exp(-2*pi*i*m/n) in long double, reduced to an angle in [0, pi/4] by the
// eight-fold symmetry of the unit circle, then rounded to float.
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

std::vector<float2> stage_table(int N, int E) {
    std::vector<float2> t((size_t)sched_tw_size(N, E) + 1);
    const int ns = sched_nstages(N, E);
    for (int s = 1; s < ns; ++s) {
        const int R = sched_radix(N, E, s), Ns = sched_ns_before(N, E, s);
        const int off = sched_tw_offset(N, E, s);
        for (int r = 1; r < R; ++r)
            for (int k = 0; k < Ns; ++k)
                t[(size_t)off + (size_t)(r - 1) * Ns + k] = host_root((int64_t)r * k, (int64_t)Ns * R);
    }
    return t;
}

float axis_scale(int64_t n, int dir, int norm) {
    if (norm == WSFFT_NORM_PAPER) return dir == WSFFT_INVERSE ? (float)(1.0 / (double)n) : 1.f;
    if (norm == WSFFT_NORM_ORTHO) return (float)(1.0 / std::sqrt((double)n));
    if (norm == WSFFT_NORM_FORWARD) return dir == WSFFT_FORWARD ? (float)(1.0 / (double)n) : 1.f;
    return 1.f;
}

cudaError_t launch(int dtype, const PassSpec &p, const void *in, void *out, const PassArgs &a,
                   cudaStream_t st) {
    switch (dtype) {
        case WSFFT_C32: return launch_pass_c32(p.kind, p.N, p.E, p.variant, in, out, a, st);
        case WSFFT_C16F: return launch_pass_c16f(p.kind, p.N, p.E, p.variant, in, out, a, st);
        default: return launch_pass_c16bf(p.kind, p.N, p.E, p.variant, in, out, a, st);
    }
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? WSFFT_SUCCESS : WSFFT_ERR_CUDA; }

}  // namespace

namespace wsfft {

const float2 *Plan::table(int N, int E) {
    auto key = std::make_pair(N, E);
    auto it = tables.find(key);
    if (it != tables.end()) return it->second;
    std::vector<float2> h = stage_table(N, E);
    float2 *d = nullptr;
    if (cudaMalloc(&d, h.size() * sizeof(float2)) != cudaSuccess) return nullptr;
    if (cudaMemcpy(d, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return nullptr;
    }
    tables[key] = d;
    return d;
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

    if (r == 1 && d[0] > 4096) {
        const int64_t n = d[0];
        const int lg = ilog2(n);
        const int64_t n1 = (int64_t)1 << ((lg + 1) / 2);  // contiguous length
        const int64_t n2 = n / n1;                         // strided length
        const float sc = axis_scale(n, dir, norm);
        // workspace holds `chunk` transforms (at most ~512 MiB)
        const int64_t per = n * elem_bytes(dtype);
        chunk = std::max<int64_t>(1, std::min<int64_t>(batch, ((int64_t)512 << 20) / per));
        work_elems = chunk * n;
        PassSpec a{};
        a.kind = PASS_STRIDED;
        a.N = (int)n2;
        a.E = default_E((int)n2);
        a.variant = true;
        a.inner = n1;
        a.npencils_per_batch = n1;
        a.src = SRC_IN;
        a.dst = DST_WORK;
        a.conj_in = inv;
        a.conj_out = false;
        a.scale = 1.f;
        a.twid_len = n;
        a.transform_elems = n;
        PassSpec b{};
        b.kind = PASS_CONTIG;
        b.N = (int)n1;
        b.E = default_E((int)n1);
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
    }
    for (auto &p : passes) {
        if (p.N > 4096 || !is_pow2(p.N)) return WSFFT_ERR_INVALID_SIZE;
        p.tw = table(p.N, p.E);
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

int Plan::run(const void *in, void *out, cudaStream_t st) {
    const int64_t eb = elem_bytes(dtype);
    for (int64_t b0 = 0; b0 < batch; b0 += chunk) {
        const int64_t nb = std::min(chunk, batch - b0);
        for (const auto &p : passes) {
            const int64_t off = b0 * p.transform_elems * eb;
            const char *src = p.src == SRC_IN ? (const char *)in + off
                              : p.src == SRC_OUT ? (const char *)out + off
                                                 : (const char *)work;
            char *dst = p.dst == DST_OUT ? (char *)out + off : (char *)work;
            PassArgs a{};
            a.npencils = p.npencils_per_batch * nb;
            a.inner = p.inner;
            a.log_inner = ilog2(p.inner);
            a.tw = p.tw;
            a.conj_in = p.conj_in ? -1.f : 1.f;
            a.sx = p.scale;
            a.sy = p.conj_out ? -p.scale : p.scale;
            a.trans_rows = p.trans_rows;
            a.tw_inv = p.twid_len ? (float)(2.0 / (double)p.twid_len) : 0.f;
            a.tw_mask = p.twid_len ? (int)(p.twid_len - 1) : 0;
            prof_begin(st);
            cudaError_t e = launch(dtype, p, src, dst, a, st);
            prof_end(st);
            if (e != cudaSuccess) return e == cudaErrorInvalidValue ? WSFFT_ERR_UNSUPPORTED : WSFFT_ERR_CUDA;
        }
    }
    return WSFFT_SUCCESS;
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
    for (auto &kv : tables) cudaFree(kv.second);
    if (work) cudaFree(work);
    if (host_buf) cudaFree(host_buf);
    if (d_status) cudaFree(d_status);
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
    cudaMemset(p->d_status, 0, sizeof(int));
    int rc = p->build_schedule();
    if (rc != WSFFT_SUCCESS) {
        delete p;
        return rc;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        delete p;
        return WSFFT_ERR_CUDA;
    }
    *plan = reinterpret_cast<wsfft_plan>(p);
    return WSFFT_SUCCESS;
}

int wsfft_plan_set_norm(wsfft_plan plan, int norm) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || norm < WSFFT_NORM_PAPER || norm > WSFFT_NORM_FORWARD) return WSFFT_ERR_INVALID_ARG;
    p->norm = norm;
    return p->build_schedule();
}

int wsfft_execute(wsfft_plan plan, const void *in, void *out, wsfft_stream stream) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || !in || !out) return WSFFT_ERR_INVALID_ARG;
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return WSFFT_ERR_INVALID_ARG;
    return p->run(in, out, (cudaStream_t)stream);
}

int wsfft_execute_host(wsfft_plan plan, const void *host_in, void *host_out, wsfft_stream stream) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || !host_in || !host_out) return WSFFT_ERR_INVALID_ARG;
    const size_t bytes = (size_t)(p->batch * p->elems * elem_bytes(p->dtype));
    if (!p->host_buf) {
        if (cudaMalloc(&p->host_buf, bytes) != cudaSuccess) {
            p->host_buf = nullptr;
            return WSFFT_ERR_ALLOC;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
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
    cudaError_t e = cudaDeviceSynchronize();
    delete p;
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    return cuda_status(e);
}

int wsfft_plan_sync_status(wsfft_plan plan, wsfft_stream stream) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p) return WSFFT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaStreamSynchronize(st) != cudaSuccess) return WSFFT_ERR_CUDA;
    int h = 0;
    if (cudaMemcpy(&h, p->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return WSFFT_ERR_CUDA;
    if (h != 0) cudaMemset(p->d_status, 0, sizeof(int));
    return h == 0 ? WSFFT_SUCCESS : WSFFT_ERR_DEVICE_TIMEOUT;
}

int wsfft_plan_passes(wsfft_plan plan, int *passes, int64_t *bytes) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p) return WSFFT_ERR_INVALID_ARG;
    if (passes) *passes = (int)p->passes.size();
    if (bytes) *bytes = (int64_t)p->passes.size() * 2 * p->batch * p->elems * elem_bytes(p->dtype);
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
    if (plan) *plan = nullptr;
    (void)count; (void)dims; (void)dtype; (void)direction;
    return WSFFT_ERR_UNSUPPORTED;
}

int wsfft_execute_ragged(wsfft_plan plan, const void *const *in, void *const *out,
                         wsfft_stream stream) {
    (void)plan; (void)in; (void)out; (void)stream;
    return WSFFT_ERR_UNSUPPORTED;
}

int wsfft_autotune(wsfft_plan plan, wsfft_stream stream) {
    (void)stream;
    return plan ? WSFFT_SUCCESS : WSFFT_ERR_INVALID_ARG;
}

}  // extern "C"
