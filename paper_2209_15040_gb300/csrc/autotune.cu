// wsfft_autotune: choose the schedule and the kernel shapes of a plan by
// timing them, and remember the choice.
//
// Search (greedy, a few dozen executes): every cube schedule the shape
// supports (the cluster-fused two-trip schedule, one launch per superstep,
// and the two-trip persistent, pipelined and warp-per-pencil schedules),
// then, for the fastest, each
// one-launch pass in turn over the (values per thread, pencils per block)
// shapes the library instantiates for its axis length.  Every candidate runs
// on temporary buffers of the plan's size: two warm-up executes, then the
// mean of three, timed with CUDA events on the caller's stream.
//
// Ragged plans: the tile shape of each axis length that occurs (two per
// length, kernel ragged.cuh) greedily, then the queue lag between an
// instance's supersteps (1, 2 or 4), on temporary buffers, timed the same
// way.
//
// Cache: when WSFFT_TUNE_CACHE names a file, each result is appended as one
// JSON object per line, keyed by device name, SM count, shape, batch, storage
// type, direction and normalisation (ragged plans: the sorted multiset of
// instance shapes instead of shape and batch); a later autotune (or plan
// creation) for the same key reads the choice back instead of timing.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/wsfft.h"
#include "pass_desc.h"
#include "plan_internal.h"

namespace wsfft {
namespace {

struct Choice {
    int mode = 0;
    std::vector<std::array<int, 3>> variants;  // pass, E, tile
};

std::string plan_key(const Plan &p) {
    cudaDeviceProp prop;
    std::string name = "unknown";
    if (cudaGetDeviceProperties(&prop, p.device) == cudaSuccess) name = prop.name;
    char buf[512];
    snprintf(buf, sizeof buf, "%s|sm%d|%lldx%lldx%lld|r%d|b%lld|t%d|d%d|n%d|l%d", name.c_str(), p.sm_count,
             (long long)p.dims[0], (long long)p.dims[1], (long long)p.dims[2], p.rank, (long long)p.batch,
             p.dtype, p.dir, p.norm, p.layout);
    return buf;
}

// Parse one cache line written by save(); returns false if the key differs.
bool parse_line(const std::string &line, const std::string &key, Choice &c) {
    const std::string kq = "\"key\": \"" + key + "\"";
    if (line.find(kq) == std::string::npos) return false;
    size_t m = line.find("\"mode\": ");
    if (m == std::string::npos) return false;
    c.mode = atoi(line.c_str() + m + 8);
    c.variants.clear();
    size_t v = line.find("\"variants\": [");
    if (v == std::string::npos) return true;
    const char *s = line.c_str() + v + 13;
    while (*s && *s != ']') {
        int a, b, d;
        if (sscanf(s, " [%d, %d, %d]", &a, &b, &d) == 3) c.variants.push_back({a, b, d});
        const char *e = strchr(s, ']');
        if (!e) break;
        s = e + 1;
        while (*s == ',' || *s == ' ') ++s;
    }
    return true;
}

bool load(const std::string &key, Choice &c) {
    const char *path = getenv("WSFFT_TUNE_CACHE");
    if (!path || !*path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char buf[4096];
    bool found = false;
    while (fgets(buf, sizeof buf, f)) {
        Choice t;
        if (parse_line(buf, key, t)) {
            c = t;  // the last entry for a key wins
            found = true;
        }
    }
    fclose(f);
    return found;
}

void save(const std::string &key, const Choice &c, double us) {
    const char *path = getenv("WSFFT_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "{\"key\": \"%s\", \"mode\": %d, \"variants\": [", key.c_str(), c.mode);
    for (size_t i = 0; i < c.variants.size(); ++i)
        fprintf(f, "%s[%d, %d, %d]", i ? ", " : "", c.variants[i][0], c.variants[i][1], c.variants[i][2]);
    fprintf(f, "], \"us\": %.2f}\n", us);
    fclose(f);
}

// Apply a choice (a candidate, or one read back from the cache file, whose
// contents are not trusted): values out of range, or a shape no kernel is
// instantiated for, leave the plan as it was and return an error.
int apply(Plan &p, const Choice &c) {
    if (c.mode < 0 || c.mode > 4) return WSFFT_ERR_INVALID_ARG;
    for (auto &v : c.variants)
        if (v[0] < 0 || v[1] < 1 || v[1] > 32 || (v[1] & (v[1] - 1)) || v[2] < 0) return WSFFT_ERR_INVALID_ARG;
    const int old_mode = p.engine_mode;
    const auto old_over = p.overrides;
    p.engine_mode = c.mode;
    p.overrides.clear();
    for (auto &v : c.variants) p.overrides[v[0]] = std::make_pair(v[1], v[2]);
    int rc = p.build_schedule();
    if (rc == WSFFT_SUCCESS && !p.overrides_launchable()) rc = WSFFT_ERR_UNSUPPORTED;
    if (rc != WSFFT_SUCCESS) {
        p.engine_mode = old_mode;
        p.overrides = old_over;
        p.build_schedule();
    }
    return rc;
}

// mean microseconds per execute, or a negative value if the schedule fails
double time_plan(Plan &p, const void *in, void *out, cudaStream_t st) {
    for (int i = 0; i < 2; ++i)
        if (p.run(in, out, st) != WSFFT_SUCCESS) return -1.0;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1.0;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return -1.0;
    }
    cudaEventRecord(e0, st);
    bool ok = true;
    for (int i = 0; i < 3 && ok; ++i) ok = p.run(in, out, st) == WSFFT_SUCCESS;
    cudaEventRecord(e1, st);
    float ms = -1.f;
    if (ok && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess) return -1.0;
    return ok && ms >= 0.f ? ms * 1e3 / 3.0 : -1.0;
}

// (kind, N, storage type) -> extra shapes instantiated by pass_launch.cuh
std::vector<std::pair<int, int>> shapes_for(int kind, int N, int dtype) {
    // tensor-core DFT-16 stage (16-bit storage only)
    if (kind == PASS_CONTIG && N == 512 && dtype != WSFFT_C32)
        return {{32, 16}, {32, 8}, {32, 32}, {16, 8}, {8, 8}, {16, TC_TILE}, {16, SPLIT_TILE + 8},
                {16, SPLIT_TILE + 16}, {8, SPLIT_TILE + 8}};
    if (kind == PASS_STRIDED && N == 512)
        return {{32, 16}, {32, 8},  {32, 32}, {16, 16}, {8, 8}, {16, 8}, {16, 32}, {8, PAIR_TILE + 16},
                {8, PAIR_TILE + 32}, {8, PAIR_TILE + 8}, {16, PAIR_TILE + 16}, {16, PAIR_TILE + 32},
                {16, SPLIT_TILE + 16}, {16, SPLIT_TILE + 32}, {8, SPLIT_TILE + 16}, {8, SPLIT_TILE + 32}};
    if (kind == PASS_STRIDED && N == 256) return {{16, 32}, {8, 16}, {8, PAIR_TILE + 16}};
    if (kind == PASS_STRIDED && N == 1024) return {{16, 8}, {32, 8}, {16, SPLIT_TILE + 8}};
    if (kind == PASS_CONTIG && N == 512)
        return {{32, 16}, {32, 8}, {32, 32}, {16, 8}, {8, 8}, {16, SPLIT_TILE + 8}, {16, SPLIT_TILE + 16}};
    if (kind == PASS_CONTIG && N == 256) return {{8, 8}};
    return {};
}

// -- ragged plans: the tile shape per axis length and the queue lag -------------

// Key of a ragged plan: device, storage type, direction, normalisation and
// the multiset of instance shapes (sorted, so the order of the instances
// does not matter), hashed (FNV-1a 64) with the count beside it.
std::string ragged_key(const Plan &p) {
    cudaDeviceProp prop;
    std::string name = "unknown";
    if (cudaGetDeviceProperties(&prop, p.device) == cudaSuccess) name = prop.name;
    std::vector<std::array<int64_t, 3>> shapes((size_t)p.rag_count);
    for (int i = 0; i < p.rag_count; ++i)
        for (int d = 0; d < 3; ++d) shapes[i][d] = p.rag_dims[3 * (size_t)i + d];
    std::sort(shapes.begin(), shapes.end());
    uint64_t h = 1469598103934665603ull;
    for (auto &sh : shapes)
        for (int d = 0; d < 3; ++d) {
            h ^= (uint64_t)sh[d];
            h *= 1099511628211ull;
        }
    char buf[512];
    snprintf(buf, sizeof buf, "%s|sm%d|ragged%d|%016llx|t%d|d%d|n%d", name.c_str(), p.sm_count, p.rag_count,
             (unsigned long long)h, p.dtype, p.dir, p.norm);
    return buf;
}

// the ragged choice is stored in the same line format: mode = lag,
// variants = [[-1, shape selection, 0]]
int apply_ragged(Plan &p, const Choice &c) {
    int sel = 0;
    for (auto &v : c.variants)
        if (v[0] == -1) sel = v[1];
    if (sel < 0 || sel > 15 || c.mode < 1 || c.mode > 64) return WSFFT_ERR_INVALID_ARG;
    p.rag_esel = sel;
    p.rag_lag = c.mode;
    return p.rag_build();
}

double time_ragged(Plan &p, const std::vector<const void *> &in, const std::vector<void *> &out, cudaStream_t st) {
    auto run = [&]() {
        return wsfft_execute_ragged(reinterpret_cast<wsfft_plan>(&p), in.data(), out.data(), (wsfft_stream)st) ==
               WSFFT_SUCCESS;
    };
    if (!run()) return -1.0;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1.0;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return -1.0;
    }
    cudaEventRecord(e0, st);
    bool ok = true;
    for (int i = 0; i < 3 && ok; ++i) ok = run();
    cudaEventRecord(e1, st);
    float ms = -1.f;
    if (ok && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess) return -1.0;
    return ok && ms >= 0.f ? ms * 1e3 / 3.0 : -1.0;
}

int autotune_ragged(Plan &p, cudaStream_t st) {
    const std::string key = ragged_key(p);
    Choice cached;
    // a cached choice that does not apply (out of range for this build) is
    // timed afresh
    if (load(key, cached) && apply_ragged(p, cached) == WSFFT_SUCCESS) return WSFFT_SUCCESS;
    const size_t eb = p.dtype == WSFFT_C32 ? 8 : 4;
    const size_t bytes = (size_t)p.elems * eb;
    char *in = nullptr, *out = nullptr;
    if (cudaMalloc(&in, bytes) != cudaSuccess) return WSFFT_ERR_ALLOC;
    if (cudaMalloc(&out, bytes) != cudaSuccess) {
        cudaFree(in);
        return WSFFT_ERR_ALLOC;
    }
    cudaMemsetAsync(in, 0, bytes, st);
    std::vector<const void *> ip((size_t)p.rag_count);
    std::vector<void *> op((size_t)p.rag_count);
    int present = 0;  // bit log2(N) - 5 for every axis length that occurs
    size_t off = 0;
    for (int i = 0; i < p.rag_count; ++i) {
        int64_t e = 1;
        for (int d = 0; d < 3; ++d) {
            const int64_t n = p.rag_dims[3 * (size_t)i + d];
            e *= n;
            int lg = 0;
            while ((int64_t)1 << lg < n) ++lg;
            present |= 1 << (lg - 5);
        }
        ip[i] = in + off;
        op[i] = out + off;
        off += (size_t)e * eb;  // a multiple of 16 bytes (axes >= 32)
    }
    const int saved_sel = p.rag_esel, saved_lag = p.rag_lag;
    Choice best;
    best.mode = saved_lag;
    best.variants = {{-1, saved_sel, 0}};
    double best_us = 1e300;
    auto consider = [&](int sel, int lag) {
        Choice c;
        c.mode = lag;
        c.variants = {{-1, sel, 0}};
        if (apply_ragged(p, c) != WSFFT_SUCCESS) return;
        const double us = time_ragged(p, ip, op, st);
        if (us > 0 && us < best_us) {
            best_us = us;
            best = c;
        }
    };
    consider(0, 1);
    for (int k = 0; k < 4; ++k)  // greedy: each present length's other shape
        if (present & (1 << k)) consider(best.variants[0][1] ^ (1 << k), best.mode);
    const int sel = best.variants[0][1];
    for (int lag : {2, 4}) consider(sel, lag);
    cudaStreamSynchronize(st);
    cudaFree(in);
    cudaFree(out);
    cudaGetLastError();
    if (best_us >= 1e300) {
        p.rag_esel = saved_sel;
        p.rag_lag = saved_lag;
        p.rag_build();
        return WSFFT_ERR_CUDA;
    }
    const int rc = apply_ragged(p, best);
    if (rc == WSFFT_SUCCESS) save(key, best, best_us);
    return rc;
}

}  // namespace

// Apply a cached choice at plan creation (no timing).  Returns true if one
// was applied.
bool autotune_apply_cached(Plan &p) {
    Choice c;
    if (p.ragged) {
        if (!load(ragged_key(p), c)) return false;
        return apply_ragged(p, c) == WSFFT_SUCCESS;
    }
    if (!load(plan_key(p), c)) return false;
    return apply(p, c) == WSFFT_SUCCESS;
}

}  // namespace wsfft

using namespace wsfft;

extern "C" int wsfft_autotune(wsfft_plan plan, wsfft_stream stream) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p) return WSFFT_ERR_INVALID_ARG;
    if (p->ragged) return autotune_ragged(*p, (cudaStream_t)stream);
    const std::string key = plan_key(*p);
    Choice cached;
    // a cached choice that does not apply (out of range, or a shape this
    // build does not instantiate) is timed afresh
    if (load(key, cached) && apply(*p, cached) == WSFFT_SUCCESS) return WSFFT_SUCCESS;

    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)(p->batch * p->elems * (p->dtype == WSFFT_C32 ? 8 : 4));
    void *in = nullptr, *out = nullptr;
    if (cudaMalloc(&in, bytes) != cudaSuccess) return WSFFT_ERR_ALLOC;
    if (cudaMalloc(&out, bytes) != cudaSuccess) {
        cudaFree(in);
        return WSFFT_ERR_ALLOC;
    }
    cudaMemsetAsync(in, 0, bytes, st);

    const int saved_mode = p->engine_mode;
    const auto saved_over = p->overrides;
    Choice best;
    double best_us = 1e300;
    for (int mode : {4, 0, 1, 2, 3}) {
        Choice c;
        c.mode = mode;
        if (apply(*p, c) != WSFFT_SUCCESS) continue;
        // a mode the shape does not support falls back to mode 0's schedule
        if (mode != 0 && p->passes.size() != 2) continue;
        const double us = time_plan(*p, in, out, st);
        if (us > 0 && us < best_us) {
            best_us = us;
            best = c;
        }
    }
    // per-pass shapes of the one-launch passes, greedily
    if (apply(*p, best) == WSFFT_SUCCESS) {
        const size_t np = p->passes.size();
        for (size_t i = 0; i < np; ++i) {
            const PassSpec ps = p->passes[i];
            if (ps.kind != PASS_CONTIG && ps.kind != PASS_STRIDED) continue;
            for (auto sh : shapes_for(ps.kind, ps.N, p->dtype)) {
                Choice c = best;
                c.variants.push_back({(int)i, sh.first, sh.second});
                if (apply(*p, c) != WSFFT_SUCCESS) continue;
                const double us = time_plan(*p, in, out, st);
                if (us > 0 && us < best_us) {
                    best_us = us;
                    best = c;
                }
            }
        }
    }
    cudaStreamSynchronize(st);
    cudaFree(in);
    cudaFree(out);
    cudaGetLastError();
    if (best_us >= 1e300) {
        p->engine_mode = saved_mode;
        p->overrides = saved_over;
        p->build_schedule();
        return WSFFT_ERR_CUDA;
    }
    const int rc = apply(*p, best);
    if (rc == WSFFT_SUCCESS) save(key, best, best_us);
    return rc;
}
