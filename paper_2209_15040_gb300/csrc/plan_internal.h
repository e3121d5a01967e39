// Library-private plan state behind the opaque wsfft_plan handle.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <utility>
#include <vector>

namespace wsfft {

enum { SRC_IN = 0, SRC_OUT = 1, SRC_WORK = 2 };
enum { DST_OUT = 0, DST_WORK = 1 };

// One superstep launch of a plan.
struct PassSpec {
    int kind;                    // PassKind
    int N, E;                    // axis length, values per thread
    bool variant;                // contiguous: transposed store; strided: four-step twiddle
    int64_t inner;               // element stride along the axis
    int64_t npencils_per_batch;  // pencils per transform
    int64_t transform_elems;     // elements per transform (batch stride)
    int src, dst;
    bool conj_in, conj_out;
    float scale;
    int64_t trans_rows;          // transposed store: rows per transform
    int64_t twid_len;            // four-step twiddle: length of the long axis
    const float2 *tw;            // device stage-twiddle table
};

struct Plan {
    int device = 0;
    int rank = 0;
    int64_t dims[3] = {1, 1, 1};
    int64_t batch = 1;
    int64_t elems = 1;  // per transform
    int dtype = 0, dir = -1, norm = 0;
    std::vector<PassSpec> passes;
    std::map<std::pair<int, int>, float2 *> tables;
    int64_t chunk = 1;        // transforms per workspace-sized chunk
    int64_t work_elems = 0;   // workspace elements needed by the schedule
    int64_t work_cap = 0;
    void *work = nullptr;
    void *host_buf = nullptr;  // device buffer for wsfft_execute_host
    int *d_status = nullptr;   // device status word (timeouts)
    std::vector<cudaEvent_t> prof_ev;  // 2 per launch slot when profiling
    int prof_used = 0;                 // launch slots recorded since the last read

    const float2 *table(int N, int E);
    int build_schedule();
    int run(const void *in, void *out, cudaStream_t st);
    // bracket one kernel launch with profiling events (no-op when off)
    void prof_begin(cudaStream_t st);
    void prof_end(cudaStream_t st);
    ~Plan();
};

}  // namespace wsfft
