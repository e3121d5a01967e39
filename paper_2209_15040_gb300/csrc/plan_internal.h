// Library-private plan state behind the opaque wsfft_plan handle.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <utility>
#include <vector>

namespace wsfft {

struct PassArgs;

enum { SRC_IN = 0, SRC_OUT = 1, SRC_WORK = 2 };
enum { DST_OUT = 0, DST_WORK = 1 };

// One superstep launch of a plan.
struct PassSpec {
    int kind;                    // PassKind
    int N, E;                    // axis length, values per thread
    int tile;                    // 0 = default tile shape, else pencils per block
    bool variant;                // contiguous: transposed store; strided: four-step twiddle
    int64_t inner;               // element stride along the axis
    int64_t npencils_per_batch;  // pencils per transform
    int64_t transform_elems;     // elements per transform (batch stride)
    int src, dst;
    bool conj_in, conj_out;
    float scale;
    int64_t trans_rows;          // transposed store: rows per transform
    int64_t twid_len;            // four-step twiddle: length of the long axis
    int twid_shift;              // four-step twiddle: bits of the low table index
    const float2 *tw;            // device stage-twiddle table
    const float2 *tw2;           // fused passes: table of the strided tiles, if it differs
    // persistent engine passes (kind PASS_ENGINE_A / PASS_ENGINE_B, PASS_PERSIST_A,
    // PASS_WP_A) and the cluster-fused pass A (PASS_SLAB_A: c_scale, s_scale)
    const void *items;           // device item table
    int nitems;
    int64_t units;               // completion counters used (pass A)
    float c_scale, s_scale;      // pass A: scale after the contiguous / strided superstep
    bool reverse;                // strided: tiles taken from the last one down
};

struct Plan {
    int device = 0;
    int rank = 0;
    int64_t dims[3] = {1, 1, 1};
    int64_t batch = 1;
    int64_t elems = 1;  // per transform
    int64_t axis_inner = 0;  // > 0: a plan of wsfft_plan_create_axis (one axis of length dims[0], stride axis_inner)
    int dtype = 0, dir = -1, norm = 0;
    std::vector<PassSpec> passes;
    std::map<int, std::pair<int, int>> overrides;  // pass index -> (E, tile)
    std::map<std::pair<int, int>, float2 *> tables;
    int64_t chunk = 1;        // transforms per workspace-sized chunk
    int64_t work_elems = 0;   // workspace elements needed by the schedule
    int64_t work_cap = 0;
    void *work = nullptr;
    void *host_buf = nullptr;  // device buffer for wsfft_execute_host
    cudaStream_t copy_stream = nullptr;      // wsfft_execute_host: host-to-device copies overlapping the supersteps
    cudaStream_t copy_out_stream = nullptr;  // and the device-to-host copies, on their own stream
    std::vector<cudaEvent_t> pipe_ev;
    int *d_status = nullptr;   // device status word (timeouts)
    cudaStream_t setup_st = nullptr;  // plan-owned stream for table uploads (synchronised per upload)
    std::map<cudaStream_t, cudaEvent_t> done_ev;  // per execute stream: recorded after the plan's last launch
    // persistent engine state
    int sm_count = 0;
    int eng_grid = 0;
    int layout = 0;                // wsfft_layout of the spectral side
    int engine_mode = 0;           // 0 one launch per superstep, 1 persistent, 2 pipelined, 3 warp-per-pencil,
                                   // 4 cluster-fused pass A
    int persist_grid = 0;          // persistent kernel blocks (all resident)
    void *d_items = nullptr;       // item tables of passes A and B
    uint32_t *d_ctr = nullptr;     // ticket and completion counters
    int64_t ctr_cap = 0;
    int64_t wait_timeout_ns = 1000000000;  // 1 s per bounded wait
    // ragged plans
    bool ragged = false;
    int rag_count = 0;
    int rag_grid = 0;
    int rag_nitems = 0;
    void *rag_items = nullptr;      // device RagItem table
    void *rag_inst = nullptr;       // device RagInst table
    void *rag_inst_host = nullptr;  // pinned host copy (pointers filled per execute)
    cudaEvent_t rag_copied = nullptr;
    bool rag_uploaded = false;
    const float2 *rag_tw[4][2] = {};  // stage tables per length 32..256 and tile shape
    std::vector<int64_t> rag_dims;     // count x 3 axis lengths
    int rag_esel = 0;                  // bit log2(N) - 5: length N uses its second tile shape
    int rag_lag = 1;                   // queue distance (instances) between an instance's supersteps
    int64_t rag_items_cap = 0;
    bool withhold = false;         // testing: drop one completion signal
    std::vector<cudaEvent_t> prof_ev;  // 2 per launch slot when profiling
    int prof_used = 0;                 // launch slots recorded since the last read

    const float2 *table(int N, int E);
    PassArgs pass_args(const PassSpec &p, int64_t npencils) const;
    const float2 *tc_table(int N);  // tensor-core contiguous superstep (tc_contig.cuh)
    std::map<int64_t, float2 *> fs_tables;        // four-step twiddle tables per long length
    const float2 *fourstep_table(int64_t L, int shift);
    int build_schedule();
    bool overrides_launchable() const;  // every pass-shape override names an instantiated kernel
    int build_engine(int64_t n0, int64_t n, bool inv);
    int build_slab(int64_t n0, int64_t n, bool inv);
    int rag_build();                   // ragged plans: instance records and tile queue
    bool slab_runs(int n);             // cluster-fused pass A resident on this device
    int slab_checked[2] = {0, 0};      // per slab edge 256 / 512: 0 unknown, 1 yes, -1 no
    int run(const void *in, void *out, cudaStream_t st);
    // host-to-device copy / zero fill on the plan's own stream, complete on
    // return (visible to kernels on any stream); a wsfft_status
    int upload(void *dst, const void *src, size_t bytes);
    int zero(void *dst, size_t bytes);
    // remember that the plan's work on `st` ends here (skipped while `st` is
    // being captured into a graph)
    void mark_done(cudaStream_t st);
    // wait for every execute of this plan and its own streams; a wsfft_status
    int wait_own_work();
    bool can_pipeline_host() const;
    int run_host_pipelined(const void *hin, void *hout, cudaStream_t st);
    // bracket one kernel launch with profiling events (no-op when off)
    void prof_begin(cudaStream_t st);
    void prof_end(cudaStream_t st);
    ~Plan();
};

// Apply a choice remembered by wsfft_autotune for this plan's key (no
// timing); true if one was applied.
bool autotune_apply_cached(Plan &p);

}  // namespace wsfft
