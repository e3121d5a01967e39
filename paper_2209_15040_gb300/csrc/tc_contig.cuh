// Tensor-core superstep along the contiguous axis for 16-bit storage,
// N = 512 (FP16 or BF16 complex, interleaved re/im).
//
// The pencil is split as n = 32*n1 + n2, k = k1 + 16*k2 (Cooley-Tukey with
// N1 = 16, N2 = 32; Section 3.1 builds the transform from such stages):
//   Y[k1][n2] = sum_n1 x[32*n1 + n2] w16^(n1*k1)                 (DFT-16)
//   X[k1 + 16*k2] = sum_n2 (w512^(n2*k1) Y[k1][n2]) w32^(n2*k2)    (DFT-32)
// The DFT-16 of every n2 is one dense product, computed on the tensor cores
// (tcgen05.mma kind::f16, FP32 accumulation in tensor memory):
//   A (M x K) = the pencil as stored: K = n1 indexes the 128-byte rows
//       (32 complex = 64 16-bit values each), M = (n2, re/im) runs along
//       the row, two pencils per M = 128 -- a TMA load with 128-byte swizzle
//       puts a tile of pencils in exactly this MN-major operand layout;
//   B (K x N) = [Re w16^(n1*k1), Im w16^(n1*k1)] over N = (k1, re/im) = 32,
//       split into a 16-bit high part and the 16-bit remainder (two MMAs
//       accumulate A*B_hi + A*B_lo, so the DFT-16 matrix is effectively
//       exact to ~2^-22; A is exact because it is the stored data).
// Row (n2, re) of D holds sum x_re * (Re w, Im w) and row (n2, im) holds
// sum x_im * (Re w, Im w); adjacent lanes combine them into Y with one
// shuffle per value.  The DFT-32 runs in registers (one thread per (pencil,
// k1)) after an exchange through shared memory, with the w512 twiddles of
// the host table.  The data path in FP32 is the same as the SIMT kernels'.
//
// Persistent, warp-specialized, one block per SM walking the tiles (8
// pencils, 16 KB each) with a stride of the grid.  The last warp is the
// producer: one lane keeps TC_STAGES TMA loads in flight and issues each
// tile's MMAs into the tensor-memory accumulator of the consumer group that
// owns the tile.  TC_GROUPS groups of four consumer warps take the tiles in
// turn (tile i of the block -> group i mod TC_GROUPS); a group reads its
// accumulator, combines it into its Y buffer in shared memory, releases the
// accumulator and runs the DFT-32 and the stores while the other groups and
// the tensor cores work on the next tiles.  mbarriers order everything: full[s] (TMA landed),
// empty[s] (the MMAs that read stage s are done), dfull[g] (accumulator g
// written), dempty[g] (accumulator g read by the group's four warps).  Every
// wait is bounded by the plan's timeout; on expiry the block records the
// failure in the status word, stops, waits (bounded) for the copies and MMAs
// it issued, frees its tensor memory and returns.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fft_core.cuh"
#include "pass_desc.h"
#include "tc.cuh"

namespace wsfft {

template <class S>
struct TcElem;
template <>
struct TcElem<__half2> {
    static constexpr bool BF16 = false;
};
template <>
struct TcElem<__nv_bfloat162> {
    static constexpr bool BF16 = true;
};

constexpr int TC_P = 8;                            // pencils per tile
constexpr int TC_STAGES = 8;                       // input ring depth
constexpr int TC_GROUPS = 2;                       // consumer groups (4 warps each)
constexpr int TC_TILE_BYTES = TC_P * 2048;         // 16 KB
constexpr int TC_YROW = 33;                        // float2 per padded Y row (32 + 1)
constexpr int TC_YBYTES = 34816;                   // one group's Y buffer (8 x 16 x 33 float2, rounded)
constexpr int TC_OFF_Y = TC_STAGES * TC_TILE_BYTES;              // 96 KB
constexpr int TC_OFF_B = TC_OFF_Y + TC_GROUPS * TC_YBYTES;       // B_hi, B_lo (1 KB each)
constexpr int TC_OFF_BAR = TC_OFF_B + 2048;                      // mbarriers, TMEM slot, flag
constexpr int TC_SMEM = TC_OFF_BAR + 256 + 1024;                 // + alignment slack
constexpr int TC_COLS = 512;                       // TC_GROUPS accumulators of 4 pairs x 32 columns
constexpr int TC_THREADS = 128 * TC_GROUPS + 32;   // consumer groups + 1 producer warp
static_assert(TC_P * 16 * TC_YROW * 8 <= TC_YBYTES, "Y buffer");
static_assert(TC_GROUPS * 128 <= TC_COLS, "accumulators fit in tensor memory");
static_assert(TC_SMEM <= 227 * 1024, "shared memory");

// barrier over one consumer group (named barrier 1 + g) that also returns
// whether any thread of the group passed v
__device__ __forceinline__ bool group_any(bool v, int g) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\t"
        "setp.ne.u32 pi, %1, 0;\n\t"
        "bar.red.or.pred po, %2, 128, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(1 + g)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void group_bar(int g) {
    asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory");
}

template <class S>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_contig512_kernel(const __grid_constant__ CUtensorMap tmap, S *__restrict__ out, PassArgs a) {
    extern __shared__ uint8_t tc_raw[];
    const uint32_t raw0 = smem_addr(tc_raw);
    uint8_t *sm = tc_raw + (((raw0 + 1023u) & ~1023u) - raw0);  // 1024-aligned (swizzle atoms)
    uint8_t *B = sm + TC_OFF_B;
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + TC_OFF_BAR);  // [TC_STAGES]
    uint64_t *empty = full + TC_STAGES;                                // [TC_STAGES]
    uint64_t *dfull = empty + TC_STAGES;                               // [TC_GROUPS]
    uint64_t *dempty = dfull + TC_GROUPS;                              // [TC_GROUPS]
    uint32_t *slot = reinterpret_cast<uint32_t *>(dempty + TC_GROUPS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t ntiles = (a.npencils + TC_P - 1) / TC_P;
    const int64_t mine = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint64_t tmo = a.timeout_ns;

    if (tid == 0) {
        for (int i = 0; i < TC_STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < TC_GROUPS; ++i) {
            mbar_init(&dfull[i], 1);
            mbar_init(&dempty[i], 4);
        }
        *abort_flag = 0;
    }
    if (warp == 0) tc_alloc(slot, TC_COLS);
    if (tid < 128) reinterpret_cast<uint4 *>(B)[tid] = __ldg(reinterpret_cast<const uint4 *>(a.tw) + tid);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;

    if (warp == 4 * TC_GROUPS) {
        // ---------------- producer ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = tc_idesc_f16(TcElem<S>::BF16, true, false, 128, 32);
            const uint64_t bh = tc_sdesc(smem_addr(B), 128, 256, TC_LAYOUT_NONE);
            const uint64_t bl = tc_sdesc(smem_addr(B + 1024), 128, 256, TC_LAYOUT_NONE);
            int64_t issued = 0;  // tiles whose TMA load was issued
            for (; issued < mine && issued < TC_STAGES; ++issued) {
                const int64_t tile = blockIdx.x + issued * gridDim.x;
                mbar_arrive_expect_tx(&full[issued], TC_TILE_BYTES);
                tma_load_2d(sm + issued * TC_TILE_BYTES, &tmap, 0, (int)(tile * TC_P * 16), &full[issued]);
            }
            int64_t mma_done_upto = 0;  // tiles whose MMAs were committed
            bool ok = true;
            for (int64_t it = 0; it < mine; ++it) {
                const int s = (int)(it % TC_STAGES), g = (int)(it % TC_GROUPS);
                if (!mbar_wait_deadline(&full[s], (uint32_t)((it / TC_STAGES) & 1), gtimer() + tmo)) ok = false;
                if (ok && it >= TC_GROUPS &&
                    !mbar_wait_deadline(&dempty[g], (uint32_t)((it / TC_GROUPS - 1) & 1), gtimer() + tmo))
                    ok = false;
                if (!ok || *abort_flag) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                uint8_t *st = sm + s * TC_TILE_BYTES;
#pragma unroll
                for (int j = 0; j < TC_P / 2; ++j) {
                    const uint64_t ad = tc_sdesc(smem_addr(st + j * 4096), 2048, 1024, TC_LAYOUT_SW128);
                    tc_mma_f16(tmem + g * 128 + 32 * j, ad, bh, idesc, 0);
                    tc_mma_f16(tmem + g * 128 + 32 * j, ad, bl, idesc, 1);
                }
                tc_commit(&dfull[g]);
                tc_commit(&empty[s]);
                mma_done_upto = it + 1;
                if (issued < mine) {
                    // refill stage s once the MMAs that read it are done
                    if (!mbar_wait_deadline(&empty[s], (uint32_t)((it / TC_STAGES) & 1), gtimer() + tmo)) {
                        ok = false;
                        break;
                    }
                    const int64_t tile = blockIdx.x + issued * gridDim.x;
                    mbar_arrive_expect_tx(&full[s], TC_TILE_BYTES);
                    tma_load_2d(st, &tmap, 0, (int)(tile * TC_P * 16), &full[s]);
                    ++issued;
                }
            }
            if (!ok) {
                atomicExch(a.status, 1);
                *abort_flag = 1;
                // drain: every load issued but not consumed, each wait bounded
                for (int64_t t = mma_done_upto; t < issued; ++t)
                    mbar_wait_deadline(&full[t % TC_STAGES], (uint32_t)((t / TC_STAGES) & 1), gtimer() + tmo);
            }
            if (mma_done_upto > 0) {  // the last MMA group (commits complete in order)
                const int64_t t = mma_done_upto - 1;
                mbar_wait_deadline(&empty[t % TC_STAGES], (uint32_t)((t / TC_STAGES) & 1), gtimer() + tmo);
            }
        }
    } else {
        // ---------------- consumer group g: tiles g, g + TC_GROUPS, ... ----------------
        const int g = warp >> 2, wq = warp & 3;  // wq: the group warp, tensor-memory lanes 32*wq..
        const int gt = tid & 127;
        float *Yf = reinterpret_cast<float *>(sm + TC_OFF_Y + g * TC_YBYTES);
        const float sgn = a.conj_in;  // -1: the input is conjugated (negates x_im)
        const int c = lane & 1;
        const float al = c ? sgn : 1.f, be = c ? 1.f : -sgn;
        const int m = 32 * wq + lane;
        const int n2 = (m & 63) >> 1;
        const int p2 = gt >> 4, k1 = gt & 15;  // DFT-32 task: (pencil, k1)
        const float2 *tw = a.tw + TC_TABLE_TW + k1;  // [n2][k1]: a warp's 16 k1 share one line
        for (int64_t it = g; it < mine; it += TC_GROUPS) {
            const bool ok = mbar_wait_deadline(&dfull[g], (uint32_t)((it / TC_GROUPS) & 1), gtimer() + tmo);
            if (!ok) {
                atomicExch(a.status, 1);
                *abort_flag = 1;
            }
            // one decision for the group's four warps (a barrier over them)
            if (group_any(!ok || *abort_flag != 0, g)) break;
            tc_fence_after();
#pragma unroll
            for (int j = 0; j < TC_P / 2; ++j) {
                uint32_t r[32];
                tc_ld_32x32b_x32(tmem + ((uint32_t)(32 * wq) << 16) + g * 128 + 32 * j, r);
                const int p = 2 * j + (m >> 6);
                float *dst = Yf + ((p * 16) * TC_YROW + n2) * 2 + c;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float mv = __uint_as_float(r[2 * q]);
                    const float ov = __shfl_xor_sync(0xffffffffu, __uint_as_float(r[2 * q + 1]), 1);
                    // even lane: Re Y = sum x_re Re w - s sum x_im Im w;
                    // odd lane:  Im Y = s sum x_im Re w + sum x_re Im w
                    dst[q * TC_YROW * 2] = fmaf(mv, al, ov * be);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&dempty[g]);
            group_bar(g);  // Y complete
            const float2 *row = reinterpret_cast<const float2 *>(Yf) + (p2 * 16 + k1) * TC_YROW;
            float2 x[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) x[q] = row[q];
            group_bar(g);  // Y free for the group's next tile
#pragma unroll
            for (int q = 1; q < 32; ++q) x[q] = cmul(x[q], __ldg(&tw[q * 16]));
            dft<32>(x);
            const int64_t pencil = (blockIdx.x + it * gridDim.x) * TC_P + p2;
            if (pencil < a.npencils) {
                S *o = out + pencil * 512 + k1;
#pragma unroll
                for (int k2 = 0; k2 < 32; ++k2)
                    Cvt<S>::template store<OP_DEF>(o + 16 * k2, make_float2(x[k2].x * a.sx, x[k2].y * a.sy));
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tc_dealloc(tmem, TC_COLS);
    }
}

}  // namespace wsfft
