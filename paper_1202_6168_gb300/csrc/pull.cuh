// pull.cuh - gather (pull) form of y = P w over the in-edges: y_k = sum of w_j
// over the in-edges j -> k, where w_j already carries the scale d/outdeg_j.
//
// Rows are binned by in-degree at graph creation so that each bin gets a
// matched mapping, every task carries a bounded amount of work, and the
// column indices stream coalesced while the gathers of w stay independent:
//   bin 1: 0..8 in-edges      256 rows per task  } edges copied contiguously in
//   bin 2: 9..32              64 rows per task   } bin order; a CTA stages the
//                                                  task's <= 2048 gathered values
//                                                  in shared memory, then one
//                                                  thread (bin 1) or 4 lanes
//                                                  (bin 2) sum each row
//   bin 3: 33..256            one warp per row (8 rows per task)
//   bin 4: 257..4096          one CTA per row
//   bin 5: > 4096             one CTA per 4096-edge segment of a row
// Rows of bins 1-4 are reduced by one owner in a fixed order (deterministic);
// a segment of bin 5 hands its partial to a per-mode handler.
#pragma once

#include "di_internal.cuh"

namespace di {

constexpr int kPullThreads = 256;
constexpr int kBin1Max = 8, kBin2Max = 32, kBin3Max = 256, kBin4Max = 4096;
constexpr int kPullSeg = 4096;

// Device view of the binned row plan (passed by value to kernels).
struct PullPlan {
    const int32_t *rows;      // bins 1..4 concatenated: row ids, ascending within a bin
    const int32_t *b12_off;   // bins 1-2: edge offsets in bin order [bin_off[2] + 1]
    const int32_t *b12_col;   // bins 1-2: in-edge sources, contiguous in bin order
    int64_t bin_off[5];       // bin b (1..4) = rows[bin_off[b-1] .. bin_off[b])
    int64_t task_off[6];      // bin b (1..5) tasks = [task_off[b-1], task_off[b])
    const int32_t *seg_row;   // bin 5: row of each segment
    const int32_t *seg_beg;   // bin 5: first in-edge of each segment
};

// Runs every task of the plan on this CTA's share (grid-stride).
//   emit(row, acc): called by exactly one thread per row of bins 1-4;
//   seg(s, row, acc): called by thread 0 of the CTA for segment s of bin 5.
// All threads of the CTA must call this (bins 4 and 5 use block reductions).
template <typename VT, typename Emit, typename Seg>
__device__ __forceinline__ void pull_plan(const PullPlan &pl, const int32_t *__restrict__ in_rp,
                                          const int32_t *__restrict__ in_col, const VT *__restrict__ w, Emit &emit,
                                          Seg &seg) {
    constexpr int kStage = 2048;            // values staged per CTA task of bins 1-2
    __shared__ VT s_val[kStage];
    __shared__ int32_t s_off[kPullThreads + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t ntasks = pl.task_off[5];
    for (int64_t task = blockIdx.x; task < ntasks; task += gridDim.x) {
        if (task < pl.task_off[2]) {                               // bins 1-2: staged in shared memory
            const bool b1 = task < pl.task_off[1];
            const int per = b1 ? kPullThreads : kPullThreads / 4;
            const int64_t i0 = b1 ? pl.bin_off[0] + (task - pl.task_off[0]) * per
                                  : pl.bin_off[1] + (task - pl.task_off[1]) * per;
            const int64_t iend = b1 ? pl.bin_off[1] : pl.bin_off[2];
            const int cnt = (int)(iend - i0 < per ? iend - i0 : per);
            for (int r = tid; r <= cnt; r += kPullThreads) s_off[r] = __ldcs(pl.b12_off + i0 + r);
            __syncthreads();
            const int32_t e0 = s_off[0];
            const int ne = s_off[cnt] - e0;                        // <= 2048 by construction
#pragma unroll
            for (int k = 0; k < kStage / kPullThreads; ++k) {
                const int e = tid + k * kPullThreads;
                if (e < ne) s_val[e] = w[__ldcs(pl.b12_col + e0 + e)];
            }
            __syncthreads();
            if (b1) {
                if (tid < cnt) {
                    const int a = s_off[tid] - e0, z = s_off[tid + 1] - e0;
                    VT acc = VT(0);
                    for (int e = a; e < z; ++e) acc += s_val[e];
                    emit(__ldcs(pl.rows + i0 + tid), acc);
                }
            } else {
                const int r = tid >> 2, sub = tid & 3;
                VT acc = VT(0);
                if (r < cnt) {
                    const int a = s_off[r] - e0, z = s_off[r + 1] - e0;
                    for (int e = a + sub; e < z; e += 4) acc += s_val[e];
                }
                acc += __shfl_xor_sync(0xffffffffu, acc, 1, 4);
                acc += __shfl_xor_sync(0xffffffffu, acc, 2, 4);
                if (r < cnt && sub == 0) emit(__ldcs(pl.rows + i0 + r), acc);
            }
            __syncthreads();
        } else if (task < pl.task_off[3]) {                        // bin 3: warp per row
            const int64_t idx = pl.bin_off[2] + (task - pl.task_off[2]) * (kPullThreads / 32) + warp;
            if (idx < pl.bin_off[3]) {
                const int32_t row = pl.rows[idx];
                const int32_t b = __ldcs(in_rp + row), e = __ldcs(in_rp + row + 1);
                VT acc = VT(0);
#pragma unroll
                for (int k = 0; k < kBin3Max / 32; ++k) {
                    const int32_t q = b + lane + 32 * k;
                    if (q < e) acc += w[__ldcs(in_col + q)];
                }
                acc = warp_sum(acc);
                if (lane == 0) emit(row, acc);
            }
        } else if (task < pl.task_off[4]) {                        // bin 4: CTA per row
            const int32_t row = pl.rows[pl.bin_off[3] + (task - pl.task_off[3])];
            const int32_t b = __ldcs(in_rp + row), e = __ldcs(in_rp + row + 1);
            VT acc = VT(0);
#pragma unroll 4
            for (int32_t q = b + tid; q < e; q += kPullThreads) acc += w[__ldcs(in_col + q)];
            double s = static_cast<double>(acc), m = 0.0;
            block_sum_max<kPullThreads>(s, m);
            if (tid == 0) emit(row, static_cast<VT>(s));
        } else {                                                   // bin 5: CTA per segment
            const int64_t sgi = task - pl.task_off[4];
            const int32_t row = pl.seg_row[sgi];
            const int32_t b = pl.seg_beg[sgi];
            const int32_t end = __ldcs(in_rp + row + 1);
            const int32_t e = b + kPullSeg < end ? b + kPullSeg : end;
            VT acc = VT(0);
#pragma unroll 4
            for (int32_t q = b + tid; q < e; q += kPullThreads) acc += w[__ldcs(in_col + q)];
            double s = static_cast<double>(acc), m = 0.0;
            block_sum_max<kPullThreads>(s, m);
            if (tid == 0) seg(sgi, row, static_cast<VT>(s));
        }
    }
}

// The plan of a graph (device pointers and offsets).
PullPlan pull_plan_of(const di_graph *g);

}  // namespace di
