// residual.cu - exact FP64 residual F = B + P H - H.
//
// Eqs. defF/defH imply that F_n + H_n - P H_n does not change with n, so
// F_n = B + P H_n - H_n for a cold start (and for any H_0 with
// F_0 = B + P H_0 - H_0).  Recomputing F from H this way in FP64 removes the
// rounding that FP32 pushes accumulate, gives the exact stopping residual
// |F|_1, and forms the warm-start fluid F_0.
//
// (P H)_k = sum over in-edges j -> k of g_j, g_j = (d / outdeg_j) H_j, in
// one of two forms:
//   source-blocked (default): the in-edges ordered by block of 2^22 sources,
//     then by destination, so that the grid gathers from one 32 MB block of
//     g at a time (L2-resident); runs of equal destination are summed per
//     thread and added with FP64 reds (k_resb_*);
//   binned: a gather over the transpose with the binned pull plan of
//     pull.cuh, with no atomics and a fixed summation order per graph object
//     (rows longer than 4096 in-edges are summed in segments whose partials
//     are added in order) (k_res_*).
#include <algorithm>

#include "di_internal.cuh"
#include "pull.cuh"

namespace di {
namespace {

__device__ void res_control(const SolveDesc *__restrict__ desc, SolveState *__restrict__ st, int mode, double s,
                            double m);

__global__ void __launch_bounds__(kResThreads) k_res_prep(const SolveDesc *__restrict__ desc,
                                                          const SolveState *__restrict__ st, int mode,
                                                          const double *__restrict__ s64,
                                                          double *__restrict__ g, int64_t n) {
    if (mode == RES_LEVEL && !st->do_recompute) return;
    const double *__restrict__ H = desc->H;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) g[i] = s64[i] * H[i];
}

// Rows of bins 1-5 of the pull plan: F = B + P H - H written by the row's
// owner; segments of the longest rows leave their partial sums in seg_part
// for k_res_long.
template <typename FT>
__global__ void __launch_bounds__(kPullThreads, 4) k_res_pull(const PullPlan pl, const SolveDesc *__restrict__ desc,
                                                           const SolveState *__restrict__ st,
                                                           const int32_t *__restrict__ in_rp,
                                                           const int32_t *__restrict__ in_col,
                                                           const double *__restrict__ g,
                                                           double *__restrict__ seg_part,
                                                           double *__restrict__ part_sum,
                                                           double *__restrict__ part_max, int mode) {
    if (mode == RES_LEVEL && !st->do_recompute) return;   // host-driven levels launch it every time
    const double *__restrict__ B = desc->B;
    const double *__restrict__ H = desc->H;
    FT *__restrict__ Ffl = (mode == RES_LEVEL || mode == RES_WARM_INIT) ? static_cast<FT *>(desc->F) : nullptr;
    double *__restrict__ F64 = mode == RES_WARM_INIT ? nullptr : desc->F_out;
    double lsum = 0.0, lmax = 0.0;
    auto emit = [&](int32_t k, double acc) {
        const double f = B[k] + acc - H[k];
        if (Ffl) Ffl[k] = static_cast<FT>(f);
        if (F64) F64[k] = f;
        const double a = fabs(f);
        lsum += a;
        lmax = fmax(lmax, a);
    };
    auto seg = [&](int64_t s, int32_t, double acc) { seg_part[s] = acc; };
    pull_plan<double>(pl, in_rp, in_col, g, emit, seg);
    block_sum_max<kPullThreads>(lsum, lmax);
    if (threadIdx.x == 0) {
        part_sum[blockIdx.x] = lsum;
        part_max[blockIdx.x] = lmax;
    }
}

// Rows longer than kPullSeg: one warp adds a row's segment partials in
// segment order, then the last CTA combines every CTA partial of both
// kernels (in a fixed order) and runs the control step of the mode.
template <typename FT>
__global__ void __launch_bounds__(kResThreads) k_res_long(
    const SolveDesc *__restrict__ desc, SolveState *__restrict__ st, const int32_t *__restrict__ lrows,
    const int32_t *__restrict__ lseg0, int n_long, const double *__restrict__ seg_part,
    double *__restrict__ part_sum, double *__restrict__ part_max, int pull_blocks, int mode) {
    if (mode == RES_LEVEL && !st->do_recompute) return;
    const double *__restrict__ B = desc->B;
    const double *__restrict__ H = desc->H;
    FT *__restrict__ Ffl = (mode == RES_LEVEL || mode == RES_WARM_INIT) ? static_cast<FT *>(desc->F) : nullptr;
    double *__restrict__ F64 = mode == RES_WARM_INIT ? nullptr : desc->F_out;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double lsum = 0.0, lmax = 0.0;
    for (int64_t r = warp; r < n_long; r += nwarps) {
        const int32_t s0 = lseg0[r], s1 = lseg0[r + 1];
        double part = 0.0;
        for (int32_t s = s0 + lane; s < s1; s += 32) part += seg_part[s];
        part = warp_sum(part);
        if (lane == 0) {
            const int32_t k = lrows[r];
            const double f = B[k] + part - H[k];
            if (Ffl) Ffl[k] = static_cast<FT>(f);
            if (F64) F64[k] = f;
            lsum += fabs(f);
            lmax = fmax(lmax, fabs(f));
        }
    }
    block_sum_max<kResThreads>(lsum, lmax);
    if (threadIdx.x == 0) {
        part_sum[pull_blocks + blockIdx.x] = lsum;
        part_max[pull_blocks + blockIdx.x] = lmax;
    }
    if (!last_block(&st->res_blocks)) return;
    // last block: deterministic combination of the partials of both kernels
    const int total = pull_blocks + gridDim.x;
    double s = 0.0, m = 0.0;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        s += part_sum[i];
        m = fmax(m, part_max[i]);
    }
    block_sum_max<kResThreads>(s, m);
    if (threadIdx.x != 0) return;
    res_control(desc, st, mode, s, m);
}

// ------------------------------------------------------------------ source-blocked form

// acc = B - H and g = (d / outdeg) H.  With the 1/N completion of dangling
// columns (Sec. 2.2) the sum of H over the dangling nodes (s = 0) goes to
// st->dang_h, one FP64 atomic per CTA.
__global__ void __launch_bounds__(kResThreads) k_resb_init(const SolveDesc *__restrict__ desc,
                                                           SolveState *__restrict__ st, int mode,
                                                           const double *__restrict__ s64, double *__restrict__ g,
                                                           double *__restrict__ acc, int64_t n) {
    if (mode == RES_LEVEL && !st->do_recompute) return;
    const double *__restrict__ B = desc->B;
    const double *__restrict__ H = desc->H;
    const bool dang = desc->dangling != 0;
    double hd = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double h = H[i];
        const double s = s64[i];
        g[i] = s * h;
        acc[i] = B[i] - h;
        if (dang && s == 0.0) hd += h;
    }
    if (dang) {
        double dummy = 0.0;
        block_sum_max<kResThreads>(hd, dummy);
        if (threadIdx.x == 0 && hd != 0.0) atomicAdd(&st->dang_h, hd);
    }
}

// acc_k += g_j over the in-edges j -> k, taken in source-blocked order: at any
// time the grid works inside one block of 2^22 sources, whose 32 MB of g stay
// in L2 while the edge arrays stream.  8 consecutive edges per thread (two
// int4 loads of each index array, 8 independent gathers; few registers, so
// 6 CTAs of 256 fit per SM to hide the latency).  Runs of equal destination
// are summed in registers, and the runs that cross lane boundaries are summed
// over the warp before their red.global.add.f64 (warp_runs_add): a
// destination of very high in-degree (a hub, up to millions of in-edges)
// would otherwise take one reduction per thread, all on one L2 address at the
// same time.
constexpr int kResbEdges = 8;

__global__ void __launch_bounds__(kResThreads, 6) k_resb_flat(const SolveState *__restrict__ st, int mode,
                                                              const int32_t *__restrict__ bcol,
                                                              const int32_t *__restrict__ brow,
                                                              const double *__restrict__ g, double *__restrict__ acc,
                                                              int64_t nnz) {
    if (mode == RES_LEVEL && !st->do_recompute) return;
    constexpr int kE = kResbEdges;
    const int lane = threadIdx.x & 31;
    const int64_t nch = (nnz + kE - 1) / kE;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // warp-uniform loop: the chunks of a warp are consecutive, lanes past the
    // end hold no edge (destination -1) and still take part in the shuffles
    for (int64_t c0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); c0 < nch; c0 += stride) {
        const int64_t e0 = (c0 + lane) * kE;
        int32_t col[kE], row[kE];
        if (e0 + kE <= nnz) {
#pragma unroll
            for (int v = 0; v < kE / 4; ++v) {
                const int4 a = __ldcs(reinterpret_cast<const int4 *>(bcol + e0) + v);
                const int4 b = __ldcs(reinterpret_cast<const int4 *>(brow + e0) + v);
                col[4 * v] = a.x; col[4 * v + 1] = a.y; col[4 * v + 2] = a.z; col[4 * v + 3] = a.w;
                row[4 * v] = b.x; row[4 * v + 1] = b.y; row[4 * v + 2] = b.z; row[4 * v + 3] = b.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < kE; ++k) {
                const bool ok = e0 + k < nnz;
                col[k] = ok ? bcol[e0 + k] : 0;
                row[k] = ok ? brow[e0 + k] : -1;
            }
        }
        double val[kE];
#pragma unroll
        for (int k = 0; k < kE; ++k) val[k] = row[k] >= 0 ? g[col[k]] : 0.0;
        warp_runs_add<kE>(row, val, acc, lane);
    }
}

// F = acc into the outputs of the mode, L1 norm and max; the last CTA runs
// the control step.
template <typename FT>
__global__ void __launch_bounds__(kResThreads) k_resb_fin(const SolveDesc *__restrict__ desc, SolveState *__restrict__ st,
                                                          int mode, const double *__restrict__ acc, int64_t n,
                                                          double *__restrict__ part_sum, double *__restrict__ part_max) {
    if (mode == RES_LEVEL && !st->do_recompute) return;
    FT *__restrict__ Ffl = (mode == RES_LEVEL || mode == RES_WARM_INIT) ? static_cast<FT *>(desc->F) : nullptr;
    double *__restrict__ F64 = mode == RES_WARM_INIT ? nullptr : desc->F_out;
    // the completed dangling columns add d/N sum_dangling H_j to every row
    const double ud = desc->dangling ? desc->d * st->dang_h / (double)n : 0.0;
    double lsum = 0.0, lmax = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double f = acc[i] + ud;
        if (Ffl) Ffl[i] = static_cast<FT>(f);
        if (F64) F64[i] = f;
        lsum += fabs(f);
        lmax = fmax(lmax, fabs(f));
    }
    block_sum_max<kResThreads>(lsum, lmax);
    if (threadIdx.x == 0) {
        part_sum[blockIdx.x] = lsum;
        part_max[blockIdx.x] = lmax;
    }
    if (!last_block(&st->res_blocks)) return;
    double s = 0.0, m = 0.0;
    for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
        s += part_sum[i];
        m = fmax(m, part_max[i]);
    }
    block_sum_max<kResThreads>(s, m);
    if (threadIdx.x != 0) return;
    st->dang_h = 0.0;                       // every CTA read it before this, the last one
    res_control(desc, st, mode, s, m);
}

// ------------------------------------------------------------------ control

// After an exact residual with L1 norm s and max m: stop, calibrate the
// scan's estimate, or (warm start) set T_0 and |F_0|_1.
__device__ void res_control(const SolveDesc *__restrict__ desc, SolveState *__restrict__ st, int mode, double s,
                            double m) {
    st->r_exact = s;
    st->max_exact = m;
    // the exact F already holds the fluid that dangling nodes drained
    if (mode == RES_LEVEL || mode == RES_WARM_INIT) st->dang_acc = 0.0;
    if (mode == RES_LEVEL) {
        st->recomputes += 1;
        st->since_recompute = 0;
        st->do_recompute = 0;
        if (!isfinite(s)) {
            st->done = 3;
        } else if (s <= desc->tol) {
            st->done = 1;
        } else if (st->confirming && st->r_confirm > 0.0) {
            // the level's estimate was too optimistic: calibrate later estimates
            st->est_scale = fmax(st->est_scale, 1.0) * fmax(s / st->r_confirm, 1.0);
        }
        st->confirming = 0;
    } else if (mode == RES_WARM_INIT) {
        // T_0 = mean |F0_i| (<= max |F0|): equal to max |F0| for a cold start
        // with uniform B; for a warm start it avoids a run of sparse levels
        // over the few largest residuals
        st->T = desc->n_nodes > 0 ? s / (double)desc->n_nodes : m;
        st->f0_l1 = s;
        if (!isfinite(s)) st->done = 3;
        else if (s <= desc->tol) st->done = 1;   // H_0 already meets the tolerance
    }
}

}  // namespace

constexpr int kResLongBlocks = 64;

int residual_grid(int sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k_res_pull<double>, kPullThreads, 0) !=
            cudaSuccess || per_sm < 1)
        per_sm = 1;
    return per_sm * sms;
}

int residual_kernels(const di_graph *) { return 3; }

int residual_partials(const di_graph *g) { return g->grid_res + kResLongBlocks; }

bool residual_blocked(const di_graph *g) { return g->res_form != 1; }

void launch_residual(di_graph *g, int fluid_fp64, ResMode mode, cudaStream_t s) {
    Workspace &ws = g->ws;
    if (residual_blocked(g)) {
        const int grid = g->grid_res;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k_resb_flat, kResThreads, 0) !=
                cudaSuccess || per_sm < 1)
            per_sm = 1;
        const int flat = (int)std::max<int64_t>(
            1, std::min<int64_t>((int64_t)per_sm * g->num_sms, (g->nnz / kResbEdges + kResThreads) / kResThreads));
        k_resb_init<<<grid, kResThreads, 0, s>>>(ws.desc, ws.st, (int)mode, g->s64, ws.g, ws.acc, g->n);
        k_resb_flat<<<flat, kResThreads, 0, s>>>(ws.st, (int)mode, g->bcol, g->brow, ws.g, ws.acc, g->nnz);
        if (fluid_fp64)
            k_resb_fin<double><<<grid, kResThreads, 0, s>>>(ws.desc, ws.st, (int)mode, ws.acc, g->n, ws.part_sum,
                                                            ws.part_max);
        else
            k_resb_fin<float><<<grid, kResThreads, 0, s>>>(ws.desc, ws.st, (int)mode, ws.acc, g->n, ws.part_sum,
                                                           ws.part_max);
        return;
    }
    const PullPlan pl = pull_plan_of(g);
    const int pull_blocks = (int)std::max<int64_t>(1, std::min<int64_t>(g->grid_res, pl.task_off[5]));
    k_res_prep<<<g->grid_res, kResThreads, 0, s>>>(ws.desc, ws.st, (int)mode, g->s64, ws.g, g->n);
    if (fluid_fp64) {
        k_res_pull<double><<<pull_blocks, kPullThreads, 0, s>>>(pl, ws.desc, ws.st, g->in_rp, g->in_col, ws.g,
                                                                ws.seg_part, ws.part_sum, ws.part_max, (int)mode);
        k_res_long<double><<<kResLongBlocks, kResThreads, 0, s>>>(ws.desc, ws.st, g->pl_lrows, g->pl_lseg0,
                                                                  g->pl_nlrows, ws.seg_part, ws.part_sum,
                                                                  ws.part_max, pull_blocks, (int)mode);
    } else {
        k_res_pull<float><<<pull_blocks, kPullThreads, 0, s>>>(pl, ws.desc, ws.st, g->in_rp, g->in_col, ws.g,
                                                               ws.seg_part, ws.part_sum, ws.part_max, (int)mode);
        k_res_long<float><<<kResLongBlocks, kResThreads, 0, s>>>(ws.desc, ws.st, g->pl_lrows, g->pl_lseg0,
                                                                 g->pl_nlrows, ws.seg_part, ws.part_sum,
                                                                 ws.part_max, pull_blocks, (int)mode);
    }
}

}  // namespace di

using namespace di;

extern "C" DI_API di_status di_residual(di_graph *g, const double *B, double d, const double *H, double *F,
                                       double *r_l1, void *stream) {
    di::NvtxRange nvtx_range("di_residual");
    clear_error();
    if (!g || !B || !H || !F) { set_error("di_residual: NULL argument"); return DI_EINVAL; }
    if (!(d > 0.0 && d < 1.0)) { set_error("di_residual: d = %g outside (0, 1)", d); return DI_EINVAL; }
    cudaStream_t s = as_stream(stream);
    DI_TRY(ensure_workspace(g));
    DI_TRY(ensure_scale(g, d, s));
    g->res_form = 0;
    DI_TRY(ensure_blocked_order(g, s));
    Workspace &ws = g->ws;
    // the workspace descriptor is shared with di_solve: stage it through the pinned mirror
    DI_CUDA_TRY(cudaStreamSynchronize(s));
    std::memset(ws.desc_h, 0, sizeof(SolveDesc));
    ws.desc_h->B = B;
    ws.desc_h->H = const_cast<double *>(H);
    ws.desc_h->F_out = F;
    ws.desc_h->d = d;
    DI_CUDA_TRY(cudaMemcpyAsync(ws.desc, ws.desc_h, sizeof(SolveDesc), cudaMemcpyHostToDevice, s));
    launch_residual(g, 1, RES_STANDALONE, s);
    DI_CUDA_TRY(cudaGetLastError());
    if (r_l1) {
        DI_CUDA_TRY(cudaMemcpyAsync(ws.st_h, ws.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        DI_CUDA_TRY(cudaStreamSynchronize(s));
        *r_l1 = ws.st_h->r_exact;
    }
    return DI_OK;
}
