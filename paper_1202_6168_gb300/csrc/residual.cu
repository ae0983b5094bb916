// residual.cu - exact FP64 residual F = B + P H - H.
//
// Eqs. defF/defH imply that F_n + H_n - P H_n does not change with n, so
// F_n = B + P H_n - H_n for a cold start (and for any H_0 with
// F_0 = B + P H_0 - H_0).  Recomputing F from H this way in FP64 removes the
// rounding that FP32 pushes accumulate, gives the exact stopping residual
// |F|_1, and forms the warm-start fluid F_0.
//
// (P H)_k = sum over in-edges j -> k of (d / outdeg_j) H_j is a gather over
// the transpose: no atomics, and a fixed summation order per graph object.
// In-rows longer than kResSeg edges are cut in segments whose partial sums
// are combined in segment order.
#include "di_internal.cuh"

namespace di {
namespace {

__global__ void __launch_bounds__(kResThreads) k_res_prep(const SolveDesc *__restrict__ desc,
                                                          const SolveState *__restrict__ st, int mode,
                                                          const double *__restrict__ s64,
                                                          double *__restrict__ g, int64_t n) {
    if (mode == RES_LEVEL && !st->do_recompute) return;
    const double *__restrict__ H = desc->H;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) g[i] = s64[i] * H[i];
}

__global__ void __launch_bounds__(kResThreads) k_res_seg(const SolveState *__restrict__ st, int mode,
                                                         const int32_t *__restrict__ in_rp,
                                                         const int32_t *__restrict__ in_col,
                                                         const int32_t *__restrict__ long_rows,
                                                         const int32_t *__restrict__ seg_row,
                                                         const int64_t *__restrict__ seg_beg, int n_seg,
                                                         const double *__restrict__ g,
                                                         double *__restrict__ seg_part) {
    if (mode == RES_LEVEL && !st->do_recompute) return;
    for (int s = blockIdx.x; s < n_seg; s += gridDim.x) {
        const int32_t row = long_rows[seg_row[s]];
        const int64_t b = seg_beg[s];
        const int64_t e = b + kResSeg < (int64_t)in_rp[row + 1] ? b + kResSeg : (int64_t)in_rp[row + 1];
        double acc = 0.0;
        for (int64_t q = b + threadIdx.x; q < e; q += kResThreads) acc += g[in_col[q]];
        double mx = 0.0;
        block_sum_max<kResThreads>(acc, mx);
        if (threadIdx.x == 0) seg_part[s] = acc;
    }
}

template <typename FT>
__global__ void __launch_bounds__(kResThreads) k_res_rows(
    const SolveDesc *__restrict__ desc, SolveState *__restrict__ st, const int32_t *__restrict__ in_rp,
    const int32_t *__restrict__ in_col, const int32_t *__restrict__ long_rows,
    const int32_t *__restrict__ long_seg0, int n_long, const double *__restrict__ seg_part,
    const double *__restrict__ g, int64_t n, double *__restrict__ part_sum, double *__restrict__ part_max,
    int mode) {
    if (mode == RES_LEVEL && !st->do_recompute) return;   // host-driven levels launch it every time
    const double *__restrict__ B = desc->B;
    const double *__restrict__ H = desc->H;
    FT *__restrict__ Ffl = (mode == RES_LEVEL || mode == RES_WARM_INIT) ? static_cast<FT *>(desc->F) : nullptr;
    double *__restrict__ F64 = mode == RES_WARM_INIT ? nullptr : desc->F_out;

    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double lsum = 0.0, lmax = 0.0;

    auto emit = [&](int64_t k, double acc) {
        const double f = B[k] + acc - H[k];
        if (Ffl) Ffl[k] = static_cast<FT>(f);
        if (F64) F64[k] = f;
        const double a = fabs(f);
        lsum += a;
        lmax = fmax(lmax, a);
    };

    for (int64_t base = warp * 32; base < n; base += nwarps * 32) {
        const int64_t k = base + lane;
        int32_t b = 0, e = 0;
        if (k < n) { b = in_rp[k]; e = in_rp[k + 1]; }
        const int len = e - b;
        double acc = 0.0;
        if (len <= 32) {
            for (int32_t q = b; q < e; ++q) acc += g[in_col[q]];
        }
        unsigned med = __ballot_sync(0xffffffffu, len > 32 && len <= kResSeg);
        while (med) {
            const int src = __ffs(med) - 1;
            med &= med - 1;
            const int32_t mb = __shfl_sync(0xffffffffu, b, src), me = __shfl_sync(0xffffffffu, e, src);
            double part = 0.0;
            for (int32_t q = mb + lane; q < me; q += 32) part += g[in_col[q]];
            part = warp_sum(part);
            if (lane == src) acc = part;
        }
        if (k < n && len <= kResSeg) emit(k, acc);
    }
    // rows split in segments: one warp per row, segment partials in order
    for (int64_t r = warp; r < n_long; r += nwarps) {
        const int32_t s0 = long_seg0[r], s1 = long_seg0[r + 1];
        double part = 0.0;
        for (int32_t s = s0 + lane; s < s1; s += 32) part += seg_part[s];
        part = warp_sum(part);
        if (lane == 0) emit(long_rows[r], part);
    }

    block_sum_max<kResThreads>(lsum, lmax);
    if (threadIdx.x == 0) {
        part_sum[blockIdx.x] = lsum;
        part_max[blockIdx.x] = lmax;
    }
    if (!last_block(&st->res_blocks)) return;
    // last block: deterministic combination of the block partials
    double s = 0.0, m = 0.0;
    for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
        s += part_sum[i];
        m = fmax(m, part_max[i]);
    }
    block_sum_max<kResThreads>(s, m);
    if (threadIdx.x != 0) return;
    st->r_exact = s;
    st->max_exact = m;
    if (mode == RES_LEVEL) {
        st->recomputes += 1;
        st->since_recompute = 0;
        st->do_recompute = 0;
        if (!isfinite(s)) {
            st->done = 3;
        } else if (s <= desc->tol) {
            st->done = 1;
        } else if (st->confirming) {
            st->force_push = 1;   // the scan's estimate was too optimistic
        }
        st->confirming = 0;
    } else if (mode == RES_WARM_INIT) {
        st->T = m;
        st->f0_l1 = s;
    }
}

}  // namespace

int residual_grid(int sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k_res_rows<double>, kResThreads, 0) !=
            cudaSuccess || per_sm < 1)
        per_sm = 1;
    return per_sm * sms;
}

int residual_kernels(const di_graph *g) { return g->n_seg > 0 ? 3 : 2; }

void launch_residual(di_graph *g, int fluid_fp64, ResMode mode, cudaStream_t s) {
    Workspace &ws = g->ws;
    k_res_prep<<<g->grid_res, kResThreads, 0, s>>>(ws.desc, ws.st, (int)mode, g->s64, ws.g, g->n);
    if (g->n_seg > 0)
        k_res_seg<<<std::min(g->n_seg, g->grid_res), kResThreads, 0, s>>>(
            ws.st, (int)mode, g->in_rp, g->in_col, g->long_rows, g->seg_row, g->seg_beg, g->n_seg, ws.g, ws.seg_part);
    if (fluid_fp64)
        k_res_rows<double><<<g->grid_res, kResThreads, 0, s>>>(ws.desc, ws.st, g->in_rp, g->in_col, g->long_rows,
                                                               g->long_seg0, g->n_long_rows, ws.seg_part, ws.g,
                                                               g->n, ws.part_sum, ws.part_max, (int)mode);
    else
        k_res_rows<float><<<g->grid_res, kResThreads, 0, s>>>(ws.desc, ws.st, g->in_rp, g->in_col, g->long_rows,
                                                              g->long_seg0, g->n_long_rows, ws.seg_part, ws.g,
                                                              g->n, ws.part_sum, ws.part_max, (int)mode);
}

}  // namespace di

using namespace di;

extern "C" DI_API di_status di_residual(di_graph *g, const double *B, double d, const double *H, double *F,
                                       double *r_l1, void *stream) {
    clear_error();
    if (!g || !B || !H || !F) { set_error("di_residual: NULL argument"); return DI_EINVAL; }
    if (!(d > 0.0 && d < 1.0)) { set_error("di_residual: d = %g outside (0, 1)", d); return DI_EINVAL; }
    cudaStream_t s = as_stream(stream);
    DI_TRY(ensure_workspace(g));
    DI_TRY(ensure_scale(g, d, s));
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
