// level_tiled.cuh - one threshold level in one launch, with the fluid of a
// node range accumulated on chip (propagation 6).
//
// A threshold level (Sec. 2.4) diffuses every node with |F_i| >= T: F_i moves
// into H_i and p_ki F_i is added to the fluid of every child k (Eqs.
// defF/defH).  On a GPU each addition is an L2 reduction, and the L2 retires
// scattered reductions at a fixed rate of sector operations whatever the word
// size, so the level's cost is its number of reduction sectors.  This kernel
// cuts that number for the two kinds of targets that repeat:
//   - targets near their source: a warp diffuses a contiguous chunk of C
//     nodes [c0, c0 + C) and adds every target in [c0 - R, c0 + C + R) to its
//     shared-memory copy of that window, flushed once per chunk with
//     coalesced reductions (eight FP32 additions per sector);
//   - targets of very high in-degree (hot slots, encoded -1 - slot in pcol):
//     added to shared memory per CTA, flushed once per launch.
// Every other target gets one red.global.add.  Each warp takes its own
// chunks, in node order across the grid, so a chunk's selection sees the
// fluid that earlier chunks of the same level sent it - through global memory or, inside the window, through
// the pending shared-memory copy, which the selection reads and the drain
// takes with the global fluid.  This is the paper's cyclic sweep (one pass in
// node order per level, fluid received earlier in the pass counted) with the
// GPU's width; any order that keeps diffusing every node converges (Sec. 2).
// Each warp pushes the rows of its 32 selected nodes edge-parallel over their
// concatenation, so column indices are loaded coalesced whatever the
// out-degrees.
#pragma once

#include "di_internal.cuh"

namespace di {

// Shared-memory layout of the tiled kernel: hot slots (padded to 4 words),
// then one fluid window of C + 2R words per warp.
constexpr int kTiledWarps = kPushThreads / 32;
__host__ __device__ inline int tiled_hot_pad(int n_hot) { return (n_hot + 3) & ~3; }
template <typename FT>
__host__ __device__ inline size_t tiled_smem(int n_hot, int chunk, int R) {
    return (size_t)(tiled_hot_pad(n_hot) + kTiledWarps * (chunk + 2 * R)) * sizeof(FT);
}

// The out-rows of the (up to) 32 nodes held one per lane (row start b, degree
// deg, weight w; deg = 0 for an idle lane), edge-parallel over their
// concatenation: edge e of the concatenation belongs to the first lane whose
// inclusive degree prefix exceeds e (5-step search over the lanes' prefixes),
// so consecutive lanes load consecutive column indices; four column loads per
// lane are issued before their additions.  Each target goes to a hot slot,
// the warp's window or a global reduction.  Returns the number of global
// reductions this lane issued.
template <typename FT>
__device__ __forceinline__ unsigned push_rows_tiled(FT *__restrict__ F, FT *s_hot, FT *w_win,
                                                    const int32_t *__restrict__ pcol, int32_t b, int deg, FT w,
                                                    int64_t wbase, unsigned span, uint64_t keep, int lane) {
    constexpr int kU = 4;
    int incl = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int32_t off = b - (incl - deg);   // column position of edge e of this lane's row: off + e
    auto src_of = [&](int e) {
        int src = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int v = __shfl_sync(0xffffffffu, incl, src + step - 1);
            if (v <= e) src += step;
        }
        return src < 31 ? src : 31;
    };
    unsigned reds = 0;
    for (int base = 0; base < total; base += 32 * kU) {
        int32_t c[kU];
        FT wv[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int e = base + 32 * u + lane;
            const int sl = src_of(e);
            const int32_t o = __shfl_sync(0xffffffffu, off, sl);
            wv[u] = __shfl_sync(0xffffffffu, w, sl);
            c[u] = e < total ? __ldcs(pcol + o + e) : INT32_MAX;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int32_t t = c[u];
            if (t == INT32_MAX) continue;
            if (t < 0) {
                atomicAdd(&s_hot[-1 - t], wv[u]);
                continue;
            }
            const uint64_t o = (uint64_t)((int64_t)t - wbase);
            if (o < span) {
                atomicAdd(&w_win[o], wv[u]);
            } else {
                red_add_keep(F + t, wv[u], keep);
                ++reds;
            }
        }
    }
    return reds;
}

__device__ __forceinline__ float fluid_exch_shared(float *p) { return atomicExch(p, 0.0f); }
__device__ __forceinline__ double fluid_exch_shared(double *p) {
    return __longlong_as_double(
        static_cast<long long>(atomicExch(reinterpret_cast<unsigned long long *>(p), 0ull)));
}

// One level (propagation 6).  Every warp takes chunks of C consecutive nodes
// (C a power of two in [32, 256]) in node order and owns a window of
// C + 2R words (R a multiple of 32, or 0); no CTA-wide barrier is taken
// until the hot slots are flushed at the end.  ctl: 1 in a CUDA graph, 2
// host-driven.  With the 1/N completion (Sec. 2.2) the fluid that dangling
// nodes drained in the previous level reaches every node here, as
// d * dang_acc / N added atomically (other warps push concurrently); what this
// level drains from dangling nodes goes to dang_next.
template <typename FT>
__global__ void __launch_bounds__(kPushThreads, sizeof(FT) == 8 ? 4 : 6) k_level_tiled(
    const SolveDesc *__restrict__ desc, SolveState *__restrict__ st, const int32_t *__restrict__ rp,
    const int32_t *__restrict__ pcol, const int32_t *__restrict__ hot_node, int n_hot, const FT *__restrict__ scale,
    int64_t n, int chunk, int R, double *__restrict__ part_sum, double *__restrict__ part_max,
    cudaGraphConditionalHandle h_while, cudaGraphConditionalHandle h_rec, int ctl) {
    {
        const int done0 = st->done;
        const int stop = done0 ? done0 : (st->level >= desc->max_levels ? 2 : 0);
        if (stop) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                st->done = stop;
                if (ctl == 1) {
                    cudaGraphSetConditional(h_rec, 0);
                    cudaGraphSetConditional(h_while, 0);
                }
            }
            return;
        }
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FT *s_hot = reinterpret_cast<FT *>(smem_raw);
    const unsigned span = (unsigned)(chunk + 2 * R);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    FT *w_win = s_hot + tiled_hot_pad(n_hot) + (size_t)warp * span;
    __shared__ double s_dang;
    for (int sl = threadIdx.x; sl < n_hot; sl += kPushThreads) s_hot[sl] = FT(0);
    for (unsigned q = lane; q < span; q += 32) w_win[q] = FT(0);
    if (threadIdx.x == 0) s_dang = 0.0;
    __syncthreads();
    FT *__restrict__ F = static_cast<FT *>(desc->F);
    double *__restrict__ H = desc->H;
    const FT Tc = thr_cast(st->T, FT(0));
    const int dangling = desc->dangling;
    const FT u = dangling ? static_cast<FT>(desc->d * st->dang_acc / (double)n) : FT(0);
    const uint64_t keep = l2_keep_policy();
    FT acc = 0, mx = 0;
    unsigned long long my_edges = 0, my_nodes = 0, my_reds = 0;
    double my_dang = 0.0;
    // chunks in node order across the grid: warp gw takes chunks gw, gw + W,
    // gw + 2W, ... (W warps in the grid; no shared counter to serialise on)
    const int64_t gwarp = (int64_t)blockIdx.x * kTiledWarps + warp, nw = (int64_t)gridDim.x * kTiledWarps;
    for (int64_t ch = gwarp;; ch += nw) {
        const int64_t c0 = ch * chunk;
        if (c0 >= n) break;
        const int64_t wbase = c0 - R;
#pragma unroll 1
        for (int k = 0; k < chunk; k += 32) {
            const int64_t i = c0 + k + lane;
            FT v = FT(0);
            if (i < n) {
                if (u != FT(0)) atomicAdd(F + i, u);
                v = __ldcg(F + i) + *(volatile FT *)&w_win[i - wbase];   // with the window's pending fluid
            }
            const FT a = fabs(v);
            acc += a;
            mx = max(mx, a);
            const bool sel = i < n && a >= Tc && a > FT(0);
            if (!__any_sync(0xffffffffu, sel)) continue;
            int32_t b = 0;
            int deg = 0;
            FT w = FT(0);
            if (sel) {
                b = __ldcs(rp + i);
                deg = __ldcs(rp + i + 1) - b;
                const FT f = atomic_exch_keep(F + i, FT(0), keep) + fluid_exch_shared(&w_win[i - wbase]);
                const double fd = static_cast<double>(f);
                __stcs(H + i, __ldcs(H + i) + fd);   // i is in one chunk only
                w = f * __ldcs(scale + i);
                my_nodes += 1;
                my_edges += static_cast<unsigned long long>(deg);
                if (deg == 0 && dangling) my_dang += fd;
            }
            my_reds += push_rows_tiled<FT>(F, s_hot, w_win, pcol, b, deg, w, wbase, span, keep, lane);
        }
        __syncwarp();
        // flush the window and clear it: consecutive lanes, consecutive nodes (coalesced)
        for (unsigned q = lane; q < span; q += 32) {
            const FT v = w_win[q];
            w_win[q] = FT(0);
            const int64_t node = wbase + q;
            const bool go = v != FT(0) && node >= 0 && node < n;
            // sectors this instruction touches: groups of 8 FP32 (4 FP64) lanes with work
            const unsigned m = __ballot_sync(0xffffffffu, go);
            if (lane == 0) {
                constexpr int per = 32 / (int)sizeof(FT);
                for (int g = 0; g < 32; g += per) my_reds += ((m >> g) & ((1u << per) - 1u)) ? 1u : 0u;
            }
            if (go) red_add_keep(F + node, v, keep);
        }
        __syncwarp();
    }
    __syncthreads();
    for (int sl = threadIdx.x; sl < n_hot; sl += kPushThreads) {
        const FT hv = s_hot[sl];
        if (hv != FT(0)) {
            red_add_keep(F + hot_node[sl], hv, keep);
            ++my_reds;
        }
    }
    cta_add_counts(&st->node_diff, my_nodes, &st->edge_diff, my_edges, &st->lvl_nodes, my_nodes, &st->red_ops,
                   my_reds);
    my_dang = warp_sum(my_dang);
    if (lane == 0 && my_dang != 0.0) atomicAdd(&s_dang, my_dang);
    double s = static_cast<double>(acc);
    double m = static_cast<double>(mx);
    block_sum_max<kPushThreads>(s, m);     // its barriers order the s_dang adds before the read below
    if (threadIdx.x == 0) {
        part_sum[blockIdx.x] = s;
        part_max[blockIdx.x] = m;
        if (s_dang != 0.0) atomicAdd(&st->dang_next, s_dang);
    }
    if (!last_block(&st->scan_blocks)) return;
    double ts = 0.0, tm = 0.0;
    for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) { ts += part_sum[i]; tm = fmax(tm, part_max[i]); }
    block_sum_max<kPushThreads>(ts, tm);
    if (threadIdx.x != 0) return;

    // control step after the level (as the fused level of propagation 5)
    const unsigned long long lnodes = st->lvl_nodes;
    double T = st->T;
    int level = st->level, since = st->since_recompute, iters = st->body_iters, phase = st->phase;
    const double est = st->est_scale > 1.0 ? st->est_scale : 1.0;
    const double tol = desc->tol, alpha = desc->alpha;
    const int max_iters = desc->max_body_iters;
    int done = 0, rec = 0;
    if (!isfinite(ts)) {
        done = 3;
    } else {
        const int level0 = level;
        threshold_step(desc->resweeps, lnodes > 0, alpha, tm, T, phase, level, since);
        if (level != level0 && refine_due(desc, st, since, ts * est)) rec = 1;
        if (ts * est <= tol) {            // the fluid read before the pushes already meets tol
            rec = 1;
            st->confirming = 1;
            st->r_confirm = ts * est;
        }
    }
    iters += 1;
    if (!done && iters >= max_iters) done = 2;
    if (done) rec = 0;
    st->r_scan = ts;
    st->max_scan = tm;
    st->T = T;
    st->level = level;
    st->since_recompute = since;
    st->body_iters = iters;
    st->phase = phase;
    st->lvl_nodes = 0;
    st->dang_acc = st->dang_next;   // reaches every node in the next level
    st->dang_next = 0.0;
    st->do_recompute = rec;
    if (done) st->done = done;
    if (ctl == 1) {
        cudaGraphSetConditional(h_rec, rec ? 1u : 0u);
        if (done) cudaGraphSetConditional(h_while, 0);
    }
}

}  // namespace di
