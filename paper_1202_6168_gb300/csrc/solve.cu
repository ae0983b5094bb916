// solve.cu - the D-iteration level loop on one GPU.
//
// One threshold level (Sec. 2.4) diffuses, at once, every node whose fluid
// satisfies |F_i| >= T (Eqs. defF/defH):
//   k_select     - drains the selected nodes (H_i += F_i, F_i = 0) into
//                  w_i = (d / outdeg_i) F_i, with the L1 norm and max of the
//                  fluid from the same read, and decides the next steps;
//   k_pull_level - dense levels: F_k += sum of w_j over the in-edges (binned
//                  gather over the transpose, no atomics);
//   k_pushw      - sparse levels: F_k += w_j for the out-edges of the active
//                  nodes (edge-parallel red.global.add; targets of very high
//                  in-degree accumulated in shared memory per CTA).
// Both propagations send the fluid the selected nodes held at the start of
// the level, so F + H - P H is unchanged by a level (the invariant that gives
// H -> X and |X - H|_1 <= |F|_1 / (1 - d)).  The levels run in a CUDA graph:
// a WHILE conditional node repeats [k_select, IF/ELSE(pull | push),
// IF(exact FP64 residual)], every decision taken by k_select's last CTA on
// the device, with no host round trip per level.
// k_scan is the frontier selection alone (di_frontier).
#include <algorithm>
#include <cmath>

#include "di_internal.cuh"
#include "level_tiled.cuh"
#include "pull.cuh"

namespace di {
namespace {

template <typename FT>
struct Acc;  // per-thread accumulation type of the scan's L1 sum
template <>
struct Acc<float> { using T = float; };
template <>
struct Acc<double> { using T = double; };


template <typename FT>
struct Vec4;   // 4 consecutive fluid values per load
template <>
struct Vec4<float> {
    float v[4];
    __device__ __forceinline__ void load(const float *p) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    __device__ __forceinline__ void store(float *p) const {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
    __device__ __forceinline__ void load_cs(const float *p) {
        const float4 t = __ldcs(reinterpret_cast<const float4 *>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    __device__ __forceinline__ void load_cg(const float *p) {
        const float4 t = __ldcg(reinterpret_cast<const float4 *>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
};
template <>
struct Vec4<double> {
    double v[4];
    __device__ __forceinline__ void load(const double *p) {
        const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    __device__ __forceinline__ void store(double *p) const {
        reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
    }
    __device__ __forceinline__ void load_cs(const double *p) {
        const double2 a = __ldcs(reinterpret_cast<const double2 *>(p)),
                      b = __ldcs(reinterpret_cast<const double2 *>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    __device__ __forceinline__ void load_cg(const double *p) {
        const double2 a = __ldcg(reinterpret_cast<const double2 *>(p)),
                      b = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};

// Loads of data that other SMs write while a persistent kernel runs: kCG
// selects ld.global.cg (L2 only), since an SM's L1 is not kept coherent with
// other SMs' writes and is only clean at a kernel launch; a kernel launched
// per phase keeps the cheaper streaming loads.
template <bool kCG, typename T>
__device__ __forceinline__ T ld_mut(const T *p) { return kCG ? __ldcg(p) : __ldcs(p); }

// Dynamic shared memory of the frontier push (propagations 3 and 7): the hot
// slots (padded to 4 words), then either the fluid window of kPushWin + 2R
// words (none when R = 0) or, for the slice-sweep variant, its queue
// (kSliceQueueCap node ids).
__host__ __device__ inline int push_hot_pad(int n_hot) { return (n_hot + 3) & ~3; }
template <typename FT>
__host__ __device__ inline size_t push_smem(int n_hot, int R, bool slice = false) {
    const size_t win = R > 0 ? (size_t)(kPushWin + 2 * R) * sizeof(FT) : 0;
    const size_t queue = slice ? (size_t)kSliceQueueCap * sizeof(int32_t) : 0;
    return (size_t)push_hot_pad(n_hot) * sizeof(FT) + (win > queue ? win : queue);
}

// ------------------------------------------------------------------ init (cold start)

template <typename FT>
__global__ void __launch_bounds__(kScanThreads) k_init(const SolveDesc *__restrict__ desc, SolveState *__restrict__ st,
                                                       int64_t n, double *__restrict__ part_sum,
                                                       double *__restrict__ part_max) {
    const double *__restrict__ B = desc->B;
    double *__restrict__ H = desc->H;
    FT *__restrict__ F = static_cast<FT *>(desc->F);
    const FT *__restrict__ iw = static_cast<const FT *>(desc->iw);
    double s = 0.0, m = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double b = B[i];
        const FT f = static_cast<FT>(b);
        F[i] = f;
        H[i] = 0.0;
        s += fabs(b);
        const FT score = iw ? fabs(f) * iw[i] : fabs(f);
        m = fmax(m, static_cast<double>(score));
    }
    block_sum_max<kScanThreads>(s, m);
    if (threadIdx.x == 0) { part_sum[blockIdx.x] = s; part_max[blockIdx.x] = m; }
    if (!last_block(&st->init_blocks)) return;
    double ts = 0.0, tm = 0.0;
    for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) { ts += part_sum[i]; tm = fmax(tm, part_max[i]); }
    block_sum_max<kScanThreads>(ts, tm);
    if (threadIdx.x == 0) {
        st->b_l1 = ts;
        st->f0_l1 = ts;
        st->r_exact = ts;   // F_0 = B exactly: this is the exact residual of H_0 = 0
        st->T = tm;         // T_0 = max |F_0| (weighted: the largest score)
        if (!isfinite(ts)) st->done = 3;
        else if (ts <= desc->tol) st->done = 1;
    }
}


// |B|_1 only (warm start)
__global__ void __launch_bounds__(kScanThreads) k_bnorm(const SolveDesc *__restrict__ desc, SolveState *__restrict__ st,
                                                        int64_t n, double *__restrict__ part_sum,
                                                        double *__restrict__ part_max) {
    const double *__restrict__ B = desc->B;
    double s = 0.0, m = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) s += fabs(B[i]);
    block_sum_max<kScanThreads>(s, m);
    if (threadIdx.x == 0) part_sum[blockIdx.x] = s;
    if (!last_block(&st->init_blocks)) return;
    double ts = 0.0;
    for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) ts += part_sum[i];
    block_sum_max<kScanThreads>(ts, m);
    if (threadIdx.x == 0) st->b_l1 = ts;
}

// ------------------------------------------------------------------ scan

// Frontier selection alone: S = { i : |F_i| >= T } compacted in node order
// within blocks of 2048 nodes (warp ballots, one prefix, one atomic per
// block), with the L1 norm and max |F_i| fused into the same read.
template <typename FT>
__global__ void __launch_bounds__(kScanThreads) k_scan(const SolveDesc *__restrict__ desc, SolveState *__restrict__ st,
                                                       int32_t *__restrict__ front, int64_t n,
                                                       double *__restrict__ part_sum, double *__restrict__ part_max) {
    using AT = typename Acc<FT>::T;
    const FT *__restrict__ F = static_cast<const FT *>(desc->F);
    const FT Tc = thr_cast(st->T, FT(0));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    __shared__ int s_cnt[kScanItems * (kScanThreads / 32)];
    __shared__ int s_base;
    AT acc = 0;
    FT mx = 0;
    for (int64_t c0 = (int64_t)blockIdx.x * kScanChunk; c0 < n; c0 += (int64_t)gridDim.x * kScanChunk) {
        unsigned masks[kScanItems];
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const int64_t idx = c0 + k * kScanThreads + threadIdx.x;
            FT v = 0;
            if (idx < n) v = fabs(F[idx]);
            const bool sel = idx < n && v >= Tc;
            masks[k] = __ballot_sync(0xffffffffu, sel);
            acc += static_cast<AT>(v);
            mx = max(mx, v);
            if (lane == 0) s_cnt[k * (kScanThreads / 32) + warp] = __popc(masks[k]);
        }
        __syncthreads();
        if (warp == 0) {   // exclusive scan of the 64 counts in node order
            const int a = s_cnt[2 * lane], b = s_cnt[2 * lane + 1];
            int incl = a + b;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int excl = incl - a - b;
            s_cnt[2 * lane] = excl;
            s_cnt[2 * lane + 1] = excl + a;
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            if (lane == 0) s_base = total ? atomicAdd(&st->nfront, total) : 0;
        }
        __syncthreads();
        const int base = s_base;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if ((masks[k] >> lane) & 1u)
                front[base + s_cnt[k * (kScanThreads / 32) + warp] + __popc(masks[k] & lt_mask)] =
                    static_cast<int32_t>(c0 + k * kScanThreads + threadIdx.x);
        }
        __syncthreads();
    }
    double s = static_cast<double>(acc);
    double m = static_cast<double>(mx);
    block_sum_max<kScanThreads>(s, m);
    if (threadIdx.x == 0) { part_sum[blockIdx.x] = s; part_max[blockIdx.x] = m; }
    if (!last_block(&st->scan_blocks)) return;
    double ts = 0.0, tm = 0.0;
    for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) { ts += part_sum[i]; tm = fmax(tm, part_max[i]); }
    block_sum_max<kScanThreads>(ts, tm);
    if (threadIdx.x != 0) return;
    st->r_scan = ts;
    st->max_scan = tm;
}

// ------------------------------------------------------------------ asynchronous push level

// Scan of one level of the asynchronous design: frontier compaction in node
// order (4 nodes per thread with vector loads, a warp prefix and one block
// prefix per 2048-node chunk) with the L1 norm and max of the fluid fused into
// the first read.  Two passes over each CTA's
// chunks - count, reserve the CTA's slice with one atomic, then write - so
// the frontier counter sees one atomic per CTA instead of one per chunk.
// Its last CTA decides the level: push the frontier (T <- T / alpha), lower T
// to the largest fluid after an empty scan, or request an exact residual to
// confirm a stop (no push).  ctl: 1 in a CUDA graph, 2 host-driven.
// Selection pass of one level (every CTA over its chunks): the frontier
// slice of the CTA and its partial |F|_1 and max in part_sum / part_max.
template <typename FT, bool kCG = false>
__device__ __forceinline__ void scan_select(const SolveDesc *__restrict__ desc, SolveState *__restrict__ st,
                                            int32_t *__restrict__ front, int64_t n, double *__restrict__ part_sum,
                                            double *__restrict__ part_max) {
    using AT = typename Acc<FT>::T;
    // not __restrict__: with the dangling completion pass 1 writes F and pass 2 reads it back
    FT *F = static_cast<FT *>(desc->F);
    const FT Tc = thr_cast(__ldcg(&st->T), FT(0));
    // 1/N completion (Sec. 2.2): the fluid that dangling nodes drained since the
    // last selection reaches every node as d / N of it; added here, before the
    // test, and stored (the last CTA clears the accumulator)
    const FT u = desc->dangling ? static_cast<FT>(desc->d * __ldcg(&st->dang_acc) / (double)n) : FT(0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // vector layout of a 2048-node chunk: item k (0, 1), thread t, nodes
    // c0 + 1024 k + 4 t + j (j = 0..3), which is node order; the fluid vector
    // is padded with zeros to a multiple of 4 nodes
    constexpr int kVItems = kScanChunk / (4 * kScanThreads);
    constexpr int kWarps = kScanThreads / 32;
    __shared__ int s_off[kVItems * kWarps];
    __shared__ int s_base, s_wcount[kWarps];
    // weighted selection (Sec. 2.4 score): |F_i| w_i >= T, w_i = 1 / ((in + 1)(out + 1))
    const FT *__restrict__ iw = static_cast<const FT *>(desc->iw);
    auto sel_mask = [&](const Vec4<FT> &f, const Vec4<FT> &w, int64_t i0) {
        unsigned msk = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const FT a = fabs(f.v[j]);
            const FT score = iw ? a * w.v[j] : a;
            if (i0 + j < n && score >= Tc && a > FT(0)) msk |= 1u << j;
        }
        return msk;
    };
    auto load_w = [&](Vec4<FT> &w, int64_t i0) {
        if (iw && i0 < n) w.load(iw + i0);
        else w.v[0] = w.v[1] = w.v[2] = w.v[3] = FT(1);
    };
    // pass 1: L1 norm, max and the number of selected nodes of all this
    // CTA's chunks; one atomic reserves the CTA's slice of the frontier
    AT acc = 0;
    FT mx = 0;
    int my_sel = 0;
    for (int64_t c0 = (int64_t)blockIdx.x * kScanChunk; c0 < n; c0 += (int64_t)gridDim.x * kScanChunk) {
        Vec4<FT> f[kVItems];
#pragma unroll
        for (int k = 0; k < kVItems; ++k) {
            const int64_t i0 = c0 + (int64_t)k * 4 * kScanThreads + 4 * threadIdx.x;
            if (i0 < n) {
                if (kCG) f[k].load_cg(F + i0);
                else f[k].load(F + i0);
            }
            else f[k].v[0] = f[k].v[1] = f[k].v[2] = f[k].v[3] = FT(0);
        }
        if (u != FT(0)) {
#pragma unroll
            for (int k = 0; k < kVItems; ++k) {
                const int64_t i0 = c0 + (int64_t)k * 4 * kScanThreads + 4 * threadIdx.x;
                if (i0 >= n) continue;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (i0 + j < n) f[k].v[j] += u;   // the zero padding past n stays zero
                f[k].store(F + i0);
            }
        }
#pragma unroll
        for (int k = 0; k < kVItems; ++k) {
            const int64_t i0 = c0 + (int64_t)k * 4 * kScanThreads + 4 * threadIdx.x;
            Vec4<FT> w;
            load_w(w, i0);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const FT a = fabs(f[k].v[j]);
                acc += static_cast<AT>(a);
                mx = max(mx, iw ? a * w.v[j] : a);   // the control lowers T against the largest score
            }
            my_sel += __popc(sel_mask(f[k], w, i0));
        }
    }
    my_sel = warp_sum(my_sel);
    if (lane == 0) s_wcount[warp] = my_sel;
    __syncthreads();
    int total = 0;   // the CTA's selected count, the same in every thread
#pragma unroll
    for (int w = 0; w < kWarps; ++w) total += s_wcount[w];
    // pass 2 (only if this CTA selected anything): the same reads, now from
    // L2, write the selected ids in node order into the CTA's slice.  Thread 0
    // reserves the slice with one atomic and waits for its result only in the
    // first chunk's serial step, so the round trip overlaps the reloads
    if (total > 0) {
        const int reserved = threadIdx.x == 0 ? atomicAdd(&st->nfront, total) : 0;
        int base = 0;
        bool first = true;
        for (int64_t c0 = (int64_t)blockIdx.x * kScanChunk; c0 < n; c0 += (int64_t)gridDim.x * kScanChunk) {
            unsigned msk[kVItems];
            int excl[kVItems];
#pragma unroll
            for (int k = 0; k < kVItems; ++k) {
                const int64_t i0 = c0 + (int64_t)k * 4 * kScanThreads + 4 * threadIdx.x;
                Vec4<FT> f, w;
                if (i0 < n) {
                    if (kCG) f.load_cg(F + i0);
                    else f.load(F + i0);
                }
                else f.v[0] = f.v[1] = f.v[2] = f.v[3] = FT(0);
                load_w(w, i0);
                msk[k] = sel_mask(f, w, i0);
                const int c = __popc(msk[k]);
                int incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += t;
                }
                excl[k] = incl - c;
                if (lane == 31) s_off[k * kWarps + warp] = incl;
            }
            __syncthreads();
            if (threadIdx.x == 0) {   // exclusive scan of the (item, warp) totals in node order
                int run = 0;
                for (int q = 0; q < kVItems * kWarps; ++q) {
                    const int v = s_off[q];
                    s_off[q] = run;
                    run += v;
                }
                s_wcount[0] = run;
                if (first) s_base = reserved;
            }
            __syncthreads();
            if (first) {
                base = s_base;
                first = false;
            }
#pragma unroll
            for (int k = 0; k < kVItems; ++k) {
                int pos = base + s_off[k * kWarps + warp] + excl[k];
                const int64_t i0 = c0 + (int64_t)k * 4 * kScanThreads + 4 * threadIdx.x;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if ((msk[k] >> j) & 1u) front[pos++] = static_cast<int32_t>(i0 + j);
            }
            base += s_wcount[0];
            __syncthreads();
        }
    }
    double s = static_cast<double>(acc);
    double m = static_cast<double>(mx);
    block_sum_max<kScanThreads>(s, m);
    if (threadIdx.x == 0) { part_sum[blockIdx.x] = s; part_max[blockIdx.x] = m; }
}

// Control step of a level after its selection pass, run by one CTA that sees
// every partial: the push (or not) and the next threshold, a stop request or
// an exact recomputation.  ctl: 1 sets the graph's conditionals, otherwise
// none are set.
__device__ __noinline__ void scan_control(const SolveDesc *__restrict__ desc, SolveState *__restrict__ st,
                                          const double *__restrict__ part_sum, const double *__restrict__ part_max,
                                          int nparts, cudaGraphConditionalHandle h_while,
                                          cudaGraphConditionalHandle h_rec, int ctl) {
    double ts = 0.0, tm = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        ts += __ldcg(part_sum + i);
        tm = fmax(tm, __ldcg(part_max + i));
    }
    block_sum_max<kScanThreads>(ts, tm);
    if (threadIdx.x != 0) return;

    // control (all loads first, one round trip; read past L1, which a
    // persistent kernel may hold stale)
    const int nf = __ldcg(&st->nfront);
    double T = __ldcg(&st->T);
    int level = __ldcg(&st->level), since = __ldcg(&st->since_recompute), iters = __ldcg(&st->body_iters),
        phase = __ldcg(&st->phase);
    const double est_raw = __ldcg(&st->est_scale);
    const double est = est_raw > 1.0 ? est_raw : 1.0;
    const double tol = desc->tol, alpha = desc->alpha;
    const int max_iters = desc->max_body_iters;
    int done = 0, rec = 0, push = 0;
    if (!isfinite(ts)) {
        done = 3;
    } else if (ts * est <= tol) {
        rec = 1;                            // stop request: confirm on the exact residual, no push
        st->confirming = 1;
        st->r_confirm = ts * est;
    } else {
        // push the frontier (if any); the next selection is at the same T
        // (a resweep) or at T / alpha, or, after an empty first pass, at the
        // first T / alpha^k <= max |F|
        push = nf;
        if (nf > 0) st->T_push = T;   // the selection's T, which the push's slice sweeps use
        const int level0 = level;
        threshold_step(desc->resweeps, nf > 0, alpha, tm, T, phase, level, since);
        if (level != level0 && refine_due(desc, st, since, ts * est)) rec = 1;
    }
    iters += 1;
    if (!done && iters >= max_iters) done = 2;
    if (done) { rec = 0; push = 0; }
    st->r_scan = ts;
    st->max_scan = tm;
    st->nfront = 0;
    st->tile_ctr = 0;
    st->tiles_done = 0;
    st->dang_acc = 0.0;                 // every CTA added it before this, the last one
    st->push_count = push;
    st->T = T;
    st->level = level;
    st->since_recompute = since;
    st->body_iters = iters;
    st->phase = phase;
    st->do_recompute = rec;
    if (done) st->done = done;
    if (ctl == 1) {
        cudaGraphSetConditional(h_rec, rec ? 1u : 0u);
        if (done) cudaGraphSetConditional(h_while, 0);
    }
}

// A stop found at the start of a level (converged, capped or not finite):
// no selection; in a graph the loop ends.
__device__ __forceinline__ bool level_stopped(const SolveDesc *__restrict__ desc, SolveState *__restrict__ st,
                                              cudaGraphConditionalHandle h_while, cudaGraphConditionalHandle h_rec,
                                              int ctl) {
    const int done0 = st->done;
    const int stop = done0 ? done0 : (st->level >= desc->max_levels ? 2 : 0);
    if (!stop) return false;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->done = stop;
        st->push_count = 0;
        if (ctl == 1) {
            cudaGraphSetConditional(h_rec, 0);
            cudaGraphSetConditional(h_while, 0);
        }
    }
    return true;
}

template <typename FT>
__global__ void __launch_bounds__(kScanThreads, 4) k_scan_level(
    const SolveDesc *__restrict__ desc, SolveState *__restrict__ st, int32_t *__restrict__ front, int64_t n,
    double *__restrict__ part_sum, double *__restrict__ part_max, cudaGraphConditionalHandle h_while,
    cudaGraphConditionalHandle h_rec, int ctl) {
    if (level_stopped(desc, st, h_while, h_rec, ctl)) return;
    scan_select<FT>(desc, st, front, n, part_sum, part_max);
    if (!last_block(&st->scan_blocks)) return;
    scan_control(desc, st, part_sum, part_max, gridDim.x, h_while, h_rec, ctl);
}

// %globaltimer (ns), and acquire / release accesses of a flag at GPU scope
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Push of the asynchronous design, for every frontier node i: f =
// atomicExch(F_i, 0) (fluid that arrives after the exchange waits for a
// later level), H_i += f in FP64, and F_k += (d / outdeg_i) f for every
// out-edge i -> k with red.global.add.  Dynamic tiles of 256 frontier
// nodes; a row is pushed by its thread (outdeg <= 16), by a warp (<= 512)
// or by the whole CTA.  Targets of very high in-degree are accumulated in
// shared memory per CTA and flushed once.
// kSlice (slice sweeps): once every frontier tile is claimed, each CTA
// sweeps its own slice of the nodes (about n / gridDim consecutive ids) at
// the level's selection threshold, up to desc->slice_sweeps times, and
// diffuses what it finds through a shared-memory queue: the nodes whose
// fluid crossed T while the level pushed, which the sequential sweep of
// Sec. 2.4 diffuses in the same sweep.  No CTA waits for another: a node
// that crosses T after its slice was swept keeps its fluid for the next
// selection.  A CTA starts its first sweep once the pushes of half the
// frontier's tiles are done (a counter the tiles' CTAs advance after a
// fence; kSliceWaitPct): all tiles are claimed by then, so every CTA it waits
// for is running, and the wait gives up after desc->wait_ns, sweeping what
// has landed.  A node
// may be drained twice in a level (a frontier tile still running and a slice
// sweep; the second drain takes what arrived since, often nothing), so H_i
// is updated with an FP64 atomic add.
template <typename FT, bool kCG = false, bool kSlice = false>
__device__ __forceinline__ void push_frontier(const SolveDesc *__restrict__ desc, SolveState *__restrict__ st,
                                              const int32_t *__restrict__ front, const int32_t *__restrict__ rp,
                                              const int32_t *__restrict__ pcol, const int32_t *__restrict__ hot_node,
                                              int n_hot, const FT *__restrict__ scale) {
    const int count = __ldcg(&st->push_count);
    if (count == 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FT *s_hot = reinterpret_cast<FT *>(smem_raw);
    // fluid window of the tile: targets in [lo - R, lo - R + span) with lo the
    // tile's first frontier node (span = kPushWin + 2R, 0 when R = 0)
    const int R = kSlice ? 0 : desc->win_R;
    const unsigned span = R > 0 ? (unsigned)(kPushWin + 2 * R) : 0u;
    FT *s_win = s_hot + push_hot_pad(n_hot);
    // slice-sweep queue (kSlice), in place of the window
    int32_t *s_sq = reinterpret_cast<int32_t *>(s_hot + push_hot_pad(n_hot));
    // thread 0's claims: the claimed tiles [s_tile, s_tile + s_unit), the next of them, the
    // number of claims, frontier exhausted
    __shared__ long long s_tile;
    __shared__ int s_unit, s_sub, s_claims, s_gdone;
    __shared__ int s_qn, s_src, s_first, s_sqn, s_sbase, s_sbt, s_sweep, s_waited;
    __shared__ long long s_pos, s_seg;
    __shared__ int32_t s_qb[kPushThreads], s_qe[kPushThreads];
    __shared__ FT s_qw[kPushThreads];
    __shared__ double s_dang;    // fluid drained from dangling nodes (1/N completion)
    double my_dang = 0.0;        // this thread's share, added to s_dang once per warp at the end

    FT *__restrict__ F = static_cast<FT *>(desc->F);
    double *__restrict__ H = desc->H;
    const int64_t n = desc->n_nodes;
    const int lane = threadIdx.x & 31;
    // the CTA's slice [s_lo, s_hi), a multiple of 4 nodes long (vector loads;
    // the fluid vector is padded with zeros to a multiple of 4)
    const int64_t per = kSlice ? ((n + gridDim.x - 1) / gridDim.x + 3) / 4 * 4 : 0;
    const int64_t s_lo = kSlice ? min(n, (int64_t)blockIdx.x * per) : 0;
    const int64_t s_hi = kSlice ? min(n, s_lo + per) : 0;
    if (threadIdx.x == 0) {   // ordered before any use by the loop's first barrier
        s_dang = 0.0;
        s_unit = 0;
        s_sub = 0;
        s_claims = 0;
        s_gdone = 0;
        s_sqn = 0;
        s_sweep = 0;
        s_waited = 0;
        s_pos = s_lo;
    }
    for (int sl = threadIdx.x; sl < n_hot; sl += kPushThreads) s_hot[sl] = FT(0);
    for (unsigned q = threadIdx.x; !kSlice && q < span; q += kPushThreads) s_win[q] = FT(0);   // (no window with slice sweeps)
    const uint64_t keep = l2_keep_policy();
    const int thread_max = desc->thread_max, warp_max = desc->warp_max;
    // sweeps only after a dense frontier (at least 1/kSliceDensity of the nodes):
    // on a sparse one the fluid that crossed T is scarce and a sweep reads all of F
    const int sweeps = kSlice && (int64_t)count * kSliceDensity >= n ? desc->slice_sweeps : 0;
    const FT Tc = kSlice ? thr_cast(__ldcg(&st->T_push), FT(0)) : FT(0);
    unsigned long long my_edges = 0, my_nodes = 0, my_reds = 0, my_slice = 0;
    int64_t wlo = 0;

    auto push1 = [&](int32_t c, FT w) {
        if (c < 0) {
            atomicAdd(&s_hot[-1 - c], w);
            return;
        }
        const uint64_t o = (uint64_t)((int64_t)c - wlo);
        if (!kSlice && o < span) {
            atomicAdd(&s_win[o], w);
        } else {
            red_add_keep(F + c, w, keep);
            ++my_reds;
        }
    };

    // thread 0 picks the work of each step: a frontier tile.  Tiles are
    // claimed in pairs, pushed one after the other (fluid a tile sends to the
    // next tile's nodes then goes with them in the same level), while more
    // than four pairs per CTA remain, and one at a time after that, so that
    // the last tiles spread over the CTAs.  A CTA's first claim is its block
    // index (no atomic at the start), later ones come from the shared
    // counter.  With
    // kSlice, a full queue batch first, then once the frontier is exhausted
    // the slice's segments of 1024 nodes (select into the queue), the queue's
    // rest after each sweep, and the next sweep
    for (;;) {
        if (threadIdx.x == 0) {
            s_qn = 0;
            int src = 2;
            const int qn = kSlice ? min(s_sqn, kSliceQueueCap) : 0;
            if (kSlice && qn >= kPushThreads) {
                src = 1;
            } else if (!s_gdone) {
                if (s_sub >= s_unit) {
                    const int64_t ntiles = ((int64_t)count + kPushThreads - 1) / kPushThreads;
                    const int64_t grid = gridDim.x;
                    const int u0 = ntiles >= 2 * grid ? 2 : 1;   // the static first claim
                    if (s_claims == 0) {
                        s_unit = u0;
                        s_tile = (int64_t)blockIdx.x * u0;
                    } else {
                        const int u = s_tile + 8 * grid < ntiles ? 2 : 1;
                        s_unit = u;
                        s_tile = grid * u0 + (int64_t)atomicAdd(&st->tile_ctr, (unsigned)u);
                    }
                    ++s_claims;
                    s_sub = 0;
                }
                const int64_t first = (s_tile + s_sub++) * kPushThreads;
                if (first < count) {
                    src = 0;
                    s_first = (int)first;
                } else {
                    s_gdone = 1;
                }
            }
            if (kSlice && src == 2 && s_gdone) {
                if (!s_waited && sweeps > 0) {
                    // half of the frontier's pushes first (bounded by the timer and a poll
                    // count): the sweep then overlaps the frontier's tail, and a node the
                    // tail pushes over T later keeps its fluid for the next selection
                    const unsigned ntiles = (unsigned)((count + kPushThreads - 1) / kPushThreads);
                    const unsigned long long t0 = global_ns(), limit = desc->wait_ns;
                    const unsigned long long max_polls = (limit >> 5) + 1024ull;
                    unsigned long long polls = 0;
                    while ((unsigned long long)ld_acquire_gpu(&st->tiles_done) * 100ull < (unsigned long long)ntiles * kSliceWaitPct &&
                           global_ns() - t0 <= limit &&
                           ++polls <= max_polls)
                        __nanosleep(64);
                    s_waited = 1;
                }
                while (s_sweep < sweeps) {
                    if (s_pos < s_hi) {
                        src = 3;
                        s_seg = s_pos;
                        s_pos += 4 * kPushThreads;
                        break;
                    }
                    if (qn > 0) {
                        src = 1;
                        break;
                    }
                    ++s_sweep;   // the slice is swept and its finds are pushed: sweep again
                    s_pos = s_lo;
                }
            }
            if (src == 1) {   // the queue's top batch
                const int bt = min(qn, kPushThreads);
                s_sbase = qn - bt;
                s_sbt = bt;
                s_sqn = qn - bt;
            }
            s_src = src;
        }
        __syncthreads();
        const int src = s_src;
        if (src == 2) break;
        if (kSlice && src == 3) {
            // select |F_i| >= T over 1024 nodes of the slice into the queue (reads
            // past L1: the other CTAs' pushes land in L2)
            const int64_t i0 = s_seg + 4 * (int64_t)threadIdx.x;
            unsigned msk = 0;
            if (i0 < s_hi) {
                Vec4<FT> f;
                f.load_cg(F + i0);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const FT a = fabs(f.v[j]);
                    if (i0 + j < s_hi && a >= Tc && a > FT(0)) msk |= 1u << j;
                }
            }
            const int c = __popc(msk);
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            int base = 0;
            if (lane == 31 && incl > 0) base = atomicAdd(&s_sqn, incl);
            int pos = __shfl_sync(0xffffffffu, base, 31) + incl - c;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if ((msk >> j) & 1u) {
                    if (pos < kSliceQueueCap) s_sq[pos] = static_cast<int32_t>(i0 + j);   // a full queue drops
                    ++pos;
                }
            __syncthreads();
            continue;
        }
        int32_t node = -1;
        if (src == 0) {
            const int64_t first = s_first;
            // the frontier of a CTA's scan slice is in node order, so in a dense
            // level the tile's nodes (and most of their near targets) fall in the window
            if (span) wlo = (int64_t)ld_mut<kCG>(front + first) - R;
            const int64_t idx = first + threadIdx.x;
            if (idx < count) node = ld_mut<kCG>(front + idx);
        } else if (kSlice && (int)threadIdx.x < s_sbt) {
            node = s_sq[s_sbase + threadIdx.x];
        }
        int32_t b = 0, e = 0;
        FT w = FT(0);
        if (node >= 0) {
            const int32_t i = node;
            b = __ldcs(rp + i);
            e = __ldcs(rp + i + 1);
            const FT f = atomic_exch_keep(F + i, FT(0), keep);
            const double fd = static_cast<double>(f);
            if (kSlice) {
                if (f != FT(0)) {
                    atomicAdd(H + i, fd);   // a node may be drained twice in a level
                    if (e == b && desc->dangling) my_dang += fd;
                    my_nodes += 1;
                    my_edges += static_cast<unsigned long long>(e - b);
                    my_slice += src == 1 ? 1u : 0u;
                } else {
                    e = b;   // drained already: nothing to send
                }
            } else {
                __stcs(H + i, ld_mut<kCG>(H + i) + fd);   // i appears once per frontier
                if (e == b && desc->dangling) my_dang += fd;   // 1/N completion
                my_nodes += 1;
                my_edges += static_cast<unsigned long long>(e - b);
            }
            w = f * __ldcs(scale + i);
        }
        const int deg = e - b;
        if (deg <= thread_max) {
            auto pw = [&](int32_t c) { push1(c, w); };
            push_range<8>(pcol, b, e, 1, pw);
        }
        const bool wrow = deg > thread_max && deg <= warp_max;
        if (__any_sync(0xffffffffu, wrow)) {
            // the warp's medium rows as one edge-parallel range: lane L's row holds
            // the edges [ex_L, ex_L + len_L) of the concatenation, and each lane
            // finds the row of its edge by a binary search over the offsets, so
            // the rows' column loads are in flight together (4 per lane)
            const int len = wrow ? deg : 0;
            int incl = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int ex = incl - len, total = __shfl_sync(0xffffffffu, incl, 31);
            for (int q0 = 0; q0 < total; q0 += 4 * 32) {
                int32_t c[4];
                FT cw[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int q = q0 + 32 * k + lane;
                    int owner = 0;   // the last lane whose offset is <= q (rows are non-empty)
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const int cand = owner + step;
                        const int cex = __shfl_sync(0xffffffffu, ex, cand & 31);
                        if (cand < 32 && cex <= q) owner = cand;
                    }
                    const int32_t ob = __shfl_sync(0xffffffffu, b, owner);
                    const int oex = __shfl_sync(0xffffffffu, ex, owner);
                    cw[k] = __shfl_sync(0xffffffffu, w, owner);
                    c[k] = q < total ? __ldcs(pcol + (int64_t)ob + (q - oex)) : 0;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (q0 + 32 * k + lane < total) push1(c[k], cw[k]);
            }
        }
        if (deg > warp_max) {
            const int slot = atomicAdd(&s_qn, 1);
            s_qb[slot] = b;
            s_qe[slot] = e;
            s_qw[slot] = w;
        }
        __syncthreads();
        const int qn = s_qn;
        for (int h = 0; h < qn; ++h) {
            const int32_t hb = s_qb[h], he = s_qe[h];
            const FT hw = s_qw[h];
            auto pw = [&](int32_t c) { push1(c, hw); };
            push_range<2>(pcol, (int64_t)hb + threadIdx.x, he, kPushThreads, pw);
        }
        __syncthreads();
        if (kSlice && src == 0 && threadIdx.x == 0) {
            __threadfence();   // the tile's adds, ordered by the barrier, before the count
            atomicAdd(&st->tiles_done, 1u);
        }
        // flush the window and clear it: consecutive threads, consecutive nodes
        // (coalesced reductions, eight FP32 or four FP64 words per sector)
        for (unsigned q = threadIdx.x; !kSlice && q < span; q += kPushThreads) {
            const FT v = s_win[q];
            s_win[q] = FT(0);
            const int64_t wnode = wlo + q;
            const bool go = v != FT(0) && wnode >= 0 && wnode < n;
            const unsigned m = __ballot_sync(0xffffffffu, go);
            if (lane == 0) {
                constexpr int per_sector = 32 / (int)sizeof(FT);
                for (int g = 0; g < 32; g += per_sector)
                    my_reds += ((m >> g) & ((1u << per_sector) - 1u)) ? 1u : 0u;
            }
            if (go) red_add_keep(F + wnode, v, keep);
        }
    }
    my_dang = warp_sum(my_dang);   // 1/N completion: one shared add per warp
    if ((threadIdx.x & 31) == 0 && my_dang != 0.0) atomicAdd(&s_dang, my_dang);
    __syncthreads();
    for (int sl = threadIdx.x; sl < n_hot; sl += kPushThreads) {
        const FT v = s_hot[sl];
        if (v != FT(0)) {
            red_add_keep(F + hot_node[sl], v, keep);
            ++my_reds;
        }
    }
    cta_add_counts(&st->node_diff, my_nodes, &st->edge_diff, my_edges, &st->red_ops, my_reds,
                   kSlice ? &st->slice_nodes : nullptr, my_slice);
    if (threadIdx.x == 0 && s_dang != 0.0) atomicAdd(&st->dang_acc, s_dang);
}

template <typename FT, bool kSlice>
__global__ void __launch_bounds__(kPushThreads, 6)
    k_push_async(const SolveDesc *__restrict__ desc, SolveState *__restrict__ st, const int32_t *__restrict__ front,
                 const int32_t *__restrict__ rp, const int32_t *__restrict__ pcol,
                 const int32_t *__restrict__ hot_node, int n_hot, const FT *__restrict__ scale) {
    // launched with programmatic dependence on the selection kernel: wait for
    // it (and its writes) before anything is read; a no-op otherwise
    asm volatile("griddepcontrol.wait;" ::: "memory");
    push_frontier<FT, false, kSlice>(desc, st, front, rp, pcol, hot_node, n_hot, scale);
}

// ------------------------------------------------------------------ persistent level loop (propagation 7)

// Grid barrier of a cooperative launch (every CTA resident).  The last CTA to
// arrive runs control() with all its threads (it sees every write made
// before the barrier), then releases the others by advancing the generation.
// The wait is bounded: after timeout_ns of %globaltimer a waiting CTA records
// the timeout and every CTA leaves the loop at its next check (no spin is
// unbounded, so a lost CTA cannot hang the device).  Returns false on a
// timeout.
template <typename Control>
__device__ __forceinline__ bool grid_barrier(SolveState *st, unsigned long long timeout_ns, Control control) {
    __shared__ unsigned s_gen;
    __shared__ int s_last, s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_gen = ld_acquire_gpu(&st->bar_gen);
        __threadfence();
        const unsigned arrived = atomicAdd(&st->bar_count, 1u) + 1u;
        s_last = arrived == gridDim.x;
        s_ok = 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        if (threadIdx.x == 0) st->bar_count = 0;
        control();
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            st_release_gpu(&st->bar_gen, s_gen + 1u);
        }
    } else if (threadIdx.x == 0) {
        const unsigned long long t0 = global_ns();
        // bounded twice: by the timer and by the number of polls (each sleeps >= ~32 ns)
        const unsigned long long max_polls = (timeout_ns >> 5) + 1024ull;
        unsigned long long polls = 0;
        while (ld_acquire_gpu(&st->bar_gen) == s_gen) {
            if (global_ns() - t0 > timeout_ns || ++polls > max_polls) {
                atomicExch(&st->timed_out, 1);
                s_ok = 0;
                break;
            }
            __nanosleep(64);
        }
    }
    // one decision per CTA (another CTA may set the flag at any time); the
    // CTA's later reads of shared state go to L2 (.cg), ordered after thread
    // 0's acquire by the block barrier
    if (threadIdx.x == 0 && __ldcg(&st->timed_out)) s_ok = 0;
    __syncthreads();
    return s_ok != 0;
}

// The level loop of propagation 3 in one cooperative launch: every pass is a
// selection phase (frontier compaction, |F|_1 and max) and, when the control
// pushes, a push phase of the asynchronous design, separated by grid
// barriers whose last CTA runs the control.  The kernel returns when the
// control asks for an exact FP64 residual (a stop to confirm or a
// refinement) or the solve ended; a CUDA graph runs the residual in an IF
// node and relaunches it in its WHILE node.  The controller also adds the
// wall time of each phase (%globaltimer) to the solve state.
template <typename FT, bool kSlice>
__global__ void __launch_bounds__(kPushThreads, sizeof(FT) == 8 ? 4 : 6) k_levels_coop(
    const SolveDesc *__restrict__ desc, SolveState *__restrict__ st, int32_t *__restrict__ front,
    const int32_t *__restrict__ rp, const int32_t *__restrict__ pcol, const int32_t *__restrict__ hot_node, int n_hot,
    const FT *__restrict__ scale, int64_t n, double *__restrict__ part_sum, double *__restrict__ part_max,
    unsigned long long timeout_ns, cudaGraphConditionalHandle h_while, cudaGraphConditionalHandle h_rec, int ctl) {
    if (level_stopped(desc, st, h_while, h_rec, ctl)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->t_mark = global_ns();
    bool ok = true;
    for (;;) {
        scan_select<FT, true>(desc, st, front, n, part_sum, part_max);
        ok = grid_barrier(st, timeout_ns, [&] {
            scan_control(desc, st, part_sum, part_max, gridDim.x, h_while, h_rec, 0);
            if (threadIdx.x == 0) {
                const unsigned long long t = global_ns();
                st->t_scan_ns = __ldcg(&st->t_scan_ns) + (t - __ldcg(&st->t_mark));
                st->t_mark = t;
                st->passes = __ldcg(&st->passes) + 1;
            }
        });
        if (!ok) break;
        if (__ldcg(&st->push_count) > 0) {
            push_frontier<FT, true, kSlice>(desc, st, front, rp, pcol, hot_node, n_hot, scale);
            ok = grid_barrier(st, timeout_ns, [&] {
                if (threadIdx.x == 0) {
                    const unsigned long long t = global_ns();
                    st->t_push_ns = __ldcg(&st->t_push_ns) + (t - __ldcg(&st->t_mark));
                    st->t_mark = t;
                }
            });
            if (!ok) break;
        }
        if (__ldcg(&st->done) || __ldcg(&st->do_recompute)) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (!ok || __ldcg(&st->timed_out)) {
            st->done = 4;          // a grid barrier gave up (here or in another CTA): DI_ETIMEOUT
            st->do_recompute = 0;
        }
        if (ctl == 1) {
            cudaGraphSetConditional(h_rec, __ldcg(&st->do_recompute) ? 1u : 0u);
            if (__ldcg(&st->done)) cudaGraphSetConditional(h_while, 0);
        }
    }
}

// Push of the asynchronous design, warp-level form: every warp claims
// kWarpGrab frontier entries with one atomic and takes them 32 at a time
// (drain: f = atomicExch(F_i, 0), H_i += f), so drains and pushes interleave
// finely and fluid that arrives before a node's turn goes with it.  A row of
// at most thread_max edges is pushed by its own lane; a longer one by the
// whole warp (coalesced column loads).  No block-wide barrier inside the
// loop; hot targets accumulate in shared memory and are flushed at the end.
constexpr int kWarpGrab = 128;

template <typename FT>
__global__ void __launch_bounds__(kPushThreads) k_push_warp(const SolveDesc *__restrict__ desc, SolveState *__restrict__ st,
                                                      const int32_t *__restrict__ front,
                                                      const int32_t *__restrict__ rp,
                                                      const int32_t *__restrict__ pcol,
                                                      const int32_t *__restrict__ hot_node, int n_hot,
                                                      const FT *__restrict__ scale) {
    const int count = st->push_count;
    if (count == 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FT *s_hot = reinterpret_cast<FT *>(smem_raw);
    __shared__ double s_dang;    // fluid drained from dangling nodes (1/N completion)
    double my_dang = 0.0;        // this thread's share, added to s_dang once per warp at the end
    if (threadIdx.x == 0) s_dang = 0.0;
    for (int sl = threadIdx.x; sl < n_hot; sl += kPushThreads) s_hot[sl] = FT(0);
    __syncthreads();
    FT *__restrict__ F = static_cast<FT *>(desc->F);
    double *__restrict__ H = desc->H;
    const int lane = threadIdx.x & 31;
    const uint64_t keep = l2_keep_policy();
    const int thread_max = desc->thread_max;
    auto push1 = [&](int32_t c, FT w) {
        if (c >= 0) red_add_keep(F + c, w, keep);
        else atomicAdd(&s_hot[-1 - c], w);
    };
    // claim size: 128 entries on large frontiers, down to 32 when the frontier
    // would leave warps idle
    const int nwarps = (int)(gridDim.x * (kPushThreads / 32));
    int grab = count / (nwarps * 4);
    grab = grab < 32 ? 32 : (grab > kWarpGrab ? kWarpGrab : grab & ~31);
    unsigned long long my_edges = 0, my_nodes = 0;
    for (;;) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(&st->tile_ctr, (unsigned)grab);
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((int64_t)base >= count) break;
#pragma unroll 1
        for (int sub = 0; sub < grab; sub += 32) {
            const int64_t idx = (int64_t)base + sub + lane;
            int32_t b = 0, e = 0;
            FT w = FT(0);
            if (idx < count) {
                const int32_t i = __ldcs(front + idx);
                b = __ldcs(rp + i);
                e = __ldcs(rp + i + 1);
                const FT f = atomic_exch_keep(F + i, FT(0), keep);
                __stcs(H + i, __ldcs(H + i) + static_cast<double>(f));   // i appears once per frontier
                w = f * __ldcs(scale + i);
                my_nodes += 1;
                my_edges += static_cast<unsigned long long>(e - b);
                if (e == b && desc->dangling) my_dang += static_cast<double>(f);   // 1/N completion
            }
            const int deg = e - b;
            if (deg <= thread_max) {
                auto pw = [&](int32_t c) { push1(c, w); };
                push_range<8>(pcol, b, e, 1, pw);
            }
            unsigned wm = __ballot_sync(0xffffffffu, deg > thread_max);
            while (wm) {
                const int src = __ffs(wm) - 1;
                wm &= wm - 1;
                const int32_t mb = __shfl_sync(0xffffffffu, b, src), me = __shfl_sync(0xffffffffu, e, src);
                const FT mw = __shfl_sync(0xffffffffu, w, src);
                auto pw = [&](int32_t c) { push1(c, mw); };
            push_range<4>(pcol, (int64_t)mb + lane, me, 32, pw);
            }
        }
    }
    my_dang = warp_sum(my_dang);   // 1/N completion: one shared add per warp
    if ((threadIdx.x & 31) == 0 && my_dang != 0.0) atomicAdd(&s_dang, my_dang);
    __syncthreads();
    for (int sl = threadIdx.x; sl < n_hot; sl += kPushThreads) {
        const FT v = s_hot[sl];
        if (v != FT(0)) red_add_keep(F + hot_node[sl], v, keep);
    }
    cta_add_counts(&st->node_diff, my_nodes, &st->edge_diff, my_edges);
    if (threadIdx.x == 0 && s_dang != 0.0) atomicAdd(&st->dang_acc, s_dang);
}

// One threshold level in one launch (propagation 5): every CTA walks its
// 2048-node chunks of the fluid in grid-stride order, selects |F_i| >= T
// (the L1 norm and max of what it reads go to the control step) and pushes
// the nodes it selected at once: f = atomicExch(F_i, 0), H_i += f, and
// F_k += (d / outdeg_i) f over the out-row, by the node's lane for a row of
// at most thread_max edges and by the whole warp for a longer one.  There is
// no frontier list and no separate scan launch; fluid that reaches a chunk
// before the CTA reads it is selected in this level, fluid that arrives
// later waits for the next (any order converges, Sec. 2).  The last CTA to
// finish runs the control step of the level.
template <typename FT>
__global__ void __launch_bounds__(kPushThreads) k_level_fused(
    const SolveDesc *__restrict__ desc, SolveState *__restrict__ st, const int32_t *__restrict__ rp,
    const int32_t *__restrict__ pcol, const int32_t *__restrict__ hot_node, int n_hot, const FT *__restrict__ scale,
    int64_t n, double *__restrict__ part_sum, double *__restrict__ part_max, cudaGraphConditionalHandle h_while,
    cudaGraphConditionalHandle h_rec, int ctl) {
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
    using AT = typename Acc<FT>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FT *s_hot = reinterpret_cast<FT *>(smem_raw);
    for (int sl = threadIdx.x; sl < n_hot; sl += kPushThreads) s_hot[sl] = FT(0);
    __syncthreads();
    FT *__restrict__ F = static_cast<FT *>(desc->F);
    double *__restrict__ H = desc->H;
    const FT Tc = thr_cast(st->T, FT(0));
    const int lane = threadIdx.x & 31;
    // 1/N completion (Sec. 2.2): the fluid dangling nodes drained in the previous
    // level reaches every node as d / N of it, added atomically (other CTAs push
    // concurrently); what this level drains goes to dang_next
    const int dangling = desc->dangling;
    const FT u = dangling ? static_cast<FT>(desc->d * st->dang_acc / (double)n) : FT(0);
    __shared__ double s_dang;
    if (threadIdx.x == 0) s_dang = 0.0;
    double my_dang = 0.0;        // this thread's share, added to s_dang once per warp at the end
    const uint64_t keep = l2_keep_policy();
    const int thread_max = desc->thread_max;
    auto push1 = [&](int32_t c, FT w) {
        if (c >= 0) red_add_keep(F + c, w, keep);
        else atomicAdd(&s_hot[-1 - c], w);
    };
    AT acc = 0;
    FT mx = 0;
    unsigned long long my_edges = 0, my_nodes = 0;
    for (int64_t c0 = (int64_t)blockIdx.x * kScanChunk; c0 < n; c0 += (int64_t)gridDim.x * kScanChunk) {
#pragma unroll 1
        for (int k = 0; k < kScanItems; ++k) {
            const int64_t idx = c0 + k * kPushThreads + threadIdx.x;
            FT v = FT(0);
            if (idx < n) {
                if (u != FT(0)) atomicAdd(F + idx, u);
                v = __ldcg(F + idx);
            }
            const FT a = fabs(v);
            acc += static_cast<AT>(a);
            mx = max(mx, a);
            const bool sel = idx < n && a >= Tc && a > FT(0);
            if (!__any_sync(0xffffffffu, sel)) continue;
            int32_t b = 0, e = 0;
            FT w = FT(0);
            if (sel) {
                b = __ldcs(rp + idx);
                e = __ldcs(rp + idx + 1);
                const FT f = atomic_exch_keep(F + idx, FT(0), keep);
                __stcs(H + idx, __ldcs(H + idx) + static_cast<double>(f));
                w = f * __ldcs(scale + idx);
                my_nodes += 1;
                my_edges += static_cast<unsigned long long>(e - b);
                if (e == b && dangling) my_dang += static_cast<double>(f);
            }
            const int deg = e - b;
            if (deg <= thread_max) {
                auto pw = [&](int32_t c) { push1(c, w); };
                push_range<8>(pcol, b, e, 1, pw);
            }
            unsigned wm = __ballot_sync(0xffffffffu, deg > thread_max);
            while (wm) {
                const int src = __ffs(wm) - 1;
                wm &= wm - 1;
                const int32_t mb = __shfl_sync(0xffffffffu, b, src), me = __shfl_sync(0xffffffffu, e, src);
                const FT mw = __shfl_sync(0xffffffffu, w, src);
                auto pw = [&](int32_t c) { push1(c, mw); };
                push_range<4>(pcol, (int64_t)mb + lane, me, 32, pw);
            }
        }
    }
    my_dang = warp_sum(my_dang);   // 1/N completion: one shared add per warp
    if ((threadIdx.x & 31) == 0 && my_dang != 0.0) atomicAdd(&s_dang, my_dang);
    __syncthreads();
    for (int sl = threadIdx.x; sl < n_hot; sl += kPushThreads) {
        const FT hv = s_hot[sl];
        if (hv != FT(0)) red_add_keep(F + hot_node[sl], hv, keep);
    }
    cta_add_counts(&st->node_diff, my_nodes, &st->edge_diff, my_edges, &st->lvl_nodes, my_nodes);
    if (threadIdx.x == 0 && s_dang != 0.0) atomicAdd(&st->dang_next, s_dang);   // after cta_add_counts' barriers
    double s = static_cast<double>(acc);
    double m = static_cast<double>(mx);
    block_sum_max<kPushThreads>(s, m);
    if (threadIdx.x == 0) { part_sum[blockIdx.x] = s; part_max[blockIdx.x] = m; }
    if (!last_block(&st->scan_blocks)) return;
    double ts = 0.0, tm = 0.0;
    for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) { ts += part_sum[i]; tm = fmax(tm, part_max[i]); }
    block_sum_max<kPushThreads>(ts, tm);
    if (threadIdx.x != 0) return;

    // control step after the level's pushes
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

// ------------------------------------------------------------------ one threshold level

constexpr int kLevelThreads = 256;
constexpr int kChunkNodes = 32;    // nodes per warp chunk of the sparse push
constexpr int kRanges = 64;        // chunk counters (contiguous node ranges)

enum : int { P2_NONE = 0, P2_PULL = 1, P2_PUSH = 2 };

// Selection and drain (Sec. 2.4 selection, Eqs. defF/defH drain): for every
// node with |F_i| >= T: H_i += F_i, F_i = 0, w_i = (d / outdeg_i) F_i; every
// other node has w_i = 0.  The same read gives the L1 norm and max of the
// fluid at the start of the level.  The last CTA then decides the next
// steps on the device: how to propagate w (gather over the in-edges when the
// active edges are a large share of all edges, scatter from the active nodes
// otherwise), the next threshold, and whether an exact FP64 residual must
// follow (FP32 fluid refresh, or confirmation of a stop).

// Selection and drain (Sec. 2.4 selection, Eqs. defF/defH drain): for every
// node with |F_i| >= T: H_i += F_i, F_i = 0, w_i = (d / outdeg_i) F_i; every
// other node has w_i = 0.  The same read gives the L1 norm and max of the
// fluid at the start of the level.  Four nodes per thread with vector loads;
// the history updates of the selected ones are independent loads/stores.
// The last CTA then decides the next steps on the device: how to propagate w
// (gather over the in-edges when the active edges are a large share of all
// edges, scatter from the active nodes otherwise), the next threshold, and
// whether an exact FP64 residual must follow (FP32 fluid refresh, or
// confirmation of a stop).
template <typename FT>
__global__ void __launch_bounds__(kLevelThreads) k_select(
    const SolveDesc *__restrict__ desc, SolveState *__restrict__ st, const int32_t *__restrict__ outdeg,
    const FT *__restrict__ scale, FT *__restrict__ w, int64_t n, int64_t nnz, double *__restrict__ part_sum,
    double *__restrict__ part_max, cudaGraphConditionalHandle h_while, cudaGraphConditionalHandle h_p2,
    cudaGraphConditionalHandle h_rec, int ctl) {
    using AT = typename Acc<FT>::T;
    {
        const int done0 = st->done;
        const int stop = done0 ? done0 : (st->level >= desc->max_levels ? 2 : 0);
        if (stop) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                st->done = stop;
                st->p2mode = P2_NONE;
                if (ctl == 1) {
                    cudaGraphSetConditional(h_p2, 0);
                    cudaGraphSetConditional(h_rec, 0);
                    cudaGraphSetConditional(h_while, 0);
                }
            }
            return;
        }
    }
    FT *__restrict__ F = static_cast<FT *>(desc->F);
    double *__restrict__ H = desc->H;
    const FT Tc = thr_cast(st->T, FT(0));
    AT acc = 0;
    FT mx = 0;
    unsigned long long my_edges = 0, my_nodes = 0;
    const int64_t n4 = n / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride) {
        const int64_t i0 = 4 * q;
        Vec4<FT> f, sc, wv;
        f.load(F + i0);
        sc.load_cs(scale + i0);
        const int4 dg = __ldcs(reinterpret_cast<const int4 *>(outdeg) + q);
        const int degs[4] = {dg.x, dg.y, dg.z, dg.w};
        unsigned selm = 0;
        double h[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const FT a = fabs(f.v[k]);
            acc += static_cast<AT>(a);
            mx = max(mx, a);
            if (a >= Tc && a > FT(0)) selm |= 1u << k;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {   // independent loads of the selected histories
            const bool sel = (selm >> k) & 1u;
            h[k] = sel ? __ldcs(H + i0 + k) : 0.0;
            wv.v[k] = sel ? f.v[k] * sc.v[k] : FT(0);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if ((selm >> k) & 1u) {
                __stcs(H + i0 + k, h[k] + static_cast<double>(f.v[k]));
                my_nodes += 1;
                my_edges += static_cast<unsigned long long>(degs[k]);
                f.v[k] = FT(0);
            }
        }
        if (selm) f.store(F + i0);
        wv.store(w + i0);
    }
    // tail (n not a multiple of 4)
    for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const FT v = F[i];
        const FT a = fabs(v);
        acc += static_cast<AT>(a);
        mx = max(mx, a);
        FT wvi = FT(0);
        if (a >= Tc && a > FT(0)) {
            __stcs(H + i, __ldcs(H + i) + static_cast<double>(v));
            F[i] = FT(0);
            wvi = v * scale[i];
            my_nodes += 1;
            my_edges += static_cast<unsigned long long>(outdeg[i]);
        }
        w[i] = wvi;
    }
    cta_add_counts(&st->node_diff, my_nodes, &st->edge_diff, my_edges, &st->lvl_nodes, my_nodes, &st->lvl_edges,
                   my_edges);
    double s = static_cast<double>(acc);
    double m = static_cast<double>(mx);
    block_sum_max<kLevelThreads>(s, m);
    if (threadIdx.x == 0) { part_sum[blockIdx.x] = s; part_max[blockIdx.x] = m; }
    if (!last_block(&st->scan_blocks)) return;
    double ts = 0.0, tm = 0.0;
    for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) { ts += part_sum[i]; tm = fmax(tm, part_max[i]); }
    block_sum_max<kLevelThreads>(ts, tm);
    if (threadIdx.x != 0) return;

    // control of the next steps (all loads first: one round trip)
    const unsigned long long lnodes = st->lvl_nodes, ledges = st->lvl_edges;
    double T = st->T;
    int level = st->level, since = st->since_recompute, iters = st->body_iters;
    const double est = st->est_scale > 1.0 ? st->est_scale : 1.0;
    const double tol = desc->tol, alpha = desc->alpha;
    const int max_iters = desc->max_body_iters;
    int done = 0, rec = 0, p2 = P2_NONE;
    if (!isfinite(ts)) {
        done = 3;
    } else {
        if (lnodes > 0) {
            level += 1;
            since += 1;
            T = T / alpha;
            p2 = desc->propagation != 2 &&
                         ledges * (unsigned long long)desc->push_ratio >= (unsigned long long)nnz
                     ? P2_PULL
                     : P2_PUSH;
            if (ledges == 0) p2 = P2_NONE;      // only dangling nodes drained
        } else if (tm > 0.0) {
            // empty level: next T is the first T / alpha^k <= max |F| (tm > 0, so
            // at most ~3600 steps from any double down to the smallest denormal)
            for (int guard = 0; T > tm && guard < 8192; ++guard) T /= alpha;
            if (T > tm) T = tm;   // alpha so close to 1 that the guard ran out
        }
        if (ts * est <= tol) {
            rec = 1;                      // stop request: confirm on the exact residual
            st->confirming = 1;
            st->r_confirm = ts * est;
        } else if (refine_due(desc, st, since, ts * est)) {
            rec = 1;
        }
    }
    iters += 1;
    if (!done && iters >= max_iters) done = 2;
    if (done) rec = 0;
    // with done set here nothing was drained (non-finite) or the cap is hit
    // after this level's drain: the propagation below still runs
    st->r_scan = ts;
    st->max_scan = tm;
    st->T = T;
    st->level = level;
    st->since_recompute = since;
    st->body_iters = iters;
    st->lvl_nodes = 0;
    st->lvl_edges = 0;
    st->p2mode = p2;
    st->do_recompute = rec;
    if (done) st->done = done;
    if (ctl == 1) {
        cudaGraphSetConditional(h_p2, p2 == P2_PULL ? 1u : 0u);
        cudaGraphSetConditional(h_rec, rec ? 1u : 0u);
        if (done) cudaGraphSetConditional(h_while, 0);
    }
}

// Dense propagation: F_k += sum of w_j over the in-edges j -> k (binned
// gather, pull.cuh).  Each row has one owner, except the longest rows whose
// segments add their partial sums with red.global.add.
template <typename FT>
__global__ void __launch_bounds__(kPullThreads, 4) k_pull_level(const PullPlan pl, const SolveDesc *__restrict__ desc,
                                                             const SolveState *__restrict__ st,
                                                             const int32_t *__restrict__ in_rp,
                                                             const int32_t *__restrict__ in_col,
                                                             const FT *__restrict__ w) {
    if (st->p2mode != P2_PULL) return;
    FT *__restrict__ F = static_cast<FT *>(desc->F);
    auto emit = [&](int32_t k, FT acc) {
        if (acc != FT(0)) F[k] += acc;
    };
    auto seg = [&](int64_t, int32_t k, FT acc) {
        if (acc != FT(0)) red_add(F + k, acc);
    };
    pull_plan<FT>(pl, in_rp, in_col, w, emit, seg);
}

// Dense propagation, flat form: each thread takes 16 consecutive in-edges
// (vector loads of their sources and destination rows), gathers the 16
// values of w independently, sums runs of equal destination and adds each
// run with one red.global.add.  Perfectly balanced whatever the in-degrees;
// the reds of a warp land on neighbouring rows.
constexpr int kFlatEdges = 16;

template <typename FT>
__global__ void __launch_bounds__(kLevelThreads) k_pull_flat(const SolveDesc *__restrict__ desc,
                                                             const SolveState *__restrict__ st,
                                                             const int32_t *__restrict__ in_col,
                                                             const int32_t *__restrict__ erow,
                                                             const FT *__restrict__ w, int64_t nnz) {
    if (st->p2mode != P2_PULL) return;
    FT *__restrict__ F = static_cast<FT *>(desc->F);
    const int64_t nchunks = (nnz + kFlatEdges - 1) / kFlatEdges;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks; c += stride) {
        const int64_t e0 = c * kFlatEdges;
        int32_t col[kFlatEdges], row[kFlatEdges];
        if (e0 + kFlatEdges <= nnz) {
#pragma unroll
            for (int v = 0; v < kFlatEdges / 4; ++v) {
                const int4 a = __ldcs(reinterpret_cast<const int4 *>(in_col + e0) + v);
                const int4 b = __ldcs(reinterpret_cast<const int4 *>(erow + e0) + v);
                col[4 * v] = a.x; col[4 * v + 1] = a.y; col[4 * v + 2] = a.z; col[4 * v + 3] = a.w;
                row[4 * v] = b.x; row[4 * v + 1] = b.y; row[4 * v + 2] = b.z; row[4 * v + 3] = b.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < kFlatEdges; ++k) {
                const bool ok = e0 + k < nnz;
                col[k] = ok ? in_col[e0 + k] : 0;
                row[k] = ok ? erow[e0 + k] : -1;
            }
        }
        FT val[kFlatEdges];
#pragma unroll
        for (int k = 0; k < kFlatEdges; ++k) val[k] = row[k] >= 0 ? w[col[k]] : FT(0);
        int32_t cur = row[0];
        FT acc = val[0];
#pragma unroll
        for (int k = 1; k < kFlatEdges; ++k) {
            if (row[k] != cur) {
                if (cur >= 0 && acc != FT(0)) red_add(F + cur, acc);
                cur = row[k];
                acc = val[k];
            } else {
                acc += val[k];
            }
        }
        if (cur >= 0 && acc != FT(0)) red_add(F + cur, acc);
    }
}

// Edge-parallel push of the out-edges of up to 32 nodes held one per lane
// (b, deg, w; deg = 0 for an idle lane).  The warp walks the concatenation
// of the 32 rows 32 edges at a time: edge e belongs to the first lane whose
// inclusive degree prefix exceeds e (5-step search over the lanes'
// prefixes), so column loads are coalesced and each lane issues an
// independent red whatever the mix of degrees.
template <typename FT>
__device__ __forceinline__ void push_rows(FT *__restrict__ F, FT *s_hot, const int32_t *__restrict__ pcol,
                                          int32_t b, int deg, FT w, int lane) {
    int incl = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int excl = incl - deg;
    const int32_t off = b - excl;   // column position of edge e of this lane's row: off + e
    auto src_of = [&](int e) {      // number of lanes whose inclusive prefix is <= e
        int src = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int v = __shfl_sync(0xffffffffu, incl, src + step - 1);
            if (v <= e) src += step;
        }
        return src < 31 ? src : 31;
    };
    auto push1 = [&](int32_t c, FT wv) {
        if (c >= 0) red_add(F + c, wv);
        else atomicAdd(&s_hot[-1 - c], wv);
    };
    for (int base = 0; base < total; base += 64) {
        const int e0 = base + lane, e1 = base + 32 + lane;
        const int s0 = src_of(e0), s1 = src_of(e1);
        const int32_t o0 = __shfl_sync(0xffffffffu, off, s0), o1 = __shfl_sync(0xffffffffu, off, s1);
        const FT w0 = __shfl_sync(0xffffffffu, w, s0), w1 = __shfl_sync(0xffffffffu, w, s1);
        const bool ok0 = e0 < total, ok1 = e1 < total;
        const int32_t c0 = ok0 ? __ldcs(pcol + o0 + e0) : 0;
        const int32_t c1 = ok1 ? __ldcs(pcol + o1 + e1) : 0;
        if (ok0) push1(c0, w0);
        if (ok1) push1(c1, w1);
    }
}

// Sparse propagation: F_k += w_j for every out-edge j -> k of the nodes with
// w_j != 0.  Warps claim 32-node chunks from kRanges range counters, find
// the active nodes with a ballot and push their rows edge-parallel.  Targets
// of very high in-degree are accumulated in shared memory per CTA and
// flushed once at the end.
template <typename FT>
__global__ void __launch_bounds__(kLevelThreads, 4) k_pushw(const SolveDesc *__restrict__ desc,
                                                            SolveState *__restrict__ st,
                                                            const int32_t *__restrict__ rp,
                                                            const int32_t *__restrict__ pcol,
                                                            const int32_t *__restrict__ hot_node, int n_hot,
                                                            const FT *__restrict__ w, int64_t n) {
    if (st->p2mode != P2_PUSH) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FT *s_hot = reinterpret_cast<FT *>(smem_raw);
    for (int sl = threadIdx.x; sl < n_hot; sl += kLevelThreads) s_hot[sl] = FT(0);
    __syncthreads();
    FT *__restrict__ F = static_cast<FT *>(desc->F);
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * kLevelThreads + threadIdx.x) >> 5);
    const int64_t nchunks = (n + kChunkNodes - 1) / kChunkNodes;
    const int nranges = (int)(nchunks < kRanges ? nchunks : kRanges);
    const int64_t per_range = (nchunks + nranges - 1) / nranges;
    for (int t = 0; t < nranges; ++t) {
        const int r = (gwarp + t) % nranges;
        const int64_t r_hi = (int64_t)(r + 1) * per_range;
        const int64_t r_end = r_hi < nchunks ? r_hi : nchunks;
        for (;;) {
            unsigned k = 0;
            if (lane == 0) k = atomicAdd(&st->rctr[r], 1u);
            k = __shfl_sync(0xffffffffu, k, 0);
            const int64_t chunk = (int64_t)r * per_range + k;
            if (chunk >= r_end) break;
            const int64_t i = chunk * kChunkNodes + lane;
            FT wv = FT(0);
            if (i < n) wv = w[i];
            if (!__ballot_sync(0xffffffffu, wv != FT(0))) continue;
            int32_t b = 0;
            int deg = 0;
            if (wv != FT(0)) {
                b = __ldcs(rp + i);
                deg = __ldcs(rp + i + 1) - b;
            }
            push_rows<FT>(F, s_hot, pcol, b, deg, wv, lane);
        }
    }
    __syncthreads();
    for (int sl = threadIdx.x; sl < n_hot; sl += kLevelThreads) {
        const FT v = s_hot[sl];
        if (v != FT(0)) red_add(F + hot_node[sl], v);
    }
    if (!last_block(&st->push_blocks)) return;
    for (int r = threadIdx.x; r < kRanges; r += kLevelThreads) st->rctr[r] = 0;
}

// ------------------------------------------------------------------ host side

// L2 access-policy windows: the sparse push scatters into the fluid F and
// the dense pull gathers from the drained vector w, so each keeps its own
// target resident while the column indices stream past it.  Attached to
// each launch, so they are captured into graph nodes and also apply to
// host-driven launches.  which: 0 = F, 1 = w.
const cudaAccessPolicyWindow *l2_window(di_graph *g, int which, int fp64, int enabled) {
    if (!enabled) return nullptr;
    const int slot = 2 * which + fp64;
    if (!g->win_ready[slot]) {
        g->win_ready[slot] = 1;
        g->win_ok[slot] = 0;
        int max_persist = 0, max_window = 0;
        cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, g->device);
        cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, g->device);
        const size_t bytes = (size_t)g->n * (fp64 ? sizeof(double) : sizeof(float));
        void *base = which == 0 ? (fp64 ? (void *)g->ws.F64 : (void *)g->ws.F32)
                                : (fp64 ? (void *)g->ws.w64 : (void *)g->ws.w32);
        if (max_persist > 0 && max_window > 0 && base) {
            const size_t limit = std::min<size_t>((size_t)max_persist, bytes);
            size_t cur = 0;
            cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
            if (cur < limit) cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, limit);
            cudaAccessPolicyWindow &w = g->win[slot];
            w.base_ptr = base;
            w.num_bytes = std::min<size_t>(bytes, (size_t)max_window);
            w.hitRatio = (float)std::min(1.0, (double)limit / (double)w.num_bytes);
            w.hitProp = cudaAccessPropertyPersisting;
            w.missProp = cudaAccessPropertyStreaming;
            g->win_ok[slot] = 1;
        }
        cudaGetLastError();   // the window is an optimisation; a refusal is not an error
    }
    return g->win_ok[slot] ? &g->win[slot] : nullptr;
}

// kPDL: programmatic dependent launch - the kernel's CTAs may be scheduled
// while the previous kernel on the stream finishes; the kernel itself waits
// for that kernel's completion (griddep_wait) before it reads anything.
template <bool kPDL = false, typename Kern, typename... Args>
void launch_ex(Kern kernel, int grid, int block, size_t smem, cudaStream_t s, const cudaAccessPolicyWindow *win,
               Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    int na = 0;
    if (win) {
        attr[na].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[na].val.accessPolicyWindow = *win;
        ++na;
    }
    if (kPDL) {
        attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[na].val.programmaticStreamSerializationAllowed = 1;
        ++na;
    }
    cfg.attrs = na ? attr : nullptr;
    cfg.numAttrs = na;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename FT>
void launch_async(di_graph *g, cudaStream_t s, cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hr, int ctl,
                  int l2, int prop, cudaEvent_t mid = nullptr) {
    Workspace &ws = g->ws;
    const cudaAccessPolicyWindow *win = l2_window(g, 0, sizeof(FT) == 8, l2);
    launch_ex(k_scan_level<FT>, g->grid_scan, kScanThreads, 0, s, nullptr, (const SolveDesc *)ws.desc, ws.st,
              ws.front, (int64_t)g->n, ws.part_sum, ws.part_max, hw, hr, ctl);
    if (mid) cudaEventRecord(mid, s);   // timing mode: end of the selection
    const FT *scale = sizeof(FT) == 4 ? reinterpret_cast<const FT *>(g->s32) : reinterpret_cast<const FT *>(g->s64);
    if (prop == 4)
        launch_ex(k_push_warp<FT>, push_grid(g), kPushThreads, g->n_hot * sizeof(FT), s, win,
                  (const SolveDesc *)ws.desc, ws.st, (const int32_t *)ws.front, (const int32_t *)g->rp,
                  (const int32_t *)g->pcol, (const int32_t *)g->hot_node, g->n_hot, scale);
    else if (g->push_slice)
        launch_ex<true>(k_push_async<FT, true>, push_grid(g, true), kPushThreads, push_smem<FT>(g->n_hot, 0, true), s,
                  win, (const SolveDesc *)ws.desc, ws.st, (const int32_t *)ws.front, (const int32_t *)g->rp,
                  (const int32_t *)g->pcol, (const int32_t *)g->hot_node, g->n_hot, scale);
    else
        launch_ex<true>(k_push_async<FT, false>, push_grid(g), kPushThreads, push_smem<FT>(g->n_hot, g->push_R), s, win,
                  (const SolveDesc *)ws.desc, ws.st, (const int32_t *)ws.front, (const int32_t *)g->rp,
                  (const int32_t *)g->pcol, (const int32_t *)g->hot_node, g->n_hot, scale);
}

template <typename FT>
void launch_fused(di_graph *g, cudaStream_t s, cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hr, int ctl,
                  int l2) {
    Workspace &ws = g->ws;
    const cudaAccessPolicyWindow *win = l2_window(g, 0, sizeof(FT) == 8, l2);
    const FT *scale = sizeof(FT) == 4 ? reinterpret_cast<const FT *>(g->s32) : reinterpret_cast<const FT *>(g->s64);
    const int grid = std::max(1, std::min(push_grid(g), (int)((g->n + kScanChunk - 1) / kScanChunk)));
    launch_ex(k_level_fused<FT>, grid, kPushThreads, g->n_hot * sizeof(FT), s, win, (const SolveDesc *)ws.desc, ws.st,
              (const int32_t *)g->rp, (const int32_t *)g->pcol, (const int32_t *)g->hot_node, g->n_hot, scale,
              (int64_t)g->n, ws.part_sum, ws.part_max, hw, hr, ctl);
}

// Chunk size and grid of the tiled level kernel for this graph and fluid
// precision (after ensure_window): the largest C in {256, ..., 32} that still
// gives every warp of the occupancy-limited grid four chunks or more.
template <typename FT>
di_status prepare_tiled(di_graph *g) {
    const int fp64 = sizeof(FT) == 8;
    if (g->tiled_chunk[fp64]) return DI_OK;
    const int R = g->win_R;
    // the attribute is per function, shared by every graph: the largest layout
    DI_CUDA_TRY(cudaFuncSetAttribute(k_level_tiled<FT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)tiled_smem<FT>(kMaxHot, 256, kMaxWinR)));
    auto grid_for_chunk = [&](int C, int *grid) -> di_status {
        const size_t smem = tiled_smem<FT>(g->n_hot, C, R);
        int per_sm = 0;
        DI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_level_tiled<FT>, kPushThreads, smem));
        *grid = std::max(1, per_sm) * g->num_sms;
        return DI_OK;
    };
    int C = 256, grid = 0;
    DI_TRY(grid_for_chunk(C, &grid));
    while (C > 32 && g->n / C < 4LL * kTiledWarps * grid) C /= 2;
    DI_TRY(grid_for_chunk(C, &grid));
    const int64_t chunks = (g->n + C - 1) / C;
    g->tiled_chunk[fp64] = C;
    g->grid_tiled[fp64] = (int)std::max<int64_t>(1, std::min<int64_t>(grid, (chunks + kTiledWarps - 1) / kTiledWarps));
    return DI_OK;
}

template <typename FT>
void launch_tiled(di_graph *g, cudaStream_t s, cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hr, int ctl,
                  int l2) {
    Workspace &ws = g->ws;
    const int fp64 = sizeof(FT) == 8;
    const cudaAccessPolicyWindow *win = l2_window(g, 0, fp64, l2);
    const FT *scale = sizeof(FT) == 4 ? reinterpret_cast<const FT *>(g->s32) : reinterpret_cast<const FT *>(g->s64);
    const int C = g->tiled_chunk[fp64], R = g->win_R;
    launch_ex(k_level_tiled<FT>, g->grid_tiled[fp64], kPushThreads, tiled_smem<FT>(g->n_hot, C, R), s, win,
              (const SolveDesc *)ws.desc, ws.st, (const int32_t *)g->rp, (const int32_t *)g->pcol,
              (const int32_t *)g->hot_node, g->n_hot, scale, (int64_t)g->n, C, R, ws.part_sum, ws.part_max, hw, hr,
              ctl);
}

// Grid of the persistent level loop: every CTA must be resident at once (a
// cooperative launch), so the occupancy maximum of the kernel with its hot
// slots, on every SM.
template <typename FT>
di_status prepare_coop(di_graph *g) {
    const int fp64 = sizeof(FT) == 8;
    int per_sm = 0;
    if (g->push_slice)
        DI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_levels_coop<FT, true>, kPushThreads,
                                                                  push_smem<FT>(g->n_hot, 0, true)));
    else
        DI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_levels_coop<FT, false>, kPushThreads,
                                                                  push_smem<FT>(g->n_hot, g->push_R)));
    if (per_sm < 1) { set_error("persistent level loop: the kernel does not fit on an SM"); return DI_ECUDA; }
    // the push shape's CTAs per SM (di_tune) caps the grid, as for the push kernels
    if (g->tune.push_ctas_per_sm > 0) per_sm = std::min(per_sm, g->tune.push_ctas_per_sm);
    g->grid_coop[fp64] = per_sm * g->num_sms;
    return DI_OK;
}

template <typename FT>
void launch_coop(di_graph *g, cudaStream_t s, cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hr, int ctl,
                 int l2, unsigned long long timeout_ns) {
    Workspace &ws = g->ws;
    const int fp64 = sizeof(FT) == 8;
    const cudaAccessPolicyWindow *win = l2_window(g, 0, fp64, l2);
    const FT *scale = sizeof(FT) == 4 ? reinterpret_cast<const FT *>(g->s32) : reinterpret_cast<const FT *>(g->s64);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g->grid_coop[fp64]);
    cfg.blockDim = dim3(kPushThreads);
    cfg.dynamicSmemBytes = g->push_slice ? push_smem<FT>(g->n_hot, 0, true) : push_smem<FT>(g->n_hot, g->push_R);
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    int na = 0;
    attr[na].id = cudaLaunchAttributeCooperative;
    attr[na].val.cooperative = 1;
    ++na;
    if (win) {
        attr[na].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[na].val.accessPolicyWindow = *win;
        ++na;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    if (g->push_slice)
        cudaLaunchKernelEx(&cfg, k_levels_coop<FT, true>, (const SolveDesc *)ws.desc, ws.st, ws.front,
                           (const int32_t *)g->rp, (const int32_t *)g->pcol, (const int32_t *)g->hot_node, g->n_hot,
                           scale, (int64_t)g->n, ws.part_sum, ws.part_max, timeout_ns, hw, hr, ctl);
    else
        cudaLaunchKernelEx(&cfg, k_levels_coop<FT, false>, (const SolveDesc *)ws.desc, ws.st, ws.front,
                           (const int32_t *)g->rp, (const int32_t *)g->pcol, (const int32_t *)g->hot_node, g->n_hot,
                           scale, (int64_t)g->n, ws.part_sum, ws.part_max, timeout_ns, hw, hr, ctl);
}

template <typename FT>
void launch_select(di_graph *g, cudaStream_t s, cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hp,
                   cudaGraphConditionalHandle hr, int ctl, int) {
    const cudaAccessPolicyWindow *win = nullptr;   // elementwise streaming pass
    Workspace &ws = g->ws;
    const FT *scale = sizeof(FT) == 4 ? reinterpret_cast<const FT *>(g->s32) : reinterpret_cast<const FT *>(g->s64);
    FT *w = sizeof(FT) == 4 ? reinterpret_cast<FT *>(ws.w32) : reinterpret_cast<FT *>(ws.w64);
    launch_ex(k_select<FT>, g->grid_select, kLevelThreads, 0, s, win, (const SolveDesc *)ws.desc, ws.st,
              (const int32_t *)g->outdeg, scale, w, (int64_t)g->n, (int64_t)g->nnz, ws.part_sum, ws.part_max, hw, hp,
              hr, ctl);
}

template <typename FT>
void launch_pull(di_graph *g, cudaStream_t s, int l2, int propagation) {
    const cudaAccessPolicyWindow *win = l2_window(g, 1, sizeof(FT) == 8, l2);
    if (propagation == 1) {
        Workspace &ws = g->ws;
        const FT *w = sizeof(FT) == 4 ? reinterpret_cast<const FT *>(ws.w32) : reinterpret_cast<const FT *>(ws.w64);
        launch_ex(k_pull_flat<FT>, g->grid_flat, kLevelThreads, 0, s, win, (const SolveDesc *)ws.desc,
                  (const SolveState *)ws.st, (const int32_t *)g->in_col, (const int32_t *)g->erow, w,
                  (int64_t)g->nnz);
        return;
    }
    Workspace &ws = g->ws;
    const FT *w = sizeof(FT) == 4 ? reinterpret_cast<const FT *>(ws.w32) : reinterpret_cast<const FT *>(ws.w64);
    launch_ex(k_pull_level<FT>, g->grid_pull, kPullThreads, 0, s, win, pull_plan_of(g), (const SolveDesc *)ws.desc,
              (const SolveState *)ws.st, (const int32_t *)g->in_rp, (const int32_t *)g->in_col, w);
}

template <typename FT>
void launch_pushw(di_graph *g, cudaStream_t s, int l2) {
    const cudaAccessPolicyWindow *win = l2_window(g, 0, sizeof(FT) == 8, l2);
    Workspace &ws = g->ws;
    const FT *w = sizeof(FT) == 4 ? reinterpret_cast<const FT *>(ws.w32) : reinterpret_cast<const FT *>(ws.w64);
    launch_ex(k_pushw<FT>, g->grid_pushw, kLevelThreads, g->n_hot * sizeof(FT), s, win, (const SolveDesc *)ws.desc,
              ws.st, (const int32_t *)g->rp, (const int32_t *)g->pcol, (const int32_t *)g->hot_node, g->n_hot, w,
              (int64_t)g->n);
}

di_status build_level_graph(di_graph *g, int fp64, int l2, int prop) {
    SolverGraph &sg = g->sg[fp64];
    if (sg.built && sg.l2 == l2 && sg.prop == prop && sg.res_form == g->res_form && sg.grid_push == push_grid(g) &&
        sg.timeout_ns == g->coop_timeout_ns && sg.grid_coop == g->grid_coop[fp64] && sg.slice == g->push_slice)
        return DI_OK;
    if (sg.built) {   // rebuilt with the other window setting
        cudaGraphExecDestroy(sg.exec);
        cudaGraphDestroy(sg.graph);
        sg = SolverGraph();
    }
    cudaStream_t cs = nullptr;
    DI_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } sgd{cs};
    const int win = l2;
    // resolve the windows now: their set-up calls are not allowed during capture
    l2_window(g, 0, fp64, win);
    l2_window(g, 1, fp64, win);
    DI_CUDA_TRY(cudaGraphCreate(&sg.graph, 0));
    DI_CUDA_TRY(cudaGraphConditionalHandleCreate(&sg.h_while, sg.graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = sg.h_while;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    DI_CUDA_TRY(cudaGraphAddNode(&wnode, sg.graph, nullptr, nullptr, 0, &wp));
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    if (prop < 3) DI_CUDA_TRY(cudaGraphConditionalHandleCreate(&sg.h_p2, body, 0, 0));
    DI_CUDA_TRY(cudaGraphConditionalHandleCreate(&sg.h_if, body, 0, 0));

    cudaGraphNodeParams pp = {};
    cudaGraphNodeParams ip = {};
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    cudaGraph_t capg = nullptr;
    cudaGraph_t ended = nullptr;
    DI_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    if (prop == 7) {
        // body: k_levels_coop (passes until a residual is due) -> IF(exact residual)
        if (fp64) launch_coop<double>(g, cs, sg.h_while, sg.h_if, 1, win, g->coop_timeout_ns);
        else launch_coop<float>(g, cs, sg.h_while, sg.h_if, 1, win, g->coop_timeout_ns);
    } else if (prop == 6) {
        // body: k_level_tiled -> IF(exact residual)
        if (fp64) launch_tiled<double>(g, cs, sg.h_while, sg.h_if, 1, win);
        else launch_tiled<float>(g, cs, sg.h_while, sg.h_if, 1, win);
    } else if (prop == 5) {
        // body: k_level_fused -> IF(exact residual)
        if (fp64) launch_fused<double>(g, cs, sg.h_while, sg.h_if, 1, win);
        else launch_fused<float>(g, cs, sg.h_while, sg.h_if, 1, win);
    } else if (prop >= 3) {
        // body: k_scan_level -> k_push_async (or k_push_warp) -> IF(exact residual)
        if (fp64) launch_async<double>(g, cs, sg.h_while, sg.h_if, 1, win, prop);
        else launch_async<float>(g, cs, sg.h_while, sg.h_if, 1, win, prop);
    } else {
        // body: k_select -> IF/ELSE(pull | push) -> IF(exact residual)
        if (fp64) launch_select<double>(g, cs, sg.h_while, sg.h_p2, sg.h_if, 1, win);
        else launch_select<float>(g, cs, sg.h_while, sg.h_p2, sg.h_if, 1, win);
        DI_CUDA_TRY(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &capg, &deps, nullptr, &ndeps));
        pp.type = cudaGraphNodeTypeConditional;
        pp.conditional.handle = sg.h_p2;
        pp.conditional.type = cudaGraphCondTypeIf;
        pp.conditional.size = 2;                  // [0]: condition != 0 (pull), [1]: else (push)
        cudaGraphNode_t pnode;
        DI_CUDA_TRY(cudaGraphAddNode(&pnode, capg, deps, nullptr, ndeps, &pp));
        DI_CUDA_TRY(cudaStreamUpdateCaptureDependencies(cs, &pnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    }
    DI_CUDA_TRY(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &capg, &deps, nullptr, &ndeps));
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = sg.h_if;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t inode;
    DI_CUDA_TRY(cudaGraphAddNode(&inode, capg, deps, nullptr, ndeps, &ip));
    DI_CUDA_TRY(cudaStreamUpdateCaptureDependencies(cs, &inode, nullptr, 1, cudaStreamSetCaptureDependencies));
    // propagations 3 and 4: kLevelsPerIter levels per WHILE iteration (fewer
    // conditional re-evaluations); when the loop ends at an earlier level, the
    // later levels' kernels return at once (their selection sees the stop)
    cudaGraphNodeParams ipk[kLevelsPerIter - 1] = {};
    const int extra_levels = (prop == 3 || prop == 4) ? kLevelsPerIter - 1 : 0;
    for (int q = 0; q < extra_levels; ++q) {
        DI_CUDA_TRY(cudaGraphConditionalHandleCreate(&sg.h_ifk[q], body, 0, 0));
        if (fp64) launch_async<double>(g, cs, sg.h_while, sg.h_ifk[q], 1, win, prop);
        else launch_async<float>(g, cs, sg.h_while, sg.h_ifk[q], 1, win, prop);
        DI_CUDA_TRY(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &capg, &deps, nullptr, &ndeps));
        ipk[q].type = cudaGraphNodeTypeConditional;
        ipk[q].conditional.handle = sg.h_ifk[q];
        ipk[q].conditional.type = cudaGraphCondTypeIf;
        ipk[q].conditional.size = 1;
        cudaGraphNode_t inode_q;
        DI_CUDA_TRY(cudaGraphAddNode(&inode_q, capg, deps, nullptr, ndeps, &ipk[q]));
        DI_CUDA_TRY(cudaStreamUpdateCaptureDependencies(cs, &inode_q, nullptr, 1, cudaStreamSetCaptureDependencies));
    }
    DI_CUDA_TRY(cudaStreamEndCapture(cs, &ended));

    if (prop < 3) {
        DI_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, pp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal));
        if (fp64) launch_pull<double>(g, cs, win, prop); else launch_pull<float>(g, cs, win, prop);
        DI_CUDA_TRY(cudaStreamEndCapture(cs, &ended));
        DI_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, pp.conditional.phGraph_out[1], nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal));
        if (fp64) launch_pushw<double>(g, cs, win); else launch_pushw<float>(g, cs, win);
        DI_CUDA_TRY(cudaStreamEndCapture(cs, &ended));
    }
    DI_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal));
    launch_residual(g, fp64, RES_LEVEL, cs);
    DI_CUDA_TRY(cudaStreamEndCapture(cs, &ended));
    for (int q = 0; q < extra_levels; ++q) {
        DI_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, ipk[q].conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal));
        launch_residual(g, fp64, RES_LEVEL, cs);
        DI_CUDA_TRY(cudaStreamEndCapture(cs, &ended));
    }

    DI_CUDA_TRY(cudaGetLastError());
    DI_CUDA_TRY(cudaGraphInstantiate(&sg.exec, sg.graph, 0));
    sg.built = true;
    sg.l2 = l2;
    sg.prop = prop;
    sg.res_form = g->res_form;
    sg.grid_push = push_grid(g);
    sg.timeout_ns = g->coop_timeout_ns;
    sg.grid_coop = g->grid_coop[fp64];
    sg.slice = g->push_slice;
    return DI_OK;
}

template <typename T>
cudaError_t dmalloc(T **p, size_t count) {
    return cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(count, 1) * sizeof(T));
}

int occupancy_grid(const void *fn, int threads, size_t smem, int sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return per_sm * sms;
}

di_status check_solve_args(di_graph *g, const double *B, double d, double tol, double *H, const di_opts *o) {
    if (!g || !B || !H) { set_error("di_solve: NULL graph, B or H"); return DI_EINVAL; }
    if (!(d > 0.0 && d < 1.0)) { set_error("di_solve: d = %g outside (0, 1)", d); return DI_EINVAL; }
    if (!(tol > 0.0) || !std::isfinite(tol)) { set_error("di_solve: tol = %g must be finite and > 0", tol); return DI_EINVAL; }
    if (!(o->alpha > 1.0) || !std::isfinite(o->alpha)) { set_error("di_solve: alpha = %g must be > 1", o->alpha); return DI_EINVAL; }
    if (o->max_levels < 0 || o->recompute_every < 0) { set_error("di_solve: negative max_levels or recompute_every"); return DI_EINVAL; }
    if (!(o->recompute_drop == 0.0 || (o->recompute_drop > 1.0 && std::isfinite(o->recompute_drop)))) {
        set_error("di_solve: recompute_drop = %g must be 0 or a finite factor > 1", o->recompute_drop);
        return DI_EINVAL;
    }
    if (o->propagation < 0 || o->propagation > 7) { set_error("di_solve: propagation = %d outside [0, 7]", o->propagation); return DI_EINVAL; }
    if (o->spin_limit < 0 || o->spin_limit > (1LL << 40)) {
        set_error("di_solve: spin_limit = %lld outside [0, 2^40] us", o->spin_limit);
        return DI_EINVAL;
    }
    if (o->exact_residual < 0 || o->exact_residual > 2) { set_error("di_solve: exact_residual = %d outside [0, 2]", o->exact_residual); return DI_EINVAL; }
    if (o->resweeps < 0 || o->resweeps > 8) { set_error("di_solve: resweeps = %d outside [0, 8]", o->resweeps); return DI_EINVAL; }
    if (o->selection < 0 || o->selection > 1) { set_error("di_solve: selection = %d outside [0, 1]", o->selection); return DI_EINVAL; }
    if (o->slice_sweeps < -1 || o->slice_sweeps > 4) {
        set_error("di_solve: slice_sweeps = %d outside [-1, 4]", o->slice_sweeps);
        return DI_EINVAL;
    }
    if (o->slice_sweeps > 0 && ((o->propagation != 3 && o->propagation != 7) || o->selection != 0)) {
        set_error("di_solve: slice sweeps need propagation 3 or 7 and selection 0 (got %d, %d)",
                  o->propagation, o->selection);
        return DI_EINVAL;
    }
    if (o->dangling < 0 || o->dangling > 1) { set_error("di_solve: dangling = %d outside [0, 1]", o->dangling); return DI_EINVAL; }
    if (o->dangling == 1 && (o->propagation < 3 || o->exact_residual == 1)) {
        set_error("di_solve: the 1/N dangling completion needs propagation 3 to 7 and exact_residual 0 or 2 "
                  "(got %d, %d)", o->propagation, o->exact_residual);
        return DI_EINVAL;
    }
    if (o->selection == 1 && o->propagation != 3 && o->propagation != 4 && o->propagation != 7) {
        set_error("di_solve: the weighted selection needs propagation 3, 4 or 7 (got %d)", o->propagation);
        return DI_EINVAL;
    }
    return DI_OK;
}

}  // namespace

// Push grid: the occupancy maximum, or the tuned CTAs per SM below it.
int push_grid(const di_graph *g, bool slice) {
    const int occ = slice ? g->grid_push_slice : g->grid_push;
    const int want = g->tune.push_ctas_per_sm > 0 ? g->tune.push_ctas_per_sm * g->num_sms : occ;
    return std::max(1, std::min(occ, want));
}

di_status ensure_workspace(di_graph *g) {
    Workspace &ws = g->ws;
    if (ws.ready) return DI_OK;
    const int64_t n = g->n;
    g->grid_scan = std::max(1, std::min<int>(occupancy_grid((const void *)k_scan_level<float>, kScanThreads, 0,
                                                            g->num_sms),
                                             (int)((n + kScanChunk - 1) / kScanChunk)));
    {
        const int sel = occupancy_grid((const void *)k_select<double>, kLevelThreads, 0, g->num_sms);
        g->grid_select =
            (int)std::max<int64_t>(1, std::min<int64_t>(sel, (n / 4 + kLevelThreads - 1) / kLevelThreads));
        const PullPlan pl = pull_plan_of(g);
        const int pull = occupancy_grid((const void *)k_pull_level<double>, kPullThreads, 0, g->num_sms);
        g->grid_pull = (int)std::max<int64_t>(1, std::min<int64_t>(pull, pl.task_off[5]));
        const int push = occupancy_grid((const void *)k_pushw<double>, kLevelThreads, kMaxHot * sizeof(double),
                                        g->num_sms);
        const int64_t chunks = (n + kChunkNodes - 1) / kChunkNodes;
        g->grid_pushw = (int)std::max<int64_t>(1, std::min<int64_t>(push, (chunks + 7) / 8));
        g->grid_push = occupancy_grid((const void *)k_push_async<double, false>, kPushThreads,
                                      push_smem<double>(kMaxHot, kMaxWinR), g->num_sms);
        g->grid_push_slice = occupancy_grid((const void *)k_push_async<double, true>, kPushThreads,
                                           push_smem<double>(kMaxHot, 0, true), g->num_sms);
        const int flat = occupancy_grid((const void *)k_pull_flat<double>, kLevelThreads, 0, g->num_sms);
        const int64_t fchunks = (g->nnz + kFlatEdges - 1) / kFlatEdges;
        g->grid_flat =
            (int)std::max<int64_t>(1, std::min<int64_t>(flat, (fchunks + kLevelThreads - 1) / kLevelThreads));
    }
    g->grid_res = residual_grid(g->num_sms);
    // one partial per CTA of every kernel that reduces across CTAs (the fused
    // level kernel runs on the push grid)
    // (the tiled kernel's grid is at most the occupancy of 256-thread CTAs, below 2048 per SM)
    const int parts = std::max({g->grid_scan, g->grid_select, residual_partials(g), g->grid_push, 8 * g->num_sms});
    const PullPlan pl = pull_plan_of(g);
    const int64_t nseg5 = pl.task_off[5] - pl.task_off[4];
    DI_CUDA_TRY(dmalloc(&ws.front, n));
    DI_CUDA_TRY(dmalloc(&ws.g, n));
    DI_CUDA_TRY(dmalloc(&ws.acc, n));
    DI_CUDA_TRY(dmalloc(&ws.seg_part, std::max<int64_t>({(int64_t)g->n_seg, nseg5, 1})));
    DI_CUDA_TRY(dmalloc(&ws.part_sum, parts));
    DI_CUDA_TRY(dmalloc(&ws.part_max, parts));
    DI_CUDA_TRY(dmalloc(&ws.desc, 1));
    DI_CUDA_TRY(dmalloc(&ws.st, 1));
    DI_CUDA_TRY(cudaMemset(ws.st, 0, sizeof(SolveState)));
    DI_CUDA_TRY(cudaMallocHost(&ws.desc_h, sizeof(SolveDesc)));
    DI_CUDA_TRY(cudaMallocHost(&ws.st_h, sizeof(SolveState)));
    DI_CUDA_TRY(cudaEventCreate(&ws.ev0));
    DI_CUDA_TRY(cudaEventCreate(&ws.ev1));
    ws.ready = true;
    return DI_OK;
}

}  // namespace di

using namespace di;

namespace {

di_status solve_impl(di_graph *g, const double *B, double d, double tol, double *H, double *F, const di_opts *opts,
                     di_stats *stats) {
    di_opts o;
    if (opts) o = *opts; else di_opts_default(&o);
    DI_TRY(check_solve_args(g, B, d, tol, H, &o));
    cudaStream_t s = as_stream(o.stream);
    int dev = -1;
    DI_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != g->device) { set_error("di_solve: graph lives on device %d, current is %d", g->device, dev); return DI_EINVAL; }
    DI_TRY(ensure_workspace(g));
    Workspace &ws = g->ws;
    const int fp64 = o.fluid_fp64 ? 1 : 0;
    // fluid vectors padded with zeros to a multiple of 4 nodes (vector loads of the selection)
    const int64_t npad = (g->n + 3) / 4 * 4;
    if (fp64 && !ws.F64) {
        DI_CUDA_TRY(dmalloc(&ws.F64, npad));
        DI_CUDA_TRY(cudaMemset(ws.F64, 0, npad * sizeof(double)));
    }
    if (fp64 && !ws.w64) DI_CUDA_TRY(dmalloc(&ws.w64, g->n));
    if (!fp64 && !ws.F32) {
        DI_CUDA_TRY(dmalloc(&ws.F32, npad));
        DI_CUDA_TRY(cudaMemset(ws.F32, 0, npad * sizeof(float)));
    }
    if (!fp64 && !ws.w32) DI_CUDA_TRY(dmalloc(&ws.w32, g->n));
    DI_TRY(ensure_scale(g, d, s));
    if (o.selection == 1) DI_TRY(ensure_selection_weights(g, s));
    g->res_form = o.exact_residual;
    if (g->res_form != 1) DI_TRY(ensure_blocked_order(g, s));
    if (o.propagation == 6) {
        DI_TRY(ensure_window(g, s));
        DI_TRY(fp64 ? prepare_tiled<double>(g) : prepare_tiled<float>(g));
    }
    g->push_R = 0;
    // slice sweeps: -1 (auto) takes one where they apply and nothing else
    // re-orders the level (no re-selection, no fluid window)
    const bool frontier_push = o.propagation == 3 || o.propagation == 7;
    const int slice_sweeps = o.slice_sweeps >= 0 ? o.slice_sweeps
                           : (frontier_push && o.selection == 0 && o.resweeps == 0 && !g->tune.push_window) ? 1 : 0;
    g->push_slice = frontier_push && slice_sweeps > 0;
    if ((o.propagation == 3 || o.propagation == 7) && g->tune.push_window && !g->push_slice) {
        // the frontier push's fluid window (its radius follows the graph's locality)
        DI_TRY(ensure_window(g, s));
        g->push_R = g->win_R;
    }
    if (o.propagation == 7) {
        DI_TRY(fp64 ? prepare_coop<double>(g) : prepare_coop<float>(g));
        g->coop_timeout_ns = (unsigned long long)o.spin_limit * 1000ull;
    }
    if (!o.timing) DI_TRY(build_level_graph(g, fp64, o.l2_window, o.propagation));

    // descriptor (the previous call has completed: every solve synchronises)
    SolveDesc &dh = *ws.desc_h;
    std::memset(&dh, 0, sizeof(dh));
    dh.B = B;
    dh.H = H;
    dh.F_out = F;
    dh.F = fp64 ? (void *)ws.F64 : (void *)ws.F32;
    dh.d = d;
    dh.tol = tol;
    dh.alpha = o.alpha;
    dh.max_levels = o.max_levels;
    dh.recompute_every = o.recompute_every;
    dh.recompute_drop = o.recompute_drop;
    dh.fluid_fp64 = fp64;
    dh.max_body_iters = (int)std::min<long long>(4LL * o.max_levels + 1000, INT32_MAX);
    dh.propagation = o.propagation;
    dh.push_ratio = o.push_ratio > 0 ? o.push_ratio : 8;
    dh.n_nodes = g->n;
    dh.thread_max = g->tune.thread_max_deg;
    dh.warp_max = g->tune.warp_max_deg;
    dh.iw = o.selection == 1 ? (fp64 ? (const void *)g->iw64 : (const void *)g->iw32) : nullptr;
    dh.dangling = o.dangling;
    dh.resweeps = o.propagation >= 3 ? o.resweeps : 0;
    dh.win_R = (o.propagation == 3 || o.propagation == 7) ? g->push_R : 0;
    dh.slice_sweeps = g->push_slice ? slice_sweeps : 0;
    dh.wait_ns = (unsigned long long)o.spin_limit * 1000ull;
    DI_CUDA_TRY(cudaEventRecord(ws.ev0, s));
    DI_CUDA_TRY(cudaMemcpyAsync(ws.desc, ws.desc_h, sizeof(SolveDesc), cudaMemcpyHostToDevice, s));
    DI_CUDA_TRY(cudaMemsetAsync(ws.st, 0, sizeof(SolveState), s));

    int warm_used = 0;
    if (o.warm_start) {
        k_bnorm<<<g->grid_scan, kScanThreads, 0, s>>>(ws.desc, ws.st, g->n, ws.part_sum, ws.part_max);
        launch_residual(g, fp64, RES_WARM_INIT, s);   // F0 = B + P H0 - H0, T0 = max |F0|
        DI_CUDA_TRY(cudaGetLastError());
        DI_CUDA_TRY(cudaMemcpyAsync(ws.st_h, ws.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        DI_CUDA_TRY(cudaStreamSynchronize(s));
        const double f0 = ws.st_h->r_exact, b1 = ws.st_h->b_l1;
        warm_used = 1;
        if (!std::isfinite(f0)) {
            if (!o.warm_fallback) {
                set_error("di_solve: warm-start fluid is not finite");
                return DI_ENONFINITE;
            }
            warm_used = 0;
        } else if (o.warm_fallback && f0 > b1) {
            warm_used = 0;
        }
        if (!warm_used) {
            DI_CUDA_TRY(cudaMemsetAsync(ws.st, 0, sizeof(SolveState), s));
            if (fp64) k_init<double><<<g->grid_scan, kScanThreads, 0, s>>>(ws.desc, ws.st, g->n, ws.part_sum, ws.part_max);
            else k_init<float><<<g->grid_scan, kScanThreads, 0, s>>>(ws.desc, ws.st, g->n, ws.part_sum, ws.part_max);
        }
    } else {
        if (fp64) k_init<double><<<g->grid_scan, kScanThreads, 0, s>>>(ws.desc, ws.st, g->n, ws.part_sum, ws.part_max);
        else k_init<float><<<g->grid_scan, kScanThreads, 0, s>>>(ws.desc, ws.st, g->n, ws.part_sum, ws.part_max);
    }
    DI_CUDA_TRY(cudaGetLastError());

    double t_level = 0.0, t_rec = 0.0, t_sel = 0.0;
    int live_iters = 0;
    long long host_launches = 0;   // timing mode: kernels launched by the host loop
    if (!o.timing) {
        DI_CUDA_TRY(cudaGraphLaunch(g->sg[fp64].exec, s));
        DI_CUDA_TRY(cudaMemcpyAsync(ws.st_h, ws.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        DI_CUDA_TRY(cudaStreamSynchronize(s));
    } else {
        // host-driven levels, a CUDA event between every two kernels
        constexpr int kBatch = 16;
        const int win = o.l2_window;
        for (cudaEvent_t &e : ws.tev)
            if (!e) DI_CUDA_TRY(cudaEventCreate(&e));
        for (;;) {
            for (int l = 0; l < kBatch; ++l) {
                NvtxRange lr("level");
                cudaEvent_t *e = ws.tev + 4 * l;
                DI_CUDA_TRY(cudaEventRecord(e[0], s));
                DI_CUDA_TRY(cudaEventRecord(e[3], s));
                if (o.propagation == 7) {
                    if (fp64) launch_coop<double>(g, s, 0, 0, 2, win, g->coop_timeout_ns);
                    else launch_coop<float>(g, s, 0, 0, 2, win, g->coop_timeout_ns);
                } else if (o.propagation == 6) {
                    if (fp64) launch_tiled<double>(g, s, 0, 0, 2, win);
                    else launch_tiled<float>(g, s, 0, 0, 2, win);
                } else if (o.propagation == 5) {
                    if (fp64) launch_fused<double>(g, s, 0, 0, 2, win);
                    else launch_fused<float>(g, s, 0, 0, 2, win);
                } else if (o.propagation >= 3) {
                    if (fp64) launch_async<double>(g, s, 0, 0, 2, win, o.propagation, e[3]);
                    else launch_async<float>(g, s, 0, 0, 2, win, o.propagation, e[3]);
                } else if (fp64) {
                    launch_select<double>(g, s, 0, 0, 0, 2, win);
                    launch_pull<double>(g, s, win, o.propagation);
                    launch_pushw<double>(g, s, win);
                } else {
                    launch_select<float>(g, s, 0, 0, 0, 2, win);
                    launch_pull<float>(g, s, win, o.propagation);
                    launch_pushw<float>(g, s, win);
                }
                DI_CUDA_TRY(cudaEventRecord(e[1], s));
                {
                    NvtxRange rr("exact residual (if due)");
                    launch_residual(g, fp64, RES_LEVEL, s);
                }
                DI_CUDA_TRY(cudaEventRecord(e[2], s));
                host_launches += (o.propagation >= 5 ? 1 : o.propagation >= 3 ? 2 : 3) + residual_kernels(g);
            }
            DI_CUDA_TRY(cudaGetLastError());
            DI_CUDA_TRY(cudaMemcpyAsync(ws.st_h, ws.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
            DI_CUDA_TRY(cudaStreamSynchronize(s));
            const int live = std::min(kBatch, ws.st_h->body_iters - live_iters);
            for (int l = 0; l < live; ++l) {
                float a = 0.f, c = 0.f, sel = 0.f;
                cudaEvent_t *e = ws.tev + 4 * l;
                DI_CUDA_TRY(cudaEventElapsedTime(&a, e[0], e[1]));
                DI_CUDA_TRY(cudaEventElapsedTime(&c, e[1], e[2]));
                DI_CUDA_TRY(cudaEventElapsedTime(&sel, e[0], e[3]));
                t_level += a * 1e-3;
                t_rec += c * 1e-3;
                t_sel += sel * 1e-3;
            }
            live_iters = ws.st_h->body_iters;
            if (ws.st_h->done) break;
        }
    }
    SolveState st = *ws.st_h;
    const bool refresh = st.done != 1 || (F != nullptr && st.recomputes == 0);
    if (refresh) {
        // level cap, non-finite residual, or converged before any exact
        // recomputation wrote F: refresh F_out and the exact residual
        launch_residual(g, fp64, RES_FINAL, s);
        DI_CUDA_TRY(cudaGetLastError());
        DI_CUDA_TRY(cudaMemcpyAsync(ws.st_h, ws.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        DI_CUDA_TRY(cudaStreamSynchronize(s));
        st.r_exact = ws.st_h->r_exact;
    }
    DI_CUDA_TRY(cudaEventRecord(ws.ev1, s));
    DI_CUDA_TRY(cudaEventSynchronize(ws.ev1));
    float ms = 0.f;
    DI_CUDA_TRY(cudaEventElapsedTime(&ms, ws.ev0, ws.ev1));

    di_status rc = DI_OK;
    if (st.done == 4) {
        rc = DI_ETIMEOUT;
        set_error("di_solve: a grid barrier of the persistent level loop waited longer than %lld us",
                  (long long)o.spin_limit);
    } else if (st.done == 3 || !std::isfinite(st.r_exact)) {
        rc = DI_ENONFINITE;
        set_error("di_solve: residual is not finite (non-finite B or H0?)");
    } else if (st.done != 1) {
        rc = DI_ENOCONV;
        set_error("di_solve: level cap %d reached with |F|_1 = %g > tol = %g", o.max_levels, st.r_exact, tol);
    }
    if (stats) {
        stats->levels = st.level;
        stats->recomputes = st.recomputes;
        stats->node_diffusions = (int64_t)st.node_diff;
        stats->edge_diffusions = (int64_t)st.edge_diff;
        stats->resid_l1 = st.r_exact;
        stats->err_bound = st.r_exact / (1.0 - d);
        stats->b_l1 = st.b_l1;
        stats->f0_l1 = st.f0_l1;
        stats->seconds = ms * 1e-3;
        stats->warm_used = warm_used;
        stats->status = rc;
        const int rk = residual_kernels(g);
        long long launches = o.warm_start ? 1 + rk + (warm_used ? 0 : 1) : 1;   // start
        if (o.timing) {
            launches += host_launches;
        } else {
            // per live level: select + one propagation kernel; the level that
            // finds the loop finished; the exact residuals
            if (o.propagation == 7)   // one persistent launch per segment between exact residuals, plus the last
                launches += (long long)st.recomputes + 1 + 1 + (long long)rk * st.recomputes;
            else if (o.propagation == 3 || o.propagation == 4)   // kLevelsPerIter levels (2 kernels each) per iteration
                launches += 2LL * kLevelsPerIter * ((st.body_iters + kLevelsPerIter) / kLevelsPerIter) +
                            (long long)rk * st.recomputes;
            else
                launches += (o.propagation >= 5 ? 1LL : 2LL) * st.body_iters + 1 + (long long)rk * st.recomputes;
        }
        if (refresh) launches += rk;        // final residual refresh
        stats->gpu_launches = launches;
        stats->level_seconds = t_level;
        stats->recompute_seconds = t_rec;
        stats->level_launches = o.timing ? live_iters : 0;
        stats->recompute_launches = st.recomputes;
        stats->body_iterations = st.body_iters;
        stats->select_seconds = t_sel;
        stats->red_ops = (int64_t)st.red_ops;
        stats->slice_nodes = (int64_t)st.slice_nodes;
        stats->slice_sweeps = g->push_slice ? slice_sweeps : 0;
        if (o.propagation == 7) {
            // the persistent loop times its own phases on the device (%globaltimer), in
            // either loop mode: selection phases and push phases of every pass
            stats->level_seconds = (double)(st.t_scan_ns + st.t_push_ns) * 1e-9;
            stats->select_seconds = (double)st.t_scan_ns * 1e-9;
            stats->level_launches = (int32_t)st.passes;
        }
    }
    return rc;
}

}  // namespace

extern "C" DI_API di_status di_solve(di_graph *g, const double *B, double d, double tol, double *H, double *F,
                                    const di_opts *opts, di_stats *stats) {
    NvtxRange range("di_solve");
    clear_error();
    return solve_impl(g, B, d, tol, H, F, opts, stats);
}

extern "C" DI_API di_status di_solve_host(di_graph *g, const double *B, double d, double tol, double *H, double *F,
                                         const di_opts *opts, di_stats *stats) {
    NvtxRange range("di_solve_host");
    clear_error();
    if (!g || !B || !H) { set_error("di_solve_host: NULL graph, B or H"); return DI_EINVAL; }
    di_opts o;
    if (opts) o = *opts; else di_opts_default(&o);
    cudaStream_t s = as_stream(o.stream);
    Workspace &ws = g->ws;
    const size_t bytes = (size_t)g->n * sizeof(double);
    if (!ws.hostB) DI_CUDA_TRY(dmalloc(&ws.hostB, g->n));
    if (!ws.hostH) DI_CUDA_TRY(dmalloc(&ws.hostH, g->n));
    if (F && !ws.hostF) DI_CUDA_TRY(dmalloc(&ws.hostF, g->n));
    DI_CUDA_TRY(cudaMemcpyAsync(ws.hostB, B, bytes, cudaMemcpyHostToDevice, s));
    if (o.warm_start) DI_CUDA_TRY(cudaMemcpyAsync(ws.hostH, H, bytes, cudaMemcpyHostToDevice, s));
    di_status rc = solve_impl(g, ws.hostB, d, tol, ws.hostH, F ? ws.hostF : nullptr, &o, stats);
    if (rc != DI_OK && rc != DI_ENOCONV) return rc;
    DI_CUDA_TRY(cudaMemcpyAsync(H, ws.hostH, bytes, cudaMemcpyDeviceToHost, s));
    if (F) DI_CUDA_TRY(cudaMemcpyAsync(F, ws.hostF, bytes, cudaMemcpyDeviceToHost, s));
    DI_CUDA_TRY(cudaStreamSynchronize(s));
    return rc;
}

extern "C" DI_API di_status di_frontier(di_graph *g, const void *F, int fluid_fp64, double T, int32_t *list,
                                       int64_t *count, double *r_l1, double *max_abs, void *stream) {
    clear_error();
    if (!g || !F || !list) { set_error("di_frontier: NULL argument"); return DI_EINVAL; }
    if (!(T >= 0.0) || !std::isfinite(T)) { set_error("di_frontier: T = %g must be finite and >= 0", T); return DI_EINVAL; }
    cudaStream_t s = as_stream(stream);
    DI_TRY(ensure_workspace(g));
    Workspace &ws = g->ws;
    DI_CUDA_TRY(cudaStreamSynchronize(s));
    std::memset(ws.desc_h, 0, sizeof(SolveDesc));
    ws.desc_h->F = const_cast<void *>(F);
    std::memset(ws.st_h, 0, sizeof(SolveState));
    ws.st_h->T = T;
    DI_CUDA_TRY(cudaMemcpyAsync(ws.desc, ws.desc_h, sizeof(SolveDesc), cudaMemcpyHostToDevice, s));
    DI_CUDA_TRY(cudaMemcpyAsync(ws.st, ws.st_h, sizeof(SolveState), cudaMemcpyHostToDevice, s));
    if (fluid_fp64)
        k_scan<double><<<g->grid_scan, kScanThreads, 0, s>>>(ws.desc, ws.st, list, g->n, ws.part_sum, ws.part_max);
    else
        k_scan<float><<<g->grid_scan, kScanThreads, 0, s>>>(ws.desc, ws.st, list, g->n, ws.part_sum, ws.part_max);
    DI_CUDA_TRY(cudaGetLastError());
    DI_CUDA_TRY(cudaMemcpyAsync(ws.st_h, ws.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    DI_CUDA_TRY(cudaStreamSynchronize(s));
    if (count) *count = ws.st_h->nfront;
    if (r_l1) *r_l1 = ws.st_h->r_scan;
    if (max_abs) *max_abs = ws.st_h->max_scan;
    return DI_OK;
}
