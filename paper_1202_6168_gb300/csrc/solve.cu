// solve.cu - the D-iteration level loop on one GPU.
//
// One threshold level (Sec. 2.4) is two kernels:
//   k_scan  - reads the fluid once: fused L1 residual sum |F_i| and max |F_i|,
//             and compaction of the frontier S = { i : |F_i| >= T } by warp
//             ballots and a block prefix (one atomic per 2048 nodes);
//   k_push  - for every i in S: f = atomicExch(F_i, 0), H_i += f (FP64),
//             and F_k += (d / outdeg_i) f for every out-edge i -> k
//             (Eqs. defF/defH), with red.global.add.  A row is pushed by one
//             thread (outdeg <= 16), one warp (<= 512) or the whole CTA.
//             Targets of very high in-degree are accumulated in shared
//             memory per CTA and flushed once, so the hottest addresses of
//             a power-law graph do not serialise the L2 atomics.
// The last block of k_scan decides the next step on the device: push, lower
// T to the largest fluid when the frontier is empty, confirm a stop request
// with an exact FP64 residual (residual.cu), or finish.  The levels run in a
// CUDA graph whose WHILE conditional node repeats [scan, push, IF(recompute)]
// until the scan reports completion: no host round trip per level.
#include <algorithm>
#include <cmath>

#include "di_internal.cuh"

namespace di {
namespace {

template <typename FT>
struct Acc;  // per-thread accumulation type of the scan's L1 sum
template <>
struct Acc<float> { using T = float; };
template <>
struct Acc<double> { using T = double; };

__device__ __forceinline__ float thr_cast(double T, float) { return __double2float_ru(T); }
__device__ __forceinline__ double thr_cast(double T, double) { return T; }

// ------------------------------------------------------------------ init (cold start)

template <typename FT>
__global__ void __launch_bounds__(kScanThreads) k_init(const SolveDesc *__restrict__ desc, SolveState *__restrict__ st,
                                                       int64_t n, double *__restrict__ part_sum,
                                                       double *__restrict__ part_max) {
    const double *__restrict__ B = desc->B;
    double *__restrict__ H = desc->H;
    FT *__restrict__ F = static_cast<FT *>(desc->F);
    double s = 0.0, m = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double b = B[i];
        const FT f = static_cast<FT>(b);
        F[i] = f;
        H[i] = 0.0;
        s += fabs(b);
        m = fmax(m, fabs(static_cast<double>(f)));
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
        st->r_exact = ts;
        st->T = tm;   // T_0 = max |F_0|
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

template <typename FT>
__global__ void __launch_bounds__(kScanThreads) k_scan(const SolveDesc *__restrict__ desc, SolveState *__restrict__ st,
                                                       int32_t *__restrict__ front, int64_t n,
                                                       double *__restrict__ part_sum, double *__restrict__ part_max,
                                                       cudaGraphConditionalHandle h_while,
                                                       cudaGraphConditionalHandle h_if, int ctl) {
    // ctl: 0 standalone frontier, 1 level loop in a CUDA graph, 2 host-driven level loop
    if (ctl && st->done) {
        if (ctl == 1 && blockIdx.x == 0 && threadIdx.x == 0) {
            cudaGraphSetConditional(h_if, 0);
            cudaGraphSetConditional(h_while, 0);
        }
        return;
    }
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
    if (!ctl) return;   // standalone frontier: the host reads nfront

    const int nf = st->nfront;
    st->nfront = 0;
    st->tile_ctr = 0;
    int push = 0, rec = 0;
    if (!isfinite(ts)) {
        st->done = 3;
    } else if (ts <= desc->tol && !st->force_push) {
        rec = 1;                  // stop request: confirm on the exact residual
        st->confirming = 1;
    } else if (st->level >= desc->max_levels) {
        st->done = 2;
    } else if (nf == 0) {
        double T = st->T;         // empty level: skip straight to the first T <= max |F|
        while (T > tm && T > 0.0) T /= desc->alpha;
        st->T = T;
    } else {
        push = nf;
        st->level += 1;
        st->force_push = 0;
        st->since_recompute += 1;
        st->T = st->T / desc->alpha;
        if (!desc->fluid_fp64 && desc->recompute_every > 0 && st->since_recompute >= desc->recompute_every) rec = 1;
    }
    st->body_iters += 1;
    if (!st->done && st->body_iters >= desc->max_body_iters) st->done = 2;
    if (st->done) { push = 0; rec = 0; }
    st->push_count = push;
    st->do_recompute = rec;
    if (ctl == 1) {
        cudaGraphSetConditional(h_if, rec ? 1u : 0u);
        if (st->done) cudaGraphSetConditional(h_while, 0);
    }
}

// ------------------------------------------------------------------ push

template <typename FT>
__global__ void __launch_bounds__(kPushThreads) k_push(const SolveDesc *__restrict__ desc, SolveState *__restrict__ st,
                                                       const int32_t *__restrict__ front,
                                                       const int32_t *__restrict__ rp,
                                                       const int32_t *__restrict__ pcol,
                                                       const int32_t *__restrict__ hot_node, int n_hot,
                                                       const FT *__restrict__ scale) {
    const int count = st->push_count;
    if (count == 0) return;
    extern __shared__ unsigned char smem_raw[];
    FT *s_hot = reinterpret_cast<FT *>(smem_raw);
    __shared__ unsigned s_tile;
    __shared__ int s_qn;
    __shared__ int32_t s_qb[kPushThreads], s_qe[kPushThreads];
    __shared__ FT s_qw[kPushThreads];

    FT *__restrict__ F = static_cast<FT *>(desc->F);
    double *__restrict__ H = desc->H;
    const int lane = threadIdx.x & 31;
    for (int sl = threadIdx.x; sl < n_hot; sl += kPushThreads) s_hot[sl] = FT(0);

    auto push1 = [&](int32_t c, FT w) {
        if (c >= 0) red_add(F + c, w);
        else atomicAdd(&s_hot[-1 - c], w);
    };

    unsigned long long my_edges = 0, my_nodes = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            s_tile = atomicAdd(&st->tile_ctr, 1u);
            s_qn = 0;
        }
        __syncthreads();
        const int64_t first = (int64_t)s_tile * kPushThreads;
        if (first >= count) break;
        const int64_t idx = first + threadIdx.x;
        int32_t b = 0, e = 0;
        FT w = FT(0);
        if (idx < count) {
            const int32_t i = front[idx];
            b = rp[i];
            e = rp[i + 1];
            const FT f = atomic_exch_fluid(F + i, FT(0));
            H[i] += static_cast<double>(f);   // i appears once per frontier
            w = f * scale[i];
            my_nodes += 1;
            my_edges += static_cast<unsigned long long>(e - b);
        }
        const int deg = e - b;
        if (deg <= kThreadMaxDeg) {
            for (int32_t q = b; q < e; ++q) push1(pcol[q], w);
        }
        unsigned wm = __ballot_sync(0xffffffffu, deg > kThreadMaxDeg && deg <= kWarpMaxDeg);
        while (wm) {
            const int src = __ffs(wm) - 1;
            wm &= wm - 1;
            const int32_t mb = __shfl_sync(0xffffffffu, b, src), me = __shfl_sync(0xffffffffu, e, src);
            const FT mw = __shfl_sync(0xffffffffu, w, src);
            for (int32_t q = mb + lane; q < me; q += 32) push1(pcol[q], mw);
        }
        if (deg > kWarpMaxDeg) {
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
            for (int32_t q = hb + threadIdx.x; q < he; q += kPushThreads) push1(pcol[q], hw);
        }
        __syncthreads();
    }
    __syncthreads();
    for (int sl = threadIdx.x; sl < n_hot; sl += kPushThreads) {
        const FT v = s_hot[sl];
        if (v != FT(0)) red_add(F + hot_node[sl], v);
    }
    my_edges = warp_sum(my_edges);
    my_nodes = warp_sum(my_nodes);
    if (lane == 0 && my_nodes) {
        atomicAdd(&st->node_diff, my_nodes);
        atomicAdd(&st->edge_diff, my_edges);
    }
}

// ------------------------------------------------------------------ host side

template <typename FT>
void launch_scan(di_graph *g, cudaStream_t s, cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hi, int ctl) {
    Workspace &ws = g->ws;
    k_scan<FT><<<g->grid_scan, kScanThreads, 0, s>>>(ws.desc, ws.st, ws.front, g->n, ws.part_sum, ws.part_max, hw,
                                                     hi, ctl);
}

template <typename FT>
void launch_push(di_graph *g, cudaStream_t s) {
    Workspace &ws = g->ws;
    const FT *scale = sizeof(FT) == 4 ? reinterpret_cast<const FT *>(g->s32) : reinterpret_cast<const FT *>(g->s64);
    k_push<FT><<<g->grid_push, kPushThreads, g->n_hot * sizeof(FT), s>>>(ws.desc, ws.st, ws.front, g->rp, g->pcol,
                                                                         g->hot_node, g->n_hot, scale);
}

di_status build_level_graph(di_graph *g, int fp64, int l2_window) {
    SolverGraph &sg = g->sg[fp64];
    if (sg.built) return DI_OK;
    cudaStream_t cs = nullptr;
    DI_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } sgd{cs};
    if (l2_window) {
        // keep the fluid vector resident in L2 while the column indices stream past it
        int max_persist = 0, max_window = 0;
        cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, g->device);
        cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, g->device);
        const size_t bytes = (size_t)g->n * (fp64 ? sizeof(double) : sizeof(float));
        if (max_persist > 0 && max_window > 0) {
            size_t limit = std::min<size_t>((size_t)max_persist, bytes);
            cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, limit);
            cudaStreamAttrValue v = {};
            v.accessPolicyWindow.base_ptr = fp64 ? (void *)g->ws.F64 : (void *)g->ws.F32;
            v.accessPolicyWindow.num_bytes = std::min<size_t>(bytes, (size_t)max_window);
            v.accessPolicyWindow.hitRatio =
                (float)std::min(1.0, (double)limit / (double)v.accessPolicyWindow.num_bytes);
            v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
            v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
            cudaStreamSetAttribute(cs, cudaStreamAttributeAccessPolicyWindow, &v);
            cudaGetLastError();   // the window is an optimisation; ignore refusal
        }
    }
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
    DI_CUDA_TRY(cudaGraphConditionalHandleCreate(&sg.h_if, body, 0, 0));

    DI_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    if (fp64) {
        launch_scan<double>(g, cs, sg.h_while, sg.h_if, 1);
        launch_push<double>(g, cs);
    } else {
        launch_scan<float>(g, cs, sg.h_while, sg.h_if, 1);
        launch_push<float>(g, cs);
    }
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    cudaGraph_t capg = nullptr;
    DI_CUDA_TRY(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &capg, &deps, nullptr, &ndeps));
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = sg.h_if;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t inode;
    DI_CUDA_TRY(cudaGraphAddNode(&inode, capg, deps, nullptr, ndeps, &ip));
    DI_CUDA_TRY(cudaStreamUpdateCaptureDependencies(cs, &inode, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t ended = nullptr;
    DI_CUDA_TRY(cudaStreamEndCapture(cs, &ended));

    cudaGraph_t ifbody = ip.conditional.phGraph_out[0];
    DI_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, ifbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    launch_residual(g, fp64, RES_LEVEL, cs);
    DI_CUDA_TRY(cudaStreamEndCapture(cs, &ended));

    DI_CUDA_TRY(cudaGraphInstantiate(&sg.exec, sg.graph, 0));
    sg.built = true;
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
    return DI_OK;
}

}  // namespace

di_status ensure_workspace(di_graph *g) {
    Workspace &ws = g->ws;
    if (ws.ready) return DI_OK;
    const int64_t n = g->n;
    g->grid_scan = std::max(1, std::min<int>(occupancy_grid((const void *)k_scan<float>, kScanThreads, 0, g->num_sms),
                                             (int)((n + kScanChunk - 1) / kScanChunk)));
    g->grid_push = occupancy_grid((const void *)k_push<double>, kPushThreads, kMaxHot * sizeof(double), g->num_sms);
    g->grid_res = residual_grid(g->num_sms);
    const int parts = std::max({g->grid_scan, g->grid_push, g->grid_res});
    DI_CUDA_TRY(dmalloc(&ws.front, n));
    DI_CUDA_TRY(dmalloc(&ws.g, n));
    DI_CUDA_TRY(dmalloc(&ws.seg_part, std::max(g->n_seg, 1)));
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
    if (fp64 && !ws.F64) DI_CUDA_TRY(dmalloc(&ws.F64, g->n));
    if (!fp64 && !ws.F32) DI_CUDA_TRY(dmalloc(&ws.F32, g->n));
    DI_TRY(ensure_scale(g, d, s));
    if (!o.timing) DI_TRY(build_level_graph(g, fp64, o.l2_window));

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
    dh.fluid_fp64 = fp64;
    dh.max_body_iters = (int)std::min<long long>(4LL * o.max_levels + 1000, INT32_MAX);
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

    double t_scan = 0.0, t_push = 0.0, t_rec = 0.0;
    int live_iters = 0;
    if (!o.timing) {
        DI_CUDA_TRY(cudaGraphLaunch(g->sg[fp64].exec, s));
        DI_CUDA_TRY(cudaMemcpyAsync(ws.st_h, ws.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        DI_CUDA_TRY(cudaStreamSynchronize(s));
    } else {
        // host-driven levels, a CUDA event between every two kernels
        constexpr int kBatch = 16;
        for (cudaEvent_t &e : ws.tev)
            if (!e) DI_CUDA_TRY(cudaEventCreate(&e));
        for (;;) {
            for (int l = 0; l < kBatch; ++l) {
                cudaEvent_t *e = ws.tev + 4 * l;
                DI_CUDA_TRY(cudaEventRecord(e[0], s));
                if (fp64) launch_scan<double>(g, s, 0, 0, 2); else launch_scan<float>(g, s, 0, 0, 2);
                DI_CUDA_TRY(cudaEventRecord(e[1], s));
                if (fp64) launch_push<double>(g, s); else launch_push<float>(g, s);
                DI_CUDA_TRY(cudaEventRecord(e[2], s));
                launch_residual(g, fp64, RES_LEVEL, s);
                DI_CUDA_TRY(cudaEventRecord(e[3], s));
            }
            DI_CUDA_TRY(cudaGetLastError());
            DI_CUDA_TRY(cudaMemcpyAsync(ws.st_h, ws.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
            DI_CUDA_TRY(cudaStreamSynchronize(s));
            const int live = std::min(kBatch, ws.st_h->body_iters - live_iters);
            for (int l = 0; l < live; ++l) {
                float a = 0.f, b = 0.f, c = 0.f;
                cudaEvent_t *e = ws.tev + 4 * l;
                DI_CUDA_TRY(cudaEventElapsedTime(&a, e[0], e[1]));
                DI_CUDA_TRY(cudaEventElapsedTime(&b, e[1], e[2]));
                DI_CUDA_TRY(cudaEventElapsedTime(&c, e[2], e[3]));
                t_scan += a * 1e-3;
                t_push += b * 1e-3;
                t_rec += c * 1e-3;
            }
            live_iters = ws.st_h->body_iters;
            if (ws.st_h->done) break;
        }
    }
    SolveState st = *ws.st_h;
    if (st.done != 1) {
        // level cap or non-finite residual: refresh F_out and the exact residual
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
    if (st.done == 3 || !std::isfinite(st.r_exact)) {
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
        long long launches = o.warm_start ? 1 + rk + (warm_used ? 0 : 1) : 1;
        launches += 2LL * st.body_iters + (long long)rk * st.recomputes;
        if (!o.timing && st.done == 1) launches += 1;   // the iteration that exits the loop
        if (st.done != 1) launches += rk;               // final residual refresh
        if (o.timing) launches = (o.warm_start ? 1 + rk + (warm_used ? 0 : 1) : 1) +
                                 (long long)(2 + rk) * st.body_iters + (st.done != 1 ? rk : 0);
        stats->gpu_launches = launches;
        stats->scan_seconds = t_scan;
        stats->push_seconds = t_push;
        stats->recompute_seconds = t_rec;
        stats->scan_launches = o.timing ? live_iters : 0;
        stats->push_launches = o.timing ? live_iters : 0;
        stats->recompute_launches = st.recomputes;
        stats->body_iterations = st.body_iters;
    }
    return rc;
}

}  // namespace

extern "C" DI_API di_status di_solve(di_graph *g, const double *B, double d, double tol, double *H, double *F,
                                    const di_opts *opts, di_stats *stats) {
    clear_error();
    return solve_impl(g, B, d, tol, H, F, opts, stats);
}

extern "C" DI_API di_status di_solve_host(di_graph *g, const double *B, double d, double tol, double *H, double *F,
                                         const di_opts *opts, di_stats *stats) {
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
        k_scan<double><<<g->grid_scan, kScanThreads, 0, s>>>(ws.desc, ws.st, list, g->n, ws.part_sum, ws.part_max, 0, 0, 0);
    else
        k_scan<float><<<g->grid_scan, kScanThreads, 0, s>>>(ws.desc, ws.st, list, g->n, ws.part_sum, ws.part_max, 0, 0, 0);
    DI_CUDA_TRY(cudaGetLastError());
    DI_CUDA_TRY(cudaMemcpyAsync(ws.st_h, ws.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    DI_CUDA_TRY(cudaStreamSynchronize(s));
    if (count) *count = ws.st_h->nfront;
    if (r_l1) *r_l1 = ws.st_h->r_scan;
    if (max_abs) *max_abs = ws.st_h->max_scan;
    return DI_OK;
}
