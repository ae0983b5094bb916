// batch.cu - many D-iteration solves (graphs x right-hand sides) in one level loop.
//
// A batch is a list of work items: right-hand side r of graph g.  Every item
// is an independent instance of X = P X + B (Eq. 1) with its own threshold
// schedule (Sec. 2.4: diffuse every node with |F_i| >= T_item, then
// T_item <- T_item / alpha) and its own stop rule |B + P H - H|_1 <= tol_item.
//
// GB300 layout: the items are laid side by side in one "union" graph, the
// disjoint union of one copy of graph g per right-hand side, every copy
// starting on a multiple of kBChunk nodes (the padding nodes are isolated and
// carry no fluid).  A scan chunk of kBChunk nodes therefore belongs to exactly
// one item, so per-item sums, maxima and frontier counts are one atomic per
// chunk, and every level of every live item runs in the same launches, which
// spread the union's edges over all SMs whatever the mix of item sizes.
//   k_bscan_level - frontier of all live items (each against its own T),
//                   per-item L1 norm / max / selected nodes and edges; its
//                   last CTA runs the control step of every item;
//   k_bpush       - asynchronous push of the frontier nodes of the items
//                   whose level goes ahead (atomicExch drain, FP64 history,
//                   red.global.add scatter);
//   k_bres_*      - exact FP64 residual F = B + P H - H of the items that
//                   asked for one (FP32 refresh or stop confirmation):
//                   edge-parallel gather over the in-edges with runs of equal
//                   destination added by one red.global.add.f64.
// The loop runs in a CUDA graph (WHILE node; IF node around the residual)
// with every decision taken on the device.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <new>
#include <vector>

#include "di_internal.cuh"

namespace di {
namespace {

constexpr int kBThreads = 256;
constexpr int kBItems = 8;                        // nodes per thread per chunk
constexpr int kBChunk = kBThreads * kBItems;      // 2048: item alignment in the union
constexpr int kBChunkShift = 11;
static_assert((1 << kBChunkShift) == kBChunk, "chunk shift");
constexpr int kBFlatEdges = 16;

// Per-item state on the device.
struct BItem {
    double T;            // threshold of the next scan
    double tol;
    double est_scale;    // calibration of the scan's running estimate
    double r_confirm;
    double r_exact;      // last exact residual
    double b_l1;
    double acc_sum;      // scan accumulators (cleared by the control step)
    unsigned long long acc_max;   // bits of max |F| (non-negative doubles order like integers)
    unsigned long long acc_nsel, acc_esel;
    double res_sum;
    unsigned long long res_max;
    unsigned long long node_diff, edge_diff;
    int level, since, recomputes, done;   // done: 0 running, 1 converged, 2 level cap, 3 non-finite
    int push, rec, confirming, pad;
    double dang_acc;     // 1/N completion: fluid drained from the item's dangling nodes since its last selection
    double dang_h;       // exact residual: sum of H over the item's dangling nodes
    double T_push;       // selection threshold of the level being pushed (the slice sweeps' T)
    int sweep;           // this level: the item's frontier is dense enough for slice sweeps
    int pad3;
};

struct BState {
    int nfront;          // frontier entries written by the current scan
    int push_count;      // frontier entries the push walks
    int body_iters;
    int pad;
    unsigned int scan_blocks, res_blocks, init_blocks, tile_ctr;
    unsigned int tiles_done, pad2;   // frontier tiles whose pushes are done (slice sweeps wait for all)
};

struct BDesc {
    double d, alpha;
    double drop;         // exact recompute when an item's |F|_1 fell this much since its last one (0 = none)
    int R, fp64, max_levels, max_body_iters, nitems, final_mode;
    int thread_max, warp_max;  // push shape
    int dangling;              // 1: dangling columns completed by d / n_t (uniform over item t's nodes)
    int slice_sweeps;          // sweeps of each push CTA's slice of the union after the frontier (0 = none)
    unsigned long long wait_ns;   // bound of the push's wait for the frontier tiles before a slice sweep
    void *F;             // union fluid (float or double)
    double *B, *H;       // union B and history
    double *tmp, *g;     // exact-residual scratch
    const double *const *pB;   // per-item caller B (device pointers)
    double *const *pH;         // per-item caller H
};

__device__ __forceinline__ float bthr(double T, float) { return __double2float_ru(T); }
__device__ __forceinline__ double bthr(double T, double) { return T; }

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *p, double v) {
    atomicMax(p, static_cast<unsigned long long>(__double_as_longlong(v)));
}
__device__ __forceinline__ double nonneg_from_bits(unsigned long long b) {
    return __longlong_as_double(static_cast<long long>(b));
}

// Block-wide sum (double), max (double) and sum (u64); results in thread 0.
__device__ __forceinline__ void block_reduce3(double &s, double &m, unsigned long long &c) {
    __shared__ double ss[kBThreads / 32], sm[kBThreads / 32];
    __shared__ unsigned long long sc[kBThreads / 32];
    s = warp_sum(s);
    m = warp_max(m);
    c = warp_sum(c);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { ss[w] = s; sm[w] = m; sc[w] = c; }
    __syncthreads();
    if (w == 0) {
        s = l < kBThreads / 32 ? ss[l] : 0.0;
        m = l < kBThreads / 32 ? sm[l] : 0.0;
        c = l < kBThreads / 32 ? sc[l] : 0ull;
        s = warp_sum(s);
        m = warp_max(m);
        c = warp_sum(c);
    }
    __syncthreads();
}

// ------------------------------------------------------------------ start

// Copies every item's B into the union (F = B, H = 0; zero on padding) and
// accumulates |B|_1 and max |F| per item; the last CTA sets T_0 = max |F_0|.
template <typename FT>
__global__ void __launch_bounds__(kBThreads) k_bstart(const BDesc *__restrict__ desc, BItem *__restrict__ items,
                                                      BState *__restrict__ st,
                                                      const int32_t *__restrict__ item_of_chunk,
                                                      const int64_t *__restrict__ base,
                                                      const int32_t *__restrict__ nloc, int64_t nchunks) {
    FT *__restrict__ F = static_cast<FT *>(desc->F);
    double *__restrict__ Bu = desc->B;
    double *__restrict__ Hu = desc->H;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int t = item_of_chunk[c];
        const double *__restrict__ Bt = desc->pB[t];
        const int64_t b0 = base[t];
        const int64_t nl = nloc[t];
        double s = 0.0, m = 0.0;
        unsigned long long z = 0;
#pragma unroll
        for (int k = 0; k < kBItems; ++k) {
            const int64_t i = (c << kBChunkShift) + k * kBThreads + threadIdx.x;
            const int64_t loc = i - b0;
            const double b = loc < nl ? Bt[loc] : 0.0;
            const FT f = static_cast<FT>(b);
            Bu[i] = b;
            F[i] = f;
            Hu[i] = 0.0;
            s += fabs(b);
            m = fmax(m, fabs(static_cast<double>(f)));
        }
        block_reduce3(s, m, z);
        if (threadIdx.x == 0) {
            atomicAdd(&items[t].acc_sum, s);
            atomic_max_nonneg(&items[t].acc_max, m);
        }
    }
    if (!last_block(&st->init_blocks)) return;
    for (int t = threadIdx.x; t < desc->nitems; t += blockDim.x) {
        BItem &it = items[t];
        const double b1 = it.acc_sum;
        it.b_l1 = b1;
        it.r_exact = b1;    // F_0 = B: the exact residual of H_0 = 0
        it.T = nonneg_from_bits(it.acc_max);
        it.acc_sum = 0.0;
        it.acc_max = 0ull;
        if (!isfinite(b1)) it.done = 3;
        else if (b1 <= it.tol) it.done = 1;
    }
}

// ------------------------------------------------------------------ one level

template <typename FT>
__global__ void __launch_bounds__(kBThreads) k_bscan_level(
    const BDesc *__restrict__ desc, BItem *__restrict__ items, BState *__restrict__ st,
    const int32_t *__restrict__ item_of_chunk, const int32_t *__restrict__ outdeg, int32_t *__restrict__ front,
    int64_t nchunks, const int64_t *__restrict__ base, const int32_t *__restrict__ nloc,
    cudaGraphConditionalHandle h_while, cudaGraphConditionalHandle h_rec, int ctl) {
    FT *__restrict__ F = static_cast<FT *>(desc->F);
    const int dangling = desc->dangling;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // one warp per 2048-node chunk, no block barrier: lane l reads nodes
    // c0 + 128 j + 4 l + v (j = 0..15, v = 0..3) with vector loads, and
    // the selected ids go to the frontier in node order (a warp scan per j)
    // after one atomic per chunk reserves the chunk's slice
    constexpr int kJ = kBChunk / 128;
    const int64_t nwarps = (int64_t)gridDim.x * (kBThreads / 32);
    for (int64_t c = (int64_t)blockIdx.x * (kBThreads / 32) + warp; c < nchunks; c += nwarps) {
        const int t = item_of_chunk[c];
        if (items[t].done) continue;                 // uniform over the warp
        const FT Tc = bthr(items[t].T, FT(0));
        const int64_t c0 = c << kBChunkShift;
        // 1/N completion (Sec. 2.2): the fluid the item's dangling nodes drained
        // since its last selection reaches each of its n_t nodes as d / n_t of it
        // (not the padding after its last node); added and stored before the test
        const int64_t b0 = base[t], nl = nloc[t];
        const FT u = dangling ? static_cast<FT>(desc->d * items[t].dang_acc / (double)nl) : FT(0);
        unsigned long long msk = 0;                  // 4 bits per j
        FT part = FT(0), mx = FT(0);
        unsigned long long esel = 0;
#pragma unroll
        for (int jj = 0; jj < kJ; ++jj) {
            const int64_t i0 = c0 + 128 * jj + 4 * lane;
            FT v[4];
            if (sizeof(FT) == 4) {
                const float4 q = *reinterpret_cast<const float4 *>(F + i0);
                v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
            } else {
                const double2 q0 = reinterpret_cast<const double2 *>(F + i0)[0];
                const double2 q1 = reinterpret_cast<const double2 *>(F + i0)[1];
                v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
            }
            if (u != FT(0)) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (i0 + k - b0 < nl) {
                        v[k] += u;
                        F[i0 + k] = v[k];
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const FT a = fabs(v[k]);
                part += a;
                mx = a > mx ? a : mx;
                if (a >= Tc && a > FT(0)) msk |= 1ull << (4 * jj + k);
            }
        }
        const int mine = __popcll(msk);
        const int total = warp_sum(mine);
        int fbase = 0;
        if (total) {
            if (lane == 0) fbase = atomicAdd(&st->nfront, total);
            fbase = __shfl_sync(0xffffffffu, fbase, 0);
            // node order: j-blocks in turn, lanes in turn inside a block
            int run = fbase;
#pragma unroll
            for (int jj = 0; jj < kJ; ++jj) {
                const unsigned m4 = (unsigned)(msk >> (4 * jj)) & 15u;
                const int cnt = __popc(m4);
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int q = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += q;
                }
                int pos = run + incl - cnt;
                const int64_t i0 = c0 + 128 * jj + 4 * lane;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if ((m4 >> k) & 1u) {
                        front[pos++] = static_cast<int32_t>(i0 + k);
                        esel += static_cast<unsigned long long>(outdeg[i0 + k]);
                    }
                run += __shfl_sync(0xffffffffu, incl, 31);
            }
        }
        // the chunk's sums (in the fluid's precision within the warp, FP64 across chunks)
        double acc = static_cast<double>(warp_sum(part));
        const double wmx = static_cast<double>(warp_max(mx));
        esel = warp_sum(esel);
        if (lane == 0) {
            BItem &it = items[t];
            atomicAdd(&it.acc_sum, acc);
            atomic_max_nonneg(&it.acc_max, wmx);
            if (total) {
                atomicAdd(&it.acc_nsel, static_cast<unsigned long long>(total));
                atomicAdd(&it.acc_esel, esel);
            }
        }
    }
    __shared__ unsigned int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(&st->scan_blocks, 1u);
        s_last = prev == gridDim.x - 1;
        if (s_last) st->scan_blocks = 0;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // control step of every item (one thread per item)
    const double alpha = desc->alpha;
    const int R = desc->R, fp64 = desc->fp64, max_levels = desc->max_levels;
    const double drop = desc->drop;
    int any_rec = 0, live = 0;
    for (int t = threadIdx.x; t < desc->nitems; t += blockDim.x) {
        BItem &it = items[t];
        int push = 0, rec = 0;
        if (!it.done) {
            const double ts = it.acc_sum, tm = nonneg_from_bits(it.acc_max);
            const unsigned long long nsel = it.acc_nsel, esel = it.acc_esel;
            const double est = it.est_scale > 1.0 ? it.est_scale : 1.0;
            double T = it.T;
            if (it.level >= max_levels) {
                it.done = 2;
            } else if (!isfinite(ts)) {
                it.done = 3;
            } else if (ts * est <= it.tol) {
                rec = 1;                       // stop request: confirm on the exact residual, no push
                it.confirming = 1;
                it.r_confirm = ts * est;
            } else if (nsel == 0) {
                if (tm > 0.0) {                  // empty level: first T / alpha^k <= max |F|
                    for (int guard = 0; T > tm && guard < 8192; ++guard) T /= alpha;
                    if (T > tm) T = tm;   // alpha so close to 1 that the guard ran out
                }
            } else {
                push = 1;
                it.level += 1;
                it.since += 1;
                it.node_diff += nsel;        // the frontier; the push adds its slice sweeps' drains
                it.edge_diff += esel;
                it.T_push = T;
                it.sweep = desc->slice_sweeps > 0 && nsel * kSliceDensity >= (unsigned long long)nloc[t];
                T /= alpha;
                // refinement: every R levels, or once |F|_1 fell by drop since the last exact value
                if (!fp64 && ((R > 0 && it.since >= R) || (drop > 0.0 && ts * est * drop <= it.r_exact))) rec = 1;
            }
            it.T = T;
        }
        it.acc_sum = 0.0;
        it.acc_max = 0ull;
        it.acc_nsel = 0ull;
        it.acc_esel = 0ull;
        it.dang_acc = 0.0;                  // applied by every chunk of this selection
        if (!push) it.sweep = 0;
        it.push = push;
        it.rec = rec;
        any_rec |= rec;
        live += (it.done == 0);
    }
    any_rec = __syncthreads_or(any_rec);
    live = __syncthreads_count(live > 0);
    if (threadIdx.x != 0) return;
    const int iters = st->body_iters + 1;
    st->body_iters = iters;
    st->push_count = st->nfront;
    st->nfront = 0;
    st->tile_ctr = 0;
    st->tiles_done = 0;
    const bool stop = live == 0 || iters >= desc->max_body_iters;
    if (ctl == 1) {
        cudaGraphSetConditional(h_rec, any_rec ? 1u : 0u);
        if (stop) cudaGraphSetConditional(h_while, 0);
    }
}

// Push of the frontier nodes whose item goes ahead this level: f =
// atomicExch(F_i, 0), H_i += f (FP64; a node is in the frontier once),
// F_k += (d / outdeg_i) f over the out-edges with red.global.add.  Dynamic
// tiles of kBThreads frontier entries; a row is pushed by its thread (<= 16
// edges), by a warp (<= 512) or by the whole CTA; very hot targets are
// accumulated in shared memory per CTA.
// kSlice (slice sweeps, as in the single-graph push): once the frontier's
// tiles are all claimed and their pushes done (a counter advanced after a
// fence; a bounded wait), each CTA sweeps its own slice of the union up to
// desc->slice_sweeps times and diffuses every node with |F_i| >= its item's
// selection threshold - the fluid that crossed it while the level pushed -
// over the chunks of the items whose frontier was dense (at least
// 1/kSliceDensity of their nodes; the others' chunks are skipped).  A node
// may then be drained twice in a level, so H_i is updated with an FP64
// atomic add.  The control counts the frontier's diffusions at its
// selection; the push counts those of its sweeps, per thread over runs of
// the same item (a slice is consecutive nodes) and summed over the warp
// before the items' counters.  A sweep starts when half the frontier's
// tiles are done, so a frontier node it drains before its own tile is
// counted twice: with sweeps the items' counts can overstate the work a
// little.
constexpr int kBSliceCap = 1536;   // slice-sweep queue entries per CTA (>= 1024 + kBThreads)

template <typename FT>
__device__ __forceinline__ void ld4_cg(const FT *p, FT v[4]);
template <>
__device__ __forceinline__ void ld4_cg<float>(const float *p, float v[4]) {
    const float4 t = __ldcg(reinterpret_cast<const float4 *>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
template <>
__device__ __forceinline__ void ld4_cg<double>(const double *p, double v[4]) {
    const double2 a = __ldcg(reinterpret_cast<const double2 *>(p)), c = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = c.x; v[3] = c.y;
}

template <typename FT, bool kSlice>
__global__ void __launch_bounds__(kBThreads) k_bpush(const BDesc *__restrict__ desc, BItem *__restrict__ items,
                                                     BState *__restrict__ st, const int32_t *__restrict__ item_of_chunk,
                                                     const int32_t *__restrict__ front, const int32_t *__restrict__ rp,
                                                     const int32_t *__restrict__ pcol,
                                                     const int32_t *__restrict__ hot_node, int n_hot,
                                                     const FT *__restrict__ scale, int64_t n_union) {
    const int count = st->push_count;
    if (count == 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FT *s_hot = reinterpret_cast<FT *>(smem_raw);
    int32_t *s_sq = reinterpret_cast<int32_t *>(s_hot + ((n_hot + 3) & ~3));   // kSlice: the queue
    __shared__ unsigned s_tile;
    __shared__ int s_qn, s_src, s_sqn, s_sbase, s_sbt, s_sweep, s_waited, s_gdone;
    __shared__ long long s_pos, s_seg;
    __shared__ int32_t s_qb[kBThreads], s_qe[kBThreads];
    __shared__ FT s_qw[kBThreads];
    FT *__restrict__ F = static_cast<FT *>(desc->F);
    double *__restrict__ H = desc->H;
    const int lane = threadIdx.x & 31;
    // the CTA's slice of the union, a multiple of 4 nodes long
    const int64_t per = kSlice ? ((n_union + gridDim.x - 1) / gridDim.x + 3) / 4 * 4 : 0;
    const int64_t s_lo = kSlice ? min(n_union, (int64_t)blockIdx.x * per) : 0;
    const int64_t s_hi = kSlice ? min(n_union, s_lo + per) : 0;
    const int sweeps = kSlice ? desc->slice_sweeps : 0;
    for (int sl = threadIdx.x; sl < n_hot; sl += kBThreads) s_hot[sl] = FT(0);
    if (threadIdx.x == 0) {   // ordered before any use by the loop's first barrier
        s_sqn = 0;
        s_sweep = 0;
        s_waited = 0;
        s_gdone = 0;
        s_pos = s_lo;
    }
    const uint64_t keep = l2_keep_policy();
    const int thread_max = desc->thread_max, warp_max = desc->warp_max;
    auto push1 = [&](int32_t c, FT w) {
        if (c >= 0) red_add_keep(F + c, w, keep);
        else atomicAdd(&s_hot[-1 - c], w);
    };
    // kSlice: the diffusions of the thread's current item, added per run
    int cnt_t = -1;
    unsigned long long cnt_nodes = 0, cnt_edges = 0;
    auto flush_counts = [&]() {
        if (cnt_t >= 0 && cnt_nodes) {
            atomicAdd(&items[cnt_t].node_diff, cnt_nodes);
            atomicAdd(&items[cnt_t].edge_diff, cnt_edges);
        }
        cnt_t = -1;
        cnt_nodes = cnt_edges = 0;
    };
    for (;;) {
        if (threadIdx.x == 0) {
            s_qn = 0;
            int src = 2;
            const int qn = kSlice ? min(s_sqn, kBSliceCap) : 0;
            if (kSlice && qn >= kBThreads) {
                src = 1;
            } else if (!s_gdone) {
                s_tile = atomicAdd(&st->tile_ctr, 1u);
                if ((int64_t)s_tile * kBThreads < count) src = 0;
                else s_gdone = 1;
            }
            if (kSlice && src == 2 && s_gdone) {
                if (!s_waited && sweeps > 0) {
                    // the frontier's pushes first (bounded by the timer and a poll count)
                    const unsigned ntiles = (unsigned)((count + kBThreads - 1) / kBThreads);
                    unsigned long long t0, now;
                    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
                    const unsigned long long limit = desc->wait_ns, max_polls = (limit >> 5) + 1024ull;
                    unsigned long long polls = 0;
                    for (;;) {
                        unsigned done_tiles;
                        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(done_tiles) : "l"(&st->tiles_done)
                                     : "memory");
                        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
                        if ((unsigned long long)done_tiles * 100ull >= (unsigned long long)ntiles * kSliceWaitPct ||
                            now - t0 > limit || ++polls > max_polls)
                            break;
                        __nanosleep(64);
                    }
                    s_waited = 1;
                }
                while (s_sweep < sweeps) {
                    // skip the chunks of items that do not sweep this level
                    while (s_pos < s_hi && !items[item_of_chunk[s_pos >> kBChunkShift]].sweep)
                        s_pos = ((s_pos >> kBChunkShift) + 1) << kBChunkShift;
                    if (s_pos < s_hi) {
                        src = 3;
                        s_seg = s_pos;
                        s_pos += 4 * kBThreads;
                        break;
                    }
                    if (qn > 0) {
                        src = 1;
                        break;
                    }
                    ++s_sweep;
                    s_pos = s_lo;
                }
            }
            if (src == 1) {
                const int bt = min(qn, kBThreads);
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
            // select |F_i| >= T_push of the node's item over 1024 nodes of the
            // slice (four consecutive nodes share a chunk, hence an item)
            const int64_t i0 = s_seg + 4 * (int64_t)threadIdx.x;
            unsigned msk = 0;
            if (i0 < s_hi) {
                const int t = item_of_chunk[i0 >> kBChunkShift];
                if (items[t].push && items[t].sweep) {
                    const FT Tc = bthr(items[t].T_push, FT(0));
                    FT v[4];
                    ld4_cg<FT>(F + i0, v);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const FT a = fabs(v[j]);
                        if (i0 + j < s_hi && a >= Tc && a > FT(0)) msk |= 1u << j;
                    }
                }
            }
            const int c = __popc(msk);
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int q = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += q;
            }
            int base = 0;
            if (lane == 31 && incl > 0) base = atomicAdd(&s_sqn, incl);
            int pos = __shfl_sync(0xffffffffu, base, 31) + incl - c;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if ((msk >> j) & 1u) {
                    if (pos < kBSliceCap) s_sq[pos] = static_cast<int32_t>(i0 + j);
                    ++pos;
                }
            __syncthreads();
            continue;
        }
        int32_t node = -1;
        if (src == 0) {
            const int64_t idx = (int64_t)s_tile * kBThreads + threadIdx.x;
            if (idx < count) node = __ldcs(front + idx);
        } else if (kSlice && (int)threadIdx.x < s_sbt) {
            node = s_sq[s_sbase + threadIdx.x];
        }
        int32_t b = 0, e = 0;
        FT w = FT(0);
        if (node >= 0) {
            const int32_t i = node;
            const int t = item_of_chunk[i >> kBChunkShift];
            if (items[t].push) {
                b = __ldcs(rp + i);
                e = __ldcs(rp + i + 1);
                const FT f = atomic_exch_keep(F + i, FT(0), keep);
                if (kSlice) {
                    if (f != FT(0)) {
                        atomicAdd(H + i, static_cast<double>(f));   // a node may be drained twice in a level
                        if (src == 1) {   // a sweep's node (the frontier's are counted at selection)
                            if (t != cnt_t) {
                                flush_counts();
                                cnt_t = t;
                            }
                            cnt_nodes += 1;
                            cnt_edges += static_cast<unsigned long long>(e - b);
                        }
                    } else {
                        e = b;   // drained already: nothing to send
                    }
                } else {
                    __stcs(H + i, __ldcs(H + i) + static_cast<double>(f));
                }
                w = f * __ldcs(scale + i);
                // 1/N completion: a selected node without out-edges is dangling (the
                // padding never holds fluid, so it is never selected)
                if (e == b && f != FT(0) && desc->dangling) atomicAdd(&items[t].dang_acc, static_cast<double>(f));
            }
        }
        const int deg = e - b;
        if (deg <= thread_max) {
            auto pw = [&](int32_t c) { push1(c, w); };
            push_range<8>(pcol, b, e, 1, pw);
        }
        const bool wrow = deg > thread_max && deg <= warp_max;
        if (__any_sync(0xffffffffu, wrow)) {
            // the warp's medium rows as one edge-parallel range (as in the
            // single-graph push): each lane finds the row of its edge by a
            // binary search over the lanes' offsets, 4 column loads in flight
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
                    int owner = 0;   // the last lane whose offset is <= q
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
            push_range<2>(pcol, (int64_t)hb + threadIdx.x, he, kBThreads, pw);
        }
        __syncthreads();
        if (kSlice && src == 0 && threadIdx.x == 0) {
            __threadfence();   // the tile's adds, ordered by the barrier, before the count
            atomicAdd(&st->tiles_done, 1u);
        }
    }
    if (kSlice) {
        // the last run of every thread: summed over the warp first when all
        // its lanes (those with a run) count for the same item, so that the
        // items' counters see one atomic per warp, not one per thread
        const int key = cnt_nodes ? cnt_t : -1;
        int k0 = key;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) k0 = max(k0, __shfl_xor_sync(0xffffffffu, k0, o));
        if (__all_sync(0xffffffffu, key == k0 || key < 0)) {
            cnt_nodes = warp_sum(cnt_nodes);
            cnt_edges = warp_sum(cnt_edges);
            cnt_t = lane == 0 ? k0 : -1;
        }
        flush_counts();
    }
    __syncthreads();
    for (int sl = threadIdx.x; sl < n_hot; sl += kBThreads) {
        const FT v = s_hot[sl];
        if (v != FT(0)) red_add_keep(F + hot_node[sl], v, keep);
    }
}

// ------------------------------------------------------------------ exact residual of the items that asked

// tmp = B - H and g = (d / outdeg) H on the chunks of items with rec set.
__global__ void __launch_bounds__(kBThreads) k_bres_prep(const BDesc *__restrict__ desc, BItem *__restrict__ items,
                                                         const int32_t *__restrict__ item_of_chunk,
                                                         const double *__restrict__ s64, const int32_t *__restrict__ rp,
                                                         const int64_t *__restrict__ base,
                                                         const int32_t *__restrict__ nloc, int64_t nchunks) {
    const double *__restrict__ B = desc->B;
    const double *__restrict__ H = desc->H;
    double *__restrict__ tmp = desc->tmp;
    double *__restrict__ g = desc->g;
    const int dangling = desc->dangling;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int t = item_of_chunk[c];
        if (!items[t].rec) continue;
        const int64_t b0 = base[t], nl = nloc[t];
        double hd = 0.0, unused = 0.0;
        unsigned long long z = 0;
#pragma unroll
        for (int k = 0; k < kBItems; ++k) {
            const int64_t i = (c << kBChunkShift) + k * kBThreads + threadIdx.x;
            const double h = H[i];
            tmp[i] = B[i] - h;
            g[i] = s64[i] * h;
            // 1/N completion: H over the item's dangling nodes (padding excluded)
            if (dangling && i - b0 < nl && rp[i + 1] == rp[i]) hd += h;
        }
        if (dangling) {
            block_reduce3(hd, unused, z);
            if (threadIdx.x == 0 && hd != 0.0) atomicAdd(&items[t].dang_h, hd);
        }
    }
}

// tmp_k += sum of g_j over the in-edges j -> k of the items with rec set:
// 16 consecutive in-edges per thread, runs of equal destination summed and
// added with one red.global.add.f64.  The in-edges of item t are the union
// in-CSR range [e_off[t], e_off[t + 1]) (items own disjoint node ranges, in
// order), so only the ranges of the items that recompute are read; chunks
// are aligned to the union's edge index (vector loads) and masked to the
// range.
__global__ void __launch_bounds__(kBThreads) k_bres_flat(const BDesc *__restrict__ desc,
                                                         const BItem *__restrict__ items, int nitems,
                                                         const int64_t *__restrict__ e_off,
                                                         const int32_t *__restrict__ in_col,
                                                         const int32_t *__restrict__ erow, int64_t nnz) {
    const double *__restrict__ g = desc->g;
    double *__restrict__ tmp = desc->tmp;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const int64_t wtid = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);   // the warp's first thread
    for (int t = 0; t < nitems; ++t) {
        if (!items[t].rec) continue;
        const int64_t eb = e_off[t], ee = e_off[t + 1];
        if (eb >= ee) continue;
        const int64_t cb = eb / kBFlatEdges, ce = (ee + kBFlatEdges - 1) / kBFlatEdges;
        // warp-uniform: lanes past ce hold no edge and still join warp_runs_add
        for (int64_t c0 = cb + wtid; c0 < ce; c0 += stride) {
            const int64_t c = c0 + lane;
            const int64_t e0 = c * kBFlatEdges;
            int32_t col[kBFlatEdges], row[kBFlatEdges];
            if (e0 + kBFlatEdges <= nnz) {
#pragma unroll
                for (int v = 0; v < kBFlatEdges / 4; ++v) {
                    const int4 a = __ldcs(reinterpret_cast<const int4 *>(in_col + e0) + v);
                    const int4 b = __ldcs(reinterpret_cast<const int4 *>(erow + e0) + v);
                    col[4 * v] = a.x; col[4 * v + 1] = a.y; col[4 * v + 2] = a.z; col[4 * v + 3] = a.w;
                    row[4 * v] = b.x; row[4 * v + 1] = b.y; row[4 * v + 2] = b.z; row[4 * v + 3] = b.w;
                }
            } else {
#pragma unroll
                for (int k = 0; k < kBFlatEdges; ++k) {
                    const bool ok = e0 + k < nnz;
                    col[k] = ok ? in_col[e0 + k] : 0;
                    row[k] = ok ? erow[e0 + k] : -1;
                }
            }
            double val[kBFlatEdges];
#pragma unroll
            for (int k = 0; k < kBFlatEdges; ++k) {
                const bool on = e0 + k >= eb && e0 + k < ee;
                if (!on) row[k] = -1;
                val[k] = on ? g[col[k]] : 0.0;
            }
            warp_runs_add<kBFlatEdges>(row, val, tmp, lane);
        }
    }
}

// F = tmp on the chunks of items with rec set (the exact residual becomes the
// fluid), per-item L1 norm and max; the last CTA runs the control step of
// those items (stop, calibration, or in final mode only the report).
template <typename FT>
__global__ void __launch_bounds__(kBThreads) k_bres_fin(const BDesc *__restrict__ desc, BItem *__restrict__ items,
                                                        BState *__restrict__ st,
                                                        const int32_t *__restrict__ item_of_chunk,
                                                        const int64_t *__restrict__ base,
                                                        const int32_t *__restrict__ nloc, int64_t nchunks) {
    FT *__restrict__ F = static_cast<FT *>(desc->F);
    const double *__restrict__ tmp = desc->tmp;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int t = item_of_chunk[c];
        if (!items[t].rec) continue;
        const int64_t b0 = base[t], nl = nloc[t];
        // 1/N completion: every node of the item gets (d / n_t) sum_dangling H_j
        const double du = desc->dangling ? desc->d * items[t].dang_h / (double)nl : 0.0;
        double s = 0.0, m = 0.0;
        unsigned long long z = 0;
#pragma unroll
        for (int k = 0; k < kBItems; ++k) {
            const int64_t i = (c << kBChunkShift) + k * kBThreads + threadIdx.x;
            const double f = i - b0 < nl ? tmp[i] + du : tmp[i];
            F[i] = static_cast<FT>(f);
            s += fabs(f);
            m = fmax(m, fabs(f));
        }
        block_reduce3(s, m, z);
        if (threadIdx.x == 0) {
            atomicAdd(&items[t].res_sum, s);
            atomic_max_nonneg(&items[t].res_max, m);
        }
    }
    if (!last_block(&st->res_blocks)) return;
    const bool final_mode = desc->final_mode != 0;
    for (int t = threadIdx.x; t < desc->nitems; t += blockDim.x) {
        BItem &it = items[t];
        if (!it.rec) continue;
        const double s = it.res_sum;
        it.r_exact = s;
        it.res_sum = 0.0;
        it.res_max = 0ull;
        it.rec = 0;
        it.dang_h = 0.0;
        it.dang_acc = 0.0;              // the exact fluid already holds what the dangling nodes drained
        if (final_mode) continue;
        it.recomputes += 1;
        it.since = 0;
        if (!isfinite(s)) {
            it.done = 3;
        } else if (s <= it.tol) {
            it.done = 1;
        } else if (it.confirming && it.r_confirm > 0.0) {
            it.est_scale = fmax(it.est_scale, 1.0) * fmax(s / it.r_confirm, 1.0);
        }
        it.confirming = 0;
    }
}

// H of every item back to the caller's buffers.
__global__ void __launch_bounds__(kBThreads) k_bfinish(const BDesc *__restrict__ desc,
                                                       const int32_t *__restrict__ item_of_chunk,
                                                       const int64_t *__restrict__ base,
                                                       const int32_t *__restrict__ nloc, int64_t nchunks) {
    const double *__restrict__ Hu = desc->H;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int t = item_of_chunk[c];
        double *__restrict__ Ht = desc->pH[t];
        const int64_t b0 = base[t], nl = nloc[t];
#pragma unroll
        for (int k = 0; k < kBItems; ++k) {
            const int64_t i = (c << kBChunkShift) + k * kBThreads + threadIdx.x;
            const int64_t loc = i - b0;
            if (loc < nl) Ht[loc] = Hu[i];
        }
    }
}

// Union construction: rows of item t = rows of its graph shifted by the
// item's first node and first edge; padding rows are empty.
__global__ void k_union_rows(const int32_t *__restrict__ rp, int64_t n, int64_t n_pad, int64_t node0, int64_t edge0,
                             int64_t *__restrict__ rp_u) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t last = rp[n];
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_pad; j += stride)
        rp_u[node0 + j] = edge0 + (j < n ? (int64_t)rp[j] : last);
}

// Targets of item t: the graph's targets (hot slots decoded) shifted by node0.
__global__ void k_union_cols(const int32_t *__restrict__ pcol, const int32_t *__restrict__ hot_node, int64_t nnz,
                             int64_t node0, int64_t edge0, int32_t *__restrict__ col_u) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        const int32_t c = pcol[e];
        const int32_t k = c >= 0 ? c : hot_node[-1 - c];
        col_u[edge0 + e] = static_cast<int32_t>(node0 + k);
    }
}

__global__ void k_set_i64(int64_t *p, int64_t v) { *p = v; }

}  // namespace
}  // namespace di

using namespace di;

struct di_batch {
    int device = 0;
    int ng = 0, nitems = 0;
    di_graph *u = nullptr;
    std::vector<int64_t> base, nloc;     // per item: first union node, nodes
    std::vector<int> graph_of;           // per item: index of its graph
    int64_t n_union = 0, nchunks = 0;
    int32_t *item_of_chunk = nullptr;
    int64_t *d_base = nullptr;
    int32_t *d_nloc = nullptr;
    int64_t *d_eoff = nullptr;           // per item: first union in-edge (nitems + 1 entries)
    double *B = nullptr, *H = nullptr, *tmp = nullptr, *g = nullptr;
    float *F32 = nullptr;
    double *F64 = nullptr;
    int32_t *front = nullptr;
    BItem *items = nullptr, *items_h = nullptr;
    BState *st = nullptr, *st_h = nullptr;
    BDesc *desc = nullptr, *desc_h = nullptr;
    const double **pB = nullptr;   // device tables [nitems]
    double **pH = nullptr;
    const double **pB_h = nullptr; // pinned mirrors
    double **pH_h = nullptr;
    int grid_scan = 0, grid_push = 0, grid_flat = 0;
    int grid_push_slice = 0;             // occupancy grid of the slice-sweep push
    int push_slice = 0;                  // the push of this call sweeps slices (opts.slice_sweeps)
    di_tune tune = {kThreadMaxDeg, kWarpMaxDeg, 0, 0};
    SolverGraph sg[2];
    int sg_l2[2] = {0, 0};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

void free_batch(di_batch *b) {
    if (!b) return;
    for (auto &sg : b->sg) {
        if (sg.exec) cudaGraphExecDestroy(sg.exec);
        if (sg.graph) cudaGraphDestroy(sg.graph);
    }
    void *dev[] = {b->item_of_chunk, b->d_base, b->d_nloc, b->d_eoff, b->B, b->H, b->tmp, b->g, b->F32, b->F64, b->front,
                   b->items, b->st, b->desc, (void *)b->pB, (void *)b->pH};
    for (void *q : dev)
        if (q) cudaFree(q);
    void *host[] = {b->items_h, b->st_h, b->desc_h, (void *)b->pB_h, (void *)b->pH_h};
    for (void *q : host)
        if (q) cudaFreeHost(q);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->u) di_graph_destroy(b->u);
    delete b;
}

int occ_grid(const void *fn, int threads, size_t smem, int sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return per_sm * sms;
}

int bpush_grid(const di_batch *b) {
    const int sms = b->u->num_sms;
    const int occ = b->push_slice ? b->grid_push_slice : b->grid_push;
    const int want = b->tune.push_ctas_per_sm > 0 ? b->tune.push_ctas_per_sm * sms : occ;
    return std::max(1, std::min(occ, want));
}

// Dynamic shared memory of the push: hot slots (padded to 4 words), then the
// slice-sweep queue.
template <typename FT>
size_t bpush_smem(int n_hot, bool slice) {
    return (size_t)((n_hot + 3) & ~3) * sizeof(FT) + (slice ? (size_t)kBSliceCap * sizeof(int32_t) : 0);
}

template <typename FT>
void launch_blevel(di_batch *b, cudaStream_t s, cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hr, int ctl) {
    di_graph *u = b->u;
    k_bscan_level<FT><<<b->grid_scan, kBThreads, 0, s>>>(b->desc, b->items, b->st, b->item_of_chunk, u->outdeg,
                                                          b->front, b->nchunks, b->d_base, b->d_nloc, hw, hr, ctl);
    const FT *scale = sizeof(FT) == 4 ? reinterpret_cast<const FT *>(u->s32) : reinterpret_cast<const FT *>(u->s64);
    if (b->push_slice)
        k_bpush<FT, true><<<bpush_grid(b), kBThreads, bpush_smem<FT>(u->n_hot, true), s>>>(
            b->desc, b->items, b->st, b->item_of_chunk, b->front, u->rp, u->pcol, u->hot_node, u->n_hot, scale,
            b->n_union);
    else
        k_bpush<FT, false><<<bpush_grid(b), kBThreads, bpush_smem<FT>(u->n_hot, false), s>>>(
            b->desc, b->items, b->st, b->item_of_chunk, b->front, u->rp, u->pcol, u->hot_node, u->n_hot, scale,
            b->n_union);
}

template <typename FT>
void launch_bres(di_batch *b, cudaStream_t s) {
    di_graph *u = b->u;
    k_bres_prep<<<b->grid_scan, kBThreads, 0, s>>>(b->desc, b->items, b->item_of_chunk, u->s64, u->rp, b->d_base,
                                                   b->d_nloc, b->nchunks);
    k_bres_flat<<<b->grid_flat, kBThreads, 0, s>>>(b->desc, b->items, b->nitems, b->d_eoff, u->in_col, u->erow,
                                                   u->nnz);
    k_bres_fin<FT><<<b->grid_scan, kBThreads, 0, s>>>(b->desc, b->items, b->st, b->item_of_chunk, b->d_base,
                                                      b->d_nloc, b->nchunks);
}

di_status build_batch_graph(di_batch *b, int fp64) {
    SolverGraph &sg = b->sg[fp64];
    if (sg.built && sg.grid_push == bpush_grid(b) && sg.slice == b->push_slice) return DI_OK;
    if (sg.built) {   // rebuilt for another push grid
        cudaGraphExecDestroy(sg.exec);
        cudaGraphDestroy(sg.graph);
        sg = SolverGraph();
    }
    cudaStream_t cs = nullptr;
    DI_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } guard{cs};
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
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    cudaGraph_t capg = nullptr, ended = nullptr;
    DI_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    if (fp64) launch_blevel<double>(b, cs, sg.h_while, sg.h_if, 1);
    else launch_blevel<float>(b, cs, sg.h_while, sg.h_if, 1);
    DI_CUDA_TRY(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &capg, &deps, nullptr, &ndeps));
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = sg.h_if;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t inode;
    DI_CUDA_TRY(cudaGraphAddNode(&inode, capg, deps, nullptr, ndeps, &ip));
    DI_CUDA_TRY(cudaStreamUpdateCaptureDependencies(cs, &inode, nullptr, 1, cudaStreamSetCaptureDependencies));
    DI_CUDA_TRY(cudaStreamEndCapture(cs, &ended));
    DI_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal));
    if (fp64) launch_bres<double>(b, cs); else launch_bres<float>(b, cs);
    DI_CUDA_TRY(cudaStreamEndCapture(cs, &ended));
    DI_CUDA_TRY(cudaGetLastError());
    DI_CUDA_TRY(cudaGraphInstantiate(&sg.exec, sg.graph, 0));
    sg.built = true;
    sg.grid_push = bpush_grid(b);
    sg.slice = b->push_slice;
    return DI_OK;
}

di_status batch_create_impl(const di_graph *const *graphs, int ng, const int *nrhs, cudaStream_t s, di_batch *b) {
    DI_CUDA_TRY(cudaGetDevice(&b->device));
    int64_t n_union = 0, nnz_union = 0;
    std::vector<int64_t> edge0;
    for (int gi = 0; gi < ng; ++gi) {
        const di_graph *g = graphs[gi];
        for (int r = 0; r < nrhs[gi]; ++r) {
            b->base.push_back(n_union);
            b->nloc.push_back(g->n);
            b->graph_of.push_back(gi);
            edge0.push_back(nnz_union);
            n_union += (g->n + kBChunk - 1) / kBChunk * kBChunk;
            nnz_union += g->nnz;
        }
    }
    b->nitems = (int)b->base.size();
    if (n_union > (int64_t)INT32_MAX || nnz_union > (int64_t)INT32_MAX) {
        set_error("di_batch_create: the batch holds %lld nodes (chunk-aligned) and %lld edges; both must be "
                  "< 2^31", (long long)n_union, (long long)nnz_union);
        return DI_EINVAL;
    }
    b->n_union = n_union;
    b->nchunks = n_union / kBChunk;
    // union CSR on the device, then the ordinary graph build (validation,
    // transpose, hot targets) on it
    int64_t *rp_u = nullptr;
    int32_t *col_u = nullptr;
    DI_CUDA_TRY(cudaMalloc(&rp_u, (n_union + 1) * sizeof(int64_t)));
    cudaError_t e = cudaMalloc(&col_u, std::max<int64_t>(nnz_union, 1) * sizeof(int32_t));
    if (e != cudaSuccess) {
        cudaFree(rp_u);
        set_error("di_batch_create: cudaMalloc of %lld edges failed: %s", (long long)nnz_union, cudaGetErrorString(e));
        return DI_ENOMEM;
    }
    struct Free2 {
        void *a, *b;
        ~Free2() { cudaFree(a); cudaFree(b); }
    } f2{rp_u, col_u};
    for (int t = 0; t < b->nitems; ++t) {
        const di_graph *g = graphs[b->graph_of[t]];
        const int64_t npad = (g->n + kBChunk - 1) / kBChunk * kBChunk;
        k_union_rows<<<(int)std::min<int64_t>((npad + 255) / 256, 4096), 256, 0, s>>>(g->rp, g->n, npad, b->base[t],
                                                                                       edge0[t], rp_u);
        if (g->nnz > 0)
            k_union_cols<<<(int)std::min<int64_t>((g->nnz + 255) / 256, 4096), 256, 0, s>>>(
                g->pcol, g->hot_node, g->nnz, b->base[t], edge0[t], col_u);
    }
    k_set_i64<<<1, 1, 0, s>>>(rp_u + n_union, nnz_union);
    DI_CUDA_TRY(cudaGetLastError());
    DI_CUDA_TRY(cudaStreamSynchronize(s));
    DI_TRY(di_graph_create(n_union, nnz_union, rp_u, col_u, 1, s, &b->u));

    std::vector<int32_t> ioc(b->nchunks);
    for (int t = 0; t < b->nitems; ++t) {
        const int64_t c0 = b->base[t] / kBChunk, c1 = (b->base[t] + (b->nloc[t] + kBChunk - 1) / kBChunk * kBChunk) / kBChunk;
        for (int64_t c = c0; c < c1; ++c) ioc[c] = t;
    }
    std::vector<int32_t> nl32(b->nitems);
    for (int t = 0; t < b->nitems; ++t) nl32[t] = (int32_t)b->nloc[t];
    DI_CUDA_TRY(cudaMalloc(&b->item_of_chunk, ioc.size() * sizeof(int32_t)));
    DI_CUDA_TRY(cudaMemcpy(b->item_of_chunk, ioc.data(), ioc.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    DI_CUDA_TRY(cudaMalloc(&b->d_base, b->nitems * sizeof(int64_t)));
    DI_CUDA_TRY(cudaMemcpy(b->d_base, b->base.data(), b->nitems * sizeof(int64_t), cudaMemcpyHostToDevice));
    DI_CUDA_TRY(cudaMalloc(&b->d_nloc, b->nitems * sizeof(int32_t)));
    DI_CUDA_TRY(cudaMemcpy(b->d_nloc, nl32.data(), b->nitems * sizeof(int32_t), cudaMemcpyHostToDevice));
    edge0.push_back(nnz_union);
    DI_CUDA_TRY(cudaMalloc(&b->d_eoff, edge0.size() * sizeof(int64_t)));
    DI_CUDA_TRY(cudaMemcpy(b->d_eoff, edge0.data(), edge0.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    const size_t nb = (size_t)n_union;
    DI_CUDA_TRY(cudaMalloc(&b->B, nb * sizeof(double)));
    DI_CUDA_TRY(cudaMalloc(&b->H, nb * sizeof(double)));
    DI_CUDA_TRY(cudaMalloc(&b->tmp, nb * sizeof(double)));
    DI_CUDA_TRY(cudaMalloc(&b->g, nb * sizeof(double)));
    DI_CUDA_TRY(cudaMalloc(&b->front, nb * sizeof(int32_t)));
    DI_CUDA_TRY(cudaMalloc(&b->items, b->nitems * sizeof(BItem)));
    DI_CUDA_TRY(cudaMalloc(&b->st, sizeof(BState)));
    DI_CUDA_TRY(cudaMalloc(&b->desc, sizeof(BDesc)));
    DI_CUDA_TRY(cudaMalloc(&b->pB, b->nitems * sizeof(double *)));
    DI_CUDA_TRY(cudaMalloc(&b->pH, b->nitems * sizeof(double *)));
    DI_CUDA_TRY(cudaMallocHost(&b->items_h, b->nitems * sizeof(BItem)));
    DI_CUDA_TRY(cudaMallocHost(&b->st_h, sizeof(BState)));
    DI_CUDA_TRY(cudaMallocHost(&b->desc_h, sizeof(BDesc)));
    DI_CUDA_TRY(cudaMallocHost(&b->pB_h, b->nitems * sizeof(double *)));
    DI_CUDA_TRY(cudaMallocHost(&b->pH_h, b->nitems * sizeof(double *)));
    DI_CUDA_TRY(cudaEventCreate(&b->ev0));
    DI_CUDA_TRY(cudaEventCreate(&b->ev1));
    const int sms = b->u->num_sms;
    b->grid_scan = (int)std::max<int64_t>(1, std::min<int64_t>(
                                                 occ_grid((const void *)k_bscan_level<double>, kBThreads, 0, sms),
                                                 b->nchunks));
    b->grid_push = occ_grid((const void *)k_bpush<double, false>, kBThreads, bpush_smem<double>(kMaxHot, false), sms);
    b->grid_push_slice = occ_grid((const void *)k_bpush<double, true>, kBThreads, bpush_smem<double>(kMaxHot, true), sms);
    const int64_t fch = (nnz_union + kBFlatEdges - 1) / kBFlatEdges;
    b->grid_flat = (int)std::max<int64_t>(
        1, std::min<int64_t>(occ_grid((const void *)k_bres_flat, kBThreads, 0, sms), (fch + kBThreads - 1) / kBThreads));
    return DI_OK;
}

}  // namespace

extern "C" DI_API di_status di_batch_create(const di_graph *const *graphs, int ng, const int *nrhs, void *stream,
                                           di_batch **out) {
    di::NvtxRange nvtx_range("di_batch_create");
    clear_error();
    if (!out) { set_error("di_batch_create: out is NULL"); return DI_EINVAL; }
    *out = nullptr;
    if (!graphs || !nrhs || ng < 1) { set_error("di_batch_create: need ng >= 1 graphs and their nrhs"); return DI_EINVAL; }
    int dev = -1;
    DI_CUDA_TRY(cudaGetDevice(&dev));
    int64_t items = 0;
    for (int gi = 0; gi < ng; ++gi) {
        if (!graphs[gi]) { set_error("di_batch_create: graph %d is NULL", gi); return DI_EINVAL; }
        if (graphs[gi]->device != dev) {
            set_error("di_batch_create: graph %d lives on device %d, current is %d", gi, graphs[gi]->device, dev);
            return DI_EINVAL;
        }
        if (nrhs[gi] < 0) { set_error("di_batch_create: nrhs[%d] = %d < 0", gi, nrhs[gi]); return DI_EINVAL; }
        items += nrhs[gi];
    }
    if (items < 1 || items > (1 << 20)) {
        set_error("di_batch_create: %lld work items; need 1 .. 2^20", (long long)items);
        return DI_EINVAL;
    }
    di_batch *b = new (std::nothrow) di_batch();
    if (!b) { set_error("di_batch_create: host allocation failed"); return DI_ENOMEM; }
    di_status rc = batch_create_impl(graphs, ng, nrhs, as_stream(stream), b);
    if (rc != DI_OK) {
        free_batch(b);
        return rc;
    }
    *out = b;
    return DI_OK;
}

extern "C" DI_API void di_batch_destroy(di_batch *b) { free_batch(b); }

extern "C" DI_API di_status di_batch_info(const di_batch *b, int *n_items, int64_t *n_union, int64_t *nnz_union) {
    clear_error();
    if (!b) { set_error("di_batch_info: NULL batch"); return DI_EINVAL; }
    if (n_items) *n_items = b->nitems;
    if (n_union) *n_union = b->n_union;
    if (nnz_union) *nnz_union = b->u->nnz;
    return DI_OK;
}

extern "C" DI_API di_status di_solve_batched(di_batch *b, const double *const *B, double d, const double *tol,
                                            double *const *H, const di_opts *opts, di_stats *item_stats,
                                            di_stats *total) {
    di::NvtxRange nvtx_range("di_solve_batched");
    clear_error();
    if (!b || !B || !H || !tol) { set_error("di_solve_batched: NULL batch, B, H or tol"); return DI_EINVAL; }
    di_opts o;
    if (opts) o = *opts; else di_opts_default(&o);
    if (!(d > 0.0 && d < 1.0)) { set_error("di_solve_batched: d = %g outside (0, 1)", d); return DI_EINVAL; }
    if (!(o.alpha > 1.0) || !std::isfinite(o.alpha)) { set_error("di_solve_batched: alpha = %g must be > 1", o.alpha); return DI_EINVAL; }
    if (o.max_levels < 0 || o.recompute_every < 0) { set_error("di_solve_batched: negative max_levels or recompute_every"); return DI_EINVAL; }
    if (!(o.recompute_drop == 0.0 || (o.recompute_drop > 1.0 && std::isfinite(o.recompute_drop)))) {
        set_error("di_solve_batched: recompute_drop = %g must be 0 or a finite factor > 1", o.recompute_drop);
        return DI_EINVAL;
    }
    if (o.warm_start) { set_error("di_solve_batched: warm starts are not supported in a batch"); return DI_EINVAL; }
    if (o.dangling < 0 || o.dangling > 1) { set_error("di_solve_batched: dangling = %d outside [0, 1]", o.dangling); return DI_EINVAL; }
    if (o.slice_sweeps < -1 || o.slice_sweeps > 4) {
        set_error("di_solve_batched: slice_sweeps = %d outside [-1, 4]", o.slice_sweeps);
        return DI_EINVAL;
    }
    if (o.spin_limit < 0 || o.spin_limit > (1LL << 40)) {
        set_error("di_solve_batched: spin_limit = %lld outside [0, 2^40] us", o.spin_limit);
        return DI_EINVAL;
    }
    for (int t = 0; t < b->nitems; ++t) {
        if (!B[t] || !H[t]) { set_error("di_solve_batched: NULL B or H of item %d", t); return DI_EINVAL; }
        if (!(tol[t] > 0.0) || !std::isfinite(tol[t])) {
            set_error("di_solve_batched: tol[%d] = %g must be finite and > 0", t, tol[t]);
            return DI_EINVAL;
        }
    }
    int dev = -1;
    DI_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != b->device) { set_error("di_solve_batched: batch lives on device %d, current is %d", b->device, dev); return DI_EINVAL; }
    cudaStream_t s = as_stream(o.stream);
    const int fp64 = o.fluid_fp64 ? 1 : 0;
    if (fp64 && !b->F64) DI_CUDA_TRY(cudaMalloc(&b->F64, (size_t)b->n_union * sizeof(double)));
    if (!fp64 && !b->F32) DI_CUDA_TRY(cudaMalloc(&b->F32, (size_t)b->n_union * sizeof(float)));
    DI_TRY(ensure_scale(b->u, d, s));
    // slice sweeps: -1 (auto) takes none in a batch.  Its items' frontiers
    // are mostly sparse (a personalised right-hand side starts from one node),
    // and on 64 graphs x 4 sources one sweep per level cut the diffusions by
    // 41% but took 260 against 230 ms: the per-level wait for the frontier
    // costs more than the diffusions it saves
    const int slice_sweeps = o.slice_sweeps >= 0 ? o.slice_sweeps : 0;
    b->push_slice = slice_sweeps > 0;
    DI_TRY(build_batch_graph(b, fp64));

    DI_CUDA_TRY(cudaStreamSynchronize(s));   // the pinned mirrors are reused call after call
    for (int t = 0; t < b->nitems; ++t) {
        b->pB_h[t] = B[t];
        b->pH_h[t] = H[t];
        std::memset(&b->items_h[t], 0, sizeof(BItem));
        b->items_h[t].tol = tol[t];
    }
    BDesc &dh = *b->desc_h;
    std::memset(&dh, 0, sizeof(dh));
    dh.d = d;
    dh.alpha = o.alpha;
    dh.R = o.recompute_every;
    dh.drop = o.recompute_drop;
    dh.fp64 = fp64;
    dh.max_levels = o.max_levels;
    dh.max_body_iters = (int)std::min<long long>(4LL * o.max_levels + 1000, INT32_MAX);
    dh.nitems = b->nitems;
    dh.thread_max = b->tune.thread_max_deg;
    dh.warp_max = b->tune.warp_max_deg;
    dh.dangling = o.dangling;
    dh.slice_sweeps = slice_sweeps;
    dh.wait_ns = (unsigned long long)o.spin_limit * 1000ull;
    dh.F = fp64 ? (void *)b->F64 : (void *)b->F32;
    dh.B = b->B;
    dh.H = b->H;
    dh.tmp = b->tmp;
    dh.g = b->g;
    dh.pB = b->pB;
    dh.pH = b->pH;
    DI_CUDA_TRY(cudaEventRecord(b->ev0, s));
    DI_CUDA_TRY(cudaMemcpyAsync(b->pB, b->pB_h, b->nitems * sizeof(double *), cudaMemcpyHostToDevice, s));
    DI_CUDA_TRY(cudaMemcpyAsync(b->pH, b->pH_h, b->nitems * sizeof(double *), cudaMemcpyHostToDevice, s));
    DI_CUDA_TRY(cudaMemcpyAsync(b->items, b->items_h, b->nitems * sizeof(BItem), cudaMemcpyHostToDevice, s));
    DI_CUDA_TRY(cudaMemcpyAsync(b->desc, b->desc_h, sizeof(BDesc), cudaMemcpyHostToDevice, s));
    DI_CUDA_TRY(cudaMemsetAsync(b->st, 0, sizeof(BState), s));
    if (fp64)
        k_bstart<double><<<b->grid_scan, kBThreads, 0, s>>>(b->desc, b->items, b->st, b->item_of_chunk, b->d_base,
                                                            b->d_nloc, b->nchunks);
    else
        k_bstart<float><<<b->grid_scan, kBThreads, 0, s>>>(b->desc, b->items, b->st, b->item_of_chunk, b->d_base,
                                                           b->d_nloc, b->nchunks);
    DI_CUDA_TRY(cudaGetLastError());
    long long launches = 1;
    if (o.timing) {
        // host-driven levels (profilers see every launch); same kernels
        for (;;) {
            for (int l = 0; l < 16; ++l) {
                if (fp64) { launch_blevel<double>(b, s, 0, 0, 2); launch_bres<double>(b, s); }
                else { launch_blevel<float>(b, s, 0, 0, 2); launch_bres<float>(b, s); }
                launches += 5;
            }
            DI_CUDA_TRY(cudaGetLastError());
            DI_CUDA_TRY(cudaMemcpyAsync(b->items_h, b->items, b->nitems * sizeof(BItem), cudaMemcpyDeviceToHost, s));
            DI_CUDA_TRY(cudaMemcpyAsync(b->st_h, b->st, sizeof(BState), cudaMemcpyDeviceToHost, s));
            DI_CUDA_TRY(cudaStreamSynchronize(s));
            bool live = false;
            for (int t = 0; t < b->nitems; ++t) live |= b->items_h[t].done == 0;
            if (!live || b->st_h->body_iters >= dh.max_body_iters) break;
        }
    } else {
        DI_CUDA_TRY(cudaGraphLaunch(b->sg[fp64].exec, s));
    }
    DI_CUDA_TRY(cudaMemcpyAsync(b->items_h, b->items, b->nitems * sizeof(BItem), cudaMemcpyDeviceToHost, s));
    DI_CUDA_TRY(cudaMemcpyAsync(b->st_h, b->st, sizeof(BState), cudaMemcpyDeviceToHost, s));
    DI_CUDA_TRY(cudaStreamSynchronize(s));
    const int body_iters = b->st_h->body_iters;
    if (!o.timing) launches += 2LL * body_iters;
    long long recomputes = 0;
    for (int t = 0; t < b->nitems; ++t) recomputes += b->items_h[t].recomputes;
    // items that did not converge: their exact residual for the report
    bool refresh = false;
    for (int t = 0; t < b->nitems; ++t) {
        BItem &it = b->items_h[t];
        it.rec = it.done != 1 ? 1 : 0;
        it.res_sum = 0.0;
        it.res_max = 0ull;
        refresh |= it.rec != 0;
    }
    if (refresh) {
        dh.final_mode = 1;
        DI_CUDA_TRY(cudaMemcpyAsync(b->desc, b->desc_h, sizeof(BDesc), cudaMemcpyHostToDevice, s));
        DI_CUDA_TRY(cudaMemcpyAsync(b->items, b->items_h, b->nitems * sizeof(BItem), cudaMemcpyHostToDevice, s));
        if (fp64) launch_bres<double>(b, s); else launch_bres<float>(b, s);
        launches += 3;
        DI_CUDA_TRY(cudaMemcpyAsync(b->items_h, b->items, b->nitems * sizeof(BItem), cudaMemcpyDeviceToHost, s));
    }
    k_bfinish<<<b->grid_scan, kBThreads, 0, s>>>(b->desc, b->item_of_chunk, b->d_base, b->d_nloc, b->nchunks);
    launches += 1;
    DI_CUDA_TRY(cudaGetLastError());
    DI_CUDA_TRY(cudaEventRecord(b->ev1, s));
    DI_CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.f;
    DI_CUDA_TRY(cudaEventElapsedTime(&ms, b->ev0, b->ev1));

    di_status rc = DI_OK;
    di_stats tot;
    std::memset(&tot, 0, sizeof(tot));
    for (int t = 0; t < b->nitems; ++t) {
        const BItem &it = b->items_h[t];
        di_status irc = DI_OK;
        if (it.done == 3 || !std::isfinite(it.r_exact)) irc = DI_ENONFINITE;
        else if (it.done != 1) irc = DI_ENOCONV;
        if (irc == DI_ENONFINITE) rc = DI_ENONFINITE;
        else if (irc == DI_ENOCONV && rc == DI_OK) rc = DI_ENOCONV;
        if (item_stats) {
            di_stats &st = item_stats[t];
            std::memset(&st, 0, sizeof(st));
            st.levels = it.level;
            st.recomputes = it.recomputes;
            st.node_diffusions = (int64_t)it.node_diff;
            st.edge_diffusions = (int64_t)it.edge_diff;
            st.resid_l1 = it.r_exact;
            st.err_bound = it.r_exact / (1.0 - d);
            st.b_l1 = it.b_l1;
            st.f0_l1 = it.b_l1;
            st.seconds = ms * 1e-3;
            st.status = irc;
        }
        tot.levels = std::max(tot.levels, it.level);
        tot.recomputes += it.recomputes;
        tot.node_diffusions += (int64_t)it.node_diff;
        tot.edge_diffusions += (int64_t)it.edge_diff;
        tot.resid_l1 += it.r_exact;
        tot.b_l1 += it.b_l1;
    }
    if (rc == DI_ENONFINITE) set_error("di_solve_batched: a residual is not finite (non-finite B?)");
    else if (rc == DI_ENOCONV) set_error("di_solve_batched: level cap %d reached by at least one item", o.max_levels);
    if (total) {
        tot.err_bound = tot.resid_l1 / (1.0 - d);
        tot.f0_l1 = tot.b_l1;
        tot.seconds = ms * 1e-3;
        tot.status = rc;
        tot.gpu_launches = launches;
        tot.body_iterations = body_iters;
        tot.recompute_launches = (int32_t)std::min<long long>(recomputes, INT32_MAX);
        *total = tot;
    }
    (void)recomputes;
    return rc;
}

extern "C" DI_API di_status di_batch_set_tune(di_batch *b, const di_tune *t) {
    clear_error();
    if (!b) { set_error("di_batch_set_tune: NULL batch"); return DI_EINVAL; }
    DI_TRY(check_tune(t, "di_batch_set_tune"));
    b->tune = *t;
    return DI_OK;
}

extern "C" DI_API di_status di_batch_get_tune(const di_batch *b, di_tune *t) {
    clear_error();
    if (!b || !t) { set_error("di_batch_get_tune: NULL argument"); return DI_EINVAL; }
    *t = b->tune;
    return DI_OK;
}

// Frontier tile shape of the batched push: times complete batched solves for
// each candidate shape and keeps the fastest.
extern "C" DI_API di_status di_batch_autotune(di_batch *b, const double *const *B, double d, const double *tol,
                                             double *const *H, const di_opts *opts, const char *cache_path,
                                             di_tune *best, double *best_seconds) {
    clear_error();
    if (!b || !B || !H || !tol) { set_error("di_batch_autotune: NULL argument"); return DI_EINVAL; }
    di_opts o;
    if (opts) o = *opts; else di_opts_default(&o);
    o.timing = 0;
    char key[160];
    std::snprintf(key, sizeof(key), "batch items=%d n=2^%d nnz=2^%d fp64=%d", b->nitems, ilog2_round(b->n_union),
                  ilog2_round(b->u->nnz), o.fluid_fp64 ? 1 : 0);
    di_tune hit;
    if (tune_cache_lookup(cache_path, key, &hit)) {
        b->tune = hit;
        if (best) *best = hit;
        if (best_seconds) *best_seconds = 0.0;
        return DI_OK;
    }
    const int occ_per_sm = std::max(1, b->grid_push / std::max(1, b->u->num_sms));
    di_tune cand[16];
    const int nc = tune_candidates(cand, 16);
    di_tune win = b->tune;
    double win_s = 1e300;
    for (int c = 0; c < nc; ++c) {
        di_tune t = cand[c];
        if (t.push_ctas_per_sm < 0) {
            if (occ_per_sm < 2) continue;
            t.push_ctas_per_sm = occ_per_sm / 2;
        }
        b->tune = t;
        double secs = 1e300;
        for (int rep = 0; rep < 2; ++rep) {   // the first solve rebuilds the level graph
            di_stats tot;
            const di_status rc = di_solve_batched(b, B, d, tol, H, &o, nullptr, &tot);
            if (rc != DI_OK && rc != DI_ENOCONV) return rc;
            if (rep > 0) secs = tot.seconds;
        }
        if (secs < win_s) { win_s = secs; win = t; }
    }
    b->tune = win;
    tune_cache_store(cache_path, key, win, win_s);
    if (best) *best = win;
    if (best_seconds) *best_seconds = win_s;
    return DI_OK;
}
