// di_internal.cuh - internal types and helpers of libdi.so (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "di.h"
#include <nvtx3/nvToolsExt.h>

namespace di {

// NVTX range for profilers' timelines (a no-op unless a tool is attached):
// every entry point, and in the host-driven level loop every level and kernel.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// ------------------------------------------------------------------ errors

void set_error(const char *fmt, ...);
void clear_error();

#define DI_CUDA_TRY(expr)                                                              \
    do {                                                                               \
        cudaError_t e_ = (expr);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            ::di::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),    \
                            __FILE__, __LINE__);                                       \
            return e_ == cudaErrorMemoryAllocation ? DI_ENOMEM : DI_ECUDA;             \
        }                                                                              \
    } while (0)

#define DI_TRY(expr)                                                                   \
    do {                                                                               \
        di_status s_ = (expr);                                                         \
        if (s_ != DI_OK) return s_;                                                    \
    } while (0)

// ------------------------------------------------------------------ tuning constants

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;                                // per thread per chunk
constexpr int kScanChunk = kScanThreads * kScanItems;       // nodes per block iteration
constexpr int kPushThreads = 256;                            // = frontier tile size
constexpr int kThreadMaxDeg = 16;   // default: out-degree <= this: one thread pushes the row
constexpr int kWarpMaxDeg = 512;    // default: <= this: one warp; above: the whole CTA
constexpr int kResThreads = 256;
constexpr int kResSeg = 8192;       // in-rows longer than this are split in segments (allocation-free path)
constexpr int kResFine = 256;       // segment length of the exact residual's long in-rows
constexpr int kMaxHot = 2048;       // privatised hot targets (shared-memory slots)
constexpr int kHotMinIndeg = 2048;  // a hot target has at least this in-degree (about 2x the push CTAs)
constexpr int kSrcBlockShift = 22;  // exact residual: sources in blocks of 2^22 nodes (32 MB of FP64 gathers)
constexpr int kWinBins = 4;         // tiled level kernel: window radii 32 .. 256 (powers of two)
constexpr int kMaxWinR = 32 << (kWinBins - 1);
constexpr int kPushWin = 1024;      // frontier push: nodes of a tile's fluid window beyond its radius
constexpr int kSliceQueueCap = 1536;   // frontier push: entries of a CTA's slice-sweep queue
constexpr int kSliceDensity = 32;      // slice sweeps follow frontiers of at least 1/32 of the nodes
constexpr int kSliceWaitPct = 50;      // a slice sweep starts once this share of the frontier's tiles is done
constexpr int kLevelsPerIter = 2;      // propagations 3, 4: levels per WHILE iteration of the level graph

// ------------------------------------------------------------------ solver state

// Everything a level kernel needs beyond its fixed graph arrays: written by
// the host before each solve (pointers change from call to call, the
// instantiated CUDA graph does not).
struct SolveDesc {
    const double *B;
    double *H;
    double *F_out;        // optional FP64 residual output
    void *F;              // internal fluid (float or double)
    double d, tol, alpha;
    int max_levels;
    int recompute_every;  // FP32 fluid: exact recompute period (levels), 0 = none
    double recompute_drop;// FP32 fluid: exact recompute when |F|_1 fell this much since the last, 0 = none
    int fluid_fp64;
    int max_body_iters;   // absolute cap on loop iterations (safety net)
    int propagation;      // 0/1 auto (binned/flat gather for dense levels), 2 push only, 3 async push
    int push_ratio;       // dense when active edges * push_ratio >= edges
    int64_t n_nodes;
    int thread_max;       // push shape: rows up to this many edges go to one thread
    int warp_max;         // ... up to this to one warp, longer ones to the CTA
    const void *iw;       // weighted selection: 1 / ((in + 1)(out + 1)) per node (FT), else NULL
    int dangling;         // 1: columns of dangling nodes completed by d/N (uniform)
    int resweeps;         // propagations 3-7: extra selections at the same T before T <- T / alpha
    int win_R;            // frontier push (propagations 3, 7): radius of the shared-memory fluid window, 0 = none
    int slice_sweeps;     // frontier push (propagations 3, 7): sweeps of each CTA's node slice after the frontier
    unsigned long long wait_ns;   // bound of the push's wait for the frontier tiles before a slice sweep
};

// Device-resident level-loop state (one per graph object).
struct SolveState {
    double T;             // threshold of the next scan
    double r_scan;        // sum |F| seen by the last scan
    double max_scan;      // max |F| seen by the last scan
    double r_exact;       // last exact FP64 residual
    double max_exact;
    double b_l1;          // |B|_1
    double f0_l1;         // |F_0|_1 of the start in use
    unsigned long long node_diff, edge_diff;
    int level;            // levels with a non-empty push
    int since_recompute;  // levels since the last exact recompute
    int recomputes;
    int nfront;           // frontier size written by the scan (reset by its control)
    int push_count;       // frontier size to push this level (0 = no push)
    int do_recompute;     // exact recompute at the end of this level
    int confirming;       // the recompute confirms a stop request
    int force_push;       // a stop request was refuted: push at least once
    int done;             // 0 running, 1 converged, 2 level cap, 3 non-finite
    int body_iters;
    int nsel;             // nodes selected in this level (all chunks)
    double est_scale;     // calibration of the scan's residual estimate (0 = 1)
    double r_confirm;     // estimate that triggered the pending confirmation
    unsigned int chunk_ctr;     // (unused)
    unsigned int rctr[64];      // chunk counters of the sparse push, one per node range
    unsigned long long lvl_nodes, lvl_edges;   // drained this level
    int p2mode;                 // propagation of this level: 0 none, 1 pull, 2 push
    unsigned int push_blocks;   // last-block counter of the sparse push
    unsigned int tile_ctr;      // dynamic tile scheduling of the push
    unsigned int scan_blocks;   // last-block counters
    unsigned int res_blocks;
    unsigned int init_blocks;
    int pad;
    double dang_acc;            // fluid drained from dangling nodes since the last selection
    double dang_h;              // exact residual: sum of H over the dangling nodes
    double dang_next;           // tiled level: dangling fluid drained in this level (for the next)
    int phase;                  // selections made at the current T (0 = the level's first)
    int timed_out;              // persistent loop: a grid barrier gave up (DI_ETIMEOUT)
    unsigned int bar_count;     // persistent loop: CTAs arrived at the current grid barrier
    unsigned int bar_gen;       // persistent loop: barrier generation (released when it changes)
    unsigned long long t_mark;  // persistent loop: %globaltimer at the last phase boundary (ns)
    unsigned long long t_scan_ns, t_push_ns;   // persistent loop: time in selection / push phases
    unsigned long long passes;  // persistent loop: selection passes made
    unsigned long long red_ops; // tiled level: global reduction sectors issued (scattered reds count one each)
    double T_push;              // selection threshold of the frontier being pushed (the slice sweeps' T)
    unsigned long long slice_nodes;  // nodes diffused by the push's slice sweeps
    unsigned int tiles_done;    // frontier tiles whose pushes are done (slice sweeps wait for all)
};

enum ResMode : int {
    RES_STANDALONE = 0,   // di_residual: FP64 F out, sum
    RES_LEVEL = 1,        // inside the level loop: only when do_recompute; control
    RES_WARM_INIT = 2,    // warm start: F0 = B + P H0 - H0 into the fluid, T0 = max
    RES_FINAL = 3         // after the loop: refresh F_out and r_exact
};

struct SolverGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle h_while = 0, h_if = 0, h_p2 = 0;
    cudaGraphConditionalHandle h_ifk[kLevelsPerIter - 1] = {};   // propagations 3, 4: the body's later levels
    bool built = false;
    int l2 = 0;           // built with the L2 window
    int prop = 0;         // built with this propagation option
    int res_form = 0;     // built with this exact-residual form
    int grid_push = 0;    // built with this push grid
    unsigned long long timeout_ns = 0;   // built with this grid-barrier bound (persistent loop)
    int grid_coop = 0;                   // built with this persistent grid
    int slice = 0;                       // built with the slice-sweep variant of the push
};

struct Workspace {
    bool ready = false;
    float *F32 = nullptr;
    double *F64 = nullptr;
    float *w32 = nullptr;          // drained fluid scaled by d/outdeg, per level
    double *w64 = nullptr;
    int32_t *front = nullptr;      // frontier list [n]
    double *g = nullptr;           // s_j H_j for the exact residual [n]
    double *acc = nullptr;         // exact residual accumulator of the source-blocked form [n]
    double *seg_part = nullptr;    // per-segment partial sums
    double *part_sum = nullptr;    // per-block partial sums
    double *part_max = nullptr;
    SolveDesc *desc = nullptr;     // device
    SolveState *st = nullptr;      // device
    SolveDesc *desc_h = nullptr;   // pinned host mirror
    SolveState *st_h = nullptr;
    double *hostB = nullptr, *hostH = nullptr, *hostF = nullptr;   // di_solve_host buffers
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t tev[64] = {};       // timing mode: 4 per level, 16 levels per batch
};

struct KpidCache;   // partition.cu: what di_solve_partitioned keeps on a graph
}  // namespace di

constexpr int kThreadMaxDegDefault = di::kThreadMaxDeg;
constexpr int kWarpMaxDegDefault = di::kWarpMaxDeg;

struct di_graph {
    int device = 0;
    int num_sms = 0;
    int64_t n = 0, nnz = 0;
    int64_t n_dangling = 0, max_outdeg = 0, max_indeg = 0;
    int n_hot = 0;
    int n_seg = 0;            // segments of the long in-rows
    int n_long_rows = 0;      // in-rows split in segments
    int32_t *rp = nullptr;        // out-CSR offsets [n+1]
    int32_t *pcol = nullptr;      // push targets [nnz]: k, or -1-slot for a hot target
    int32_t *hot_node = nullptr;  // [n_hot]
    int32_t *in_rp = nullptr;     // in-CSR offsets [n+1]
    int32_t *in_col = nullptr;    // in-CSR sources [nnz]
    int32_t *long_rows = nullptr; // [n_long_rows] ids of split in-rows
    int32_t *long_seg0 = nullptr; // [n_long_rows + 1] first segment of each
    int32_t *seg_row = nullptr;   // [n_seg] in-row of each segment (index in long_rows)
    int64_t *seg_beg = nullptr;   // [n_seg] first in-edge of each segment
    // the same table with kResFine-edge segments (exact residual of the solver)
    int n_fseg = 0, n_frows = 0;
    int32_t *frows = nullptr, *fseg0 = nullptr, *fseg_row = nullptr;
    int64_t *fseg_beg = nullptr;
    // binned pull plan over the in-edges (pull.cuh): device arrays and offsets
    int32_t *pl_rows = nullptr, *pl_seg_row = nullptr, *pl_seg_beg = nullptr;
    int32_t *pl_b12_off = nullptr, *pl_b12_col = nullptr;   // bins 1-2 edges in bin order
    int32_t *outdeg = nullptr;                            // [n] out-degrees
    int32_t *erow = nullptr;                              // [nnz] destination row of each in-edge
    // in-edges in source-blocked order (source block of 2^kSrcBlockShift
    // nodes, then destination row): bcol = source, brow = destination.  Built
    // on first use; with one block they alias in_col / erow.
    int32_t *bcol = nullptr, *brow = nullptr;
    int n_src_blocks = 1;
    int res_form = 0;             // exact residual: 0 auto, 1 binned gather, 2 source-blocked flat gather
    int32_t *pl_lrows = nullptr, *pl_lseg0 = nullptr;   // rows of bin 5 and their first segment
    int pl_nlrows = 0;
    int64_t pl_bin_off[5] = {0, 0, 0, 0, 0};
    int64_t pl_task_off[6] = {0, 0, 0, 0, 0, 0};
    // d / outdeg, cached for the last damping factor used
    double scale_d = -1.0;
    float *s32 = nullptr;
    double *s64 = nullptr;
    // tiled level kernel: radius of the shared-memory fluid window (-1 = not yet chosen),
    // nodes per chunk and grid (per fluid precision)
    int win_R = -1;
    int tiled_chunk[2] = {0, 0}, grid_tiled[2] = {0, 0};
    // persistent level loop: cooperative grid (per fluid precision) and grid-barrier bound
    int grid_coop[2] = {0, 0};
    unsigned long long coop_timeout_ns = 0;
    int push_R = 0;               // frontier push: window radius in use (0 = none)
    di::KpidCache *kpid = nullptr;   // di_solve_partitioned: ranges, buffers and round graph of the last K
    int push_slice = 0;           // frontier push: the slice-sweep variant in use (opts.slice_sweeps > 0)
    int grid_push_slice = 0;      // occupancy grid of the slice-sweep variant
    // weighted selection (Sec. 2.4 score): 1 / ((in + 1)(out + 1)), built on first use
    float *iw32 = nullptr;
    double *iw64 = nullptr;
    // grid sizes (persistent kernels)
    int grid_scan = 0, grid_push = 0, grid_res = 0, grid_level = 0;
    int grid_select = 0, grid_pull = 0, grid_pushw = 0, grid_flat = 0;
    int level_items = 8;          // nodes per thread per chunk of the fused level kernel
    di::Workspace ws;
    di_tune tune = {kThreadMaxDegDefault, kWarpMaxDegDefault, 0, 0};   // push shape (di_autotune)
    di::SolverGraph sg[2];        // [fluid_fp64]
    cudaAccessPolicyWindow win[4] = {};   // L2 windows: [2 * (0: F, 1: w) + fluid_fp64]
    int win_ready[4] = {0, 0, 0, 0}, win_ok[4] = {0, 0, 0, 0};
};

namespace di {

// ------------------------------------------------------------------ device helpers

__device__ __forceinline__ void red_add(float *addr, float v) {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add(double *addr, double v) {
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(addr), "d"(v) : "memory");
}

// Adds each thread's kE (destination, value) pairs into acc, for pairs sorted
// by destination along the warp (lane l holds the l-th group of kE consecutive
// edges; destination -1 = no edge, value 0, skipped wherever it is).  Runs of equal
// destination are summed in registers; a thread's first run, when it
// continues the previous lane's last run, goes to that lane, and the last runs
// are summed over lanes of equal destination: a destination whose in-edges
// span many lanes (a hub) takes one reduction per warp, not one per thread
// on the same L2 address.  All 32 lanes must call it together.
template <int kE>
__device__ __forceinline__ void warp_runs_add(const int32_t (&row)[kE], const double (&val)[kE], double *acc,
                                              int lane) {
    constexpr unsigned kFull = 0xffffffffu;
    int32_t kA = -1, kB = row[0];
    double sA = 0.0, sB = val[0];
    bool first_open = true;
#pragma unroll
    for (int k = 1; k < kE; ++k) {
        if (row[k] != kB) {
            if (first_open) {   // the first run closes (a key of -1 is then dropped below)
                kA = kB;
                sA = sB;
                first_open = false;
            } else if (kB >= 0) {
                red_add(acc + kB, sB);
            }
            kB = row[k];
            sB = val[k];
        } else {
            sB += val[k];
        }
    }
    const int32_t kA_next = __shfl_down_sync(kFull, kA, 1);
    const double sA_next = __shfl_down_sync(kFull, sA, 1);
    const int32_t kB_prev = __shfl_up_sync(kFull, kB, 1);
    if (lane < 31 && kA_next >= 0 && kA_next == kB) sB += sA_next;
    if (kA >= 0 && !(lane > 0 && kA == kB_prev)) red_add(acc + kA, sA);
    // segmented sum of the last runs; segments are numbered from their heads,
    // so only neighbouring lanes merge.  The steps stop once no segment is
    // longer than the distance (FP64 adds are scarce on this part): none when
    // every lane heads its own segment
    const bool head = lane == 0 || kB != kB_prev;
    const unsigned heads = __ballot_sync(kFull, head);
    double v = sB;
    if (heads != kFull) {
        const int seg = __popc(heads & (kFull >> (31 - lane)));
#pragma unroll 1
        for (int o = 1; o < 32; o <<= 1) {
            const double w = __shfl_down_sync(kFull, v, o);
            const int s2 = __shfl_down_sync(kFull, seg, o);
            const bool same = lane + o < 32 && s2 == seg;
            if (same) v += w;
            if (!__any_sync(kFull, same)) break;
        }
    }
    if (head && kB >= 0) red_add(acc + kB, v);
}

// L2 policy "evict last" for the fluid vector: the scatter target stays in
// L2 while the column indices, offsets and histories stream past it.
__device__ __forceinline__ uint64_t l2_keep_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void red_add_keep(float *addr, float v, uint64_t pol) {
    asm volatile("red.global.add.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(addr), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void red_add_keep(double *addr, double v, uint64_t pol) {
    asm volatile("red.global.add.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(addr), "d"(v), "l"(pol) : "memory");
}
// fetch-and-add with the same policy: returns the target's value before the add
__device__ __forceinline__ float atom_add_keep(float *addr, float v, uint64_t pol) {
    float old;
    asm volatile("atom.global.add.L2::cache_hint.f32 %0, [%1], %2, %3;"
                 : "=f"(old) : "l"(addr), "f"(v), "l"(pol) : "memory");
    return old;
}
__device__ __forceinline__ double atom_add_keep(double *addr, double v, uint64_t pol) {
    double old;
    asm volatile("atom.global.add.L2::cache_hint.f64 %0, [%1], %2, %3;"
                 : "=d"(old) : "l"(addr), "d"(v), "l"(pol) : "memory");
    return old;
}
__device__ __forceinline__ float atomic_exch_keep(float *p, float v, uint64_t pol) {
    uint32_t old;
    asm volatile("atom.global.exch.L2::cache_hint.b32 %0, [%1], %2, %3;"
                 : "=r"(old) : "l"(p), "r"(__float_as_uint(v)), "l"(pol) : "memory");
    return __uint_as_float(old);
}
__device__ __forceinline__ double atomic_exch_keep(double *p, double v, uint64_t pol) {
    unsigned long long old;
    asm volatile("atom.global.exch.L2::cache_hint.b64 %0, [%1], %2, %3;"
                 : "=l"(old) : "l"(p), "l"(static_cast<unsigned long long>(__double_as_longlong(v))), "l"(pol)
                 : "memory");
    return __longlong_as_double(static_cast<long long>(old));
}

__device__ __forceinline__ float atomic_exch_fluid(float *p, float v) { return atomicExch(p, v); }
__device__ __forceinline__ double atomic_exch_fluid(double *p, double v) {
    unsigned long long old = atomicExch(reinterpret_cast<unsigned long long *>(p),
                                        static_cast<unsigned long long>(__double_as_longlong(v)));
    return __longlong_as_double(static_cast<long long>(old));
}

// Calls push(c) for the targets c = pcol[q], q = first, first + step, ...
// < end.  The column indices are loaded kBatch at a time before their
// pushes are issued, so the loads of a batch are in flight together (the
// pushes are volatile asm with a memory clobber, which would otherwise
// serialise each load behind the previous push).
template <int kBatch, typename Push>
__device__ __forceinline__ void push_range(const int32_t *__restrict__ pcol, int64_t first, int64_t end, int step,
                                           Push &push) {
    for (int64_t q0 = first; q0 < end; q0 += (int64_t)kBatch * step) {
        int32_t c[kBatch];
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            const int64_t q = q0 + (int64_t)k * step;
            c[k] = q < end ? __ldcs(pcol + q) : 0;
        }
#pragma unroll
        for (int k = 0; k < kBatch; ++k)
            if (q0 + (int64_t)k * step < end) push(c[k]);
    }
}

// Threshold in the fluid's precision: a float threshold is rounded up, so
// |F_i| >= T in FP32 never selects a node the FP64 comparison would not.
__device__ __forceinline__ float thr_cast(double T, float) { return __double2float_ru(T); }
__device__ __forceinline__ double thr_cast(double T, double) { return T; }

// Exact recomputation as iterative refinement (FP32 fluid only): every
// recompute_every levels, and whenever the running |F|_1 estimate r has
// fallen by the factor recompute_drop since the last exact residual.  The
// FP32 pushes round each target to 2^-24 of its value, so the drift they add
// between two recomputations stays a small multiple of 2^-24 * recompute_drop
// of the current residual.
__device__ __forceinline__ bool refine_due(const SolveDesc *__restrict__ desc, const SolveState *__restrict__ st,
                                           int since, double r) {
    if (desc->fluid_fp64) return false;
    const int R = desc->recompute_every;
    const double drop = desc->recompute_drop;
    return (R > 0 && since >= R) || (drop > 0.0 && r * drop <= __ldcg(&st->r_exact));
}

// Threshold schedule after one selection pass (Sec. 2.4): a level starts at
// T; after its pass the level is re-selected at the same T up to `resweeps`
// times (nodes that crossed T while the level pushed - the fluid a
// sequential sweep would have met later in the same sweep), then T <- T /
// alpha.  A pass that selects nothing ends the level; an empty first pass
// lowers T to the first T / alpha^k <= the largest fluid tm (an empty sweep
// changes nothing).  level counts threshold levels that diffused, since the
// levels since the last exact recomputation.
__device__ __forceinline__ void lower_threshold(double &T, double alpha, double tm) {
    if (tm > 0.0) {
        for (int guard = 0; T > tm && guard < 8192; ++guard) T /= alpha;
        if (T > tm) T = tm;   // alpha so close to 1 that the guard ran out
    }
}
__device__ __forceinline__ void threshold_step(int resweeps, bool pushed, double alpha, double tm, double &T,
                                               int &phase, int &level, int &since) {
    if (pushed) {
        if (phase == 0) {
            level += 1;
            since += 1;
        }
        if (phase < resweeps) {
            phase += 1;
        } else {
            phase = 0;
            T /= alpha;
        }
    } else {
        if (phase > 0) {
            phase = 0;
            T /= alpha;
        }
        lower_threshold(T, alpha, tm);
    }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum and max of one double per thread; result valid in thread 0.
template <int THREADS>
__device__ __forceinline__ void block_sum_max(double &s, double &m) {
    __shared__ double ss[THREADS / 32], sm[THREADS / 32];
    s = warp_sum(s);
    m = warp_max(m);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { ss[w] = s; sm[w] = m; }
    __syncthreads();
    if (w == 0) {
        s = l < THREADS / 32 ? ss[l] : 0.0;
        m = l < THREADS / 32 ? sm[l] : 0.0;
        s = warp_sum(s);
        m = warp_max(m);
    }
    __syncthreads();
}

// Adds this CTA's per-thread counts to up to four device counters with one
// global atomic per counter and CTA (the same-address atomics of every warp
// would serialise at one L2 slice).  Every thread of the CTA must call it.
__device__ __forceinline__ void cta_add_counts(unsigned long long *c0, unsigned long long v0, unsigned long long *c1,
                                               unsigned long long v1, unsigned long long *c2 = nullptr,
                                               unsigned long long v2 = 0, unsigned long long *c3 = nullptr,
                                               unsigned long long v3 = 0) {
    __shared__ unsigned long long s_c[4];
    if (threadIdx.x < 4) s_c[threadIdx.x] = 0ull;
    __syncthreads();
    v0 = warp_sum(v0);
    v1 = warp_sum(v1);
    v2 = warp_sum(v2);
    v3 = warp_sum(v3);
    if ((threadIdx.x & 31) == 0) {
        if (v0) atomicAdd(&s_c[0], v0);
        if (v1) atomicAdd(&s_c[1], v1);
        if (v2) atomicAdd(&s_c[2], v2);
        if (v3) atomicAdd(&s_c[3], v3);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_c[0] && c0) atomicAdd(c0, s_c[0]);
        if (s_c[1] && c1) atomicAdd(c1, s_c[1]);
        if (s_c[2] && c2) atomicAdd(c2, s_c[2]);
        if (s_c[3] && c3) atomicAdd(c3, s_c[3]);
    }
}

// Marks this block done; returns true in every thread of the last block to
// finish (the one that sees all partials).  counter must start at 0 and is
// reset to 0 by the last block.
__device__ __forceinline__ bool last_block(unsigned int *counter) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int prev = atomicAdd(counter, 1u);
        is_last = (prev == gridDim.x - 1);
        if (is_last) *counter = 0;
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

// ------------------------------------------------------------------ cross-TU entry points

// graph.cu: (re)compute d / outdeg for damping d
di_status ensure_scale(di_graph *g, double d, cudaStream_t s);
// graph.cu: the source-blocked in-edge order of the exact residual (lazy)
di_status ensure_blocked_order(di_graph *g, cudaStream_t s);
// graph.cu: the selection weights 1 / ((in + 1)(out + 1)) (lazy)
di_status ensure_selection_weights(di_graph *g, cudaStream_t s);
// graph.cu: the window radius of the tiled level kernel (lazy)
di_status ensure_window(di_graph *g, cudaStream_t s);
// solve.cu
di_status ensure_workspace(di_graph *g);
int push_grid(const di_graph *g, bool slice = false);
void free_kpid_cache(di_graph *g);   // partition.cu
// tune.cu: validation of a push shape, candidates, and the JSON-lines cache
di_status check_tune(const di_tune *t, const char *who);
int tune_candidates(di_tune *out, int cap);
bool tune_cache_lookup(const char *path, const char *key, di_tune *out);
void tune_cache_store(const char *path, const char *key, const di_tune &t, double seconds);
int ilog2_round(int64_t v);
// residual.cu: launch the exact-residual kernels (prep, segments, rows)
void launch_residual(di_graph *g, int fluid_fp64, ResMode mode, cudaStream_t s);
int residual_grid(int sms);
int residual_kernels(const di_graph *g);
int residual_partials(const di_graph *g);
// batched / warm-start modules register nothing here yet

inline cudaStream_t as_stream(void *p) { return reinterpret_cast<cudaStream_t>(p); }

}  // namespace di
