// partition.cu - the K-PID asynchronous D-iteration of Secs. 2.3-2.6 on one GPU.
//
// The nodes are split into K contiguous ranges Omega_k (uniform, or cost
// balanced so that every range holds about L / K out-edges, Sec. 2.3).  The
// PID of range k keeps its own threshold T_k and diffuses its nodes to their
// children inside Omega_k only (the algorithm (*) of Sec. 2.5); the fluid it
// owes to other ranges is carried by H - H_old and transmitted, as
// P (H - H_old) restricted to external children, once the amount s_k exceeds
// r_k / K (Eq. send).  A range that receives fluid rescales its threshold by
// (r_k + received) / r_k, or sets it to the received amount when it held no
// fluid (Sec. 2.6).  On one GPU every PID runs in the same
// launches, one round (one threshold level of every range) at a time:
//   k_pscan  - selection |F_i| >= T_k, per-range |F|_1, max and count; its
//              last CTA runs the control of every range (threshold, the
//              transmission decision) and the stop request;
//   k_ppush  - drain f = atomicExch(F_i, 0), H_i += f, local children only;
//              the fluid owed to other ranges accumulates into s_k;
//   k_psend  - transmission of the ranges that decided to send; its last
//              CTA rescales the thresholds of the receivers;
//   exact residual (residual.cu) as the stop test and refinement: it
//              contains the fluid still owed, so H_old is reset with it.
// The rounds run on the device: a CUDA graph holds a WHILE node around
// [k_pscan -> k_ppush -> k_psend -> IF(k_phold -> exact residual)], and
// k_pscan's last CTA sets both conditions.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "di_internal.cuh"

namespace di {
namespace {

constexpr int kMaxParts = 64;
constexpr int kPThreads = 256;
constexpr int kPThreadRow = 16;   // rows up to this many edges go to one thread, longer ones to a warp

// Per-range state on the device.  Sums are cleared by the step that consumes them.
struct PartState {
    double T[kMaxParts];                 // threshold of the next selection
    double r[kMaxParts];                 // |F|_1 over the range, from the selection
    unsigned long long m[kMaxParts];     // max |F| (bits; non-negative doubles order like integers)
    unsigned long long sel[kMaxParts];   // nodes selected
    double s[kMaxParts];                 // fluid owed to other ranges since the last transmission
    double rdec[kMaxParts];              // |F|_1 at the last transmission decision
    double recv[kMaxParts];              // fluid received in this round's transmissions
    unsigned long long ops[kMaxParts];   // elementary diffusions of the range's PID
    unsigned long long sends[kMaxParts]; // transmissions of the range's PID
    int send[kMaxParts];                 // this round: transmit
    // 1/N completion (Sec. 2.2): the per-node amount every node of range k gets
    // at its next selection (completed columns' local parts and received
    // parts), and the sending ranges' sum of H - H_old over their dangling nodes
    double pend[kMaxParts];
    double dsend[kMaxParts];
    int any_send;
    int K;
    unsigned int scan_blocks, send_blocks, init_blocks;
};

__device__ __forceinline__ double bits_to_double(unsigned long long b) {
    return __longlong_as_double(static_cast<long long>(b));
}
__device__ __forceinline__ unsigned long long double_to_bits(double v) {
    return static_cast<unsigned long long>(__double_as_longlong(v));
}

// Node range of CTA b: [b * span, min(n, (b + 1) * span)), span a multiple of
// the block size; threads interleave inside it, so a thread meets few range
// boundaries and flushes its per-range sums rarely.
__device__ __forceinline__ int64_t cta_span(int64_t n) {
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    return (per + kPThreads - 1) / kPThreads * kPThreads;
}

// The range of node j: the last k with bounds[k] <= j (bounds in shared
// memory, K + 1 entries, non-decreasing; at most 7 steps for K <= 64).
__device__ __forceinline__ int range_of(const int64_t *s_b, int K, int64_t j) {
    int lo = 0, hi = K;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (j >= s_b[mid]) lo = mid;
        else hi = mid;
    }
    return lo;
}

// F = B (FP32 fluid), H = H_old = 0, |B|_1, and T_k = max |B_i| over Omega_k.
__global__ void __launch_bounds__(kPThreads) k_pinit(const SolveDesc *__restrict__ desc, SolveState *__restrict__ st,
                                                     PartState *__restrict__ ps, const uint8_t *__restrict__ part_of,
                                                     double *__restrict__ H_old, int64_t n,
                                                     double *__restrict__ part_sum) {
    __shared__ unsigned long long s_m[kMaxParts];
    const int K = ps->K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) s_m[k] = 0ull;
    __syncthreads();
    const double *__restrict__ B = desc->B;
    double *__restrict__ H = desc->H;
    float *__restrict__ F = static_cast<float *>(desc->F);
    const int64_t span = cta_span(n), lo = (int64_t)blockIdx.x * span;
    const int64_t hi = lo + span < n ? lo + span : n;
    double sum = 0.0, mx = 0.0;
    int cur = -1;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kPThreads) {
        const int k = part_of[i];
        if (k != cur) {
            if (cur >= 0 && mx > 0.0) atomicMax(&s_m[cur], double_to_bits(mx));
            cur = k;
            mx = 0.0;
        }
        const double b = B[i];
        F[i] = static_cast<float>(b);
        H[i] = 0.0;
        H_old[i] = 0.0;
        sum += fabs(b);
        mx = fmax(mx, fabs(b));
    }
    if (cur >= 0 && mx > 0.0) atomicMax(&s_m[cur], double_to_bits(mx));
    double dummy = 0.0;
    block_sum_max<kPThreads>(sum, dummy);
    if (threadIdx.x == 0) part_sum[blockIdx.x] = sum;
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x)
        if (s_m[k]) atomicMax(&ps->m[k], s_m[k]);
    if (!last_block(&ps->init_blocks)) return;
    double ts = 0.0;
    for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) ts += part_sum[i];
    block_sum_max<kPThreads>(ts, dummy);
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        ps->T[k] = bits_to_double(ps->m[k]);   // T_k = max |F_i| over Omega_k (0: the range idles)
        ps->m[k] = 0ull;
    }
    if (threadIdx.x == 0) {
        st->b_l1 = ts;
        st->f0_l1 = ts;
        st->r_exact = ts;
        if (!isfinite(ts)) st->done = 3;
        else if (ts <= desc->tol) st->done = 1;
    }
}

// Selection of every range against its own T_k, in two passes over the CTA's
// node span (count, one atomic for the CTA's slice of the frontier, write);
// per-range |F|_1, max and count.  The last CTA runs the control.
__global__ void __launch_bounds__(kPThreads) k_pscan(const SolveDesc *__restrict__ desc, SolveState *__restrict__ st,
                                                     PartState *__restrict__ ps, const uint8_t *__restrict__ part_of,
                                                     int32_t *__restrict__ front, int64_t n,
                                                     cudaGraphConditionalHandle h_while,
                                                     cudaGraphConditionalHandle h_rec, int ctl) {
    if (st->done) {                                     // converged, capped or not finite: end the loop
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->push_count = 0;
            ps->any_send = 0;
            if (ctl == 1) {
                cudaGraphSetConditional(h_rec, 0);
                cudaGraphSetConditional(h_while, 0);
            }
        }
        return;
    }
    __shared__ float s_T[kMaxParts];
    __shared__ float s_u[kMaxParts];   // 1/N completion: the range's pending uniform add
    __shared__ double s_r[kMaxParts];
    __shared__ unsigned s_m[kMaxParts], s_sel[kMaxParts];   // max |F| as float bits (non-negative floats order like integers)
    __shared__ int s_warp[kPThreads / 32];
    __shared__ int s_base;
    const int K = ps->K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        s_T[k] = __double2float_ru(ps->T[k]);   // |F_i| >= T in FP32: T rounded up to a float
        s_u[k] = static_cast<float>(ps->pend[k]);
        s_r[k] = 0.0;
        s_m[k] = 0u;
        s_sel[k] = 0u;
    }
    __syncthreads();
    // not __restrict__: with the 1/N completion pass 1 writes F and pass 2 reads it back
    float *F = static_cast<float *>(desc->F);
    const int64_t span = cta_span(n), lo = (int64_t)blockIdx.x * span;
    const int64_t hi = lo + span < n ? lo + span : n;
    // pass 1: sums and counts, per thread for its current range; a range
    // change flushes the thread's sums (rare: a CTA's span meets few range
    // bounds), the last flush is reduced over the warp first when all its
    // lanes end in the same range
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double r = 0.0;
    float mx = 0.f;
    unsigned nsel = 0;
    int cur = -1, mine = 0;
    auto flush = [&]() {
        if (cur < 0) return;
        if (r != 0.0) atomicAdd(&s_r[cur], r);
        if (mx > 0.f) atomicMax(&s_m[cur], __float_as_uint(mx));
        if (nsel) atomicAdd(&s_sel[cur], nsel);
        r = 0.0;
        mx = 0.f;
        nsel = 0;
    };
    for (int64_t i = lo + threadIdx.x; i < hi; i += kPThreads) {
        const int k = part_of[i];
        if (k != cur) {
            flush();
            cur = k;
        }
        float v = F[i];
        if (s_u[k] != 0.f) {   // the range's completed columns, added before the test
            v += s_u[k];
            F[i] = v;
        }
        const float a = fabsf(v);
        r += a;
        mx = fmaxf(mx, a);
        if (a >= s_T[k] && a > 0.f) {
            ++nsel;
            ++mine;
        }
    }
    {
        const int c0 = __shfl_sync(0xffffffffu, cur, 0);
        if (__all_sync(0xffffffffu, cur == c0)) {
            r = warp_sum(r);
            mx = warp_max(mx);
            nsel = warp_sum(nsel);
            if (lane != 0) cur = -1;   // lane 0 flushes the warp's sums
        }
        flush();
    }
    // exclusive prefix of the per-thread counts, one atomic for the CTA's slice
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < kPThreads / 32; ++w) {
            const int v = s_warp[w];
            s_warp[w] = run;
            run += v;
        }
        s_base = run ? atomicAdd(&st->nfront, run) : 0;
    }
    __syncthreads();
    // pass 2: the same reads (from L2), write the selected ids
    int pos = s_base + s_warp[warp] + incl - mine;
    if (mine)
        for (int64_t i = lo + threadIdx.x; i < hi; i += kPThreads) {
            const float a = fabsf(F[i]);
            if (a >= s_T[part_of[i]] && a > 0.f) front[pos++] = static_cast<int32_t>(i);
        }
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        if (s_r[k] != 0.0) atomicAdd(&ps->r[k], s_r[k]);
        if (s_m[k]) atomicMax(&ps->m[k], double_to_bits(static_cast<double>(__uint_as_float(s_m[k]))));
        if (s_sel[k]) atomicAdd(&ps->sel[k], (unsigned long long)s_sel[k]);
    }
    if (!last_block(&ps->scan_blocks)) return;

    // control of every range (one thread each), then of the solve
    __shared__ double s_tot[kMaxParts];
    __shared__ int s_snd[kMaxParts];
    __shared__ int s_stop;
    const double alpha = desc->alpha;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const double rk = ps->r[k], mk = bits_to_double(ps->m[k]), sk = ps->s[k];
        double T = ps->T[k];
        if (ps->sel[k] > 0) {
            T /= alpha;                                 // the range swept at T: next level T / alpha
        } else if (mk > 0.0) {                          // empty sweep: first T / alpha^j <= max |F|
            for (int guard = 0; T > mk && guard < 8192; ++guard) T /= alpha;
            if (T > mk) T = mk;                         // alpha so close to 1 that the guard ran out
        }
        ps->T[k] = T;
        s_snd[k] = sk > 0.0 && sk > rk / (double)K;     // Eq. send
        ps->rdec[k] = rk;
        s_tot[k] = rk + sk;
        ps->r[k] = 0.0;
        ps->m[k] = 0ull;
        ps->sel[k] = 0ull;
        ps->pend[k] = 0.0;                              // added by every CTA of this selection
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double total = 0.0;
        int any = 0;
        for (int k = 0; k < K; ++k) {
            total += s_tot[k];
            any |= s_snd[k];
        }
        const double est = st->est_scale > 1.0 ? st->est_scale : 1.0;
        const double tol = desc->tol, drop = desc->recompute_drop;
        int done = 0, rec = 0, stop = 0, push = st->nfront;
        if (!isfinite(total)) {
            done = 3;
        } else if (total * est <= tol) {                // stop request: confirm on the exact residual
            rec = 1;
            stop = 1;
            st->confirming = 1;
            st->r_confirm = total * est;
            push = 0;
            any = 0;
        } else if (drop > 0.0 && total * est * drop <= st->r_exact) {
            rec = 1;                                     // refinement of the FP32 fluid
        }
        if (push > 0) st->level += 1;
        st->body_iters += 1;
        if (!done && st->body_iters >= desc->max_body_iters) done = 2;
        if (!done && st->level >= desc->max_levels && !rec) done = 2;
        if (done) {
            rec = 0;
            push = 0;
            any = 0;
            st->done = done;
        }
        st->push_count = push;
        st->do_recompute = rec;
        st->nfront = 0;
        st->tile_ctr = 0;
        ps->any_send = any;
        s_stop = stop || done;
        if (ctl == 1) {   // in a CUDA graph; host-driven rounds read st instead
            cudaGraphSetConditional(h_rec, rec ? 1u : 0u);
            if (done) cudaGraphSetConditional(h_while, 0);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) ps->send[k] = s_stop ? 0 : s_snd[k];
}

__device__ __forceinline__ int32_t push_target(const int32_t *__restrict__ pcol, const int32_t *__restrict__ hot_node,
                                               int64_t e) {
    const int32_t c = pcol[e];
    return c >= 0 ? c : hot_node[-1 - c];
}

// Drain of the frontier, one lane per node; a lane's row goes to its local
// children, and rows longer than 32 edges are walked by the whole warp.
// The fluid owed to other ranges, |w| per external child, accumulates in s_k.
__global__ void __launch_bounds__(kPThreads) k_ppush(const SolveDesc *__restrict__ desc, SolveState *__restrict__ st,
                                                     PartState *__restrict__ ps, const uint8_t *__restrict__ part_of,
                                                     const int64_t *__restrict__ bounds,
                                                     const int32_t *__restrict__ front, const int32_t *__restrict__ rp,
                                                     const int32_t *__restrict__ pcol,
                                                     const int32_t *__restrict__ hot_node, int n_hot,
                                                     const float *__restrict__ scale) {
    const int count = st->push_count;
    if (count == 0) return;
    // per range: fluid owed (FP32 in the CTA, FP64 across CTAs) and diffusions
    __shared__ float s_s[kMaxParts];
    __shared__ unsigned s_ops[kMaxParts];
    __shared__ int64_t s_b[kMaxParts + 1];
    __shared__ float s_dang[kMaxParts];     // 1/N completion: fluid drained from the range's dangling nodes
    __shared__ unsigned s_dcnt[kMaxParts];  // ... and their number
    // targets of very high in-degree (hot slots, encoded -1 - slot in pcol)
    // are accumulated per CTA in shared memory and flushed once, as in the
    // main push: hot-node ranges, then the sums
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *s_hot = reinterpret_cast<float *>(smem_raw);
    uint8_t *s_hot_part = reinterpret_cast<uint8_t *>(s_hot + n_hot);
    const int K = ps->K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        s_s[k] = 0.f;
        s_ops[k] = 0u;
        s_dang[k] = 0.f;
        s_dcnt[k] = 0u;
    }
    for (int k = threadIdx.x; k <= K; k += blockDim.x) s_b[k] = bounds[k];
    const bool dangling = desc->dangling != 0;
    const double dN = desc->d / (double)desc->n_nodes;
    for (int sl = threadIdx.x; sl < n_hot; sl += blockDim.x) {
        s_hot[sl] = 0.f;
        s_hot_part[sl] = part_of[hot_node[sl]];
    }
    __syncthreads();
    float *__restrict__ F = static_cast<float *>(desc->F);
    double *__restrict__ H = desc->H;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long my_nodes = 0, my_edges = 0;
    // one target of a row of range k (children [lo, hi)): inside the range it
    // is diffused (hot targets in their shared-memory slot), outside it only
    // counts towards the fluid owed
    auto push1 = [&](int32_t c, float w, int k, int64_t lo, int64_t hi, unsigned &loc, unsigned &ext) {
        if (c < 0) {
            if (s_hot_part[-1 - c] == k) {
                atomicAdd(&s_hot[-1 - c], w);
                ++loc;
            } else {
                ++ext;
            }
        } else if (c >= lo && c < hi) {
            red_add(F + c, w);
            ++loc;
        } else {
            ++ext;
        }
    };
    for (int64_t base = warp * 32; base < count; base += nwarps * 32) {
        const int64_t idx = base + lane;
        int32_t b = 0, e = 0;
        int k = 0;
        float w = 0.f, w_dang = 0.f;
        if (idx < count) {
            const int32_t i = front[idx];
            k = part_of[i];
            b = rp[i];
            e = rp[i + 1];
            const float f = atomicExch(F + i, 0.f);
            H[i] += static_cast<double>(f);
            w = f * scale[i];
            w_dang = f;
            my_nodes += 1;
        }
        const int deg = e - b;
        unsigned loc = 0, ext = 0;
        // a drained dangling node with the 1/N completion: its column's part in
        // the range is a pending uniform add, the rest (N - n_k rows of d/N) is owed
        float dl = idx < count && deg == 0 && dangling ? w_dang : 0.f;
        unsigned dc = dl != 0.f ? 1u : 0u;
        if (deg <= kPThreadRow) {
            // the row by its thread, 8 column loads in flight
            const int64_t lo = s_b[k], hi = s_b[k + 1];
            for (int32_t q0 = b; q0 < e; q0 += 8) {
                int32_t c[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) c[t] = q0 + t < e ? __ldcs(pcol + q0 + t) : 0;
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if (q0 + t < e) push1(c[t], w, k, lo, hi, loc, ext);
            }
        }
        {
            // the thread rows' counts (all lanes; zero for the others), reduced
            // over the warp first when its lanes share a range
            float owed = fabsf(w) * static_cast<float>(ext);
            if (dl != 0.f) owed += fabsf(dl) * static_cast<float>(dN * (double)(desc->n_nodes - (s_b[k + 1] - s_b[k])));
            int kk = k;
            const int k0 = __shfl_sync(0xffffffffu, k, 0);
            if (__all_sync(0xffffffffu, k == k0)) {
                loc = warp_sum(loc);
                owed = warp_sum(owed);
                dl = warp_sum(dl);
                dc = warp_sum(dc);
                if (lane != 0) kk = -1;
            }
            if (kk >= 0) {
                if (loc) atomicAdd(&s_ops[kk], loc);
                if (owed != 0.f) atomicAdd(&s_s[kk], owed);
                if (dc) {
                    atomicAdd(&s_dang[kk], dl);
                    atomicAdd(&s_dcnt[kk], dc);
                }
                my_edges += loc;
            }
        }
        unsigned big = __ballot_sync(0xffffffffu, deg > kPThreadRow);
        while (big) {
            // a longer row by the whole warp, 4 column loads in flight per lane
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int32_t mb = __shfl_sync(0xffffffffu, b, src), me = __shfl_sync(0xffffffffu, e, src);
            const float mw = __shfl_sync(0xffffffffu, w, src);
            const int mk = __shfl_sync(0xffffffffu, k, src);
            const int64_t lo = s_b[mk], hi = s_b[mk + 1];
            unsigned loc = 0, ext = 0;
            for (int32_t q0 = mb + lane; q0 < me; q0 += 4 * 32) {
                int32_t c[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) c[t] = q0 + 32 * t < me ? __ldcs(pcol + q0 + 32 * t) : 0;
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (q0 + 32 * t < me) push1(c[t], mw, mk, lo, hi, loc, ext);
            }
            loc = warp_sum(loc);
            ext = warp_sum(ext);
            if (lane == 0) {
                if (loc) atomicAdd(&s_ops[mk], loc);
                if (ext) atomicAdd(&s_s[mk], fabsf(mw) * static_cast<float>(ext));
                my_edges += loc;
            }
        }
    }
    my_nodes = warp_sum(my_nodes);
    my_edges = warp_sum(my_edges);
    if (lane == 0 && my_nodes) {
        atomicAdd(&st->node_diff, my_nodes);
        atomicAdd(&st->edge_diff, my_edges);
    }
    __syncthreads();
    for (int sl = threadIdx.x; sl < n_hot; sl += blockDim.x) {
        const float v = s_hot[sl];
        if (v != 0.f) red_add(F + hot_node[sl], v);
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        unsigned long long ops = s_ops[k];
        if (s_dcnt[k]) {   // completed columns: n_k local rows, a pending uniform add
            atomicAdd(&ps->pend[k], dN * static_cast<double>(s_dang[k]));
            ops += (unsigned long long)s_dcnt[k] * (unsigned long long)(s_b[k + 1] - s_b[k]);
        }
        if (s_s[k] != 0.f) atomicAdd(&ps->s[k], static_cast<double>(s_s[k]));
        if (ops) atomicAdd(&ps->ops[k], ops);
    }
}

// Transmission of the ranges with send[k]: for every node i of such a range,
// F_j += (d / outdeg_i)(H_i - H_old_i) for its children j outside the range,
// and H_old_i = H_i.  The last CTA rescales the receivers' thresholds.
__global__ void __launch_bounds__(kPThreads) k_psend(const SolveDesc *__restrict__ desc, SolveState *__restrict__ st,
                                                     PartState *__restrict__ ps, const uint8_t *__restrict__ part_of,
                                                     const int64_t *__restrict__ bounds,
                                                     const int32_t *__restrict__ rp, const int32_t *__restrict__ pcol,
                                                     const int32_t *__restrict__ hot_node,
                                                     const double *__restrict__ scale64, double *__restrict__ H_old,
                                                     int64_t n) {
    if (!ps->any_send) return;
    __shared__ int s_send[kMaxParts];
    __shared__ float s_recv[kMaxParts];       // received per range (FP32 in the CTA, FP64 across CTAs)
    __shared__ unsigned s_ops[kMaxParts];
    __shared__ int64_t s_b[kMaxParts + 1];
    __shared__ double s_dh[kMaxParts];        // 1/N completion: H - H_old over the range's dangling nodes
    __shared__ unsigned s_dcnt[kMaxParts];
    const int K = ps->K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        s_send[k] = ps->send[k];
        s_recv[k] = 0.f;
        s_ops[k] = 0u;
        s_dh[k] = 0.0;
        s_dcnt[k] = 0u;
    }
    const bool dangling = desc->dangling != 0;
    for (int k = threadIdx.x; k <= K; k += blockDim.x) s_b[k] = bounds[k];
    __syncthreads();
    float *__restrict__ F = static_cast<float *>(desc->F);
    const double *__restrict__ H = desc->H;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long my_edges = 0;
    // one child j of a transmitting row of range k: sent if outside the range;
    // the amount a receiving range gets is summed in registers over runs of
    // children in the same range (rkj, racc) and added to shared memory per run
    int rkj = -1;
    float racc = 0.f;
    auto flush_recv = [&]() {
        if (rkj >= 0) atomicAdd(&s_recv[rkj], racc);
        rkj = -1;
        racc = 0.f;
    };
    auto send1 = [&](int32_t j, float w, int64_t lo, int64_t hi, unsigned &sent) {
        if (j >= lo && j < hi) return;
        red_add(F + j, w);
        const int kj = range_of(s_b, K, j);
        if (kj != rkj) {
            flush_recv();
            rkj = kj;
        }
        racc += fabsf(w);
        ++sent;
    };
    for (int64_t base = warp * 32; base < n; base += nwarps * 32) {
        const int64_t i = base + lane;
        int32_t b = 0, e = 0;
        int k = 0;
        float w = 0.f;
        double ddh = 0.0;   // a dangling node's H - H_old (1/N completion)
        if (i < n) {
            k = part_of[i];
            if (s_send[k]) {
                const double h = H[i], dh = h - H_old[i];
                H_old[i] = h;
                if (dh != 0.0) {
                    w = static_cast<float>(scale64[i] * dh);
                    b = rp[i];
                    e = rp[i + 1];
                    if (b == e && dangling) ddh = dh;
                }
            }
        }
        if (dangling && __any_sync(0xffffffffu, ddh != 0.0)) {
            // the completed columns' owed rows: summed per range over the warp
            // when its lanes share one (their rows go to every node outside it)
            unsigned dc = ddh != 0.0 ? 1u : 0u;
            int kk = k;
            const int k0 = __shfl_sync(0xffffffffu, k, 0);
            if (__all_sync(0xffffffffu, k == k0)) {
                ddh = warp_sum(ddh);
                dc = warp_sum(dc);
                if (lane != 0) kk = -1;
            }
            if (kk >= 0 && dc) {
                atomicAdd(&s_dh[kk], ddh);
                atomicAdd(&s_dcnt[kk], dc);
            }
        }
        const int deg = e - b;
        if (deg <= kPThreadRow) {
            const int64_t lo = s_b[k], hi = s_b[k + 1];
            unsigned sent = 0;
            for (int32_t q0 = b; q0 < e; q0 += 8) {
                int32_t c[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) c[t] = q0 + t < e ? push_target(pcol, hot_node, q0 + t) : 0;
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if (q0 + t < e) send1(c[t], w, lo, hi, sent);
            }
            if (sent) atomicAdd(&s_ops[k], sent);
            my_edges += sent;
        }
        unsigned big = __ballot_sync(0xffffffffu, deg > kPThreadRow);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int32_t mb = __shfl_sync(0xffffffffu, b, src), me = __shfl_sync(0xffffffffu, e, src);
            const float mw = __shfl_sync(0xffffffffu, w, src);
            const int mk = __shfl_sync(0xffffffffu, k, src);
            const int64_t lo = s_b[mk], hi = s_b[mk + 1];
            unsigned sent = 0;
            for (int32_t q0 = mb + lane; q0 < me; q0 += 4 * 32) {
                int32_t c[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) c[t] = q0 + 32 * t < me ? push_target(pcol, hot_node, q0 + 32 * t) : 0;
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (q0 + 32 * t < me) send1(c[t], mw, lo, hi, sent);
            }
            sent = warp_sum(sent);
            if (lane == 0 && sent) {
                atomicAdd(&s_ops[mk], sent);
                my_edges += sent;
            }
        }
    }
    flush_recv();
    my_edges = warp_sum(my_edges);
    if (lane == 0 && my_edges) atomicAdd(&st->edge_diff, my_edges);
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        if (s_recv[k] != 0.f) atomicAdd(&ps->recv[k], static_cast<double>(s_recv[k]));
        unsigned long long ops = s_ops[k];
        if (s_dcnt[k]) {   // N - n_k transmitted rows per completed column
            atomicAdd(&ps->dsend[k], s_dh[k]);
            ops += (unsigned long long)s_dcnt[k] * (unsigned long long)(n - (s_b[k + 1] - s_b[k]));
        }
        if (ops) atomicAdd(&ps->ops[k], ops);
    }
    if (!last_block(&ps->send_blocks)) return;
    if (dangling) {
        // the completed columns' transmissions land on every node outside the
        // sender's range: a pending uniform add per receiving range
        if (threadIdx.x == 0) {
            const double dN = desc->d / (double)n;
            for (int k = 0; k < K; ++k) {
                const double q = dN * ps->dsend[k];
                if (q == 0.0) continue;
                for (int k2 = 0; k2 < K; ++k2) {
                    if (k2 == k) continue;
                    ps->pend[k2] += q;
                    ps->recv[k2] += fabs(q) * (double)(s_b[k2 + 1] - s_b[k2]);
                }
                ps->dsend[k] = 0.0;
            }
        }
        __syncthreads();
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        if (ps->send[k]) {
            ps->sends[k] += 1;
            ps->s[k] = 0.0;
            ps->send[k] = 0;
        }
        const double rv = ps->recv[k];
        if (rv > 0.0) {
            // Sec. 2.6: scale T_k by (r_k + received) / r_k; a range that held
            // no fluid takes T_k = received (the next selection's empty-sweep
            // rule lowers a T above every |F_i| to the first T / alpha^j below
            // the max)
            const double rd = ps->rdec[k];
            ps->T[k] = rd > 0.0 ? ps->T[k] * (rd + rv) / rd : rv;
            ps->recv[k] = 0.0;
        }
    }
    if (threadIdx.x == 0) ps->any_send = 0;
}

// Before an exact residual: it will hold every fluid still owed, so H_old = H
// and the owed amounts are cleared.
__global__ void __launch_bounds__(kPThreads) k_phold(const SolveDesc *__restrict__ desc,
                                                     const SolveState *__restrict__ st, PartState *__restrict__ ps,
                                                     double *__restrict__ H_old, int64_t n) {
    if (!st->do_recompute) return;
    const double *__restrict__ H = desc->H;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) H_old[i] = H[i];
    if (blockIdx.x == 0)
        for (int k = threadIdx.x; k < ps->K; k += blockDim.x) {
            ps->s[k] = 0.0;
            ps->pend[k] = 0.0;   // the exact residual holds the pending completed parts as well
            ps->dsend[k] = 0.0;
        }
}

// Range boundaries (host): uniform w_k = floor(k N / K), or the first node at
// which the out-edge prefix sum reaches k L / K (cost balanced).
std::vector<int64_t> partition_bounds(const std::vector<int32_t> &rp, int64_t n, int K, int kind) {
    std::vector<int64_t> b(K + 1, 0);
    const int64_t L = rp[n];
    for (int k = 1; k < K; ++k) {
        if (kind == 0) {
            b[k] = (int64_t)k * n / K;
        } else {
            const double target = (double)k * (double)L / (double)K;
            int64_t lo = b[k - 1], hi = n;                  // first j >= b[k-1] with rp[j] >= target
            while (lo < hi) {
                const int64_t mid = (lo + hi) / 2;
                if ((double)rp[mid] >= target) hi = mid; else lo = mid + 1;
            }
            b[k] = lo;
        }
    }
    b[K] = n;
    return b;
}

}  // namespace

// What di_solve_partitioned keeps on a graph between calls.
struct KpidCache {
    int K = -1, kind = -1;            // ranges loaded in part_of / bounds
    int grid = 0, res_form = -1;      // the round graph was built for these
    std::vector<int64_t> bounds_h;
    uint8_t *part_of = nullptr;       // [n] range of every node
    int64_t *bounds = nullptr;        // [kMaxParts + 1] range bounds
    double *H_old = nullptr;          // [n] history at the last transmission
    PartState *ps = nullptr, *ps_h = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

void free_kpid_cache(di_graph *g) {
    KpidCache *kc = g->kpid;
    if (!kc) return;
    if (kc->exec) cudaGraphExecDestroy(kc->exec);
    if (kc->graph) cudaGraphDestroy(kc->graph);
    if (kc->part_of) cudaFree(kc->part_of);
    if (kc->bounds) cudaFree(kc->bounds);
    if (kc->H_old) cudaFree(kc->H_old);
    if (kc->ps) cudaFree(kc->ps);
    if (kc->ps_h) cudaFreeHost(kc->ps_h);
    delete kc;
    g->kpid = nullptr;
}

}  // namespace di

using namespace di;

extern "C" DI_API di_status di_solve_partitioned(di_graph *g, const double *B, double d, double tol, double *H,
                                                double *F, const di_opts *opts, int32_t K, int32_t kind,
                                                int64_t *pid_ops, int64_t *pid_sends, di_stats *stats) {
    di::NvtxRange nvtx_range("di_solve_partitioned");
    clear_error();
    if (!g || !B || !H) { set_error("di_solve_partitioned: NULL graph, B or H"); return DI_EINVAL; }
    di_opts o;
    if (opts) o = *opts; else di_opts_default(&o);
    if (!(d > 0.0 && d < 1.0)) { set_error("di_solve_partitioned: d = %g outside (0, 1)", d); return DI_EINVAL; }
    if (!(tol > 0.0) || !std::isfinite(tol)) { set_error("di_solve_partitioned: tol = %g must be finite and > 0", tol); return DI_EINVAL; }
    if (!(o.alpha > 1.0) || !std::isfinite(o.alpha)) { set_error("di_solve_partitioned: alpha = %g must be > 1", o.alpha); return DI_EINVAL; }
    if (K < 1 || K > kMaxParts) { set_error("di_solve_partitioned: K = %d outside [1, %d]", K, kMaxParts); return DI_EINVAL; }
    if (kind < 0 || kind > 1) { set_error("di_solve_partitioned: kind = %d outside [0, 1]", kind); return DI_EINVAL; }
    if (o.fluid_fp64 || o.warm_start || o.dangling < 0 || o.dangling > 1 || o.selection || o.max_levels < 0 ||
        !(o.recompute_drop == 0.0 || (o.recompute_drop > 1.0 && std::isfinite(o.recompute_drop)))) {
        set_error("di_solve_partitioned: supports FP32 fluid from a cold start with the plain selection and "
                  "dangling 0 or 1; recompute_drop must be 0 or > 1");
        return DI_EINVAL;
    }
    if (g->n > (int64_t)INT32_MAX) { set_error("di_solve_partitioned: too many nodes"); return DI_EINVAL; }
    cudaStream_t s = as_stream(o.stream);
    DI_CUDA_TRY(cudaSetDevice(g->device));
    DI_TRY(ensure_workspace(g));
    DI_TRY(ensure_scale(g, d, s));
    g->res_form = 0;
    DI_TRY(ensure_blocked_order(g, s));
    Workspace &ws = g->ws;
    const int64_t n = g->n;
    if (!ws.F32) {
        const int64_t npad = (n + 3) / 4 * 4;
        DI_CUDA_TRY(cudaMalloc(&ws.F32, npad * sizeof(float)));
        DI_CUDA_TRY(cudaMemsetAsync(ws.F32, 0, npad * sizeof(float), s));
    }

    // ranges, node -> range table and round graph: kept on the graph object
    // and reused while K, the partition kind, the grid and the residual form
    // are unchanged (the buffers do not depend on K, so a new K only reloads
    // the tables)
    if (!g->kpid) g->kpid = new KpidCache();
    KpidCache &kc = *g->kpid;
    if (!kc.part_of) {
        DI_CUDA_TRY(cudaMalloc(&kc.part_of, n > 0 ? n : 1));
        DI_CUDA_TRY(cudaMalloc(&kc.bounds, (kMaxParts + 1) * sizeof(int64_t)));
        DI_CUDA_TRY(cudaMalloc(&kc.H_old, (n > 0 ? n : 1) * sizeof(double)));
        DI_CUDA_TRY(cudaMalloc(&kc.ps, sizeof(PartState)));
        DI_CUDA_TRY(cudaMallocHost(&kc.ps_h, sizeof(PartState)));
    }
    if (kc.K != K || kc.kind != kind) {
        std::vector<int32_t> rp(n + 1);
        DI_CUDA_TRY(cudaMemcpyAsync(rp.data(), g->rp, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        DI_CUDA_TRY(cudaStreamSynchronize(s));
        kc.bounds_h = partition_bounds(rp, n, K, kind);
        std::vector<uint8_t> part(n > 0 ? n : 1, 0);
        for (int k = 0; k < K; ++k)
            for (int64_t i = kc.bounds_h[k]; i < kc.bounds_h[k + 1]; ++i) part[i] = static_cast<uint8_t>(k);
        DI_CUDA_TRY(cudaMemcpy(kc.part_of, part.data(), part.size(), cudaMemcpyHostToDevice));
        DI_CUDA_TRY(cudaMemcpy(kc.bounds, kc.bounds_h.data(), (K + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
        kc.K = K;
        kc.kind = kind;
    }
    std::memset(kc.ps_h, 0, sizeof(PartState));
    kc.ps_h->K = K;
    DI_CUDA_TRY(cudaMemcpyAsync(kc.ps, kc.ps_h, sizeof(PartState), cudaMemcpyHostToDevice, s));

    // descriptor and state (the previous call on this graph has completed: every solve synchronises)
    SolveDesc &dh = *ws.desc_h;
    std::memset(&dh, 0, sizeof(dh));
    dh.B = B;
    dh.H = H;
    dh.F_out = F;
    dh.F = ws.F32;
    dh.d = d;
    dh.tol = tol;
    dh.alpha = o.alpha;
    dh.max_levels = o.max_levels;
    dh.recompute_drop = o.recompute_drop;
    dh.max_body_iters = (int)std::min<long long>(4LL * o.max_levels + 1000, INT32_MAX);
    dh.n_nodes = n;
    dh.dangling = o.dangling;
    DI_CUDA_TRY(cudaEventRecord(ws.ev0, s));
    DI_CUDA_TRY(cudaMemcpyAsync(ws.desc, ws.desc_h, sizeof(SolveDesc), cudaMemcpyHostToDevice, s));
    DI_CUDA_TRY(cudaMemsetAsync(ws.st, 0, sizeof(SolveState), s));

    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k_ppush, kPThreads,
                                                      (size_t)g->n_hot * (sizeof(float) + 1)) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    // k_pinit leaves one partial per CTA in part_sum, which holds as many as
    // the largest grid of the workspace
    const int64_t parts = std::max({g->grid_scan, g->grid_select, residual_partials(g), g->grid_push});
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>({(int64_t)per_sm * g->num_sms, (n + kPThreads - 1) / kPThreads, parts}));
    k_pinit<<<grid, kPThreads, 0, s>>>(ws.desc, ws.st, kc.ps, kc.part_of, kc.H_old, n, ws.part_sum);
    DI_CUDA_TRY(cudaGetLastError());

    const size_t hot_smem = (size_t)g->n_hot * (sizeof(float) + 1);
    double t_scan = 0.0, t_push = 0.0, t_send = 0.0, t_res = 0.0;
    int timed_rounds = 0;
    if (o.timing) {
        // host-driven rounds with a CUDA event around every kernel (profilers
        // see the kernels; the residual kernels return at once unless k_pscan
        // asked for a recompute)
        cudaEvent_t ev[5];
        for (auto &e : ev) e = nullptr;
        struct EventGuard {
            cudaEvent_t *e;
            ~EventGuard() {
                for (int q = 0; q < 5; ++q)
                    if (e[q]) cudaEventDestroy(e[q]);
            }
        } eg{ev};
        for (auto &e : ev) DI_CUDA_TRY(cudaEventCreate(&e));
        const cudaGraphConditionalHandle none = 0;
        for (;;) {
            DI_CUDA_TRY(cudaEventRecord(ev[0], s));
            k_pscan<<<grid, kPThreads, 0, s>>>(ws.desc, ws.st, kc.ps, kc.part_of, ws.front, n, none, none, 2);
            DI_CUDA_TRY(cudaEventRecord(ev[1], s));
            k_ppush<<<grid, kPThreads, hot_smem, s>>>(ws.desc, ws.st, kc.ps, kc.part_of, kc.bounds, ws.front, g->rp,
                                                      g->pcol, g->hot_node, g->n_hot, g->s32);
            DI_CUDA_TRY(cudaEventRecord(ev[2], s));
            k_psend<<<grid, kPThreads, 0, s>>>(ws.desc, ws.st, kc.ps, kc.part_of, kc.bounds, g->rp, g->pcol,
                                               g->hot_node, g->s64, kc.H_old, n);
            DI_CUDA_TRY(cudaEventRecord(ev[3], s));
            k_phold<<<grid, kPThreads, 0, s>>>(ws.desc, ws.st, kc.ps, kc.H_old, n);
            launch_residual(g, 0, RES_LEVEL, s);
            DI_CUDA_TRY(cudaEventRecord(ev[4], s));
            DI_CUDA_TRY(cudaGetLastError());
            DI_CUDA_TRY(cudaMemcpyAsync(ws.st_h, ws.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
            DI_CUDA_TRY(cudaStreamSynchronize(s));
            float t[4] = {0.f, 0.f, 0.f, 0.f};
            for (int q = 0; q < 4; ++q) DI_CUDA_TRY(cudaEventElapsedTime(&t[q], ev[q], ev[q + 1]));
            t_scan += 1e-3 * t[0];
            t_push += 1e-3 * t[1];
            t_send += 1e-3 * t[2];
            t_res += 1e-3 * t[3];
            ++timed_rounds;
            if (ws.st_h->done) break;
        }
    } else {
    // the rounds as a CUDA graph: WHILE [scan -> push -> send -> IF(hold -> exact residual)]
    if (!kc.exec || kc.grid != grid || kc.res_form != g->res_form) {
        if (kc.exec) cudaGraphExecDestroy(kc.exec);
        if (kc.graph) cudaGraphDestroy(kc.graph);
        kc.exec = nullptr;
        kc.graph = nullptr;
        struct StreamGuard {
            cudaStream_t cs = nullptr;
            ~StreamGuard() {
                if (cs) cudaStreamDestroy(cs);
            }
        } sg;
        DI_CUDA_TRY(cudaStreamCreateWithFlags(&sg.cs, cudaStreamNonBlocking));
        DI_CUDA_TRY(cudaGraphCreate(&kc.graph, 0));
        cudaGraphConditionalHandle h_while, h_if;
        DI_CUDA_TRY(cudaGraphConditionalHandleCreate(&h_while, kc.graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams wp = {};
        wp.type = cudaGraphNodeTypeConditional;
        wp.conditional.handle = h_while;
        wp.conditional.type = cudaGraphCondTypeWhile;
        wp.conditional.size = 1;
        cudaGraphNode_t wnode;
        DI_CUDA_TRY(cudaGraphAddNode(&wnode, kc.graph, nullptr, nullptr, 0, &wp));
        cudaGraph_t body = wp.conditional.phGraph_out[0];
        DI_CUDA_TRY(cudaGraphConditionalHandleCreate(&h_if, body, 0, 0));
        DI_CUDA_TRY(cudaStreamBeginCaptureToGraph(sg.cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        k_pscan<<<grid, kPThreads, 0, sg.cs>>>(ws.desc, ws.st, kc.ps, kc.part_of, ws.front, n, h_while, h_if, 1);
        k_ppush<<<grid, kPThreads, hot_smem, sg.cs>>>(ws.desc, ws.st, kc.ps, kc.part_of, kc.bounds, ws.front, g->rp,
                                                      g->pcol, g->hot_node, g->n_hot, g->s32);
        k_psend<<<grid, kPThreads, 0, sg.cs>>>(ws.desc, ws.st, kc.ps, kc.part_of, kc.bounds, g->rp, g->pcol,
                                               g->hot_node, g->s64, kc.H_old, n);
        cudaStreamCaptureStatus cst;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        cudaGraph_t capg = nullptr, ended = nullptr;
        DI_CUDA_TRY(cudaStreamGetCaptureInfo(sg.cs, &cst, nullptr, &capg, &deps, nullptr, &ndeps));
        cudaGraphNodeParams ip = {};
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = h_if;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        cudaGraphNode_t inode;
        DI_CUDA_TRY(cudaGraphAddNode(&inode, capg, deps, nullptr, ndeps, &ip));
        DI_CUDA_TRY(cudaStreamUpdateCaptureDependencies(sg.cs, &inode, nullptr, 1, cudaStreamSetCaptureDependencies));
        DI_CUDA_TRY(cudaStreamEndCapture(sg.cs, &ended));
        DI_CUDA_TRY(cudaStreamBeginCaptureToGraph(sg.cs, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal));
        k_phold<<<grid, kPThreads, 0, sg.cs>>>(ws.desc, ws.st, kc.ps, kc.H_old, n);
        launch_residual(g, 0, RES_LEVEL, sg.cs);
        DI_CUDA_TRY(cudaStreamEndCapture(sg.cs, &ended));
        DI_CUDA_TRY(cudaGetLastError());
        DI_CUDA_TRY(cudaGraphInstantiate(&kc.exec, kc.graph, 0));
        kc.grid = grid;
        kc.res_form = g->res_form;
    }
    DI_CUDA_TRY(cudaGraphLaunch(kc.exec, s));
    }
    DI_CUDA_TRY(cudaMemcpyAsync(ws.st_h, ws.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    DI_CUDA_TRY(cudaStreamSynchronize(s));
    // k_pinit; the three kernels of every round, and of the round that ends
    // the loop; the IF body's when a recompute ran
    long long launches = o.timing ? 1 + (4LL + residual_kernels(g)) * timed_rounds
                                  : 1 + 3LL * (ws.st_h->body_iters + 1) + (1LL + residual_kernels(g)) * ws.st_h->recomputes;
    SolveState st = *ws.st_h;
    const bool refresh = st.done != 1 || (F != nullptr && st.recomputes == 0);
    if (refresh) {
        launch_residual(g, 0, RES_FINAL, s);
        DI_CUDA_TRY(cudaGetLastError());
        launches += residual_kernels(g);
        DI_CUDA_TRY(cudaMemcpyAsync(ws.st_h, ws.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        DI_CUDA_TRY(cudaStreamSynchronize(s));
        st.r_exact = ws.st_h->r_exact;
    }
    DI_CUDA_TRY(cudaMemcpyAsync(kc.ps_h, kc.ps, sizeof(PartState), cudaMemcpyDeviceToHost, s));
    DI_CUDA_TRY(cudaEventRecord(ws.ev1, s));
    DI_CUDA_TRY(cudaEventSynchronize(ws.ev1));
    float ms = 0.f;
    DI_CUDA_TRY(cudaEventElapsedTime(&ms, ws.ev0, ws.ev1));
    for (int k = 0; k < K; ++k) {
        if (pid_ops) pid_ops[k] = (int64_t)kc.ps_h->ops[k];
        if (pid_sends) pid_sends[k] = (int64_t)kc.ps_h->sends[k];
    }
    di_status rc = DI_OK;
    if (st.done == 3 || !std::isfinite(st.r_exact)) {
        rc = DI_ENONFINITE;
        set_error("di_solve_partitioned: residual is not finite");
    } else if (st.done != 1) {
        rc = DI_ENOCONV;
        set_error("di_solve_partitioned: level cap %d reached with |F|_1 = %g > tol = %g", o.max_levels, st.r_exact, tol);
    }
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->levels = st.level;
        stats->recomputes = st.recomputes;
        stats->node_diffusions = (int64_t)st.node_diff;
        stats->edge_diffusions = (int64_t)st.edge_diff;
        stats->resid_l1 = st.r_exact;
        stats->err_bound = st.r_exact / (1.0 - d);
        stats->b_l1 = st.b_l1;
        stats->f0_l1 = st.f0_l1;
        stats->seconds = ms * 1e-3;
        stats->status = rc;
        stats->gpu_launches = launches;
        stats->body_iterations = st.body_iters;
        if (o.timing) {
            stats->select_seconds = t_scan;
            stats->level_seconds = t_scan + t_push + t_send;
            stats->recompute_seconds = t_res;
            stats->level_launches = timed_rounds;
            stats->recompute_launches = st.recomputes;
        }
    }
    return rc;
}
