// warmstart.cu - learned warm start H0 for the D-iteration.
//
// Any H0 is a valid start: the fluid F0 = B + P H0 - H0 (the invariant of
// Eqs. defF/defH) is drained by the same threshold levels, and the bound
// |X - H|_1 <= |F|_1 / (1 - d) still holds with signed fluid.  A small
// network predicts y_i = log(N x_i) from per-node structural features, so
// that H0_i = exp(y_i) / N starts the solve close to X.
//
//   k_feat_node / k_feat_hop<1,2> - features from degree aggregates over the
//       in-edges (row gathers on the transpose, FP32 arithmetic with
//       compensated sums): log in/out-degree, 1- and 2-hop mean and
//       max of neighbour log-degree, log(1 + N (Q u)_i), log(1 + N (Q^2 u)_i),
//       N B_i;
//   k_mlp_fwd  - the network 9 -> 64 -> 64 -> 1 (ReLU) on the tensor cores:
//       mma.sync m16n8k16 with BF16 operands and FP32 accumulation, one warp
//       per 16 nodes, the first layer's accumulators re-packed in registers as
//       the second layer's A operand; the last layer is a quad reduction.  It
//       writes y, or H0 = exp(y)/N, or (training) y and the activations;
//   k_mlp_bwd  - gradient of the mean squared error, FP32 on the CUDA cores
//       (the dW reductions run over the minibatch; 0.5 GFLOP per step);
//   k_adam     - Adam with bias correction on FP32 master weights.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <new>
#include <vector>

#include "di_internal.cuh"
#include "pull.cuh"

namespace di {
namespace {

constexpr int kNF = DI_MODEL_NFEAT;       // 9 raw features
constexpr int kK1 = 16;                   // first-layer width (features zero-padded)
constexpr int kHid = 64;
constexpr int kNP = DI_MODEL_NPARAM;      // 5313 parameters
constexpr int kOffW1 = 0, kOffB1 = kHid * kK1, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid,
              kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid;
static_assert(kOffB3 + 1 == kNP, "parameter layout");
constexpr int kFwdThreads = 128;          // 4 warps x 16 nodes per tile
constexpr int kBwdThreads = 256;
constexpr int kBwdRows = 16;
constexpr int kFeatThreads = 256;

// ------------------------------------------------------------------ features

// Feature arithmetic is FP32: GB300 runs FP64 at a small fraction of the
// FP32 rate (an FP64 sum per in-edge kept its FP64 pipe 84% busy), and the
// features feed a BF16 network.  Sums over in-edges are compensated
// (Neumaier): the running sum carries its rounding errors in a second float,
// so the result is within about 2 units in the last place of the exact sum
// of the (non-negative) terms whatever the row length.
struct CSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x;
        c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
        s = t;
    }
    __device__ __forceinline__ void add(const CSum &o) {
        add(o.s);
        c += o.c;
    }
    __device__ __forceinline__ float value() const { return s + c; }
};

__device__ __forceinline__ CSum warp_csum(CSum v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        CSum w;
        w.s = __shfl_xor_sync(0xffffffffu, v.s, o);
        w.c = __shfl_xor_sync(0xffffffffu, v.c, o);
        v.add(w);
    }
    return v;
}
//
// Per-node temporaries, 16 bytes each, so that a gather over an in-edge
// j -> i reads one 32-byte sector: t1[j] = (x0_j, s_j, x1_j, x8_j) with
// x0 = log(1 + indeg), s = 1 / outdeg (0 for a dangling node), x1 =
// log(1 + outdeg), x8 = N B; t2[j] = (x2_j, x3_j, s_j a1_j, a1_j) from the
// first hop.  Only the second hop writes the 36-byte feature rows, each one
// whole: writing a few columns per pass made DRAM fill and write back the
// whole feature array on every pass.
__host__ __device__ __forceinline__ int64_t tmp_floats(int64_t n) { return 8 * n; }

__global__ void __launch_bounds__(kFeatThreads) k_feat_node(const int32_t *__restrict__ rp,
                                                            const int32_t *__restrict__ in_rp,
                                                            const double *__restrict__ B, int64_t n,
                                                            float4 *__restrict__ t1) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int indeg = in_rp[i + 1] - in_rp[i];
        const int outdeg = rp[i + 1] - rp[i];
        t1[i] = make_float4(log1pf((float)indeg), outdeg > 0 ? 1.0f / (float)outdeg : 0.0f, log1pf((float)outdeg),
                            (float)((double)n * B[i]));
    }
}

// Value of in-edge j -> i for each hop (all values are >= 0):
//   HOP 1: (ld_j, ld_j, s_j) summed, maximised, summed -> x2, x3, a1
//   HOP 2: (x2_j, x3_j, s_j a1_j)                      -> x4, x5, a2
template <int HOP>
struct FeatVal;
template <>
struct FeatVal<1> {
    float4 v;
    __device__ __forceinline__ void load(const float4 *__restrict__ t1, const float4 *__restrict__, int32_t j) {
        v = __ldg(t1 + j);
    }
    __device__ __forceinline__ void visit(CSum &u, float &m, CSum &w) const {
        u.add(v.x);
        m = fmaxf(m, v.x);
        w.add(v.y);
    }
};
template <>
struct FeatVal<2> {
    float4 v;
    __device__ __forceinline__ void load(const float4 *__restrict__, const float4 *__restrict__ t2, int32_t j) {
        v = __ldg(t2 + j);
    }
    __device__ __forceinline__ void visit(CSum &u, float &m, CSum &w) const {
        u.add(v.x);
        m = fmaxf(m, v.y);
        w.add(v.z);
    }
};

// In-edges [b, e) of one row in order, four gathers issued before they are
// accumulated (the sums keep the edge order).
template <int HOP>
__device__ __forceinline__ void feat_row(const int32_t *__restrict__ in_col, int32_t b, int32_t e,
                                         const float4 *__restrict__ t1, const float4 *__restrict__ t2, CSum &u,
                                         float &m, CSum &w) {
    int32_t q = b;
    for (; q + 4 <= e; q += 4) {
        FeatVal<HOP> x[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) x[k].load(t1, t2, __ldg(in_col + q + k));
#pragma unroll
        for (int k = 0; k < 4; ++k) x[k].visit(u, m, w);
    }
    for (; q < e; ++q) {
        FeatVal<HOP> x;
        x.load(t1, t2, __ldg(in_col + q));
        x.visit(u, m, w);
    }
}

// Outputs of node i from its in-row sums (u, w), max m and length len: the
// first hop fills t2[i], the second writes the node's whole feature row.
template <int HOP>
__device__ __forceinline__ void feat_emit(const float4 *__restrict__ t1, float4 *__restrict__ t2,
                                          float *__restrict__ feat, int64_t i, int len, float u, float m, float w) {
    const float mean = len > 0 ? u / (float)len : 0.0f;
    if (HOP == 1) {
        t2[i] = make_float4(mean, m, t1[i].y * w, w);
    } else {
        const float4 a = t1[i], b = t2[i];
        float *__restrict__ f = feat + i * kNF;
        f[0] = a.x;
        f[1] = a.z;
        f[2] = b.x;
        f[3] = b.y;
        f[4] = mean;
        f[5] = m;
        f[6] = log1pf(b.w);
        f[7] = log1pf(w);
        f[8] = a.w;
    }
}

// One hop over the in-edges of every node, one warp per 32 nodes: a row of
// at most 32 in-edges is reduced by its lane, one of up to kBin4Max by the
// whole warp.  Longer rows (a handful of hubs) are left to k_feat_seg /
// k_feat_long, which split them over CTAs.
template <int HOP>
__global__ void __launch_bounds__(kFeatThreads) k_feat_hop(const int32_t *__restrict__ in_rp,
                                                           const int32_t *__restrict__ in_col, int64_t n,
                                                           float *__restrict__ feat, float4 *__restrict__ t1,
                                                           float4 *__restrict__ t2) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * 32; base < n; base += nwarps * 32) {
        const int64_t i = base + lane;
        int32_t b = 0, e = 0;
        if (i < n) { b = in_rp[i]; e = in_rp[i + 1]; }
        const int len = e - b;
        CSum u, w;
        float m = 0.f;
        if (len <= 32) feat_row<HOP>(in_col, b, e, t1, t2, u, m, w);
        unsigned big = __ballot_sync(0xffffffffu, len > 32 && len <= kBin4Max);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int32_t mb = __shfl_sync(0xffffffffu, b, src), me = __shfl_sync(0xffffffffu, e, src);
            CSum pu, pw;
            float pm = 0.f;
            for (int32_t q = mb + lane; q < me; q += 32) {
                FeatVal<HOP> x;
                x.load(t1, t2, __ldg(in_col + q));
                x.visit(pu, pm, pw);
            }
            pu = warp_csum(pu);
            pm = warp_max(pm);
            pw = warp_csum(pw);
            if (lane == src) { u = pu; m = pm; w = pw; }
        }
        if (i < n && len <= kBin4Max) feat_emit<HOP>(t1, t2, feat, i, len, u.value(), m, w.value());
    }
}

// In-rows longer than kBin4Max: one CTA per kPullSeg-edge segment (the pull
// plan's bin 5) adds its partial sums and max into lacc[3 r .. 3 r + 2] of
// its long row r (max as the bits of a non-negative double).
template <int HOP>
__global__ void __launch_bounds__(kFeatThreads) k_feat_seg(const int32_t *__restrict__ seg_row,
                                                           const int32_t *__restrict__ seg_beg,
                                                           const int32_t *__restrict__ lseg0, int n_long,
                                                           int64_t nseg, const int32_t *__restrict__ in_rp,
                                                           const int32_t *__restrict__ in_col,
                                                           const float4 *__restrict__ t1,
                                                           const float4 *__restrict__ t2, double *__restrict__ lacc) {
    __shared__ CSum su[kFeatThreads / 32], sv[kFeatThreads / 32];
    __shared__ float sm[kFeatThreads / 32];
    for (int64_t sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
        const int32_t row = seg_row[sg];
        const int32_t b = seg_beg[sg];
        const int32_t end = in_rp[row + 1];
        const int32_t e = b + kPullSeg < end ? b + kPullSeg : end;
        CSum cu, cv;
        float cm = 0.f;
        for (int32_t q = b + threadIdx.x; q < e; q += kFeatThreads) {
            FeatVal<HOP> x;
            x.load(t1, t2, __ldg(in_col + q));
            x.visit(cu, cm, cv);
        }
        cu = warp_csum(cu);
        cm = warp_max(cm);
        cv = warp_csum(cv);
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        if (l == 0) { su[w] = cu; sm[w] = cm; sv[w] = cv; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 1; k < kFeatThreads / 32; ++k) { cu.add(su[k]); cm = fmaxf(cm, sm[k]); cv.add(sv[k]); }
            // one FP64 atomic per segment: the few hub rows add their segments exactly
            const double u = (double)cu.s + (double)cu.c, m = (double)cm, v = (double)cv.s + (double)cv.c;
            int lo = 0, hi = n_long;                 // long row r: lseg0[r] <= sg < lseg0[r + 1]
            while (hi - lo > 1) {
                const int mid = (lo + hi) / 2;
                if (lseg0[mid] <= sg) lo = mid; else hi = mid;
            }
            atomicAdd(&lacc[3 * lo], u);
            atomicMax(reinterpret_cast<unsigned long long *>(&lacc[3 * lo + 1]),
                      static_cast<unsigned long long>(__double_as_longlong(m)));
            atomicAdd(&lacc[3 * lo + 2], v);
        }
        __syncthreads();
    }
}

template <int HOP>
__global__ void k_feat_long(const int32_t *__restrict__ lrows, int n_long, const int32_t *__restrict__ in_rp,
                            const double *__restrict__ lacc, const float4 *__restrict__ t1,
                            float4 *__restrict__ t2, float *__restrict__ feat) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_long; r += gridDim.x * blockDim.x) {
        const int32_t i = lrows[r];
        feat_emit<HOP>(t1, t2, feat, i, in_rp[i + 1] - in_rp[i], (float)lacc[3 * r], (float)lacc[3 * r + 1],
                       (float)lacc[3 * r + 2]);
    }
}

// ------------------------------------------------------------------ network

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // .x (low half) = lo
    return *reinterpret_cast<uint32_t *>(&v);
}

// D += A B for one m16n8k16 tile: A 16x16 BF16 (row), B 16x8 BF16 (col), FP32.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

enum FwdMode : int { FWD_Y = 0, FWD_H0 = 1, FWD_TRAIN = 2 };

struct FwdArgs {
    const float *feat;        // [nodes][9] raw features
    const int32_t *idx;       // training: node of each row; else NULL (row = node)
    int64_t nrows;
    const float *theta;       // FP32 parameters (biases, w3, b3 used directly)
    const __nv_bfloat16 *wbf; // BF16 W1 [64][16] then W2 [64][64]
    const float *norm;        // mu[9], sd[9]
    float *y;                 // FWD_Y / FWD_TRAIN: prediction per row
    double *h0;               // FWD_H0: expf(y) / N per node
    double inv_n;
    // training
    const float *target;      // per node
    __nv_bfloat16 *xs;        // [rows][16]
    __nv_bfloat16 *h1;        // [rows][64]
    float *h2;                // [rows][64]
    double *loss_sum;
};

template <int MODE>
__global__ void __launch_bounds__(kFwdThreads) k_mlp_fwd(const FwdArgs a) {
    __shared__ __align__(16) __nv_bfloat16 sW1[kHid][kK1 + 8];    // row stride 48 B: conflict-free B loads
    __shared__ __align__(16) __nv_bfloat16 sW2[kHid][kHid + 8];   // row stride 144 B
    __shared__ float sb1[kHid], sb2[kHid], sw3[kHid], smu[kNF], ssd[kNF];
    __shared__ float sb3;
    for (int q = threadIdx.x; q < kHid * kK1; q += blockDim.x) sW1[q / kK1][q % kK1] = a.wbf[q];
    for (int q = threadIdx.x; q < kHid * kHid; q += blockDim.x) sW2[q / kHid][q % kHid] = a.wbf[kHid * kK1 + q];
    for (int q = threadIdx.x; q < kHid; q += blockDim.x) {
        sb1[q] = a.theta[kOffB1 + q];
        sb2[q] = a.theta[kOffB2 + q];
        sw3[q] = a.theta[kOffW3 + q];
    }
    if (threadIdx.x < kNF) {
        smu[threadIdx.x] = a.norm[threadIdx.x];
        ssd[threadIdx.x] = a.norm[kNF + threadIdx.x];
    }
    if (threadIdx.x == 0) sb3 = a.theta[kOffB3];
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tig = lane & 3;
    const int64_t ntiles = (a.nrows + 15) / 16;
    double my_loss = 0.0;
    for (int64_t tile = (int64_t)blockIdx.x * (kFwdThreads / 32) + warp; tile < ntiles;
         tile += (int64_t)gridDim.x * (kFwdThreads / 32)) {
        const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
        const bool v0 = r0 < a.nrows, v1 = r1 < a.nrows;
        int64_t n0 = r0, n1 = r1;
        if (MODE == FWD_TRAIN) {
            n0 = v0 ? a.idx[r0] : 0;
            n1 = v1 ? a.idx[r1] : 0;
        }
        // layer-1 A operand: standardised features, columns 2tig, 2tig+1, 2tig+8, 2tig+9
        auto feat_at = [&](bool v, int64_t node, int c) -> float {
            if (!v || c >= kNF) return 0.f;
            return (a.feat[node * kNF + c] - smu[c]) / ssd[c];
        };
        uint32_t A1[4];
        A1[0] = pack_bf16(feat_at(v0, n0, 2 * tig), feat_at(v0, n0, 2 * tig + 1));
        A1[1] = pack_bf16(feat_at(v1, n1, 2 * tig), feat_at(v1, n1, 2 * tig + 1));
        A1[2] = pack_bf16(feat_at(v0, n0, 2 * tig + 8), feat_at(v0, n0, 2 * tig + 9));
        A1[3] = pack_bf16(feat_at(v1, n1, 2 * tig + 8), feat_at(v1, n1, 2 * tig + 9));
        float acc1[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            acc1[nt][0] = acc1[nt][1] = acc1[nt][2] = acc1[nt][3] = 0.f;
            const uint32_t b0 = *reinterpret_cast<const uint32_t *>(&sW1[nt * 8 + g][2 * tig]);
            const uint32_t b1 = *reinterpret_cast<const uint32_t *>(&sW1[nt * 8 + g][8 + 2 * tig]);
            mma_bf16(acc1[nt], A1, b0, b1);
        }
        // bias + ReLU, rounded to BF16 in the layout of the layer-2 A operand
        uint32_t A2[4][4];
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int nt = 2 * ks + half;
                const int c = nt * 8 + 2 * tig;
                const float e0 = fmaxf(acc1[nt][0] + sb1[c], 0.f), e1 = fmaxf(acc1[nt][1] + sb1[c + 1], 0.f);
                const float e2 = fmaxf(acc1[nt][2] + sb1[c], 0.f), e3 = fmaxf(acc1[nt][3] + sb1[c + 1], 0.f);
                A2[ks][2 * half + 0] = pack_bf16(e0, e1);   // row g
                A2[ks][2 * half + 1] = pack_bf16(e2, e3);   // row g + 8
            }
        }
        float acc2[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) acc2[nt][0] = acc2[nt][1] = acc2[nt][2] = acc2[nt][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            const uint32_t A[4] = {A2[ks][0], A2[ks][1], A2[ks][2], A2[ks][3]};
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const uint32_t b0 = *reinterpret_cast<const uint32_t *>(&sW2[nt * 8 + g][ks * 16 + 2 * tig]);
                const uint32_t b1 = *reinterpret_cast<const uint32_t *>(&sW2[nt * 8 + g][ks * 16 + 8 + 2 * tig]);
                mma_bf16(acc2[nt], A, b0, b1);
            }
        }
        // layer 3 (FP32): y = w3 . relu(z2) + b3, reduced over the quad
        float p0 = 0.f, p1 = 0.f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int c = nt * 8 + 2 * tig;
            acc2[nt][0] = fmaxf(acc2[nt][0] + sb2[c], 0.f);
            acc2[nt][1] = fmaxf(acc2[nt][1] + sb2[c + 1], 0.f);
            acc2[nt][2] = fmaxf(acc2[nt][2] + sb2[c], 0.f);
            acc2[nt][3] = fmaxf(acc2[nt][3] + sb2[c + 1], 0.f);
            p0 += sw3[c] * acc2[nt][0] + sw3[c + 1] * acc2[nt][1];
            p1 += sw3[c] * acc2[nt][2] + sw3[c + 1] * acc2[nt][3];
        }
        p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
        p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
        p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
        p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
        const float y0 = p0 + sb3, y1 = p1 + sb3;
        if (MODE == FWD_H0) {
            // H0 is only a start (F0 is formed from it exactly), so the
            // exponential is taken in FP32: an FP64 exp per node would run on
            // GB300's narrow FP64 pipe
            if (tig == 0) {
                if (v0) a.h0[r0] = (double)expf(y0) * a.inv_n;
                if (v1) a.h0[r1] = (double)expf(y1) * a.inv_n;
            }
            continue;
        }
        if (tig == 0) {
            if (v0) a.y[r0] = y0;
            if (v1) a.y[r1] = y1;
        }
        if (MODE != FWD_TRAIN) continue;
        // activations for the backward pass (row = minibatch position)
        if (v0) {
            uint32_t *xs0 = reinterpret_cast<uint32_t *>(a.xs + r0 * kK1);
            xs0[tig] = A1[0];
            xs0[4 + tig] = A1[2];
            uint32_t *h10 = reinterpret_cast<uint32_t *>(a.h1 + r0 * kHid);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                h10[ks * 8 + tig] = A2[ks][0];
                h10[ks * 8 + 4 + tig] = A2[ks][2];
            }
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
                *reinterpret_cast<float2 *>(a.h2 + r0 * kHid + nt * 8 + 2 * tig) = make_float2(acc2[nt][0], acc2[nt][1]);
        }
        if (v1) {
            uint32_t *xs1 = reinterpret_cast<uint32_t *>(a.xs + r1 * kK1);
            xs1[tig] = A1[1];
            xs1[4 + tig] = A1[3];
            uint32_t *h11 = reinterpret_cast<uint32_t *>(a.h1 + r1 * kHid);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                h11[ks * 8 + tig] = A2[ks][1];
                h11[ks * 8 + 4 + tig] = A2[ks][3];
            }
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
                *reinterpret_cast<float2 *>(a.h2 + r1 * kHid + nt * 8 + 2 * tig) = make_float2(acc2[nt][2], acc2[nt][3]);
        }
        if (tig == 0) {
            if (v0) { const double e = (double)y0 - (double)a.target[n0]; my_loss += e * e; }
            if (v1) { const double e = (double)y1 - (double)a.target[n1]; my_loss += e * e; }
        }
    }
    if (MODE == FWD_TRAIN) {
        my_loss = warp_sum(my_loss);
        if (lane == 0 && my_loss != 0.0) atomicAdd(a.loss_sum, my_loss);
    }
}

struct BwdArgs {
    const int32_t *idx;       // node of each row (target lookup)
    int64_t nrows;
    float inv_m2;             // 2 / M
    const float *theta;
    const __nv_bfloat16 *wbf;
    const float *target;
    const float *y;
    const __nv_bfloat16 *xs, *h1;
    const float *h2;
    float *grad;              // [kNP], accumulated with atomics
};

// Gradient of (1/M) sum (y - t)^2 over 16-row tiles (FP32):
//   dy = 2 (y - t) / M;  dz2 = dy w3 [z2 > 0];  dh1 = W2^T dz2;  dz1 = dh1 [z1 > 0];
//   dW2 += dz2 h1^T, dW1 += dz1 x^T, biases and w3 likewise.
// Every thread keeps its share of the weight gradients in registers across
// the tiles it visits and adds them to grad once at the end.
__global__ void __launch_bounds__(kBwdThreads) k_mlp_bwd(const BwdArgs a) {
    __shared__ float sW2[kHid][kHid + 1];
    __shared__ float sw3[kHid];
    __shared__ float sh1[kBwdRows][kHid], sh2[kBwdRows][kHid], sdz2[kBwdRows][kHid], sdz1[kBwdRows][kHid];
    __shared__ float sx[kBwdRows][kK1], sdy[kBwdRows];
    const int t = threadIdx.x;
    for (int q = t; q < kHid * kHid; q += kBwdThreads)
        sW2[q / kHid][q % kHid] = __bfloat162float(a.wbf[kHid * kK1 + q]);
    for (int q = t; q < kHid; q += kBwdThreads) sw3[q] = a.theta[kOffW3 + q];
    __syncthreads();
    // register accumulators: dW2 (16 per thread), dW1 (4 per thread), vectors (threads < 64)
    const int j2 = t >> 2, k2 = (t & 3) * 16;      // dW2[j2][k2 .. k2+15]
    const int j1 = t >> 2, k1 = (t & 3) * 4;       // dW1[j1][k1 .. k1+3]
    float gW2[16], gW1[4];
#pragma unroll
    for (int q = 0; q < 16; ++q) gW2[q] = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) gW1[q] = 0.f;
    float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f;
    const int64_t ntiles = (a.nrows + kBwdRows - 1) / kBwdRows;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t row0 = tile * kBwdRows;
        if (t < kBwdRows) {
            const int64_t r = row0 + t;
            float dy = 0.f;
            if (r < a.nrows) dy = (a.y[r] - a.target[a.idx[r]]) * a.inv_m2;
            sdy[t] = dy;
        }
        for (int q = t; q < kBwdRows * kHid; q += kBwdThreads) {
            const int rr = q / kHid, c = q % kHid;
            const int64_t r = row0 + rr;
            const bool ok = r < a.nrows;
            sh1[rr][c] = ok ? __bfloat162float(a.h1[r * kHid + c]) : 0.f;
            sh2[rr][c] = ok ? a.h2[r * kHid + c] : 0.f;
        }
        for (int q = t; q < kBwdRows * kK1; q += kBwdThreads) {
            const int rr = q / kK1, c = q % kK1;
            const int64_t r = row0 + rr;
            sx[rr][c] = r < a.nrows ? __bfloat162float(a.xs[r * kK1 + c]) : 0.f;
        }
        __syncthreads();
        for (int q = t; q < kBwdRows * kHid; q += kBwdThreads) {
            const int rr = q / kHid, c = q % kHid;
            sdz2[rr][c] = sh2[rr][c] > 0.f ? sdy[rr] * sw3[c] : 0.f;
        }
        __syncthreads();
        {   // dh1 = W2^T dz2, dz1 = dh1 [h1 > 0]
            const int k = t & (kHid - 1), rg = t >> 6;
#pragma unroll
            for (int rr = rg; rr < kBwdRows; rr += kBwdThreads / kHid) {
                float s = 0.f;
#pragma unroll 8
                for (int j = 0; j < kHid; ++j) s += sdz2[rr][j] * sW2[j][k];
                sdz1[rr][k] = sh1[rr][k] > 0.f ? s : 0.f;
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < kBwdRows; ++rr) {
            const float d2 = sdz2[rr][j2];
#pragma unroll
            for (int q = 0; q < 16; ++q) gW2[q] += d2 * sh1[rr][k2 + q];
            const float d1 = sdz1[rr][j1];
#pragma unroll
            for (int q = 0; q < 4; ++q) gW1[q] += d1 * sx[rr][k1 + q];
        }
        if (t < kHid) {
            for (int rr = 0; rr < kBwdRows; ++rr) {
                gb2 += sdz2[rr][t];
                gb1 += sdz1[rr][t];
                gw3 += sdy[rr] * sh2[rr][t];
            }
        } else if (t == kHid) {
            for (int rr = 0; rr < kBwdRows; ++rr) gb3 += sdy[rr];
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) atomicAdd(&a.grad[kOffW2 + j2 * kHid + k2 + q], gW2[q]);
#pragma unroll
    for (int q = 0; q < 4; ++q) atomicAdd(&a.grad[kOffW1 + j1 * kK1 + k1 + q], gW1[q]);
    if (t < kHid) {
        atomicAdd(&a.grad[kOffB1 + t], gb1);
        atomicAdd(&a.grad[kOffB2 + t], gb2);
        atomicAdd(&a.grad[kOffW3 + t], gw3);
    } else if (t == kHid) {
        atomicAdd(&a.grad[kOffB3], gb3);
    }
}

// Adam: m = b1 m + (1 - b1) g; v = b2 v + (1 - b2) g^2;
// theta -= lr (m / bc1) / (sqrt(v / bc2) + eps), bc = 1 - beta^step.
// (1 - beta) comes from the host, formed in FP64: 1 - 0.999f in FP32 would
// be off by 1.3e-5 relative.
__global__ void k_adam(float *__restrict__ theta, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ grad, int np, float lr, float beta1, float beta2, float omb1,
                       float omb2, float eps, float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gr = grad[i];
    const float mi = beta1 * m[i] + omb1 * gr;
    const float vi = beta2 * v[i] + omb2 * gr * gr;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// BF16 copies of W1 and W2 (the tensor-core operands).
__global__ void k_pack_weights(const float *__restrict__ theta, __nv_bfloat16 *__restrict__ wbf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kHid * kK1) wbf[i] = __float2bfloat16_rn(theta[kOffW1 + i]);
    else if (i < kHid * kK1 + kHid * kHid) wbf[i] = __float2bfloat16_rn(theta[kOffW2 + i - kHid * kK1]);
}

// Training target log(N x_i).
__global__ void k_target(const double *__restrict__ X, int64_t n, float *__restrict__ y) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        y[i] = (float)log((double)n * fmax(X[i], 1e-300));
}

// Column sums and sums of squares of the features, and the target sum (FP64).
__global__ void __launch_bounds__(256) k_colstats(const float *__restrict__ feat, const float *__restrict__ y,
                                                  int64_t n, double *__restrict__ acc) {
    double s[kNF], q[kNF], ys = 0.0;
#pragma unroll
    for (int c = 0; c < kNF; ++c) s[c] = q[c] = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
#pragma unroll
        for (int c = 0; c < kNF; ++c) {
            const double v = feat[i * kNF + c];
            s[c] += v;
            q[c] += v * v;
        }
        ys += y[i];
    }
#pragma unroll
    for (int c = 0; c < kNF; ++c) {
        s[c] = warp_sum(s[c]);
        q[c] = warp_sum(q[c]);
    }
    ys = warp_sum(ys);
    if ((threadIdx.x & 31) == 0) {
        for (int c = 0; c < kNF; ++c) {
            atomicAdd(&acc[c], s[c]);
            atomicAdd(&acc[kNF + c], q[c]);
        }
        atomicAdd(&acc[2 * kNF], ys);
    }
}

// Minibatch rows drawn with replacement: node = SplitMix64(seed, counter) mod n_total.
__global__ void k_sample(int32_t *__restrict__ idx, int64_t m, uint64_t seed, uint64_t step, int64_t n_total) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    uint64_t z = seed + (step * (uint64_t)m + (uint64_t)r + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    idx[r] = (int32_t)(z % (uint64_t)n_total);
}

}  // namespace
}  // namespace di

using namespace di;

struct di_model {
    int device = 0;
    float norm_h[2 * kNF];          // mu, sd (host copy)
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *norm = nullptr;
    __nv_bfloat16 *wbf = nullptr;
    long long step = 0;
    double last_loss = 0.0;
    // scratch, grown on demand
    int64_t feat_cap = 0;
    float *feat = nullptr;
    float *ftmp = nullptr;
    int64_t row_cap = 0;
    int32_t *idx = nullptr;
    float *y = nullptr;
    __nv_bfloat16 *xs = nullptr, *h1 = nullptr;
    float *h2 = nullptr;
    double *dacc = nullptr;         // [2 * kNF + 2]
    int lacc_cap = 0;
    double *lacc = nullptr;         // [3 * long in-rows] partial sums of the features' long rows
};

namespace {

void free_model(di_model *m) {
    if (!m) return;
    void *p[] = {m->theta, m->m, m->v, m->grad, m->norm, m->wbf, m->feat, m->ftmp, m->idx, m->y,
                 m->xs, m->h1, m->h2, m->dacc, m->lacc};
    for (void *q : p)
        if (q) cudaFree(q);
    delete m;
}

di_status ensure_feat(di_model *m, int64_t n) {
    if (n <= m->feat_cap) return DI_OK;
    if (m->feat) cudaFree(m->feat);
    if (m->ftmp) cudaFree(m->ftmp);
    m->feat = nullptr;
    m->ftmp = nullptr;
    m->feat_cap = 0;
    DI_CUDA_TRY(cudaMalloc(&m->feat, (size_t)n * kNF * sizeof(float)));
    DI_CUDA_TRY(cudaMalloc(&m->ftmp, (size_t)tmp_floats(n) * sizeof(float)));
    m->feat_cap = n;
    return DI_OK;
}

di_status ensure_rows(di_model *m, int64_t rows) {
    if (rows <= m->row_cap) return DI_OK;
    void *old[] = {m->idx, m->y, m->xs, m->h1, m->h2};
    for (void *q : old)
        if (q) cudaFree(q);
    m->idx = nullptr; m->y = nullptr; m->xs = nullptr; m->h1 = nullptr; m->h2 = nullptr;
    m->row_cap = 0;
    DI_CUDA_TRY(cudaMalloc(&m->idx, (size_t)rows * sizeof(int32_t)));
    DI_CUDA_TRY(cudaMalloc(&m->y, (size_t)rows * sizeof(float)));
    DI_CUDA_TRY(cudaMalloc(&m->xs, (size_t)rows * kK1 * sizeof(__nv_bfloat16)));
    DI_CUDA_TRY(cudaMalloc(&m->h1, (size_t)rows * kHid * sizeof(__nv_bfloat16)));
    DI_CUDA_TRY(cudaMalloc(&m->h2, (size_t)rows * kHid * sizeof(float)));
    m->row_cap = rows;
    return DI_OK;
}

int grid_of(int64_t items, int per_block, int cap) {
    int64_t b = (items + per_block - 1) / per_block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

int sm_count(int dev) {
    int s = 0;
    cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
    return s > 0 ? s : 1;
}

// features of graph g into feat (device [n][9])
di_status features_into(di_model *m, di_graph *g, const double *B, float *feat, cudaStream_t s) {
    DI_TRY(ensure_feat(m, g->n));
    const int n_long = g->pl_nlrows;
    const int64_t nseg = g->pl_task_off[5] - g->pl_task_off[4];
    if (n_long > m->lacc_cap) {
        if (m->lacc) cudaFree(m->lacc);
        m->lacc = nullptr;
        m->lacc_cap = 0;
        DI_CUDA_TRY(cudaMalloc(&m->lacc, (size_t)3 * n_long * sizeof(double)));
        m->lacc_cap = n_long;
    }
    const int cap = g->num_sms * 8;
    float4 *t1 = reinterpret_cast<float4 *>(m->ftmp);
    float4 *t2 = reinterpret_cast<float4 *>(m->ftmp) + g->n;
    k_feat_node<<<grid_of(g->n, kFeatThreads, cap), kFeatThreads, 0, s>>>(g->rp, g->in_rp, B, g->n, t1);
    const int hop_grid = grid_of((g->n + 31) / 32, kFeatThreads / 32, cap);
    const int seg_grid = (int)std::max<int64_t>(1, std::min<int64_t>(nseg, cap));
    const int long_grid = grid_of(n_long, 128, cap);
    k_feat_hop<1><<<hop_grid, kFeatThreads, 0, s>>>(g->in_rp, g->in_col, g->n, feat, t1, t2);
    if (n_long > 0) {
        DI_CUDA_TRY(cudaMemsetAsync(m->lacc, 0, (size_t)3 * n_long * sizeof(double), s));
        k_feat_seg<1><<<seg_grid, kFeatThreads, 0, s>>>(g->pl_seg_row, g->pl_seg_beg, g->pl_lseg0, n_long, nseg,
                                                        g->in_rp, g->in_col, t1, t2, m->lacc);
        k_feat_long<1><<<long_grid, 128, 0, s>>>(g->pl_lrows, n_long, g->in_rp, m->lacc, t1, t2, feat);
    }
    k_feat_hop<2><<<hop_grid, kFeatThreads, 0, s>>>(g->in_rp, g->in_col, g->n, feat, t1, t2);
    if (n_long > 0) {
        DI_CUDA_TRY(cudaMemsetAsync(m->lacc, 0, (size_t)3 * n_long * sizeof(double), s));
        k_feat_seg<2><<<seg_grid, kFeatThreads, 0, s>>>(g->pl_seg_row, g->pl_seg_beg, g->pl_lseg0, n_long, nseg,
                                                        g->in_rp, g->in_col, t1, t2, m->lacc);
        k_feat_long<2><<<long_grid, 128, 0, s>>>(g->pl_lrows, n_long, g->in_rp, m->lacc, t1, t2, feat);
    }
    DI_CUDA_TRY(cudaGetLastError());
    return DI_OK;
}

FwdArgs fwd_args(const di_model *m) {
    FwdArgs a = {};
    a.theta = m->theta;
    a.wbf = m->wbf;
    a.norm = m->norm;
    return a;
}

int fwd_grid(int dev, int64_t rows) {
    return grid_of((rows + 15) / 16, kFwdThreads / 32, sm_count(dev) * 8);
}

// forward (training mode) + backward over `rows` rows into m->grad (zeroed here)
di_status grad_pass(di_model *m, const float *feat, const float *target, int64_t rows, double *loss_dev,
                    cudaStream_t s) {
    FwdArgs a = fwd_args(m);
    a.feat = feat;
    a.idx = m->idx;
    a.nrows = rows;
    a.y = m->y;
    a.target = target;
    a.xs = m->xs;
    a.h1 = m->h1;
    a.h2 = m->h2;
    a.loss_sum = loss_dev;
    k_mlp_fwd<FWD_TRAIN><<<fwd_grid(m->device, rows), kFwdThreads, 0, s>>>(a);
    DI_CUDA_TRY(cudaMemsetAsync(m->grad, 0, kNP * sizeof(float), s));
    BwdArgs b = {};
    b.idx = m->idx;
    b.nrows = rows;
    b.inv_m2 = (float)(2.0 / (double)rows);
    b.theta = m->theta;
    b.wbf = m->wbf;
    b.target = target;
    b.y = m->y;
    b.xs = m->xs;
    b.h1 = m->h1;
    b.h2 = m->h2;
    b.grad = m->grad;
    k_mlp_bwd<<<grid_of((rows + kBwdRows - 1) / kBwdRows, 1, sm_count(m->device) * 2), kBwdThreads, 0, s>>>(b);
    DI_CUDA_TRY(cudaGetLastError());
    return DI_OK;
}

void adam_launch(di_model *m, const di_train_opts &o, cudaStream_t s) {
    m->step += 1;
    const double bc1 = 1.0 - std::pow(o.beta1, (double)m->step);
    const double bc2 = 1.0 - std::pow(o.beta2, (double)m->step);
    k_adam<<<(kNP + 255) / 256, 256, 0, s>>>(m->theta, m->m, m->v, m->grad, kNP, (float)o.lr, (float)o.beta1,
                                             (float)o.beta2, (float)(1.0 - o.beta1), (float)(1.0 - o.beta2),
                                             (float)o.eps, (float)bc1, (float)bc2);
    k_pack_weights<<<(kHid * kK1 + kHid * kHid + 255) / 256, 256, 0, s>>>(m->theta, m->wbf);
}

// uniform He initialisation U(-sqrt(6/fan_in), sqrt(6/fan_in)) from SplitMix64
void init_params(std::vector<float> &th, uint64_t seed) {
    uint64_t x = seed;
    auto next = [&]() {
        uint64_t z = (x += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);   // [0, 1)
    };
    th.assign(kNP, 0.f);
    const double l1 = std::sqrt(6.0 / kNF), l2 = std::sqrt(6.0 / kHid);
    for (int j = 0; j < kHid; ++j)
        for (int k = 0; k < kNF; ++k) th[kOffW1 + j * kK1 + k] = (float)((2.0 * next() - 1.0) * l1);
    for (int q = 0; q < kHid * kHid; ++q) th[kOffW2 + q] = (float)((2.0 * next() - 1.0) * l2);
    for (int q = 0; q < kHid; ++q) th[kOffW3 + q] = (float)((2.0 * next() - 1.0) * l2);
}

di_status upload_state(di_model *m, const float *state_host) {
    std::memcpy(m->norm_h, state_host, sizeof(m->norm_h));
    DI_CUDA_TRY(cudaMemcpy(m->norm, state_host, 2 * kNF * sizeof(float), cudaMemcpyHostToDevice));
    DI_CUDA_TRY(cudaMemcpy(m->theta, state_host + 2 * kNF, kNP * sizeof(float), cudaMemcpyHostToDevice));
    k_pack_weights<<<(kHid * kK1 + kHid * kHid + 255) / 256, 256>>>(m->theta, m->wbf);
    DI_CUDA_TRY(cudaGetLastError());
    DI_CUDA_TRY(cudaDeviceSynchronize());
    return DI_OK;
}

di_status model_new(di_model **out) {
    di_model *m = new (std::nothrow) di_model();
    if (!m) { set_error("model: host allocation failed"); return DI_ENOMEM; }
    struct Guard {
        di_model *m;
        bool keep = false;
        ~Guard() { if (!keep) free_model(m); }
    } guard{m};
    DI_CUDA_TRY(cudaGetDevice(&m->device));
    DI_CUDA_TRY(cudaMalloc(&m->theta, kNP * sizeof(float)));
    DI_CUDA_TRY(cudaMalloc(&m->m, kNP * sizeof(float)));
    DI_CUDA_TRY(cudaMalloc(&m->v, kNP * sizeof(float)));
    DI_CUDA_TRY(cudaMalloc(&m->grad, kNP * sizeof(float)));
    DI_CUDA_TRY(cudaMalloc(&m->norm, 2 * kNF * sizeof(float)));
    DI_CUDA_TRY(cudaMalloc(&m->wbf, (kHid * kK1 + kHid * kHid) * sizeof(__nv_bfloat16)));
    DI_CUDA_TRY(cudaMalloc(&m->dacc, (2 * kNF + 2) * sizeof(double)));
    DI_CUDA_TRY(cudaMemset(m->m, 0, kNP * sizeof(float)));
    DI_CUDA_TRY(cudaMemset(m->v, 0, kNP * sizeof(float)));
    guard.keep = true;
    *out = m;
    return DI_OK;
}

di_status check_model(const di_model *m, const char *who) {
    if (!m) { set_error("%s: NULL model", who); return DI_EINVAL; }
    int dev = -1;
    DI_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != m->device) { set_error("%s: model lives on device %d, current is %d", who, m->device, dev); return DI_EINVAL; }
    return DI_OK;
}

constexpr uint32_t kMagic = 0x53574944u;   // "DIWS"
constexpr uint32_t kVersion = 1;

}  // namespace

extern "C" DI_API di_status di_train_opts_default(di_train_opts *o) {
    if (!o) { set_error("di_train_opts_default: NULL"); return DI_EINVAL; }
    std::memset(o, 0, sizeof(*o));
    o->epochs = 4;
    o->batch = 65536;
    o->lr = 1e-3;
    o->beta1 = 0.9;
    o->beta2 = 0.999;
    o->eps = 1e-8;
    o->seed = 1;
    o->stream = nullptr;
    return DI_OK;
}

extern "C" DI_API di_status di_model_create(uint64_t seed, di_model **out) {
    clear_error();
    if (!out) { set_error("di_model_create: out is NULL"); return DI_EINVAL; }
    *out = nullptr;
    di_model *m = nullptr;
    DI_TRY(model_new(&m));
    std::vector<float> state(DI_MODEL_STATE, 0.f);
    for (int c = 0; c < kNF; ++c) state[kNF + c] = 1.f;    // identity standardisation
    std::vector<float> th;
    init_params(th, seed);
    std::copy(th.begin(), th.end(), state.begin() + 2 * kNF);
    di_status rc = upload_state(m, state.data());
    if (rc != DI_OK) { free_model(m); return rc; }
    *out = m;
    return DI_OK;
}

extern "C" DI_API void di_model_destroy(di_model *m) { free_model(m); }

extern "C" DI_API di_status di_model_get(const di_model *m, float *state) {
    clear_error();
    DI_TRY(check_model(m, "di_model_get"));
    if (!state) { set_error("di_model_get: NULL state"); return DI_EINVAL; }
    std::memcpy(state, m->norm_h, sizeof(m->norm_h));
    DI_CUDA_TRY(cudaMemcpy(state + 2 * kNF, m->theta, kNP * sizeof(float), cudaMemcpyDeviceToHost));
    return DI_OK;
}

extern "C" DI_API di_status di_model_set(di_model *m, const float *state) {
    clear_error();
    DI_TRY(check_model(m, "di_model_set"));
    if (!state) { set_error("di_model_set: NULL state"); return DI_EINVAL; }
    for (int c = 0; c < kNF; ++c)
        if (!(state[kNF + c] > 0.f) || !std::isfinite(state[c])) {
            set_error("di_model_set: feature %d has mu = %g, sd = %g (sd must be > 0)", c, state[c], state[kNF + c]);
            return DI_EINVAL;
        }
    return upload_state(m, state);
}

extern "C" DI_API di_status di_features(di_model *m, di_graph *g, const double *B, float *feat, void *stream) {
    di::NvtxRange nvtx_range("di_features");
    clear_error();
    DI_TRY(check_model(m, "di_features"));
    if (!g || !B || !feat) { set_error("di_features: NULL argument"); return DI_EINVAL; }
    if (g->device != m->device) { set_error("di_features: graph and model on different devices"); return DI_EINVAL; }
    return features_into(m, g, B, feat, as_stream(stream));
}

extern "C" DI_API di_status di_mlp_forward(const di_model *m, const float *feat, int64_t n, float *y, void *stream) {
    di::NvtxRange nvtx_range("di_mlp_forward");
    clear_error();
    DI_TRY(check_model(m, "di_mlp_forward"));
    if (!feat || !y || n < 1) { set_error("di_mlp_forward: NULL argument or n < 1"); return DI_EINVAL; }
    FwdArgs a = fwd_args(m);
    a.feat = feat;
    a.nrows = n;
    a.y = y;
    k_mlp_fwd<FWD_Y><<<fwd_grid(m->device, n), kFwdThreads, 0, as_stream(stream)>>>(a);
    DI_CUDA_TRY(cudaGetLastError());
    return DI_OK;
}

extern "C" DI_API di_status di_mlp_grad(di_model *m, const float *feat, const float *target, int64_t n, float *grad,
                                       double *loss, void *stream) {
    clear_error();
    DI_TRY(check_model(m, "di_mlp_grad"));
    if (!feat || !target || !grad || n < 1 || n > INT32_MAX) {
        set_error("di_mlp_grad: NULL argument or n outside [1, 2^31)");
        return DI_EINVAL;
    }
    cudaStream_t s = as_stream(stream);
    DI_TRY(ensure_rows(m, n));
    std::vector<int32_t> iota(n);
    for (int64_t i = 0; i < n; ++i) iota[i] = (int32_t)i;
    DI_CUDA_TRY(cudaMemcpyAsync(m->idx, iota.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    DI_CUDA_TRY(cudaMemsetAsync(m->dacc, 0, sizeof(double), s));
    DI_TRY(grad_pass(m, feat, target, n, m->dacc, s));
    double l = 0.0;
    DI_CUDA_TRY(cudaMemcpyAsync(grad, m->grad, kNP * sizeof(float), cudaMemcpyDeviceToHost, s));
    DI_CUDA_TRY(cudaMemcpyAsync(&l, m->dacc, sizeof(double), cudaMemcpyDeviceToHost, s));
    DI_CUDA_TRY(cudaStreamSynchronize(s));
    if (loss) *loss = l / (double)n;
    return DI_OK;
}

extern "C" DI_API di_status di_model_adam(di_model *m, const float *grad, const di_train_opts *opts) {
    clear_error();
    DI_TRY(check_model(m, "di_model_adam"));
    if (!grad) { set_error("di_model_adam: NULL grad"); return DI_EINVAL; }
    di_train_opts o;
    if (opts) o = *opts; else di_train_opts_default(&o);
    cudaStream_t s = as_stream(o.stream);
    DI_CUDA_TRY(cudaMemcpyAsync(m->grad, grad, kNP * sizeof(float), cudaMemcpyHostToDevice, s));
    adam_launch(m, o, s);
    DI_CUDA_TRY(cudaGetLastError());
    DI_CUDA_TRY(cudaStreamSynchronize(s));
    return DI_OK;
}

extern "C" DI_API di_status di_warmstart_train(di_model *m, di_graph *const *graphs, int ng, const double *const *B,
                                              const double *const *X, const di_train_opts *opts, double *final_loss) {
    di::NvtxRange nvtx_range("di_warmstart_train");
    clear_error();
    DI_TRY(check_model(m, "di_warmstart_train"));
    if (!graphs || !B || !X || ng < 1) { set_error("di_warmstart_train: need ng >= 1 graphs with B and X"); return DI_EINVAL; }
    di_train_opts o;
    if (opts) o = *opts; else di_train_opts_default(&o);
    if (o.epochs < 1 || o.batch < 16 || !(o.lr > 0.0) || !(o.beta1 >= 0.0 && o.beta1 < 1.0) ||
        !(o.beta2 >= 0.0 && o.beta2 < 1.0) || !(o.eps > 0.0)) {
        set_error("di_warmstart_train: bad options (epochs >= 1, batch >= 16, lr > 0, beta in [0,1), eps > 0)");
        return DI_EINVAL;
    }
    int64_t total = 0, maxn = 0;
    for (int i = 0; i < ng; ++i) {
        if (!graphs[i] || !B[i] || !X[i]) { set_error("di_warmstart_train: NULL graph, B or X %d", i); return DI_EINVAL; }
        if (graphs[i]->device != m->device) { set_error("di_warmstart_train: graph %d on another device", i); return DI_EINVAL; }
        total += graphs[i]->n;
        maxn = std::max<int64_t>(maxn, graphs[i]->n);
    }
    if (total > INT32_MAX) { set_error("di_warmstart_train: %lld training nodes exceed 2^31", (long long)total); return DI_EINVAL; }
    cudaStream_t s = as_stream(o.stream);
    float *feat_all = nullptr, *tgt = nullptr;
    DI_CUDA_TRY(cudaMalloc(&feat_all, (size_t)total * kNF * sizeof(float)));
    struct FreeOnExit {
        void *a = nullptr, *b = nullptr;
        ~FreeOnExit() { if (a) cudaFree(a); if (b) cudaFree(b); }
    } fo;
    fo.a = feat_all;
    DI_CUDA_TRY(cudaMalloc(&tgt, (size_t)total * sizeof(float)));
    fo.b = tgt;
    int64_t off = 0;
    for (int i = 0; i < ng; ++i) {
        di_graph *g = graphs[i];
        DI_TRY(features_into(m, g, B[i], feat_all + off * kNF, s));
        k_target<<<grid_of(g->n, 256, g->num_sms * 8), 256, 0, s>>>(X[i], g->n, tgt + off);
        off += g->n;
    }
    // standardisation statistics of the training features; b3 starts at the mean target
    DI_CUDA_TRY(cudaMemsetAsync(m->dacc, 0, (2 * kNF + 2) * sizeof(double), s));
    k_colstats<<<grid_of(total, 256, sm_count(m->device) * 4), 256, 0, s>>>(feat_all, tgt, total, m->dacc);
    double acc[2 * kNF + 2];
    DI_CUDA_TRY(cudaMemcpyAsync(acc, m->dacc, sizeof(acc), cudaMemcpyDeviceToHost, s));
    DI_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<float> state(DI_MODEL_STATE);
    DI_CUDA_TRY(cudaMemcpy(state.data() + 2 * kNF, m->theta, kNP * sizeof(float), cudaMemcpyDeviceToHost));
    for (int c = 0; c < kNF; ++c) {
        const double mu = acc[c] / (double)total;
        const double var = std::max(acc[kNF + c] / (double)total - mu * mu, 0.0);
        const double sd = std::sqrt(var);
        state[c] = (float)mu;
        state[kNF + c] = sd > 1e-6 * std::max(1.0, std::fabs(mu)) ? (float)sd : 1.f;
    }
    if (m->step == 0) state[2 * kNF + kOffB3] = (float)(acc[2 * kNF] / (double)total);
    DI_TRY(upload_state(m, state.data()));

    const int64_t M = std::min<int64_t>(o.batch, total);
    DI_TRY(ensure_rows(m, M));
    const int64_t steps_per_epoch = (total + M - 1) / M;
    double loss_last_epoch = 0.0;
    for (int ep = 0; ep < o.epochs; ++ep) {
        DI_CUDA_TRY(cudaMemsetAsync(m->dacc, 0, sizeof(double), s));
        for (int64_t st = 0; st < steps_per_epoch; ++st) {
            const uint64_t counter = (uint64_t)ep * (uint64_t)steps_per_epoch + (uint64_t)st;
            k_sample<<<(int)((M + 255) / 256), 256, 0, s>>>(m->idx, M, o.seed, counter, total);
            DI_TRY(grad_pass(m, feat_all, tgt, M, m->dacc, s));
            adam_launch(m, o, s);
        }
        DI_CUDA_TRY(cudaGetLastError());
        double l = 0.0;
        DI_CUDA_TRY(cudaMemcpyAsync(&l, m->dacc, sizeof(double), cudaMemcpyDeviceToHost, s));
        DI_CUDA_TRY(cudaStreamSynchronize(s));
        loss_last_epoch = l / (double)(M * steps_per_epoch);
    }
    m->last_loss = loss_last_epoch;
    if (final_loss) *final_loss = loss_last_epoch;
    return DI_OK;
}

extern "C" DI_API di_status di_warmstart_infer(di_model *m, di_graph *g, const double *B, double *H0, void *stream) {
    di::NvtxRange nvtx_range("di_warmstart_infer");
    clear_error();
    DI_TRY(check_model(m, "di_warmstart_infer"));
    if (!g || !B || !H0) { set_error("di_warmstart_infer: NULL argument"); return DI_EINVAL; }
    if (g->device != m->device) { set_error("di_warmstart_infer: graph and model on different devices"); return DI_EINVAL; }
    cudaStream_t s = as_stream(stream);
    DI_TRY(ensure_feat(m, g->n));
    DI_TRY(features_into(m, g, B, m->feat, s));
    FwdArgs a = fwd_args(m);
    a.feat = m->feat;
    a.nrows = g->n;
    a.h0 = H0;
    a.inv_n = 1.0 / (double)g->n;
    k_mlp_fwd<FWD_H0><<<fwd_grid(m->device, g->n), kFwdThreads, 0, s>>>(a);
    DI_CUDA_TRY(cudaGetLastError());
    return DI_OK;
}

extern "C" DI_API di_status di_warmstart_save(const di_model *m, const char *path) {
    clear_error();
    DI_TRY(check_model(m, "di_warmstart_save"));
    if (!path) { set_error("di_warmstart_save: NULL path"); return DI_EINVAL; }
    std::vector<float> th(kNP), mm(kNP), vv(kNP);
    DI_CUDA_TRY(cudaMemcpy(th.data(), m->theta, kNP * sizeof(float), cudaMemcpyDeviceToHost));
    DI_CUDA_TRY(cudaMemcpy(mm.data(), m->m, kNP * sizeof(float), cudaMemcpyDeviceToHost));
    DI_CUDA_TRY(cudaMemcpy(vv.data(), m->v, kNP * sizeof(float), cudaMemcpyDeviceToHost));
    FILE *f = std::fopen(path, "wb");
    if (!f) { set_error("di_warmstart_save: cannot open %s", path); return DI_EINVAL; }
    const uint32_t hdr[4] = {kMagic, kVersion, (uint32_t)kNF, (uint32_t)kNP};
    const int64_t step = m->step;
    bool ok = std::fwrite(hdr, sizeof(hdr), 1, f) == 1 && std::fwrite(&step, sizeof(step), 1, f) == 1 &&
              std::fwrite(m->norm_h, sizeof(m->norm_h), 1, f) == 1 &&
              std::fwrite(th.data(), sizeof(float), kNP, f) == (size_t)kNP &&
              std::fwrite(mm.data(), sizeof(float), kNP, f) == (size_t)kNP &&
              std::fwrite(vv.data(), sizeof(float), kNP, f) == (size_t)kNP;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) { set_error("di_warmstart_save: write to %s failed", path); return DI_EINVAL; }
    return DI_OK;
}

extern "C" DI_API di_status di_warmstart_load(const char *path, di_model **out) {
    clear_error();
    if (!path || !out) { set_error("di_warmstart_load: NULL argument"); return DI_EINVAL; }
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) { set_error("di_warmstart_load: cannot open %s", path); return DI_EINVAL; }
    uint32_t hdr[4] = {0, 0, 0, 0};
    int64_t step = 0;
    std::vector<float> state(DI_MODEL_STATE), mm(kNP), vv(kNP);
    bool ok = std::fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == kMagic && hdr[1] == kVersion &&
              hdr[2] == (uint32_t)kNF && hdr[3] == (uint32_t)kNP && std::fread(&step, sizeof(step), 1, f) == 1 &&
              std::fread(state.data(), sizeof(float), DI_MODEL_STATE, f) == (size_t)DI_MODEL_STATE &&
              std::fread(mm.data(), sizeof(float), kNP, f) == (size_t)kNP &&
              std::fread(vv.data(), sizeof(float), kNP, f) == (size_t)kNP;
    std::fclose(f);
    if (!ok) { set_error("di_warmstart_load: %s is not a model file of this version", path); return DI_EINVAL; }
    di_model *m = nullptr;
    DI_TRY(model_new(&m));
    di_status rc = upload_state(m, state.data());
    if (rc == DI_OK) {
        cudaError_t e1 = cudaMemcpy(m->m, mm.data(), kNP * sizeof(float), cudaMemcpyHostToDevice);
        cudaError_t e2 = cudaMemcpy(m->v, vv.data(), kNP * sizeof(float), cudaMemcpyHostToDevice);
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            set_error("di_warmstart_load: upload failed: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
            rc = DI_ECUDA;
        }
    }
    if (rc != DI_OK) { free_model(m); return rc; }
    m->step = step;
    *out = m;
    return DI_OK;
}
