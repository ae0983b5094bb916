// graph.cu - device form of P (Sec. 2.2): out-CSR for the push, in-CSR
// (transpose) for the exact residual, d/outdeg scales, hot-target slots.
#include <algorithm>
#include <vector>

#include "di_internal.cuh"
#include "pull.cuh"

namespace di {
namespace {

constexpr int kThreads = 256;

int grid_for(int64_t items, int per_block, int cap) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return static_cast<int>(b);
}

// Validation: row_ptr[0] == 0, non-decreasing, row_ptr[n] == nnz, col in [0, n).
__global__ void k_validate(const int64_t *__restrict__ rp, const int32_t *__restrict__ col, int64_t n,
                           int64_t nnz, unsigned long long *bad) {
    unsigned long long b = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        if (rp[i + 1] < rp[i]) ++b;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (rp[0] != 0) ++b;
        if (rp[n] != nnz) ++b;
    }
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        int32_t c = col[e];
        if (c < 0 || c >= n) ++b;
    }
    b = warp_sum(b);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(bad, b);
}

// int64 offsets -> int32, plus out-degree statistics.
__global__ void k_offsets32(const int64_t *__restrict__ rp64, int32_t *__restrict__ rp32, int64_t n,
                            unsigned long long *n_dangling, int *max_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long dang = 0;
    int mx = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride) {
        rp32[i] = static_cast<int32_t>(rp64[i]);
        if (i < n) {
            int deg = static_cast<int>(rp64[i + 1] - rp64[i]);
            if (deg == 0) ++dang;
            mx = max(mx, deg);
        }
    }
    dang = warp_sum(dang);
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) {
        if (dang) atomicAdd(n_dangling, dang);
        atomicMax(max_out, mx);
    }
}

// In-degree histogram over all edges.
__global__ void k_indeg(const int32_t *__restrict__ col, int64_t nnz, int32_t *__restrict__ cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride)
        atomicAdd(&cnt[col[e]], 1);
}

__global__ void k_count_ge(const int32_t *__restrict__ cnt, int64_t n, int t, unsigned long long *out,
                           int *max_in) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long c = 0;
    int mx = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int v = cnt[i];
        if (v >= t) ++c;
        mx = max(mx, v);
    }
    c = warp_sum(c);
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) {
        if (c) atomicAdd(out, c);
        if (max_in) atomicMax(max_in, mx);
    }
}

// Exclusive scan of int32 counts in chunks: per-chunk sums, host scan of the
// chunk sums, then a per-chunk scan that adds the chunk offset.
constexpr int kScanChunkElems = 4096;   // per block: 256 threads x 16

__global__ void k_chunk_sums(const int32_t *__restrict__ cnt, int64_t n, int64_t *__restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanChunkElems;
    int64_t s = 0;
    for (int k = threadIdx.x; k < kScanChunkElems; k += blockDim.x) {
        int64_t i = base + k;
        if (i < n) s += cnt[i];
    }
    s = warp_sum(s);
    __shared__ int64_t ws[kThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += ws[w];
        sums[blockIdx.x] = t;
    }
}

__global__ void k_chunk_scan(const int32_t *__restrict__ cnt, int64_t n, const int64_t *__restrict__ offs,
                             int32_t *__restrict__ out) {
    // each thread owns 16 consecutive elements of the chunk
    constexpr int kPer = kScanChunkElems / kThreads;
    const int64_t base = (int64_t)blockIdx.x * kScanChunkElems + (int64_t)threadIdx.x * kPer;
    int32_t v[kPer];
    int64_t local = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        int64_t i = base + k;
        v[k] = i < n ? cnt[i] : 0;
        local += v[k];
    }
    // exclusive scan of `local` across the block
    __shared__ int64_t sh[kThreads];
    sh[threadIdx.x] = local;
    __syncthreads();
    for (int o = 1; o < kThreads; o <<= 1) {
        int64_t add = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += add;
        __syncthreads();
    }
    int64_t run = offs[blockIdx.x] + sh[threadIdx.x] - local;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = static_cast<int32_t>(run);
        run += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kThreads - 1) out[n] = static_cast<int32_t>(run);
}

// Fill the transpose: edge j -> k becomes in-edge k <- j.  One thread per row.
__global__ void k_fill_in(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, int64_t n,
                          int32_t *__restrict__ cursor, int32_t *__restrict__ in_col) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        for (int32_t e = rp[j]; e < rp[j + 1]; ++e) {
            int32_t pos = atomicAdd(&cursor[col[e]], 1);
            in_col[pos] = static_cast<int32_t>(j);
        }
    }
}

__global__ void k_assign_hot(const int32_t *__restrict__ cnt, int64_t n, int t, int32_t *__restrict__ slot_of,
                             int32_t *__restrict__ hot_node, int *n_hot) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int s = -1;
        if (cnt[i] >= t) {
            s = atomicAdd(n_hot, 1);
            hot_node[s] = static_cast<int32_t>(i);
        }
        slot_of[i] = s;
    }
}

__global__ void k_encode_hot(int32_t *__restrict__ pcol, int64_t nnz, const int32_t *__restrict__ slot_of) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        int s = slot_of[pcol[e]];
        if (s >= 0) pcol[e] = -1 - s;
    }
}

// Contiguous copy of the in-edges of the rows of bins 1-2, in bin order.
__global__ void k_copy_rows(const int32_t *__restrict__ rows, int64_t nrows, const int32_t *__restrict__ in_rp,
                            const int32_t *__restrict__ in_col, const int32_t *__restrict__ off,
                            int32_t *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrows; i += stride) {
        const int32_t r = rows[i], b = in_rp[r], e = in_rp[r + 1], o = off[i];
        for (int32_t q = b; q < e; ++q) out[o + (q - b)] = in_col[q];
    }
}

// Destination row of every in-edge (the flat gather's run keys).
__global__ void k_erow(const int32_t *__restrict__ in_rp, int64_t n, int32_t *__restrict__ erow) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride)
        for (int32_t q = in_rp[k]; q < in_rp[k + 1]; ++q) erow[q] = (int32_t)k;
}

// Source-blocked order of the in-edges, one source block at a time: count,
// per destination row k, the in-edges whose source lies in [lo, hi), then
// copy them in row order (the order inside a row is the in-CSR order).
__global__ void k_blk_count(const int32_t *__restrict__ in_rp, const int32_t *__restrict__ in_col, int64_t n,
                            int32_t lo, int32_t hi, int32_t *__restrict__ cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        int32_t c = 0;
        for (int32_t q = in_rp[k]; q < in_rp[k + 1]; ++q) {
            const int32_t j = in_col[q];
            c += (j >= lo && j < hi) ? 1 : 0;
        }
        cnt[k] = c;
    }
}

__global__ void k_blk_fill(const int32_t *__restrict__ in_rp, const int32_t *__restrict__ in_col, int64_t n,
                           int32_t lo, int32_t hi, const int32_t *__restrict__ off, int64_t base,
                           int32_t *__restrict__ bcol, int32_t *__restrict__ brow) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        int64_t pos = base + off[k];
        for (int32_t q = in_rp[k]; q < in_rp[k + 1]; ++q) {
            const int32_t j = in_col[q];
            if (j >= lo && j < hi) {
                bcol[pos] = j;
                brow[pos] = static_cast<int32_t>(k);
                ++pos;
            }
        }
    }
}

// 1 / ((in + 1)(out + 1)) in FP64 and its FP32 rounding.
__global__ void k_sel_weights(const int32_t *__restrict__ rp, const int32_t *__restrict__ in_rp, int64_t n,
                              double *__restrict__ w64, float *__restrict__ w32) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double in = (double)(in_rp[i + 1] - in_rp[i]), out = (double)(rp[i + 1] - rp[i]);
        const double w = 1.0 / ((in + 1.0) * (out + 1.0));
        w64[i] = w;
        w32[i] = (float)w;
    }
}

__global__ void k_outdeg(const int32_t *__restrict__ rp, int64_t n, int32_t *__restrict__ deg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) deg[i] = rp[i + 1] - rp[i];
}

// Locality of the edges for the window of the tiled level kernel: counts of
// the edges j -> k with |k - j| <= 32 << b for b = 0 .. kWinBins - 1 (hot
// targets decoded through hot_node).  One thread per row, per-CTA counters.
__global__ void k_win_hist(const int32_t *__restrict__ rp, const int32_t *__restrict__ pcol,
                           const int32_t *__restrict__ hot_node, int64_t n, unsigned long long *__restrict__ out) {
    __shared__ unsigned long long s_c[kWinBins];
    for (int b = threadIdx.x; b < kWinBins; b += blockDim.x) s_c[b] = 0ull;
    __syncthreads();
    unsigned long long c[kWinBins] = {};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        for (int32_t e = rp[j]; e < rp[j + 1]; ++e) {
            const int32_t code = pcol[e];
            const int64_t k = code >= 0 ? code : hot_node[-1 - code];
            const int64_t dist = k > j ? k - j : j - k;
#pragma unroll
            for (int b = 0; b < kWinBins; ++b) c[b] += dist <= (int64_t(32) << b) ? 1ull : 0ull;
        }
    }
#pragma unroll
    for (int b = 0; b < kWinBins; ++b)
        if (c[b]) atomicAdd(&s_c[b], c[b]);
    __syncthreads();
    for (int b = threadIdx.x; b < kWinBins; b += blockDim.x)
        if (s_c[b]) atomicAdd(&out[b], s_c[b]);
}

// d / outdeg (0 for a dangling node) in FP64 and its FP32 rounding.
__global__ void k_scale(const int32_t *__restrict__ rp, int64_t n, double d, double *__restrict__ s64,
                        float *__restrict__ s32) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int deg = rp[i + 1] - rp[i];
        double s = deg > 0 ? d / (double)deg : 0.0;
        s64[i] = s;
        s32[i] = (float)s;
    }
}

struct DevPtrs {
    std::vector<void *> p;
    ~DevPtrs() {
        for (void *q : p) cudaFree(q);
    }
    template <typename T>
    cudaError_t alloc(T **out, size_t count) {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
        if (e == cudaSuccess) p.push_back(q);
        *out = static_cast<T *>(q);
        return e;
    }
    void release(void *q) {
        auto it = std::find(p.begin(), p.end(), q);
        if (it != p.end()) p.erase(it);
    }
};

void free_graph(di_graph *g) {
    if (!g) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != g->device) cudaSetDevice(g->device);
    for (auto &sg : g->sg) {
        if (sg.exec) cudaGraphExecDestroy(sg.exec);
        if (sg.graph) cudaGraphDestroy(sg.graph);
    }
    free_kpid_cache(g);
    void *dev[] = {g->rp, g->pcol, g->hot_node, g->in_rp, g->in_col, g->long_rows, g->long_seg0,
                   g->seg_row, g->seg_beg, g->frows, g->fseg0, g->fseg_row, g->fseg_beg,
                   g->pl_rows, g->pl_seg_row, g->pl_seg_beg, g->pl_lrows, g->pl_lseg0, g->pl_b12_off,
                   g->pl_b12_col, g->outdeg, g->erow, g->s32, g->s64, g->iw32, g->iw64, g->ws.F32, g->ws.F64, g->ws.w32, g->ws.w64, g->ws.front, g->ws.g, g->ws.acc,
                   g->ws.seg_part, g->ws.part_sum, g->ws.part_max, g->ws.desc, g->ws.st,
                   g->ws.hostB, g->ws.hostH, g->ws.hostF};
    for (void *q : dev)
        if (q) cudaFree(q);
    if (g->n_src_blocks > 1) {
        if (g->bcol) cudaFree(g->bcol);
        if (g->brow) cudaFree(g->brow);
    }
    if (g->ws.desc_h) cudaFreeHost(g->ws.desc_h);
    if (g->ws.st_h) cudaFreeHost(g->ws.st_h);
    if (g->ws.ev0) cudaEventDestroy(g->ws.ev0);
    if (g->ws.ev1) cudaEventDestroy(g->ws.ev1);
    for (cudaEvent_t e : g->ws.tev)
        if (e) cudaEventDestroy(e);
    if (cur >= 0 && cur != g->device) cudaSetDevice(cur);
    delete g;
}

// Rows of in-degree > seg_len, cut in segments of seg_len in-edges:
// rows[r] = row id, seg0[r] = first segment of row r (seg0[n_rows] = n_seg),
// seg_row[s] = r, seg_beg[s] = first in-edge of segment s.
di_status build_segments(const std::vector<int32_t> &hin, int seg_len, int *n_rows, int *n_seg, int32_t **d_rows,
                         int32_t **d_seg0, int32_t **d_seg_row, int64_t **d_seg_beg) {
    const int64_t n = (int64_t)hin.size() - 1;
    std::vector<int32_t> rows, seg0, segrow;
    std::vector<int64_t> segbeg;
    for (int64_t k = 0; k < n; ++k) {
        const int64_t len = (int64_t)hin[k + 1] - hin[k];
        if (len > seg_len) {
            seg0.push_back(static_cast<int32_t>(segrow.size()));
            for (int64_t b = hin[k]; b < hin[k + 1]; b += seg_len) {
                segrow.push_back(static_cast<int32_t>(rows.size()));
                segbeg.push_back(b);
            }
            rows.push_back(static_cast<int32_t>(k));
        }
    }
    seg0.push_back(static_cast<int32_t>(segrow.size()));
    *n_rows = static_cast<int>(rows.size());
    *n_seg = static_cast<int>(segrow.size());
    DI_CUDA_TRY(cudaMalloc(d_rows, std::max<size_t>(rows.size(), 1) * sizeof(int32_t)));
    DI_CUDA_TRY(cudaMalloc(d_seg0, seg0.size() * sizeof(int32_t)));
    DI_CUDA_TRY(cudaMalloc(d_seg_row, std::max<size_t>(segrow.size(), 1) * sizeof(int32_t)));
    DI_CUDA_TRY(cudaMalloc(d_seg_beg, std::max<size_t>(segbeg.size(), 1) * sizeof(int64_t)));
    if (!rows.empty()) {
        DI_CUDA_TRY(cudaMemcpy(*d_rows, rows.data(), rows.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        DI_CUDA_TRY(cudaMemcpy(*d_seg_row, segrow.data(), segrow.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        DI_CUDA_TRY(cudaMemcpy(*d_seg_beg, segbeg.data(), segbeg.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    }
    DI_CUDA_TRY(cudaMemcpy(*d_seg0, seg0.data(), seg0.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    return DI_OK;
}

// Binned pull plan (pull.cuh) from the host copy of the in-CSR offsets.
di_status build_pull_plan(di_graph *g, const std::vector<int32_t> &hin) {
    const int64_t n = (int64_t)hin.size() - 1;
    std::vector<int32_t> bins[4], segrow, segbeg, lrows, lseg0;
    for (int64_t k = 0; k < n; ++k) {
        const int64_t len = (int64_t)hin[k + 1] - hin[k];
        if (len <= kBin1Max) bins[0].push_back((int32_t)k);
        else if (len <= kBin2Max) bins[1].push_back((int32_t)k);
        else if (len <= kBin3Max) bins[2].push_back((int32_t)k);
        else if (len <= kBin4Max) bins[3].push_back((int32_t)k);
        else {
            lseg0.push_back((int32_t)segrow.size());
            lrows.push_back((int32_t)k);
            for (int64_t b = hin[k]; b < hin[k + 1]; b += kPullSeg) {
                segrow.push_back((int32_t)k);
                segbeg.push_back((int32_t)b);
            }
        }
    }
    lseg0.push_back((int32_t)segrow.size());
    std::vector<int32_t> rows;
    rows.reserve(n);
    g->pl_bin_off[0] = 0;
    for (int b = 0; b < 4; ++b) {
        rows.insert(rows.end(), bins[b].begin(), bins[b].end());
        g->pl_bin_off[b + 1] = (int64_t)rows.size();
    }
    const int64_t per_task[4] = {kPullThreads, kPullThreads / 4, kPullThreads / 32, 1};
    g->pl_task_off[0] = 0;
    for (int b = 0; b < 4; ++b)
        g->pl_task_off[b + 1] = g->pl_task_off[b] + ((int64_t)bins[b].size() + per_task[b] - 1) / per_task[b];
    g->pl_task_off[5] = g->pl_task_off[4] + (int64_t)segrow.size();
    g->pl_nlrows = (int)lrows.size();
    // bins 1-2: offsets of their edges once copied contiguously in bin order
    const int64_t n12 = g->pl_bin_off[2];
    std::vector<int32_t> off12(n12 + 1);
    int64_t run = 0;
    for (int64_t i = 0; i < n12; ++i) {
        off12[i] = (int32_t)run;
        run += (int64_t)hin[rows[i] + 1] - hin[rows[i]];
    }
    off12[n12] = (int32_t)run;
    auto up = [](int32_t **d, const std::vector<int32_t> &h) -> di_status {
        DI_CUDA_TRY(cudaMalloc(d, std::max<size_t>(h.size(), 1) * sizeof(int32_t)));
        if (!h.empty()) DI_CUDA_TRY(cudaMemcpy(*d, h.data(), h.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        return DI_OK;
    };
    DI_TRY(up(&g->pl_rows, rows));
    DI_TRY(up(&g->pl_seg_row, segrow));
    DI_TRY(up(&g->pl_seg_beg, segbeg));
    DI_TRY(up(&g->pl_lrows, lrows));
    DI_TRY(up(&g->pl_lseg0, lseg0));
    DI_TRY(up(&g->pl_b12_off, off12));
    DI_CUDA_TRY(cudaMalloc(&g->pl_b12_col, std::max<int64_t>(run, 1) * sizeof(int32_t)));
    if (n12 > 0)
        k_copy_rows<<<(int)std::min<int64_t>((n12 + 255) / 256, 4096), 256>>>(g->pl_rows, n12, g->in_rp, g->in_col,
                                                                              g->pl_b12_off, g->pl_b12_col);
    DI_CUDA_TRY(cudaGetLastError());
    DI_CUDA_TRY(cudaDeviceSynchronize());   // graph creation is synchronous
    return DI_OK;
}

}  // namespace

// Builds, on first use, the in-edges in source-blocked order (blocks of
// 2^kSrcBlockShift sources, then destination row).  With one block it is the
// in-CSR order itself.
di_status ensure_blocked_order(di_graph *g, cudaStream_t s) {
    if (g->bcol) return DI_OK;
    const int64_t n = g->n, nnz = g->nnz;
    g->n_src_blocks = (int)((n + (1LL << kSrcBlockShift) - 1) >> kSrcBlockShift);
    if (g->n_src_blocks <= 1 || nnz == 0) {
        g->n_src_blocks = 1;
        g->bcol = g->in_col;
        g->brow = g->erow;
        return DI_OK;
    }
    DevPtrs tmp;
    int32_t *cnt = nullptr, *off = nullptr, *bcol = nullptr, *brow = nullptr;
    const int nchunks = static_cast<int>((n + kScanChunkElems - 1) / kScanChunkElems);
    int64_t *chunk = nullptr;
    DI_CUDA_TRY(tmp.alloc(&cnt, n));
    DI_CUDA_TRY(tmp.alloc(&off, n + 1));
    DI_CUDA_TRY(tmp.alloc(&chunk, nchunks));
    DI_CUDA_TRY(tmp.alloc(&bcol, nnz));
    DI_CUDA_TRY(tmp.alloc(&brow, nnz));
    const int cap = g->num_sms * 16;
    std::vector<int64_t> hc(nchunks);
    int64_t base = 0;
    for (int b = 0; b < g->n_src_blocks; ++b) {
        const int64_t lo64 = (int64_t)b << kSrcBlockShift;
        const int32_t lo = (int32_t)lo64, hi = (int32_t)std::min<int64_t>(n, lo64 + (1LL << kSrcBlockShift));
        k_blk_count<<<grid_for(n, kThreads, cap), kThreads, 0, s>>>(g->in_rp, g->in_col, n, lo, hi, cnt);
        k_chunk_sums<<<nchunks, kThreads, 0, s>>>(cnt, n, chunk);
        DI_CUDA_TRY(cudaMemcpyAsync(hc.data(), chunk, nchunks * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        DI_CUDA_TRY(cudaStreamSynchronize(s));
        int64_t run = 0;
        for (int c = 0; c < nchunks; ++c) {
            const int64_t v = hc[c];
            hc[c] = run;
            run += v;
        }
        DI_CUDA_TRY(cudaMemcpyAsync(chunk, hc.data(), nchunks * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        k_chunk_scan<<<nchunks, kThreads, 0, s>>>(cnt, n, chunk, off);
        k_blk_fill<<<grid_for(n, kThreads, cap), kThreads, 0, s>>>(g->in_rp, g->in_col, n, lo, hi, off, base, bcol,
                                                                   brow);
        base += run;
    }
    DI_CUDA_TRY(cudaGetLastError());
    DI_CUDA_TRY(cudaStreamSynchronize(s));
    if (base != nnz) {
        set_error("blocked order: placed %lld of %lld in-edges", (long long)base, (long long)nnz);
        return DI_ECUDA;
    }
    tmp.release(bcol);
    tmp.release(brow);
    g->bcol = bcol;
    g->brow = brow;
    return DI_OK;
}

di_status ensure_selection_weights(di_graph *g, cudaStream_t s) {
    if (g->iw64) return DI_OK;
    const int64_t npad = (g->n + 3) / 4 * 4;   // padded like the fluid (vector loads)
    DI_CUDA_TRY(cudaMalloc(&g->iw64, npad * sizeof(double)));
    DI_CUDA_TRY(cudaMalloc(&g->iw32, npad * sizeof(float)));
    DI_CUDA_TRY(cudaMemsetAsync(g->iw64, 0, npad * sizeof(double), s));
    DI_CUDA_TRY(cudaMemsetAsync(g->iw32, 0, npad * sizeof(float), s));
    k_sel_weights<<<grid_for(g->n, kThreads, g->num_sms * 16), kThreads, 0, s>>>(g->rp, g->in_rp, g->n, g->iw64,
                                                                                g->iw32);
    DI_CUDA_TRY(cudaGetLastError());
    return DI_OK;
}

PullPlan pull_plan_of(const di_graph *g) {
    PullPlan p;
    p.rows = g->pl_rows;
    p.b12_off = g->pl_b12_off;
    p.b12_col = g->pl_b12_col;
    for (int b = 0; b < 5; ++b) p.bin_off[b] = g->pl_bin_off[b];
    for (int b = 0; b < 6; ++b) p.task_off[b] = g->pl_task_off[b];
    p.seg_row = g->pl_seg_row;
    p.seg_beg = g->pl_seg_beg;
    return p;
}

// Radius R of the fluid window of the tiled level kernel: the smallest
// 32 << b whose edges |k - j| <= R are at least 90% of those within
// kMaxWinR; 0 (no window) when fewer than 2% of the edges are that local.
// Lazy, once.
di_status ensure_window(di_graph *g, cudaStream_t s) {
    if (g->win_R >= 0) return DI_OK;
    unsigned long long *cnt = nullptr;
    DI_CUDA_TRY(cudaMalloc(&cnt, kWinBins * sizeof(unsigned long long)));
    unsigned long long h[kWinBins] = {};
    cudaError_t e = cudaMemsetAsync(cnt, 0, kWinBins * sizeof(unsigned long long), s);
    if (e == cudaSuccess && g->nnz > 0) {
        k_win_hist<<<grid_for(g->n, kThreads, g->num_sms * 8), kThreads, 0, s>>>(g->rp, g->pcol, g->hot_node, g->n,
                                                                                cnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(cnt);
    DI_CUDA_TRY(e);
    const unsigned long long all = h[kWinBins - 1];
    int R = 0;
    if (g->nnz > 0 && (double)all >= 0.02 * (double)g->nnz) {
        int b = 0;
        while (b < kWinBins - 1 && (double)h[b] < 0.9 * (double)all) ++b;
        R = 32 << b;
    }
    g->win_R = R;
    return DI_OK;
}

di_status ensure_scale(di_graph *g, double d, cudaStream_t s) {
    if (g->s64 && g->scale_d == d) return DI_OK;
    if (!g->s64) {
        DI_CUDA_TRY(cudaMalloc(&g->s64, std::max<int64_t>(g->n, 1) * sizeof(double)));
        DI_CUDA_TRY(cudaMalloc(&g->s32, std::max<int64_t>(g->n, 1) * sizeof(float)));
    }
    k_scale<<<grid_for(g->n, kThreads, 4 * g->num_sms * 8), kThreads, 0, s>>>(g->rp, g->n, d, g->s64, g->s32);
    DI_CUDA_TRY(cudaGetLastError());
    g->scale_d = d;
    return DI_OK;
}

}  // namespace di

using namespace di;

extern "C" DI_API di_status di_graph_create(int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                                           int on_device, void *stream, di_graph **out) {
    di::NvtxRange nvtx_range("di_graph_create");
    clear_error();
    if (!out) { set_error("di_graph_create: out is NULL"); return DI_EINVAL; }
    *out = nullptr;
    if (n < 1 || n > INT32_MAX) { set_error("di_graph_create: n = %lld outside [1, 2^31-1]", (long long)n); return DI_EINVAL; }
    if (nnz < 0 || nnz > INT32_MAX) { set_error("di_graph_create: nnz = %lld outside [0, 2^31-1]", (long long)nnz); return DI_EINVAL; }
    if (!row_ptr || (nnz > 0 && !col)) { set_error("di_graph_create: NULL row_ptr or col"); return DI_EINVAL; }
    cudaStream_t s = as_stream(stream);

    di_graph *g = new (std::nothrow) di_graph();
    if (!g) { set_error("di_graph_create: host allocation failed"); return DI_ENOMEM; }
    struct Guard {
        di_graph *g;
        bool keep = false;
        ~Guard() { if (!keep) free_graph(g); }
    } guard{g};

    DI_CUDA_TRY(cudaGetDevice(&g->device));
    DI_CUDA_TRY(cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device));
    g->n = n;
    g->nnz = nnz;
    const int cap = g->num_sms * 16;

    DevPtrs tmp;
    int64_t *rp64 = nullptr;
    unsigned long long *cnt64 = nullptr;   // [0] bad, [1] dangling, [2] count_ge
    int *ints = nullptr;                   // [0] max_out, [1] max_in, [2] n_hot
    int32_t *cnt = nullptr, *slot_of = nullptr;
    DI_CUDA_TRY(tmp.alloc(&rp64, n + 1));
    DI_CUDA_TRY(tmp.alloc(&cnt64, 4));
    DI_CUDA_TRY(tmp.alloc(&ints, 4));
    DI_CUDA_TRY(cudaMalloc(&g->rp, (n + 1) * sizeof(int32_t)));
    DI_CUDA_TRY(cudaMalloc(&g->pcol, std::max<int64_t>(nnz, 1) * sizeof(int32_t)));
    DI_CUDA_TRY(cudaMalloc(&g->in_rp, (n + 1) * sizeof(int32_t)));
    DI_CUDA_TRY(cudaMalloc(&g->in_col, std::max<int64_t>(nnz, 1) * sizeof(int32_t)));

    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    DI_CUDA_TRY(cudaMemcpyAsync(rp64, row_ptr, (n + 1) * sizeof(int64_t), kind, s));
    if (nnz > 0) DI_CUDA_TRY(cudaMemcpyAsync(g->pcol, col, nnz * sizeof(int32_t), kind, s));
    DI_CUDA_TRY(cudaMemsetAsync(cnt64, 0, 4 * sizeof(unsigned long long), s));
    DI_CUDA_TRY(cudaMemsetAsync(ints, 0, 4 * sizeof(int), s));

    // 1. validate
    k_validate<<<grid_for(std::max(n, nnz), kThreads, cap), kThreads, 0, s>>>(rp64, g->pcol, n, nnz, cnt64);
    unsigned long long bad = 0;
    DI_CUDA_TRY(cudaMemcpyAsync(&bad, cnt64, sizeof(bad), cudaMemcpyDeviceToHost, s));
    DI_CUDA_TRY(cudaStreamSynchronize(s));
    if (bad) {
        set_error("di_graph_create: %llu violation(s) of the CSR contract (row_ptr[0]=0, non-decreasing, "
                  "row_ptr[n]=nnz, 0<=col<n)", bad);
        return DI_EINVAL;
    }
    // 2. int32 offsets and out-degree statistics
    k_offsets32<<<grid_for(n + 1, kThreads, cap), kThreads, 0, s>>>(rp64, g->rp, n, cnt64 + 1, ints);
    DI_CUDA_TRY(cudaMalloc(&g->outdeg, n * sizeof(int32_t)));
    k_outdeg<<<grid_for(n, kThreads, cap), kThreads, 0, s>>>(g->rp, n, g->outdeg);
    // 3. in-degrees
    DI_CUDA_TRY(tmp.alloc(&cnt, n));
    DI_CUDA_TRY(cudaMemsetAsync(cnt, 0, n * sizeof(int32_t), s));
    if (nnz > 0) k_indeg<<<grid_for(nnz, kThreads, cap), kThreads, 0, s>>>(g->pcol, nnz, cnt);
    // 4. in-CSR offsets
    const int nchunks = static_cast<int>((n + kScanChunkElems - 1) / kScanChunkElems);
    int64_t *chunk = nullptr;
    DI_CUDA_TRY(tmp.alloc(&chunk, nchunks));
    k_chunk_sums<<<nchunks, kThreads, 0, s>>>(cnt, n, chunk);
    std::vector<int64_t> hchunk(nchunks);
    DI_CUDA_TRY(cudaMemcpyAsync(hchunk.data(), chunk, nchunks * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    DI_CUDA_TRY(cudaStreamSynchronize(s));
    int64_t run = 0;
    for (int c = 0; c < nchunks; ++c) {
        int64_t v = hchunk[c];
        hchunk[c] = run;
        run += v;
    }
    if (run != nnz) { set_error("di_graph_create: in-degree total %lld != nnz", (long long)run); return DI_ECUDA; }
    DI_CUDA_TRY(cudaMemcpyAsync(chunk, hchunk.data(), nchunks * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    k_chunk_scan<<<nchunks, kThreads, 0, s>>>(cnt, n, chunk, g->in_rp);
    // 5. fill the transpose (cursor = copy of in_rp)
    int32_t *cursor = nullptr;
    DI_CUDA_TRY(tmp.alloc(&cursor, n + 1));
    DI_CUDA_TRY(cudaMemcpyAsync(cursor, g->in_rp, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    k_fill_in<<<grid_for(n, kThreads, cap), kThreads, 0, s>>>(g->rp, g->pcol, n, cursor, g->in_col);

    DI_CUDA_TRY(cudaMalloc(&g->erow, std::max<int64_t>(nnz, 1) * sizeof(int32_t)));
    k_erow<<<grid_for(n, kThreads, cap), kThreads, 0, s>>>(g->in_rp, n, g->erow);
    // 6. hot targets: the smallest threshold t >= kHotMinIndeg with at most
    //    kMaxHot nodes of in-degree >= t (binary search on t)
    int lo = kHotMinIndeg, hi = INT32_MAX;
    auto count_ge = [&](int t, unsigned long long *res, int *mx) -> di_status {
        DI_CUDA_TRY(cudaMemsetAsync(cnt64 + 2, 0, sizeof(unsigned long long), s));
        k_count_ge<<<grid_for(n, kThreads, cap), kThreads, 0, s>>>(cnt, n, t, cnt64 + 2, mx);
        DI_CUDA_TRY(cudaMemcpyAsync(res, cnt64 + 2, sizeof(*res), cudaMemcpyDeviceToHost, s));
        DI_CUDA_TRY(cudaStreamSynchronize(s));
        return DI_OK;
    };
    unsigned long long c_lo = 0;
    DI_TRY(count_ge(lo, &c_lo, ints + 1));
    int hstats[3] = {0, 0, 0};
    unsigned long long hdang = 0;
    DI_CUDA_TRY(cudaMemcpy(hstats, ints, 2 * sizeof(int), cudaMemcpyDeviceToHost));
    DI_CUDA_TRY(cudaMemcpy(&hdang, cnt64 + 1, sizeof(hdang), cudaMemcpyDeviceToHost));
    g->max_outdeg = hstats[0];
    g->max_indeg = hstats[1];
    g->n_dangling = static_cast<int64_t>(hdang);
    int t_hot = lo;
    if (c_lo > (unsigned long long)kMaxHot) {
        hi = std::max(lo, hstats[1]) + 1;   // count_ge(hi) == 0
        while (hi - lo > 1) {
            int mid = lo + (hi - lo) / 2;
            unsigned long long c = 0;
            DI_TRY(count_ge(mid, &c, nullptr));
            if (c > (unsigned long long)kMaxHot) lo = mid; else hi = mid;
        }
        t_hot = hi;
    }
    DI_CUDA_TRY(cudaMalloc(&g->hot_node, kMaxHot * sizeof(int32_t)));
    DI_CUDA_TRY(tmp.alloc(&slot_of, n));
    k_assign_hot<<<grid_for(n, kThreads, cap), kThreads, 0, s>>>(cnt, n, t_hot, slot_of, g->hot_node, ints + 2);
    if (nnz > 0) k_encode_hot<<<grid_for(nnz, kThreads, cap), kThreads, 0, s>>>(g->pcol, nnz, slot_of);
    int nh = 0;
    DI_CUDA_TRY(cudaMemcpyAsync(&nh, ints + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
    DI_CUDA_TRY(cudaStreamSynchronize(s));
    g->n_hot = nh;

    // 8. segments of the long in-rows (exact residual load balance), two granularities
    {
        std::vector<int32_t> hin(n + 1);
        DI_CUDA_TRY(cudaMemcpy(hin.data(), g->in_rp, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
        DI_TRY(build_segments(hin, kResSeg, &g->n_long_rows, &g->n_seg, &g->long_rows, &g->long_seg0, &g->seg_row,
                              &g->seg_beg));
        DI_TRY(build_pull_plan(g, hin));
    }
    DI_CUDA_TRY(cudaGetLastError());
    DI_CUDA_TRY(cudaStreamSynchronize(s));
    guard.keep = true;
    *out = g;
    return DI_OK;
}

extern "C" DI_API void di_graph_destroy(di_graph *g) { free_graph(g); }

extern "C" DI_API di_status di_graph_info(const di_graph *g, int64_t *n, int64_t *nnz, int64_t *n_dangling,
                                         int64_t *max_outdeg, int64_t *max_indeg, int64_t *n_hot) {
    clear_error();
    if (!g) { set_error("di_graph_info: NULL graph"); return DI_EINVAL; }
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    if (n_dangling) *n_dangling = g->n_dangling;
    if (max_outdeg) *max_outdeg = g->max_outdeg;
    if (max_indeg) *max_indeg = g->max_indeg;
    if (n_hot) *n_hot = g->n_hot;
    return DI_OK;
}
