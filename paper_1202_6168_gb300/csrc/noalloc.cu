// noalloc.cu - exact residual F = B + P H - H that allocates no memory.
//
// Some callers cannot call cudaMalloc on their hot path: a serving loop
// under a fixed device-memory budget that was reserved at start-up, code
// running while another component owns the allocator (a caching allocator,
// a memory pool being torn down), or a process that must not trigger the
// implicit synchronisation cudaMalloc/cudaFree can cause.  For them this
// file provides di_residual_noalloc: the same computation as di_residual,
// but its scratch memory is a file-scope static device array instead of
// buffers the library allocates on first use.
//
// The array is part of the library's device image, so every GPU that loads
// libdi.so holds it (kScratchBytes = 8,430,080 bytes) until the process exits.
// Its size caps the graphs this entry point accepts: at most kMaxN nodes and
// kMaxSeg segments of long in-rows; larger graphs get DI_EINVAL.
//
// Host code cannot use the array's name as a device address (in host code
// it names a host-side stand-in).  The first call on each device therefore
// resolves the array's device address with cudaGetSymbolAddress while that
// device is current, checks the result, caches it per device, and passes it
// to the kernels.  That first call should come before any stream capture.
//
// Every call shares the one array and it keeps the last call's contents.
// The completion counter, the only part that must start at zero, is cleared
// by each call (a cudaMemsetAsync on the stream, which allocates nothing).
// Calls that overlap on the GPU (on different streams, or from several
// threads) race on the array and give wrong results: serialise them.
#include <algorithm>
#include <mutex>

#include "di_internal.cuh"

namespace di {
namespace {

constexpr int64_t kMaxN = 1 << 20;       // nodes
constexpr int kMaxSeg = 4096;            // segments of in-rows longer than kResSeg
constexpr int kMaxBlocks = 1024;         // grid of the row kernel
constexpr size_t kAlign = 256;

constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
// layout of the scratch array
constexpr size_t kOffG = 0;                                                  // double[kMaxN]
constexpr size_t kOffSeg = align_up(kOffG + sizeof(double) * kMaxN);         // double[kMaxSeg]
constexpr size_t kOffPart = align_up(kOffSeg + sizeof(double) * kMaxSeg);    // double[kMaxBlocks]
constexpr size_t kOffCounter = align_up(kOffPart + sizeof(double) * kMaxBlocks);  // unsigned
constexpr size_t kOffResult = align_up(kOffCounter + sizeof(unsigned int));  // double
constexpr size_t kScratchBytes = align_up(kOffResult + sizeof(double));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
unsigned char *g_addr[kMaxDevices] = {};

// g_j = (d / outdeg_j) H_j, 0 for a dangling j (same arithmetic as the
// allocating path: the quotient first, then the product)
__global__ void __launch_bounds__(kResThreads) k_na_prep(const int32_t *__restrict__ rp,
                                                         const double *__restrict__ H, double d, int64_t n,
                                                         double *__restrict__ g) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int deg = rp[i + 1] - rp[i];
        const double s = deg > 0 ? d / (double)deg : 0.0;
        g[i] = s * H[i];
    }
}

__global__ void __launch_bounds__(kResThreads) k_na_seg(const int32_t *__restrict__ in_rp,
                                                        const int32_t *__restrict__ in_col,
                                                        const int32_t *__restrict__ long_rows,
                                                        const int32_t *__restrict__ seg_row,
                                                        const int64_t *__restrict__ seg_beg, int n_seg,
                                                        const double *__restrict__ g,
                                                        double *__restrict__ seg_part) {
    for (int s = blockIdx.x; s < n_seg; s += gridDim.x) {
        const int32_t row = long_rows[seg_row[s]];
        const int64_t b = seg_beg[s];
        const int64_t end = (int64_t)in_rp[row + 1];
        const int64_t e = b + kResSeg < end ? b + kResSeg : end;
        double acc = 0.0;
        for (int64_t q = b + threadIdx.x; q < e; q += kResThreads) acc += g[in_col[q]];
        double mx = 0.0;
        block_sum_max<kResThreads>(acc, mx);
        if (threadIdx.x == 0) seg_part[s] = acc;
    }
}

__global__ void __launch_bounds__(kResThreads) k_na_rows(
    const double *__restrict__ B, const double *__restrict__ H, double *__restrict__ F,
    const int32_t *__restrict__ in_rp, const int32_t *__restrict__ in_col, const int32_t *__restrict__ long_rows,
    const int32_t *__restrict__ long_seg0, int n_long, const double *__restrict__ seg_part,
    const double *__restrict__ g, int64_t n, double *__restrict__ part_sum, unsigned int *__restrict__ counter,
    double *__restrict__ result) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double lsum = 0.0;
    auto emit = [&](int64_t k, double acc) {
        const double f = B[k] + acc - H[k];
        F[k] = f;
        lsum += fabs(f);
    };
    for (int64_t base = warp * 32; base < n; base += nwarps * 32) {
        const int64_t k = base + lane;
        int32_t b = 0, e = 0;
        if (k < n) { b = in_rp[k]; e = in_rp[k + 1]; }
        const int len = e - b;
        double acc = 0.0;
        if (len <= 32)
            for (int32_t q = b; q < e; ++q) acc += g[in_col[q]];
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
    for (int64_t r = warp; r < n_long; r += nwarps) {
        const int32_t s0 = long_seg0[r], s1 = long_seg0[r + 1];
        double part = 0.0;
        for (int32_t s = s0 + lane; s < s1; s += 32) part += seg_part[s];
        part = warp_sum(part);
        if (lane == 0) emit(long_rows[r], part);
    }
    double m = 0.0;
    block_sum_max<kResThreads>(lsum, m);
    if (threadIdx.x == 0) part_sum[blockIdx.x] = lsum;
    if (!last_block(counter)) return;
    double s = 0.0;
    for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) s += part_sum[i];
    block_sum_max<kResThreads>(s, m);
    if (threadIdx.x == 0) *result = s;
}

// Device address of the scratch array on the current device (resolved once
// per device, with that device current).
di_status scratch_address(unsigned char **out) {
    int dev = -1;
    DI_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("di_residual_noalloc: device %d outside the supported range [0, %d)", dev, kMaxDevices);
        return DI_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("di_residual_noalloc: cudaGetSymbolAddress of the scratch array failed on device %d: %s",
                      dev, cudaGetErrorString(e));
            return DI_ECUDA;
        }
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return DI_OK;
}

}  // namespace
}  // namespace di

using namespace di;

extern "C" DI_API di_status di_residual_noalloc(const di_graph *g, const double *B, double d, const double *H,
                                               double *F, double *r_l1, void *stream) {
    di::NvtxRange nvtx_range("di_residual_noalloc");
    clear_error();
    if (!g || !B || !H || !F) { set_error("di_residual_noalloc: NULL argument"); return DI_EINVAL; }
    if (!(d > 0.0 && d < 1.0)) { set_error("di_residual_noalloc: d = %g outside (0, 1)", d); return DI_EINVAL; }
    if (g->n > kMaxN) {
        set_error("di_residual_noalloc: n = %lld exceeds the fixed scratch capacity of %lld nodes "
                  "(use di_residual)", (long long)g->n, (long long)kMaxN);
        return DI_EINVAL;
    }
    if (g->n_seg > kMaxSeg) {
        set_error("di_residual_noalloc: %d in-row segments exceed the fixed scratch capacity of %d "
                  "(use di_residual)", g->n_seg, kMaxSeg);
        return DI_EINVAL;
    }
    int dev = -1;
    DI_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != g->device) {
        set_error("di_residual_noalloc: graph lives on device %d, current is %d", g->device, dev);
        return DI_EINVAL;
    }
    unsigned char *base = nullptr;
    DI_TRY(scratch_address(&base));
    double *gvec = reinterpret_cast<double *>(base + kOffG);
    double *seg = reinterpret_cast<double *>(base + kOffSeg);
    double *part = reinterpret_cast<double *>(base + kOffPart);
    unsigned int *counter = reinterpret_cast<unsigned int *>(base + kOffCounter);
    double *result = reinterpret_cast<double *>(base + kOffResult);

    cudaStream_t s = as_stream(stream);
    const int grid = std::min(kMaxBlocks, std::max(1, g->num_sms * 4));
    DI_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned int), s));
    k_na_prep<<<grid, kResThreads, 0, s>>>(g->rp, H, d, g->n, gvec);
    if (g->n_seg > 0)
        k_na_seg<<<std::min(g->n_seg, grid), kResThreads, 0, s>>>(g->in_rp, g->in_col, g->long_rows, g->seg_row,
                                                                   g->seg_beg, g->n_seg, gvec, seg);
    k_na_rows<<<grid, kResThreads, 0, s>>>(B, H, F, g->in_rp, g->in_col, g->long_rows, g->long_seg0,
                                           g->n_long_rows, seg, gvec, g->n, part, counter, result);
    DI_CUDA_TRY(cudaGetLastError());
    if (r_l1) {
        DI_CUDA_TRY(cudaMemcpyAsync(r_l1, result, sizeof(double), cudaMemcpyDeviceToHost, s));
        DI_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return DI_OK;
}
