// probe.cu - ceilings of the memory operations the push and the exact residual
// are built from, measured on the device that runs them.
//
// The push of a threshold level (Sec. 2.4 selection, Eq. defF update) is one
// red.global.add per out-edge into the fluid vector at an irregular target,
// and the exact residual (Eqs. defF/defH invariant) is one gather of s_j H_j
// per in-edge.  Their roofline is therefore not only the HBM copy bandwidth:
// with the fluid held in L2, the binding limit is the rate at which the SMs
// and the L2 process scattered single-word operations.  di_probe_l2 measures
// that rate for the exact operation the kernels issue (same cache-policy
// hint, same word size), over an array the caller sizes (a 2^24-float array
// is the 64 MB fluid of a 2^24-node graph).
#include <algorithm>
#include <cmath>

#include "di_internal.cuh"

namespace di {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeUnroll = 8;

// Per-thread stream of pseudo-random slots: a 32-bit LCG whose output is
// mixed (xorshift of the high bits down) so that low bits are not periodic;
// slot = mixed & mask with mask = slots - 1 (slots a power of two).
__device__ __forceinline__ uint32_t next_slot(uint32_t &x, uint32_t mask) {
    x = x * 1664525u + 1013904223u;
    uint32_t y = x ^ (x >> 15);
    y *= 0x2c1b3c6du;
    y ^= y >> 12;
    return y & mask;
}

// mode 0: red.global.add.f32 at random slots (L2 evict-last, as the push)
// mode 1: red.global.add.f64 at random slots (the FP64-fluid push)
// mode 2: 4-byte loads at random slots (gathers), summed so they stay live
// mode 3: red.global.add.f32 at consecutive slots per warp (coalesced), the
//         contrast that shows the per-address cost of the scattered form
// mode 4: atom.global.add.f32 at random slots (fetch-and-add: the old value
//         returns to the thread and is summed so that it stays live)
template <int kMode>
__global__ void __launch_bounds__(kProbeThreads) k_probe(void *arr, uint32_t mask, int iters, uint32_t seed,
                                                         float *sink) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t x = (t + 1u) * 0x9E3779B9u ^ seed;
    const uint64_t keep = l2_keep_policy();
    float acc = 0.f;
    const uint32_t nthreads = gridDim.x * blockDim.x;
    for (int k = 0; k < iters; k += kProbeUnroll) {
        uint32_t slot[kProbeUnroll];
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) {
            if (kMode == 3) slot[u] = (t + (uint32_t)(k + u) * nthreads) & mask;
            else slot[u] = next_slot(x, mask);
        }
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) {
            if (kMode == 0 || kMode == 3) red_add_keep(static_cast<float *>(arr) + slot[u], 1.0f, keep);
            else if (kMode == 1) red_add_keep(static_cast<double *>(arr) + slot[u], 1.0, keep);
            else if (kMode == 4) acc += atom_add_keep(static_cast<float *>(arr) + slot[u], 1.0f, keep);
            else acc += __ldcg(static_cast<const float *>(arr) + slot[u]);
        }
    }
    if ((kMode == 2 || kMode == 4) && acc == -1.0f) *sink = acc;   // never true (values >= 0): keeps the results
}

}  // namespace
}  // namespace di

using namespace di;

extern "C" DI_API di_status di_probe_l2(int mode, int64_t slots, int64_t ops, double *ops_per_s, double *seconds,
                                        void *stream) {
    clear_error();
    if (mode < 0 || mode > 4) { set_error("di_probe_l2: mode %d outside [0, 4]", mode); return DI_EINVAL; }
    if (slots < 1024 || slots > (int64_t(1) << 30) || (slots & (slots - 1))) {
        set_error("di_probe_l2: slots = %lld must be a power of two in [2^10, 2^30]", (long long)slots);
        return DI_EINVAL;
    }
    if (ops < 1 || ops > (int64_t(1) << 40)) { set_error("di_probe_l2: ops = %lld outside [1, 2^40]", (long long)ops); return DI_EINVAL; }
    if (!ops_per_s) { set_error("di_probe_l2: NULL ops_per_s"); return DI_EINVAL; }
    cudaStream_t s = as_stream(stream);
    int dev = 0, sms = 0, per_sm = 0;
    DI_CUDA_TRY(cudaGetDevice(&dev));
    DI_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const void *fn = mode == 0 ? (const void *)k_probe<0> : mode == 1 ? (const void *)k_probe<1>
                   : mode == 2 ? (const void *)k_probe<2> : mode == 3 ? (const void *)k_probe<3>
                                                                       : (const void *)k_probe<4>;
    DI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kProbeThreads, 0));
    const int grid = std::max(1, per_sm) * sms;
    const int64_t threads = (int64_t)grid * kProbeThreads;
    int64_t iters = (ops + threads - 1) / threads;
    iters = (iters + kProbeUnroll - 1) / kProbeUnroll * kProbeUnroll;
    if (iters > (int64_t(1) << 30)) { set_error("di_probe_l2: too many ops per thread"); return DI_EINVAL; }
    const size_t bytes = (size_t)slots * (mode == 1 ? sizeof(double) : sizeof(float));
    void *arr = nullptr;
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    di_status rc = DI_OK;
    float best = 0.f;
    auto fail = [&](cudaError_t e, const char *what) {
        set_error("di_probe_l2: %s failed: %s", what, cudaGetErrorString(e));
        rc = e == cudaErrorMemoryAllocation ? DI_ENOMEM : DI_ECUDA;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&arr, bytes)) != cudaSuccess) { fail(e, "cudaMalloc"); goto done; }
    if ((e = cudaMalloc(&sink, sizeof(float))) != cudaSuccess) { fail(e, "cudaMalloc"); goto done; }
    if ((e = cudaMemsetAsync(arr, 0, bytes, s)) != cudaSuccess) { fail(e, "cudaMemsetAsync"); goto done; }
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        fail(e, "cudaEventCreate");
        goto done;
    }
    // one warm-up launch (the array enters L2), then the best of three
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, s);
        const uint32_t mask = (uint32_t)(slots - 1), seed = 0x5bd1e995u * (uint32_t)(rep + 1);
        switch (mode) {
            case 0: k_probe<0><<<grid, kProbeThreads, 0, s>>>(arr, mask, (int)iters, seed, sink); break;
            case 1: k_probe<1><<<grid, kProbeThreads, 0, s>>>(arr, mask, (int)iters, seed, sink); break;
            case 2: k_probe<2><<<grid, kProbeThreads, 0, s>>>(arr, mask, (int)iters, seed, sink); break;
            case 3: k_probe<3><<<grid, kProbeThreads, 0, s>>>(arr, mask, (int)iters, seed, sink); break;
            default: k_probe<4><<<grid, kProbeThreads, 0, s>>>(arr, mask, (int)iters, seed, sink); break;
        }
        cudaEventRecord(e1, s);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { fail(e, "k_probe"); goto done; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    *ops_per_s = (double)threads * (double)iters / (best * 1e-3);
    if (seconds) *seconds = best * 1e-3;
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (arr) cudaFree(arr);
    if (sink) cudaFree(sink);
    return rc;
}
