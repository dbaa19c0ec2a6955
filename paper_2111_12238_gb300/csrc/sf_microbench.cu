// Measurement kernels for the roofline of the executor (not part of the method): the FP64 /
// FP32 fused multiply-add rate of this GPU, and the latency of one hand-off of a value between
// two SMs through L2 (the cheapest possible dependence hop: one relaxed store, one polling
// relaxed load, no fences). Timed by the caller with CUDA events around the launch.
#include <algorithm>

#include "sf_exec.cuh"

#define SF_API extern "C" __attribute__((visibility("default")))

namespace sf {
namespace {

constexpr int kFmaChains = 8;   // independent accumulators per thread (covers the FMA latency)

template <typename T>
__global__ void __launch_bounds__(256) k_fma_rate(int iters, T seed, T *sink) {
    T acc[kFmaChains];
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) acc[c] = seed + T(threadIdx.x + c);
    const T m = T(0.999999), ad = T(1e-7);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kFmaChains; ++c) acc[c] = fma(acc[c], m, ad);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) s += acc[c];
    if (s == T(-1)) sink[threadIdx.x] = s;   // never true for these operands; keeps the chains live
}

// Ping-pong of one word between block 0 and block 1 (one lane each) through L2: block 0 writes
// the odd values, block 1 the even ones, each after seeing the previous value. Both blocks are
// resident (cooperative launch, one block per SM by its shared-memory request). Every poll is
// bounded: after timeout_ns without progress the lane records the failure in out[1] and stops;
// the other lane then runs out of time as well. out[0] = elapsed ns of `hops` hand-offs.
__global__ void k_hop(int hops, unsigned *word, unsigned long long timeout_ns, unsigned long long *out) {
    extern __shared__ unsigned char pad[];
    (void)pad;
    if (threadIdx.x != 0 || blockIdx.x > 1) return;
    const unsigned me = blockIdx.x;
    unsigned long long t_start = global_ns();
    unsigned long long t_last = t_start;
    for (unsigned v = me; v < (unsigned)hops; v += 2) {
        // wait until the word holds v (the previous hand-off), then write v + 1
        while (ld_relaxed_u32(word) != v) {
            const unsigned long long t = global_ns();
            if (t - t_last > timeout_ns) {
                atomicExch(out + 1, 1ull);
                return;
            }
        }
        if (v == 0 && me == 0) t_start = global_ns();
        st_relaxed_u32(word, v + 1);
        t_last = global_ns();
    }
    if (me == 0) {
        // the last hand-off is complete when the word reaches hops
        while (ld_relaxed_u32(word) != (unsigned)hops && (hops & 1) == 0) {
            if (global_ns() - t_last > timeout_ns) {
                atomicExch(out + 1, 1ull);
                return;
            }
        }
        out[0] = global_ns() - t_start;
    }
}

}  // namespace
}  // namespace sf

using namespace sf;

// FMA-rate kernel: blocks x 256 threads, each running kFmaChains independent FMA chains of
// `iters` steps (2 flops each): flops = blocks * 256 * 8 * iters * 2. sink: device buffer of
// at least 256 elements of the dtype (never written in practice). Asynchronous on `stream`.
SF_API sf_status sf_bench_fma(sf_dtype dt, int32_t blocks, int32_t iters, void *sink, void *stream) {
    if ((dt != SF_F64 && dt != SF_F32) || blocks < 1 || iters < 1 || !sink) return SF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (dt == SF_F64) k_fma_rate<double><<<blocks, 256, 0, s>>>(iters, 1.0, (double *)sink);
    else k_fma_rate<float><<<blocks, 256, 0, s>>>(iters, 1.0f, (float *)sink);
    return cudaGetLastError() == cudaSuccess ? SF_OK : SF_ERR_CUDA;
}

// Hand-off latency kernel: `hops` (even, >= 2) alternating hand-offs of one word between two
// SMs. word: one zeroed device uint32; out: two zeroed device uint64 (out[0] receives the
// elapsed ns, out[1] = 1 if a poll ran out of time). Asynchronous on `stream`.
SF_API sf_status sf_bench_hop(int32_t hops, void *word, void *out, void *stream) {
    if (hops < 2 || (hops & 1) || !word || !out) return SF_ERR_INVALID_ARG;
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // more than half of an SM's shared memory: the two blocks land on two SMs
    const int smem = std::max(0, smem_max / 2 + 1024);
    if (cudaFuncSetAttribute((const void *)k_hop, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return SF_ERR_CUDA;
    unsigned long long tmo = 1000000000ull;
    int h = hops;
    unsigned *w = (unsigned *)word;
    unsigned long long *o = (unsigned long long *)out;
    void *args[] = {(void *)&h, (void *)&w, (void *)&tmo, (void *)&o};
    if (cudaLaunchCooperativeKernel((const void *)k_hop, dim3(2), dim3(32), args, (size_t)smem, (cudaStream_t)stream) !=
        cudaSuccess)
        return SF_ERR_CUDA;
    return SF_OK;
}
