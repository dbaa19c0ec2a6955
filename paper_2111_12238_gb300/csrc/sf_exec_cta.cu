// Single-CTA executor (exec_mode 5, one right-hand side): every instance of the system (the
// whole system for sf_inspect, each independent instance of a block-diagonal batch) runs its
// joint DAG on one CTA, with no waits on other CTAs. A CTA stages into shared memory what fits
// of, in this order: the right-hand side (as x), the level segments and vertex order of its
// block of the row-block order (one block per instance), and L's row pointers, columns and
// values with each diagonal entry replaced by its reciprocal. What does not fit is read from
// global memory, x then living in the output buffer. The CTA walks its segments: the SpTRSV rows
// of a segment are independent of each other, so the threads take one row each, read the x_j
// they need, and a barrier of those threads separates the segments. With everything staged,
// nothing on that dependence chain touches global memory. For SpTRSV -> SpMV a quarter of the
// warps run the second kernel's rows instead, concurrently with the solve: a row of segment g
// waits (in shared memory) until the solver threads have finished the segments before g, then
// reads M from global memory and x on chip, so M's loads overlap the solve rather than
// following it. x_save is written out after the last wavefront. The intermediate x never leaves
// the SM: the barrier between wavefronts is a CTA barrier instead of a hand-off through L2.
// Blocks are launched costliest first (most segments), so that the long instances start in the
// first wave of a batch. The only wait, on the solver's progress counter, is bounded.
#include <algorithm>
#include <atomic>

#include "sf_exec.cuh"

namespace sf {

namespace {

constexpr int kCtaMaxThreads = 1024;
constexpr int kStageUnroll = 8;    // independent loads in flight per thread while staging
constexpr int kMaxDevices = 64;
constexpr size_t kCtlBytes = 16;   // progress counter of the solver threads, ahead of the layout
constexpr int kSpmvPrefetch = 8;   // entries of an SpMV row loaded before its wait

__device__ __forceinline__ unsigned ld_relaxed_cta_shared(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_cta_shared(unsigned *p, unsigned v) {
    asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}
// barrier 1 among the first `count` threads (a multiple of 32) of the CTA
__device__ __forceinline__ void solver_barrier(int count) { asm volatile("bar.sync 1, %0;" ::"r"(count) : "memory"); }

__host__ __device__ __forceinline__ size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// dst[i] = src[i] - shift for i < n, with kStageUnroll loads in flight per thread.
template <typename E>
__device__ __forceinline__ void stage(E *__restrict__ dst, const E *__restrict__ src, long long n, E shift = E(0)) {
    for (long long base = threadIdx.x; base < n; base += (long long)kStageUnroll * blockDim.x) {
        E v[kStageUnroll];
#pragma unroll
        for (int u = 0; u < kStageUnroll; ++u) {
            const long long e = base + (long long)u * blockDim.x;
            if (e < n) v[u] = __ldg(src + e);
        }
#pragma unroll
        for (int u = 0; u < kStageUnroll; ++u) {
            const long long e = base + (long long)u * blockDim.x;
            if (e < n) dst[e] = v[u] - shift;
        }
    }
}

// One block (instance): rows [r0, r1), positions [p0, p1) of the order, segments [s0, s1),
// L entries [e0, e1). LV: 0 nothing staged (x in the output buffer), 1 x, 2 x and the order,
// 3 x, the order and L. Shared-memory layout after the kCtlBytes control word, each part
// 16-byte aligned: x[r1 - r0] (T), segment pointers [s1 - s0 + 1], order [p1 - p0], L values
// [e1 - e0] (T), L columns [e1 - e0] (relative to r0), L row pointers [r1 - r0 + 1] (relative
// to e0).
template <typename T, int LV>
__device__ void cta_block(const ExecArgs &a, int mode, int r0, int r1, int p0, int p1, int s0, int s1, int e0, int e1,
                          unsigned char *smem_all) {
    const int nr = r1 - r0;
    const int ne = e1 - e0;
    T *xg = mode == M_TRSV ? (T *)a.y : (T *)a.xs;   // x in global memory (the output)
    unsigned *done = (unsigned *)smem_all;           // segments the solver threads have finished
    unsigned char *smem = smem_all + kCtlBytes;
    size_t off = 0;
    T *sx = (T *)smem;
    off += align16(sizeof(T) * (size_t)nr);
    int *sseg = (int *)(smem + off);
    off += align16(sizeof(int) * ((size_t)(s1 - s0) + 1));
    int *sord = (int *)(smem + off);
    off += align16(sizeof(int) * (size_t)(p1 - p0));
    T *slv = (T *)(smem + off);
    off += align16(sizeof(T) * (size_t)ne);
    int *slc = (int *)(smem + off);
    off += align16(sizeof(int) * (size_t)ne);
    int *srp = (int *)(smem + off);
    const T *Lv = (const T *)a.Lv;
    const T *b = (const T *)a.b;
    if constexpr (LV >= 2) {
        stage<int>(sseg, a.seg_ptr + s0, (long long)(s1 - s0) + 1);
        stage<int>(sord, a.order + p0, p1 - p0);
    }
    if constexpr (LV >= 3) {
        stage<T>(slv, Lv + e0, ne);
        stage<int>(slc, a.Lci + e0, ne, r0);
        stage<int>(srp, a.Lrp + r0, (long long)nr + 1, e0);
    }
    // x starts as b (a row then subtracts its sum in place and scales)
    if constexpr (LV >= 1) stage<T>(sx, b + r0, nr);
    else
        for (int i = threadIdx.x; i < nr; i += blockDim.x) xg[r0 + i] = __ldg(b + r0 + i);
    if (threadIdx.x == 0) *done = 0u;
    __syncthreads();
    if constexpr (LV >= 3) {
        // diagonal entries to reciprocals, off the dependence chain
        for (int i = threadIdx.x; i < nr; i += blockDim.x) {
            const int dg = srp[i + 1] - 1;
            const T d = slv[dg];
            if (d == T(0)) record_error(a.st, SF_ERR_NONFINITE, r0 + i);
            slv[dg] = T(1) / d;
        }
        __syncthreads();
    }
    // solver threads: the SpTRSV rows; for SpTRSV -> SpMV the last quarter of the warps run the
    // SpMV rows concurrently
    const int ns = mode == M_TRSV_SPMV ? (int)blockDim.x - (int)blockDim.x / 4 : (int)blockDim.x;
    const int tid = threadIdx.x;
    if (tid < ns) {
        for (int g = s0; g < s1; ++g) {
            const int q0 = LV >= 2 ? sseg[g - s0] : a.seg_ptr[g];
            const int q1 = LV >= 2 ? sseg[g - s0 + 1] : a.seg_ptr[g + 1];
            for (int q = q0 + tid; q < q1; q += ns) {
                const unsigned o = (unsigned)(LV >= 2 ? sord[q - p0] : a.order[q]);
                if (o >> 31) continue;   // SpMV row
                // SpTRSV row: x_i = (b_i - sum_{j<i} L_ij x_j) / L_ii
                const int row = (int)o;
                if constexpr (LV >= 3) {
                    const int li = row - r0;
                    const int rs = srp[li], dg = srp[li + 1] - 1;
                    // b_i - L_i1 x_1 - L_i2 x_2 - ...: one dependent FP64 operation per entry
                    T t = sx[li];
                    for (int e = rs; e < dg; ++e) t = fma(-slv[e], sx[slc[e]], t);
                    sx[li] = t * slv[dg];
                } else {
                    const int rs = __ldg(a.Lrp + row), dg = __ldg(a.Lrp + row + 1) - 1;
                    T acc = T(0);
                    for (int e = rs; e < dg; ++e) {
                        const int j = __ldg(a.Lci + e);
                        acc += __ldg(Lv + e) * (LV >= 1 ? sx[j - r0] : xg[j]);
                    }
                    const T d = __ldg(Lv + dg);
                    if (d == T(0)) record_error(a.st, SF_ERR_NONFINITE, row);
                    if constexpr (LV >= 1) sx[row - r0] = (sx[row - r0] - acc) / d;
                    else xg[row] = (xg[row] - acc) / d;
                }
            }
            solver_barrier(ns);
            if (tid == 0) st_release_cta_shared(done, (unsigned)(g - s0 + 1));
        }
    } else {
        // SpMV rows: y_i = sum_j M_ij x_j. Each thread takes every nsp-th position of the block;
        // a row's pattern and first kSpmvPrefetch values are loaded before it waits until the
        // segments before its own are done, so only the on-chip x reads follow the wait.
        const int nsp = (int)blockDim.x - ns, st = tid - ns;
        const T *Mv = (const T *)a.Mv;
        T *y = (T *)a.y;
        constexpr int P = kSpmvPrefetch;
        int g = s0;             // segment of position q (q only grows)
        unsigned seen = 0;      // segments known to be done
        unsigned long long t0 = 0;
        for (int q = p0 + st; q < p1; q += nsp) {
            const unsigned o = (unsigned)(LV >= 2 ? sord[q - p0] : a.order[q]);
            if (!(o >> 31)) continue;
            while ((LV >= 2 ? sseg[g + 1 - s0] : a.seg_ptr[g + 1]) <= q) ++g;
            const int row = (int)(o & 0x7fffffffu);
            const int ms = __ldg(a.Mrp + row), me = __ldg(a.Mrp + row + 1);
            int jc[P];
            T mv[P];
#pragma unroll
            for (int u = 0; u < P; ++u) {
                jc[u] = ms + u < me ? __ldg(a.Mci + ms + u) : r0;
                mv[u] = ms + u < me ? __ldg(Mv + ms + u) : T(0);
            }
            if (seen < (unsigned)(g - s0)) {
                // poll with a short sleep (the solver warps keep the issue slots), then acquire
                bool ok = true;
                for (unsigned it = 0; (seen = ld_relaxed_cta_shared(done)) < (unsigned)(g - s0); ++it) {
                    __nanosleep(64);
                    if ((it & 15u) == 15u) {
                        const unsigned long long now = global_ns();
                        if (t0 == 0) t0 = now;
                        else if (now - t0 > a.timeout_ns) {
                            record_error(a.st, SF_ERR_TIMEOUT, row);
                            ok = false;
                            break;
                        }
                    }
                }
                if (!ok) break;
                asm volatile("fence.acq_rel.cta;" ::: "memory");
                t0 = 0;
            }
            T acc = T(0);
#pragma unroll
            for (int u = 0; u < P; ++u)
                if (ms + u < me) acc += mv[u] * (LV >= 1 ? sx[jc[u] - r0] : xg[jc[u]]);
            for (int e = ms + P; e < me; ++e) {
                const int j = __ldg(a.Mci + e);
                acc += __ldg(Mv + e) * (LV >= 1 ? sx[j - r0] : xg[j]);
            }
            y[row] = acc;
        }
    }
    __syncthreads();
    if constexpr (LV >= 1)
        for (int i = tid; i < nr; i += blockDim.x) xg[r0 + i] = sx[i];
}

// One CTA per block of the per-instance row-block order (block bperm[blockIdx.x]); `budget`
// bytes of dynamic shared memory decide what the block stages.
template <typename T>
__global__ void __launch_bounds__(kCtaMaxThreads, 1)
    k_cta_exec(const ExecArgs a, int mode, const int *__restrict__ inst_ptr, const int *__restrict__ bperm,
               unsigned budget) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int blk = bperm ? __ldg(bperm + blockIdx.x) : (int)blockIdx.x;
    const int r0 = __ldg(inst_ptr + blk), r1 = __ldg(inst_ptr + blk + 1);
    const int p0 = __ldg(a.block_ptr + blk), p1 = __ldg(a.block_ptr + blk + 1);
    const int s0 = __ldg(a.block_seg + blk), s1 = __ldg(a.block_seg + blk + 1);
    const int e0 = __ldg(a.Lrp + r0), e1 = __ldg(a.Lrp + r1);
    const size_t nr = (size_t)(r1 - r0), ne = (size_t)(e1 - e0);
    if (budget < kCtlBytes) return;   // the launcher never asks for less
    const size_t need1 = kCtlBytes + align16(sizeof(T) * nr);
    const size_t need2 = need1 + align16(sizeof(int) * ((size_t)(s1 - s0) + 1)) + align16(sizeof(int) * (size_t)(p1 - p0));
    const size_t need3 = need2 + align16(sizeof(T) * ne) + align16(sizeof(int) * ne) + align16(sizeof(int) * (nr + 1));
    if (need3 <= budget) cta_block<T, 3>(a, mode, r0, r1, p0, p1, s0, s1, e0, e1, smem);
    else if (need2 <= budget) cta_block<T, 2>(a, mode, r0, r1, p0, p1, s0, s1, e0, e1, smem);
    else if (need1 <= budget) cta_block<T, 1>(a, mode, r0, r1, p0, p1, s0, s1, e0, e1, smem);
    else cta_block<T, 0>(a, mode, r0, r1, p0, p1, s0, s1, e0, e1, smem);
}

}  // namespace

// Launches the single-CTA executor over the a.n_blocks blocks of the per-instance order:
// cta_per_sm CTAs of 1024 / cta_per_sm threads share an SM (0: one when the blocks fit in one
// wave, else two), each with an equal share of the SM's shared memory.
cudaError_t launch_cta_exec(int mode, int dtype, const int *inst_ptr, const int *bperm, int cta_per_sm, int sms,
                            cudaStream_t s, const ExecArgs &a, cudaEvent_t ev_start, cudaEvent_t ev_stop) {
    int dev = 0, smax = 0, ssm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&ssm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const int cps = cta_per_sm > 0 ? cta_per_sm : (a.n_blocks > sms ? 2 : 1);
    const int threads = kCtaMaxThreads / cps;
    // 1 KB of each CTA's shared memory is reserved by the system
    const int budget = (int)(std::min<long long>(smax, (long long)ssm / cps - 1024) & ~15LL);
    if (budget < 16) return cudaErrorInvalidValue;
    const void *f = dtype == 0 ? (const void *)k_cta_exec<double> : (const void *)k_cta_exec<float>;
    // the opt-in shared-memory size is set once per device and kernel to the largest request
    static std::atomic<int> opted[kMaxDevices][2];
    cudaError_t e = cudaSuccess;
    if (dev >= kMaxDevices || opted[dev][dtype].load() < budget) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, budget);
        if (e != cudaSuccess) return e;
        if (dev < kMaxDevices) {
            int cur = opted[dev][dtype].load();
            while (cur < budget && !opted[dev][dtype].compare_exchange_weak(cur, budget)) {
            }
        }
    }
    unsigned ub = (unsigned)budget;
    void *args[] = {(void *)&a, (void *)&mode, (void *)&inst_ptr, (void *)&bperm, (void *)&ub};
    if (ev_start && (e = cudaEventRecord(ev_start, s)) != cudaSuccess) return e;
    if (a.n_blocks > 0 &&
        (e = cudaLaunchKernel(f, dim3((unsigned)a.n_blocks), dim3((unsigned)threads), args, (size_t)budget, s)) !=
            cudaSuccess)
        return e;
    if (ev_stop) return cudaEventRecord(ev_stop, s);
    return cudaSuccess;
}

}  // namespace sf
