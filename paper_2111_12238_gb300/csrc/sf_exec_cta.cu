// Single-CTA executor (exec_mode 5, one right-hand side): every instance of the system (the
// whole system for sf_inspect, each independent instance of a block-diagonal batch) runs its
// joint DAG on one CTA, with no waits on other CTAs. A CTA stages into shared memory what fits
// of, in this order: the right-hand side (as x), the level segments and vertex order of its
// block of the row-block order (one block per instance), and L's row pointers, columns and
// values with each diagonal entry replaced by its reciprocal. What does not fit is read from
// global memory, x then living in the output buffer. The CTA walks its segments: the SpTRSV rows
// of a segment are independent of each other, so the threads take one row each, read the x_j
// they need, and a CTA barrier separates the segments. With everything staged, nothing on that
// dependence chain touches global memory. The intermediate x stays on chip: the barrier between
// wavefronts is a CTA barrier instead of a hand-off through L2. The second kernel's (SpMV) rows
// are sinks of the joint DAG. For a single system they run on helper CTAs of the same
// (cooperative) launch, on other SMs, while the solve goes on: the solving CTA also publishes
// each x_i by value (one relaxed store into a flag buffer whose reset pattern means "not yet",
// no fence); a helper thread loads an SpMV row's pattern and first values, then polls the x_j it
// needs (bounded) and adds them up. The SpMV's FP64 work then neither competes with the solve
// for the one SM's FP64 pipe nor follows it. The last CTA of the launch to finish resets the
// flag buffer for the next launch. For a batch (one
// block per instance, launched costliest first) an instance's SpMV rows run after its last
// wavefront on its own CTA, several rows per thread at once with x on chip, M prefetched into
// L2 while the block was staged.
#include <algorithm>
#include <atomic>
#include <mutex>

#include "sf_exec.cuh"

namespace sf {

namespace {

constexpr int kCtaMaxThreads = 1024;
constexpr int kStageUnroll = 8;    // independent loads in flight per thread while staging
constexpr int kMaxDevices = 64;
constexpr int kRowsInFlight = 4;   // SpMV rows a thread works on together after the solve
constexpr int kLine = 128;         // bytes per L2 prefetch

__device__ __forceinline__ double unset_value(double) { return __longlong_as_double(-1LL); }
__device__ __forceinline__ float unset_value(float) { return __uint_as_float(0xffffffffu); }

// Asks L2 for the bytes [p, p + bytes) of a global array, one line per request, spread over the
// CTA's threads (addresses stay inside the array).
__device__ __forceinline__ void prefetch_l2(const void *p, size_t bytes) {
    const char *c = (const char *)p;
    for (size_t o = (size_t)threadIdx.x * kLine; o < bytes; o += (size_t)blockDim.x * kLine)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(c + o));
}

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
// 3 x, the order and L. Shared-memory layout, each part 16-byte aligned: x[r1 - r0] (T),
// segment pointers [s1 - s0 + 1], order [p1 - p0], L values [e1 - e0] (T), L columns [e1 - e0]
// (relative to r0), L row pointers [r1 - r0 + 1] (relative to e0).
template <typename T, int LV>
__device__ void cta_block(const ExecArgs &a, int mode, int r0, int r1, int p0, int p1, int s0, int s1, int e0, int e1,
                          T *vb, unsigned char *smem) {
    const bool publish = vb != nullptr;
    const int nr = r1 - r0;
    const int ne = e1 - e0;
    T *xg = mode == M_TRSV ? (T *)a.y : (T *)a.xs;   // x in global memory (the output)
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
    if (mode == M_TRSV_SPMV && !publish) {
        // M's rows of the block, read after the solve: on their way to L2 meanwhile
        const int m0 = __ldg(a.Mrp + r0), m1 = __ldg(a.Mrp + r1);
        prefetch_l2(a.Mrp + r0, sizeof(int) * ((size_t)nr + 1));
        prefetch_l2(a.Mci + m0, sizeof(int) * (size_t)(m1 - m0));
        prefetch_l2((const T *)a.Mv + m0, sizeof(T) * (size_t)(m1 - m0));
    }
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
    const int tid = threadIdx.x;
    for (int g = s0; g < s1; ++g) {
        const int q0 = LV >= 2 ? sseg[g - s0] : a.seg_ptr[g];
        const int q1 = LV >= 2 ? sseg[g - s0 + 1] : a.seg_ptr[g + 1];
        for (int q = q0 + tid; q < q1; q += blockDim.x) {
            const unsigned o = (unsigned)(LV >= 2 ? sord[q - p0] : a.order[q]);
            if (o >> 31) continue;   // SpMV row: after the last wavefront
            // SpTRSV row: x_i = (b_i - sum_{j<i} L_ij x_j) / L_ii
            const int row = (int)o;
            if constexpr (LV >= 3) {
                const int li = row - r0;
                const int rs = srp[li], dg = srp[li + 1] - 1;
                // b_i - L_i1 x_1 - L_i2 x_2 - ...: one dependent FP64 operation per entry
                T t = sx[li];
                for (int e = rs; e < dg; ++e) t = fma(-slv[e], sx[slc[e]], t);
                t *= slv[dg];
                sx[li] = t;
                if (publish) put_value(vb + row, t);
            } else {
                const int rs = __ldg(a.Lrp + row), dg = __ldg(a.Lrp + row + 1) - 1;
                T acc = T(0);
                for (int e = rs; e < dg; ++e) {
                    const int j = __ldg(a.Lci + e);
                    acc += __ldg(Lv + e) * (LV >= 1 ? sx[j - r0] : xg[j]);
                }
                const T d = __ldg(Lv + dg);
                if (d == T(0)) record_error(a.st, SF_ERR_NONFINITE, row);
                T xi;
                if constexpr (LV >= 1) {
                    xi = (sx[row - r0] - acc) / d;
                    sx[row - r0] = xi;
                } else {
                    xi = (xg[row] - acc) / d;
                    xg[row] = xi;
                }
                if (publish) put_value(vb + row, xi);
            }
        }
        __syncthreads();
    }
    if constexpr (LV >= 1)
        for (int i = tid; i < nr; i += blockDim.x) xg[r0 + i] = sx[i];
    if (mode != M_TRSV_SPMV || publish) return;
    // y = M x over the block's rows: kRowsInFlight rows per thread at a time, their entries
    // loaded together
    constexpr int R = kRowsInFlight;
    const T *Mv = (const T *)a.Mv;
    T *y = (T *)a.y;
    for (int i0 = r0 + tid; i0 < r1; i0 += R * blockDim.x) {
        int ms[R], me[R];
        int len = 0;
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int i = i0 + u * blockDim.x;
            ms[u] = i < r1 ? __ldg(a.Mrp + i) : 0;
            me[u] = i < r1 ? __ldg(a.Mrp + i + 1) : 0;
            len = max(len, me[u] - ms[u]);
        }
        T acc[R];
#pragma unroll
        for (int u = 0; u < R; ++u) acc[u] = T(0);
        for (int t = 0; t < len; ++t) {
#pragma unroll
            for (int u = 0; u < R; ++u)
                if (ms[u] + t < me[u]) {
                    const int j = __ldg(a.Mci + ms[u] + t);
                    acc[u] += __ldg(Mv + ms[u] + t) * (LV >= 1 ? sx[j - r0] : xg[j]);
                }
        }
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < r1) y[i] = acc[u];
        }
    }
}

// Runs one block with as much of it staged as `budget` bytes allow.
template <typename T>
__device__ __forceinline__ void cta_dispatch(const ExecArgs &a, int mode, int r0, int r1, int p0, int p1, int s0,
                                             int s1, int e0, int e1, T *vb, unsigned budget, unsigned char *smem) {
    const size_t nr = (size_t)(r1 - r0), ne = (size_t)(e1 - e0);
    const size_t need1 = align16(sizeof(T) * nr);
    const size_t need2 = need1 + align16(sizeof(int) * ((size_t)(s1 - s0) + 1)) + align16(sizeof(int) * (size_t)(p1 - p0));
    const size_t need3 = need2 + align16(sizeof(T) * ne) + align16(sizeof(int) * ne) + align16(sizeof(int) * (nr + 1));
    if (need3 <= budget) cta_block<T, 3>(a, mode, r0, r1, p0, p1, s0, s1, e0, e1, vb, smem);
    else if (need2 <= budget) cta_block<T, 2>(a, mode, r0, r1, p0, p1, s0, s1, e0, e1, vb, smem);
    else if (need1 <= budget) cta_block<T, 1>(a, mode, r0, r1, p0, p1, s0, s1, e0, e1, vb, smem);
    else cta_block<T, 0>(a, mode, r0, r1, p0, p1, s0, s1, e0, e1, vb, smem);
}

// Helper CTA h (of `helpers`) of a single-system SpTRSV -> SpMV launch: every (helpers *
// blockDim)-th position of the order from its own offset (so rows come roughly in the order
// their inputs are solved); an SpMV row's pattern and first kHelpPrefetch values are loaded,
// then its x_j are read from the flag buffer vb, the first kHelpPrefetch together, each
// polled again until it is set (bounded by the launch's timeout).
constexpr int kHelpPrefetch = 6;
template <typename T>
__device__ __forceinline__ bool poll_value(const T *p, T &v, const ExecArgs &a, unsigned long long &t0, int row) {
    for (unsigned it = 0;; ++it) {
        v = ld_relaxed_val(p);
        if (!is_unset(v)) return true;
        __nanosleep(32);
        if ((it & 15u) == 15u) {
            const unsigned long long now = global_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > a.timeout_ns) {
                record_error(a.st, SF_ERR_TIMEOUT, row);
                return false;
            }
        }
    }
}
template <typename T>
__device__ void cta_helper(const ExecArgs &a, int h, int helpers, int p0, int p1, const T *vb) {
    const T *Mv = (const T *)a.Mv;
    T *y = (T *)a.y;
    constexpr int P = kHelpPrefetch;
    const int stride = helpers * (int)blockDim.x;
    for (int q = p0 + h * (int)blockDim.x + (int)threadIdx.x; q < p1; q += stride) {
        const unsigned o = (unsigned)__ldg(a.order + q);
        if (!(o >> 31)) continue;
        const int row = (int)(o & 0x7fffffffu);
        const int ms = __ldg(a.Mrp + row), me = __ldg(a.Mrp + row + 1);
        int jc[P];
        T mv[P];
#pragma unroll
        for (int u = 0; u < P; ++u) {
            jc[u] = ms + u < me ? __ldg(a.Mci + ms + u) : row;
            mv[u] = ms + u < me ? __ldg(Mv + ms + u) : T(0);
        }
        // the first P operands are loaded together and only the unpublished ones polled again
        int jw[P];
        T xv[P];
#pragma unroll
        for (int u = 0; u < P; ++u) jw[u] = ms + u < me ? jc[u] : -1;
        if (!wait_values<T, P>(vb, jw, xv, a.st, a.timeout_ns, row)) return;
        unsigned long long t0 = 0;
        T acc = T(0);
#pragma unroll
        for (int u = 0; u < P; ++u)
            if (ms + u < me) acc += mv[u] * xv[u];
        for (int e = ms + P; e < me; ++e) {
            T xv;
            if (!poll_value(vb + __ldg(a.Mci + e), xv, a, t0, row)) return;
            acc += __ldg(Mv + e) * xv;
        }
        y[row] = acc;
    }
}

// One CTA per block of the per-instance row-block order (block bperm[blockIdx.x]); `budget`
// bytes of dynamic shared memory decide what the block stages. With helpers > 0 (one block):
// CTA 0 solves and publishes x into the flag buffer vb, CTAs 1 .. helpers run the SpMV rows,
// and the last CTA to finish resets vb for the next launch.
template <typename T>
__global__ void __launch_bounds__(kCtaMaxThreads, 1)
    k_cta_exec(const ExecArgs a, int mode, const int *__restrict__ inst_ptr, const int *__restrict__ bperm,
               unsigned budget, int helpers, T *vb) {
    extern __shared__ __align__(16) unsigned char smem[];
    if (helpers > 0) {
        const int r0 = __ldg(inst_ptr), r1 = __ldg(inst_ptr + 1);
        const int p0 = __ldg(a.block_ptr), p1 = __ldg(a.block_ptr + 1);
        const int s0 = __ldg(a.block_seg), s1 = __ldg(a.block_seg + 1);
        if (blockIdx.x == 0) {
            const int e0 = __ldg(a.Lrp + r0), e1 = __ldg(a.Lrp + r1);
            cta_dispatch<T>(a, mode, r0, r1, p0, p1, s0, s1, e0, e1, vb, budget, smem);
        } else {
            cta_helper<T>(a, (int)blockIdx.x - 1, helpers, p0, p1, vb);
        }
        __shared__ bool last;
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            last = atomicAdd(&a.st->cta_exit, 1u) == gridDim.x - 1;
        }
        __syncthreads();
        if (last) {
            // every CTA is done with vb: back to the reset pattern (all bits set)
            __threadfence();
            for (int i = r0 + (int)threadIdx.x; i < r1; i += blockDim.x) st_relaxed_val(vb + i, unset_value(T(0)));
            if (threadIdx.x == 0) st_relaxed_u32(&a.st->cta_exit, 0u);
        }
        return;
    }
    const int blk = bperm ? __ldg(bperm + blockIdx.x) : (int)blockIdx.x;
    const int r0 = __ldg(inst_ptr + blk), r1 = __ldg(inst_ptr + blk + 1);
    const int p0 = __ldg(a.block_ptr + blk), p1 = __ldg(a.block_ptr + blk + 1);
    const int s0 = __ldg(a.block_seg + blk), s1 = __ldg(a.block_seg + blk + 1);
    const int e0 = __ldg(a.Lrp + r0), e1 = __ldg(a.Lrp + r1);
    cta_dispatch<T>(a, mode, r0, r1, p0, p1, s0, s1, e0, e1, (T *)nullptr, budget, smem);
}

}  // namespace

// Launches the single-CTA executor over the a.n_blocks blocks of the per-instance order:
// cta_per_sm CTAs of 1024 / cta_per_sm threads share an SM (0: one when the blocks fit in one
// wave, else two), each with an equal share of the SM's shared memory.
cudaError_t launch_cta_exec(int mode, int dtype, const int *inst_ptr, const int *bperm, int cta_per_sm, int sms,
                            void *vbuf, cudaStream_t s, const ExecArgs &a, cudaEvent_t ev_start, cudaEvent_t ev_stop) {
    int dev = 0;
    cudaGetDevice(&dev);
    const int cps = cta_per_sm > 0 ? cta_per_sm : (a.n_blocks > sms ? 2 : 1);
    const int threads = kCtaMaxThreads / cps;
    const void *f = dtype == 0 ? (const void *)k_cta_exec<double> : (const void *)k_cta_exec<float>;
    // device limits and the kernel's static shared memory, looked up once per device and type
    // (the per-call queries cost microseconds on a launch that takes tens of them)
    struct Limits {
        int smax, ssm;
        long long stat;
    };
    static std::mutex mu;
    static Limits lim[kMaxDevices][2];
    static bool have[kMaxDevices][2];
    Limits L{};
    cudaError_t e = cudaSuccess;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev < kMaxDevices && have[dev][dtype]) {
            L = lim[dev][dtype];
        } else {
            cudaDeviceGetAttribute(&L.smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            cudaDeviceGetAttribute(&L.ssm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
            cudaFuncAttributes fa{};
            e = cudaFuncGetAttributes(&fa, f);
            if (e != cudaSuccess) return e;
            L.stat = (long long)fa.sharedSizeBytes;
            if (dev < kMaxDevices) {
                lim[dev][dtype] = L;
                have[dev][dtype] = true;
            }
        }
    }
    const int smax = L.smax, ssm = L.ssm;
    // 1 KB of each CTA's shared memory is reserved by the system; the kernel's static shared
    // memory comes out of the same budget
    const long long stat = L.stat;
    const int budget = (int)(std::min<long long>(smax - stat, (long long)ssm / cps - 1024 - stat) & ~15LL);
    if (budget < 16) return cudaErrorInvalidValue;
    // the opt-in shared-memory size is set once per device and kernel to the largest request
    static std::atomic<int> opted[kMaxDevices][2];
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
    // a single SpTRSV -> SpMV system: helper CTAs for the SpMV rows, about 2048 positions each
    int helpers = 0;
    if (mode == M_TRSV_SPMV && a.n_blocks == 1 && vbuf) {
        const long long nv = 2LL * a.n;
        helpers = (int)std::min<long long>(std::max(sms - 1, 1), std::max(1LL, (nv + 2047) / 2048));
    }
    void *vb = helpers > 0 ? vbuf : nullptr;
    void *args[] = {(void *)&a, (void *)&mode, (void *)&inst_ptr, (void *)&bperm, (void *)&ub, (void *)&helpers,
                    (void *)&vb};
    if (ev_start && (e = cudaEventRecord(ev_start, s)) != cudaSuccess) return e;
    if (helpers > 0) {
        // the helpers wait for CTA 0: every CTA of the launch must be resident
        e = cudaLaunchCooperativeKernel(f, dim3((unsigned)(1 + helpers)), dim3((unsigned)threads), args,
                                        (size_t)budget, s);
        if (e != cudaSuccess) return e;
    } else if (a.n_blocks > 0 &&
               (e = cudaLaunchKernel(f, dim3((unsigned)a.n_blocks), dim3((unsigned)threads), args, (size_t)budget,
                                     s)) != cudaSuccess) {
        return e;
    }
    if (ev_stop) return cudaEventRecord(ev_stop, s);
    return cudaSuccess;
}

}  // namespace sf
