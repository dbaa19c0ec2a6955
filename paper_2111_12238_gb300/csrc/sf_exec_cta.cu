// Single-CTA executor for small systems (exec_mode 5, one right-hand side): the whole joint DAG
// runs on one SM. The CTA first stages into shared memory the right-hand side (as x), the level
// segments and the vertex order of the row-block order (one block holding every row) and, when
// they fit as well, L's row pointers, columns and values, with each diagonal entry replaced by
// its reciprocal. It then walks the segments: the SpTRSV rows of a segment are independent of
// each other, so the threads take one row each, read the x_j they need from shared memory, and a
// __syncthreads() separates the segments. Nothing on that dependence chain touches global memory
// when everything is staged: x_save is written out after the last wavefront, and the
// second-kernel (SpMV) rows, sinks of the joint DAG, run after it too, every thread on several
// rows at once with x still in shared memory (their latest placement in the fused order). The
// intermediate x never leaves the SM: the barrier between wavefronts is a CTA barrier instead of
// a hand-off through L2. No waits on other CTAs, so nothing to bound.
#include <algorithm>
#include <atomic>

#include "sf_exec.cuh"

namespace sf {

namespace {

constexpr int kCtaThreads = 1024;
constexpr int kStageUnroll = 8;   // independent loads in flight per thread while staging
constexpr int kMaxDevices = 64;
constexpr int kRowsInFlight = 4;   // SpMV rows a thread works on together after the solve

__device__ __forceinline__ size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// Copies n elements from global to shared memory with kStageUnroll loads in flight per thread.
template <typename E>
__device__ __forceinline__ void stage(E *__restrict__ dst, const E *__restrict__ src, long long n) {
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
            if (e < n) dst[e] = v[u];
        }
    }
}

// Shared-memory layout, each part 16-byte aligned: x[n] (T); when OS: segment pointers
// [segs + 1] and the vertex order [nv] (int); when LS: L values [nnz] (T, the diagonal entry of
// each row replaced by its reciprocal), L columns [nnz] (int), L row pointers [n + 1] (int).
template <typename T, bool OS, bool LS>
__global__ void __launch_bounds__(kCtaThreads, 1)
    k_cta_exec(const ExecArgs a, int mode, long long nnzL, long long nv, int segs) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = a.n;
    size_t off = 0;
    T *x = (T *)smem;
    off = align16(sizeof(T) * (size_t)n);
    int *s_seg = (int *)(smem + off);
    if (OS) off += align16(sizeof(int) * ((size_t)segs + 1));
    int *s_order = (int *)(smem + off);
    if (OS) off += align16(sizeof(int) * (size_t)nv);
    T *s_lv = (T *)(smem + off);
    if (LS) off += align16(sizeof(T) * (size_t)nnzL);
    int *s_lc = (int *)(smem + off);
    if (LS) off += align16(sizeof(int) * (size_t)nnzL);
    int *s_lrp = (int *)(smem + off);
    const T *Lv = (const T *)a.Lv;
    if constexpr (OS) {
        stage<int>(s_seg, a.seg_ptr, (long long)segs + 1);
        stage<int>(s_order, a.order, nv);
    }
    if constexpr (LS) {
        stage<T>(s_lv, Lv, nnzL);
        stage<int>(s_lc, a.Lci, nnzL);
        stage<int>(s_lrp, a.Lrp, (long long)n + 1);
    }
    // x starts as b (a row then subtracts its sum in place and scales)
    stage<T>(x, (const T *)a.b, n);
    __syncthreads();
    if constexpr (LS) {
        // diagonal entries to reciprocals, off the dependence chain
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int dg = s_lrp[i + 1] - 1;
            const T d = s_lv[dg];
            if (d == T(0)) record_error(a.st, SF_ERR_NONFINITE, i);
            s_lv[dg] = T(1) / d;
        }
        __syncthreads();
    }
    const int *seg = OS ? s_seg : a.seg_ptr;
    const int *ord = OS ? s_order : a.order;
    const int *rp = LS ? s_lrp : a.Lrp;
    const int *ci = LS ? s_lc : a.Lci;
    const T *lv = LS ? s_lv : Lv;
    for (int g = 0; g < segs; ++g) {
        const int q0 = seg[g], q1 = seg[g + 1];
        for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
            const unsigned o = (unsigned)ord[q];
            if (o >> 31) continue;   // SpMV row: after the last wavefront
            // SpTRSV row: x_i = (b_i - sum_{j<i} L_ij x_j) / L_ii
            const int row = (int)o;
            const int rs = rp[row], dg = rp[row + 1] - 1;
            T acc = T(0);
            for (int e = rs; e < dg; ++e) acc += lv[e] * x[ci[e]];
            if constexpr (LS) {
                x[row] = (x[row] - acc) * lv[dg];
            } else {
                const T d = lv[dg];
                if (d == T(0)) record_error(a.st, SF_ERR_NONFINITE, row);
                x[row] = (x[row] - acc) / d;
            }
        }
        __syncthreads();
    }
    T *out_x = mode == M_TRSV ? (T *)a.y : (T *)a.xs;
    if (out_x)
        for (int i = threadIdx.x; i < n; i += blockDim.x) out_x[i] = x[i];
    if (mode != M_TRSV_SPMV) return;
    // y = M x: kRowsInFlight rows per thread at a time, their entries loaded together
    constexpr int R = kRowsInFlight;
    const T *Mv = (const T *)a.Mv;
    T *y = (T *)a.y;
    for (int i0 = threadIdx.x; i0 < n; i0 += R * blockDim.x) {
        int ms[R], me[R];
        int len = 0;
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int i = i0 + u * blockDim.x;
            ms[u] = i < n ? __ldg(a.Mrp + i) : 0;
            me[u] = i < n ? __ldg(a.Mrp + i + 1) : 0;
            len = max(len, me[u] - ms[u]);
        }
        T acc[R];
#pragma unroll
        for (int u = 0; u < R; ++u) acc[u] = T(0);
        for (int t = 0; t < len; ++t) {
#pragma unroll
            for (int u = 0; u < R; ++u)
                if (ms[u] + t < me[u]) acc[u] += __ldg(Mv + ms[u] + t) * x[__ldg(a.Mci + ms[u] + t)];
        }
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < n) y[i] = acc[u];
        }
    }
}

size_t bytes_x(size_t es, int n) { return (es * (size_t)n + 15) & ~(size_t)15; }
size_t bytes_order(long long nv, int segs) {
    return ((4 * ((size_t)segs + 1) + 15) & ~(size_t)15) + ((4 * (size_t)nv + 15) & ~(size_t)15);
}
size_t bytes_L(size_t es, int n, long long nnzL) {
    return ((es * (size_t)nnzL + 15) & ~(size_t)15) + ((4 * (size_t)nnzL + 15) & ~(size_t)15) +
           ((4 * ((size_t)n + 1) + 15) & ~(size_t)15);
}

template <typename T>
const void *cta_kernel(bool os, bool ls) {
    if (os) return ls ? (const void *)k_cta_exec<T, true, true> : (const void *)k_cta_exec<T, true, false>;
    return ls ? (const void *)k_cta_exec<T, false, true> : (const void *)k_cta_exec<T, false, false>;
}

}  // namespace

// Launches the single-CTA executor. Shared memory holds x, then (when they fit) the segments and
// the order, then (when they fit too) L; what does not fit is read from global memory.
// cudaErrorInvalidValue when x alone does not fit.
cudaError_t launch_cta_exec(int mode, int dtype, long long nnzL, long long nv, int segs, cudaStream_t s,
                            const ExecArgs &a, cudaEvent_t ev_start, cudaEvent_t ev_stop) {
    int dev = 0, smax = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t es = dtype == 0 ? 8 : 4;
    size_t smem = bytes_x(es, a.n);
    if (smem > (size_t)smax) return cudaErrorInvalidValue;
    const bool os = smem + bytes_order(nv, segs) <= (size_t)smax;
    if (os) smem += bytes_order(nv, segs);
    const bool ls = smem + bytes_L(es, a.n, nnzL) <= (size_t)smax;
    if (ls) smem += bytes_L(es, a.n, nnzL);
    const void *f = dtype == 0 ? cta_kernel<double>(os, ls) : cta_kernel<float>(os, ls);
    // the opt-in shared-memory size is set once per device and kernel to the largest request
    static std::atomic<int> opted[kMaxDevices][2][2][2];
    cudaError_t e = cudaSuccess;
    if (dev >= kMaxDevices || opted[dev][dtype][os][ls].load() < (int)smem) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev < kMaxDevices) {
            int cur = opted[dev][dtype][os][ls].load();
            while (cur < (int)smem && !opted[dev][dtype][os][ls].compare_exchange_weak(cur, (int)smem)) {
            }
        }
    }
    void *args[] = {(void *)&a, (void *)&mode, (void *)&nnzL, (void *)&nv, (void *)&segs};
    if (ev_start && (e = cudaEventRecord(ev_start, s)) != cudaSuccess) return e;
    if ((e = cudaLaunchKernel(f, dim3(1), dim3(kCtaThreads), args, smem, s)) != cudaSuccess) return e;
    if (ev_stop) return cudaEventRecord(ev_stop, s);
    return cudaSuccess;
}

}  // namespace sf
