// Row-block executor: double-precision kernels, launch and occupancy (k = 1; one, two, four
// or thirty-two lanes per row).
#include <algorithm>

#include "sf_block_inst.cuh"

namespace sf {

const void *block_kernel_f64(int mode, int lpr) { return block_kernel_t<double>(mode, lpr); }
const void *block_ws_kernel_f64(int mode) { return block_ws_kernel_t<double>(mode); }
const void *block_tma_kernel_f64(int mode, int which) { return block_tma_kernel_t<double>(mode, which); }

namespace {

const void *block_kernel(int mode, int dtype, int lpr) {
    return dtype == 0 ? block_kernel_f64(mode, lpr) : block_kernel_f32(mode, lpr);
}

}  // namespace

template <typename T>
__global__ void __launch_bounds__(256) k_rdiag(int n, int k, const int *__restrict__ Lrp, const T *__restrict__ Lv,
                                               T *vec, T *__restrict__ rdiag, ExecState *st,
                                               const int *__restrict__ diag_at, T *vec2) {
    const long long nk = (long long)n * k;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nk; t += (long long)gridDim.x * blockDim.x) {
        vec[t] = unset_value<T>();
        if (vec2) vec2[t] = unset_value<T>();
        if (t < n) {
            const int i = (int)t;
            const T d = Lv[diag_at ? __ldg(diag_at + i) : __ldg(Lrp + i + 1) - 1];
            if (d == T(0)) record_error(st, SF_ERR_NONFINITE, i);
            rdiag[i] = T(1) / d;
        }
    }
}

cudaError_t launch_rdiag(int dtype, int n, int k, const int *Lrp, const void *Lv, void *vec, void *rdiag,
                         ExecState *st, cudaStream_t s, const int *diag_at, void *vec2) {
    const long long nk = (long long)n * k;
    const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>((nk + 255) / 256, 65535LL));
    if (dtype == 0)
        k_rdiag<double><<<grid, 256, 0, s>>>(n, k, Lrp, (const double *)Lv, (double *)vec, (double *)rdiag, st,
                                             diag_at, (double *)vec2);
    else
        k_rdiag<float><<<grid, 256, 0, s>>>(n, k, Lrp, (const float *)Lv, (float *)vec, (float *)rdiag, st, diag_at,
                                            (float *)vec2);
    return cudaGetLastError();
}

size_t block_exec_smem(int mode, int dtype, int block_rows) {
    (void)mode;
    return (size_t)block_rows * (dtype == 0 ? 8 : 4);
}

int block_exec_occupancy(int mode, int dtype, int lpr, int block_rows, int threads) {
    const void *f = lpr ? block_kernel(mode, dtype, lpr) : nullptr;
    if (!f || threads < 32 || threads > kBlockMaxThreads || threads % 32) return 0;
    const size_t smem = block_exec_smem(mode, dtype, block_rows);
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

size_t block_ws_smem(int dtype, int rows, int nc) {
    const size_t es = dtype == 0 ? 8 : 4;
    const size_t stage = dtype == 0 ? ws_stage_bytes<double>(nc) : ws_stage_bytes<float>(nc);
    return (((size_t)rows * es + 15) & ~(size_t)15) + (size_t)kWsStages * stage + ws_desc_bytes(nc);
}

int block_ws_fits(int mode, int dtype, int rows, int nc) {
    const void *f = dtype == 0 ? block_ws_kernel_f64(mode) : block_ws_kernel_f32(mode);
    if (!f || nc < 32 || nc > kWsMaxConsumers || (nc & (nc - 1))) return 0;
    const size_t smem = block_ws_smem(dtype, rows, nc);
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, nc + kWsProducers, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

cudaError_t launch_block_ws(int mode, int dtype, int blocks, int nc, cudaStream_t s, const ExecArgs &a,
                            cudaEvent_t ev_start, cudaEvent_t ev_stop) {
    const void *prep = block_kernel(mode, dtype, 0);
    const void *f = dtype == 0 ? block_ws_kernel_f64(mode) : block_ws_kernel_f32(mode);
    if (!prep || !f || nc < 32 || nc > kWsMaxConsumers || (nc & (nc - 1))) return cudaErrorInvalidValue;
    void *args[] = {(void *)&a};
    const long long pb = std::min<long long>(((long long)a.n + 255) / 256, 65535LL);
    cudaError_t e = cudaLaunchKernel(prep, dim3((unsigned)std::max<long long>(pb, 1)), dim3(256), args, 0, s);
    if (e != cudaSuccess) return e;
    const size_t smem = block_ws_smem(dtype, std::min(a.block_rows, a.n), nc);
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (ev_start && (e = cudaEventRecord(ev_start, s)) != cudaSuccess) return e;
    e = cudaLaunchCooperativeKernel(f, dim3(blocks), dim3(nc + kWsProducers), args, smem, s);
    if (e != cudaSuccess) return e;
    return ev_stop ? cudaEventRecord(ev_stop, s) : cudaSuccess;
}

cudaError_t launch_block_exec(int mode, int dtype, int lpr, int blocks, int threads, cudaStream_t s,
                              const ExecArgs &a, cudaEvent_t ev_start, cudaEvent_t ev_stop) {
    const void *prep = block_kernel(mode, dtype, 0);
    const void *f = lpr ? block_kernel(mode, dtype, lpr) : nullptr;
    if (!prep || !f || threads < 32 || threads > kBlockMaxThreads || threads % 32) return cudaErrorInvalidValue;
    void *args[] = {(void *)&a};
    // pre-pass: value-flag reset, independent parts and reciprocal diagonals of all rows
    const long long pb = std::min<long long>(((long long)a.n + 255) / 256, 65535LL);
    cudaError_t e = cudaLaunchKernel(prep, dim3((unsigned)std::max<long long>(pb, 1)), dim3(256), args, 0, s);
    if (e != cudaSuccess) return e;
    const size_t smem = block_exec_smem(mode, dtype, std::min(a.block_rows, a.n));
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (ev_start && (e = cudaEventRecord(ev_start, s)) != cudaSuccess) return e;
    e = cudaLaunchCooperativeKernel(f, dim3(blocks), dim3(threads), args, smem, s);
    if (e != cudaSuccess) return e;
    return ev_stop ? cudaEventRecord(ev_stop, s) : cudaSuccess;
}

// Pattern part of the packed records: for every position q of the row-block order its order
// entry, entry range and first kTmaU column indices (of L, M, L^T or M^T by kind and kernel).
__global__ void __launch_bounds__(256) k_pack_pattern(int kind, long long nv, int nvp, const int *__restrict__ border,
                                                      const int2 *__restrict__ bdesc, const int *__restrict__ Lci,
                                                      const int *__restrict__ Mci, const int *__restrict__ LTci,
                                                      const int *__restrict__ MTci, PackMeta *__restrict__ meta,
                                                      int *__restrict__ cols) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nvp; t += (long long)gridDim.x * blockDim.x) {
        const int q = (int)t;
        PackMeta md{-1, 0, 0, 0};
        const int *ci = nullptr;
        int cnt = 0;
        if (q < nv) {
            const unsigned o = (unsigned)border[q];
            const int2 dd = bdesc[q];
            const bool tag = (o >> 31) != 0;
            md = PackMeta{(int)o, dd.x, dd.y, 0};
            if (kind == K_SEP) ci = tag ? Mci : Lci;
            else if (kind == K_PAIRED) ci = Lci;
            else if (kind == K_PAIRED_T) ci = LTci;
            else ci = tag ? MTci : LTci;
            cnt = min(dd.y - dd.x, kTmaU);
        }
        meta[q] = md;
#pragma unroll
        for (int u = 0; u < kTmaU; ++u) cols[(size_t)u * nvp + q] = u < cnt ? ci[md.rs + u] : 0;
    }
}

cudaError_t pack_pattern(int kind, long long nv, int nvp, const int *border, const int2 *bdesc, const int *Lci,
                         const int *Mci, const int *LTci, const int *MTci, void *meta, int *cols, cudaStream_t s) {
    const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(((long long)nvp + 255) / 256, 65535LL));
    k_pack_pattern<<<grid, 256, 0, s>>>(kind, nv, nvp, border, bdesc, Lci, Mci, LTci, MTci, (PackMeta *)meta, cols);
    return cudaGetLastError();
}

size_t block_tma_smem(int dtype, int rows, int nc) {
    const size_t es = dtype == 0 ? 8 : 4;
    const size_t stage = dtype == 0 ? tma_stage_bytes<double>(nc) : tma_stage_bytes<float>(nc);
    return (((size_t)rows * es + 15) & ~(size_t)15) + (size_t)kTmaStages * stage;
}

int block_tma_fits(int mode, int dtype, int rows, int nc) {
    const void *f = dtype == 0 ? block_tma_kernel_f64(mode, 0) : block_tma_kernel_f32(mode, 0);
    if (!f || nc < 32 || nc > kTmaMaxConsumers || (nc & (nc - 1))) return 0;
    const size_t smem = block_tma_smem(dtype, rows, nc);
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, nc + kTmaProducers, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

cudaError_t launch_block_tma(int mode, int dtype, int blocks, int nc, cudaStream_t s, const ExecArgs &a,
                             cudaEvent_t ev_start, cudaEvent_t ev_stop) {
    const void *prep = block_kernel(mode, dtype, 0);
    const void *pack = dtype == 0 ? block_tma_kernel_f64(mode, 1) : block_tma_kernel_f32(mode, 1);
    const void *f = dtype == 0 ? block_tma_kernel_f64(mode, 0) : block_tma_kernel_f32(mode, 0);
    if (!prep || !pack || !f || nc < 32 || nc > kTmaMaxConsumers || (nc & (nc - 1))) return cudaErrorInvalidValue;
    void *args[] = {(void *)&a};
    const long long pb = std::min<long long>(((long long)a.n + 255) / 256, 65535LL);
    cudaError_t e = cudaLaunchKernel(prep, dim3((unsigned)std::max<long long>(pb, 1)), dim3(256), args, 0, s);
    if (e != cudaSuccess) return e;
    const long long vb = std::min<long long>(((long long)a.pack_stride + 255) / 256, 65535LL);
    e = cudaLaunchKernel(pack, dim3((unsigned)std::max<long long>(vb, 1)), dim3(256), args, 0, s);
    if (e != cudaSuccess) return e;
    const size_t smem = block_tma_smem(dtype, std::min(a.block_rows, a.n), nc);
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (ev_start && (e = cudaEventRecord(ev_start, s)) != cudaSuccess) return e;
    e = cudaLaunchCooperativeKernel(f, dim3(blocks), dim3(nc + kTmaProducers), args, smem, s);
    if (e != cudaSuccess) return e;
    return ev_stop ? cudaEventRecord(ev_stop, s) : cudaSuccess;
}

}  // namespace sf
