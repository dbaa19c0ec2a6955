// Executor instantiations: the adjoint pass of SpTRSV -> SpMV (that of SpMV -> SpTRSV is in
// sf_exec_adj2.cu), plus the adjoint's two streaming helpers (values in transposed order,
// and the pattern-restricted value gradients, one thread per entry).
#include <algorithm>
#include <cstdint>

#include "sf_exec.cuh"

namespace sf {

cudaError_t launch_exec_adj(int mode, int dtype, int lpr, bool vf, int team, int minb, int blocks, cudaStream_t s,
                            const ExecArgs &a) {
    if (mode == M_ADJ_TRSV_SPMV) return launch_mode<M_ADJ_TRSV_SPMV>(dtype, lpr, vf, team, minb, blocks, s, a);
    if (mode == M_ADJ_SPMV_TRSV) return launch_exec_adj2(dtype, lpr, vf, team, minb, blocks, s, a);
    return cudaErrorInvalidValue;
}

int occupancy_adj(int mode, int dtype, int lpr, bool vf, int team, int minb) {
    if (mode == M_ADJ_TRSV_SPMV) return blocks_per_sm_mode<M_ADJ_TRSV_SPMV>(dtype, lpr, vf, team, minb);
    return occupancy_adj2(dtype, lpr, vf, team, minb);
}

template <typename T>
__global__ void k_gather_vals(long long nnz, const int *__restrict__ perm, const T *__restrict__ src,
                              T *__restrict__ dst) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nnz; t += (long long)gridDim.x * blockDim.x)
        dst[t] = __ldg(src + __ldg(perm + t));
}

cudaError_t launch_gather_vals(int dtype, long long nnz, const int *perm, const void *src, void *dst, cudaStream_t s) {
    if (nnz <= 0) return cudaSuccess;
    long long blocks = (nnz + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    if (dtype == 0) k_gather_vals<double><<<(unsigned)blocks, 256, 0, s>>>(nnz, perm, (const double *)src, (double *)dst);
    else k_gather_vals<float><<<(unsigned)blocks, 256, 0, s>>>(nnz, perm, (const float *)src, (float *)dst);
    return cudaGetLastError();
}

// out[e] = sign * sum_c coef[i*k+c] * vec[ci[e]*k+c] for every entry e (row i = row_of[e]):
// the pattern-restricted outer products of the adjoint's value gradients. One thread per entry,
// consecutive threads on consecutive entries (coalesced pattern reads and stores; the coef row
// is shared by a row's entries and stays in L1), the k products of an entry summed in column
// order from V-wide vector loads (V = 2 doubles or 4 floats when k allows the alignment), so a
// thread has k / V independent loads in flight and no lane waits on another.
template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float4; };

template <typename T, bool VEC>
__global__ void __launch_bounds__(256) k_grad_entries(long long nnz, int k, const int *__restrict__ row_of,
                                                      const int *__restrict__ ci, const T *__restrict__ coef,
                                                      const T *__restrict__ vec, T sign, T *__restrict__ out) {
    using VT = typename Vec2<T>::type;
    constexpr int V = sizeof(VT) / sizeof(T);
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
         e += (long long)gridDim.x * blockDim.x) {
        const T *a = coef + (size_t)__ldg(row_of + e) * k;
        const T *b = vec + (size_t)__ldg(ci + e) * k;
        T sum = T(0);
        if constexpr (VEC) {
#pragma unroll 4
            for (int c = 0; c < k; c += V) {
                const VT va = __ldg((const VT *)(a + c)), vb = __ldg((const VT *)(b + c));
                if constexpr (V == 2) {
                    sum += va.x * vb.x;
                    sum += va.y * vb.y;
                } else {
                    sum += va.x * vb.x;
                    sum += va.y * vb.y;
                    sum += va.z * vb.z;
                    sum += va.w * vb.w;
                }
            }
        } else {
#pragma unroll 4
            for (int c = 0; c < k; ++c) sum += __ldg(a + c) * __ldg(b + c);
        }
        out[e] = sign * sum;
    }
}

cudaError_t launch_grad_entries(int dtype, long long nnz, int k, const int *row_of, const int *ci, const void *coef,
                                const void *vec, double sign, void *out, cudaStream_t s) {
    if (nnz <= 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long blocks = std::max<long long>(1, std::min<long long>((nnz + 255) / 256, (long long)sms * 32));
    // vector loads need every row of coef and vec to start on a 16-byte boundary
    const int V = dtype == 0 ? 2 : 4;
    const bool vec_ok = k % V == 0 && ((uintptr_t)coef % 16) == 0 && ((uintptr_t)vec % 16) == 0;
    if (dtype == 0) {
        if (vec_ok)
            k_grad_entries<double, true><<<(unsigned)blocks, 256, 0, s>>>(nnz, k, row_of, ci, (const double *)coef,
                                                                         (const double *)vec, sign, (double *)out);
        else
            k_grad_entries<double, false><<<(unsigned)blocks, 256, 0, s>>>(nnz, k, row_of, ci, (const double *)coef,
                                                                          (const double *)vec, sign, (double *)out);
    } else {
        if (vec_ok)
            k_grad_entries<float, true><<<(unsigned)blocks, 256, 0, s>>>(nnz, k, row_of, ci, (const float *)coef,
                                                                        (const float *)vec, (float)sign, (float *)out);
        else
            k_grad_entries<float, false><<<(unsigned)blocks, 256, 0, s>>>(nnz, k, row_of, ci, (const float *)coef,
                                                                         (const float *)vec, (float)sign, (float *)out);
    }
    return cudaGetLastError();
}

}  // namespace sf
