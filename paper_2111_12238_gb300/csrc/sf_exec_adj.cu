// Executor instantiations: the adjoint pass of SpTRSV -> SpMV (that of SpMV -> SpTRSV is in
// sf_exec_adj2.cu), plus the adjoint's two streaming helpers (values in transposed order,
// and the pattern-restricted value gradients).
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

// out[e] = sign * sum_c coef[i*k+c] * vec[ci[e]*k+c] for every entry e of row i; one group of
// LPR lanes per row, rows in order (coalesced over the pattern).
template <typename T, int LPR>
__global__ void __launch_bounds__(256) k_grad_rows(int n, int k, int kt, const int *__restrict__ rp,
                                                   const int *__restrict__ ci, const T *__restrict__ coef,
                                                   const T *__restrict__ vec, T sign, T *__restrict__ out) {
    constexpr int G = 32 / LPR;
    const int lane = threadIdx.x & 31, grp = lane / LPR, gl = lane % LPR, gbase = grp * LPR;
    const long long warp = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r0 = warp * G; r0 < n; r0 += nwarps * G) {
        const long long i = r0 + grp;
        if (i >= n) continue;
        const T *cr = coef + (size_t)i * k;
        grad_row<T, LPR>(ci, __ldg(rp + i), __ldg(rp + i + 1), [&](int c) { return __ldg(cr + c); }, vec, k, kt, gl,
                         gbase, sign, out);
    }
}

cudaError_t launch_grad_rows(int dtype, int n, long long nnz, int k, const int *rp, const int *ci, const void *coef,
                             const void *vec, double sign, void *out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int kt = 1;
    while (kt < k && kt < 32) kt <<= 1;
    const long long mean = (nnz + n - 1) / n;
    int lpr = kt;
    while (lpr < 32 && lpr * 4 < mean * kt) lpr <<= 1;    // about four entries per slice
    const long long groups_per_block = 8LL * (32 / lpr);
    long long blocks = (n + groups_per_block - 1) / groups_per_block;
    if (blocks > (long long)sms * 16) blocks = (long long)sms * 16;
#define SF_G(T, L) k_grad_rows<T, L><<<(unsigned)blocks, 256, 0, s>>>(n, k, kt, rp, ci, (const T *)coef, (const T *)vec, (T)sign, (T *)out); return cudaGetLastError()
    if (dtype == 0) {
        switch (lpr) {
            case 1: SF_G(double, 1); case 2: SF_G(double, 2); case 4: SF_G(double, 4);
            case 8: SF_G(double, 8); case 16: SF_G(double, 16); case 32: SF_G(double, 32);
        }
    } else {
        switch (lpr) {
            case 1: SF_G(float, 1); case 2: SF_G(float, 2); case 4: SF_G(float, 4);
            case 8: SF_G(float, 8); case 16: SF_G(float, 16); case 32: SF_G(float, 32);
        }
    }
#undef SF_G
    return cudaErrorInvalidValue;
}

}  // namespace sf
