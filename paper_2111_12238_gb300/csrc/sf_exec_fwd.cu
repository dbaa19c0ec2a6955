// Executor instantiations: SpTRSV -> SpMV (separated items; SpTRSV alone is in
// sf_exec_trsv.cu), plus the plain SpMV kernel of the unfused two-launch path.
#include "sf_exec.cuh"

namespace sf {

cudaError_t launch_exec_fwd(int mode, int dtype, int lpr, bool vf, int team, int minb, int blocks, cudaStream_t s,
                            const ExecArgs &a) {
    if (mode == M_TRSV_SPMV) return launch_mode<M_TRSV_SPMV>(dtype, lpr, vf, team, minb, blocks, s, a);
    if (mode == M_TRSV) return launch_exec_trsv(dtype, lpr, vf, team, minb, blocks, s, a);
    return cudaErrorInvalidValue;
}

int occupancy_fwd(int mode, int dtype, int lpr, bool vf, int team, int minb) {
    if (mode == M_TRSV_SPMV) return blocks_per_sm_mode<M_TRSV_SPMV>(dtype, lpr, vf, team, minb);
    return occupancy_trsv(dtype, lpr, vf, team, minb);
}

// y = M x or y = b - M x, one group of LPR lanes per row, rows in order (no
// dependences, so no flags): the SpMV kernel optimised on its own.
template <typename T, int LPR>
__global__ void __launch_bounds__(256) k_spmv(int nrows, int k, int kt, const int *__restrict__ rp,
                                              const int *__restrict__ ci, const T *__restrict__ v,
                                              const T *__restrict__ x, const T *__restrict__ b, T *__restrict__ y) {
    constexpr int G = 32 / LPR;
    const int lane = threadIdx.x & 31, grp = lane / LPR, gl = lane % LPR;
    const unsigned gmask = (LPR == 32) ? 0xffffffffu : (((1u << LPR) - 1u) << (grp * LPR));
    const int S = LPR / kt, s = gl / kt, cl = gl % kt;
    const long long warp = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    bool dummy = true;
    for (long long r0 = warp * G; r0 < nrows; r0 += nwarps * G) {
        const long long row = r0 + grp;
        if (row >= nrows) continue;
        const int rs = rp[row], re = rp[row + 1];
        for (int c0 = 0; c0 < k; c0 += kt) {
            const int c = c0 + cl;
            const bool act = c < k;
            T acc = row_dot<T, D_NONE, false>(ci, nullptr, v, rs + s, re, S, x, k, c, act, nullptr, 0u, nullptr,
                                             0ull, (int)row, dummy);
            acc = slice_sum<LPR>(acc, kt, gmask);
            if (s == 0 && act) {
                const size_t o = (size_t)row * k + c;
                y[o] = b ? b[o] - acc : acc;
            }
        }
    }
}

cudaError_t launch_spmv(int dtype, int lpr, int kt, int nrows, int k, const int *rp, const int *ci, const void *v,
                        const void *x, const void *b, void *y, cudaStream_t s) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long groups = nrows;
    const long long warps_needed = (groups + (32 / lpr) - 1) / (32 / lpr);
    long long blocks = (warps_needed + 7) / 8;
    const long long cap = (long long)sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
#define SF_SPMV(T, L) k_spmv<T, L><<<(int)blocks, 256, 0, s>>>(nrows, k, kt, rp, ci, (const T *)v, (const T *)x, (const T *)b, (T *)y); return cudaGetLastError()
    if (dtype == 0) {
        switch (lpr) {
            case 1: SF_SPMV(double, 1); case 2: SF_SPMV(double, 2); case 4: SF_SPMV(double, 4);
            case 8: SF_SPMV(double, 8); case 16: SF_SPMV(double, 16); case 32: SF_SPMV(double, 32);
        }
    } else {
        switch (lpr) {
            case 1: SF_SPMV(float, 1); case 2: SF_SPMV(float, 2); case 4: SF_SPMV(float, 4);
            case 8: SF_SPMV(float, 8); case 16: SF_SPMV(float, 16); case 32: SF_SPMV(float, 32);
        }
    }
#undef SF_SPMV
    return cudaErrorInvalidValue;
}

}  // namespace sf
