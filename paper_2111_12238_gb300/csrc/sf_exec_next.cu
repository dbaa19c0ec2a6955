// Executor instantiations of Table 2 combinations 1 (SpTRSV -> SpTRSV, paired rows, any lane
// count, value or epoch flags) and 6 (SpILU0 -> SpTRSV, whole-warp rows with value flags only).
#include "sf_exec.cuh"

namespace sf {

namespace {

const void *ilu0_kernel(int dtype, int minb) {
    if (minb >= kMinBlocksHigh)
        return dtype == 0 ? (const void *)k_exec<M_ILU0_TRSV, double, 32, true, 32, kMinBlocksIc0>
                          : (const void *)k_exec<M_ILU0_TRSV, float, 32, true, 32, kMinBlocksIc0>;
    return dtype == 0 ? (const void *)k_exec<M_ILU0_TRSV, double, 32, true, 32, kMinBlocksDefault>
                      : (const void *)k_exec<M_ILU0_TRSV, float, 32, true, 32, kMinBlocksDefault>;
}

}  // namespace

cudaError_t launch_exec_next(int mode, int dtype, int lpr, bool vf, int team, int minb, int blocks, cudaStream_t s,
                             const ExecArgs &a) {
    if (mode == M_TRSV_TRSV) return launch_mode<M_TRSV_TRSV>(dtype, lpr, vf, team, minb, blocks, s, a);
    if (mode != M_ILU0_TRSV || lpr != 32 || !vf) return cudaErrorInvalidValue;
    void *args[] = {(void *)&a};
    const void *f = ilu0_kernel(dtype, minb);
    if (a.dynamic) return cudaLaunchKernel(f, dim3(blocks), dim3(kExecThreads), args, 0, s);
    return cudaLaunchCooperativeKernel(f, dim3(blocks), dim3(kExecThreads), args, 0, s);
}

int occupancy_next(int mode, int dtype, int lpr, bool vf, int team, int minb) {
    if (mode == M_TRSV_TRSV) return blocks_per_sm_mode<M_TRSV_TRSV>(dtype, lpr, vf, team, minb);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ilu0_kernel(dtype, minb), kExecThreads, 0) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

}  // namespace sf
