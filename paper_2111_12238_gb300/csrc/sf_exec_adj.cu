// Executor instantiations: the two adjoint passes.
#include "sf_exec.cuh"

namespace sf {

cudaError_t launch_exec_adj(int mode, int dtype, int lpr, bool vf, int blocks, cudaStream_t s, const ExecArgs &a) {
    if (mode == M_ADJ_TRSV_SPMV) return launch_mode<M_ADJ_TRSV_SPMV>(dtype, lpr, vf, blocks, s, a);
    if (mode == M_ADJ_SPMV_TRSV) return launch_mode<M_ADJ_SPMV_TRSV>(dtype, lpr, vf, blocks, s, a);
    return cudaErrorInvalidValue;
}

int occupancy_adj(int mode, int dtype, int lpr, bool vf) {
    if (mode == M_ADJ_TRSV_SPMV) return blocks_per_sm_mode<M_ADJ_TRSV_SPMV>(dtype, lpr, vf);
    return blocks_per_sm_mode<M_ADJ_SPMV_TRSV>(dtype, lpr, vf);
}

}  // namespace sf
