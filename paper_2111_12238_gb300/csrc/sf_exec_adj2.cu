// Executor instantiations: the adjoint pass of SpMV -> SpTRSV.
#include "sf_exec.cuh"

namespace sf {

cudaError_t launch_exec_adj2(int dtype, int lpr, bool vf, int team, int minb, int blocks, cudaStream_t s,
                             const ExecArgs &a) {
    return launch_mode<M_ADJ_SPMV_TRSV>(dtype, lpr, vf, team, minb, blocks, s, a);
}

int occupancy_adj2(int dtype, int lpr, bool vf, int team, int minb) {
    return blocks_per_sm_mode<M_ADJ_SPMV_TRSV>(dtype, lpr, vf, team, minb);
}

}  // namespace sf
