// Executor instantiations: the paired modes SpMV -> SpTRSV and SpIC0 -> SpTRSV, and
// SpIC0 alone.
#include "sf_exec.cuh"

namespace sf {

cudaError_t launch_exec_pair(int mode, int dtype, int lpr, bool vf, int team, int minb, int blocks, cudaStream_t s,
                            const ExecArgs &a) {
    if (mode == M_SPMV_TRSV) return launch_mode<M_SPMV_TRSV>(dtype, lpr, vf, team, minb, blocks, s, a);
    if (mode == M_IC0_TRSV) return launch_mode<M_IC0_TRSV>(dtype, lpr, vf, team, minb, blocks, s, a);
    if (mode == M_IC0) return launch_mode<M_IC0>(dtype, lpr, vf, team, minb, blocks, s, a);
    return cudaErrorInvalidValue;
}

int occupancy_pair(int mode, int dtype, int lpr, bool vf, int team, int minb) {
    if (mode == M_SPMV_TRSV) return blocks_per_sm_mode<M_SPMV_TRSV>(dtype, lpr, vf, team, minb);
    if (mode == M_IC0_TRSV) return blocks_per_sm_mode<M_IC0_TRSV>(dtype, lpr, vf, team, minb);
    return blocks_per_sm_mode<M_IC0>(dtype, lpr, vf, team, minb);
}

}  // namespace sf
