// Executor instantiations: the paired mode SpMV -> SpTRSV; the IC0 modes are in
// sf_exec_ic0.cu and sf_exec_ic0_alone.cu (separate translation units compile in parallel).
#include "sf_exec.cuh"

namespace sf {

cudaError_t launch_exec_pair(int mode, int dtype, int lpr, bool vf, int team, int minb, int blocks, cudaStream_t s,
                            const ExecArgs &a) {
    if (mode == M_SPMV_TRSV) return launch_mode<M_SPMV_TRSV>(dtype, lpr, vf, team, minb, blocks, s, a);
    if (mode == M_IC0_TRSV || mode == M_IC0) return launch_exec_ic0(mode, dtype, lpr, vf, team, minb, blocks, s, a);
    return cudaErrorInvalidValue;
}

int occupancy_pair(int mode, int dtype, int lpr, bool vf, int team, int minb) {
    if (mode == M_SPMV_TRSV) return blocks_per_sm_mode<M_SPMV_TRSV>(dtype, lpr, vf, team, minb);
    return occupancy_ic0(mode, dtype, lpr, vf, team, minb);
}

}  // namespace sf
