// Executor instantiations: the paired mode SpIC0 -> SpTRSV; dispatch of both IC0 modes.
#include "sf_exec.cuh"

namespace sf {

cudaError_t launch_exec_ic0(int mode, int dtype, int lpr, bool vf, int team, int minb, int blocks, cudaStream_t s,
                            const ExecArgs &a) {
    if (mode == M_IC0_TRSV) return launch_mode<M_IC0_TRSV>(dtype, lpr, vf, team, minb, blocks, s, a);
    if (mode == M_IC0) return launch_exec_ic0_alone(dtype, lpr, vf, team, minb, blocks, s, a);
    return cudaErrorInvalidValue;
}

int occupancy_ic0(int mode, int dtype, int lpr, bool vf, int team, int minb) {
    if (mode == M_IC0_TRSV) return blocks_per_sm_mode<M_IC0_TRSV>(dtype, lpr, vf, team, minb);
    return occupancy_ic0_alone(dtype, lpr, vf, team, minb);
}

}  // namespace sf
