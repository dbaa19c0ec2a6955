// Executor instantiations: SpTRSV alone (the solve pass of the unfused path).
#include "sf_exec.cuh"

namespace sf {

cudaError_t launch_exec_trsv(int dtype, int lpr, bool vf, int team, int minb, int blocks, cudaStream_t s,
                             const ExecArgs &a) {
    return launch_mode<M_TRSV>(dtype, lpr, vf, team, minb, blocks, s, a);
}

int occupancy_trsv(int dtype, int lpr, bool vf, int team, int minb) {
    return blocks_per_sm_mode<M_TRSV>(dtype, lpr, vf, team, minb);
}

}  // namespace sf
