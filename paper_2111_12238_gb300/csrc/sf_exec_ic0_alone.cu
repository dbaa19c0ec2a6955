// Executor instantiations: SpIC0 alone (the factor pass of the unfused path).
#include "sf_exec.cuh"

namespace sf {

cudaError_t launch_exec_ic0_alone(int dtype, int lpr, bool vf, int team, int minb, int blocks, cudaStream_t s,
                                  const ExecArgs &a) {
    return launch_mode<M_IC0>(dtype, lpr, vf, team, minb, blocks, s, a);
}

int occupancy_ic0_alone(int dtype, int lpr, bool vf, int team, int minb) {
    return blocks_per_sm_mode<M_IC0>(dtype, lpr, vf, team, minb);
}

}  // namespace sf
