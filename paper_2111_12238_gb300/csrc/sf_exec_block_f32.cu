// Row-block executor kernels, single precision.
#include "sf_block_inst.cuh"

namespace sf {
const void *block_kernel_f32(int mode, int lpr) { return block_kernel_t<float>(mode, lpr); }
const void *block_ws_kernel_f32(int mode) { return block_ws_kernel_t<float>(mode); }
const void *block_tma_kernel_f32(int mode, int which) { return block_tma_kernel_t<float>(mode, which); }
}  // namespace sf
