// nmc_rp8.cu -- mode-update kernels for padded rank 8.
#include "launch_rp.cuh"

namespace ntc {
template cudaError_t launch_mode_rp<8>(int, bool, const ModeArgs&, const ModePlan&, Launcher&, bool);
}  // namespace ntc
