// nmc_rp16.cu -- mode-update kernels for padded rank 16.
#include "launch_rp.cuh"

namespace ntc {
template cudaError_t launch_mode_rp<16>(int, bool, const ModeArgs&, const ModePlan&, Launcher&, bool);
}  // namespace ntc
