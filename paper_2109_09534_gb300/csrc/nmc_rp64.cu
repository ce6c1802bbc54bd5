// nmc_rp64.cu -- mode-update kernels for padded rank 64.
#include "launch_rp.cuh"

namespace ntc {
template cudaError_t launch_mode_rp<64>(int, bool, const ModeArgs&, const ModePlan&, Launcher&, bool);
}  // namespace ntc
