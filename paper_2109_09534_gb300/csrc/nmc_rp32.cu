// nmc_rp32.cu -- mode-update kernels for padded rank 32.
#include "launch_rp.cuh"

namespace ntc {
template cudaError_t launch_mode_rp<32>(int, bool, const ModeArgs&, const ModePlan&, Launcher&, bool);
}  // namespace ntc
