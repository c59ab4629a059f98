// Build-pass instantiations for BF16 feature storage (one translation unit per
// storage type so that they compile in parallel).
#include "pilot_build_impl.cuh"
#include "pilot_level_impl.cuh"

namespace pilot {
template cudaError_t launch_build_dtype<PILOT_BF16>(const BuildParams&, cudaStream_t);
template cudaError_t launch_build_fused_dtype<PILOT_BF16>(const FusedBuildParams&, cudaStream_t);
template cudaError_t launch_level_persistent_dtype<PILOT_BF16>(int, int, const LevelArgs&, int, cudaStream_t);
template cudaError_t level_persistent_occupancy<PILOT_BF16>(int, int, int*);
}  // namespace pilot
