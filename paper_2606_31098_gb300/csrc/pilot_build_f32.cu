// Build-pass instantiations for F32 feature storage (one translation unit per
// storage type so that they compile in parallel).
#include "pilot_build_impl.cuh"
#include "pilot_level_impl.cuh"

namespace pilot {
template cudaError_t launch_build_dtype<PILOT_F32>(const BuildParams&, cudaStream_t);
template cudaError_t launch_build_fused_dtype<PILOT_F32>(const FusedBuildParams&, cudaStream_t);
template cudaError_t launch_level_persistent_dtype<PILOT_F32>(int, int, const LevelArgs&, int, cudaStream_t);
template cudaError_t level_persistent_occupancy<PILOT_F32>(int, int, int*);
}  // namespace pilot
