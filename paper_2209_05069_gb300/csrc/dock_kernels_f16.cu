// FP16 pocket-grid instantiations of the fused docking kernel (all five atom buckets).
#include "dock_kernels.cuh"

namespace dockgpu {
template cudaError_t launch_bucket_t<true>(int, const PocketDev&, const BatchDev&, const ParamsDev&, const uint32_t*,
                                           int, const LaunchCfg&, cudaStream_t, bool);
}  // namespace dockgpu
