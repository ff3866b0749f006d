// Instantiates the docking kernel for one grid type (DOCK_INST_GT: 0 FP32, 1 FP16, 2 int16), one
// number of warps per work item (DOCK_INST_G) and one pose tile (DOCK_INST_T: poses or angles a lane
// scores per pass), all five atom buckets.  The build compiles this file once per combination so
// the instantiations compile in parallel.
#include "dock_kernels.cuh"

#if !defined(DOCK_INST_GT) || !defined(DOCK_INST_G) || !defined(DOCK_INST_T)
#error "compile with -DDOCK_INST_GT=<0|1|2> -DDOCK_INST_G=<1|2|4|8> -DDOCK_INST_T=<1|2>"
#endif

namespace dockgpu {

#define DOCK_CAT2(a, b, c, d) a##b##_##c##_##d
#define DOCK_CAT(a, b, c, d) DOCK_CAT2(a, b, c, d)
#define DOCK_INST_NAME DOCK_CAT(launch_bucket_f, DOCK_INST_GT, DOCK_INST_G, DOCK_INST_T)

cudaError_t DOCK_INST_NAME(int bucket, const PocketDev& pk, const BatchDev& b, const ParamsDev& p,
                           const uint32_t* items, int n_items, const LaunchCfg& cfg, cudaStream_t s,
                           bool set_attributes) {
  constexpr int GT = DOCK_INST_GT;
  constexpr int G = DOCK_INST_G;
  constexpr int T = DOCK_INST_T;
  switch (bucket) {
    case 0: return launch_t<32, GT, G, T>(pk, b, p, items, n_items, cfg, s, set_attributes);
    case 1: return launch_t<64, GT, G, T>(pk, b, p, items, n_items, cfg, s, set_attributes);
    case 2: return launch_t<96, GT, G, T>(pk, b, p, items, n_items, cfg, s, set_attributes);
    case 3: return launch_t<128, GT, G, T>(pk, b, p, items, n_items, cfg, s, set_attributes);
    case 4: return launch_t<160, GT, G, T>(pk, b, p, items, n_items, cfg, s, set_attributes);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dockgpu
