// Instantiates the latency form's kernels for one grid type (DOCK_INST_GT: 0 FP32, 1 FP16, 2 int16),
// all five atom buckets; the build compiles this file once per grid type.
#include "dock_latency.cuh"

#if !defined(DOCK_INST_GT)
#error "compile with -DDOCK_INST_GT=<0|1|2>"
#endif

namespace dockgpu {

#define DOCK_LCAT2(a, b) a##b
#define DOCK_LCAT(a, b) DOCK_LCAT2(a, b)

cudaError_t DOCK_LCAT(launch_latency_f, DOCK_INST_GT)(int bucket, const PocketDev& pk, const BatchDev& b,
                                                      const ParamsDev& p, int l, const LatScratch& sc, cudaStream_t s,
                                                      int* launches) {
  constexpr int GT = DOCK_INST_GT;
  switch (bucket) {
    case 0: return lat_launch_t<32, GT>(pk, b, p, l, sc, s, launches);
    case 1: return lat_launch_t<64, GT>(pk, b, p, l, sc, s, launches);
    case 2: return lat_launch_t<96, GT>(pk, b, p, l, sc, s, launches);
    case 3: return lat_launch_t<128, GT>(pk, b, p, l, sc, s, launches);
    case 4: return lat_launch_t<160, GT>(pk, b, p, l, sc, s, launches);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dockgpu
