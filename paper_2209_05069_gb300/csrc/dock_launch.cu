// Pocket packing kernel and the dispatch from (bucket, grid dtype) to kernel instantiations.
#include <cuda_fp16.h>

#include "dock_internal.h"

namespace dockgpu {

// One instantiation per (grid type, warps per item, pose tile), from dock_kernels_inst.cu; the
// tile of 2 exists for 1 and 2 warps per item (larger groups already hold many angles in flight).
#define DOCK_DECLARE_INST(f, g, t)                                                                          \
  cudaError_t launch_bucket_f##f##_##g##_##t(int bucket, const PocketDev& pk, const BatchDev& b, const ParamsDev& p, \
                                             const uint32_t* items, int n_items, const LaunchCfg& cfg,            \
                                             cudaStream_t s, bool set_attributes);
#define DOCK_DECLARE_GT(f) \
  DOCK_DECLARE_INST(f, 1, 1) DOCK_DECLARE_INST(f, 2, 1) DOCK_DECLARE_INST(f, 4, 1) DOCK_DECLARE_INST(f, 8, 1) \
  DOCK_DECLARE_INST(f, 1, 2) DOCK_DECLARE_INST(f, 2, 2)
DOCK_DECLARE_GT(0)
DOCK_DECLARE_GT(1)
DOCK_DECLARE_GT(2)

// The latency form, one instantiation per grid type, from dock_latency_inst.cu.
#define DOCK_DECLARE_LAT(f)                                                                                \
  cudaError_t launch_latency_f##f(int bucket, const PocketDev& pk, const BatchDev& b, const ParamsDev& p, int l, \
                                  const LatScratch& sc, cudaStream_t s, int* launches);
DOCK_DECLARE_LAT(0)
DOCK_DECLARE_LAT(1)
DOCK_DECLARE_LAT(2)

// Cell c = (k*(ny-1) + j)*(nx-1) + i gathers the 8 corner voxels of the grid cell whose lower
// corner is voxel (i, j, k); the extra last cell is all zeros (positions outside the grid).
__global__ void pack_pocket_kernel(const float* __restrict__ v, void* cells, int nx, int ny, int nz, int f16) {
  const long long nc = (long long)(nx - 1) * (ny - 1) * (nz - 1);
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c <= nc; c += (long long)gridDim.x * blockDim.x) {
    float q[8];
    if (c == nc) {
#pragma unroll
      for (int t = 0; t < 8; ++t) q[t] = 0.f;
    } else {
      const long long i = c % (nx - 1), j = (c / (nx - 1)) % (ny - 1), k = c / ((long long)(nx - 1) * (ny - 1));
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const long long di = t & 1, dj = (t >> 1) & 1, dk = (t >> 2) & 1;
        q[t] = v[((k + dk) * ny + (j + dj)) * nx + (i + di)];
      }
    }
    if (f16) {
      __half2 h[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) h[t] = __halves2half2(__float2half_rn(q[2 * t]), __float2half_rn(q[2 * t + 1]));
      reinterpret_cast<uint4*>(cells)[c] = *reinterpret_cast<const uint4*>(h);
    } else {
      float4* o = reinterpret_cast<float4*>(cells) + 2 * c;
      o[0] = make_float4(q[0], q[1], q[2], q[3]);
      o[1] = make_float4(q[4], q[5], q[6], q[7]);
    }
  }
}

cudaError_t launch_pack_pocket(const float* values, void* cells, int nx, int ny, int nz, int f16, cudaStream_t s) {
  const long long nc = (long long)(nx - 1) * (ny - 1) * (nz - 1) + 1;
  const int threads = 256;
  const long long want = (nc + threads - 1) / threads;
  const int blocks = (int)(want < 65536 ? want : 65536);
  pack_pocket_kernel<<<blocks, threads, 0, s>>>(values, cells, nx, ny, nz, f16);
  return cudaGetLastError();
}

cudaError_t launch_dock_bucket(int bucket, const PocketDev& pk, const BatchDev& b, const ParamsDev& p,
                               const uint32_t* items, int n_items, const LaunchCfg& cfg, cudaStream_t s,
                               bool set_attributes) {
  if (n_items <= 0 && !set_attributes) return cudaSuccess;
  const int key = cfg.warps_per_item * 10 + (cfg.tile == 2 ? 2 : 1);
#define DOCK_DISPATCH_GT(f)                                                                        \
  switch (key) {                                                                                   \
    case 11: return launch_bucket_f##f##_1_1(bucket, pk, b, p, items, n_items, cfg, s, set_attributes); \
    case 21: return launch_bucket_f##f##_2_1(bucket, pk, b, p, items, n_items, cfg, s, set_attributes); \
    case 41: return launch_bucket_f##f##_4_1(bucket, pk, b, p, items, n_items, cfg, s, set_attributes); \
    case 81: return launch_bucket_f##f##_8_1(bucket, pk, b, p, items, n_items, cfg, s, set_attributes); \
    case 12: return launch_bucket_f##f##_1_2(bucket, pk, b, p, items, n_items, cfg, s, set_attributes); \
    case 22: return launch_bucket_f##f##_2_2(bucket, pk, b, p, items, n_items, cfg, s, set_attributes); \
  }
  if (pk.dtype == 2) {
    DOCK_DISPATCH_GT(2)
  } else if (pk.dtype == 1) {
    DOCK_DISPATCH_GT(1)
  } else {
    DOCK_DISPATCH_GT(0)
  }
#undef DOCK_DISPATCH_GT
  return cudaErrorInvalidValue;
}

cudaError_t launch_latency_ligand(int bucket, const PocketDev& pk, const BatchDev& b, const ParamsDev& p, int l,
                                  const LatScratch& sc, cudaStream_t s, int* launches) {
  switch (pk.dtype) {
    case 0: return launch_latency_f0(bucket, pk, b, p, l, sc, s, launches);
    case 1: return launch_latency_f1(bucket, pk, b, p, l, sc, s, launches);
    case 2: return launch_latency_f2(bucket, pk, b, p, l, sc, s, launches);
  }
  return cudaErrorInvalidValue;
}

}  // namespace dockgpu
