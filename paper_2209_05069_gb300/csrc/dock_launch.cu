// Pocket packing kernel and the dispatch from (bucket, grid dtype) to kernel instantiations.
#include <cuda_fp16.h>

#include "dock_internal.h"

namespace dockgpu {

// One instantiation per (grid type, warps per item), from dock_kernels_inst.cu.
#define DOCK_DECLARE_INST(f, g)                                                                        \
  cudaError_t launch_bucket_f##f##_##g(int bucket, const PocketDev& pk, const BatchDev& b, const ParamsDev& p, \
                                      const uint32_t* items, int n_items, const LaunchCfg& cfg, cudaStream_t s, \
                                      bool set_attributes);
DOCK_DECLARE_INST(0, 1)
DOCK_DECLARE_INST(0, 2)
DOCK_DECLARE_INST(0, 4)
DOCK_DECLARE_INST(0, 8)
DOCK_DECLARE_INST(1, 1)
DOCK_DECLARE_INST(1, 2)
DOCK_DECLARE_INST(1, 4)
DOCK_DECLARE_INST(1, 8)
DOCK_DECLARE_INST(2, 1)
DOCK_DECLARE_INST(2, 2)
DOCK_DECLARE_INST(2, 4)
DOCK_DECLARE_INST(2, 8)

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
  const int g = cfg.warps_per_item;
  if (pk.dtype == 2) {
    switch (g) {
      case 1: return launch_bucket_f2_1(bucket, pk, b, p, items, n_items, cfg, s, set_attributes);
      case 2: return launch_bucket_f2_2(bucket, pk, b, p, items, n_items, cfg, s, set_attributes);
      case 4: return launch_bucket_f2_4(bucket, pk, b, p, items, n_items, cfg, s, set_attributes);
      case 8: return launch_bucket_f2_8(bucket, pk, b, p, items, n_items, cfg, s, set_attributes);
    }
  } else if (pk.dtype == 1) {
    switch (g) {
      case 1: return launch_bucket_f1_1(bucket, pk, b, p, items, n_items, cfg, s, set_attributes);
      case 2: return launch_bucket_f1_2(bucket, pk, b, p, items, n_items, cfg, s, set_attributes);
      case 4: return launch_bucket_f1_4(bucket, pk, b, p, items, n_items, cfg, s, set_attributes);
      case 8: return launch_bucket_f1_8(bucket, pk, b, p, items, n_items, cfg, s, set_attributes);
    }
  } else {
    switch (g) {
      case 1: return launch_bucket_f0_1(bucket, pk, b, p, items, n_items, cfg, s, set_attributes);
      case 2: return launch_bucket_f0_2(bucket, pk, b, p, items, n_items, cfg, s, set_attributes);
      case 4: return launch_bucket_f0_4(bucket, pk, b, p, items, n_items, cfg, s, set_attributes);
      case 8: return launch_bucket_f0_8(bucket, pk, b, p, items, n_items, cfg, s, set_attributes);
    }
  }
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
