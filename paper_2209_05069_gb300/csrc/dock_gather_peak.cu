// Stand-alone pocket-gather rate: the roofline denominator of the docking kernel, measured on the
// GPU it runs on.  No counterpart in the paper (measurement only).
//
// The docking kernel is bound by scattered pocket lookups (one corner-packed cell, or one int16
// voxel, per atom per pose).  This kernel issues the same lookups — the same lookup<GT> code on the
// same pocket layout — at independent uniformly random positions inside the pocket's nonzero box,
// so that every lookup is a scattered access, and does nothing else: no bump check, no torsion
// geometry, no argmax.  Its lookups per second are the hardware's rate for scattered lookups of
// that layout.  Lookups of the docking kernel that fall in a sector a neighbouring lane also reads
// (neighbouring torsion angles move an atom by less than a cell) can push it a little above this
// rate; the int16 grid, whose 2-byte voxels put many neighbours in one sector, far above it.
#include "dock.h"
#include "dock_kernels.cuh"

namespace dockgpu {
namespace {

constexpr int kPeakLookups = 8192;  // per lane: 2.5 G lookups per run on 152 SMs
constexpr int kPeakBlocksPerSM = 8;
constexpr int kPeakThreads = 256;

// Uniform float in [lo, hi) from the next output of a 32-bit LCG (Numerical Recipes constants),
// without the conversion unit: the top 23 bits become the mantissa of a float in [1, 2).
__device__ __forceinline__ float next_uniform(unsigned& state, float lo, float span) {
  state = state * 1664525u + 1013904223u;
  return fmaf(__uint_as_float(0x3F800000u | (state >> 9)) - 1.0f, span, lo);
}

template <int GT>
__global__ void __launch_bounds__(kPeakThreads) gather_peak_kernel(PocketDev pk, float* out) {
  const GridK g = make_gridk(pk);
  const int lane = threadIdx.x & 31;
  const unsigned tid = (unsigned)(blockIdx.x * blockDim.x + threadIdx.x);
  unsigned state = tid * 2654435761u + 12345u;
  // the nonzero box in grid coordinates (for the integer grid: its stored box, in the box-relative
  // coordinates its lookup takes)
  const float lx = GT == 2 ? 0.f : pk.lox, ly = GT == 2 ? 0.f : pk.loy, lz = GT == 2 ? 0.f : pk.loz;
  const float sx = fmaxf(pk.hix - pk.lox, 0.f), sy = fmaxf(pk.hiy - pk.loy, 0.f), sz = fmaxf(pk.hiz - pk.loz, 0.f);
  float acc = 0.f;
#pragma unroll 4
  for (int k = 0; k < kPeakLookups; ++k) {
    const float u = next_uniform(state, lx, sx);
    const float v = next_uniform(state, ly, sy);
    const float w = next_uniform(state, lz, sz);
    acc += lookup<GT>(g, u, v, w);
  }
  acc = warp_sum(acc);
  if (lane == 0) out[tid >> 5] = acc;
}

}  // namespace
}  // namespace dockgpu

extern "C" int dock_gather_peak(dock_ctx* ctx, int32_t pocket_id, double* lookups_per_s) {
  using namespace dockgpu;
  if (!ctx) return DOCK_ERR_INVALID;
  if (!lookups_per_s) return record_error(ctx, DOCK_ERR_INVALID, "lookups_per_s is NULL");
  PocketDev pk;
  cudaStream_t s;
  int rc = pocket_view(ctx, pocket_id, &pk, &s);
  if (rc != DOCK_OK) return rc;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * kPeakBlocksPerSM;
  const int warps = blocks * kPeakThreads / 32;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(float) * warps);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first run warms up
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
      if (pk.dtype == 2)
        gather_peak_kernel<2><<<blocks, kPeakThreads, 0, s>>>(pk, out);
      else if (pk.dtype == 1)
        gather_peak_kernel<1><<<blocks, kPeakThreads, 0, s>>>(pk, out);
      else
        gather_peak_kernel<0><<<blocks, kPeakThreads, 0, s>>>(pk, out);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (e != cudaSuccess) return record_error(ctx, DOCK_ERR_CUDA, cudaGetErrorString(e));
  const double lookups = (double)warps * 32 * kPeakLookups;
  *lookups_per_s = lookups / (best * 1e-3);
  return DOCK_OK;
}
