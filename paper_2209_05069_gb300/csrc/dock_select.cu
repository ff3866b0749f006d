// Select Poses (Alg. 1, after the restart loop) as its own kernel, launched after the docking
// kernels of a batch when more than one pose per ligand is kept.  Keeping it out of the docking
// kernel leaves that kernel's register budget (and so its occupancy) untouched.
#include <math_constants.h>

#include "dock_kernels.cuh"

namespace dockgpu {

// Select Poses (Alg. 1, after the restart loop): walks a ligand's restarts in order of final score
// (ties: lowest restart) and keeps a pose when its RMSD to every pose kept so far is at least the
// threshold, until K poses are kept.  RMSD compares the same atoms of two poses in the pocket
// frame, without superposition: sum of squared distances >= n * threshold^2.  Run by one warp (the
// ligand's warp of select_kernel) after every restart's pose is in rs_xyz; slots past the last
// kept pose get restart -1, score -inf and a zero pose.
__device__ void select_poses(const BatchDev& bd, const ParamsDev& p, int l, int a0, int n, float s0, int r0,
                             int lane) {
  int kept[16];  // lane-uniform
  kept[0] = r0;
  int nk = 1;
  float ls = s0;
  int lr = r0;
  const float* sc = bd.restart_score + (size_t)l * p.R;
  const float* rs = bd.rs_xyz + (size_t)a0 * p.R * 3;
  const float lim = (float)n * p.sel_rmsd2;
  while (nk < p.K) {
    // next restart in ranked order after (ls, lr)
    float s = -CUDART_INF_F;
    int r = 0x7fffffff;
    for (int q = lane; q < p.R; q += 32) {
      const float v = __ldcg(sc + q);
      const bool after = v < ls || (v == ls && q > lr);
      if (after && (v > s || (v == s && q < r))) {
        s = v;
        r = q;
      }
    }
    warp_argmax(s, r);
    if (r == 0x7fffffff) break;  // every restart examined
    ls = s;
    lr = r;
    const float* xr = rs + (size_t)r * n * 3;
    bool far = true;
    for (int k = 0; k < nk && far; ++k) {
      const float* xk = rs + (size_t)kept[k] * n * 3;
      float d = 0.f;
      for (int i = lane; i < n; i += 32) {
        const float dx = __ldcg(xr + 3 * i) - __ldcg(xk + 3 * i);
        const float dy = __ldcg(xr + 3 * i + 1) - __ldcg(xk + 3 * i + 1);
        const float dz = __ldcg(xr + 3 * i + 2) - __ldcg(xk + 3 * i + 2);
        d += dx * dx + dy * dy + dz * dz;
      }
      far = warp_sum(d) >= lim;
    }
    if (far) kept[nk++] = r;
  }
  for (int k = 0; k < p.K; ++k) {
    const int r = k < nk ? kept[k] : -1;
    if (lane == 0) {
      bd.select_restart[(size_t)l * p.K + k] = r;
      bd.select_score[(size_t)l * p.K + k] = r >= 0 ? __ldcg(sc + r) : -CUDART_INF_F;
    }
    float* dst = bd.select_xyz + ((size_t)a0 * p.K + (size_t)k * n) * 3;
    const float* src = rs + (size_t)(r >= 0 ? r : 0) * n * 3;
    for (int i = lane; i < 3 * n; i += 32) dst[i] = r >= 0 ? __ldcg(src + i) : 0.f;
  }
}

// One warp per ligand.
__global__ void __launch_bounds__(256) select_kernel(BatchDev bd, ParamsDev p) {
  const int l = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (l >= bd.n_lig) return;
  const int4 h = bd.hdr[l];
  const int r0 = __ldcg(bd.best_restart + l);
  select_poses(bd, p, l, h.x, h.y, __ldcg(bd.best_score + l), r0, threadIdx.x & 31);
}

cudaError_t launch_select(const BatchDev& bd, const ParamsDev& p, cudaStream_t s) {
  if (bd.select_restart == nullptr || bd.n_lig == 0) return cudaSuccess;
  const int wpb = 8;
  select_kernel<<<(bd.n_lig + wpb - 1) / wpb, 32 * wpb, 0, s>>>(bd, p);
  return cudaGetLastError();
}

}  // namespace dockgpu
