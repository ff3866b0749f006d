// The latency form (arXiv 2209.05069 Section 4.1): one ligand spread over the whole GPU.
//
// The paper's latency design docks one ligand at a time with many small kernels, so that a single
// ligand finishes as soon as possible.  Here one ligand takes two kernels, stream-ordered, each
// with one block of 8 warps per (restart, 8 alignment passes):
//  1. lat_align_torsion_kernel: the rigid alignment (Alg. 1's two rotation loops) of all R restarts
//     at once, R x ceil(N*N/32) passes of 32 poses, one pass per warp over every SM; each warp
//     writes its best pose (score, flat index) to a candidate slot.  The last block of a restart to
//     finish (a counter, no waiting) picks the best candidate (highest score, lowest index), moves
//     the pose there and sweeps every rotatable bond in order (Alg. 1's fragment loop) with its 8
//     warps: all 256 angles of a bond in flight and the bump check shared by the warps;
//  2. lat_post_final_kernel: the post-optimisation alignment spread the same way; the last block of
//     a restart applies it, scores the final pose and counts its clashes (all 8 warps, exclusion
//     bitsets in shared memory), and the last restart to finish picks the best restart.
// Every pose is scored with the batched kernel's own arithmetic (lookup's steps, torsion_phase,
// pose_score; the alignment passes only issue their loads earlier) and a (score, index) argmax is
// exact whatever its grouping, so the latency form's results equal the batched form's bit for bit.
#pragma once

#include "dock_kernels.cuh"

namespace dockgpu {

constexpr int kLatWarps = 8;  // warps per block: alignment passes per block, warps per torsion sweep
// Lookups a lane has in flight in the latency form's alignment passes: a lone ligand leaves the GPU
// mostly idle, so each lane issues the loads of kLatUnroll atoms before it sums any of them.
#ifndef DOCK_LAT_UNROLL
#define DOCK_LAT_UNROLL 8
#endif
constexpr int kLatUnroll = DOCK_LAT_UNROLL;

// Alignment passes per restart, and blocks per restart.
__host__ __device__ __forceinline__ int lat_passes(int N) { return (N * N + 31) / 32; }
__host__ __device__ __forceinline__ int lat_chunks(int N) { return (lat_passes(N) + kLatWarps - 1) / kLatWarps; }

// align_pass<GT, 1> with the lookups of U atoms issued before any of them is summed
// (sum_lookups_ilp): the same values summed in the same order, with U loads in flight per lane.
template <int GT, int U>
__device__ __forceinline__ void lat_align_pass(const float4* rel, int n, const float2* tab, int N, const GridK& g,
                                               float tx, float ty, float tz, int f0, int lane, float& best, int& bidx) {
  const float ih = g.inv_h;
  const int NN = N * N;
  const int f = f0 + lane;
  const bool act = f < NN;
  const int ff = act ? f : 0;
  const int i = ff / N, j = ff - (ff / N) * N;
  const float2 ca = tab[i], cb = tab[j];  // (cos, sin)
  const float r00 = cb.x * ih, r01 = cb.y * ca.y * ih, r02 = cb.y * ca.x * ih;
  const float r11 = ca.x * ih, r12 = -ca.y * ih;
  const float r20 = -cb.y * ih, r21 = cb.x * ca.y * ih, r22 = cb.x * ca.x * ih;
  const typename Acc<GT>::type sa = sum_lookups_ilp<GT, U>(g, n, [&](int a) {
    const float4 d = rel[a];
    return make_float3(fmaf(r00, d.x, fmaf(r01, d.y, fmaf(r02, d.z, tx))), fmaf(r11, d.y, fmaf(r12, d.z, ty)),
                       fmaf(r20, d.x, fmaf(r21, d.y, fmaf(r22, d.z, tz))));
  });
  const float s = (float)sa;
  if (act && s > best) {
    best = s;
    bidx = f;
  }
  DOCK_CNT(if (lane == 0) cnt_add(kCntAlignPoses, 32);)
}

// Best candidate of a restart (highest score, lowest index on ties); every lane of the calling
// warp gets it.
__device__ __forceinline__ int lat_pick(const float2* cand, int passes, int lane) {
  float best = -CUDART_INF_F;
  int idx = 0x7fffffff;
  for (int q = lane; q < passes; q += 32) {
    const float2 c = __ldcg(cand + q);
    const int i = __float_as_int(c.y);
    if (c.x > best || (c.x == best && i < idx)) {
      best = c.x;
      idx = i;
    }
  }
  warp_argmax(best, idx);
  return idx;
}

// Counter build: adds the warp's counts to the launch's totals (nothing in the normal build).
__device__ __forceinline__ void lat_flush(const ParamsDev& p) {
  DOCK_CNT(__syncwarp(); const int w = threadIdx.x >> 5, lane = threadIdx.x & 31; if (lane < kCnt && p.exec) {
    const unsigned long long v = g_cnt_smem[w][lane];
    if (v) atomicAdd(p.exec + lane, v);
    g_cnt_smem[w][lane] = 0;
  } __syncwarp();)
}

__device__ __forceinline__ void lat_count_init() {
  DOCK_CNT(if ((threadIdx.x & 31) < kCnt) g_cnt_smem[threadIdx.x >> 5][threadIdx.x & 31] = 0; __syncwarp();)
}

// Shared memory of both kernels: angle tables, the item, the other warps' bump-pair buffers and
// the ligand's exclusion bitsets.
template <int MAXN>
struct LatSmem {
  static __host__ __device__ size_t tables(int N, int A) { return align16(sizeof(float2) * (size_t)(N + A)); }
  static __host__ __device__ size_t bytes(int N, int A) {
    return tables(N, A) + sizeof(ItemSmem<MAXN>) + (size_t)(kLatWarps - 1) * PairCap<MAXN>::value * sizeof(float4) +
           (size_t)MAXN * kMaskWords * sizeof(uint32_t) + 16;
  }
};

__device__ __forceinline__ void lat_tables(float2* tab, int N, int A) {
  for (int t = threadIdx.x; t < N + A; t += blockDim.x) {
    float sn, cs;
    if (t < N)
      sincospif((float)(2 * t) / (float)N, &sn, &cs);
    else
      sincospif((float)(2 * (t - N)) / (float)A, &sn, &cs);
    tab[t] = make_float2(cs, sn);
  }
}

// The alignment passes of this block (restart r, chunk c): warp w scores pass c * 8 + w of the pose
// whose centroid-relative coordinates are in ws.u.rel and writes its best to the candidates; then
// returns whether this block is the last of restart r to finish (it then sees every candidate).
template <int MAXN, int GT>
__device__ __forceinline__ bool lat_passes_then_last(ItemSmem<MAXN>& ws, const float2* tab, const ParamsDev& p,
                                                     const GridK& g, int n, int r, int chunk, const LatScratch& sc,
                                                     int* flag) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int passes = lat_passes(p.N);
  const int q = chunk * kLatWarps + warp;
  if (q < passes) {
    const float3 t = centre_grid(ws.bc, g);
    float best = -CUDART_INF_F;
    int bidx = 0x7fffffff;
    lat_align_pass<GT, kLatUnroll>(ws.u.rel, n, tab, p.N, g, t.x, t.y, t.z, q * 32, lane, best, bidx);
    warp_argmax(best, bidx);
    if (lane == 0) sc.cand[(size_t)r * passes + q] = make_float2(best, __int_as_float(bidx));
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(sc.done + r, 1u);
    const bool last = prev == (unsigned)(lat_chunks(p.N) - 1);
    if (last) sc.done[r] = 0;  // ready for the next kernel or ligand
    *flag = last;
  }
  __syncthreads();
  const bool last = *flag != 0;
  if (last) __threadfence();
  return last;
}

// Kernel 1.  Block b: restart b / chunks, alignment chunk b % chunks.
template <int MAXN, int GT>
__global__ void __launch_bounds__(kLatWarps * 32) lat_align_torsion_kernel(PocketDev pk, BatchDev bd, ParamsDev p,
                                                                           int l, LatScratch sc) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* tab_al = reinterpret_cast<float2*>(smem);
  float2* tab_to = tab_al + p.N;
  ItemSmem<MAXN>& ws = *reinterpret_cast<ItemSmem<MAXN>*>(smem + LatSmem<MAXN>::tables(p.N, p.A));
  float4* xp = reinterpret_cast<float4*>(&ws + 1);
  int* flag = reinterpret_cast<int*>(xp + (kLatWarps - 1) * PairCap<MAXN>::value);
  lat_count_init();
  lat_tables(tab_al, p.N, p.A);
  const int chunks = lat_chunks(p.N);
  const int r = blockIdx.x / chunks, chunk = blockIdx.x - r * chunks;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int4 h = bd.hdr[l];
  const int a0 = h.x, n = h.y, rb0 = h.z, B = h.w;
  const GridK g = make_gridk(pk);
  for (int i = threadIdx.x; i < n; i += blockDim.x) ws.pos[i] = make_float4(bd.x[a0 + i], bd.y[a0 + i], bd.z[a0 + i], 0.f);
  __syncthreads();
  if (warp == 0) {
    start_pose(ws, n, bd.ids[l], p.seed, r, pk, lane);
    __syncwarp();
    align_centre(ws, n, lane);
  }
  __syncthreads();
  if (lat_passes_then_last<MAXN, GT>(ws, tab_al, p, g, n, r, chunk, sc, flag)) {
    // the restart's alignment choice, then its torsion sweep with the block's 8 warps
    const int ai = lat_pick(sc.cand + (size_t)r * lat_passes(p.N), lat_passes(p.N), lane);
    const float4 cc = ws.bc;
    align_move(ws, n, tab_al, p.N, ai, make_float3(cc.x, cc.y, cc.z), threadIdx.x, blockDim.x);
    __syncthreads();
    float4* xpairs = warp > 0 ? xp + (warp - 1) * PairCap<MAXN>::value : nullptr;
    for (int bi = 0; bi < B; ++bi) {
      const uint32_t ab = __ldg(bd.rot_ab + rb0 + bi);
      int rej = 0;
      // the bump check is shared by the warps whenever there is a pair to test (the same result:
      // an angle bumps if any pair bumps)
      const int k = torsion_phase<MAXN, GT, kLatWarps, 1, 1, 4, kLatUnroll>(ws, n, (int)(ab & 0xffffu), (int)(ab >> 16),
                                                          bd.mask + (size_t)(rb0 + bi) * kMaskWords, tab_to, p.A,
                                                          p.dc2, p.early_exit != 0, g, warp, lane, 0, xpairs, rej);
      if (warp == 0 && lane == 0) {
        const size_t o = (size_t)rb0 * p.R + (size_t)r * B + bi;
        bd.tors_idx[o] = k;
        bd.rejected[o] = rej;
      }
    }
    if (threadIdx.x == 0) bd.align_idx[(size_t)l * p.R + r] = ai;
    for (int i = threadIdx.x; i < n; i += blockDim.x) sc.pose[(size_t)r * kMaxAtoms + i] = ws.pos[i];
  }
  lat_flush(p);
}

// Kernel 2.  Block b: restart b / chunks, post-alignment chunk b % chunks (one block per restart
// and no passes without post_align).
template <int MAXN, int GT>
__global__ void __launch_bounds__(kLatWarps * 32) lat_post_final_kernel(PocketDev pk, BatchDev bd, ParamsDev p, int l,
                                                                        LatScratch sc) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* tab = reinterpret_cast<float2*>(smem);
  ItemSmem<MAXN>& ws = *reinterpret_cast<ItemSmem<MAXN>*>(smem + LatSmem<MAXN>::tables(p.N, 0));
  float4* xp = reinterpret_cast<float4*>(&ws + 1);
  int* flag = reinterpret_cast<int*>(xp + (kLatWarps - 1) * PairCap<MAXN>::value);
  uint32_t* excl = reinterpret_cast<uint32_t*>(flag + 4);
  __shared__ int clash_part[kLatWarps];
  lat_count_init();
  lat_tables(tab, p.N, 0);
  const int chunks = p.post_align ? lat_chunks(p.N) : 1;
  const int r = blockIdx.x / chunks, chunk = blockIdx.x - r * chunks;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int4 h = bd.hdr[l];
  const int a0 = h.x, n = h.y;
  const GridK g = make_gridk(pk);
  for (int i = threadIdx.x; i < n; i += blockDim.x) ws.pos[i] = __ldcg(sc.pose + (size_t)r * kMaxAtoms + i);
  __syncthreads();
  int pi = -1;
  if (p.post_align) {
    if (warp == 0) align_centre(ws, n, lane);
    __syncthreads();
    if (!lat_passes_then_last<MAXN, GT>(ws, tab, p, g, n, r, chunk, sc, flag)) {
      lat_flush(p);
      return;
    }
    pi = lat_pick(sc.cand + (size_t)r * lat_passes(p.N), lat_passes(p.N), lane);
    const float4 cc = ws.bc;
    align_move(ws, n, tab, p.N, pi, make_float3(cc.x, cc.y, cc.z), threadIdx.x, blockDim.x);
  }
  // final score (warp 0, the batched kernel's summation) and clash count (all warps, integers)
  for (int t = threadIdx.x; t < n * kMaskWords; t += blockDim.x) excl[t] = __ldg(bd.excl + (size_t)a0 * kMaskWords + t);
  __syncthreads();
  int c = 0;
  for (int i = warp; i < n; i += kLatWarps) {
    const float4 pa = ws.pos[i];
    for (int j = i + 1 + lane; j < n; j += 32) {
      if ((excl[i * kMaskWords + (j >> 5)] >> (j & 31)) & 1u) continue;
      const float4 q = ws.pos[j];
      const float dx = pa.x - q.x, dy = pa.y - q.y, dz = pa.z - q.z;
      c += (dx * dx + dy * dy + dz * dz) < p.dc2;
    }
  }
  c = warp_sum_i(c);
  if (lane == 0) clash_part[warp] = c;
  __syncthreads();
  if (warp == 0) {
    const float s = pose_score<MAXN, GT>(ws, n, g, lane);
    int cc = 0;
#pragma unroll
    for (int w = 0; w < kLatWarps; ++w) cc += clash_part[w];
    const int ai = __ldcg(bd.align_idx + (size_t)l * p.R + r);
    finish_restart<MAXN>(ws, bd, p, l, r, ai, pi, s, cc, lane);
  }
  lat_flush(p);
}

// Queues ligand l's latency-form kernels on stream s; returns the first error.  l < 0 only applies
// the kernels' shared-memory attributes (outside a stream capture).
template <int MAXN, int GT>
cudaError_t lat_launch_t(const PocketDev& pk, const BatchDev& bd, const ParamsDev& p, int l, const LatScratch& sc,
                         cudaStream_t s, int* launches) {
  const size_t sm1 = LatSmem<MAXN>::bytes(p.N, p.A), sm2 = LatSmem<MAXN>::bytes(p.N, 0);
  if (l < 0) {
    cudaError_t e = cudaFuncSetAttribute(lat_align_torsion_kernel<MAXN, GT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(lat_post_final_kernel<MAXN, GT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
    return e;
  }
  const int chunks = lat_chunks(p.N);
  lat_align_torsion_kernel<MAXN, GT><<<p.R * chunks, kLatWarps * 32, sm1, s>>>(pk, bd, p, l, sc);
  lat_post_final_kernel<MAXN, GT><<<p.R * (p.post_align ? chunks : 1), kLatWarps * 32, sm2, s>>>(pk, bd, p, l, sc);
  *launches += 2;
  return cudaGetLastError();
}

}  // namespace dockgpu
