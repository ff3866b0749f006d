// Fused docking kernel (arXiv 2209.05069, Alg. 1), one warp per (ligand, restart).
//
// Per work item the warp runs: starting pose -> rigid alignment over N x N x/y angles (the rotation loops)
// -> torsion sweep of every rotatable bond in order with bump check (the fragment loop) -> optional
// second rigid alignment -> final score and clash count.  The last warp of a ligand to finish
// picks the best restart.  Geometry is FP32; the pocket grid is read through corner-packed cells
// (one 32-byte FP32 or 16-byte FP16 load per trilinear lookup) or, for an integer grid, as int16
// voxels (one 2-byte load of the nearest voxel).  Template parameter GT: 0 FP32, 1 FP16, 2 int16.
//
// Mapping onto the warp (the paper's batched design gives one warp one ligand, lanes over atoms;
// here lanes own poses so every lane stays busy whatever the ligand size):
//  * alignment: lane = one of the N*N rotations; the lane rotates every atom (broadcast from
//    shared memory) and sums its lookups; a warp argmax picks the pose.
//  * torsion sweep: lane = one torsion angle.  The moving atoms' positions are written as
//    x(theta) = c + cos(theta) r + sin(theta) w (c on the axis, r and w perpendicular), so one
//    angle costs 6 FMA per atom before its lookup.  For the bump check every moving/fixed pair
//    has d^2(theta) = C + Pa cos(theta) + Pb sin(theta); pairs whose minimum over theta stays
//    above d_c^2 are dropped once per bond and each angle tests only the remaining pairs.
#pragma once

#include <cuda_fp16.h>
#include <math_constants.h>

#include <mutex>

#include "dock_internal.h"

// Register budget of the docking kernel.  dock_kernel: blocks of up to 256 threads, 4 of them
// resident per SM (64 registers, a few spilled bytes outside the lookup loops).  Left to itself
// ptxas takes 66-80 registers with 2-8 warps per item and over 100 with one; the bound measured
// 7-15% faster with 2 or 4 warps per item and 19-43% faster with 8 on databases of 10^2-10^4
// ligands.  dock_kernel_wide, the entry point of the FP32 grid with one warp per item: 96
// registers (5 blocks of 128 threads per SM).  A sweep of one cap for every instantiation (64, 72,
// 80, 96) on the uneven size mix and on 80-150-atom molecules kept 64 for the FP16 and int16 grids
// and for 2 or more warps per item; FP32 with one warp per item and a pose tile of 2 ran 1-4% faster
// per bucket at 96, the fastest shape of the 64-atom FP32 bucket.  A register cap (__maxnreg__) in
// place of the launch bound generates other code: 64 registers that way made small serving batches
// (8 warps per item) 8% slower at the median, so the bound stays.  DOCK_MAXNREG caps both entry
// points at one count instead.
#ifdef DOCK_MAXNREG
#define DOCK_KERNEL_BOUNDS __maxnreg__(DOCK_MAXNREG)
#define DOCK_KERNEL_WIDE_BOUNDS __maxnreg__(DOCK_MAXNREG)
#else
#define DOCK_KERNEL_BOUNDS __launch_bounds__(256, 4)
#define DOCK_KERNEL_WIDE_BOUNDS __maxnreg__(96)
#endif

// PTX load used for one FP32 corner-packed cell (32 bytes, one sector).
#ifndef DOCK_CELL_LOAD_F32
#define DOCK_CELL_LOAD_F32 "ld.global.nc.v8.f32"
#endif

namespace dockgpu {

constexpr unsigned kFull = 0xffffffffu;

// ---- executed-work counters (the counter build, DOCK_COUNT_WORK) ---------------------------------
// Each warp adds its events to its own shared-memory slot (one lane per warp-wide event); after each
// work item the slot is added to the launch's global counters.  In the normal build DOCK_CNT(...)
// expands to nothing, so the product kernels carry no trace of it.
#ifdef DOCK_COUNT_WORK
static __shared__ unsigned long long g_cnt_smem[8][kCnt];
static_assert(kCnt <= 32, "one lane per counter flushes a warp's slot");
__device__ __forceinline__ void cnt_add(int k, unsigned long long v) {
  if (v) atomicAdd(&g_cnt_smem[threadIdx.x >> 5][k], v);
}
// Lookup event of the active lanes: evaluated, loads issued, distinct sectors of those loads.
__device__ __forceinline__ void cnt_lookup(bool issued, unsigned long long addr) {
  const unsigned act = __activemask();
  const int lane = threadIdx.x & 31;
  const unsigned issue = __ballot_sync(act, issued);
  const unsigned long long sec = issued ? (addr >> 5) : ~0ull;
  const unsigned m = __match_any_sync(act, sec);
  const unsigned leaders = __ballot_sync(act, issued && lane == __ffs(m) - 1);
  const unsigned long long line = issued ? (addr >> 7) : ~0ull;
  const unsigned ml = __match_any_sync(act, line);
  const unsigned line_leaders = __ballot_sync(act, issued && lane == __ffs(ml) - 1);
  if (lane == __ffs(act) - 1) {
    cnt_add(kCntLookups, __popc(act));
    cnt_add(kCntLoads, __popc(issue));
    cnt_add(kCntSectors, __popc(leaders));
    cnt_add(kCntLines, __popc(line_leaders));
  }
}
#define DOCK_CNT(...) __VA_ARGS__
#else
#define DOCK_CNT(...)
#endif

// ---- small warp helpers ------------------------------------------------------------------------

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Warp-wide (max score, lowest index among equal scores); every lane gets the result.
__device__ __forceinline__ void warp_argmax(float& s, int& idx) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const float s2 = __shfl_xor_sync(kFull, s, o);
    const int i2 = __shfl_xor_sync(kFull, idx, o);
    if (s2 > s || (s2 == s && i2 < idx)) {
      s = s2;
      idx = i2;
    }
  }
}

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): output number k >= 1 of the generator
// started from `state`.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long state, unsigned long long k) {
  unsigned long long z = state + k * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Starting orientation of restart r: identity for r = 0, else Shoemake's uniform random
// rotation (Graphics Gems III) from three SplitMix64 draws keyed by the ligand id and the seed.
__device__ __forceinline__ void restart_rotation(unsigned long long id, unsigned long long seed, int r, float R[9]) {
  if (r == 0) {
    R[0] = 1.f; R[1] = 0.f; R[2] = 0.f;
    R[3] = 0.f; R[4] = 1.f; R[5] = 0.f;
    R[6] = 0.f; R[7] = 0.f; R[8] = 1.f;
    return;
  }
  const unsigned long long key = splitmix64(seed ^ id, 1ull);
  float u[3];
#pragma unroll
  for (int t = 0; t < 3; ++t)
    u[t] = (float)(unsigned)(splitmix64(key, (unsigned long long)(3 * r + t + 1)) >> 40) * (1.0f / 16777216.0f);
  const float a = sqrtf(1.0f - u[0]), b = sqrtf(u[0]);
  float s1, c1, s2, c2;
  sincospif(2.0f * u[1], &s1, &c1);
  sincospif(2.0f * u[2], &s2, &c2);
  const float qx = a * s1, qy = a * c1, qz = b * s2, qw = b * c2;
  R[0] = 1.f - 2.f * (qy * qy + qz * qz); R[1] = 2.f * (qx * qy - qw * qz); R[2] = 2.f * (qx * qz + qw * qy);
  R[3] = 2.f * (qx * qy + qw * qz); R[4] = 1.f - 2.f * (qx * qx + qz * qz); R[5] = 2.f * (qy * qz - qw * qx);
  R[6] = 2.f * (qx * qz - qw * qy); R[7] = 2.f * (qy * qz + qw * qx); R[8] = 1.f - 2.f * (qx * qx + qy * qy);
}

// ---- pocket lookups ------------------------------------------------------------------------------

struct GridK {
  const void* cells;       // integer grid: the stored box of voxels (nonzero voxels and a zero border)
  int nx1, ny1;            // cells per row / per column (n - 1); stored box row / column length for int16
  int imax, jmax, kmax;    // largest lower-corner index (n - 2)
  float lox, loy, loz;     // grid-coordinate box outside which every lookup is exactly 0
  float hix, hiy, hiz;
  int ihix, ihiy, ihiz;    // integer grid: largest box-relative voxel index
  float inv_h, ox, oy, oz;
  int zero_cell;           // trilinear grids: the all-zero cell past the last one
};

__device__ __forceinline__ GridK make_gridk(const PocketDev& p) {
  GridK g;
  g.cells = p.cells;
  g.nx1 = p.nx - 1;
  g.ny1 = p.ny - 1;
  g.imax = p.nx - 2;
  g.jmax = p.ny - 2;
  g.kmax = p.nz - 2;
  g.lox = p.lox;
  g.loy = p.loy;
  g.loz = p.loz;
  g.hix = p.hix;
  g.hiy = p.hiy;
  g.hiz = p.hiz;
  g.ihix = g.ihiy = g.ihiz = 0;
  g.zero_cell = (p.nx - 1) * (p.ny - 1) * (p.nz - 1);
  g.inv_h = p.inv_h;
  g.ox = p.ox;
  g.oy = p.oy;
  g.oz = p.oz;
  if (p.dtype == 2) {
    // stored box [lo, hi] per axis: row and column length, largest box-relative index
    g.nx1 = (int)p.hix - (int)p.lox + 1;
    g.ny1 = (int)p.hiy - (int)p.loy + 1;
    g.ihix = g.nx1 - 1;
    g.ihiy = g.ny1 - 1;
    g.ihiz = (int)p.hiz - (int)p.loz;
    // the origin moves to the stored box's first voxel, so the voxel indices the kernel computes
    // are box-relative, and the +1/2 of the nearest-voxel rounding floor(u + 1/2) is folded into
    // it too, so every grid coordinate arrives shifted and a lookup only floors it
    g.ox = p.ox + p.spacing * (p.lox - 0.5f);
    g.oy = p.oy + p.spacing * (p.loy - 0.5f);
    g.oz = p.oz + p.spacing * (p.loz - 0.5f);
  }
  return g;
}

// Trilinear interpolation at grid coordinates (u, v, w); 0 outside [0, n-1] on any axis.  Inside
// the grid but outside the box of nonzero voxels the value is exactly 0 too, so no load is issued.
// Integer grid (GT == 2): the value of the nearest voxel, index floor(u + 1/2) per axis (half-way
// reads the upper voxel), 0 outside the grid; only the nonzero voxels and a zero border are
// stored, and the index is clamped into that box.  Its coordinates arrive relative to the box and
// shifted by +1/2 (make_gridk moves the origin), so u here is u + 1/2 - (first stored voxel).
// Integer values are exact in FP32 and their sums stay exact below 2^24, so every score of an
// integer grid is exact whatever the summation order.
constexpr float kRound = 12582912.0f;  // 1.5 * 2^23: kRound + q has unit spacing for |q| < 2^22

// Integer grid: the int16 value of the nearest voxel.  One round-down conversion per axis
// (saturating) to a box-relative index, clamped by one unsigned min: an index past the box lands on
// its far border, a negative one wraps to it, and the border is zero.
__device__ __forceinline__ int voxel_value(const GridK& g, float u, float v, float w) {
  const unsigned i = min((unsigned)__float2int_rd(u), (unsigned)g.ihix);
  const unsigned j = min((unsigned)__float2int_rd(v), (unsigned)g.ihiy);
  const unsigned k = min((unsigned)__float2int_rd(w), (unsigned)g.ihiz);
  const short* a = reinterpret_cast<const short*>(g.cells) + (k * (unsigned)g.ny1 + j) * (unsigned)g.nx1 + i;
  DOCK_CNT(cnt_lookup(true, (unsigned long long)a);)
  return __ldg(a);
}

// A trilinear lookup in three steps, shared by lookup() and the latency form's batched fetches
// (lat_lookups): the cell and fractional position, the cell's 8 corner values (one load), the
// interpolation.  An atom outside the box of nonzero voxels has value exactly 0.
struct CellPos {
  int cell;         // corner-packed cell index (meaningful when inside)
  float tx, ty, tz;
  bool inside;
};

__device__ __forceinline__ CellPos cell_pos(const GridK& g, float u, float v, float w) {
  CellPos c;
  c.inside = (u >= g.lox) & (v >= g.loy) & (w >= g.loz) & (u <= g.hix) & (v <= g.hiy) & (w <= g.hiz);
  const int i0 = min(__float2int_rd(u), g.imax);
  const int j0 = min(__float2int_rd(v), g.jmax);
  const int k0 = min(__float2int_rd(w), g.kmax);
  c.tx = u - (float)i0;
  c.ty = v - (float)j0;
  c.tz = w - (float)k0;
  c.cell = (k0 * g.ny1 + j0) * g.nx1 + i0;
  return c;
}

// The 8 corner values of an FP32 cell (one 256-bit load).
template <int GT>
__device__ __forceinline__ void load_cell(const GridK& g, int cell, float (&c)[8]) {
  const float* p = reinterpret_cast<const float*>(g.cells) + 8 * (size_t)cell;
  asm(DOCK_CELL_LOAD_F32 " {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=f"(c[0]), "=f"(c[1]), "=f"(c[2]), "=f"(c[3]), "=f"(c[4]), "=f"(c[5]), "=f"(c[6]), "=f"(c[7])
      : "l"(p));
}

// An FP16 cell (one 128-bit load) as the 4 x-interpolation inputs it feeds: the lower corner's value
// b and the difference d = upper - lower along x, for (dj, dk) = (0,0), (1,0), (0,1), (1,1).  d comes
// from the mixed-precision subtraction (the f16 operand converted exactly, then one FP32 rounding:
// the value that converting both corners and subtracting gives, with one conversion fewer).
struct CellF16 {
  float b[4], d[4];
};

__device__ __forceinline__ void load_cell_f16(const GridK& g, int cell, CellF16& v) {
  const uint4 q = __ldg(reinterpret_cast<const uint4*>(g.cells) + cell);
  const unsigned h[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int t = 0; t < 4; ++t)
    asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
        "cvt.f32.f16 %0, lo;\n\tsub.rn.f32.f16 %1, hi, %0;\n\t}"
        : "=&f"(v.b[t]), "=f"(v.d[t])
        : "r"(h[t]));
}

// trilerp of an FP16 cell: the same operations in the same order.
__device__ __forceinline__ float trilerp_f16(const CellF16& v, const CellPos& cp) {
  const float c00 = fmaf(cp.tx, v.d[0], v.b[0]);
  const float c10 = fmaf(cp.tx, v.d[1], v.b[1]);
  const float c01 = fmaf(cp.tx, v.d[2], v.b[2]);
  const float c11 = fmaf(cp.tx, v.d[3], v.b[3]);
  const float d0 = fmaf(cp.ty, c10 - c00, c00);
  const float d1 = fmaf(cp.ty, c11 - c01, c01);
  return cp.inside ? fmaf(cp.tz, d1 - d0, d0) : 0.f;
}

__device__ __forceinline__ float trilerp(const float (&c)[8], const CellPos& cp) {
  const float c00 = fmaf(cp.tx, c[1] - c[0], c[0]);
  const float c10 = fmaf(cp.tx, c[3] - c[2], c[2]);
  const float c01 = fmaf(cp.tx, c[5] - c[4], c[4]);
  const float c11 = fmaf(cp.tx, c[7] - c[6], c[6]);
  const float d0 = fmaf(cp.ty, c10 - c00, c00);
  const float d1 = fmaf(cp.ty, c11 - c01, c01);
  return cp.inside ? fmaf(cp.tz, d1 - d0, d0) : 0.f;
}

template <int GT>
__device__ __forceinline__ float lookup(const GridK& g, float u, float v, float w) {
  if (GT == 2) {
    const int q = voxel_value(g, u, v, w);
    return __int_as_float(__float_as_int(kRound) + q) - kRound;  // exact int16 -> float
  }
  const CellPos cp = cell_pos(g, u, v, w);
  DOCK_CNT(cnt_lookup(cp.inside, (unsigned long long)g.cells + (unsigned long long)cp.cell * (GT == 1 ? 16u : 32u));)
  if constexpr (GT == 1) {
    CellF16 c = {};
    if (cp.inside) load_cell_f16(g, cp.cell, c);
    return trilerp_f16(c, cp);
  } else {
    float c[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (cp.inside) load_cell<GT>(g, cp.cell, c);
    return trilerp(c, cp);
  }
}

// The type a pose's lookups are summed in: float for the trilinear grids; int for the integer
// grid, whose sums are exact integers (|sum| <= 160 * 32767 < 2^24), converted to float once per
// pose, which is exact too.
template <int GT>
struct Acc {
  using type = float;
};
template <>
struct Acc<2> {
  using type = int;
};

template <int GT>
__device__ __forceinline__ typename Acc<GT>::type lookup_acc(const GridK& g, float u, float v, float w) {
  if constexpr (GT == 2)
    return voxel_value(g, u, v, w);
  else
    return lookup<GT>(g, u, v, w);
}

// The sum of the lookups at positions pos(0), ..., pos(m - 1), in that order, with the loads of U
// positions issued before any of them is summed (a position outside the box reads the all-zero cell
// instead of skipping its load): the values and the sum of lookup_acc, with U loads in flight per
// lane.  For the latency form, whose lone warps cannot hide load latency behind other warps.
template <int GT, int U, class Pos>
__device__ __forceinline__ typename Acc<GT>::type sum_lookups_ilp(const GridK& g, int m, const Pos& pos) {
  typename Acc<GT>::type sa = 0;
  for (int e0 = 0; e0 < m; e0 += U) {
    if constexpr (GT == 2) {
      int q[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const float3 p = pos(min(e0 + k, m - 1));
        q[k] = voxel_value(g, p.x, p.y, p.z);
      }
#pragma unroll
      for (int k = 0; k < U; ++k)
        if (e0 + k < m) sa += q[k];
    } else if constexpr (GT == 1) {
      CellPos cp[U];
      CellF16 c[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const float3 p = pos(min(e0 + k, m - 1));
        cp[k] = cell_pos(g, p.x, p.y, p.z);
        const int cell = cp[k].inside ? cp[k].cell : g.zero_cell;
        DOCK_CNT(cnt_lookup(true, (unsigned long long)g.cells + (unsigned long long)cell * 16u);)
        load_cell_f16(g, cell, c[k]);
      }
#pragma unroll
      for (int k = 0; k < U; ++k)
        if (e0 + k < m) sa += trilerp_f16(c[k], cp[k]);
    } else {
      CellPos cp[U];
      float c[U][8];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const float3 p = pos(min(e0 + k, m - 1));
        cp[k] = cell_pos(g, p.x, p.y, p.z);
        const int cell = cp[k].inside ? cp[k].cell : g.zero_cell;
        DOCK_CNT(cnt_lookup(true, (unsigned long long)g.cells + (unsigned long long)cell * (GT == 1 ? 16u : 32u));)
        load_cell<GT>(g, cell, c[k]);
      }
#pragma unroll
      for (int k = 0; k < U; ++k)
        if (e0 + k < m) sa += trilerp(c[k], cp[k]);
    }
  }
  return sa;
}

// Lookup at a position in Angstrom.
template <int GT>
__device__ __forceinline__ typename Acc<GT>::type lookup_at(const GridK& g, float x, float y, float z) {
  return lookup_acc<GT>(g, (x - g.ox) * g.inv_h, (y - g.oy) * g.inv_h, (z - g.oz) * g.inv_h);
}

// ---- per-item shared memory ----------------------------------------------------------------------

// Moving/fixed atom pairs from which the bump check of one bond is split over the item's warps.
constexpr int kSplitPairs = 256;

// Bump pairs held in shared memory at once; more are processed in chunks of this size.  Larger
// molecules have bonds with thousands of moving/fixed pairs, so their chunks are larger (each chunk
// costs a walk over the bond's angle passes).
template <int MAXN>
struct PairCap {
  static constexpr int value = MAXN >= 96 ? 64 : 32;
};

// Shared memory of one work item, used by the G warps that dock it.
template <int MAXN>
struct __align__(16) ItemSmem {
  float4 pos[MAXN];                 // current pose (w unused)
  union {
    float4 rel[MAXN];               // alignment: pose relative to its centroid
    struct {
      float4 B[MAXN];               // torsion: circle centre of each moving atom, grid units (w = atom)
      float4 R[MAXN];               //          in-plane radius vector r / h, and (u x r / h).x
      float2 W[MAXN];               //          (u x r / h).y, .z
    } mov;
  } u;
  float4 pairs[PairCap<MAXN>::value];  // active bump pairs (C, Pa, Pb, -)
  unsigned char fixed_idx[(MAXN + 15) / 16 * 16];
  // exchange between the warps of the item
  float xs[8];                      // each warp's best score
  int xi[8];                        // and its index
  unsigned clash[32];               // per lane: bump bits of its angle passes (current bond)
  float4 bc;                        // a broadcast vector (centroid)
  int bi[4];                        // broadcast integers: moving-atom count, -, fixed-atom count, work item
};

// Barrier of the G warps docking one item (named barrier 1 + group; a warp barrier when G = 1).
template <int G>
__device__ __forceinline__ void group_sync(int grp) {
  if (G == 1)
    __syncwarp();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(G * 32) : "memory");
}

// Argmax (highest score, lowest index on ties) over the G warps of an item; every thread of the
// group gets the result.  The order of the comparison does not change the result.
template <int MAXN, int G>
__device__ __forceinline__ void group_argmax(ItemSmem<MAXN>& ws, float& best, int& idx, int wig, int lane, int grp) {
  warp_argmax(best, idx);
  if (G == 1) return;
  if (lane == 0) {
    ws.xs[wig] = best;
    ws.xi[wig] = idx;
  }
  group_sync<G>(grp);
  float b = ws.xs[0];
  int i = ws.xi[0];
#pragma unroll
  for (int w = 1; w < G; ++w) {
    const float s2 = ws.xs[w];
    const int i2 = ws.xi[w];
    if (s2 > b || (s2 == b && i2 < i)) {
      b = s2;
      i = i2;
    }
  }
  best = b;
  idx = i;
  group_sync<G>(grp);
}

__device__ __forceinline__ float3 warp_centroid(const float4* pos, int n, int lane) {
  float sx = 0.f, sy = 0.f, sz = 0.f;
  for (int i = lane; i < n; i += 32) {
    const float4 q = pos[i];
    sx += q.x;
    sy += q.y;
    sz += q.z;
  }
  const float inv = 1.0f / (float)n;
  return make_float3(warp_sum(sx) * inv, warp_sum(sy) * inv, warp_sum(sz) * inv);
}

// ---- rigid alignment (Alg. 1, the two rotation loops) ---------------------------------------------

// The alignment in three steps, shared by the batched kernel (align_phase) and the latency form's
// kernels, so that both evaluate every pose with the same operations:
//  1. align_centre (one warp): centroid c of the current pose into ws.bc, the pose relative to it
//     into ws.u.rel;
//  2. align_pass (one warp): scores the 32 poses f0 + lane, pose (i, j) = c + Ry(2 pi j / N)
//     Rx(2 pi i / N) (P - c), and folds them into the lane's (best, index);
//  3. align_move: moves the ligand to the chosen flat index i*N + j.
template <int MAXN>
__device__ __forceinline__ void align_centre(ItemSmem<MAXN>& ws, int n, int lane) {
  const float3 c = warp_centroid(ws.pos, n, lane);
  for (int i = lane; i < n; i += 32) {
    const float4 q = ws.pos[i];
    ws.u.rel[i] = make_float4(q.x - c.x, q.y - c.y, q.z - c.z, 0.f);
  }
  if (lane == 0) ws.bc = make_float4(c.x, c.y, c.z, 0.f);
}

// T (the pose tile) poses per lane: f0 + lane + 32 t, t < T; each atom's coordinates are read from
// shared memory once for the T poses, which keep T independent lookup chains in flight.  Every
// pose's sum is formed in atom order whatever T is, and a lane meets its poses in increasing index.
// U is the atom loop's unrolling (lookups issued ahead of their sums); it changes no result.
template <int GT, int T, int U = (T == 1 ? 4 : 2)>
__device__ __forceinline__ void align_pass(const float4* rel, int n, const float2* tab, int N, const GridK& g,
                                           float tx, float ty, float tz, int f0, int lane, float& best, int& bidx) {
  const float ih = g.inv_h;
  const int NN = N * N;
  int f[T];
  bool act[T];
  float r00[T], r01[T], r02[T], r11[T], r12[T], r20[T], r21[T], r22[T];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    f[t] = f0 + lane + 32 * t;
    act[t] = f[t] < NN;
    const int ff = act[t] ? f[t] : 0;
    const int i = ff / N, j = ff - (ff / N) * N;
    const float2 ca = tab[i], cb = tab[j];  // (cos, sin)
    r00[t] = cb.x * ih, r01[t] = cb.y * ca.y * ih, r02[t] = cb.y * ca.x * ih;
    r11[t] = ca.x * ih, r12[t] = -ca.y * ih;
    r20[t] = -cb.y * ih, r21[t] = cb.x * ca.y * ih, r22[t] = cb.x * ca.x * ih;
  }
  typename Acc<GT>::type sa[T];
#pragma unroll
  for (int t = 0; t < T; ++t) sa[t] = 0;
#pragma unroll(U)
  for (int a = 0; a < n; ++a) {
    const float4 d = rel[a];
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const float u = fmaf(r00[t], d.x, fmaf(r01[t], d.y, fmaf(r02[t], d.z, tx)));
      const float v = fmaf(r11[t], d.y, fmaf(r12[t], d.z, ty));
      const float w = fmaf(r20[t], d.x, fmaf(r21[t], d.y, fmaf(r22[t], d.z, tz)));
      sa[t] += lookup_acc<GT>(g, u, v, w);
    }
  }
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const float s = (float)sa[t];
    if (act[t] && s > best) {
      best = s;
      bidx = f[t];
    }
  }
  DOCK_CNT(if (lane == 0) cnt_add(kCntAlignPoses, 32 * T);)
}

template <int MAXN>
__device__ __forceinline__ void align_move(ItemSmem<MAXN>& ws, int n, const float2* tab, int N, int bidx, float3 c,
                                           int first, int stride) {
  const int i = bidx / N, j = bidx - (bidx / N) * N;
  const float2 ca = tab[i], cb = tab[j];
  for (int a = first; a < n; a += stride) {
    const float4 d = ws.u.rel[a];
    const float x = cb.x * d.x + cb.y * ca.y * d.y + cb.y * ca.x * d.z;
    const float y = ca.x * d.y - ca.y * d.z;
    const float z = -cb.y * d.x + cb.x * ca.y * d.y + cb.x * ca.x * d.z;
    ws.pos[a] = make_float4(c.x + x, c.y + y, c.z + z, 0.f);
  }
}

// Grid coordinates of the centroid in ws.bc (the translation part of every alignment pose).
__device__ __forceinline__ float3 centre_grid(const float4& cc, const GridK& g) {
  return make_float3((cc.x - g.ox) * g.inv_h, (cc.y - g.oy) * g.inv_h, (cc.z - g.oz) * g.inv_h);
}

// Scores pose (i, j) for all N*N pairs (one pose per lane; the item's warps share the passes),
// moves the ligand to the best one (ties: lowest i*N + j) and returns its flat index.  The
// centroid is summed by warp 0 alone, so the result does not depend on the number of warps.
template <int MAXN, int GT, int G, int T>
__device__ int align_phase(ItemSmem<MAXN>& ws, int n, const float2* tab, int N, const GridK& g, int wig, int lane,
                           int grp) {
  if (wig == 0) align_centre(ws, n, lane);
  group_sync<G>(grp);
  const float4 cc = ws.bc;
  const float3 c = make_float3(cc.x, cc.y, cc.z);
  const float3 t = centre_grid(cc, g);
  const int NN = N * N;
  float best = -CUDART_INF_F;
  int bidx = 0x7fffffff;
  for (int f0 = wig * 32 * T; f0 < NN; f0 += 32 * G * T)
    align_pass<GT, T>(ws.u.rel, n, tab, N, g, t.x, t.y, t.z, f0, lane, best, bidx);
  group_argmax<MAXN, G>(ws, best, bidx, wig, lane, grp);
  align_move(ws, n, tab, N, bidx, c, wig * 32 + lane, 32 * G);
  group_sync<G>(grp);
  return bidx;
}

// ---- torsion sweep (Alg. 1, the fragment loop) ---------------------------------------------------

// Bit q of the result: the angle of pass q owned by this lane (k = 32 q + lane) bumps in one of
// the `cnt` pairs.  `prior` holds bits already known from earlier pair chunks.  Each lane keeps the
// smallest d^2 it has seen; the warp votes on "every live angle bumps" at the start of a pass and
// after every 8 pairs in both modes, and only acts on the vote (skipping the rest) with early_exit.
// Even and odd pairs fold into two independent chains of minima, merged at each vote, which halves
// the chain's latency; the minimum, and so every bit, is the same.
__device__ __forceinline__ unsigned check_pairs(const float4* pairs, int cnt, const float2* tab, int A, int nq,
                                                float dc2, bool early_exit, unsigned prior, int lane) {
  __syncwarp();
  unsigned bits = 0;
  for (int q = 0; q < nq; ++q) {
    const int k = q * 32 + lane;
    const bool live = k < A;
    const float2 cs = tab[live ? k : 0];
    float dmin = ((prior >> q) & 1u) ? -1.0f : CUDART_INF_F;
    const bool all_bump = __all_sync(kFull, dmin < dc2 || !live);
    if (!(early_exit && all_bump)) {
      DOCK_CNT(int e_run = 0;)
      float d1 = CUDART_INF_F;  // odd pairs: two independent chains of minima, merged at each vote
      for (int e = 0; e < cnt; e += 2) {
        const float4 P = pairs[e];
        dmin = fminf(dmin, fmaf(P.z, cs.y, fmaf(P.y, cs.x, P.x)));
        if (e + 1 < cnt) {
          const float4 Q = pairs[e + 1];
          d1 = fminf(d1, fmaf(Q.z, cs.y, fmaf(Q.y, cs.x, Q.x)));
        }
        DOCK_CNT(e_run += min(2, cnt - e);)
        if ((e & 7) == 6) {
          dmin = fminf(dmin, d1);
          const bool all = __all_sync(kFull, dmin < dc2 || !live);
          if (early_exit && all) break;
        }
      }
      dmin = fminf(dmin, d1);
      DOCK_CNT(const unsigned nl = __popc(__ballot_sync(kFull, live)); if (lane == 0) cnt_add(kCntPairTests,
                                                                                                (unsigned long long)nl * e_run);)
    }
    if (live && dmin < dc2) bits |= 1u << q;
  }
  __syncwarp();
  return bits;
}

// Sweeps rotatable bond (a, b): angles theta_k = 2 pi k / A about the axis a -> b through b move
// the atoms of `maskw` (the side holding b).  Chooses the best-scoring angle without a bump
// (ties: lowest k; none: k = 0), applies it, and returns k; `rejected` = angles with a bump.
// Warp 0 lists the moving atoms; the item's warps share the bump check and the scoring passes.
template <int MAXN, int GT, int G, int SPLIT = kSplitPairs, int T = 1, int U = (T == 1 ? 4 : 2), int ILP = 0>
__device__ int torsion_phase(ItemSmem<MAXN>& ws, int n, int a, int b, const uint32_t* __restrict__ maskw,
                             const float2* tab, int A, float dc2, bool early_exit, const GridK& g, int wig, int lane,
                             int grp, float4* xpairs, int& rejected) {
  constexpr int CAP = PairCap<MAXN>::value;
  const float4 pa = ws.pos[a], pb = ws.pos[b];
  float ux = pb.x - pa.x, uy = pb.y - pa.y, uz = pb.z - pa.z;
  const float inv_len = 1.0f / sqrtf(ux * ux + uy * uy + uz * uz);
  ux *= inv_len;
  uy *= inv_len;
  uz *= inv_len;
  const float ih = g.inv_h;
  const int nq = (A + 31) >> 5;

  const unsigned lt = lanemask_lt();
  // With many moving/fixed pairs the bump check is split over the item's warps.  Every warp counts
  // the moving side from the mask itself (b is on it, a is not), so the choice needs no barrier.
  int msize = 0;
  for (int w = 0; w * 32 < n; ++w) msize += __popc(__ldg(maskw + w));
  const bool split = G > 1 && (msize - 1) * (n - msize - 1) >= SPLIT;

  int m = 0, f = 0;
  if (wig == 0) {
    // moving atoms except b (their circle data) and fixed atoms except a (their indices)
    for (int base = 0; base < n; base += 32) {
      const int i = base + lane;
      const uint32_t word = __ldg(maskw + (base >> 5));
      const bool in = i < n;
      const bool mv = in && ((word >> lane) & 1u);
      const bool is_m = mv && i != b;
      const bool is_f = in && !mv && i != a;
      const unsigned bm = __ballot_sync(kFull, is_m), bf = __ballot_sync(kFull, is_f);
      if (is_m) {
        const float4 q = ws.pos[i];
        const float vx = q.x - pb.x, vy = q.y - pb.y, vz = q.z - pb.z;
        const float t = vx * ux + vy * uy + vz * uz;
        const float rx = vx - t * ux, ry = vy - t * uy, rz = vz - t * uz;
        const float wx = uy * rz - uz * ry, wy = uz * rx - ux * rz, wz = ux * ry - uy * rx;
        const int k = m + __popc(bm & lt);
        ws.u.mov.B[k] = make_float4((pb.x + t * ux - g.ox) * ih, (pb.y + t * uy - g.oy) * ih,
                                    (pb.z + t * uz - g.oz) * ih, __int_as_float(i));
        ws.u.mov.R[k] = make_float4(rx * ih, ry * ih, rz * ih, wx * ih);
        ws.u.mov.W[k] = make_float2(wy * ih, wz * ih);
      }
      if (is_f) ws.fixed_idx[f + __popc(bf & lt)] = (unsigned char)i;
      m += __popc(bm);
      f += __popc(bf);
    }
    if (split) ws.clash[lane] = 0u;
    if (lane == 0) {
      ws.bi[0] = m;
      ws.bi[2] = f;
    }
    __syncwarp();
  }
  if (split) {
    group_sync<G>(grp);
    m = ws.bi[0];
    f = ws.bi[2];
  }

  // bump check: collect pairs that can come within d_c, test each angle against them.  Split, the
  // G warps take interleaved blocks of 32 pairs into their own pair buffers; an angle bumps if any
  // pair bumps, so OR-ing the warps' bits gives the single-warp result exactly.
  if (wig == 0 || split) {
    const int ways = split ? G : 1;
    float4* pairs = wig == 0 ? ws.pairs : xpairs;
    const int npairs = m * f;
    unsigned clash_bits = 0;
    int cnt = 0;
    for (int p0 = wig * 32; p0 < npairs; p0 += 32 * ways) {
      const int pi = p0 + lane;
      bool act = false;
      float C = 0.f, Pa = 0.f, Pb = 0.f;
      if (pi < npairs) {
        const int km = pi / f, kf = pi - (pi / f) * f;
        const int i = __float_as_int(ws.u.mov.B[km].w);
        const float4 q = ws.pos[i], xj = ws.pos[ws.fixed_idx[kf]];
        const float vx = q.x - pb.x, vy = q.y - pb.y, vz = q.z - pb.z;
        const float t = vx * ux + vy * uy + vz * uz;
        const float rx = vx - t * ux, ry = vy - t * uy, rz = vz - t * uz;
        const float wx = uy * rz - uz * ry, wy = uz * rx - ux * rz, wz = ux * ry - uy * rx;
        const float ex = pb.x + t * ux - xj.x, ey = pb.y + t * uy - xj.y, ez = pb.z + t * uz - xj.z;
        C = ex * ex + ey * ey + ez * ez + (rx * rx + ry * ry + rz * rz);
        Pa = 2.f * (ex * rx + ey * ry + ez * rz);
        Pb = 2.f * (ex * wx + ey * wy + ez * wz);
        // keep the pair unless its closest approach clears d_c by more than FP32 rounding
        act = C - sqrtf(Pa * Pa + Pb * Pb) < dc2 + 1e-3f + 1e-5f * C;
      }
      const unsigned bal = __ballot_sync(kFull, act);
      const int na = __popc(bal);
      if (cnt + na > CAP) {
        clash_bits |= check_pairs(pairs, cnt, tab, A, nq, dc2, early_exit, clash_bits, lane);
        cnt = 0;
      }
      if (act) pairs[cnt + __popc(bal & lt)] = make_float4(C, Pa, Pb, 0.f);
      cnt += na;
    }
    clash_bits |= check_pairs(pairs, cnt, tab, A, nq, dc2, early_exit, clash_bits, lane);
    if (!split)
      ws.clash[lane] = clash_bits;
    else if (clash_bits)
      atomicOr(&ws.clash[lane], clash_bits);
  }
  group_sync<G>(grp);
  m = ws.bi[0];
  const unsigned clash_bits = ws.clash[lane];
  {
    int rej = 0;
    for (int q = 0; q < nq; ++q) rej += __popc(__ballot_sync(kFull, (clash_bits >> q) & 1u));
    rejected = rej;
  }

  // score every accepted angle: sum of lookups over the moving atoms (the rest is constant).  A group
  // is T passes of 32 angles (the angle tile): each lane scores angles (q0 + t) * 32 + lane, t < T,
  // reading each moving atom's circle data once for the T angles; a group is skipped (early exit)
  // when none of its angles is accepted.
  float best = -CUDART_INF_F;
  int bk = 0x7fffffff;
  for (int q0 = wig * T; q0 < nq; q0 += G * T) {
    int k[T];
    bool valid[T];
    bool any = false;
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const int q = q0 + t;
      k[t] = q * 32 + lane;
      valid[t] = q < nq && k[t] < A && !((clash_bits >> (q < nq ? q : 0)) & 1u);
      any |= valid[t];
    }
    const bool any_valid = __any_sync(kFull, any);
    if (early_exit && !any_valid) continue;
    DOCK_CNT(unsigned nv = 0;
#pragma unroll
             for (int t = 0; t < T; ++t) nv += __popc(__ballot_sync(kFull, valid[t])); if (lane == 0) {
               cnt_add(kCntTorsionAngles, 32 * T);
               cnt_add(kCntAnglesAccepted, nv);
             })
    float2 cs[T];
#pragma unroll
    for (int t = 0; t < T; ++t) cs[t] = tab[k[t] < A ? k[t] : 0];
    typename Acc<GT>::type sa[T];
#pragma unroll
    for (int t = 0; t < T; ++t) sa[t] = 0;
    if constexpr (ILP > 0) {  // the latency form: ILP lookups of the lane's angle in flight
      static_assert(T == 1, "grouped fetches score one angle per lane");
      const float2 c0 = cs[0];
      sa[0] = sum_lookups_ilp<GT, ILP>(g, m, [&](int e) {
        const float4 Bq = ws.u.mov.B[e], Rq = ws.u.mov.R[e];
        const float2 Wq = ws.u.mov.W[e];
        return make_float3(fmaf(c0.y, Rq.w, fmaf(c0.x, Rq.x, Bq.x)), fmaf(c0.y, Wq.x, fmaf(c0.x, Rq.y, Bq.y)),
                           fmaf(c0.y, Wq.y, fmaf(c0.x, Rq.z, Bq.z)));
      });
    } else {
#pragma unroll(U)
      for (int e = 0; e < m; ++e) {
        const float4 Bq = ws.u.mov.B[e], Rq = ws.u.mov.R[e];
        const float2 Wq = ws.u.mov.W[e];
#pragma unroll
        for (int t = 0; t < T; ++t) {
          const float u = fmaf(cs[t].y, Rq.w, fmaf(cs[t].x, Rq.x, Bq.x));
          const float v = fmaf(cs[t].y, Wq.x, fmaf(cs[t].x, Rq.y, Bq.y));
          const float w = fmaf(cs[t].y, Wq.y, fmaf(cs[t].x, Rq.z, Bq.z));
          sa[t] += lookup_acc<GT>(g, u, v, w);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const float s = (float)sa[t];
      if (valid[t] && s > best) {
        best = s;
        bk = k[t];
      }
    }
  }
  group_argmax<MAXN, G>(ws, best, bk, wig, lane, grp);
  const int kstar = (best == -CUDART_INF_F) ? 0 : bk;

  // apply theta_k* to the moving atoms (k = 0 leaves the pose unchanged)
  if (kstar != 0) {
    const float2 cs = tab[kstar];
    for (int e = wig * 32 + lane; e < m; e += 32 * G) {
      const int i = __float_as_int(ws.u.mov.B[e].w);
      const float4 q = ws.pos[i];
      const float vx = q.x - pb.x, vy = q.y - pb.y, vz = q.z - pb.z;
      const float t = vx * ux + vy * uy + vz * uz;
      const float rx = vx - t * ux, ry = vy - t * uy, rz = vz - t * uz;
      const float wx = uy * rz - uz * ry, wy = uz * rx - ux * rz, wz = ux * ry - uy * rx;
      ws.pos[i] = make_float4(pb.x + t * ux + cs.x * rx + cs.y * wx, pb.y + t * uy + cs.x * ry + cs.y * wy,
                              pb.z + t * uz + cs.x * rz + cs.y * wz, 0.f);
    }
  }
  group_sync<G>(grp);
  return kstar;
}

// ---- final score and clash count ------------------------------------------------------------------

template <int MAXN, int GT>
__device__ float pose_score(const ItemSmem<MAXN>& ws, int n, const GridK& g, int lane) {
  typename Acc<GT>::type s = 0;
  for (int i = lane; i < n; i += 32) {
    const float4 q = ws.pos[i];
    s += lookup_at<GT>(g, q.x, q.y, q.z);
  }
  return warp_sum((float)s);
}

// Pairs more than two bonds apart (excl bit clear) closer than d_c.
template <int MAXN>
__device__ int clash_count(const ItemSmem<MAXN>& ws, int n, const uint32_t* __restrict__ excl, float dc2, int lane) {
  int c = 0;
  for (int i = 0; i < n; ++i) {
    const float4 p = ws.pos[i];
    for (int j = i + 1 + lane; j < n; j += 32) {
      const uint32_t ex = __ldg(excl + (size_t)i * kMaskWords + (j >> 5));
      if ((ex >> (j & 31)) & 1u) continue;
      const float4 q = ws.pos[j];
      const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
      c += (dx * dx + dy * dy + dz * dz) < dc2;
    }
  }
  return warp_sum_i(c);
}

// Starting pose (Alg. 1 Generate_Starting_Pose): centroid to the pocket centre, restart r's
// orientation about it.  One warp.
template <int MAXN>
__device__ __forceinline__ void start_pose(ItemSmem<MAXN>& ws, int n, unsigned long long id, unsigned long long seed,
                                           int r, const PocketDev& pk, int lane) {
  const float3 c0 = warp_centroid(ws.pos, n, lane);
  float S[9];
  restart_rotation(id, seed, r, S);
  for (int i = lane; i < n; i += 32) {
    const float4 q = ws.pos[i];
    const float dx = q.x - c0.x, dy = q.y - c0.y, dz = q.z - c0.z;
    ws.pos[i] = make_float4(pk.cx + S[0] * dx + S[1] * dy + S[2] * dz, pk.cy + S[3] * dx + S[4] * dy + S[5] * dz,
                            pk.cz + S[6] * dx + S[7] * dy + S[8] * dz, 0.f);
  }
}

template <int MAXN>
__device__ void finish_restart(const ItemSmem<MAXN>& ws, const BatchDev& bd, const ParamsDev& p, int l, int r, int ai,
                               int pi, float s, int cc, int lane);

// ---- the kernel --------------------------------------------------------------------------------------

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Docks one (ligand, restart) with the G warps of group `grp` (wig = warp within the group).
template <int MAXN, int GT, int G, int T>
__device__ void dock_item(ItemSmem<MAXN>& ws, float4* xpairs, const float2* tab_al, const float2* tab_to,
                          const PocketDev& pk, const BatchDev& bd, const ParamsDev& p, uint32_t item, int wig, int lane,
                          int grp) {
  const int l = (int)(item >> kRestartBits);
  const int r = (int)(item & ((1u << kRestartBits) - 1));
  const int4 h = bd.hdr[l];
  const int a0 = h.x, n = h.y, rb0 = h.z, B = h.w;
  const GridK g = make_gridk(pk);
  DOCK_CNT(if (wig == 0 && lane == 0) cnt_add(kCntItems, 1);)

  for (int i = wig * 32 + lane; i < n; i += 32 * G)
    ws.pos[i] = make_float4(bd.x[a0 + i], bd.y[a0 + i], bd.z[a0 + i], 0.f);
  group_sync<G>(grp);

  if (wig == 0) start_pose(ws, n, bd.ids[l], p.seed, r, pk, lane);
  group_sync<G>(grp);

  const int ai = align_phase<MAXN, GT, G, T>(ws, n, tab_al, p.N, g, wig, lane, grp);

  for (int bi = 0; bi < B; ++bi) {
    const uint32_t ab = __ldg(bd.rot_ab + rb0 + bi);
    int rej = 0;
    const int k = torsion_phase<MAXN, GT, G, kSplitPairs, T>(ws, n, (int)(ab & 0xffffu), (int)(ab >> 16),
                                              bd.mask + (size_t)(rb0 + bi) * kMaskWords, tab_to, p.A, p.dc2,
                                              p.early_exit != 0, g, wig, lane, grp, xpairs, rej);
    if (wig == 0 && lane == 0) {
      const size_t o = (size_t)rb0 * p.R + (size_t)r * B + bi;
      bd.tors_idx[o] = k;
      bd.rejected[o] = rej;
    }
  }

  const int pi = p.post_align ? align_phase<MAXN, GT, G, T>(ws, n, tab_al, p.N, g, wig, lane, grp) : -1;
  if (wig != 0) return;  // the rest is warp 0's
  const float s = pose_score<MAXN, GT>(ws, n, g, lane);
  const int cc = clash_count<MAXN>(ws, n, bd.excl + (size_t)a0 * kMaskWords, p.dc2, lane);
  finish_restart<MAXN>(ws, bd, p, l, r, ai, pi, s, cc, lane);
}

// Writes the restart's outputs (final score s, clash count cc, alignment choices) and final pose;
// the last restart of the ligand to finish picks the best one (ties: lowest restart).  One warp.
template <int MAXN>
__device__ void finish_restart(const ItemSmem<MAXN>& ws, const BatchDev& bd, const ParamsDev& p, int l, int r, int ai,
                               int pi, float s, int cc, int lane) {
  const int4 h = bd.hdr[l];
  const int a0 = h.x, n = h.y;
  const size_t o = (size_t)l * p.R + r;
  if (lane == 0) {
    bd.restart_score[o] = s;
    bd.restart_clash[o] = cc;
    bd.align_idx[o] = ai;
    bd.post_idx[o] = pi;
  }
  float* rx = bd.rs_xyz + ((size_t)a0 * p.R + (size_t)r * n) * 3;
  for (int i = lane; i < n; i += 32) {
    const float4 q = ws.pos[i];
    rx[3 * i] = q.x;
    rx[3 * i + 1] = q.y;
    rx[3 * i + 2] = q.z;
  }

  // the last restart of the ligand to finish picks the best one (ties: lowest restart)
  __threadfence();
  __syncwarp();
  unsigned prev = 0;
  if (lane == 0) prev = atomicAdd(bd.done + l, 1u);
  prev = __shfl_sync(kFull, prev, 0);
  if (prev != (unsigned)(p.R - 1)) return;
  __syncwarp();
  __threadfence();
  float best = -CUDART_INF_F;
  int br = 0x7fffffff;
  for (int q = lane; q < p.R; q += 32) {
    const float v = __ldcg(bd.restart_score + (size_t)l * p.R + q);
    if (v > best) {
      best = v;
      br = q;
    }
  }
  warp_argmax(best, br);
  const float* src = bd.rs_xyz + ((size_t)a0 * p.R + (size_t)br * n) * 3;
  for (int i = lane; i < 3 * n; i += 32) bd.out_xyz[(size_t)a0 * 3 + i] = __ldcg(src + i);
  if (lane == 0) {
    bd.best_score[l] = best;
    bd.best_restart[l] = br;
    bd.clash[l] = __ldcg(bd.restart_clash + (size_t)l * p.R + br);
    bd.done[l] = 0;
  }
}

template <int MAXN>
__host__ __device__ constexpr size_t table_bytes(int N, int A) {
  return align16((size_t)(N + A) * sizeof(float2));
}

// G warps per work item, wpb / G items per block.  With next_item == nullptr group q of block b
// takes item b*(wpb/G) + q; otherwise (persistent form) every group pulls items from the counter
// until the list is exhausted.
//
// One kernel body, two entry points with their own register budgets.  The body is a macro so that
// each entry point is compiled as this kernel written out in full: moving it into a device function
// called by both, even an inlined one, changed the code generated for the 8-warps-per-item kernel of
// small serving batches (ptxas reserved all 16 named barriers for it instead of 2, and their median
// latency rose 8%).
#define DOCK_KERNEL_DEFINE(NAME, BOUNDS)                                                                                     \
  template <int MAXN, int GT, int G, int T>                                                                                  \
  __global__ void BOUNDS NAME(PocketDev pk, BatchDev bd, ParamsDev p, const uint32_t* __restrict__ items,                    \
                              int n_items, int wpb, unsigned* next_item) {                                                   \
  extern __shared__ __align__(16) unsigned char smem[];                                                                      \
  float2* tab_al = reinterpret_cast<float2*>(smem);                                                                          \
  float2* tab_to = tab_al + p.N;                                                                                             \
  for (int t = threadIdx.x; t < p.N + p.A; t += blockDim.x) {                                                                \
    float s, c;                                                                                                              \
    if (t < p.N)                                                                                                             \
      sincospif((float)(2 * t) / (float)p.N, &s, &c);                                                                        \
    else                                                                                                                     \
      sincospif((float)(2 * (t - p.N)) / (float)p.A, &s, &c);                                                                \
    tab_al[t] = make_float2(c, s);                                                                                           \
  }                                                                                                                          \
  __syncthreads();                                                                                                           \
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;                                                                \
  const int grp = warp / G, wig = warp - grp * G;                                                                            \
  DOCK_CNT(if (lane < kCnt) g_cnt_smem[warp][lane] = 0; __syncwarp();)                                                       \
/* counter build: after each item the warp adds its slot to the launch's counters */                                         \
  auto flush = [&]() {                                                                                                       \
    DOCK_CNT(__syncwarp(); if (lane < kCnt && p.exec) {                                                                      \
      const unsigned long long v = g_cnt_smem[warp][lane];                                                                   \
      if (v) atomicAdd(p.exec + lane, v);                                                                                    \
      g_cnt_smem[warp][lane] = 0;                                                                                            \
    } __syncwarp();)                                                                                                         \
  };                                                                                                                         \
  ItemSmem<MAXN>* items_smem = reinterpret_cast<ItemSmem<MAXN>*>(smem + table_bytes<MAXN>(p.N, p.A));                        \
  ItemSmem<MAXN>& ws = items_smem[grp];                                                                                      \
/* bump-pair buffers of the warps other than each item's warp 0 (which uses ws.pairs) */                                     \
  float4* xpairs = G > 1 && wig > 0                                                                                          \
                       ? reinterpret_cast<float4*>(items_smem + wpb / G) + (grp * (G - 1) + wig - 1) * PairCap<MAXN>::value  \
                       : nullptr;                                                                                            \
  if (next_item == nullptr) {                                                                                                \
    const int item = blockIdx.x * (wpb / G) + grp;                                                                           \
    if (item >= n_items) return;                                                                                             \
    dock_item<MAXN, GT, G, T>(ws, xpairs, tab_al, tab_to, pk, bd, p, items[item], wig, lane, grp);                           \
    flush();                                                                                                                 \
    return;                                                                                                                  \
  }                                                                                                                          \
  for (;;) {                                                                                                                 \
/* warp 0 of the group has finished the previous item before anyone takes the next one */                                    \
    if (wig == 0 && lane == 0) ws.bi[3] = (int)atomicAdd(next_item, 1u);                                                     \
    group_sync<G>(grp);                                                                                                      \
    const unsigned it = (unsigned)ws.bi[3];                                                                                  \
    group_sync<G>(grp);                                                                                                      \
    if (it >= (unsigned)n_items) return;                                                                                     \
    dock_item<MAXN, GT, G, T>(ws, xpairs, tab_al, tab_to, pk, bd, p, items[it], wig, lane, grp);                             \
    flush();                                                                                                                 \
  }                                                                                                                          \
  }

template <int MAXN>
inline size_t smem_bytes_for(const ParamsDev& p, int wpb, int G) {
  return table_bytes<MAXN>(p.N, p.A) + (size_t)(wpb / G) * sizeof(ItemSmem<MAXN>) +
         (size_t)(wpb - wpb / G) * PairCap<MAXN>::value * sizeof(float4);  // other warps' pair buffers
}

// Resident blocks per SM of each kernel shape, recorded when attributes are applied (outside any
// stream capture) and read by persistent launches.
struct ResidentCache {
  int key[64][5];
  int blocks[64];
  int n;
};

DOCK_KERNEL_DEFINE(dock_kernel, DOCK_KERNEL_BOUNDS)
DOCK_KERNEL_DEFINE(dock_kernel_wide, DOCK_KERNEL_WIDE_BOUNDS)

// The entry point of an instantiation (only the one taken is instantiated).
template <int MAXN, int GT, int G, int T>
constexpr auto dock_kernel_entry() {
  if constexpr (GT == 0 && G == 1)
    return &dock_kernel_wide<MAXN, GT, G, T>;
  else
    return &dock_kernel<MAXN, GT, G, T>;
}

template <int MAXN, int GT, int G, int T>
cudaError_t launch_t(const PocketDev& pk, const BatchDev& b, const ParamsDev& p, const uint32_t* items, int n_items,
                     const LaunchCfg& cfg, cudaStream_t s, bool set_attributes) {
  constexpr auto kernel = dock_kernel_entry<MAXN, GT, G, T>();
  static ResidentCache cache = {};
  static std::mutex cache_mu;
  const int wpb = cfg.warps_per_block;
  const size_t smem = smem_bytes_for<MAXN>(p, wpb, G);
  int dev = 0;
  cudaGetDevice(&dev);
  auto lookup_resident = [&](int* out) {
    std::lock_guard<std::mutex> lk(cache_mu);
    for (int i = 0; i < cache.n; ++i)
      if (cache.key[i][0] == wpb && cache.key[i][1] == (int)smem && cache.key[i][2] == cfg.smem_carveout &&
          cache.key[i][3] == dev) {
        *out = cache.blocks[i];
        return true;
      }
    return false;
  };
  if (set_attributes) {
    cudaError_t e =
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cfg.smem_carveout >= 0 ? cfg.smem_carveout : (int)cudaSharedmemCarveoutDefault);
    if (e != cudaSuccess) return e;
    int resident = 0;
    if (cfg.persistent && !lookup_resident(&resident)) {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, kernel, wpb * 32, smem);
      if (e != cudaSuccess) return e;
      std::lock_guard<std::mutex> lk(cache_mu);
      if (cache.n < 64) {
        cache.key[cache.n][0] = wpb;
        cache.key[cache.n][1] = (int)smem;
        cache.key[cache.n][2] = cfg.smem_carveout;
        cache.key[cache.n][3] = dev;
        cache.blocks[cache.n++] = resident;
      }
    }
  }
  if (n_items <= 0) return cudaSuccess;
  const int per_block = wpb / G;
  int blocks = (n_items + per_block - 1) / per_block;
  unsigned* counter = nullptr;
  if (cfg.persistent && b.next_item) {
    int resident = 0, sms = 0;
    if (!lookup_resident(&resident) || resident < 1) resident = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    blocks = blocks < resident * sms ? blocks : resident * sms;
    counter = b.next_item + cfg.counter_slot;
  }
  kernel<<<blocks, wpb * 32, smem, s>>>(pk, b, p, items, n_items, wpb, counter);
  return cudaGetLastError();
}

}  // namespace dockgpu
