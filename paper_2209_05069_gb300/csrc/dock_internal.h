// Internal interface between the host runtime (dock_host.cpp) and the CUDA kernels
// (dock_kernels_*.cu).  Not part of the public C-ABI (include/dock.h).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace dockgpu {

constexpr int kMaskWords = 5;         // 160-atom bitsets
constexpr int kMaxAtoms = 160;
constexpr int kRestartBits = 10;      // work item = ligand << 10 | restart
constexpr int kNumBuckets = 5;        // atom-count buckets (0,32], (32,64], ..., (128,160]

inline int bucket_of(int n_atoms) { return (n_atoms - 1) / 32; }

// Pocket grid in device memory, stored as corner-packed cells: cell (i, j, k) for
// i < nx-1, j < ny-1, k < nz-1 holds the 8 voxel values of its corners in the order
// (di, dj, dk) = (0,0,0), (1,0,0), (0,1,0), (1,1,0), (0,0,1), (1,0,1), (0,1,1), (1,1,1),
// so one trilinear lookup is one 32-byte (FP32) or 16-byte (FP16) load.  One extra all-zero
// cell at index (nx-1)(ny-1)(nz-1) serves every position outside the grid.
struct PocketDev {
  const void* cells;
  int nx, ny, nz;
  int dtype;              // DOCK_GRID_F32 (32-byte cells), _F16 (16-byte cells) or _I16 (int16 voxels)
  float spacing, inv_h;
  float ox, oy, oz;       // grid origin (Angstrom)
  float cx, cy, cz;       // pocket centre = origin + spacing * (n - 1) / 2
  // Grid coordinates outside [lo, hi] on any axis have all 8 corner voxels zero (or lie outside
  // the grid), so their lookup is exactly 0 and is skipped: lo = max(0, first nonzero voxel - 1),
  // hi = min(n - 1, last nonzero voxel + 1); lo > hi for an all-zero grid.  Integer grid: `cells`
  // holds voxels lo..hi of a box one voxel wider than the nonzero voxels on every side (its border
  // is zero; for an all-zero grid lo = -1, hi = 0), and a nearest-voxel index is clamped into it.
  float lox, loy, loz, hix, hiy, hiz;
};

// Packed ligands and result arrays of one batch, all in device memory.
struct BatchDev {
  int n_lig;
  const int4* hdr;                  // {atom_off, n_atoms, rot_off, n_rot}
  const unsigned long long* ids;
  const float* x;                   // SoA coordinates, indexed by atom_off + i
  const float* y;
  const float* z;
  const uint32_t* rot_ab;           // rotatable bond: a | b << 16, indexed by rot_off + bond
  const uint32_t* mask;             // moving-side bitset of each rotatable bond [rot][5]
  const uint32_t* excl;             // atoms within two bonds (and self) of each atom [atom][5]
  // results
  float* restart_score;             // [n_lig * R]
  int* restart_clash;               // [n_lig * R]
  int* align_idx;                   // [n_lig * R]
  int* post_idx;                    // [n_lig * R]
  int* tors_idx;                    // [rot_total * R]: rot_off*R + r*B + b
  int* rejected;                    // [rot_total * R]
  float* best_score;                // [n_lig]
  int* best_restart;                // [n_lig]
  float* out_xyz;                   // [atom_total * 3]
  int* clash;                       // [n_lig]
  int* select_restart;              // [n_lig * K] (nullptr: Select Poses output skipped)
  float* select_score;              // [n_lig * K]
  float* select_xyz;                // [atom_total * K * 3]: (atom_off*K + k*n)*3
  // scratch (global memory besides inputs and outputs)
  float* rs_xyz;                    // final pose of every restart: (atom_off*R + r*n)*3
  unsigned* done;                   // finished restarts per ligand; the last one resets it to 0
  unsigned* next_item;              // per-bucket work counters of persistent launches (zeroed before
                                    // each launch); nullptr: no persistent launches
};

struct ParamsDev {
  int R, N, A;                      // restarts, alignment steps per axis, torsion steps
  float dc2;                        // squared bump threshold
  int post_align, early_exit;
  unsigned long long seed;
  int K;                            // Select Poses: poses kept per ligand
  float sel_rmsd2;                  // squared RMSD threshold of Select Poses
  unsigned long long* exec;         // executed-work counters (kCnt of them) of a library built with
                                    // DOCK_COUNT_WORK; nullptr (and never read) otherwise
};

// Executed-work counters of the counter build, in the order of dock_exec_work (include/dock.h).
enum : int {
  kCntItems = 0,        // ligand-restarts docked
  kCntAlignPoses,       // alignment pose lanes evaluated (idle lanes of a last pass included)
  kCntTorsionAngles,    // torsion angle lanes of the scoring passes run
  kCntAnglesAccepted,   // of which accepted by the bump check
  kCntLookups,          // pocket lookups evaluated (lane level)
  kCntLoads,            // of which issued a global load (inside the stored box)
  kCntSectors,          // distinct 32-byte sectors of those loads, per warp-wide load instruction
  kCntPairTests,        // bump-pair distance tests evaluated (angle lanes x pairs)
  kCntLines,            // distinct 128-byte lines of those loads, per warp-wide load instruction
  kCnt
};

// Kernel launch configuration for one atom bucket.
struct LaunchCfg {
  int warps_per_block;   // 1..8, a multiple of warps_per_item
  int smem_carveout;     // preferred shared-memory share of L1/shared, percent; -1 = driver default
  int persistent;        // 1: grid sized to the resident blocks, items pulled from a counter
  int counter_slot;      // which of BatchDev::next_item this launch uses (its bucket)
  int warps_per_item;    // warps docking one (ligand, restart): 1, 2, 4 or 8
  int tile;              // poses (alignment) or angles (torsion) one lane scores per pass: 1, or 2
                         // with 1 or 2 warps per item
};

// Builds the corner-packed cell array from voxel values (both in device memory).
cudaError_t launch_pack_pocket(const float* values, void* cells, int nx, int ny, int nz, int f16,
                               cudaStream_t s);

// Docks the work items (ligand << 10 | restart) of one atom bucket.  Every item of a ligand must
// be in the same launch or in launches ordered on one stream (the last finished restart of a
// ligand picks its best restart).
// With set_attributes the kernel's shared-memory attributes are (re)applied first; a launch being
// captured into a CUDA graph passes false after applying them with n_items = 0 outside the capture.
cudaError_t launch_dock_bucket(int bucket, const PocketDev& pk, const BatchDev& b, const ParamsDev& p,
                               const uint32_t* items, int n_items, const LaunchCfg& cfg, cudaStream_t s,
                               bool set_attributes = true);

// Scratch of the latency form (one ligand spread over the GPU; device memory of the batch, reused
// ligand after ligand on one stream).
struct LatScratch {
  float2* cand;    // [R * ceil(N*N/32)]: best (score, flat index as int bits) of each alignment pass
  float4* pose;    // [R * kMaxAtoms]: each restart's pose between the kernels
  unsigned* done;  // [R]: alignment blocks of each restart finished (zeroed before a batch; the last
                   // block of a restart resets its count)
};

// Bytes of LatScratch for R restarts and N alignment angles per axis (256-byte aligned parts).
inline size_t latency_cand_bytes(int R, int N) {
  return ((size_t)8 * R * (((size_t)N * N + 31) / 32) + 255) & ~size_t(255);
}
inline size_t latency_scratch_bytes(int R, int N) {
  return latency_cand_bytes(R, N) + (size_t)16 * R * kMaxAtoms + (((size_t)4 * R + 255) & ~size_t(255));
}

inline LatScratch latency_scratch(void* base, int R, int N) {
  LatScratch s;
  unsigned char* b = static_cast<unsigned char*>(base);
  s.cand = reinterpret_cast<float2*>(b);
  s.pose = reinterpret_cast<float4*>(b + latency_cand_bytes(R, N));
  s.done = reinterpret_cast<unsigned*>(b + latency_cand_bytes(R, N) + (size_t)16 * R * kMaxAtoms);
  return s;
}

// Queues the latency form's kernels (alignment over every SM, torsion sweep per restart,
// post-alignment over every SM, final score and best restart) for ligand l of a batch on stream s;
// adds the kernels launched to *launches.  Ligands of one batch must be queued on one stream.
cudaError_t launch_latency_ligand(int bucket, const PocketDev& pk, const BatchDev& b, const ParamsDev& p, int l,
                                  const LatScratch& sc, cudaStream_t s, int* launches);

// Select Poses over every ligand of a batch (no-op when b.select_restart is null); queued after
// the batch's docking kernels on stream s.
cudaError_t launch_select(const BatchDev& b, const ParamsDev& p, cudaStream_t s);

// ---- read-only view of a prepared batch, for the allocation-free entry point (dock_noalloc.cu) ----

struct BatchView {
  PocketDev pocket;
  BatchDev inputs;                  // input pointers filled; result and scratch pointers left to the caller
  ParamsDev params;
  LaunchCfg cfg[kNumBuckets];
  int n_items[kNumBuckets];
  int item_off[kNumBuckets];
  const uint32_t* items;            // device work items
  int n_lig;
  size_t atoms;
  size_t rots;
  int device;
  cudaStream_t ctx_stream;
};

}  // namespace dockgpu

struct dock_ctx;
struct dock_batch;

#include <functional>

namespace dockgpu {

// Under the context lock: fills a BatchView for (pocket_id, batch), makes the context's device
// current and calls launch(view, stream) with `stream` (NULL: the context's stream).  When launch
// returns >= 0 the batch's completion event is recorded on the stream (dock_batch_wait and
// dock_batch_destroy then wait for this work) and the pocket notes the use, so an unload frees it
// only after the work.  Returns launch's result, or an error code with the last error set.
int with_batch_view(dock_ctx* ctx, int pocket_id, const dock_batch* b, void* stream,
                    const std::function<int(const BatchView&, cudaStream_t)>& launch);

// Device address of the allocation-free entry point's fixed scratch array on `device` (made
// current by the caller), looked up once per device; the context creation calls it so that the
// array is loaded then, not in a docking call.
cudaError_t noalloc_scratch_address(int device, void** out);

// Sets the context's last-error message and returns `code`.
int record_error(dock_ctx* ctx, int code, const char* msg);
// The same, for code that already holds the context lock (inside with_batch_view's launch).
int record_error_locked(dock_ctx* ctx, int code, const char* msg);

// Copies a loaded pocket's device view under the context lock and makes the context's device
// current; also returns the context's stream.  DOCK_OK or DOCK_ERR_NOPOCKET (last error set).
int pocket_view(dock_ctx* ctx, int pocket_id, PocketDev* pk, cudaStream_t* stream);

}  // namespace dockgpu
