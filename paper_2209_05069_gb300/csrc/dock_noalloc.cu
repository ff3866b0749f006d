// Allocation-free launch (dock_batch_launch_noalloc): the docking kernel with its scratch in a
// fixed device array instead of per-batch device memory, for callers that cannot allocate when
// they dock.  Nothing here calls cudaMalloc, cudaFree or an allocating library routine.
#include <cstdio>
#include <mutex>

#include "dock.h"
#include "dock_internal.h"

namespace {

// The scratch: completion counters first (one per ligand, 256-byte aligned block), then each
// restart's final pose.  Every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[DOCK_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

namespace dockgpu {

// In host code the array's name is only a host-side stand-in, so its device address is looked up
// once per device (with that device current).  The first lookup loads the array's module, which
// takes its DOCK_NOALLOC_SCRATCH_BYTES of device memory; dock_create makes that lookup.
cudaError_t noalloc_scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

}  // namespace dockgpu

extern "C" int dock_batch_launch_noalloc(dock_ctx* ctx, int32_t pocket_id, const dock_batch* batch,
                                         const dock_device_results* out, void* stream) {
  using namespace dockgpu;
  if (!ctx) return DOCK_ERR_INVALID;
  if (!out || !out->score || !out->best_restart || !out->xyz || !out->clash_count || !out->restart_score ||
      !out->restart_clash || !out->align_idx || !out->post_idx || !out->torsion_idx || !out->rejected)
    return record_error(ctx, DOCK_ERR_INVALID, "every dock_device_results pointer is required");
  // runs under the context lock, so the pocket stays loaded while the kernels are queued; the
  // batch's completion event and the pocket's use are recorded after them
  return with_batch_view(ctx, pocket_id, batch, stream, [&](const BatchView& v, cudaStream_t s) -> int {
    const size_t counters = (4 * (size_t)v.n_lig + 255) & ~size_t(255);
    const size_t need = counters + 12 * v.atoms * (size_t)v.params.R;
    if (need > DOCK_NOALLOC_SCRATCH_BYTES) {
      char msg[200];
      snprintf(msg, sizeof msg, "batch needs %zu bytes of scratch, the allocation-free limit is %u", need,
               (unsigned)DOCK_NOALLOC_SCRATCH_BYTES);
      return record_error_locked(ctx, DOCK_ERR_INVALID, msg);
    }
    void* base = nullptr;
    cudaError_t e = noalloc_scratch_address(v.device, &base);
    if (e != cudaSuccess) return record_error_locked(ctx, DOCK_ERR_CUDA, cudaGetErrorString(e));
    BatchDev bd = v.inputs;
    bd.best_score = out->score;
    bd.best_restart = out->best_restart;
    bd.out_xyz = out->xyz;
    bd.clash = out->clash_count;
    bd.restart_score = out->restart_score;
    bd.restart_clash = out->restart_clash;
    bd.align_idx = out->align_idx;
    bd.post_idx = out->post_idx;
    bd.tors_idx = out->torsion_idx;
    bd.rejected = out->rejected;
    bd.select_restart = nullptr;  // Select Poses output is not part of this call
    bd.select_score = nullptr;
    bd.select_xyz = nullptr;
    bd.done = static_cast<unsigned*>(base);
    bd.next_item = nullptr;  // launches here are never persistent
    bd.rs_xyz = reinterpret_cast<float*>(static_cast<unsigned char*>(base) + counters);
    // the counters must start at zero; the previous call may have left anything there
    e = cudaMemsetAsync(bd.done, 0, counters, s);
    if (e != cudaSuccess) return record_error_locked(ctx, DOCK_ERR_CUDA, cudaGetErrorString(e));
    int launches = 0;
    for (int b = 0; b < kNumBuckets; ++b) {
      if (!v.n_items[b]) continue;
      LaunchCfg cfg = v.cfg[b];
      cfg.persistent = 0;
      e = launch_dock_bucket(b, v.pocket, bd, v.params, v.items + v.item_off[b], v.n_items[b], cfg, s);
      if (e != cudaSuccess) return record_error_locked(ctx, DOCK_ERR_CUDA, cudaGetErrorString(e));
      ++launches;
    }
    return launches;
  });
}
