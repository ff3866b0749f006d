// Host runtime of libdock.so: the C-ABI of include/dock.h.
//
// Ingest validates each ligand and precomputes, per rotatable bond, the bitset of the side that
// moves (the component holding b once bond (a, b) is cut; Section 1: a rotatable bond splits the
// ligand in two) and, per atom, the bitset of atoms within two bonds (excluded from the final
// clash count).  A batch is laid out in one device arena [inputs | results | scratch] mirrored by
// one pinned host buffer [inputs | results], so a batch moves with one H2D and one D2H copy.
// Work items are (ligand, restart) pairs grouped into five atom-count buckets (Section 4.2 uses
// the same (0,32], ..., (128,160] bins), each bucket sorted by estimated cost, largest first.
//
// The serving loop (continuous batching): submitted ligands wait in a FIFO; whenever one of the
// context's streams is free, the loop packs the waiting ligands that share the head's pocket and
// parameters (from any number of submissions) into a batch that fits the stream's share of the
// device-memory budget, uploads it, launches it and queues the copy back.  Batches on different
// streams overlap on the device; results are scattered to their submissions as batches finish.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <functional>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <unistd.h>

#include <cuda_runtime.h>

#include "dock.h"
#include "dock_internal.h"

using namespace dockgpu;

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// ---- validated, packed ligands ------------------------------------------------------------------

// Allocator whose resize() leaves new elements uninitialised: ingest sizes each array once and
// its threads write every element, so zero-filling first would only add a serial pass.
template <class T>
struct NoInit : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = NoInit<U>;
  };
  NoInit() = default;
  template <class U>
  NoInit(const NoInit<U>&) noexcept {}
  template <class U>
  void construct(U* q) noexcept {
    ::new ((void*)q) U;
  }
  template <class U, class... A>
  void construct(U* q, A&&... a) {
    ::new ((void*)q) U(std::forward<A>(a)...);
  }
};
template <class T>
using Buf = std::vector<T, NoInit<T>>;

struct Packed {
  int n_lig = 0;
  Buf<int> atom_off{0}, rot_off{0};
  Buf<uint64_t> ids;
  Buf<float> x, y, z;
  Buf<uint32_t> rot_ab, mask, excl;
  Buf<int64_t> cost;
  uint64_t moving = 0;  // sum over rotatable bonds of (moving atoms - 1)
};

std::string fmt(const char* f, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, f);
  vsnprintf(buf, sizeof buf, f, ap);
  va_end(ap);
  return buf;
}

bool check_params(const dock_params* p, std::string& err) {
  if (!p) return err = "params is NULL", false;
  if (p->restarts < 1 || p->restarts > DOCK_MAX_RESTARTS) return err = fmt("restarts=%d out of [1,%d]", p->restarts, DOCK_MAX_RESTARTS), false;
  if (p->align_steps < 1 || p->align_steps > DOCK_MAX_ALIGN_STEPS)
    return err = fmt("align_steps=%d out of [1,%d]", p->align_steps, DOCK_MAX_ALIGN_STEPS), false;
  if (p->torsion_steps < 1 || p->torsion_steps > DOCK_MAX_TORSION_STEPS)
    return err = fmt("torsion_steps=%d out of [1,%d]", p->torsion_steps, DOCK_MAX_TORSION_STEPS), false;
  if (!(p->clash_dist >= 0.f) || !std::isfinite(p->clash_dist)) return err = "clash_dist must be finite and >= 0", false;
  if ((p->post_align != 0 && p->post_align != 1) || (p->early_exit != 0 && p->early_exit != 1))
    return err = "post_align and early_exit must be 0 or 1", false;
  const int k = p->select_k <= 0 ? 1 : p->select_k;
  if (k > 16 || k > p->restarts) return err = fmt("select_k=%d out of [1, min(16, restarts)]", p->select_k), false;
  if (!(p->select_rmsd >= 0.f) || !std::isfinite(p->select_rmsd)) return err = "select_rmsd must be finite and >= 0", false;
  if (p->outputs != DOCK_OUTPUT_FULL && p->outputs != DOCK_OUTPUT_BEST)
    return err = "outputs must be DOCK_OUTPUT_FULL or DOCK_OUTPUT_BEST", false;
  return true;
}

using Bits = uint32_t[kMaskWords];

inline void set_bit(uint32_t* b, int i) { b[i >> 5] |= 1u << (i & 31); }
inline bool get_bit(const uint32_t* b, int i) { return (b[i >> 5] >> (i & 31)) & 1u; }

// Host worker threads shared by every context of the process, started on first use, so that
// preparing a submission does not pay for creating and joining threads.  run(n, f) calls f(0) ..
// f(n-1), the caller taking part, and returns when all calls are done.  One job runs at a time;
// a caller that finds the pool busy (another thread's submission) runs its tasks itself, and so
// does a forked child process, which inherits the pool but not its threads.
class WorkPool {
 public:
  static WorkPool& get() {
    static WorkPool pool;
    return pool;
  }
  int workers() const { return (int)threads_.size(); }

  void run(int n, const std::function<void(int)>& f) {
    std::unique_lock<std::mutex> busy(run_mu_, std::try_to_lock);
    if (!busy.owns_lock() || threads_.empty() || n <= 1 || ::getpid() != pid_) {
      for (int i = 0; i < n; ++i) f(i);
      return;
    }
    {
      std::lock_guard<std::mutex> g(mu_);
      job_ = &f;
      n_ = n;
      next_ = 0;
      done_ = 0;
      ++generation_;
    }
    cv_.notify_all();
    work();
    std::unique_lock<std::mutex> g(mu_);
    done_cv_.wait(g, [&] { return done_ == n_; });
    job_ = nullptr;
  }

  ~WorkPool() {
    if (::getpid() != pid_) return;  // a forked child has none of these threads
    {
      std::lock_guard<std::mutex> g(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : threads_) t.join();
  }

 private:
  WorkPool() : pid_(::getpid()) {
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    for (int i = 0; i < std::min(hw, 16) - 1; ++i) threads_.emplace_back([this] { loop(); });
  }

  // takes tasks of the current job until none is left
  void work() {
    for (;;) {
      int i;
      const std::function<void(int)>* f;
      {
        std::lock_guard<std::mutex> g(mu_);
        if (!job_ || next_ >= n_) return;
        i = next_++;
        f = job_;
      }
      (*f)(i);
      std::lock_guard<std::mutex> g(mu_);
      if (++done_ == n_) done_cv_.notify_all();
    }
  }

  void loop() {
    uint64_t seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> g(mu_);
        cv_.wait(g, [&] { return stop_ || generation_ != seen; });
        if (stop_) return;
        seen = generation_;
      }
      work();
    }
  }

  const pid_t pid_;
  std::mutex run_mu_, mu_;
  std::condition_variable cv_, done_cv_;
  std::vector<std::thread> threads_;
  const std::function<void(int)>* job_ = nullptr;
  int n_ = 0, next_ = 0, done_ = 0;
  uint64_t generation_ = 0;
  bool stop_ = false;
};

// Validates ligands [l0, l1) and writes them into `out`, whose arrays are already sized and whose
// atom_off / rot_off already hold every ligand's offsets.  Adds the range's moving-atom count to
// `moving`.  On failure `err` names the ligand and the field and `bad` is that ligand's index.
bool prepare_range(const dock_ligand_batch* lb, const dock_params* p, int l0, int l1, Packed& out, uint64_t& moving,
                   std::string& err, int& bad) {
  const int N = p->align_steps, A = p->torsion_steps;
  std::array<uint32_t, kMaskWords> adj[DOCK_MAX_ATOMS];
  int l = l0;
  auto fail = [&](std::string msg) {
    err = std::move(msg);
    bad = l;
    return false;
  };
  for (; l < l1; ++l) {
    const int a0 = lb->atom_off[l], n = lb->atom_off[l + 1] - a0;
    const int b0 = lb->bond_off[l], nb = lb->bond_off[l + 1] - b0;
    const int r0 = lb->rot_off[l], nr = lb->rot_off[l + 1] - r0;
    if (n < 1 || n > DOCK_MAX_ATOMS) return fail(fmt("ligand %d: atoms=%d out of [1,%d]", l, n, DOCK_MAX_ATOMS));
    if (nb < 0 || nb > DOCK_MAX_BONDS) return fail(fmt("ligand %d: bonds=%d out of [0,%d]", l, nb, DOCK_MAX_BONDS));
    if (nr < 0 || nr > DOCK_MAX_ROT) return fail(fmt("ligand %d: rot_bonds=%d out of [0,%d]", l, nr, DOCK_MAX_ROT));
    for (int i = 0; i < 3 * n; ++i)
      if (!std::isfinite(lb->xyz[3 * (size_t)a0 + i])) return fail(fmt("ligand %d: xyz[%d] not finite", l, i / 3));
    for (int i = 0; i < n; ++i) adj[i] = {};
    for (int e = 0; e < nb; ++e) {
      const int u = lb->bonds[2 * (size_t)(b0 + e)], v = lb->bonds[2 * (size_t)(b0 + e) + 1];
      if (u < 0 || v < 0 || u >= n || v >= n || u == v)
        return fail(fmt("ligand %d: bonds[%d]=(%d,%d) invalid for %d atoms", l, e, u, v, n));
      if (get_bit(adj[u].data(), v)) return fail(fmt("ligand %d: bonds[%d]=(%d,%d) repeated", l, e, u, v));
      set_bit(adj[u].data(), v);
      set_bit(adj[v].data(), u);
    }
    const size_t ta = (size_t)out.atom_off[l], tr = (size_t)out.rot_off[l];
    int64_t moved = 0;
    for (int k = 0; k < nr; ++k) {
      const int a = lb->rot_bonds[2 * (size_t)(r0 + k)], b = lb->rot_bonds[2 * (size_t)(r0 + k) + 1];
      if (a < 0 || b < 0 || a >= n || b >= n || !get_bit(adj[a].data(), b))
        return fail(fmt("ligand %d: rot_bonds[%d]=(%d,%d) is not a bond", l, k, a, b));
      // side holding b once the bond a-b is cut (breadth-first over the bond bitsets)
      uint32_t seen[kMaskWords] = {0}, front[kMaskWords] = {0};
      set_bit(seen, b);
      set_bit(front, b);
      bool any = true;
      while (any) {
        uint32_t next[kMaskWords] = {0};
        for (int w = 0; w < kMaskWords; ++w)
          for (uint32_t bits = front[w]; bits; bits &= bits - 1) {
            const int v = w * 32 + __builtin_ctz(bits);
            for (int q = 0; q < kMaskWords; ++q) {
              uint32_t nb_bits = adj[v][q];
              if (v == b && q == (a >> 5)) nb_bits &= ~(1u << (a & 31));  // the cut edge
              next[q] |= nb_bits;
            }
          }
        any = false;
        for (int q = 0; q < kMaskWords; ++q) {
          next[q] &= ~seen[q];
          seen[q] |= next[q];
          front[q] = next[q];
          any |= next[q] != 0;
        }
      }
      if (get_bit(seen, a)) return fail(fmt("ligand %d: rot_bonds[%d]=(%d,%d) is not a bridge", l, k, a, b));
      int m = 0;
      for (int q = 0; q < kMaskWords; ++q) {
        out.mask[(tr + k) * kMaskWords + q] = seen[q];
        m += __builtin_popcount(seen[q]);
      }
      out.rot_ab[tr + k] = (uint32_t)a | ((uint32_t)b << 16);
      moved += m;
      moving += (uint64_t)(m - 1);
    }
    for (int i = 0; i < n; ++i) {
      uint32_t ex[kMaskWords] = {0};
      set_bit(ex, i);
      for (int q = 0; q < kMaskWords; ++q) ex[q] |= adj[i][q];
      for (int w = 0; w < kMaskWords; ++w)
        for (uint32_t bits = adj[i][w]; bits; bits &= bits - 1) {
          const int j = w * 32 + __builtin_ctz(bits);
          for (int q = 0; q < kMaskWords; ++q) ex[q] |= adj[j][q];
        }
      for (int q = 0; q < kMaskWords; ++q) out.excl[(ta + i) * kMaskWords + q] = ex[q];
      out.x[ta + i] = lb->xyz[3 * (size_t)(a0 + i)];
      out.y[ta + i] = lb->xyz[3 * (size_t)(a0 + i) + 1];
      out.z[ta + i] = lb->xyz[3 * (size_t)(a0 + i) + 2];
    }
    out.ids[l] = lb->ids[l];
    out.cost[l] = (int64_t)(1 + p->post_align) * N * N * n + (int64_t)A * 2 * moved + 64;
  }
  return true;
}

// Validates ligands and packs them into `out` (which must be empty).  The offsets come first, from
// the ligand counts alone (a ligand whose counts are out of range gets none, and fails below before
// it writes), so every array is sized once and large submissions are prepared in tasks of 256
// ligands by the host worker pool, each writing its own range in place.  On failure `err` names
// the first bad ligand and the field.
bool prepare(const dock_ligand_batch* lb, const dock_params* p, Packed& out, std::string& err) {
  if (!check_params(p, err)) return false;
  if (!lb) return err = "ligand batch is NULL", false;
  const int L = lb->n_lig;
  if (L < 0) return err = "n_lig < 0", false;
  if (L == 0) return true;
  if (!lb->atom_off || !lb->xyz || !lb->bond_off || !lb->rot_off || !lb->ids || (lb->bond_off[L] > 0 && !lb->bonds) ||
      (lb->rot_off[L] > 0 && !lb->rot_bonds))
    return err = "a ligand array pointer is NULL", false;
  if (lb->atom_off[0] != 0 || lb->bond_off[0] != 0 || lb->rot_off[0] != 0)
    return err = "atom_off[0], bond_off[0] and rot_off[0] must be 0", false;
  out.atom_off.resize((size_t)L + 1);
  out.rot_off.resize((size_t)L + 1);
  for (int l = 0; l < L; ++l) {
    const int n = lb->atom_off[l + 1] - lb->atom_off[l], nr = lb->rot_off[l + 1] - lb->rot_off[l];
    const bool in_range = n >= 1 && n <= DOCK_MAX_ATOMS && nr >= 0 && nr <= DOCK_MAX_ROT;
    out.atom_off[l + 1] = out.atom_off[l] + (in_range ? n : 0);
    out.rot_off[l + 1] = out.rot_off[l] + (in_range ? nr : 0);
  }
  const size_t atoms = (size_t)out.atom_off[L], rots = (size_t)out.rot_off[L];
  out.ids.resize(L);
  out.cost.resize(L);
  out.x.resize(atoms);
  out.y.resize(atoms);
  out.z.resize(atoms);
  out.excl.resize(atoms * kMaskWords);
  out.rot_ab.resize(rots);
  out.mask.resize(rots * kMaskWords);
  constexpr int kPerTask = 256;
  const int T = std::max(1, (L + kPerTask - 1) / kPerTask);
  std::vector<std::string> errs(T);
  std::vector<int> bads(T, -1);
  std::vector<uint64_t> moving(T, 0);
  std::vector<char> ok(T, 1);
  const std::function<void(int)> run = [&](int t) {
    const int a = (int)((int64_t)L * t / T), b = (int)((int64_t)L * (t + 1) / T);
    ok[t] = prepare_range(lb, p, a, b, out, moving[t], errs[t], bads[t]);
  };
  WorkPool::get().run(T, run);
  for (int t = 0; t < T; ++t)  // the first failing range holds the first bad ligand
    if (!ok[t]) return out = Packed{}, err = errs[t], false;
  for (uint64_t m : moving) out.moving += m;
  out.n_lig = L;
  return true;
}

// ---- batch layout: one device arena and its pinned mirror ---------------------------------------

struct Layout {
  size_t hdr, ids, x, y, z, rot_ab, mask, excl, items, in_end;
  size_t restart_score, restart_clash, align_idx, post_idx, tors_idx, rejected, best_score, best_restart, out_xyz,
      clash, select_restart, select_score, select_xyz, out_end;
  size_t rs_xyz, done, counters, lat, total;
  size_t sel_k;  // poses Select Poses keeps per ligand; 0 when it keeps only the best one, whose
                 // outputs are then copied from the best-restart arrays instead of a second copy
  // first result byte copied back: every output, or (DOCK_OUTPUT_BEST) only the per-ligand ones,
  // which the layout keeps contiguous at the end of the result region
  size_t out_begin(int outputs) const { return outputs == DOCK_OUTPUT_BEST ? best_score : in_end; }
};

Layout make_layout(size_t L, size_t atoms, size_t rots, size_t R, size_t K, size_t lat_bytes) {
  Layout y{};
  y.sel_k = K > 1 ? K : 0;
  K = y.sel_k;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t r = o;
    o = (o + bytes + 255) & ~size_t(255);
    return r;
  };
  y.hdr = take(16 * L);
  y.ids = take(8 * L);
  y.x = take(4 * atoms);
  y.y = take(4 * atoms);
  y.z = take(4 * atoms);
  y.rot_ab = take(4 * rots);
  y.mask = take(4 * kMaskWords * rots);
  y.excl = take(4 * kMaskWords * atoms);
  y.items = take(4 * L * R);
  y.in_end = o;
  y.restart_score = take(4 * L * R);
  y.restart_clash = take(4 * L * R);
  y.align_idx = take(4 * L * R);
  y.post_idx = take(4 * L * R);
  y.tors_idx = take(4 * rots * R);
  y.rejected = take(4 * rots * R);
  y.best_score = take(4 * L);
  y.best_restart = take(4 * L);
  y.out_xyz = take(12 * atoms);
  y.clash = take(4 * L);
  y.select_restart = take(4 * L * K);
  y.select_score = take(4 * L * K);
  y.select_xyz = take(12 * atoms * K);
  y.out_end = o;
  y.rs_xyz = take(12 * atoms * R);
  y.done = take(4 * L);
  y.counters = take(4 * kNumBuckets);
  y.lat = take(lat_bytes);  // the latency form's scratch (one ligand at a time)
  y.total = std::max<size_t>(o, 256);  // an empty batch still gets valid (non-NULL) buffers
  y.out_end = std::max<size_t>(y.out_end, 256);
  return y;
}

struct LigRef {
  const Packed* pk;
  int l;
};

struct Plan {
  int n_lig = 0, atoms = 0, rots = 0;
  int n_items[kNumBuckets] = {0}, item_off[kNumBuckets] = {0};
  int64_t bucket_cost[kNumBuckets] = {0};  // estimated work per bucket (launch order, heaviest first)
  std::vector<int> lig_item_off;  // first item of each ligand (its R items are consecutive)
  std::vector<int> lig_atom_off, lig_rot_off;
};

// Reorders the ligand indices `v` by descending cost, equal costs in their given order: the order
// of a stable comparison sort, from a least-significant-digit radix sort (11-bit digits, stopping
// after the highest digit in use), a few times faster on the tens of thousands of ligands of a
// large batch.
void sort_by_cost_desc(std::vector<int>& v, const std::vector<int64_t>& cost) {
  if (v.size() < 2) return;
  int64_t hi = 0;
  for (int i : v) hi = std::max(hi, cost[i]);
  std::vector<std::pair<uint64_t, int>> a(v.size()), t(v.size());
  uint64_t span = 0;
  for (size_t k = 0; k < v.size(); ++k) {
    a[k] = {(uint64_t)(hi - cost[v[k]]), v[k]};
    span |= a[k].first;
  }
  constexpr int kDigit = 11, kBins = 1 << kDigit;
  for (int shift = 0; shift < 64 && (span >> shift); shift += kDigit) {
    std::vector<size_t> cnt(kBins + 1, 0);
    for (const auto& e : a) ++cnt[((e.first >> shift) & (kBins - 1)) + 1];
    for (int d = 0; d < kBins; ++d) cnt[d + 1] += cnt[d];
    for (const auto& e : a) t[cnt[(e.first >> shift) & (kBins - 1)]++] = e;
    a.swap(t);
  }
  for (size_t k = 0; k < v.size(); ++k) v[k] = a[k].second;
}

// Writes the inputs of `ligs` into the host mirror and fills the plan.
void fill_inputs(char* h, const Layout& y, const std::vector<LigRef>& ligs, int R, Plan& plan) {
  const int L = (int)ligs.size();
  plan.n_lig = L;
  plan.lig_atom_off.assign(L + 1, 0);
  plan.lig_rot_off.assign(L + 1, 0);
  int4* hdr = reinterpret_cast<int4*>(h + y.hdr);
  uint64_t* ids = reinterpret_cast<uint64_t*>(h + y.ids);
  float* xs = reinterpret_cast<float*>(h + y.x);
  float* ys = reinterpret_cast<float*>(h + y.y);
  float* zs = reinterpret_cast<float*>(h + y.z);
  uint32_t* rab = reinterpret_cast<uint32_t*>(h + y.rot_ab);
  uint32_t* msk = reinterpret_cast<uint32_t*>(h + y.mask);
  uint32_t* exc = reinterpret_cast<uint32_t*>(h + y.excl);
  std::vector<int> bucket_ligs[kNumBuckets];
  std::vector<int64_t> cost(L);
  // Consecutive ligands of one submission are contiguous in its packed arrays and land contiguously
  // here, so each such run is copied with one memcpy per array.
  auto copy_run = [&](int i0, int i1) {
    const Packed& P = *ligs[i0].pk;
    const int l0 = ligs[i0].l, l1 = ligs[i1 - 1].l + 1;
    const size_t pa = P.atom_off[l0], na = P.atom_off[l1] - pa, pr = P.rot_off[l0], nr = P.rot_off[l1] - pr;
    const size_t ao = plan.lig_atom_off[i0], ro = plan.lig_rot_off[i0];
    std::memcpy(ids + i0, P.ids.data() + l0, 8 * (size_t)(i1 - i0));
    std::memcpy(xs + ao, P.x.data() + pa, 4 * na);
    std::memcpy(ys + ao, P.y.data() + pa, 4 * na);
    std::memcpy(zs + ao, P.z.data() + pa, 4 * na);
    std::memcpy(exc + ao * kMaskWords, P.excl.data() + pa * kMaskWords, 4 * na * kMaskWords);
    if (nr) {
      std::memcpy(rab + ro, P.rot_ab.data() + pr, 4 * nr);
      std::memcpy(msk + ro * kMaskWords, P.mask.data() + pr * kMaskWords, 4 * nr * kMaskWords);
    }
  };
  int ao = 0, ro = 0, run = 0;
  for (int i = 0; i < L; ++i) {
    const Packed& P = *ligs[i].pk;
    const int l = ligs[i].l;
    if (i > run && (ligs[i].pk != ligs[i - 1].pk || l != ligs[i - 1].l + 1)) {
      copy_run(run, i);
      run = i;
    }
    cost[i] = P.cost[l];
    const int n = P.atom_off[l + 1] - P.atom_off[l], B = P.rot_off[l + 1] - P.rot_off[l];
    hdr[i] = make_int4(ao, n, ro, B);
    bucket_ligs[bucket_of(n)].push_back(i);
    ao += n;
    ro += B;
    plan.lig_atom_off[i + 1] = ao;
    plan.lig_rot_off[i + 1] = ro;
  }
  if (L > run) copy_run(run, L);
  plan.atoms = ao;
  plan.rots = ro;
  uint32_t* items = reinterpret_cast<uint32_t*>(h + y.items);
  plan.lig_item_off.assign(L, 0);
  int it = 0;
  for (int b = 0; b < kNumBuckets; ++b) {
    auto& v = bucket_ligs[b];
    sort_by_cost_desc(v, cost);
    plan.item_off[b] = it;
    plan.bucket_cost[b] = 0;
    for (int i : v) {
      plan.bucket_cost[b] += cost[i] * R;
      plan.lig_item_off[i] = it;
      for (int r = 0; r < R; ++r) items[it++] = ((uint32_t)i << kRestartBits) | (uint32_t)r;
    }
    plan.n_items[b] = it - plan.item_off[b];
  }
}

BatchDev batch_pointers(char* d, const Layout& y, int L) {
  BatchDev b{};
  b.n_lig = L;
  b.hdr = reinterpret_cast<const int4*>(d + y.hdr);
  b.ids = reinterpret_cast<const unsigned long long*>(d + y.ids);
  b.x = reinterpret_cast<const float*>(d + y.x);
  b.y = reinterpret_cast<const float*>(d + y.y);
  b.z = reinterpret_cast<const float*>(d + y.z);
  b.rot_ab = reinterpret_cast<const uint32_t*>(d + y.rot_ab);
  b.mask = reinterpret_cast<const uint32_t*>(d + y.mask);
  b.excl = reinterpret_cast<const uint32_t*>(d + y.excl);
  b.restart_score = reinterpret_cast<float*>(d + y.restart_score);
  b.restart_clash = reinterpret_cast<int*>(d + y.restart_clash);
  b.align_idx = reinterpret_cast<int*>(d + y.align_idx);
  b.post_idx = reinterpret_cast<int*>(d + y.post_idx);
  b.tors_idx = reinterpret_cast<int*>(d + y.tors_idx);
  b.rejected = reinterpret_cast<int*>(d + y.rejected);
  b.best_score = reinterpret_cast<float*>(d + y.best_score);
  b.best_restart = reinterpret_cast<int*>(d + y.best_restart);
  b.out_xyz = reinterpret_cast<float*>(d + y.out_xyz);
  b.clash = reinterpret_cast<int*>(d + y.clash);
  if (y.sel_k) {
    b.select_restart = reinterpret_cast<int*>(d + y.select_restart);
    b.select_score = reinterpret_cast<float*>(d + y.select_score);
    b.select_xyz = reinterpret_cast<float*>(d + y.select_xyz);
  }
  b.rs_xyz = reinterpret_cast<float*>(d + y.rs_xyz);
  b.done = reinterpret_cast<unsigned*>(d + y.done);
  b.next_item = reinterpret_cast<unsigned*>(d + y.counters);
  return b;
}

ParamsDev params_dev(const dock_params& p) {
  ParamsDev d{};
  d.R = p.restarts;
  d.N = p.align_steps;
  d.A = p.torsion_steps;
  d.dc2 = p.clash_dist * p.clash_dist;
  d.post_align = p.post_align;
  d.early_exit = p.early_exit;
  d.seed = p.seed;
  d.K = p.select_k <= 0 ? 1 : p.select_k;
  d.sel_rmsd2 = p.select_rmsd * p.select_rmsd;
  return d;
}

bool same_params(const dock_params& a, const dock_params& b) {
  return a.restarts == b.restarts && a.align_steps == b.align_steps && a.torsion_steps == b.torsion_steps &&
         a.clash_dist == b.clash_dist && a.post_align == b.post_align && a.early_exit == b.early_exit &&
         a.seed == b.seed && a.select_k == b.select_k && a.select_rmsd == b.select_rmsd && a.outputs == b.outputs;
}

struct Pocket {
  PocketDev dev{};
  void* cells = nullptr;       // stream-ordered allocation (cudaMallocAsync on the context's stream)
  std::vector<cudaEvent_t> uses;  // recorded after launches that read the pocket, pruned as they finish
  bool closed = false;         // unloaded: unknown to new calls, kept for ligands already submitted
  int64_t queued = 0;          // submitted ligands naming the pocket that the serving loop has not
                               // admitted yet; a closed pocket is released when this reaches 0
};

// Streams and events that let the bucket kernels of one batch run side by side: the heaviest
// bucket runs on the caller's stream, the others on their own streams forked from it and joined
// back before the caller's stream goes on.
struct Fork {
  cudaStream_t aux[kNumBuckets] = {};
  cudaEvent_t forked = nullptr;
  cudaEvent_t joined[kNumBuckets] = {};

  cudaError_t create() {
    cudaError_t e = cudaEventCreateWithFlags(&forked, cudaEventDisableTiming);
    for (int b = 0; b < kNumBuckets && e == cudaSuccess; ++b) {
      e = cudaStreamCreateWithFlags(&aux[b], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&joined[b], cudaEventDisableTiming);
    }
    return e;
  }
  void destroy() {
    for (int b = 0; b < kNumBuckets; ++b) {
      if (aux[b]) cudaStreamDestroy(aux[b]);
      if (joined[b]) cudaEventDestroy(joined[b]);
    }
    if (forked) cudaEventDestroy(forked);
  }
};

struct Ticket {
  uint64_t id = 0;
  int pocket = 0;
  dock_params params{};
  Packed pk;
  int64_t t_submit = 0;
  int n_admitted = 0, n_done = 0;
  std::vector<float> score, xyz, restart_score, select_score, select_xyz;
  std::vector<int32_t> best_restart, clash, restart_clash, align_idx, post_idx, tors_idx, rejected, select_restart;
  std::vector<int64_t> lat;
  int K = 1;
  bool full = true;  // DOCK_OUTPUT_FULL: per-restart and per-bond outputs kept
};

struct Slot {
  cudaStream_t stream = nullptr;
  Fork fork;
  cudaEvent_t ev = nullptr;
  char* dev = nullptr;
  size_t dev_cap = 0;
  char* host = nullptr;
  size_t host_cap = 0;
  bool busy = false;
  int64_t t_launch = 0;
  Layout y{};
  Plan plan;
  std::vector<std::pair<uint64_t, int>> members;  // (ticket, ligand index in the ticket)
  int R = 0;
};

int cuda_status(cudaError_t e) { return e == cudaErrorMemoryAllocation ? DOCK_ERR_NOMEM : DOCK_ERR_CUDA; }

}  // namespace

// ---- the context -------------------------------------------------------------------------------------

struct dock_batch {
  int n_lig = 0;
  dock_work work{};
  // the batched launch sequence captured as a CUDA graph, for the pocket and launch shapes it was
  // captured with
  cudaGraphExec_t gexec[3] = {};   // per form (DOCK_FORM_BATCHED, -, DOCK_FORM_LATENCY)
  int graph_pocket[3] = {-1, -1, -1};
  uint64_t graph_version[3] = {};
  int graph_kernels[3] = {};
  dock_params params{};
  Layout y{};
  Plan plan;
  char* dev = nullptr;
  char* host = nullptr;
  cudaEvent_t ev = nullptr;
  bool launched = false;
};

struct dock_ctx {
  dock_config cfg{};
  int device = 0;
  cudaStream_t stream = nullptr;
  Fork fork;  // for dock_batch_launch
  std::mutex mu;
  std::condition_variable work_cv, done_cv;
  std::string last_error;
  std::unordered_map<int, Pocket> pockets;
  int next_pocket = 1;
  std::unordered_map<uint64_t, std::unique_ptr<Ticket>> tickets;
  std::deque<uint64_t> pending;  // tickets with ligands not yet admitted, FIFO
  uint64_t next_ticket = 1;
  int64_t queued = 0;            // ligands submitted but not yet admitted
  std::vector<Slot> slots;
  std::thread server;
  bool stop = false;
  int fatal = 0;
  std::string fatal_msg;
  LaunchCfg launch_cfg[kNumBuckets];
  int64_t latency_items = 0;  // serving batches of at most this many items use latency_launch
  int64_t latency_form_ligands = 0;  // serving batches of at most this many ligands: latency form
  uint64_t launch_version = 1;   // bumped by dock_set_launch (invalidates captured graphs)
  cudaStream_t capture_stream = nullptr;
  Fork capture_fork;
  dock_stats stats{};
  std::vector<cudaEvent_t> spare_events;  // recycled pocket-use events
  unsigned long long* exec = nullptr;  // executed-work counters (counter build only)

  int fail(int code, const std::string& msg) {
    last_error = msg;
    return code;
  }
  int cuda_fail(cudaError_t e, const char* what) {
    return fail(cuda_status(e), fmt("%s: %s", what, cudaGetErrorString(e)));
  }
};

namespace {

// Default launch shape of a bucket: 8 warps per block, driver carveout, persistent, two warps per
// item, the shape the autotuner settles on for the uneven database and for most uniform batches.
LaunchCfg default_launch(int bucket) { return LaunchCfg{8, -1, 1, bucket, 2, 1}; }

// Records, on stream s, that work queued there reads pocket P (context lock held).  Events of
// finished uses are recycled first, so the list holds only launches that may still be running.
void note_use(dock_ctx* ctx, Pocket& P, cudaStream_t s) {
  size_t keep = 0;
  for (cudaEvent_t e : P.uses) {
    if (cudaEventQuery(e) == cudaSuccess)
      ctx->spare_events.push_back(e);
    else
      P.uses[keep++] = e;
  }
  P.uses.resize(keep);
  cudaEvent_t e = nullptr;
  if (!ctx->spare_events.empty()) {
    e = ctx->spare_events.back();
    ctx->spare_events.pop_back();
  } else if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
    e = nullptr;
  }
  if (e && cudaEventRecord(e, s) == cudaSuccess) {
    P.uses.push_back(e);
    return;
  }
  if (e) ctx->spare_events.push_back(e);
  // the use cannot be recorded: let it finish now, so that a later unload cannot free the pocket
  // under it (reached only when the runtime cannot create or record an event)
  cudaStreamSynchronize(s);
}

// The loaded (not unloaded) pocket `id`, or nullptr.
Pocket* open_pocket(dock_ctx* ctx, int id) {
  auto it = ctx->pockets.find(id);
  return it == ctx->pockets.end() || it->second.closed ? nullptr : &it->second;
}

// Frees pocket P once every launch that reads it has finished, without blocking the host: the
// context's stream waits for each recorded use and the memory is freed in stream order there.
void release_pocket(dock_ctx* ctx, Pocket& P) {
  for (cudaEvent_t e : P.uses) {
    cudaStreamWaitEvent(ctx->stream, e, 0);
    ctx->spare_events.push_back(e);  // the wait has captured the event's state; it may be reused
  }
  P.uses.clear();
  if (P.cells) cudaFreeAsync(P.cells, ctx->stream);
  P.cells = nullptr;
}

// Launches every bucket of a prepared batch; the work is complete when stream s reaches the point
// after the call.  Returns launches or a negative error.
// The latency-oriented launch shape: one ligand-restart per block of 8 warps, all 8 on it.
LaunchCfg latency_launch(int bucket) { return LaunchCfg{8, -1, 0, bucket, 8, 1}; }

int launch_batch(dock_ctx* ctx, const PocketDev& pk, char* dev, const Layout& y, const Plan& plan,
                 const dock_params& prm, int form, cudaStream_t s, Fork* fork, std::string& err,
                 bool set_attributes = true, bool latency_shape = false) {
  const BatchDev bd = batch_pointers(dev, y, plan.n_lig);
  ParamsDev pd = params_dev(prm);
  pd.exec = ctx->exec;
  const uint32_t* items = reinterpret_cast<const uint32_t*>(dev + y.items);
  int launches = 0;
  if (form == DOCK_FORM_BATCHED) {
    int order[kNumBuckets], nb = 0;
    for (int b = 0; b < kNumBuckets; ++b)
      if (plan.n_items[b]) order[nb++] = b;
    std::sort(order, order + nb, [&](int p, int q) { return plan.bucket_cost[p] > plan.bucket_cost[q]; });
    cudaError_t e = cudaSuccess;
    bool any_persistent = false;
    auto shape = [&](int b) { return latency_shape ? latency_launch(b) : ctx->launch_cfg[b]; };
    for (int i = 0; i < nb; ++i) any_persistent |= shape(order[i]).persistent != 0;
    if (any_persistent) e = cudaMemsetAsync(bd.next_item, 0, 4 * kNumBuckets, s);
    if (nb > 1 && e == cudaSuccess) e = cudaEventRecord(fork->forked, s);
    for (int i = 0; i < nb && e == cudaSuccess; ++i) {
      const int b = order[i];
      cudaStream_t t = i == 0 ? s : fork->aux[b];
      if (i > 0) e = cudaStreamWaitEvent(t, fork->forked, 0);
      LaunchCfg cfg = shape(b);
      cfg.counter_slot = b;
      if (e == cudaSuccess)
        e = launch_dock_bucket(b, pk, bd, pd, items + plan.item_off[b], plan.n_items[b], cfg, t, set_attributes);
      if (e == cudaSuccess && i > 0) e = cudaEventRecord(fork->joined[b], t);
      if (e == cudaSuccess) ++launches;
    }
    for (int i = 1; i < nb && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(s, fork->joined[order[i]], 0);
    if (e == cudaSuccess && bd.select_restart && plan.n_lig) {
      e = launch_select(bd, pd, s);
      if (e == cudaSuccess) ++launches;
    }
    if (e != cudaSuccess) return err = fmt("dock kernel launch: %s", cudaGetErrorString(e)), cuda_status(e);
    ctx->stats.kernel_launches += launches;
  } else if (form == DOCK_FORM_LATENCY) {
    // one ligand at a time over the whole GPU, all on stream s (they share the latency scratch)
    const LatScratch sc = latency_scratch(dev + y.lat, prm.restarts, prm.align_steps);
    if (plan.n_lig) {  // the per-restart block counters reset themselves after their first use
      const cudaError_t e = cudaMemsetAsync(sc.done, 0, 4 * (size_t)prm.restarts, s);
      if (e != cudaSuccess) return err = fmt("latency scratch: %s", cudaGetErrorString(e)), cuda_status(e);
    }
    for (int k = 0; k < kNumBuckets && set_attributes; ++k)
      if (plan.n_items[k]) {
        const cudaError_t e = launch_latency_ligand(k, pk, bd, pd, -1, sc, s, nullptr);
        if (e != cudaSuccess) return err = fmt("latency kernel attributes: %s", cudaGetErrorString(e)), cuda_status(e);
      }
    for (int i = 0; i < plan.n_lig; ++i) {
      const int n = plan.lig_atom_off[i + 1] - plan.lig_atom_off[i];
      const cudaError_t e = launch_latency_ligand(bucket_of(n), pk, bd, pd, i, sc, s, &launches);
      if (e != cudaSuccess) return err = fmt("latency kernel launch: %s", cudaGetErrorString(e)), cuda_status(e);
    }
    if (bd.select_restart && plan.n_lig) {
      const cudaError_t e = launch_select(bd, pd, s);
      if (e != cudaSuccess) return err = fmt("select kernel launch: %s", cudaGetErrorString(e)), cuda_status(e);
      ++launches;
    }
    ctx->stats.kernel_launches += launches;
  } else {
    for (int i = 0; i < plan.n_lig; ++i) {
      const int n = plan.lig_atom_off[i + 1] - plan.lig_atom_off[i];
      LaunchCfg cfg = ctx->launch_cfg[bucket_of(n)];
      cfg.persistent = 0;  // the plain form: one launch per ligand, one warp per restart
      const cudaError_t e = launch_dock_bucket(bucket_of(n), pk, bd, pd, items + plan.lig_item_off[i], prm.restarts,
                                               cfg, s);
      if (e != cudaSuccess) return err = fmt("dock kernel launch: %s", cudaGetErrorString(e)), cuda_status(e);
      ++launches;
    }
    if (bd.select_restart && plan.n_lig) {
      const cudaError_t e = launch_select(bd, pd, s);
      if (e != cudaSuccess) return err = fmt("select kernel launch: %s", cudaGetErrorString(e)), cuda_status(e);
      ++launches;
    }
    ctx->stats.kernel_launches += launches;
  }
  return launches;
}

// Copies results of ligands [0, L) of a finished batch mirror into caller buffers laid out like
// the batch (the plan's offsets equal the caller's offsets for a batch made from one submission).
void copy_results(const char* h, const Layout& y, const Plan& plan, int R, dock_result_buffers* o) {
  const size_t L = plan.n_lig, A = plan.atoms, Q = plan.rots;
  if (o->score) std::memcpy(o->score, h + y.best_score, 4 * L);
  if (o->best_restart) std::memcpy(o->best_restart, h + y.best_restart, 4 * L);
  if (o->xyz) std::memcpy(o->xyz, h + y.out_xyz, 12 * A);
  if (o->clash_count) std::memcpy(o->clash_count, h + y.clash, 4 * L);
  if (o->restart_score) std::memcpy(o->restart_score, h + y.restart_score, 4 * L * R);
  if (o->restart_clash) std::memcpy(o->restart_clash, h + y.restart_clash, 4 * L * R);
  if (o->align_idx) std::memcpy(o->align_idx, h + y.align_idx, 4 * L * R);
  if (o->post_idx) std::memcpy(o->post_idx, h + y.post_idx, 4 * L * R);
  if (o->torsion_idx) std::memcpy(o->torsion_idx, h + y.tors_idx, 4 * Q * R);
  if (o->rejected) std::memcpy(o->rejected, h + y.rejected, 4 * Q * R);
  const size_t K = y.sel_k;
  if (o->select_restart) std::memcpy(o->select_restart, h + (K ? y.select_restart : y.best_restart), 4 * L * (K ? K : 1));
  if (o->select_score) std::memcpy(o->select_score, h + (K ? y.select_score : y.best_score), 4 * L * (K ? K : 1));
  if (o->select_xyz) std::memcpy(o->select_xyz, h + (K ? y.select_xyz : y.out_xyz), 12 * A * (K ? K : 1));
}

// Launches a prepared batch through a CUDA graph of its launch sequence (DOCK_FORM_BATCHED: the
// bucket kernels; DOCK_FORM_LATENCY: every ligand's kernels in order) captured on first use and
// re-captured when the pocket or the launch shapes change.  Returns kernels per launch or a
// negative error.
int graph_launch(dock_ctx* ctx, int pocket_id, const PocketDev& pk, dock_batch* b, cudaStream_t s, std::string& err,
                 int form = DOCK_FORM_BATCHED) {
  cudaGraphExec_t& gexec = b->gexec[form];
  if (!gexec || b->graph_pocket[form] != pocket_id || b->graph_version[form] != ctx->launch_version) {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
    const BatchDev bd = batch_pointers(b->dev, b->y, b->plan.n_lig);
    ParamsDev pd = params_dev(b->params);
    pd.exec = ctx->exec;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kNumBuckets && e == cudaSuccess; ++k)  // attributes outside the capture
      if (b->plan.n_items[k]) {
        e = form == DOCK_FORM_BATCHED
                ? launch_dock_bucket(k, pk, bd, pd, nullptr, 0, ctx->launch_cfg[k], s, true)
                : launch_latency_ligand(k, pk, bd, pd, -1, LatScratch{}, s, nullptr);
      }
    if (e != cudaSuccess) return err = fmt("kernel attributes: %s", cudaGetErrorString(e)), cuda_status(e);
    e = cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return err = fmt("begin capture: %s", cudaGetErrorString(e)), cuda_status(e);
    const uint64_t before = ctx->stats.kernel_launches;
    const int rc = launch_batch(ctx, pk, b->dev, b->y, b->plan, b->params, form, ctx->capture_stream,
                                &ctx->capture_fork, err, false);
    ctx->stats.kernel_launches = before;  // nothing ran yet
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(ctx->capture_stream, &g);
    if (rc < 0) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      gexec = nullptr;
      return err = fmt("graph capture: %s", cudaGetErrorString(e)), cuda_status(e);
    }
    b->graph_pocket[form] = pocket_id;
    b->graph_version[form] = ctx->launch_version;
    b->graph_kernels[form] = rc;
  }
  const cudaError_t e = cudaGraphLaunch(gexec, s);
  if (e != cudaSuccess) return err = fmt("graph launch: %s", cudaGetErrorString(e)), cuda_status(e);
  ctx->stats.kernel_launches += b->graph_kernels[form];
  ctx->stats.graph_launches += 1;
  return b->graph_kernels[form];
}

// Latency-form batches of up to this many ligands run from a captured graph (four kernel nodes per
// ligand); larger ones are launched directly.
constexpr int kLatencyGraphLigands = 256;

// ---- serving loop ------------------------------------------------------------------------------------

void scatter_slot(dock_ctx* ctx, Slot& s) {
  const char* h = s.host;
  const Layout& y = s.y;
  const int R = s.R;
  const int64_t t = now_ns();
  for (size_t i = 0; i < s.members.size(); ++i) {
    auto it = ctx->tickets.find(s.members[i].first);
    if (it == ctx->tickets.end()) continue;
    Ticket& T = *it->second;
    const int l = s.members[i].second;
    const int n = T.pk.atom_off[l + 1] - T.pk.atom_off[l], B = T.pk.rot_off[l + 1] - T.pk.rot_off[l];
    const int ta = T.pk.atom_off[l], tr = T.pk.rot_off[l];
    const int ba = s.plan.lig_atom_off[i], br = s.plan.lig_rot_off[i];
    T.score[l] = reinterpret_cast<const float*>(h + y.best_score)[i];
    T.best_restart[l] = reinterpret_cast<const int*>(h + y.best_restart)[i];
    T.clash[l] = reinterpret_cast<const int*>(h + y.clash)[i];
    std::memcpy(&T.xyz[3 * (size_t)ta], h + y.out_xyz + 12 * (size_t)ba, 12 * (size_t)n);
    if (T.full) {
      std::memcpy(&T.restart_score[(size_t)l * R], h + y.restart_score + 4 * i * R, 4 * (size_t)R);
      std::memcpy(&T.restart_clash[(size_t)l * R], h + y.restart_clash + 4 * i * R, 4 * (size_t)R);
      std::memcpy(&T.align_idx[(size_t)l * R], h + y.align_idx + 4 * i * R, 4 * (size_t)R);
      std::memcpy(&T.post_idx[(size_t)l * R], h + y.post_idx + 4 * i * R, 4 * (size_t)R);
      if (B) {
        std::memcpy(&T.tors_idx[(size_t)tr * R], h + y.tors_idx + 4 * (size_t)br * R, 4 * (size_t)B * R);
        std::memcpy(&T.rejected[(size_t)tr * R], h + y.rejected + 4 * (size_t)br * R, 4 * (size_t)B * R);
      }
    }
    if (const size_t K = y.sel_k) {
      std::memcpy(&T.select_restart[l * K], h + y.select_restart + 4 * i * K, 4 * K);
      std::memcpy(&T.select_score[l * K], h + y.select_score + 4 * i * K, 4 * K);
      std::memcpy(&T.select_xyz[3 * (size_t)ta * K], h + y.select_xyz + 12 * (size_t)ba * K, 12 * (size_t)n * K);
    } else {
      T.select_restart[l] = T.best_restart[l];
      T.select_score[l] = T.score[l];
      std::memcpy(&T.select_xyz[3 * (size_t)ta], &T.xyz[3 * (size_t)ta], 12 * (size_t)n);
    }
    T.lat[l] = t - T.t_submit;
    ++T.n_done;
    ++ctx->stats.ligands_done;
  }
  s.members.clear();
  s.busy = false;
  ctx->stats.scatter_ns += (uint64_t)(now_ns() - t);
}

// Capacity for a buffer that must hold `need` bytes: the next power of four from 4 MiB, but no
// more than `limit` (and never less than `need`).  Pinning host memory stalls the whole process's
// memory mapping while it runs, so a slot should grow in few, large steps.
size_t grown_capacity(size_t need, size_t limit) {
  size_t c = size_t(4) << 20;
  while (c < need) c <<= 2;
  return std::max(need, std::min(c, limit));
}

// Packs waiting ligands into slot s and launches them.  Returns true if a batch was launched.
bool admit(dock_ctx* ctx, Slot& s, std::unique_lock<std::mutex>& lk) {
  while (!ctx->pending.empty()) {  // drop finished heads
    auto it = ctx->tickets.find(ctx->pending.front());
    if (it != ctx->tickets.end() && it->second->n_admitted < it->second->pk.n_lig) break;
    ctx->pending.pop_front();
  }
  if (ctx->pending.empty()) return false;
  Ticket& head = *ctx->tickets[ctx->pending.front()];
  const int pocket = head.pocket;
  const dock_params prm = head.params;
  const size_t cap = ctx->cfg.hbm_budget_bytes / ctx->slots.size();
  const int R = prm.restarts;
  const int K = params_dev(prm).K;
  const size_t lat = latency_scratch_bytes(R, prm.align_steps);
  std::vector<LigRef> refs;
  s.members.clear();
  size_t L = 0, atoms = 0, rots = 0;
  for (uint64_t tid : ctx->pending) {
    auto it = ctx->tickets.find(tid);
    if (it == ctx->tickets.end()) continue;
    Ticket& T = *it->second;
    if (T.pocket != pocket || !same_params(T.params, prm)) continue;
    while (T.n_admitted < T.pk.n_lig && (int)L < ctx->cfg.max_batch_ligands) {
      const int l = T.n_admitted;
      const size_t n = T.pk.atom_off[l + 1] - T.pk.atom_off[l], B = T.pk.rot_off[l + 1] - T.pk.rot_off[l];
      if (L > 0 && make_layout(L + 1, atoms + n, rots + B, R, K, lat).total > cap) break;
      refs.push_back({&T.pk, l});
      s.members.push_back({tid, l});
      ++L;
      atoms += n;
      rots += B;
      ++T.n_admitted;
      --ctx->queued;
    }
    if ((int)L >= ctx->cfg.max_batch_ligands) break;
  }
  if (L == 0) return false;
  s.y = make_layout(L, atoms, rots, R, K, lat);
  s.R = R;
  cudaError_t e = cudaSuccess;
  if (s.y.total > s.dev_cap || s.y.out_end > s.host_cap) {
    // A slot that must grow is sized for a full batch (max_batch_ligands) of ligands like these,
    // in steps of four and within its share of the budget, so it grows about once.  The context
    // lock is released meanwhile: pinning host memory takes milliseconds and submit, poll and
    // results must not wait for it.  Nothing else touches an idle slot, and the tickets of its
    // members stay until their ligands are done.  Device memory is stream-ordered, so freeing it
    // waits for nothing but the slot's own (finished) work.
    const size_t maxL = (size_t)ctx->cfg.max_batch_ligands;
    const Layout full = make_layout(maxL, atoms * maxL / L, rots * maxL / L, R, K, lat);
    lk.unlock();
    const int64_t t_grow = now_ns();
    if (s.y.total > s.dev_cap) {
      if (s.dev) cudaFreeAsync(s.dev, s.stream);
      s.dev = nullptr;
      s.dev_cap = 0;
      const size_t want = std::max(s.y.total, std::min(grown_capacity(full.total, cap), cap));
      e = cudaMallocAsync(reinterpret_cast<void**>(&s.dev), want, s.stream);
      if (e == cudaSuccess) s.dev_cap = want;
    }
    if (e == cudaSuccess && s.y.out_end > s.host_cap) {
      if (s.host) cudaFreeHost(s.host);
      s.host = nullptr;
      s.host_cap = 0;
      const size_t want = std::max(s.y.out_end, std::min(grown_capacity(full.out_end, cap), cap));
      e = cudaHostAlloc(reinterpret_cast<void**>(&s.host), want, cudaHostAllocDefault);
      if (e == cudaSuccess) s.host_cap = want;
    }
    const uint64_t dt = (uint64_t)(now_ns() - t_grow);
    lk.lock();
    ctx->stats.slot_grows += 1;
    ctx->stats.slot_grow_ns += dt;
  }
  auto pit = ctx->pockets.find(pocket);  // after the lock may have been released (closed or not)
  if (pit != ctx->pockets.end()) pit->second.queued -= (int64_t)L;
  std::string err;
  int rc = 0;
  if (e == cudaSuccess && pit != ctx->pockets.end()) {
    const int64_t t0 = now_ns();
    fill_inputs(s.host, s.y, refs, R, s.plan);
    ctx->stats.fill_ns += (uint64_t)(now_ns() - t0);
    e = cudaMemcpyAsync(s.dev, s.host, s.y.in_end, cudaMemcpyHostToDevice, s.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.dev + s.y.done, 0, 4 * L, s.stream);
    if (e == cudaSuccess) {
      // a small batch (light load) finishes sooner with the latency-oriented shape, and a batch of
      // at most latency_form_ligands ligands sooner still in the latency form (one ligand at a
      // time over the whole GPU)
      const bool lat_form = (int64_t)L <= ctx->latency_form_ligands;
      const bool latency = (int64_t)L * R <= ctx->latency_items;
      rc = launch_batch(ctx, pit->second.dev, s.dev, s.y, s.plan, prm, lat_form ? DOCK_FORM_LATENCY : DOCK_FORM_BATCHED,
                        s.stream, &s.fork, err, true, latency);
      if (rc >= 0) note_use(ctx, pit->second, s.stream);
      if (rc >= 0 && lat_form) ctx->stats.latency_form_batches += 1;
      else if (rc >= 0 && latency) ctx->stats.latency_batches += 1;
      if (rc >= 0)
        e = cudaMemcpyAsync(s.host + s.y.out_begin(prm.outputs), s.dev + s.y.out_begin(prm.outputs),
                            s.y.out_end - s.y.out_begin(prm.outputs), cudaMemcpyDeviceToHost,
                            s.stream);
    }
    if (e == cudaSuccess && rc >= 0) e = cudaEventRecord(s.ev, s.stream);
    if (pit->second.closed && pit->second.queued == 0) {  // its last queued ligands are on their way
      release_pocket(ctx, pit->second);
      ctx->pockets.erase(pit);
    }
  } else if (e == cudaSuccess) {
    err = fmt("pocket %d was unloaded while work for it was queued", pocket);
    rc = DOCK_ERR_NOPOCKET;
  }
  if (e != cudaSuccess || rc < 0) {
    ctx->fatal = e != cudaSuccess ? cuda_status(e) : rc;
    ctx->fatal_msg = e != cudaSuccess ? fmt("serving batch: %s", cudaGetErrorString(e)) : err;
    s.members.clear();
    return false;
  }
  s.busy = true;
  s.t_launch = now_ns();
  ctx->stats.batches += 1;
  ctx->stats.h2d_bytes += s.y.in_end;
  ctx->stats.d2h_bytes += s.y.out_end - s.y.out_begin(prm.outputs);
  return true;
}

void serve_loop(dock_ctx* ctx) {
  cudaSetDevice(ctx->device);
  std::unique_lock<std::mutex> lk(ctx->mu);
  while (!ctx->stop) {
    bool progress = false, any_busy = false;
    for (Slot& s : ctx->slots) {
      if (!s.busy) continue;
      const cudaError_t q = cudaEventQuery(s.ev);
      if (q == cudaSuccess) {
        scatter_slot(ctx, s);
        progress = true;
      } else if (q != cudaErrorNotReady) {
        ctx->fatal = cuda_status(q);
        ctx->fatal_msg = fmt("serving batch failed: %s", cudaGetErrorString(q));
        s.members.clear();
        s.busy = false;
        progress = true;
      } else {
        any_busy = true;
        // watchdog: a batch that runs past the stall limit stops admission; its work is left to
        // finish (a kernel cannot be cancelled) and unfinished tickets report DOCK_ERR_TIMEOUT
        const int64_t ran_ms = (now_ns() - s.t_launch) / 1000000;
        if (!ctx->fatal && ran_ms > ctx->cfg.stall_timeout_ms) {
          ctx->fatal = DOCK_ERR_TIMEOUT;
          ctx->fatal_msg = fmt("serving batch of %zu ligands still running after %lld ms (stall_timeout_ms %d)",
                               s.members.size(), (long long)ran_ms, ctx->cfg.stall_timeout_ms);
          progress = true;
        }
      }
    }
    if (progress) ctx->done_cv.notify_all();
    if (!ctx->fatal)
      for (Slot& s : ctx->slots)
        if (!s.busy && admit(ctx, s, lk)) {
          progress = true;
          any_busy = true;
        }
    if (ctx->fatal) ctx->done_cv.notify_all();
    if (progress) continue;
    if (any_busy) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    } else {
      ctx->work_cv.wait_for(lk, std::chrono::milliseconds(50));
    }
  }
}

}  // namespace

// ================================================================================================
// C-ABI
// ================================================================================================

extern "C" {

int dock_create(const dock_config* cfg, dock_ctx** out) {
  if (!out) return DOCK_ERR_INVALID;
  *out = nullptr;
  auto ctx = std::make_unique<dock_ctx>();
  if (cfg) ctx->cfg = *cfg;
  dock_config& c = ctx->cfg;
  if (c.n_streams <= 0) c.n_streams = 4;
  if (c.hbm_budget_bytes == 0) c.hbm_budget_bytes = 8ull << 30;
  if (c.max_batch_ligands <= 0) c.max_batch_ligands = 4096;
  if (c.max_queued_ligands <= 0) c.max_queued_ligands = 4000000;
  if (c.stall_timeout_ms <= 0) c.stall_timeout_ms = 120000;
  if (c.n_streams > 64 || c.max_batch_ligands > (1 << 21)) return DOCK_ERR_INVALID;
  ctx->device = c.device;
  for (int b = 0; b < kNumBuckets; ++b) ctx->launch_cfg[b] = default_launch(b);
  cudaError_t e = cudaSetDevice(c.device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = ctx->fork.create();
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = ctx->capture_fork.create();
  ctx->slots.resize(c.n_streams);
  for (Slot& s : ctx->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = s.fork.create();
  }
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device);
  void* scratch = nullptr;  // loads the allocation-free entry point's fixed array now, not in a docking call
  if (e == cudaSuccess) e = noalloc_scratch_address(c.device, &scratch);
#ifdef DOCK_COUNT_WORK
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&ctx->exec), sizeof(unsigned long long) * kCnt);
  if (e == cudaSuccess) e = cudaMemset(ctx->exec, 0, sizeof(unsigned long long) * kCnt);
#endif
  if (e != cudaSuccess) {
    dock_destroy(ctx.release());
    return DOCK_ERR_CUDA;
  }
  ctx->latency_items = c.serve_latency_items < 0 ? 0 : c.serve_latency_items > 0 ? c.serve_latency_items : 2 * 4 * sms;
  ctx->latency_form_ligands = c.serve_latency_form < 0 ? 0 : c.serve_latency_form > 0 ? c.serve_latency_form : 1;
  if (!c.serve_off) ctx->server = std::thread(serve_loop, ctx.get());
  *out = ctx.release();
  return DOCK_OK;
}

int dock_destroy(dock_ctx* ctx) {
  if (!ctx) return DOCK_ERR_INVALID;
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->stop = true;
  }
  ctx->work_cv.notify_all();
  if (ctx->server.joinable()) ctx->server.join();
  cudaSetDevice(ctx->device);
  for (Slot& s : ctx->slots) {
    if (s.dev) cudaFreeAsync(s.dev, s.stream);  // stream-ordered, like its allocation
    if (s.stream) cudaStreamSynchronize(s.stream);
    if (s.host) cudaFreeHost(s.host);
    if (s.ev) cudaEventDestroy(s.ev);
    if (s.stream) cudaStreamDestroy(s.stream);
    s.fork.destroy();
  }
  if (ctx->stream) {
    for (auto& kv : ctx->pockets) release_pocket(ctx, kv.second);
    cudaStreamSynchronize(ctx->stream);
  }
  ctx->pockets.clear();
  for (cudaEvent_t e : ctx->spare_events) cudaEventDestroy(e);
  if (ctx->exec) cudaFree(ctx->exec);
  ctx->fork.destroy();
  ctx->capture_fork.destroy();
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return DOCK_OK;
}

const char* dock_last_error(dock_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

int dock_set_launch(dock_ctx* ctx, int32_t bucket, const dock_launch_shape* sh) {
  if (!ctx) return DOCK_ERR_INVALID;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (bucket < 0 || bucket >= kNumBuckets) return ctx->fail(DOCK_ERR_INVALID, fmt("bucket %d out of [0,4]", bucket));
  if (!sh) {
    ctx->launch_cfg[bucket] = default_launch(bucket);
    ++ctx->launch_version;
    return DOCK_OK;
  }
  const int g = sh->warps_per_item;
  if (g != 1 && g != 2 && g != 4 && g != 8) return ctx->fail(DOCK_ERR_INVALID, "warps_per_item must be 1, 2, 4 or 8");
  if (sh->warps_per_block < 1 || sh->warps_per_block > 8 || sh->warps_per_block % g)
    return ctx->fail(DOCK_ERR_INVALID,
                     fmt("warps_per_block %d must be in [1,8] and a multiple of warps_per_item", sh->warps_per_block));
  if (sh->smem_carveout_pct < -1 || sh->smem_carveout_pct > 100)
    return ctx->fail(DOCK_ERR_INVALID, fmt("smem_carveout_pct %d out of [-1,100]", sh->smem_carveout_pct));
  if (sh->persistent != 0 && sh->persistent != 1) return ctx->fail(DOCK_ERR_INVALID, "persistent must be 0 or 1");
  const int tile = sh->pose_tile <= 0 ? 1 : sh->pose_tile;
  if (tile != 1 && (tile != 2 || g > 2))
    return ctx->fail(DOCK_ERR_INVALID, "pose_tile must be 1, or 2 with 1 or 2 warps per item");
  ctx->launch_cfg[bucket] = LaunchCfg{sh->warps_per_block, sh->smem_carveout_pct, sh->persistent, bucket, g, tile};
  ++ctx->launch_version;
  return DOCK_OK;
}

int dock_get_launch(dock_ctx* ctx, int32_t bucket, dock_launch_shape* sh) {
  if (!ctx) return DOCK_ERR_INVALID;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (bucket < 0 || bucket >= kNumBuckets || !sh) return ctx->fail(DOCK_ERR_INVALID, "bad bucket or NULL shape");
  const LaunchCfg& c = ctx->launch_cfg[bucket];
  *sh = dock_launch_shape{c.warps_per_block, c.smem_carveout, c.persistent, c.warps_per_item, c.tile};
  return DOCK_OK;
}

int dock_get_stats(dock_ctx* ctx, dock_stats* out) {
  if (!ctx || !out) return DOCK_ERR_INVALID;
  std::lock_guard<std::mutex> lk(ctx->mu);
  *out = ctx->stats;
  return DOCK_OK;
}

int dock_load_pocket(dock_ctx* ctx, const dock_grid_desc* g, const float* host_values, int32_t* pocket_id) {
  if (!ctx) return DOCK_ERR_INVALID;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!g || !host_values || !pocket_id) return ctx->fail(DOCK_ERR_INVALID, "grid, values and pocket_id must be non-NULL");
  if (g->nx < 2 || g->ny < 2 || g->nz < 2) return ctx->fail(DOCK_ERR_INVALID, "grid dimensions must be >= 2");
  if (!(g->spacing > 0.f) || !std::isfinite(g->spacing)) return ctx->fail(DOCK_ERR_INVALID, "spacing must be > 0");
  if (g->dtype != DOCK_GRID_F32 && g->dtype != DOCK_GRID_F16 && g->dtype != DOCK_GRID_I16)
    return ctx->fail(DOCK_ERR_INVALID, "unknown grid dtype");
  const size_t nv = (size_t)g->nx * g->ny * g->nz;
  const size_t ncell = (size_t)(g->nx - 1) * (g->ny - 1) * (g->nz - 1) + 1;
  if (ncell > (size_t)0x7fffffff) return ctx->fail(DOCK_ERR_INVALID, "grid too large");
  for (size_t i = 0; i < nv; ++i)
    if (!std::isfinite(host_values[i])) return ctx->fail(DOCK_ERR_INVALID, fmt("grid value %zu not finite", i));
  const bool i16 = g->dtype == DOCK_GRID_I16;
  std::vector<int16_t> ints;
  if (i16) {
    ints.resize(nv);
    for (size_t i = 0; i < nv; ++i) {
      const float v = host_values[i];
      if (v != std::nearbyint(v) || v < -32768.f || v > 32767.f)
        return ctx->fail(DOCK_ERR_INVALID, fmt("integer grid value %zu (%g) is not an int16", i, (double)v));
      ints[i] = (int16_t)v;
    }
  }
  // box of nonzero voxels
  int lo[3] = {g->nx, g->ny, g->nz}, hi[3] = {-1, -1, -1};
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i)
        if (host_values[((size_t)k * g->ny + j) * g->nx + i] != 0.f) {
          const int q[3] = {i, j, k};
          for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], q[a]);
            hi[a] = std::max(hi[a], q[a]);
          }
        }
  const bool empty = hi[0] < 0;
  if (empty)
    for (int a = 0; a < 3; ++a) lo[a] = 0, hi[a] = -1;
  cudaSetDevice(ctx->device);
  float* tmp = nullptr;
  Pocket P;
  cudaError_t e = cudaSuccess;
  if (i16) {
    // int16 voxels, x fastest, read one at a time (no corner packing).  Only the box of nonzero
    // voxels is stored, with a border of zero voxels one wide, so a lookup clamps its voxel index
    // into [lo - 1, hi + 1] per axis instead of testing it: every voxel outside the box is zero.
    const int bx = hi[0] - lo[0] + 3, by = hi[1] - lo[1] + 3, bz = hi[2] - lo[2] + 3;
    std::vector<int16_t> box((size_t)bx * by * bz, 0);
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i)
          box[((size_t)(k - lo[2] + 1) * by + (j - lo[1] + 1)) * bx + (i - lo[0] + 1)] =
              ints[((size_t)k * g->ny + j) * g->nx + i];
    // stream-ordered, so that dock_unload_pocket can free it after its last use without a device sync
    e = cudaMallocAsync(&P.cells, box.size() * sizeof(int16_t), ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(P.cells, box.data(), box.size() * sizeof(int16_t), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  } else {
    e = cudaMallocAsync(reinterpret_cast<void**>(&tmp), nv * sizeof(float), ctx->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&P.cells, ncell * (g->dtype == DOCK_GRID_F16 ? 16 : 32), ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, host_values, nv * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = launch_pack_pocket(tmp, P.cells, g->nx, g->ny, g->nz, g->dtype == DOCK_GRID_F16, ctx->stream);
    if (tmp) cudaFreeAsync(tmp, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  }
  if (e != cudaSuccess) {
    if (P.cells) cudaFreeAsync(P.cells, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    return ctx->cuda_fail(e, "load pocket");
  }
  PocketDev& d = P.dev;
  d.cells = P.cells;
  d.nx = g->nx;
  d.ny = g->ny;
  d.nz = g->nz;
  d.dtype = g->dtype;
  d.spacing = g->spacing;
  d.inv_h = 1.0f / g->spacing;
  d.ox = g->origin[0];
  d.oy = g->origin[1];
  d.oz = g->origin[2];
  d.cx = g->origin[0] + g->spacing * (float)(g->nx - 1) * 0.5f;
  d.cy = g->origin[1] + g->spacing * (float)(g->ny - 1) * 0.5f;
  d.cz = g->origin[2] + g->spacing * (float)(g->nz - 1) * 0.5f;
  // trilinear grids: the box of nonzero voxels widened by one voxel and clipped to the grid
  // (lookups outside are 0); integer grid: the stored box with its zero border
  const int dim[3] = {g->nx, g->ny, g->nz};
  float blo[3], bhi[3];
  for (int a = 0; a < 3; ++a) {
    if (i16) {
      blo[a] = (float)(lo[a] - 1);
      bhi[a] = (float)(hi[a] + 1);
    } else if (empty) {  // all-zero grid: an empty box
      blo[a] = 1.f;
      bhi[a] = 0.f;
    } else {
      blo[a] = (float)std::max(0, lo[a] - 1);
      bhi[a] = (float)std::min(dim[a] - 1, hi[a] + 1);
    }
  }
  d.lox = blo[0];
  d.loy = blo[1];
  d.loz = blo[2];
  d.hix = bhi[0];
  d.hiy = bhi[1];
  d.hiz = bhi[2];
  const int id = ctx->next_pocket++;
  ctx->pockets[id] = P;
  *pocket_id = id;
  return DOCK_OK;
}

int dock_unload_pocket(dock_ctx* ctx, int32_t pocket_id) {
  if (!ctx) return DOCK_ERR_INVALID;
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->pockets.find(pocket_id);
  if (it == ctx->pockets.end() || it->second.closed)
    return ctx->fail(DOCK_ERR_NOPOCKET, fmt("unknown pocket %d", pocket_id));
  cudaSetDevice(ctx->device);
  // no device-wide wait and nothing blocks while the lock is held: ligands already submitted for
  // the pocket are still docked (the serving loop releases it after admitting the last of them),
  // and the memory is freed in stream order after the launches that read it (their recorded uses)
  it->second.closed = true;
  if (it->second.queued == 0) {
    release_pocket(ctx, it->second);
    ctx->pockets.erase(it);
  }
  return DOCK_OK;
}

int dock_validate_ligands(const dock_ligand_batch* lb, const dock_params* p, char* err, size_t err_len) {
  Packed pk;
  std::string msg;
  const bool ok = prepare(lb, p, pk, msg);
  if (err && err_len) {
    std::strncpy(err, ok ? "" : msg.c_str(), err_len - 1);
    err[err_len - 1] = 0;
  }
  return ok ? DOCK_OK : DOCK_ERR_INVALID;
}

int dock_submit_ligands(dock_ctx* ctx, int32_t pocket_id, const dock_ligand_batch* lb, const dock_params* p,
                        uint64_t* ticket) {
  if (!ctx) return DOCK_ERR_INVALID;
  if (!ticket) return ctx->fail(DOCK_ERR_INVALID, "ticket is NULL");
  if (ctx->cfg.serve_off) return ctx->fail(DOCK_ERR_INVALID, "context was created with serve_off");
  auto T = std::make_unique<Ticket>();
  T->t_submit = now_ns();
  std::string err;
  if (!prepare(lb, p, T->pk, err)) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    return ctx->fail(DOCK_ERR_INVALID, err);
  }
  const uint64_t prep_ns = (uint64_t)(now_ns() - T->t_submit);
  const int L = T->pk.n_lig;
  const int R = p->restarts;
  T->pocket = pocket_id;
  T->params = *p;
  T->score.assign(L, 0.f);
  T->best_restart.assign(L, -1);
  T->clash.assign(L, 0);
  T->xyz.assign(3 * (size_t)T->pk.atom_off[L], 0.f);
  T->full = p->outputs == DOCK_OUTPUT_FULL;
  if (T->full) {  // per-restart and per-bond outputs, kept only when asked for
    T->restart_score.assign((size_t)L * R, 0.f);
    T->restart_clash.assign((size_t)L * R, 0);
    T->align_idx.assign((size_t)L * R, 0);
    T->post_idx.assign((size_t)L * R, 0);
    T->tors_idx.assign((size_t)T->pk.rot_off[L] * R, 0);
    T->rejected.assign((size_t)T->pk.rot_off[L] * R, 0);
  }
  T->lat.assign(L, 0);
  T->K = params_dev(*p).K;
  T->select_restart.assign((size_t)L * T->K, -1);
  T->select_score.assign((size_t)L * T->K, 0.f);
  T->select_xyz.assign(3 * (size_t)T->pk.atom_off[L] * T->K, 0.f);
  std::lock_guard<std::mutex> lk(ctx->mu);
  Pocket* P = open_pocket(ctx, pocket_id);
  if (!P) return ctx->fail(DOCK_ERR_NOPOCKET, fmt("unknown pocket %d", pocket_id));
  if (ctx->queued + L > ctx->cfg.max_queued_ligands)
    return ctx->fail(DOCK_ERR_BUSY, fmt("queue full: %lld ligands waiting", (long long)ctx->queued));
  const uint64_t id = ctx->next_ticket++;
  T->id = id;
  ctx->queued += L;
  P->queued += L;
  ctx->stats.ligands_submitted += L;
  ctx->stats.prep_ns += prep_ns;
  if (L > 0) ctx->pending.push_back(id);
  ctx->tickets[id] = std::move(T);
  *ticket = id;
  ctx->work_cv.notify_all();
  return DOCK_OK;
}

int dock_poll(dock_ctx* ctx, uint64_t ticket, int32_t timeout_ms, dock_status* st) {
  if (!ctx) return DOCK_ERR_INVALID;
  std::unique_lock<std::mutex> lk(ctx->mu);
  auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms > 0 ? timeout_ms : 0);
  for (;;) {
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) return ctx->fail(DOCK_ERR_UNKNOWN_TICKET, fmt("unknown ticket %llu", (unsigned long long)ticket));
    Ticket& T = *it->second;
    if (st) {
      st->pending = T.n_done < T.pk.n_lig;
      st->n_done = T.n_done;
      st->n_total = T.pk.n_lig;
    }
    if (T.n_done == T.pk.n_lig) return DOCK_OK;
    if (ctx->fatal) return ctx->fail(ctx->fatal, ctx->fatal_msg);
    if (timeout_ms == 0) return DOCK_PENDING;
    if (timeout_ms > 0) {
      if (ctx->done_cv.wait_until(lk, deadline) == std::cv_status::timeout) {
        auto it2 = ctx->tickets.find(ticket);
        if (it2 != ctx->tickets.end() && it2->second->n_done == it2->second->pk.n_lig) continue;
        return DOCK_PENDING;
      }
    } else {
      ctx->done_cv.wait_for(lk, std::chrono::milliseconds(100));
    }
  }
}

int dock_results(dock_ctx* ctx, uint64_t ticket, dock_result_buffers* o) {
  if (!ctx) return DOCK_ERR_INVALID;
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->tickets.find(ticket);
  if (it == ctx->tickets.end()) return ctx->fail(DOCK_ERR_UNKNOWN_TICKET, fmt("unknown ticket %llu", (unsigned long long)ticket));
  if (!o) return ctx->fail(DOCK_ERR_INVALID, "result buffers are NULL");
  Ticket& T = *it->second;
  if (T.n_done < T.pk.n_lig) return DOCK_PENDING;
  if (!T.full && (o->restart_score || o->restart_clash || o->align_idx || o->post_idx || o->torsion_idx || o->rejected))
    return ctx->fail(DOCK_ERR_INVALID, "ticket submitted with DOCK_OUTPUT_BEST: per-restart outputs were not kept");
  const size_t L = T.pk.n_lig;
  auto cp = [](void* dst, const void* src, size_t bytes) {
    if (dst && bytes) std::memcpy(dst, src, bytes);
  };
  cp(o->score, T.score.data(), 4 * L);
  cp(o->best_restart, T.best_restart.data(), 4 * L);
  cp(o->xyz, T.xyz.data(), 4 * T.xyz.size());
  cp(o->clash_count, T.clash.data(), 4 * L);
  cp(o->restart_score, T.restart_score.data(), 4 * T.restart_score.size());
  cp(o->restart_clash, T.restart_clash.data(), 4 * T.restart_clash.size());
  cp(o->align_idx, T.align_idx.data(), 4 * T.align_idx.size());
  cp(o->post_idx, T.post_idx.data(), 4 * T.post_idx.size());
  cp(o->torsion_idx, T.tors_idx.data(), 4 * T.tors_idx.size());
  cp(o->rejected, T.rejected.data(), 4 * T.rejected.size());
  cp(o->latency_ns, T.lat.data(), 8 * L);
  cp(o->select_restart, T.select_restart.data(), 4 * T.select_restart.size());
  cp(o->select_score, T.select_score.data(), 4 * T.select_score.size());
  cp(o->select_xyz, T.select_xyz.data(), 4 * T.select_xyz.size());
  ctx->tickets.erase(it);
  return DOCK_OK;
}

int dock_batch_create(dock_ctx* ctx, const dock_ligand_batch* lb, const dock_params* p, dock_batch** out) {
  if (!ctx) return DOCK_ERR_INVALID;
  if (!out) return ctx->fail(DOCK_ERR_INVALID, "out is NULL");
  *out = nullptr;
  auto P = std::make_unique<Packed>();
  std::string err;
  const int64_t t0 = now_ns();
  if (!prepare(lb, p, *P, err)) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    return ctx->fail(DOCK_ERR_INVALID, err);
  }
  const uint64_t prep_ns = (uint64_t)(now_ns() - t0);
  auto b = std::make_unique<dock_batch>();
  b->n_lig = P->n_lig;
  b->params = *p;
  const int R = p->restarts;
  const uint64_t atoms = (uint64_t)P->atom_off.back();
  b->work.items = (uint64_t)P->n_lig * R;
  b->work.lookups_align = (uint64_t)R * (1 + p->post_align) * p->align_steps * p->align_steps * atoms;
  b->work.lookups_torsion = (uint64_t)R * p->torsion_steps * P->moving;
  b->work.lookups_final = (uint64_t)R * atoms;
  b->y = make_layout(P->n_lig, P->atom_off.back(), P->rot_off.back(), R, params_dev(*p).K,
                     latency_scratch_bytes(R, p->align_steps));
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  cudaError_t e = cudaMalloc(&b->dev, b->y.total);
  if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&b->host), b->y.out_end, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
  if (e == cudaSuccess) {
    std::vector<LigRef> refs(P->n_lig);
    for (int l = 0; l < P->n_lig; ++l) refs[l] = {P.get(), l};
    fill_inputs(b->host, b->y, refs, R, b->plan);
    e = cudaMemcpyAsync(b->dev, b->host, b->y.in_end, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->dev + b->y.done, 0, 4 * (size_t)P->n_lig, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  }
  if (e != cudaSuccess) {
    if (b->dev) cudaFree(b->dev);
    if (b->host) cudaFreeHost(b->host);
    if (b->ev) cudaEventDestroy(b->ev);
    return ctx->cuda_fail(e, "batch create");
  }
  ctx->stats.batches += 1;
  ctx->stats.h2d_bytes += b->y.in_end;
  ctx->stats.prep_ns += prep_ns;
  *out = b.release();
  return DOCK_OK;
}

int dock_batch_launch(dock_ctx* ctx, int32_t pocket_id, dock_batch* b, int32_t form, void* stream) {
  if (!ctx) return DOCK_ERR_INVALID;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!b) return ctx->fail(DOCK_ERR_INVALID, "batch is NULL");
  if (form != DOCK_FORM_BATCHED && form != DOCK_FORM_PER_LIGAND && form != DOCK_FORM_LATENCY)
    return ctx->fail(DOCK_ERR_INVALID, "unknown form");
  Pocket* P = open_pocket(ctx, pocket_id);
  if (!P) return ctx->fail(DOCK_ERR_NOPOCKET, fmt("unknown pocket %d", pocket_id));
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
  cudaSetDevice(ctx->device);
  std::string err;
  const bool graph = form == DOCK_FORM_BATCHED || (form == DOCK_FORM_LATENCY && b->n_lig <= kLatencyGraphLigands);
  const int rc = graph ? graph_launch(ctx, pocket_id, P->dev, b, s, err, form)
                       : launch_batch(ctx, P->dev, b->dev, b->y, b->plan, b->params, form, s, &ctx->fork, err);
  if (rc < 0) return ctx->fail(rc, err);
  const cudaError_t e = cudaEventRecord(b->ev, s);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "event record");
  b->launched = true;
  note_use(ctx, *P, s);
  return rc;
}

int dock_batch_results(dock_ctx* ctx, dock_batch* b, dock_result_buffers* o) {
  if (!ctx) return DOCK_ERR_INVALID;
  if (!b || !o) return ctx->fail(DOCK_ERR_INVALID, "batch and result buffers must be non-NULL");
  if (!b->launched) return ctx->fail(DOCK_ERR_INVALID, "batch was never launched");
  if (b->params.outputs == DOCK_OUTPUT_BEST &&
      (o->restart_score || o->restart_clash || o->align_idx || o->post_idx || o->torsion_idx || o->rejected))
    return ctx->fail(DOCK_ERR_INVALID, "batch created with DOCK_OUTPUT_BEST: per-restart outputs are not copied back");
  cudaSetDevice(ctx->device);
  const size_t o0 = b->y.out_begin(b->params.outputs);
  cudaError_t e = cudaEventSynchronize(b->ev);
  if (e == cudaSuccess) e = cudaMemcpy(b->host + o0, b->dev + o0, b->y.out_end - o0, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    return ctx->cuda_fail(e, "batch results");
  }
  copy_results(b->host, b->y, b->plan, b->params.restarts, o);
  if (o->latency_ns) std::memset(o->latency_ns, 0, 8 * (size_t)b->n_lig);
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->stats.d2h_bytes += b->y.out_end - b->y.out_begin(b->params.outputs);
  ctx->stats.ligands_done += b->n_lig;
  return DOCK_OK;
}

int dock_exec_counters(dock_ctx* ctx, dock_exec_work* out, int32_t reset) {
  if (!ctx) return DOCK_ERR_INVALID;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!out) return ctx->fail(DOCK_ERR_INVALID, "out is NULL");
  if (!ctx->exec)
    return ctx->fail(DOCK_ERR_INVALID, "this library was built without work counters (libdock_count.so has them)");
  static_assert(sizeof(dock_exec_work) == sizeof(unsigned long long) * kCnt, "dock_exec_work layout");
  cudaSetDevice(ctx->device);
  cudaError_t e = cudaMemcpyAsync(out, ctx->exec, sizeof(dock_exec_work), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess && reset) e = cudaMemsetAsync(ctx->exec, 0, sizeof(dock_exec_work), ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "read work counters");
  return DOCK_OK;
}

int dock_batch_work(const dock_batch* b, dock_work* out) {
  if (!b || !out) return DOCK_ERR_INVALID;
  *out = b->work;
  return DOCK_OK;
}

int dock_batch_wait(dock_ctx* ctx, dock_batch* b) {
  if (!ctx) return DOCK_ERR_INVALID;
  if (!b) return ctx->fail(DOCK_ERR_INVALID, "batch is NULL");
  if (!b->launched) return DOCK_OK;
  cudaSetDevice(ctx->device);
  const cudaError_t e = cudaEventSynchronize(b->ev);
  if (e != cudaSuccess) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    return ctx->cuda_fail(e, "batch wait");
  }
  return DOCK_OK;
}

int dock_batch_destroy(dock_ctx* ctx, dock_batch* b) {
  if (!ctx || !b) return DOCK_ERR_INVALID;
  cudaSetDevice(ctx->device);
  if (b->launched) cudaEventSynchronize(b->ev);
  for (cudaGraphExec_t g : b->gexec)
    if (g) cudaGraphExecDestroy(g);
  cudaFree(b->dev);
  cudaFreeHost(b->host);
  cudaEventDestroy(b->ev);
  delete b;
  return DOCK_OK;
}

}  // extern "C"

// ---- internal view for the allocation-free entry point (dock_noalloc.cu) ---------------------------

namespace dockgpu {

int with_batch_view(dock_ctx* ctx, int pocket_id, const dock_batch* b, void* stream,
                    const std::function<int(const BatchView&, cudaStream_t)>& launch) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!b) return ctx->fail(DOCK_ERR_INVALID, "batch is NULL");
  Pocket* P = open_pocket(ctx, pocket_id);
  if (!P) return ctx->fail(DOCK_ERR_NOPOCKET, fmt("unknown pocket %d", pocket_id));
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "set device");
  BatchView view;
  BatchView* v = &view;
  v->pocket = P->dev;
  v->inputs = batch_pointers(b->dev, b->y, b->n_lig);
  v->params = params_dev(b->params);
  v->params.exec = ctx->exec;
  for (int k = 0; k < kNumBuckets; ++k) {
    v->cfg[k] = ctx->launch_cfg[k];
    v->n_items[k] = b->plan.n_items[k];
    v->item_off[k] = b->plan.item_off[k];
  }
  v->items = reinterpret_cast<const uint32_t*>(b->dev + b->y.items);
  v->n_lig = b->n_lig;
  v->atoms = (size_t)b->plan.atoms;
  v->rots = (size_t)b->plan.rots;
  v->device = ctx->device;
  v->ctx_stream = ctx->stream;
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
  const int rc = launch(view, s);
  // recorded even when a later launch of the call failed: the earlier ones may be running.  The
  // batch is logically const for the caller; its completion event is bookkeeping
  dock_batch* mb = const_cast<dock_batch*>(b);
  e = cudaEventRecord(mb->ev, s);
  if (e == cudaSuccess) mb->launched = true;
  note_use(ctx, *P, s);
  if (rc < 0) return rc;
  if (e != cudaSuccess) return ctx->cuda_fail(e, "event record");
  return rc;
}

int record_error_locked(dock_ctx* ctx, int code, const char* msg) { return ctx->fail(code, msg); }

int record_error(dock_ctx* ctx, int code, const char* msg) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  return ctx->fail(code, msg);
}

int pocket_view(dock_ctx* ctx, int pocket_id, PocketDev* pk, cudaStream_t* stream) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  Pocket* P = open_pocket(ctx, pocket_id);
  if (!P) return ctx->fail(DOCK_ERR_NOPOCKET, fmt("unknown pocket %d", pocket_id));
  const cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "set device");
  *pk = P->dev;
  *stream = ctx->stream;
  return DOCK_OK;
}

}  // namespace dockgpu
