/*
 * dock.h - C-ABI of the GB300 geometric docking library (libdock.so).
 *
 * The library docks ligands into a pocket with the method of Vitali et al., "GPU-optimized
 * Approaches to Molecular Docking-based Virtual Screening in Drug Discovery" (arXiv 2209.05069),
 * Alg. 1: for each of N restarts a starting pose, a rigid alignment over a grid of x/y rotation
 * angles, a sequential sweep of every rotatable bond through a set of torsion angles with an
 * intra-ligand bump check, an optional second rigid alignment, and the final pose score; the
 * best restart is reported.  As in Alg. 1's problem statement (Section 4), a pocket and each
 * ligand's initial pose go in and the scores of the poses evaluated come out.
 * The asynchronous submit / poll / results shape follows the batched design of Section 4.2, where
 * host threads push ligands and the GPU consumes them in batches.
 *
 * Conventions
 *  - Every call returns an int status: DOCK_OK (0), DOCK_PENDING (1), or a negative DOCK_ERR_*.
 *    No call throws across the ABI.  dock_last_error() gives a one-line message for the last
 *    failing call on the context (ligand index and field for validation errors).
 *  - Host pointers are only read during the call (inputs are copied before return) unless stated.
 *  - All device memory is owned by the context; callers never free library memory.
 *  - A context is bound to one CUDA device.  All calls on one context are thread-safe.
 *  - Geometry on the device is FP32; no FP64 runs on the device.
 */
#ifndef DOCK_H
#define DOCK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------------ */
#define DOCK_OK 0
#define DOCK_PENDING 1               /* work not finished yet (dock_poll, dock_results) */
#define DOCK_ERR_INVALID (-1)        /* bad argument or ligand; see dock_last_error */
#define DOCK_ERR_NOMEM (-2)          /* device or pinned allocation failed, or over budget */
#define DOCK_ERR_BUSY (-3)           /* admission queue full; retry after polling */
#define DOCK_ERR_NOPOCKET (-4)       /* unknown pocket id */
#define DOCK_ERR_UNKNOWN_TICKET (-5) /* ticket never issued or already released */
#define DOCK_ERR_TIMEOUT (-6)        /* dock_poll timed out, or the serving loop stalled */
#define DOCK_ERR_CUDA (-7)           /* a CUDA call failed; the message names it */

/* ---- limits -------------------------------------------------------------------------------- */
#define DOCK_MAX_ATOMS 160           /* largest ligand (Section 4.2 buckets end at 160 atoms) */
#define DOCK_MAX_ROT 64              /* rotatable bonds per ligand */
#define DOCK_MAX_BONDS 512           /* bonds per ligand */
#define DOCK_MAX_RESTARTS 1024
#define DOCK_MAX_ALIGN_STEPS 128     /* rigid-alignment angles per axis */
#define DOCK_MAX_TORSION_STEPS 1024  /* angles per rotatable bond */

typedef struct dock_ctx dock_ctx;

/* Context configuration.  Zero fields take the stated defaults. */
typedef struct {
  int32_t device;             /* CUDA device ordinal */
  int32_t n_streams;          /* streams the serving loop spreads batches over (default 4) */
  uint64_t hbm_budget_bytes;  /* device bytes in-flight ligand state may hold (default 8 GiB) */
  int32_t max_batch_ligands;  /* most ligands one serving launch takes (default 4096) */
  int32_t max_queued_ligands; /* most ligands waiting for admission before submit says BUSY
                                 (default 4,000,000) */
  int32_t serve_off;          /* 1: no serving thread (only the dock_batch_* calls work) */
  int32_t stall_timeout_ms;   /* a serving batch still running after this long puts the context in
                                 the stalled state: nothing more is admitted and dock_poll returns
                                 DOCK_ERR_TIMEOUT for unfinished tickets (default 120000) */
  int32_t serve_latency_items; /* serving batches of at most this many ligand-restarts run with the
                                 latency-oriented launch shape (8 warps per ligand-restart, one per
                                 block, not persistent), larger ones with the dock_set_launch shapes:
                                 a small batch then finishes sooner, a large one keeps the
                                 throughput shape.  0: twice the items 8-warp blocks fill the GPU
                                 with at once (4 blocks per SM); -1: never */
  int32_t serve_latency_form; /* serving batches of at most this many ligands are docked in the
                                 latency form (DOCK_FORM_LATENCY: one ligand at a time over the whole
                                 GPU), which finishes a lone ligand soonest.  0: 1 ligand; -1: never */
  int32_t reserved;
} dock_config;

/* Pocket grid (Section 4.1: a read-only 3-D field indexed by atom x, y, z).  Voxel (i, j, k)
 * sits at origin + spacing * (i, j, k); host_values[(k*ny + j)*nx + i] (x fastest). */
#define DOCK_GRID_F32 0
#define DOCK_GRID_F16 1              /* stored as FP16 on the device (values rounded to nearest) */
#define DOCK_GRID_I16 2              /* integer grid (Section 5.5: the score sums integer values):
                                        host values must be integers in [-32768, 32767], stored as
                                        int16; an atom reads its nearest voxel, index
                                        floor((x - origin) / spacing + 1/2) per axis (half-way reads
                                        the upper voxel), 0 outside the grid.  Scores are exact
                                        integers (held in float) */
typedef struct {
  int32_t nx, ny, nz;         /* each >= 2 */
  float spacing;              /* > 0, Angstrom */
  float origin[3];
  int32_t dtype;              /* DOCK_GRID_F32, DOCK_GRID_F16 or DOCK_GRID_I16 */
} dock_grid_desc;

/* Docking parameters (Alg. 1). */
typedef struct {
  int32_t restarts;           /* N starting poses (Alg. 1 outer loop), >= 1 */
  int32_t align_steps;        /* rigid-alignment angles per axis: 360/align_steps degree steps
                                 (Alg. 1 uses 12 degrees, i.e. 30) */
  int32_t torsion_steps;      /* angles per rotatable bond: 360/torsion_steps degree steps */
  float clash_dist;           /* bump threshold d_c (Angstrom): a pair closer than d_c bumps */
  int32_t post_align;         /* 1: repeat the rigid alignment after the torsion sweep */
  int32_t early_exit;         /* 1: stop testing an angle's pairs at its first bump and skip
                                 scoring rejected angles (results are identical either way) */
  uint64_t seed;              /* keys the restart orientations together with the ligand id */
  int32_t select_k;           /* Select Poses (Alg. 1, after the restart loop): keep up to this many restart poses
                                 per ligand (<= 0 means 1, at most 16 and at most restarts) */
  float select_rmsd;          /* ... accepting a pose (in order of final score, ties: lowest restart)
                                 only if its RMSD to every pose already kept is >= this (Angstrom) */
  int32_t outputs;            /* DOCK_OUTPUT_FULL (0): every output of dock_result_buffers is kept;
                                 DOCK_OUTPUT_BEST (1): only the per-ligand ones (score, best restart,
                                 pose, clash count, Select Poses, latency) are copied back and kept,
                                 and asking dock_results / dock_batch_results for a per-restart or
                                 per-bond output is an error */
} dock_params;

#define DOCK_OUTPUT_FULL 0
#define DOCK_OUTPUT_BEST 1

/* A batch of ligands in CSR form (host memory).  Atom, bond and rotatable-bond indices are local
 * to their ligand.  Rotatable bond (a, b) must be a bond whose removal splits the ligand; the
 * side holding b is the one its torsion moves. */
typedef struct {
  int32_t n_lig;
  const int32_t* atom_off;    /* [n_lig+1], non-decreasing, atom_off[0] = 0 */
  const float* xyz;           /* [atom_off[n_lig]*3]: x, y, z of each atom */
  const int32_t* bond_off;    /* [n_lig+1] */
  const int32_t* bonds;       /* [bond_off[n_lig]*2] */
  const int32_t* rot_off;     /* [n_lig+1] */
  const int32_t* rot_bonds;   /* [rot_off[n_lig]*2] as (a, b) */
  const uint64_t* ids;        /* [n_lig] ligand ids (key the restart orientations) */
} dock_ligand_batch;

/* Caller-allocated result buffers (host memory).  R = restarts.  NULL optional fields are
 * skipped.  Per-bond arrays of ligand l hold restart r, bond b at (rot_off[l]*R + r*B_l + b). */
typedef struct {
  float* score;               /* [n_lig] best final score over the restarts */
  int32_t* best_restart;      /* [n_lig] restart with that score (ties: lowest index) */
  float* xyz;                 /* [atom_off[n_lig]*3] final pose of the best restart */
  int32_t* clash_count;       /* [n_lig] pairs > 2 bonds apart closer than d_c, best pose */
  float* restart_score;       /* [n_lig*R] optional */
  int32_t* restart_clash;     /* [n_lig*R] optional */
  int32_t* align_idx;         /* [n_lig*R] optional: chosen alignment i*align_steps + j */
  int32_t* post_idx;          /* [n_lig*R] optional: post-optimisation alignment, -1 if off */
  int32_t* torsion_idx;       /* [rot_off[n_lig]*R] optional: chosen torsion angle index */
  int32_t* rejected;          /* [rot_off[n_lig]*R] optional: angles rejected by the bump check */
  int64_t* latency_ns;        /* [n_lig] optional: submit -> completion seen by the host */
  int32_t* select_restart;    /* [n_lig*K] optional: restarts kept by Select Poses, -1 past the end */
  float* select_score;        /* [n_lig*K] optional: their final scores */
  float* select_xyz;          /* [atom_off[n_lig]*K*3] optional: their poses; ligand l, pose k at
                                 (atom_off[l]*K + k*n_l)*3 */
} dock_result_buffers;

typedef struct {
  int32_t pending;            /* 1 while any ligand of the ticket is unfinished */
  int32_t n_done;
  int32_t n_total;
} dock_status;

/* ---- context ------------------------------------------------------------------------------ */

/* Creates a context on cfg->device (NULL cfg: all defaults).  Errors: DOCK_ERR_INVALID,
 * DOCK_ERR_CUDA. */
int dock_create(const dock_config* cfg, dock_ctx** out);

/* Stops the serving loop, waits for launched work, frees all device and pinned memory. */
int dock_destroy(dock_ctx* ctx);

/* One-line description of the last error on ctx ("" if none).  Valid until the next call. */
const char* dock_last_error(dock_ctx* ctx);

/* Cumulative counters of a context since dock_create (metrics; Section 5 reports throughput). */
typedef struct {
  uint64_t ligands_submitted;  /* through dock_submit_ligands */
  uint64_t ligands_done;       /* results ready, serving loop and batches */
  uint64_t batches;            /* batches uploaded (serving batches and dock_batch_create) */
  uint64_t kernel_launches;    /* docking kernel launches queued */
  uint64_t h2d_bytes;          /* ligand input bytes copied host -> device */
  uint64_t d2h_bytes;          /* result bytes copied device -> host */
  uint64_t graph_launches;     /* batched launches replayed from a captured CUDA graph */
  uint64_t prep_ns;            /* host time validating and packing ligands (submit, batch create) */
  uint64_t fill_ns;            /* serving loop: host time writing batches into pinned staging */
  uint64_t scatter_ns;         /* serving loop: host time copying finished batches to tickets */
  uint64_t latency_batches;    /* serving batches launched with the latency-oriented shape */
  uint64_t slot_grows;         /* serving loop: times a stream slot's buffers had to grow */
  uint64_t slot_grow_ns;       /* and the host time those reallocations took */
  uint64_t latency_form_batches; /* serving batches docked in the latency form */
} dock_stats;

/* Copies the context's counters into *out. */
int dock_get_stats(dock_ctx* ctx, dock_stats* out);

/* Launch shape of the docking kernel for one atom bucket (0: <=32 atoms, 1: <=64, 2: <=96,
 * 3: <=128, 4: <=160).  Results do not depend on the launch shape (tested bit for bit). */
typedef struct {
  int32_t warps_per_block;    /* 1..8 (default 8) */
  int32_t smem_carveout_pct;  /* preferred shared-memory share of the SM's L1/shared capacity,
                                 percent; -1 = driver default.  A lower share leaves more L1 cache
                                 for pocket lookups and fewer resident blocks. */
  int32_t persistent;         /* 1: the grid holds only the blocks the GPU runs at once and each
                                 item group pulls ligand-restarts from a counter until the bucket is
                                 done (default); 0: one item group per ligand-restart */
  int32_t warps_per_item;     /* warps that dock one ligand-restart together: 1, 2 (default), 4 or
                                 8, dividing warps_per_block.  More warps per item shorten each
                                 ligand's time on the GPU (the latency-oriented shape) */
  int32_t pose_tile;          /* alignment poses, and torsion angles, one lane scores per pass: 1
                                 (default; 0 means 1) or 2 (with 1 or 2 warps per item): each atom is
                                 read once for both and two lookup chains are in flight */
} dock_launch_shape;

/* Sets the launch shape of one bucket; applies to launches queued after the call.  shape == NULL
 * restores the bucket's default.  Error: DOCK_ERR_INVALID. */
int dock_set_launch(dock_ctx* ctx, int32_t bucket, const dock_launch_shape* shape);

/* Reads the launch shape of one bucket.  Error: DOCK_ERR_INVALID. */
int dock_get_launch(dock_ctx* ctx, int32_t bucket, dock_launch_shape* shape);

/* ---- pocket -------------------------------------------------------------------------------- */

/* Uploads a pocket grid (Section 4.1: the pocket is shared read-only by all ligands) and builds
 * its device layout; the grid stays resident until dock_unload_pocket.  The caller keeps
 * host_values.  Errors: DOCK_ERR_INVALID (a dimension < 2, spacing <= 0, unknown dtype, a value
 * not finite, or for DOCK_GRID_I16 not an integer in [-32768, 32767]), DOCK_ERR_NOMEM,
 * DOCK_ERR_CUDA. */
int dock_load_pocket(dock_ctx* ctx, const dock_grid_desc* grid, const float* host_values, int32_t* pocket_id);

/* Unloads a pocket: later calls naming it get DOCK_ERR_NOPOCKET.  Returns at once.  Ligands already
 * submitted for it are still docked (the serving loop keeps the pocket until it has admitted the last
 * of them), and its device memory is freed in stream order once every launch that reads it (serving
 * batches, dock_batch_launch, dock_batch_launch_noalloc) has finished: work in flight completes
 * normally and nothing else on the context or the device waits.  Error: DOCK_ERR_NOPOCKET. */
int dock_unload_pocket(dock_ctx* ctx, int32_t pocket_id);

/* ---- validation (host only, no context or GPU needed) -------------------------------------- */

/* Runs the checks dock_submit_ligands applies to ligands and params, without docking.  Returns
 * DOCK_OK or DOCK_ERR_INVALID; on error writes a one-line message (ligand index and field) into
 * err (may be NULL) truncated to err_len bytes including the terminator. */
int dock_validate_ligands(const dock_ligand_batch* ligands, const dock_params* params, char* err, size_t err_len);

/* ---- asynchronous docking (serving) -------------------------------------------------------- */

/* Queues a batch of ligands for docking into pocket_id and returns at once with a ticket.
 * The inputs are validated and copied before return (each ligand: 1 <= atoms <= 160, bonds
 * <= 512 within range, rotatable bonds <= 64 and each a bridge of the bond graph).  The serving
 * loop admits queued ligands as device memory (hbm_budget_bytes) frees up, packs them with other
 * tickets' ligands into batches and overlaps batches on several streams.  Results do not depend
 * on which ligands share a batch.  Errors: DOCK_ERR_INVALID (message names ligand and field),
 * DOCK_ERR_NOPOCKET, DOCK_ERR_BUSY (queue full), DOCK_ERR_NOMEM. */
int dock_submit_ligands(dock_ctx* ctx, int32_t pocket_id, const dock_ligand_batch* ligands,
                        const dock_params* params, uint64_t* ticket);

/* Waits up to timeout_ms (0: do not wait, < 0: wait without limit) for a ticket.  Returns
 * DOCK_OK when every ligand is done, DOCK_PENDING otherwise; st (may be NULL) gets progress.
 * Errors: DOCK_ERR_UNKNOWN_TICKET, DOCK_ERR_TIMEOUT (the serving loop reported a stall),
 * DOCK_ERR_CUDA. */
int dock_poll(dock_ctx* ctx, uint64_t ticket, int32_t timeout_ms, dock_status* st);

/* Copies a finished ticket's results into caller buffers sized for the submitted batch and
 * releases the ticket.  Returns DOCK_PENDING (nothing copied, ticket kept) if unfinished.
 * Errors: DOCK_ERR_UNKNOWN_TICKET. */
int dock_results(dock_ctx* ctx, uint64_t ticket, dock_result_buffers* out);

/* ---- device-resident batches (one launch over inputs already in device memory) ------------- */

typedef struct dock_batch dock_batch;

#define DOCK_FORM_BATCHED 0      /* bucketed batched launches, one warp per ligand-restart */
#define DOCK_FORM_PER_LIGAND 1   /* one launch per ligand (the plain per-ligand form) */
#define DOCK_FORM_LATENCY 2      /* the latency form (Section 4.1): one ligand at a time spread over
                                    the whole GPU; each ligand's R x N^2 alignment poses are dealt to
                                    every SM (one pass of 32 poses per warp), the best pose of each
                                    restart is reduced exactly (highest score, lowest index) by the
                                    last of its blocks to finish, which then runs the restart's
                                    torsion sweep with all angles of a bond in flight; the
                                    post-alignment and final scoring follow the same way.  Results
                                    equal the batched form's bit for bit */

/* Validates and packs ligands for params into device memory owned by ctx (synchronous upload).
 * Errors as dock_submit_ligands, plus DOCK_ERR_NOMEM. */
int dock_batch_create(dock_ctx* ctx, const dock_ligand_batch* ligands, const dock_params* params,
                      dock_batch** out);

/* Docks a prepared batch into pocket_id on `stream` (a cudaStream_t; NULL = the context's own
 * stream).  Inputs and results stay in device memory; the call returns once the work is queued.
 * `form` selects DOCK_FORM_BATCHED or DOCK_FORM_PER_LIGAND.  The batched form's launch sequence
 * (one kernel per non-empty atom bucket, forked across streams and joined) is captured into a CUDA
 * graph on its first launch and replayed afterwards; it is captured again when the pocket or the
 * launch shapes (dock_set_launch) change.  DOCK_FORM_LATENCY queues two kernels per ligand, from a
 * CUDA graph captured the same way for batches of up to 256 ligands and directly for larger ones.
 * Returns the number of kernel launches queued (>= 0) or
 * an error: DOCK_ERR_NOPOCKET, DOCK_ERR_INVALID, DOCK_ERR_CUDA. */
int dock_batch_launch(dock_ctx* ctx, int32_t pocket_id, dock_batch* batch, int32_t form, void* stream);

/* Waits until the batch's last launched work has finished (no copy). */
int dock_batch_wait(dock_ctx* ctx, dock_batch* batch);

/* Waits for the batch's launched work and copies its results to caller host buffers. */
int dock_batch_results(dock_ctx* ctx, dock_batch* batch, dock_result_buffers* out);

/* Algorithmic work of one launch of a prepared batch: the pocket lookups (trilinear
 * interpolations) the method performs, counted with every torsion angle scored. */
typedef struct {
  uint64_t items;            /* (ligand, restart) work items */
  uint64_t lookups_align;    /* rigid alignment: (1 + post_align) * align_steps^2 * atoms per item */
  uint64_t lookups_torsion;  /* torsion sweep: torsion_steps * (moving atoms - 1) per bond per item */
  uint64_t lookups_final;    /* final pose score: atoms per item */
} dock_work;

int dock_batch_work(const dock_batch* batch, dock_work* out);

/* Work the docking kernels actually executed (measurement; no counterpart in the paper).  Only the
 * counter build of the library (libdock_count.so, the same sources compiled with DOCK_COUNT_WORK)
 * counts; its kernels add these totals over every launch of the context.  Early exit and the
 * skipped loads outside the pocket's nonzero box make them differ from dock_work's algorithmic
 * counts.  Lane-level counts include idle lanes of a last partial pass. */
typedef struct {
  uint64_t items;            /* ligand-restarts docked */
  uint64_t align_poses;      /* alignment pose lanes evaluated (both alignments) */
  uint64_t torsion_angles;   /* torsion angle lanes of the scoring passes run */
  uint64_t angles_accepted;  /* of those, angles the bump check accepted (the ones Alg. 1 scores) */
  uint64_t lookups;          /* pocket lookups evaluated */
  uint64_t loads;            /* of those, lookups that issued a global load (inside the stored box) */
  uint64_t sectors;          /* distinct 32-byte sectors those loads read, counted per warp-wide load */
  uint64_t pair_tests;       /* bump-check distance tests evaluated (angle lanes x pairs) */
  uint64_t lines;            /* distinct 128-byte lines those loads read, counted per warp-wide load */
} dock_exec_work;

/* Copies the counters into *out (waits for the context's stream; call after the launches to count
 * have finished, e.g. after dock_batch_wait) and zeroes them if reset != 0.  Error:
 * DOCK_ERR_INVALID (NULL, or a library built without counters). */
int dock_exec_counters(dock_ctx* ctx, dock_exec_work* out, int32_t reset);

/* ---- allocation-free launch ----------------------------------------------------------------
 *
 * The paper has no counterpart to this call; it exists for callers that cannot allocate device
 * memory at the time they dock: a process whose device memory is owned by another allocator (a
 * framework's caching pool holding the GPU), a latency-critical loop that must not pay for
 * cudaMalloc/cudaFree (both can synchronize the whole device), or code under a policy that forbids
 * allocation after start-up.  It docks a prepared batch like dock_batch_launch(DOCK_FORM_BATCHED),
 * with results written to device buffers the caller owns, and calls no cudaMalloc, cudaFree or
 * other allocating routine.  The kernel's scratch (each restart's final pose and each ligand's
 * count of finished restarts) lives in one fixed array of DOCK_NOALLOC_SCRATCH_BYTES inside the
 * library, which every GPU that loads the library holds until the process exits.
 *
 * When memory is taken: the first dock_create on a device looks up the array's device address,
 * which loads it, so its DOCK_NOALLOC_SCRATCH_BYTES are taken then, not in a docking call.  With
 * CUDA's lazy module loading (the default) the first launch of each docking kernel in a process also
 * loads that kernel's code; a caller that must not allocate at docking time docks one batch of
 * the same shape at set-up (through either launch call) or runs with CUDA_MODULE_LOADING=EAGER.
 *
 * A batch fits if 256-byte-rounded (4 * ligands) + 12 * atoms * restarts <= that size; larger
 * batches are rejected with DOCK_ERR_INVALID and nothing runs.  Select Poses (select_k > 1) is not
 * part of this call: only the outputs of dock_device_results are written; a caller wanting
 * several poses per ligand selects them from the per-restart scores itself or uses
 * dock_batch_launch.  Every call, from every context of the process, shares the one array and it
 * keeps the last call's contents: the call clears the counters it needs on `stream` before its
 * kernels, and calls whose work overlaps on the GPU (different streams, or another context) race
 * on the array, so order them on one stream or wait between them.  The call records the batch's
 * completion event on `stream`, so dock_batch_wait and dock_batch_destroy wait for its work. */
#define DOCK_NOALLOC_SCRATCH_BYTES (16u << 20)

/* Caller-owned device buffers for dock_batch_launch_noalloc, laid out like dock_result_buffers;
 * every pointer is required. */
typedef struct {
  float* score;               /* [n_lig] */
  int32_t* best_restart;      /* [n_lig] */
  float* xyz;                 /* [atom_off[n_lig]*3] */
  int32_t* clash_count;       /* [n_lig] */
  float* restart_score;       /* [n_lig*R] */
  int32_t* restart_clash;     /* [n_lig*R] */
  int32_t* align_idx;         /* [n_lig*R] */
  int32_t* post_idx;          /* [n_lig*R] */
  int32_t* torsion_idx;       /* [rot_off[n_lig]*R] */
  int32_t* rejected;          /* [rot_off[n_lig]*R] */
} dock_device_results;

/* Queues the batch's kernels on `stream` (a cudaStream_t; NULL = the context's stream) and returns
 * the number of kernel launches (>= 0) once queued.  Results are in `out` when the stream reaches
 * that point.  Errors: DOCK_ERR_INVALID (NULL argument, batch over the scratch size),
 * DOCK_ERR_NOPOCKET, DOCK_ERR_CUDA. */
int dock_batch_launch_noalloc(dock_ctx* ctx, int32_t pocket_id, const dock_batch* batch,
                              const dock_device_results* out, void* stream);

/* Frees a prepared batch (waits for its launched work first). */
int dock_batch_destroy(dock_ctx* ctx, dock_batch* batch);

/* ---- measurement (no counterpart in the paper) ------------------------------------------------ */

/* Measures the rate of scattered pocket lookups on this GPU, the roof of the docking kernel: the
 * same trilinear (or nearest-voxel) lookup code on the same device layout of pocket `pocket_id`, at
 * independent uniformly random positions inside the pocket's nonzero box, with no other work.
 * Runs four launches of a few milliseconds each on the context's stream, synchronously, and
 * allocates a few KB of device memory.  *lookups_per_s receives the best of three timed runs.  Errors:
 * DOCK_ERR_INVALID (NULL), DOCK_ERR_NOPOCKET, DOCK_ERR_CUDA. */
int dock_gather_peak(dock_ctx* ctx, int32_t pocket_id, double* lookups_per_s);

#ifdef __cplusplus
}
#endif

#endif /* DOCK_H */
