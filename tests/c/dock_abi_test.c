/*
 * dock_abi_test.c - a plain C11 client of include/dock.h (test infrastructure).
 *
 * Compiled against the public header alone and linked with libdock.so, it checks the boundary the
 * way a C caller sees it:
 *   dock_abi_test layout            prints sizeof and offsetof of every struct of the C-ABI, one
 *                                   "struct.field offset size" line each, for comparison with the
 *                                   Python binding's ctypes mirrors (no GPU needed);
 *   dock_abi_test dock IN OUT       docks one batch through dock_create, dock_load_pocket,
 *                                   dock_submit_ligands, dock_poll and dock_results, reading the
 *                                   pocket, parameters and ligands from IN and writing every result
 *                                   array to OUT (little-endian, the layout below).
 *
 * IN:  i32 nx ny nz dtype; f32 spacing ox oy oz; f32 values[nx*ny*nz];
 *      i32 restarts align_steps torsion_steps post_align early_exit select_k outputs;
 *      f32 clash_dist select_rmsd; u64 seed;
 *      i32 n_lig; i32 atom_off[n+1]; f32 xyz[3*atoms]; i32 bond_off[n+1]; i32 bonds[2*bonds];
 *      i32 rot_off[n+1]; i32 rot[2*rot]; u64 ids[n]
 * OUT: f32 score[n]; i32 best_restart[n]; f32 xyz[3*atoms]; i32 clash_count[n];
 *      f32 restart_score[n*R]; i32 restart_clash[n*R] align_idx[n*R] post_idx[n*R];
 *      i32 torsion_idx[rot*R] rejected[rot*R]
 * Exit status 0 on success; a failing call prints its status and dock_last_error.
 */
#include <stddef.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "dock.h"

#define FIELD(T, f) printf("%s.%s %zu %zu\n", #T, #f, offsetof(T, f), sizeof(((T*)0)->f))
#define SIZE(T) printf("%s %zu %zu\n", #T, (size_t)0, sizeof(T))

static int layout(void) {
  SIZE(dock_config);
  FIELD(dock_config, device); FIELD(dock_config, n_streams); FIELD(dock_config, hbm_budget_bytes);
  FIELD(dock_config, max_batch_ligands); FIELD(dock_config, max_queued_ligands); FIELD(dock_config, serve_off);
  FIELD(dock_config, stall_timeout_ms); FIELD(dock_config, serve_latency_items);
  FIELD(dock_config, serve_latency_form); FIELD(dock_config, reserved);
  SIZE(dock_grid_desc);
  FIELD(dock_grid_desc, nx); FIELD(dock_grid_desc, ny); FIELD(dock_grid_desc, nz); FIELD(dock_grid_desc, spacing);
  FIELD(dock_grid_desc, origin); FIELD(dock_grid_desc, dtype);
  SIZE(dock_params);
  FIELD(dock_params, restarts); FIELD(dock_params, align_steps); FIELD(dock_params, torsion_steps);
  FIELD(dock_params, clash_dist); FIELD(dock_params, post_align); FIELD(dock_params, early_exit);
  FIELD(dock_params, seed); FIELD(dock_params, select_k); FIELD(dock_params, select_rmsd);
  FIELD(dock_params, outputs);
  SIZE(dock_ligand_batch);
  FIELD(dock_ligand_batch, n_lig); FIELD(dock_ligand_batch, atom_off); FIELD(dock_ligand_batch, xyz);
  FIELD(dock_ligand_batch, bond_off); FIELD(dock_ligand_batch, bonds); FIELD(dock_ligand_batch, rot_off);
  FIELD(dock_ligand_batch, rot_bonds); FIELD(dock_ligand_batch, ids);
  SIZE(dock_result_buffers);
  FIELD(dock_result_buffers, score); FIELD(dock_result_buffers, best_restart); FIELD(dock_result_buffers, xyz);
  FIELD(dock_result_buffers, clash_count); FIELD(dock_result_buffers, restart_score);
  FIELD(dock_result_buffers, restart_clash); FIELD(dock_result_buffers, align_idx);
  FIELD(dock_result_buffers, post_idx); FIELD(dock_result_buffers, torsion_idx); FIELD(dock_result_buffers, rejected);
  FIELD(dock_result_buffers, latency_ns); FIELD(dock_result_buffers, select_restart);
  FIELD(dock_result_buffers, select_score); FIELD(dock_result_buffers, select_xyz);
  SIZE(dock_status);
  FIELD(dock_status, pending); FIELD(dock_status, n_done); FIELD(dock_status, n_total);
  SIZE(dock_stats);
  FIELD(dock_stats, ligands_submitted); FIELD(dock_stats, ligands_done); FIELD(dock_stats, batches);
  FIELD(dock_stats, kernel_launches); FIELD(dock_stats, h2d_bytes); FIELD(dock_stats, d2h_bytes);
  FIELD(dock_stats, graph_launches); FIELD(dock_stats, prep_ns); FIELD(dock_stats, fill_ns);
  FIELD(dock_stats, scatter_ns); FIELD(dock_stats, latency_batches); FIELD(dock_stats, slot_grows);
  FIELD(dock_stats, slot_grow_ns); FIELD(dock_stats, latency_form_batches);
  SIZE(dock_launch_shape);
  FIELD(dock_launch_shape, warps_per_block); FIELD(dock_launch_shape, smem_carveout_pct);
  FIELD(dock_launch_shape, persistent); FIELD(dock_launch_shape, warps_per_item);
  FIELD(dock_launch_shape, pose_tile);
  SIZE(dock_work);
  FIELD(dock_work, items); FIELD(dock_work, lookups_align); FIELD(dock_work, lookups_torsion);
  FIELD(dock_work, lookups_final);
  SIZE(dock_exec_work);
  FIELD(dock_exec_work, items); FIELD(dock_exec_work, align_poses); FIELD(dock_exec_work, torsion_angles);
  FIELD(dock_exec_work, angles_accepted); FIELD(dock_exec_work, lookups); FIELD(dock_exec_work, loads);
  FIELD(dock_exec_work, sectors); FIELD(dock_exec_work, pair_tests); FIELD(dock_exec_work, lines);
  SIZE(dock_device_results);
  FIELD(dock_device_results, score); FIELD(dock_device_results, best_restart); FIELD(dock_device_results, xyz);
  FIELD(dock_device_results, clash_count); FIELD(dock_device_results, restart_score);
  FIELD(dock_device_results, restart_clash); FIELD(dock_device_results, align_idx);
  FIELD(dock_device_results, post_idx); FIELD(dock_device_results, torsion_idx);
  FIELD(dock_device_results, rejected);
  return 0;
}

static void* read_n(FILE* f, size_t elem, size_t n) {
  void* p = malloc(elem * (n ? n : 1));
  if (!p || fread(p, elem, n, f) != n) {
    fprintf(stderr, "short read\n");
    exit(2);
  }
  return p;
}

static int32_t read_i32(FILE* f) {
  int32_t v;
  if (fread(&v, 4, 1, f) != 1) exit(2);
  return v;
}

static float read_f32(FILE* f) {
  float v;
  if (fread(&v, 4, 1, f) != 1) exit(2);
  return v;
}

static int check(dock_ctx* ctx, int rc, const char* what) {
  if (rc < 0) {
    fprintf(stderr, "%s failed with %d: %s\n", what, rc, ctx ? dock_last_error(ctx) : "");
    exit(3);
  }
  return rc;
}

static int dock(const char* in_path, const char* out_path) {
  FILE* f = fopen(in_path, "rb");
  if (!f) return 2;
  dock_grid_desc g;
  g.nx = read_i32(f);
  g.ny = read_i32(f);
  g.nz = read_i32(f);
  g.dtype = read_i32(f);
  g.spacing = read_f32(f);
  for (int a = 0; a < 3; ++a) g.origin[a] = read_f32(f);
  float* values = read_n(f, 4, (size_t)g.nx * g.ny * g.nz);
  dock_params p;
  memset(&p, 0, sizeof p);
  p.restarts = read_i32(f);
  p.align_steps = read_i32(f);
  p.torsion_steps = read_i32(f);
  p.post_align = read_i32(f);
  p.early_exit = read_i32(f);
  p.select_k = read_i32(f);
  p.outputs = read_i32(f);
  p.clash_dist = read_f32(f);
  p.select_rmsd = read_f32(f);
  if (fread(&p.seed, 8, 1, f) != 1) return 2;
  dock_ligand_batch lb;
  lb.n_lig = read_i32(f);
  const size_t n = (size_t)lb.n_lig;
  int32_t* atom_off = read_n(f, 4, n + 1);
  float* xyz = read_n(f, 4, 3 * (size_t)atom_off[n]);
  int32_t* bond_off = read_n(f, 4, n + 1);
  int32_t* bonds = read_n(f, 4, 2 * (size_t)bond_off[n]);
  int32_t* rot_off = read_n(f, 4, n + 1);
  int32_t* rot = read_n(f, 4, 2 * (size_t)rot_off[n]);
  uint64_t* ids = read_n(f, 8, n);
  fclose(f);
  lb.atom_off = atom_off;
  lb.xyz = xyz;
  lb.bond_off = bond_off;
  lb.bonds = bonds;
  lb.rot_off = rot_off;
  lb.rot_bonds = rot;
  lb.ids = ids;

  dock_config cfg;
  memset(&cfg, 0, sizeof cfg);  /* every zero field takes its default */
  dock_ctx* ctx = NULL;
  check(NULL, dock_create(&cfg, &ctx), "dock_create");
  int32_t pocket = -1;
  check(ctx, dock_load_pocket(ctx, &g, values, &pocket), "dock_load_pocket");
  uint64_t ticket = 0;
  check(ctx, dock_submit_ligands(ctx, pocket, &lb, &p, &ticket), "dock_submit_ligands");
  dock_status st;
  int rc;
  while ((rc = check(ctx, dock_poll(ctx, ticket, 1000, &st), "dock_poll")) == DOCK_PENDING) {
  }
  if (st.pending || st.n_done != lb.n_lig || st.n_total != lb.n_lig) {
    fprintf(stderr, "dock_poll status %d %d %d\n", st.pending, st.n_done, st.n_total);
    return 4;
  }
  const size_t R = (size_t)p.restarts, atoms = (size_t)atom_off[n], nrot = (size_t)rot_off[n];
  dock_result_buffers o;
  memset(&o, 0, sizeof o);
  o.score = calloc(n + 1, 4);
  o.best_restart = calloc(n + 1, 4);
  o.xyz = calloc(3 * atoms + 1, 4);
  o.clash_count = calloc(n + 1, 4);
  o.restart_score = calloc(n * R + 1, 4);
  o.restart_clash = calloc(n * R + 1, 4);
  o.align_idx = calloc(n * R + 1, 4);
  o.post_idx = calloc(n * R + 1, 4);
  o.torsion_idx = calloc(nrot * R + 1, 4);
  o.rejected = calloc(nrot * R + 1, 4);
  check(ctx, dock_results(ctx, ticket, &o), "dock_results");
  FILE* w = fopen(out_path, "wb");
  if (!w) return 2;
  fwrite(o.score, 4, n, w);
  fwrite(o.best_restart, 4, n, w);
  fwrite(o.xyz, 4, 3 * atoms, w);
  fwrite(o.clash_count, 4, n, w);
  fwrite(o.restart_score, 4, n * R, w);
  fwrite(o.restart_clash, 4, n * R, w);
  fwrite(o.align_idx, 4, n * R, w);
  fwrite(o.post_idx, 4, n * R, w);
  fwrite(o.torsion_idx, 4, nrot * R, w);
  fwrite(o.rejected, 4, nrot * R, w);
  fclose(w);
  check(ctx, dock_unload_pocket(ctx, pocket), "dock_unload_pocket");
  check(ctx, dock_destroy(ctx), "dock_destroy");
  return 0;
}

int main(int argc, char** argv) {
  if (argc == 2 && strcmp(argv[1], "layout") == 0) return layout();
  if (argc == 4 && strcmp(argv[1], "dock") == 0) return dock(argv[2], argv[3]);
  fprintf(stderr, "usage: %s layout | dock IN OUT\n", argv[0]);
  return 1;
}
