// FP64 reference implementation of the geometric docking hot path (arXiv 2209.05069, Alg. 1).
//
// TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library is checked against.
// Only the tests, the smoke check and the CPU-baseline leg of the benchmark may load it; the
// product library never links, loads or calls it, and it shares no code with the CUDA path.
//
// Plain, slow and literal: double precision everywhere, one ligand at a time, no blocking, no
// precomputed tables, every pair and every angle evaluated in the order the method states.
//
// Readings of points the paper leaves open (each is also pinned by a test in tests/):
//  * Score (Alg. 1 Evaluate_Score / Score; pocket grid indexed by atom x, y, z, Section 4.1):
//    the sum over all atoms of the trilinear interpolation of the pocket grid.  Per axis
//    u = (x - origin)/h; an atom with u < 0 or u > G-1 on any axis contributes 0;
//    i0 = min(floor(u), G-2), t = u - i0.
//  * Objective: maximise (Section 4 keeps the angle with the highest score).
//  * Starting pose (Alg. 1 Generate_Starting_Pose, not defined in the paper): the centroid is
//    moved to the pocket centre (the grid's geometric centre); restart 0 keeps the input
//    orientation, restart r >= 1 is rotated by Shoemake's uniform random quaternion (Graphics
//    Gems III, 1992) built from three counter-based SplitMix64 draws (Steele, Lea and Flood,
//    OOPSLA 2014) keyed by the ligand id and the seed.
//  * Rigid alignment (Alg. 1, the two rotation loops): angles 0, 360/N, ..., 360(N-1)/N on each axis
//    (0 to 360 step 12 is 30 angles: 360 equals 0).  Pose (i, j) = c + Ry(beta_j) Rx(alpha_i)
//    (P - c), c the centroid of the current pose, evaluated directly (not by incremental steps).
//    Best pose = highest score, ties to the lowest flat index i*N + j.
//  * Torsion sweep (Alg. 1, the fragment loop): rotatable bonds in input order; bond (a, b) moves the
//    side M_b that holds b once the bond is cut; theta_k = 2 pi k / A for k in [0, A) about the
//    axis a -> b through b (right-handed, Rodrigues), relative to the current conformation.
//  * Bump check (Alg. 1 CheckBump, Section 5.5): an angle is rejected when some moving atom
//    i in M_b \ {b} and fixed atom j in F_b \ {a} have |x_i - x_j|^2 < d_c^2; every other pair
//    keeps its distance under the torsion.  The chosen angle is the best-scoring accepted one,
//    ties to the lowest k; with no accepted angle the conformation is kept (k = 0).
//  * After the torsion sweep the rigid alignment is repeated on the optimised pose (flag
//    post_align), then the final pose is scored.  Best restart = highest final score, ties to
//    the lowest restart index.  Final clash count = atom pairs more than two bonds apart with
//    |x_i - x_j|^2 < d_c^2.
//  * Integer grid (Section 5.5 remarks that the score sums integer values; the mapping from a
//    position to a value is not given): in mode 1 an atom reads the value of its nearest voxel,
//    per axis i = floor(u + 1/2) (a position half-way between two voxels reads the upper one), and
//    contributes 0 when i < 0 or i > G-1 on any axis.  Scores are sums of integers, so every
//    ordering of the sum gives the same value; what FP32 can change is which voxel an atom near a
//    half-way plane reads.  Each score therefore also carries the range of values it takes when
//    every coordinate moves by up to eps_voxel grid units, and each decision reports whether it is
//    the only possible one over those ranges (robust) and whether a forced choice is a possible
//    one (possible).
//  * Select Poses (Alg. 1, after the restart loop; the paper names the step but gives neither the
//    number of poses kept nor the similarity test): restarts in order of final score (ties to the
//    lowest restart) are kept greedily when the RMSD of their pose to every pose already kept is
//    at least a threshold, until K are kept.  RMSD = sqrt(mean over atoms of |x_i - y_i|^2) between
//    the two poses of the same ligand in the pocket frame (no superposition).  K and the threshold
//    are parameters; K = 1 keeps the best restart alone.
//
// Pins (tests/test_oracle_pins.py, tests/test_oracle_mutants.py): each step above is pinned by a
// closed form, an invariant, a library routine or brute force.  The whole docking of a ligand
// (oracle_dock_ligand) has no published worked example to compare with (the paper's numbers are all in
// figures): end to end it is "parity unpinned" beyond those component pins.
//
// Besides the results, every decision reports its margin (score gap, distance to the clash
// threshold) so a caller can tell decisions that FP32 rounding cannot flip from those it can.
// A caller may also force the decisions (replay): the oracle then follows the given choices and
// reports how each compares with the best choice available in double precision.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>

namespace {

const double kPi = 3.14159265358979323846264338327950288;
const double kInf = std::numeric_limits<double>::infinity();

struct Grid {
  int dim[3];
  double h;
  double origin[3];
  const double* v;  // v[(k*ny + j)*nx + i]
  int mode = 0;     // 0: trilinear interpolation, 1: nearest voxel (integer grid)
  double eps = 0;   // mode 1: coordinate uncertainty, grid units, for the score ranges
};

struct V3 {
  double x, y, z;
};
V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }

struct M3 {
  double m[3][3];
};
V3 mul(const M3& R, V3 a) {
  return {R.m[0][0] * a.x + R.m[0][1] * a.y + R.m[0][2] * a.z,
          R.m[1][0] * a.x + R.m[1][1] * a.y + R.m[1][2] * a.z,
          R.m[2][0] * a.x + R.m[2][1] * a.y + R.m[2][2] * a.z};
}
M3 mul(const M3& A, const M3& B) {
  M3 C;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      C.m[i][j] = 0;
      for (int k = 0; k < 3; ++k) C.m[i][j] += A.m[i][k] * B.m[k][j];
    }
  return C;
}

// ---- score: sum of trilinear grid lookups ---------------------------------------------------

double trilinear(const Grid& g, V3 p) {
  const double x[3] = {p.x, p.y, p.z};
  int i0[3];
  double t[3];
  for (int a = 0; a < 3; ++a) {
    const double u = (x[a] - g.origin[a]) / g.h;
    if (!(u >= 0.0 && u <= (double)(g.dim[a] - 1))) return 0.0;
    int i = (int)std::floor(u);
    if (i > g.dim[a] - 2) i = g.dim[a] - 2;
    i0[a] = i;
    t[a] = u - (double)i;
  }
  double s = 0.0;
  for (int dk = 0; dk < 2; ++dk)
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) {
        const double w = (di ? t[0] : 1.0 - t[0]) * (dj ? t[1] : 1.0 - t[1]) * (dk ? t[2] : 1.0 - t[2]);
        const size_t idx = ((size_t)(i0[2] + dk) * g.dim[1] + (size_t)(i0[1] + dj)) * g.dim[0] + (i0[0] + di);
        s += w * g.v[idx];
      }
  return s;
}

// Nearest-voxel value at p (mode 1) and its range over positions within eps grid units per axis.
struct Sc {
  double s, lo, hi;
};

Sc nearest(const Grid& g, V3 p) {
  const double x[3] = {p.x, p.y, p.z};
  int nom[3], first[3], last[3];
  for (int a = 0; a < 3; ++a) {
    const double u = (x[a] - g.origin[a]) / g.h;
    nom[a] = (int)std::floor(u + 0.5);
    first[a] = (int)std::floor(u - g.eps + 0.5);
    last[a] = (int)std::floor(u + g.eps + 0.5);
  }
  auto value = [&](const int* q) {
    for (int a = 0; a < 3; ++a)
      if (q[a] < 0 || q[a] > g.dim[a] - 1) return 0.0;
    return g.v[((size_t)q[2] * g.dim[1] + (size_t)q[1]) * g.dim[0] + q[0]];
  };
  Sc r = {value(nom), kInf, -kInf};
  int q[3];
  for (q[2] = first[2]; q[2] <= last[2]; ++q[2])
    for (q[1] = first[1]; q[1] <= last[1]; ++q[1])
      for (q[0] = first[0]; q[0] <= last[0]; ++q[0]) {
        const double v = value(q);
        r.lo = std::min(r.lo, v);
        r.hi = std::max(r.hi, v);
      }
  return r;
}

// Score of a pose with its range (mode 0: lo = hi = s).
Sc score_range(const Grid& g, const std::vector<V3>& P) {
  Sc r = {0, 0, 0};
  for (const V3& p : P) {
    if (g.mode == 1) {
      const Sc a = nearest(g, p);
      r.s += a.s;
      r.lo += a.lo;
      r.hi += a.hi;
    } else {
      const double t = trilinear(g, p);
      r.s += t;
      r.lo += t;
      r.hi += t;
    }
  }
  return r;
}

double score(const Grid& g, const std::vector<V3>& P) {
  if (g.mode == 1) return score_range(g, P).s;
  double s = 0.0;
  for (const V3& p : P) s += trilinear(g, p);
  return s;
}

// Over score ranges: choice c is the only possible argmax (ties to the lowest index) when its
// lowest value beats every other candidate's highest (strictly for lower indices); it is a
// possible argmax when its highest value reaches every other candidate's lowest (strictly for
// lower indices).  cand[j] = 0 leaves j out.
bool only_possible(const std::vector<Sc>& r, const std::vector<char>& cand, int c) {
  for (int j = 0; j < (int)r.size(); ++j) {
    if (j == c || !cand[j]) continue;
    if (j < c ? !(r[c].lo > r[j].hi) : !(r[c].lo >= r[j].hi)) return false;
  }
  return true;
}
bool possible(const std::vector<Sc>& r, const std::vector<char>& cand, int c) {
  for (int j = 0; j < (int)r.size(); ++j) {
    if (j == c || !cand[j]) continue;
    if (j < c ? !(r[c].hi > r[j].lo) : !(r[c].hi >= r[j].lo)) return false;
  }
  return true;
}

V3 centroid(const std::vector<V3>& P) {
  V3 c = {0, 0, 0};
  for (const V3& p : P) c = c + p;
  return (1.0 / (double)P.size()) * c;
}

// ---- rotations -------------------------------------------------------------------------------

M3 rot_x(double a) {
  const double c = std::cos(a), s = std::sin(a);
  return {{{1, 0, 0}, {0, c, -s}, {0, s, c}}};
}
M3 rot_y(double b) {
  const double c = std::cos(b), s = std::sin(b);
  return {{{c, 0, s}, {0, 1, 0}, {-s, 0, c}}};
}

// Rodrigues: rotate v by angle th about the unit axis u (right-handed).
V3 rodrigues(V3 v, V3 u, double th) {
  const double c = std::cos(th), s = std::sin(th);
  return c * v + s * cross(u, v) + ((1.0 - c) * dot(u, v)) * u;
}

// SplitMix64 output number `k` (k >= 1) of the generator started from `state`.
uint64_t splitmix64(uint64_t state, uint64_t k) {
  uint64_t z = state + k * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Restart r's starting orientation: identity for r = 0, else Shoemake's uniform quaternion from
// u_t = top 24 bits of draw (3r + t + 1) of a SplitMix64 stream whose start is the first draw of
// the SplitMix64 stream started at seed ^ id (hashing the key keeps the streams of neighbouring
// ligand ids from overlapping).
M3 restart_rotation(uint64_t id, uint64_t seed, int r) {
  if (r == 0) return {{{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}};
  const uint64_t key = splitmix64(seed ^ id, 1);
  double u[3];
  for (int t = 0; t < 3; ++t)
    u[t] = (double)(splitmix64(key, (uint64_t)(3 * r + t + 1)) >> 40) * (1.0 / 16777216.0);
  const double a = std::sqrt(1.0 - u[0]), b = std::sqrt(u[0]);
  const double qx = a * std::sin(2 * kPi * u[1]), qy = a * std::cos(2 * kPi * u[1]);
  const double qz = b * std::sin(2 * kPi * u[2]), qw = b * std::cos(2 * kPi * u[2]);
  M3 R = {{{1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)},
           {2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)},
           {2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)}}};
  return R;
}

// ---- ligand graph ------------------------------------------------------------------------------

struct Graph {
  int n;
  std::vector<std::vector<int>> adj;
};

int build_graph(int n, int nb, const int32_t* bonds, Graph& G) {
  G.n = n;
  G.adj.assign(n, {});
  for (int e = 0; e < nb; ++e) {
    const int a = bonds[2 * e], b = bonds[2 * e + 1];
    if (a < 0 || b < 0 || a >= n || b >= n || a == b) return -1;
    G.adj[a].push_back(b);
    G.adj[b].push_back(a);
  }
  return 0;
}

// Moving side of bond (a, b): atoms reachable from b without crossing the edge a-b.
// Returns -1 if (a, b) is not a bond, -2 if the bond is not a bridge (a reachable from b).
int moving_set(const Graph& G, int a, int b, std::vector<char>& in_m) {
  if (a < 0 || b < 0 || a >= G.n || b >= G.n) return -1;
  if (std::find(G.adj[a].begin(), G.adj[a].end(), b) == G.adj[a].end()) return -1;
  in_m.assign(G.n, 0);
  std::vector<int> stack = {b};
  in_m[b] = 1;
  while (!stack.empty()) {
    const int x = stack.back();
    stack.pop_back();
    for (int y : G.adj[x]) {
      if (x == b && y == a) continue;  // the cut edge
      if (!in_m[y]) {
        in_m[y] = 1;
        stack.push_back(y);
      }
    }
  }
  return in_m[a] ? -2 : 0;
}

// Graph distance capped at 3 (0 = same atom, 1 = bonded, 2 = 1-3, 3 = farther).
std::vector<std::vector<int>> graph_dist3(const Graph& G) {
  std::vector<std::vector<int>> d(G.n, std::vector<int>(G.n, 3));
  for (int s = 0; s < G.n; ++s) {
    d[s][s] = 0;
    for (int x : G.adj[s]) {
      if (d[s][x] > 1) d[s][x] = 1;
      for (int y : G.adj[x])
        if (d[s][y] > 2) d[s][y] = 2;
    }
  }
  return d;
}

int clash_count(const std::vector<V3>& P, const std::vector<std::vector<int>>& gd, double dc,
                double* min_margin) {
  int c = 0;
  double mm = kInf;
  for (size_t i = 0; i < P.size(); ++i)
    for (size_t j = i + 1; j < P.size(); ++j) {
      if (gd[i][j] < 3) continue;
      const V3 d = P[i] - P[j];
      const double d2 = dot(d, d);
      if (d2 < dc * dc) ++c;
      mm = std::min(mm, std::fabs(std::sqrt(d2) - dc));
    }
  if (min_margin) *min_margin = mm;
  return c;
}

// ---- alignment ---------------------------------------------------------------------------------

std::vector<V3> align_pose(const std::vector<V3>& P, V3 c, int N, int i, int j) {
  const M3 R = mul(rot_y(2 * kPi * j / N), rot_x(2 * kPi * i / N));
  std::vector<V3> Q(P.size());
  for (size_t a = 0; a < P.size(); ++a) Q[a] = c + mul(R, P[a] - c);
  return Q;
}

struct AlignOut {
  int chosen;
  double best, second, forced_score;
  int robust = -1, possible = -1;  // mode 1 only (see only_possible / possible)
};

// Scores all N*N poses; chooses the best (or `forced` when >= 0) and moves P there.
AlignOut align(const Grid& g, std::vector<V3>& P, int N, int forced) {
  const V3 c = centroid(P);
  AlignOut o = {-1, -kInf, -kInf, -kInf};
  std::vector<double> s(N * N);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      s[i * N + j] = score(g, align_pose(P, c, N, i, j));
      if (s[i * N + j] > o.best) {
        o.second = o.best;
        o.best = s[i * N + j];
        o.chosen = i * N + j;
      } else if (s[i * N + j] > o.second) {
        o.second = s[i * N + j];
      }
    }
  if (g.mode == 1) {
    std::vector<Sc> r(N * N);
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) r[i * N + j] = score_range(g, align_pose(P, c, N, i, j));
    const std::vector<char> all(N * N, 1);
    o.robust = only_possible(r, all, o.chosen);
    o.possible = possible(r, all, forced >= 0 ? forced : o.chosen);
  }
  if (forced >= 0) {
    o.chosen = forced;
    o.forced_score = s[forced];
  }
  P = align_pose(P, c, N, o.chosen / N, o.chosen % N);
  return o;
}

// ---- torsion -------------------------------------------------------------------------------------

std::vector<V3> torsion_pose(const std::vector<V3>& P, const std::vector<char>& in_m, int a, int b, double th) {
  const V3 axis = P[b] - P[a];
  const V3 u = (1.0 / std::sqrt(dot(axis, axis))) * axis;
  std::vector<V3> Q = P;
  for (size_t i = 0; i < P.size(); ++i)
    if (in_m[i]) Q[i] = P[b] + rodrigues(P[i] - P[b], u, th);
  return Q;
}

struct TorsionOut {
  int chosen;
  int rejected;          // angles with a bump
  int n_ambiguous;       // angles whose worst pair lies within eps_clash of the threshold
  int robust_valid;      // angles accepted with every pair farther than d_c + eps_clash
  double best, second;   // best and second-best accepted scores
  double best_robust;    // best score among robustly accepted angles
  double forced_score;   // score of the forced angle
  double forced_margin;  // min over checked pairs of (d - d_c) at the forced angle
  double max_margin;     // max over angles of that min
  int robust = -1;       // mode 1: no angle on the bump threshold and the choice is the only possible one
  int possible = -1;     // mode 1: the forced (else chosen) angle is a possible choice
};

TorsionOut torsion(const Grid& g, std::vector<V3>& P, const Graph& G, int a, int b, int A, double dc,
                   double eps_clash, int forced, int* err) {
  std::vector<char> in_m;
  *err = moving_set(G, a, b, in_m);
  TorsionOut o = {0, 0, 0, 0, -kInf, -kInf, -kInf, -kInf, kInf, -kInf};
  if (*err) return o;
  int chosen = -1;
  std::vector<Sc> range(A);
  // no bump / every pair beyond d_c + eps_clash / no pair below d_c - eps_clash
  std::vector<char> accepted(A, 0), clear(A, 0), not_clearly_bumping(A, 0);
  for (int k = 0; k < A; ++k) {
    const std::vector<V3> Q = torsion_pose(P, in_m, a, b, 2 * kPi * k / A);
    bool bump = false;
    double margin = kInf;  // min over checked pairs of (d - d_c)
    for (int i = 0; i < G.n; ++i) {
      if (!in_m[i] || i == b) continue;
      for (int j = 0; j < G.n; ++j) {
        if (in_m[j] || j == a) continue;
        const V3 d = Q[i] - Q[j];
        const double d2 = dot(d, d);
        if (d2 < dc * dc) bump = true;
        margin = std::min(margin, std::sqrt(d2) - dc);
      }
    }
    const double s = score(g, Q);
    if (g.mode == 1) range[k] = score_range(g, Q);
    accepted[k] = !bump;
    clear[k] = margin > eps_clash;
    not_clearly_bumping[k] = margin >= -eps_clash;
    o.max_margin = std::max(o.max_margin, margin);
    if (std::fabs(margin) <= eps_clash) ++o.n_ambiguous;
    if (k == forced) {
      o.forced_score = s;
      o.forced_margin = margin;
    }
    if (bump) {
      ++o.rejected;
      continue;
    }
    if (margin > eps_clash) {
      ++o.robust_valid;
      o.best_robust = std::max(o.best_robust, s);
    }
    if (s > o.best) {
      o.second = o.best;
      o.best = s;
      chosen = k;
    } else if (s > o.second) {
      o.second = s;
    }
  }
  if (g.mode == 1) {
    // with no angle on the bump threshold the accepted set is certain
    o.robust = o.n_ambiguous == 0 && (chosen < 0 || only_possible(range, accepted, chosen));
    const int f = forced >= 0 ? forced : (chosen >= 0 ? chosen : 0);
    if (o.robust_valid == 0)  // every angle bumps or sits on the threshold
      o.possible = f == 0 || not_clearly_bumping[f];
    else
      o.possible = not_clearly_bumping[f] && possible(range, clear, f);
  }
  o.chosen = forced >= 0 ? forced : (chosen >= 0 ? chosen : 0);
  P = torsion_pose(P, in_m, a, b, 2 * kPi * o.chosen / A);
  return o;
}

}  // namespace

// ================================================================================================
// C API (called through ctypes by oracle/oracle.py)
// ================================================================================================

extern "C" {

struct oracle_grid {
  int32_t nx, ny, nz;
  double spacing;
  double origin[3];
  const double* values;  // x fastest
  int32_t mode;          // 0: trilinear, 1: nearest voxel (integer grid)
};

struct oracle_params {
  int32_t restarts;
  int32_t align_steps;    // N: angles per axis
  int32_t torsion_steps;  // A: angles per rotatable bond
  int32_t post_align;
  double clash_dist;
  uint64_t seed;
  double eps_clash;  // A: distance to the threshold below which a clash decision is ambiguous
  double eps_voxel;  // grid units: coordinate uncertainty behind the mode-1 score ranges
};

// Per-ligand outputs, caller-allocated.  R = restarts, B = rotatable bonds, n = atoms.
struct oracle_out {
  double* best_score;       // [1]
  int32_t* best_restart;    // [1]
  double* restart_score;    // [R]
  int32_t* align_idx;       // [R]   flat i*N + j of the first alignment
  int32_t* post_idx;        // [R]   flat index of the post-optimisation alignment (-1 if off)
  int32_t* torsion_idx;     // [R*B] chosen k per bond
  int32_t* rejected;        // [R*B] angles rejected by the bump check
  int32_t* clash;           // [R]   final-pose clash count
  double* restart_xyz;      // [R*n*3] final pose of every restart
  // decision margins
  double* align_best;       // [R] best and second-best alignment scores
  double* align_second;     // [R]
  double* align_forced;     // [R] score of the forced alignment (replay)
  double* post_best;        // [R]
  double* post_second;      // [R]
  double* post_forced;      // [R]
  double* tors_best;        // [R*B] best / second accepted score
  double* tors_second;      // [R*B]
  double* tors_best_robust; // [R*B]
  double* tors_forced;      // [R*B] score of the forced angle
  double* tors_forced_margin;  // [R*B]
  double* tors_max_margin;     // [R*B]
  int32_t* tors_ambiguous;     // [R*B]
  int32_t* tors_robust_valid;  // [R*B]
  double* clash_margin;        // [R] min |d - d_c| over final-pose pairs counted for clashes
  // mode 1 (integer grid) only; -1 in mode 0
  int32_t* align_robust;       // [R] the alignment chosen is the only possible one
  int32_t* align_possible;     // [R] the forced alignment is a possible one
  int32_t* post_robust;        // [R]
  int32_t* post_possible;      // [R]
  int32_t* tors_robust;        // [R*B]
  int32_t* tors_possible;      // [R*B]
  double* score_lo;            // [R] range of the final score (both = the score in mode 0)
  double* score_hi;            // [R]
};

// Error codes: -1 bad bond index, -2 rotatable bond is not a bridge, -3 bad sizes.
int oracle_dock_ligand(const oracle_grid* gd, int32_t n, const float* xyz, int32_t nb, const int32_t* bonds,
                       int32_t nrot, const int32_t* rot, uint64_t id, const oracle_params* p,
                       const int32_t* forced_align, const int32_t* forced_post, const int32_t* forced_tors,
                       oracle_out* out) {
  if (n < 1 || nb < 0 || nrot < 0 || p->restarts < 1 || p->align_steps < 1 || p->torsion_steps < 1) return -3;
  if (gd->nx < 2 || gd->ny < 2 || gd->nz < 2 || !(gd->spacing > 0)) return -3;
  const Grid g = {{gd->nx, gd->ny, gd->nz}, gd->spacing, {gd->origin[0], gd->origin[1], gd->origin[2]}, gd->values,
                  gd->mode, p->eps_voxel};
  if (g.mode != 0 && g.mode != 1) return -3;
  Graph G;
  if (build_graph(n, nb, bonds, G)) return -1;
  const auto gdist = graph_dist3(G);
  std::vector<V3> P0(n);
  for (int i = 0; i < n; ++i) P0[i] = {(double)xyz[3 * i], (double)xyz[3 * i + 1], (double)xyz[3 * i + 2]};
  const V3 pocket_centre = {g.origin[0] + g.h * (g.dim[0] - 1) / 2.0, g.origin[1] + g.h * (g.dim[1] - 1) / 2.0,
                            g.origin[2] + g.h * (g.dim[2] - 1) / 2.0};
  const int R = p->restarts, N = p->align_steps, A = p->torsion_steps;
  int best_r = -1;
  double best_s = -kInf;
  for (int r = 0; r < R; ++r) {
    // starting pose
    const M3 S = restart_rotation(id, p->seed, r);
    const V3 c0 = centroid(P0);
    std::vector<V3> P(n);
    for (int i = 0; i < n; ++i) P[i] = pocket_centre + mul(S, P0[i] - c0);
    // rigid alignment
    const AlignOut al = align(g, P, N, forced_align ? forced_align[r] : -1);
    out->align_idx[r] = al.chosen;
    out->align_best[r] = al.best;
    out->align_second[r] = al.second;
    out->align_forced[r] = al.forced_score;
    out->align_robust[r] = al.robust;
    out->align_possible[r] = al.possible;
    // torsion sweep, bonds in input order
    for (int bi = 0; bi < nrot; ++bi) {
      int err = 0;
      const int fk = forced_tors ? forced_tors[r * nrot + bi] : -1;
      const TorsionOut t = torsion(g, P, G, rot[2 * bi], rot[2 * bi + 1], A, p->clash_dist, p->eps_clash, fk, &err);
      if (err) return err;
      const int o = r * nrot + bi;
      out->torsion_idx[o] = t.chosen;
      out->rejected[o] = t.rejected;
      out->tors_best[o] = t.best;
      out->tors_second[o] = t.second;
      out->tors_best_robust[o] = t.best_robust;
      out->tors_forced[o] = t.forced_score;
      out->tors_forced_margin[o] = t.forced_margin;
      out->tors_max_margin[o] = t.max_margin;
      out->tors_ambiguous[o] = t.n_ambiguous;
      out->tors_robust_valid[o] = t.robust_valid;
      out->tors_robust[o] = t.robust;
      out->tors_possible[o] = t.possible;
    }
    // rigid alignment of the optimised pose
    if (p->post_align) {
      const AlignOut pa = align(g, P, N, forced_post ? forced_post[r] : -1);
      out->post_idx[r] = pa.chosen;
      out->post_best[r] = pa.best;
      out->post_second[r] = pa.second;
      out->post_forced[r] = pa.forced_score;
      out->post_robust[r] = pa.robust;
      out->post_possible[r] = pa.possible;
    } else {
      out->post_idx[r] = -1;
      out->post_best[r] = out->post_second[r] = out->post_forced[r] = -kInf;
      out->post_robust[r] = out->post_possible[r] = -1;
    }
    // final score and clash count
    const double s = score(g, P);
    const Sc range = score_range(g, P);
    out->restart_score[r] = s;
    out->score_lo[r] = range.lo;
    out->score_hi[r] = range.hi;
    out->clash[r] = clash_count(P, gdist, p->clash_dist, &out->clash_margin[r]);
    for (int i = 0; i < n; ++i) {
      out->restart_xyz[(size_t)(r * n + i) * 3 + 0] = P[i].x;
      out->restart_xyz[(size_t)(r * n + i) * 3 + 1] = P[i].y;
      out->restart_xyz[(size_t)(r * n + i) * 3 + 2] = P[i].z;
    }
    if (s > best_s) {
      best_s = s;
      best_r = r;
    }
  }
  *out->best_score = best_s;
  *out->best_restart = best_r;
  return 0;
}

// Select Poses over one ligand's restarts.  score[R], xyz[R*n*3] (restart r, atom i at
// (r*n + i)*3).  Writes sel[K] (-1 past the last kept pose) and returns the number kept.
// rmsd_margin: over every keep/drop decision, how far the decision is from flipping (for a kept
// pose the smallest RMSD - threshold to the kept poses; for a dropped one the largest threshold -
// RMSD); score_margin: the smallest gap between consecutive scores in ranked order among the
// restarts examined and the next one (0 for a tie).  Returns -3 for bad sizes.
int oracle_select_poses(int32_t R, int32_t n, const double* score, const double* xyz, int32_t K, double thr,
                        int32_t* sel, double* rmsd_margin, double* score_margin) {
  if (R < 1 || n < 1 || K < 1 || !(thr >= 0)) return -3;
  std::vector<int> order(R);
  for (int r = 0; r < R; ++r) order[r] = r;
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    if (score[a] != score[b]) return score[a] > score[b];
    return a < b;
  });
  auto rmsd = [&](int a, int b) {
    double ss = 0;
    for (int i = 0; i < n; ++i)
      for (int c = 0; c < 3; ++c) {
        const double d = xyz[((size_t)a * n + i) * 3 + c] - xyz[((size_t)b * n + i) * 3 + c];
        ss += d * d;
      }
    return std::sqrt(ss / n);
  };
  std::vector<int> kept;
  double rm = kInf;
  int examined = 0;
  for (int t = 0; t < R && (int)kept.size() < K; ++t) {
    const int r = order[t];
    examined = t + 1;
    double nearest = kInf;
    for (int k : kept) nearest = std::min(nearest, rmsd(r, k));
    if (kept.empty() || nearest >= thr) {
      kept.push_back(r);
      if (!std::isinf(nearest)) rm = std::min(rm, nearest - thr);
    } else {
      rm = std::min(rm, thr - nearest);
    }
  }
  double sm = kInf;
  for (int t = 0; t + 1 < R && t < examined; ++t) sm = std::min(sm, score[order[t]] - score[order[t + 1]]);
  for (int k = 0; k < K; ++k) sel[k] = k < (int)kept.size() ? kept[k] : -1;
  *rmsd_margin = rm;
  *score_margin = sm;
  return (int)kept.size();
}

// ---- building blocks, exposed so each can be pinned on its own ------------------------------------

double oracle_score(const oracle_grid* gd, int32_t n, const double* xyz) {
  const Grid g = {{gd->nx, gd->ny, gd->nz}, gd->spacing, {gd->origin[0], gd->origin[1], gd->origin[2]}, gd->values,
                  gd->mode, 0.0};
  std::vector<V3> P(n);
  for (int i = 0; i < n; ++i) P[i] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
  return score(g, P);
}

// Mode-1 score of a pose and its range when every coordinate moves by up to eps grid units.
double oracle_score_range(const oracle_grid* gd, int32_t n, const double* xyz, double eps, double* lo, double* hi) {
  const Grid g = {{gd->nx, gd->ny, gd->nz}, gd->spacing, {gd->origin[0], gd->origin[1], gd->origin[2]}, gd->values,
                  gd->mode, eps};
  std::vector<V3> P(n);
  for (int i = 0; i < n; ++i) P[i] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
  const Sc r = score_range(g, P);
  *lo = r.lo;
  *hi = r.hi;
  return r.s;
}

uint64_t oracle_splitmix64(uint64_t state, uint64_t k) { return splitmix64(state, k); }

void oracle_restart_rotation(uint64_t id, uint64_t seed, int32_t r, double* R9) {
  const M3 R = restart_rotation(id, seed, r);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R9[3 * i + j] = R.m[i][j];
}

void oracle_align_pose(int32_t n, const double* xyz, int32_t N, int32_t i, int32_t j, double* out) {
  std::vector<V3> P(n);
  for (int a = 0; a < n; ++a) P[a] = {xyz[3 * a], xyz[3 * a + 1], xyz[3 * a + 2]};
  const std::vector<V3> Q = align_pose(P, centroid(P), N, i, j);
  for (int a = 0; a < n; ++a) {
    out[3 * a] = Q[a].x;
    out[3 * a + 1] = Q[a].y;
    out[3 * a + 2] = Q[a].z;
  }
}

int oracle_moving_set(int32_t n, int32_t nb, const int32_t* bonds, int32_t a, int32_t b, int32_t* mask) {
  Graph G;
  if (build_graph(n, nb, bonds, G)) return -1;
  std::vector<char> in_m;
  const int e = moving_set(G, a, b, in_m);
  if (e) return e;
  for (int i = 0; i < n; ++i) mask[i] = in_m[i];
  return 0;
}

int oracle_torsion_pose(int32_t n, const double* xyz, int32_t nb, const int32_t* bonds, int32_t a, int32_t b,
                        int32_t A, int32_t k, double* out) {
  Graph G;
  if (build_graph(n, nb, bonds, G)) return -1;
  std::vector<char> in_m;
  const int e = moving_set(G, a, b, in_m);
  if (e) return e;
  std::vector<V3> P(n);
  for (int i = 0; i < n; ++i) P[i] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
  const std::vector<V3> Q = torsion_pose(P, in_m, a, b, 2 * kPi * k / A);
  for (int i = 0; i < n; ++i) {
    out[3 * i] = Q[i].x;
    out[3 * i + 1] = Q[i].y;
    out[3 * i + 2] = Q[i].z;
  }
  return 0;
}

// Number of angles of the sweep of bond (a, b) rejected by the bump check (the restricted
// moving x fixed pair set), for a pose given in double precision.
int oracle_rejected_angles(int32_t n, const double* xyz, int32_t nb, const int32_t* bonds, int32_t a, int32_t b,
                           int32_t A, double dc) {
  Graph G;
  if (build_graph(n, nb, bonds, G)) return -1;
  std::vector<char> in_m;
  const int e = moving_set(G, a, b, in_m);
  if (e) return e;
  std::vector<V3> P(n);
  for (int i = 0; i < n; ++i) P[i] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
  int rej = 0;
  for (int k = 0; k < A; ++k) {
    const std::vector<V3> Q = torsion_pose(P, in_m, a, b, 2 * kPi * k / A);
    bool bump = false;
    for (int i = 0; i < n && !bump; ++i) {
      if (!in_m[i] || i == b) continue;
      for (int j = 0; j < n; ++j) {
        if (in_m[j] || j == a) continue;
        const V3 d = Q[i] - Q[j];
        if (dot(d, d) < dc * dc) {
          bump = true;
          break;
        }
      }
    }
    rej += bump;
  }
  return rej;
}

int oracle_clash_count(int32_t n, const double* xyz, int32_t nb, const int32_t* bonds, double dc) {
  Graph G;
  if (build_graph(n, nb, bonds, G)) return -1;
  std::vector<V3> P(n);
  for (int i = 0; i < n; ++i) P[i] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
  return clash_count(P, graph_dist3(G), dc, nullptr);
}

}  // extern "C"
