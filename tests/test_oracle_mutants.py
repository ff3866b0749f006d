"""The oracle's pins catch plausible mistakes (CPU only).

Each mutant is the oracle's source with one plausible mistake planted in a copy (a flipped sign, a
transposed operand, a dropped term, a wrong index, an off-by-one boundary or tie rule); the copy is
compiled on its own and every pin of tests/test_oracle_pins.py is run against it.  A mutant must
fail at least one pin.  The oracle in oracle/ is never modified.
"""
import inspect
import os
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

from . import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "dock_oracle.cpp")

MUTANTS = {
    "rot_x sign": ("return {{{1, 0, 0}, {0, c, -s}, {0, s, c}}};", "return {{{1, 0, 0}, {0, c, s}, {0, -s, c}}};"),
    "rot_y sign": ("return {{{c, 0, s}, {0, 1, 0}, {-s, 0, c}}};", "return {{{c, 0, -s}, {0, 1, 0}, {s, 0, c}}};"),
    "alignment order Rx Ry": ("mul(rot_y(2 * kPi * j / N), rot_x(2 * kPi * i / N))",
                              "mul(rot_x(2 * kPi * i / N), rot_y(2 * kPi * j / N))"),
    "rodrigues cross operands": ("s * cross(u, v)", "s * cross(v, u)"),
    "rodrigues axial term dropped": ("+ ((1.0 - c) * dot(u, v)) * u", "+ 0.0 * u"),
    "torsion axis reversed": ("const V3 axis = P[b] - P[a];", "const V3 axis = P[a] - P[b];"),
    "torsion half angles": ("torsion_pose(P, in_m, a, b, 2 * kPi * k / A);\n    bool bump = false;\n    double margin",
                            "torsion_pose(P, in_m, a, b, kPi * k / A);\n    bool bump = false;\n    double margin"),
    "trilinear weight swapped": ("(di ? t[0] : 1.0 - t[0])", "(di ? 1.0 - t[0] : t[0])"),
    "trilinear index transposed": ("(size_t)(i0[1] + dj)) * g.dim[0]", "(size_t)(i0[1] + di)) * g.dim[0]"),
    "grid edge excluded": ("u <= (double)(g.dim[a] - 1)", "u < (double)(g.dim[a] - 1)"),
    "cell index not clamped": ("if (i > g.dim[a] - 2) i = g.dim[a] - 2;", "if (i > g.dim[a] - 1) i = g.dim[a] - 1;"),
    "alignment ties to highest index": ("      if (s[i * N + j] > o.best) {", "      if (s[i * N + j] >= o.best) {"),
    "restart ties to highest index": ("    if (s > best_s) {", "    if (s >= best_s) {"),
    "start pose keeps offset": ("P[i] = pocket_centre + mul(S, P0[i] - c0);", "P[i] = pocket_centre + mul(S, P0[i]);"),
    "clash count includes 1-3": ("if (gd[i][j] < 3) continue;", "if (gd[i][j] < 2) continue;"),
    "splitmix constant": ("z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;", "z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ull;"),
    "shoemake sin/cos swapped": ("const double qx = a * std::sin(2 * kPi * u[1]), qy = a * std::cos(2 * kPi * u[1]);",
                                 "const double qx = a * std::cos(2 * kPi * u[1]), qy = a * std::cos(2 * kPi * u[1]);"),
    "moving side is a's side": ("std::vector<int> stack = {b};\n  in_m[b] = 1;", "std::vector<int> stack = {a};\n  in_m[a] = 1;"),
    "bump threshold not squared": ("if (d2 < dc * dc) bump = true;", "if (d2 < dc) bump = true;"),
    "select ties to highest restart": ("    return a < b;\n  });", "    return a > b;\n  });"),
    "select rmsd over coordinates": ("return std::sqrt(ss / n);", "return std::sqrt(ss / (3 * n));"),
    "select rmsd not rooted": ("return std::sqrt(ss / n);", "return ss / n;"),
    "select strict threshold": ("if (kept.empty() || nearest >= thr) {", "if (kept.empty() || nearest > thr) {"),
    "nearest voxel rounds down": ("nom[a] = (int)std::floor(u + 0.5);", "nom[a] = (int)std::floor(u);"),
    "nearest half-way to the lower voxel": ("nom[a] = (int)std::floor(u + 0.5);", "nom[a] = (int)std::ceil(u - 0.5);"),
    "nearest last voxel excluded": ("if (q[a] < 0 || q[a] > g.dim[a] - 1) return 0.0;",
                                    "if (q[a] < 0 || q[a] > g.dim[a] - 2) return 0.0;"),
    "nearest index transposed": ("return g.v[((size_t)q[2] * g.dim[1] + (size_t)q[1]) * g.dim[0] + q[0]];",
                                 "return g.v[((size_t)q[2] * g.dim[1] + (size_t)q[0]) * g.dim[0] + q[1]];"),
    "score range ignores eps": ("first[a] = (int)std::floor(u - g.eps + 0.5);", "first[a] = (int)std::floor(u + 0.5);"),
    "possible ignores the tie order": ("if (j < c ? !(r[c].hi > r[j].lo) : !(r[c].hi >= r[j].lo)) return false;",
                                       "if (!(r[c].hi >= r[j].lo)) return false;"),
    "only-possible ignores the tie order": ("if (j < c ? !(r[c].lo > r[j].hi) : !(r[c].lo >= r[j].hi)) return false;",
                                            "if (!(r[c].lo > r[j].hi)) return false;"),
    "no-valid-angle fallback": ("o.chosen = forced >= 0 ? forced : (chosen >= 0 ? chosen : 0);",
                                "o.chosen = forced >= 0 ? forced : (chosen >= 0 ? chosen : A - 1);"),
    "torsion ties to highest angle": ("    if (s > o.best) {\n      o.second = o.best;\n      o.best = s;\n      chosen = k;",
                                      "    if (s >= o.best) {\n      o.second = o.best;\n      o.best = s;\n      chosen = k;"),
    "bump check includes the moving bond atom": (
        "      if (!in_m[i] || i == b) continue;\n      for (int j = 0; j < G.n; ++j) {",
        "      if (!in_m[i]) continue;\n      for (int j = 0; j < G.n; ++j) {"),
    "bump check includes the fixed bond atom": (
        "        if (in_m[j] || j == a) continue;\n        const V3 d = Q[i] - Q[j];\n        const double d2",
        "        if (in_m[j]) continue;\n        const V3 d = Q[i] - Q[j];\n        const double d2"),
    "post-alignment skipped": ("    if (p->post_align) {", "    if (false) {"),
    "alignment pivot at the first atom": ("AlignOut align(const Grid& g, std::vector<V3>& P, int N, int forced) {\n  const V3 c = centroid(P);",
                                          "AlignOut align(const Grid& g, std::vector<V3>& P, int N, int forced) {\n  const V3 c = P[0];"),
    "restart streams not keyed by ligand": ("const uint64_t key = splitmix64(seed ^ id, 1);", "const uint64_t key = splitmix64(seed, 1);"),
    "grid lower edge excluded": ("if (!(u >= 0.0 && u <= (double)(g.dim[a] - 1))) return 0.0;",
                                 "if (!(u > 0.0 && u <= (double)(g.dim[a] - 1))) return 0.0;"),
    "select compares with the last kept pose only": ("    for (int k : kept) nearest = std::min(nearest, rmsd(r, k));",
                                                     "    if (!kept.empty()) nearest = rmsd(r, kept.back());"),
    "rotatable bonds swept in reverse order": ("    for (int bi = 0; bi < nrot; ++bi) {",
                                               "    for (int bj = 0; bj < nrot; ++bj) {\n      const int bi = nrot - 1 - bj;"),
    "alignment angles closed at 360": ("const M3 R = mul(rot_y(2 * kPi * j / N), rot_x(2 * kPi * i / N));",
                                       "const M3 R = mul(rot_y(2 * kPi * j / (N - 1)), rot_x(2 * kPi * i / (N - 1)));"),
}


def _pin_functions():
    return [(n, f) for n, f in inspect.getmembers(pins, inspect.isfunction)
            if n.startswith("test_") and list(inspect.signature(f).parameters) == ["oracle"]]


@pytest.fixture(scope="module")
def mutant_libs():
    src = open(SRC).read()
    for name, (old, new) in MUTANTS.items():
        assert src.count(old) == 1, f"mutant '{name}' no longer matches the oracle source"
    tmp = tempfile.mkdtemp(prefix="oracle_mutants_")
    from oracle import oracle as O

    def build(item):
        i, (name, (old, new)) = item
        return name, O.build_source(src.replace(old, new), os.path.join(tmp, f"mutant{i}.so"))
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        return dict(ex.map(build, enumerate(MUTANTS.items())))


def test_every_planted_mistake_fails_a_pin(oracle, mutant_libs):
    survivors = {}
    try:
        for name, path in mutant_libs.items():
            oracle.use_library(path)
            failed = []
            for pname, fn in _pin_functions():
                try:
                    fn(oracle)
                except Exception:
                    failed.append(pname)
            if not failed:
                survivors[name] = path
    finally:
        oracle.use_library(None)
    assert not survivors, f"mutants no pin catches: {sorted(survivors)}"
    # the real oracle passes them all again
    for pname, fn in _pin_functions():
        fn(oracle)
