"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test checks one building block, or the whole method, of arXiv 2209.05069 Alg. 1 against a
closed form, an invariant, a library routine (scipy's trilinear ``map_coordinates`` and
``Rotation``, networkx graph algorithms) or brute force on tiny inputs.
"""
import itertools
import math
import os

import networkx as nx
import numpy as np
import pytest
from scipy.ndimage import map_coordinates
from scipy.spatial.transform import Rotation

from paper_2209_05069_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---- independent helpers (library routines, no oracle code) ------------------------------------

def lib_trilinear(pocket_values, spacing, origin, pts):
    """scipy order-1 interpolation; mode='constant' gives 0 outside [0, G-1] on any axis."""
    pts = np.asarray(pts, np.float64).reshape(-1, 3)
    u = (pts - np.asarray(origin)) / spacing
    return map_coordinates(np.asarray(pocket_values, np.float64), [u[:, 2], u[:, 1], u[:, 0]],
                           order=1, mode="constant", cval=0.0)


def graph_of(n, bonds):
    G = nx.Graph()
    G.add_nodes_from(range(n))
    G.add_edges_from([tuple(map(int, b)) for b in bonds])
    return G


def lib_moving_side(n, bonds, a, b):
    G = graph_of(n, bonds)
    G.remove_edge(a, b)
    side = nx.node_connected_component(G, b)
    m = np.zeros(n, bool)
    m[list(side)] = True
    return m


def lib_torsion(xyz, moving, a, b, theta):
    u = xyz[b] - xyz[a]
    u = u / np.linalg.norm(u)
    out = xyz.copy()
    out[moving] = Rotation.from_rotvec(theta * u).apply(xyz[moving] - xyz[b]) + xyz[b]
    return out


def lib_far_pairs(n, bonds):
    """Pairs (i < j) more than two bonds apart (networkx shortest paths)."""
    d = dict(nx.all_pairs_shortest_path_length(graph_of(n, bonds), cutoff=2))
    return [(i, j) for i in range(n) for j in range(i + 1, n) if j not in d[i]]


def small_pocket(G=24, h=0.5, seed=3, noise=0.2, R=5.0):
    return synth.make_pocket(G, h, R, noise, seed)


def tiny_ligands(count, n_lo, n_hi, b, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    while len(out) < count:
        n = int(rng.integers(n_lo, n_hi + 1))
        xyz, bonds, rot, clipped = synth.make_ligand(rng, n, b)
        if not clipped:
            out.append((xyz, bonds, rot, len(out)))
    return out


# ---- SplitMix64 and the starting pose ----------------------------------------------------------

def test_splitmix64_known_answers(oracle):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 6
    for seed, k, val in rows:
        assert oracle.splitmix64(int(seed), int(k)) == int(val)


def test_restart_rotation_is_identity_for_restart_zero(oracle):
    for lid in (0, 7, 123456789):
        assert np.array_equal(oracle.restart_rotation(lid, 99, 0), np.eye(3))


def test_restart_rotations_are_proper_and_uniform(oracle):
    # Haar-uniform rotations: orthonormal, det +1, E[R_ij] = 0 and E[R_ij^2] = 1/3.
    Rs = np.array([oracle.restart_rotation(lid, 2209, r) for lid in range(400) for r in range(1, 31)])
    assert np.allclose(np.einsum("nij,nkj->nik", Rs, Rs), np.eye(3), atol=1e-12)
    assert np.allclose(np.linalg.det(Rs), 1.0, atol=1e-12)
    assert np.abs(Rs.mean(axis=0)).max() < 0.03
    assert np.abs((Rs ** 2).mean(axis=0) - 1.0 / 3.0).max() < 0.02
    # distinct restarts and distinct ligands draw distinct orientations
    assert len({tuple(np.round(R, 9).ravel()) for R in Rs}) == len(Rs)


# ---- score (sum of trilinear lookups) ------------------------------------------------------------

def test_score_constant_grid(oracle):
    c = 0.625
    pk = synth.make_field_pocket((10, 11, 12), 0.5, (-2.0, -2.5, -3.0), lambda x, y, z: c + 0 * x)
    g = oracle.GridView.of(pk)
    rng = np.random.default_rng(1)
    lo = pk.origin
    hi = pk.origin + pk.spacing * (np.array(pk.dims) - 1)
    pts = lo + rng.random((50, 3)) * (hi - lo)
    assert oracle.score(g, pts) == pytest.approx(50 * c, rel=1e-14)
    # atoms outside the grid contribute nothing; the far corner itself is inside
    assert oracle.score(g, [hi + [1e-9, 0, 0]]) == 0.0
    assert oracle.score(g, [lo - [0, 1e-9, 0]]) == 0.0
    assert oracle.score(g, [hi]) == pytest.approx(c, rel=1e-14)


def test_score_linear_grid_is_exact(oracle):
    gvec, d = np.array([0.3, -1.1, 0.7]), 2.5
    pk = synth.make_field_pocket((9, 8, 7), 0.75, (-3.0, -2.0, -1.5), lambda x, y, z: gvec[0] * x + gvec[1] * y + gvec[2] * z + d)
    # float32 storage of an affine field is not affine; keep the values in double
    zz, yy, xx = np.meshgrid(*[pk.origin[a] + pk.spacing * np.arange(pk.dims[a]) for a in (2, 1, 0)], indexing="ij")
    v = gvec[0] * xx + gvec[1] * yy + gvec[2] * zz + d
    g = oracle.GridView(v, pk.spacing, pk.origin)
    rng = np.random.default_rng(2)
    hi = pk.origin + pk.spacing * (np.array(pk.dims) - 1)
    pts = pk.origin + rng.random((40, 3)) * (hi - pk.origin)
    assert oracle.score(g, pts) == pytest.approx(float(gvec @ pts.sum(0) + 40 * d), rel=1e-12)


def test_score_matches_library_trilinear(oracle):
    pk = small_pocket()
    g = oracle.GridView.of(pk)
    rng = np.random.default_rng(3)
    span = pk.spacing * (np.array(pk.dims) - 1)
    pts = pk.origin - 1.0 + rng.random((400, 3)) * (span + 2.0)  # some atoms fall outside
    ref = lib_trilinear(pk.values, pk.spacing, pk.origin, pts)
    got = np.array([oracle.score(g, p[None]) for p in pts])
    assert np.abs(got - ref).max() < 1e-12
    assert (ref == 0).sum() > 10 and (ref != 0).sum() > 100


def test_score_on_far_faces_reads_only_the_grid(oracle):
    # atoms exactly on the far faces, edges and corner of the grid interpolate inside it; the grid
    # sits in a buffer poisoned with NaN after its end, so any read past the grid shows up
    G, h = 6, 0.5
    rng = np.random.default_rng(8)
    buf = np.full(G ** 3 + 64, np.nan)
    buf[:G ** 3] = rng.random(G ** 3)
    vals = buf[:G ** 3].reshape(G, G, G)
    g = oracle.GridView(vals, h, (0.0, 0.0, 0.0))
    assert g.values.ctypes.data == buf.ctypes.data   # the view was not copied
    far = h * (G - 1)
    pts = [(far, far, far), (far, 1.2, far), (far, far, 0.7), (0.3, far, far), (far, 0.0, 0.0), (1.1, 0.9, far)]
    for p in pts:
        got = oracle.score(g, [p])
        assert np.isfinite(got)
        assert abs(got - lib_trilinear(vals, h, (0, 0, 0), [p])[0]) < 1e-12


def test_score_quadratic_sphere_closed_form(oracle):
    # noise-free sphere grid 1 - (r/R)^2: on a cell whose corners all lie inside R, trilinear of
    # X^2 equals X^2 + (X - X0)(X0 + h - X), so interpolated f = f_exact - sum_axes (X-X0)(X0+h-X)/R^2
    w = synth.WORKLOADS["tiny"]
    pk = synth.make_pocket(w.grid, w.spacing, w.radius, 0.0, 1)
    v64 = None
    ax = pk.origin[0] + pk.spacing * np.arange(w.grid)
    zz, yy, xx = np.meshgrid(ax, ax, ax, indexing="ij")
    r = np.sqrt(xx ** 2 + yy ** 2 + zz ** 2)
    v64 = np.where(r < w.radius, 1.0 - (r / w.radius) ** 2, 0.0)
    g = oracle.GridView(v64, pk.spacing, pk.origin)
    rng = np.random.default_rng(4)
    pts = (rng.random((300, 3)) - 0.5) * 2 * 6.0 / np.sqrt(3)  # |p| <= 6 < R - cell diagonal
    h, R = pk.spacing, w.radius
    X0 = pk.origin + h * np.floor((pts - pk.origin) / h)
    expect = 1.0 - (pts ** 2).sum(1) / R ** 2 - ((pts - X0) * (X0 + h - pts)).sum(1) / R ** 2
    got = np.array([oracle.score(g, p[None]) for p in pts])
    assert np.abs(got - expect).max() < 1e-12


# ---- rigid alignment poses ------------------------------------------------------------------------

def test_align_pose_quarter_turns(oracle):
    rng = np.random.default_rng(5)
    P = rng.normal(size=(9, 3)) * 2 + [1.0, -2.0, 0.5]
    c = P.mean(0)
    d = P - c
    assert np.allclose(oracle.align_pose(P, 4, 0, 0), P, atol=1e-14)
    # Rx(90 deg): (x, y, z) -> (x, -z, y)
    assert np.allclose(oracle.align_pose(P, 4, 1, 0), c + np.stack([d[:, 0], -d[:, 2], d[:, 1]], 1), atol=1e-12)
    # Ry(90 deg): (x, y, z) -> (z, y, -x)
    assert np.allclose(oracle.align_pose(P, 4, 0, 1), c + np.stack([d[:, 2], d[:, 1], -d[:, 0]], 1), atol=1e-12)


def test_align_pose_matches_library_composition(oracle):
    rng = np.random.default_rng(6)
    P = rng.normal(size=(15, 3)) * 3
    c = P.mean(0)
    N = 30
    for (i, j) in [(1, 0), (0, 1), (7, 13), (29, 29), (12, 5)]:
        R = Rotation.from_euler("y", 2 * math.pi * j / N) * Rotation.from_euler("x", 2 * math.pi * i / N)
        Q = oracle.align_pose(P, N, i, j)
        assert np.allclose(Q, c + R.apply(P - c), atol=1e-12)
        # rigid: pairwise distances and centroid preserved
        dP = np.linalg.norm(P[:, None] - P[None], axis=-1)
        dQ = np.linalg.norm(Q[:, None] - Q[None], axis=-1)
        assert np.abs(dP - dQ).max() < 1e-12
        assert np.allclose(Q.mean(0), c, atol=1e-12)


# ---- moving side and torsion ----------------------------------------------------------------------

def test_moving_set_matches_graph_component(oracle):
    for xyz, bonds, rot, _ in tiny_ligands(20, 12, 40, 4, 7):
        for a, b in rot:
            assert np.array_equal(oracle.moving_set(len(xyz), bonds, int(a), int(b)),
                                  lib_moving_side(len(xyz), bonds, int(a), int(b)))


def test_moving_set_rejects_ring_bond_and_bad_bond(oracle):
    ring = [(0, 1), (1, 2), (2, 3), (3, 0), (3, 4)]
    with pytest.raises(ValueError, match="-2"):
        oracle.moving_set(5, ring, 0, 1)
    with pytest.raises(ValueError, match="-1"):
        oracle.moving_set(5, ring, 0, 2)
    assert oracle.moving_set(5, ring, 3, 4).tolist() == [False, False, False, False, True]


def test_torsion_pose_matches_library_rotation_and_invariants(oracle):
    for xyz, bonds, rot, _ in tiny_ligands(10, 15, 30, 3, 8):
        P = xyz.astype(np.float64)
        n = len(P)
        for a, b in rot:
            a, b = int(a), int(b)
            m = lib_moving_side(n, bonds, a, b)
            for A, k in [(64, 0), (64, 1), (64, 17), (4, 2), (256, 255)]:
                Q = oracle.torsion_pose(P, bonds, a, b, A, k)
                assert np.allclose(Q, lib_torsion(P, m, a, b, 2 * math.pi * k / A), atol=1e-12)
                # bond lengths and distances within each side are unchanged; the fixed side stays put
                bl = lambda X: np.linalg.norm(X[bonds[:, 0]] - X[bonds[:, 1]], axis=1)
                assert np.abs(bl(P) - bl(Q)).max() < 1e-12
                assert np.array_equal(Q[~m], P[~m])
                for S in (m, ~m):
                    dP = np.linalg.norm(P[S][:, None] - P[S][None], axis=-1)
                    dQ = np.linalg.norm(Q[S][:, None] - Q[S][None], axis=-1)
                    assert np.abs(dP - dQ).max() < 1e-12


def test_half_turn_closed_form(oracle):
    # theta = pi: v -> 2 (u.v) u - v about the pivot b
    P = np.array([[0.0, 0, 0], [1.5, 0, 0], [2.0, 1.4, 0.0], [2.7, 1.9, 1.1]])
    bonds = [(0, 1), (1, 2), (2, 3)]
    Q = oracle.torsion_pose(P, bonds, 0, 1, 8, 4)
    u = np.array([1.0, 0, 0])
    v = P[2:] - P[1]
    assert np.allclose(Q[2:], P[1] + 2 * (v @ u)[:, None] * u - v, atol=1e-14)


# ---- bump check and clash count -----------------------------------------------------------------------

def test_clash_count_brute_force(oracle):
    rng = np.random.default_rng(9)
    for xyz, bonds, rot, _ in tiny_ligands(10, 20, 40, 3, 10):
        P = xyz.astype(np.float64) + rng.normal(scale=0.6, size=xyz.shape)  # jostle to create clashes
        pairs = lib_far_pairs(len(P), bonds)
        for dc in (1.5, 2.0, 3.0):
            brute = sum(1 for i, j in pairs if np.sum((P[i] - P[j]) ** 2) < dc * dc)
            assert oracle.clash_count(P, bonds, dc) == brute


def test_restricted_bump_check_equals_all_pairs_check(oracle):
    # from a clash-free start only pairs across the bond change distance, so checking
    # M_b\{b} x F_b\{a} decides the same as checking every pair more than two bonds apart
    checked = 0
    for xyz, bonds, rot, _ in tiny_ligands(12, 15, 35, 3, 11):
        P = xyz.astype(np.float64)
        n = len(P)
        pairs = np.array(lib_far_pairs(n, bonds))
        for dc in (2.0, 2.6):
            d0 = np.linalg.norm(P[pairs[:, 0]] - P[pairs[:, 1]], axis=1)
            if (d0 < dc).any():
                continue
            for a, b in rot:
                a, b = int(a), int(b)
                m = lib_moving_side(n, bonds, a, b)
                A = 32
                brute = 0
                for k in range(A):
                    Q = lib_torsion(P, m, a, b, 2 * math.pi * k / A)
                    brute += int((np.linalg.norm(Q[pairs[:, 0]] - Q[pairs[:, 1]], axis=1) < dc).any())
                assert oracle.rejected_angles(P, bonds, a, b, A, dc) == brute
                checked += 1
    assert checked > 10


def test_contacts_with_the_bond_atoms_do_not_reject_angles(oracle):
    # The bond atoms a and b lie on the rotation axis, so their distances to the other side never
    # change under the torsion: a pre-existing contact of b with a fixed atom, or of a moving atom
    # with a, must not reject every angle.  Here b sits 1.93 A from fixed atom 2 and moving atom 3
    # sits 1.93 A from a (both below d_c = 2.0 A); only the pair (3, 2) changes distance, and only
    # its approaches may reject angles.
    c80, s80 = math.cos(math.radians(80)), math.sin(math.radians(80))
    P = np.array([[0.0, 0.0, 0.0],                      # a
                  [1.5, 0.0, 0.0],                      # b
                  [1.5 * c80, 1.5 * s80, 0.0],          # fixed, bonded to a
                  [1.5 - 1.5 * c80, -1.5 * s80, 0.0]])  # moving, bonded to b
    bonds = np.array([[0, 1], [0, 2], [1, 3]], np.int32)
    dc, A = 2.0, 72
    assert np.linalg.norm(P[1] - P[2]) < dc and np.linalg.norm(P[3] - P[0]) < dc
    m = lib_moving_side(4, bonds, 0, 1)
    expected = sum(1 for k in range(A)
                   if np.linalg.norm(lib_torsion(P, m, 0, 1, 2 * math.pi * k / A)[3] - P[2]) < dc)
    assert 0 < expected < A
    assert oracle.rejected_angles(P, bonds, 0, 1, A, dc) == expected
    # the same through the whole method: rigid moves keep every internal distance, so the sweep of
    # this bond rejects the same number of angles after the placement and the alignment
    g = oracle.GridView.of(small_pocket(G=40, h=0.5, R=8.0))
    p = oracle.Params(restarts=1, align_steps=6, torsion_steps=A, clash_dist=dc, post_align=0, seed=3)
    r = oracle.dock_ligand(g, P.astype(np.float32), bonds, np.array([[0, 1]], np.int32), 7, p)
    assert int(np.asarray(r["rejected"]).reshape(-1)[0]) == expected


# ---- whole method --------------------------------------------------------------------------------------

def _params(oracle, **kw):
    base = dict(restarts=4, align_steps=30, torsion_steps=32, clash_dist=2.0, post_align=1, seed=11)
    base.update(kw)
    return oracle.Params(**base)


def test_dock_constant_grid_ties_resolve_to_lowest_index(oracle):
    c = 0.25
    pk = synth.make_field_pocket((48, 48, 48), 0.5, (-11.75,) * 3, lambda x, y, z: c + 0 * x)
    g = oracle.GridView.of(pk)
    for xyz, bonds, rot, lid in tiny_ligands(4, 15, 25, 3, 12):
        r = oracle.dock_ligand(g, xyz, bonds, rot, lid, _params(oracle))
        n = len(xyz)
        assert np.allclose(r["restart_score"], n * c, rtol=1e-13)
        assert r["best_restart"] == 0
        assert (r["align_idx"] == 0).all() and (r["post_idx"] == 0).all()
        # every accepted angle ties, so each bond takes its lowest accepted angle
        # (angle 0 is the current, clash-free conformation)
        assert (r["torsion_idx"] == 0).all()


def test_dock_bond_with_no_accepted_angle_keeps_the_conformation(oracle):
    # with a bump threshold longer than the ligand every angle of every bond bumps: each bond keeps
    # angle 0, rejects all A angles, and the final pose equals that of the same ligand docked with
    # no rotatable bonds at all
    pk = small_pocket(G=40, h=0.5, R=8.0)
    g = oracle.GridView.of(pk)
    A = 24
    for xyz, bonds, rot, lid in tiny_ligands(3, 12, 20, 3, 21):
        p = _params(oracle, restarts=2, align_steps=6, torsion_steps=A, clash_dist=40.0)
        r = oracle.dock_ligand(g, xyz, bonds, rot, lid, p)
        r0 = oracle.dock_ligand(g, xyz, bonds, np.zeros((0, 2), np.int32), lid, p)
        assert (r["torsion_idx"] == 0).all() and (r["rejected"] == A).all()
        assert np.allclose(r["restart_xyz"], r0["restart_xyz"], rtol=0, atol=1e-12)


def test_dock_restart_zero_is_a_pure_translation(oracle):
    pk = small_pocket(G=40, h=0.5, R=8.0)
    g = oracle.GridView.of(pk)
    xyz, bonds, _, lid = tiny_ligands(1, 20, 20, 0, 13)[0]
    r = oracle.dock_ligand(g, xyz, bonds, np.zeros((0, 2), np.int32), lid, _params(oracle, restarts=1, align_steps=1, post_align=0))
    centre = pk.origin + pk.spacing * (np.array(pk.dims) - 1) / 2
    P = xyz.astype(np.float64)
    assert np.allclose(r["restart_xyz"][0], P - P.mean(0) + centre, atol=1e-12)
    assert r["restart_score"][0] == pytest.approx(lib_trilinear(pk.values, pk.spacing, pk.origin, r["restart_xyz"][0]).sum(), rel=1e-12)


def test_dock_alignment_is_the_brute_force_best_pose(oracle):
    pk = small_pocket(G=40, h=0.5, R=8.0, noise=0.3)
    g = oracle.GridView.of(pk)
    N = 6
    for xyz, bonds, _, lid in tiny_ligands(3, 12, 20, 0, 14):
        r = oracle.dock_ligand(g, xyz, bonds, np.zeros((0, 2), np.int32), lid, _params(oracle, restarts=3, align_steps=N, post_align=0))
        for rr in range(3):
            S = oracle.restart_rotation(lid, 11, rr)
            centre = pk.origin + pk.spacing * (np.array(pk.dims) - 1) / 2
            X = xyz.astype(np.float64)
            P = centre + (X - X.mean(0)) @ S.T
            c = P.mean(0)
            scores = []
            for i in range(N):
                for j in range(N):
                    R = Rotation.from_euler("y", 2 * math.pi * j / N) * Rotation.from_euler("x", 2 * math.pi * i / N)
                    scores.append(lib_trilinear(pk.values, pk.spacing, pk.origin, c + R.apply(P - c)).sum())
            assert r["align_idx"][rr] == int(np.argmax(scores))
            assert r["restart_score"][rr] == pytest.approx(max(scores), rel=1e-12)


def test_dock_linear_grid_torsion_closed_form(oracle):
    # affine grid f = g.x + d: the score of a torsion angle is S + g.sum_M(x_b + h u + cos t r + sin t w),
    # so the best angle maximises cos(theta - phi) with phi = atan2(g.sum w, g.sum r)
    gvec = np.array([0.8, -0.35, 0.5])
    G, h = 64, 0.5
    o = np.full(3, -h * (G - 1) / 2)
    ax = o[0] + h * np.arange(G)
    zz, yy, xx = np.meshgrid(ax, ax, ax, indexing="ij")
    g = oracle.GridView(gvec[0] * xx + gvec[1] * yy + gvec[2] * zz + 3.0, h, o)
    A = 64
    for xyz, bonds, rot, lid in tiny_ligands(5, 15, 30, 4, 15):
        r = oracle.dock_ligand(g, xyz, bonds, rot, lid, _params(oracle, restarts=1, align_steps=1, post_align=0,
                                                                 clash_dist=0.0, torsion_steps=A))
        P = xyz.astype(np.float64) - xyz.astype(np.float64).mean(0)  # restart 0: centroid to the centre (0)
        n = len(P)
        for bi, (a, b) in enumerate(rot):
            a, b = int(a), int(b)
            m = lib_moving_side(n, bonds, a, b)
            u = (P[b] - P[a]) / np.linalg.norm(P[b] - P[a])
            v = P[m] - P[b]
            rr = v - np.outer(v @ u, u)
            ww = np.cross(u, rr)
            phi = math.atan2(gvec @ ww.sum(0), gvec @ rr.sum(0))
            vals = np.cos(2 * math.pi * np.arange(A) / A - phi)
            k = int(np.argmax(vals))
            assert r["torsion_idx"][0, bi] == k
            P = lib_torsion(P, m, a, b, 2 * math.pi * k / A)
        assert np.allclose(r["restart_xyz"][0], P, atol=1e-10)
        assert r["restart_score"][0] == pytest.approx(gvec @ P.sum(0) + 3.0 * n, rel=1e-12)


def _brute_scores(pk, P, bonds, rot, A, dc):
    """All A^B angle combinations applied in bond order: final scores and validity per combination."""
    n = len(P)
    res = {}
    for combo in itertools.product(range(A), repeat=len(rot)):
        Q = P.copy()
        ok = True
        for (a, b), k in zip(rot, combo):
            a, b = int(a), int(b)
            m = lib_moving_side(n, bonds, a, b)
            Q = lib_torsion(Q, m, a, b, 2 * math.pi * k / A)
            mi = [i for i in range(n) if m[i] and i != b]
            fj = [j for j in range(n) if not m[j] and j != a]
            d2 = ((Q[mi][:, None] - Q[fj][None]) ** 2).sum(-1)
            ok = ok and not (d2 < dc * dc).any()
        res[combo] = (lib_trilinear(pk.values, pk.spacing, pk.origin, Q).sum(), ok)
    return res


def test_dock_torsion_against_brute_force_on_tiny_ligands(oracle):
    pk = small_pocket(G=40, h=0.5, R=8.0, noise=0.3)
    g = oracle.GridView.of(pk)
    centre = pk.origin + pk.spacing * (np.array(pk.dims) - 1) / 2
    A, dc = 12, 2.0
    seen_multi = 0
    for nb in (1, 2, 3):
        for xyz, bonds, rot, lid in tiny_ligands(3, 8, 10, nb, 16 + nb):
            r = oracle.dock_ligand(g, xyz, bonds, rot, lid, _params(oracle, restarts=1, align_steps=1, post_align=0,
                                                                     torsion_steps=A, clash_dist=dc))
            P = xyz.astype(np.float64) - xyz.astype(np.float64).mean(0) + centre
            brute = _brute_scores(pk, P, bonds, rot, A, dc)
            valid = {c: s for c, (s, ok) in brute.items() if ok}
            greedy = tuple(int(k) for k in r["torsion_idx"][0])
            if len(rot) == 1:
                # one bond: the greedy sweep is the exhaustive search
                best = max(valid.items(), key=lambda kv: (kv[1], -kv[0][0]))[0] if valid else (0,)
                assert greedy == best
            else:
                seen_multi += 1
                # the first greedy step is the best single step; the greedy end is no better than
                # the best combination (the paper rejects the combinatorial search, Section 4)
                one = _brute_scores(pk, P, bonds, rot[:1], A, dc)
                first = {c[0]: s1 for c, (s1, ok1) in one.items() if ok1}
                if first:
                    assert greedy[0] == max(first.items(), key=lambda kv: (kv[1], -kv[0]))[0]
                if valid:
                    assert r["restart_score"][0] <= max(valid.values()) + 1e-12
            assert r["restart_score"][0] == pytest.approx(brute[greedy][0], rel=1e-12)
    assert seen_multi >= 3


def test_dock_forced_replay_reproduces_free_run(oracle):
    w = synth.WORKLOADS["tiny"]
    pk = synth.workload_pocket(w)
    g = oracle.GridView.of(pk)
    db = synth.make_db(w, 3)
    p = _params(oracle, restarts=3, torsion_steps=64)
    for l in range(db.n_lig):
        free = oracle.dock_ligand(g, *db.ligand(l), p)
        rep = oracle.dock_ligand(g, *db.ligand(l), p, forced_align=free["align_idx"], forced_post=free["post_idx"],
                                 forced_tors=free["torsion_idx"])
        for k in ("restart_score", "restart_xyz", "rejected", "clash"):
            assert np.array_equal(free[k], rep[k])
        assert np.array_equal(rep["align_forced"], free["align_best"])
        has_valid = free["tors_best"] > -np.inf
        assert np.array_equal(rep["tors_forced"][has_valid], free["tors_best"][has_valid])


def test_post_align_flag(oracle):
    w = synth.WORKLOADS["tiny"]
    pk = synth.workload_pocket(w)
    g = oracle.GridView.of(pk)
    db = synth.make_db(w, 1)
    r = oracle.dock_ligand(g, *db.ligand(0), _params(oracle, restarts=2, post_align=0))
    assert (r["post_idx"] == -1).all()
    r1 = oracle.dock_ligand(g, *db.ligand(0), _params(oracle, restarts=2, post_align=1))
    assert (r1["post_idx"] >= 0).all()
    assert (r1["restart_score"] >= r["restart_score"] - 1e-12).all()  # index 0 (identity) is among the poses


def test_dock_rejects_invalid_inputs(oracle):
    pk = small_pocket()
    g = oracle.GridView.of(pk)
    xyz = np.zeros((5, 3), np.float32)
    xyz[:, 0] = np.arange(5) * 1.5
    ring = [(0, 1), (1, 2), (2, 3), (3, 0), (3, 4)]
    with pytest.raises(ValueError, match="-2"):
        oracle.dock_ligand(g, xyz, ring, [(0, 1)], 0, _params(oracle, restarts=1, align_steps=1))
    with pytest.raises(ValueError, match="-1"):
        oracle.dock_ligand(g, xyz, [(0, 9)], [], 0, _params(oracle, restarts=1, align_steps=1))


# ---- Select Poses ------------------------------------------------------------------------------

def _shifted_poses(shifts_x, n=5):
    """Poses of one ligand that differ by a rigid shift along x.  Coordinates are multiples of 1/8,
    so every difference, square and mean below is exact: the RMSD of two poses is |dx| exactly."""
    base = (np.arange(3 * n, dtype=np.float64).reshape(n, 3) * 0.125) - 1.0
    return np.stack([base + np.array([sx, 0.0, 0.0]) for sx in shifts_x])


def test_select_poses_hand_worked_translation_family(oracle):
    xyz = _shifted_poses([0.0, 1.0, 2.5, 3.0, 6.0])
    # ranked 0..4; threshold 2: 1 is 1.0 from 0 (dropped), 2 is 2.5 from 0 (kept), 3 is 0.5 from 2
    # (dropped), 4 is 3.5 from 2 (kept)
    r = oracle.select_poses([5, 4, 3, 2, 1], xyz, 5, 2.0)
    assert list(r["sel"]) == [0, 2, 4, -1, -1] and r["n_kept"] == 3
    assert r["rmsd_margin"] == pytest.approx(0.5, abs=1e-12)
    assert r["score_margin"] == pytest.approx(1.0, abs=1e-12)
    assert list(oracle.select_poses([5, 4, 3, 2, 1], xyz, 2, 2.0)["sel"]) == [0, 2]
    # scores reorder the walk: 1 (x=1), 3 (x=3, exactly 2.0 from 1: kept, the test is >=),
    # 4 (x=6, kept), 2 (x=2.5, 0.5 from 3), 0 (x=0, 1.0 from 1)
    r = oracle.select_poses([1, 5, 2, 4, 3], xyz, 5, 2.0)
    assert list(r["sel"]) == [1, 3, 4, -1, -1]
    assert r["rmsd_margin"] == 0.0


def test_select_poses_rmsd_is_root_mean_square_over_atoms(oracle):
    # one atom of four moved by 3 A: RMSD = sqrt(9 / 4) = 1.5 exactly
    a = _shifted_poses([0.0], n=4)[0]
    b = a.copy()
    b[0, 0] += 3.0
    xyz = np.stack([a, b])
    assert list(oracle.select_poses([2, 1], xyz, 2, 1.5)["sel"]) == [0, 1]
    assert list(oracle.select_poses([2, 1], xyz, 2, 1.5 + 1e-9)["sel"]) == [0, -1]
    assert list(oracle.select_poses([2, 1], xyz, 2, 1.5 - 1e-9)["sel"]) == [0, 1]


def test_select_poses_zero_threshold_is_the_score_ranking(oracle):
    rng = np.random.default_rng(5)
    for R in (1, 3, 17, 40):
        score = rng.integers(0, 6, R).astype(np.float64)      # many ties
        xyz = rng.normal(size=(R, 7, 3))
        xyz[R // 2] = xyz[0]                                  # identical poses are RMSD 0 >= 0
        order = np.lexsort((np.arange(R), -score))            # score descending, ties lowest index
        for K in (1, min(4, R), R):
            r = oracle.select_poses(score, xyz, K, 0.0)
            assert list(r["sel"]) == list(order[:K]) and r["n_kept"] == K


def test_select_poses_single_pose_is_the_best_restart(oracle):
    pk = small_pocket(G=40, h=0.5, R=8.0)
    g = oracle.GridView.of(pk)
    for xyz, bonds, rot, lid in tiny_ligands(3, 10, 18, 2, 31):
        d = oracle.dock_ligand(g, xyz, bonds, rot, lid, _params(oracle, restarts=6, align_steps=6, torsion_steps=8))
        r = oracle.select_poses(d["restart_score"], d["restart_xyz"], 1, 2.0)
        assert list(r["sel"]) == [d["best_restart"]]


def test_select_poses_greedy_properties(oracle):
    """On random instances the kept set is what the greedy rule fixes: kept poses are pairwise at
    least the threshold apart and keep the score order; every restart examined but dropped lies
    closer than the threshold to a pose kept before it; fewer than K kept means all were examined."""
    rng = np.random.default_rng(9)
    for trial in range(60):
        R, n, K = int(rng.integers(2, 20)), int(rng.integers(1, 9)), int(rng.integers(1, 8))
        thr = float(rng.uniform(0.2, 2.0))
        score = rng.normal(size=R).round(1)
        xyz = rng.normal(scale=0.8, size=(R, n, 3))
        r = oracle.select_poses(score, xyz, K, thr)
        sel = [s for s in r["sel"] if s >= 0]
        assert len(sel) == r["n_kept"] and all(s == -1 for s in r["sel"][len(sel):])

        def rmsd(a, b):
            return np.sqrt(((xyz[a] - xyz[b]) ** 2).sum(axis=1).mean())
        order = list(np.lexsort((np.arange(R), -score)))
        assert [o for o in order if o in sel] == sel
        for i, a in enumerate(sel):
            for b in sel[:i]:
                assert rmsd(a, b) >= thr
        last = order.index(sel[-1]) if len(sel) == K else R - 1
        for t in range(last + 1):
            o = order[t]
            if o not in sel:
                assert any(rmsd(o, k) < thr for k in sel if order.index(k) < t)


# ---- integer grid: nearest-voxel score -----------------------------------------------------------

def lib_nearest(pocket_values, spacing, origin, pts):
    """scipy's nearest-neighbour grid interpolator; 0 outside the voxel centres' span."""
    from scipy.interpolate import RegularGridInterpolator
    v = np.asarray(pocket_values, np.float64)
    axes = [np.arange(d, dtype=np.float64) for d in v.shape]
    f = RegularGridInterpolator(axes, v, method="nearest", bounds_error=False, fill_value=0.0)
    u = (np.asarray(pts, np.float64).reshape(-1, 3) - np.asarray(origin)) / spacing
    return f(u[:, ::-1])


def _one_voxel_grid(oracle, value=7.0):
    v = np.zeros((6, 6, 6))
    v[4, 3, 2] = value                       # voxel (i, j, k) = (2, 3, 4)
    return oracle.GridView(v, 0.5, (-1.0, -1.0, -1.0), mode=1), np.array([0.0, 0.5, 1.0])


def test_nearest_voxel_reads_the_voxel_whose_cube_holds_the_atom(oracle):
    g, centre = _one_voxel_grid(oracle)
    for axis in range(3):
        e = np.zeros(3)
        e[axis] = 0.5                        # one voxel spacing; every position below is exact
        assert oracle.score(g, [centre]) == 7.0
        assert oracle.score(g, [centre + 0.49 * e]) == 7.0
        assert oracle.score(g, [centre - 0.49 * e]) == 7.0
        assert oracle.score(g, [centre + 0.51 * e]) == 0.0
        assert oracle.score(g, [centre - 0.51 * e]) == 0.0
        # half-way between two voxels the upper one is read
        assert oracle.score(g, [centre - 0.5 * e]) == 7.0
        assert oracle.score(g, [centre + 0.5 * e]) == 0.0
    assert oracle.score(g, [centre, centre + [0.1, -0.2, 0.2], centre + [0.5, 0, 0]]) == 14.0


def test_nearest_voxel_grid_edges(oracle):
    g = oracle.GridView(np.ones((4, 4, 4)), 1.0, (0.0, 0.0, 0.0), mode=1)
    mid = np.array([1.0, 2.0, 1.0])
    for axis in range(3):
        for u, want in [(-0.5, 1.0), (-0.5 - 1e-9, 0.0), (3.5 - 1e-9, 1.0), (3.5, 0.0), (0.0, 1.0), (3.0, 1.0)]:
            p = mid.copy()
            p[axis] = u
            assert oracle.score(g, [p]) == want, (axis, u)


def test_nearest_voxel_matches_library_interpolator(oracle):
    rng = np.random.default_rng(41)
    v = rng.integers(-50, 50, size=(9, 11, 13)).astype(np.float64)
    g = oracle.GridView(v, 0.375, (-1.0, 2.0, -3.0), mode=1)
    for _ in range(20):
        u = rng.uniform(0, 1, size=(30, 3)) * (np.array([13, 11, 9]) - 1)   # inside the centres' span
        pts = (-1.0, 2.0, -3.0) + 0.375 * u
        assert oracle.score(g, pts) == lib_nearest(v, 0.375, (-1.0, 2.0, -3.0), pts).sum()


def test_nearest_voxel_score_range(oracle):
    v = np.zeros((6, 6, 6))
    v[4, 3, 2], v[4, 3, 3], v[4, 4, 2], v[4, 4, 3] = 7, -2, 5, 11     # (i, j) in {2, 3} x {3, 4} at k = 4
    g = oracle.GridView(v, 0.5, (-1.0, -1.0, -1.0), mode=1)
    centre = np.array([0.0, 0.5, 1.0])                                # voxel (2, 3, 4)
    assert oracle.score_range(g, [centre + [0.1, 0.05, 0]], 1e-4) == (7.0, 7.0, 7.0)
    # 3e-5 grid units past the x half-way plane: reads voxel 3 (-2), could read voxel 2 (7)
    s, lo, hi = oracle.score_range(g, [centre + [0.25 + 1.5e-5, 0.1, 0]], 1e-4)
    assert (s, lo, hi) == (-2.0, -2.0, 7.0)
    assert oracle.score_range(g, [centre + [0.25 + 1.5e-5, 0.1, 0]], 0.0) == (-2.0, -2.0, -2.0)
    # near two half-way planes: any of the four voxels
    s, lo, hi = oracle.score_range(g, [centre + [0.25 - 1.5e-5, 0.25 + 1.5e-5, 0]], 1e-4)
    assert (s, lo, hi) == (5.0, -2.0, 11.0)
    # ranges add over atoms
    s, lo, hi = oracle.score_range(g, [centre, centre + [0.25 + 1.5e-5, 0.1, 0]], 1e-4)
    assert (s, lo, hi) == (5.0, 5.0, 14.0)


def _int_params(oracle, **kw):
    base = dict(restarts=3, align_steps=6, torsion_steps=16, clash_dist=2.0, post_align=1, seed=11)
    base.update(kw)
    return oracle.Params(**base)


def test_dock_integer_constant_grid_ties_and_decision_flags(oracle):
    v = np.full((48, 48, 48), 5.0)
    g = oracle.GridView(v, 0.5, (-11.75,) * 3, mode=1)
    for xyz, bonds, rot, lid in tiny_ligands(3, 12, 20, 2, 33):
        p = _int_params(oracle)
        r = oracle.dock_ligand(g, xyz, bonds, rot, lid, p)
        n = len(xyz)
        assert (r["restart_score"] == 5.0 * n).all() and (r["score_lo"] == r["score_hi"]).all()
        assert (r["align_idx"] == 0).all() and (r["post_idx"] == 0).all() and (r["torsion_idx"] == 0).all()
        # every alternative ties, and ties go to the lowest index: the choice is the only one
        assert (r["align_robust"] == 1).all() and (r["post_robust"] == 1).all() and (r["tors_robust"] == 1).all()
        # forcing a higher index loses the tie
        f = oracle.dock_ligand(g, xyz, bonds, rot, lid, p, forced_align=[3] * 3, forced_post=[0] * 3,
                               forced_tors=np.full(3 * len(rot), 5))
        assert (f["align_possible"] == 0).all() and (f["post_possible"] == 1).all()
        assert (f["tors_possible"][f["tors_robust_valid"] > 1] == 0).all()


def test_dock_integer_grid_alignment_is_the_brute_force_best_pose(oracle):
    pk = small_pocket(G=40, h=0.5, R=8.0, noise=0.3).integer(1000)
    g = oracle.GridView.of(pk, nearest=True)
    N = 6
    for xyz, bonds, _, lid in tiny_ligands(3, 12, 20, 0, 15):
        r = oracle.dock_ligand(g, xyz, bonds, np.zeros((0, 2), np.int32), lid,
                               _params(oracle, restarts=3, align_steps=N, post_align=0))
        assert (r["restart_score"] == np.rint(r["restart_score"])).all()
        for rr in range(3):
            S = oracle.restart_rotation(lid, 11, rr)
            centre = pk.origin + pk.spacing * (np.array(pk.dims) - 1) / 2
            X = xyz.astype(np.float64)
            P = centre + (X - X.mean(0)) @ S.T
            c = P.mean(0)
            scores = []
            for i in range(N):
                for j in range(N):
                    R = Rotation.from_euler("y", 2 * math.pi * j / N) * Rotation.from_euler("x", 2 * math.pi * i / N)
                    scores.append(lib_nearest(pk.values, pk.spacing, pk.origin, c + R.apply(P - c)).sum())
            assert r["align_idx"][rr] == int(np.argmax(scores))      # first maximum: ties to the lowest
            assert r["restart_score"][rr] == max(scores)


def test_dock_integer_grid_flags_agree_with_forced_replay(oracle):
    """Where a decision is the only possible one, replaying it is possible and any other choice
    is not; a free run's own choices are always possible."""
    pk = small_pocket(G=40, h=0.5, R=8.0, noise=0.3).integer(1000)
    g = oracle.GridView.of(pk, nearest=True)
    for xyz, bonds, rot, lid in tiny_ligands(3, 14, 22, 3, 16):
        p = _int_params(oracle, restarts=4)
        r = oracle.dock_ligand(g, xyz, bonds, rot, lid, p)
        assert (r["align_possible"] == 1).all() and (r["post_possible"] == 1).all() and (r["tors_possible"] == 1).all()
        assert (r["align_robust"] >= 0).all() and (r["tors_robust"] >= 0).all()
        other = (r["align_idx"] + 1) % 36
        f = oracle.dock_ligand(g, xyz, bonds, rot, lid, p, forced_align=other, forced_post=r["post_idx"],
                               forced_tors=r["torsion_idx"].reshape(-1))
        robust = r["align_robust"] == 1
        assert (f["align_possible"][robust] == 0).all()
