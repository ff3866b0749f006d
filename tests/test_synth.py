"""The seeded synthetic inputs follow the recipe the design states (CPU).

These are input-generator checks, not parity: prefix stability, bond geometry, clash-free starts,
rotatable bonds that are bridges with at least two atoms per side, the pocket field, the integer
pocket, and the tiled databases and arrival streams of the plateau and serving runs.
"""
import networkx as nx
import numpy as np

from paper_2209_05069_gb300 import synth


def test_database_prefixes_are_stable():
    w = synth.WORKLOADS["uneven"]
    a, b = synth.make_db(w, 60), synth.make_db(w, 25)
    assert np.array_equal(a.atom_off[:26], b.atom_off) and np.array_equal(a.xyz[:b.atom_off[-1]], b.xyz)
    assert np.array_equal(a.rot[:b.rot_off[-1]], b.rot) and np.array_equal(a.ids[:25], b.ids)


def test_ligand_geometry_and_rotatable_bonds():
    w = synth.WORKLOADS["uneven"]
    db = synth.make_db(w, 80)
    for l in range(db.n_lig):
        xyz, bonds, rot, _ = db.ligand(l)
        n = len(xyz)
        assert 10 <= n <= 80 and len(rot) <= 20
        d = np.linalg.norm(xyz[bonds[:, 0]] - xyz[bonds[:, 1]], axis=1)
        assert np.allclose(d, 1.5, atol=1e-4)                       # bond length
        G = nx.Graph(list(map(tuple, bonds)))
        G.add_nodes_from(range(n))
        assert nx.is_tree(G) and max(dict(G.degree()).values()) <= 4
        far = dict(nx.all_pairs_shortest_path_length(G))
        for i in range(n):                                          # clash-free start beyond 1-3
            for j in range(i + 1, n):
                if far[i][j] > 2:
                    assert np.linalg.norm(xyz[i] - xyz[j]) >= 2.0 - 1e-4
        for a, b in rot:                                            # bridges, >= 2 atoms per side
            H = G.copy()
            H.remove_edge(int(a), int(b))
            side_b = nx.node_connected_component(H, int(b))
            assert int(a) not in side_b and 2 <= len(side_b) <= n - 2
            assert len(side_b) <= n - len(side_b)                   # the smaller side moves


def test_pocket_field_and_integer_pocket():
    w = synth.WORKLOADS["tiny"]
    pk = synth.workload_pocket(w)
    nz, ny, nx_ = pk.values.shape
    assert (nx_, ny, nz) == (w.grid,) * 3
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx_), indexing="ij")
    x = pk.origin[0] + pk.spacing * i
    y = pk.origin[1] + pk.spacing * j
    z = pk.origin[2] + pk.spacing * k
    r = np.sqrt(x ** 2 + y ** 2 + z ** 2)
    inside = r < w.radius
    base = 1.0 - (r / w.radius) ** 2
    assert (pk.values[~inside] == 0).all()
    excess = pk.values[inside] - base[inside]
    assert excess.min() >= -1e-6 and excess.max() <= w.noise + 1e-6   # 1 - (r/R)^2 + U(0, noise)
    q = pk.integer(1000)
    assert (q.values == np.rint(q.values)).all() and q.values.max() <= 32767
    assert np.abs(q.values - 1000 * pk.values.astype(np.float64)).max() <= 0.5


def test_tiled_database_and_arrivals():
    pool = synth.make_db(synth.WORKLOADS["uneven"], 7)
    db = synth.tile_db(pool, 20, first_id=100)
    assert db.n_lig == 20 and list(db.ids) == list(range(100, 120))
    for l in range(20):
        assert np.array_equal(db.ligand(l)[0], pool.ligand(l % 7)[0])
    t = synth.poisson_arrivals(1000.0, 20000, seed=3)
    gaps = np.diff(t)
    assert (gaps >= 0).all() and abs(gaps.mean() - 1e-3) < 5e-5     # mean inter-arrival 1/rate
