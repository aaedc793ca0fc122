"""Pins of the oracle's initial-structure generation from a triangular mesh
and of its velocity quench ("Initial structure generation": proteins on the
mesh's vertices and edges, lipids sampled uniformly on its faces, a minimum
distance enforced, then a velocity quench), checked by routes other than the
oracle's own code: Euler's formula, geometry of the inputs, brute-force
distances and the statistics of uniform sampling."""
import math

import numpy as np
import pytest

import oracle
from synth import membranes as M

A_LIP = math.sqrt(3.0) / 2.0 * 1.12 ** 2


def build(v, f, **kw):
    return oracle.mesh_build(v, f, **kw)


def chains(out, nl, nv):
    """Junction pairs joined by each chain, read from the bond list."""
    adj = {}
    for a, b in out["bonds"].tolist():
        adj.setdefault(a, []).append(b)
        adj.setdefault(b, []).append(a)
    pairs = []
    for j in range(nl, nl + nv):
        for nxt in adj.get(j, []):
            prev, cur = j, nxt
            while cur >= nl + nv:                      # walk the beads
                a, b = adj[cur]
                prev, cur = cur, (b if a == prev else a)
            if j < cur:
                pairs.append((j - nl, cur - nl))
    return pairs


def test_closed_mesh_edges_once_each_and_euler():
    v, f = M.icosphere_mesh(3, 10.0)
    beads = 3
    out = build(v, f, beads=beads, d_min=0.0, d_ll=0.0)
    typ = out["type"]
    nl, nv = int((typ == 0).sum()), int((typ == 1).sum())
    ne = int((typ == 2).sum()) // beads
    assert nv == len(v) and nv - ne + len(f) == 2                  # Euler: V - E + F = 2
    assert len(out["bonds"]) == ne * (beads + 1)
    mesh_edges = {tuple(sorted((int(f[t, i]), int(f[t, (i + 1) % 3])))) for t in range(len(f)) for i in range(3)}
    got = chains(out, nl, nv)
    assert sorted(got) == sorted(mesh_edges) and len(set(got)) == len(got)
    # ids: lipids, then junctions, then spectrin
    assert (typ[:nl] == 0).all() and (typ[nl:nl + nv] == 1).all() and (typ[nl + nv:] == 2).all()


def test_open_mesh_single_triangle():
    v = np.array([[0.0, 0.0, 0.0], [30.0, 0.0, 0.0], [0.0, 20.0, 0.0]])
    f = np.array([[0, 1, 2]], np.int32)
    out = build(v, f, beads=2, d_min=0.0, d_ll=0.0, offset=0.0)
    typ = out["type"]
    assert (typ == 1).sum() == 3 and (typ == 2).sum() == 3 * 2 and len(out["bonds"]) == 3 * 3
    lam = 0.5 * 30.0 * 20.0 / A_LIP
    assert (typ == 0).sum() in (math.floor(lam), math.floor(lam) + 1)


def test_samples_lie_in_their_triangles_and_are_uniform():
    """One large triangle: every sample has non-negative barycentric
    coordinates, and the share of samples in the medial sub-triangle (a
    quarter of the area) is 1/4 within four standard deviations; the
    director is the unit normal of the face (here +z)."""
    a, b, c = np.array([0.0, 0.0, 0.0]), np.array([200.0, 0.0, 0.0]), np.array([40.0, 150.0, 0.0])
    out = build(np.array([a, b, c]), np.array([[0, 1, 2]], np.int32), beads=0, d_min=0.0, d_ll=0.0, offset=0.0,
                seed=11)
    lip = out["type"] == 0
    p, n = out["pos"][lip], out["ori"][lip]
    T = np.column_stack([b - a, c - a])[:2]
    lam = np.linalg.solve(T, (p - a)[:, :2].T).T
    assert (lam >= -1e-12).all() and (lam.sum(1) <= 1 + 1e-12).all()
    inner = (lam[:, 0] <= 0.5) & (lam[:, 1] <= 0.5) & (lam.sum(1) >= 0.5)
    share, N = inner.mean(), len(p)
    assert abs(share - 0.25) < 4 * math.sqrt(0.25 * 0.75 / N), share
    assert np.allclose(n, [0.0, 0.0, 1.0])


def test_face_counts_follow_the_area():
    """Without drops, each face holds floor(A/a) or floor(A/a) + 1 lipids and
    the total is the expected sum within four standard deviations of the
    Bernoulli rounding."""
    v, f = M.icosphere_mesh(6, 25.0)
    out = build(v, f, beads=0, d_min=0.0, d_ll=0.0, seed=3)
    e1, e2 = v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]]
    lam = 0.5 * np.linalg.norm(np.cross(e1, e2), axis=1) / A_LIP
    nl = int((out["type"] == 0).sum())
    frac = lam - np.floor(lam)
    assert np.floor(lam).sum() <= nl <= np.ceil(lam).sum()
    assert abs(nl - lam.sum()) < 4 * math.sqrt((frac * (1 - frac)).sum()) + 1


def test_directors_outward_and_junctions_inside():
    """Lipid directors are unit and point outward; junctions sit `offset`
    inside the surface along the vertex normal: exactly radial on an
    octahedron (every vertex's faces are symmetric about its radius), and
    radial to the mesh's irregularity on an icosphere."""
    R, off = 15.0, 1.0
    v, f = M.icosphere_mesh(5, R)
    out = build(v, f, beads=2, offset=off)
    typ, p, n = out["type"], out["pos"], out["ori"]
    lip = typ == 0
    assert np.allclose(np.linalg.norm(n[lip], axis=1), 1.0)
    assert (np.einsum("ij,ij->i", n[lip], p[lip]) > 0).all()
    rj = np.linalg.norm(p[typ == 1], axis=1)
    assert np.abs(rj - (R - off)).max() < 1e-3
    ov = np.array([[R, 0, 0], [-R, 0, 0], [0, R, 0], [0, -R, 0], [0, 0, R], [0, 0, -R]], float)
    of = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4], [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]], np.int32)
    out = build(ov, of, beads=0, offset=off)
    pj = out["pos"][out["type"] == 1]
    assert np.abs(pj - ov * (R - off) / R).max() < 1e-12


def test_chain_spacing_and_rest_length():
    v, f = M.icosphere_mesh(2, 12.0)
    beads, slack = 4, 1.03
    out = build(v, f, beads=beads, slack=slack)
    p = out["pos"]
    for (a, b), r0 in zip(out["bonds"].tolist(), out["r0"]):
        d = np.linalg.norm(p[a] - p[b])
        assert r0 == pytest.approx(slack * d, rel=1e-12)               # evenly spaced beads


def test_minimum_distances_hold():
    v, f = M.icosphere_mesh(4, 12.0)
    d_min, d_ll = 1.05, 0.6
    out = build(v, f, beads=3, offset=1.0, d_min=d_min, d_ll=d_ll, seed=7)
    typ, p = out["type"], out["pos"]
    L, P = p[typ == 0], p[typ != 0]
    dlp = np.linalg.norm(L[:, None, :] - P[None, :, :], axis=2)
    assert dlp.min() >= d_min
    dll = np.linalg.norm(L[:, None, :] - L[None, :, :], axis=2) + np.eye(len(L)) * 1e9
    assert dll.min() >= d_ll
    # everything dropped when the protein distance exceeds the mesh
    none = build(v, f, beads=3, d_min=100.0, d_ll=0.0)
    assert (none["type"] == 0).sum() == 0


def test_quench_separates_an_overlapping_pair():
    """Two lipids at 0.5 sigma (deep in the repulsive core) move apart under
    the quench and stop near the minimum of the pair potential; every step
    lowers the energy."""
    pos = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]])
    ori = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]])
    mem = M.Membrane(pos, np.zeros((2, 3)), ori, np.zeros((2, 3)), np.zeros(2, np.uint8),
                     np.arange(2, dtype=np.uint32), np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(0),
                     (0.0, 0.0, 0.0), (0, 0, 0), 1, 0.0)
    s = oracle.OracleSystem(oracle.model(), oracle.run(kT=0.0, n_centroids=1, seed=0))
    s.load(mem)
    s.init_cells()
    e_prev = s.compute_forces()[0]
    for _ in range(6):
        fmax = s.quench(50, 0.01)
        e = s.compute_forces()[0]
        assert e <= e_prev + 1e-12
        e_prev = e
    r = np.linalg.norm(np.diff(s.state()["pos"], axis=0))
    assert abs(r - 2.0 ** (1.0 / 6.0)) < 1e-9 and e_prev == pytest.approx(-1.0, abs=1e-12) and fmax < 1e-8
    assert np.abs(s.state()["vel"]).max() == 0.0


# --------------------------------------------------------------------------- bilayer proteins on the mesh

def test_membrane_proteins_on_vertices_edges_and_faces():
    """Glycophorin on every vertex (at the vertex, along the vertex normal),
    immobile band-3 on every edge (at its midpoint), mobile band-3 among the
    face samples; the bilayer first in id order, then junctions and
    spectrin ("Initial structure generation")."""
    R = 12.0
    v, f = M.icosphere_mesh(3, R)
    beads = 3
    out = build(v, f, beads=beads, glycophorin=1, band3_edges=1, band3_fraction=0.25, seed=4)
    typ, p, n = out["type"], out["pos"], out["ori"]
    nv = len(v)
    ne = nv + len(f) - 2                                            # Euler
    cnt = np.bincount(typ, minlength=5)
    assert cnt[4] == nv and cnt[1] == nv and cnt[2] == ne * beads
    nb3_face = cnt[3] - ne
    nface = cnt[0] + nb3_face
    assert abs(nb3_face - 0.25 * nface) < 5 * math.sqrt(nface * 0.25 * 0.75)
    nbil = cnt[0] + cnt[3] + cnt[4]
    assert np.isin(typ[:nbil], (0, 3, 4)).all() and np.isin(typ[nbil:], (1, 2)).all()
    gly = np.flatnonzero(typ == 4)
    assert np.array_equal(p[gly], v)                                # exactly the vertices, in order
    assert np.allclose(np.linalg.norm(n[gly], axis=1), 1.0)
    assert (np.einsum("ij,ij->i", n[gly], p[gly]) > 0).all()        # outward
    # the edges' band-3: one per mesh edge, at its midpoint
    e3 = gly[-1] + 1 + np.arange(ne)
    assert (typ[e3] == 3).all()
    mid = {tuple(np.round((v[a] + v[b]) * 0.5, 12)) for a, b in
           {tuple(sorted((int(f[t, i]), int(f[t, (i + 1) % 3])))) for t in range(len(f)) for i in range(3)}}
    assert {tuple(np.round(x, 12)) for x in p[e3]} == mid
    assert np.allclose(np.linalg.norm(n[e3], axis=1), 1.0)
    assert (np.einsum("ij,ij->i", n[e3], p[e3]) > 0).all()


def test_anchor_bonds_start_at_rest_and_join_the_right_partners():
    """Each glycophorin is bonded to the junction `offset` beneath it, each
    edge band-3 to the middle bead of its own edge's chain; every anchor's
    rest length is its length at construction, with constant kb_anchor."""
    R, off, beads = 12.0, 1.0, 3
    v, f = M.icosphere_mesh(2, R)
    out = build(v, f, beads=beads, offset=off, glycophorin=1, band3_edges=1, kb_anchor=37.0, d_min=0.0, d_ll=0.0)
    typ, p = out["type"], out["pos"]
    bonds, r0, kb = out["bonds"], out["r0"], out["kb"]
    bil = np.isin(typ, (0, 3, 4))
    anchor = bil[bonds[:, 0]] != bil[bonds[:, 1]]
    nv = len(v)
    ne = nv + len(f) - 2
    assert anchor.sum() == nv + ne and (kb[anchor] == 37.0).all() and (kb[~anchor] == 100.0).all()
    # the anchors follow the chains' bonds
    assert not anchor[: (~anchor).sum()].any()
    for (a, b), r in zip(bonds[anchor].tolist(), r0[anchor]):
        assert r == pytest.approx(np.linalg.norm(p[a] - p[b]), rel=1e-15)
        if typ[a] == 4:
            assert typ[b] == 1
            assert r == pytest.approx(off, rel=1e-12)               # the junction beneath the vertex
        else:
            assert typ[a] == 3 and typ[b] == 2
            # beads = 3: the middle bead is the chain's centre, below the edge's midpoint
            assert r == pytest.approx(off, abs=0.2)
    # each edge band-3's bead is the middle one of the chain joining that
    # edge's two junctions
    nbil = int(bil.sum())
    chain_adj = {}
    for x, y in bonds[~anchor].tolist():
        chain_adj.setdefault(x, []).append(y)
        chain_adj.setdefault(y, []).append(x)
    for (a, b) in bonds[anchor].tolist():
        if typ[a] != 3:
            continue
        ends, steps = [], []
        for first in chain_adj[b]:
            prev, cur, k = b, first, 1
            while typ[cur] == 2:
                nxt = [q for q in chain_adj[cur] if q != prev]
                prev, cur, k = cur, nxt[0], k + 1
            ends.append(cur - nbil)                                  # junction id -> vertex index
            steps.append(k)
        assert steps == [2, 2]                                       # the middle of three beads
        assert np.array_equal(p[a], (v[ends[0]] + v[ends[1]]) * 0.5)


def test_face_band3_do_not_move_the_samples():
    """The band-3 share only relabels face samples: positions and
    directors are those of the lipid-only build, and the shares 0 and 1
    give all lipids and all band-3."""
    v, f = M.icosphere_mesh(3, 10.0)
    a = build(v, f, beads=2, seed=9)
    b = build(v, f, beads=2, seed=9, band3_fraction=0.4)
    assert np.array_equal(a["pos"], b["pos"]) and np.array_equal(a["ori"], b["ori"])
    face = a["type"] == 0
    assert set(np.unique(b["type"][face]).tolist()) == {0, 3}
    c = build(v, f, beads=2, seed=9, band3_fraction=1.0)
    assert (c["type"][face] == 3).all()


def test_minimum_distance_holds_against_the_surface_proteins():
    v, f = M.icosphere_mesh(4, 12.0)
    d_min = 0.9
    out = build(v, f, beads=3, d_min=d_min, d_ll=0.3, glycophorin=1, band3_edges=1, band3_fraction=0.1, seed=2)
    typ, p = out["type"], out["pos"]
    nv = len(v)
    ne = nv + len(f) - 2
    nbil = int(np.isin(typ, (0, 3, 4)).sum())
    face = np.arange(nbil - nv - ne)                                 # the kept face samples
    prot = np.arange(nbil - nv - ne, len(typ))                       # every protein particle
    d = np.linalg.norm(p[face][:, None, :] - p[prot][None, :, :], axis=2)
    assert d.min() >= d_min


def test_band3_on_edges_needs_beads():
    v, f = M.icosphere_mesh(1, 10.0)
    with pytest.raises(ValueError):
        build(v, f, beads=0, band3_edges=1)
