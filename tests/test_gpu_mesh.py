"""Initial structure from a triangular mesh and the velocity quench on the
GPU ("Initial structure generation"), through the C ABI, against the FP64
oracle.

The builder draws its random variates from Philox4x32-10 counted by (face,
sample) and writes its FP64 arithmetic operation by operation, so every
output array -- positions, directors, types, bonds, rest lengths -- must
equal the oracle's bit for bit.  The quench runs on FP32 forces and is not a
smooth map (a velocity is zeroed wherever v.F changes sign, and capped
where it is large), so FP32 force errors flip single decisions: after 30
steps on the 3k-particle vesicle positions agree to RMS <= 1e-3 sigma
(measured 1.5e-4) and the potential energy to 1e-3 relative, and the
quench's effect is checked directly: the largest force falls.
"""
import numpy as np
import pytest

import oracle
from synth import membranes as M

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_1701_02059_gb300")
from paper_1701_02059_gb300 import _native  # noqa: E402

MESHES = {
    "icosphere-f4": (lambda: M.icosphere_mesh(4, 12.0), dict(beads=3, seed=5)),
    "icosphere-f8": (lambda: M.icosphere_mesh(8, 22.0), dict(beads=4, d_min=0.8, d_ll=0.2, seed=9)),
    "biconcave-600": (lambda: M.biconcave_mesh(600, 20_000), dict(beads=4, seed=2)),
    "triangle-open": (lambda: (np.array([[0.0, 0.0, 0.0], [30.0, 0.0, 0.0], [0.0, 20.0, 0.0]]),
                               np.array([[0, 1, 2]], np.int32)), dict(beads=2, d_min=0.0, d_ll=0.0, offset=0.0)),
    # the bilayer's proteins: glycophorin on the vertices, band-3 on the
    # edges and among the face samples, anchored to the network
    "icosphere-f6-proteins": (lambda: M.icosphere_mesh(6, 14.0),
                              dict(beads=3, seed=6, glycophorin=1, band3_edges=1, band3_fraction=0.1, kb_anchor=40.0)),
    "biconcave-600-proteins": (lambda: M.biconcave_mesh(600, 20_000),
                               dict(beads=4, seed=3, glycophorin=1, band3_edges=1, band3_fraction=0.05)),
    "triangle-open-band3": (lambda: (np.array([[0.0, 0.0, 0.0], [30.0, 0.0, 0.0], [0.0, 20.0, 0.0]]),
                                     np.array([[0, 1, 2]], np.int32)), dict(beads=1, band3_edges=1, band3_fraction=0.5)),
}


@pytest.mark.parametrize("name", list(MESHES))
def test_mesh_build_equals_oracle(name):
    make, kw = MESHES[name]
    v, f = make()
    got = G.mesh_build(v, f, **kw)
    want = oracle.mesh_build(v, f, **kw)
    for k in ("pos", "ori", "type", "bonds", "r0", "kb"):
        assert got[k].shape == want[k].shape, k
        assert np.array_equal(got[k], want[k]), f"{k}: {np.flatnonzero(got[k].ravel() != want[k].ravel())[:5]}"


def test_mesh_build_rejects_bad_meshes():
    v, f = M.icosphere_mesh(2, 10.0)
    bad = f.copy()
    bad[3, 1] = len(v)
    with pytest.raises(G.OrbcError) as e:
        G.mesh_build(v, bad)
    assert e.value.code == _native.ORBC_E_ARG
    deg = f.copy()
    deg[0] = [deg[0, 0], deg[0, 0], deg[0, 1]]
    with pytest.raises(G.OrbcError) as e:
        G.mesh_build(v, deg)
    assert e.value.code == _native.ORBC_E_ARG
    for kw in (dict(beads=0, band3_edges=1), dict(band3_fraction=1.5), dict(kb_anchor=-1.0)):
        with pytest.raises(G.OrbcError) as e:
            G.mesh_build(v, f, **kw)
        assert e.value.code == _native.ORBC_E_ARG, kw


def _membrane(out, kT=0.0, K=None):
    n = len(out["type"])
    return M.Membrane(out["pos"], np.zeros((n, 3)), np.where(np.isin(out["type"], M.BILAYER)[:, None], out["ori"], 0.0),
                      np.zeros((n, 3)), out["type"], np.arange(n, dtype=np.uint32), out["bonds"], out["r0"],
                      out["kb"], np.zeros(3), np.zeros(3, np.int32), K or max(1, n // 61), kT)


def test_quench_matches_oracle_and_removes_collisions():
    v, f = M.icosphere_mesh(6, 14.0)
    out = G.mesh_build(v, f, beads=3, seed=3)
    mem = _membrane(out)
    g = G.System(G.make_params(kT=0.0, n_centroids=mem.n_centroids, seed=0))
    g.load_membrane(mem)
    g.init_cells()
    g.compute_forces()
    f0 = np.linalg.norm(g.forces()[0], axis=1).max()
    fm = g.quench(30, 0.01)
    o = oracle.OracleSystem(oracle.model(), oracle.run(kT=0.0, n_centroids=mem.n_centroids, seed=0))
    o.load(mem)
    o.init_cells()
    fo = o.quench(30, 0.01)
    sg, so = g.state(), o.state()
    rms = np.sqrt(((sg["pos"] - so["pos"]) ** 2).sum(1).mean())
    assert rms <= 1e-3, rms
    eg, eo = g.compute_forces(energies=True), o.compute_forces()
    assert abs(eg[0] + eg[1] - eo[0] - eo[1]) <= 1e-3 * abs(eo[0] + eo[1])
    assert fm < 0.2 * f0 and fo < 0.2 * f0
    assert np.abs(sg["vel"]).max() == 0.0 and np.abs(sg["angvel"]).max() == 0.0 and sg["step"] == 0
    g.close()


def test_red_cell_from_a_mesh():
    """The biconcave cell of the 4M workload built the paper's way: a
    33,000-vertex triangulation, lipids sampled on its faces.  Counts follow
    the face areas, the minimum distances hold on sampled lipids, and the
    system initialises and quenches."""
    from scipy.spatial import cKDTree
    v, f = M.biconcave_mesh(33_000)
    out = G.mesh_build(v, f, beads=4, seed=2)
    typ = out["type"]
    nl, nv, ns = int((typ == 0).sum()), int((typ == 1).sum()), int((typ == 2).sum())
    assert nv == 33_000 and ns == 4 * (3 * nv - 6) and len(out["bonds"]) == 5 * (3 * nv - 6)
    e1, e2 = v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]]
    expect = 0.5 * np.linalg.norm(np.cross(e1, e2), axis=1).sum() / (np.sqrt(3) / 2 * 1.12 ** 2)
    assert 0.85 * expect < nl < expect
    pos = out["pos"]
    rng = np.random.default_rng(0)
    sample = rng.choice(nl, 20_000, replace=False)
    dl, _ = cKDTree(pos[:nl]).query(pos[sample], k=2)
    assert dl[:, 1].min() >= 0.2
    dp, _ = cKDTree(pos[nl:]).query(pos[sample], k=1)
    assert dp.min() >= 0.8
    mem = _membrane(out, K=65_536)
    g = G.System(G.make_params(kT=0.0, n_centroids=65_536, seed=2))
    g.load_membrane(mem)
    g.init_cells()
    g.compute_forces()
    f0 = np.linalg.norm(g.forces()[0], axis=1).max()
    fm = g.quench(20, 0.01)
    assert np.isfinite(fm) and fm < f0
    g.close()


def test_protein_set_from_a_mesh_quenches_and_runs_like_the_oracle():
    """The full protein set built the paper's way (glycophorin on the
    vertices, immobile band-3 on the edges, mobile band-3 on the faces, all
    anchored): quenched on the GPU and in the oracle, then 20 Langevin steps
    from the oracle's quenched state agree within the FP32-force tolerance."""
    v, f = M.icosphere_mesh(6, 14.0)
    out = G.mesh_build(v, f, beads=3, seed=8, glycophorin=1, band3_edges=1, band3_fraction=0.1)
    mem = _membrane(out)
    g = G.System(G.make_params(kT=0.0, n_centroids=mem.n_centroids, seed=0))
    g.load_membrane(mem)
    g.init_cells()
    g.compute_forces()
    f0 = np.linalg.norm(g.forces()[0], axis=1).max()
    fm = g.quench(30, 0.01)
    o = oracle.OracleSystem(oracle.model(), oracle.run(kT=0.0, n_centroids=mem.n_centroids, seed=0))
    o.load(mem)
    o.init_cells()
    fo = o.quench(30, 0.01)
    assert fm < 0.2 * f0 and fo < 0.2 * f0
    so = o.state()
    q = mem.copy()
    q.pos, q.ori, q.kT = so["pos"], so["ori"], 0.2
    a = G.System(G.make_params(kT=0.2, n_centroids=mem.n_centroids, seed=4))
    a.load_membrane(q)
    b = oracle.OracleSystem(oracle.model(), oracle.run(kT=0.2, n_centroids=mem.n_centroids, seed=4))
    b.load(q)
    a.init_cells()
    b.init_cells()
    a.integrate(20)
    b.integrate(20)
    rms = np.sqrt(((a.state()["pos"] - b.state()["pos"]) ** 2).sum(1).mean())
    assert rms <= 1e-5, rms
    g.close()
    a.close()
