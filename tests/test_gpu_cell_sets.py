"""Separate Voronoi cell set for the proteins of a detached cytoskeleton on
the GPU (through the C ABI) against the FP64 oracle.

Tolerances as for the shared cells: cells, permutation, centroids, radii,
neighbouring cells and the pair set bit-exact; forces e_F <= 1e-5 (FP32
forces) and <= 1e-8 (FP64); 100-step trajectories <= 1e-5 sigma RMS (FP32
forces) and <= 1e-9 sigma (FP64).  Between the two cell layouts on the GPU
the forces, and so the trajectories, are bit-identical: the pair set does
not depend on the cells and the force sums are exact integers (the energies
agree to 1e-12: their FP64 per-particle partials follow the rows' order).
"""
import numpy as np
import pytest

import oracle
from synth import membranes as M

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_1701_02059_gb300")
from paper_1701_02059_gb300 import _native  # noqa: E402

KP = 12


def partly_detached():
    return M.vesicle(3000, 5, f=2, chain_beads=5, n_centroids=50, detach_upper=4.0)


def fully_detached():
    return M.vesicle(3000, 7, f=2, chain_beads=5, n_centroids=50, net_offset=5.0)


WORKLOADS = {"partly": partly_detached, "fully": fully_detached}


def pair(mem, kp=KP, precision=0, **kw):
    g = G.System(G.make_params(kT=mem.kT, n_centroids=mem.n_centroids, n_protein_centroids=kp, box=mem.box,
                               periodic=mem.periodic, seed=0, precision=precision, **kw))
    g.load_membrane(mem)
    m = oracle.model(box=mem.box, periodic=mem.periodic)
    o = oracle.OracleSystem(m, oracle.run(kT=mem.kT, n_centroids=mem.n_centroids, n_protein_centroids=kp, seed=0,
                                          **kw))
    o.load(mem)
    return g, m, o


def assert_cells_equal(g, o):
    a, b = g.cells(), o.cells()
    for k in ("cell_of_id", "slot_ids", "centroids", "start", "radius", "adj_ptr", "adj"):
        assert a[k].shape == b[k].shape, k
        assert np.array_equal(a[k], b[k]), f"{k} differs at {np.flatnonzero(a[k].ravel() != b[k].ravel())[:5]}"


def sorted_pairs(p):
    p = np.sort(np.asarray(p, np.int64), axis=1)
    return p[np.lexsort((p[:, 1], p[:, 0]))].astype(np.uint32)


def force_error(Fg, Fo):
    frms = np.sqrt((Fo ** 2).sum(1).mean())
    return (np.linalg.norm(Fg - Fo, axis=1) / np.maximum(np.linalg.norm(Fo, axis=1), frms)).max(), frms


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_cells_pairs_and_forces_match_oracle(name):
    mem = WORKLOADS[name]()
    g, m, o = pair(mem)
    g.init_cells()
    o.init_cells()
    assert_cells_equal(g, o)
    c = g.cells()
    lip = mem.type == 0
    assert (c["cell_of_id"][lip] < mem.n_centroids).all() and (c["cell_of_id"][~lip] >= mem.n_centroids).all()
    assert np.array_equal(g.pairs(), sorted_pairs(o.pairs()))
    g.compute_forces()
    o.compute_forces()
    Fg, Tg = g.forces()
    Fo, To = o.forces()
    ef, frms = force_error(Fg, Fo)
    assert ef <= 1e-5, ef
    g.close()


@pytest.mark.parametrize("precision", [G.F32_FORCE_F64_STATE, G.F64_ALL])
def test_trajectory_matches_oracle_and_cells_stay_exact(precision):
    mem = partly_detached()
    g, m, o = pair(mem, precision=precision)
    g.init_cells()
    o.init_cells()
    g.integrate(100)
    o.integrate(100)
    sg, so = g.state(), o.state()
    assert sg["step"] == so["step"] == 100
    rms = np.sqrt(((sg["pos"] - so["pos"]) ** 2).sum(1).mean())
    assert rms <= (1e-9 if precision == G.F64_ALL else 1e-5), rms
    # the GPU's own state: each particle in the nearest centroid of its set,
    # and the pair set equal to the O(N^2) search
    c = g.cells()
    KL = mem.n_centroids
    lip = mem.type == 0
    want_l = oracle.assign_brute(sg["pos"][lip], c["centroids"][:KL], mem.box, mem.periodic)
    want_p = oracle.assign_brute(sg["pos"][~lip], c["centroids"][KL:], mem.box, mem.periodic) + KL
    assert np.array_equal(c["cell_of_id"][lip], want_l) and np.array_equal(c["cell_of_id"][~lip], want_p)
    brute = sorted_pairs(oracle.pairs_brute(m, sg["pos"], mem.type, mem.id, mem.bonds))
    assert np.array_equal(g.pairs(), brute)
    g.close()


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_separate_and_shared_cells_give_identical_trajectories(name):
    mem = WORKLOADS[name]()
    a = G.System(G.make_params(kT=mem.kT, n_centroids=mem.n_centroids, n_protein_centroids=KP, seed=3))
    b = G.System(G.make_params(kT=mem.kT, n_centroids=mem.n_centroids, seed=3))
    for s in (a, b):
        s.load_membrane(mem)
        s.init_cells()
    ea, eb = a.compute_forces(energies=True), b.compute_forces(energies=True)
    Fa, Ta = a.forces()
    Fb, Tb = b.forces()
    assert np.array_equal(Fa, Fb) and np.array_equal(Ta, Tb)
    # energies: FP64 per-particle partials summed in the order of each
    # layout's neighbour rows
    assert np.allclose(ea, eb, rtol=1e-12, atol=0)
    a.integrate(50)
    b.integrate(50)
    sa, sb = a.state(), b.state()
    for k in ("pos", "vel", "ori", "angvel"):
        assert np.array_equal(sa[k], sb[k]), k
    # the detached proteins widen the shared lipid cells, not their own
    Ra, Rb = a.cells()["radius"], b.cells()["radius"]
    assert Ra[: mem.n_centroids].max() < Rb.max()
    a.close()
    b.close()


def test_separate_cells_refuse_mixed_ids_lipid_bonds_and_the_arena():
    mem = partly_detached()
    p = G.make_params(kT=mem.kT, n_centroids=mem.n_centroids, n_protein_centroids=KP)
    # ids not type-major
    g = G.System(p)
    ids = mem.id.copy()
    ids[[0, -1]] = ids[[-1, 0]]
    g.set_particles(mem.pos, mem.vel, mem.ori, mem.angvel, mem.type, ids)
    with pytest.raises(G.OrbcError) as e:
        g.init_cells()
    assert e.value.code == _native.ORBC_E_ARG
    g.close()
    # a bond that ends on a lipid
    g = G.System(p)
    g.set_particles(mem.pos, mem.vel, mem.ori, mem.angvel, mem.type, mem.id)
    bonds = np.vstack([mem.bonds, [[0, mem.n - 1]]]).astype(np.int32)
    g.set_bonds(bonds, np.append(mem.r0, 1.0), np.append(mem.kb, 1.0))
    with pytest.raises(G.OrbcError) as e:
        g.init_cells()
    assert e.value.code == _native.ORBC_E_ARG
    g.close()
    arena = G.Arena(1 << 30)
    with pytest.raises(G.OrbcError):
        arena.admit(p, mem, 10)
    arena.close()


# --------------------------------------------------------------------------- full-size 4M cell, detached network

def test_rbc_detached_separate_cells_sampled():
    """The 4,000,000-particle cell with its network 6 sigma inside: with a
    protein cell set of its own, sampled particles of each set sit in the
    nearest centroid of their set, and steps run clean."""
    mem = M.rbc_4m_detached()
    kp = 8192
    g = G.System(G.make_params(kT=mem.kT, n_centroids=mem.n_centroids, n_protein_centroids=kp, seed=2))
    g.load_membrane(mem)
    g.init_cells()
    g.integrate(3)
    st = g.state()
    c = g.cells()
    KL = mem.n_centroids
    rng = np.random.default_rng(5)
    lip = np.flatnonzero(mem.type == 0)
    pro = np.flatnonzero(mem.type != 0)
    il, ip = rng.choice(lip, 800, replace=False), rng.choice(pro, 800, replace=False)
    assert np.array_equal(c["cell_of_id"][il], oracle.assign_brute(st["pos"][il], c["centroids"][:KL], mem.box,
                                                                   mem.periodic))
    assert np.array_equal(c["cell_of_id"][ip], oracle.assign_brute(st["pos"][ip], c["centroids"][KL:], mem.box,
                                                                   mem.periodic) + KL)
    assert np.isfinite(st["pos"]).all()
    g.close()
