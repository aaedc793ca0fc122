"""Pins of the oracle's separate Voronoi cell set for the proteins ("Force
Evaluation": a cell with a detached cytoskeleton gets a second set of
Voronoi cells for its proteins), checked by brute force: every particle sits
in the nearest centroid of its own set, each set's cells hold one kind of
particle, the pair set equals the O(N^2) search, centroids move to the mean
of their members, each set runs along its own Morton curve, and the forces
equal those of the shared cells (the pair set is the same)."""
import numpy as np
import pytest

import oracle
from synth import membranes as M

KP = 6


def detached(upper=4.0, offset=1.0):
    return M.vesicle(1500, 5, kT=0.2, f=2, chain_beads=4, n_centroids=24, net_offset=offset, detach_upper=upper)


def make(mem, kp=KP, **kw):
    m = oracle.model(box=mem.box, periodic=mem.periodic)
    s = oracle.OracleSystem(m, oracle.run(kT=mem.kT, n_centroids=mem.n_centroids, n_protein_centroids=kp, seed=0,
                                          **kw))
    s.load(mem)
    s.init_cells()
    return m, s


def sorted_pairs(p):
    p = np.sort(np.asarray(p, np.int64), axis=1)
    return p[np.lexsort((p[:, 1], p[:, 0]))]


def check_sets(mem, s):
    c = s.cells()
    st = s.state()
    KL = mem.n_centroids
    lip = mem.type == 0
    cell = c["cell_of_id"]
    assert (cell[lip] < KL).all() and (cell[~lip] >= KL).all()
    # nearest centroid of the own set, lowest index on ties (brute force)
    want_l = oracle.assign_brute(st["pos"][lip], c["centroids"][:KL], mem.box, mem.periodic)
    want_p = oracle.assign_brute(st["pos"][~lip], c["centroids"][KL:], mem.box, mem.periodic) + KL
    assert np.array_equal(cell[lip], want_l) and np.array_equal(cell[~lip], want_p)
    return c


@pytest.mark.parametrize("upper,offset", [(4.0, 1.0), (0.0, 5.0), (0.0, 1.0)])
def test_each_particle_in_the_nearest_centroid_of_its_set(upper, offset):
    mem = detached(upper, offset)
    m, s = make(mem)
    check_sets(mem, s)
    s.integrate(10)
    check_sets(mem, s)


@pytest.mark.parametrize("upper,offset", [(4.0, 1.0), (0.0, 5.0)])
def test_pair_set_equals_brute_force(upper, offset):
    mem = detached(upper, offset)
    m, s = make(mem)
    for _ in range(2):
        st = s.state()
        brute = sorted_pairs(oracle.pairs_brute(m, st["pos"], mem.type, mem.id, mem.bonds))
        assert len(brute) > 1000
        assert np.array_equal(sorted_pairs(s.pairs()), brute)
        s.integrate(8)


def test_centroids_are_member_means_and_sets_follow_their_own_morton_curves():
    mem = detached()
    m, s = make(mem, n_lloyd_init=3)
    c0 = s.cells()
    x = s.state()["pos"]
    s.rebuild()
    c1 = s.cells()
    KL = mem.n_centroids
    # new centroids = means of the old members (on the state grid), as a set per cell set
    means = np.array([x[c0["cell_of_id"] == k].mean(0) for k in range(KL + KP)])
    for lo, hi in ((0, KL), (KL, KL + KP)):
        a = np.sort(np.round(means[lo:hi], 9), axis=0)
        b = np.sort(np.round(c1["centroids"][lo:hi], 9), axis=0)
        assert np.allclose(a, b, atol=1e-9)
        keys = oracle.morton_keys(c1["centroids"][lo:hi])
        assert np.all(np.diff(keys.astype(np.float64)) >= 0)


def test_forces_equal_the_shared_cells():
    """The pair set does not depend on the cells, so the forces of both cell
    layouts agree to the FP64 summation order."""
    mem = detached()
    _, a = make(mem, kp=KP)
    _, b = make(mem, kp=0)
    ea, eb = a.compute_forces(), b.compute_forces()
    Fa, Ta = a.forces()
    Fb, Tb = b.forces()
    scale = np.abs(Fb).max()
    assert np.abs(Fa - Fb).max() < 1e-12 * scale and np.abs(Ta - Tb).max() < 1e-12 * max(1.0, np.abs(Tb).max())
    assert ea[0] == pytest.approx(eb[0], rel=1e-12)
    # detached proteins inflate the shared lipid cells; their own cells do not
    Ra, Rb = a.cells()["radius"], b.cells()["radius"]
    assert Ra[: mem.n_centroids].max() < Rb.max()


def test_more_protein_centroids_than_proteins_is_refused():
    mem = detached()
    m = oracle.model()
    s = oracle.OracleSystem(m, oracle.run(kT=mem.kT, n_centroids=mem.n_centroids,
                                          n_protein_centroids=int((mem.type != 0).sum()) + 1))
    s.load(mem)
    with pytest.raises(RuntimeError):
        s.init_cells()
