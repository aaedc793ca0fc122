"""Pins of the oracle's bilayer proteins (band-3 and glycophorin) against
closed forms, invariances and brute force.

The two-component model places glycophorin and band-3 in the bilayer
("Initial structure generation"); the paper prints none of the cited model's
constants, so the oracle reads them as oriented bilayer particles that meet
other bilayer particles through the lipid potential with the well depth and
cutoff of their species pair, and the cytoskeleton through the WCA term, the
anchoring bonds excluding their 1-2 and 1-3 pairs from it.  Each test below
checks one of these statements by a route other than the oracle's formulas:
the tail's closed form at an interior point with the pair's own constants,
the relabelling invariance of the default table, the cutoff decided by brute
force, the exclusions of an anchor, and the thermostat's equipartition for
the proteins' rotations.
"""
import math

import numpy as np
import pytest

import oracle
from synth import membranes as M

RMIN = 2.0 ** (1.0 / 6.0)
L, B3, GP, J, S = M.LIPID, M.BAND3, M.GLYCOPHORIN, M.JUNCTION, M.SPECTRIN
SPECIES = {L: 0, B3: 1, GP: 2}


def table(eps_lb=2.5, rc_lb=3.0, eps_bg=0.7, rc_bg=2.2, eps_bb=1.8, rc_bb=0.0):
    """A symmetric table that differs from the lipid pair in every entry
    that involves a protein (rc 0: the lipid-lipid cutoff)."""
    te = np.zeros((3, 3))
    tr = np.zeros((3, 3))
    te[0, 1] = te[1, 0] = eps_lb
    tr[0, 1] = tr[1, 0] = rc_lb
    te[1, 2] = te[2, 1] = eps_bg
    tr[1, 2] = tr[2, 1] = rc_bg
    te[1, 1] = eps_bb
    tr[1, 1] = rc_bb
    return te, tr


@pytest.mark.parametrize("ti,tj", [(B3, L), (L, B3), (B3, GP), (GP, B3), (B3, B3), (GP, GP), (GP, L)])
def test_species_pair_tail_interior_closed_form(ti, tj):
    """Halfway through the well of the species pair (aligned directors
    perpendicular to the separation, phi = 1): U = -eps_ab 2^-zeta and the
    radial pull eps_ab 2 zeta cos^(2 zeta - 1) sin (pi/2)/(rc_ab - r_min) at
    theta = pi/4, with the pair's own eps_ab and rc_ab (pairs without a
    table entry take the lipid-lipid ones)."""
    te, tr = table()
    m = oracle.model(eps=1.0, rc=2.6, zeta=4, mem_eps=te, mem_rc=tr)
    a, b = SPECIES[ti], SPECIES[tj]
    eps = te[a, b] or 1.0
    rc = tr[a, b] or 2.6
    r = 0.5 * (RMIN + rc)
    U, F, Ti, Tj = oracle.pair_terms(m, ti, tj, [r, 0, 0], [0, 0, 1], [0, 0, 1])
    assert U == pytest.approx(-eps * 2.0 ** -4, rel=1e-13)
    w = (math.pi / 2.0) / (rc - RMIN)
    c = s = math.sqrt(0.5)
    assert F[0] == pytest.approx(eps * 8 * c ** 7 * s * w, rel=1e-12)
    assert abs(F[1]) < 1e-14 and abs(F[2]) < 1e-14
    assert np.abs(Ti).max() < 1e-14 and np.abs(Tj).max() < 1e-14


def test_species_pair_core_closed_form():
    """Inside r_min with phi = 1 the pair energy is eps_ab [(r_min/r)^4 -
    2 (r_min/r)^2]: at (r_min/r)^2 = sqrt 2 that is eps_ab (2 - 2 sqrt 2)."""
    te, tr = table()
    m = oracle.model(mem_eps=te, mem_rc=tr)
    r = RMIN / 2.0 ** 0.25
    for ti, tj, eps in ((B3, L, 2.5), (B3, GP, 0.7), (L, L, 1.0), (GP, GP, 1.0)):
        U, _, _, _ = oracle.pair_terms(m, ti, tj, [0, r, 0], [0, 0, 1], [0, 0, 1])
        assert U == pytest.approx(eps * (2.0 - 2.0 * math.sqrt(2.0)), rel=1e-13)


def test_membrane_proteins_meet_the_cytoskeleton_through_wca():
    """A band-3 or glycophorin particle and a spectrin bead: the textbook WCA
    point U(sigma) = eps_wca with the lipid-protein size, no torque."""
    m = oracle.model(eps_wca=1.3, sigma_wca=1.0)
    for t in (B3, GP, L):
        U, F, Ti, _ = oracle.pair_terms(m, t, S, [1.0, 0, 0], [0, 0, 1], [0, 0, 0])
        assert U == pytest.approx(1.3, rel=1e-14)
        assert F[0] == pytest.approx(-4 * 1.3 * 6, rel=1e-13)     # -dU/dr at r = sigma, pushes i to -x
        assert np.abs(Ti).max() == 0.0


def test_default_table_makes_a_protein_a_relabelled_lipid():
    """With no table every bilayer species pair is the lipid pair, so
    relabelling lipids as band-3 or glycophorin leaves every pair term, the
    pair set and the forces unchanged, bit for bit."""
    mem = M.patch(2, 11, kT=0.2, n_centroids=64)
    rng = np.random.default_rng(3)
    relab = mem.copy()
    lip = np.flatnonzero(mem.type == L)
    pick = rng.choice(lip, 200, replace=False)
    relab.type[pick[:120]] = B3
    relab.type[pick[120:]] = GP
    m = oracle.model(box=mem.box, periodic=mem.periodic)
    out = []
    for mm in (mem, relab):
        s = oracle.OracleSystem(m, oracle.run(kT=mem.kT, n_centroids=mem.n_centroids, seed=0))
        s.load(mm)
        s.init_cells()
        e = s.compute_forces()
        out.append((s.forces(), e, s.pairs()))
    (Fa, Ta), ea, pa = out[0]
    (Fb, Tb), eb, pb = out[1]
    assert np.array_equal(Fa, Fb) and np.array_equal(Ta, Tb)
    assert np.array_equal(np.asarray(ea)[:2], np.asarray(eb)[:2])
    assert np.array_equal(pa, pb)


def test_species_cutoff_decides_the_pair_set_by_brute_force():
    """A band-3 and a lipid interact up to the table's 3.0 sigma, two lipids
    only to 2.6: pairs at 2.8 sigma exist for the first and not the second,
    and the search cutoff is the table's largest."""
    te, tr = table()
    m = oracle.model(mem_eps=te, mem_rc=tr)
    x = np.array([[0.0, 0, 0], [2.8, 0, 0], [0, 30, 0], [2.8, 30, 0], [0, 60, 0], [2.999999, 60, 0],
                  [0, 90, 0], [3.000001, 90, 0]])
    typ = np.array([B3, L, L, L, L, B3, B3, L], np.uint8)
    pairs = {tuple(p) for p in oracle.pairs_brute(m, x, typ, np.arange(8, dtype=np.uint32)).tolist()}
    assert pairs == {(0, 1), (4, 5)}
    assert oracle.lib().or_search_cutoff(oracle.C.byref(m)) == 3.0


def test_anchor_bond_excludes_its_one_two_and_one_three_pairs():
    """Glycophorin anchored to a junction that starts a spectrin chain: the
    glycophorin-junction pair (1-2) and the glycophorin-bead pair (1-3)
    carry no WCA term although inside its range; an unanchored band-3 at the
    same distance from the bead does; bilayer pairs are never excluded, even
    when bonded."""
    m = oracle.model()
    x = np.array([[0.0, 0.0, 0.95],    # 0 glycophorin, above the junction
                  [0.0, 0.0, 0.0],     # 1 junction
                  [0.55, 0.0, 0.0],    # 2 spectrin bead bonded to the junction
                  [0.55, 0.0, 0.9],    # 3 band-3, not anchored, above the bead
                  [1.6, 0.0, 1.0]])    # 4 lipid bonded to the glycophorin (never excluded)
    typ = np.array([GP, J, S, B3, L], np.uint8)
    ids = np.arange(5, dtype=np.uint32)
    bonds = np.array([[0, 1], [1, 2], [0, 4]], np.int32)
    pairs = {tuple(p) for p in oracle.pairs_brute(m, x, typ, ids, bonds).tolist()}
    assert (0, 1) not in pairs and (0, 2) not in pairs
    assert (2, 3) in pairs and (1, 3) in pairs
    assert (0, 4) in pairs and (0, 3) in pairs
    # without the anchor the glycophorin-junction and -bead pairs interact
    pairs = {tuple(p) for p in oracle.pairs_brute(m, x, typ, ids, bonds[1:]).tolist()}
    assert (0, 1) in pairs and (0, 2) in pairs


def test_bilayer_proteins_rotate_and_thermalise():
    """The thermostat acts on the proteins' directors as on the lipids':
    isolated band-3 and glycophorin particles (farther apart than any
    cutoff) reach the rotational equipartition kT (two degrees of freedom)
    while junctions keep zero angular velocity."""
    n = 216
    g = np.stack(np.meshgrid(*[np.arange(6)] * 3, indexing="ij"), -1).reshape(-1, 3) * 4.0
    typ = np.array([B3, GP, J] * (n // 3), np.uint8)
    ori = np.where((typ == J)[:, None], 0.0, np.array([0.0, 0.0, 1.0]))
    mem = M.Membrane(pos=g.astype(float), vel=np.zeros((n, 3)), ori=ori, angvel=np.zeros((n, 3)), type=typ,
                     id=np.arange(n, dtype=np.uint32), bonds=np.zeros((0, 2), np.int32), r0=np.zeros(0),
                     kb=np.zeros(0), box=np.zeros(3), periodic=np.zeros(3, np.int32), n_centroids=8, kT=0.3)
    m = oracle.model()
    s = oracle.OracleSystem(m, oracle.run(kT=0.3, n_centroids=8, seed=5, gamma_r=2.0))
    s.load(mem)
    s.init_cells()
    s.integrate(200)
    kr = []
    for _ in range(40):
        s.integrate(25)
        st = s.state()
        w = st["angvel"]
        kr.append(0.5 * (w[typ != J] ** 2).sum(1).mean())
        assert np.abs(w[typ == J]).max() == 0.0
        assert np.abs((w * st["ori"]).sum(1)).max() < 1e-9
    assert np.mean(kr) == pytest.approx(0.3, rel=0.06)
