"""Pins of the FP64 oracle against what the mathematics and the paper fix.

Each test checks the oracle by a route other than its own formulas:
published known-answer vectors, closed-form values, finite differences of
the energy, conservation laws, brute force on tiny inputs, library routines
(numpy stable argsort), and the statistical statements of the paper.
"""
import math
import os

import numpy as np
import pytest

import oracle
from synth import membranes as M

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RMIN = 2.0 ** (1.0 / 6.0)


def unit(v):
    v = np.asarray(v, float)
    return v / np.linalg.norm(v)


# --------------------------------------------------------------------------- Philox

def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


def test_noise_is_unit_variance_uniform():
    xs = np.array([oracle.noise3(12345, 7, i, 3, 0) for i in range(20000)]).ravel()
    lim = math.sqrt(3.0)
    assert xs.min() > -lim and xs.max() < lim
    assert abs(xs.mean()) < 0.02
    assert abs(xs.var() - 1.0) < 0.02
    # distinct substreams / steps / instances give different words
    a = oracle.noise3(1, 0, 5, 10, 0)
    assert not np.array_equal(a, oracle.noise3(1, 0, 5, 10, 1))
    assert not np.array_equal(a, oracle.noise3(1, 0, 5, 11, 0))
    assert not np.array_equal(a, oracle.noise3(1, 1, 5, 10, 0))


# --------------------------------------------------------------------------- pair potential

def test_lipid_pair_closed_form_minimum():
    """Two lipids at r = r_min with parallel normals perpendicular to the
    separation: a = 1, phi = 1, so U = -eps and the force and torques vanish."""
    m = oracle.model()
    U, F, Ti, Tj = oracle.lipid_pair(m, [RMIN, 0, 0], [0, 0, 1], [0, 0, 1])
    assert U == pytest.approx(-1.0, abs=1e-14)
    assert np.abs(F).max() < 1e-13 and np.abs(Ti).max() < 1e-14 and np.abs(Tj).max() < 1e-14


def test_lipid_pair_closed_form_inner_zero():
    """At r = r_min / sqrt(2): (r_min/r)^2 = 2 so u_R = eps (4 - 4) = 0; with
    phi = 1 the energy is 0 and the radial force is 8 eps / r, repulsive."""
    m = oracle.model()
    r = RMIN / math.sqrt(2.0)
    U, F, _, _ = oracle.lipid_pair(m, [0, r, 0], [1, 0, 0], [1, 0, 0])
    assert U == pytest.approx(0.0, abs=1e-13)
    # j sits at +y from i, so the repulsive force on i points to -y
    assert F[1] == pytest.approx(-8.0 / r, rel=1e-13)
    assert abs(F[0]) < 1e-13 and abs(F[2]) < 1e-13


def test_lipid_pair_vanishes_at_cutoff():
    m = oracle.model()
    rng = np.random.default_rng(0)
    for _ in range(5):
        d = unit(rng.normal(size=3)) * m.rc
        U, F, Ti, Tj = oracle.lipid_pair(m, d, unit(rng.normal(size=3)), unit(rng.normal(size=3)))
        assert abs(U) < 1e-30 and np.abs(F).max() < 1e-12 and np.abs(Ti).max() < 1e-12


def test_lipid_pair_antiparallel_tilted_phi():
    """Normals along the separation (n_i = n_j = rh): a = 1 - 1 = 0 so
    phi = 1 - mu; at r_min U = -eps phi = eps (mu - 1)."""
    m = oracle.model()
    U, _, _, _ = oracle.lipid_pair(m, [RMIN, 0, 0], [1, 0, 0], [1, 0, 0])
    assert U == pytest.approx(m.mu - 1.0, abs=1e-13)


@pytest.mark.parametrize("zeta", [2, 3, 4])
def test_lipid_pair_attractive_tail_interior_closed_form(zeta):
    """Inside the attractive well, with aligned normals perpendicular to the
    separation (a = 1, phi = 1), U = -eps cos^(2 zeta)(theta) with
    theta = (pi/2)(r - r_min)/(r_c - r_min).  Halfway between r_min and r_c
    theta = pi/4, so U = -eps 2^-zeta; one third of the way theta = pi/6, so
    U = -eps (3/4)^zeta.  The radial force is -dU/dr =
    -eps 2 zeta cos^(2 zeta - 1) sin (pi/2)/(r_c - r_min), pulling i towards
    j.  A wrong exponent (cos^zeta, cos^(2 zeta - 2)) or a wrong width
    ((pi/2)/r_c) moves every one of these values."""
    eps, rc = 1.5, 2.6
    m = oracle.model(eps=eps, rc=rc, zeta=zeta)
    w = (math.pi / 2.0) / (rc - RMIN)
    for frac, c, s in ((0.5, math.sqrt(0.5), math.sqrt(0.5)), (1.0 / 3.0, math.sqrt(3.0) / 2.0, 0.5)):
        r = RMIN + frac * (rc - RMIN)
        # j sits at +x from i; normals along z, perpendicular to the separation
        U, F, Ti, Tj = oracle.lipid_pair(m, [r, 0, 0], [0, 0, 1], [0, 0, 1])
        assert U == pytest.approx(-eps * c ** (2 * zeta), rel=1e-13)
        fr = eps * 2 * zeta * c ** (2 * zeta - 1) * s * w
        assert F[0] == pytest.approx(fr, rel=1e-12)       # attractive: towards +x
        assert abs(F[1]) < 1e-14 and abs(F[2]) < 1e-14
        assert np.abs(Ti).max() < 1e-14 and np.abs(Tj).max() < 1e-14
    # halfway, the energy is exactly -eps 2^-zeta
    U, _, _, _ = oracle.lipid_pair(m, [0, 0.5 * (RMIN + rc), 0], [1, 0, 0], [1, 0, 0])
    assert U == pytest.approx(-eps * 2.0 ** -zeta, rel=1e-13)


def test_lipid_pair_attractive_tail_scales_with_phi():
    """Halfway through the well, a tilt that lowers a scales the tail by
    phi = 1 + mu (a - 1) and adds the angular force and torques: with n_i
    along z and n_j tilted by alpha about the separation axis x, rh = -x and
    a = cos(alpha), so U = -eps 2^-zeta (1 + mu (cos(alpha) - 1))."""
    m = oracle.model()
    r = 0.5 * (RMIN + m.rc)
    for alpha in (0.1, 0.4, 1.0):
        nj = [0.0, -math.sin(alpha), math.cos(alpha)]
        U, _, Ti, Tj = oracle.lipid_pair(m, [r, 0, 0], [0, 0, 1], nj)
        phi = 1.0 + m.mu * (math.cos(alpha) - 1.0)
        assert U == pytest.approx(-(2.0 ** -m.zeta) * phi, rel=1e-12)
        # the torques twist the directors back towards each other about x
        g = -(2.0 ** -m.zeta)
        assert Ti[0] == pytest.approx(-g * m.mu * math.sin(alpha), rel=1e-12)
        assert Tj[0] == pytest.approx(g * m.mu * math.sin(alpha), rel=1e-12)


@pytest.mark.parametrize("delta", [0.1, -0.05])
def test_bond_closed_form(delta):
    """One harmonic bond stretched (or compressed) by delta from its rest
    length: U = kb delta^2 / 2 and the force on each end has magnitude
    kb |delta|, pulling the ends together when stretched.  Checked on the
    term itself and through the system force routine (both ends, energy,
    virial W = -kb delta r)."""
    kb, r0 = 100.0, 0.57
    r = r0 + delta
    u = unit([0.3, -0.4, 1.2])
    U, Fa = oracle.bond_pair(u * r, kb, r0)
    assert U == pytest.approx(0.5 * kb * delta * delta, rel=1e-13)
    np.testing.assert_allclose(Fa, kb * delta * u, rtol=1e-12, atol=1e-14)
    m = oracle.model()
    x = np.array([[1.0, 2.0, 3.0], [1.0, 2.0, 3.0] + u * r])
    typ = np.array([2, 2], np.uint8)
    F, T, e = oracle.forces_from_pairs(m, x, np.zeros((2, 3)), typ, np.zeros((0, 2), np.int32),
                                       bond_idx=np.array([[0, 1]]), r0=np.array([r0]), kb=np.array([kb]))
    np.testing.assert_allclose(F[0], kb * delta * u, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(F[1], -kb * delta * u, rtol=1e-12, atol=1e-14)
    assert e[1] == pytest.approx(0.5 * kb * delta * delta, rel=1e-13)
    assert e[4] == pytest.approx(-kb * delta * r, rel=1e-12)
    assert np.abs(T).max() == 0.0


def test_wca_textbook_points():
    """WCA at r = s: LJ is 0 so U = eps, and the force is 24 eps/s; at
    r = 2^(1/6) s both vanish (LJ minimum).  s = sigma_wca for a
    lipid-protein pair, sigma_pp for a protein-protein pair."""
    m = oracle.model(sigma_wca=1.0, sigma_pp=0.5)
    U, F, _, _ = oracle.pair_terms(m, 0, 2, [0, 0, 1.0], [0, 0, 1], [0, 0, 0])
    assert U == pytest.approx(1.0, abs=1e-14)
    assert F[2] == pytest.approx(-24.0, rel=1e-14)
    U, F, _, _ = oracle.pair_terms(m, 0, 2, [RMIN, 0, 0], [0, 0, 1], [0, 0, 0])
    assert abs(U) < 1e-14 and np.abs(F).max() < 1e-12
    U, F, _, _ = oracle.pair_terms(m, 1, 2, [0, 0.5, 0], [0, 0, 0], [0, 0, 0])
    assert U == pytest.approx(1.0, abs=1e-14)
    assert F[1] == pytest.approx(-48.0, rel=1e-14)
    U, F, _, _ = oracle.pair_terms(m, 2, 2, [0, 0, 0.5 * RMIN], [0, 0, 0], [0, 0, 0])
    assert abs(U) < 1e-14 and np.abs(F).max() < 1e-11


def _rotate(n, axis, ang):
    axis = unit(axis)
    return n * math.cos(ang) + np.cross(axis, n) * math.sin(ang) + axis * np.dot(axis, n) * (1 - math.cos(ang))


@pytest.mark.parametrize("s0", [0.0, 0.2])
def test_lipid_pair_finite_difference(s0):
    """Central differences of U give the force on i and the torques."""
    m = oracle.model(sin_theta0=s0)
    rng = np.random.default_rng(1 + int(s0 * 10))
    h = 1e-6
    for trial in range(40):
        r = rng.uniform(0.8, 2.55)
        d = unit(rng.normal(size=3)) * r
        ni, nj = unit(rng.normal(size=3)), unit(rng.normal(size=3))
        U, F, Ti, Tj = oracle.lipid_pair(m, d, ni, nj)
        # force on i: moving x_i by +e changes d = x_j - x_i by -e
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            up = oracle.lipid_pair(m, d - e, ni, nj)[0]
            dn = oracle.lipid_pair(m, d + e, ni, nj)[0]
            assert -(up - dn) / (2 * h) == pytest.approx(F[k], abs=2e-6 * (1 + abs(F[k])))
        # torque on i about each axis: dU/dang = -tau . axis
        for k in range(3):
            ax = np.eye(3)[k]
            up = oracle.lipid_pair(m, d, _rotate(ni, ax, h), nj)[0]
            dn = oracle.lipid_pair(m, d, _rotate(ni, ax, -h), nj)[0]
            assert -(up - dn) / (2 * h) == pytest.approx(Ti[k], abs=2e-6 * (1 + abs(Ti[k])))
            up = oracle.lipid_pair(m, d, ni, _rotate(nj, ax, h))[0]
            dn = oracle.lipid_pair(m, d, ni, _rotate(nj, ax, -h))[0]
            assert -(up - dn) / (2 * h) == pytest.approx(Tj[k], abs=2e-6 * (1 + abs(Tj[k])))


def test_pair_conserves_momentum_and_angular_momentum():
    """Per pair: F_j = -F_i, and r_i x F_i + r_j x F_j + tau_i + tau_j = 0."""
    m = oracle.model(sin_theta0=0.15)
    rng = np.random.default_rng(3)
    for _ in range(50):
        xi = rng.normal(size=3)
        d = unit(rng.normal(size=3)) * rng.uniform(0.8, 2.55)
        xj = xi + d
        ni, nj = unit(rng.normal(size=3)), unit(rng.normal(size=3))
        _, F, Ti, Tj = oracle.lipid_pair(m, d, ni, nj)
        L = np.cross(xi, F) + np.cross(xj, -F) + Ti + Tj
        assert np.abs(L).max() < 1e-12 * (1 + np.abs(F).max() * np.abs(xj).max())
        # torques are perpendicular to their directors
        assert abs(np.dot(Ti, ni)) < 1e-12 and abs(np.dot(Tj, nj)) < 1e-12


def test_potential_is_c1_at_rmin():
    m = oracle.model()
    ni, nj = unit([0.1, 0.2, 1.0]), unit([-0.2, 0.1, 1.0])
    dirv = unit([1.0, 0.3, 0.1])
    lo = oracle.lipid_pair(m, dirv * (RMIN - 1e-9), ni, nj)
    hi = oracle.lipid_pair(m, dirv * (RMIN + 1e-9), ni, nj)
    assert lo[0] == pytest.approx(hi[0], abs=1e-8)
    assert np.abs(lo[1] - hi[1]).max() < 1e-6


# --------------------------------------------------------------------------- tiny systems

def tiny_vesicle(n_lipids=600, seed=5, f=1, beads=3):
    mem = M.vesicle(n_lipids, seed, kT=0.2, f=f, chain_beads=beads, n_centroids=12)
    return mem


def tiny_patch():
    return M.patch(2, 11, kT=0.2, n_centroids=64)


def make_sys(mem, **run_kw):
    m = oracle.model(box=mem.box, periodic=mem.periodic)
    kw = dict(kT=mem.kT, n_centroids=mem.n_centroids, seed=0)
    kw.update(run_kw)
    r = oracle.run(**kw)
    s = oracle.OracleSystem(m, r)
    s.load(mem)
    return m, s


def sorted_pairs(p):
    p = np.sort(np.asarray(p, np.int64), axis=1)
    return p[np.lexsort((p[:, 1], p[:, 0]))]


@pytest.mark.parametrize("which", ["vesicle", "patch"])
def test_cell_list_pairs_equal_brute_force(which):
    mem = tiny_vesicle() if which == "vesicle" else tiny_patch()
    m, s = make_sys(mem)
    s.init_cells()
    st = s.state()
    brute = sorted_pairs(oracle.pairs_brute(m, st["pos"], mem.type, mem.id, mem.bonds))
    cells = sorted_pairs(s.pairs())
    assert len(brute) > 1000
    assert np.array_equal(brute, cells)
    # still exact after integration and several rebuilds
    s.integrate(15)
    st = s.state()
    brute = sorted_pairs(oracle.pairs_brute(m, st["pos"], mem.type, mem.id, mem.bonds))
    assert np.array_equal(brute, sorted_pairs(s.pairs()))


def test_bonded_pairs_are_excluded_and_bonds_act():
    mem = tiny_vesicle()
    m, s = make_sys(mem)
    s.init_cells()
    pairs = {tuple(p) for p in s.pairs().tolist()}
    for a, b in mem.bonds.tolist():
        assert (min(a, b), max(a, b)) not in pairs


def test_half_list_newton3_equals_per_particle_double_computation():
    """The paper's race-free scheme computes cross-patch pairs twice; the
    result must equal the serial Newton's-3rd-law sum."""
    mem = tiny_vesicle()
    m, s = make_sys(mem)
    s.init_cells()
    e_full = s.compute_forces()
    F_full, T_full = s.forces()
    st = s.state()
    pairs = oracle.pairs_brute(m, st["pos"], mem.type, mem.id, mem.bonds)
    F, T, e = oracle.forces_from_pairs(m, st["pos"], st["ori"], mem.type, pairs, mem.bonds, mem.r0, mem.kb)
    scale = np.abs(F).max()
    assert np.abs(F - F_full).max() < 1e-12 * scale
    assert np.abs(T - T_full).max() < 1e-12 * max(1.0, np.abs(T).max())
    assert e[0] == pytest.approx(e_full[0], rel=1e-12)
    assert e[1] == pytest.approx(e_full[1], rel=1e-12)
    assert e[4] == pytest.approx(e_full[4], rel=1e-10)


def test_total_force_and_torque_vanish():
    """Isolated (non-periodic) vesicle: Newton's third law gives sum F = 0 and
    total angular momentum change sum (r x F + tau) = 0."""
    mem = tiny_vesicle()
    m, s = make_sys(mem)
    s.init_cells()
    s.compute_forces()
    F, T = s.forces()
    x = s.state()["pos"]
    scale = np.abs(F).max() * len(F)
    assert np.abs(F.sum(0)).max() < 1e-13 * scale
    L = (np.cross(x, F) + T).sum(0)
    assert np.abs(L).max() < 1e-12 * scale * np.abs(x).max()


def test_system_forces_finite_difference():
    """Central differences of the total potential (pairs + bonds) of a small
    vesicle give the forces; rotations of a director give the torque."""
    mem = tiny_vesicle(n_lipids=300, f=1, beads=2)
    m, s = make_sys(mem)
    s.init_cells()
    s.compute_forces()
    F, T = s.forces()
    rng = np.random.default_rng(4)
    h = 1e-5

    def energy(pos, ori):
        t = oracle.OracleSystem(m, s.r)
        t.set_particles(pos, mem.vel, ori, mem.angvel, mem.type, mem.id)
        t.set_bonds(mem.bonds, mem.r0, mem.kb)
        t.init_cells()
        e = t.compute_forces()
        return e[0] + e[1]

    st = s.state()
    for i in rng.choice(mem.n, 6, replace=False):
        for k in range(3):
            p1, p2 = st["pos"].copy(), st["pos"].copy()
            p1[i, k] += h
            p2[i, k] -= h
            fd = -(energy(p1, st["ori"]) - energy(p2, st["ori"])) / (2 * h)
            assert fd == pytest.approx(F[i, k], abs=1e-5 * (1 + abs(F[i, k])))
    lip = np.flatnonzero(mem.type == 0)
    for i in rng.choice(lip, 4, replace=False):
        for k in range(3):
            ax = np.eye(3)[k]
            o1, o2 = st["ori"].copy(), st["ori"].copy()
            o1[i] = _rotate(o1[i], ax, h)
            o2[i] = _rotate(o2[i], ax, -h)
            fd = -(energy(st["pos"], o1) - energy(st["pos"], o2)) / (2 * h)
            assert fd == pytest.approx(T[i, k], abs=1e-5 * (1 + abs(T[i, k])))


def test_virial_is_minus_the_dilation_derivative():
    """Under x -> lambda x with the directors held, dU/dlambda at 1 is
    sum_i x_i . grad_i U = -sum_i x_i . F_i, so the reported virial W (pairs
    and bonds) equals minus the central difference of U in lambda."""
    mem = tiny_vesicle(n_lipids=300, f=1, beads=2)
    m, s = make_sys(mem)
    s.init_cells()
    e = s.compute_forces()
    st = s.state()

    def energy(lam):
        t = oracle.OracleSystem(m, s.r)
        t.set_particles(lam * st["pos"], mem.vel, st["ori"], mem.angvel, mem.type, mem.id)
        t.set_bonds(mem.bonds, mem.r0, mem.kb)
        t.init_cells()
        u = t.compute_forces()
        return u[0] + u[1]

    h = 1e-6
    w_fd = -(energy(1.0 + h) - energy(1.0 - h)) / (2 * h)
    assert abs(e[4]) > 1.0
    assert w_fd == pytest.approx(e[4], rel=1e-5, abs=1e-6)


# --------------------------------------------------------------------------- Voronoi cells

def _random_points(rng, n, L):
    return rng.uniform(0, L, size=(n, 3))


@pytest.mark.parametrize("periodic", [(0, 0, 0), (1, 1, 0), (1, 1, 1)])
def test_kdtree_equals_brute_force_argmin(periodic):
    rng = np.random.default_rng(sum(periodic))
    box = np.array([20.0, 17.0, 13.0])
    c = _random_points(rng, 300, 1.0) * box
    x = rng.uniform(-15, 35, size=(4000, 3))
    # exact ties: duplicate some centroids (lowest index must win)
    c[150:160] = c[10:20]
    x[:10] = c[10:20]
    a = oracle.assign_brute(x, c, box, periodic)
    b = oracle.assign_kdtree(x, c, box, periodic)
    assert np.array_equal(a, b)
    assert np.all(a[:10] == np.arange(10, 20))


def test_voronoi_invariant_after_init_and_rebuilds():
    """Every particle lies in the cell of its nearest centroid (ties to the
    lowest index), after initialisation and after each rebuild."""
    mem = tiny_patch()
    m, s = make_sys(mem)
    s.init_cells()
    for it in range(3):
        cl = s.cells()
        st = s.state()
        want = oracle.assign_brute(st["pos"], cl["centroids"], mem.box, mem.periodic)
        assert np.array_equal(cl["cell_of_id"], want)
        s.integrate(5)


def test_cells_are_approximately_equally_populated():
    """The paper: Voronoi cells of the k-means clustering are approximately
    equally populated and follow the membrane.  Reading: no empty cell and
    occupancy CV < 0.5 after initialisation."""
    for mem in (tiny_patch(), M.vesicle(8000, 3, f=2, chain_beads=5, n_centroids=128)):
        _, s = make_sys(mem)
        s.init_cells()
        cnt = np.diff(s.cells()["start"])
        assert cnt.min() > 0
        assert cnt.std() / cnt.mean() < 0.5


def test_lloyd_step_is_the_member_mean():
    """The M-step moves each centroid to the mean of its lipids (checked with
    numpy's mean, within the 2^-40 grid rounding)."""
    rng = np.random.default_rng(7)
    x = rng.normal(size=(500, 3)) * 5
    typ = (rng.random(500) < 0.8).astype(np.uint8) * 0
    typ[::7] = 2
    c = x[rng.choice(500, 20, replace=False)].copy()
    c = np.round(c * 2.0 ** 40) / 2.0 ** 40
    cell = oracle.assign_brute(x, c, np.zeros(3), (0, 0, 0))
    c2 = oracle.lloyd(x, typ, cell, c, np.zeros(3), (0, 0, 0))
    for k in range(20):
        sel = (cell == k) & (typ == 0)
        if sel.any():
            assert np.abs(c2[k] - x[sel].mean(0)).max() < 4e-12
        else:
            assert np.array_equal(c2[k], c[k])


def test_lloyd_fixed_point():
    """Repeated E/M steps reach a fixed point where every centroid is the mean
    of its lipids and no centroid moves."""
    rng = np.random.default_rng(8)
    x = rng.normal(size=(400, 3)) * 4
    typ = np.zeros(400, np.uint8)
    c = np.round(x[:16] * 2.0 ** 40) / 2.0 ** 40
    z = np.zeros(3)
    for it in range(200):
        cell = oracle.assign_brute(x, c, z, (0, 0, 0))
        c2 = oracle.lloyd(x, typ, cell, c, z, (0, 0, 0))
        if np.array_equal(c2, c):
            break
        c = c2
    assert np.abs(c2 - c).max() < 1e-12


def test_lloyd_periodic_wraps_and_uses_minimum_image():
    box = np.array([10.0, 10.0, 0.0])
    x = np.array([[9.8, 5.0, 0.0], [0.2, 5.0, 0.0]])   # straddle the boundary
    c = np.array([[9.9, 5.0, 0.0]])
    c = np.round(c * 2.0 ** 40) / 2.0 ** 40
    c2 = oracle.lloyd(x, np.zeros(2, np.uint8), np.zeros(2, np.int32), c, box, (1, 1, 0))
    assert c2[0, 0] == pytest.approx(0.0, abs=1e-11) or c2[0, 0] == pytest.approx(10.0, abs=1e-11)
    assert 0.0 <= c2[0, 0] < 10.0


def test_morton_key_interleave_and_order():
    # 2x2x2 corners: x is the least significant interleaved bit
    c = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0], [0, 0, 1], [1, 0, 1], [0, 1, 1], [1, 1, 1]], float)
    keys = oracle.morton_keys(c)
    top = np.uint64(2 ** 21 - 1)
    spread = lambda v: sum(((int(v) >> b) & 1) << (3 * b) for b in range(21))
    want = [spread(top * int(q[0])) | (spread(top * int(q[1])) << 1) | (spread(top * int(q[2])) << 2) for q in c]
    assert keys.tolist() == want
    perm = np.random.default_rng(0).permutation(8)
    order = oracle.morton_order(c[perm])
    assert np.array_equal(perm[order], np.arange(8))
    # equal keys keep the old index order
    d = np.zeros((5, 3))
    assert oracle.morton_order(d).tolist() == [0, 1, 2, 3, 4]


def test_counting_sort_is_stable():
    rng = np.random.default_rng(9)
    cell = rng.integers(0, 37, size=5000).astype(np.int32)
    perm, start = oracle.counting_sort(cell, 40)
    assert np.array_equal(perm, np.argsort(cell, kind="stable"))
    assert np.array_equal(start, np.concatenate([[0], np.cumsum(np.bincount(cell, minlength=40))]))


def test_adjacency_is_conservative_symmetric_reflexive():
    mem = tiny_patch()
    m, s = make_sys(mem)
    s.init_cells()
    cl = s.cells()
    K = len(cl["centroids"])
    nbr = [set(cl["adj"][cl["adj_ptr"][k]:cl["adj_ptr"][k + 1]].tolist()) for k in range(K)]
    for k in range(K):
        assert k in nbr[k]
        for j in nbr[k]:
            assert k in nbr[j]
    st = s.state()
    cell = cl["cell_of_id"]
    rs = 2.6
    x = st["pos"]
    pairs = oracle.pairs_brute(oracle.model(rc=rs, sigma_wca=rs / RMIN, box=mem.box, periodic=mem.periodic),
                               x, np.zeros(mem.n, np.uint8), mem.id)
    for i, j in pairs:
        assert cell[j] in nbr[cell[i]]


def test_state_is_quantised_to_grid():
    mem = tiny_vesicle()
    _, s = make_sys(mem)
    st = s.state()
    q = st["pos"] * 2.0 ** 40
    assert np.array_equal(q, np.round(q))
    assert np.abs(st["pos"] - mem.pos).max() <= 2.0 ** -41 * 1.0000001


# --------------------------------------------------------------------------- integrator

def _nve_energy_error(mem, dt, T):
    m, s = make_sys(mem, dt=dt, gamma_t=0.0, gamma_r=0.0, kT=0.0)
    s.init_cells()
    e0 = s.compute_forces()
    E0 = e0[0] + e0[1] + e0[2] + e0[3]
    nsteps = int(round(T / dt))
    devs = []
    for chunk in range(4):
        s.integrate(nsteps // 4)
        e = s.compute_forces()
        devs.append(abs(e[0] + e[1] + e[2] + e[3] - E0))
    return max(devs)


def test_nve_energy_error_scales_as_dt_squared():
    """At gamma = 0 the integrator is velocity Verlet with Cayley rotations:
    the energy error over a fixed time falls ~4x when dt halves."""
    mem = tiny_vesicle(n_lipids=400, f=1, beads=2)
    errs = [_nve_energy_error(mem, dt, 0.2) for dt in (0.004, 0.002, 0.001)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 2.5 < r1 < 6.0 and 2.5 < r2 < 6.0, errs


def test_langevin_equipartition():
    """BAOAB at kT: translational kinetic energy per particle -> 3/2 kT and
    rotational per lipid -> kT (two degrees of freedom)."""
    mem = tiny_patch()
    m, s = make_sys(mem, kT=0.2, gamma_t=1.0, gamma_r=1.0)
    s.init_cells()
    s.integrate(100)
    kt, kr = [], []
    for _ in range(20):
        s.integrate(10)
        e = s.compute_forces()
        kt.append(e[2] / mem.n)
        kr.append(e[3] / mem.n_lipids)
    assert np.mean(kt) == pytest.approx(1.5 * 0.2, rel=0.06)
    assert np.mean(kr) == pytest.approx(0.2, rel=0.06)


def _rodrigues(n, axis, theta):
    u = unit(axis)
    return n * math.cos(theta) + np.cross(u, n) * math.sin(theta) + u * np.dot(u, n) * (1.0 - math.cos(theta))


def test_free_lipids_drift_and_rotate_in_closed_form():
    """Two lipids farther apart than the cutoff, kT = 0 and no friction: no
    force, torque or noise acts, so each step moves x by dt v and turns n
    about omega (right-handed, dn/dt = omega x n) through twice the angle
    of one half-step Cayley map with a = (dt/2) omega / 2, i.e. by
    4 atan(dt |omega| / 4); v and omega stay constant."""
    d = [unit([0.0, 0.0, 1.0]), unit([1.0, 2.0, -0.5])]
    w = [np.array([1.5, -0.7, 0.0]), 0.0 * d[1]]
    w[1] = np.cross(d[1], unit([0.3, -1.0, 2.0])) * 2.2          # perpendicular to its director
    mem = M.Membrane(pos=np.array([[0.0, 0.0, 0.0], [9.0, -4.0, 3.0]]), vel=np.array([[0.3, -0.2, 0.1], [-0.4, 0.0, 0.25]]),
                     ori=np.array(d), angvel=np.array(w), type=np.zeros(2, np.uint8), id=np.array([0, 1], np.uint32),
                     bonds=np.zeros((0, 2), np.int32), r0=np.zeros(0), kb=np.zeros(0),
                     box=np.array([100.0, 100.0, 100.0]), periodic=np.zeros(3, np.int32), n_centroids=2, kT=0.0)
    dt, steps = 0.01, 60
    _, s = make_sys(mem, dt=dt, kT=0.0, gamma_t=0.0, gamma_r=0.0)
    s.init_cells()
    s0 = s.state()
    e = s.compute_forces()
    assert e[0] == 0.0 and e[1] == 0.0          # no pair or bond energy: nothing in range
    s.integrate(steps)
    st = s.state()
    assert st["step"] == steps
    assert np.abs(st["pos"] - (s0["pos"] + steps * dt * s0["vel"])).max() < 1e-12
    assert np.abs(st["vel"] - s0["vel"]).max() < 1e-15
    for i in range(2):
        om = s0["angvel"][i]
        theta = steps * 4.0 * math.atan(dt * np.linalg.norm(om) / 4.0)
        expect = _rodrigues(unit(s0["ori"][i]), om, theta)
        assert np.abs(st["ori"][i] - expect).max() < 1e-10, i
        assert np.abs(st["angvel"][i] - om).max() < 1e-10, i
    # the turn is not the small-angle one: the Cayley angle differs from |omega| t
    om = s0["angvel"][0]
    naive = _rodrigues(unit(s0["ori"][0]), om, steps * dt * np.linalg.norm(om))
    assert np.abs(st["ori"][0] - naive).max() > 1e-8


def test_free_lipids_relax_at_the_friction_rate():
    """kT = 0 with friction: the O step multiplies v by exp(-gamma_t dt) and
    omega by exp(-gamma_r dt) once per step, so v and omega decay as
    exp(-gamma t); x gains (dt/2)(v_j + v_j+1) and n turns through the two
    half-step Cayley angles of omega before and after that step's O."""
    dn = unit([0.2, -0.4, 1.0])
    om0 = np.cross(dn, unit([1.0, 0.5, 0.0])) * 1.8
    mem = M.Membrane(pos=np.array([[1.0, 2.0, -3.0]]), vel=np.array([[0.5, -0.25, 0.75]]), ori=dn[None, :],
                     angvel=om0[None, :], type=np.zeros(1, np.uint8), id=np.array([0], np.uint32),
                     bonds=np.zeros((0, 2), np.int32), r0=np.zeros(0), kb=np.zeros(0),
                     box=np.array([100.0, 100.0, 100.0]), periodic=np.zeros(3, np.int32), n_centroids=1, kT=0.0)
    dt, steps, gt, gr = 0.01, 40, 1.5, 4.0
    _, s = make_sys(mem, dt=dt, kT=0.0, gamma_t=gt, gamma_r=gr)
    s.init_cells()
    s0 = s.state()
    s.integrate(steps)
    st = s.state()
    ct, cr = math.exp(-gt * dt), math.exp(-gr * dt)
    v0, w0 = s0["vel"][0], s0["angvel"][0]
    assert np.abs(st["vel"][0] - ct ** steps * v0).max() < 1e-13
    assert np.abs(st["angvel"][0] - cr ** steps * w0).max() < 1e-10
    x = s0["pos"][0] + 0.5 * dt * sum(ct ** j + ct ** (j + 1) for j in range(steps)) * v0
    assert np.abs(st["pos"][0] - x).max() < 1e-12
    wn = np.linalg.norm(w0)
    theta = sum(2.0 * math.atan(0.25 * dt * wn * cr ** j) + 2.0 * math.atan(0.25 * dt * wn * cr ** (j + 1))
                for j in range(steps))
    assert np.abs(st["ori"][0] - _rodrigues(unit(s0["ori"][0]), w0, theta)).max() < 1e-10
    # exp(-gamma dt / 2) per step would leave v visibly larger
    assert np.abs(st["vel"][0] - math.exp(-0.5 * gt * dt) ** steps * v0).max() > 1e-3


def test_directors_stay_unit_and_angular_velocity_perpendicular():
    mem = tiny_patch()
    _, s = make_sys(mem)
    s.init_cells()
    s.integrate(30)
    st = s.state()
    lip = mem.type == 0
    assert np.abs(np.linalg.norm(st["ori"][lip], axis=1) - 1).max() < 1e-14
    assert np.abs(np.sum(st["ori"][lip] * st["angvel"][lip], axis=1)).max() < 1e-14


def test_trajectory_is_deterministic():
    mem = tiny_patch()
    _, a = make_sys(mem)
    a.init_cells()
    a.integrate(20)
    _, b = make_sys(mem)
    b.init_cells()
    b.integrate(20)
    sa, sb = a.state(), b.state()
    for k in ("pos", "vel", "ori", "angvel"):
        assert np.array_equal(sa[k], sb[k])


def test_skin_cadence_gives_the_same_pair_set():
    """Rebuilding every 5 steps with a skin still finds exactly the brute-force
    pair set (the adjacency is conservative while no particle has moved more
    than the skin)."""
    mem = tiny_patch()
    m, s = make_sys(mem, rebuild_every=5, skin=0.3)
    s.init_cells()
    for _ in range(3):
        s.integrate(3)
        st = s.state()
        brute = sorted_pairs(oracle.pairs_brute(m, st["pos"], mem.type, mem.id, mem.bonds))
        assert np.array_equal(brute, sorted_pairs(s.pairs()))


def test_spontaneous_curvature_term_closed_form():
    """With s0 = sin(theta0) and normals tilted towards each other by theta0
    (n_i = (-s0, 0, c0) at +x of n_j = (s0, 0, c0)): a = (1 - s0^2) + 2 s0^2
    - s0^2 = 1, so phi = 1 and U(r_min) = -eps.  With parallel normals
    perpendicular to the separation a = 1 - s0^2 instead."""
    s0 = 0.2
    c0 = math.sqrt(1 - s0 * s0)
    m = oracle.model(sin_theta0=s0)
    # d = x_j - x_i = -r_min x  (i sits at +x of j)
    U, F, _, _ = oracle.lipid_pair(m, [-RMIN, 0, 0], [-s0, 0, c0], [s0, 0, c0])
    assert U == pytest.approx(-1.0, abs=1e-13)
    U, _, _, _ = oracle.lipid_pair(m, [-RMIN, 0, 0], [0, 0, 1], [0, 0, 1])
    assert U == pytest.approx(-(1.0 - m.mu * s0 * s0), abs=1e-13)


def test_periodic_minimum_image_against_scipy():
    """Pair search and nearest centroid in a periodic box agree with scipy's
    periodic k-d tree (an independent minimum-image implementation)."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(21)
    box = np.array([9.0, 11.0, 7.5])
    x = rng.uniform(0, 1, size=(700, 3)) * box
    x[:50] += box * rng.integers(-2, 3, size=(50, 3))      # unwrapped copies
    m = oracle.model(rc=2.0, sigma_wca=2.0 / RMIN, box=box, periodic=(1, 1, 1))
    got = sorted_pairs(oracle.pairs_brute(m, x, np.zeros(700, np.uint8), np.arange(700, dtype=np.uint32)))
    t = cKDTree(np.mod(x, box), boxsize=box)
    want = sorted_pairs(np.array(sorted(t.query_pairs(2.0))))
    assert np.array_equal(got, want)
    c = rng.uniform(0, 1, size=(40, 3)) * box
    a = oracle.assign_brute(x, c, box, (1, 1, 1))
    _, b = cKDTree(c, boxsize=box).query(np.mod(x, box), k=1)
    assert np.array_equal(a, b)


def test_one_three_exclusion():
    """Spectrin beads two bonds apart (sharing a bond partner) carry no
    excluded-volume term; three bonds apart they do."""
    m = oracle.model(sigma_pp=0.5)
    # chain 0-1-2-3 folded so that 1-3 pairs and the 1-4 pair are inside the cutoff
    x = np.array([[0.0, 0.0, 0.0], [0.35, 0.0, 0.0], [0.35, 0.35, 0.0], [0.0, 0.35, 0.0]])
    typ = np.full(4, 2, np.uint8)
    ids = np.arange(4, dtype=np.uint32)
    bonds = np.array([[0, 1], [1, 2], [2, 3]], np.int32)
    pairs = {tuple(p) for p in oracle.pairs_brute(m, x, typ, ids, bonds).tolist()}
    assert (0, 2) not in pairs and (1, 3) not in pairs      # 1-3
    assert (0, 3) in pairs                                  # 1-4
    assert (0, 1) not in pairs                              # 1-2
