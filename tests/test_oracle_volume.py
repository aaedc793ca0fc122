"""Pins of the oracle's harmonic volume constraint and height map
("Validation and Benchmark": a harmonic volume constraint holds the cell's
surface-to-volume ratio; the fluctuation dh(x, y) is read along the upper rim
of the cell), checked by routes other than the oracle's own formulas: the
volume of a sphere and of a polyhedron in closed form, invariance under the
reference point for a centrally symmetric surface, the virtual work of a
dilation against the closed-form volume change, and numpy's weighted 2-D
histogram and a sine's bin means.
"""
import math

import numpy as np
import pytest

import oracle
from synth import membranes as M


def lipid_sphere(f=6, R=12.0):
    """Lipids on the vertices of a frequency-f icosphere of radius R (a
    centrally symmetric point set) with radial directors; a = 4 pi R^2 / N."""
    v, _ = M.icosphere(f)
    n = len(v)
    pos, ori = v * R, v.copy()
    typ = np.zeros(n, np.uint8)
    z = np.zeros((n, 3))
    return pos, ori, typ, 4.0 * math.pi * R * R / n


def make(pos, ori, typ, bonds=None, r0=None, kb=None, n_centroids=8):
    m = oracle.model()
    s = oracle.OracleSystem(m, oracle.run(kT=0.0, n_centroids=n_centroids, seed=0))
    z = np.zeros_like(pos)
    s.set_particles(pos, z, ori, z, typ, np.arange(len(typ), dtype=np.uint32))
    if bonds is not None:
        s.set_bonds(bonds, r0, kb)
    else:
        s.set_bonds(np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(0))
    s.init_cells()
    return s


def test_volume_of_a_sphere_closed_form():
    R = 12.0
    pos, ori, typ, a = lipid_sphere(6, R)
    s = make(pos, ori, typ)
    V = s.volume(a, [0.0, 0.0, 0.0])
    assert V == pytest.approx(4.0 / 3.0 * math.pi * R ** 3, rel=1e-12)


@pytest.mark.parametrize("xc", [[3.0, -2.0, 1.5], [-7.0, 0.5, 4.0]])
def test_volume_independent_of_reference_point_for_a_symmetric_surface(xc):
    """sum_i a n_i = 0 for a centrally symmetric set, so the reference point
    drops out of V."""
    pos, ori, typ, a = lipid_sphere(6, 12.0)
    s = make(pos, ori, typ)
    assert s.volume(a, xc) == pytest.approx(s.volume(a, [0.0, 0.0, 0.0]), rel=1e-10)


def test_volume_of_an_ellipsoidal_polyhedron():
    """Lipids sampled on the faces of a triangulated ellipsoid carry the
    face normal, so (x - x_c).n is constant over a face: V tends to the
    polyhedron's volume (1/6) sum det(a, b, c) as the face counts follow the
    face areas, whatever the reference point."""
    v, f = M.icosphere_mesh(6, 1.0)
    v = v * np.array([30.0, 22.0, 12.0])
    out = oracle.mesh_build(v, f, beads=1, d_min=0.0, d_ll=0.0, seed=3)
    lip = out["type"] == 0
    pos, ori = out["pos"][lip], out["ori"][lip]
    tri = v[f]
    V_poly = np.einsum("ij,ij->i", tri[:, 0], np.cross(tri[:, 1], tri[:, 2])).sum() / 6.0
    A = 0.5 * np.linalg.norm(np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0]), axis=1).sum()
    s = make(pos, ori, np.zeros(len(pos), np.uint8), n_centroids=32)
    a = A / len(pos)
    for xc in ([0.0, 0.0, 0.0], [5.0, -3.0, 2.0]):
        assert s.volume(a, xc) == pytest.approx(V_poly, rel=3e-3)


def test_constraint_energy_closed_form_and_inactive_for_proteins():
    """U_V = k_V (V - V0)^2 / 2 with V = 4/3 pi R^3 (the sphere's closed
    form, not the oracle's sum); the constraint acts on lipids only and
    exerts no torque, so every torque and a protein's force are unchanged."""
    R = 12.0
    pos, ori, typ, a = lipid_sphere(6, R)
    # one protein at the centre, far from every lipid
    pos = np.vstack([pos, [[0.0, 0.0, 0.0]]])
    ori = np.vstack([ori, [[0.0, 0.0, 0.0]]])
    typ = np.append(typ, np.uint8(1))
    s = make(pos, ori, typ)
    e0 = s.compute_forces()
    F0, T0 = s.forces()
    Vs = 4.0 / 3.0 * math.pi * R ** 3
    kv, V0 = 0.02, 0.93 * Vs
    s.set_volume(kv, V0, a, [0.0, 0.0, 0.0])
    e1 = s.compute_forces()
    F1, T1 = s.forces()
    assert e1[1] - e0[1] == pytest.approx(0.5 * kv * (Vs - V0) ** 2, rel=1e-11)
    assert e1[0] == e0[0] and e1[4] == e0[4]                 # pair energy and virial untouched
    assert np.array_equal(F1[-1], F0[-1]) and np.array_equal(T1, T0)
    # V > V0 pushes every lipid inward along its director
    dF = F1[:-1] - F0[:-1]
    assert (np.einsum("ij,ij->i", dF, ori[:-1]) < 0).all()
    assert np.abs(np.cross(dF, ori[:-1])).max() < 1e-12 * np.abs(dF).max()
    # switching it off restores the forces exactly
    s.set_volume(0.0, V0, a, [0.0, 0.0, 0.0])
    s.compute_forces()
    F2, T2 = s.forces()
    assert np.array_equal(F2, F0) and np.array_equal(T2, T0)


def _ellipsoid_lipids(seed=3):
    v, f = M.icosphere_mesh(6, 1.0)
    v = v * np.array([30.0, 22.0, 12.0])
    out = oracle.mesh_build(v, f, beads=1, d_min=0.0, d_ll=0.0, seed=seed)
    lip = out["type"] == 0
    tri = v[f]
    V_poly = np.einsum("ij,ij->i", tri[:, 0], np.cross(tri[:, 1], tri[:, 2])).sum() / 6.0
    A = 0.5 * np.linalg.norm(np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0]), axis=1).sum()
    return out["pos"][lip], out["ori"][lip], V_poly, A


def test_constraint_force_does_the_virtual_work_of_a_dilation():
    """Under the dilation x -> x_c + (1 + e)(x - x_c) the enclosed volume of
    any shape grows by 3 e V, so the work of forces that derive from
    U_V(true volume) is -k_V (V - V0) 3 e V_poly: checked against the
    polyhedron's closed-form volume, and a uniform translation (no volume
    change) does no work.  A force of a/3 per lipid, a sign error or a
    dropped term fails."""
    pos, ori, V_poly, A = _ellipsoid_lipids()
    s = make(pos, ori, np.zeros(len(pos), np.uint8), n_centroids=32)
    a = A / len(pos)
    xc = np.array([5.0, -3.0, 2.0])
    s.compute_forces()
    F0, T0 = s.forces()
    kv, V0 = 1e-3, 0.9 * V_poly
    s.set_volume(kv, V0, a, xc)
    s.compute_forces()
    F1, T1 = s.forces()
    dF = F1 - F0
    V = s.volume(a, xc)
    x = s.state()["pos"]
    work = np.einsum("ij,ij->", dF, x - xc)                    # per unit e
    assert work == pytest.approx(-kv * (V - V0) * 3.0 * V_poly, rel=5e-3)
    # a translation does no work up to the face counts' rounding (a closed
    # polyhedron's area-weighted normals sum to zero)
    assert np.linalg.norm(dF.sum(0)) < 2e-3 * np.linalg.norm(dF, axis=1).sum()
    assert np.array_equal(T1, T0)


def test_constraint_drives_the_volume_toward_v0():
    """Overdamped Langevin steps at kT = 0 with the constraint on: a vesicle
    whose target volume is 3% below its own shrinks toward it, and the
    constraint energy falls."""
    mem = M.vesicle(600, 5, kT=0.0, f=1, chain_beads=3, n_centroids=12)
    m = oracle.model()
    s = oracle.OracleSystem(m, oracle.run(kT=0.0, n_centroids=mem.n_centroids, seed=0, dt=0.005))
    s.load(mem)
    s.init_cells()
    lip = mem.type == 0
    R = mem.meta["R"]
    a = 4.0 * math.pi * R * R / lip.sum()
    V_start = s.volume(a, [0.0, 0.0, 0.0])
    V0 = 0.97 * V_start
    s.set_volume(0.05, V0, a, [0.0, 0.0, 0.0])
    u0 = s.compute_forces()
    s.integrate(300)
    V_end = s.volume(a, [0.0, 0.0, 0.0])
    assert V_end < V_start - 0.3 * (V_start - V0)
    assert abs(V_end - V0) < abs(V_start - V0)


# --------------------------------------------------------------------------- height map

def lattice_patch(nx=60, ny=40, step=0.5, z=lambda x, y: 0.0 * x):
    xs, ys = np.meshgrid((np.arange(nx) + 0.5) * step, (np.arange(ny) + 0.5) * step)
    x, y = xs.ravel(), ys.ravel()
    pos = np.stack([x, y, z(x, y)], 1)
    ori = np.tile([0.0, 0.0, 1.0], (len(x), 1))
    return pos, ori


def test_height_map_equals_weighted_histogram():
    """Bin sums and counts of a random cloud equal numpy's weighted 2-D
    histogram over the selected lipids (above z_min, in the annulus)."""
    rng = np.random.default_rng(2)
    n = 3000
    pos = np.column_stack([rng.uniform(-20, 20, n), rng.uniform(-20, 20, n), rng.normal(1.0, 2.0, n)])
    ori = np.tile([0.0, 0.0, 1.0], (n, 1))
    typ = np.zeros(n, np.uint8)
    typ[::7] = 2                                                # proteins are never counted
    s = make(pos, ori, typ, n_centroids=16)
    st = s.state()["pos"]
    x0, y0, dx, dy, nx, ny = -18.0, -15.0, 3.0, 2.5, 12, 12
    z_min, axis, r_in, r_out = 0.0, (1.0, -2.0), 4.0, 16.0
    h, cnt = s.height_map(x0, y0, dx, dy, nx, ny, z_min, axis, r_in, r_out)
    rho = np.hypot(st[:, 0] - axis[0], st[:, 1] - axis[1])
    sel = (typ == 0) & (st[:, 2] > z_min) & (rho >= r_in) & (rho < r_out)
    edges = (x0 + dx * np.arange(nx + 1), y0 + dy * np.arange(ny + 1))
    c_ref, _, _ = np.histogram2d(st[sel, 0], st[sel, 1], bins=edges)
    s_ref, _, _ = np.histogram2d(st[sel, 0], st[sel, 1], bins=edges, weights=st[sel, 2])
    assert np.array_equal(cnt, c_ref.T.astype(np.int32))
    full = cnt > 0
    assert np.allclose(h[full], (s_ref.T[full] / c_ref.T[full]), rtol=0, atol=1e-12)
    assert (h[~full] == 0).all()
    assert cnt.sum() > 500


def test_height_map_bin_means_of_a_sine():
    """z = A sin(k x) on a fine lattice: each bin's mean is the sine's
    average over the bin, A (cos k x_a - cos k x_b) / (k dx), to the
    lattice's midpoint-rule error."""
    A, lam = 0.8, 15.0
    k = 2 * math.pi / lam
    pos, ori = lattice_patch(120, 40, 0.25, lambda x, y: 2.0 + A * np.sin(k * x))
    s = make(pos, ori, np.zeros(len(pos), np.uint8), n_centroids=16)
    dx = 2.5
    h, cnt = s.height_map(0.0, 0.0, dx, 10.0, 12, 1, 0.0, (0.0, 0.0), 0.0, 1e9)
    xa = dx * np.arange(12)
    exact = 2.0 + A * (np.cos(k * xa) - np.cos(k * (xa + dx))) / (k * dx)
    assert (cnt == 10 * 40).all()
    assert np.abs(h[0] - exact).max() < A * (k * 0.25) ** 2 / 24 * 1.01 + 1e-12
