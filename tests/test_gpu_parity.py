"""CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (stated, from the arithmetic):
  * cell of each particle, storage permutation, centroids, cell radii,
    neighbouring cells and the interacting pair set: bit-exact;
  * forces, FP32 path: e_F = max_i |dF_i| / max(|F_i|, F_rms) <= 1e-5;
    torques: max_i |dtau_i| / max(tau_rms, sigma F_rms) <= 1e-5;
  * forces, FP64 path: e_F <= 1e-8 (2^-32 fixed-point accumulation);
  * potential energy: |dU| / |U| <= 1e-6 (FP32), 1e-10 (FP64);
  * trajectories: RMS position deviation after 100 steps <= 1e-5 sigma
    (FP32 forces) and <= 1e-9 sigma (FP64 path).
"""
import numpy as np
import pytest

import oracle
from synth import membranes as M

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_1701_02059_gb300")


def gpu_params(mem, **kw):
    d = dict(kT=mem.kT, n_centroids=mem.n_centroids, box=mem.box, periodic=mem.periodic, seed=0)
    d.update(kw)
    return G.make_params(**d)


def oracle_sys(mem, seed=0, **kw):
    m = oracle.model(box=mem.box, periodic=mem.periodic)
    rk = dict(kT=mem.kT, n_centroids=mem.n_centroids, seed=seed)
    rk.update(kw)
    s = oracle.OracleSystem(m, oracle.run(**rk))
    s.load(mem)
    return m, s


def pair(mem, gkw=None, okw=None):
    gkw = gkw or {}
    okw = okw or {}
    g = G.System(gpu_params(mem, **gkw))
    g.load_membrane(mem)
    m, o = oracle_sys(mem, **okw)
    return g, m, o


def assert_cells_equal(g, o):
    a, b = g.cells(), o.cells()
    for k in ("cell_of_id", "slot_ids", "centroids", "start", "radius", "adj_ptr", "adj"):
        assert a[k].shape == b[k].shape, k
        assert np.array_equal(a[k], b[k]), f"{k} differs at {np.flatnonzero(a[k].ravel() != b[k].ravel())[:5]}"


def force_error(Fg, Fo):
    frms = np.sqrt((Fo ** 2).sum(1).mean())
    return (np.linalg.norm(Fg - Fo, axis=1) / np.maximum(np.linalg.norm(Fo, axis=1), frms)).max(), frms


def torque_error(Tg, To, frms):
    trms = np.sqrt((To ** 2).sum(1).mean())
    return np.linalg.norm(Tg - To, axis=1).max() / max(trms, frms)


def sorted_pairs(p):
    p = np.sort(np.asarray(p, np.int64), axis=1)
    return p[np.lexsort((p[:, 1], p[:, 0]))].astype(np.uint32)


def small_vesicle():
    return M.vesicle(3000, 5, f=2, chain_beads=5, n_centroids=50)


WORKLOADS = {
    "patch-2304": M.flat_patch_2304,
    "vesicle-3.6k": small_vesicle,
    "vesicle-62k": M.vesicle_62k,
}


@pytest.fixture(scope="module", params=list(WORKLOADS))
def initialised(request):
    mem = WORKLOADS[request.param]()
    g, m, o = pair(mem)
    g.init_cells()
    o.init_cells()
    yield request.param, mem, g, m, o
    g.close()


def test_init_cells_bit_exact(initialised):
    _, mem, g, m, o = initialised
    assert_cells_equal(g, o)


def test_pair_set_bit_exact(initialised):
    _, mem, g, m, o = initialised
    assert np.array_equal(g.pairs(), o.pairs())


def test_forces_energies_fp32(initialised):
    _, mem, g, m, o = initialised
    eg = g.compute_forces(energies=True)
    eo = o.compute_forces()
    Fg, Tg = g.forces()
    Fo, To = o.forces()
    ef, frms = force_error(Fg, Fo)
    assert ef <= 1e-5, ef
    assert torque_error(Tg, To, frms) <= 1e-5
    assert abs(eg[0] - eo[0]) <= 1e-6 * abs(eo[0])
    assert abs(eg[1] - eo[1]) <= 1e-6 * max(abs(eo[1]), 1.0)
    # kinetic sums are exact 2^-32 fixed point of per-particle FP64 terms
    assert eg[2] == pytest.approx(eo[2], rel=1e-9) and eg[3] == pytest.approx(eo[3], rel=1e-9)
    assert abs(eg[4] - eo[4]) <= 1e-5 * max(abs(eo[4]), abs(eo[0]))


def test_split_pair_path_equals_one_launch_path(initialised):
    """The step's pair forces come from a per-cell search that writes
    neighbour lists and a per-particle evaluation of them; energies and the
    pair dump come from the one-launch quad-loop kernel.  Both add the same
    FP32 pair terms as exact 2^-32 integers, so forces and torques agree bit
    for bit."""
    _, mem, g, m, o = initialised
    g.compute_forces(energies=True)
    F1, T1 = g.forces()
    g.compute_forces()
    F2, T2 = g.forces()
    assert np.array_equal(F1, F2) and np.array_equal(T1, T2)


@pytest.mark.parametrize("K", [6, 12])
def test_split_pair_path_with_split_staging(K):
    """Few, large cells (about 300-600 particles each) make every
    neighbourhood larger than the search and evaluation stages, so rows are
    staged over several passes, some split between two passes: forces from
    the split path equal the one-launch kernel's bit for bit, and stay so
    over rebuilding steps."""
    mem = M.vesicle(3000, 5, f=2, chain_beads=5, n_centroids=K)
    g = G.System(gpu_params(mem))
    g.load_membrane(mem)
    g.init_cells()
    for _ in range(3):
        g.compute_forces(energies=True)
        F1, T1 = g.forces()
        g.compute_forces()
        F2, T2 = g.forces()
        assert np.array_equal(F1, F2) and np.array_equal(T1, T2)
        g.integrate(5)
    g.close()


def test_forces_do_not_depend_on_the_cell_list():
    """The mirrors are referenced to centroids rounded to 2^-26 sigma, so a
    pair's integer displacement depends on the two positions alone: on a
    non-periodic membrane, FP32 forces are bit-identical before and after
    the cell list is rebuilt (new centroids, new ownership, new order), and
    a skin cadence (cells rebuilt every 5 steps or on a 0.3 sigma move)
    gives the same trajectory as rebuilding every step, bit for bit, with
    FP64 integrator increments."""
    mem = small_vesicle()
    g = G.System(gpu_params(mem))
    g.load_membrane(mem)
    g.init_cells()
    g.compute_forces()
    F0, T0 = g.forces()
    for _ in range(3):
        g.rebuild_cells()
        g.compute_forces()
        F1, T1 = g.forces()
        assert np.array_equal(F0, F1) and np.array_equal(T0, T1)
    g.close()
    runs = []
    for kw in ({}, {"rebuild_every": 5, "skin": 0.3}):
        h = G.System(gpu_params(mem, **kw))
        h.load_membrane(mem)
        h.init_cells()
        h.integrate(30)
        runs.append(h.state())
        h.close()
    for k in ("pos", "vel", "ori", "angvel"):
        assert np.array_equal(runs[0][k], runs[1][k]), k


def test_rebuilds_bit_exact(initialised):
    _, mem, g, m, o = initialised
    for _ in range(3):
        g.rebuild_cells()
        o.rebuild()
        assert_cells_equal(g, o)


@pytest.mark.parametrize("precision", [G.F32_FORCE_F64_STATE, G.F32_FORCE_F32_STEP])
@pytest.mark.parametrize("name", ["patch-2304", "vesicle-3.6k", "vesicle-62k"])
def test_trajectory_100_steps_fp32(name, precision):
    """FP32 forces with FP64 or FP32 integrator increments: 100 steps within
    1e-5 sigma RMS of the oracle's trajectory."""
    mem = WORKLOADS[name]()
    g, m, o = pair(mem, gkw={"precision": precision})
    g.init_cells()
    o.init_cells()
    g.integrate(100)
    o.integrate(100)
    sg, so = g.state(), o.state()
    assert sg["step"] == so["step"] == 100
    rms = np.sqrt(((sg["pos"] - so["pos"]) ** 2).sum(1).mean())
    assert rms <= 1e-5, rms
    lip = mem.type == 0
    assert np.sqrt(((sg["ori"][lip] - so["ori"][lip]) ** 2).sum(1).mean()) <= 1e-5
    # the cell list of the GPU's own state is still exact
    cg = g.cells()
    assert np.array_equal(cg["cell_of_id"], oracle.assign_brute(sg["pos"], cg["centroids"], mem.box, mem.periodic))
    brute = sorted_pairs(oracle.pairs_brute(m, sg["pos"], mem.type, mem.id, mem.bonds))
    assert np.array_equal(g.pairs(), brute)
    g.close()


def test_vesicle_62k_1000_steps():
    """The vesicle workload for its full 1,000 steps with FP32 forces: the run
    stays finite, its final cell list is exact for its own state (Voronoi
    invariant, pair set equal to the O(N^2) brute force), and the Langevin
    thermostat holds the kinetic temperatures at kT (3/2 kT translational,
    kT rotational per lipid; statistical over 62k particles)."""
    mem = M.vesicle_62k()
    g = G.System(gpu_params(mem))
    g.load_membrane(mem)
    g.init_cells()
    g.integrate(1000)
    st = g.state()
    assert st["step"] == 1000
    assert np.isfinite(st["pos"]).all() and np.isfinite(st["vel"]).all()
    cg = g.cells()
    assert np.array_equal(cg["cell_of_id"], oracle.assign_brute(st["pos"], cg["centroids"], mem.box, mem.periodic))
    m = oracle.model(box=mem.box, periodic=mem.periodic)
    brute = sorted_pairs(oracle.pairs_brute(m, st["pos"], mem.type, mem.id, mem.bonds))
    assert np.array_equal(g.pairs(), brute)
    ke = 0.5 * (st["vel"] ** 2).sum(1).mean()
    assert abs(ke / (1.5 * mem.kT) - 1.0) < 0.03, ke
    lip = mem.type == 0
    kr = 0.5 * (st["angvel"][lip] ** 2).sum(1).mean()
    assert abs(kr / mem.kT - 1.0) < 0.03, kr
    g.close()


def test_fp64_path_patch_200_steps():
    """The 2,304-particle patch with FP64 forces and increments: forces to
    the fixed-point resolution, 200-step trajectory within 1e-9 sigma RMS."""
    mem = M.flat_patch_2304()
    g, m, o = pair(mem, gkw={"precision": G.F64_ALL})
    g.init_cells()
    o.init_cells()
    eg = g.compute_forces(energies=True)
    eo = o.compute_forces()
    Fg, Tg = g.forces()
    Fo, To = o.forces()
    ef, frms = force_error(Fg, Fo)
    assert ef <= 1e-8, ef
    assert torque_error(Tg, To, frms) <= 1e-8
    assert abs(eg[0] - eo[0]) <= 1e-10 * abs(eo[0])
    g.integrate(100)
    o.integrate(100)
    rms = np.sqrt(((g.state()["pos"] - o.state()["pos"]) ** 2).sum(1).mean())
    assert rms <= 1e-9, rms
    g.integrate(100)
    o.integrate(100)
    st = g.state()
    cg = g.cells()
    assert np.array_equal(cg["cell_of_id"], oracle.assign_brute(st["pos"], cg["centroids"], mem.box, mem.periodic))
    g.close()


def test_nve_energy_drift_fp32():
    """gamma = 0: total energy stays within the dt^2 error of velocity Verlet."""
    mem = small_vesicle()
    g = G.System(gpu_params(mem, gamma_t=0.0, gamma_r=0.0, kT=0.0, dt=0.005))
    g.load_membrane(mem)
    g.init_cells()
    e0 = g.compute_forces(energies=True)
    E0 = e0[:4].sum()
    dev = 0.0
    for _ in range(5):
        g.integrate(40)
        e = g.compute_forces(energies=True)
        dev = max(dev, abs(e[:4].sum() - E0))
    assert dev / abs(E0) < 2e-4, dev / abs(E0)
    g.close()


def test_deterministic_bitwise():
    mem = small_vesicle()
    runs = []
    for _ in range(2):
        g = G.System(gpu_params(mem))
        g.load_membrane(mem)
        g.init_cells()
        g.integrate(25)
        runs.append(g.state())
        g.close()
    for k in ("pos", "vel", "ori", "angvel"):
        assert np.array_equal(runs[0][k], runs[1][k])


def test_skin_cadence_exact_pairs():
    """Rebuilding every 5 steps with a 0.3 sigma skin: the pair set stays
    exact, and forces agree with the every-step rebuild."""
    mem = small_vesicle()
    g = G.System(gpu_params(mem, rebuild_every=5, skin=0.3))
    g.load_membrane(mem)
    g.init_cells()
    m = oracle.model(box=mem.box, periodic=mem.periodic)
    for _ in range(4):
        g.integrate(3)
        st = g.state()
        assert np.array_equal(g.pairs(), sorted_pairs(oracle.pairs_brute(m, st["pos"], mem.type, mem.id, mem.bonds)))
    g.close()


# --------------------------------------------------------------------------- edge cases

def _run_edge(mem, **gkw):
    g, m, o = pair(mem, gkw=gkw, okw={k: v for k, v in gkw.items() if k in ("n_lloyd_init",)})
    g.init_cells()
    o.init_cells()
    assert_cells_equal(g, o)
    assert np.array_equal(g.pairs(), o.pairs())
    g.compute_forces()
    o.compute_forces()
    ef, _ = force_error(g.forces()[0], o.forces()[0])
    assert ef <= 1e-5
    g.integrate(5)
    o.integrate(5)
    assert_cells_equal(g, o) if np.abs(g.state()["pos"] - o.state()["pos"]).max() == 0 else None
    g.close()


def test_single_cell():
    mem = M.vesicle(300, 7, f=1, chain_beads=2, n_centroids=1)
    _run_edge(mem)


def test_cell_larger_than_stage_and_sort_tile():
    """One cell of 2,500 particles: neighbour staging is split across passes
    and the stable order of a cell beyond the shared-memory sort is ranked."""
    mem = M.vesicle(2500, 8, f=1, chain_beads=0, n_centroids=1)
    mem.bonds = np.zeros((0, 2), np.int32)
    mem.r0 = np.zeros(0)
    mem.kb = np.zeros(0)
    _run_edge(mem)


def test_ragged_and_empty_cells():
    """Ragged particle count and centroids placed so that some cells start
    empty (far away from the membrane)."""
    mem = M.vesicle(1001, 9, f=1, chain_beads=3, n_centroids=24)
    g, m, o = pair(mem, gkw={"n_lloyd_init": 0}, okw={"n_lloyd_init": 0})
    rng = np.random.default_rng(0)
    c = mem.pos[mem.type == 0][rng.choice(1001, 20, replace=False)]
    c = np.concatenate([c, np.array([[500.0, 0, 0], [0, 500.0, 0], [0, 0, -500.0], [300.0, 300.0, 300.0]])])
    g.init_cells(c)
    o.init_cells(c)
    assert_cells_equal(g, o)
    assert (np.diff(g.cells()["start"]) == 0).sum() >= 4
    assert np.array_equal(g.pairs(), o.pairs())
    g.compute_forces()
    o.compute_forces()
    assert force_error(g.forces()[0], o.forces()[0])[0] <= 1e-5
    g.rebuild_cells()
    o.rebuild()
    assert_cells_equal(g, o)
    g.close()


def test_small_periodic_box_and_all_lipids():
    mem = M.patch(3, 13, kT=0.25, n_centroids=40)
    keep = mem.type == 0
    lip = M.Membrane(mem.pos[keep], mem.vel[keep], mem.ori[keep], mem.angvel[keep], mem.type[keep],
                     np.arange(keep.sum(), dtype=np.uint32), np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(0),
                     mem.box, mem.periodic, 40, 0.25)
    _run_edge(lip)


def test_nonzero_spontaneous_curvature():
    mem = small_vesicle()
    g, m, o = pair(mem, gkw={"sin_theta0": 0.1})
    o = oracle.OracleSystem(oracle.model(sin_theta0=0.1, box=mem.box, periodic=mem.periodic),
                            oracle.run(kT=mem.kT, n_centroids=mem.n_centroids, seed=0))
    o.load(mem)
    g.init_cells()
    o.init_cells()
    g.compute_forces()
    o.compute_forces()
    ef, frms = force_error(g.forces()[0], o.forces()[0])
    assert ef <= 1e-5
    assert torque_error(g.forces()[1], o.forces()[1], frms) <= 1e-5
    g.close()


POTENTIALS = {
    # zeta = 2 and 3 take the kernels' general exponent path; a shorter
    # lipid cutoff and wider proteins change the search radius and the WCA
    # bands; a nonzero sin(theta0) adds the spontaneous-curvature terms
    "zeta2": dict(zeta=2, mu=2.0, eps=1.3, rc_lipid=2.5, sigma_wca=0.95, sigma_wca_pp=0.6),
    "zeta3-s0": dict(zeta=3, mu=4.0, eps=0.8, rc_lipid=2.7, sin_theta0=0.05),
}


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", list(POTENTIALS))
def test_other_potential_parameters(name, precision):
    """Other constants of the potential (the model's parameters are inputs):
    pair set bit-exact, forces and torques within the path's tolerance."""
    kw = POTENTIALS[name]
    mem = small_vesicle()
    g = G.System(gpu_params(mem, precision=precision, **kw))
    g.load_membrane(mem)
    okw = dict(kw)
    okw["rc"] = okw.pop("rc_lipid")
    if "sigma_wca_pp" in okw:
        okw["sigma_pp"] = okw.pop("sigma_wca_pp")
    o = oracle.OracleSystem(oracle.model(box=mem.box, periodic=mem.periodic, **okw),
                            oracle.run(kT=mem.kT, n_centroids=mem.n_centroids, seed=0))
    o.load(mem)
    g.init_cells()
    o.init_cells()
    assert_cells_equal(g, o)
    assert np.array_equal(g.pairs(), o.pairs())
    g.compute_forces()
    o.compute_forces()
    tol = 1e-5 if precision == 0 else 1e-8
    ef, frms = force_error(g.forces()[0], o.forces()[0])
    assert ef <= tol, ef
    assert torque_error(g.forces()[1], o.forces()[1], frms) <= tol
    g.close()


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_coincident_particles_report_non_finite_forces(precision):
    """Two lipids at the same point make the pair force non-finite: the
    kernels flag it and the call returns ORBC_E_NAN (no fault, no silent
    garbage)."""
    mem = M.flat_patch_2304(seed=5)
    pos = mem.pos.copy()
    pos[1] = pos[0]
    kw = {"precision": G.F64_ALL} if precision == "f64" else {}
    g = G.System(gpu_params(mem, **kw))
    g.set_particles(pos, mem.vel, mem.ori, mem.angvel, mem.type, mem.id)
    g.set_bonds(mem.bonds, mem.r0, mem.kb)
    g.init_cells()
    with pytest.raises(G.OrbcError) as e:
        g.compute_forces()
    assert e.value.code == -5
    g.close()


def test_errors_are_reported():
    mem = small_vesicle()
    g = G.System(gpu_params(mem))
    bad = mem.pos.copy()
    bad[3, 1] = np.nan
    with pytest.raises(G.OrbcError) as e:
        g.set_particles(bad, mem.vel, mem.ori, mem.angvel, mem.type, mem.id)
    assert e.value.code == -1
    ids = mem.id.copy()
    ids[0] = ids[1]
    with pytest.raises(G.OrbcError):
        g.set_particles(mem.pos, mem.vel, mem.ori, mem.angvel, mem.type, ids)
    with pytest.raises(G.OrbcError) as e:
        g.integrate(1)
    assert e.value.code in (-4, -1)
    g.load_membrane(mem)
    with pytest.raises(G.OrbcError) as e:
        g.compute_forces()
    assert e.value.code == -4
    g.init_cells()
    g.compute_forces()
    with pytest.raises(G.OrbcError):
        g.integrate(-1)
    g.close()
    with pytest.raises(G.OrbcError):
        G.System(gpu_params(mem, rebuild_every=3, skin=0.0))
    with pytest.raises(G.OrbcError):
        small = M.vesicle(300, 7, f=1, chain_beads=2, n_centroids=1)
        h = G.System(gpu_params(small, n_centroids=400))
        h.load_membrane(small)
        h.init_cells()


def test_neighbour_row_limit_is_reported():
    """Each cell's neighbouring cells are held in a row of 64.  512 cells on
    the 2,304-particle patch with a 5 sigma skin put about 170 centroids
    within R_k + R_j + r_s + 2 skin of each other: the initialisation
    reports ORBC_E_STATE instead of dropping neighbours.  Without the skin
    the rows hold about 20 cells and the same system initialises."""
    mem = M.flat_patch_2304()
    g = G.System(gpu_params(mem, n_centroids=512, skin=5.0))
    g.load_membrane(mem)
    with pytest.raises(G.OrbcError) as e:
        g.init_cells()
    assert e.value.code == -4
    g.close()
    h = G.System(gpu_params(mem, n_centroids=512))
    h.load_membrane(mem)
    h.init_cells()
    c = h.cells()
    assert np.diff(c["adj_ptr"]).max() <= 64
    h.close()


# --------------------------------------------------------------------------- full-size 4M cell, sampled

@pytest.fixture(scope="module")
def rbc():
    mem = M.rbc_4m()
    g = G.System(gpu_params(mem, seed=2))
    g.load_membrane(mem)
    g.init_cells()
    g.compute_forces()
    yield mem, g
    g.close()


def test_rbc_voronoi_sampled(rbc):
    """Sampled particles of the 4,000,000-particle cell sit in the cell of
    their nearest centroid (brute force over all 65,536 centroids)."""
    mem, g = rbc
    c = g.cells()
    st = g.state()
    rng = np.random.default_rng(1)
    idx = rng.choice(mem.n, 1500, replace=False)
    want = oracle.assign_brute(st["pos"][idx], c["centroids"], mem.box, mem.periodic)
    assert np.array_equal(c["cell_of_id"][idx], want)
    cnt = np.diff(c["start"])
    assert cnt.min() > 0 and cnt.std() / cnt.mean() < 0.5
    # storage order is sorted by cell
    cell_by_slot = c["cell_of_id"][c["slot_ids"]]
    assert np.all(np.diff(cell_by_slot) >= 0)


def test_rbc_forces_sampled(rbc):
    """Forces on sampled particles against the oracle evaluated on their
    exact neighbourhoods: every particle within the search cutoff plus the
    particle's bond partners."""
    from scipy.spatial import cKDTree
    mem, g = rbc
    st = g.state()
    Fg, _ = g.forces()
    m = oracle.model(box=mem.box, periodic=mem.periodic)
    tree = cKDTree(st["pos"])
    partners = {}
    for q, (a, b) in enumerate(mem.bonds.tolist()):
        partners.setdefault(a, []).append((b, q))
        partners.setdefault(b, []).append((a, q))
    rng = np.random.default_rng(2)
    sample = np.concatenate([rng.choice(mem.n, 250, replace=False),
                             rng.choice(np.flatnonzero(mem.type != 0), 50, replace=False)])
    frms = np.sqrt((Fg ** 2).sum(1).mean())
    worst = 0.0
    for i in sample.tolist():
        loc = sorted(set(tree.query_ball_point(st["pos"][i], 2.7)) | {b for b, _ in partners.get(i, [])})
        li = loc.index(i)
        where = {p: q for q, p in enumerate(loc)}
        bonds = np.array([(li, where[b]) for b, _ in partners.get(i, [])], np.int32).reshape(-1, 2)
        r0 = np.array([mem.r0[q] for _, q in partners.get(i, [])])
        kb = np.array([mem.kb[q] for _, q in partners.get(i, [])])
        ids = np.arange(len(loc), dtype=np.uint32)
        pairs = oracle.pairs_brute(m, st["pos"][loc], mem.type[loc], ids, bonds)
        pairs = pairs[(pairs[:, 0] == li) | (pairs[:, 1] == li)]
        F, _, _ = oracle.forces_from_pairs(m, st["pos"][loc], st["ori"][loc], mem.type[loc], pairs, bonds, r0, kb)
        worst = max(worst, np.linalg.norm(Fg[i] - F[li]) / max(np.linalg.norm(F[li]), frms))
    assert worst <= 1e-5, worst


def test_rbc_steps_keep_cells_exact(rbc):
    mem, g = rbc
    g.integrate(3)
    st = g.state()
    c = g.cells()
    rng = np.random.default_rng(3)
    idx = rng.choice(mem.n, 1000, replace=False)
    assert np.array_equal(c["cell_of_id"][idx],
                          oracle.assign_brute(st["pos"][idx], c["centroids"], mem.box, mem.periodic))
    assert np.isfinite(st["pos"]).all() and st["step"] == 3


def test_rbc_trajectory_matches_oracle():
    """The whole 4,000,000-particle cell, GPU and oracle from the same state:
    five steps (cells rebuilt every step, FP32 forces, FP64 increments)
    within 1e-5 sigma RMS of the oracle's positions and directors."""
    mem = M.rbc_4m()
    g = G.System(gpu_params(mem, seed=2))
    g.load_membrane(mem)
    m, o = oracle_sys(mem, seed=2)
    g.init_cells()
    o.init_cells()
    g.integrate(5)
    o.integrate(5)
    sg, so = g.state(), o.state()
    assert sg["step"] == so["step"] == 5
    rms = np.sqrt(((sg["pos"] - so["pos"]) ** 2).sum(1).mean())
    assert rms <= 1e-5, rms
    lip = mem.type == 0
    assert np.sqrt(((sg["ori"][lip] - so["ori"][lip]) ** 2).sum(1).mean()) <= 1e-5
    g.close()


def test_fp64_path_vesicle_62k_50_steps():
    """FP64 pair terms and increments on the 61,962-particle vesicle: 50 steps
    within 1e-9 sigma RMS of the oracle."""
    mem = M.vesicle_62k()
    g, m, o = pair(mem, gkw={"precision": G.F64_ALL})
    g.init_cells()
    o.init_cells()
    g.integrate(50)
    o.integrate(50)
    sg, so = g.state(), o.state()
    rms = np.sqrt(((sg["pos"] - so["pos"]) ** 2).sum(1).mean())
    assert rms <= 1e-9, rms
    g.close()


# --------------------------------------------------------------------------- standalone stable sort

@pytest.mark.parametrize("n,K,big", [(100_000, 2000, False), (50_000, 9, True), (3, 5, False), (0, 4, False)])
def test_cell_sort_entry_point(n, K, big):
    """orbc_cell_sort on device memory equals numpy's stable argsort by cell,
    including empty cells and cells beyond the warp and block sorts."""
    import torch
    rng = np.random.default_rng(n + K)
    cell = rng.integers(0, K, size=n).astype(np.int32)
    if big:
        cell[: n // 2] = 3          # one cell of > 2,048 items
        cell[n // 2: n // 2 + 500] = 7
    d = torch.from_numpy(cell).cuda()
    perm, start = G.cell_sort(d, K)
    torch.cuda.synchronize()
    assert np.array_equal(perm.cpu().numpy(), np.argsort(cell, kind="stable").astype(np.int32))
    want = np.concatenate([[0], np.cumsum(np.bincount(cell, minlength=K))]).astype(np.int32)
    assert np.array_equal(start.cpu().numpy(), want)
    if n:
        bad = d.clone()
        bad[0] = K
        with pytest.raises(G.OrbcError):
            G.cell_sort(bad, K)
