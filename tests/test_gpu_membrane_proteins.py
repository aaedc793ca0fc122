"""The two-component model's bilayer proteins on the GPU (through the C ABI)
against the FP64 oracle: band-3 and glycophorin as oriented bilayer
particles with their own well depths and cutoffs per species pair, anchored
to the spectrin network by bonds that exclude their 1-2 and 1-3 pairs from
the WCA term ("Initial structure generation"; "Force Evaluation": protein
interactions through the lipid cells with their own cutoffs).

Tolerances as for the lipid-only model: cells, permutation, centroids,
radii, neighbouring cells and the pair set bit-exact; forces and torques
e_F <= 1e-5 (FP32 forces) and <= 1e-8 (FP64); 100-step trajectories
<= 1e-5 sigma RMS (FP32 forces) and <= 1e-9 sigma (FP64).  With the default
table a protein is a relabelled lipid, so relabelling leaves forces and
trajectories bit-identical (the species-pair evaluation against the
lipid-only one).
"""
import math

import numpy as np
import pytest

import oracle
from synth import membranes as M

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_1701_02059_gb300")
from paper_1701_02059_gb300 import _native  # noqa: E402
from test_gpu_ties import exact_distance_pair, grid  # noqa: E402

# well depth and cutoff per bilayer species pair (lipid, band-3, glycophorin);
# 0: the lipid-lipid value
TE = np.array([[0.0, 1.2, 0.9], [1.2, 1.4, 1.1], [0.9, 1.1, 0.0]])
TR = np.array([[0.0, 2.8, 0.0], [2.8, 2.9, 2.7], [0.0, 2.7, 0.0]])


def vesicle_proteins():
    return M.with_membrane_proteins(M.vesicle(3000, 5, f=2, chain_beads=5, n_centroids=50), seed=1)


def patch_proteins():
    return M.with_membrane_proteins(M.flat_patch_2304(), seed=2)


WORKLOADS = {"vesicle": vesicle_proteins, "patch": patch_proteins}


def pair(mem, precision=0, table=True, **kw):
    tab = dict(eps_mem=TE, rc_mem=TR) if table else {}
    g = G.System(G.make_params(kT=mem.kT, n_centroids=mem.n_centroids, box=mem.box, periodic=mem.periodic, seed=0,
                               precision=precision, **tab, **kw))
    g.load_membrane(mem)
    m = oracle.model(box=mem.box, periodic=mem.periodic, mem_eps=TE if table else None, mem_rc=TR if table else None)
    o = oracle.OracleSystem(m, oracle.run(kT=mem.kT, n_centroids=mem.n_centroids, seed=0, **kw))
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


def errors(g, o):
    Fg, Tg = g.forces()
    Fo, To = o.forces()
    frms = np.sqrt((Fo ** 2).sum(1).mean())
    ef = (np.linalg.norm(Fg - Fo, axis=1) / np.maximum(np.linalg.norm(Fo, axis=1), frms)).max()
    trms = np.sqrt((To ** 2).sum(1).mean())
    et = np.linalg.norm(Tg - To, axis=1).max() / max(trms, frms)
    return ef, et


def test_workloads_hold_the_protein_set():
    for name, make in WORKLOADS.items():
        mem = make()
        cnt = np.bincount(mem.type, minlength=5)
        assert cnt[M.BAND3] > 0 and cnt[M.GLYCOPHORIN] > 0, name
        bil = np.isin(mem.type, M.BILAYER)
        anchors = bil[mem.bonds[:, 0]] != bil[mem.bonds[:, 1]]
        assert anchors.sum() > 0, name


@pytest.mark.parametrize("name", list(WORKLOADS))
@pytest.mark.parametrize("precision", [G.F32_FORCE_F64_STATE, G.F64_ALL])
def test_cells_pairs_forces_energies_match_oracle(name, precision):
    mem = WORKLOADS[name]()
    g, m, o = pair(mem, precision=precision)
    g.init_cells()
    o.init_cells()
    assert_cells_equal(g, o)
    pairs = g.pairs()
    assert np.array_equal(pairs, sorted_pairs(o.pairs()))
    # every anchor's own pair is absent from the pair set (1-2 exclusion),
    # while band-3-lipid pairs beyond the lipid cutoff are present
    ps = {tuple(p) for p in pairs.tolist()}
    bil = np.isin(mem.type, M.BILAYER)
    for a, b in mem.bonds[bil[mem.bonds[:, 0]] != bil[mem.bonds[:, 1]]].tolist():
        assert (min(a, b), max(a, b)) not in ps
    st = o.state()
    far = [p for p in ps if {mem.type[p[0]], mem.type[p[1]]} == {M.BAND3, M.LIPID}
           and np.linalg.norm(st["pos"][p[0]] - st["pos"][p[1]]) > 2.6]
    assert len(far) > 0
    eg = g.compute_forces(energies=True)
    eo = o.compute_forces()
    ef, et = errors(g, o)
    tol = 1e-8 if precision == G.F64_ALL else 1e-5
    assert ef <= tol and et <= tol, (ef, et)
    assert abs(eg[0] - eo[0]) <= 1e-6 * abs(eo[0])
    assert abs(eg[1] - eo[1]) <= 1e-6 * max(abs(eo[1]), 1.0)
    assert eg[3] == pytest.approx(eo[3], rel=1e-9)
    g.close()


@pytest.mark.parametrize("precision", [G.F32_FORCE_F64_STATE, G.F64_ALL])
def test_trajectory_100_steps_matches_oracle(precision):
    mem = vesicle_proteins()
    g, m, o = pair(mem, precision=precision)
    g.init_cells()
    o.init_cells()
    g.integrate(100)
    o.integrate(100)
    sg, so = g.state(), o.state()
    assert sg["step"] == so["step"] == 100
    tol = 1e-9 if precision == G.F64_ALL else 1e-5
    rms = np.sqrt(((sg["pos"] - so["pos"]) ** 2).sum(1).mean())
    assert rms <= tol, rms
    pro = np.isin(mem.type, (M.BAND3, M.GLYCOPHORIN))
    assert np.sqrt(((sg["ori"][pro] - so["ori"][pro]) ** 2).sum(1).mean()) <= tol
    # the proteins' directors turned (they carry the rotational integrator)
    assert np.abs(sg["ori"][pro] - mem.ori[pro]).max() > 1e-3
    # the GPU's own cells still exact after 100 rebuilds
    c = g.cells()
    assert np.array_equal(c["cell_of_id"], oracle.assign_brute(sg["pos"], c["centroids"], mem.box, mem.periodic))
    assert np.array_equal(g.pairs(), sorted_pairs(oracle.pairs_brute(m, sg["pos"], mem.type, mem.id, mem.bonds)))
    g.close()


@pytest.mark.parametrize("precision", [G.F32_FORCE_F64_STATE, G.F32_FORCE_F32_STEP])
def test_default_table_relabelling_is_bit_identical(precision):
    """Lipids relabelled as band-3 and glycophorin with no table: the
    species-pair evaluation gives the lipid-only evaluation's forces,
    energies and 30-step trajectory bit for bit."""
    mem = M.vesicle(3000, 5, f=2, chain_beads=5, n_centroids=50)
    relab = mem.copy()
    rng = np.random.default_rng(4)
    pick = rng.choice(np.flatnonzero(mem.type == M.LIPID), 300, replace=False)
    relab.type[pick[:200]] = M.BAND3
    relab.type[pick[200:]] = M.GLYCOPHORIN
    out = []
    for mm in (mem, relab):
        g = G.System(G.make_params(kT=mm.kT, n_centroids=mm.n_centroids, seed=6, precision=precision))
        g.load_membrane(mm)
        g.init_cells()
        e = g.compute_forces(energies=True)
        F = g.forces()
        g.integrate(30)
        out.append((e, F, g.state(), g.forces()))
        g.close()
    (ea, Fa, sa, Ga), (eb, Fb, sb, Gb) = out
    assert np.array_equal(ea, eb)
    for x, y in zip(Fa + Ga, Fb + Gb):
        assert np.array_equal(x, y)
    for k in ("pos", "vel", "ori", "angvel"):
        assert np.array_equal(sa[k], sb[k]), k


SPECIES = {M.LIPID: 0, M.BAND3: 1, M.GLYCOPHORIN: 2}


def cutoff_of(ti, tj):
    if ti in SPECIES and tj in SPECIES:
        return TR[SPECIES[ti], SPECIES[tj]] or 2.6
    if ti in SPECIES or tj in SPECIES:
        return 2.0 ** (1.0 / 6.0)
    return 0.5 * 2.0 ** (1.0 / 6.0)


@pytest.mark.parametrize("precision", [G.F32_FORCE_F64_STATE, G.F64_ALL, G.F32_FORCE_F32_STEP])
def test_species_cutoffs_at_and_around_the_boundary(precision):
    """Probe pairs of every bilayer species pair and a band-3-spectrin pair
    at d^2 == r_c^2 exactly (excluded: the test is strict) and at
    r_c -+ 1e-7 and -+ 2e-6 sigma, near 700 sigma from the origin: the pair
    set equals the oracle's brute force, which includes exactly the probes
    inside."""
    probes = [(M.BAND3, M.LIPID), (M.BAND3, M.BAND3), (M.BAND3, M.GLYCOPHORIN), (M.GLYCOPHORIN, M.LIPID),
              (M.GLYCOPHORIN, M.GLYCOPHORIN), (M.BAND3, M.SPECTRIN)]
    pos, typ, cents = [], [], []
    x0, y0 = 700.0, 700.0
    q = 0
    for ti, tj in probes:
        rc = cutoff_of(ti, tj)
        offsets = [exact_distance_pair(rc * rc, axes) for axes in ((0, 1), (2, 0))]
        u = np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)
        offsets += [grid((rc + dr) * u) for dr in (-1e-7, 1e-7, -2e-6, 2e-6)]
        for d in offsets:
            base = grid([x0 + 10.0 * q, y0, 0.0])
            pos += [base, base + d]
            typ += [ti, tj]
            cents.append(base + grid(d / 2) + np.array([0.0, 0.0, 0.5]))
            q += 1
    npb = len(pos)
    # lipids near every centroid, at least 0.9 sigma from every other
    # particle, so that the forces have their usual scale
    rng = np.random.default_rng(7)
    for c in cents:
        placed = 0
        while placed < 3:
            p = grid(np.asarray(c) + rng.uniform(-1.5, 1.5, 3) * np.array([1, 1, 0.3]))
            if np.linalg.norm(np.asarray(pos) - p, axis=1).min() < 0.9:
                continue
            pos.append(p)
            typ.append(M.LIPID)
            placed += 1
    n = len(pos)
    ori = np.zeros((n, 3))
    ori[np.isin(typ, M.BILAYER), 2] = 1.0
    mem = M.Membrane(np.array(pos), np.zeros((n, 3)), ori, np.zeros((n, 3)), np.array(typ, np.uint8),
                     np.arange(n, dtype=np.uint32), np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(0),
                     np.zeros(3), np.zeros(3, np.int32), len(cents), 0.2)
    g, m, o = pair(mem, precision=precision, n_lloyd_init=0)
    g.init_cells(np.array(cents))
    o.init_cells(np.array(cents))
    assert_cells_equal(g, o)
    st = o.state()
    brute = sorted_pairs(oracle.pairs_brute(m, st["pos"], mem.type, mem.id))
    assert np.array_equal(g.pairs(), brute)
    ps = {tuple(p) for p in brute.tolist()}
    inside = 0
    for k in range(0, npb, 2):
        d = st["pos"][k + 1] - st["pos"][k]
        d2 = d[0] * d[0]
        d2 = d2 + d[1] * d[1]
        d2 = d2 + d[2] * d[2]
        want = d2 < cutoff_of(int(mem.type[k]), int(mem.type[k + 1])) ** 2
        assert ((k, k + 1) in ps) == want
        inside += want
    assert inside == 2 * len(probes)
    g.compute_forces()
    o.compute_forces()
    ef, et = errors(g, o)
    assert ef <= (1e-8 if precision == G.F64_ALL else 1e-5), ef
    g.close()


def test_volume_and_separate_cells_take_the_bilayer():
    """The enclosed volume sums over every bilayer particle, and a separate
    protein cell set puts band-3 and glycophorin in the bilayer's cells; a
    network without anchors (detached) matches the oracle exactly."""
    mem = M.with_membrane_proteins(M.vesicle(3000, 7, f=2, chain_beads=5, n_centroids=50, net_offset=5.0), seed=3,
                                   glycophorin=False, anchored_beads=0.0, mobile_band3=0.1)
    assert (mem.type == M.BAND3).sum() > 200
    g, m, o = pair(mem, n_protein_centroids=12)
    g.init_cells()
    o.init_cells()
    assert_cells_equal(g, o)
    c = g.cells()
    bil = np.isin(mem.type, M.BILAYER)
    assert (c["cell_of_id"][bil] < mem.n_centroids).all() and (c["cell_of_id"][~bil] >= mem.n_centroids).all()
    assert np.array_equal(g.pairs(), sorted_pairs(o.pairs()))
    center = np.zeros(3)
    vg = g.volume(1.0, center)
    vo = o.volume(1.0, center)
    n = mem.n
    assert abs(vg - vo) <= n * (2.0 ** -49 + 2.0 ** -52 * abs(vo))
    # every bilayer particle counts: relabelling the band-3 as lipids
    # leaves the volume unchanged
    lip_only = mem.copy()
    lip_only.type[lip_only.type == M.BAND3] = M.LIPID
    assert vo == pytest.approx(oracle_volume_of(lip_only), rel=1e-12)
    g.integrate(20)
    o.integrate(20)
    assert np.sqrt(((g.state()["pos"] - o.state()["pos"]) ** 2).sum(1).mean()) <= 1e-5
    g.close()


def oracle_volume_of(mem):
    m = oracle.model(box=mem.box, periodic=mem.periodic)
    o = oracle.OracleSystem(m, oracle.run(kT=mem.kT, n_centroids=mem.n_centroids, seed=0))
    o.load(mem)
    return o.volume(1.0, np.zeros(3))


def test_invalid_species_tables_and_types_are_refused():
    bad = [dict(eps_mem=[[0, 1, 0], [2, 0, 0], [0, 0, 0]]),          # asymmetric
           dict(eps_mem=[[1.5, 0, 0], [0, 0, 0], [0, 0, 0]]),        # lipid-lipid entry set
           dict(rc_mem=[[0, 1.0, 0], [1.0, 0, 0], [0, 0, 0]]),       # cutoff inside r_min
           dict(eps_mem=[[0, -1, 0], [-1, 0, 0], [0, 0, 0]]),        # negative
           dict(rc_mem=[[0, np.nan, 0], [np.nan, 0, 0], [0, 0, 0]])]  # not finite
    for kw in bad:
        with pytest.raises(G.OrbcError) as e:
            G.System(G.make_params(**kw))
        assert e.value.code == _native.ORBC_E_ARG, kw
    mem = vesicle_proteins()
    g = G.System(G.make_params(kT=mem.kT, n_centroids=mem.n_centroids))
    typ = mem.type.copy()
    typ[0] = 5
    with pytest.raises(G.OrbcError) as e:
        g.set_particles(mem.pos, mem.vel, mem.ori, mem.angvel, typ, mem.id)
    assert e.value.code == _native.ORBC_E_ARG
    # anchors with a separate protein cell set are refused (a detached network
    # has none)
    g2 = G.System(G.make_params(kT=mem.kT, n_centroids=mem.n_centroids, n_protein_centroids=8))
    g2.load_membrane(mem)
    with pytest.raises(G.OrbcError) as e:
        g2.init_cells()
    assert e.value.code == _native.ORBC_E_ARG
    g.close()
    g2.close()


# --------------------------------------------------------------------------- full-size 4M cell with the protein set

def test_rbc_proteins_trajectory_matches_oracle():
    """The 4,000,000-particle cell with 33,000 glycophorin, anchored and
    mobile band-3 and the species table: five steps on the GPU and in the
    oracle from the same state within 1e-5 sigma RMS."""
    mem = M.rbc_4m_proteins()
    g, m, o = pair(mem)
    g.init_cells()
    o.init_cells()
    g.integrate(5)
    o.integrate(5)
    sg, so = g.state(), o.state()
    rms = np.sqrt(((sg["pos"] - so["pos"]) ** 2).sum(1).mean())
    assert rms <= 1e-5, rms
    bil = np.isin(mem.type, M.BILAYER)
    assert np.sqrt(((sg["ori"][bil] - so["ori"][bil]) ** 2).sum(1).mean()) <= 1e-5
    g.close()


def test_anchored_lipids_take_the_exclusions():
    """Lipids (no band-3 or glycophorin) bonded to the junctions beneath
    them: their bilayer-cytoskeleton pairs within the anchor's 1-2 and 1-3
    reach lose the WCA term on the GPU as in the oracle."""
    mem = M.with_membrane_proteins(M.vesicle(3000, 5, f=2, chain_beads=5, n_centroids=50), seed=5,
                                   anchored_beads=0.1, mobile_band3=0.0)
    mem.type[np.isin(mem.type, (M.BAND3, M.GLYCOPHORIN))] = M.LIPID
    g, m, o = pair(mem, table=False)
    g.init_cells()
    o.init_cells()
    assert np.array_equal(g.pairs(), sorted_pairs(o.pairs()))
    bil = mem.type == M.LIPID
    ps = {tuple(p) for p in g.pairs().tolist()}
    for a, b in mem.bonds[bil[mem.bonds[:, 0]] != bil[mem.bonds[:, 1]]].tolist():
        assert (min(a, b), max(a, b)) not in ps
    g.compute_forces()
    o.compute_forces()
    ef, et = errors(g, o)
    assert ef <= 1e-5 and et <= 1e-5, (ef, et)
    g.integrate(30)
    o.integrate(30)
    assert np.sqrt(((g.state()["pos"] - o.state()["pos"]) ** 2).sum(1).mean()) <= 1e-5
    g.close()


@pytest.mark.parametrize("zeta,s0", [(3, 0.0), (4, 0.05)])
def test_species_pairs_with_other_potential_parameters(zeta, s0):
    """The species-pair evaluation's general instantiation (another tail
    exponent, a spontaneous-curvature term) against the oracle: pair set
    bit-exact, forces within the FP32 tolerance, 50-step trajectory."""
    mem = vesicle_proteins()
    tab = dict(eps_mem=TE, rc_mem=TR)
    g = G.System(G.make_params(kT=mem.kT, n_centroids=mem.n_centroids, seed=0, zeta=zeta, sin_theta0=s0, **tab))
    g.load_membrane(mem)
    m = oracle.model(zeta=zeta, sin_theta0=s0, mem_eps=TE, mem_rc=TR)
    o = oracle.OracleSystem(m, oracle.run(kT=mem.kT, n_centroids=mem.n_centroids, seed=0))
    o.load(mem)
    g.init_cells()
    o.init_cells()
    assert np.array_equal(g.pairs(), sorted_pairs(o.pairs()))
    g.compute_forces()
    o.compute_forces()
    ef, et = errors(g, o)
    assert ef <= 1e-5 and et <= 1e-5, (ef, et)
    g.integrate(50)
    o.integrate(50)
    assert np.sqrt(((g.state()["pos"] - o.state()["pos"]) ** 2).sum(1).mean()) <= 1e-5
    g.close()
