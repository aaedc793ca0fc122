"""Harmonic volume constraint and upper-rim height map on the GPU (through
the C ABI) against the FP64 oracle.

Tolerances (stated, from the arithmetic):
  * volume query (FP64 terms each rounded to 2^-48 sigma^3 before an exact
    integer sum; the oracle sums its FP64 terms serially):
    |dV| <= N_lipid (2^-49 + 2^-52 |V|), the rounding of the GPU's terms
    plus the serial-summation bound with sum |term| <= 2 |V|;
  * forces and torques with the constraint on: the pair tolerances, FP32
    forces e_F <= 1e-5, FP64 everywhere e_F <= 1e-8;
  * bond + constraint energy: relative 1e-6 (FP32 terms of V), 1e-10 (FP64);
  * 100-step trajectories: RMS position deviation <= 1e-5 sigma (FP32
    forces), <= 1e-9 sigma (FP64 everywhere);
  * height map: bin counts bit-exact (every decision in FP64 with correctly
    rounded operations on the same state on both sides), bin means within
    1e-12 of the largest |z| (integer sum against a serial FP64 sum).
"""
import math

import numpy as np
import pytest

import oracle
from synth import membranes as M

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_1701_02059_gb300")
from paper_1701_02059_gb300 import _native  # noqa: E402

A_LIP = M.AREA_PER_LIPID


def vesicle():
    return M.vesicle(3000, 5, f=2, chain_beads=5, n_centroids=50)


def pair(mem, precision=0, seed=0):
    g = G.System(G.make_params(kT=mem.kT, n_centroids=mem.n_centroids, box=mem.box, periodic=mem.periodic,
                               seed=seed, precision=precision))
    g.load_membrane(mem)
    m = oracle.model(box=mem.box, periodic=mem.periodic)
    o = oracle.OracleSystem(m, oracle.run(kT=mem.kT, n_centroids=mem.n_centroids, seed=seed))
    o.load(mem)
    return g, o


def volume_close(vg, vo, n_lip):
    return abs(vg - vo) <= n_lip * (2.0 ** -49 + 2.0 ** -52 * abs(vo))


def force_error(Fg, Fo):
    frms = np.sqrt((Fo ** 2).sum(1).mean())
    return (np.linalg.norm(Fg - Fo, axis=1) / np.maximum(np.linalg.norm(Fo, axis=1), frms)).max(), frms


XC = (0.25, -0.5, 0.375)          # on the state grid, off the vesicle's centre


def test_volume_query_matches_oracle():
    mem = vesicle()
    g, o = pair(mem)
    for xc in ((0.0, 0.0, 0.0), XC):
        assert volume_close(g.volume(A_LIP, xc), o.volume(A_LIP, xc), int((mem.type == 0).sum()))
    R = mem.meta["R"]
    # a nearly spherical vesicle of radius R encloses about 4/3 pi R^3
    assert g.volume(A_LIP, XC) == pytest.approx(4.0 / 3.0 * math.pi * R ** 3, rel=0.02)
    g.close()


@pytest.mark.parametrize("precision", [G.F32_FORCE_F64_STATE, G.F64_ALL, G.F32_FORCE_F32_STEP])
def test_constraint_forces_and_energy_match_oracle(precision):
    mem = vesicle()
    g, o = pair(mem, precision)
    V = o.volume(A_LIP, XC)
    kv, V0 = 0.02, 0.97 * V
    g.set_volume_constraint(kv, V0, A_LIP, XC)
    o.set_volume(kv, V0, A_LIP, XC)
    g.init_cells()
    o.init_cells()
    eg = g.compute_forces(energies=True)
    eo = o.compute_forces()
    Fg, Tg = g.forces()
    Fo, To = o.forces()
    tol = 1e-8 if precision == G.F64_ALL else 1e-5
    ef, frms = force_error(Fg, Fo)
    assert ef <= tol, ef
    trms = np.sqrt((To ** 2).sum(1).mean())
    assert np.linalg.norm(Tg - To, axis=1).max() / max(trms, frms) <= tol
    u_v = 0.5 * kv * (V - V0) ** 2
    assert u_v > 0.1 * abs(eo[1])                   # the constraint is a visible part of the bond energy
    assert eg[1] == pytest.approx(eo[1], rel=1e-10 if precision == G.F64_ALL else 1e-6)
    assert eg[0] == pytest.approx(eo[0], rel=1e-10 if precision == G.F64_ALL else 1e-6)
    g.close()


@pytest.mark.parametrize("precision", [G.F32_FORCE_F64_STATE, G.F64_ALL])
def test_trajectory_with_constraint_matches_oracle(precision):
    mem = vesicle()
    g, o = pair(mem, precision)
    V = o.volume(A_LIP, XC)
    g.set_volume_constraint(0.01, 0.95 * V, A_LIP, XC)
    o.set_volume(0.01, 0.95 * V, A_LIP, XC)
    g.init_cells()
    o.init_cells()
    g.integrate(100)
    o.integrate(100)
    sg, so = g.state(), o.state()
    rms = np.sqrt(((sg["pos"] - so["pos"]) ** 2).sum(1).mean())
    assert rms <= (1e-9 if precision == G.F64_ALL else 1e-5), rms
    # the constraint acted: the vesicle shrank toward V0
    assert g.volume(A_LIP, XC) < V - 1e-3 * V
    g.close()


def test_constraint_off_is_bit_identical_and_survives_reload():
    mem = vesicle()
    g, _ = pair(mem)
    g.init_cells()
    g.compute_forces()
    F0, T0 = g.forces()
    V = g.volume(A_LIP, XC)
    g.set_volume_constraint(0.02, 0.97 * V, A_LIP, XC)
    g.compute_forces()
    F1, _ = g.forces()
    assert not np.array_equal(F0, F1)
    g.set_volume_constraint(0.0, 0.0, 0.0, XC)
    g.compute_forces()
    F2, T2 = g.forces()
    assert np.array_equal(F0, F2) and np.array_equal(T0, T2)
    # the setting is kept when the particles are loaded again
    g.set_volume_constraint(0.02, 0.97 * V, A_LIP, XC)
    g.load_membrane(mem)
    g.init_cells()
    g.compute_forces()
    F3, _ = g.forces()
    assert np.array_equal(F1, F3)
    g.close()


def test_constraint_argument_errors():
    mem = M.flat_patch_2304()
    g = G.System(G.make_params(kT=mem.kT, n_centroids=mem.n_centroids, box=mem.box, periodic=mem.periodic))
    g.load_membrane(mem)
    with pytest.raises(G.OrbcError) as e:
        g.set_volume_constraint(0.1, 100.0, A_LIP, (0, 0, 0))      # periodic box
    assert e.value.code == _native.ORBC_E_ARG
    g.close()
    mem = vesicle()
    g, _ = pair(mem)
    for bad in ((-1.0, 1.0, A_LIP), (0.1, 1.0, 0.0), (0.1, float("nan"), A_LIP)):
        with pytest.raises(G.OrbcError) as e:
            g.set_volume_constraint(*bad, (0, 0, 0))
        assert e.value.code == _native.ORBC_E_ARG
    with pytest.raises(G.OrbcError):
        g.height_map(0, 0, 0.0, 1.0, 4, 4, 0.0)
    with pytest.raises(G.OrbcError):
        g.height_map(0, 0, 1.0, 1.0, 0, 4, 0.0)
    g.close()


def _height_cases(R):
    return [
        # x0, y0, dx, dy, nx, ny, z_min, axis, rho_in, rho_out
        (-R, -R, 2.0, 2.0, int(R), int(R), 0.0, (0.0, 0.0), 0.3 * R, 0.9 * R),        # few hundred bins: shared path
        (-R, -R, 0.5, 0.5, 4 * int(R), 4 * int(R), 0.2 * R, (1.0, -2.0), 0.0, 1e9),    # > 1024 bins: global path
        (-R, -R, 2.0, 2.0, 8, 8, 2.0 * R, (0.0, 0.0), 0.0, 1e9),                        # nothing selected
    ]


def test_height_map_matches_oracle_on_the_gpu_state():
    mem = vesicle()
    g, _ = pair(mem)
    g.init_cells()
    g.integrate(30)
    st = g.state()
    m = oracle.model()
    o = oracle.OracleSystem(m, oracle.run(kT=mem.kT, n_centroids=mem.n_centroids))
    o.set_particles(st["pos"], st["vel"], st["ori"], st["angvel"], mem.type, mem.id)
    R = mem.meta["R"]
    totals = []
    for case in _height_cases(R):
        hg, cg = g.height_map(*case)
        ho, co = o.height_map(*case)
        assert np.array_equal(cg, co), case
        assert np.abs(hg - ho).max() <= 1e-12 * R
        totals.append(int(cg.sum()))
    assert totals[0] > 200 and totals[1] > 200 and totals[2] == 0
    g.close()


# --------------------------------------------------------------------------- full-size 4M cell

@pytest.fixture(scope="module")
def rbc():
    mem = M.rbc_4m()
    g = G.System(G.make_params(kT=mem.kT, n_centroids=mem.n_centroids, box=mem.box, periodic=mem.periodic, seed=2))
    g.load_membrane(mem)
    g.init_cells()
    yield mem, g
    g.close()


def test_rbc_volume_and_height_map_full_size(rbc):
    """The 4,000,000-particle cell: the volume query and an upper-rim height
    map equal the oracle's on the same (grid-exact) state, and a constrained
    step runs clean."""
    mem, g = rbc
    st = g.state()
    o = oracle.OracleSystem(oracle.model(), oracle.run(kT=mem.kT, n_centroids=mem.n_centroids))
    o.set_particles(st["pos"], st["vel"], st["ori"], st["angvel"], mem.type, mem.id)
    V = g.volume(A_LIP, (0.0, 0.0, 0.0))
    assert volume_close(V, o.volume(A_LIP, (0.0, 0.0, 0.0)), int((mem.type == 0).sum()))
    s = mem.meta["sigma_per_um"]
    # the Evans-Fung cell encloses about 94 um^3
    assert V / s ** 3 == pytest.approx(94.0, rel=0.05)
    rim = (-4.0 * s, -4.0 * s, 0.25 * s, 0.25 * s, 32, 32, 0.0, (0.0, 0.0), 2.5 * s, 3.9 * s)
    hg, cg = g.height_map(*rim)
    ho, co = o.height_map(*rim)
    assert np.array_equal(cg, co) and cg.sum() > 100_000
    assert np.abs(hg - ho).max() <= 1e-12 * 4.0 * s
    g.set_volume_constraint(1e-6, V, A_LIP, (0.0, 0.0, 0.0))
    g.integrate(3)
    assert np.isfinite(g.state()["pos"]).all()
    g.set_volume_constraint(0.0, 0.0, 0.0, (0.0, 0.0, 0.0))
