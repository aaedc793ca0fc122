"""The fused step (each force launch runs the next step's B-A-O-A update in
its epilogue) against the separate launches: the same trajectory bit for
bit, in both FP32-force modes, with bonds, proteins, a periodic box, the
volume constraint, the skin cadence and separate protein cells; and the
fused path against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from synth import membranes as M

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_1701_02059_gb300")


def vesicle():
    return M.vesicle(3000, 5, f=2, chain_beads=5, n_centroids=50)


def run(mem, fuse, steps, vol=None, **kw):
    d = dict(kT=mem.kT, n_centroids=mem.n_centroids, box=mem.box, periodic=mem.periodic, seed=9)
    d.update(kw)
    g = G.System(G.make_params(**d))
    g.set_step_fusion(fuse)
    g.load_membrane(mem)
    if vol is not None:
        g.set_volume_constraint(*vol)
    g.init_cells()
    g.integrate(steps)
    g.integrate(3)          # a second call: the pipeline restarts from valid forces
    st = g.state()
    F, T = g.forces()
    g.close()
    return st, F, T


CASES = {
    "vesicle-f64-increments": (vesicle, {}, None),
    "vesicle-f32-increments": (vesicle, {"precision": G.F32_FORCE_F32_STEP}, None),
    "patch-periodic": (M.flat_patch_2304, {}, None),
    "vesicle-volume": (vesicle, {}, (0.01, 17000.0, M.AREA_PER_LIPID, (0.0, 0.0, 0.0))),
    "vesicle-cadence": (vesicle, {"rebuild_every": 5, "skin": 0.3}, None),
    "detached-separate-cells": (lambda: M.vesicle(3000, 5, f=2, chain_beads=5, n_centroids=50, detach_upper=4.0),
                                {"n_protein_centroids": 12}, None),
}


@pytest.mark.parametrize("name", list(CASES))
def test_fused_and_separate_launches_are_bit_identical(name):
    make, kw, vol = CASES[name]
    mem = make()
    a = run(mem, True, 40, vol, **kw)
    b = run(mem, False, 40, vol, **kw)
    for k in ("pos", "vel", "ori", "angvel", "step"):
        assert np.array_equal(a[0][k], b[0][k]), k
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_fused_trajectory_matches_oracle():
    mem = vesicle()
    g = G.System(G.make_params(kT=mem.kT, n_centroids=mem.n_centroids, seed=0))
    g.load_membrane(mem)
    m = oracle.model()
    o = oracle.OracleSystem(m, oracle.run(kT=mem.kT, n_centroids=mem.n_centroids, seed=0))
    o.load(mem)
    g.init_cells()
    o.init_cells()
    g.integrate(100)
    o.integrate(100)
    sg, so = g.state(), o.state()
    rms = np.sqrt(((sg["pos"] - so["pos"]) ** 2).sum(1).mean())
    assert sg["step"] == so["step"] == 100 and rms <= 1e-5, rms
    g.close()
