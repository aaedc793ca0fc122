"""Long constant-energy runs (gamma = 0, no noise) of a 3,642-particle
vesicle for 10^4 steps at dt = 0.005: the total energy of the GPU path in
its two FP32-force modes against the FP64 oracle's own, at the same dt.

The integrator is BAOAB with the friction switched off, i.e. velocity
Verlet with Cayley rotations ("Software Overview": force and torque, then
position and orientation update); its energy error is bounded (no secular
drift) at O(dt^2).  The FP32 pair forces are not exact gradients, and FP32
increments add rounding on every update, so each mode gets its own stated
bound on max_t |E(t) - E(0)| / |E(0)|:

  * oracle (FP64 forces and increments):                   <= 1e-4
  * FP32 forces, FP64 increments (ORBC_F32_FORCE_F64_STATE): <= 1e-4
  * FP32 forces, FP32 increments (ORBC_F32_FORCE_F32_STEP):  <= 2e-4

and the GPU's largest excursion may exceed the oracle's by at most 5e-5
of |E(0)| in the FP64-increment mode.
"""
import json
import os

import numpy as np
import pytest

import oracle
from synth import membranes as M

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_1701_02059_gb300")

STEPS, EVERY, DT = 10_000, 1_000, 0.005


def vesicle():
    return M.vesicle(3000, 5, f=2, chain_beads=5, n_centroids=50)


def gpu_energy_series(mem, precision):
    p = G.make_params(kT=0.0, gamma_t=0.0, gamma_r=0.0, dt=DT, n_centroids=mem.n_centroids, box=mem.box,
                      periodic=mem.periodic, seed=0, precision=precision)
    g = G.System(p)
    g.load_membrane(mem)
    g.init_cells()
    out = [g.compute_forces(energies=True)[:4].sum()]
    for _ in range(STEPS // EVERY):
        g.integrate(EVERY)
        out.append(g.compute_forces(energies=True)[:4].sum())
    g.close()
    return np.array(out)


def oracle_energy_series(mem):
    o = oracle.OracleSystem(oracle.model(box=mem.box, periodic=mem.periodic),
                            oracle.run(kT=0.0, gamma_t=0.0, gamma_r=0.0, dt=DT, n_centroids=mem.n_centroids, seed=0))
    o.load(mem)
    o.init_cells()
    out = [o.compute_forces()[:4].sum()]
    for _ in range(STEPS // EVERY):
        o.integrate(EVERY)
        out.append(o.compute_forces()[:4].sum())
    return np.array(out)


def excursion(E):
    return float(np.abs(E - E[0]).max() / abs(E[0]))


def test_nve_energy_over_ten_thousand_steps():
    mem = vesicle()
    e_split = gpu_energy_series(mem, G.F32_FORCE_F64_STATE)
    e_f32 = gpu_energy_series(mem, G.F32_FORCE_F32_STEP)
    e_orc = oracle_energy_series(mem)
    d = {"oracle": excursion(e_orc), "f32_force_f64_step": excursion(e_split), "f32_force_f32_step": excursion(e_f32)}
    out = os.environ.get("ORBC_NVE_REPORT")
    if out:
        with open(out, "w") as f:
            json.dump({"excursions": d, "oracle": e_orc.tolist(), "f32_force_f64_step": e_split.tolist(),
                       "f32_force_f32_step": e_f32.tolist()}, f, indent=1)
    assert np.isfinite(e_split).all() and np.isfinite(e_f32).all()
    assert d["oracle"] <= 1e-4, d
    assert d["f32_force_f64_step"] <= 1e-4, d
    assert d["f32_force_f32_step"] <= 2e-4, d
    assert d["f32_force_f64_step"] <= d["oracle"] + 5e-5, d
