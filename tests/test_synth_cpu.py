"""The seeded synthetic workloads against their stated recipes: particle,
junction, bead and bond counts, centroid counts, boxes, geometry, thermal
initial velocities and determinism.  The benchmark's and the parity tests'
inputs come from these generators, so a drift here would silently change
the measured workload."""
import math

import numpy as np
import pytest

from synth import membranes as M

SPACING = 1.12
AREA_PER_LIPID = math.sqrt(3.0) / 2.0 * SPACING ** 2


def _common(mem):
    n = mem.n
    assert mem.pos.shape == (n, 3) and mem.vel.shape == (n, 3) and mem.ori.shape == (n, 3)
    assert np.array_equal(np.sort(mem.id), np.arange(n))
    assert set(np.unique(mem.type)) <= {0, 1, 2}
    lip = mem.type == 0
    assert np.abs(np.linalg.norm(mem.ori[lip], axis=1) - 1.0).max() < 1e-12
    assert np.abs(np.sum(mem.ori[lip] * mem.angvel[lip], axis=1)).max() < 1e-12
    b = np.asarray(mem.bonds)
    assert b.ndim == 2 and b.shape[1] == 2 and len(b) == len(mem.r0) == len(mem.kb)
    if len(b):
        assert b.min() >= 0 and b.max() < n and np.all(b[:, 0] != b[:, 1])
        assert np.all(mem.r0 > 0) and np.all(mem.kb > 0)


def _median_6nn(p):
    """Median distance to the six nearest neighbours (1.12 sigma on a
    hexagonal packing; the single nearest is shorter once jittered)."""
    from scipy.spatial import cKDTree
    d, _ = cKDTree(p).query(p, k=7)
    return float(np.median(d[:, 1:]))


def test_flat_patch_2304():
    mem = M.flat_patch_2304()
    _common(mem)
    counts = np.bincount(mem.type, minlength=3)
    assert mem.n == 2304 and counts.tolist() == [2048, 16, 240]      # 32 x 64 lipids, 16 junctions, 24 chains of 10
    assert len(mem.r0) == 24 * 11 and mem.n_centroids == 64 and mem.kT == 0.2
    assert mem.box[0] == pytest.approx(32 * SPACING) and mem.box[1] == pytest.approx(64 * SPACING * math.sqrt(3) / 2)
    assert mem.periodic.tolist() == [1, 1, 0]
    lp = mem.pos[mem.type == 0]
    assert _median_6nn(lp) == pytest.approx(SPACING, abs=0.02)
    # the network lies 1 sigma below the lipid sheet
    assert np.mean(mem.pos[mem.type == 1][:, 2]) == pytest.approx(np.mean(lp[:, 2]) - 1.0, abs=0.05)


def test_vesicle_62k():
    mem = M.vesicle_62k()
    _common(mem)
    counts = np.bincount(mem.type, minlength=3)
    # frequency-6 icosphere: 10 f^2 + 2 junctions, 30 f^2 edges of 20 beads (21 bonds each)
    assert counts.tolist() == [40000, 362, 1080 * 20] and mem.n == 61962
    assert len(mem.r0) == 1080 * 21 and mem.n_centroids == 1024
    R = math.sqrt(40000 * AREA_PER_LIPID / (4 * math.pi))
    rl = np.linalg.norm(mem.pos[mem.type == 0], axis=1)
    assert np.median(rl) == pytest.approx(R, abs=0.01) and R == pytest.approx(58.80, abs=0.01)
    assert np.median(np.linalg.norm(mem.pos[mem.type == 1], axis=1)) == pytest.approx(R - 1.0, abs=0.01)
    # outward directors
    lp = mem.pos[mem.type == 0]
    assert np.min(np.sum(lp * mem.ori[mem.type == 0], axis=1) / rl) > 0.99


def test_rbc_4m():
    mem = M.rbc_4m()
    _common(mem)
    counts = np.bincount(mem.type, minlength=3)
    assert mem.n == 4_000_000 and counts[0] == 3_571_024 and counts[1] == 33_000
    # 4-bead chains on the triangulation's edges, 5 bonds each
    assert counts[2] == 4 * mem.meta["n_edges"] and len(mem.r0) == 5 * mem.meta["n_edges"]
    assert mem.n_centroids == 65_536 and mem.periodic.tolist() == [0, 0, 0]
    # the surface is scaled so that each lipid has the area of a 1.12 sigma hexagonal packing
    area_sigma2 = mem.meta["area_um2"] * mem.meta["sigma_per_um"] ** 2
    assert area_sigma2 == pytest.approx(counts[0] * AREA_PER_LIPID, rel=1e-3)
    # lipid spacing close to 1.12 sigma: every lipid of a slab through the cell
    lp = mem.pos[mem.type == 0]
    slab = lp[np.abs(lp[:, 0]) < 20.0]
    assert _median_6nn(slab) == pytest.approx(SPACING, abs=0.05)
    # thermal start: 3/2 kT translational per particle, kT rotational per lipid
    assert np.mean(0.5 * np.sum(mem.vel ** 2, axis=1)) == pytest.approx(1.5 * mem.kT, rel=0.01)
    assert np.mean(0.5 * np.sum(mem.angvel[mem.type == 0] ** 2, axis=1)) == pytest.approx(mem.kT, rel=0.01)


def test_generators_are_deterministic():
    a, b = M.vesicle(3000, 5, f=2, chain_beads=5, n_centroids=50), M.vesicle(3000, 5, f=2, chain_beads=5, n_centroids=50)
    for k in ("pos", "vel", "ori", "angvel", "type", "id", "bonds", "r0", "kb"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
    c = M.vesicle(3000, 6, f=2, chain_beads=5, n_centroids=50)
    assert not np.array_equal(a.vel, c.vel)


def test_ensemble_members():
    sizes = []
    for i in range(64):
        m = M.ensemble_member(i)
        sizes.append(m.n)
        assert 4000 <= m.n <= 260_000, (i, m.n)
        assert m.n_centroids == max(1, round(m.n / 61)) or abs(m.n_centroids - m.n / 61) <= 1
        assert 0.1 <= m.kT <= 0.3
        if i < 4:
            _common(m)
    # log-uniform sizes: both ends of [5k, 200k] are represented
    assert min(sizes) < 20_000 and max(sizes) > 80_000


def test_request_stream():
    rs = M.request_stream(256)
    assert len(rs) == 256
    t = [r["arrival_s"] for r in rs]
    assert all(t[i] <= t[i + 1] for i in range(255)) and t[0] >= 0
    assert all(100 <= r["steps"] <= 2000 for r in rs)
    n = np.array([r["n_est"] for r in rs])
    assert n.min() >= 5_000 and n.max() <= 1_300_000
    assert np.median(n) > 50_000
