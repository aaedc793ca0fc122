"""Batched arena on the GPU: instances of uneven size packed into one batch,
admitted while others run, stepped by graph replay, retired when done.

The batch only concatenates per-instance work (per-cell kernels, per-
particle integrator, exact integer force sums, noise keyed by instance, id
and step), so every instance must come out bit-identical to the same
membrane run alone through the plain system API for the same number of
steps.  The plain system itself is held to the FP64 oracle by
test_gpu_parity.py.
"""
import numpy as np
import pytest

from synth import membranes as M

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_1701_02059_gb300")
from paper_1701_02059_gb300 import _native  # noqa: E402


def members():
    """Three uneven membranes: flat patches and a closed vesicle, each with
    its own temperature, seed and Philox instance word."""
    a = M.flat_patch_2304(seed=11)
    b = M.vesicle(3000, 12, kT=0.15, f=2, chain_beads=5, n_centroids=50)
    c = M.patch(3, 13, kT=0.25, n_centroids=85)
    return [a, b, c]


def params(mem, i, precision=G.F32_FORCE_F64_STATE):
    return G.make_params(kT=mem.kT, n_centroids=mem.n_centroids, box=mem.box, periodic=mem.periodic,
                         seed=1000 + i, instance=i, precision=precision)


def alone(mem, i, nsteps, precision=G.F32_FORCE_F64_STATE):
    g = G.System(params(mem, i, precision))
    g.load_membrane(mem)
    g.init_cells()
    g.integrate(nsteps)
    st = g.state()
    g.close()
    return st


def assert_same(a, b):
    for k in ("pos", "vel", "ori", "angvel"):
        assert np.array_equal(a[k], b[k]), f"{k}: max |diff| {np.abs(a[k] - b[k]).max()}"
    assert a["step"] == b["step"]


@pytest.mark.parametrize("graphs", [True, False])
def test_continuous_batching_equals_alone(graphs):
    mems = members()
    targets = [7, 12, 20]
    ar = G.Arena(8 << 30)
    s0 = ar.admit(params(mems[0], 0), mems[0], targets[0])
    s1 = ar.admit(params(mems[1], 1), mems[1], targets[1])
    assert ar.info()["pending"] == 2
    done = {}
    # first batch: instances 0 and 1, at most 5 steps per call
    assert ar.run(5, graphs) == 5
    assert ar.info()["resident"] == 2
    # instance 2 arrives while the others are resident
    s2 = ar.admit(params(mems[2], 2), mems[2], targets[2])
    slots = {s0: 0, s1: 1, s2: 2}
    calls = 0
    while len(done) < 3:
        ran = ar.run(5, graphs)
        calls += 1
        assert calls < 20
        for s in ar.poll():
            done[slots[s]] = ar.retire(s)
        if ran == 0:
            assert ar.info()["resident"] == 0
    assert ar.info() == {"resident": 0, "pending": 0, "done": 0, "particles": 0, "bytes": 0}
    assert ar.launch_count() > 0
    for i, mem in enumerate(mems):
        assert done[i]["step"] == targets[i]
        assert_same(done[i], alone(mem, i, targets[i]))
    ar.close()


def test_fp64_arena_equals_alone():
    mems = members()[:2]
    ar = G.Arena(8 << 30, precision=G.F64_ALL)
    slots = [ar.admit(params(m, i, G.F64_ALL), m, 6) for i, m in enumerate(mems)]
    assert ar.run(10) == 6
    got = {s: ar.retire(s) for s in ar.poll()}
    for i, m in enumerate(mems):
        assert_same(got[slots[i]], alone(m, i, 6, G.F64_ALL))


def test_mixed_potentials_in_one_batch_equal_alone():
    """Instances with other constants of the potential (zeta, mu, sin theta0)
    share a batch: the batch takes the kernels' general paths, which must
    reproduce each instance's own specialised run bit for bit."""
    mems = members()[:2]
    extra = [{}, dict(zeta=2, mu=2.5, sin_theta0=0.05)]

    def prm(i):
        return G.make_params(kT=mems[i].kT, n_centroids=mems[i].n_centroids, box=mems[i].box,
                             periodic=mems[i].periodic, seed=1000 + i, instance=i, **extra[i])

    ar = G.Arena(8 << 30)
    slots = [ar.admit(prm(i), m, 6) for i, m in enumerate(mems)]
    assert ar.run(10) == 6
    got = {s: ar.retire(s) for s in ar.poll()}
    ar.close()
    for i, m in enumerate(mems):
        g = G.System(prm(i))
        g.load_membrane(m)
        g.init_cells()
        g.integrate(6)
        assert_same(got[slots[i]], g.state())
        g.close()


def test_admission_respects_the_budget():
    mem = M.flat_patch_2304(seed=3)
    ar = G.Arena(8 << 30)
    s = ar.admit(params(mem, 0), mem, 3)
    per_instance = ar.info()["bytes"]
    assert per_instance > 0
    ar.close()
    # room for one instance only
    tight = G.Arena(int(per_instance * 1.5))
    s = tight.admit(params(mem, 0), mem, 3)
    with pytest.raises(G.OrbcError) as e:
        tight.admit(params(mem, 1), mem, 3)
    assert e.value.code == _native.ORBC_E_NOMEM
    assert tight.run(10) == 3
    assert tight.poll() == [s]
    tight.retire(s)
    # the freed budget admits the next request
    s2 = tight.admit(params(mem, 1), mem, 2)
    assert tight.run(10) == 2
    assert tight.poll() == [s2]
    tight.close()


def test_arena_rejects_invalid_requests():
    mem = M.flat_patch_2304(seed=4)
    ar = G.Arena(8 << 30)
    with pytest.raises(G.OrbcError) as e:
        ar.admit(params(mem, 0, G.F64_ALL), mem, 3)        # precision differs from the arena's
    assert e.value.code == _native.ORBC_E_ARG
    with pytest.raises(G.OrbcError) as e:
        ar.admit(params(mem, 0), mem, 0)                    # no steps
    assert e.value.code == _native.ORBC_E_ARG
    with pytest.raises(G.OrbcError) as e:
        ar.run(0)
    assert e.value.code == _native.ORBC_E_ARG
    with pytest.raises(G.OrbcError) as e:
        ar.retire(7)                                        # no such finished slot
    assert e.value.code == _native.ORBC_E_ARG
    assert ar.run(3) == 0                                   # nothing resident
    ar.close()


def test_overlapping_instances_stay_separate():
    """Five vesicles of the same radius around the same origin, with
    instance boundaries inside warps: the batch must never let one
    instance's particles or cells meet another's."""
    mems = [M.vesicle(3000, 40 + i, kT=0.2, f=2, chain_beads=5, n_centroids=60) for i in range(5)]
    assert any(m.n % 32 for m in mems)
    ar = G.Arena(8 << 30)
    slots = [ar.admit(params(m, i), m, 8) for i, m in enumerate(mems)]
    assert ar.run(3) == 3
    assert ar.run(10) == 5
    got = {s: ar.retire(s) for s in ar.poll()}
    for i, m in enumerate(mems):
        assert_same(got[slots[i]], alone(m, i, 8))
    ar.close()


def runaway_patch(seed=31):
    """A 2,304-particle patch with one spectrin bond made stiff (k_b = 10^6)
    and stretched 0.01 sigma past its rest length: admissible (a 10^4 force
    at admission), but the two beads overshoot each other with growing
    amplitude and the bond force passes the 2^24 range limit within a few
    steps."""
    m = M.flat_patch_2304(seed=seed)
    i, j = (int(x) for x in m.bonds[0])
    r = float(np.linalg.norm(m.pos[j] - m.pos[i]))
    m.kb = m.kb.copy()
    m.r0 = m.r0.copy()
    m.kb[0] = 1.0e6
    m.r0[0] = r - 0.01
    return m


@pytest.mark.parametrize("graphs", [True, False])
def test_failing_instance_is_isolated(graphs):
    """One instance that blows up fails alone: poll reports it, retire
    returns ORBC_E_NAN for it, and the others finish bit-identical to their
    runs alone."""
    mems = members()
    bad = runaway_patch()
    steps = 12
    ar = G.Arena(8 << 30)
    slots = [ar.admit(params(m, i), m, steps) for i, m in enumerate(mems)]
    sbad = ar.admit(params(bad, 9), bad, steps)
    got, failed = {}, {}
    for _ in range(20):
        ar.run(2, graphs)
        for s in ar.poll():
            try:
                got[s] = ar.retire(s)
            except G.OrbcError as e:
                failed[s] = e.code
        if len(got) + len(failed) == 4:
            break
    assert failed == {sbad: _native.ORBC_E_NAN}
    for i, m in enumerate(mems):
        assert_same(got[slots[i]], alone(m, i, steps))
    ar.close()
    # the runaway instance alone fails the plain system with the same code
    g = G.System(params(bad, 9))
    g.load_membrane(bad)
    g.init_cells()
    with pytest.raises(G.OrbcError) as e:
        g.integrate(steps)
    assert e.value.code == _native.ORBC_E_NAN
    g.close()
