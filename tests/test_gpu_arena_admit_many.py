"""Admission of many instances at once (orbc_arena_admit_many): the library
validates, quantises and initialises several requests concurrently, each on
a stream of its own, and must leave the arena exactly as admitting them one
after the other would: the same instances, bit-identical trajectories, the
same budget decisions, an admitted prefix when a request fails."""
import numpy as np
import pytest

from synth import membranes as M

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_1701_02059_gb300")
from paper_1701_02059_gb300 import _native  # noqa: E402


def members():
    a = M.flat_patch_2304(seed=21)
    b = M.vesicle(3000, 22, kT=0.15, f=2, chain_beads=5, n_centroids=50)
    c = M.patch(3, 23, kT=0.25, n_centroids=85)
    return [a, b, c, M.flat_patch_2304(seed=24), M.patch(2, 25, kT=0.2, n_centroids=40), M.flat_patch_2304(seed=26)]


def params(mem, i):
    return G.make_params(kT=mem.kT, n_centroids=mem.n_centroids, box=mem.box, periodic=mem.periodic,
                         seed=2000 + i, instance=i)


def alone(mem, i, nsteps):
    g = G.System(params(mem, i))
    g.load_membrane(mem)
    g.init_cells()
    g.integrate(nsteps)
    st = g.state()
    g.close()
    return st


def drain(ar, slot_of):
    done, calls = {}, 0
    while len(done) < len(slot_of):
        ar.run(5)
        calls += 1
        assert calls < 40
        for s in ar.poll():
            done[slot_of[s]] = ar.retire(s)
    return done


@pytest.mark.parametrize("threads", [1, 4, 8])
def test_admit_many_equals_alone(threads):
    mems = members()
    targets = [5, 9, 7, 4, 8, 6]
    ar = G.Arena(8 << 30)
    slots = ar.admit_many([(params(m, i), m, targets[i]) for i, m in enumerate(mems)], threads)
    assert len(slots) == len(mems) and len(set(slots)) == len(mems)
    info = ar.info()
    assert info["pending"] == len(mems)
    assert info["bytes"] == sum(ar.slot_bytes(s) for s in slots)
    done = drain(ar, {s: i for i, s in enumerate(slots)})
    assert ar.info()["bytes"] == 0
    ar.close()
    for i, m in enumerate(mems):
        assert done[i]["step"] == targets[i]
        a, b = done[i], alone(m, i, targets[i])
        for k in ("pos", "vel", "ori", "angvel"):
            assert np.array_equal(a[k], b[k]), f"instance {i} {k}"


def test_admit_many_matches_one_at_a_time_under_a_binding_budget():
    mems = [M.flat_patch_2304(seed=30 + i) for i in range(5)]
    items = [(params(m, i), m, 3) for i, m in enumerate(mems)]
    probe = G.Arena(8 << 30)
    per = probe.slot_bytes(probe.admit(*items[0]))
    probe.close()
    budget = int(per * 2.6)
    # one after the other: the budget refuses the first request that does not fit
    seq = G.Arena(budget)
    n_seq = 0
    for it in items:
        try:
            seq.admit(*it)
            n_seq += 1
        except G.OrbcError as e:
            assert e.code == _native.ORBC_E_NOMEM
            break
    seq.close()
    assert 1 <= n_seq < len(items)
    ar = G.Arena(budget)
    with pytest.raises(G.OrbcError) as e:
        ar.admit_many(items, 4)
    assert e.value.code == _native.ORBC_E_NOMEM
    assert len(e.value.slots) == n_seq
    assert ar.info()["pending"] == n_seq and ar.info()["bytes"] <= budget
    # retiring frees room for the rest, admitted in order
    done = drain(ar, {s: i for i, s in enumerate(e.value.slots)})
    assert sorted(done) == list(range(n_seq))
    rest = ar.admit_many(items[n_seq:n_seq + 1], 4)
    assert len(rest) == 1
    ar.close()


def test_admit_many_stops_at_the_first_invalid_request():
    mems = members()[:4]
    items = [(params(m, i), m, 4) for i, m in enumerate(mems)]
    items[2] = (items[2][0], items[2][1], 0)                 # no steps: invalid
    ar = G.Arena(8 << 30)
    with pytest.raises(G.OrbcError) as e:
        ar.admit_many(items, 4)
    assert e.value.code == _native.ORBC_E_ARG
    assert "request 2" in str(e.value)
    assert len(e.value.slots) == 2
    assert ar.info()["pending"] == 2
    assert ar.info()["bytes"] == sum(ar.slot_bytes(s) for s in e.value.slots)
    done = drain(ar, {s: i for i, s in enumerate(e.value.slots)})
    for i in range(2):
        b = alone(mems[i], i, 4)
        assert np.array_equal(done[i]["pos"], b["pos"])
    ar.close()


def test_admit_many_edge_cases():
    ar = G.Arena(8 << 30)
    assert ar.admit_many([], 4) == []
    assert ar.info()["pending"] == 0
    with pytest.raises(G.OrbcError) as e:
        ar.slot_bytes(0)                                     # no such slot yet
    assert e.value.code == _native.ORBC_E_ARG
    m = M.flat_patch_2304(seed=40)
    s = ar.admit_many([(params(m, 0), m, 2)], 0)             # threads <= 0: the default
    assert len(s) == 1 and ar.slot_bytes(s[0]) > 0
    assert ar.run(5) == 2
    ar.retire(ar.poll()[0])
    assert ar.slot_bytes(s[0]) == 0                          # a free slot holds nothing
    ar.close()
