"""Host logic of the served-stream comparison (no GPU): the first-come-
first-served completion model that the plain form is timed against, and the
continuous-batching loop's admission under an HBM budget that binds (a fake
arena in place of the C ABI)."""
import numpy as np

from paper_1701_02059_gb300 import serving


def test_fifo_completion_times():
    # three jobs: the second arrives while the first is served, the third
    # after the server went idle
    services = [2.0, 1.0, 0.5]
    arrivals = [0.0, 1.0, 10.0]
    lat = serving.fifo(services, arrivals)
    assert np.allclose(lat, [2.0, 2.0, 0.5])


def test_fifo_serves_in_arrival_order_not_list_order():
    services = [1.0, 1.0]
    arrivals = [5.0, 0.0]          # the second job arrives first
    lat = serving.fifo(services, arrivals)
    assert np.allclose(lat, [1.0, 1.0])
    lat = serving.fifo([3.0, 1.0], [0.5, 0.0])
    assert np.allclose(lat, [3.5, 1.0])


def test_percentiles_summary():
    s = serving._percentiles([1.0, 2.0, 3.0, 4.0])
    assert s["p50_s"] == 2.5 and s["max_s"] == 4.0 and s["mean_s"] == 2.5


class _FakeArena:
    """Stands in for the C-ABI arena: a byte budget, bytes per particle,
    and steps advanced per run call; admission over budget raises
    ORBC_E_NOMEM like orbc_arena_admit."""
    BYTES_PER_PARTICLE = 300
    log = []

    def __init__(self, budget, precision=None, stream=None):
        self.budget, self.used, self.left, self.size, self.next = budget, 0, {}, {}, 0
        _FakeArena.log = []

    def admit(self, params, mem, nsteps):
        need = mem.n * self.BYTES_PER_PARTICLE
        if self.used + need > self.budget:
            raise serving.OrbcError(serving.ORBC_E_NOMEM, "over budget")
        s = self.next
        self.next += 1
        self.used += need
        self.left[s], self.size[s] = nsteps, need
        _FakeArena.log.append(("admit", params, self.used))
        return s

    def admit_many(self, items, threads=4):
        # the library's contract: an admitted prefix, then the first
        # failure raised with the prefix's slots
        slots = []
        for params, mem, nsteps in items:
            try:
                slots.append(self.admit(params, mem, nsteps))
            except serving.OrbcError as e:
                e.slots = slots
                raise
        return slots

    def slot_bytes(self, s):
        return self.size.get(s, 0)

    def run(self, max_steps, graphs=True):
        k = min(min(self.left.values()), max_steps)
        for s in self.left:
            self.left[s] -= k
        return k

    def poll(self):
        return sorted(s for s, v in self.left.items() if v == 0)

    def retire(self, s):
        del self.left[s]
        self.used -= self.size.pop(s)
        _FakeArena.log.append(("retire", s, self.used))
        return {}

    def launch_count(self):
        return 0

    def info(self):
        return {"resident": len(self.left), "pending": 0, "done": 0, "particles": 0, "bytes": self.used}

    def stats(self):
        return {"repack_s": 0.0, "repacks": 0, "steps": 0}

    def close(self):
        pass


class _Mem:
    def __init__(self, n):
        self.n = n


def test_batched_loop_under_a_binding_budget(monkeypatch):
    """With room for two requests at a time, the loop never exceeds the
    budget, admits in arrival order as retirements free memory, and finishes
    every request."""
    monkeypatch.setattr(serving, "Arena", _FakeArena)
    per = 1000 * _FakeArena.BYTES_PER_PARTICLE
    jobs = [{"params": i, "mem": _Mem(1000), "steps": 10 + 5 * i, "arrival_s": 0.0} for i in range(6)]
    rec, summary, _ = serving.serve_batched(jobs, 2 * per, max_steps=5)
    assert all(r is not None and r["latency_s"] >= 0 for r in rec)
    assert summary["particle_steps"] == sum(1000 * j["steps"] for j in jobs)
    admits = [e for e in _FakeArena.log if e[0] == "admit"]
    assert [e[1] for e in admits] == list(range(6))          # arrival (here: list) order
    assert max(e[2] for e in _FakeArena.log) <= 2 * per        # never over budget
    assert sum(1 for e in _FakeArena.log if e[0] == "retire") == 6
    # admissions after the first two wait for a retirement
    first_retire = next(k for k, e in enumerate(_FakeArena.log) if e[0] == "retire")
    assert sum(1 for e in _FakeArena.log[:first_retire] if e[0] == "admit") == 2
    # the summary reports the budget binding: refused admissions, the peak
    # reserved bytes at the budget and the largest single request
    assert summary["budget_refusals"] >= 1
    assert summary["peak_reserved_bytes"] == 2 * per
    assert summary["largest_request_bytes"] == per


def test_request_larger_than_the_budget_is_refused(monkeypatch):
    import pytest
    monkeypatch.setattr(serving, "Arena", _FakeArena)
    jobs = [{"params": 0, "mem": _Mem(5000), "steps": 3, "arrival_s": 0.0}]
    with pytest.raises(RuntimeError, match="does not fit"):
        serving.serve_batched(jobs, 1000 * _FakeArena.BYTES_PER_PARTICLE)
