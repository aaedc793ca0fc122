"""Served stream on the GPU: requests arrive over time, join the running
batch as they arrive, leave it when done; each result must be bit-identical
to the same request served alone by the plain one-system form."""
import numpy as np
import pytest

from synth import membranes as M

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_1701_02059_gb300")
from paper_1701_02059_gb300 import serving  # noqa: E402


def jobs():
    mems = [M.flat_patch_2304(seed=21), M.vesicle(2500, 22, kT=0.12, f=2, chain_beads=5, n_centroids=40),
            M.patch(3, 23, kT=0.28, n_centroids=85), M.vesicle(4000, 24, kT=0.3, f=2, chain_beads=6, n_centroids=65)]
    arrivals = [0.0, 0.0, 0.02, 0.05]
    steps = [6, 9, 13, 4]
    out = []
    for i, m in enumerate(mems):
        p = G.make_params(kT=m.kT, n_centroids=m.n_centroids, box=m.box, periodic=m.periodic, seed=77, instance=i)
        out.append({"params": p, "mem": m, "steps": steps[i], "arrival_s": arrivals[i]})
    return out


def test_served_results_equal_alone():
    js = jobs()
    rec_b, sum_b, st_b = serving.serve_batched(js, 8 << 30, max_steps=3, keep_states=True)
    rec_p, sum_p, st_p = serving.serve_plain(js, keep_states=True)
    for i in range(len(js)):
        for k in ("pos", "vel", "ori", "angvel"):
            assert np.array_equal(st_b[i][k], st_p[i][k]), (i, k)
        assert st_b[i]["step"] == st_p[i]["step"] == js[i]["steps"]
        assert rec_b[i]["latency_s"] > 0 and rec_p[i]["latency_s"] > 0
    work = sum(j["mem"].n * j["steps"] for j in js)
    assert sum_b["particle_steps"] == sum_p["particle_steps"] == work
    assert sum_b["p99_s"] >= sum_b["p50_s"] > 0
    assert sum_b["gpu_launches"] > 0


def test_tight_budget_queues_requests_and_still_serves_them():
    js = jobs()
    # room for the largest request and a little more (admission reserves
    # an instance's arrays half as much again for its set-up): the others
    # wait for it
    probe = G.Arena(8 << 30)
    need = []
    for j in js:
        s = probe.admit(j["params"], j["mem"], 1)
        need.append(probe.info()["bytes"] - sum(need))
    probe.close()
    budget = int(max(need) * 1.6)
    assert budget < sum(need)
    for j in js:
        j["arrival_s"] = 0.0     # all at once: only the budget holds them back
    rec, summary, states = serving.serve_batched(js, budget, max_steps=4, keep_states=True)
    _, _, alone = serving.serve_plain(js, keep_states=True)
    for i in range(len(js)):
        assert np.array_equal(states[i]["pos"], alone[i]["pos"])
    # the budget cannot hold every request at once: some were admitted only
    # after an earlier one had finished and freed its memory
    first_done = min(r["done_s"] for r in rec)
    assert sum(r["admitted_s"] < first_done for r in rec) < len(js)
    assert summary["budget_refusals"] >= 1 and summary["peak_reserved_bytes"] <= budget
