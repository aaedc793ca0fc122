"""Request loops over the batched arena (continuous batching) and over the
plain one-system-per-request form, for the ensemble and served-stream
workloads.  Orchestration only: admission, stepping and retirement are calls
into the C ABI (orbc_arena_*, orbc_*); no arithmetic of the method runs here.

A job is a dict with ``params`` (orbc_params), ``mem`` (a membrane with the
host arrays of orbc_set_particles / orbc_set_bonds), ``steps`` and
``arrival_s`` (seconds after the start of the stream).
"""
from __future__ import annotations

import time

import numpy as np

from . import Arena, OrbcError, System
from ._native import ORBC_E_NOMEM, F32_FORCE_F64_STATE


def _percentiles(lat):
    lat = np.asarray(lat, float)
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "max_s": float(lat.max()), "mean_s": float(lat.mean())}


def serve_batched(jobs, hbm_budget_bytes: int, max_steps: int = 50, graphs: bool = True, keep_states: bool = False,
                  precision: int = F32_FORCE_F64_STATE, stream: int | None = None, admit_threads: int = 8):
    """Continuous batching: requests are admitted as they arrive and as the
    budget allows, every resident request advances in one batched launch per
    phase, finished ones are retired.  Returns per-job records (latency =
    completion time - arrival time) and a summary."""
    arena = Arena(hbm_budget_bytes, precision, stream)
    order = sorted(range(len(jobs)), key=lambda i: jobs[i]["arrival_s"])
    waiting = list(order)
    slot_job = {}
    rec = [None] * len(jobs)
    states = [None] * len(jobs)
    t0 = time.perf_counter()
    work = 0
    spent = {"admit_s": 0.0, "run_s": 0.0, "retire_s": 0.0, "idle_s": 0.0}
    mem_stats = {"peak_reserved_bytes": 0, "largest_request_bytes": 0, "budget_refusals": 0}
    while waiting or slot_job:
        now = time.perf_counter() - t0
        # admit everything that has arrived, in arrival order, while it fits;
        # the library initialises up to admit_threads of them at once
        arrived = []
        while len(arrived) < len(waiting) and jobs[waiting[len(arrived)]]["arrival_s"] <= now:
            arrived.append(waiting[len(arrived)])
        if arrived:
            ta = time.perf_counter()
            refused = None
            try:
                slots = arena.admit_many([(jobs[i]["params"], jobs[i]["mem"], jobs[i]["steps"]) for i in arrived],
                                         admit_threads)
            except OrbcError as e:
                if e.code != ORBC_E_NOMEM:
                    raise
                slots, refused = e.slots, e
            spent["admit_s"] += time.perf_counter() - ta
            for i, s in zip(arrived, slots):
                mem_stats["largest_request_bytes"] = max(mem_stats["largest_request_bytes"], arena.slot_bytes(s))
                slot_job[s] = i
                waiting.pop(0)
                rec[i] = {"arrival_s": jobs[i]["arrival_s"], "admitted_s": time.perf_counter() - t0}
            mem_stats["peak_reserved_bytes"] = max(mem_stats["peak_reserved_bytes"], arena.info()["bytes"])
            if refused is not None:
                mem_stats["budget_refusals"] += 1
                if not slot_job:
                    raise RuntimeError(f"request {waiting[0]} does not fit the HBM budget on an empty GPU") from refused
        if slot_job:
            tr = time.perf_counter()
            arena.run(max_steps, graphs)
            spent["run_s"] += time.perf_counter() - tr
            for s in arena.poll():
                i = slot_job.pop(s)
                tt = time.perf_counter()
                try:
                    st = arena.retire(s)
                except OrbcError as e:
                    # the request failed alone (its own data raised a device
                    # flag); the others carry on
                    st = None
                    rec[i]["error"] = e.code
                spent["retire_s"] += time.perf_counter() - tt
                if keep_states:
                    states[i] = st
                done = time.perf_counter() - t0
                rec[i]["done_s"] = done
                rec[i]["latency_s"] = done - jobs[i]["arrival_s"]
                if st is not None:
                    work += jobs[i]["mem"].n * jobs[i]["steps"]
        elif waiting:
            ti = time.perf_counter()
            time.sleep(max(0.0, min(0.05, jobs[waiting[0]]["arrival_s"] - (time.perf_counter() - t0))))
            spent["idle_s"] += time.perf_counter() - ti
    total = time.perf_counter() - t0
    launches = arena.launch_count()
    inner = arena.stats()
    arena.close()
    summary = _percentiles([r["latency_s"] for r in rec])
    busy = spent["admit_s"] + spent["run_s"] + spent["retire_s"]
    # the same two throughputs as the plain form: over the makespan (arrival
    # gaps included) and over the time the server was busy
    summary.update({"makespan_s": total, "busy_s": busy, "particle_steps": work, "particle_steps_per_s": work / total,
                    "busy_particle_steps_per_s": work / busy if busy > 0 else 0.0, "gpu_launches": launches})
    summary.update({k: round(v, 3) for k, v in spent.items()})
    summary.update({"repack_s": round(inner["repack_s"], 3), "repacks": inner["repacks"],
                    "batched_steps": inner["steps"]})
    summary.update(mem_stats)
    summary["failed"] = sum(1 for r in rec if "error" in r)
    return rec, summary, states


def fifo(services, arrivals):
    """Completion latencies of a single first-come-first-served server with
    the given service and arrival times."""
    order = np.argsort(np.asarray(arrivals, float), kind="stable")
    clock = 0.0
    lat = np.zeros(len(services))
    for i in order:
        clock = max(clock, arrivals[i]) + services[i]
        lat[i] = clock - arrivals[i]
    return lat


def serve_plain(jobs, keep_states: bool = False, stream: int | None = None):
    """The plain form: one system per request, one request at a time, first
    come first served.  Each request's service time (set-up, k-means
    initialisation, steps, state read-back) is measured; completion times
    follow from the arrival times and the FIFO order."""
    order = sorted(range(len(jobs)), key=lambda i: jobs[i]["arrival_s"])
    rec = [None] * len(jobs)
    states = [None] * len(jobs)
    clock = 0.0
    busy = 0.0
    work = 0
    for i in order:
        j = jobs[i]
        t = time.perf_counter()
        g = System(j["params"], stream=stream)
        g.load_membrane(j["mem"])
        g.init_cells()
        g.integrate(j["steps"])
        st = g.state()
        g.close()
        service = time.perf_counter() - t
        if keep_states:
            states[i] = st
        start = max(clock, j["arrival_s"])
        clock = start + service
        busy += service
        work += j["mem"].n * j["steps"]
        rec[i] = {"arrival_s": j["arrival_s"], "start_s": start, "done_s": clock, "service_s": service,
                  "latency_s": clock - j["arrival_s"]}
    summary = _percentiles([r["latency_s"] for r in rec])
    summary.update({"makespan_s": clock, "busy_s": busy, "particle_steps": work, "particle_steps_per_s": work / clock,
                    "busy_particle_steps_per_s": work / busy})
    return rec, summary, states
