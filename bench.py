"""Throughput of the Voronoi-cell-list CGMD step on a 4,000,000-particle
biconcave red cell (Evans-Fung shape, 65,536 Voronoi cells, FP32 forces with
64-bit fixed-point state, cells rebuilt every step).

One JSON line on stdout (rank 0).  A step is one pass of the whole hot path:
B-A-O-A update, Voronoi rebuild (M-step, Morton relabel, E-step, stable sort,
radii, neighbouring cells), pair + bond forces, final B.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload rbc-4m|rbc-1m|rbc-1m-proteins|vesicle-62k|patch-2304] [--precision f32|f64]

--impl reference times the FP64 CPU oracle on this machine's host cores on a
bounded sample of the same workload.  Under torchrun (N > 1) every rank runs
an independent replica (the path is replicas-only across GPUs) and value is
the total particle-steps/s over all ranks; the reference arm runs on rank 0.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s at 4M-particle RBC"
UNIT = "particle-steps/s"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_COUNT = 152
FP32_LANES = 128
MAX_SM_MHZ = 2070.0
# algorithmic work of the hot loop (per half-list pair and per half-list
# candidate test), counted from the pair expression
FLOP_PER_PAIR = 100.0
FLOP_PER_CANDIDATE = 9.0
# FP64 arithmetic of the integrator's B-A-O-A per step (both half kicks, both
# drifts with their Cayley maps and the renormalisation, the
# Ornstein-Uhlenbeck update with its noise scaling), counted from the
# kernel's expressions with FMA = 2 and a division as 1: per lipid (the
# angular kick 15, first drift's Cayley map 32 and second drift's 36 with the
# Cayley factor's three-term series and the renormalisation's exact integer
# norm, the angular Ornstein-Uhlenbeck update 21); a point particle has none.
# The translational kick, the drifts and the velocity's Ornstein-Uhlenbeck
# update are exact 128-bit integer products (and a sum of two) of the int64
# state with the FP64 constants (integer pipes, one rounding) and are not
# FP64 flops; the int64 <-> FP64 conversions (about 40 per lipid) use the
# FP64 pipe but are not counted.
FLOP64_PER_LIPID_STEP = 104.0
FLOP64_PER_BEAD_STEP = 0.0
# FP64 peak: the recipe's nominal GB300 figure (no measured FP64 peak exists)
FP64_TFLOPS = 1.25
# algorithmic HBM bytes of one step per particle (cells rebuilt every step):
# B-A-O-A 240, M-step 24, E-step 32, histogram/scatter/per-cell order 16,
# gather 238 (state in and out, mirrors, slot), pair kernel 80 (mirrors in,
# force and torque out); the final half kick runs once per integrate call
STEP_BYTES_PER_PARTICLE = 630.0
PAIR_BYTES_PER_PARTICLE = 80.0
# cell-list cadence of the skin variant
CADENCE_EVERY = 10
CADENCE_SKIN = 0.3
# harmonic volume constraint of the constrained variant: k_V (eps/sigma^6),
# V0 = the cell's initial volume; the upper-rim height map on a 32 x 32 grid
# of 0.25 um bins over the annulus 2.5-3.9 um, upper half
VOL_KV = 1e-6
# the detached-network variant: the 4M cell with its junctions 6 sigma inside
# the lipid surface, run with the lipid cells shared and with a protein cell
# set of its own (about 52 proteins per cell)
DETACHED_KP = 8192


def workload(name: str):
    from synth import membranes as M
    if name == "rbc-4m":
        return M.rbc_4m()
    if name == "rbc-1m":
        # the same biconcave cell at a quarter of the particles (profiling captures)
        return M.biconcave(n_lipids=892_756, n_junctions=8_250, n_centroids=16_384, seed=2, name="rbc-1m")
    if name == "rbc-1m-proteins":
        # the 1M cell with the protein set of the 4M protein variant (profiling captures)
        return M.with_membrane_proteins(workload("rbc-1m"), seed=102)
    if name == "vesicle-62k":
        return M.vesicle_62k()
    if name == "patch-2304":
        return M.flat_patch_2304()
    raise SystemExit(f"unknown workload {name}")


PRECISION = {"f32": ("F32_FORCE_F64_STATE", "FP32 pair/bond forces; FP64 integrator increments and energy/virial "
                                             "partials; int64 fixed-point state (2^-40) and force sums (2^-32)"),
             "f64": ("F64_ALL", "FP64 pair/bond forces and integrator increments; int64 fixed-point state"),
             "f32step": ("F32_FORCE_F32_STEP", "FP32 pair/bond forces and FP32 integrator increments; int64 "
                                               "fixed-point state")}


def params_for(mem, precision: str, G, **kw):
    import numpy as np
    if np.isin(mem.type, (3, 4)).any():
        # band-3 or glycophorin: the species table of the protein variant
        kw.setdefault("eps_mem", PROTEIN_EPS)
        kw.setdefault("rc_mem", PROTEIN_RC)
    return G.make_params(kT=mem.kT, n_centroids=mem.n_centroids, box=mem.box, periodic=mem.periodic,
                         seed=2, precision=getattr(G, PRECISION[precision][0]), **kw)


def oracle_params(mem, oracle):
    import numpy as np
    tab = dict(mem_eps=PROTEIN_EPS, mem_rc=PROTEIN_RC) if np.isin(mem.type, (3, 4)).any() else {}
    return (oracle.model(box=mem.box, periodic=mem.periodic, **tab),
            oracle.run(kT=mem.kT, n_centroids=mem.n_centroids, seed=2))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed
    region. ``start`` returns once the sampler has produced its first row, so
    it is already running when the region opens; ``region`` brackets the
    region in host time; the summary takes the rows that arrived inside it
    (with the rows just before and after for the throttle reasons)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 50
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index: int, exe: str = "nvidia-smi"):
        self.gpu = gpu_index
        self.exe = exe
        self.rows = []          # (host time of arrival, fields)
        self.proc = None
        self.t0 = self.t1 = None

    def start(self, wait_s: float = 5.0):
        try:
            self.proc = subprocess.Popen([self.exe, f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
            return
        t = time.perf_counter()
        while not self.rows and self.proc.poll() is None and time.perf_counter() - t < wait_s:
            time.sleep(0.005)

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.perf_counter(), [t.strip() for t in line.split(",")]))

    def region(self, begin: bool):
        if begin:
            self.t0 = time.perf_counter()
        else:
            self.t1 = time.perf_counter()

    def stop(self):
        if self.proc:
            # one more interval so that a row taken at the region's end arrives
            time.sleep(self.INTERVAL_MS * 1.5e-3)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = list(self.rows)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        t0 = self.t0 if self.t0 is not None else rows[0][0]
        t1 = self.t1 if self.t1 is not None else rows[-1][0]
        inside = [r for t, r in rows if t0 <= t <= t1]
        before = [r for t, r in rows if t < t0][-1:]
        after = [r for t, r in rows if t > t1][:1]
        # a region shorter than the sampling interval: the nearest row after it
        use = inside or after or before
        num = lambda x: x.replace(".", "").isdigit()
        sm = sorted(float(r[1]) for r in use if len(r) > 1 and num(r[1]))
        mx = max((float(r[2]) for r in use if len(r) > 2 and num(r[2])), default=None)
        reasons = set()
        for r in before + inside + after:
            for q, nm in enumerate(self.REASONS):
                if len(r) > 5 + q and r[5 + q].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(inside), "interval_ms": self.INTERVAL_MS}


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def algorithmic_work(g, mem):
    """Half-list pairs and candidate tests of the quad loop over cells."""
    import numpy as np
    c = g.cells()
    cnt = np.diff(c["start"]).astype(np.int64)
    ptr, adj = c["adj_ptr"], c["adj"]
    cand = 0
    for k in range(len(cnt)):
        js = adj[ptr[k]:ptr[k + 1]]
        js = js[js >= k]
        cand += int(sum(cnt[k] * cnt[j] if j != k else cnt[k] * (cnt[k] - 1) // 2 for j in js))
    npairs = g.pair_count()
    return npairs, cand


def kernel_traffic(kernel: str, n_particles: int):
    """DRAM bytes per launch of a kernel, from the committed ncu summary of
    the same kernel revision (profiles/<kernel>_rbc-1m.md, a line
    "traffic_bytes_per_particle: X (kernel REV)"): bytes per particle
    measured on the 1M-particle cell, scaled by the particles one launch
    processes.  None when there is no summary of this revision."""
    import re
    path = os.path.join(ROOT, "profiles", f"{kernel}_rbc-1m.md")
    if not os.path.exists(path):
        return None
    m = re.search(r"^traffic_bytes_per_particle:\s*([0-9.eE+]+)\s*\(kernel (\S+)\)", open(path).read(), re.M)
    if not m or m.group(2) != KERNEL_REV.get(kernel):
        return None
    return round(float(m.group(1)) * n_particles)


def max_over_ranks(ms: float, world: int) -> float:
    """The slowest rank's time (replicas run independently; this all-reduce
    is the only cross-rank exchange, and it happens outside the timed work)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(particles_per_rank: int, steps: int, world: int, ms: float) -> float:
    """Particle-steps per second of all ranks together over the slowest rank's time."""
    return particles_per_rank * steps * world / (ms * 1e-3)


def run_ours(args, rank, world):
    import numpy as np
    import torch
    import paper_1701_02059_gb300 as G

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    mem = workload(args.workload)
    stream = torch.cuda.Stream()
    g = G.System(params_for(mem, args.precision, G), stream=stream.cuda_stream)
    g.load_membrane(mem)
    g.init_cells()
    g.integrate(args.warmup)
    # per-kernel timing (CUDA events recorded by the library on its stream)
    g.set_timing(True)
    clocks = ClockSampler(dev)
    clocks.start()              # running before the ranks meet at the barrier
    launches0 = g.launch_count()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.region(True)
    ev0.record(stream)
    g.integrate(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks.region(False)
    clocks.stop()
    ms = ev0.elapsed_time(ev1)
    launches = g.launch_count() - launches0
    times = g.kernel_times()
    g.set_timing(False)
    ms = max_over_ranks(ms, world)
    value = whole_job_rate(mem.n, args.steps, world, ms)

    # work counts of the step: half-list pairs and quad-loop candidate tests
    # (counted from the cell list), lipids and point particles
    npairs, ncand = algorithmic_work(g, mem)
    n_lip = int((mem.type == 0).sum())
    n_bead = mem.n - n_lip
    peak32 = SM_COUNT * FP32_LANES * 2 * MAX_SM_MHZ * 1e6 / 1e12
    pk_meas, src = peaks()
    hbm = float(pk_meas.get("hbm_gbs", 6800.0)) * 1e9
    f64_step = args.precision in ("f32", "f64")
    per = lambda name: times.get(name, {"ms": 0.0, "launches": 1})["ms"] / max(times.get(name, {}).get("launches", 1), 1)
    flops_pair = npairs * FLOP_PER_PAIR
    flops_search = ncand * FLOP_PER_CANDIDATE
    flops64 = n_lip * FLOP64_PER_LIPID_STEP + n_bead * FLOP64_PER_BEAD_STEP
    # candidates for the dominant single kernel: the list search, the pair
    # evaluation and the B-A-O-A update, each against its own bound
    cands = {
        "k_pair_search": {"ms": per("pair_search"), "bound": "alu", "unit": "TFLOP/s", "work": flops_search,
                          "peak": peak32, "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"},
        "k_pair_eval": {"ms": per("pairs"), "bound": "alu", "unit": "TFLOP/s", "work": flops_pair, "peak": peak32,
                        "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"},
    }
    if f64_step:
        cands["k_baoa_d"] = {"ms": per("integrate_baoa"), "bound": "alu", "unit": "TFLOP/s", "work": flops64,
                             "peak": FP64_TFLOPS, "peak_source": "nominal GB300 FP64 (no measured FP64 peak)",
                             "dtype": "f64"}
    else:
        cands["k_baoa"] = {"ms": per("integrate_baoa"), "bound": "hbm", "unit": "GB/s",
                           "work": 240.0 * mem.n, "peak": hbm / 1e9, "peak_source": f"{src} copy bandwidth"}
    dom = max(cands, key=lambda k: cands[k]["ms"])
    d = cands[dom]
    achieved = d["work"] / (d["ms"] * 1e-3) / (1e12 if d["unit"] == "TFLOP/s" else 1e9)
    roof = {"bound": d["bound"], "kernel": dom, "achieved": round(achieved, 3), "peak": round(d["peak"], 2),
            "unit": d["unit"], "frac": round(achieved / d["peak"], 4), "traffic": kernel_traffic(dom, mem.n),
            "peak_source": d["peak_source"], "work_per_launch": d["work"], "kernel_ms": round(d["ms"], 4)}
    # the pair stage (list search + evaluation) against the FP32 peak
    pair_ms = per("pair_search") + per("pairs")
    pair_roof = {"kernels": ["k_pair_search", "k_pair_eval"], "ms": round(pair_ms, 4),
                 "flops_per_step": flops_pair + flops_search, "half_list_pairs": npairs,
                 "half_list_candidates": ncand,
                 "achieved_tflops": round((flops_pair + flops_search) / (pair_ms * 1e-3) / 1e12, 3),
                 "peak_tflops": round(peak32, 2),
                 "frac": round((flops_pair + flops_search) / (pair_ms * 1e-3) / 1e12 / peak32, 4),
                 "eval_frac": round(flops_pair / (per("pairs") * 1e-3) / 1e12 / peak32, 4)}
    breakdown = {k: round(v["ms"] / max(v["launches"], 1), 4) for k, v in times.items()}
    # step roofline: each phase at the larger of its HBM time and its
    # arithmetic time (FP32 pair work; FP64 integrator work when the step
    # computes its increments in FP64)
    t_int = max(240.0 * mem.n / hbm, flops64 / (FP64_TFLOPS * 1e12) if f64_step else 0.0)
    t_rest = (STEP_BYTES_PER_PARTICLE - 240.0 - PAIR_BYTES_PER_PARTICLE) * mem.n / hbm
    t_pair = max(PAIR_BYTES_PER_PARTICLE * mem.n / hbm, (flops_pair + flops_search) / (peak32 * 1e12))
    t_roof = t_int + t_rest + t_pair
    step_roof = {"t_roof_ms": round(t_roof * 1e3, 4), "t_measured_ms": round(ms / args.steps, 4),
                 "frac": round(t_roof * 1e3 / (ms / args.steps), 4), "hbm_gbs": hbm / 1e9, "hbm_source": src,
                 "bytes_per_particle": STEP_BYTES_PER_PARTICLE,
                 "phases_ms": {"integrator": round(t_int * 1e3, 4), "rebuild": round(t_rest * 1e3, 4),
                               "pairs": round(t_pair * 1e3, 4)},
                 "fp64_tflops": FP64_TFLOPS if f64_step else None}

    g.close()

    def variant(prec, nsteps, setup=None, **kw):
        """The same step in another precision mode (or cell-list cadence, or
        with the volume constraint), a few steps on the same workload."""
        pv = params_for(mem, prec, G)
        for k, val in kw.items():
            setattr(pv, k, val)
        gv = G.System(pv, stream=stream.cuda_stream)
        gv.load_membrane(mem)
        if setup is not None:
            setup(gv)
        gv.init_cells()
        gv.integrate(3)
        gv.set_timing(True)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        gv.integrate(nsteps)
        f1.record(stream)
        torch.cuda.synchronize()
        fms = f0.elapsed_time(f1)
        kt = {k: round(v["ms"] / max(v["launches"], 1), 4) for k, v in gv.kernel_times().items()}
        gv.close()
        return {"value": round(mem.n * nsteps / (fms * 1e-3), 1), "unit": UNIT, "steps": nsteps,
                "ms_per_step": round(fms / nsteps, 4), "precision": PRECISION[prec][1],
                "kernel_ms_per_launch": kt}

    # the FP64-everywhere variant (FP64 pair terms and increments) and the
    # FP32-increment variant of the same step
    f64 = f32step = None
    if args.precision == "f32" and not args.no_f64:
        f64 = variant("f64", max(2, args.steps // 4)) | {"dtype": "f64"}
    cadence = None
    if args.precision == "f32" and not args.no_variants:
        f32step = variant("f32step", args.steps) | {"dtype": "f32"}
        f32step["cost_of_fp64_increments_ms_per_step"] = round(ms / args.steps - f32step["ms_per_step"], 4)
        # the cell list rebuilt every 10 steps or as soon as a particle has
        # moved more than the skin (the neighbour lists are searched with the
        # cutoff plus two skins, so the pair set stays exact); the search runs
        # only with the rebuild
        cadence = variant(args.precision, 4 * args.steps, rebuild_every=CADENCE_EVERY, skin=CADENCE_SKIN) | {
            "rebuild_every": CADENCE_EVERY, "skin_sigma": CADENCE_SKIN, "dtype": "f32",
            "speedup_over_every_step": None}
        cadence["speedup_over_every_step"] = round((ms / args.steps) / cadence["ms_per_step"], 3)
    volume = detached = proteins = None
    if args.precision == "f32" and not args.no_variants and args.workload == "rbc-4m":
        volume = volume_variant(mem, G, torch, stream, variant, args.steps, ms / args.steps)
        detached = detached_variant(G, torch, stream, args.steps)
        proteins = protein_variant(G, torch, stream, args.steps, ms / args.steps)
    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        # the user's arrays in page-locked host memory, made before the timed region
        def pinned(a):
            a = np.ascontiguousarray(a)
            buf = torch.empty(max(a.nbytes, 1), dtype=torch.uint8, pin_memory=True).numpy()
            out = buf[:a.nbytes].view(a.dtype).reshape(a.shape)
            out[...] = a
            return out
        pmem = dataclasses.replace(mem, **{k: pinned(getattr(mem, k))
                                           for k in ("pos", "vel", "ori", "angvel", "type", "id", "bonds", "r0", "kb")})
        pout = {k: pinned(np.empty((mem.n, 3))) for k in ("pos", "vel", "ori", "angvel")}
        h2d = sum(a.nbytes for a in (pmem.pos, pmem.vel, pmem.ori, pmem.angvel, pmem.type, pmem.id, pmem.bonds,
                                     pmem.r0, pmem.kb))
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record(stream)
        g2 = G.System(params_for(mem, args.precision, G), stream=stream.cuda_stream)
        g2.load_membrane(pmem)
        ev[1].record(stream)
        g2.init_cells()
        ev[2].record(stream)
        g2.integrate(args.steps)
        ev[3].record(stream)
        st = g2.state(out=pout)
        ev[4].record(stream)
        torch.cuda.synchronize()
        ems = ev[0].elapsed_time(ev[4])
        phases = {k: round(ev[i].elapsed_time(ev[i + 1]), 2)
                  for i, k in enumerate(("upload_ms", "init_cells_ms", "steps_ms", "read_back_ms"))}
        d2h = sum(st[k].nbytes for k in ("pos", "vel", "ori", "angvel"))
        e2e = {"value": mem.n * args.steps * world / (ems * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "includes": "upload, k-means initialisation, steps, state read-back", "phases": phases,
               "host_buffers": "page-locked (allocated before the timed region)"}
        g2.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(mem, budget_s=args.cpu_budget)
    ens = None
    if rank == 0 and world == 1 and not args.no_ensemble and args.workload == "rbc-4m":
        ens = run_ensemble(steps=args.ensemble_steps, budget_gb=args.budget_gb)
    serve = None
    if rank == 0 and world == 1 and not args.no_serve and args.workload == "rbc-4m":
        serve = serve_leg(args.serve_requests, args.load, args.budget_gb, args.max_steps)

    line = {"metric": METRIC if args.workload == "rbc-4m" else f"particle-steps/s at {args.workload}",
            "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "f64" else "f32", "data": "synthetic",
            "config": {"workload": args.workload, "particles": mem.n, "voronoi_cells": mem.n_centroids,
                       "precision": PRECISION[args.precision][1],
                       "rebuild_every": 1, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (resident state, forces and mirrors ~1.4 GB)"},
            "roofline": roof, "kernel_ms_per_launch": breakdown, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks.summary(), "step_roofline": step_roof, "pair_roofline": pair_roof, "fp64_variant": f64,
            "f32_increment_variant": f32step, "skin_cadence_variant": cadence, "volume_variant": volume,
            "detached_variant": detached, "protein_variant": proteins,
            "ensemble": ens, "serve": serve}
    return line


# Bilayer species table of the protein-set variant (lipid, band-3,
# glycophorin; 0 = the lipid-lipid value).  The paper prints none of the
# cited model's constants: these only exercise the species-pair path with
# cutoffs wider than the lipids' (a wider search) and unequal well depths.
PROTEIN_EPS = [[0.0, 1.2, 0.9], [1.2, 1.4, 1.1], [0.9, 1.1, 0.0]]
PROTEIN_RC = [[0.0, 2.8, 0.0], [2.8, 2.9, 2.7], [0.0, 2.7, 0.0]]


def protein_variant(G, torch, stream, steps, plain_ms):
    """The 4M cell with the two-component model's full protein set (33,000
    glycophorin bonded to the junctions, band-3 bonded to a quarter of the
    spectrin beads, 5 % of the other lipids as mobile band-3) and the species
    table above, every step rebuilt."""
    import numpy as np
    from synth import membranes as M
    mem = M.rbc_4m_proteins()
    cnt = np.bincount(mem.type, minlength=5)
    p = params_for(mem, "f32", G, eps_mem=PROTEIN_EPS, rc_mem=PROTEIN_RC)
    g = G.System(p, stream=stream.cuda_stream)
    g.load_membrane(mem)
    g.init_cells()
    g.integrate(3)
    g.set_timing(True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.integrate(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1)
    kt = {k: round(v["ms"] / max(v["launches"], 1), 4) for k, v in g.kernel_times().items()}
    g.close()
    return {"workload": "rbc-4m with glycophorin, anchored and mobile band-3", "particles": mem.n,
            "lipids": int(cnt[0]), "band3": int(cnt[3]), "glycophorin": int(cnt[4]),
            "anchor_bonds": int(len(mem.bonds) - len(M.rbc_4m().bonds)),
            "eps_mem": PROTEIN_EPS, "rc_mem": PROTEIN_RC, "dtype": "f32",
            "value": round(mem.n * steps / (t * 1e-3), 1), "unit": UNIT, "ms_per_step": round(t / steps, 4),
            "cost_over_lipid_only_ms_per_step": round(t / steps - plain_ms, 4), "kernel_ms_per_launch": kt}


def detached_variant(G, torch, stream, steps):
    """The 4M cell with a detached protein network, every step rebuilt, with
    the lipid cells shared by the proteins and with a protein cell set of
    its own (the same trajectory bit for bit)."""
    from synth import membranes as M
    mem = M.rbc_4m_detached()
    out = {"workload": "rbc-4m, junctions 6 sigma inside the lipid surface", "particles": mem.n,
           "lipid_cells": mem.n_centroids, "protein_cells": DETACHED_KP}
    for name, kp in (("shared_cells", 0), ("separate_cells", DETACHED_KP)):
        p = params_for(mem, "f32", G)
        p.n_protein_centroids = kp
        g = G.System(p, stream=stream.cuda_stream)
        g.load_membrane(mem)
        g.init_cells()
        g.integrate(3)
        g.set_timing(True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.integrate(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        kt = {k: round(v["ms"] / max(v["launches"], 1), 4) for k, v in g.kernel_times().items()}
        R = g.cells()["radius"]
        g.close()
        out[name] = {"value": round(mem.n * steps / (t * 1e-3), 1), "unit": UNIT, "ms_per_step": round(t / steps, 4),
                     "largest_lipid_cell_radius": round(float(R[:mem.n_centroids].max()), 3),
                     "kernel_ms_per_launch": kt}
    out["speedup_of_separate_cells"] = round(out["shared_cells"]["ms_per_step"] / out["separate_cells"]["ms_per_step"], 3)
    return out


def volume_variant(mem, G, torch, stream, variant, steps, plain_ms):
    """The headline step with the harmonic volume constraint on (V0 = the
    initial volume), and the cost of one upper-rim height map."""
    from synth.membranes import AREA_PER_LIPID
    a = float(AREA_PER_LIPID)
    s = float(mem.meta["sigma_per_um"])

    def on(gv):
        gv.set_volume_constraint(VOL_KV, gv.volume(a, (0.0, 0.0, 0.0)), a, (0.0, 0.0, 0.0))

    out = variant("f32", steps, setup=on) | {"dtype": "f32", "kv": VOL_KV, "v0": "initial volume",
                                              "area_per_lipid": a}
    out["cost_of_constraint_ms_per_step"] = round(out["ms_per_step"] - plain_ms, 4)
    # height map: time a few calls on the same stream
    pv = params_for(mem, "f32", G)
    gv = G.System(pv, stream=stream.cuda_stream)
    gv.load_membrane(mem)
    gv.init_cells()
    rim = (-4.0 * s, -4.0 * s, 0.25 * s, 0.25 * s, 32, 32, 0.0, (0.0, 0.0), 2.5 * s, 3.9 * s)
    gv.height_map(*rim)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = 10
    for _ in range(reps):
        h, c = gv.height_map(*rim)
    t1 = time.perf_counter()
    gv.close()
    out["height_map"] = {"ms_per_call": round((t1 - t0) * 1e3 / reps, 4), "bins": "32 x 32, 0.25 um",
                         "lipids_binned": int(c.sum()), "includes": "launch, scratch, copy back, host means"}
    return out


def cpu_baseline(mem, budget_s=30.0, steps=None):
    """The FP64 oracle as it stands, on this machine's host cores: k-means
    initialisation (untimed), then whole steps until the budget is spent."""
    import oracle
    m, r = oracle_params(mem, oracle)
    s = oracle.OracleSystem(m, r)
    s.load(mem)
    s.init_cells()
    s.compute_forces()
    done, t0 = 0, time.perf_counter()
    while True:
        s.integrate(1)
        done += 1
        el = time.perf_counter() - t0
        if (steps is not None and done >= steps) or (steps is None and (el > budget_s or done >= 3)) or el > budget_s:
            break
    el = time.perf_counter() - t0
    return {"value": round(mem.n * done / el, 1), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{done} whole step(s) of the {mem.n}-particle workload after k-means initialisation, {el:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    mem = workload(args.workload)
    import oracle
    m, r = oracle_params(mem, oracle)
    s = oracle.OracleSystem(m, r)
    s.load(mem)
    s.init_cells()
    s.compute_forces()
    # bounded sample: warm-up and timed steps capped so the run ends within minutes
    t = time.perf_counter()
    s.integrate(1)
    per = time.perf_counter() - t
    w = max(0, min(args.warmup, int(30.0 / max(per, 1e-9))) - 1)
    if w:
        s.integrate(w)
    k = max(1, min(args.steps, int(120.0 / max(per, 1e-9))))
    t = time.perf_counter()
    s.integrate(k)
    el = time.perf_counter() - t
    value = mem.n * k / el
    sample = f"{k} of {args.steps} timed steps (budget 120 s) of the {mem.n}-particle workload, {min(args.warmup, w + 1)} warm-up"
    return {"metric": METRIC if args.workload == "rbc-4m" else f"particle-steps/s at {args.workload}",
            "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": k, "warmup": args.warmup,
            "ms_per_step": round(el / k * 1e3, 2), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "particles": mem.n, "voronoi_cells": mem.n_centroids},
            "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# revisions of the kernels whose ncu summaries are committed under profiles/
KERNEL_REV = {"k_pair_search": "search-v7", "k_pair_eval": "eval-v4", "k_baoa_d": "baoa-d-v7"}


def ensemble_jobs(n_instances: int, steps: int):
    """The uneven ensemble: patches and vesicles, N log-uniform in [5k, 200k],
    kT in [0.1, 0.3], seed 3000 + i; all submitted at once."""
    import paper_1701_02059_gb300 as G
    from synth import membranes as M
    jobs = []
    for i in range(n_instances):
        m = M.ensemble_member(i)
        p = G.make_params(kT=m.kT, n_centroids=m.n_centroids, box=m.box, periodic=m.periodic, seed=3000 + i,
                          instance=i)
        jobs.append({"params": p, "mem": m, "steps": steps, "arrival_s": 0.0})
    return jobs


# size classes of the ensemble's members for the autotuner (particles)
SIZE_CLASSES = (20_000, 80_000)


def run_ensemble(n_instances=64, steps=500, budget_gb=120.0, max_steps=500):
    """Batched arena against one-instance-per-launch on the same GPU; the
    cell size (particles per Voronoi cell) and the pair evaluation's CTAs per
    SM are the autotuner's choice for the largest member of each size class
    (below 20k, 20k-80k, above 80k particles)."""
    import torch
    import paper_1701_02059_gb300 as G
    from paper_1701_02059_gb300 import serving
    jobs = ensemble_jobs(n_instances, steps)
    cls = lambda n: sum(n >= c for c in SIZE_CLASSES)
    tuned = {}
    for c in sorted({cls(j["mem"].n) for j in jobs}):
        big = max((j for j in jobs if cls(j["mem"].n) == c), key=lambda j: j["mem"].n)
        K, ctas, _ = G.autotune(big["params"], big["mem"], steps=10)
        tuned[c] = (big["mem"].n / K, ctas)
    for j in jobs:
        ppc, ctas = tuned[cls(j["mem"].n)]
        j["params"].n_centroids = max(1, round(j["mem"].n / ppc))
        j["params"].eval_ctas = ctas
    ppc = sum(j["mem"].n for j in jobs) / sum(j["params"].n_centroids for j in jobs)
    torch.cuda.synchronize()
    _, sb, _ = serving.serve_batched(jobs, int(budget_gb * 2**30), max_steps=max_steps)
    _, sp, _ = serving.serve_plain(jobs)
    keep = ("p50_s", "p99_s", "makespan_s", "particle_steps_per_s")
    return {"instances": n_instances, "steps": steps, "particles": sum(j["mem"].n for j in jobs),
            "particles_per_cell": round(ppc, 1),
            "tuned_per_size_class": {f"class {c}": {"particles_per_cell": round(v[0], 1), "eval_ctas": v[1]}
                                     for c, v in sorted(tuned.items())},
            "batched": {k: round(sb[k], 4) for k in keep} | {"gpu_launches": sb["gpu_launches"]}
            | {k: sb[k] for k in ("admit_s", "run_s", "retire_s", "repack_s", "batched_steps")},
            "plain": {k: round(sp[k], 4) for k in keep},
            "p99_speedup": round(sp["p99_s"] / sb["p99_s"], 3),
            "throughput_speedup": round(sb["particle_steps_per_s"] / sp["particle_steps_per_s"], 3),
            "timing": "wall clock from submission to retirement, host arrays in and out (set-up, k-means "
                      "initialisation, steps, state read-back included)"}


def run_serving(args):
    """Served request stream: Poisson arrivals at load x the plain form's
    measured throughput, continuous batching against FIFO one-at-a-time."""
    import numpy as np
    from paper_1701_02059_gb300 import serving
    reqs, jobs = serve_jobs(args.requests)
    # plain form: measured service times, then FIFO against the arrivals
    recp, sp, _ = serving.serve_plain(jobs)
    services = [r["service_s"] for r in recp]
    C = sp["particle_steps_per_s"]
    mean_work = float(np.mean([j["mem"].n * j["steps"] for j in jobs]))
    rate = args.load * C / mean_work
    arrivals = [r["arrival_s"] / rate for r in reqs]          # unit-rate Poisson times rescaled
    for j, a in zip(jobs, arrivals):
        j["arrival_s"] = a
    lat_p = serving.fifo(services, arrivals)
    _, sb, _ = serving.serve_batched(jobs, int(args.budget_gb * 2**30), max_steps=args.max_steps)
    work = sum(j["mem"].n * j["steps"] for j in jobs)
    # both forms: throughput over the makespan (arrival gaps included) and
    # over the time the server was busy
    span_p = float(np.max(np.asarray(arrivals) + lat_p))
    plain = {"p50_s": round(float(np.percentile(lat_p, 50)), 4), "p99_s": round(float(np.percentile(lat_p, 99)), 4),
             "makespan_s": round(span_p, 4), "particle_steps_per_s": round(work / span_p, 1),
             "busy_particle_steps_per_s": round(C, 1)}
    batched = {k: round(sb[k], 4) for k in ("p50_s", "p99_s", "makespan_s", "particle_steps_per_s",
                                           "busy_particle_steps_per_s", "admit_s", "run_s", "retire_s", "idle_s",
                                           "repack_s", "repacks", "batched_steps")}
    return {"metric": "p99 completion latency of a served request stream", "value": batched["p99_s"], "unit": "s",
            "n_gpus": 1, "steps": None, "warmup": 0, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serve", "requests": len(jobs), "particles": sum(j["mem"].n for j in jobs),
                       "particle_steps": work, "rate_per_s": round(rate, 4), "load": args.load,
                       "hbm_budget_gb": args.budget_gb, "max_steps_per_launch": args.max_steps},
            "serving": {"batched": batched | {"gpu_launches": sb["gpu_launches"]}, "plain_fifo": plain,
                        "p99_speedup": round(plain["p99_s"] / batched["p99_s"], 3)},
            "gpu_launches": sb["gpu_launches"]}


def serve_jobs(n_requests: int):
    """The served-stream requests (Poisson order, sizes log-uniform in
    [10k, 1M] particles, steps in {100..2000})."""
    import paper_1701_02059_gb300 as G
    from synth import membranes as M
    reqs = M.request_stream(n_requests=n_requests, rate_per_s=1.0, seed=4)
    jobs = []
    for i, r in enumerate(reqs):
        m = r["build"]()
        p = G.make_params(kT=m.kT, n_centroids=m.n_centroids, box=m.box, periodic=m.periodic, seed=40_000 + i,
                          instance=i)
        jobs.append({"params": p, "mem": m, "steps": r["steps"], "arrival_s": 0.0})
    return reqs, jobs


def serve_leg(n_requests: int, load: float, budget_gb: float, max_steps: int):
    """Served stream inside the default run: Poisson arrivals at load x the
    plain form's measured throughput; continuous batching at the full HBM
    budget and at a budget below the resident peak that pass reached (so
    that admission waits for memory), against the first-come-first-served
    plain server."""
    import numpy as np
    from paper_1701_02059_gb300 import serving
    reqs, jobs = serve_jobs(n_requests)
    recp, sp, _ = serving.serve_plain(jobs)
    services = [r["service_s"] for r in recp]
    C = sp["particle_steps_per_s"]
    mean_work = float(np.mean([j["mem"].n * j["steps"] for j in jobs]))
    rate = load * C / mean_work
    arrivals = [r["arrival_s"] / rate for r in reqs]
    for j, a in zip(jobs, arrivals):
        j["arrival_s"] = a
    lat_p = serving.fifo(services, arrivals)
    span_p = float(np.max(np.asarray(arrivals) + lat_p))
    work = sum(j["mem"].n * j["steps"] for j in jobs)
    keep = ("p50_s", "p99_s", "makespan_s", "particle_steps_per_s", "busy_particle_steps_per_s", "repacks",
            "batched_steps", "peak_reserved_bytes", "largest_request_bytes", "budget_refusals")
    _, full, _ = serving.serve_batched(jobs, int(budget_gb * 2**30), max_steps=max_steps)
    # a budget that binds: half the resident peak of the first pass, and no
    # less than twice the largest request (admission reserves an instance's
    # arrays, half as much again for its set-up, and its carried copy)
    tight = max(int(0.5 * full["peak_reserved_bytes"]), int(2.0 * full["largest_request_bytes"]))
    _, bound, _ = serving.serve_batched(jobs, tight, max_steps=max_steps)
    plain = {"p50_s": round(float(np.percentile(lat_p, 50)), 4), "p99_s": round(float(np.percentile(lat_p, 99)), 4),
             "makespan_s": round(span_p, 4), "particle_steps_per_s": round(work / span_p, 1),
             "busy_particle_steps_per_s": round(C, 1)}
    rnd = lambda d: {k: (round(d[k], 4) if isinstance(d[k], float) else d[k]) for k in keep}
    return {"requests": len(jobs), "particles": sum(j["mem"].n for j in jobs), "particle_steps": work,
            "rate_per_s": round(rate, 4), "load": load, "max_steps_per_launch": max_steps,
            "batched": rnd(full) | {"hbm_budget_gb": budget_gb},
            "batched_tight": rnd(bound) | {"hbm_budget_gb": round(tight / 2**30, 3),
                                           "budget_bound": bool(bound["budget_refusals"] > 0)},
            "plain_fifo": plain,
            "p99_speedup": round(plain["p99_s"] / full["p99_s"], 3),
            "timing": "wall clock from arrival to retirement, host arrays in and out"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="rbc-4m")
    ap.add_argument("--precision", choices=list(PRECISION), default="f32")
    ap.add_argument("--cpu-budget", type=float, default=25.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the batched-vs-plain ensemble comparison")
    ap.add_argument("--no-f64", action="store_true", help="skip the FP64-everywhere variant")
    ap.add_argument("--no-variants", action="store_true", help="skip the FP32-increment and skin-cadence variants")
    ap.add_argument("--no-serve", action="store_true", help="skip the served-stream leg")
    ap.add_argument("--serve-requests", type=int, default=32, help="requests of the served-stream leg")
    ap.add_argument("--ensemble-steps", type=int, default=500)
    ap.add_argument("--requests", type=int, default=32, help="served-stream requests (workload serve)")
    ap.add_argument("--load", type=float, default=0.8, help="arrival rate / plain-form throughput (workload serve)")
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--max-steps", type=int, default=50, help="steps per arena launch (workload serve)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    elif args.workload == "serve":
        line = run_serving(args) if rank == 0 else None
    else:
        line = run_ours(args, rank, world)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
