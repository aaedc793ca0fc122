"""GB300-native hot path of OpenRBC's Voronoi-cell-list coarse-grained MD
(arXiv 1701.02059): adaptive Voronoi cell list, orientation-dependent lipid
pair forces for the bilayer's lipids and proteins (band-3, glycophorin),
spectrin and anchor bonds and a BAOAB Langevin integrator, all in CUDA
kernels for sm_103a behind the C ABI of include/orbc.h.

``System`` is a thin wrapper over that ABI (host numpy arrays in, host numpy
arrays out); it does no arithmetic of its own.  ``fluctuation`` holds the
host-side analysis of a series of height maps.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native
from ._native import (BAND3, F32_FORCE_F32_STEP, F32_FORCE_F64_STATE, F64_ALL, GLYCOPHORIN, JUNCTION, LIPID, SPECTRIN,
                      OrbcError, Params, default_params, load)

__all__ = ["System", "Arena", "autotune", "Params", "default_params", "load", "OrbcError", "F32_FORCE_F64_STATE", "F64_ALL",
           "F32_FORCE_F32_STEP", "LIPID", "JUNCTION", "SPECTRIN", "BAND3", "GLYCOPHORIN"]


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def make_params(**kw) -> Params:
    """orbc_params with the library defaults, overridden by keyword
    (eps_mem, rc_mem: 3 x 3 tables over the bilayer species lipid, band-3,
    glycophorin)."""
    p = default_params()
    for k, v in kw.items():
        if k in ("box", "periodic"):
            for a in range(3):
                getattr(p, k)[a] = v[a]
        elif k in ("eps_mem", "rc_mem"):
            t = np.asarray(v, np.float64).reshape(3, 3)
            for a in range(3):
                for b in range(3):
                    getattr(p, k)[a][b] = float(t[a, b])
        else:
            setattr(p, k, v)
    return p


def mesh_build(verts, faces, stream=None, **kw):
    """orbc_mesh_build: particles and bonds of a membrane on a triangular
    mesh (keywords: the orbc_mesh_params fields).  Returns dict(pos, ori,
    type, bonds, r0, kb) in id order."""
    from ._native import MeshParams
    L = load()
    mp = MeshParams()
    L.orbc_default_mesh_params(C.byref(mp))
    for k, v in kw.items():
        setattr(mp, k, v)
    v = np.ascontiguousarray(verts, np.float64)
    f = np.ascontiguousarray(faces, np.int32)
    n, nb = C.c_longlong(0), C.c_longlong(0)
    st = C.c_void_p(stream) if stream else None
    rc = L.orbc_mesh_build(C.byref(mp), len(v), _p(v), len(f), _p(f), 0, None, None, None, C.byref(n), 0, None, None,
                           None, C.byref(nb), st)
    if rc != 0:
        raise OrbcError(rc, "orbc_mesh_build")
    out = {"pos": np.zeros((n.value, 3)), "ori": np.zeros((n.value, 3)), "type": np.zeros(n.value, np.uint8),
           "bonds": np.zeros((nb.value, 2), np.int32), "r0": np.zeros(nb.value), "kb": np.zeros(nb.value)}
    rc = L.orbc_mesh_build(C.byref(mp), len(v), _p(v), len(f), _p(f), n.value, _p(out["pos"]), _p(out["ori"]),
                           _p(out["type"]), C.byref(n), nb.value, _p(out["bonds"]), _p(out["r0"]), _p(out["kb"]),
                           C.byref(nb), st)
    if rc != 0:
        raise OrbcError(rc, "orbc_mesh_build")
    return out


def cell_sort(cell, K: int, stream=None):
    """Stable sort of device int32 cell ids (torch tensor on CUDA) through
    orbc_cell_sort; returns (perm, cell_start) as device tensors."""
    import torch
    assert cell.is_cuda and cell.dtype == torch.int32 and cell.is_contiguous()
    n = cell.numel()
    perm = torch.empty(n, dtype=torch.int32, device=cell.device)
    start = torch.empty(K + 1, dtype=torch.int32, device=cell.device)
    s = stream if stream is not None else torch.cuda.current_stream(cell.device).cuda_stream
    rc = load().orbc_cell_sort(C.c_void_p(cell.data_ptr()), n, K, C.c_void_p(perm.data_ptr()),
                               C.c_void_p(start.data_ptr()), C.c_void_p(s))
    if rc != 0:
        raise OrbcError(rc, "orbc_cell_sort")
    return perm, start


def autotune(params: Params, mem, steps: int = 10, cache: str | None = None):
    """orbc_autotune: the centroid count (cell-tile shape) and the pair
    evaluation's CTAs per SM with the fastest step for this membrane;
    returns (n_centroids, eval_ctas, ms_per_step)."""
    arrs = [np.ascontiguousarray(mem.pos, np.float64), np.ascontiguousarray(mem.vel, np.float64),
            np.ascontiguousarray(mem.ori, np.float64), np.ascontiguousarray(mem.angvel, np.float64),
            np.ascontiguousarray(mem.type, np.uint8), np.ascontiguousarray(mem.id, np.uint32)]
    ij = np.ascontiguousarray(mem.bonds, np.int32)
    r0 = np.ascontiguousarray(mem.r0, np.float64)
    kb = np.ascontiguousarray(mem.kb, np.float64)
    K = C.c_int(0)
    ctas = C.c_int(0)
    ms = C.c_double(0.0)
    rc = load().orbc_autotune(C.byref(params), len(arrs[4]), *[_p(a) for a in arrs], len(r0), _p(ij), _p(r0), _p(kb),
                              int(steps), cache.encode() if cache else None, C.byref(K), C.byref(ctas), C.byref(ms))
    if rc != 0:
        raise OrbcError(rc, "orbc_autotune")
    return K.value, ctas.value, ms.value


class System:
    """One membrane on the GPU.  Methods map one to one onto the C ABI."""

    def __init__(self, params: Params, stream: int | None = None):
        self._L = load()
        self._h = C.c_void_p()
        self._check(self._L.orbc_create(C.byref(params), C.c_void_p(stream) if stream else None, C.byref(self._h)),
                    "orbc_create")
        self.params = params
        self.n = 0
        self.K = params.n_centroids + params.n_protein_centroids   # lipid cells, then protein cells

    def _check(self, rc, what):
        if rc != 0:
            msg = self._L.orbc_last_error(self._h).decode() if self._h else what
            raise OrbcError(rc, f"{what}: {msg}")

    def close(self):
        if self._h:
            self._L.orbc_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -------------------------------------------------------------- set-up
    def set_particles(self, pos, vel, ori, angvel, typ, ids):
        arrs = [np.ascontiguousarray(pos, np.float64), np.ascontiguousarray(vel, np.float64),
                np.ascontiguousarray(ori, np.float64), np.ascontiguousarray(angvel, np.float64),
                np.ascontiguousarray(typ, np.uint8), np.ascontiguousarray(ids, np.uint32)]
        self.n = len(arrs[4])
        self._check(self._L.orbc_set_particles(self._h, self.n, *[_p(a) for a in arrs]), "orbc_set_particles")

    def set_bonds(self, ij, r0, kb):
        ij = np.ascontiguousarray(ij, np.int32)
        r0 = np.ascontiguousarray(r0, np.float64)
        kb = np.ascontiguousarray(kb, np.float64)
        self._check(self._L.orbc_set_bonds(self._h, len(r0), _p(ij), _p(r0), _p(kb)), "orbc_set_bonds")

    def load_membrane(self, mem):
        self.set_particles(mem.pos, mem.vel, mem.ori, mem.angvel, mem.type, mem.id)
        if len(mem.r0):
            self.set_bonds(mem.bonds, mem.r0, mem.kb)

    def init_cells(self, centroids=None):
        c = None if centroids is None else np.ascontiguousarray(centroids, np.float64)
        self._check(self._L.orbc_init_cells(self._h, _p(c)), "orbc_init_cells")

    # -------------------------------------------------------------- the path
    def rebuild_cells(self):
        self._check(self._L.orbc_rebuild_cells(self._h), "orbc_rebuild_cells")

    def compute_forces(self, energies: bool = False):
        e = np.zeros(5) if energies else None
        self._check(self._L.orbc_compute_forces(self._h, _p(e)), "orbc_compute_forces")
        return e

    def integrate(self, nsteps: int):
        self._check(self._L.orbc_integrate(self._h, int(nsteps)), "orbc_integrate")

    def quench(self, nsteps: int, dt: float, max_move: float = 0.02, max_turn: float = 0.05) -> float:
        """orbc_quench: velocity quench; returns the largest |F| at the end."""
        fm = C.c_double(0.0)
        self._check(self._L.orbc_quench(self._h, int(nsteps), float(dt), float(max_move), float(max_turn),
                                        C.byref(fm)), "orbc_quench")
        return fm.value

    def set_step_fusion(self, on: bool):
        """orbc_set_step_fusion: run each step's update in the previous force
        launch's epilogue, or as a launch of its own (the default)."""
        self._check(self._L.orbc_set_step_fusion(self._h, int(bool(on))), "orbc_set_step_fusion")

    def set_volume_constraint(self, kv: float, v0: float, area_per_lipid: float, center=(0.0, 0.0, 0.0)):
        """orbc_set_volume_constraint: U_V = kv (V - v0)^2 / 2 on the lipid
        volume V (kv = 0 switches it off)."""
        c = np.ascontiguousarray(center, np.float64)
        self._check(self._L.orbc_set_volume_constraint(self._h, float(kv), float(v0), float(area_per_lipid), _p(c)),
                    "orbc_set_volume_constraint")

    def volume(self, area_per_lipid: float, center=(0.0, 0.0, 0.0)) -> float:
        """orbc_get_volume: the enclosed lipid volume of the current state."""
        c = np.ascontiguousarray(center, np.float64)
        V = C.c_double(0.0)
        self._check(self._L.orbc_get_volume(self._h, float(area_per_lipid), _p(c), C.byref(V)), "orbc_get_volume")
        return V.value

    def height_map(self, x0, y0, dx, dy, nx, ny, z_min, axis=(0.0, 0.0), rho_in=0.0, rho_out=float("inf")):
        """orbc_height_map: mean z and count per (x, y) bin of the lipids
        above z_min in the annulus rho_in <= rho < rho_out; arrays [ny, nx]."""
        a = np.ascontiguousarray(axis, np.float64)
        h, cnt = np.zeros(nx * ny), np.zeros(nx * ny, np.int32)
        self._check(self._L.orbc_height_map(self._h, float(x0), float(y0), float(dx), float(dy), int(nx), int(ny),
                                            float(z_min), _p(a), float(rho_in), float(rho_out), _p(h), _p(cnt)),
                    "orbc_height_map")
        return h.reshape(ny, nx), cnt.reshape(ny, nx)

    # -------------------------------------------------------------- getters
    def state(self, out=None):
        """orbc_get_state: positions, velocities, directors and angular
        velocities in id order. ``out`` (optional) maps those four names to
        caller-owned C-contiguous float64 [n, 3] arrays (pinned memory makes
        the copy run at the link's full rate); they are filled and returned."""
        n = self.n
        if out is None:
            pos, vel, ori, w = (np.empty((n, 3)) for _ in range(4))
        else:
            pos, vel, ori, w = (out[k] for k in ("pos", "vel", "ori", "angvel"))
            for a in (pos, vel, ori, w):
                if a.dtype != np.float64 or a.shape != (n, 3) or not a.flags.c_contiguous or not a.flags.writeable:
                    raise ValueError("state(out=...) wants writeable C-contiguous float64 [n, 3] arrays")
        step = C.c_longlong(0)
        self._check(self._L.orbc_get_state(self._h, _p(pos), _p(vel), _p(ori), _p(w), C.byref(step)), "orbc_get_state")
        return {"pos": pos, "vel": vel, "ori": ori, "angvel": w, "step": step.value}

    # -------------------------------------------------------------- device tensors
    def set_particles_tensors(self, pos, vel, ori, angvel, typ, ids):
        """orbc_set_particles_device from CUDA tensors (float64 [n,3] x4,
        uint8 [n], int32/uint32 [n]), on the system's stream."""
        ts = [pos, vel, ori, angvel, typ, ids]
        for t in ts:
            assert t.is_cuda and t.is_contiguous()
        self.n = int(typ.numel())
        self._check(self._L.orbc_set_particles_device(self._h, self.n, *[C.c_void_p(t.data_ptr()) for t in ts]),
                    "orbc_set_particles_device")

    def state_tensors(self, device=None):
        """orbc_get_state_device: the state in id order as CUDA float64 tensors."""
        import torch
        out = [torch.empty((self.n, 3), dtype=torch.float64, device=device or "cuda") for _ in range(4)]
        self._check(self._L.orbc_get_state_device(self._h, *[C.c_void_p(t.data_ptr()) for t in out]),
                    "orbc_get_state_device")
        return dict(zip(("pos", "vel", "ori", "angvel"), out))

    def force_tensors(self, device=None):
        """orbc_get_forces_device: forces and torques in id order as CUDA tensors."""
        import torch
        F = torch.empty((self.n, 3), dtype=torch.float64, device=device or "cuda")
        T = torch.empty((self.n, 3), dtype=torch.float64, device=device or "cuda")
        self._check(self._L.orbc_get_forces_device(self._h, C.c_void_p(F.data_ptr()), C.c_void_p(T.data_ptr())),
                    "orbc_get_forces_device")
        return F, T

    def forces(self):
        F, T = np.zeros((self.n, 3)), np.zeros((self.n, 3))
        self._check(self._L.orbc_get_forces(self._h, _p(F), _p(T)), "orbc_get_forces")
        return F, T

    def cells(self):
        n, K = self.n, self.K
        L = C.c_longlong(0)
        self._check(self._L.orbc_get_adjacency_len(self._h, C.byref(L)), "orbc_get_adjacency_len")
        cell = np.zeros(n, np.int32)
        slots = np.zeros(n, np.uint32)
        c = np.zeros((K, 3))
        start = np.zeros(K + 1, np.int32)
        R = np.zeros(K)
        ptr = np.zeros(K + 1, np.int32)
        adj = np.zeros(max(L.value, 1), np.int32)
        self._check(self._L.orbc_get_cells(self._h, _p(cell), _p(slots), _p(c), _p(start), _p(R), _p(ptr), _p(adj)),
                    "orbc_get_cells")
        return {"cell_of_id": cell, "slot_ids": slots, "centroids": c, "start": start, "radius": R, "adj_ptr": ptr,
                "adj": adj[:L.value]}

    def pair_count(self) -> int:
        cnt = C.c_longlong(0)
        self._check(self._L.orbc_dump_pairs(self._h, 0, None, C.byref(cnt)), "orbc_dump_pairs")
        return cnt.value

    def pairs(self):
        cnt = C.c_longlong(0)
        self._check(self._L.orbc_dump_pairs(self._h, 0, None, C.byref(cnt)), "orbc_dump_pairs")
        out = np.zeros((max(cnt.value, 1), 2), np.uint32)
        self._check(self._L.orbc_dump_pairs(self._h, cnt.value, _p(out), C.byref(cnt)), "orbc_dump_pairs")
        return out[:cnt.value]

    def set_timing(self, on: bool):
        self._check(self._L.orbc_set_timing(self._h, 1 if on else 0), "orbc_set_timing")

    def set_wait_test(self, extra_tx_bytes: int = 0, max_polls: int = 1 << 22):
        """orbc_set_wait_test: make the staging waits run out (test of the
        bounded waits); (0, 1 << 22) is normal operation."""
        self._check(self._L.orbc_set_wait_test(self._h, int(extra_tx_bytes), int(max_polls)), "orbc_set_wait_test")

    def launch_count(self) -> int:
        c = C.c_longlong(0)
        self._check(self._L.orbc_get_launch_count(self._h, C.byref(c)), "orbc_get_launch_count")
        return c.value

    def kernel_times(self):
        buf = C.create_string_buffer(4096)
        ms = (C.c_float * 64)()
        cnt = C.c_int(0)
        self._check(self._L.orbc_get_kernel_times(self._h, buf, 4096, ms, 64, C.byref(cnt)), "orbc_get_kernel_times")
        out = {}
        names = buf.value.decode().split(",") if buf.value else []
        for q, nm in enumerate(names[:cnt.value]):
            name, launches = nm.rsplit(":", 1)
            out[name] = {"ms": float(ms[q]), "launches": int(launches)}
        return out


class Arena:
    """Batched, continuously batched instances on one GPU (orbc_arena_*)."""

    def __init__(self, hbm_budget_bytes: int, precision: int = F32_FORCE_F64_STATE, stream: int | None = None):
        self._L = load()
        self._h = C.c_void_p()
        rc = self._L.orbc_arena_create(int(hbm_budget_bytes), int(precision), C.c_void_p(stream) if stream else None,
                                       C.byref(self._h))
        if rc != 0:
            raise OrbcError(rc, "orbc_arena_create")
        self.n_of_slot = {}

    def _check(self, rc, what):
        if rc != 0:
            raise OrbcError(rc, f"{what}: {self._L.orbc_arena_last_error(self._h).decode()}")

    def close(self):
        if self._h:
            self._L.orbc_arena_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def admit(self, params: Params, mem, nsteps: int) -> int:
        """Admit a membrane (synth.membranes.Membrane-like) for nsteps steps;
        returns its slot.  Raises OrbcError(ORBC_E_NOMEM) when over budget."""
        arrs = [np.ascontiguousarray(mem.pos, np.float64), np.ascontiguousarray(mem.vel, np.float64),
                np.ascontiguousarray(mem.ori, np.float64), np.ascontiguousarray(mem.angvel, np.float64),
                np.ascontiguousarray(mem.type, np.uint8), np.ascontiguousarray(mem.id, np.uint32)]
        ij = np.ascontiguousarray(mem.bonds, np.int32)
        r0 = np.ascontiguousarray(mem.r0, np.float64)
        kb = np.ascontiguousarray(mem.kb, np.float64)
        slot = C.c_int(-1)
        self._check(self._L.orbc_arena_admit(self._h, C.byref(params), len(arrs[4]), *[_p(a) for a in arrs], len(r0),
                                             _p(ij), _p(r0), _p(kb), int(nsteps), C.byref(slot)), "orbc_arena_admit")
        self.n_of_slot[slot.value] = len(arrs[4])
        return slot.value

    def admit_many(self, items, threads: int = 8):
        """Admit [(params, mem, nsteps), ...] in order, up to `threads`
        initialised at once; returns the admitted prefix's slots.  When a
        request fails, raises OrbcError for it with .slots = that prefix."""
        from ._native import ArenaRequest
        keep, reqs = [], (ArenaRequest * max(len(items), 1))()
        for k, (params, mem, nsteps) in enumerate(items):
            arrs = [np.ascontiguousarray(mem.pos, np.float64), np.ascontiguousarray(mem.vel, np.float64),
                    np.ascontiguousarray(mem.ori, np.float64), np.ascontiguousarray(mem.angvel, np.float64),
                    np.ascontiguousarray(mem.type, np.uint8), np.ascontiguousarray(mem.id, np.uint32),
                    np.ascontiguousarray(mem.bonds, np.int32), np.ascontiguousarray(mem.r0, np.float64),
                    np.ascontiguousarray(mem.kb, np.float64)]
            keep.append((params, arrs))
            r = reqs[k]
            r.params = C.pointer(params)
            r.n = len(arrs[4])
            r.pos, r.vel, r.ori, r.angvel, r.type, r.id = (_p(a) for a in arrs[:6])
            r.nb = len(arrs[7])
            r.ij, r.r0, r.kb = _p(arrs[6]), _p(arrs[7]), _p(arrs[8])
            r.nsteps = int(nsteps)
        slots = np.full(max(len(items), 1), -1, np.int32)
        done = C.c_int(0)
        rc = self._L.orbc_arena_admit_many(self._h, reqs, len(items), int(threads), _p(slots), C.byref(done))
        out = [int(x) for x in slots[:done.value]]
        for k, s in enumerate(out):
            self.n_of_slot[s] = reqs[k].n
        if rc != 0:
            e = OrbcError(rc, f"orbc_arena_admit_many: {self._L.orbc_arena_last_error(self._h).decode()}")
            e.slots = out
            raise e
        return out

    def slot_bytes(self, slot: int) -> int:
        b = C.c_ulonglong(0)
        self._check(self._L.orbc_arena_slot_bytes(self._h, int(slot), C.byref(b)), "orbc_arena_slot_bytes")
        return b.value

    def run(self, max_steps: int, graphs: bool = True) -> int:
        s = C.c_int(0)
        self._check(self._L.orbc_arena_run(self._h, int(max_steps), 1 if graphs else 0, C.byref(s)), "orbc_arena_run")
        return s.value

    def poll(self):
        n = C.c_int(0)
        self._check(self._L.orbc_arena_poll(self._h, None, 0, C.byref(n)), "orbc_arena_poll")
        out = np.zeros(max(n.value, 1), np.int32)
        self._check(self._L.orbc_arena_poll(self._h, _p(out), n.value, C.byref(n)), "orbc_arena_poll")
        return [int(x) for x in out[:n.value]]

    def retire(self, slot: int):
        n = self.n_of_slot.get(slot, 0)
        pos, vel, ori, w = (np.zeros((n, 3)) for _ in range(4))
        step = C.c_longlong(0)
        self._check(self._L.orbc_arena_retire(self._h, int(slot), _p(pos), _p(vel), _p(ori), _p(w), C.byref(step)),
                    "orbc_arena_retire")
        self.n_of_slot.pop(slot, None)
        return {"pos": pos, "vel": vel, "ori": ori, "angvel": w, "step": step.value}

    def info(self):
        r, p, d = C.c_int(0), C.c_int(0), C.c_int(0)
        np_, b = C.c_longlong(0), C.c_ulonglong(0)
        self._check(self._L.orbc_arena_info(self._h, C.byref(r), C.byref(p), C.byref(d), C.byref(np_), C.byref(b)),
                    "orbc_arena_info")
        return {"resident": r.value, "pending": p.value, "done": d.value, "particles": np_.value, "bytes": b.value}

    def launch_count(self) -> int:
        return int(self._L.orbc_arena_launch_count(self._h))

    def stats(self):
        rp, st = C.c_double(0.0), C.c_double(0.0)
        nr, ns = C.c_longlong(0), C.c_longlong(0)
        self._check(self._L.orbc_arena_stats(self._h, C.byref(rp), C.byref(st), C.byref(nr), C.byref(ns)),
                    "orbc_arena_stats")
        return {"repack_s": rp.value, "step_s": st.value, "repacks": nr.value, "steps": ns.value}
