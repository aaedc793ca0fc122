"""Python access to the FP64 CPU oracle (``orbc_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg use it; the CUDA product path never does.  It
shares no code with the CUDA library (own C source, own ctypes structures).

``build()`` compiles the C source with ``-O2 -ffp-contract=off -fopenmp``
(no fused multiply-add, so every FP64 operation is the plain IEEE one).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "orbc_oracle.c")
SRC_MESH = os.path.join(HERE, "orbc_oracle_mesh.c")
LIB = os.path.join(HERE, "liborbc_oracle.so")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place; returns its path."""
    stale = not os.path.exists(LIB) or any(os.path.getmtime(LIB) < os.path.getmtime(x) for x in (SRC, SRC_MESH))
    if force or stale:
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, SRC, SRC_MESH, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


class Model(C.Structure):
    _fields_ = [("eps", C.c_double), ("rmin", C.c_double), ("rc", C.c_double), ("mu", C.c_double),
                ("sin_theta0", C.c_double), ("zeta", C.c_int), ("pad0", C.c_int),
                ("eps_wca", C.c_double), ("sigma_wca", C.c_double), ("sigma_pp", C.c_double),
                ("box", C.c_double * 3), ("periodic", C.c_int * 3), ("pad1", C.c_int),
                ("mem_eps", C.c_double * 9), ("mem_rc", C.c_double * 9)]


class Run(C.Structure):
    _fields_ = [("dt", C.c_double), ("kT", C.c_double), ("gamma_t", C.c_double), ("gamma_r", C.c_double),
                ("mass", C.c_double), ("inertia", C.c_double), ("skin", C.c_double),
                ("seed", C.c_ulonglong), ("instance", C.c_uint), ("rebuild_every", C.c_int),
                ("n_centroids", C.c_int), ("n_lloyd_init", C.c_int), ("n_protein_centroids", C.c_int)]


TWO_SIXTH = 2.0 ** (1.0 / 6.0)


def model(eps=1.0, sigma=1.0, rc=2.6, zeta=4, mu=3.0, sin_theta0=0.0, eps_wca=1.0, sigma_wca=1.0, sigma_pp=0.5,
          box=(0.0, 0.0, 0.0), periodic=(0, 0, 0), mem_eps=None, mem_rc=None) -> Model:
    """mem_eps, mem_rc: symmetric 3 x 3 tables over the bilayer species
    (lipid, band-3, glycophorin) of the lipid potential's well depth and
    cutoff; an entry of 0 (or no table) takes the lipid-lipid value, and the
    lipid-lipid entry is always (eps, rc)."""
    m = Model()
    m.eps, m.rmin, m.rc, m.mu, m.sin_theta0, m.zeta = eps, TWO_SIXTH * sigma, rc, mu, sin_theta0, zeta
    m.eps_wca, m.sigma_wca, m.sigma_pp = eps_wca, sigma_wca, sigma_pp
    for k in range(3):
        m.box[k] = float(box[k])
        m.periodic[k] = int(periodic[k])
    te = np.zeros((3, 3)) if mem_eps is None else np.asarray(mem_eps, float).reshape(3, 3)
    tr = np.zeros((3, 3)) if mem_rc is None else np.asarray(mem_rc, float).reshape(3, 3)
    for a in range(3):
        for b in range(3):
            lip = a == 0 and b == 0
            m.mem_eps[3 * a + b] = eps if (lip or te[a, b] == 0) else float(te[a, b])
            m.mem_rc[3 * a + b] = rc if (lip or tr[a, b] == 0) else float(tr[a, b])
    return m


def run(dt=0.01, kT=0.2, gamma_t=1.0, gamma_r=1.0, mass=1.0, inertia=1.0, skin=0.0, seed=0, instance=0,
        rebuild_every=1, n_centroids=64, n_lloyd_init=10, n_protein_centroids=0) -> Run:
    r = Run()
    r.dt, r.kT, r.gamma_t, r.gamma_r, r.mass, r.inertia, r.skin = dt, kT, gamma_t, gamma_r, mass, inertia, skin
    r.seed, r.instance, r.rebuild_every, r.n_centroids, r.n_lloyd_init = seed, instance, rebuild_every, n_centroids, n_lloyd_init
    r.n_protein_centroids = n_protein_centroids
    return r


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            P = C.c_void_p
            L.or_sys_create.restype = P
            L.or_sys_create.argtypes = [C.POINTER(Model), C.POINTER(Run)]
            L.or_sys_destroy.argtypes = [P]
            L.or_sys_set_particles.argtypes = [P, C.c_int, P, P, P, P, P, P]
            L.or_sys_set_bonds.argtypes = [P, C.c_int, P, P, P]
            L.or_sys_init_cells.argtypes = [P, P]
            L.or_sys_rebuild.argtypes = [P]
            L.or_sys_compute_forces.argtypes = [P, P]
            L.or_sys_integrate.argtypes = [P, C.c_int]
            L.or_sys_set_volume.argtypes = [P, C.c_double, C.c_double, C.c_double, P]
            L.or_sys_volume.restype = C.c_double
            L.or_sys_volume.argtypes = [P, C.c_double, P]
            L.or_height_map.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int,
                                        C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, P, P]
            L.or_sys_quench.argtypes = [P, C.c_int, C.c_double, C.c_double, C.c_double, P]
            L.or_mesh_build.argtypes = [C.c_int, P, C.c_int, P, C.c_double, C.c_int, C.c_double, C.c_double,
                                        C.c_double, C.c_double, C.c_double, C.c_ulonglong, C.c_double, C.c_int,
                                        C.c_int, C.c_double, C.c_longlong, P, P, P, P, C.c_longlong, P, P, P, P]
            L.or_sys_get_state.argtypes = [P, P, P, P, P, P]
            L.or_sys_get_forces.argtypes = [P, P, P]
            L.or_sys_get_cells.argtypes = [P, P, P, P, P, P, P, P]
            L.or_sys_pairs.restype = C.c_longlong
            L.or_sys_pairs.argtypes = [P, C.c_longlong, P]
            L.or_sys_n.argtypes = [P]
            L.or_sys_k.argtypes = [P]
            L.or_sys_adj_len.argtypes = [P]
            L.or_sys_adj_len.restype = C.c_longlong
            L.or_sys_rebuilds.argtypes = [P]
            L.or_sys_rebuilds.restype = C.c_longlong
            L.or_philox4x32_10.argtypes = [P, P, P]
            L.or_noise3.argtypes = [C.c_ulonglong, C.c_uint, C.c_uint, C.c_ulonglong, C.c_uint, P]
            L.or_lipid_pair.restype = C.c_double
            L.or_lipid_pair.argtypes = [C.POINTER(Model), P, C.c_double, P, P, P, P, P]
            L.or_wca_pair.restype = C.c_double
            L.or_wca_pair.argtypes = [C.POINTER(Model), P, C.c_double, P]
            L.or_pair_terms.restype = C.c_double
            L.or_pair_terms.argtypes = [C.POINTER(Model), C.c_int, C.c_int, P, C.c_double, P, P, P, P, P]
            L.or_bond_pair.restype = C.c_double
            L.or_bond_pair.argtypes = [P, C.c_double, C.c_double, P]
            L.or_pairs_brute.restype = C.c_longlong
            L.or_pairs_brute.argtypes = [C.POINTER(Model), C.c_int, P, P, P, C.c_int, P, C.c_longlong, P]
            L.or_forces_from_pairs.argtypes = [C.POINTER(Model), C.c_int, P, P, P, C.c_longlong, P, C.c_int, P,
                                               P, P, P, P, P]
            L.or_assign_brute.argtypes = [C.c_int, P, C.c_int, P, P, P, P]
            L.or_assign_kdtree.argtypes = [C.c_int, P, C.c_int, P, P, P, P]
            L.or_lloyd.argtypes = [C.c_int, P, P, P, C.c_int, P, P, P, P]
            L.or_morton_keys.argtypes = [C.c_int, P, P]
            L.or_morton_order.argtypes = [C.c_int, P, P]
            L.or_counting_sort.argtypes = [C.c_int, P, C.c_int, P, P]
            L.or_cell_radius.argtypes = [P, C.c_int, P, P, P, P, P]
            L.or_adjacency.restype = C.c_longlong
            L.or_adjacency.argtypes = [C.c_int, P, P, C.c_double, C.c_double, P, P, P, P, C.c_longlong]
            L.or_search_cutoff.restype = C.c_double
            L.or_search_cutoff.argtypes = [C.POINTER(Model)]
            L.or_to_grid.restype = C.c_longlong
            L.or_to_grid.argtypes = [C.c_double]
            L.or_from_grid.restype = C.c_double
            L.or_from_grid.argtypes = [C.c_longlong]
            L.or_num_threads.restype = C.c_int
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# --------------------------------------------------------------------------- free functions

def philox4x32_10(counter, key):
    c = _c(counter, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def noise3(seed, instance, pid, step, sub):
    out = np.zeros(3)
    lib().or_noise3(seed, instance, pid, step, sub, _p(out))
    return out


def lipid_pair(m: Model, d, ni, nj):
    d = _c(d, np.float64)
    ni = _c(ni, np.float64)
    nj = _c(nj, np.float64)
    Fi, Ti, Tj = np.zeros(3), np.zeros(3), np.zeros(3)
    r2 = float(d[0] * d[0] + d[1] * d[1] + d[2] * d[2])
    U = lib().or_lipid_pair(C.byref(m), _p(d), r2, _p(ni), _p(nj), _p(Fi), _p(Ti), _p(Tj))
    return U, Fi, Ti, Tj


def pair_terms(m: Model, ti, tj, d, ni, nj):
    d = _c(d, np.float64)
    ni = _c(ni, np.float64)
    nj = _c(nj, np.float64)
    Fi, Ti, Tj = np.zeros(3), np.zeros(3), np.zeros(3)
    r2 = float(d[0] * d[0] + d[1] * d[1] + d[2] * d[2])
    U = lib().or_pair_terms(C.byref(m), int(ti), int(tj), _p(d), r2, _p(ni), _p(nj), _p(Fi), _p(Ti), _p(Tj))
    return U, Fi, Ti, Tj


def bond_pair(d, kb, r0):
    """Harmonic bond term; d = x_b - x_a.  Returns (U, force on a)."""
    d = _c(d, np.float64)
    Fa = np.zeros(3)
    U = lib().or_bond_pair(_p(d), float(kb), float(r0), _p(Fa))
    return U, Fa


def mesh_build(verts, faces, spacing=1.12, beads=4, slack=1.03, kb=100.0, offset=1.0, d_min=0.8, d_ll=0.2, seed=0,
               band3_fraction=0.0, glycophorin=0, band3_edges=0, kb_anchor=50.0):
    """Particles and bonds of a triangular mesh (readings M1-M11 of
    orbc_oracle_mesh.c): returns dict(pos, ori, type, bonds, r0, kb)."""
    v = _c(verts, np.float64)
    f = _c(faces, np.int32)
    n, nb = C.c_longlong(0), C.c_longlong(0)
    args = (len(v), _p(v), len(f), _p(f), float(spacing), int(beads), float(slack), float(kb), float(offset),
            float(d_min), float(d_ll), int(seed), float(band3_fraction), int(glycophorin), int(band3_edges),
            float(kb_anchor))
    if lib().or_mesh_build(*args, 0, None, None, None, C.byref(n), 0, None, None, None, C.byref(nb)) != 0:
        raise ValueError("invalid mesh")
    pos, ori = np.zeros((n.value, 3)), np.zeros((n.value, 3))
    typ = np.zeros(n.value, np.uint8)
    bonds = np.zeros((nb.value, 2), np.int32)
    r0, kbo = np.zeros(nb.value), np.zeros(nb.value)
    lib().or_mesh_build(*args, n.value, _p(pos), _p(ori), _p(typ), C.byref(n), nb.value, _p(bonds), _p(r0),
                        _p(kbo), C.byref(nb))
    return {"pos": pos, "ori": ori, "type": typ, "bonds": bonds, "r0": r0, "kb": kbo}


def pairs_brute(m: Model, x, typ, ids, bonds=None):
    x = _c(x, np.float64)
    typ = _c(typ, np.uint8)
    ids = _c(ids, np.uint32)
    nb = 0 if bonds is None else len(bonds)
    b = _c(bonds if nb else np.zeros((1, 2)), np.int32)
    n = len(typ)
    cnt = lib().or_pairs_brute(C.byref(m), n, _p(x), _p(typ), _p(ids), nb, _p(b), 0, None)
    pairs = np.zeros((max(cnt, 1), 2), np.int32)
    lib().or_pairs_brute(C.byref(m), n, _p(x), _p(typ), _p(ids), nb, _p(b), cnt, _p(pairs))
    return pairs[:cnt]


def forces_from_pairs(m: Model, x, ori, typ, pairs, bond_idx=None, r0=None, kb=None):
    x = _c(x, np.float64)
    ori = _c(ori, np.float64)
    typ = _c(typ, np.uint8)
    pairs = _c(pairs, np.int32)
    n = len(typ)
    nb = 0 if bond_idx is None else len(bond_idx)
    bi = _c(bond_idx if nb else np.zeros((1, 2)), np.int32)
    r0 = _c(r0 if nb else np.zeros(1), np.float64)
    kb = _c(kb if nb else np.zeros(1), np.float64)
    F, T, e = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(5)
    lib().or_forces_from_pairs(C.byref(m), n, _p(x), _p(ori), _p(typ), len(pairs), _p(pairs), nb, _p(bi), _p(r0),
                               _p(kb), _p(F), _p(T), _p(e))
    return F, T, e


def assign_brute(x, c, box, periodic):
    x, c = _c(x, np.float64), _c(c, np.float64)
    box, per = _c(box, np.float64), _c(periodic, np.int32)
    out = np.zeros(len(x), np.int32)
    lib().or_assign_brute(len(x), _p(x), len(c), _p(c), _p(box), _p(per), _p(out))
    return out


def assign_kdtree(x, c, box, periodic):
    x, c = _c(x, np.float64), _c(c, np.float64)
    box, per = _c(box, np.float64), _c(periodic, np.int32)
    out = np.zeros(len(x), np.int32)
    lib().or_assign_kdtree(len(x), _p(x), len(c), _p(c), _p(box), _p(per), _p(out))
    return out


def lloyd(x, typ, cell, c, box, periodic):
    x, c = _c(x, np.float64), _c(c, np.float64)
    typ, cell = _c(typ, np.uint8), _c(cell, np.int32)
    box, per = _c(box, np.float64), _c(periodic, np.int32)
    out = np.zeros_like(c)
    lib().or_lloyd(len(x), _p(x), _p(typ), _p(cell), len(c), _p(c), _p(out), _p(box), _p(per))
    return out


def morton_keys(c):
    c = _c(c, np.float64)
    out = np.zeros(len(c), np.uint64)
    lib().or_morton_keys(len(c), _p(c), _p(out))
    return out


def morton_order(c):
    c = _c(c, np.float64)
    out = np.zeros(len(c), np.int32)
    lib().or_morton_order(len(c), _p(c), _p(out))
    return out


def counting_sort(cell, K):
    cell = _c(cell, np.int32)
    perm = np.zeros(len(cell), np.int32)
    start = np.zeros(K + 1, np.int32)
    lib().or_counting_sort(len(cell), _p(cell), K, _p(perm), _p(start))
    return perm, start


def cell_radius(x_sorted, start, c, box, periodic):
    x, c = _c(x_sorted, np.float64), _c(c, np.float64)
    start = _c(start, np.int32)
    box, per = _c(box, np.float64), _c(periodic, np.int32)
    R = np.zeros(len(c))
    lib().or_cell_radius(_p(x), len(c), _p(start), _p(c), _p(box), _p(per), _p(R))
    return R


def adjacency(c, R, rs, skin, box, periodic):
    c, R = _c(c, np.float64), _c(R, np.float64)
    box, per = _c(box, np.float64), _c(periodic, np.int32)
    K = len(c)
    ptr = np.zeros(K + 1, np.int32)
    tot = lib().or_adjacency(K, _p(c), _p(R), rs, skin, _p(box), _p(per), _p(ptr), None, 0)
    adj = np.zeros(max(tot, 1), np.int32)
    lib().or_adjacency(K, _p(c), _p(R), rs, skin, _p(box), _p(per), _p(ptr), _p(adj), tot)
    return ptr, adj[:tot]


def to_grid(v):
    return lib().or_to_grid(float(v))


def num_threads():
    return lib().or_num_threads()


# --------------------------------------------------------------------------- the system

class OracleSystem:
    """FP64 reference of the whole path: set particles and bonds, initialise
    the Voronoi cells, rebuild, compute forces, integrate N steps.  Getters
    return arrays in particle-id order."""

    def __init__(self, m: Model, r: Run):
        self.m, self.r = m, r
        self._h = lib().or_sys_create(C.byref(m), C.byref(r))
        self.n = 0

    def __del__(self):
        try:
            if self._h:
                lib().or_sys_destroy(self._h)
                self._h = None
        except Exception:
            pass

    def set_particles(self, pos, vel, ori, angvel, typ, ids):
        self._keep = [_c(pos, np.float64), _c(vel, np.float64), _c(ori, np.float64), _c(angvel, np.float64),
                      _c(typ, np.uint8), _c(ids, np.uint32)]
        self.n = len(self._keep[4])
        lib().or_sys_set_particles(self._h, self.n, *[_p(a) for a in self._keep])

    def set_bonds(self, ij, r0, kb):
        ij, r0, kb = _c(ij, np.int32), _c(r0, np.float64), _c(kb, np.float64)
        lib().or_sys_set_bonds(self._h, len(r0), _p(ij), _p(r0), _p(kb))

    def load(self, mem):
        """Particles and bonds of a ``synth.membranes.Membrane``."""
        self.set_particles(mem.pos, mem.vel, mem.ori, mem.angvel, mem.type, mem.id)
        self.set_bonds(mem.bonds, mem.r0, mem.kb)

    def init_cells(self, centroids=None):
        c = None if centroids is None else _c(centroids, np.float64)
        rc = lib().or_sys_init_cells(self._h, _p(c) if c is not None else None)
        if rc != 0:
            raise RuntimeError("oracle init_cells failed")

    def rebuild(self):
        if lib().or_sys_rebuild(self._h) != 0:
            raise RuntimeError("oracle rebuild failed")

    def compute_forces(self):
        e = np.zeros(5)
        if lib().or_sys_compute_forces(self._h, _p(e)) != 0:
            raise RuntimeError("oracle compute_forces failed")
        return e

    def integrate(self, nsteps):
        if lib().or_sys_integrate(self._h, int(nsteps)) != 0:
            raise RuntimeError("oracle integrate failed")

    def set_volume(self, kv, v0, area, center):
        """Harmonic volume constraint (readings V1-V2); kv = 0 switches it off."""
        c = _c(center, np.float64)
        lib().or_sys_set_volume(self._h, float(kv), float(v0), float(area), _p(c))

    def volume(self, area, center):
        c = _c(center, np.float64)
        return lib().or_sys_volume(self._h, float(area), _p(c))

    def height_map(self, x0, y0, dx, dy, nx, ny, z_min, axis, rho_in, rho_out):
        """Mean z per (x, y) bin of the upper-rim lipids (reading H1)."""
        h, cnt = np.zeros(nx * ny), np.zeros(nx * ny, np.int32)
        lib().or_height_map(self._h, float(x0), float(y0), float(dx), float(dy), int(nx), int(ny), float(z_min),
                            float(axis[0]), float(axis[1]), float(rho_in), float(rho_out), _p(h), _p(cnt))
        return h.reshape(ny, nx), cnt.reshape(ny, nx)

    def quench(self, nsteps, dt, max_move=0.02, max_turn=0.05):
        """Velocity quench (reading M7); returns the largest |F| at the end."""
        fm = np.zeros(1)
        if lib().or_sys_quench(self._h, int(nsteps), float(dt), float(max_move), float(max_turn), _p(fm)) != 0:
            raise RuntimeError("oracle quench failed")
        return float(fm[0])

    def state(self):
        n = self.n
        pos, vel, ori, w = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
        step = C.c_longlong(0)
        lib().or_sys_get_state(self._h, _p(pos), _p(vel), _p(ori), _p(w), C.byref(step))
        return {"pos": pos, "vel": vel, "ori": ori, "angvel": w, "step": step.value}

    def forces(self):
        n = self.n
        F, T = np.zeros((n, 3)), np.zeros((n, 3))
        lib().or_sys_get_forces(self._h, _p(F), _p(T))
        return F, T

    def cells(self):
        n, K = self.n, lib().or_sys_k(self._h)
        L = lib().or_sys_adj_len(self._h)
        cell_of_id = np.zeros(n, np.int32)
        slot_ids = np.zeros(n, np.uint32)
        c = np.zeros((K, 3))
        start = np.zeros(K + 1, np.int32)
        R = np.zeros(K)
        ptr = np.zeros(K + 1, np.int32)
        adj = np.zeros(max(L, 1), np.int32)
        lib().or_sys_get_cells(self._h, _p(cell_of_id), _p(slot_ids), _p(c), _p(start), _p(R), _p(ptr), _p(adj))
        return {"cell_of_id": cell_of_id, "slot_ids": slot_ids, "centroids": c, "start": start, "radius": R,
                "adj_ptr": ptr, "adj": adj[:L]}

    def pairs(self):
        cnt = lib().or_sys_pairs(self._h, 0, None)
        out = np.zeros((max(cnt, 1), 2), np.uint32)
        lib().or_sys_pairs(self._h, cnt, _p(out))
        return out[:cnt]

    def rebuilds(self):
        return lib().or_sys_rebuilds(self._h)
