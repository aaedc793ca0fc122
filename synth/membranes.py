"""Seeded synthetic membranes shaped like the paper's workloads.

These generators build the initial states that both the CUDA library and the
FP64 oracle consume.  They contain none of the simulation method's arithmetic
(no potential, no cell list, no integrator): only geometry and random draws.

Particle types follow the two-component red-cell model the paper simulates
(Introduction; "Initial structure generation"): lipids (type 0) carry an
orientation, spectrin-network junctions (type 1) and spectrin beads (type 2)
are point particles linked by harmonic bonds; band-3 (type 3) and
glycophorin (type 4) sit in the bilayer with an orientation like the lipids
(``with_membrane_proteins``).

Every system is returned as a ``Membrane`` with host numpy arrays in id order:

* ``pos``, ``vel`` float64 [N, 3]; ``ori`` float64 [N, 3] (unit vector for
  lipids, zero for proteins); ``angvel`` float64 [N, 3] (perpendicular to
  ``ori`` for lipids, zero for proteins);
* ``type`` uint8 [N]; ``id`` uint32 [N] (= 0..N-1);
* ``bonds`` int32 [nb, 2] (particle ids), ``r0`` and ``kb`` float64 [nb];
* ``box`` float64 [3] and ``periodic`` int32 [3];
* ``n_centroids`` (Voronoi cell count) and ``kT``.

Geometry readings (the paper gives shapes, not recipes):

* Flat patch: jittered hexagonal lipid lattice at 1.12 sigma spacing, periodic
  in x and y, with a honeycomb spectrin network 1 sigma below it.
* Vesicle: Fibonacci-sphere lipids, icosphere spectrin network 1 sigma inside.
* Biconcave cell: the Evans & Fung (1972) red-cell profile, lipids on a
  Fibonacci lattice taken over the surface's area distribution (area-uniform
  and free of overlaps, which i.i.d. sampling would need the paper's
  minimum-distance rejection and velocity quench to remove).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LIPID, JUNCTION, SPECTRIN, BAND3, GLYCOPHORIN = 0, 1, 2, 3, 4
BILAYER = (LIPID, BAND3, GLYCOPHORIN)

LIPID_SPACING = 1.12                     # nearest-neighbour lipid distance (sigma)
ROW_PITCH = LIPID_SPACING * math.sqrt(3.0) / 2.0
AREA_PER_LIPID = math.sqrt(3.0) / 2.0 * LIPID_SPACING ** 2   # 1.08634 sigma^2
GOLDEN_ANGLE = math.pi * (3.0 - math.sqrt(5.0))


@dataclass
class Membrane:
    pos: np.ndarray
    vel: np.ndarray
    ori: np.ndarray
    angvel: np.ndarray
    type: np.ndarray
    id: np.ndarray
    bonds: np.ndarray
    r0: np.ndarray
    kb: np.ndarray
    box: np.ndarray
    periodic: np.ndarray
    n_centroids: int
    kT: float
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_lipids(self) -> int:
        return int(np.count_nonzero(self.type == LIPID))

    @property
    def n_bilayer(self) -> int:
        """Particles with a director: lipids and membrane proteins."""
        return int(np.count_nonzero(np.isin(self.type, BILAYER)))

    def copy(self) -> "Membrane":
        return Membrane(self.pos.copy(), self.vel.copy(), self.ori.copy(), self.angvel.copy(),
                        self.type.copy(), self.id.copy(), self.bonds.copy(), self.r0.copy(),
                        self.kb.copy(), self.box.copy(), self.periodic.copy(), self.n_centroids,
                        self.kT, self.name, dict(self.meta))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _thermal(rng, ori, typ, kT, mass=1.0, inertia=1.0):
    """Maxwell velocities (variance kT/m per axis) and, for lipids, angular
    velocities perpendicular to the orientation (variance kT/I per axis)."""
    n = typ.shape[0]
    vel = rng.normal(0.0, math.sqrt(kT / mass), size=(n, 3))
    w = rng.normal(0.0, math.sqrt(kT / inertia), size=(n, 3))
    w -= np.sum(w * ori, axis=1, keepdims=True) * ori
    w[typ != LIPID] = 0.0
    return vel, w


def _chains(junction_pos, edges, beads_per_chain, first_junction_id, first_bead_id,
            r0_fn, kb, project=None):
    """Beads evenly spaced on the chord of every network edge, with the bond
    path junction-bead-...-bead-junction."""
    ne = len(edges)
    t = np.arange(1, beads_per_chain + 1, dtype=np.float64) / (beads_per_chain + 1)
    a = junction_pos[edges[:, 0]]
    b = junction_pos[edges[:, 1]]
    beads = a[:, None, :] + (b - a)[:, None, :] * t[None, :, None]
    beads = beads.reshape(-1, 3)
    if project is not None:
        beads = project(beads)
    L = np.linalg.norm(b - a, axis=1)
    bonds = []
    r0 = []
    for e in range(ne):
        ids = [first_junction_id + int(edges[e, 0])]
        ids += [first_bead_id + e * beads_per_chain + q for q in range(beads_per_chain)]
        ids += [first_junction_id + int(edges[e, 1])]
        for q in range(len(ids) - 1):
            bonds.append((ids[q], ids[q + 1]))
            r0.append(r0_fn(L[e]))
    bonds = np.asarray(bonds, dtype=np.int32).reshape(-1, 2)
    r0 = np.asarray(r0, dtype=np.float64)
    return beads, bonds, r0, np.full(r0.shape, kb, dtype=np.float64)


def _assemble(name, lipid_pos, lipid_ori, junc_pos, bead_pos, bonds, r0, kb, box, periodic,
              n_centroids, kT, rng, meta=None):
    nl, nj, ns = len(lipid_pos), len(junc_pos), len(bead_pos)
    pos = np.concatenate([lipid_pos, junc_pos, bead_pos]).astype(np.float64)
    ori = np.zeros_like(pos)
    ori[:nl] = lipid_ori
    typ = np.concatenate([np.full(nl, LIPID), np.full(nj, JUNCTION), np.full(ns, SPECTRIN)]).astype(np.uint8)
    vel, angvel = _thermal(rng, ori, typ, kT)
    ids = np.arange(pos.shape[0], dtype=np.uint32)
    return Membrane(pos, vel, ori, angvel, typ, ids, bonds, r0, kb,
                    np.asarray(box, dtype=np.float64), np.asarray(periodic, dtype=np.int32),
                    int(n_centroids), float(kT), name, meta or {})


# --------------------------------------------------------------------------- flat patch

def honeycomb(m: int, b: float):
    """Honeycomb (3-connected) network of m x m rectangular units of size
    sqrt(3) b x 3 b, four vertices per unit, periodic.  Returns vertex xy and
    the 6 m^2 edges."""
    w, h = math.sqrt(3.0) * b, 3.0 * b
    base = np.array([[0.0, 0.0], [0.0, b], [w / 2, 1.5 * b], [w / 2, 2.5 * b]])
    verts = []
    for ux in range(m):
        for uy in range(m):
            verts.append(base + np.array([ux * w, uy * h]))
    verts = np.concatenate(verts)

    def vid(ux, uy, s):
        return ((ux % m) * m + (uy % m)) * 4 + s

    edges = []
    for ux in range(m):
        for uy in range(m):
            edges.append((vid(ux, uy, 0), vid(ux, uy, 1)))          # vertical
            edges.append((vid(ux, uy, 1), vid(ux, uy, 2)))          # up-right
            edges.append((vid(ux, uy, 2), vid(ux, uy, 3)))          # vertical
            edges.append((vid(ux, uy, 3), vid(ux, uy + 1, 0)))      # to next unit (up-left)
            edges.append((vid(ux, uy, 1), vid(ux - 1, uy, 2)))      # up-left to left unit
            edges.append((vid(ux, uy, 3), vid(ux + 1, uy + 1, 0)))  # up-right to diagonal unit
    return verts, np.asarray(edges, dtype=np.int64)


def patch(m: int, seed: int, kT: float = 0.2, n_centroids: int | None = None,
          jitter: float = 0.05, tilt_deg: float = 5.0, chain_beads: int = 10,
          bond_r0: float = 1.0, kb: float = 100.0, name: str = "patch") -> Membrane:
    """Flat periodic patch: 16m x 32m lipids, 4m^2 junctions, 6m^2 chains of
    `chain_beads` beads; N = 576 m^2 for 10-bead chains (m = 2 is the
    2,304-particle patch)."""
    rng = _rng(seed)
    nx, ny = 16 * m, 32 * m
    Lx, Ly = nx * LIPID_SPACING, ny * ROW_PITCH
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    x = ii * LIPID_SPACING + (jj % 2) * (LIPID_SPACING / 2)
    y = jj * ROW_PITCH
    lp = np.stack([x.ravel(), y.ravel(), np.zeros(nx * ny)], axis=1)
    lp[:, :2] += rng.normal(0.0, jitter, size=(nx * ny, 2))
    tilt = math.radians(tilt_deg)
    lo = np.zeros((nx * ny, 3))
    lo[:, :2] = rng.normal(0.0, tilt, size=(nx * ny, 2))
    lo[:, 2] = 1.0
    lo /= np.linalg.norm(lo, axis=1, keepdims=True)
    b = Lx / (m * math.sqrt(3.0))
    vxy, edges = honeycomb(m, b)
    # shift so no junction sits exactly on a lattice row, then wrap into the box
    vxy = vxy + np.array([0.25 * LIPID_SPACING, 0.25 * ROW_PITCH])
    jp = np.stack([vxy[:, 0] % Lx, vxy[:, 1] % Ly, np.full(len(vxy), -1.0)], axis=1)
    # chains follow the minimum-image chord between junctions
    a = jp[edges[:, 0]]
    d = jp[edges[:, 1]] - a
    d[:, 0] -= Lx * np.round(d[:, 0] / Lx)
    d[:, 1] -= Ly * np.round(d[:, 1] / Ly)
    t = np.arange(1, chain_beads + 1) / (chain_beads + 1)
    beads = (a[:, None, :] + d[:, None, :] * t[None, :, None]).reshape(-1, 3)
    beads[:, 0] %= Lx
    beads[:, 1] %= Ly
    nl, nj = nx * ny, len(jp)
    bonds, r0 = [], []
    for e in range(len(edges)):
        ids = [nl + int(edges[e, 0])] + [nl + nj + e * chain_beads + q for q in range(chain_beads)] \
              + [nl + int(edges[e, 1])]
        for q in range(len(ids) - 1):
            bonds.append((ids[q], ids[q + 1]))
            r0.append(bond_r0)
    bonds = np.asarray(bonds, dtype=np.int32)
    r0 = np.asarray(r0)
    if n_centroids is None:
        n_centroids = max(1, round((nl + nj + len(beads)) / 36))
    return _assemble(name, lp, lo, jp, beads, bonds, r0, np.full(len(r0), kb), [Lx, Ly, 0.0],
                     [1, 1, 0], n_centroids, kT, rng, {"m": m})


# --------------------------------------------------------------------------- vesicle

def fibonacci_sphere(n: int) -> np.ndarray:
    k = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * k + 1.0) / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = k * GOLDEN_ANGLE
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def icosphere(f: int):
    """Frequency-f geodesic icosphere on the unit sphere: V = 10 f^2 + 2,
    E = 30 f^2.  Returns (vertices, edges)."""
    p = (1.0 + math.sqrt(5.0)) / 2.0
    v0 = np.array([[-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0], [0, -1, p], [0, 1, p],
                   [0, -1, -p], [0, 1, -p], [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1]],
                  dtype=np.float64)
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
             (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
             (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    key_of = {}
    verts = []
    edges = set()

    def vertex(pnt):
        q = pnt / np.linalg.norm(pnt)
        key = tuple(np.round(q, 9))
        if key not in key_of:
            key_of[key] = len(verts)
            verts.append(q)
        return key_of[key]

    for (a, b, c) in faces:
        A, B, C = v0[a], v0[b], v0[c]
        idx = {}
        for i in range(f + 1):
            for j in range(f + 1 - i):
                k = f - i - j
                idx[(i, j)] = vertex((i * A + j * B + k * C) / f)
        for i in range(f + 1):
            for j in range(f + 1 - i):
                for (di, dj) in ((1, 0), (0, 1), (1, -1)):
                    q = (i + di, j + dj)
                    if q in idx:
                        u, w = idx[(i, j)], idx[q]
                        edges.add((min(u, w), max(u, w)))
    return np.asarray(verts), np.asarray(sorted(edges), dtype=np.int64)


def icosphere_mesh(f: int, radius: float = 1.0):
    """Frequency-f geodesic icosphere as a triangle mesh: vertices on the
    sphere of the given radius and faces wound counter-clockwise seen from
    outside (V = 10 f^2 + 2, F = 20 f^2)."""
    p = (1.0 + math.sqrt(5.0)) / 2.0
    v0 = np.array([[-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0], [0, -1, p], [0, 1, p],
                   [0, -1, -p], [0, 1, -p], [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1]],
                  dtype=np.float64)
    base = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
            (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
            (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    key_of, verts, faces = {}, [], []

    def vertex(pnt):
        q = pnt / np.linalg.norm(pnt)
        key = tuple(np.round(q, 9))
        if key not in key_of:
            key_of[key] = len(verts)
            verts.append(q)
        return key_of[key]

    for (a, b, c) in base:
        A, B, C = v0[a], v0[b], v0[c]
        if np.dot(np.cross(B - A, C - A), A + B + C) < 0:      # wind outward
            B, C = C, B
        P = {}
        for i in range(f + 1):
            for j in range(f + 1 - i):
                P[(i, j)] = vertex((i * A + j * B + (f - i - j) * C) / f)
        for i in range(f):
            for j in range(f - i):
                faces.append((P[(i, j)], P[(i + 1, j)], P[(i, j + 1)]))
                if i + j <= f - 2:
                    faces.append((P[(i + 1, j + 1)], P[(i, j + 1)], P[(i + 1, j)]))
    return np.asarray(verts) * radius, np.asarray(faces, dtype=np.int32)


def biconcave_mesh(n_vertices: int, n_lipids: int = 3_571_024):
    """Triangulated biconcave red-cell surface (Evans-Fung profile) at the
    lipid scale of biconcave(): n_vertices points spread by area, joined by
    the convex hull of their unit-sphere images, faces wound outward."""
    from scipy.spatial import ConvexHull
    cdf = _AreaCDF()
    scale = math.sqrt(n_lipids * AREA_PER_LIPID / cdf.total)
    pos, _, sph = _ef_points(n_vertices, cdf, scale)
    faces = ConvexHull(sph).simplices.astype(np.int32)
    a, b, c = sph[faces[:, 0]], sph[faces[:, 1]], sph[faces[:, 2]]
    inward = np.einsum("ij,ij->i", np.cross(b - a, c - a), a + b + c) < 0
    faces[inward] = faces[inward][:, [0, 2, 1]]
    return pos, faces


def vesicle(n_lipids: int, seed: int, kT: float = 0.2, f: int | None = None,
            chain_beads: int = 20, slack: float = 0.03, kb: float = 100.0,
            n_centroids: int | None = None, jitter: float = 0.05, name: str = "vesicle",
            net_offset: float = 1.0, detach_upper: float = 0.0) -> Membrane:
    """Closed vesicle: Fibonacci-sphere lipids at 1.12 sigma spacing with
    outward orientations; icosphere spectrin network net_offset sigma inside
    (1 sigma: attached).  detach_upper > 0 moves the junctions of the upper
    hemisphere (z > 0) that much further in (a partly detached network; its
    chains then run straight between their junctions)."""
    rng = _rng(seed)
    R = math.sqrt(n_lipids * AREA_PER_LIPID / (4.0 * math.pi))
    u = fibonacci_sphere(n_lipids)
    lp = u * R
    noise = rng.normal(0.0, jitter, size=lp.shape)
    noise -= np.sum(noise * u, axis=1, keepdims=True) * u      # tangent jitter only
    lp = lp + noise
    lo = lp / np.linalg.norm(lp, axis=1, keepdims=True)
    if f is None:
        f = max(1, round(math.sqrt(n_lipids / 1105.0)))
    Rn = R - net_offset
    vj, edges = icosphere(f)
    jp = vj * Rn
    if detach_upper > 0.0:
        jp[vj[:, 2] > 0.0] *= (Rn - detach_upper) / Rn
    beads, bonds, r0, kbs = _chains(jp, edges, chain_beads, n_lipids, n_lipids + len(jp),
                                    lambda L: (1.0 + slack) * L / (chain_beads + 1), kb,
                                    project=None if detach_upper > 0.0 else
                                    (lambda q: q * (Rn / np.linalg.norm(q, axis=1, keepdims=True))))
    if n_centroids is None:
        n_centroids = max(1, round((n_lipids + len(jp) + len(beads)) / 61))
    return _assemble(name, lp, lo, jp, beads, bonds, r0, kbs, [0.0, 0.0, 0.0], [0, 0, 0],
                     n_centroids, kT, rng, {"f": f, "R": R})


# --------------------------------------------------------------------------- biconcave cell

# Evans & Fung (1972) red-cell thickness profile, micrometres:
#   thickness(r) = sqrt(1 - (r/R0)^2) * (C0 + C2 (r/R0)^2 + C4 (r/R0)^4),  z = +-thickness/2
EF_R0, EF_C0, EF_C2, EF_C4 = 3.91, 0.81, 7.83, -4.39


def _ef_meridian(t):
    """Meridian of the biconcave surface parametrised by t in [0, pi]:
    r = R0 sin t, z = cos(t) P(sin^2 t) / 2.  Returns r, z, dr/dt, dz/dt."""
    s, c = np.sin(t), np.cos(t)
    s2 = s * s
    P = EF_C0 + EF_C2 * s2 + EF_C4 * s2 * s2
    dP = (EF_C2 + 2.0 * EF_C4 * s2) * 2.0 * s * c
    r = EF_R0 * s
    z = 0.5 * c * P
    dr = EF_R0 * c
    dz = 0.5 * (-s * P + c * dP)
    return r, z, dr, dz


class _AreaCDF:
    def __init__(self, n_grid=400001):
        t = np.linspace(0.0, math.pi, n_grid)
        r, _, dr, dz = _ef_meridian(t)
        dA = 2.0 * math.pi * r * np.sqrt(dr * dr + dz * dz)
        A = np.concatenate([[0.0], np.cumsum(0.5 * (dA[1:] + dA[:-1]) * np.diff(t))])
        self.t, self.A, self.total = t, A, A[-1]

    def t_of_fraction(self, u):
        return np.interp(u * self.total, self.A, self.t)


def _ef_points(n, cdf, scale):
    """n points of a Fibonacci lattice over the biconcave surface's area
    distribution.  Returns positions (sigma), outward normals and the unit-
    sphere points with the same lattice indices (for triangulation)."""
    k = np.arange(n, dtype=np.float64)
    u = (k + 0.5) / n
    phi = k * GOLDEN_ANGLE
    t = cdf.t_of_fraction(u)
    r, z, dr, dz = _ef_meridian(t)
    nr, nz = -dz, dr
    nn = np.sqrt(nr * nr + nz * nz)
    nr, nz = nr / nn, nz / nn
    cp, sp = np.cos(phi), np.sin(phi)
    pos = np.stack([r * cp, r * sp, z], axis=1) * scale
    nrm = np.stack([nr * cp, nr * sp, nz], axis=1)
    zs = 1.0 - 2.0 * u
    rs = np.sqrt(np.maximum(0.0, 1.0 - zs * zs))
    sphere = np.stack([rs * cp, rs * sp, zs], axis=1)
    return pos, nrm, sphere


def biconcave(n_lipids: int = 3_571_024, n_junctions: int = 33_000, seed: int = 2,
              kT: float = 0.2, chain_beads: int = 4, slack: float = 0.03, kb: float = 100.0,
              n_centroids: int = 65_536, jitter: float = 0.05, name: str = "rbc",
              net_offset: float = 1.0) -> Membrane:
    """Whole biconcave red cell (Evans-Fung profile, diameter 7.82 um) mapped
    to reduced units so the lipid area per particle is that of a 1.12 sigma
    hexagonal packing.  Junctions form a triangulated network 1 sigma inside
    the lipid surface (net_offset sigma: 1 is attached, more is a detached
    network); every network edge carries `chain_beads` beads."""
    from scipy.spatial import ConvexHull

    rng = _rng(seed)
    cdf = _AreaCDF()
    scale = math.sqrt(n_lipids * AREA_PER_LIPID / cdf.total)      # sigma per micrometre
    lp, lo, _ = _ef_points(n_lipids, cdf, scale)
    noise = rng.normal(0.0, jitter, size=lp.shape)
    noise -= np.sum(noise * lo, axis=1, keepdims=True) * lo
    lp = lp + noise
    jpos, jn, jsph = _ef_points(n_junctions, cdf, scale)
    jpos = jpos - net_offset * jn                                   # net_offset sigma inside
    hull = ConvexHull(jsph)
    e = np.concatenate([hull.simplices[:, [0, 1]], hull.simplices[:, [1, 2]], hull.simplices[:, [2, 0]]])
    e.sort(axis=1)
    edges = np.unique(e, axis=0).astype(np.int64)
    beads, bonds, r0, kbs = _chains(jpos, edges, chain_beads, n_lipids, n_lipids + n_junctions,
                                    lambda L: (1.0 + slack) * L / (chain_beads + 1), kb)
    return _assemble(name, lp, lo, jpos, beads, bonds, r0, kbs, [0.0, 0.0, 0.0], [0, 0, 0],
                     n_centroids, kT, rng,
                     {"sigma_per_um": scale, "n_edges": len(edges), "area_um2": cdf.total})


# --------------------------------------------------------------------------- the five workloads

def flat_patch_2304(seed: int = 0) -> Membrane:
    """2,304-particle flat patch: 2,048 lipids, 16 junctions, 24 ten-bead
    chains, 64 Voronoi centroids, kT = 0.2."""
    return patch(2, seed, kT=0.2, n_centroids=64, name="patch-2304")


def vesicle_62k(seed: int = 1) -> Membrane:
    """61,962-particle vesicle: 40,000 lipids, 362-junction icosphere network
    with 20-bead chains at 3% slack, 1,024 Voronoi centroids."""
    return vesicle(40_000, seed, kT=0.2, f=6, chain_beads=20, n_centroids=1024, name="vesicle-62k")


def rbc_4m(seed: int = 2) -> Membrane:
    """4,000,000-particle biconcave red cell: 3,571,024 lipids, 33,000
    junctions, 98,994 four-bead chains, 65,536 Voronoi centroids."""
    return biconcave(seed=seed)


def rbc_4m_detached(seed: int = 2, depth: float = 6.0) -> Membrane:
    """The 4,000,000-particle cell with its whole protein network detached:
    the junctions `depth` sigma inside the lipid surface instead of 1."""
    return biconcave(seed=seed, net_offset=depth, name="rbc-detached")


def ensemble_member(i: int) -> Membrane:
    """Member i of the 64-instance uneven ensemble: patch or vesicle with
    particle count log-uniform in [5,000, 200,000] and kT in [0.1, 0.3]."""
    rng = _rng(3000 + i)
    is_patch = rng.random() < 0.5
    n_target = math.exp(rng.uniform(math.log(5_000), math.log(200_000)))
    kT = float(rng.uniform(0.1, 0.3))
    seed = 3000 + i
    if is_patch:
        m = max(3, round(math.sqrt(n_target / 576.0)))
        mem = patch(m, seed, kT=kT, name=f"ens{i}-patch")
    else:
        nl = max(2000, round(n_target / 1.55))
        mem = vesicle(nl, seed, kT=kT, name=f"ens{i}-vesicle")
    mem.n_centroids = max(1, round(mem.n / 61))
    return mem


def request_stream(n_requests: int = 256, rate_per_s: float = 1.0, seed: int = 4):
    """Served-stream workload: Poisson arrival times at `rate_per_s`, each
    request a patch or vesicle with N log-uniform in [10,000, 1,000,000] and
    a step count uniform in {100..2000}.  Returns a list of dicts with the
    arrival time, the step count and a builder for the membrane."""
    rng = _rng(seed)
    t = 0.0
    out = []
    for r in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        n_target = math.exp(rng.uniform(math.log(10_000), math.log(1_000_000)))
        steps = int(rng.integers(100, 2001))
        is_patch = rng.random() < 0.5
        kT = float(rng.uniform(0.1, 0.3))
        s = 40_000 + r
        if is_patch:
            m = max(3, round(math.sqrt(n_target / 576.0)))
            build = (lambda m=m, s=s, kT=kT, r=r: _with_cells(patch(m, s, kT=kT, name=f"req{r}-patch")))
            n_est = 576 * m * m
        else:
            nl = max(2000, round(n_target / 1.55))
            build = (lambda nl=nl, s=s, kT=kT, r=r: _with_cells(vesicle(nl, s, kT=kT, name=f"req{r}-vesicle")))
            n_est = int(nl * 1.55)
        out.append({"arrival_s": t, "steps": steps, "n_est": n_est, "build": build, "kT": kT})
    return out


def with_membrane_proteins(mem: Membrane, seed: int = 0, glycophorin: bool = True, anchored_beads: float = 0.25,
                           mobile_band3: float = 0.05, kb_anchor: float = 50.0) -> Membrane:
    """The membrane with the two-component model's bilayer proteins
    ("Initial structure generation": glycophorin bound to the actin
    junctions, immobile band-3 bound to the spectrin, mobile band-3 free in
    the bilayer), made by relabelling lipids, so that every id keeps its
    place and the bilayer still holds ids 0..N_B-1:

    * glycophorin: for each junction, the nearest lipid not yet taken, joined
      to it by an anchor bond;
    * immobile band-3: for a seeded share `anchored_beads` of the spectrin
      beads, the nearest lipid not yet taken, joined to the bead;
    * mobile band-3: a seeded share `mobile_band3` of the remaining lipids.

    Anchor bonds start at rest (r0 = the distance at construction) with
    constant kb_anchor.  Geometry and random draws only."""
    from scipy.spatial import cKDTree
    out = mem.copy()
    rng = _rng(seed)
    lip = np.flatnonzero(out.type == LIPID)
    taken = np.zeros(out.n, bool)
    tree = cKDTree(out.pos[lip])
    anchors = []
    targets = []
    if glycophorin:
        targets += [(int(i), GLYCOPHORIN) for i in np.flatnonzero(out.type == JUNCTION)]
    beads = np.flatnonzero(out.type == SPECTRIN)
    if anchored_beads > 0 and len(beads):
        pick = np.sort(rng.choice(beads, int(round(anchored_beads * len(beads))), replace=False))
        targets += [(int(i), BAND3) for i in pick]
    for p, t in targets:
        k = 8
        while True:
            _, q = tree.query(out.pos[p], k=min(k, len(lip)))
            free = [lip[j] for j in np.atleast_1d(q) if not taken[lip[j]]]
            if free or k >= len(lip):
                break
            k *= 4
        if not free:
            continue
        m = int(free[0])
        taken[m] = True
        out.type[m] = t
        anchors.append((int(out.id[m]), int(out.id[p]), float(np.linalg.norm(out.pos[m] - out.pos[p]))))
    rest = np.flatnonzero((out.type == LIPID) & ~taken)
    if mobile_band3 > 0 and len(rest):
        out.type[rng.choice(rest, int(round(mobile_band3 * len(rest))), replace=False)] = BAND3
    if anchors:
        a = np.array([[x[0], x[1]] for x in anchors], np.int32)
        out.bonds = np.vstack([out.bonds, a]).astype(np.int32)
        out.r0 = np.concatenate([out.r0, [x[2] for x in anchors]])
        out.kb = np.concatenate([out.kb, np.full(len(anchors), kb_anchor)])
    out.name = (mem.name or "membrane") + "+proteins"
    return out


def rbc_4m_proteins(seed: int = 2) -> Membrane:
    """The 4,000,000-particle cell with the full protein set: 33,000
    glycophorin (one per junction), immobile band-3 on a quarter of the
    spectrin beads and 5 % of the other lipids as mobile band-3."""
    return with_membrane_proteins(biconcave(seed=seed), seed=seed + 100)


def _with_cells(mem: Membrane) -> Membrane:
    mem.n_centroids = max(1, round(mem.n / 61))
    return mem
