"""Constructed boundary cases of the two exact decisions of the method, on
the GPU through the C ABI against the FP64 oracle.

* Nearest centroid ("Spatial Searching Algorithm": each particle belongs to
  the Voronoi cell of its closest centroid).  Particles sit exactly on the
  bisector of two, three or four centroids on the 2^-40 grid (also through
  the minimum image across a periodic face), where the reading is the
  lowest centroid index; and 1e-7 sigma and 2e-6 sigma off a bisector,
  inside the FP32 kernels' rounding band, where the FP64 distances decide.
* Pair inclusion ("Force Evaluation": particles within the cutoff of their
  type pair interact).  Pairs at d^2 == r_c^2 exactly in FP64 (excluded:
  the test is strict), and at r_c -+ 1e-7 sigma and r_c -+ 2e-6 sigma, for
  lipid-lipid (r_c), lipid-protein (2^(1/6) sigma_wca) and protein-protein
  (2^(1/6) sigma_pp) pairs, placed near 700 sigma from the origin where FP32
  spacing is widest.

Cell of every particle, storage permutation, centroids, radii, neighbouring
cells and the pair set must be bit-exact in every precision mode.
"""
import math

import numpy as np
import pytest

import oracle
from synth import membranes as M

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_1701_02059_gb300")

Q = 2.0 ** 40
TWO_SIXTH = 1.122462048309373


def grid(v):
    """Nearest point of the 2^-40 grid (both sides hold the state there)."""
    return np.round(np.asarray(v, np.float64) * Q) / Q


def exact_distance_pair(target2, axes):
    """Grid displacement whose FP64 squared distance, evaluated as
    ((dx*dx + dy*dy) + dz*dz), equals target2 exactly: a main component a
    and a small one b (about 0.01 sigma, so that one grid step of b moves
    the sum by a few FP64 ulps and some step lands on target2), placed on
    the two given axes; the third component is zero."""
    b0 = 0.01
    a0 = float(grid(math.sqrt(target2 - b0 * b0)))
    for k in range(0, 20000):
        a = a0 - k / Q
        rem = target2 - a * a
        if rem <= 0:
            continue
        bc = float(grid(math.sqrt(rem)))
        for t in range(-2, 3):
            b = bc + t / Q
            d = np.zeros(3)
            d[axes[0]] = a
            d[axes[1]] = b
            s = d[0] * d[0]
            s = s + d[1] * d[1]
            s = s + d[2] * d[2]
            if s == target2:
                return d
    raise AssertionError("no exact grid displacement found")


def cutoffs(m):
    rc_ll = m.rc
    rc_lp = TWO_SIXTH * m.sigma_wca
    rc_pp = TWO_SIXTH * m.sigma_pp
    return {(0, 0): rc_ll, (0, 2): rc_lp, (2, 2): rc_pp, (1, 2): rc_pp}


def build_nonperiodic():
    """Pair probes near (700, 700, 0) and centroid-tie probes near
    (700, 760, 0); one centroid per probe group plus the tie centroids."""
    m = oracle.model()
    cut = cutoffs(m)
    pos, typ, cents = [], [], []
    x0, y0 = 700.0, 700.0
    g = 0
    for (ti, tj) in [(0, 0), (0, 2), (2, 2), (1, 2)]:
        rc = cut[(ti, tj)]
        offsets = []
        # exactly at the cutoff (FP64 d^2 == rc*rc), along two directions
        for axes in ((0, 1), (2, 0)):
            offsets.append(exact_distance_pair(rc * rc, axes))
        # inside the FP32 band and just outside it, on both sides
        for dr in (-1e-7, 1e-7, -2e-6, 2e-6):
            u = np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)
            offsets.append(grid((rc + dr) * u))
        for d in offsets:
            base = grid([x0 + 10.0 * g, y0, 0.0])
            pos += [base, base + d]
            typ += [ti, tj]
            cents.append(base + grid(d / 2) + np.array([0.0, 0.0, 0.5]))
            g += 1
    # exact ties between centroids: a particle on the bisector of two, the
    # centre of three and of four centroids, and particles 1e-7 / 2e-6 off a
    # bisector (h = 4 sigma apart from the tie point)
    X, Y = 700.0, 760.0
    h = 4.0
    tie_c = [[X - h, Y, 0], [X + h, Y, 0], [X, Y + h, 0], [X, Y - h, 0]]
    cents += [grid(c) for c in tie_c]
    tie_p = [[X, Y, 0.0],                          # four-way tie
             [X + 1.5, Y + 1.5, 0.0],              # on the bisector of (X + h, Y) and (X, Y + h)
             [X - 1.25, Y - 1.25, 0.25],           # on the bisector of (X - h, Y) and (X, Y - h)
             [X + 1.0 + 1e-7, Y + 1.0, 0.0], [X - 1.0 - 1e-7, Y - 1.0, 0.0],
             [X + 1.0 + 2e-6, Y + 1.0, 0.1], [X - 1.0 + 2e-6, Y + 1.0, -0.1]]
    # a three-way tie: three centroids at distance h along x, y and z
    X3, Y3 = 760.0, 760.0
    cents += [grid(c) for c in ([X3 + h, Y3, 0.0], [X3, Y3 + h, 0.0], [X3, Y3, h])]
    tie_p += [[X3, Y3, 0.0]]
    for p in tie_p:
        pos.append(grid(p))
        typ.append(0)
    # lipids near every centroid so that no cell is far from its members,
    # each at least 0.9 sigma from every other particle
    rng = np.random.default_rng(7)
    for c in cents:
        placed = 0
        while placed < 3:
            p = grid(np.asarray(c) + rng.uniform(-1.5, 1.5, 3) * np.array([1, 1, 0.3]))
            if np.linalg.norm(np.asarray(pos) - p, axis=1).min() < 0.9:
                continue
            pos.append(p)
            typ.append(0)
            placed += 1
    return _membrane(np.array(pos), np.array(typ, np.uint8), np.array(cents), box=(0, 0, 0), periodic=(0, 0, 0))


def build_periodic():
    """A box periodic in x and y (40 x 36 sigma): centroids that tie only
    through the minimum image across the x = 0 and y = 0 faces."""
    L = (40.0, 36.0, 0.0)
    cents = [[1.0, 18.0, 0.0], [39.0, 18.0, 0.0],        # tie at x = 0 through the face
             [20.0, 1.5, 0.0], [20.0, 34.5, 0.0],        # tie at y = 0 through the face
             [10.0, 10.0, 0.0], [30.0, 26.0, 0.0], [10.0, 26.0, 0.0], [30.0, 10.0, 0.0]]
    # on the face bisectors (exact ties, two each), and 1e-7 / 2e-6 sigma
    # off them on either side of the face; all at least 1.5 sigma apart
    pos = [[0.0, 18.0, 0.0], [0.0, 16.5, 0.5], [1e-7, 20.5, 0.0], [40.0 - 1e-7, 13.5, 0.0],
           [20.0, 0.0, 0.0], [21.5, 0.0, -0.5], [23.5, 36.0 - 2e-6, 0.0], [18.5, 2e-6, 0.0]]
    rng = np.random.default_rng(8)
    for c in cents:
        placed = 0
        while placed < 4:
            p = np.asarray(c) + rng.uniform(-2.5, 2.5, 3) * np.array([1, 1, 0.2])
            p[:2] = np.mod(p[:2], L[:2])
            d = np.asarray(pos) - p
            d[:, :2] -= np.asarray(L[:2]) * np.rint(d[:, :2] / np.asarray(L[:2]))
            if np.linalg.norm(d, axis=1).min() < 0.9:
                continue
            pos.append(p)
            placed += 1
    pos = grid(np.array(pos))
    typ = np.zeros(len(pos), np.uint8)
    return _membrane(pos, typ, grid(np.array(cents)), box=L, periodic=(1, 1, 0))


def _membrane(pos, typ, cents, box, periodic):
    n = len(pos)
    ori = np.zeros((n, 3))
    ori[:, 2] = 1.0
    zeros = np.zeros((n, 3))
    mem = M.Membrane(pos, zeros.copy(), ori, zeros.copy(), typ, np.arange(n, dtype=np.uint32),
                     np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(0), tuple(box), tuple(periodic),
                     len(cents), 0.2)
    return mem, cents


def sorted_pairs(p):
    p = np.sort(np.asarray(p, np.int64), axis=1)
    return p[np.lexsort((p[:, 1], p[:, 0]))].astype(np.uint32)


def run_both(mem, cents, precision):
    p = G.make_params(kT=0.2, n_centroids=len(cents), box=mem.box, periodic=mem.periodic, seed=0, n_lloyd_init=0,
                      precision=precision)
    g = G.System(p)
    g.load_membrane(mem)
    g.init_cells(cents)
    o = oracle.OracleSystem(oracle.model(box=mem.box, periodic=mem.periodic),
                            oracle.run(kT=0.2, n_centroids=len(cents), seed=0, n_lloyd_init=0))
    o.load(mem)
    o.init_cells(cents)
    return g, o


def assert_cells_equal(g, o):
    a, b = g.cells(), o.cells()
    for k in ("cell_of_id", "slot_ids", "centroids", "start", "radius", "adj_ptr", "adj"):
        assert a[k].shape == b[k].shape, k
        assert np.array_equal(a[k], b[k]), f"{k} differs at {np.flatnonzero(a[k].ravel() != b[k].ravel())[:5]}"


PRECISIONS = [G.F32_FORCE_F64_STATE, G.F64_ALL, G.F32_FORCE_F32_STEP]


@pytest.mark.parametrize("precision", PRECISIONS)
def test_cutoff_and_bisector_cases_nonperiodic(precision):
    mem, cents = build_nonperiodic()
    m = oracle.model()
    g, o = run_both(mem, cents, precision)
    assert_cells_equal(g, o)
    st = o.state()
    # the construction: ties are exact in FP64 and each has its expected winner
    c = o.cells()
    assign = oracle.assign_brute(st["pos"], c["centroids"], mem.box, mem.periodic)
    assert np.array_equal(c["cell_of_id"], assign)
    ntie = []
    for pid in range(48, 56):
        d = st["pos"][pid] - c["centroids"]
        d2 = d[:, 0] * d[:, 0]
        d2 = d2 + d[:, 1] * d[:, 1]
        d2 = d2 + d[:, 2] * d[:, 2]
        ntie.append(int((d2 == d2.min()).sum()))
    # four-way, two-way (twice), none (the off-bisector four), three-way
    assert ntie == [4, 2, 2, 1, 1, 1, 1, 3], ntie
    brute = sorted_pairs(oracle.pairs_brute(m, st["pos"], mem.type, mem.id))
    assert np.array_equal(o.pairs(), brute)
    assert np.array_equal(g.pairs(), brute)
    # every probe pair at exactly r_c or outside the band-crossing distance
    # is absent, every one 1e-7 / 2e-6 inside is present
    cut = cutoffs(m)
    want_in = 0
    pairs = {tuple(p) for p in brute.tolist()}
    for q in range(0, 2 * 24, 2):
        ti, tj = int(mem.type[q]), int(mem.type[q + 1])
        d = st["pos"][q + 1] - st["pos"][q]
        d2 = d[0] * d[0]
        d2 = d2 + d[1] * d[1]
        d2 = d2 + d[2] * d[2]
        inside = d2 < cut[(ti, tj)] ** 2
        assert ((q, q + 1) in pairs) == inside
        want_in += inside
    assert want_in == 8     # the -1e-7 and -2e-6 probes of the four type pairs
    # forces within the mode's tolerance on the same cell list
    g.compute_forces()
    o.compute_forces()
    Fg, Fo = g.forces()[0], o.forces()[0]
    frms = max(np.sqrt((Fo ** 2).sum(1).mean()), 1e-12)
    err = (np.linalg.norm(Fg - Fo, axis=1) / np.maximum(np.linalg.norm(Fo, axis=1), frms)).max()
    assert err <= (1e-8 if precision == G.F64_ALL else 1e-5), err
    g.close()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_ties_through_the_periodic_faces(precision):
    mem, cents = build_periodic()
    g, o = run_both(mem, cents, precision)
    assert_cells_equal(g, o)
    st = o.state()
    c = o.cells()
    assert np.array_equal(c["cell_of_id"], oracle.assign_brute(st["pos"], c["centroids"], mem.box, mem.periodic))
    # the particles on the face bisectors tie between two cells and go to
    # the lower index of the two
    for pid, (ca, cb) in ((0, (0, 1)), (4, (2, 3))):
        d2 = []
        for k in range(len(cents)):
            d = st["pos"][pid] - c["centroids"][k]
            for a in range(2):
                d[a] = d[a] - mem.box[a] * np.rint(d[a] / mem.box[a])
            s = d[0] * d[0]
            s = s + d[1] * d[1]
            s = s + d[2] * d[2]
            d2.append(s)
        d2 = np.array(d2)
        best = np.flatnonzero(d2 == d2.min())
        assert len(best) >= 2, "construction lost its exact tie"
        assert g.cells()["cell_of_id"][pid] == best.min()
    assert np.array_equal(g.pairs(), o.pairs())
    g.rebuild_cells()
    o.rebuild()
    assert_cells_equal(g, o)
    g.close()
