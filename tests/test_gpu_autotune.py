"""Autotuner of the cell-tile shape and of the pair evaluation's launch shape
on the GPU: it returns the centroid count of one of the candidate
particles-per-cell sizes and one of the compiled occupancies, answers a
system of the same shape from its cache file without timing again, the
system it picks keeps the exact pair set of any other cell count, and the
launch shape leaves the forces unchanged bit for bit."""
import numpy as np
import pytest

import oracle
from synth import membranes as M

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_1701_02059_gb300")
from paper_1701_02059_gb300 import _native  # noqa: E402


def test_autotune_picks_a_candidate_in_both_dimensions_and_caches(tmp_path):
    mem = M.patch(4, 31, n_centroids=150)
    p = G.make_params(kT=mem.kT, box=mem.box, periodic=mem.periodic, seed=9)
    cache = str(tmp_path / "tiles.txt")
    K, ctas, ms = G.autotune(p, mem, steps=5, cache=cache)
    n = mem.n
    assert K in {max(1, round(n / c)) for c in (32, 45, 61, 80, 100)}
    assert ctas in (5, 7) and ms > 0
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and lines[0].split()[1:3] == [str(K), str(ctas)]
    # same shape: answered from the cache (same numbers, no new line)
    assert G.autotune(p, mem, steps=5, cache=cache) == (K, ctas, float(lines[0].split()[3]))
    assert len(open(cache).read().splitlines()) == 1
    # the chosen cell count and launch shape give the brute-force pair set
    g = G.System(G.make_params(kT=mem.kT, box=mem.box, periodic=mem.periodic, seed=9, n_centroids=K, eval_ctas=ctas))
    g.load_membrane(mem)
    g.init_cells()
    m = oracle.model(box=mem.box, periodic=mem.periodic)
    pairs = np.sort(oracle.pairs_brute(m, mem.pos, mem.type, mem.id, mem.bonds).astype(np.int64), axis=1)
    brute = pairs[np.lexsort((pairs[:, 1], pairs[:, 0]))].astype(np.uint32)
    assert np.array_equal(g.pairs(), brute)
    g.close()


def test_eval_launch_shape_leaves_trajectories_unchanged():
    mem = M.vesicle(3000, 5, f=2, chain_beads=5, n_centroids=50)
    out = []
    for ctas in (5, 7):
        g = G.System(G.make_params(kT=mem.kT, n_centroids=mem.n_centroids, seed=4, eval_ctas=ctas))
        g.load_membrane(mem)
        g.init_cells()
        g.integrate(20)
        out.append((g.state(), g.forces()))
        g.close()
    (sa, fa), (sb, fb) = out
    for k in ("pos", "vel", "ori", "angvel"):
        assert np.array_equal(sa[k], sb[k])
    assert np.array_equal(fa[0], fb[0]) and np.array_equal(fa[1], fb[1])
    with pytest.raises(G.OrbcError) as e:
        G.System(G.make_params(eval_ctas=6))
    assert e.value.code == _native.ORBC_E_ARG
