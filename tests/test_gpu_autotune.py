"""Autotuner of the cell-tile shape on the GPU: it returns the centroid count
of one of the candidate particles-per-cell sizes, answers a system of the
same shape from its cache file without timing again, and the system it picks
keeps the exact pair set of any other cell count."""
import numpy as np
import pytest

import oracle
from synth import membranes as M

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_1701_02059_gb300")


def test_autotune_picks_a_candidate_and_caches(tmp_path):
    mem = M.patch(4, 31, n_centroids=150)
    p = G.make_params(kT=mem.kT, box=mem.box, periodic=mem.periodic, seed=9)
    cache = str(tmp_path / "tiles.txt")
    K, ms = G.autotune(p, mem, steps=5, cache=cache)
    n = mem.n
    assert K in {max(1, round(n / c)) for c in (32, 45, 61, 80, 100)}
    assert ms > 0
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and lines[0].split()[1] == str(K)
    # same shape: answered from the cache (same numbers, no new line)
    K2, ms2 = G.autotune(p, mem, steps=5, cache=cache)
    assert (K2, ms2) == (K, float(lines[0].split()[2]))
    assert len(open(cache).read().splitlines()) == 1
    # the chosen cell count gives the brute-force pair set
    g = G.System(G.make_params(kT=mem.kT, box=mem.box, periodic=mem.periodic, seed=9, n_centroids=K))
    g.load_membrane(mem)
    g.init_cells()
    m = oracle.model(box=mem.box, periodic=mem.periodic)
    pairs = np.sort(oracle.pairs_brute(m, mem.pos, mem.type, mem.id, mem.bonds).astype(np.int64), axis=1)
    brute = pairs[np.lexsort((pairs[:, 1], pairs[:, 0]))].astype(np.uint32)
    assert np.array_equal(g.pairs(), brute)
    g.close()
