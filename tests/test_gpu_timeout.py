"""The bounded waits of the pair kernels on the GPU.

Every kernel wait on a shared-memory staging barrier has an iteration
limit; when it runs out the kernel records a timeout, waits (bounded) for
its copies and leaves, and the call returns ORBC_E_TIMEOUT with the context
intact.  orbc_set_wait_test makes the barrier expect 16 bytes more than the
copies bring, so every copy lands and only the barrier count is short: the
wait runs out after the shortened limit.  The handle must stay usable:
with normal settings the next call gives the same forces as before.
"""
import numpy as np
import pytest

from synth import membranes as M

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_1701_02059_gb300")
from paper_1701_02059_gb300 import _native  # noqa: E402


def test_staging_wait_runs_out_and_the_handle_stays_usable():
    mem = M.vesicle(3000, 41, f=2, chain_beads=5, n_centroids=50)
    g = G.System(G.make_params(kT=mem.kT, n_centroids=mem.n_centroids, box=mem.box, periodic=mem.periodic, seed=41))
    g.load_membrane(mem)
    g.init_cells()
    g.compute_forces()
    F0, T0 = g.forces()
    g.set_wait_test(extra_tx_bytes=16, max_polls=4096)
    g.rebuild_cells()                         # the next call searches the neighbour lists again
    with pytest.raises(G.OrbcError) as e:
        g.compute_forces()                    # the split path's list search waits
    assert e.value.code == _native.ORBC_E_TIMEOUT
    with pytest.raises(G.OrbcError) as e:
        g.compute_forces(energies=True)       # the one-launch kernel waits the same way
    assert e.value.code == _native.ORBC_E_TIMEOUT
    g.set_wait_test(0, 1 << 22)
    g.compute_forces()                        # forces do not depend on the cell list
    F1, T1 = g.forces()
    assert np.array_equal(F0, F1) and np.array_equal(T0, T1)
    g.integrate(3)
    assert g.state()["step"] == 3
    g.close()


def test_wait_test_arguments_are_checked():
    mem = M.flat_patch_2304(seed=41)
    g = G.System(G.make_params(kT=mem.kT, n_centroids=mem.n_centroids, box=mem.box, periodic=mem.periodic))
    for extra, polls in ((8, 100), (16, 0), (8192, 100), (0, (1 << 22) + 1)):
        with pytest.raises(G.OrbcError) as e:
            g.set_wait_test(extra, polls)
        assert e.value.code == _native.ORBC_E_ARG
    g.close()
