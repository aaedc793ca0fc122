"""Device-pointer variants of the boundary (orbc_set_particles_device,
orbc_get_state_device, orbc_get_forces_device) against the host-pointer
calls: the same system set up either way steps identically, and the device
getters return exactly the host getters' values (both are the fixed-point
state scaled by a power of two)."""
import numpy as np
import pytest

from synth import membranes as M

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_1701_02059_gb300")
torch = pytest.importorskip("torch")


def params(mem):
    return G.make_params(kT=mem.kT, n_centroids=mem.n_centroids, box=mem.box, periodic=mem.periodic, seed=3)


def device_system(mem):
    g = G.System(params(mem))
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dt)).cuda()
    g.set_particles_tensors(t(mem.pos, np.float64), t(mem.vel, np.float64), t(mem.ori, np.float64),
                            t(mem.angvel, np.float64), t(mem.type, np.uint8), t(mem.id, np.int32))
    if len(mem.r0):
        g.set_bonds(mem.bonds, mem.r0, mem.kb)
    return g


@pytest.mark.parametrize("name", ["patch-2304", "vesicle-3.6k"])
def test_device_io_matches_host_io(name):
    mem = M.flat_patch_2304() if name == "patch-2304" else M.vesicle(3000, 5, f=2, chain_beads=5, n_centroids=50)
    h = G.System(params(mem))
    h.load_membrane(mem)
    d = device_system(mem)
    for g in (h, d):
        g.init_cells()
        g.integrate(20)
        g.compute_forces()
    sh, sd = h.state(), d.state_tensors()
    for k in ("pos", "vel", "ori", "angvel"):
        assert np.array_equal(sh[k], sd[k].cpu().numpy()), k
    Fh, Th = h.forces()
    Fd, Td = d.force_tensors()
    assert np.array_equal(Fh, Fd.cpu().numpy())
    assert np.array_equal(Th, Td.cpu().numpy())
    # NULL outputs are skipped
    assert d._L.orbc_get_state_device(d._h, None, None, None, None) == 0
    h.close()
    d.close()


def test_device_getters_need_state():
    mem = M.flat_patch_2304()
    g = G.System(params(mem))
    with pytest.raises(RuntimeError):
        g.state_tensors()
    g.load_membrane(mem)
    with pytest.raises(RuntimeError):
        g.force_tensors()
    g.close()


def test_lazy_setup_keeps_the_trajectory():
    """The device set-up is deferred to the first call that needs it: the
    state reads back right after set_particles, and setting the bonds again
    after some steps keeps the stepped state (the host copy is refreshed
    from the device first)."""
    mem = M.flat_patch_2304()
    g = G.System(params(mem))
    g.set_particles(mem.pos, mem.vel, mem.ori, mem.angvel, mem.type, mem.id)
    st0 = g.state()
    assert np.array_equal(st0["pos"], np.rint(mem.pos * 2.0 ** 40) / 2.0 ** 40)
    g.set_bonds(mem.bonds, mem.r0, mem.kb)
    g.init_cells()
    g.integrate(5)
    st5 = g.state()
    g.set_bonds(mem.bonds, mem.r0, mem.kb)
    g.init_cells()
    st5b = g.state()
    for k in ("pos", "vel", "ori", "angvel"):
        assert np.array_equal(st5[k], st5b[k]), k
    assert st5b["step"] == 5
    g.close()


def test_too_many_bonds_on_one_particle_is_rejected():
    """A particle with more than 8 bonds is refused when the device lists are
    built (the first call that needs the device), with ORBC_E_ARG."""
    mem = M.flat_patch_2304()
    g = G.System(params(mem))
    g.set_particles(mem.pos, mem.vel, mem.ori, mem.angvel, mem.type, mem.id)
    hub = 0
    ij = np.array([[hub, j] for j in range(1, 11)], np.int32)
    g.set_bonds(ij, np.ones(len(ij)), np.ones(len(ij)))
    with pytest.raises(G.OrbcError) as e:
        g.init_cells()
    assert e.value.code == -1
    g.close()


def test_pinned_host_buffers_match_pageable():
    """Page-locked inputs and caller-owned page-locked outputs give the same
    trajectory and state as ordinary numpy arrays."""
    import dataclasses
    mem = M.flat_patch_2304()

    def pinned(a):
        a = np.ascontiguousarray(a)
        buf = torch.empty(max(a.nbytes, 1), dtype=torch.uint8, pin_memory=True).numpy()
        out = buf[:a.nbytes].view(a.dtype).reshape(a.shape)
        out[...] = a
        return out

    pm = dataclasses.replace(mem, **{k: pinned(getattr(mem, k))
                                     for k in ("pos", "vel", "ori", "angvel", "type", "id", "bonds", "r0", "kb")})
    out = {k: pinned(np.full((mem.n, 3), np.nan)) for k in ("pos", "vel", "ori", "angvel")}
    a, b = G.System(params(mem)), G.System(params(mem))
    a.load_membrane(mem)
    b.load_membrane(pm)
    for g in (a, b):
        g.init_cells()
        g.integrate(10)
    sa, sb = a.state(), b.state(out=out)
    assert sb["step"] == sa["step"] == 10
    for k in ("pos", "vel", "ori", "angvel"):
        assert sb[k] is out[k]
        assert np.array_equal(sa[k], out[k]), k
    with pytest.raises(ValueError):
        b.state(out={k: np.empty((mem.n, 3), np.float32) for k in out})
    a.close()
    b.close()
