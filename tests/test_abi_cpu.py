"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads,
exports every entry point that include/orbc.h declares, and its pure-host
calls behave."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "orbc.h")


def declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"ORBC_API\s+[\w\s\*]+?\b(orbc_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1701_02059_gb300 import build
    path = build.build()
    return path


def test_header_declares_the_boundary():
    names = declared()
    for want in ("orbc_create", "orbc_set_particles", "orbc_set_bonds", "orbc_init_cells", "orbc_rebuild_cells",
                 "orbc_compute_forces", "orbc_integrate", "orbc_get_state", "orbc_get_forces", "orbc_get_cells",
                 "orbc_dump_pairs", "orbc_last_error", "orbc_destroy"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (orbc_\w+)", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing


def test_binding_covers_the_exports(lib):
    from paper_1701_02059_gb300 import _native
    assert sorted(_native.EXPORTS) == declared()


def test_default_params_on_host(lib):
    from paper_1701_02059_gb300 import _native
    p = _native.default_params()
    assert (p.eps, p.sigma, p.rc_lipid, p.mu, p.zeta) == (1.0, 1.0, 2.6, 3.0, 4)
    assert (p.dt, p.kT, p.n_centroids, p.n_lloyd_init, p.rebuild_every) == (0.01, 0.2, 64, 10, 1)
    assert p.precision == 0 and tuple(p.periodic) == (0, 0, 0)
    # the ctypes mirror has the C layout (size checked against the compiler)
    src = '#include <stdio.h>\n#include "orbc.h"\nint main(){printf("%zu", sizeof(orbc_params));return 0;}\n'
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "s")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        size = int(subprocess.run([exe], capture_output=True, text=True, check=True).stdout)
    assert C.sizeof(_native.Params) == size


def test_null_handles_are_rejected(lib):
    from paper_1701_02059_gb300 import _native
    L = _native.load()
    assert L.orbc_create(None, None, None) == _native.ORBC_E_ARG
    assert L.orbc_integrate(None, 1) == _native.ORBC_E_ARG
    assert L.orbc_compute_forces(None, None) == _native.ORBC_E_ARG
    assert L.orbc_set_particles_device(None, 1, None, None, None, None, None, None) == _native.ORBC_E_ARG
    assert L.orbc_get_state_device(None, None, None, None, None) == _native.ORBC_E_ARG
    assert L.orbc_get_forces_device(None, None, None) == _native.ORBC_E_ARG
    assert L.orbc_last_error(None) == b"null handle"
    L.orbc_destroy(None)


def test_arena_null_handles_and_arguments_are_rejected(lib):
    from paper_1701_02059_gb300 import _native
    L = _native.load()
    h = C.c_void_p()
    assert L.orbc_arena_create(0, 0, None, C.byref(h)) == _native.ORBC_E_ARG       # no budget
    assert L.orbc_arena_create(1 << 30, 7, None, C.byref(h)) == _native.ORBC_E_ARG  # unknown precision
    assert L.orbc_arena_create(1 << 30, 0, None, None) == _native.ORBC_E_ARG
    assert not h
    n = C.c_int(0)
    assert L.orbc_arena_run(None, 1, 1, C.byref(n)) == _native.ORBC_E_ARG
    assert L.orbc_arena_poll(None, None, 0, C.byref(n)) == _native.ORBC_E_ARG
    assert L.orbc_arena_retire(None, 0, None, None, None, None, None) == _native.ORBC_E_ARG
    slot = C.c_int(5)
    p = _native.default_params()
    assert L.orbc_arena_admit(None, C.byref(p), 1, None, None, None, None, None, None, 0, None, None, None, 1,
                              C.byref(slot)) == _native.ORBC_E_ARG
    assert L.orbc_arena_info(None, None, None, None, None, None) == _native.ORBC_E_ARG
    done = C.c_int(3)
    reqs = (_native.ArenaRequest * 1)()
    slots = (C.c_int * 1)()
    assert L.orbc_arena_admit_many(None, reqs, 1, 4, slots, C.byref(done)) == _native.ORBC_E_ARG
    b = C.c_ulonglong(7)
    assert L.orbc_arena_slot_bytes(None, 0, C.byref(b)) == _native.ORBC_E_ARG and b.value == 7
    assert L.orbc_arena_launch_count(None) == -1
    assert L.orbc_arena_stats(None, None, None, None, None) == _native.ORBC_E_ARG
    assert L.orbc_arena_last_error(None) == b"null handle"
    L.orbc_arena_destroy(None)


def test_autotune_rejects_bad_arguments(lib):
    from paper_1701_02059_gb300 import _native
    L = _native.load()
    p = _native.default_params()
    K = C.c_int(0)
    assert L.orbc_autotune(None, 1, None, None, None, None, None, None, 0, None, None, None, 5, None, C.byref(K),
                           None, None) == _native.ORBC_E_ARG
    assert L.orbc_autotune(C.byref(p), 1, None, None, None, None, None, None, 0, None, None, None, 0, None, C.byref(K),
                           None, None) == _native.ORBC_E_ARG                # no timed steps
    assert L.orbc_autotune(C.byref(p), 1, None, None, None, None, None, None, 0, None, None, None, 5, None, None,
                           None, None) == _native.ORBC_E_ARG                # no output
    assert L.orbc_autotune(C.byref(p), 4, None, None, None, None, None, None, 0, None, None, None, 5, None, C.byref(K),
                           None, None) == _native.ORBC_E_ARG                # null particle arrays


def test_ctypes_mirrors_have_the_c_layout():
    """Every struct the binding passes across the boundary has the size and
    field offsets the C compiler gives the header's declaration."""
    from paper_1701_02059_gb300 import _native
    import tempfile
    mirrors = {"orbc_params": _native.Params, "orbc_mesh_params": _native.MeshParams,
               "orbc_arena_request": _native.ArenaRequest}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "orbc.h"', 'int main(void) {']
    expect = []
    for cname, ct in mirrors.items():
        lines.append(f'    printf("%zu\\n", sizeof({cname}));')
        expect.append(C.sizeof(ct))
        for f in ct._fields_:
            lines.append(f'    printf("%zu\\n", offsetof({cname}, {f[0]}));')
            expect.append(getattr(ct, f[0]).offset)
    lines += ['    return 0;', '}']
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        open(c, "w").write("\n".join(lines) + "\n")
        exe = os.path.join(d, "layout")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        got = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert got == expect
