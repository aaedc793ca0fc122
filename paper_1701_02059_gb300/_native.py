"""ctypes binding of liborbc.so (the C ABI of include/orbc.h).

Argument marshalling only: every step of the hot path runs in the CUDA
library.  Loading fails loudly when the library is missing; there is no CPU
fallback."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liborbc.so")

ORBC_OK, ORBC_E_ARG, ORBC_E_NOMEM, ORBC_E_CUDA, ORBC_E_STATE, ORBC_E_NAN, ORBC_E_TIMEOUT = 0, -1, -2, -3, -4, -5, -6
# particle types (orbc.h): lipid, junction (actin), spectrin bead, band-3, glycophorin
LIPID, JUNCTION, SPECTRIN, BAND3, GLYCOPHORIN = 0, 1, 2, 3, 4
F32_FORCE_F64_STATE, F64_ALL, F32_FORCE_F32_STEP = 0, 1, 2
STATUS_NAMES = {0: "ORBC_OK", -1: "ORBC_E_ARG", -2: "ORBC_E_NOMEM", -3: "ORBC_E_CUDA", -4: "ORBC_E_STATE",
                -5: "ORBC_E_NAN", -6: "ORBC_E_TIMEOUT"}

EXPORTS = [
    "orbc_default_params", "orbc_create", "orbc_set_particles", "orbc_set_bonds", "orbc_init_cells",
    "orbc_rebuild_cells", "orbc_compute_forces", "orbc_integrate", "orbc_get_state", "orbc_get_forces",
    "orbc_get_cells", "orbc_get_adjacency_len", "orbc_dump_pairs", "orbc_set_timing", "orbc_set_wait_test", "orbc_get_kernel_times",
    "orbc_get_launch_count", "orbc_last_error", "orbc_destroy", "orbc_cell_sort", "orbc_cell_sort_noalloc",
    "orbc_arena_create", "orbc_arena_admit", "orbc_arena_admit_many", "orbc_arena_slot_bytes", "orbc_arena_run", "orbc_arena_poll", "orbc_arena_retire",
    "orbc_arena_info", "orbc_arena_launch_count", "orbc_arena_last_error", "orbc_arena_destroy",
    "orbc_autotune", "orbc_arena_stats", "orbc_set_particles_device", "orbc_get_state_device",
    "orbc_get_forces_device", "orbc_default_mesh_params", "orbc_mesh_build", "orbc_quench",
    "orbc_set_volume_constraint", "orbc_get_volume", "orbc_height_map", "orbc_set_step_fusion",
]
_NOT_INT = {"orbc_default_params": None, "orbc_default_mesh_params": None, "orbc_last_error": C.c_char_p, "orbc_destroy": None,
            "orbc_arena_launch_count": C.c_longlong, "orbc_arena_last_error": C.c_char_p, "orbc_arena_destroy": None}


class Params(C.Structure):
    """Mirror of orbc_params."""
    _fields_ = [("eps", C.c_double), ("sigma", C.c_double), ("rc_lipid", C.c_double), ("mu", C.c_double),
                ("sin_theta0", C.c_double), ("zeta", C.c_int), ("pad0", C.c_int),
                ("eps_wca", C.c_double), ("sigma_wca", C.c_double), ("sigma_wca_pp", C.c_double),
                ("dt", C.c_double), ("kT", C.c_double), ("gamma_t", C.c_double), ("gamma_r", C.c_double),
                ("mass", C.c_double), ("inertia", C.c_double),
                ("box", C.c_double * 3), ("periodic", C.c_int * 3),
                ("n_centroids", C.c_int), ("n_lloyd_init", C.c_int), ("rebuild_every", C.c_int),
                ("skin", C.c_double), ("grid_h", C.c_double), ("seed", C.c_ulonglong), ("instance", C.c_uint),
                ("precision", C.c_int), ("n_protein_centroids", C.c_int), ("eval_ctas", C.c_int),
                ("eps_mem", (C.c_double * 3) * 3), ("rc_mem", (C.c_double * 3) * 3)]


class ArenaRequest(C.Structure):
    """orbc_arena_request: one request of orbc_arena_admit_many."""
    _fields_ = [("params", C.POINTER(Params)), ("n", C.c_int), ("pos", C.c_void_p), ("vel", C.c_void_p),
                ("ori", C.c_void_p), ("angvel", C.c_void_p), ("type", C.c_void_p), ("id", C.c_void_p),
                ("nb", C.c_int), ("ij", C.c_void_p), ("r0", C.c_void_p), ("kb", C.c_void_p), ("nsteps", C.c_longlong)]


class MeshParams(C.Structure):
    """Mirror of orbc_mesh_params."""
    _fields_ = [("spacing", C.c_double), ("slack", C.c_double), ("kb", C.c_double), ("offset", C.c_double),
                ("d_min", C.c_double), ("d_ll", C.c_double), ("beads", C.c_int), ("pad0", C.c_int),
                ("seed", C.c_ulonglong), ("band3_fraction", C.c_double), ("kb_anchor", C.c_double),
                ("glycophorin", C.c_int), ("band3_edges", C.c_int)]


class OrbcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(path: str | None = None):
    """Load liborbc.so (built by paper_1701_02059_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"liborbc.so not found at {p}: build it with python -m paper_1701_02059_gb300.build")
    L = C.CDLL(p)
    V = C.c_void_p
    L.orbc_default_params.argtypes = [C.POINTER(Params)]
    L.orbc_default_params.restype = None
    L.orbc_create.argtypes = [C.POINTER(Params), V, C.POINTER(V)]
    L.orbc_set_particles.argtypes = [V, C.c_int, V, V, V, V, V, V]
    L.orbc_set_bonds.argtypes = [V, C.c_int, V, V, V]
    L.orbc_init_cells.argtypes = [V, V]
    L.orbc_rebuild_cells.argtypes = [V]
    L.orbc_compute_forces.argtypes = [V, V]
    L.orbc_integrate.argtypes = [V, C.c_int]
    L.orbc_get_state.argtypes = [V, V, V, V, V, V]
    L.orbc_get_forces.argtypes = [V, V, V]
    L.orbc_get_cells.argtypes = [V, V, V, V, V, V, V, V]
    L.orbc_get_adjacency_len.argtypes = [V, C.POINTER(C.c_longlong)]
    L.orbc_dump_pairs.argtypes = [V, C.c_longlong, V, C.POINTER(C.c_longlong)]
    L.orbc_set_timing.argtypes = [V, C.c_int]
    L.orbc_set_wait_test.argtypes = [V, C.c_uint, C.c_uint]
    L.orbc_default_mesh_params.argtypes = [V]
    L.orbc_mesh_build.argtypes = [V, C.c_int, V, C.c_int, V, C.c_longlong, V, V, V, V, C.c_longlong, V, V, V, V, V]
    L.orbc_quench.argtypes = [V, C.c_int, C.c_double, C.c_double, C.c_double, V]
    L.orbc_set_volume_constraint.argtypes = [V, C.c_double, C.c_double, C.c_double, V]
    L.orbc_set_step_fusion.argtypes = [V, C.c_int]
    L.orbc_get_volume.argtypes = [V, C.c_double, V, C.POINTER(C.c_double)]
    L.orbc_height_map.argtypes = [V, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, C.c_double,
                                  V, C.c_double, C.c_double, V, V]
    L.orbc_get_kernel_times.argtypes = [V, C.c_char_p, C.c_int, V, C.c_int, C.POINTER(C.c_int)]
    L.orbc_get_launch_count.argtypes = [V, C.POINTER(C.c_longlong)]
    L.orbc_cell_sort.argtypes = [V, C.c_int, C.c_int, V, V, V]
    L.orbc_cell_sort_noalloc.argtypes = [V, C.c_int, C.c_int, V, V, V]
    L.orbc_last_error.argtypes = [V]
    L.orbc_last_error.restype = C.c_char_p
    L.orbc_destroy.argtypes = [V]
    L.orbc_arena_create.argtypes = [C.c_ulonglong, C.c_int, V, C.POINTER(V)]
    L.orbc_arena_admit.argtypes = [V, C.POINTER(Params), C.c_int, V, V, V, V, V, V, C.c_int, V, V, V,
                                   C.c_longlong, C.POINTER(C.c_int)]
    L.orbc_arena_admit_many.argtypes = [V, C.POINTER(ArenaRequest), C.c_int, C.c_int, V, C.POINTER(C.c_int)]
    L.orbc_arena_slot_bytes.argtypes = [V, C.c_int, C.POINTER(C.c_ulonglong)]
    L.orbc_arena_run.argtypes = [V, C.c_int, C.c_int, C.POINTER(C.c_int)]
    L.orbc_arena_poll.argtypes = [V, V, C.c_int, C.POINTER(C.c_int)]
    L.orbc_arena_retire.argtypes = [V, C.c_int, V, V, V, V, C.POINTER(C.c_longlong)]
    L.orbc_arena_info.argtypes = [V, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                  C.POINTER(C.c_longlong), C.POINTER(C.c_ulonglong)]
    L.orbc_arena_launch_count.argtypes = [V]
    L.orbc_arena_last_error.argtypes = [V]
    L.orbc_arena_destroy.argtypes = [V]
    L.orbc_set_particles_device.argtypes = [V, C.c_int, V, V, V, V, V, V]
    L.orbc_get_state_device.argtypes = [V, V, V, V, V]
    L.orbc_get_forces_device.argtypes = [V, V, V]
    L.orbc_arena_stats.argtypes = [V, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                                   C.POINTER(C.c_longlong)]
    L.orbc_autotune.argtypes = [C.POINTER(Params), C.c_int, V, V, V, V, V, V, C.c_int, V, V, V, C.c_int, C.c_char_p,
                                C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)]
    for name in EXPORTS:
        getattr(L, name).restype = _NOT_INT.get(name, C.c_int) if name in _NOT_INT else C.c_int
    _lib = L
    return L


def default_params() -> Params:
    p = Params()
    load().orbc_default_params(C.byref(p))
    return p
