"""ctypes binding of the C ABI declared in include/fep3m.h (argument marshalling only)."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfep3m.so")

FEP3M_OK, FEP3M_EINVAL, FEP3M_ENOTNEUTRAL, FEP3M_ENOMEM, FEP3M_ECUDA, FEP3M_ENOCONV, FEP3M_ESTATE, FEP3M_ETIMEOUT = \
    0, -1, -2, -3, -4, -5, -6, -7
FEP3M_FP64, FEP3M_MIXED = 0, 1
FEP3M_NEUTRALIZE = 1
FEP3M_CUDA_CORES = 2
FEP3M_MULTIGRID = 4
FEP3M_ONE_ELEMENT = 8
FEP3M_DIRICHLET = 16
FEP3M_NEUMANN = 32
FEP3M_NEUMANN_NGL = 8


class Config(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double), ("n_el", ctypes.c_int), ("q", ctypes.c_int), ("n_sr", ctypes.c_int),
                ("precision", ctypes.c_int), ("mg_rtol", ctypes.c_double), ("mg_max_cycles", ctypes.c_int),
                ("table_pad", ctypes.c_int), ("flags", ctypes.c_uint)]


class Stats(ctypes.Structure):
    _fields_ = [("n_particles", ctypes.c_int64), ("mg_levels", ctypes.c_int), ("mg_iterations", ctypes.c_int),
                ("refine_steps", ctypes.c_int), ("mg_rel_residual", ctypes.c_double),
                ("adj_iterations", ctypes.c_int), ("adj_rel_residual", ctypes.c_double),
                ("singular_pairs", ctypes.c_int64), ("nonempty_elements", ctypes.c_int64),
                ("max_per_element", ctypes.c_int), ("ms_bin", ctypes.c_double), ("ms_assemble", ctypes.c_double),
                ("ms_solve", ctypes.c_double), ("ms_pair", ctypes.c_double), ("ms_adjoint", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("screen_element_pairs", ctypes.c_int64),
                ("screen_charge_pairs", ctypes.c_int64), ("ms_pair_screen", ctypes.c_double),
                ("ms_pair_eval", ctypes.c_double), ("ms_inner_solve", ctypes.c_double), ("solve_rhs", ctypes.c_int)]


P = ctypes.c_void_p
SIGNATURES = {
    "fep3m_create": (ctypes.c_int, [ctypes.POINTER(Config), P, ctypes.POINTER(P)]),
    "fep3m_set_particles": (ctypes.c_int, [P, ctypes.c_int64, P, P]),
    "fep3m_compute": (ctypes.c_int, [P, P, P, P]),
    "fep3m_vjp": (ctypes.c_int, [P, ctypes.c_double, P, P, P]),
    "fep3m_get_stats": (ctypes.c_int, [P, ctypes.POINTER(Stats)]),
    "fep3m_set_timing": (ctypes.c_int, [P, ctypes.c_int]),
    "fep3m_get_binning": (ctypes.c_int, [P, P, P, P, P]),
    "fep3m_get_mesh": (ctypes.c_int, [P, P, P, P]),
    "fep3m_solve_mesh": (ctypes.c_int, [P, P, P]),
    "fep3m_get_table": (ctypes.c_int, [P, P]),
    "fep3m_set_boundary": (ctypes.c_int, [P, P]),
    "fep3m_mesh_eigenbasis": (ctypes.c_int, [ctypes.c_int, P, P]),
    "fep3m_mesh_eigenbasis_order": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, P, P]),
    "fep3m_screen_type_table": (ctypes.c_int, [ctypes.c_int] * 6 + [P]),
    "fep3m_screen_node_table": (ctypes.c_int, [ctypes.c_int] * 3 + [P]),
    "fep3m_screen_weight_poly": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, P]),
    "fep3m_box_eigenbasis": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P]),
    "fep3m_load_vector_static": (ctypes.c_int, [ctypes.c_double, ctypes.c_int, ctypes.c_int64, P, P, P, P]),
    "fep3m_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "fep3m_destroy": (None, [P]),
}

_lib = None


def load():
    """Load libfep3m.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libfep3m.so is not built (run __graft_entry__.build()); the FE-P3M path has no "
                           "CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class FEP3MError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        msg = load().fep3m_strerror(status).decode()
        super().__init__("%s: %s (status %d)" % (what, msg, status))


def check(status, what, allow=()):
    if status != FEP3M_OK and status not in allow:
        raise FEP3MError(status, what)
    return status
