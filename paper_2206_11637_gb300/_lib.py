"""ctypes binding of libpflbm.so (include/pflbm.h): argument marshalling only.

Every step of the PFLBM path runs in the library's CUDA kernels.  Loading fails
loudly when the library has not been built; there is no CPU fallback.
"""
import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpflbm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "pflbm.h")

PFL_OK, PFL_ERR_ARG, PFL_ERR_CUDA, PFL_ERR_OOM, PFL_ERR_UNSTABLE, PFL_ERR_STATE = range(6)
PFL_SPEED_LIMIT = 0.3
PFL_FP64, PFL_FP32, PFL_FP16S = 0, 1, 2
PFL_PERIODIC, PFL_NOSLIP = 0, 1
PFL_MRT, PFL_BGK = 0, 1
PFL_ENGINE_AUTO, PFL_ENGINE_INPLACE = 0, 1
STATUS_NAMES = {0: "PFL_OK", 1: "PFL_ERR_ARG", 2: "PFL_ERR_CUDA", 3: "PFL_ERR_OOM", 4: "PFL_ERR_UNSTABLE",
                5: "PFL_ERR_STATE"}


class pfl_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("bc", ctypes.c_int * 6),
                ("rho_h", ctypes.c_double), ("rho_l", ctypes.c_double),
                ("nu_h", ctypes.c_double), ("nu_l", ctypes.c_double),
                ("sigma", ctypes.c_double), ("mobility", ctypes.c_double), ("xi", ctypes.c_double),
                ("gravity", ctypes.c_double * 3),
                ("precision", ctypes.c_int), ("collision", ctypes.c_int), ("engine", ctypes.c_int),
                ("h_lattice", ctypes.c_int), ("solids", ctypes.c_int),
                ("hydrostatic", ctypes.c_int), ("p_level", ctypes.c_double)]


class PFLError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None


def load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libpflbm.so is not built (run __graft_entry__.build() or "
                           "python -m paper_2206_11637_gb300.build); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    P, D, I, S = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_size_t
    PP = ctypes.POINTER(pfl_params)
    lib.pfl_workspace_bytes.restype = S
    lib.pfl_workspace_bytes.argtypes = [PP]
    lib.pfl_hydrostatic_pstar.restype = I
    lib.pfl_hydrostatic_pstar.argtypes = [PP, P, P]
    lib.pfl_init.restype = I
    lib.pfl_init.argtypes = [PP, P, P, P, P, S, P, ctypes.POINTER(P)]
    lib.pfl_step.restype = I
    lib.pfl_step.argtypes = [P, I]
    lib.pfl_set_graph_steps.restype = I
    lib.pfl_set_graph_steps.argtypes = [P, I]
    lib.pfl_fields.restype = I
    lib.pfl_fields.argtypes = [P, P, P, P, P]
    lib.pfl_populations.restype = I
    lib.pfl_populations.argtypes = [P, P, P]
    lib.pfl_set_populations.restype = I
    lib.pfl_set_populations.argtypes = [P, P, P]
    lib.pfl_set_solid.restype = I
    lib.pfl_set_solid.argtypes = [P, P]
    lib.pfl_interface_height.restype = I
    lib.pfl_interface_height.argtypes = [P, I, I, P]
    lib.pfl_state_bytes.restype = ctypes.c_size_t
    lib.pfl_state_bytes.argtypes = [P]
    lib.pfl_save.restype = I
    lib.pfl_save.argtypes = [P, P, ctypes.c_size_t]
    lib.pfl_load.restype = I
    lib.pfl_load.argtypes = [P, P, ctypes.c_size_t]
    lib.pfl_diag.restype = I
    lib.pfl_diag.argtypes = [P, P, ctypes.POINTER(ctypes.c_longlong)]
    lib.pfl_max_speed.restype = I
    lib.pfl_max_speed.argtypes = [P, P]
    lib.pfl_adjoint_workspace_bytes.restype = S
    lib.pfl_adjoint_workspace_bytes.argtypes = [P, I]
    lib.pfl_adjoint.restype = I
    lib.pfl_adjoint.argtypes = [P, I, I, P, P, P, S, P, P]
    lib.pfl_phi_moments_static.restype = I
    lib.pfl_phi_moments_static.argtypes = [P, I, I, I, I, P, ctypes.POINTER(ctypes.c_longlong), P]
    lib.pfl_batch_workspace_bytes.restype = S
    lib.pfl_batch_workspace_bytes.argtypes = [P, I]
    lib.pfl_batch_init.restype = I
    lib.pfl_batch_init.argtypes = [P, I, P, P, P, P, S, P, I, ctypes.POINTER(P)]
    lib.pfl_batch_step.restype = I
    lib.pfl_batch_step.argtypes = [P, I]
    lib.pfl_batch_fields.restype = I
    lib.pfl_batch_fields.argtypes = [P, I, P, P, P, P]
    lib.pfl_batch_diag.restype = I
    lib.pfl_batch_diag.argtypes = [P, P, P]
    lib.pfl_batch_shapes.restype = I
    lib.pfl_batch_shapes.argtypes = [P, P, P, P]
    lib.pfl_batch_set_shape.restype = I
    lib.pfl_batch_set_shape.argtypes = [P, I, I, I, I, I]
    lib.pfl_batch_time.restype = ctypes.c_longlong
    lib.pfl_batch_time.argtypes = [P]
    lib.pfl_batch_destroy.restype = None
    lib.pfl_batch_destroy.argtypes = [P]
    lib.pfl_kernel_times.restype = I
    lib.pfl_kernel_times.argtypes = [P, I, P]
    lib.pfl_time.restype = ctypes.c_longlong
    lib.pfl_time.argtypes = [P]
    lib.pfl_destroy.restype = None
    lib.pfl_destroy.argtypes = [P]
    lib.pfl_last_error.restype = ctypes.c_char_p
    lib.pfl_last_error.argtypes = []
    lib.pfl_version.restype = I
    lib.pfl_version.argtypes = []
    _lib = lib
    return lib


def check(status):
    if status != PFL_OK:
        raise PFLError(status, load().pfl_last_error().decode())
    return status


def declared_symbols():
    """Names of the functions declared in include/pflbm.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pfl_[a-z_]+)\s*\(", text)))
