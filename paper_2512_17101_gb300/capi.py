"""ctypes declarations of libdg's C ABI (include/dg.h).

Loading fails loudly if libdg.so has not been built: there is no fallback.
"""

from __future__ import annotations

import ctypes
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libdg.so")

DG_OK = 0
DG_ERR_INVALID_ARG = -1
DG_ERR_CUDA = -2
DG_ERR_NO_CONVERGENCE = -3
DG_ERR_NONPHYSICAL = -4
DG_ERR_TIMEOUT = -5
DG_ERR_OOM = -6
DG_ERR_UNSUPPORTED = -7
DG_STATUS_NONPHYSICAL = 1
DG_STATUS_NO_CONVERGENCE = 2
DG_STATUS_TIMEOUT = 4
DG_BC_SLIP_WALL, DG_BC_NOSLIP_WALL, DG_BC_INFLOW, DG_BC_OUTFLOW = 1, 2, 3, 4
DG_MAX_ORDER = 4
DG_MAX_SPECIES = 8
DG_MAX_OVERINT_POINTS = 12
DG_OVERINT_DEFAULT = -1
DG_GEO_STRIDE = 26
DG_GAS_PERFECT = 0
DG_GAS_NASA7 = 1
DG_PREC_FP64 = 0
DG_PREC_MIXED = 1
DG_TSEED_INPUT = 0
DG_TSEED_CONST = 1
DG_TSEED_MLP = 2
DG_MLP_PARAMS = 4801
DG_MESH_HOST_ONLY = 1
DG_BATCH_AUTOTUNE = 1
DG_STATIC_SCRATCH_NODES = 1 << 19
DG_KERNEL_VISCOUS = 0
DG_KERNEL_RHS = 1
DG_KERNEL_TEMPERATURE = 2
DG_KERNEL_PRIMS = 3
DG_NUM_KERNELS = 5
KERNEL_NAMES = ('viscous', 'rhs', 'temperature', 'prims', 'av')

c_int32, c_int64, c_uint32, c_double, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double, \
    ctypes.c_void_p


class dg_mesh_desc(ctypes.Structure):
    _fields_ = [("K", c_int32), ("N", c_int32), ("ref_nodes", c_void_p), ("vertices", c_void_p),
                ("period", c_double * 3), ("flags", c_int32), ("face_bc", c_void_p),
                ("EToV", c_void_p), ("EToE", c_void_p), ("EToF", c_void_p), ("vmapP", c_void_p),
                ("Dr", c_void_p), ("Ds", c_void_p), ("Dt", c_void_p), ("LIFT", c_void_p), ("Fmask", c_void_p),
                ("geo", c_void_p)]


class dg_av_params(ctypes.Structure):
    _fields_ = [("eps0", c_double), ("s0", c_double), ("kappa", c_double)]


class dg_gas_desc(ctypes.Structure):
    _fields_ = [("model", c_int32), ("gamma", c_double), ("R", c_double), ("mu", c_double), ("Pr", c_double),
                ("nspecies", c_int32), ("W", c_void_p), ("nasa7", c_void_p), ("R_universal", c_double),
                ("newton_tol", c_double), ("newton_max_it", c_int32), ("Sc", c_double)]


class dg_mesh_tables(ctypes.Structure):
    _fields_ = [("K", c_int32), ("N", c_int32), ("ops_dev", c_void_p), ("fmask_dev", c_void_p),
                ("geo_dev", c_void_p), ("vmapP_dev", c_void_p)]


class dg_mlp_norm(ctypes.Structure):
    _fields_ = [("e_mean", c_double), ("e_scale", c_double), ("T_mean", c_double), ("T_scale", c_double),
                ("T_min", c_double), ("T_max", c_double)]


class dg_mlp_train_opts(ctypes.Structure):
    _fields_ = [("epochs", c_int32), ("batch", c_int32), ("lr", ctypes.c_float), ("lr_decay", ctypes.c_float)]


class dg_batch_case(ctypes.Structure):
    _fields_ = [("mesh", c_void_p), ("gas", c_void_p), ("dt", c_double), ("q_dev", c_void_p)]


class dg_opts(ctypes.Structure):
    _fields_ = [("precision", c_int32), ("t_seed", c_int32), ("t_const", c_double), ("viscous_given", c_int32),
                ("wait_polls", c_int32), ("elem_range", c_int32), ("elem_begin", c_int32),
                ("elem_end", c_int32), ("prims_given", c_int32), ("reserved", c_int32 * 2)]


# name -> (restype, argtypes); every entry point declared in include/dg.h
class dg_hex_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("L", ctypes.c_double * 3), ("N", ctypes.c_int32),
                ("nodes1d", ctypes.c_void_p), ("bc", ctypes.c_int32 * 6)]


SIGNATURES = {
    "dg_mesh_upload": (c_int32, [ctypes.POINTER(dg_mesh_desc), ctypes.POINTER(c_void_p)]),
    "dg_mesh_free": (c_int32, [c_void_p]),
    "dg_mesh_info": (c_int32, [c_void_p, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32),
                               ctypes.POINTER(c_int32), ctypes.POINTER(c_int32)]),
    "dg_mesh_operators": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dg_mesh_connectivity": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "dg_mesh_face_pairs": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "dg_mesh_set_inflow": (c_int32, [c_void_p, c_void_p, c_int32]),
    "dg_mesh_set_av": (c_int32, [c_void_p, c_void_p]),
    "dg_mesh_set_overint": (c_int32, [c_void_p, c_int32]),
    "dg_tet_quadrature": (c_int32, [c_int32, c_void_p, c_void_p]),
    "dg_gather_elements": (c_int32, [c_void_p, c_int32, ctypes.c_int64, c_int32, c_void_p, c_int32, c_void_p,
                                     c_void_p]),
    "dg_scatter_elements": (c_int32, [c_void_p, c_int32, ctypes.c_int64, c_int32, c_void_p, c_int32, c_void_p,
                                      c_void_p]),
    "dg_viscous_flux": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "dg_viscous_flux_range": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p]),
    "dg_primitives": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p]),
    "dg_integrals": (c_int32, [c_void_p, c_void_p, c_int32, ctypes.c_int64, c_void_p, c_void_p]),
    "dg_max_rate": (c_int32, [c_void_p, c_void_p, c_void_p, ctypes.c_int64, c_void_p, c_void_p]),
    "dg_mesh_viscous_buffer": (c_int32, [c_void_p, ctypes.POINTER(c_void_p)]),
    "dg_av_viscosity": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "dg_mesh_status": (c_int32, [c_void_p, ctypes.POINTER(c_uint32), c_int32]),
    "dg_mesh_set_timing": (c_int32, [c_void_p, c_int32]),
    "dg_mesh_kernel_times": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32]),
    "dg_gas_create": (c_int32, [ctypes.POINTER(dg_gas_desc), ctypes.POINTER(c_void_p)]),
    "dg_gas_free": (c_int32, [c_void_p]),
    "dg_gas_status": (c_int32, [c_void_p, ctypes.POINTER(c_uint32), c_int32]),
    "dg_rhs": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, ctypes.POINTER(dg_opts), c_void_p]),
    "dg_rk_stage": (c_int32, [c_void_p, c_void_p, c_int32, c_double, c_void_p, c_void_p, c_void_p, c_void_p,
                              ctypes.POINTER(dg_opts), c_void_p]),
    "dg_lsrk4_coefficients": (c_int32, [c_void_p, c_void_p]),
    "dg_temperature": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, ctypes.POINTER(dg_opts),
                                 c_void_p]),
    "dg_mixture_energy": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dg_mlp_set": (c_int32, [c_void_p, c_void_p, ctypes.POINTER(dg_mlp_norm)]),
    "dg_mlp_get": (c_int32, [c_void_p, c_void_p, ctypes.POINTER(dg_mlp_norm)]),
    "dg_mlp_loss_grad": (c_int32, [c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dg_fp64_fma_rate": (c_int32, [c_void_p]),
    "dg_mlp_adam_step": (c_int32, [c_int32, ctypes.c_float, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dg_mlp_train": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p,
                               ctypes.POINTER(dg_mlp_train_opts), c_void_p]),
    "dg_mlp_guess": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p]),
    "dg_batch_create": (c_int32, [ctypes.POINTER(dg_batch_case), c_int32, c_int32, ctypes.POINTER(c_void_p)]),
    "dg_batch_step": (c_int32, [c_void_p, c_int32, c_void_p]),
    "dg_batch_tiles": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "dg_batch_status": (c_int32, [c_void_p, ctypes.POINTER(c_uint32), c_int32]),
    "dg_batch_free": (c_int32, [c_void_p]),
    "dg_rk_stage_noalloc": (c_int32, [ctypes.POINTER(dg_mesh_tables), ctypes.POINTER(dg_gas_desc), c_int32,
                                      c_double, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dg_hex_mesh_create": (ctypes.c_int, [ctypes.POINTER(dg_hex_desc), ctypes.POINTER(ctypes.c_void_p)]),
    "dg_hex_mesh_free": (ctypes.c_int, [ctypes.c_void_p]),
    "dg_hex_operators": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "dg_hex_rhs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "dg_hex_rk_stage": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_double,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "dg_hex_advection_rhs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p]),
    "dg_hex_advection_rk_stage": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_double,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "dg_hex_set_inflow": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "dg_hex_set_av": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "dg_hex_set_overintegration": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "dg_hex_av_viscosity": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "dg_hex_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32), ctypes.c_int]),
    "dg_round_to_float": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "dg_widen_to_double": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "dg_split_to_float_pair": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                              ctypes.c_void_p]),
    "dg_last_error": (ctypes.c_char_p, []),
}


class DGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libdg error {code}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libdg.so (once) and declare its signatures; raises ImportError if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code: int) -> None:
    if code != DG_OK:
        msg = load().dg_last_error()
        raise DGError(code, msg.decode() if msg else "")
