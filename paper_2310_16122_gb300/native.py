"""ctypes binding of libcrk's C ABI (include/crk.h): the same names, argument marshalling only.

Every compute step runs in the CUDA library.  Loading fails loudly when
libcrk.so has not been built (``python -c "import __graft_entry__ as g;
g.build()"`` builds it); there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libcrk.so")

CRK_OK = 0
CRK_EINVAL = -1
CRK_ENOMEM = -2
CRK_ECUDA = -3
CRK_EBOX = -4
CRK_ESTATE = -5
CRK_ETIMEOUT = -6
CRK_ETOOLARGE = -7
NOALLOC_MAX_PARTICLES = 1 << 21
# bits of the leaves' status word (crk_leaves_status)
LEAVES_STATUS = {1: "bad position", 2: "bad h", 4: "gas count", 8: "leaf size", 16: "h_max", 32: "candidates",
                 64: "image capacity", 128: "group capacity", 256: "list capacity", 512: "internal"}
KERNELS = {"geometry": 0, "corrections": 1, "hydro": 2, "gravity": 3, "gravity_adjoint": 4, "geometry_adjoint": 5,
           "extras": 6, "accel": 7, "energy": 8}
N_KERNELS = 9
VARIANT_LISTS = 0
VARIANT_TILES = 1
VARIANT_TILES16 = 2
VARIANT_TILES8 = 3
VARIANT_RING16 = 4
VARIANT_HALFWARP_SHFL = 5
VARIANT_HALFWARP_SMEM = 6
VARIANT_HALFWARP_LOAD = 7
VARIANT_SPLIT8 = 8
N_VARIANTS = 9
TUNE_COLS = N_VARIANTS + 7  # per kernel: variant timings, launch mode off/on, depth 32/64/96, warps 4/2
STATUS_NAMES = {0: "CRK_OK", -1: "CRK_EINVAL", -2: "CRK_ENOMEM", -3: "CRK_ECUDA", -4: "CRK_EBOX",
                -5: "CRK_ESTATE", -6: "CRK_ETIMEOUT", -7: "CRK_ETOOLARGE"}


class CrkError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class crk_particles(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("species", ctypes.c_void_p), ("n", ctypes.c_int64), ("box", ctypes.c_float)]


class crk_leaf_params(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("cells_per_side", ctypes.c_int), ("max_leaf", ctypes.c_int),
                ("r_cut_grav", ctypes.c_float)]


class crk_grav_params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_float), ("r_cut", ctypes.c_float), ("poly", ctypes.c_float * 6)]


class crk_hydro_params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_float), ("alpha", ctypes.c_float), ("beta", ctypes.c_float),
                ("eta2", ctypes.c_float)]


class crk_batch(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("species", ctypes.c_void_p), ("n", ctypes.c_int64), ("nbox", ctypes.c_int),
                ("box_start", ctypes.POINTER(ctypes.c_int64)), ("box_side", ctypes.POINTER(ctypes.c_float))]


class crk_advance_params(ctypes.Structure):
    _fields_ = [("cfl", ctypes.c_float), ("dt_max", ctypes.c_float), ("dt_fixed", ctypes.c_float),
                ("sig_beta", ctypes.c_float), ("limited", ctypes.c_int), ("gravity", ctypes.c_int)]


class crk_chain_adjoint_io(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p) for name in (
        "m", "v3", "u", "dvbar3", "dubar", "dvdt3", "dudt", "xbar3", "mbar", "vbar3", "ubar", "n_singular")]


class crk_step_io(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p) for name in (
        "m", "v3", "u", "V", "rho", "A", "B", "gradA", "gradB", "dvdt3", "dudt", "conservation", "a3", "abar3",
        "gx3_grav", "gm_grav", "rhobar", "Vbar", "gx3_geom", "gm_geom", "n_singular", "pair_count")] + [
        ("extras", ctypes.c_int), ("rho_r", ctypes.c_void_p), ("dvdx", ctypes.c_void_p),
        ("swept_count", ctypes.c_void_p)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64

# name -> argument types (all return int unless listed in _VOID / _STR)
SIGNATURES = {
    "crk_create": [ctypes.POINTER(_P), _I, _P],
    "crk_destroy": [_P],
    "crk_set_stream": [_P, _P],
    "crk_last_error": [_P],
    "crk_version": [],
    "crk_launch_count": [_P, ctypes.POINTER(_I64)],
    "crk_set_trace": [_P, _I],
    "crk_set_variant": [_P, _I, _I],
    "crk_set_persistent": [_P, _I],
    "crk_set_launch": [_P, _I, _I, _I, _I],
    "crk_get_launch": [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "crk_get_variant": [_P, _I, ctypes.POINTER(_I)],
    "crk_build_leaves": [_P, ctypes.POINTER(crk_particles), _P, ctypes.POINTER(crk_leaf_params), ctypes.POINTER(_P)],
    "crk_build_leaves_batch": [_P, ctypes.POINTER(crk_batch), _P, ctypes.POINTER(crk_leaf_params),
                               ctypes.POINTER(_P)],
    "crk_leaves_info": [_P, ctypes.POINTER(_I64)],
    "crk_leaves_export": [_P, _P, _P, _P, _P, _P, _P, _P],
    "crk_leaves_free": [_P, _P],
    "crk_geometry": [_P, _P, _P, _P, _P, _P],
    "crk_corrections": [_P, _P, _P, _P, _P, _P, _P, _P],
    "crk_hydro": [_P, _P, ctypes.POINTER(crk_hydro_params)] + [_P] * 13,
    "crk_extras": [_P] * 12,
    "crk_hydro_limited": [_P, _P, ctypes.POINTER(crk_hydro_params)] + [_P] * 14,
    "crk_hydro_accel": [_P, _P, ctypes.POINTER(crk_hydro_params)] + [_P] * 10 + [ctypes.c_float] + [_P] * 4,
    "crk_hydro_energy": [_P, _P, ctypes.POINTER(crk_hydro_params)] + [_P] * 14,
    "crk_timestep": [_P, _P, ctypes.c_float, ctypes.c_float, _P],
    "crk_corrections_adjoint": [_P] * 10,
    "crk_hydro_chain_adjoint": [_P, _P, ctypes.POINTER(crk_hydro_params), ctypes.POINTER(crk_chain_adjoint_io)],
    "crk_hydro_adjoint": [_P, _P, ctypes.POINTER(crk_hydro_params)] + [_P] * 21,
    "crk_advance": [_P, _I64, ctypes.c_float] + [_P] * 8 + [ctypes.POINTER(crk_leaf_params),
                                                           ctypes.POINTER(crk_hydro_params),
                                                           ctypes.POINTER(crk_grav_params),
                                                           ctypes.POINTER(crk_advance_params), _P, _P, _P],
    "grav_short": [_P, _P, ctypes.POINTER(crk_grav_params), _P, _P, _P],
    "grav_short_adjoint": [_P, _P, ctypes.POINTER(crk_grav_params), _P, _P, _P, _P],
    "crk_geometry_adjoint": [_P, _P, _P, _P, _P, _P, _P, _P],
    "grav_short_noalloc": [_P, _P, ctypes.POINTER(crk_grav_params), _P, _P],
    "crk_step": [_P, _P, ctypes.POINTER(crk_grav_params), ctypes.POINTER(crk_hydro_params),
                 ctypes.POINTER(crk_step_io)],
    "crk_step_graph_create": [_P, _P, ctypes.POINTER(crk_grav_params), ctypes.POINTER(crk_hydro_params),
                              ctypes.POINTER(crk_step_io), ctypes.POINTER(_P)],
    "crk_graph_launch": [_P],
    "crk_rebuild_step_graph_create": [_P, _P, ctypes.POINTER(crk_batch), _P, ctypes.POINTER(crk_grav_params),
                                      ctypes.POINTER(crk_hydro_params), ctypes.POINTER(crk_step_io), ctypes.POINTER(_P)],
    "crk_leaves_rebuild": [_P, _P, ctypes.POINTER(crk_particles), _P],
    "crk_leaves_rebuild_batch": [_P, _P, ctypes.POINTER(crk_batch), _P],
    "crk_leaves_status": [_P, _P, ctypes.POINTER(_I)],
    "crk_step_profile": [_P, _I],
    "crk_step_profile_read": [_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_I)],
    "crk_graph_destroy": [_P],
    "crk_tune": [_P, _P, ctypes.POINTER(crk_grav_params), ctypes.POINTER(crk_hydro_params),
                 ctypes.POINTER(crk_step_io), _I, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_I)],
}
_VOID = {"crk_destroy", "crk_leaves_free", "crk_graph_destroy"}
_STR = {"crk_last_error", "crk_version"}

_lib = None


def lib() -> ctypes.CDLL:
    """Load libcrk.so (once).  Raises if the library has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libcrk.so not found at {LIB_PATH}: build it with paper_2310_16122_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = None if name in _VOID else (ctypes.c_char_p if name in _STR else ctypes.c_int)
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(SIGNATURES)


def check(status: int, ctx=None) -> None:
    if status != CRK_OK:
        msg = lib().crk_last_error(ctx).decode() if ctx else ""
        raise CrkError(status, msg)
