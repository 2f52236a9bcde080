"""ctypes binding of libirk.so (argument marshalling only).

Every computation runs in the CUDA library; this module converts Python
arguments (torch tensors on the GPU or the CPU, NumPy arrays) into the plain
pointers and sizes of the C ABI declared in include/irk.h, and turns non-zero
status codes into exceptions.  If the shared library is missing the import of
this module fails loudly: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libirk.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "irk.h")

IRK_OK, IRK_EINVAL, IRK_ENOMEM, IRK_ECUDA, IRK_ENOCONV, IRK_ENONFINITE = 0, -1, -2, -3, -4, -5
PC = {"diag": 0, "lower": 1, "upper": 2, "rana_ld": 3, "monolithic": 4}
PREC = {"fp64": 0, "fp32": 1, "bf16": 2}
ORTH = {"cgs2": 0, "dgks": 1, "cgs": 2}
SOLVER = {"fgmres": 0, "dirk_cg": 1}
SPLIT = {"ai": 0, "ia": 1}
MAX_STAGES = 4
_ERRNAMES = {-1: "IRK_EINVAL", -2: "IRK_ENOMEM", -3: "IRK_ECUDA", -4: "IRK_ENOCONV", -5: "IRK_ENONFINITE"}


class IRKError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class irk_mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_cells", C.c_int), ("levels", C.c_int), ("kappa", C.POINTER(C.c_double))]


class irk_tableau(C.Structure):
    _fields_ = [("s", C.c_int), ("A", C.POINTER(C.c_double)), ("b", C.POINTER(C.c_double)),
                ("c", C.POINTER(C.c_double))]


class irk_options(C.Structure):
    _fields_ = [("precond", C.c_int), ("vcycle_prec", C.c_int), ("nu_pre", C.c_int), ("nu_post", C.c_int),
                ("omega", C.c_double), ("rtol", C.c_double), ("restart", C.c_int), ("maxit", C.c_int),
                ("orth", C.c_int), ("solver", C.c_int), ("splitting", C.c_int), ("warm_start", C.c_int)]


class irk_stats(C.Structure):
    _fields_ = [("fgmres_its", C.c_int), ("vcycles", C.c_int), ("rel_resid", C.c_double), ("converged", C.c_int)]

    def as_dict(self) -> dict:
        return {"fgmres_its": self.fgmres_its, "vcycles": self.vcycles, "rel_resid": self.rel_resid,
                "converged": bool(self.converged)}


K_CLASSES = ["stage_apply", "jacobi", "residual", "restrict", "prolong", "coarse", "multidot", "axpy",
             "block_rhs", "other", "mg_coarse", "mg_tail"]
_NK = len(K_CLASSES)


class irk_perf(C.Structure):
    _fields_ = [("launches", C.c_longlong), ("class_launches", C.c_longlong * _NK), ("class_bytes", C.c_double * _NK),
                ("class_flops", C.c_double * _NK), ("timed_launches", C.c_longlong * _NK),
                ("timed_ms", C.c_double * _NK), ("timed_bytes", C.c_double * _NK), ("timed_flops", C.c_double * _NK)]

    def as_dict(self) -> dict:
        out = {"launches": int(self.launches), "classes": {}}
        for i, name in enumerate(K_CLASSES):
            out["classes"][name] = {
                "launches": int(self.class_launches[i]), "bytes": self.class_bytes[i], "flops": self.class_flops[i],
                "timed_launches": int(self.timed_launches[i]), "timed_ms": self.timed_ms[i],
                "timed_bytes": self.timed_bytes[i], "timed_flops": self.timed_flops[i]}
        return out


_P = C.c_void_p
_SIGNATURES = {
    "irk_default_options": (None, [C.POINTER(irk_options)]),
    "irk_create": (C.c_int, [C.POINTER(_P), C.POINTER(irk_mesh), C.POINTER(irk_tableau), C.c_double,
                             C.POINTER(irk_options), _P]),
    "irk_destroy": (C.c_int, [_P]),
    "irk_set_kappa": (C.c_int, [_P, _P]),
    "irk_reset_initial_guess": (C.c_int, [_P]),
    "irk_step": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, C.POINTER(irk_stats)]),
    "irk_step_dirichlet": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, C.POINTER(irk_stats)]),
    "irk_solve": (C.c_int, [_P, _P, _P, C.POINTER(irk_stats)]),
    "irk_apply_operator": (C.c_int, [_P, _P, _P, C.c_int]),
    "irk_apply_mass": (C.c_int, [_P, _P, _P]),
    "irk_apply_preconditioner": (C.c_int, [_P, _P, _P, C.c_int]),
    "irk_apply_preconditioner_noalloc": (C.c_int, [_P, _P, _P, C.c_int]),
    "irk_step_adjoint": (C.c_int, [_P, _P, _P, _P, _P, _P, C.POINTER(irk_stats)]),
    "irk_perf_select": (C.c_int, [_P, C.c_uint]),
    "irk_perf_read": (C.c_int, [_P, C.POINTER(irk_perf)]),
    "irk_last_error": (C.c_char_p, []),
}


def header_symbols(path: str = HEADER) -> list[str]:
    """Names of the functions declared in include/irk.h."""
    text = open(path).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(irk_\w+)\s*\(", text, re.M)))


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libirk.so not found at {path}: run paper_2403_08084_gb300/build.py (no fallback exists)")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = load()


def check(code: int) -> int:
    if code != IRK_OK:
        raise IRKError(code, lib.irk_last_error().decode())
    return code


def ptr(x, dtype_size: int = 8, count: int | None = None):
    """Raw pointer of a contiguous float64 buffer (torch tensor, NumPy array) or None."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):  # torch.Tensor
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if x.element_size() != dtype_size:
            raise ValueError(f"expected {dtype_size}-byte elements, got {x.dtype}")
        if count is not None and x.numel() != count:
            raise ValueError(f"expected {count} elements, got {x.numel()}")
        return C.c_void_p(x.data_ptr())
    if hasattr(x, "ctypes"):  # numpy.ndarray
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if x.itemsize != dtype_size:
            raise ValueError(f"expected {dtype_size}-byte elements, got {x.dtype}")
        if count is not None and x.size != count:
            raise ValueError(f"expected {count} elements, got {x.size}")
        return C.c_void_p(x.ctypes.data)
    raise TypeError(f"unsupported buffer type {type(x)}")


def dbl_array(values) -> C.Array:
    vals = [float(v) for v in values]
    return (C.c_double * len(vals))(*vals)
