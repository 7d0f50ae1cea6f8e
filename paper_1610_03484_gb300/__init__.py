"""Python binding of librve (C ABI in include/rve.h): argument marshalling only.

Every step of the homogenisation runs inside librve's CUDA kernels; this
module converts numpy arrays to pointers and error codes to exceptions.  There
is no CPU fallback: if librve.so is missing or no GB300 is visible, calls fail
with ``RveError``.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# RVE_LIBRARY selects another build of the library (the checking build, librve_check.so)
LIB_PATH = os.environ.get("RVE_LIBRARY") or os.path.join(HERE, "librve.so")

RVE_OK = 0
ERRORS = {
    -1: "INVALID_ARGUMENT", -2: "BAD_MESH", -3: "NOT_SPD", -4: "NOT_CONVERGED", -5: "NUMERIC",
    -6: "CUDA", -7: "NO_DEVICE", -8: "OUT_OF_MEMORY", -9: "STATE", -10: "TIMEOUT", -11: "BOUNDS",
}
BC_DIRICHLET, BC_PERIODIC, BC_NEUMANN = 0, 1, 2
PREC_FP64, PREC_MIXED = 0, 1
MODE_PCG = 0
KERNEL_AUTO, KERNEL_CUDA_CORE, KERNEL_TENSOR = 0, 1, 2


class RveError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        super().__init__(f"{where}: RVE_ERR_{ERRORS.get(code, code)} ({detail})")


class Options(C.Structure):
    _fields_ = [("device", C.c_int), ("precision", C.c_int), ("rtol", C.c_double),
                ("max_iter", C.c_int), ("inner_rtol", C.c_double), ("max_refine", C.c_int),
                ("check_every", C.c_int), ("batch", C.c_int), ("stream", C.c_void_p), ("profile", C.c_int),
                ("warm_start", C.c_int), ("transport_once", C.c_int), ("operator_kernel", C.c_int),
                ("deterministic", C.c_int)]


class MatrixProps(C.Structure):
    _fields_ = [("E", C.c_double), ("nu", C.c_double), ("k", C.c_double), ("d", C.c_double)]


class YarnProps(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("E1", "E2", "G12", "nu12", "nu23", "k1", "k2", "d1", "d2")]


class Degradation(C.Structure):
    _fields_ = [("beta", C.c_double), ("Tg_C", C.c_double), ("c_sat_wt", C.c_double),
                ("apply_to_yarn", C.c_int)]


class MacroStats(C.Structure):
    _fields_ = [("iterations_T", C.c_int32), ("iterations_c", C.c_int32), ("converged", C.c_int32),
                ("gauss_points_unencodable", C.c_int32), ("rel_residual_T", C.c_double),
                ("rel_residual_c", C.c_double), ("seconds", C.c_double), ("handover_max_err", C.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class MacroMechStats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("rel_residual", C.c_double),
                ("seconds", C.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class MeshStats(C.Structure):
    _fields_ = [("n_vertices", C.c_int64), ("n_edges", C.c_int64), ("n_faces", C.c_int64),
                ("n_tets", C.c_int64), ("n_scalar_dofs", C.c_int64), ("n_constrained", C.c_int64),
                ("p", C.c_int32), ("bc", C.c_int32), ("volume", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("iterations_mech", C.c_int32), ("iterations_scalar", C.c_int32),
                ("refine_sweeps", C.c_int32), ("converged", C.c_int32),
                ("rel_residual_mech", C.c_double), ("rel_residual_scalar", C.c_double),
                ("hill_mandel_mech", C.c_double), ("hill_mandel_scalar", C.c_double),
                ("seconds", C.c_double), ("kernel_launches", C.c_int64), ("op_ms", C.c_double),
                ("op_launches", C.c_int64), ("op_bytes", C.c_double), ("op_flops", C.c_double),
                ("update_ms", C.c_double), ("update_bytes", C.c_double), ("pupdate_ms", C.c_double),
                ("pupdate_bytes", C.c_double), ("finalize_ms", C.c_double),
                ("residual_ms", C.c_double), ("residual_launches", C.c_int64),
                ("op_active_frac", C.c_double),
                ("op_class_ms", C.c_double * 6), ("op_class_launches", C.c_int64 * 6),
                ("op_class_bytes", C.c_double * 6), ("op_class_flops", C.c_double * 6),
                ("op_class_active_frac", C.c_double * 6),
                ("graph_host_ms", C.c_double), ("graphs", C.c_int64)]

    def as_dict(self):
        return {n: (list(v) if isinstance(v, C.Array) else v)
                for n, v in ((n, getattr(self, n)) for n, _ in self._fields_)}


_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "rve_strerror": (C.c_char_p, [C.c_int]),
    "rve_last_error": (C.c_char_p, []),
    "rve_default_options": (None, [C.POINTER(Options)]),
    "rve_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Options)]),
    "rve_destroy": (C.c_int, [C.c_void_p]),
    "rve_set_options": (C.c_int, [C.c_void_p, C.POINTER(Options)]),
    "rve_get_options": (C.c_int, [C.c_void_p, C.POINTER(Options)]),
    "rve_mesh_load": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]),
    "rve_mesh_free": (C.c_int, [C.c_void_p, C.c_void_p]),
    "rve_mesh_info": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(MeshStats)]),
    "rve_set_materials": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(MatrixProps), C.POINTER(YarnProps),
                                    C.c_double, C.c_double, C.c_double, C.POINTER(Degradation)]),
    "rve_set_bc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "rve_homogenise": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.POINTER(Stats)]),
    "rve_macro_create": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                   C.POINTER(C.c_void_p)]),
    "rve_macro_free": (C.c_int, [C.c_void_p, C.c_void_p]),
    "rve_macro_set_transport": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]),
    "rve_macro_set_face": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_double]),
    "rve_macro_reset": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_double]),
    "rve_macro_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_double, C.c_int,
                                 C.POINTER(MacroStats)]),
    "rve_macro_gauss_dev": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                      C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)]),
    "rve_macro_get": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p]),
    "rve_macro_set_held": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rve_macro_solve_steady": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.POINTER(MacroStats)]),
    "rve_macro_gradients": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "rve_macro_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rve_macro_mech_set_bc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rve_macro_mech_set_u": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "rve_macro_mech_set_traction": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "rve_macro_mech_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_int,
                                       C.POINTER(MacroMechStats)]),
    "rve_macro_mech_get": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rve_fibre_directions": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                       C.c_int, C.c_void_p, C.c_double, C.c_void_p]),
    "macro_update_gauss_points_w": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int64, C.c_void_p,
                                              C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_int, C.POINTER(Stats)]),
    "macro_update_gauss_points_w_dev": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int64, C.c_void_p,
                                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                                  C.c_int, C.POINTER(Stats)]),
    "rve_apply_operator_mixed": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_void_p]),
    "rve_homogenise_weak": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.POINTER(Stats)]),
    "rve_partition_blocks": (C.c_int, [C.c_int64, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "rve_autotune_schedule": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_int32),
                                        C.POINTER(C.c_int32), C.c_void_p]),
    "rve_surrogate_set_fused": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "rve_surrogate_predict_dev": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.c_void_p]),
    "rve_autotune_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_int, C.POINTER(C.c_int32), C.c_void_p]),
    "macro_update_gauss_points": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int64, C.c_void_p,
                                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.c_void_p, C.c_int, C.POINTER(Stats)]),
    "macro_update_gauss_points_dev": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int64, C.c_void_p,
                                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                                C.POINTER(Stats)]),
    "rve_degradation_factor": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.POINTER(Degradation), C.c_void_p]),
    "rve_mesh_get_tensors": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rve_apply_operator": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "rve_mesh_get_dofmap": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rve_mesh_get_colouring": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]),
    "rve_debug_bounds": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_int32), C.c_int]),
    "rve_debug_set_node_bound": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "rve_debug_galerkin_solve": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]),
    "rve_operator_energy_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                              C.c_void_p]),
    "rve_surrogate_create": (C.c_int, [C.c_void_p, C.c_int, C.c_uint64, C.POINTER(C.c_void_p)]),
    "rve_surrogate_free": (C.c_int, [C.c_void_p, C.c_void_p]),
    "rve_gauss_point_features": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_void_p]),
    "rve_surrogate_train": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_uint64, C.c_void_p]),
    "rve_surrogate_gradients": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.POINTER(C.c_double)]),
    "rve_surrogate_predict": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p]),
    "rve_surrogate_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)]),
    "rve_surrogate_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]),
    "macro_update_gauss_points_surrogate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                                                      C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                                      C.POINTER(Stats)]),
}


def load_library(path: str = LIB_PATH):
    """Load librve.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RveError(-6, "load_library", f"{path} not built; run __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


def partition_blocks(cost, n_ranks: int):
    """Contiguous cost-balanced blocks (rve_partition_blocks): (offsets [n+1], imbalance)."""
    lib = load_library()
    c = np.ascontiguousarray(cost, np.float64)
    off = np.zeros(int(n_ranks) + 1, np.int64)
    imb = C.c_double()
    _check(lib.rve_partition_blocks(len(c), _ptr(c), int(n_ranks), _ptr(off), C.byref(imb)), "rve_partition_blocks")
    return off, imb.value


def _check(rc: int, where: str, allow=()):
    if rc != RVE_OK and rc not in allow:
        detail = _lib.rve_last_error().decode(errors="replace") if _lib else ""
        raise RveError(rc, where, detail)
    return rc


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def galerkin_solve(G, g, rel: float = 1e-12) -> np.ndarray:
    """c = G^+ g as the energy-optimal warm start solves it (rve_debug_galerkin_solve);
    host only."""
    G = np.ascontiguousarray(G, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    n = g.shape[0]
    if G.shape != (n, n):
        raise ValueError("G must be n x n with n = len(g)")
    c = np.zeros(n)
    _check(load_library().rve_debug_galerkin_solve(n, _ptr(G), _ptr(g), float(rel), _ptr(c)),
           "rve_debug_galerkin_solve")
    return c


def default_options() -> Options:
    lib = load_library()
    o = Options()
    lib.rve_default_options(C.byref(o))
    return o


@dataclass
class Result:
    C: np.ndarray
    K: np.ndarray
    D: np.ndarray
    stats: dict
    code: int


class Context:
    """One librve context (device + stream).  Use as a context manager."""

    def __init__(self, precision=PREC_FP64, rtol=1e-10, max_iter=20000, inner_rtol=1e-6,
                 max_refine=4, check_every=16, batch=0, stream=None, device=0, profile=False,
                 warm_start=4, transport_once=False, operator_kernel=KERNEL_AUTO, deterministic=False):
        lib = load_library()
        o = default_options()
        o.device, o.precision, o.rtol, o.max_iter = device, precision, rtol, max_iter
        o.inner_rtol, o.max_refine, o.check_every, o.batch = inner_rtol, max_refine, check_every, batch
        o.stream = stream
        o.profile = int(profile)
        o.warm_start = (4 if warm_start else 0) if isinstance(warm_start, bool) else int(warm_start)
        o.transport_once = int(transport_once)
        o.operator_kernel = int(operator_kernel)
        o.deterministic = int(deterministic)
        h = C.c_void_p()
        _check(lib.rve_create(C.byref(h), C.byref(o)), "rve_create")
        self.h = h
        self.lib = lib

    def get_options(self) -> dict:
        o = Options()
        _check(self.lib.rve_get_options(self.h, C.byref(o)), "rve_get_options")
        return {n: getattr(o, n) for n, _ in Options._fields_ if n not in ("device", "stream")}

    def set_options(self, **kw):
        o = Options()
        _check(self.lib.rve_get_options(self.h, C.byref(o)), "rve_get_options")
        for k, v in kw.items():
            setattr(o, k, v)
        _check(self.lib.rve_set_options(self.h, C.byref(o)), "rve_set_options")

    def debug_bounds(self, reset: bool = False) -> dict:
        """Counters of the checking build (checking_build = 0 in a release build)."""
        cb, n, fe, fc = C.c_int32(), C.c_int64(), C.c_int64(), C.c_int32()
        _check(self.lib.rve_debug_bounds(self.h, C.byref(cb), C.byref(n), C.byref(fe), C.byref(fc), int(reset)),
               "rve_debug_bounds")
        return {"checking_build": cb.value, "violations": n.value, "first_element": fe.value,
                "first_column": fc.value}

    def close(self):
        if self.h:
            self.lib.rve_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------------------- mesh
    def mesh_load(self, xyz, tets, p, phase=None, fibre_dir=None) -> "Mesh":
        xyz = np.ascontiguousarray(xyz, np.float64)
        tets = np.ascontiguousarray(tets, np.int32)
        ph = None if phase is None else np.ascontiguousarray(phase, np.uint8)
        fd = None if fibre_dir is None else np.ascontiguousarray(fibre_dir, np.float64)
        h = C.c_void_p()
        _check(self.lib.rve_mesh_load(self.h, _ptr(xyz), len(xyz), _ptr(tets), len(tets), _ptr(ph), _ptr(fd),
                                      int(p), C.byref(h)), "rve_mesh_load")
        return Mesh(self, h, len(tets), int(p))

    def macro_load(self, xyz, tets) -> "Macro":
        xyz = np.ascontiguousarray(xyz, np.float64)
        tets = np.ascontiguousarray(tets, np.int32)
        h = C.c_void_p()
        _check(self.lib.rve_macro_create(self.h, _ptr(xyz), len(xyz), _ptr(tets), len(tets), C.byref(h)),
               "rve_macro_create")
        return Macro(self, h, len(xyz), len(tets))

    def fibre_directions(self, xyz, tets, yarn_of_tet, yarn_axis, dir_in, rtol=1e-12):
        """Yarn directions from potential flow along each yarn (Sec. 6); matrix
        tetrahedra keep dir_in."""
        xyz = np.ascontiguousarray(xyz, np.float64)
        tets = np.ascontiguousarray(tets, np.int32)
        yid = np.ascontiguousarray(yarn_of_tet, np.int32)
        ax = np.ascontiguousarray(yarn_axis, np.int32)
        d = np.array(dir_in, np.float64, copy=True, order="C")
        _check(self.lib.rve_fibre_directions(self.h, _ptr(xyz), len(xyz), _ptr(tets), len(tets), _ptr(yid), len(ax),
                                             _ptr(ax), float(rtol), _ptr(d)), "rve_fibre_directions")
        return d

    def degradation_factor(self, T_C, c_wt, t_h, beta=-0.001682, Tg_C=126.0, c_sat_wt=1.5):
        T = np.ascontiguousarray(T_C, np.float64)
        c = np.ascontiguousarray(c_wt, np.float64)
        t = np.ascontiguousarray(t_h, np.float64)
        out = np.zeros_like(T)
        dg = Degradation(beta, Tg_C, c_sat_wt, 0)
        _check(self.lib.rve_degradation_factor(self.h, len(T), _ptr(T), _ptr(c), _ptr(t), C.byref(dg),
                                               _ptr(out)), "rve_degradation_factor")
        return out

    def macro_update(self, meshes, T_C, c_wt, t_h, mesh_id, allow_not_converged=False):
        G = len(T_C)
        arr = (C.c_void_p * len(meshes))(*[m.h for m in meshes])
        T = np.ascontiguousarray(T_C, np.float64)
        c = np.ascontiguousarray(c_wt, np.float64)
        t = np.ascontiguousarray(t_h, np.float64)
        mid = np.ascontiguousarray(mesh_id, np.int32)
        Cc = np.zeros((G, 6, 6))
        Kk = np.zeros((G, 3, 3))
        Dd = np.zeros((G, 3, 3))
        st = np.zeros(G, np.int32)
        s = Stats()
        allow = (-4,) if allow_not_converged else ()
        rc = _check(self.lib.macro_update_gauss_points(self.h, arr, len(meshes), G, _ptr(T), _ptr(c), _ptr(t),
                                                       _ptr(mid), _ptr(Cc), _ptr(Kk), _ptr(Dd), _ptr(st),
                                                       MODE_PCG, C.byref(s)),
                    "macro_update_gauss_points", allow)
        return Cc, Kk, Dd, st, s.as_dict(), rc

    def macro_update_w(self, meshes, W, mesh_id, allow_not_converged=False):
        """Batched evaluation with the degradation factor 1 - omega given per point."""
        G = len(W)
        arr = (C.c_void_p * len(meshes))(*[m.h for m in meshes])
        w = np.ascontiguousarray(W, np.float64)
        mid = np.ascontiguousarray(mesh_id, np.int32)
        Cc, Kk, Dd = np.zeros((G, 6, 6)), np.zeros((G, 3, 3)), np.zeros((G, 3, 3))
        st = np.zeros(G, np.int32)
        s = Stats()
        allow = (-4,) if allow_not_converged else ()
        rc = _check(self.lib.macro_update_gauss_points_w(self.h, arr, len(meshes), G, _ptr(w), _ptr(mid), _ptr(Cc),
                                                         _ptr(Kk), _ptr(Dd), _ptr(st), MODE_PCG, C.byref(s)),
                    "macro_update_gauss_points_w", allow)
        return Cc, Kk, Dd, st, s.as_dict(), rc

    def macro_update_w_dev(self, meshes, W_dev, mesh_id, C_dev, K_dev, D_dev, status_dev):
        """Device-pointer form of macro_update_w (mesh_id is a host array)."""
        arr = (C.c_void_p * len(meshes))(*[m.h for m in meshes])
        mid = np.ascontiguousarray(mesh_id, np.int32)
        s = Stats()
        rc = _check(self.lib.macro_update_gauss_points_w_dev(self.h, arr, len(meshes), len(mid), C.c_void_p(W_dev),
                                                             _ptr(mid), C.c_void_p(C_dev), C.c_void_p(K_dev),
                                                             C.c_void_p(D_dev), C.c_void_p(status_dev), MODE_PCG,
                                                             C.byref(s)),
                    "macro_update_gauss_points_w_dev")
        return s.as_dict(), rc

    def features(self, mesh, T_C, c_wt, t_h):
        T = np.ascontiguousarray(T_C, np.float64)
        c = np.ascontiguousarray(c_wt, np.float64)
        t = np.ascontiguousarray(t_h, np.float64)
        f = np.zeros((len(T), 8))
        _check(self.lib.rve_gauss_point_features(self.h, mesh.h, len(T), _ptr(T), _ptr(c), _ptr(t), _ptr(f)),
               "rve_gauss_point_features")
        return f

    def macro_update_surrogate(self, meshes, surrogates, tau, T_C, c_wt, t_h, mesh_id):
        G = len(T_C)
        arr = (C.c_void_p * len(meshes))(*[m.h for m in meshes])
        sarr = (C.c_void_p * len(meshes))(*[(s.h if s is not None else None) for s in surrogates])
        T = np.ascontiguousarray(T_C, np.float64)
        c = np.ascontiguousarray(c_wt, np.float64)
        t = np.ascontiguousarray(t_h, np.float64)
        mid = np.ascontiguousarray(mesh_id, np.int32)
        Cc, Kk, Dd = np.zeros((G, 6, 6)), np.zeros((G, 3, 3)), np.zeros((G, 3, 3))
        st = np.zeros(G, np.int32)
        fb = np.zeros(G, np.uint8)
        s = Stats()
        rc = _check(self.lib.macro_update_gauss_points_surrogate(self.h, arr, sarr, len(meshes), float(tau), G,
                                                                 _ptr(T), _ptr(c), _ptr(t), _ptr(mid), _ptr(Cc),
                                                                 _ptr(Kk), _ptr(Dd), _ptr(st), _ptr(fb), C.byref(s)),
                    "macro_update_gauss_points_surrogate", (-4,))
        return Cc, Kk, Dd, st, fb, s.as_dict(), rc

    def macro_update_dev(self, meshes, T_dev, c_dev, t_dev, mesh_id_host, C_dev, K_dev, D_dev, status_dev):
        """Device-pointer variant: every *_dev argument is an integer device address."""
        G = len(mesh_id_host)
        arr = (C.c_void_p * len(meshes))(*[m.h for m in meshes])
        mid = np.ascontiguousarray(mesh_id_host, np.int32)
        s = Stats()
        rc = _check(self.lib.macro_update_gauss_points_dev(self.h, arr, len(meshes), G, C.c_void_p(T_dev),
                                                           C.c_void_p(c_dev), C.c_void_p(t_dev), _ptr(mid),
                                                           C.c_void_p(C_dev), C.c_void_p(K_dev),
                                                           C.c_void_p(D_dev), C.c_void_p(status_dev),
                                                           MODE_PCG, C.byref(s)),
                    "macro_update_gauss_points_dev", (-4,))
        return s.as_dict(), rc


class Surrogate:
    """Ensemble MLP surrogate (see include/rve.h); training and inference on the GPU."""

    N_OUT = 33

    def __init__(self, ctx: "Context", members=4, seed=0):
        h = C.c_void_p()
        _check(ctx.lib.rve_surrogate_create(ctx.h, int(members), int(seed), C.byref(h)), "rve_surrogate_create")
        self.ctx, self.h, self.members = ctx, h, members

    def free(self):
        if self.h:
            self.ctx.lib.rve_surrogate_free(self.ctx.h, self.h)
            self.h = None

    def __del__(self):
        try:
            if self.ctx.h:
                self.free()
        except Exception:
            pass

    def train(self, feat, Cc, Kk, Dd, epochs=100, batch=256, lr=1e-3, seed=0):
        feat = np.ascontiguousarray(feat, np.float64)
        Cc = np.ascontiguousarray(Cc, np.float64).reshape(-1, 36)
        Kk = np.ascontiguousarray(Kk, np.float64).reshape(-1, 9)
        Dd = np.ascontiguousarray(Dd, np.float64).reshape(-1, 9)
        hist = np.zeros(epochs)
        _check(self.ctx.lib.rve_surrogate_train(self.ctx.h, self.h, len(feat), _ptr(feat), _ptr(Cc), _ptr(Kk),
                                                _ptr(Dd), int(epochs), int(batch), float(lr), int(seed), _ptr(hist)),
               "rve_surrogate_train")
        return hist

    def gradients(self, member, feat, target_factors):
        feat = np.ascontiguousarray(feat, np.float64)
        tf = np.ascontiguousarray(target_factors, np.float32)
        n = len(feat)
        g = np.zeros(self.param_count(), np.float32)
        loss = C.c_double()
        _check(self.ctx.lib.rve_surrogate_gradients(self.ctx.h, self.h, int(member), n, _ptr(feat), _ptr(tf),
                                                    _ptr(g), C.byref(loss)), "rve_surrogate_gradients")
        return g, loss.value

    def predict(self, feat):
        feat = np.ascontiguousarray(feat, np.float64)
        n = len(feat)
        Cc, Kk, Dd, sp = np.zeros((n, 6, 6)), np.zeros((n, 3, 3)), np.zeros((n, 3, 3)), np.zeros(n)
        _check(self.ctx.lib.rve_surrogate_predict(self.ctx.h, self.h, n, _ptr(feat), _ptr(Cc), _ptr(Kk), _ptr(Dd),
                                                  _ptr(sp)), "rve_surrogate_predict")
        return Cc, Kk, Dd, sp

    def set_fused(self, fused: bool):
        """Inference path: the fused whole-network kernel (default) or one GEMM per layer."""
        _check(self.ctx.lib.rve_surrogate_set_fused(self.ctx.h, self.h, int(bool(fused))), "rve_surrogate_set_fused")

    def predict_dev(self, n: int, feat_dev: int, C_dev: int, K_dev: int, D_dev: int, spread_dev: int):
        """Device-pointer inference (integer device addresses), on the context's stream."""
        _check(self.ctx.lib.rve_surrogate_predict_dev(self.ctx.h, self.h, int(n), C.c_void_p(feat_dev),
                                                      C.c_void_p(C_dev), C.c_void_p(K_dev), C.c_void_p(D_dev),
                                                      C.c_void_p(spread_dev)), "rve_surrogate_predict_dev")

    def get_params(self) -> np.ndarray:
        n = C.c_int64()
        _check(self.ctx.lib.rve_surrogate_get_params(self.ctx.h, self.h, None, C.byref(n)), "rve_surrogate_get_params")
        buf = np.zeros(n.value, np.float32)
        _check(self.ctx.lib.rve_surrogate_get_params(self.ctx.h, self.h, _ptr(buf), C.byref(n)),
               "rve_surrogate_get_params")
        return buf

    def set_params(self, buf):
        buf = np.ascontiguousarray(buf, np.float32)
        _check(self.ctx.lib.rve_surrogate_set_params(self.ctx.h, self.h, _ptr(buf), len(buf)),
               "rve_surrogate_set_params")

    HEADER = 52

    def param_count(self):
        return (len(self.get_params()) - self.HEADER) // self.members


class Mesh:
    def __init__(self, ctx: Context, h, nt: int, p: int):
        self.ctx, self.h, self.nt, self.p = ctx, h, nt, p

    def free(self):
        if self.h:
            self.ctx.lib.rve_mesh_free(self.ctx.h, self.h)
            self.h = None

    def __del__(self):
        try:
            if self.ctx.h:
                self.free()
        except Exception:
            pass

    def info(self) -> dict:
        s = MeshStats()
        _check(self.ctx.lib.rve_mesh_info(self.ctx.h, self.h, C.byref(s)), "rve_mesh_info")
        return {n: getattr(s, n) for n, _ in s._fields_}

    def set_materials(self, matrix, yarn, T_C=20.0, c_wt=0.0, t_h=0.0, beta=-0.001682, Tg_C=126.0,
                      c_sat_wt=1.5, apply_to_yarn=False):
        mp = MatrixProps(matrix.E, matrix.nu, matrix.k, matrix.d)
        yp = YarnProps(yarn.E1, yarn.E2, yarn.G12, yarn.nu12, yarn.nu23, yarn.k1, yarn.k2, yarn.d1, yarn.d2)
        dg = Degradation(beta, Tg_C, c_sat_wt, int(apply_to_yarn))
        _check(self.ctx.lib.rve_set_materials(self.ctx.h, self.h, C.byref(mp), C.byref(yp), T_C, c_wt, t_h,
                                              C.byref(dg)), "rve_set_materials")

    def set_bc(self, bc: int):
        _check(self.ctx.lib.rve_set_bc(self.ctx.h, self.h, int(bc)), "rve_set_bc")

    def autotune_batch(self, T_C, c_wt, t_h, candidates=None):
        """Time candidate batch sizes on sample states of this mesh and keep the
        fastest for later batched calls; returns (best, {candidate: rate})."""
        T = np.ascontiguousarray(T_C, np.float64)
        cw = np.ascontiguousarray(c_wt, np.float64)
        th = np.ascontiguousarray(t_h, np.float64)
        cand = np.ascontiguousarray(candidates if candidates is not None else [8, 16, 32, 64, 128, 256],
                                    np.int32)
        rates = np.zeros(len(cand))
        best = C.c_int32(0)
        _check(self.ctx.lib.rve_autotune_batch(self.ctx.h, self.h, len(T), _ptr(T), _ptr(cw), _ptr(th),
                                                _ptr(cand), len(cand), C.byref(best), _ptr(rates)),
               "rve_autotune_batch")
        return int(best.value), {int(b): float(r) for b, r in zip(cand, rates)}

    def autotune_schedule(self, T_C, c_wt, t_h, batches, kernels=(KERNEL_CUDA_CORE, KERNEL_TENSOR)):
        """Time (operator kernel, batch size) pairs on sample states of this mesh and keep
        the choice for later batched calls; returns (batch, kernel, {(kernel, batch): rate})."""
        T = np.ascontiguousarray(T_C, np.float64)
        cw = np.ascontiguousarray(c_wt, np.float64)
        th = np.ascontiguousarray(t_h, np.float64)
        bc = np.ascontiguousarray(batches, np.int32)
        kc = np.ascontiguousarray(kernels, np.int32)
        rates = np.zeros(len(bc) * len(kc))
        bb, bk = C.c_int32(0), C.c_int32(0)
        _check(self.ctx.lib.rve_autotune_schedule(self.ctx.h, self.h, len(T), _ptr(T), _ptr(cw), _ptr(th), _ptr(bc),
                                                  len(bc), _ptr(kc), len(kc), C.byref(bb), C.byref(bk), _ptr(rates)),
               "rve_autotune_schedule")
        rr = rates.reshape(len(kc), len(bc))
        return int(bb.value), int(bk.value), {(int(k), int(b)): float(rr[i, j]) for i, k in enumerate(kc)
                                              for j, b in enumerate(bc)}

    def homogenise_weak(self):
        """(sigma-route tensors C, K, D via the multipliers, energy-form C, K, D)."""
        out = [np.zeros((6, 6)), np.zeros((3, 3)), np.zeros((3, 3)), np.zeros((6, 6)), np.zeros((3, 3)),
               np.zeros((3, 3))]
        s = Stats()
        _check(self.ctx.lib.rve_homogenise_weak(self.ctx.h, self.h, *[_ptr(a) for a in out], C.byref(s)),
               "rve_homogenise_weak")
        return out

    def homogenise(self, allow_not_converged=False) -> Result:
        Cc = np.zeros((6, 6))
        Kk = np.zeros((3, 3))
        Dd = np.zeros((3, 3))
        s = Stats()
        allow = (-4,) if allow_not_converged else ()
        rc = _check(self.ctx.lib.rve_homogenise(self.ctx.h, self.h, _ptr(Cc), _ptr(Kk), _ptr(Dd), C.byref(s)),
                    "rve_homogenise", allow)
        return Result(Cc, Kk, Dd, s.as_dict(), rc)

    def tensors(self):
        D = np.zeros((self.nt, 6, 6))
        K = np.zeros((self.nt, 3, 3))
        Dd = np.zeros((self.nt, 3, 3))
        _check(self.ctx.lib.rve_mesh_get_tensors(self.ctx.h, self.h, _ptr(D), _ptr(K), _ptr(Dd)),
               "rve_mesh_get_tensors")
        return D, K, Dd

    def apply_operator(self, field: int, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, np.float64)
        ncols = x.shape[-1]
        y = np.zeros_like(x)
        _check(self.ctx.lib.rve_apply_operator(self.ctx.h, self.h, int(field), int(ncols), _ptr(x), _ptr(y)),
               "rve_apply_operator")
        return y

    def apply_operator_mixed(self, x: np.ndarray, kernel: int = 0, scale=None, active=None):
        """The FP32 mechanics operator of the mixed-precision inner solve: kernel 0
        tensor cores, 1 CUDA cores.  Returns (y, energy per column)."""
        x = np.ascontiguousarray(x, np.float64)
        ncols = x.shape[-1]
        y = np.zeros_like(x)
        en = np.zeros(ncols)
        sc = None if scale is None else np.ascontiguousarray(scale, np.float64)
        act = None if active is None else np.ascontiguousarray(active, np.int32)
        _check(self.ctx.lib.rve_apply_operator_mixed(self.ctx.h, self.h, int(kernel), int(ncols), _ptr(x), _ptr(sc),
                                                     _ptr(act), _ptr(y), _ptr(en)), "rve_apply_operator_mixed")
        return y, en

    def operator_energy_noalloc(self, field: int, ncols: int, x_dev: int, y_dev: int, energy_dev: int):
        """Allocation-free operator apply on caller-owned device buffers (integer
        device addresses); enqueued on the context's stream."""
        _check(self.ctx.lib.rve_operator_energy_noalloc(self.ctx.h, self.h, int(field), int(ncols),
                                                        C.c_void_p(x_dev), C.c_void_p(y_dev),
                                                        C.c_void_p(energy_dev)),
               "rve_operator_energy_noalloc")

    def dofmap(self):
        ne = {1: 4, 2: 10, 3: 20}[self.p]
        ed = np.zeros((self.nt, ne), np.int32)
        lv = np.zeros((self.nt, 4), np.int32)
        _check(self.ctx.lib.rve_mesh_get_dofmap(self.ctx.h, self.h, _ptr(ed), _ptr(lv)), "rve_mesh_get_dofmap")
        return ed, lv

    def colouring(self):
        """(colour of every element, number of colours) of the current DOF map."""
        col = np.zeros(self.nt, np.int32)
        n = C.c_int32()
        _check(self.ctx.lib.rve_mesh_get_colouring(self.ctx.h, self.h, _ptr(col), C.byref(n)),
               "rve_mesh_get_colouring")
        return col, n.value

    def debug_set_node_bound(self, n_nodes: int):
        _check(self.ctx.lib.rve_debug_set_node_bound(self.ctx.h, self.h, int(n_nodes)), "rve_debug_set_node_bound")


__all__ = ["Context", "Mesh", "Surrogate", "RveError", "load_library", "exported_symbols", "galerkin_solve", "BC_DIRICHLET", "BC_PERIODIC",
           "BC_NEUMANN", "PREC_FP64", "PREC_MIXED", "Options", "Stats"]


class Macro:
    """The coupled macro step (heat and moisture transport, Gauss-point degradation)."""

    def __init__(self, ctx: "Context", h, nv: int, nt: int):
        self.ctx, self.h, self.nv, self.nt = ctx, h, nv, nt

    def free(self):
        if self.h:
            self.ctx.lib.rve_macro_free(self.ctx.h, self.h)
            self.h = None

    def set_transport(self, K_T, rho_cp, D_c):
        KT = np.ascontiguousarray(K_T, np.float64).reshape(9)
        Dc = np.ascontiguousarray(D_c, np.float64).reshape(9)
        _check(self.ctx.lib.rve_macro_set_transport(self.ctx.h, self.h, _ptr(KT), float(rho_cp), _ptr(Dc)),
               "rve_macro_set_transport")

    def set_face(self, mask, T_C, c_wt):
        m = np.ascontiguousarray(mask, np.uint8)
        _check(self.ctx.lib.rve_macro_set_face(self.ctx.h, self.h, _ptr(m), float(T_C), float(c_wt)),
               "rve_macro_set_face")

    def set_held(self, mask, values):
        m = np.ascontiguousarray(mask, np.uint8)
        v = np.ascontiguousarray(values, np.float64).reshape(-1)
        _check(self.ctx.lib.rve_macro_set_held(self.ctx.h, self.h, _ptr(m), _ptr(v)), "rve_macro_set_held")

    def solve_steady(self, rtol=1e-12, max_iter=20000):
        st = MacroStats()
        _check(self.ctx.lib.rve_macro_solve_steady(self.ctx.h, self.h, float(rtol), int(max_iter), C.byref(st)),
               "rve_macro_solve_steady")
        return st.as_dict()

    def gradients(self, field=0):
        g = np.zeros((self.nt, 3))
        _check(self.ctx.lib.rve_macro_gradients(self.ctx.h, self.h, int(field), _ptr(g)), "rve_macro_gradients")
        return g

    def reset(self, T0_C, c0_wt):
        _check(self.ctx.lib.rve_macro_reset(self.ctx.h, self.h, float(T0_C), float(c0_wt)), "rve_macro_reset")

    def step(self, dt_h, rtol=1e-12, max_iter=5000, beta=-0.001682, Tg_C=126.0, c_sat_wt=1.5):
        dg = Degradation(beta, Tg_C, c_sat_wt, 0)
        st = MacroStats()
        _check(self.ctx.lib.rve_macro_step(self.ctx.h, self.h, float(dt_h), C.byref(dg), float(rtol),
                                           int(max_iter), C.byref(st)), "rve_macro_step")
        return st.as_dict()

    def set_state(self, T, c, W, beta=-0.001682, Tg_C=126.0, c_sat_wt=1.5):
        """Resume from a saved state: nodal T and c [nv], Gauss-point 1 - omega [nt, 4]
        (as returned by get())."""
        Tn = np.ascontiguousarray(T, np.float64).reshape(-1)
        cn = np.ascontiguousarray(c, np.float64).reshape(-1)
        Wg = np.ascontiguousarray(W, np.float64).reshape(-1)
        if Tn.size != self.nv or cn.size != self.nv or Wg.size != self.nt * 4:
            raise ValueError("T and c need nv entries, W nt * 4")
        dg = Degradation(beta, Tg_C, c_sat_wt, 0)
        _check(self.ctx.lib.rve_macro_set_state(self.ctx.h, self.h, _ptr(Tn), _ptr(cn), _ptr(Wg), C.byref(dg)),
               "rve_macro_set_state")

    def gauss_dev(self):
        """Device addresses of the Gauss-point T, c, 1 - omega and t_eq arrays [nt * 4]."""
        ptrs = [C.c_void_p() for _ in range(4)]
        _check(self.ctx.lib.rve_macro_gauss_dev(self.ctx.h, self.h, *[C.byref(p) for p in ptrs]),
               "rve_macro_gauss_dev")
        return [p.value for p in ptrs]

    def get(self):
        T = np.zeros(self.nv)
        c = np.zeros(self.nv)
        g = [np.zeros(self.nt * 4) for _ in range(4)]
        _check(self.ctx.lib.rve_macro_get(self.ctx.h, self.h, _ptr(T), _ptr(c), *[_ptr(a) for a in g]),
               "rve_macro_get")
        return dict(T=T, c=c, Tg=g[0].reshape(-1, 4), cg=g[1].reshape(-1, 4), W=g[2].reshape(-1, 4),
                    t_eq=g[3].reshape(-1, 4))

    # macro mechanics of the nested FE^2 step (Sec. 5)
    def mech_set_bc(self, fixed, values=None):
        """fixed [nv, 3] (held DOFs) at values [nv, 3] (m; None = 0)."""
        f = np.ascontiguousarray(fixed, np.uint8).reshape(-1)
        v = None if values is None else np.ascontiguousarray(values, np.float64).reshape(-1)
        if f.size != self.nv * 3 or (v is not None and v.size != self.nv * 3):
            raise ValueError("fixed and values must have nv * 3 entries")
        _check(self.ctx.lib.rve_macro_mech_set_bc(self.ctx.h, self.h, _ptr(f), _ptr(v) if v is not None else None),
               "rve_macro_mech_set_bc")

    def mech_set_u(self, u=None):
        """Starting displacement of the next solve ([nv, 3], m; None = rest)."""
        v = None if u is None else np.ascontiguousarray(u, np.float64).reshape(-1)
        if v is not None and v.size != self.nv * 3:
            raise ValueError("u must have nv * 3 entries")
        _check(self.ctx.lib.rve_macro_mech_set_u(self.ctx.h, self.h, _ptr(v)), "rve_macro_mech_set_u")

    def mech_set_traction(self, face_nodes, t, add=False):
        m = np.ascontiguousarray(face_nodes, np.uint8).reshape(-1)
        tv = np.ascontiguousarray(t, np.float64).reshape(3)
        if m.size != self.nv:
            raise ValueError("face_nodes must have nv entries")
        _check(self.ctx.lib.rve_macro_mech_set_traction(self.ctx.h, self.h, _ptr(m), _ptr(tv), int(bool(add))),
               "rve_macro_mech_set_traction")

    def mech_solve(self, C_gp, rtol=1e-12, max_iter=20000):
        """C_gp: host array [nt, 4, 6, 6] (or [nt * 4, 6, 6]), or an integer device
        address of that layout (e.g. the C output of Context.macro_update_dev)."""
        st = MacroMechStats()
        if isinstance(C_gp, int):
            ptr, on_dev = C.c_void_p(C_gp), 1
        else:
            arr = np.ascontiguousarray(C_gp, np.float64).reshape(-1)
            if arr.size != self.nt * 4 * 36:
                raise ValueError("C_gp must have nt * 4 * 36 entries")
            ptr, on_dev = _ptr(arr), 0
        _check(self.ctx.lib.rve_macro_mech_solve(self.ctx.h, self.h, ptr, on_dev, float(rtol), int(max_iter),
                                                 C.byref(st)), "rve_macro_mech_solve")
        return st.as_dict()

    def mech_get(self):
        u = np.zeros((self.nv, 3))
        sig = np.zeros((self.nt, 4, 6))
        f = np.zeros((self.nv, 3))
        _check(self.ctx.lib.rve_macro_mech_get(self.ctx.h, self.h, _ptr(u), _ptr(sig), _ptr(f)),
               "rve_macro_mech_get")
        return dict(u=u, stress=sig, load=f)
