"""ctypes binding of the C ABI declared in ``include/tfeti.h``.

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  Device buffers are passed as raw pointers; torch tensors (CUDA,
float64/uint8, contiguous) are accepted wherever a device pointer is expected.
The library is built in-tree by ``build.py``; if it is missing the import of
this module raises, so there is no silent fallback.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))

TFETI_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of memory", 4: "non-positive pivot",
          5: "singular coarse problem", 6: "not converged", 7: "PCGP breakdown", 8: "non-finite value",
          9: "bounded device wait timed out"}
PRECOND_NONE, PRECOND_LUMPED, PRECOND_DIRICHLET = 0, 1, 2
COARSE_AUTO, COARSE_DENSE, COARSE_PLANES = 0, 1, 2
MLP_PARAMS = 4801
MAX_NEWTON = 64
FACES = ("x0", "x1", "y0", "y1", "z0", "z1")


class Problem(C.Structure):
    _fields_ = [("nel", C.c_int32 * 3), ("length", C.c_double * 3), ("nsub", C.c_int32 * 3),
                ("cuts", C.POINTER(C.c_int32) * 3), ("young", C.c_double), ("poisson", C.c_double),
                ("sigma_y", C.c_double), ("hardening", C.c_double), ("dirichlet", C.c_int32 * 6),
                ("traction_face", C.c_int32), ("precond", C.c_int32), ("coarse", C.c_int32)]


class Sizes(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("n_sub", "n_dof", "n_elements", "n_gp", "n_mult", "n_coarse", "n_nodes",
                                         "n_copy", "max_band", "device_bytes")]


class PcgInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("used_lambda0", C.c_int32),
                ("f_applies", C.c_int32), ("r0_norm", C.c_double), ("w_norm", C.c_double), ("seconds", C.c_double),
                ("f32_applies", C.c_int32), ("outer_iterations", C.c_int32)]


class StepInfo(C.Structure):
    _fields_ = [("newton", C.c_int32), ("converged", C.c_int32), ("pcg", C.c_int32 * MAX_NEWTON),
                ("plastic", C.c_int64 * MAX_NEWTON), ("criterion", C.c_double * MAX_NEWTON),
                ("refactored", C.c_int32 * MAX_NEWTON), ("plastic_committed", C.c_int64), ("seconds", C.c_double),
                ("outer", C.c_int32 * MAX_NEWTON), ("history", C.c_int32 * MAX_NEWTON)]

    def as_dict(self) -> dict:
        n = self.newton
        return {"newton": n, "converged": bool(self.converged), "pcg": list(self.pcg[:n]),
                "plastic": list(self.plastic[:n]), "criterion": list(self.criterion[:n]),
                "refactored": list(self.refactored[:n]), "plastic_committed": self.plastic_committed,
                "seconds": self.seconds, "outer": list(self.outer[:n]), "history": list(self.history[:n])}


class Timing(C.Structure):
    _fields_ = [("f_apply_ms_total", C.c_double), ("f_apply_launches", C.c_int64), ("f_apply_bytes", C.c_double),
                ("f_apply_flops", C.c_double), ("factor_ms_total", C.c_double), ("factor_launches", C.c_int64),
                ("kernel_launches", C.c_int64), ("schur_ms_total", C.c_double), ("schur_launches", C.c_int64),
                ("schur_flops_total", C.c_double), ("schur_bytes_total", C.c_double), ("inner_ms_total", C.c_double),
                ("inner_iterations", C.c_int64), ("inner_body_runs", C.c_int64)]


_P = C.c_void_p
_D = C.c_double
_I = C.c_int32
# name -> (restype, argtypes)
SIGNATURES = {
    "tfeti_plan_create": (C.c_int, [C.POINTER(Problem), C.POINTER(_P)]),
    "tfeti_plan_destroy": (C.c_int, [_P]),
    "tfeti_plan_sizes": (C.c_int, [_P, C.POINTER(Sizes)]),
    "tfeti_plan_export_B": (C.c_int, [_P, _P, _P, _P, C.POINTER(C.c_int64)]),
    "tfeti_plan_export_subdomains": (C.c_int, [_P, _P]),
    "tfeti_plan_export_fixing": (C.c_int, [_P, _P]),
    "tfeti_setup": (C.c_int, [C.POINTER(Problem), _P, C.POINTER(_P)]),
    "tfeti_setup_case": (C.c_int, [_P, _D, _D, _P, C.POINTER(_P)]),
    "tfeti_destroy": (C.c_int, [_P]),
    "tfeti_sizes_get": (C.c_int, [_P, C.POINTER(Sizes)]),
    "tfeti_last_error": (C.c_char_p, [_P]),
    "tfeti_status_str": (C.c_char_p, [C.c_int]),
    "tfeti_traction_load": (C.c_int, [_P, _P, _P]),
    "tfeti_return_map": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "tfeti_assemble_tangent": (C.c_int, [_P, _P, _P, _P]),
    "tfeti_dual_pcg": (C.c_int, [_P, _P, _P, _P, _P, _D, _I, C.POINTER(PcgInfo)]),
    "ssn_time_step": (C.c_int, [_P, _P, _I, _D, _D, _I, _I, C.POINTER(StepInfo)]),
    "ssn_time_step_cases": (C.c_int, [_P, _I, _P, _I, _D, _D, _I, _I, _P]),
    "tfeti_first_yield_traction": (C.c_int, [_P, _P, _D, C.POINTER(_D)]),
    "tfeti_set_precision": (C.c_int, [_P, _I, _D]),
    "tfeti_set_graphs": (C.c_int, [_P, _I]),
    "tfeti_set_fapply": (C.c_int, [_P, _I]),
    "tfeti_set_schur_format": (C.c_int, [_P, _I]),
    "tfeti_set_schur_threshold": (C.c_int, [_P, _I]),
    "tfeti_set_deflation": (C.c_int, [_P, _I]),
    "tfeti_set_woodbury": (C.c_int, [_P, _I]),
    "tfeti_set_fused_inner": (C.c_int, [_P, _I]),
    "tfeti_get_fused_inner": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "tfeti_get_woodbury_stats": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "tfeti_get_deflation_stats": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "tfeti_get_tuning": (C.c_int, [_P, _P, _P, _P]),
    "tfeti_set_recycling": (C.c_int, [_P, _I]),
    "tfeti_set_learned": (C.c_int, [_P, _I, _I, _D]),
    "tfeti_mlp_weights": (C.c_int, [_P, _P]),
    "tfeti_mlp_predict": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "tfeti_mlp_train": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _I]),
    "tfeti_get_state": (C.c_int, [_P, _P, _P, _P]),
    "tfeti_set_state": (C.c_int, [_P, _P, _P, _P]),
    "tfeti_apply_F": (C.c_int, [_P, _P, _P]),
    "tfeti_apply_F32": (C.c_int, [_P, _P, _P]),
    "tfeti_apply_projector": (C.c_int, [_P, _P, _P]),
    "tfeti_apply_precond": (C.c_int, [_P, _P, _P]),
    "tfeti_apply_N": (C.c_int, [_P, _P, _P]),
    "tfeti_apply_kdag": (C.c_int, [_P, _P, _P]),
    "tfeti_apply_K": (C.c_int, [_P, _P, _P]),
    "tfeti_apply_projector_noalloc": (C.c_int, [_P, _P, _P]),
    "tfeti_timing_get": (C.c_int, [_P, C.POINTER(Timing)]),
    "tfeti_timing_reset": (C.c_int, [_P, _I]),
    "tfeti_check_bounded_wait": (C.c_int, [_P, C.c_int64, C.POINTER(_I)]),
    "tfeti_measure_fp64_fma": (C.c_int, [_P, _I, C.POINTER(C.c_double)]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load the in-tree shared library (building it first if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"TFETI CUDA library not built: {path}")
        _build.build()
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class TfetiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def make_problem(workload, material: dict | None = None, precond: int = PRECOND_LUMPED, coarse: int = COARSE_AUTO):
    """Fill a Problem struct from a ``workloads.Workload`` (sizes, cuts, material, masks)."""
    pr = Problem()
    mat = dict(workload.material if material is None else material)
    keep = []
    for d in range(3):
        pr.nel[d] = workload.nel[d]
        pr.length[d] = workload.length[d]
        cuts = workload.cuts[d]
        pr.nsub[d] = len(cuts) - 1
        arr = (C.c_int32 * len(cuts))(*cuts)
        keep.append(arr)
        pr.cuts[d] = C.cast(arr, C.POINTER(C.c_int32))
    pr.young, pr.poisson = mat["young"], mat["poisson"]
    pr.sigma_y, pr.hardening = mat["sigma_y"], mat["hardening"]
    for f, m in enumerate(workload.dirichlet_masks()):
        pr.dirichlet[f] = m
    pr.traction_face = FACES.index(workload.traction_face)
    pr.precond = precond
    pr.coarse = coarse
    pr._keep = keep
    return pr


class Plan:
    """Host-only plan (no GPU): sizes, B, subdomains and fixing dofs."""

    def __init__(self, workload, **kw):
        self.lib = load()
        self.problem = make_problem(workload, **kw)
        h = _P()
        st = self.lib.tfeti_plan_create(C.byref(self.problem), C.byref(h))
        if st != TFETI_OK:
            raise TfetiError(st, "tfeti_plan_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.tfeti_plan_destroy(self.h)
            self.h = None

    __del__ = close

    def sizes(self) -> dict:
        s = Sizes()
        self.lib.tfeti_plan_sizes(self.h, C.byref(s))
        return {k: getattr(s, k) for k, _ in Sizes._fields_}

    def export_B(self):
        import numpy as np
        nnz = C.c_int64()
        self.lib.tfeti_plan_export_B(self.h, None, None, None, C.byref(nnz))
        rows = np.zeros(nnz.value, dtype=np.int64)
        cols = np.zeros(nnz.value, dtype=np.int64)
        vals = np.zeros(nnz.value, dtype=np.float64)
        self.lib.tfeti_plan_export_B(self.h, rows.ctypes.data, cols.ctypes.data, vals.ctypes.data, C.byref(nnz))
        return rows, cols, vals

    def export_subdomains(self):
        import numpy as np
        out = np.zeros((self.sizes()["n_sub"], 9), dtype=np.int64)
        self.lib.tfeti_plan_export_subdomains(self.h, out.ctypes.data)
        return out

    def export_fixing(self):
        import numpy as np
        out = np.zeros((self.sizes()["n_sub"], 6), dtype=np.int32)
        self.lib.tfeti_plan_export_fixing(self.h, out.ctypes.data)
        return out


class Context:
    """A device context (``tfeti_setup``) with thin wrappers of every C-ABI call."""

    def __init__(self, workload, stream=None, **kw):
        self.lib = load()
        self.problem = make_problem(workload, **kw)
        h = _P()
        st = self.lib.tfeti_setup(C.byref(self.problem), _ptr_stream(stream), C.byref(h))
        if st != TFETI_OK:
            raise TfetiError(st, "tfeti_setup")
        self.h = h
        s = Sizes()
        self.lib.tfeti_sizes_get(self.h, C.byref(s))
        self.sizes = {k: getattr(s, k) for k, _ in Sizes._fields_}

    @classmethod
    def case_of(cls, base: "Context", sigma_y: float, hardening: float, stream=None) -> "Context":
        """A case context (``tfeti_setup_case``) sharing base's read-only set-up; it keeps
        a reference to base so that base outlives it."""
        obj = cls.__new__(cls)
        obj.lib = base.lib
        obj.problem = Problem.from_buffer_copy(base.problem)
        obj.problem.sigma_y = sigma_y
        obj.problem.hardening = hardening
        obj._base = base
        h = _P()
        st = obj.lib.tfeti_setup_case(base.h, sigma_y, hardening, _ptr_stream(stream), C.byref(h))
        if st != TFETI_OK:
            obj.h = None
            raise TfetiError(st, f"tfeti_setup_case: {base.lib.tfeti_last_error(base.h).decode()}")
        obj.h = h
        s = Sizes()
        obj.lib.tfeti_sizes_get(obj.h, C.byref(s))
        obj.sizes = {k: getattr(s, k) for k, _ in Sizes._fields_}
        return obj

    def close(self):
        if getattr(self, "h", None):
            self.lib.tfeti_destroy(self.h)
            self.h = None

    __del__ = close

    def _check(self, st, name):
        if st != TFETI_OK:
            raise TfetiError(st, f"{name}: {self.lib.tfeti_last_error(self.h).decode()}")
        return st

    def traction_load(self, t, f_out):
        arr = (C.c_double * 3)(*t)
        return self._check(self.lib.tfeti_traction_load(self.h, C.cast(arr, _P), _ptr(f_out)), "tfeti_traction_load")

    def return_map(self, du, dsigma, dkappa, plastic, Dtan=None):
        return self._check(self.lib.tfeti_return_map(self.h, _ptr(du), _ptr(dsigma), _ptr(dkappa), _ptr(plastic),
                                                     _ptr(Dtan)), "tfeti_return_map")

    def assemble_tangent(self, du, df, f_out=None):
        return self._check(self.lib.tfeti_assemble_tangent(self.h, _ptr(du), _ptr(df), _ptr(f_out)),
                           "tfeti_assemble_tangent")

    def dual_pcg(self, f, u_out, lambda_out=None, lambda0=None, rtol=1e-8, maxit=5000, check=True):
        info = PcgInfo()
        st = self.lib.tfeti_dual_pcg(self.h, _ptr(f), _ptr(u_out), _ptr(lambda_out), _ptr(lambda0), rtol, maxit,
                                     C.byref(info))
        if check:
            self._check(st, "tfeti_dual_pcg")
        return {k: getattr(info, k) for k, _ in PcgInfo._fields_} | {"status": st}

    def time_step(self, df, newton_tol, pcg_rtol, newton_maxit=30, pcg_maxit=5000, df_on_host=False, check=True):
        info = StepInfo()
        st = self.lib.ssn_time_step(self.h, _ptr(df), 1 if df_on_host else 0, newton_tol, pcg_rtol, newton_maxit,
                                    pcg_maxit, C.byref(info))
        if check:
            self._check(st, "ssn_time_step")
        return info.as_dict() | {"status": st}

    def set_precision(self, mixed: bool, inner_rtol: float = 1e-4):
        """FP64 dual solve (default) or FP64-refined PCGP with FP32 inner F-applies."""
        return self._check(self.lib.tfeti_set_precision(self.h, 1 if mixed else 0, inner_rtol), "tfeti_set_precision")

    def set_recycling(self, q: int):
        """Start each dual solve from the best combination of the last q solutions (0: off)."""
        return self._check(self.lib.tfeti_set_recycling(self.h, int(q)), "tfeti_set_recycling")

    def set_learned(self, enable: bool, epochs: int = 8, lr: float = 1e-3):
        """Per-interface MLP prediction in the history start of every load step's first Newton solve."""
        return self._check(self.lib.tfeti_set_learned(self.h, 1 if enable else 0, int(epochs), float(lr)),
                           "tfeti_set_learned")

    def mlp_weights(self):
        out = (C.c_float * MLP_PARAMS)()
        self._check(self.lib.tfeti_mlp_weights(self.h, C.cast(out, _P)), "tfeti_mlp_weights")
        return list(out)

    def mlp_predict(self, la, lb, d, pf_now, pf_prev, scal, y):
        sc = (C.c_float * 4)(*scal)
        return self._check(self.lib.tfeti_mlp_predict(self.h, _ptr(la), _ptr(lb), _ptr(d), _ptr(pf_now), _ptr(pf_prev),
                                                      C.cast(sc, _P), _ptr(y)), "tfeti_mlp_predict")

    def mlp_train(self, la, lb, d, pf_now, pf_prev, scal, target, steps):
        sc = (C.c_float * 4)(*scal)
        return self._check(self.lib.tfeti_mlp_train(self.h, _ptr(la), _ptr(lb), _ptr(d), _ptr(pf_now), _ptr(pf_prev),
                                                    C.cast(sc, _P), _ptr(target), int(steps)), "tfeti_mlp_train")

    def set_fapply(self, schur: bool):
        """FP64 F-apply of elastic subdomains by their shape's dual Schur block (DGEMM) or banded solves."""
        return self._check(self.lib.tfeti_set_fapply(self.h, 1 if schur else 0), "tfeti_set_fapply")

    def set_schur_format(self, bf16: bool):
        """Inner Schur apply of the mixed mode with BF16 S (two MMAs per step) or TF32 x 3 (default)."""
        return self._check(self.lib.tfeti_set_schur_format(self.h, 1 if bf16 else 0), "tfeti_set_schur_format")

    def set_woodbury(self, mode):
        """Plastic subdomains on their shape's elastic factor + a Woodbury correction: 0 (or False) off,
        1 in the inner FP32 F-apply only, 2 (or True, the default) also in the FP64 solves, which
        leaves them out of the refactorisation."""
        m = 2 if mode is True else 0 if mode is False else int(mode)
        return self._check(self.lib.tfeti_set_woodbury(self.h, m), "tfeti_set_woodbury")

    def set_fused_inner(self, enable: bool):
        """The inner PCGP iteration as one cooperative launch between two F-applies (default off)."""
        return self._check(self.lib.tfeti_set_fused_inner(self.h, 1 if enable else 0), "tfeti_set_fused_inner")

    def fused_inner_active(self) -> bool:
        v = C.c_int32()
        self._check(self.lib.tfeti_get_fused_inner(self.h, C.byref(v)), "tfeti_get_fused_inner")
        return bool(v.value)

    def woodbury_stats(self) -> dict:
        a, b = C.c_int64(), C.c_int64()
        self.lib.tfeti_get_woodbury_stats(self.h, C.byref(a), C.byref(b))
        return {"subdomains": a.value, "fallbacks": b.value}

    def set_deflation(self, k: int):
        """Deflate the inner PCGP with up to k vectors (network prediction, stored solutions); 0: off."""
        return self._check(self.lib.tfeti_set_deflation(self.h, int(k)), "tfeti_set_deflation")

    def deflation_stats(self) -> dict:
        a, b, f = C.c_int64(), C.c_int64(), C.c_int64()
        self.lib.tfeti_get_deflation_stats(self.h, C.byref(a), C.byref(b), C.byref(f))
        return {"setups": a.value, "vectors": b.value, "fallbacks": f.value}

    def set_schur_threshold(self, threshold: int):
        """Shapes with >= threshold subdomains use their Schur block in the inner F-apply (0: tune)."""
        return self._check(self.lib.tfeti_set_schur_threshold(self.h, int(threshold)), "tfeti_set_schur_threshold")

    def tuning(self) -> dict:
        t, n = C.c_int32(), C.c_int32()
        ms = (C.c_float * 4)()
        self.lib.tfeti_get_tuning(self.h, C.byref(t), C.byref(n), C.cast(ms, _P))
        return {"schur_threshold": t.value, "n_schur_shapes": n.value, "tune_ms": list(ms)}

    def set_graphs(self, enable: bool):
        """Inner PCGP of the mixed mode as one CUDA graph launch (default) or kernel by kernel."""
        return self._check(self.lib.tfeti_set_graphs(self.h, 1 if enable else 0), "tfeti_set_graphs")

    def first_yield_traction(self, direction, rtol=1e-12) -> float:
        arr = (C.c_double * 3)(*direction)
        out = C.c_double()
        self._check(self.lib.tfeti_first_yield_traction(self.h, C.cast(arr, _P), rtol, C.byref(out)),
                    "tfeti_first_yield_traction")
        return out.value

    def get_state(self, u=None, sigma=None, kappa=None):
        return self._check(self.lib.tfeti_get_state(self.h, _ptr(u), _ptr(sigma), _ptr(kappa)), "tfeti_get_state")

    def set_state(self, u=None, sigma=None, kappa=None):
        return self._check(self.lib.tfeti_set_state(self.h, _ptr(u), _ptr(sigma), _ptr(kappa)), "tfeti_set_state")

    def apply(self, which: str, x, y):
        fn = getattr(self.lib, "tfeti_apply_" + which)
        return self._check(fn(self.h, _ptr(x), _ptr(y)), "tfeti_apply_" + which)

    def apply_projector_noalloc(self, x, y):
        """P_N x through the entry point that keeps its work vectors in static device memory."""
        return self._check(self.lib.tfeti_apply_projector_noalloc(self.h, _ptr(x), _ptr(y)),
                           "tfeti_apply_projector_noalloc")

    def timing(self) -> dict:
        t = Timing()
        self.lib.tfeti_timing_get(self.h, C.byref(t))
        return {k: getattr(t, k) for k, _ in Timing._fields_}

    def timing_reset(self, events: bool):
        self.lib.tfeti_timing_reset(self.h, 1 if events else 0)


def time_step_cases(ctxs, dfs, newton_tol, pcg_rtol, newton_maxit=30, pcg_maxit=5000, df_on_host=False,
                    check=True):
    """``ssn_time_step_cases``: one time step of every context in ``ctxs`` (distinct, each
    on its own stream), case k with load increment ``dfs[k]``; returns one info dict per case."""
    n = len(ctxs)
    lib = load()
    hs = (_P * n)(*[c.h for c in ctxs])
    ps = (_P * n)(*[_ptr(d) for d in dfs])
    infos = (StepInfo * n)()
    st = lib.ssn_time_step_cases(C.cast(hs, _P), n, C.cast(ps, _P), 1 if df_on_host else 0, newton_tol, pcg_rtol,
                                 newton_maxit, pcg_maxit, C.cast(infos, _P))
    if check and st != TFETI_OK:
        msgs = "; ".join(f"case {k}: {lib.tfeti_last_error(c.h).decode()}" for k, c in enumerate(ctxs))
        raise TfetiError(st, f"ssn_time_step_cases: {msgs}")
    return [infos[k].as_dict() | {"status": st} for k in range(n)]


def measure_fp64_fma(stream=None, iters=20000) -> float:
    """FP64 FMA rate of the current device in TFLOP/s (``tfeti_measure_fp64_fma``)."""
    out = C.c_double()
    st = load().tfeti_measure_fp64_fma(_ptr_stream(stream), int(iters), C.byref(out))
    if st != TFETI_OK:
        raise TfetiError(st, "tfeti_measure_fp64_fma")
    return out.value


def _ptr_stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)
