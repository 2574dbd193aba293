"""Thin Python binding of libmfto.so (the C ABI declared in include/mfto.h).

Argument marshalling only: every step runs in the library's CUDA kernels.
Device arrays are torch tensors on a CUDA device (torch supplies the memory
and the stream); the functions carry the C names without the ``mfto_``
prefix.  Loading fails loudly when the library is missing -- there is no CPU
path.
"""
from __future__ import annotations

import ctypes as C
import os
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
LIB_PATH = HERE / "libmfto.so"

(OK, INVALID_ARG, CUDA_ERROR, OOM, NOT_CONVERGED, STALLED, BREAKDOWN, UNSUPPORTED,
 TOO_LARGE) = range(9)
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA_ERROR", 3: "OOM", 4: "NOT_CONVERGED",
                5: "STALLED", 6: "BREAKDOWN", 7: "UNSUPPORTED", 8: "TOO_LARGE"}
NOALLOC_MAX_ELEMENTS = 2048 * 256

(FORM_F64, FORM_F32, FORM_TF32, FORM_TF32X3, FORM_BF16, FORM_BF16X3, FORM_F16,
 FORM_F16X3) = range(8)
FORMS = {"f64": FORM_F64, "f32": FORM_F32, "tf32": FORM_TF32, "tf32x3": FORM_TF32X3,
         "bf16": FORM_BF16, "bf16x3": FORM_BF16X3, "f16": FORM_F16, "f16x3": FORM_F16X3}
IR_RESTART, IR_CONTINUE = 0, 1


class Mesh(C.Structure):
    _fields_ = [("nelx", C.c_int32), ("nely", C.c_int32), ("nelz", C.c_int32),
                ("h", C.c_double)]


class Params(C.Structure):
    _fields_ = [("E0", C.c_double), ("Emin", C.c_double), ("nu", C.c_double),
                ("penal", C.c_double), ("rmin", C.c_double), ("volfrac", C.c_double),
                ("move", C.c_double), ("rtol", C.c_double), ("maxit", C.c_int32),
                ("check_every", C.c_int32), ("max_rhs", C.c_int32)]


class SolveStats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("status", C.c_int32),
                ("rel_residual", C.c_double), ("fnorm", C.c_double)]


class IterStats(C.Structure):
    _fields_ = [("compliance", C.c_double), ("change", C.c_double), ("volume", C.c_double),
                ("grayness", C.c_double), ("lambda_", C.c_double),
                ("cg_iterations", C.c_int32), ("cg_status", C.c_int32),
                ("rel_residual", C.c_double)]


class IrStats(C.Structure):
    _fields_ = [("outer_iterations", C.c_int32), ("inner_iterations", C.c_int32),
                ("status", C.c_int32), ("kv_f64", C.c_int32), ("rel_residual", C.c_double),
                ("fnorm", C.c_double), ("history", C.c_double * 64)]


class KappaParams(C.Structure):
    _fields_ = [("power_maxit", C.c_int32), ("power_tol", C.c_double),
                ("inverse_maxit", C.c_int32), ("inverse_tol", C.c_double),
                ("inner_rtol", C.c_double), ("inner_maxit", C.c_int32)]


class GmgParams(C.Structure):
    _fields_ = [("max_levels", C.c_int32), ("coarse_max_dofs", C.c_int32),
                ("nu_pre", C.c_int32), ("nu_post", C.c_int32), ("omega", C.c_double),
                ("mixed", C.c_int32), ("inner_tol", C.c_double),
                ("smoother_form", C.c_int32), ("matfree_level1", C.c_int32),
                ("continue_dir", C.c_int32), ("cheb_degree", C.c_int32)]


GMG_MAX_LEVELS = 10

class KappaStats(C.Structure):
    _fields_ = [("lambda_max", C.c_double), ("lambda_min", C.c_double), ("kappa", C.c_double),
                ("power_steps", C.c_int32), ("inverse_steps", C.c_int32),
                ("inner_iterations", C.c_int32), ("inner_capped", C.c_int32)]


class ProtocolParams(C.Structure):
    _fields_ = [("n_iter", C.c_int32), ("rmin0", C.c_double), ("eta", C.c_double),
                ("restart_factor", C.c_double), ("select_min_penal", C.c_double),
                ("select_max_gray", C.c_double), ("cold_start", C.c_int32)]


class ProtocolStats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("selected_iteration", C.c_int32),
                ("selected_compliance", C.c_double), ("restarts", C.c_int32),
                ("cg_iterations", C.c_int32)]


class LearnedStats(C.Structure):
    _fields_ = [("outer_iterations", C.c_int32), ("inner_iterations", C.c_int32),
                ("fp64_iterations", C.c_int32), ("nn_calls", C.c_int32),
                ("fallback", C.c_int32), ("status", C.c_int32),
                ("rel_residual", C.c_double), ("fnorm", C.c_double), ("nn_ms", C.c_double),
                ("history", C.c_double * 64)]


class MftoError(RuntimeError):
    def __init__(self, fn, code, msg=""):
        super().__init__(f"{fn} -> {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None

# name -> (restype, argtypes); the full exported surface of include/mfto.h
_P = C.c_void_p
SIGNATURES = {
    "mfto_version": (C.c_char_p, []),
    "mfto_default_params": (None, [C.POINTER(Params)]),
    "mfto_unit_ke": (C.c_int32, [C.c_double, C.c_double, C.c_double, _P]),
    "mfto_edof": (C.c_int32, [C.POINTER(Mesh), _P]),
    "mfto_filter_stencil": (C.c_int32, [C.c_double, C.c_int32, _P, _P, C.POINTER(C.c_int32)]),
    "mfto_create": (C.c_int32, [C.POINTER(Mesh), C.POINTER(Params), _P, _P, C.POINTER(_P)]),
    "mfto_destroy": (C.c_int32, [_P]),
    "mfto_set_params": (C.c_int32, [_P, C.POINTER(Params)]),
    "mfto_last_error": (C.c_char_p, [_P]),
    "mfto_sizes": (C.c_int32, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                               C.POINTER(C.c_int64)]),
    "mfto_simp_modulus": (C.c_int32, [_P, C.c_int32, _P, _P]),
    "mfto_kv": (C.c_int32, [_P, C.c_int32, _P, _P, _P]),
    "mfto_jacobi_diag": (C.c_int32, [_P, C.c_int32, _P, _P]),
    "mfto_set_kv_variant": (C.c_int32, [_P, C.c_int32]),
    "mfto_set_cg_engine": (C.c_int32, [_P, C.c_int32]),
    "mfto_set_ir_mode": (C.c_int32, [_P, C.c_int32]),
    "mfto_default_kappa_params": (None, [C.POINTER(KappaParams)]),
    "mfto_default_gmg_params": (None, [C.POINTER(GmgParams)]),
    "mfto_device_bytes": (C.c_int32, [_P, C.POINTER(C.c_int64)]),
    "mfto_gmg_params_in_use": (C.c_int32, [_P, C.POINTER(GmgParams)]),
    "mfto_gmg_solve_multi": (C.c_int32, [_P, _P, _P, _P, C.c_int32, _P]),
    "mfto_gmg_setup": (C.c_int32, [_P, _P, C.POINTER(GmgParams)]),
    "mfto_gmg_levels": (C.c_int32, [_P, C.POINTER(C.c_int32), _P]),
    "mfto_gmg_apply": (C.c_int32, [_P, C.c_int32, _P, _P]),
    "mfto_gmg_vcycle": (C.c_int32, [_P, _P, _P]),
    "mfto_gmg_solve": (C.c_int32, [_P, _P, _P, _P, C.POINTER(SolveStats)]),
    "mfto_set_gmg_solver": (C.c_int32, [_P, C.c_int32, C.POINTER(GmgParams)]),
    "mfto_set_projection": (C.c_int32, [_P, C.c_double, C.c_double]),
    "mfto_project": (C.c_int32, [_P, _P, _P, _P]),
    "mfto_default_protocol_params": (None, [C.POINTER(ProtocolParams)]),
    "mfto_simp_protocol": (C.c_int32, [_P, _P, _P, _P, _P, C.POINTER(ProtocolParams), _P, _P,
                                       _P, C.POINTER(ProtocolStats)]),
    "mfto_kappa": (C.c_int32, [_P, _P, _P, _P, _P, C.POINTER(KappaParams), C.POINTER(KappaStats)]),
    "mfto_set_kv_shape": (C.c_int32, [_P, C.c_int32, C.c_int32]),
    "mfto_kv_autotune": (C.c_int32, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                     C.POINTER(C.c_float)]),
    "mfto_cg_timing_read": (C.c_int32, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                        C.POINTER(C.c_double)]),
    "mfto_cg_kv_time": (C.c_int32, [_P, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_double)]),
    "mfto_pcg": (C.c_int32, [_P, _P, _P, _P, C.POINTER(SolveStats)]),
    "mfto_ir_solve": (C.c_int32, [_P, C.c_int32, C.c_double, _P, _P, _P, C.POINTER(IrStats)]),
    "mfto_set_solver": (C.c_int32, [_P, C.c_int32, C.c_double, C.c_int32, C.c_int32]),
    "mfto_kv_multi": (C.c_int32, [_P, C.c_int32, _P, _P, _P, C.c_int32]),
    "mfto_batch_create": (C.c_int32, [C.c_int32, C.POINTER(Mesh), C.POINTER(Params), _P, _P,
                                      C.POINTER(_P)]),
    "mfto_batch_destroy": (C.c_int32, [_P]),
    "mfto_batch_last_error": (C.c_char_p, [_P]),
    "mfto_batch_layout": (C.c_int32, [_P, _P, _P]),
    "mfto_batch_kv": (C.c_int32, [_P, C.c_int32, _P, _P, _P]),
    "mfto_batch_autotune": (C.c_int32, [_P, C.c_int32, _P, C.POINTER(C.c_int32)]),
    "mfto_batch_set_shape": (C.c_int32, [_P, C.c_int32]),
    "mfto_batch_solve": (C.c_int32, [_P, C.c_double, _P, _P, _P, C.c_int32, C.c_int32,
                                     C.POINTER(IrStats)]),
    "mfto_batch_launch_count": (C.c_int32, [_P, C.POINTER(C.c_int64)]),
    "mfto_batch_set_ir_mode": (C.c_int32, [_P, C.c_int32]),
    "mfto_ebe_create": (C.c_int32, [C.c_int64, C.c_int64, _P, _P, _P]),
    "mfto_ebe_destroy": (C.c_int32, [_P]),
    "mfto_ebe_last_error": (C.c_char_p, [_P]),
    "mfto_ebe_kv": (C.c_int32, [_P, C.c_int32, _P, _P, _P, _P, _P]),
    "mfto_ebe_launch_count": (C.c_int32, [_P, C.POINTER(C.c_int64)]),
    "mfto_ir_solve_multi": (C.c_int32, [_P, C.c_double, _P, _P, _P, C.c_int32,
                                        C.POINTER(IrStats)]),
    "mfto_filter": (C.c_int32, [_P, _P, _P, C.c_int32]),
    "mfto_compliance_sens": (C.c_int32, [_P, _P, _P, C.POINTER(C.c_double), _P]),
    "mfto_oc_update": (C.c_int32, [_P, _P, _P, _P, C.POINTER(IterStats)]),
    "mfto_simp_step": (C.c_int32, [_P, _P, _P, _P, _P, C.POINTER(IterStats)]),
    "mfto_launch_count": (C.c_int32, [_P, C.POINTER(C.c_int64)]),
    "mfto_fma_probe": (C.c_int32, [C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_double)]),
    "mfto_compliance_sens_noalloc": (C.c_int32, [C.POINTER(Mesh), C.c_double, C.c_double,
                                                 C.c_double, C.c_double, _P, _P, _P,
                                                 C.POINTER(C.c_double), _P]),
    "mfto_kv_timing": (C.c_int32, [_P, C.c_int32]),
    "mfto_nn_create": (C.c_int32, [C.c_int32, C.c_int32, C.c_int64, C.c_int64, C.c_uint64, _P,
                                   C.POINTER(_P)]),
    "mfto_nn_destroy": (C.c_int32, [_P]),
    "mfto_nn_last_error": (C.c_char_p, [_P]),
    "mfto_nn_num_params": (C.c_int32, [_P, C.POINTER(C.c_int64)]),
    "mfto_nn_get_params": (C.c_int32, [_P, _P]),
    "mfto_nn_set_params": (C.c_int32, [_P, _P]),
    "mfto_nn_forward": (C.c_int32, [_P, C.c_int32, C.c_int32, C.c_int32, _P, _P]),
    "mfto_nn_gradient": (C.c_int32, [_P, C.c_int32, C.c_int32, C.c_int32, _P, _P, _P,
                                     C.POINTER(C.c_double), _P]),
    "mfto_nn_train_step": (C.c_int32, [_P, C.c_int32, C.c_int32, C.c_int32, _P, _P, _P,
                                       C.c_float, C.POINTER(C.c_double)]),
    "mfto_nn_launch_count": (C.c_int32, [_P, C.POINTER(C.c_int64)]),
    "mfto_nn_set_tensor_cores": (C.c_int32, [_P, C.c_int32]),
    "mfto_nn_tc_status": (C.c_int32, [_P, C.POINTER(C.c_int32)]),
    "mfto_nn_grid": (C.c_int32, [C.POINTER(Mesh), C.c_int32, _P]),
    "mfto_nn_features": (C.c_int32, [_P, C.c_int32, _P, _P, _P]),
    "mfto_nn_target": (C.c_int32, [_P, C.c_int32, _P, _P, _P]),
    "mfto_nn_to_dofs": (C.c_int32, [_P, C.c_int32, _P, _P]),
    "mfto_nn_sample": (C.c_int32, [_P, C.c_int32, _P, _P, _P, _P, C.c_int32, _P, _P, _P]),
    "mfto_set_learned": (C.c_int32, [_P, _P, C.c_int32]),
    "mfto_nn_train_energy": (C.c_int32, [_P, _P, _P, _P, _P, C.c_double, C.c_float,
                                         C.POINTER(C.c_double)]),
    "mfto_learned_solve": (C.c_int32, [_P, _P, _P, _P, _P, C.POINTER(LearnedStats)]),
    "mfto_kv_timing_read": (C.c_int32, [_P, C.c_int32, C.POINTER(C.c_int64),
                                        C.POINTER(C.c_double)]),
}


def lib() -> C.CDLL:
    """Load libmfto.so (built by paper_2604_18020_gb300.build); raise if absent."""
    global _lib
    if _lib is None:
        path = Path(os.environ.get("MFTO_LIB", LIB_PATH))
        if not path.exists():
            raise RuntimeError(f"{path} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(str(path))
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(fn, code, handle=None):
    if code != OK:
        msg = ""
        if handle:
            raw = lib().mfto_last_error(handle)
            msg = raw.decode() if raw else ""
        raise MftoError(fn, code, msg)


def default_protocol_params(**kw) -> ProtocolParams:
    p = ProtocolParams()
    lib().mfto_default_protocol_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def default_kappa_params(**kw) -> KappaParams:
    p = KappaParams()
    lib().mfto_default_kappa_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def default_params(**kw) -> Params:
    p = Params()
    lib().mfto_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


# ------------------------------------------------------------------ host calls

def default_gmg_params(**kw) -> GmgParams:
    p = GmgParams()
    lib().mfto_default_gmg_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def unit_ke(E0=1.0, nu=0.3, h=1.0) -> np.ndarray:
    out = np.zeros(576)
    _check("mfto_unit_ke", lib().mfto_unit_ke(E0, nu, h, out.ctypes.data))
    return out.reshape(24, 24)


def edof(nelx, nely, nelz) -> np.ndarray:
    m = Mesh(nelx, nely, nelz, 1.0)
    out = np.zeros(nelx * nely * nelz * 24, dtype=np.int32)
    _check("mfto_edof", lib().mfto_edof(C.byref(m), out.ctypes.data))
    return out.reshape(-1, 24)


def filter_stencil(rmin):
    n = C.c_int32(0)
    lib().mfto_filter_stencil(rmin, 0, None, None, C.byref(n))
    off = np.zeros(3 * n.value, dtype=np.int32)
    w = np.zeros(n.value)
    _check("mfto_filter_stencil",
           lib().mfto_filter_stencil(rmin, n.value, off.ctypes.data, w.ctypes.data, C.byref(n)))
    return off.reshape(-1, 3), w


def fma_probe(form=FORM_F64, blocks=0, iters=4096):
    """FMA-pipe peak probe: returns (FMA/s, elapsed ms)."""
    import torch
    if blocks <= 0:
        blocks = 8 * torch.cuda.get_device_properties(0).multi_processor_count
    ms = C.c_double()
    _check("mfto_fma_probe", lib().mfto_fma_probe(form, blocks, iters, C.byref(ms)))
    return blocks * 256.0 * iters * 8 / (ms.value * 1e-3), ms.value


def compliance_sens_noalloc(nelx, nely, nelz, rho_phys, u, dc=None, E0=1.0, Emin=1e-9,
                            nu=0.3, penal=3.0, h=1.0, stream=None) -> float:
    """Compliance (returned) and sensitivities (into dc) without a handle and
    without any device allocation by the library; see
    mfto_compliance_sens_noalloc in include/mfto.h for who needs it, its
    524,288-element capacity and why overlapping calls race."""
    import torch
    n_elem = nelx * nely * nelz
    n_dof = 3 * (nelx + 1) * (nely + 1) * (nelz + 1)
    st = stream if stream is not None else torch.cuda.current_stream()
    # the library launches on the current device: every array and the stream
    # must live there
    cur = torch.cuda.current_device()
    for name, t in (("rho_phys", rho_phys), ("u", u), ("dc", dc)):
        if t is not None and t.is_cuda and t.device.index != cur:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is "
                             f"cuda:{cur}")
    if st.device.index != cur:
        raise ValueError(f"the stream is on cuda:{st.device.index}, the current device is "
                         f"cuda:{cur}")
    c = C.c_double()
    m = Mesh(nelx, nely, nelz, h)
    code = lib().mfto_compliance_sens_noalloc(
        C.byref(m), E0, Emin, nu, penal, _ptr(rho_phys, torch.float64, n_elem, "rho_phys"),
        _ptr(u, torch.float64, n_dof, "u"), _ptr(dc, torch.float64, n_elem, "dc"), C.byref(c),
        C.c_void_p(st.cuda_stream))
    if code == TOO_LARGE:
        raise MftoError("mfto_compliance_sens_noalloc", code,
                        f"mesh has {n_elem} elements; this entry point takes at most "
                        f"{NOALLOC_MAX_ELEMENTS}")
    _check("mfto_compliance_sens_noalloc", code)
    return c.value


# ----------------------------------------------------------------- the handle

def _ptr(t, dtype=None, numel=None, name="tensor"):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return t.data_ptr()


class Handle:
    """Owns one mfto_handle (mesh, parameters, fixed set, device workspace)."""

    def __init__(self, nelx, nely, nelz, fixed, params: Params | None = None, h=1.0,
                 stream=None):
        import torch
        self.mesh = Mesh(nelx, nely, nelz, h)
        self.params = params if params is not None else default_params()
        fixed = np.ascontiguousarray(fixed, dtype=np.uint8)
        self.n_elem = nelx * nely * nelz
        self.n_node = (nelx + 1) * (nely + 1) * (nelz + 1)
        self.n_dof = 3 * self.n_node
        if fixed.size != self.n_node:
            raise ValueError(f"fixed mask must have {self.n_node} entries")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        hp = C.c_void_p()
        code = lib().mfto_create(C.byref(self.mesh), C.byref(self.params), fixed.ctypes.data,
                                 C.c_void_p(self.stream.cuda_stream), C.byref(hp))
        _check("mfto_create", code)
        self._h = hp

    def close(self):
        if getattr(self, "_h", None):
            lib().mfto_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- helpers
    def _dt(self, form):
        import torch
        return torch.float64 if form == FORM_F64 else torch.float32

    def set_params(self, params: Params):
        _check("mfto_set_params", lib().mfto_set_params(self._h, C.byref(params)), self._h)
        self.params = params

    def sizes(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        _check("mfto_sizes", lib().mfto_sizes(self._h, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    # ---- device steps
    def simp_modulus(self, rho_phys, E, form=FORM_F64):
        import torch
        _check("mfto_simp_modulus", lib().mfto_simp_modulus(
            self._h, form, _ptr(rho_phys, torch.float64, self.n_elem, "rho_phys"),
            _ptr(E, self._dt(form), self.n_elem, "E")), self._h)

    def kv(self, E, v, y, form=FORM_F64):
        dt = self._dt(form)
        _check("mfto_kv", lib().mfto_kv(
            self._h, form, _ptr(E, dt, self.n_elem, "E"), _ptr(v, dt, self.n_dof, "v"),
            _ptr(y, dt, self.n_dof, "y")), self._h)

    def set_kv_variant(self, variant: int):
        _check("mfto_set_kv_variant", lib().mfto_set_kv_variant(self._h, variant), self._h)

    def set_cg_engine(self, engine: int):
        """FP32 inner CG: 1 = one persistent cooperative kernel per solve,
        0 = per-iteration kernels replayed from a CUDA graph."""
        _check("mfto_set_cg_engine", lib().mfto_set_cg_engine(self._h, engine), self._h)

    def set_projection(self, beta: float, eta: float = 0.5):
        _check("mfto_set_projection", lib().mfto_set_projection(self._h, beta, eta), self._h)

    def project(self, rho_bar, rho_phys=None, dc=None):
        import torch
        _check("mfto_project", lib().mfto_project(
            self._h, _ptr(rho_bar, torch.float64, self.n_elem, "rho_bar"),
            _ptr(rho_phys, torch.float64, self.n_elem, "rho_phys") if rho_phys is not None else None,
            _ptr(dc, torch.float64, self.n_elem, "dc") if dc is not None else None), self._h)

    def simp_protocol(self, rho, u, f, rho_selected, params):
        """The SIMP-120 continuation protocol; returns (stats, compliance,
        grayness, restarted) with the per-iteration host histories."""
        import torch
        n = params.n_iter
        comp = np.zeros(n)
        gray = np.zeros(n)
        rest = np.zeros(n, dtype=np.int32)
        st = ProtocolStats()
        _check("mfto_simp_protocol", lib().mfto_simp_protocol(
            self._h, _ptr(rho, torch.float64, self.n_elem, "rho"),
            _ptr(u, torch.float64, self.n_dof, "u"), _ptr(f, torch.float64, self.n_dof, "f"),
            _ptr(rho_selected, torch.float64, self.n_elem, "rho_selected"), C.byref(params),
            comp.ctypes.data, gray.ctypes.data, rest.ctypes.data, C.byref(st)), self._h)
        return st, comp, gray, rest

    def kappa(self, E, v_power, v_inverse, params=None) -> KappaStats:
        """Condition-number estimate of K(E) on the free DOFs; v_power and
        v_inverse (FP64 device vectors, seeded by the caller) are overwritten
        with the final unit iterates."""
        import torch
        st = KappaStats()
        work = torch.empty(self.n_dof, dtype=torch.float64, device=E.device)
        prm = params if params is not None else default_kappa_params()
        _check("mfto_kappa", lib().mfto_kappa(
            self._h, _ptr(E, torch.float64, self.n_elem, "E"),
            _ptr(v_power, torch.float64, self.n_dof, "v_power"),
            _ptr(v_inverse, torch.float64, self.n_dof, "v_inverse"),
            _ptr(work, torch.float64, self.n_dof, "work"), C.byref(prm), C.byref(st)), self._h)
        return st

    def device_bytes(self) -> int:
        """Device memory the handle holds (workspace and optional parts)."""
        n = C.c_int64()
        _check("mfto_device_bytes", lib().mfto_device_bytes(self._h, C.byref(n)), self._h)
        return n.value

    # ---- geometric multigrid
    def gmg_setup(self, E, params=None):
        import torch
        _check("mfto_gmg_setup", lib().mfto_gmg_setup(
            self._h, _ptr(E, torch.float64, self.n_elem, "E"),
            C.byref(params) if params is not None else None), self._h)

    def gmg_params_in_use(self) -> GmgParams:
        """The last setup's parameters with its automatic choices resolved."""
        p = GmgParams()
        _check("mfto_gmg_params_in_use", lib().mfto_gmg_params_in_use(self._h, C.byref(p)),
               self._h)
        return p

    def gmg_levels(self):
        n = C.c_int32()
        dims = np.zeros(3 * GMG_MAX_LEVELS, dtype=np.int32)
        _check("mfto_gmg_levels", lib().mfto_gmg_levels(self._h, C.byref(n), dims.ctypes.data),
               self._h)
        return [tuple(int(x) for x in dims[3 * l:3 * l + 3]) for l in range(n.value)]

    def gmg_apply(self, level, x, y):
        import torch
        _check("mfto_gmg_apply", lib().mfto_gmg_apply(
            self._h, level, _ptr(x, torch.float32, None, "x"), _ptr(y, torch.float32, None, "y")),
            self._h)

    def gmg_vcycle(self, r, z):
        import torch
        _check("mfto_gmg_vcycle", lib().mfto_gmg_vcycle(
            self._h, _ptr(r, torch.float32, self.n_dof, "r"), _ptr(z, torch.float32, self.n_dof, "z")),
            self._h)

    def gmg_solve(self, E, f, u) -> SolveStats:
        import torch
        st = SolveStats()
        _check("mfto_gmg_solve", lib().mfto_gmg_solve(
            self._h, _ptr(E, torch.float64, self.n_elem, "E"),
            _ptr(f, torch.float64, self.n_dof, "f"), _ptr(u, torch.float64, self.n_dof, "u"),
            C.byref(st)), self._h)
        return st

    def gmg_solve_multi(self, E, F, U, nrhs):
        """nrhs load cases (F, U: [nrhs * n_dof] FP64) on one hierarchy."""
        import torch
        st = (SolveStats * nrhs)()
        _check("mfto_gmg_solve_multi", lib().mfto_gmg_solve_multi(
            self._h, _ptr(E, torch.float64, self.n_elem, "E"),
            _ptr(F, torch.float64, nrhs * self.n_dof, "F"),
            _ptr(U, torch.float64, nrhs * self.n_dof, "U"), nrhs, st), self._h)
        return list(st)

    def set_gmg_solver(self, on=True, params=None):
        _check("mfto_set_gmg_solver", lib().mfto_set_gmg_solver(
            self._h, 1 if on else 0, C.byref(params) if params is not None else None), self._h)

    def set_ir_mode(self, mode: int):
        """IR_RESTART (0): each inner CG starts with p = z; IR_CONTINUE (1): it
        keeps the previous search direction (reliable updating)."""
        _check("mfto_set_ir_mode", lib().mfto_set_ir_mode(self._h, mode), self._h)

    def set_kv_shape(self, nzc: int, kind: int):
        """Pin the FP32 column K.v launch shape (nzc 0 = automatic, kind 0 or 1)."""
        _check("mfto_set_kv_shape", lib().mfto_set_kv_shape(self._h, nzc, kind), self._h)

    def kv_autotune(self):
        """Pick the fastest z-chunk and kernel kind of the FP32 column K.v;
        returns (nzc, kind, us)."""
        n, mb, us = C.c_int32(), C.c_int32(), C.c_float()
        _check("mfto_kv_autotune", lib().mfto_kv_autotune(self._h, C.byref(n), C.byref(mb),
                                                          C.byref(us)), self._h)
        return n.value, mb.value, us.value

    def jacobi_diag(self, E, d, form=FORM_F64):
        dt = self._dt(form)
        _check("mfto_jacobi_diag", lib().mfto_jacobi_diag(
            self._h, form, _ptr(E, dt, self.n_elem, "E"), _ptr(d, dt, self.n_dof, "diag")),
            self._h)

    def pcg(self, E, f, u) -> SolveStats:
        import torch
        st = SolveStats()
        _check("mfto_pcg", lib().mfto_pcg(
            self._h, _ptr(E, torch.float64, self.n_elem, "E"),
            _ptr(f, torch.float64, self.n_dof, "f"), _ptr(u, torch.float64, self.n_dof, "u"),
            C.byref(st)), self._h)
        return st

    def ir_solve(self, E, f, u, inner=FORM_F32, inner_tol=1e-2) -> IrStats:
        import torch
        st = IrStats()
        _check("mfto_ir_solve", lib().mfto_ir_solve(
            self._h, inner, inner_tol, _ptr(E, torch.float64, self.n_elem, "E"),
            _ptr(f, torch.float64, self.n_dof, "f"), _ptr(u, torch.float64, self.n_dof, "u"),
            C.byref(st)), self._h)
        return st

    def kv_multi(self, E, V, Y, nrhs, form=FORM_F64):
        dt = self._dt(form)
        _check("mfto_kv_multi", lib().mfto_kv_multi(
            self._h, form, _ptr(E, dt, self.n_elem, "E"), _ptr(V, dt, nrhs * self.n_dof, "V"),
            _ptr(Y, dt, nrhs * self.n_dof, "Y"), nrhs), self._h)

    def ir_solve_multi(self, E, F, U, nrhs, inner_tol=1e-2):
        import torch
        st = (IrStats * nrhs)()
        _check("mfto_ir_solve_multi", lib().mfto_ir_solve_multi(
            self._h, inner_tol, _ptr(E, torch.float64, self.n_elem, "E"),
            _ptr(F, torch.float64, nrhs * self.n_dof, "F"),
            _ptr(U, torch.float64, nrhs * self.n_dof, "U"), nrhs, st), self._h)
        return list(st)

    def set_solver(self, form=FORM_F64, inner_tol=1e-2, inner_maxit=10000, max_outer=50):
        _check("mfto_set_solver", lib().mfto_set_solver(self._h, form, inner_tol, inner_maxit,
                                                        max_outer), self._h)

    def filter(self, x, y, transpose=False):
        import torch
        _check("mfto_filter", lib().mfto_filter(
            self._h, _ptr(x, torch.float64, self.n_elem, "x"),
            _ptr(y, torch.float64, self.n_elem, "y"), 1 if transpose else 0), self._h)

    def compliance_sens(self, rho_phys, u, dc=None) -> float:
        import torch
        c = C.c_double()
        _check("mfto_compliance_sens", lib().mfto_compliance_sens(
            self._h, _ptr(rho_phys, torch.float64, self.n_elem, "rho_phys"),
            _ptr(u, torch.float64, self.n_dof, "u"), C.byref(c),
            _ptr(dc, torch.float64, self.n_elem, "dc")), self._h)
        return c.value

    def oc_update(self, rho, dc, rho_new) -> IterStats:
        import torch
        st = IterStats()
        _check("mfto_oc_update", lib().mfto_oc_update(
            self._h, _ptr(rho, torch.float64, self.n_elem, "rho"),
            _ptr(dc, torch.float64, self.n_elem, "dc"),
            _ptr(rho_new, torch.float64, self.n_elem, "rho_new"), C.byref(st)), self._h)
        return st

    def simp_step(self, rho, u, f, rho_phys=None) -> IterStats:
        import torch
        st = IterStats()
        _check("mfto_simp_step", lib().mfto_simp_step(
            self._h, _ptr(rho, torch.float64, self.n_elem, "rho"),
            _ptr(u, torch.float64, self.n_dof, "u"), _ptr(f, torch.float64, self.n_dof, "f"),
            _ptr(rho_phys, torch.float64, self.n_elem, "rho_phys"), C.byref(st)), self._h)
        return st

    # ---- timing
    def launch_count(self) -> int:
        n = C.c_int64()
        _check("mfto_launch_count", lib().mfto_launch_count(self._h, C.byref(n)), self._h)
        return n.value

    def kv_timing(self, on: bool):
        _check("mfto_kv_timing", lib().mfto_kv_timing(self._h, 1 if on else 0), self._h)

    def kv_timing_read(self, form=FORM_F64):
        n, ms = C.c_int64(), C.c_double()
        _check("mfto_kv_timing_read",
               lib().mfto_kv_timing_read(self._h, form, C.byref(n), C.byref(ms)), self._h)
        return n.value, ms.value

    def cg_timing_read(self):
        """(launches, CG iterations, device ms) of the timed persistent CG launches."""
        n, it, ms = C.c_int64(), C.c_int64(), C.c_double()
        _check("mfto_cg_timing_read",
               lib().mfto_cg_timing_read(self._h, C.byref(n), C.byref(it), C.byref(ms)), self._h)
        return n.value, it.value, ms.value

    def cg_kv_time(self, launches=64, reps=5, events=False):
        """Microseconds per launch of the FP32 CG K.v, timed over a graph of
        back-to-back launches (mfto_cg_kv_time; overwrites the FP32 work
        vectors); with events, the mean interval between event nodes placed
        around every launch of that graph."""
        us = C.c_double()
        _check("mfto_cg_kv_time",
               lib().mfto_cg_kv_time(self._h, launches, reps, int(bool(events)), C.byref(us)),
               self._h)
        return us.value

    # ---- learned part
    def nn_grid(self, levels=4):
        return nn_grid(self.mesh.nelx, self.mesh.nely, self.mesh.nelz, levels)

    def _vox(self, levels):
        D, H, W = self.nn_grid(levels)
        return D * H * W

    def nn_features(self, rho_phys, load, x, levels=4):
        import torch
        _check("mfto_nn_features", lib().mfto_nn_features(
            self._h, levels, _ptr(rho_phys, torch.float64, self.n_elem, "rho_phys"),
            _ptr(load, torch.float64, self.n_dof, "load"),
            _ptr(x, torch.float32, 4 * self._vox(levels), "x")), self._h)

    def nn_target(self, u, y, mask, levels=4):
        import torch
        V = self._vox(levels)
        _check("mfto_nn_target", lib().mfto_nn_target(
            self._h, levels, _ptr(u, torch.float64, self.n_dof, "u"),
            _ptr(y, torch.float32, 3 * V, "y"), _ptr(mask, torch.float32, 3 * V, "mask")),
            self._h)

    def nn_to_dofs(self, y, c, levels=4):
        import torch
        _check("mfto_nn_to_dofs", lib().mfto_nn_to_dofs(
            self._h, levels, _ptr(y, torch.float32, 3 * self._vox(levels), "y"),
            _ptr(c, torch.float64, self.n_dof, "c")), self._h)

    def nn_sample(self, E, rho_phys, f, u_star, k_iters, x, y, mask, levels=4):
        import torch
        V = self._vox(levels)
        _check("mfto_nn_sample", lib().mfto_nn_sample(
            self._h, levels, _ptr(E, torch.float64, self.n_elem, "E"),
            _ptr(rho_phys, torch.float64, self.n_elem, "rho_phys"),
            _ptr(f, torch.float64, self.n_dof, "f"), _ptr(u_star, torch.float64, self.n_dof, "u"),
            k_iters, _ptr(x, torch.float32, 4 * V, "x"), _ptr(y, torch.float32, 3 * V, "y"),
            _ptr(mask, torch.float32, 3 * V, "mask")), self._h)

    def nn_train_energy(self, net, E, rho_phys, f, compliance, lr=1e-3, want_loss=True):
        import torch
        loss = C.c_double()
        _check("mfto_nn_train_energy", lib().mfto_nn_train_energy(
            self._h, net._n, _ptr(E, torch.float64, self.n_elem, "E"),
            _ptr(rho_phys, torch.float64, self.n_elem, "rho_phys"),
            _ptr(f, torch.float64, self.n_dof, "f"), compliance, lr,
            C.byref(loss) if want_loss else None), self._h)
        return loss.value if want_loss else None

    def set_learned(self, net, every=0):
        self._net = net   # keep the network alive while attached
        _check("mfto_set_learned", lib().mfto_set_learned(
            self._h, net._n if net is not None else None, every), self._h)

    def learned_solve(self, E, rho_phys, f, u) -> LearnedStats:
        import torch
        st = LearnedStats()
        _check("mfto_learned_solve", lib().mfto_learned_solve(
            self._h, _ptr(E, torch.float64, self.n_elem, "E"),
            _ptr(rho_phys, torch.float64, self.n_elem, "rho_phys"),
            _ptr(f, torch.float64, self.n_dof, "f"), _ptr(u, torch.float64, self.n_dof, "u"),
            C.byref(st)), self._h)
        return st


def nn_grid(nelx, nely, nelz, levels=4):
    dims = np.zeros(3, dtype=np.int32)
    m = Mesh(nelx, nely, nelz, 1.0)
    _check("mfto_nn_grid", lib().mfto_nn_grid(C.byref(m), levels, dims.ctypes.data))
    return tuple(int(d) for d in dims)


class Net:
    """Owns one mfto_nn (the U-Net of the learned solve)."""

    def __init__(self, base=14, levels=4, max_voxels=1, max_train_voxels=0, seed=0, stream=None):
        import torch
        self.base, self.levels = base, levels
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        np_ = C.c_void_p()
        _check("mfto_nn_create", lib().mfto_nn_create(
            base, levels, int(max_voxels), int(max_train_voxels), seed,
            C.c_void_p(self.stream.cuda_stream), C.byref(np_)))
        self._n = np_
        cnt = C.c_int64()
        self._chk("mfto_nn_num_params", lib().mfto_nn_num_params(self._n, C.byref(cnt)))
        self.num_params = cnt.value

    def _chk(self, fn, code):
        if code != OK:
            raw = lib().mfto_nn_last_error(self._n) if getattr(self, "_n", None) else b""
            raise MftoError(fn, code, raw.decode() if raw else "")

    def close(self):
        if getattr(self, "_n", None):
            lib().mfto_nn_destroy(self._n)
            self._n = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.num_params, dtype=np.float32)
        self._chk("mfto_nn_get_params", lib().mfto_nn_get_params(self._n, out.ctypes.data))
        return out

    def set_params(self, params):
        params = np.ascontiguousarray(params, dtype=np.float32)
        if params.size != self.num_params:
            raise ValueError(f"expected {self.num_params} parameters, got {params.size}")
        self._chk("mfto_nn_set_params", lib().mfto_nn_set_params(self._n, params.ctypes.data))

    def set_tensor_cores(self, on: bool):
        """3x3x3 convolutions of the forward pass on tcgen05 (True, default)
        or on the FP32 FMA pipe (False)."""
        self._chk("mfto_nn_set_tensor_cores", lib().mfto_nn_set_tensor_cores(self._n, int(bool(on))))

    def tc_gave_up(self) -> bool:
        """True if a tensor-core convolution gave up waiting for its MMAs."""
        v = C.c_int32()
        self._chk("mfto_nn_tc_status", lib().mfto_nn_tc_status(self._n, C.byref(v)))
        return bool(v.value)

    def forward(self, x, out, dims):
        import torch
        D, H, W = dims
        V = D * H * W
        self._chk("mfto_nn_forward", lib().mfto_nn_forward(
            self._n, D, H, W, _ptr(x, torch.float32, 4 * V, "x"),
            _ptr(out, torch.float32, 3 * V, "out")))

    def gradient(self, x, target, mask, dims):
        """(loss, gradient as a float32 numpy vector)"""
        import torch
        D, H, W = dims
        V = D * H * W
        loss = C.c_double()
        g = np.zeros(self.num_params, dtype=np.float32)
        self._chk("mfto_nn_gradient", lib().mfto_nn_gradient(
            self._n, D, H, W, _ptr(x, torch.float32, 4 * V, "x"),
            _ptr(target, torch.float32, 3 * V, "target"), _ptr(mask, torch.float32, 3 * V, "mask"),
            C.byref(loss), g.ctypes.data))
        return loss.value, g

    def train_step(self, x, target, mask, dims, lr=1e-3, want_loss=True):
        import torch
        D, H, W = dims
        V = D * H * W
        loss = C.c_double()
        self._chk("mfto_nn_train_step", lib().mfto_nn_train_step(
            self._n, D, H, W, _ptr(x, torch.float32, 4 * V, "x"),
            _ptr(target, torch.float32, 3 * V, "target"), _ptr(mask, torch.float32, 3 * V, "mask"),
            lr, C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def launch_count(self):
        n = C.c_int64()
        self._chk("mfto_nn_launch_count", lib().mfto_nn_launch_count(self._n, C.byref(n)))
        return n.value


EBE_STAGED_F64, EBE_FUSED_F64, EBE_FUSED_F32 = 0, 1, 2


class Ebe:
    """Owns one mfto_ebe: K.v over an arbitrary element DOF table (int32
    [n_elem, 24]), staged FP64 or fused FP64 / FP32, with atomic scatter."""

    def __init__(self, n_elem, n_dof, KE=None, stream=None):
        import torch
        self.n_elem, self.n_dof = int(n_elem), int(n_dof)
        ke = np.ascontiguousarray(unit_ke() if KE is None else np.asarray(KE, np.float64))
        assert ke.shape == (24, 24)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ep = C.c_void_p()
        _check("mfto_ebe_create", lib().mfto_ebe_create(self.n_elem, self.n_dof, ke.ctypes.data,
                                                        C.c_void_p(self.stream.cuda_stream),
                                                        C.byref(ep)))
        self._e = ep

    def _chk(self, fn, code):
        if code != OK:
            raw = lib().mfto_ebe_last_error(self._e) if getattr(self, "_e", None) else b""
            raise MftoError(fn, code, raw.decode() if raw else "")

    def kv(self, variant, edof, E, v, y, timed=False):
        """y = K(E) v; with timed=True returns the device times in ms
        ([gather, contraction, scatter] staged, [total] fused)."""
        import torch
        dt = torch.float32 if variant == EBE_FUSED_F32 else torch.float64
        ms = np.zeros(3, dtype=np.float32)
        self._chk("mfto_ebe_kv", lib().mfto_ebe_kv(
            self._e, variant, _ptr(edof, torch.int32, 24 * self.n_elem, "edof"),
            _ptr(E, dt, self.n_elem, "E"), _ptr(v, dt, self.n_dof, "v"),
            _ptr(y, dt, self.n_dof, "y"), ms.ctypes.data if timed else None))
        if timed:
            return [float(x) for x in (ms if variant == EBE_STAGED_F64 else ms[:1])]
        return None

    def launch_count(self):
        n = C.c_int64()
        self._chk("mfto_ebe_launch_count", lib().mfto_ebe_launch_count(self._e, C.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "_e", None):
            lib().mfto_ebe_destroy(self._e)
            self._e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Owns one mfto_batch: many independent meshes solved together."""

    def __init__(self, meshes, fixed_masks, params: Params | None = None, h=1.0, stream=None):
        import torch
        self.count = len(meshes)
        self.meshes = (Mesh * self.count)(*[Mesh(a, b, c, h) for (a, b, c) in meshes])
        self.params = params if params is not None else default_params()
        fixed = np.ascontiguousarray(np.concatenate([np.asarray(f, np.uint8) for f in fixed_masks]))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        bp = C.c_void_p()
        code = lib().mfto_batch_create(self.count, self.meshes, C.byref(self.params),
                                       fixed.ctypes.data, C.c_void_p(self.stream.cuda_stream),
                                       C.byref(bp))
        _check("mfto_batch_create", code)
        self._b = bp
        eo = np.zeros(self.count + 1, dtype=np.int64)
        do = np.zeros(self.count + 1, dtype=np.int64)
        self._chk("mfto_batch_layout", lib().mfto_batch_layout(self._b, eo.ctypes.data,
                                                               do.ctypes.data))
        self.elem_off, self.dof_off = eo, do
        self.n_elem, self.n_dof = int(eo[-1]), int(do[-1])

    def _chk(self, fn, code):
        if code != OK:
            raw = lib().mfto_batch_last_error(self._b) if getattr(self, "_b", None) else b""
            raise MftoError(fn, code, raw.decode() if raw else "")

    def close(self):
        if getattr(self, "_b", None):
            lib().mfto_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def kv(self, E, V, Y, form=FORM_F64):
        import torch
        dt = torch.float64 if form == FORM_F64 else torch.float32
        self._chk("mfto_batch_kv", lib().mfto_batch_kv(
            self._b, form, _ptr(E, dt, self.n_elem, "E"), _ptr(V, dt, self.n_dof, "V"),
            _ptr(Y, dt, self.n_dof, "Y")))

    def autotune(self, reps=5):
        ms = np.zeros(4)
        ch = C.c_int32()
        self._chk("mfto_batch_autotune", lib().mfto_batch_autotune(self._b, reps, ms.ctypes.data,
                                                                   C.byref(ch)))
        return ch.value, ms

    def set_shape(self, shape):
        self._chk("mfto_batch_set_shape", lib().mfto_batch_set_shape(self._b, shape))

    def solve(self, E, F, U, inner_tol=1e-2, inner_maxit=10000, max_outer=50):
        import torch
        st = (IrStats * self.count)()
        self._chk("mfto_batch_solve", lib().mfto_batch_solve(
            self._b, inner_tol, _ptr(E, torch.float64, self.n_elem, "E"),
            _ptr(F, torch.float64, self.n_dof, "F"), _ptr(U, torch.float64, self.n_dof, "U"),
            inner_maxit, max_outer, st))
        return list(st)

    def set_ir_mode(self, mode):
        self._chk("mfto_batch_set_ir_mode", lib().mfto_batch_set_ir_mode(self._b, mode))

    def launch_count(self):
        n = C.c_int64()
        self._chk("mfto_batch_launch_count", lib().mfto_batch_launch_count(self._b, C.byref(n)))
        return n.value
