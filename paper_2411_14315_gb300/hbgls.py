"""Thin Python binding of libhbgls (the C ABI declared in include/hbgls.h).

Argument marshalling only: every step of the method runs in the library's CUDA kernels.  Importing
this module does not load the library; the first call does, and raises if libhbgls.so has not been
built (there is no fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libhbgls.so")

HB_OK = 0
STATUS = {0: "HB_OK", 1: "HB_ERR_INVALID_ARG", 2: "HB_ERR_MESH", 3: "HB_ERR_CUDA", 4: "HB_ERR_OOM",
          5: "HB_ERR_NOT_CONVERGED", 6: "HB_ERR_NAN", 7: "HB_ERR_TIMEOUT", 8: "HB_ERR_STATE"}

PAPER, EXACT, ASSEMBLED = 0, 1, 2
FP64, FP32 = 0, 1


class HBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class hb_mesh(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_tets", C.c_int64), ("n_faces", C.c_int64),
                ("xyz", C.POINTER(C.c_double)), ("tets", C.POINTER(C.c_int32)),
                ("faces", C.POINTER(C.c_int32)), ("face_tag", C.POINTER(C.c_int32))]


class hb_solve_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("rtol", C.c_double), ("switch_rtol", C.c_double),
                ("gmres_rtol_pseudo", C.c_double), ("gmres_rtol_newton", C.c_double),
                ("gmres_restart", C.c_int), ("max_gmres", C.c_int), ("max_steps", C.c_int),
                ("dt_pseudo", C.c_double), ("cfl", C.c_double), ("use_learned", C.c_int),
                ("verbose", C.c_int), ("ser", C.c_int), ("ser_max", C.c_double), ("r_ref", C.c_double),
                ("assembled", C.c_int), ("precond", C.c_int), ("line_search", C.c_int),
                ("scatter", C.c_int), ("backflow_beta", C.c_double)]


class hb_report(C.Structure):
    _fields_ = [("steps", C.c_int), ("newton_steps", C.c_int), ("gmres_iters", C.c_int),
                ("jv_calls", C.c_int), ("residual_calls", C.c_int), ("res0", C.c_double),
                ("res_final", C.c_double), ("seconds", C.c_double), ("dt_pseudo", C.c_double),
                ("status", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hb_march_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("steps_per_period", C.c_int), ("periods", C.c_int),
                ("rho_inf", C.c_double), ("newton_rtol", C.c_double), ("newton_max", C.c_int),
                ("gmres_rtol", C.c_double), ("gmres_restart", C.c_int), ("max_gmres", C.c_int),
                ("tau_acceleration", C.c_int), ("verbose", C.c_int)]


class hb_march_report(C.Structure):
    _fields_ = [("steps", C.c_int), ("newton_iters", C.c_int), ("gmres_iters", C.c_int), ("jv_calls", C.c_int),
                ("seconds", C.c_double), ("period_change", C.c_double), ("max_newton_rel", C.c_double),
                ("status", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hb_info(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_tets", C.c_int64), ("n_faces", C.c_int64),
                ("n_dirichlet_nodes", C.c_int64), ("n_neumann_faces", C.c_int64), ("n_h", C.c_int),
                ("N", C.c_int), ("n_patches32", C.c_int), ("n_patches64", C.c_int),
                ("patch_nodes_max32", C.c_int), ("patch_elems_max32", C.c_int),
                ("device_bytes", C.c_int64), ("h_char", C.c_double), ("u_ref", C.c_double),
                ("p_ref", C.c_double), ("assembled_pairs", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_DP = C.POINTER(C.c_double)
_VP = C.c_void_p
_P = C.c_void_p
# name -> (argtypes, restype); every entry point declared in include/hbgls.h
SIGNATURES = {
    "hb_create": ([C.POINTER(hb_mesh), C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, _VP,
                   C.POINTER(_P)], C.c_int),
    "hb_destroy": ([_P], C.c_int),
    "hb_last_error": ([], C.c_char_p),
    "hb_set_inflow": ([_P, C.c_int, _DP, _DP, _DP], C.c_int),
    "hb_set_outlet_pressure": ([_P, C.c_int, _DP, _DP], C.c_int),
    "hb_set_inflow_harmonics": ([_P, C.c_int, _DP], C.c_int),
    "hb_set_outlet_resistance": ([_P, C.c_int, C.c_double, _DP, _DP], C.c_int),
    "hb_set_backflow": ([_P, C.c_double], C.c_int),
    "hb_set_stabilization": ([_P, C.c_int, C.c_double], C.c_int),
    "hb_set_initial": ([_P, _DP], C.c_int),
    "hb_set_instances": ([_P, _DP], C.c_int),
    "hb_default_opts": ([C.POINTER(hb_solve_opts)], C.c_int),
    "hb_solve": ([_P, C.POINTER(hb_solve_opts), C.POINTER(hb_report)], C.c_int),
    "hb_get_harmonics": ([_P, _DP], C.c_int),
    "hb_get_instances": ([_P, _DP], C.c_int),
    "hb_default_march_opts": ([C.POINTER(hb_march_opts)], C.c_int),
    "hb_march": ([_P, C.POINTER(hb_march_opts), C.POINTER(hb_march_report)], C.c_int),
    "hb_get_march_samples": ([_P, _DP], C.c_int),
    "hb_assemble_dev": ([_P, _VP, C.c_int, _VP], C.c_int),
    "hb_time_residual": ([_P, _DP, _DP, _DP, C.c_int, C.c_double, C.c_double], C.c_int),
    "hb_time_jv": ([_P, _DP, _DP, _DP, C.c_int, C.c_double, C.c_double], C.c_int),
    "hb_residual": ([_P, _DP, _DP, C.c_int], C.c_int),
    "hb_jv": ([_P, _DP, _DP, _DP, C.c_int, C.c_int, C.c_double], C.c_int),
    "hb_jacobi_diag": ([_P, _DP, _DP, C.c_int, C.c_double], C.c_int),
    "hb_jv_f32": ([_P, C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_int, C.c_double],
                  C.c_int),
    "hb_residual_dev": ([_P, _VP, _VP, C.c_int, _VP], C.c_int),
    "hb_jv_dev": ([_P, _VP, _VP, _VP, C.c_int, C.c_int, C.c_double, _VP], C.c_int),
    "hb_jacobi_diag_dev": ([_P, _VP, _VP, C.c_int, C.c_double, _VP], C.c_int),
    "hb_get_info": ([_P, C.POINTER(hb_info)], C.c_int),
    "hb_launch_count": ([_P], C.c_int64),
    "hb_set_launch_variant": ([_P, C.c_int], C.c_int),
    "hb_get_launch_variant": ([_P], C.c_int),
    "hb_set_spectral_path": ([_P, C.c_int], C.c_int),
    "hb_get_spectral_path": ([_P], C.c_int),
    "hb_set_scatter": ([_P, C.c_int], C.c_int),
    "hb_get_scatter": ([_P], C.c_int),
    "hb_profile_elem": ([_P, C.c_int], C.c_int),
    "hb_profile_read": ([_P, C.POINTER(C.c_double), C.POINTER(C.c_int64)], C.c_int),
    "hb_jv_dev_noalloc": ([_P, _VP, _VP, _VP, C.c_int, C.c_int, C.c_double, _VP], C.c_int),
    "hb_mpnn_create": ([C.c_void_p, C.c_int, C.POINTER(_P)], C.c_int),
    "hb_mpnn_destroy": ([_P], C.c_int),
    "hb_mpnn_set_tensor_cores": ([_P, C.c_int], C.c_int),
    "hb_mpnn_num_params": ([_P], C.c_int64),
    "hb_mpnn_get_params": ([_P, C.POINTER(C.c_float)], C.c_int),
    "hb_mpnn_set_params": ([_P, C.POINTER(C.c_float)], C.c_int),
    "hb_mpnn_loss_grad": ([_P, _P, _DP, C.POINTER(C.c_float), C.POINTER(C.c_float)], C.c_int),
    "hb_mpnn_train_step": ([_P, _P, _DP, C.c_float, C.POINTER(C.c_float)], C.c_int),
    "hb_mpnn_predict": ([_P, _P, _DP], C.c_int),
    "hb_mpnn_graph": ([_P, _P, C.POINTER(C.c_float), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                       C.POINTER(C.c_float), C.POINTER(C.c_int64)], C.c_int),
    "hb_mpnn_warm_start": ([_P, _P], C.c_int),
    "hb_attach_learned": ([_P, _P], C.c_int),
    "hb_batch_create": ([C.POINTER(_P), C.c_int, C.c_int, C.POINTER(_P)], C.c_int),
    "hb_batch_destroy": ([_P], C.c_int),
    "hb_batch_jv_dev": ([_P, C.POINTER(_VP), C.POINTER(_VP), C.POINTER(_VP), C.c_int, C.c_double, _VP], C.c_int),
    "hb_batch_launch_count": ([_P], C.c_int64),
    "hb_batch_set_grouping": ([_P, C.c_int], C.c_int),
    "hb_tune_patches": ([_P, C.c_int, C.POINTER(C.c_int), C.c_int, C.c_int, C.POINTER(C.c_int),
                         C.POINTER(C.c_double)], C.c_int),
}


class hb_mpnn_config(C.Structure):
    _fields_ = [("hidden", C.c_int), ("layers", C.c_int), ("n_h", C.c_int), ("seed", C.c_int),
                ("p_scale", C.c_double)]

_lib = None


def lib():
    """Load libhbgls.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libhbgls.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(st: int):
    if st != HB_OK:
        raise HBError(st, lib().hb_last_error().decode())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != tuple(shape):
        a = a.reshape(shape)
    return a


_CUDA_STREAM_LEGACY = 1     # cudaStreamLegacy: the legacy default stream


def _stream_handle(stream):
    """cudaStream_t of a torch stream (or a raw handle).  A torch stream whose handle is 0 is the legacy
    default stream and is passed as cudaStreamLegacy, because a NULL handle means "the problem's own
    stream" in the C ABI."""
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        h = int(stream.cuda_stream)
        return C.c_void_p(h if h != 0 else _CUDA_STREAM_LEGACY)
    h = int(stream)
    return C.c_void_p(h) if h != 0 else None


class Problem:
    """One HB problem on one device (hb_create .. hb_destroy)."""

    def __init__(self, xyz, tets, faces, face_tag, rho: float, mu: float, T: float, n_h: int,
                 device: int = 0, stream=None):
        self._xyz = _f64(xyz)
        self._tets = np.ascontiguousarray(tets, dtype=np.int32)
        self._faces = np.ascontiguousarray(faces, dtype=np.int32)
        self._tag = np.ascontiguousarray(face_tag, dtype=np.int32)
        m = hb_mesh(self._xyz.shape[0], self._tets.shape[0], self._faces.shape[0], _dptr(self._xyz),
                    self._tets.ctypes.data_as(C.POINTER(C.c_int32)),
                    self._faces.ctypes.data_as(C.POINTER(C.c_int32)),
                    self._tag.ctypes.data_as(C.POINTER(C.c_int32)))
        h = _P()
        _check(lib().hb_create(C.byref(m), rho, mu, T, n_h, device, _stream_handle(stream), C.byref(h)))
        self._h = h
        self.rho, self.mu, self.T = float(rho), float(mu), float(T)
        self.n_nodes = int(self._xyz.shape[0])
        self.n_h = int(n_h)
        self.N = 2 * self.n_h + 1
        self.shape = (self.n_nodes, 4, self.N)

    @classmethod
    def from_mesh(cls, mesh, rho, mu, T, n_h, **kw):
        return cls(mesh.xyz, mesh.tets, mesh.faces, mesh.face_tag, rho, mu, T, n_h, **kw)

    @classmethod
    def from_spec(cls, spec, **kw):
        """Create a problem from a workload spec (paper_2411_14315_gb300.workloads.Spec)."""
        m = spec.mesh
        p = cls(m.xyz, m.tets, m.faces, spec.face_tag, spec.rho, spec.mu, spec.T, spec.n_h, **kw)
        p.set_backflow(spec.beta)
        for tag, prof, a, b in spec.inflows:
            p.set_inflow(tag, prof, a, b)
        for tag, harm in getattr(spec, "inflows_harm", []):
            p.set_inflow_harmonics(tag, harm)
        for tag, a, b in spec.outlets_p:
            p.set_outlet_pressure(tag, a, b)
        for tag, R, a, b in spec.outlets_r:
            p.set_outlet_resistance(tag, R, a, b)
        return p

    def close(self):
        if getattr(self, "_h", None):
            lib().hb_destroy(self._h)
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

    # boundary conditions -------------------------------------------------------------------------
    def _wave(self, a, b):
        a = _f64(a)
        b = _f64(b)
        if a.shape != (self.n_h + 1,) or b.shape != (self.n_h + 1,):
            raise ValueError("waveform arrays need n_h + 1 entries")
        return a, b

    def set_inflow(self, tag: int, profile, a, b):
        a, b = self._wave(a, b)
        prof = None if profile is None else _f64(profile, (self.n_nodes, 3))
        _check(lib().hb_set_inflow(self._h, tag, None if prof is None else _dptr(prof), _dptr(a), _dptr(b)))

    def set_inflow_harmonics(self, tag: int, harmonics):
        h = _f64(harmonics, (self.n_nodes, 3, 2 * self.n_h + 1))
        _check(lib().hb_set_inflow_harmonics(self._h, tag, _dptr(h)))

    def set_outlet_pressure(self, tag: int, a, b):
        a, b = self._wave(a, b)
        _check(lib().hb_set_outlet_pressure(self._h, tag, _dptr(a), _dptr(b)))

    def set_outlet_resistance(self, tag: int, R: float, a, b):
        a, b = self._wave(a, b)
        _check(lib().hb_set_outlet_resistance(self._h, tag, R, _dptr(a), _dptr(b)))

    def set_backflow(self, beta: float):
        _check(lib().hb_set_backflow(self._h, beta))

    def set_stabilization(self, variant: int = 0, ct_dt: float = 0.0):
        """hb_set_stabilization: 0 = GLS as printed, 1 = full RBVMS; ct_dt (1/dt)^2 under the root of tau."""
        _check(lib().hb_set_stabilization(self._h, int(variant), float(ct_dt)))

    def set_initial(self, harmonics=None):
        hm = None if harmonics is None else _f64(harmonics, (self.n_nodes, 4, 2 * self.n_h + 1))
        _check(lib().hb_set_initial(self._h, None if hm is None else _dptr(hm)))

    def set_instances(self, y=None):
        yy = None if y is None else _f64(y, self.shape)
        _check(lib().hb_set_instances(self._h, None if yy is None else _dptr(yy)))

    # hot path, host buffers ------------------------------------------------------------------------
    def residual(self, y, precision: int = FP64):
        y = _f64(y, self.shape)
        r = np.empty(self.shape)
        _check(lib().hb_residual(self._h, _dptr(y), _dptr(r), precision))
        return r

    def jv(self, y, v, kind: int = PAPER, precision: int = FP64, shift: float = 0.0, out=None):
        y = _f64(y, self.shape)
        v = _f64(v, self.shape)
        r = np.empty(self.shape) if out is None else out
        _check(lib().hb_jv(self._h, _dptr(y), _dptr(v), _dptr(r), kind, precision, shift))
        return r

    def jv_f32(self, y, v, kind: int = PAPER, shift: float = 0.0, out=None):
        """hb_jv_f32: FP32 host buffers in and out (FP32 kernels)."""
        y = np.ascontiguousarray(y, dtype=np.float32).reshape(self.shape)
        v = np.ascontiguousarray(v, dtype=np.float32).reshape(self.shape)
        r = np.empty(self.shape, dtype=np.float32) if out is None else out
        fp = C.POINTER(C.c_float)
        _check(lib().hb_jv_f32(self._h, y.ctypes.data_as(fp), v.ctypes.data_as(fp), r.ctypes.data_as(fp), kind,
                               shift))
        return r

    def jacobi_diag(self, y, precision: int = FP64, shift: float = 0.0):
        y = _f64(y, self.shape)
        d = np.empty(self.shape)
        _check(lib().hb_jacobi_diag(self._h, _dptr(y), _dptr(d), precision, shift))
        return d

    # hot path, device buffers (torch tensors of float64 / float32, instance layout) --------------
    def residual_dev(self, y, r, precision: int, stream=None):
        _check(lib().hb_residual_dev(self._h, y.data_ptr(), r.data_ptr(), precision, _stream_handle(stream)))

    def jv_dev(self, y, v, out, kind: int, precision: int, shift: float = 0.0, stream=None):
        _check(lib().hb_jv_dev(self._h, y.data_ptr(), v.data_ptr(), out.data_ptr(), kind, precision, shift,
                               _stream_handle(stream)))

    def assemble_dev(self, y, precision: int, stream=None):
        """Assemble the paper tangent at the device state y (hb_assemble_dev); kind 2 then applies it."""
        _check(lib().hb_assemble_dev(self._h, y.data_ptr(), precision, _stream_handle(stream)))

    def jv_dev_noalloc(self, y, v, out, kind: int, precision: int, shift: float = 0.0, stream=None):
        """hb_jv_dev without any device allocation (see include/hbgls.h for the conditions)."""
        _check(lib().hb_jv_dev_noalloc(self._h, y.data_ptr(), v.data_ptr(), out.data_ptr(), kind, precision,
                                       shift, _stream_handle(stream)))

    def jacobi_diag_dev(self, y, d, precision: int, shift: float = 0.0, stream=None):
        _check(lib().hb_jacobi_diag_dev(self._h, y.data_ptr(), d.data_ptr(), precision, shift,
                                        _stream_handle(stream)))

    # solve -----------------------------------------------------------------------------------------
    @staticmethod
    def default_opts(**kw) -> hb_solve_opts:
        o = hb_solve_opts()
        _check(lib().hb_default_opts(C.byref(o)))
        for k, v in kw.items():
            setattr(o, k, v)
        return o

    def solve(self, opts: hb_solve_opts | None = None, check: bool = True, **kw):
        o = opts if opts is not None else self.default_opts(**kw)
        rep = hb_report()
        st = lib().hb_solve(self._h, C.byref(o), C.byref(rep))
        if check:
            _check(st)
        return rep.as_dict()

    def harmonics(self):
        out = np.empty((self.n_nodes, 4, 2 * self.n_h + 1))
        _check(lib().hb_get_harmonics(self._h, _dptr(out)))
        return out

    def instances(self):
        out = np.empty(self.shape)
        _check(lib().hb_get_instances(self._h, _dptr(out)))
        return out

    def march(self, check: bool = True, **kw):
        """Time-domain march (hb_march); keyword arguments set hb_march_opts fields."""
        o = hb_march_opts()
        _check(lib().hb_default_march_opts(C.byref(o)))
        for k, v in kw.items():
            setattr(o, k, v)
        rep = hb_march_report()
        st = lib().hb_march(self._h, C.byref(o), C.byref(rep))
        if check:
            _check(st)
        return rep.as_dict()

    def time_residual(self, y, ydot, t: float, omega2: float = 0.0, precision: int = 0):
        """Residual of one time level [n_nodes, 4] (hb_time_residual)."""
        y = np.ascontiguousarray(y, dtype=np.float64)
        yd = np.ascontiguousarray(ydot, dtype=np.float64)
        out = np.empty((self.n_nodes, 4))
        _check(lib().hb_time_residual(self._h, _dptr(y), _dptr(yd), _dptr(out), precision, t, omega2))
        return out

    def time_jv(self, y, v, omega2: float = 0.0, shift: float = 0.0, precision: int = 0):
        """Paper tangent of one time level along v [n_nodes, 4] (hb_time_jv)."""
        y = np.ascontiguousarray(y, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.empty((self.n_nodes, 4))
        _check(lib().hb_time_jv(self._h, _dptr(y), _dptr(v), _dptr(out), precision, omega2, shift))
        return out

    def march_samples(self):
        """State of the last march at the N instance times of its last period, [n_nodes, 4, N]."""
        out = np.empty(self.shape)
        _check(lib().hb_get_march_samples(self._h, _dptr(out)))
        return out

    def info(self):
        i = hb_info()
        _check(lib().hb_get_info(self._h, C.byref(i)))
        return i.as_dict()

    def launch_count(self) -> int:
        return int(lib().hb_launch_count(self._h))

    def set_launch_variant(self, variant: int):
        _check(lib().hb_set_launch_variant(self._h, int(variant)))

    def set_spectral_path(self, path: int):
        """hb_set_spectral_path: 0 = tcgen05, 1 = mma.sync, 2 = FP32 FMAs (FP32, N = 9, 13, 21)."""
        _check(lib().hb_set_spectral_path(self._h, int(path)))

    def spectral_path(self) -> int:
        return int(lib().hb_get_spectral_path(self._h))

    def set_scatter(self, scatter: int):
        """hb_set_scatter: 0 = deterministic (per-element slots, fixed-order gather), 1 = atomic."""
        _check(lib().hb_set_scatter(self._h, int(scatter)))

    def scatter(self) -> int:
        return int(lib().hb_get_scatter(self._h))

    def launch_variant(self) -> int:
        return int(lib().hb_get_launch_variant(self._h))

    def tune_patches(self, precision: int, candidates, reps: int = 5):
        """Autotune the element patch node cap; returns (best cap, ms per element pass)."""
        c = (C.c_int * len(candidates))(*[int(x) for x in candidates])
        best = C.c_int()
        ms = C.c_double()
        _check(lib().hb_tune_patches(self._h, precision, c, len(candidates), reps, C.byref(best), C.byref(ms)))
        return best.value, ms.value

    def profile_elem(self, enable: bool):
        _check(lib().hb_profile_elem(self._h, int(bool(enable))))

    def profile_read(self):
        """(total milliseconds, launches) of the element kernel since profiling was enabled / read."""
        ms = C.c_double()
        n = C.c_int64()
        _check(lib().hb_profile_read(self._h, C.byref(ms), C.byref(n)))
        return ms.value, n.value


class MPNN:
    """Learned warm-start network (hb_mpnn_*): message passing over the mesh graph, BF16 weights."""

    F_IN, F_E = 32, 4

    def __init__(self, n_h: int, hidden: int = 64, layers: int = 3, seed: int = 0, device: int = 0,
                 p_scale: float = 1.0):
        cfg = hb_mpnn_config(hidden, layers, n_h, seed, p_scale)
        h = _P()
        _check(lib().hb_mpnn_create(C.cast(C.pointer(cfg), C.c_void_p), device, C.byref(h)))
        self._h = h
        self.n_h, self.hidden, self.layers = n_h, hidden, layers
        self.f_out = 4 * (2 * n_h + 1)

    def close(self):
        if getattr(self, "_h", None):
            lib().hb_mpnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tensor_cores(self, enable: bool):
        """hb_mpnn_set_tensor_cores: forward MLPs on the tensor cores (True) or on FP32 FMAs (False)."""
        _check(lib().hb_mpnn_set_tensor_cores(self._h, int(bool(enable))))

    @property
    def num_params(self) -> int:
        return int(lib().hb_mpnn_num_params(self._h))

    def get_params(self) -> np.ndarray:
        out = np.empty(self.num_params, dtype=np.float32)
        _check(lib().hb_mpnn_get_params(self._h, out.ctypes.data_as(C.POINTER(C.c_float))))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(lib().hb_mpnn_set_params(self._h, p.ctypes.data_as(C.POINTER(C.c_float))))

    def loss_grad(self, problem: "Problem", target, want_grad: bool = True):
        t = _f64(target)
        loss = C.c_float()
        g = np.empty(self.num_params, dtype=np.float32) if want_grad else None
        _check(lib().hb_mpnn_loss_grad(self._h, problem._h, _dptr(t), C.byref(loss),
                                       g.ctypes.data_as(C.POINTER(C.c_float)) if want_grad else None))
        return loss.value, g

    def train_step(self, problem: "Problem", target, lr: float) -> float:
        t = _f64(target)
        loss = C.c_float()
        _check(lib().hb_mpnn_train_step(self._h, problem._h, _dptr(t), lr, C.byref(loss)))
        return loss.value

    def predict(self, problem: "Problem") -> np.ndarray:
        out = np.empty((problem.n_nodes, 4, 2 * self.n_h + 1))
        _check(lib().hb_mpnn_predict(self._h, problem._h, _dptr(out)))
        return out

    def graph(self, problem: "Problem"):
        ne = C.c_int64()
        _check(lib().hb_mpnn_graph(self._h, problem._h, None, None, None, None, C.byref(ne)))
        n = problem.n_nodes
        x = np.empty((n, self.F_IN), dtype=np.float32)
        src = np.empty(ne.value, dtype=np.int32)
        dst = np.empty(ne.value, dtype=np.int32)
        e = np.empty((ne.value, self.F_E), dtype=np.float32)
        fp = C.POINTER(C.c_float)
        ip = C.POINTER(C.c_int32)
        _check(lib().hb_mpnn_graph(self._h, problem._h, x.ctypes.data_as(fp), src.ctypes.data_as(ip),
                                   dst.ctypes.data_as(ip), e.ctypes.data_as(fp), C.byref(ne)))
        return x, src, dst, e

    def warm_start(self, problem: "Problem"):
        _check(lib().hb_mpnn_warm_start(self._h, problem._h))

    def attach(self, problem: "Problem"):
        _check(lib().hb_attach_learned(problem._h, self._h))


class Batch:
    """Many problems whose operator is applied in one captured graph (hb_batch_*)."""

    def __init__(self, problems, precision: int = FP32):
        self.problems = list(problems)
        arr = (_P * len(self.problems))(*[p._h for p in self.problems])
        h = _P()
        _check(lib().hb_batch_create(arr, len(self.problems), precision, C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().hb_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def jv_dev(self, ys, vs, outs, kind: int, shift: float = 0.0, stream=None):
        n = len(self.problems)
        mk = lambda ts: (_VP * n)(*[t.data_ptr() for t in ts])  # noqa: E731
        _check(lib().hb_batch_jv_dev(self._h, mk(ys), mk(vs), mk(outs), kind, shift, _stream_handle(stream)))

    def launch_count(self) -> int:
        return int(lib().hb_batch_launch_count(self._h))

    def set_grouping(self, grouping: int):
        """hb_batch_set_grouping: 0 = one element launch over every N, 1 = one launch per N, 2 = every
        member's own operator on parallel graph branches."""
        _check(lib().hb_batch_set_grouping(self._h, int(grouping)))
