"""Thin Python binding of libpim (include/pim.h) over ctypes.

Argument marshalling only: every step of the apply runs in the CUDA library.
The functions carry the C names (pim_plan_create, pim_set_points, pim_apply,
pim_apply_adjoint, pim_destroy, ...); `Plan` wraps them for torch tensors or
numpy arrays.  If the library is missing or fails to load, importing works
but every call raises: there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpim.so")

PIM_OK, PIM_ERR_ARG, PIM_ERR_UNSUPPORTED, PIM_ERR_ANOMALY, PIM_ERR_NOT_NEUTRAL, PIM_ERR_OUT_OF_CELL, \
    PIM_ERR_STATE, PIM_ERR_OOM, PIM_ERR_CUDA, PIM_ERR_TIMEOUT, PIM_ERR_DEVICE = range(11)
PIM_FP64, PIM_FP32_MIXED = 0, 1
PIM_CORR_FP64, PIM_CORR_DOUBLE_FLOAT, PIM_CORR_FP32, PIM_CORR_COMPACT = 0, 1, 2, 3

# symbols declared in include/pim.h
EXPORTS = ["pim_options_default", "pim_status_string", "pim_last_error", "pim_plan_create", "pim_set_points",
           "pim_apply", "pim_apply_adjoint", "pim_last_device_status", "pim_plan_info", "pim_set_profiling",
           "pim_stage_times", "pim_stage_name", "pim_position_grad", "pim_position_grad_reuse", "pim_update_positions",
           "pim_apply_noalloc", "pim_set_points_observers", "pim_apply_observers", "pim_apply_observers_adjoint",
           "pim_apply_batched", "pim_debug_copy", "pim_destroy"]
STAGES = ["permute", "spread", "fft", "gather_correct", "far", "apply", "lf_exact", "lf_grid", "corr_multi",
          "lf_tc_gemm"]


class pim_options(ctypes.Structure):
    _fields_ = [("far_n", ctypes.c_int * 3), ("far_p", ctypes.c_int), ("corr_radius", ctypes.c_int),
                ("corr_cube", ctypes.c_int), ("corr_mode", ctypes.c_int),
                ("neutral_tol", ctypes.c_double), ("series_tol", ctypes.c_double), ("mem_cap", ctypes.c_size_t),
                ("autotune", ctypes.c_int), ("with_gradient", ctypes.c_int), ("corr_split", ctypes.c_int),
                ("gather_variant", ctypes.c_int), ("corr_listfree", ctypes.c_int), ("k_imag", ctypes.c_double),
                ("k0_imag", ctypes.c_double * 3), ("lf_tensor_cores", ctypes.c_int)]


class pim_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("nf", ctypes.c_int * 3), ("p", ctypes.c_int), ("pf", ctypes.c_int),
                ("corr_radius", ctypes.c_int), ("precision", ctypes.c_int), ("corr_mode", ctypes.c_int),
                ("periodic_mask", ctypes.c_int), ("near_layers", ctypes.c_int), ("N", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("device_bytes", ctypes.c_size_t), ("plan_ms", ctypes.c_double),
                ("points_ms", ctypes.c_double), ("launches", ctypes.c_int64), ("gather_variant", ctypes.c_int),
                ("gather_variants", ctypes.c_int), ("lf_boxes", ctypes.c_int64), ("lf_points", ctypes.c_int64),
                ("lf_pairs", ctypes.c_int64), ("lf_tc_boxes", ctypes.c_int64)]


class PimError(RuntimeError):
    def __init__(self, status, where, msg=""):
        self.status = status
        name = _lib.pim_status_string(status).decode() if _lib is not None else str(status)
        super().__init__("%s: %s%s" % (where, name, (" (" + msg + ")") if msg else ""))


_lib = None
_load_error = None


def load(path=LIB_PATH):
    """Loads libpim.so and declares the C signatures."""
    global _lib, _load_error
    if _lib is not None:
        return _lib
    try:
        lib = ctypes.CDLL(path)
    except OSError as e:
        _load_error = str(e)
        raise RuntimeError("libpim.so not loadable (%s); build it with __graft_entry__.build()" % e)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.pim_options_default.argtypes = [ctypes.POINTER(pim_options)]
    lib.pim_options_default.restype = None
    lib.pim_status_string.argtypes = [i32]
    lib.pim_status_string.restype = ctypes.c_char_p
    lib.pim_last_error.argtypes = []
    lib.pim_last_error.restype = ctypes.c_char_p
    lib.pim_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(dbl), ctypes.c_uint, dbl,
                                    ctypes.POINTER(dbl), ctypes.POINTER(dbl), i32, i32, i32,
                                    ctypes.POINTER(pim_options), vp]
    lib.pim_plan_create.restype = i32
    lib.pim_set_points.argtypes = [vp, i64, vp]
    lib.pim_set_points.restype = i32
    lib.pim_apply.argtypes = [vp, vp, vp, i32, vp]
    lib.pim_apply.restype = i32
    lib.pim_apply_adjoint.argtypes = [vp, vp, vp, i32, vp]
    lib.pim_apply_adjoint.restype = i32
    lib.pim_last_device_status.argtypes = [vp]
    lib.pim_last_device_status.restype = i32
    lib.pim_plan_info.argtypes = [vp, ctypes.POINTER(pim_info)]
    lib.pim_plan_info.restype = i32
    lib.pim_set_profiling.argtypes = [vp, i32]
    lib.pim_set_profiling.restype = i32
    lib.pim_stage_times.argtypes = [vp, ctypes.POINTER(dbl), i32, ctypes.POINTER(i64)]
    lib.pim_stage_times.restype = i32
    lib.pim_stage_name.argtypes = [i32]
    lib.pim_stage_name.restype = ctypes.c_char_p
    lib.pim_position_grad.argtypes = [vp, vp, vp, vp, i32, vp]
    lib.pim_position_grad.restype = i32
    lib.pim_position_grad_reuse.argtypes = [vp, vp, vp, vp, vp]
    lib.pim_position_grad_reuse.restype = i32
    lib.pim_update_positions.argtypes = [vp, vp]
    lib.pim_update_positions.restype = i32
    lib.pim_set_points_observers.argtypes = [vp, i64, vp, i64, vp]
    lib.pim_set_points_observers.restype = i32
    lib.pim_apply_observers.argtypes = [vp, vp, vp, i32, vp]
    lib.pim_apply_observers.restype = i32
    lib.pim_apply_observers_adjoint.argtypes = [vp, vp, vp, i32, vp]
    lib.pim_apply_observers_adjoint.restype = i32
    lib.pim_apply_batched.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), i32, i32, vp]
    lib.pim_apply_batched.restype = i32
    lib.pim_apply_noalloc.argtypes = [vp, vp, vp, i32, i32, vp]
    lib.pim_apply_noalloc.restype = i32
    lib.pim_debug_copy.argtypes = [vp, i32, vp, ctypes.c_size_t]
    lib.pim_debug_copy.restype = i32
    lib.pim_destroy.argtypes = [vp]
    lib.pim_destroy.restype = None
    _lib = lib
    return lib


def _check(st, where):
    if st != PIM_OK:
        raise PimError(st, where, _lib.pim_last_error().decode())


def _ptr(x):
    """Device or host address of a torch tensor or numpy array (contiguous)."""
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError("expected a torch tensor or numpy array")


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


# ---------------------------------------------------------------------------
# C-named functions
# ---------------------------------------------------------------------------
def pim_options_default():
    lib = load()
    o = pim_options()
    lib.pim_options_default(ctypes.byref(o))
    return o


def pim_plan_create(lattice, periodic_mask, k, k0, h, p, near_layers, prec, opt=None, stream=None):
    lib = load()
    lat = (ctypes.c_double * 9)(*np.asarray(lattice, np.float64).ravel())
    k0a = (ctypes.c_double * 3)(*np.asarray(k0, np.float64))
    ha = (ctypes.c_double * 3)(*np.asarray(h, np.float64))
    out = ctypes.c_void_p()
    st = lib.pim_plan_create(ctypes.byref(out), lat, int(periodic_mask), float(k), k0a, ha, int(p),
                             int(near_layers), int(prec), ctypes.byref(opt) if opt is not None else None,
                             _stream_ptr(stream))
    _check(st, "pim_plan_create")
    return out


def pim_set_points(plan, N, xyz):
    _check(load().pim_set_points(plan, int(N), _ptr(xyz)), "pim_set_points")


def pim_apply(plan, q, u, nrhs=1, stream=None):
    _check(load().pim_apply(plan, _ptr(q), _ptr(u), int(nrhs), _stream_ptr(stream)), "pim_apply")


def pim_apply_adjoint(plan, v, w, nrhs=1, stream=None):
    _check(load().pim_apply_adjoint(plan, _ptr(v), _ptr(w), int(nrhs), _stream_ptr(stream)), "pim_apply_adjoint")


def pim_last_device_status(plan):
    return load().pim_last_device_status(plan)


def pim_plan_info(plan):
    info = pim_info()
    _check(load().pim_plan_info(plan, ctypes.byref(info)), "pim_plan_info")
    return info


def pim_set_profiling(plan, on):
    _check(load().pim_set_profiling(plan, int(on)), "pim_set_profiling")


def pim_stage_times(plan):
    """{stage name: total ms} and the number of applies timed."""
    ms = (ctypes.c_double * len(STAGES))()
    cnt = ctypes.c_int64()
    _check(load().pim_stage_times(plan, ms, len(STAGES), ctypes.byref(cnt)), "pim_stage_times")
    return {STAGES[i]: ms[i] for i in range(len(STAGES))}, cnt.value


def pim_stage_name(stage):
    r = load().pim_stage_name(int(stage))
    return r.decode() if r is not None else None


def pim_position_grad(plan, q, g, grad_xyz, nrhs=1, stream=None):
    _check(load().pim_position_grad(plan, _ptr(q), _ptr(g), _ptr(grad_xyz), int(nrhs), _stream_ptr(stream)),
           "pim_position_grad")


def pim_position_grad_reuse(plan, q, g, grad_xyz, stream=None):
    _check(load().pim_position_grad_reuse(plan, _ptr(q), _ptr(g), _ptr(grad_xyz), _stream_ptr(stream)),
           "pim_position_grad_reuse")


def pim_set_points_observers(plan, N, xyz, M, obs):
    _check(load().pim_set_points_observers(plan, ctypes.c_int64(int(N)), _ptr(xyz), ctypes.c_int64(int(M)), _ptr(obs)),
           "pim_set_points_observers")


def pim_apply_observers(plan, q, u, nrhs=1, stream=None):
    _check(load().pim_apply_observers(plan, _ptr(q), _ptr(u), int(nrhs), _stream_ptr(stream)), "pim_apply_observers")


def pim_apply_observers_adjoint(plan, v, w, nrhs=1, stream=None):
    _check(load().pim_apply_observers_adjoint(plan, _ptr(v), _ptr(w), int(nrhs), _stream_ptr(stream)),
           "pim_apply_observers_adjoint")


def pim_update_positions(plan, xyz):
    _check(load().pim_update_positions(plan, _ptr(xyz)), "pim_update_positions")


def pim_apply_batched(plans, qs, us, nrhs=1, adjoint=False, stream=None):
    """plans: list of Plan or handles; qs, us: lists of device tensors."""
    n = len(plans)
    hs = [p._h if isinstance(p, Plan) else p for p in plans]
    P = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in hs])
    Q = (ctypes.c_void_p * n)(*[_ptr(x).value for x in qs])
    U = (ctypes.c_void_p * n)(*[_ptr(x).value for x in us])
    _check(load().pim_apply_batched(n, P, Q, U, int(nrhs), 1 if adjoint else 0, _stream_ptr(stream)),
           "pim_apply_batched")


def pim_apply_noalloc(plan, q, u, nrhs=1, adjoint=False, stream=None):
    _check(load().pim_apply_noalloc(plan, _ptr(q), _ptr(u), int(nrhs), 1 if adjoint else 0, _stream_ptr(stream)),
           "pim_apply_noalloc")


def pim_debug_copy(plan, what, out):
    _check(load().pim_debug_copy(plan, int(what), _ptr(out), out.nbytes), "pim_debug_copy")


def pim_destroy(plan):
    if plan:
        load().pim_destroy(plan)


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------
class Plan:
    """An FFT-PIM plan for one cell, grid and point set.

    D          cell extents (D_x, D_y, D_z); the lattice is diag(D)
    pdims      periodic axes, e.g. (0, 1)
    k, k0      wavenumber and phase-shift vector (the paper's k_0 and
               k_x0, k_y0, k_z0); complex values allowed (Im k <= 0)
    n          near grid nodes per axis (h = D / (n - 1))
    p          near Lagrange degree; layers = near-image layers i_d
    precision  "fp64" or "fp32"
    b, nf, pf, corr_mode, cube, listfree: options (None = library default)
    """

    def __init__(self, D, pdims, k, k0, n, p=4, layers=1, precision="fp32", b=None, nf=None, pf=None,
                 corr_mode=None, cube=False, listfree=None, lf_tensor_cores=None, neutral_tol=None, mem_cap=0,
                 autotune=None,
                 with_gradient=False, gather_variant=None, corr_split=None, stream=None):
        self.D = np.asarray(D, np.float64)
        self.n = np.asarray(n, np.int64)
        self.pdims = tuple(pdims)
        self.k = complex(k) if np.iscomplexobj(k) and complex(k).imag != 0 else float(np.real(k))
        k0c = np.asarray(k0, np.complex128)
        self.k0 = k0c if np.any(k0c.imag != 0) else k0c.real.copy()
        self.precision = precision
        opt = pim_options_default()
        opt.k_imag = float(np.imag(self.k))
        for d in range(3):
            opt.k0_imag[d] = float(k0c[d].imag)
        if b is not None:
            opt.corr_radius = int(b)
        if nf is not None:
            for d in range(3):
                opt.far_n[d] = int(nf[d])
        if pf is not None:
            opt.far_p = int(pf)
        if corr_mode is not None:
            opt.corr_mode = int(corr_mode)
        if listfree is not None:
            opt.corr_listfree = int(listfree)
        if lf_tensor_cores is not None:
            opt.lf_tensor_cores = 1 if lf_tensor_cores else 0
        if neutral_tol is not None:
            opt.neutral_tol = float(neutral_tol)
        opt.corr_cube = 1 if cube else 0
        if autotune is not None:
            opt.autotune = 1 if autotune else 0
        opt.with_gradient = 1 if with_gradient else 0
        if gather_variant is not None:
            opt.gather_variant = int(gather_variant)
        if corr_split is not None:
            opt.corr_split = int(corr_split)
        opt.mem_cap = int(mem_cap)
        mask = sum(1 << d for d in self.pdims)
        h = self.D / (self.n - 1)
        prec = PIM_FP64 if precision == "fp64" else PIM_FP32_MIXED
        self.real = self.k == 0 and not np.any(self.k0 != 0)
        self._h = pim_plan_create(np.diag(self.D), mask, float(np.real(self.k)), np.real(k0c), h, p, layers, prec, opt,
                                  stream)
        self.N = 0

    def set_points(self, xyz):
        """xyz: (N, 3) float64 positions (torch tensor on the GPU or numpy)."""
        self.N = int(xyz.shape[0])
        pim_set_points(self._h, self.N, xyz)

    def set_points_observers(self, xyz, obs):
        """N sources xyz (N, 3) and M observers obs (M, 3), float64 (torch on
        the GPU or numpy): one point set, sources first."""
        self.N_src, self.M_obs = int(xyz.shape[0]), int(obs.shape[0])
        self.N = self.N_src + self.M_obs
        pim_set_points_observers(self._h, self.N_src, xyz, self.M_obs, obs)

    def apply_observers(self, q, stream=None, adjoint=False):
        """Potentials at the observers from source strengths q ([N] or
        [N, nrhs]); adjoint=True maps observer values ([M] or [M, nrhs]) to
        the sources."""
        nrhs = 1 if q.ndim == 1 else int(q.shape[1])
        rows = self.N_src if adjoint else self.M_obs
        shape = (rows,) if q.ndim == 1 else (rows, nrhs)
        if hasattr(q, "data_ptr") and not isinstance(q, np.ndarray):
            import torch
            out = torch.empty(shape, dtype=q.dtype, device=q.device)
        else:
            out = np.empty(shape, q.dtype)
        (pim_apply_observers_adjoint if adjoint else pim_apply_observers)(self._h, q, out, nrhs, stream)
        return out

    def dtype_np(self):
        if self.real:
            return np.float64 if self.precision == "fp64" else np.float32
        return np.complex128 if self.precision == "fp64" else np.complex64

    def apply(self, q, out=None, stream=None, adjoint=False):
        """u = A q (or A^H q).  q: [N] or [N, nrhs] torch tensor or numpy
        array of the plan dtype; a new array/tensor is returned unless out
        is given."""
        nrhs = 1 if q.ndim == 1 else int(q.shape[1])
        if out is None:
            if hasattr(q, "data_ptr") and not isinstance(q, np.ndarray):
                import torch
                out = torch.empty_like(q)
            else:
                out = np.empty_like(q)
        f = pim_apply_adjoint if adjoint else pim_apply
        f(self._h, q, out, nrhs, stream)
        if not adjoint:
            self.forward_applies = getattr(self, "forward_applies", 0) + 1
        return out

    def apply_adjoint(self, v, out=None, stream=None):
        return self.apply(v, out, stream, adjoint=True)

    def position_grad(self, q, g, out=None, stream=None):
        """(N, 3) float64: d/dx Re sum conj(g) (A q) with the discrete
        structure frozen (plan created with with_gradient=True)."""
        nrhs = 1 if q.ndim == 1 else int(q.shape[1])
        if out is None:
            if hasattr(q, "data_ptr") and not isinstance(q, np.ndarray):
                import torch
                out = torch.empty((self.N, 3), dtype=torch.float64, device=q.device)
            else:
                out = np.empty((self.N, 3), np.float64)
        pim_position_grad(self._h, q, g, out, nrhs, stream)
        return out

    def position_grad_reuse(self, q, g, out=None, stream=None):
        """position_grad for one right-hand side after apply(q) and
        apply_adjoint(g) on this plan, reusing their grid potentials (q and g
        must be the arrays those applies read)."""
        if out is None:
            if hasattr(q, "data_ptr") and not isinstance(q, np.ndarray):
                import torch
                out = torch.empty((self.N, 3), dtype=torch.float64, device=q.device)
            else:
                out = np.empty((self.N, 3), np.float64)
        pim_position_grad_reuse(self._h, q, g, out, stream)
        return out

    def update_positions(self, xyz):
        """New positions with the stencils, boxes and correction list kept."""
        pim_update_positions(self._h, xyz)

    def set_profiling(self, on=True):
        pim_set_profiling(self._h, on)

    def stage_times(self):
        return pim_stage_times(self._h)

    def device_status(self):
        return pim_last_device_status(self._h)

    def info(self):
        return pim_plan_info(self._h)

    def debug(self, what):
        info = self.info()
        n = tuple(info.n)
        G = n[0] * n[1] * n[2]
        cdt = np.complex128 if self.precision == "fp64" else np.complex64
        if what == 0:
            nf = tuple(info.nf)
            out = np.empty((2 * nf[2] - 1, 2 * nf[1] - 1, 2 * nf[0] - 1), np.complex128)
        elif what in (1, 2):
            out = np.empty((n[2], n[1], n[0]), cdt)
        elif what == 3:
            out = np.empty(info.N, np.int32)
        elif what == 4:
            out = np.empty(info.N + 1, np.int64)
        elif what == 5:
            out = np.empty(info.nnz, np.uint32)
        elif what == 6:
            out = np.empty(info.nnz, np.complex128)
        elif what == 7:
            out = np.empty(info.N, np.int32)
        else:
            raise ValueError(what)
        pim_debug_copy(self._h, what, out)
        return out

    def close(self):
        if getattr(self, "_h", None):
            pim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
