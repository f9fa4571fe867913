"""ctypes binding of libextconv.so: argument marshalling only.

Every function here forwards to the C entry point of the same name
(declared in include/extconv.h); the computation happens in the library's
CUDA kernels.  Arrays may be torch tensors (device or host) or numpy arrays
(host); their data pointers are passed through unchanged.  If the library
has not been built, importing works but every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libextconv.so")

EXT_OK = 0
EXT_ERR_INVALID_ARG = 1
EXT_ERR_UNSUPPORTED = 2
EXT_ERR_CUDA = 3
EXT_ERR_OOM = 4
EXT_ERR_TIMEOUT = 5
EXT_ERR_CHECKPOINT = 6

EXT_FILTER_ANALYTIC_GAUSSPOW = 0
EXT_FILTER_TABLE = 1
EXT_FILTER_SAMPLED = 2

EXT_PREC_FP32 = 0
EXT_PREC_BF16X3 = 1
EXT_PREC_DEFAULT = -1

EXT_TUNE_OFF = 0
EXT_TUNE_ON = 1
EXT_FAULT_NONE = 0
EXT_FAULT_ALLOC = 1

EXPORTED = (
    "ext_status_string", "ext_last_error", "ext_plan_create", "ext_plan_destroy", "ext_plan_trim",
    "ext_plan_profile", "ext_plan_profile_read", "ext_plan_sync",
    "ext_filter_so2_decompose", "ext_conv_so2", "ext_corr_so2", "ext_corr_so2_components",
    "ext_sweep_so2", "ext_sweep_so2_noalloc", "ext_conv_scale", "ext_batch_corr_so2",
    "ext_so3_channels", "ext_so3_wigner", "ext_corr_so3_components", "ext_sweep_so3", "ext_corr_so3",
    "ext_mlp_create", "ext_mlp_destroy", "ext_mlp_set_params", "ext_mlp_get_params", "ext_mlp_forward",
    "ext_mlp_grads", "ext_mlp_train", "ext_so3_upper_bound", "ext_so3_refined_bound", "ext_so3_gather", "ext_so3_augment", "ext_so3_refine",
    "ext_so3_propose", "ext_corr_so3_propose", "ext_gradient_field", "ext_consensus_radius",
    "ext_consensus_filter", "ext_ght_detect", "ext_conv_so2_normalized", "ext_filter_so2_energy",
    "ext_corr_so2_subset", "ext_conv_so3", "ext_conv_similarity", "ext_options_init", "ext_plan_selftest_timeout",
    "ext_select_components", "ext_mlp_save", "ext_mlp_load", "ext_mlp_checkpoint_info", "ext_sweep_so3_grid",
    "ext_corr_so3_grid",
)


class ExtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class ext_image_desc(ctypes.Structure):
    pass


class ext_options(ctypes.Structure):
    _fields_ = [
        ("device", ctypes.c_int), ("precision", ctypes.c_int), ("wait_budget_ns", ctypes.c_uint64),
        ("autotune", ctypes.c_int), ("tune_cache", ctypes.c_char_p), ("fault_inject", ctypes.c_int),
        ("fault_after", ctypes.c_int),
    ]


class ext_filter_so2(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_int), ("R", ctypes.c_int), ("kind", ctypes.c_int),
        ("a", ctypes.POINTER(ctypes.c_double)), ("sigma", ctypes.c_double),
        ("fk", ctypes.POINTER(ctypes.c_double)), ("n_r", ctypes.c_int), ("dr", ctypes.c_double),
        ("img", ctypes.POINTER(ctypes.c_double)), ("n_theta", ctypes.c_int),
    ]


ext_image_desc._fields_ = [
    ("H", ctypes.c_void_p), ("h", ctypes.c_int), ("w", ctypes.c_int), ("F", ctypes.POINTER(ext_filter_so2)),
    ("n_angles", ctypes.c_int), ("max_out", ctypes.c_void_p), ("argmax", ctypes.c_void_p),
]

_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libextconv.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        fp = ctypes.POINTER(ext_filter_so2)
        L.ext_status_string.restype = ctypes.c_char_p
        L.ext_status_string.argtypes = [i32]
        L.ext_last_error.restype = ctypes.c_char_p
        L.ext_last_error.argtypes = []
        L.ext_options_init.argtypes = [ctypes.POINTER(ext_options)]
        L.ext_options_init.restype = None
        L.ext_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ext_options)]
        L.ext_plan_selftest_timeout.argtypes = [vp, vp]
        L.ext_select_components.argtypes = [vp, i32, i32, vp, ctypes.POINTER(i32)]
        L.ext_mlp_save.argtypes = [vp, ctypes.c_char_p]
        L.ext_mlp_load.argtypes = [vp, ctypes.c_char_p]
        L.ext_mlp_checkpoint_info.argtypes = [ctypes.c_char_p, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                              ctypes.POINTER(i64)]
        L.ext_plan_destroy.argtypes = [vp]
        L.ext_plan_trim.argtypes = [vp]
        L.ext_plan_profile.argtypes = [vp, i32]
        L.ext_plan_sync.argtypes = [vp, vp]
        L.ext_plan_profile_read.argtypes = [vp, i32, vp, vp, vp, ctypes.POINTER(i32)]
        L.ext_filter_so2_decompose.argtypes = [vp, fp, vp, i64, ctypes.POINTER(i32)]
        L.ext_conv_so2.argtypes = [vp, vp, i32, i32, fp, vp, vp, vp]
        L.ext_corr_so2.argtypes = [vp, vp, i32, i32, fp, vp, i32, vp, vp, i32, vp]
        L.ext_corr_so2_components.argtypes = [vp, vp, i32, i32, fp, vp, vp]
        L.ext_sweep_so2.argtypes = [vp, vp, i64, i32, i32, vp, vp, i32, vp]
        L.ext_sweep_so2_noalloc.argtypes = [vp, i64, i32, i32, vp, vp, vp]
        L.ext_batch_corr_so2.argtypes = [vp, ctypes.POINTER(ext_image_desc), i32, i32, vp]
        L.ext_so3_channels.argtypes = [i32]
        L.ext_so3_wigner.argtypes = [vp, vp, i32, i32, vp]
        L.ext_corr_so3_components.argtypes = [vp, vp, i32, i32, i32, vp, i32, i32, ctypes.c_double, i32, vp, vp]
        L.ext_sweep_so3.argtypes = [vp, vp, i64, i32, vp, i32, vp, vp, i32, vp]
        L.ext_corr_so3.argtypes = [vp, vp, i32, i32, i32, vp, i32, i32, ctypes.c_double, i32, vp, i32, vp, vp, i32, vp]
        L.ext_sweep_so3_grid.argtypes = [vp, vp, i64, i32, vp, i32, i32, vp, vp, i32, vp]
        L.ext_corr_so3_grid.argtypes = [vp, vp, i32, i32, i32, vp, i32, i32, ctypes.c_double, i32, vp, i32, i32, vp,
                                        vp, i32, vp]
        L.ext_conv_so3.argtypes = [vp, vp, i32, i32, i32, vp, i32, i32, ctypes.c_double, i32, vp, vp, vp]
        L.ext_conv_similarity.argtypes = [vp, vp, i32, i32, i32, vp, i32, i32, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, vp, vp, i32, vp, vp]
        dbl, f32 = ctypes.c_double, ctypes.c_float
        L.ext_mlp_create.argtypes = [vp, i32, i32, ctypes.POINTER(vp)]
        L.ext_mlp_destroy.argtypes = [vp]
        L.ext_mlp_set_params.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.ext_mlp_get_params.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.ext_mlp_forward.argtypes = [vp, vp, i32, vp, vp]
        L.ext_mlp_grads.argtypes = [vp, vp, vp, i32, vp, vp, vp]
        L.ext_mlp_train.argtypes = [vp, vp, vp, i32, i32, vp, vp, i32, i32, f32, vp, vp]
        L.ext_so3_upper_bound.argtypes = [vp, vp, i64, i32, vp, vp]
        L.ext_so3_refined_bound.argtypes = [vp, vp, i32, i32, vp, vp]
        L.ext_so3_gather.argtypes = [vp, vp, i64, i32, vp, i32, vp, vp]
        L.ext_so3_augment.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, vp]
        L.ext_so3_refine.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp]
        L.ext_so3_propose.argtypes = [vp, vp, i64, i32, vp, vp, i32, f32, vp, vp, vp, i32, vp, vp]
        L.ext_corr_so3_propose.argtypes = [vp, vp, i32, i32, i32, vp, i32, i32, dbl, i32, vp, vp, i32, f32, vp, vp,
                                           vp, i32, vp, vp]
        L.ext_conv_scale.argtypes = [vp, vp, i32, i32, i32, vp, i32, dbl, dbl, dbl, dbl, vp, i32, vp, vp]
        L.ext_gradient_field.argtypes = [vp, vp, i32, i32, vp, vp, vp]
        L.ext_consensus_radius.argtypes = [dbl]
        L.ext_consensus_filter.argtypes = [vp, vp, i32, i32, i32, i32, dbl, vp, vp]
        L.ext_ght_detect.argtypes = [vp, vp, i32, i32, fp, vp, vp]
        L.ext_conv_so2_normalized.argtypes = [vp, vp, i32, i32, i32, fp, vp, vp, vp]
        L.ext_filter_so2_energy.argtypes = [vp, fp, vp]
        L.ext_corr_so2_subset.argtypes = [vp, vp, i32, i32, fp, vp, i32, i32, vp, vp, i32, vp]
        for name in EXPORTED:
            if name not in ("ext_status_string", "ext_last_error", "ext_so3_channels", "ext_consensus_radius",
                            "ext_options_init"):
                getattr(L, name).restype = i32
        _lib = L
    return _lib


def _check(status):
    if status != EXT_OK:
        L = lib()
        raise ExtError(status, f"{L.ext_status_string(status).decode()}: {L.ext_last_error().decode()}")


def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy arrays must be C-contiguous")
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class FilterSO2:
    """Owns the host arrays an ext_filter_so2 points to."""

    def __init__(self, K, R, kind, a=None, sigma=0.0, fk=None, dr=0.0, img=None, n_theta=0):
        self.K, self.R, self.kind = int(K), int(R), int(kind)
        self._a = None if a is None else np.ascontiguousarray(np.asarray(a, np.complex128)).view(np.float64)
        self._fk = None if fk is None else np.ascontiguousarray(np.asarray(fk, np.complex128)).view(np.float64)
        self._img = None if img is None else np.ascontiguousarray(np.asarray(img, np.float64))
        dp = ctypes.POINTER(ctypes.c_double)
        self.struct = ext_filter_so2(
            self.K, self.R, self.kind,
            self._a.ctypes.data_as(dp) if self._a is not None else None, float(sigma),
            self._fk.ctypes.data_as(dp) if self._fk is not None else None,
            0 if fk is None else int(np.asarray(fk).shape[1]), float(dr),
            self._img.ctypes.data_as(dp) if self._img is not None else None, int(n_theta))

    @classmethod
    def analytic(cls, a, sigma, R):
        a = np.asarray(a, np.complex128)
        return cls((len(a) - 1) // 2, R, EXT_FILTER_ANALYTIC_GAUSSPOW, a=a, sigma=sigma)

    @classmethod
    def table(cls, fk, dr, R):
        fk = np.asarray(fk, np.complex128)
        return cls((fk.shape[0] - 1) // 2, R, EXT_FILTER_TABLE, fk=fk, dr=dr)

    @classmethod
    def sampled(cls, img, K, dr, n_theta):
        img = np.asarray(img, np.float64)
        return cls(K, (img.shape[0] - 1) // 2, EXT_FILTER_SAMPLED, img=img, dr=dr, n_theta=n_theta)

    def ref(self):
        return ctypes.byref(self.struct)


class Plan:
    """A plan (ext_plan) on `device`; the keyword options map to ext_options:
    precision (default sweep precision), wait_budget_ns, autotune (bool),
    tune_cache (path), fault_inject / fault_after (host-side injection of an
    allocation failure, for tests)."""

    def __init__(self, device: int = 0, precision=None, wait_budget_ns=None, autotune=False, tune_cache=None,
                 fault_inject=None, fault_after=0):
        import weakref
        self.handle = ctypes.c_void_p()
        self._nets = weakref.WeakSet()
        opts = ext_options()
        lib().ext_options_init(ctypes.byref(opts))
        opts.device = int(device)
        if precision is not None:
            opts.precision = int(precision)
        if wait_budget_ns is not None:
            opts.wait_budget_ns = int(wait_budget_ns)
        opts.autotune = EXT_TUNE_ON if autotune else EXT_TUNE_OFF
        self._tune_cache = None if tune_cache is None else os.fsencode(tune_cache)
        opts.tune_cache = self._tune_cache
        if fault_inject is not None:
            opts.fault_inject = int(fault_inject)
            opts.fault_after = int(fault_after)
        _check(lib().ext_plan_create(ctypes.byref(self.handle), ctypes.byref(opts)))

    def selftest_timeout(self, stream=None):
        _check(lib().ext_plan_selftest_timeout(self.handle, _stream(stream)))

    def close(self):
        if self.handle:
            for net in list(self._nets):      # networks use the plan: close them first
                net.close()
            lib().ext_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def trim(self):
        _check(lib().ext_plan_trim(self.handle))

    def sync(self, stream=None):
        _check(lib().ext_plan_sync(self.handle, _stream(stream)))

    def profile(self, enable: bool):
        _check(lib().ext_plan_profile(self.handle, 1 if enable else 0))

    def profile_read(self):
        """{kernel name: (total ms, launches)} since the last read."""
        n_max = 64
        names = ctypes.create_string_buffer(64 * n_max)
        ms = np.zeros(n_max, np.float64)
        cnt = np.zeros(n_max, np.int64)
        n = ctypes.c_int(0)
        _check(lib().ext_plan_profile_read(self.handle, n_max, names, _ptr(ms), _ptr(cnt), ctypes.byref(n)))
        out = {}
        for i in range(n.value):
            name = names.raw[64 * i:64 * i + 64].split(b"\0", 1)[0].decode()
            out[name] = (float(ms[i]), int(cnt[i]))
        return out

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ext_filter_so2_decompose(plan: Plan, F: FilterSO2):
    nk = 2 * F.K + 1
    cap = 2 * nk * 100000
    out = np.zeros(cap, np.float64)
    n_r = ctypes.c_int(0)
    _check(lib().ext_filter_so2_decompose(plan.handle, F.ref(), _ptr(out), cap, ctypes.byref(n_r)))
    return out[: 2 * nk * n_r.value].view(np.complex128).reshape(nk, n_r.value)


def ext_conv_so2(plan: Plan, H, h, w, F: FilterSO2, alpha, out, stream=None):
    _check(lib().ext_conv_so2(plan.handle, _ptr(H), int(h), int(w), F.ref(), _ptr(alpha), _ptr(out),
                              _stream(stream)))


def ext_corr_so2(plan: Plan, H, h, w, F: FilterSO2, alpha, n_angles, out_or_max, argmax, precision=EXT_PREC_FP32,
                 stream=None):
    _check(lib().ext_corr_so2(plan.handle, _ptr(H), int(h), int(w), F.ref(), _ptr(alpha), int(n_angles),
                              _ptr(out_or_max), _ptr(argmax), int(precision), _stream(stream)))


def ext_corr_so2_components(plan: Plan, H, h, w, F: FilterSO2, G, stream=None):
    _check(lib().ext_corr_so2_components(plan.handle, _ptr(H), int(h), int(w), F.ref(), _ptr(G),
                                         _stream(stream)))


def ext_sweep_so2(plan: Plan, G, n_pix, K, n_angles, max_out, argmax, precision=EXT_PREC_FP32, stream=None):
    _check(lib().ext_sweep_so2(plan.handle, _ptr(G), int(n_pix), int(K), int(n_angles), _ptr(max_out),
                               _ptr(argmax), int(precision), _stream(stream)))


def ext_sweep_so2_noalloc(G, n_pix, K, n_angles, max_out, argmax, stream=None):
    """Allocation-free FP32 sweep (device buffers only; see include/extconv.h)."""
    _check(lib().ext_sweep_so2_noalloc(_ptr(G), int(n_pix), int(K), int(n_angles), _ptr(max_out), _ptr(argmax),
                                       _stream(stream)))


def ext_conv_scale(plan: Plan, H, channels, h, w, mellin_c, log_period, r_min, r_max, centre_tap, s, mode, out,
                   stream=None):
    """Scale-adaptive extended convolution / smoothing (see include/extconv.h)."""
    c = np.ascontiguousarray(np.asarray(mellin_c, np.complex128)).view(np.float64)
    _check(lib().ext_conv_scale(plan.handle, _ptr(H), int(channels), int(h), int(w), _ptr(c), int(len(c) // 2),
                                float(log_period), float(r_min), float(r_max), float(centre_tap), _ptr(s), int(mode),
                                _ptr(out), _stream(stream)))


class BatchDescriptors:
    """The ext_image_desc array of a batch, built once: pass it instead of
    the item list to ext_batch_corr_so2 to skip re-marshalling the same
    buffers and filters on every call."""

    def __init__(self, items):
        self.items = list(items)
        self.arr = (ext_image_desc * len(self.items))()
        for i, (H, h, w, F, J, mx, am) in enumerate(self.items):
            self.arr[i] = ext_image_desc(_ptr(H), int(h), int(w), ctypes.pointer(F.struct), int(J), _ptr(mx),
                                         _ptr(am))


def ext_batch_corr_so2(plan: Plan, items, precision=EXT_PREC_BF16X3, stream=None):
    """items: sequence of (H, h, w, FilterSO2, n_angles, max_out, argmax) with device tensors, or a
    BatchDescriptors of such a sequence."""
    batch = items if isinstance(items, BatchDescriptors) else BatchDescriptors(items)
    _check(lib().ext_batch_corr_so2(plan.handle, batch.arr, len(batch.items), int(precision), _stream(stream)))


def so3_pack_tables(tables):
    """List over l of (2l+1, n_r) complex arrays -> contiguous (L+1)^2 x n_r complex128."""
    return np.ascontiguousarray(np.concatenate([np.asarray(t, np.complex128) for t in tables], axis=0))


def ext_so3_channels(L):
    return int(lib().ext_so3_channels(int(L)))


def ext_so3_wigner(plan: Plan, quats, L):
    q = np.ascontiguousarray(np.asarray(quats, np.float64).reshape(-1, 4))
    per = (L + 1) * (2 * L + 1) * (2 * L + 3) // 3
    out = np.zeros((q.shape[0], per), np.complex128)
    _check(lib().ext_so3_wigner(plan.handle, _ptr(q), q.shape[0], int(L), _ptr(out.view(np.float64))))
    return out


def ext_corr_so3_components(plan: Plan, V, nz, ny, nx, tables, dr, R, G, stream=None):
    t = so3_pack_tables(tables)
    L = len(tables) - 1
    _check(lib().ext_corr_so3_components(plan.handle, _ptr(V), int(nz), int(ny), int(nx), _ptr(t.view(np.float64)),
                                         L, t.shape[1], float(dr), int(R), _ptr(G), _stream(stream)))


def ext_sweep_so3(plan: Plan, G, n_vox, L, quats, max_out, argmax, precision=EXT_PREC_BF16X3, stream=None):
    q = np.ascontiguousarray(np.asarray(quats, np.float64).reshape(-1, 4))
    _check(lib().ext_sweep_so3(plan.handle, _ptr(G), int(n_vox), int(L), _ptr(q), q.shape[0], _ptr(max_out),
                               _ptr(argmax), int(precision), _stream(stream)))


def ext_corr_so3(plan: Plan, V, nz, ny, nx, tables, dr, R, quats, max_out, argmax, precision=EXT_PREC_BF16X3,
                 stream=None):
    t = so3_pack_tables(tables)
    L = len(tables) - 1
    q = np.ascontiguousarray(np.asarray(quats, np.float64).reshape(-1, 4))
    _check(lib().ext_corr_so3(plan.handle, _ptr(V), int(nz), int(ny), int(nx), _ptr(t.view(np.float64)), L, t.shape[1],
                              float(dr), int(R), _ptr(q), q.shape[0], _ptr(max_out), _ptr(argmax), int(precision),
                              _stream(stream)))


def ext_sweep_so3_grid(plan: Plan, G, n_vox, L, dir_quats, n_psi, max_out, argmax, precision=EXT_PREC_BF16X3,
                       stream=None):
    q = np.ascontiguousarray(np.asarray(dir_quats, np.float64).reshape(-1, 4))
    _check(lib().ext_sweep_so3_grid(plan.handle, _ptr(G), int(n_vox), int(L), _ptr(q), q.shape[0], int(n_psi),
                                    _ptr(max_out), _ptr(argmax), int(precision), _stream(stream)))


def ext_corr_so3_grid(plan: Plan, V, nz, ny, nx, tables, dr, R, dir_quats, n_psi, max_out, argmax,
                      precision=EXT_PREC_BF16X3, stream=None):
    t = so3_pack_tables(tables)
    L = len(tables) - 1
    q = np.ascontiguousarray(np.asarray(dir_quats, np.float64).reshape(-1, 4))
    _check(lib().ext_corr_so3_grid(plan.handle, _ptr(V), int(nz), int(ny), int(nx), _ptr(t.view(np.float64)), L,
                                   t.shape[1], float(dr), int(R), _ptr(q), q.shape[0], int(n_psi), _ptr(max_out),
                                   _ptr(argmax), int(precision), _stream(stream)))


def ext_conv_similarity(plan: Plan, H, channels, h, w, coef, log_period, r_min, r_max, centre_tap, alpha, s, mode,
                        out, stream=None):
    """Extended convolution with rotation and scale fields; coef complex
    [K + 1][2 n_h - 1] (row k, column j + n_h - 1)."""
    c = np.ascontiguousarray(np.asarray(coef, np.complex128))
    K, nj = c.shape
    _check(lib().ext_conv_similarity(plan.handle, _ptr(H), int(channels), int(h), int(w), _ptr(c.view(np.float64)),
                                     K - 1, (nj + 1) // 2, float(log_period), float(r_min), float(r_max),
                                     float(centre_tap), _ptr(alpha), _ptr(s), int(mode), _ptr(out), _stream(stream)))


def ext_conv_so3(plan: Plan, V, nz, ny, nx, tables, dr, R, quats, out, stream=None):
    """SO(3) extended convolution (scatter) with one quaternion (w, x, y, z)
    per voxel; quats float32 [nz*ny*nx][4], host array or device tensor."""
    t = so3_pack_tables(tables)
    L = len(tables) - 1
    if isinstance(quats, np.ndarray):
        quats = np.ascontiguousarray(quats, np.float32)
    _check(lib().ext_conv_so3(plan.handle, _ptr(V), int(nz), int(ny), int(nx), _ptr(t.view(np.float64)), L, t.shape[1],
                              float(dr), int(R), _ptr(quats), _ptr(out), _stream(stream)))


class MLP:
    """The proposal network (ext_mlp): n_in -> hidden -> hidden -> 4, owned by a plan."""

    def __init__(self, plan: Plan, n_in: int, hidden: int = 256):
        self.plan = plan
        self.n_in, self.hidden = int(n_in), int(hidden)
        self.handle = ctypes.c_void_p()
        _check(lib().ext_mlp_create(plan.handle, self.n_in, self.hidden, ctypes.byref(self.handle)))
        plan._nets.add(self)

    def close(self):
        if self.handle:
            lib().ext_mlp_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        """p: dict W1, b1, W2, b2, W3, b3 (arrays or tensors, FP32 on host or device)."""
        arrs = [p[k] for k in ("W1", "b1", "W2", "b2", "W3", "b3")]
        arrs = [np.ascontiguousarray(np.asarray(a, np.float32)) if not hasattr(a, "data_ptr") else a for a in arrs]
        _check(lib().ext_mlp_set_params(self.handle, *[_ptr(a) for a in arrs]))

    def get_params(self):
        H, n = self.hidden, self.n_in
        out = dict(W1=np.zeros((H, n), np.float32), b1=np.zeros(H, np.float32), W2=np.zeros((H, H), np.float32),
                   b2=np.zeros(H, np.float32), W3=np.zeros((4, H), np.float32), b3=np.zeros(4, np.float32))
        _check(lib().ext_mlp_get_params(self.handle, *[_ptr(out[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]))
        return out

    def n_params(self):
        H, n = self.hidden, self.n_in
        return H * n + H + H * H + H + 4 * H + 4

    def save(self, path):
        _check(lib().ext_mlp_save(self.handle, os.fsencode(path)))

    def load(self, path):
        _check(lib().ext_mlp_load(self.handle, os.fsencode(path)))


def ext_mlp_checkpoint_info(path):
    """(n_in, hidden, step) of a checkpoint file, checked on the host alone."""
    n_in, hidden, step = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int64(0)
    _check(lib().ext_mlp_checkpoint_info(os.fsencode(path), ctypes.byref(n_in), ctypes.byref(hidden),
                                         ctypes.byref(step)))
    return n_in.value, hidden.value, step.value


def ext_select_components(energy, budget):
    """The component list of ext_select_components for energies E_0..E_K."""
    E = np.ascontiguousarray(np.asarray(energy, np.float64))
    K = len(E) - 1
    ks = np.zeros(max(K + 1, 1), np.int32)
    n = ctypes.c_int(0)
    _check(lib().ext_select_components(_ptr(E), int(K), int(budget), _ptr(ks), ctypes.byref(n)))
    return [int(k) for k in ks[:n.value]]


def ext_mlp_forward(net: MLP, X, n, q, stream=None):
    _check(lib().ext_mlp_forward(net.handle, _ptr(X), int(n), _ptr(q), _stream(stream)))


def ext_mlp_grads(net: MLP, X, qt, n, loss, grads, stream=None):
    _check(lib().ext_mlp_grads(net.handle, _ptr(X), _ptr(qt), int(n), _ptr(loss), _ptr(grads), _stream(stream)))


def ext_mlp_train(net: MLP, X, qt, n_train, L, rows, Q, steps, batch, lr, losses, stream=None):
    _check(lib().ext_mlp_train(net.handle, _ptr(X), _ptr(qt), int(n_train), int(L), _ptr(rows), _ptr(Q), int(steps),
                               int(batch), float(lr), _ptr(losses), _stream(stream)))


def ext_so3_upper_bound(plan: Plan, G, n_vox, L, ub, stream=None):
    _check(lib().ext_so3_upper_bound(plan.handle, _ptr(G), int(n_vox), int(L), _ptr(ub), _stream(stream)))


def ext_so3_refined_bound(plan: Plan, X, n, L, out, stream=None):
    _check(lib().ext_so3_refined_bound(plan.handle, _ptr(X), int(n), int(L), _ptr(out), _stream(stream)))


def ext_so3_gather(plan: Plan, G, n_vox, L, vox, n, X, stream=None):
    _check(lib().ext_so3_gather(plan.handle, _ptr(G), int(n_vox), int(L), _ptr(vox), int(n), _ptr(X),
                                _stream(stream)))


def ext_so3_augment(plan: Plan, X, n, L, Q, q_in, X_out, q_out, stream=None):
    _check(lib().ext_so3_augment(plan.handle, _ptr(X), int(n), int(L), _ptr(Q), _ptr(q_in), _ptr(X_out), _ptr(q_out),
                                 _stream(stream)))


def ext_so3_refine(plan: Plan, X, n, L, q0, q_out, s_out, stream=None):
    _check(lib().ext_so3_refine(plan.handle, _ptr(X), int(n), int(L), _ptr(q0), _ptr(q_out), _ptr(s_out),
                                _stream(stream)))


def ext_so3_propose(plan: Plan, G, n_vox, L, net, quats, bound, score, quat=None, grid_idx=None,
                    precision=EXT_PREC_BF16X3, stream=None):
    """Returns (voxels with UB >= bound, candidates, swept candidates)."""
    q = np.ascontiguousarray(np.asarray(quats, np.float64).reshape(-1, 4))
    counts = np.zeros(3, np.int64)
    _check(lib().ext_so3_propose(plan.handle, _ptr(G), int(n_vox), int(L), net.handle if net is not None else None,
                                 _ptr(q), q.shape[0], float(bound), _ptr(score), _ptr(quat), _ptr(grid_idx),
                                 int(precision), _ptr(counts), _stream(stream)))
    return int(counts[0]), int(counts[1]), int(counts[2])


def ext_corr_so3_propose(plan: Plan, V, nz, ny, nx, tables, dr, R, net, quats, bound, score, quat=None, grid_idx=None,
                         precision=EXT_PREC_BF16X3, stream=None):
    """Returns (voxels with UB >= bound, candidates, swept candidates)."""
    t = so3_pack_tables(tables)
    L = len(tables) - 1
    q = np.ascontiguousarray(np.asarray(quats, np.float64).reshape(-1, 4))
    counts = np.zeros(3, np.int64)
    _check(lib().ext_corr_so3_propose(plan.handle, _ptr(V), int(nz), int(ny), int(nx), _ptr(t.view(np.float64)), L,
                                      t.shape[1], float(dr), int(R), net.handle if net is not None else None, _ptr(q),
                                      q.shape[0], float(bound), _ptr(score), _ptr(quat), _ptr(grid_idx),
                                      int(precision), _ptr(counts), _stream(stream)))
    return int(counts[0]), int(counts[1]), int(counts[2])


def ext_gradient_field(plan: Plan, I, h, w, H_out, theta_out, stream=None):
    _check(lib().ext_gradient_field(plan.handle, _ptr(I), int(h), int(w), _ptr(H_out), _ptr(theta_out),
                                    _stream(stream)))


def ext_consensus_radius(eps):
    return int(lib().ext_consensus_radius(float(eps)))


def ext_consensus_filter(plan: Plan, P, hp, wp, cy, cx, eps, F_out, stream=None):
    _check(lib().ext_consensus_filter(plan.handle, _ptr(P), int(hp), int(wp), int(cy), int(cx), float(eps),
                                      _ptr(F_out), _stream(stream)))


def ext_ght_detect(plan: Plan, I, h, w, F: FilterSO2, out, stream=None):
    _check(lib().ext_ght_detect(plan.handle, _ptr(I), int(h), int(w), F.ref(), _ptr(out), _stream(stream)))


def ext_conv_so2_normalized(plan: Plan, H, channels, h, w, F: FilterSO2, alpha, out, stream=None):
    _check(lib().ext_conv_so2_normalized(plan.handle, _ptr(H), int(channels), int(h), int(w), F.ref(), _ptr(alpha),
                                         _ptr(out), _stream(stream)))


def ext_filter_so2_energy(plan: Plan, F: FilterSO2):
    """Lattice energies E_k, k = 0..K, of the filter's angular components (float64 array)."""
    E = np.zeros(F.K + 1, np.float64)
    _check(lib().ext_filter_so2_energy(plan.handle, F.ref(), _ptr(E)))
    return E


def ext_corr_so2_subset(plan: Plan, H, h, w, F: FilterSO2, ks, n_angles, max_out, argmax, precision=EXT_PREC_FP32,
                        stream=None):
    k = np.ascontiguousarray(np.asarray(ks, np.int32))
    _check(lib().ext_corr_so2_subset(plan.handle, _ptr(H), int(h), int(w), F.ref(), _ptr(k), int(len(k)),
                                     int(n_angles), _ptr(max_out), _ptr(argmax), int(precision), _stream(stream)))
