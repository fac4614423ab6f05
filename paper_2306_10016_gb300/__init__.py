"""Hybrid dealiased convolution on GB300: Python binding of libhdc.so.

Argument marshalling only.  Every step of the convolution runs in the CUDA
kernels of ``libhdc.so`` (see ``include/hdc.h`` for the C ABI); PyTorch
supplies device memory and streams.  There is no CPU fallback: if the
library is missing or no GPU is present, the calls raise.

    import torch, paper_2306_10016_gb300 as hdc
    h = hdc.conv1d(f, g, m=512)              # f, g: (L,) or (B, L) complex cuda
    h = hdc.conv2d(f, g, m=(1024, 1024))     # f, g: (Lx, Ly) or (B, Lx, Ly)

Parameters follow Section 2.5 of the paper, per axis: M (padded length,
default 2L-1), m (FFT size), p and q (0: ceil(L/m), ceil(M/m)), D (residues
per pass, 0: q) and inplace (the result overwrites f).

Beyond the two-input convolution: ``convnd_window`` (slices of the linear
convolution), ``conv2d_hermitian``, ``convnd_unequal`` (unequal lengths,
residue matching), ``convnd_multi`` (n-fold product or pairwise sum of up to
8 inputs), ``convnd_real`` (real inputs), ``BatchedPlan`` (many 1-D
convolutions in one launch), ``convnd_residues`` (one rank's share),
``conv1d_noalloc`` and ``convnd_host``; searches ``tune``, ``tune_unequal``,
``tune_multi``, ``tune_real``, ``tune_random``, ``tune_proxy`` and the plan
modes of ``Plan`` (including the learned predictor, ``MLP``).
"""
from __future__ import annotations

import ctypes as C
import os

from . import build_ext as _build_ext

HDC_C64 = 0
HDC_C128 = 1

HDC_FIXED = 0
HDC_TUNE_EXHAUSTIVE = 1
HDC_PREDICT_MLP = 2
HDC_EXPLICIT = 3
HDC_TUNE_CACHED_ONLY = 4
HDC_PREDICT_MLP_SEARCH = 5
HDC_TUNE_RANDOM = 6
HDC_TUNE_PROXY = 7

HDC_OK = 0
HDC_ERR_PARAM = -1
HDC_ERR_ALIAS = -2
HDC_ERR_UNSUPPORTED_SIZE = -3
HDC_ERR_DTYPE = -4
HDC_ERR_ALLOC = -5
HDC_ERR_CUDA = -6
HDC_ERR_TIMEOUT = -7
HDC_ERR_NOT_TUNED = -8
HDC_ERR_WORKSPACE = -9
HDC_ERR_NOT_PREPARED = -10
HDC_MULTI_PRODUCT = 0
HDC_MULTI_DOT = 1
_MULTI_OPS = {"product": HDC_MULTI_PRODUCT, "dot": HDC_MULTI_DOT, HDC_MULTI_PRODUCT: HDC_MULTI_PRODUCT,
              HDC_MULTI_DOT: HDC_MULTI_DOT}

LIB_PATH = _build_ext.LIB
# the predictor network trained on this GPU's grid-search timings (a
# checkpoint of hdc_mlp_save) and the dataset it was trained on
MLP_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "mlp_gb300.bin")
MLP_DATASET = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "mlp_dataset_gb300.json.gz")

_i64 = C.c_int64
_i64p = C.POINTER(C.c_int64)
_vp = C.c_void_p
_sz = C.c_size_t

# (name, restype, argtypes) of every entry point declared in include/hdc.h
_SIGS = [
    ("hdc_strerror", C.c_char_p, [C.c_int]),
    ("hdc_version", C.c_int, []),
    ("hdc_is_good_size", C.c_int, [_i64]),
    ("hdc_next_good_size", _i64, [_i64]),
    ("hdc_derive_params", C.c_int, [_i64, _i64, _i64, _i64p, _i64p]),
    ("hdc_explicit_params", C.c_int, [_i64, _i64, _i64p, _i64p, _i64p]),
    ("hdc_validate_axis", C.c_int, [_i64, _i64, _i64, _i64, _i64, _i64, C.c_int, _i64p, _i64p, _i64p]),
    ("hdc_max_fft_size", _i64, [C.c_int]),
    ("hdc_max_padded_size", _i64, [C.c_int]),
    ("hdc_max_outer_fft_size", _i64, [C.c_int]),
    ("hdc_fft_stages", C.c_int, [_i64, C.c_int, C.c_int, C.POINTER(C.c_int), C.c_int]),
    ("hdc_workspace_size", C.c_int, [C.c_int, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, C.c_int, _i64,
                                     C.c_int, C.POINTER(_sz)]),
    ("hdc_conv1d", C.c_int, [_vp, _vp, _vp, _i64, _i64, _i64, _i64, _i64, _i64, C.c_int, C.c_int, _i64,
                             _vp, _sz, _vp]),
    ("hdc_conv2d", C.c_int, [_vp, _vp, _vp, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, C.c_int, C.c_int,
                             _i64, _vp, _sz, _vp]),
    ("hdc_conv3d", C.c_int, [_vp, _vp, _vp, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, C.c_int, C.c_int,
                             _i64, _vp, _sz, _vp]),
    ("hdc_convnd", C.c_int, [C.c_int, _vp, _vp, _vp, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, C.c_int,
                             C.c_int, _i64, _vp, _sz, _vp]),
    ("hdc_release_caches", C.c_int, []),
    ("hdc_prepare", C.c_int, [C.c_int, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, C.c_int, _i64]),
    ("hdc_prepare_window", C.c_int, [C.c_int, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, C.c_int,
                                     _i64]),
    ("hdc_prepare_hermitian", C.c_int, [_i64, _i64p, _i64p, C.c_int, _i64]),
    ("hdc_prepare_unequal", C.c_int, [C.c_int, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, C.c_int,
                                      _i64]),
    ("hdc_prepare_multi", C.c_int, [C.c_int, C.c_int, C.c_int, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, C.c_int,
                                    _i64]),
    ("hdc_prepare_real", C.c_int, [C.c_int, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, C.c_int, _i64]),
    ("hdc_probe_fma", C.c_int, [C.c_int, _i64, C.c_int, C.c_int, _vp, _vp, C.POINTER(C.c_double)]),
    ("hdc_conv1d_noalloc", C.c_int, [_vp, _vp, _vp, _i64, _i64, _i64, _i64, _i64, _i64, C.c_int, _i64, _vp]),
]



class Tuple(C.Structure):
    """hdc_tuple: one axis' (m, p, q, D), its model flops and measured ms."""
    _fields_ = [("m", C.c_int64), ("p", C.c_int64), ("q", C.c_int64), ("D", C.c_int64),
                ("model_flops", C.c_double), ("ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class UTuple(C.Structure):
    """hdc_unequal_tuple: one axis' (m, lam, qg, D) of the unequal-length
    path, its model flops and measured ms."""
    _fields_ = [("m", C.c_int64), ("lam", C.c_int64), ("q", C.c_int64), ("D", C.c_int64),
                ("model_flops", C.c_double), ("ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_tp = C.POINTER(Tuple)
_utp = C.POINTER(UTuple)
_SIGS += [
    ("hdc_tune_real_workspace_size", C.c_int, [C.c_int, _i64p, _i64p, C.c_int, _i64, C.c_double, _i64,
                                               C.POINTER(_sz)]),
    ("hdc_tune_real", C.c_int, [C.c_int, _i64p, _i64p, C.c_int, _i64, _vp, _vp, _vp, _vp, _sz, C.c_int, C.c_int,
                                C.c_double, _i64, _vp, _tp, _tp, _i64, _i64p]),
    ("hdc_tune_convnd_random", C.c_int, [C.c_int, _i64p, _i64p, C.c_int, _i64, _vp, _vp, _vp, _vp, _sz, C.c_int,
                                         C.c_int, C.c_double, _i64, _i64, C.c_uint64, _vp, _tp, _tp, _i64, _i64p]),
    ("hdc_tune_convnd_proxy", C.c_int, [C.c_int, _i64p, _i64p, C.c_int, _i64, _vp, _vp, _vp, _vp, _sz, C.c_int,
                                        C.c_int, C.c_double, _i64, _i64, _vp, _tp, _i64p]),
    ("hdc_tune_multi_workspace_size", C.c_int, [C.c_int, C.c_int, C.c_int, _i64p, _i64p, C.c_int, _i64, C.c_double,
                                                _i64, C.POINTER(_sz)]),
    ("hdc_tune_multi", C.c_int, [C.c_int, C.c_int, C.c_int, _i64p, _i64p, C.c_int, _i64, C.POINTER(_vp), _vp, _vp,
                                 _sz, C.c_int, C.c_int, C.c_double, _i64, _vp, _tp, _tp, _i64, _i64p]),
    ("hdc_tune_unequal_candidates", C.c_int, [_i64, _i64, _i64, C.c_int, C.c_double, _i64, _utp, _i64, _i64p]),
    ("hdc_tune_unequal_workspace_size", C.c_int, [C.c_int, _i64p, _i64p, _i64p, C.c_int, _i64, C.c_double, _i64,
                                                  C.POINTER(_sz)]),
    ("hdc_tune_unequal", C.c_int, [C.c_int, _i64p, _i64p, _i64p, C.c_int, _i64, _vp, _vp, _vp, _vp, _sz, C.c_int,
                                   C.c_int, C.c_double, _i64, C.c_char_p, _vp, _utp, _utp, _i64, _i64p]),
    ("hdc_workspace_size_host", C.c_int, [C.c_int, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, C.c_int, _i64,
                                          C.POINTER(_sz)]),
    ("hdc_convnd_host", C.c_int, [C.c_int, _vp, _vp, _vp, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, C.c_int,
                                  _i64, _vp, _sz, _vp]),
    ("hdc_tune_candidates", C.c_int, [_i64, _i64, C.c_int, C.c_double, _i64, _tp, _i64, _i64p]),
    ("hdc_tune_workspace_size", C.c_int, [C.c_int, _i64p, _i64p, C.c_int, _i64, C.c_double, _i64,
                                          C.POINTER(_sz)]),
    ("hdc_tune_convnd", C.c_int, [C.c_int, _i64p, _i64p, C.c_int, _i64, _vp, _vp, _vp, _vp, _sz, C.c_int, C.c_int,
                                  C.c_double, _i64, _vp, _tp, _tp, _i64, _i64p]),
    ("hdc_tune_conv1d", C.c_int, [_i64, _i64, C.c_int, _i64, _vp, _vp, _vp, _vp, _sz, C.c_int, C.c_int, C.c_double,
                                  _i64, _vp, _tp, _tp, _i64, _i64p]),
    ("hdc_plan_create", C.c_int, [C.POINTER(_vp), C.c_int, _i64p, _i64p, _i64p, _i64p, C.c_int, _i64, C.c_int,
                                  C.c_char_p, _vp]),
    ("hdc_plan_params", C.c_int, [_vp, _i64p, _i64p, _i64p, _i64p]),
    ("hdc_plan_workspace", _sz, [_vp]),
    ("hdc_plan_execute", C.c_int, [_vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    ("hdc_plan_destroy", C.c_int, [_vp]),
    ("hdc_batched_create", C.c_int, [C.POINTER(_vp), _i64, _i64p, _i64p, C.c_int]),
    ("hdc_batched_workspace", _sz, [_vp]),
    ("hdc_batched_params", C.c_int, [_vp, _i64p, _i64p, _i64p, _i64p, _i64p]),
    ("hdc_batched_execute", C.c_int, [_vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    ("hdc_batched_status", C.c_int, [_vp, C.POINTER(C.c_int)]),
    ("hdc_batched_phase_ms", C.c_int, [_vp, C.POINTER(C.c_double)]),
    ("hdc_batched_set_barrier", C.c_int, [_vp, C.c_longlong, C.c_int]),
    ("hdc_batched_destroy", C.c_int, [_vp]),
    ("hdc_batched_tune", C.c_int, [_i64, _i64p, C.c_int, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp), C.c_int,
                                   C.c_int, _vp, _i64p, C.POINTER(C.c_double)]),
    ("hdc_workspace_size_window", C.c_int, [C.c_int, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p,
                                            C.c_int, _i64, C.POINTER(_sz)]),
    ("hdc_convnd_window", C.c_int, [C.c_int, _vp, _vp, _vp, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p,
                                    C.c_int, _i64, _vp, _sz, _vp]),
    ("hdc_validate_unequal_axis", C.c_int, [_i64, _i64, _i64, _i64, _i64, _i64, C.c_int, _i64p, _i64p, _i64p,
                                            _i64p]),
    ("hdc_workspace_size_unequal", C.c_int, [C.c_int, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p,
                                             C.c_int, _i64, C.POINTER(_sz)]),
    ("hdc_convnd_unequal", C.c_int, [C.c_int, _vp, _vp, _vp, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p,
                                     _i64p, C.c_int, _i64, _vp, _sz, _vp]),
    ("hdc_workspace_size_multi", C.c_int, [C.c_int, C.c_int, C.c_int, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p,
                                           C.c_int, _i64, C.POINTER(_sz)]),
    ("hdc_convnd_multi", C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(_vp), _vp, _i64p, _i64p, _i64p, _i64p,
                                   _i64p, _i64p, C.c_int, _i64, _vp, _sz, _vp]),
    ("hdc_workspace_size_real", C.c_int, [C.c_int, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, C.c_int, _i64,
                                          C.POINTER(_sz)]),
    ("hdc_convnd_real", C.c_int, [C.c_int, _vp, _vp, _vp, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, C.c_int, _i64,
                                  _vp, _sz, _vp]),
    ("hdc_workspace_size_hermitian", C.c_int, [_i64, _i64p, _i64p, C.c_int, _i64, C.POINTER(_sz)]),
    ("hdc_conv2d_hermitian", C.c_int, [_vp, _vp, _vp, _i64, _i64p, _i64p, C.c_int, _i64, _vp, _sz, _vp]),
    ("hdc_mlp_create", C.c_int, [C.POINTER(_vp), C.c_int, C.c_int, C.c_int]),
    ("hdc_mlp_num_params", C.c_int, [_vp]),
    ("hdc_mlp_set_params", C.c_int, [_vp, C.POINTER(C.c_float)]),
    ("hdc_mlp_get_params", C.c_int, [_vp, C.POINTER(C.c_float)]),
    ("hdc_mlp_get_grads", C.c_int, [_vp, C.POINTER(C.c_float)]),
    ("hdc_mlp_forward", C.c_int, [_vp, _vp, _i64, _vp, _vp]),
    ("hdc_mlp_loss_grad", C.c_int, [_vp, _vp, _vp, _vp, _i64, C.c_int, _vp, _vp]),
    ("hdc_mlp_adam", C.c_int, [_vp, C.c_float, C.c_float, C.c_float, C.c_float, _vp]),
    ("hdc_mlp_save", C.c_int, [_vp, C.c_char_p]),
    ("hdc_mlp_load", C.c_int, [_vp, C.c_char_p]),
    ("hdc_mlp_destroy", C.c_int, [_vp]),
    ("hdc_mlp_num_q_classes", C.c_int, []),
    ("hdc_mlp_q_class", _i64, [C.c_int]),
    ("hdc_mlp_q_to_class", C.c_int, [_i64]),
    ("hdc_mlp_axis_features", C.c_int, [C.c_int, _i64p, _i64p, C.c_int, _i64, C.POINTER(C.c_float)]),
    ("hdc_plan_timed", _i64, [_vp]),
    ("hdc_mlp_decode_class", C.c_int, [C.c_int, C.c_int, _i64, _i64, C.c_int, _i64, _i64p, _i64p, _i64p, _i64p]),
    ("hdc_mlp_decode_axis", C.c_int, [C.POINTER(C.c_float), C.c_int, _i64, _i64, C.c_int, _i64, C.c_int, _i64p,
                                      _i64p, _i64p, _i64p]),
    ("hdc_convnd_residues", C.c_int, [C.c_int, _vp, _vp, _vp, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p, _i64, _i64,
                                      C.c_int, _i64, _vp, _sz, _vp]),
    ("hdc_last_cuda_error", C.c_int, []),
    ("hdc_last_cuda_error_name", C.c_char_p, []),
    ("hdc_set_tma", C.c_int, [C.c_int]),
    ("hdc_set_cluster", C.c_int, [C.c_int]),
    ("hdc_device_status", C.c_int, [C.POINTER(C.c_int), C.c_int]),
    ("hdc_stats_reset", C.c_int, []),
    ("hdc_stats_timing", C.c_int, [C.c_int]),
    ("hdc_stats_kernel_count", C.c_int, []),
    ("hdc_stats_kernel_name", C.c_char_p, [C.c_int]),
    ("hdc_stats_total_launches", _i64, []),
    ("hdc_stats_get", C.c_int, [C.c_int, _i64p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                C.POINTER(C.c_double)]),
]

_lib = None


class HDCError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = strerror(code) if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")


def build(force: bool = False) -> str:
    """Compile libhdc.so for sm_103a (nvcc) if it is missing or stale."""
    return _build_ext.build(force=force)


def lib() -> C.CDLL:
    """The loaded libhdc.so.  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2306_10016_gb300.build() "
                               "(there is no fallback implementation)")
        L = C.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, what: str) -> None:
    if rc != HDC_OK:
        if rc == HDC_ERR_CUDA:
            what = f"{what} [{lib().hdc_last_cuda_error_name().decode()}]"
        raise HDCError(rc, what)


def _arr(vals):
    if vals is None:
        return None  # NULL: the library's default for that argument
    a = (C.c_int64 * len(vals))(*[int(v) for v in vals])
    return a


# ------------------------------------------------------------ host helpers

def strerror(code: int) -> str:
    return lib().hdc_strerror(int(code)).decode()


def is_good_size(n: int) -> bool:
    return bool(lib().hdc_is_good_size(int(n)))


def next_good_size(n: int) -> int:
    return int(lib().hdc_next_good_size(int(n)))


def derive_params(L: int, M: int, m: int):
    p, q = C.c_int64(), C.c_int64()
    _check(lib().hdc_derive_params(L, M, m, C.byref(p), C.byref(q)), "derive_params")
    return p.value, q.value


def explicit_params(L: int, M: int):
    m, p, q = C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib().hdc_explicit_params(L, M, C.byref(m), C.byref(p), C.byref(q)), "explicit_params")
    return m.value, p.value, q.value


def validate_axis(L, M, m, p=0, q=0, D=0, dtype=HDC_C128):
    """Returns the status code and the resolved (p, q, D)."""
    po, qo, Do = C.c_int64(), C.c_int64(), C.c_int64()
    rc = lib().hdc_validate_axis(L, M, m, p, q, D, dtype, C.byref(po), C.byref(qo), C.byref(Do))
    return rc, (po.value, qo.value, Do.value)


def max_fft_size(dtype=HDC_C128) -> int:
    return int(lib().hdc_max_fft_size(dtype))


def max_padded_size(dtype=HDC_C128) -> int:
    return int(lib().hdc_max_padded_size(dtype))


FFT_ROWS, FFT_COLS, FFT_OTHER = 0, 1, 2


def fft_stages(n: int, dtype=HDC_C128, kind=FFT_ROWS) -> list:
    """hdc_fft_stages: the radices, first stage first, of the n-point
    transform a kernel of the given kind runs (host only)."""
    buf = (C.c_int * 32)()
    rc = lib().hdc_fft_stages(n, dtype, kind, buf, 32)
    if rc < 0:
        _check(rc, "hdc_fft_stages")
    return list(buf[:rc])


def _per_axis(v, dims, name):
    if v is None:
        return None
    if isinstance(v, (list, tuple)):
        if len(v) != dims:
            raise ValueError(f"{name} needs {dims} entries")
        return [int(x) for x in v]
    return [int(v)] * dims


def workspace_size(L, M, m, p=0, q=0, D=0, dtype=HDC_C128, batch=1, inplace=False) -> int:
    dims = len(L)
    M, m, p, q, D = (_per_axis(v, dims, n) for v, n in ((M, "M"), (m, "m"), (p, "p"), (q, "q"), (D, "D")))
    nb = C.c_size_t()
    rc = lib().hdc_workspace_size(dims, _arr(L), _arr(M), _arr(m), _arr(p), _arr(q), _arr(D), dtype,
                                  int(batch), int(bool(inplace)), C.byref(nb))
    _check(rc, "workspace_size")
    return nb.value


# ------------------------------------------------------- torch entry points

def _torch():
    import torch
    return torch


def dtype_code(t) -> int:
    torch = _torch()
    if t == torch.complex128:
        return HDC_C128
    if t == torch.complex64:
        return HDC_C64
    raise TypeError(f"unsupported dtype {t}: use torch.complex64 or torch.complex128")


_PREPARED = set()
_CLUSTER_MODE = [1]     # the route rule of hdc_set_cluster: it decides which tables a call reads


def _plain(a):
    if a is None or isinstance(a, (int, float)):
        return a
    try:
        return tuple(a)
    except TypeError:
        return repr(a)


def _prepare(name: str, *args) -> None:
    """Make the twiddle tables a convolution call reads (hdc_prepare*) on the
    current device, unless a stream capture is running: the convolution
    calls themselves allocate nothing, and a table made during a capture
    would break it (the call then fails with HDC_ERR_NOT_PREPARED).  Calls
    already prepared on this device are remembered, so a repeated call costs
    a set lookup."""
    torch = _torch()
    key = (name, torch.cuda.current_device(), _CLUSTER_MODE[0], tuple(_plain(a) for a in args))
    if key in _PREPARED:
        return
    if torch.cuda.is_current_stream_capturing():
        return
    _check(getattr(lib(), name)(*args), name)
    _PREPARED.add(key)


def prepare(L, m, M=None, p=0, q=0, D=0, dtype=HDC_C128, batch=1) -> None:
    """hdc_prepare: the twiddle tables of convnd / conv1d-3d / convnd_host /
    convnd_residues for these per-axis parameters (lists) on the current
    device."""
    dims = len(L)
    Mv = _per_axis(M, dims, "M") or [2 * int(x) - 1 for x in L]
    _check(lib().hdc_prepare(dims, _arr(L), _arr(Mv), _arr(_per_axis(m, dims, "m")), _arr(_per_axis(p, dims, "p")),
                             _arr(_per_axis(q, dims, "q")), _arr(_per_axis(D, dims, "D")), dtype, batch),
           "hdc_prepare")


def convnd(f, g, dims: int, m, M=None, p=0, q=0, D=0, out=None, inplace=False, workspace=None,
           stream=None):
    """First L outputs per axis of the linear convolution of f and g over
    their last `dims` axes; leading axes are a batch.  Returns the output
    tensor (f itself when inplace)."""
    torch = _torch()
    if not (f.is_cuda and g.is_cuda):
        raise ValueError("f and g must be CUDA tensors (there is no CPU path)")
    if f.shape != g.shape or f.dtype != g.dtype:
        raise ValueError("f and g must have the same shape and dtype")
    if f.dim() < dims:
        raise ValueError(f"need at least {dims} axes")
    if not (f.is_contiguous() and g.is_contiguous()):
        raise ValueError("f and g must be contiguous")
    dt = dtype_code(f.dtype)
    L = [int(x) for x in f.shape[f.dim() - dims:]]
    batch = 1
    for x in f.shape[: f.dim() - dims]:
        batch *= int(x)
    Mv = _per_axis(M, dims, "M") or [2 * l - 1 for l in L]
    mv = _per_axis(m, dims, "m")
    pv = _per_axis(p, dims, "p")
    qv = _per_axis(q, dims, "q")
    Dv = _per_axis(D, dims, "D")
    if inplace:
        h = f
    else:
        h = out if out is not None else torch.empty_like(f)
        if h.shape != f.shape or h.dtype != f.dtype or not h.is_contiguous() or not h.is_cuda:
            raise ValueError("out must match f")
    nbytes = workspace_size(L, Mv, mv, pv, qv, Dv, dt, batch, inplace)
    if workspace is None or workspace.numel() * workspace.element_size() < nbytes:
        workspace = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=f.device)
    st = stream if stream is not None else torch.cuda.current_stream(f.device)
    with torch.cuda.device(f.device):
        _prepare("hdc_prepare", dims, _arr(L), _arr(Mv), _arr(mv), _arr(pv), _arr(qv), _arr(Dv), dt, batch)
        rc = lib().hdc_convnd(dims, f.data_ptr(), g.data_ptr(), h.data_ptr(), _arr(L), _arr(Mv), _arr(mv),
                              _arr(pv), _arr(qv), _arr(Dv), int(bool(inplace)), dt, batch,
                              workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                              st.cuda_stream)
    _check(rc, "hdc_convnd")
    return h


def convnd_window(f, g, dims, m, o, Lw, M=None, p=0, q=0, D=0, out=None, workspace=None, stream=None):
    """Outputs [o, o + Lw) per axis of the linear convolution of f and g
    over their last `dims` axes (hdc_convnd_window); M defaults to 2L - 1."""
    torch = _torch()
    if not (f.is_cuda and g.is_cuda) or f.shape != g.shape or f.dtype != g.dtype:
        raise ValueError("f and g must be CUDA tensors of one shape and dtype")
    dt = dtype_code(f.dtype)
    L = [int(x) for x in f.shape[f.dim() - dims:]]
    lead = list(f.shape[: f.dim() - dims])
    batch = 1
    for x in lead:
        batch *= int(x)
    Mv = _per_axis(M, dims, "M") or [2 * l - 1 for l in L]
    mv, pv, qv, Dv, ov, Lwv = (_per_axis(v, dims, n) for v, n in ((m, "m"), (p, "p"), (q, "q"), (D, "D"),
                                                                  (o, "o"), (Lw, "Lw")))
    h = out if out is not None else torch.empty(lead + Lwv, dtype=f.dtype, device=f.device)
    nb = C.c_size_t()
    _check(lib().hdc_workspace_size_window(dims, _arr(L), _arr(Mv), _arr(mv), _arr(pv), _arr(qv), _arr(Dv), _arr(ov),
                                           _arr(Lwv), dt, batch, C.byref(nb)), "workspace_size_window")
    if workspace is None or workspace.numel() * workspace.element_size() < nb.value:
        workspace = torch.empty(max(1, nb.value), dtype=torch.uint8, device=f.device)
    st = stream if stream is not None else torch.cuda.current_stream(f.device)
    with torch.cuda.device(f.device):
        _prepare("hdc_prepare_window", dims, _arr(L), _arr(Mv), _arr(mv), _arr(pv), _arr(qv), _arr(Dv), _arr(ov),
                 _arr(Lwv), dt, batch)
        _check(lib().hdc_convnd_window(dims, f.data_ptr(), g.data_ptr(), h.data_ptr(), _arr(L), _arr(Mv), _arr(mv),
                                       _arr(pv), _arr(qv), _arr(Dv), _arr(ov), _arr(Lwv), dt, batch,
                                       workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                       st.cuda_stream), "hdc_convnd_window")
    return h


def _multi_op(op) -> int:
    if op not in _MULTI_OPS:
        raise ValueError("op must be 'product' or 'dot'")
    return _MULTI_OPS[op]


def workspace_size_multi(n, L, m, op="product", M=None, p=0, q=0, D=0, dtype=HDC_C128, batch=1) -> int:
    dims = len(L)
    mv, Mv, pv, qv, Dv = (_per_axis(v, dims, k) for v, k in ((m, "m"), (M, "M"), (p, "p"), (q, "q"), (D, "D")))
    nb = C.c_size_t()
    _check(lib().hdc_workspace_size_multi(dims, int(n), _multi_op(op), _arr(L), _arr(Mv), _arr(mv), _arr(pv),
                                          _arr(qv), _arr(Dv), dtype, int(batch), C.byref(nb)), "workspace_size_multi")
    return nb.value


def convnd_multi(xs, dims, m, op="product", M=None, p=0, q=0, D=0, out=None, workspace=None, stream=None):
    """First L outputs per axis over the last `dims` axes of the n-fold
    convolution xs[0] * ... * xs[n-1] (op 'product') or of the sum of
    pairwise convolutions xs[0] * xs[1] + xs[2] * xs[3] + ... (op 'dot');
    xs: a list of 2..8 CUDA tensors of one shape and dtype (leading axes
    are a batch).  hdc_convnd_multi."""
    torch = _torch()
    xs = list(xs)
    n = len(xs)
    x0 = xs[0]
    for x in xs:
        if not x.is_cuda or x.shape != x0.shape or x.dtype != x0.dtype or not x.is_contiguous():
            raise ValueError("inputs must be contiguous CUDA tensors of one shape and dtype")
    dt = dtype_code(x0.dtype)
    L = [int(v) for v in x0.shape[x0.dim() - dims:]]
    batch = 1
    for v in x0.shape[: x0.dim() - dims]:
        batch *= int(v)
    mv, Mv, pv, qv, Dv = (_per_axis(v, dims, k) for v, k in ((m, "m"), (M, "M"), (p, "p"), (q, "q"), (D, "D")))
    h = out if out is not None else torch.empty_like(x0)
    nb = C.c_size_t()
    opc = _multi_op(op)
    _check(lib().hdc_workspace_size_multi(dims, n, opc, _arr(L), _arr(Mv), _arr(mv), _arr(pv), _arr(qv), _arr(Dv), dt,
                                          batch, C.byref(nb)), "workspace_size_multi")
    if workspace is None or workspace.numel() * workspace.element_size() < nb.value:
        workspace = torch.empty(max(1, nb.value), dtype=torch.uint8, device=x0.device)
    ptrs = (_vp * n)(*[x.data_ptr() for x in xs])
    st = stream if stream is not None else torch.cuda.current_stream(x0.device)
    with torch.cuda.device(x0.device):
        _prepare("hdc_prepare_multi", dims, n, opc, _arr(L), _arr(Mv), _arr(mv), _arr(pv), _arr(qv), _arr(Dv), dt,
                 batch)
        _check(lib().hdc_convnd_multi(dims, n, opc, ptrs, h.data_ptr(), _arr(L), _arr(Mv), _arr(mv), _arr(pv), _arr(qv),
                                      _arr(Dv), dt, batch, workspace.data_ptr(),
                                      workspace.numel() * workspace.element_size(), st.cuda_stream),
               "hdc_convnd_multi")
    return h


def workspace_size_real(L, m, M=None, p=0, q=0, D=0, dtype=HDC_C128, batch=1) -> int:
    dims = len(L)
    mv, Mv, pv, qv, Dv = (_per_axis(v, dims, k) for v, k in ((m, "m"), (M, "M"), (p, "p"), (q, "q"), (D, "D")))
    Mv = Mv or [2 * l - 1 for l in L]
    nb = C.c_size_t()
    _check(lib().hdc_workspace_size_real(dims, _arr(L), _arr(Mv), _arr(mv), _arr(pv), _arr(qv), _arr(Dv), dtype,
                                         int(batch), C.byref(nb)), "workspace_size_real")
    return nb.value


def convnd_real(f, g, dims, m, M=None, p=0, q=0, D=0, out=None, workspace=None, stream=None):
    """First L outputs per axis of the convolution of REAL f and g (float64
    or float32 CUDA tensors of one shape) over their last `dims` axes, by the
    packed transform of f + i g and conjugate residue pairs
    (hdc_convnd_real); the result is real."""
    torch = _torch()
    if not (f.is_cuda and g.is_cuda) or f.shape != g.shape or f.dtype != g.dtype:
        raise ValueError("f and g must be CUDA tensors of one shape and dtype")
    if not (f.is_contiguous() and g.is_contiguous()):
        raise ValueError("f and g must be contiguous")
    if f.dtype == torch.float64:
        dt = HDC_C128
    elif f.dtype == torch.float32:
        dt = HDC_C64
    else:
        raise TypeError(f"unsupported dtype {f.dtype}: use torch.float32 or torch.float64")
    L = [int(x) for x in f.shape[f.dim() - dims:]]
    batch = 1
    for x in f.shape[: f.dim() - dims]:
        batch *= int(x)
    mv, Mv, pv, qv, Dv = (_per_axis(v, dims, k) for v, k in ((m, "m"), (M, "M"), (p, "p"), (q, "q"), (D, "D")))
    Mv = Mv or [2 * l - 1 for l in L]
    h = out if out is not None else torch.empty_like(f)
    nb = C.c_size_t()
    _check(lib().hdc_workspace_size_real(dims, _arr(L), _arr(Mv), _arr(mv), _arr(pv), _arr(qv), _arr(Dv), dt, batch,
                                         C.byref(nb)), "workspace_size_real")
    if workspace is None or workspace.numel() * workspace.element_size() < nb.value:
        workspace = torch.empty(max(1, nb.value), dtype=torch.uint8, device=f.device)
    st = stream if stream is not None else torch.cuda.current_stream(f.device)
    with torch.cuda.device(f.device):
        _prepare("hdc_prepare_real", dims, _arr(L), _arr(Mv), _arr(mv), _arr(pv), _arr(qv), _arr(Dv), dt, batch)
        _check(lib().hdc_convnd_real(dims, f.data_ptr(), g.data_ptr(), h.data_ptr(), _arr(L), _arr(Mv), _arr(mv),
                                     _arr(pv), _arr(qv), _arr(Dv), dt, batch, workspace.data_ptr(),
                                     workspace.numel() * workspace.element_size(), st.cuda_stream),
               "hdc_convnd_real")
    return h


def validate_unequal_axis(Lf, Lg, m, lam=1, M=0, D=0, dtype=HDC_C128):
    """(pf, pg, qg, D) of one unequal-length axis (hdc_validate_unequal_axis);
    raises HdcError when the tuple is invalid."""
    pf, pg, qg, Do = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib().hdc_validate_unequal_axis(int(Lf), int(Lg), int(M or 0), int(m), int(lam), int(D), dtype,
                                           C.byref(pf), C.byref(pg), C.byref(qg), C.byref(Do)),
           "validate_unequal_axis")
    return pf.value, pg.value, qg.value, Do.value


def workspace_size_unequal(Lf, Lg, m, lam=1, M=None, D=0, o=None, Lw=None, dtype=HDC_C128, batch=1) -> int:
    dims = len(Lf)
    mv, lv, Mv, Dv, ov, Lwv = (_per_axis(v, dims, n) for v, n in ((m, "m"), (lam, "lam"), (M, "M"), (D, "D"),
                                                                  (o, "o"), (Lw, "Lw")))
    nb = C.c_size_t()
    _check(lib().hdc_workspace_size_unequal(dims, _arr(Lf), _arr(Lg), _arr(Mv), _arr(mv), _arr(lv), _arr(Dv),
                                            _arr(ov), _arr(Lwv), dtype, int(batch), C.byref(nb)),
           "workspace_size_unequal")
    return nb.value


def convnd_unequal(f, g, dims, m, lam=1, M=None, D=0, o=None, Lw=None, out=None, workspace=None, stream=None):
    """Convolution of f and g of different lengths over their last `dims`
    axes (hdc_convnd_unequal): f at m points, g at lam * m points per axis,
    residues matched; leading axes (equal for f and g) are a batch.  Output
    per axis: the window [o, o + Lw) of the linear convolution (default: the
    first Lg outputs)."""
    torch = _torch()
    if not (f.is_cuda and g.is_cuda) or f.dtype != g.dtype:
        raise ValueError("f and g must be CUDA tensors of one dtype")
    if not (f.is_contiguous() and g.is_contiguous()):
        raise ValueError("f and g must be contiguous")
    if f.dim() < dims or g.dim() != f.dim() or f.shape[: f.dim() - dims] != g.shape[: g.dim() - dims]:
        raise ValueError("f and g need the same leading (batch) axes")
    dt = dtype_code(f.dtype)
    Lf = [int(x) for x in f.shape[f.dim() - dims:]]
    Lg = [int(x) for x in g.shape[g.dim() - dims:]]
    lead = list(f.shape[: f.dim() - dims])
    batch = 1
    for x in lead:
        batch *= int(x)
    mv, lv, Mv, Dv, ov, Lwv = (_per_axis(v, dims, n) for v, n in ((m, "m"), (lam, "lam"), (M, "M"), (D, "D"),
                                                                  (o, "o"), (Lw, "Lw")))
    shape = Lwv if Lwv is not None else Lg
    h = out if out is not None else torch.empty(lead + shape, dtype=f.dtype, device=f.device)
    nb = C.c_size_t()
    _check(lib().hdc_workspace_size_unequal(dims, _arr(Lf), _arr(Lg), _arr(Mv), _arr(mv), _arr(lv), _arr(Dv),
                                            _arr(ov), _arr(Lwv), dt, batch, C.byref(nb)), "workspace_size_unequal")
    if workspace is None or workspace.numel() * workspace.element_size() < nb.value:
        workspace = torch.empty(max(1, nb.value), dtype=torch.uint8, device=f.device)
    st = stream if stream is not None else torch.cuda.current_stream(f.device)
    with torch.cuda.device(f.device):
        _prepare("hdc_prepare_unequal", dims, _arr(Lf), _arr(Lg), _arr(Mv), _arr(mv), _arr(lv), _arr(Dv), _arr(ov),
                 _arr(Lwv), dt, batch)
        _check(lib().hdc_convnd_unequal(dims, f.data_ptr(), g.data_ptr(), h.data_ptr(), _arr(Lf), _arr(Lg),
                                        _arr(Mv), _arr(mv), _arr(lv), _arr(Dv), _arr(ov), _arr(Lwv), dt, batch,
                                        workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                        st.cuda_stream), "hdc_convnd_unequal")
    return h


def conv2d_hermitian(f, g, m=None, D=0, out=None, workspace=None, stream=None):
    """Centered Hermitian 2-D convolution of half-plane spectra (2K-1, K)
    (leading axes: batch), padding 3/2; m per axis defaults to K."""
    torch = _torch()
    if not (f.is_cuda and g.is_cuda) or f.shape != g.shape or f.dtype != g.dtype:
        raise ValueError("f and g must be CUDA tensors of one shape and dtype")
    K = int(f.shape[-1])
    if int(f.shape[-2]) != 2 * K - 1:
        raise ValueError("half-plane spectra have shape (2K-1, K)")
    batch = f.numel() // ((2 * K - 1) * K)
    dt = dtype_code(f.dtype)
    mv = _arr(_per_axis(m if m is not None else K, 2, "m"))
    Dv = _arr(_per_axis(D, 2, "D"))
    h = out if out is not None else torch.empty_like(f)
    nb = C.c_size_t()
    _check(lib().hdc_workspace_size_hermitian(K, mv, Dv, dt, batch, C.byref(nb)), "workspace_size_hermitian")
    if workspace is None or workspace.numel() * workspace.element_size() < nb.value:
        workspace = torch.empty(max(1, nb.value), dtype=torch.uint8, device=f.device)
    st = stream if stream is not None else torch.cuda.current_stream(f.device)
    with torch.cuda.device(f.device):
        _prepare("hdc_prepare_hermitian", K, mv, Dv, dt, batch)
        _check(lib().hdc_conv2d_hermitian(f.data_ptr(), g.data_ptr(), h.data_ptr(), K, mv, Dv, dt, batch,
                                          workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                          st.cuda_stream), "hdc_conv2d_hermitian")
    return h


def convnd_residues(f, g, dims, m, r_lo, r_hi, M=None, p=0, q=0, D=0, out=None, workspace=None, stream=None):
    """The share of residues [r_lo, r_hi) of axis 0 (hdc_convnd_residues);
    the shares of disjoint ranges add up to the convolution."""
    torch = _torch()
    if not (f.is_cuda and g.is_cuda) or f.shape != g.shape or f.dtype != g.dtype:
        raise ValueError("f and g must be CUDA tensors of one shape and dtype")
    dt = dtype_code(f.dtype)
    L = [int(x) for x in f.shape[f.dim() - dims:]]
    batch = 1
    for x in f.shape[: f.dim() - dims]:
        batch *= int(x)
    Mv = _per_axis(M, dims, "M") or [2 * l - 1 for l in L]
    mv, pv, qv, Dv = (_per_axis(v, dims, n) for v, n in ((m, "m"), (p, "p"), (q, "q"), (D, "D")))
    h = out if out is not None else torch.empty_like(f)
    nbytes = workspace_size(L, Mv, mv, pv, qv, Dv, dt, batch)
    if workspace is None or workspace.numel() * workspace.element_size() < nbytes:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=f.device)
    st = stream if stream is not None else torch.cuda.current_stream(f.device)
    with torch.cuda.device(f.device):
        _prepare("hdc_prepare", dims, _arr(L), _arr(Mv), _arr(mv), _arr(pv), _arr(qv), _arr(Dv), dt, batch)
        _check(lib().hdc_convnd_residues(dims, f.data_ptr(), g.data_ptr(), h.data_ptr(), _arr(L), _arr(Mv), _arr(mv),
                                         _arr(pv), _arr(qv), _arr(Dv), int(r_lo), int(r_hi), dt, batch,
                                         workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                         st.cuda_stream), "hdc_convnd_residues")
    return h


def conv1d(f, g, m, M=None, p=0, q=0, D=0, **kw):
    return convnd(f, g, 1, m, M, p, q, D, **kw)


def conv2d(f, g, m, M=None, p=0, q=0, D=0, **kw):
    return convnd(f, g, 2, m, M, p, q, D, **kw)


def conv3d(f, g, m, M=None, p=0, q=0, D=0, **kw):
    return convnd(f, g, 3, m, M, p, q, D, **kw)


def probe_fma_peak(dtype=HDC_C128, iters=1 << 16, blocks=None, threads=256, reps=5, device=None):
    """Measured vector FMA throughput in TFLOP/s (best of reps launches)."""
    torch = _torch()
    dev = torch.device(device or "cuda")
    props = torch.cuda.get_device_properties(dev)
    blocks = blocks or props.multi_processor_count * 8
    out = torch.empty(blocks * threads, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream(dev)
    fl = C.c_double()
    best = 0.0
    with torch.cuda.device(dev):
        for i in range(reps + 1):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            _check(lib().hdc_probe_fma(dtype, iters, blocks, threads, out.data_ptr(), st.cuda_stream,
                                       C.byref(fl)), "probe_fma")
            e1.record(st)
            e1.synchronize()
            if i:
                best = max(best, fl.value / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    return best


# ------------------------------------------------------------- host buffers

def workspace_size_host(L, M, m, p=0, q=0, D=0, dtype=HDC_C128, batch=1) -> int:
    dims = len(L)
    M, m, p, q, D = (_per_axis(v, dims, n) for v, n in ((M, "M"), (m, "m"), (p, "p"), (q, "q"), (D, "D")))
    nb = C.c_size_t()
    _check(lib().hdc_workspace_size_host(dims, _arr(L), _arr(M), _arr(m), _arr(p), _arr(q), _arr(D), dtype,
                                         int(batch), C.byref(nb)), "workspace_size_host")
    return nb.value


def convnd_host(f, g, h, dims, m, M=None, p=0, q=0, D=0, workspace=None, stream=None, sync=True):
    """The convolution on host tensors f, g -> h (CPU torch tensors, pinned
    for overlap); copies in, convolution and copy out all run through one C
    call on the device.  With sync (default) the stream is synchronised
    before returning; without it h is valid once the stream has reached this
    point, so calls on several streams (each with its own workspace) overlap
    one call's copies with another's kernels."""
    torch = _torch()
    for t in (f, g, h):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError("convnd_host takes contiguous host tensors")
    dt = dtype_code(f.dtype)
    L = [int(x) for x in f.shape[f.dim() - dims:]]
    batch = 1
    for x in f.shape[: f.dim() - dims]:
        batch *= int(x)
    Mv = _per_axis(M, dims, "M") or [2 * l - 1 for l in L]
    args = [_per_axis(v, dims, n) for v, n in ((m, "m"), (p, "p"), (q, "q"), (D, "D"))]
    nbytes = workspace_size_host(L, Mv, *args, dtype=dt, batch=batch)
    if workspace is None or workspace.numel() * workspace.element_size() < nbytes:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = stream if stream is not None else torch.cuda.current_stream(workspace.device)
    with torch.cuda.device(workspace.device):
        _prepare("hdc_prepare", dims, _arr(L), _arr(Mv), *[_arr(a) for a in args], dt, batch)
    _check(lib().hdc_convnd_host(dims, f.data_ptr(), g.data_ptr(), h.data_ptr(), _arr(L), _arr(Mv),
                                 *[_arr(a) for a in args], dt, batch, workspace.data_ptr(),
                                 workspace.numel() * workspace.element_size(), st.cuda_stream), "convnd_host")
    if sync:
        st.synchronize()
    return h


# -------------------------------------------------------- parameter search

def tune_candidates(L: int, M: int, dtype=HDC_C128, max_ratio=2.0, m_min=16):
    n = C.c_int64()
    _check(lib().hdc_tune_candidates(L, M, dtype, max_ratio, m_min, None, 0, C.byref(n)), "tune_candidates")
    buf = (Tuple * max(1, n.value))()
    _check(lib().hdc_tune_candidates(L, M, dtype, max_ratio, m_min, buf, n.value, C.byref(n)), "tune_candidates")
    return [buf[i].as_dict() for i in range(n.value)]


def tune(f, g, dims, M=None, max_ratio=2.0, m_min=16, warmup=1, reps=3, out=None, stream=None):
    """Grid search (Section 4.2) on the given device tensors; returns
    (best per axis, trials) where trials is a list of per-axis dict lists."""
    torch = _torch()
    dt = dtype_code(f.dtype)
    L = [int(x) for x in f.shape[f.dim() - dims:]]
    batch = 1
    for x in f.shape[: f.dim() - dims]:
        batch *= int(x)
    Mv = _per_axis(M, dims, "M") or [2 * l - 1 for l in L]
    nb = C.c_size_t()
    _check(lib().hdc_tune_workspace_size(dims, _arr(L), _arr(Mv), dt, batch, max_ratio, m_min, C.byref(nb)),
           "tune_workspace_size")
    ws = torch.empty(max(1, nb.value), dtype=torch.uint8, device=f.device)
    h = out if out is not None else torch.empty_like(f)
    cap = 4096
    best = (Tuple * dims)()
    trials = (Tuple * (cap * dims))()
    nt = C.c_int64()
    st = stream if stream is not None else torch.cuda.current_stream(f.device)
    with torch.cuda.device(f.device):
        _check(lib().hdc_tune_convnd(dims, _arr(L), _arr(Mv), dt, batch, f.data_ptr(), g.data_ptr(), h.data_ptr(),
                                     ws.data_ptr(), nb.value, warmup, reps, max_ratio, m_min, st.cuda_stream, best,
                                     trials, cap, C.byref(nt)), "tune_convnd")
    tr = [[trials[i * dims + a].as_dict() for a in range(dims)] for i in range(min(nt.value, cap))]
    return [best[a].as_dict() for a in range(dims)], tr


def _tune_setup(f, g, dims, M, max_ratio, m_min):
    torch = _torch()
    dt = dtype_code(f.dtype)
    L = [int(x) for x in f.shape[f.dim() - dims:]]
    batch = 1
    for x in f.shape[: f.dim() - dims]:
        batch *= int(x)
    Mv = _per_axis(M, dims, "M") or [2 * l - 1 for l in L]
    nb = C.c_size_t()
    _check(lib().hdc_tune_workspace_size(dims, _arr(L), _arr(Mv), dt, batch, max_ratio, m_min, C.byref(nb)),
           "tune_workspace_size")
    ws = torch.empty(max(1, nb.value), dtype=torch.uint8, device=f.device)
    return dt, L, batch, Mv, ws, nb.value


def tune_real(f, g, dims, M=None, max_ratio=1.5, m_min=16, warmup=1, reps=3, stream=None):
    """Grid search of (m, D) per axis for hdc_convnd_real on real CUDA
    tensors f, g; returns (best per axis, trials)."""
    torch = _torch()
    dt = HDC_C128 if f.dtype == torch.float64 else HDC_C64
    L = [int(x) for x in f.shape[f.dim() - dims:]]
    batch = 1
    for x in f.shape[: f.dim() - dims]:
        batch *= int(x)
    Mv = _per_axis(M, dims, "M") or [2 * l - 1 for l in L]
    nb = C.c_size_t()
    _check(lib().hdc_tune_real_workspace_size(dims, _arr(L), _arr(Mv), dt, batch, max_ratio, m_min, C.byref(nb)),
           "tune_real_workspace_size")
    ws = torch.empty(max(1, nb.value), dtype=torch.uint8, device=f.device)
    h = torch.empty_like(f)
    cap = 4096
    best = (Tuple * dims)()
    trials = (Tuple * (cap * dims))()
    nt = C.c_int64()
    st = stream if stream is not None else torch.cuda.current_stream(f.device)
    with torch.cuda.device(f.device):
        _check(lib().hdc_tune_real(dims, _arr(L), _arr(Mv), dt, batch, f.data_ptr(), g.data_ptr(), h.data_ptr(),
                                   ws.data_ptr(), nb.value, warmup, reps, max_ratio, m_min, st.cuda_stream, best,
                                   trials, cap, C.byref(nt)), "tune_real")
    tr = [[trials[i * dims + a].as_dict() for a in range(dims)] for i in range(min(nt.value, cap))]
    return [best[a].as_dict() for a in range(dims)], tr


def tune_random(f, g, dims, n_samples=0, seed=230610016, M=None, max_ratio=2.0, m_min=16, warmup=1, reps=3,
                stream=None):
    """Random search (Section 4.3, A1): n_samples candidates per axis (0: a
    quarter, at least 3) drawn with a seeded SplitMix64 stream, then the
    separable search; returns (best per axis, trials)."""
    torch = _torch()
    dt, L, batch, Mv, ws, wsb = _tune_setup(f, g, dims, M, max_ratio, m_min)
    h = torch.empty_like(f)
    cap = 4096
    best = (Tuple * dims)()
    trials = (Tuple * (cap * dims))()
    nt = C.c_int64()
    st = stream if stream is not None else torch.cuda.current_stream(f.device)
    with torch.cuda.device(f.device):
        _check(lib().hdc_tune_convnd_random(dims, _arr(L), _arr(Mv), dt, batch, f.data_ptr(), g.data_ptr(),
                                            h.data_ptr(), ws.data_ptr(), wsb, warmup, reps, max_ratio, m_min,
                                            int(n_samples), int(seed), st.cuda_stream, best, trials, cap,
                                            C.byref(nt)), "tune_convnd_random")
    tr = [[trials[i * dims + a].as_dict() for a in range(dims)] for i in range(min(nt.value, cap))]
    return [best[a].as_dict() for a in range(dims)], tr


def tune_proxy(f, g, dims, Lproxy=32, M=None, max_ratio=2.0, m_min=16, warmup=1, reps=3, stream=None):
    """Per axis, the separable search on the rectangle with every other axis
    cut to Lproxy points (Section 6.3 heuristic); returns (best per axis,
    number of timed configurations)."""
    torch = _torch()
    dt, L, batch, Mv, ws, wsb = _tune_setup(f, g, dims, M, max_ratio, m_min)
    h = torch.empty_like(f)
    best = (Tuple * dims)()
    nt = C.c_int64()
    st = stream if stream is not None else torch.cuda.current_stream(f.device)
    with torch.cuda.device(f.device):
        _check(lib().hdc_tune_convnd_proxy(dims, _arr(L), _arr(Mv), dt, batch, f.data_ptr(), g.data_ptr(),
                                           h.data_ptr(), ws.data_ptr(), wsb, warmup, reps, max_ratio, m_min,
                                           int(Lproxy), st.cuda_stream, best, C.byref(nt)), "tune_convnd_proxy")
    return [best[a].as_dict() for a in range(dims)], nt.value


def tune_unequal_candidates(Lf: int, Lg: int, M: int = 0, dtype=HDC_C128, max_ratio=1.5, m_min=16):
    """Candidate (m, lam, qg) of one unequal-length axis, by model flops."""
    n = C.c_int64()
    _check(lib().hdc_tune_unequal_candidates(Lf, Lg, M, dtype, max_ratio, m_min, None, 0, C.byref(n)),
           "tune_unequal_candidates")
    buf = (UTuple * max(1, n.value))()
    _check(lib().hdc_tune_unequal_candidates(Lf, Lg, M, dtype, max_ratio, m_min, buf, n.value, C.byref(n)),
           "tune_unequal_candidates")
    return [buf[i].as_dict() for i in range(n.value)]


def tune_unequal(f, g, dims, M=None, max_ratio=1.5, m_min=16, warmup=1, reps=3, tuning_db=None, stream=None):
    """Grid search of (m, lam, D) per axis for hdc_convnd_unequal on the given
    device tensors (first Lg outputs); returns (best per axis, trials).  With
    tuning_db, a stored result is returned without timing (trials empty)."""
    torch = _torch()
    dt = dtype_code(f.dtype)
    Lf = [int(x) for x in f.shape[f.dim() - dims:]]
    Lg = [int(x) for x in g.shape[g.dim() - dims:]]
    batch = 1
    for x in f.shape[: f.dim() - dims]:
        batch *= int(x)
    Mv = _per_axis(M, dims, "M")
    nb = C.c_size_t()
    _check(lib().hdc_tune_unequal_workspace_size(dims, _arr(Lf), _arr(Lg), _arr(Mv), dt, batch, max_ratio, m_min,
                                                 C.byref(nb)), "tune_unequal_workspace_size")
    ws = torch.empty(max(1, nb.value), dtype=torch.uint8, device=f.device)
    h = torch.empty(list(g.shape), dtype=g.dtype, device=g.device)
    cap = 4096
    best = (UTuple * dims)()
    trials = (UTuple * (cap * dims))()
    nt = C.c_int64()
    st = stream if stream is not None else torch.cuda.current_stream(f.device)
    db = os.fsencode(tuning_db) if tuning_db else None
    with torch.cuda.device(f.device):
        _check(lib().hdc_tune_unequal(dims, _arr(Lf), _arr(Lg), _arr(Mv), dt, batch, f.data_ptr(), g.data_ptr(),
                                      h.data_ptr(), ws.data_ptr(), nb.value, warmup, reps, max_ratio, m_min, db,
                                      st.cuda_stream, best, trials, cap, C.byref(nt)), "tune_unequal")
    tr = [[trials[i * dims + a].as_dict() for a in range(dims)] for i in range(min(nt.value, cap))]
    return [best[a].as_dict() for a in range(dims)], tr


def tune_multi(xs, dims, op="product", M=None, max_ratio=1.5, m_min=16, warmup=1, reps=3, stream=None):
    """Grid search of (m, D) per axis for hdc_convnd_multi with operator op
    on the given inputs (a list of 2..8 CUDA tensors of one shape); returns
    (best per axis, trials)."""
    torch = _torch()
    xs = list(xs)
    n = len(xs)
    x0 = xs[0]
    dt = dtype_code(x0.dtype)
    L = [int(v) for v in x0.shape[x0.dim() - dims:]]
    batch = 1
    for v in x0.shape[: x0.dim() - dims]:
        batch *= int(v)
    opc = _multi_op(op)
    k = n if opc == HDC_MULTI_PRODUCT else 2
    Mv = _per_axis(M, dims, "M") or [k * (l - 1) + 1 for l in L]
    nb = C.c_size_t()
    _check(lib().hdc_tune_multi_workspace_size(dims, n, opc, _arr(L), _arr(Mv), dt, batch, max_ratio, m_min,
                                               C.byref(nb)), "tune_multi_workspace_size")
    ws = torch.empty(max(1, nb.value), dtype=torch.uint8, device=x0.device)
    h = torch.empty_like(x0)
    cap = 4096
    best = (Tuple * dims)()
    trials = (Tuple * (cap * dims))()
    nt = C.c_int64()
    ptrs = (_vp * n)(*[x.data_ptr() for x in xs])
    st = stream if stream is not None else torch.cuda.current_stream(x0.device)
    with torch.cuda.device(x0.device):
        _check(lib().hdc_tune_multi(dims, n, opc, _arr(L), _arr(Mv), dt, batch, ptrs, h.data_ptr(), ws.data_ptr(),
                                    nb.value, warmup, reps, max_ratio, m_min, st.cuda_stream, best, trials, cap,
                                    C.byref(nt)), "tune_multi")
    tr = [[trials[i * dims + a].as_dict() for a in range(dims)] for i in range(min(nt.value, cap))]
    return [best[a].as_dict() for a in range(dims)], tr


class Plan:
    """(m, p, q, D) per axis fixed for one problem shape (hdc_plan_*)."""

    def __init__(self, L, M=None, dtype=HDC_C128, batch=1, mode=HDC_TUNE_EXHAUSTIVE, m=None, D=None,
                 tuning_db=None, stream=None):
        torch = _torch()
        self.L = [int(x) for x in L]
        self.dims = len(self.L)
        self.M = _per_axis(M, self.dims, "M") or [2 * l - 1 for l in self.L]
        self.dtype = dtype
        self.batch = int(batch)
        h = C.c_void_p()
        st = stream if stream is not None else torch.cuda.current_stream()
        mm = _arr(_per_axis(m, self.dims, "m")) if m is not None else None
        DD = _arr(_per_axis(D, self.dims, "D")) if D is not None else None
        if tuning_db is None and mode in (HDC_PREDICT_MLP, HDC_PREDICT_MLP_SEARCH):
            tuning_db = MLP_WEIGHTS
        db = tuning_db.encode() if tuning_db else None
        _check(lib().hdc_plan_create(C.byref(h), self.dims, _arr(self.L), _arr(self.M), mm, DD, dtype, self.batch,
                                     mode, db, st.cuda_stream), "plan_create")
        self._h = h

    @property
    def params(self):
        arrs = [(C.c_int64 * self.dims)() for _ in range(4)]
        _check(lib().hdc_plan_params(self._h, *arrs), "plan_params")
        return [dict(m=arrs[0][i], p=arrs[1][i], q=arrs[2][i], D=arrs[3][i]) for i in range(self.dims)]

    @property
    def workspace_bytes(self) -> int:
        return int(lib().hdc_plan_workspace(self._h))

    @property
    def timed(self) -> int:
        """Configurations timed while the plan was made."""
        return int(lib().hdc_plan_timed(self._h))

    def execute(self, f, g, out=None, workspace=None, stream=None):
        torch = _torch()
        h = out if out is not None else torch.empty_like(f)
        nbytes = self.workspace_bytes
        if workspace is None or workspace.numel() * workspace.element_size() < nbytes:
            workspace = torch.empty(nbytes, dtype=torch.uint8, device=f.device)
        st = stream if stream is not None else torch.cuda.current_stream(f.device)
        _check(lib().hdc_plan_execute(self._h, f.data_ptr(), g.data_ptr(), h.data_ptr(), workspace.data_ptr(),
                                      workspace.numel() * workspace.element_size(), st.cuda_stream), "plan_execute")
        return h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.hdc_plan_destroy(self._h)
            self._h = None


# --------------------------------------------------------- batched plans

def _ptr_arrays(ts):
    return (C.c_void_p * len(ts))(*[t.data_ptr() for t in ts])


def batched_tune(fs, gs, hs, reps=3, max_cands=12, stream=None):
    """Per-size-class m for the batched kernel (hdc_batched_tune) on the
    given lists of device tensors; returns (m list, summed best ms)."""
    torch = _torch()
    n = len(fs)
    L = _arr([int(t.shape[-1]) for t in fs])
    m = (C.c_int64 * n)()
    ms = C.c_double()
    st = stream if stream is not None else torch.cuda.current_stream(fs[0].device)
    _check(lib().hdc_batched_tune(n, L, dtype_code(fs[0].dtype), _ptr_arrays(fs), _ptr_arrays(gs), _ptr_arrays(hs),
                                  reps, max_cands, st.cuda_stream, m, C.byref(ms)), "batched_tune")
    return list(m), ms.value


class BatchedPlan:
    """n 1-D convolutions of lengths L (M = 2L-1) and FFT sizes m in one
    persistent launch (hdc_batched_*)."""

    def __init__(self, L, m, dtype=HDC_C128):
        self.L = [int(x) for x in L]
        self.n = len(self.L)
        h = C.c_void_p()
        _check(lib().hdc_batched_create(C.byref(h), self.n, _arr(self.L), _arr(m), dtype), "batched_create")
        self._h = h
        self.dtype = dtype
        self._ptrs = None

    @property
    def workspace_bytes(self) -> int:
        return int(lib().hdc_batched_workspace(self._h))

    @property
    def params(self):
        arrs = [(C.c_int64 * self.n)() for _ in range(5)]
        _check(lib().hdc_batched_params(self._h, *arrs), "batched_params")
        return [dict(L=self.L[i], m=arrs[0][i], p=arrs[1][i], q=arrs[2][i], m1=arrs[3][i], m2=arrs[4][i])
                for i in range(self.n)]

    def bind(self, fs, gs, hs):
        """Device arrays of the n input/output pointers (kept by the plan, so a
        captured launch keeps reading valid arrays)."""
        torch = _torch()
        dev = fs[0].device
        self._ptrs = [torch.tensor([t.data_ptr() for t in ts], dtype=torch.int64, device=dev) for ts in (fs, gs, hs)]
        return self._ptrs

    def execute(self, workspace, stream=None):
        torch = _torch()
        if self._ptrs is None:
            raise RuntimeError("bind() the input and output tensors first")
        st = stream if stream is not None else torch.cuda.current_stream(workspace.device)
        pf, pg, ph = self._ptrs
        _check(lib().hdc_batched_execute(self._h, pf.data_ptr(), pg.data_ptr(), ph.data_ptr(), workspace.data_ptr(),
                                         workspace.numel() * workspace.element_size(), st.cuda_stream),
               "batched_execute")

    @staticmethod
    def status(workspace) -> int:
        v = C.c_int()
        _check(lib().hdc_batched_status(workspace.data_ptr(), C.byref(v)), "batched_status")
        return v.value

    @staticmethod
    def phase_ms(workspace) -> list:
        """Durations (ms) of the last execute's four phases: column folds and
        FFTs, rows, inverse column FFTs, unfolds."""
        v = (C.c_double * 4)()
        _check(lib().hdc_batched_phase_ms(workspace.data_ptr(), v), "batched_phase_ms")
        return [float(x) for x in v]

    def set_barrier(self, spin_limit: int, extra_arrivals: int = 0):
        _check(lib().hdc_batched_set_barrier(self._h, int(spin_limit), int(extra_arrivals)), "batched_set_barrier")

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.hdc_batched_destroy(self._h)
            self._h = None


# ------------------------------------------------------ learned predictor

MLP_FEATURES = 12
MLP_HIDDEN = 64


def mlp_q_classes():
    return [int(lib().hdc_mlp_q_class(k)) for k in range(lib().hdc_mlp_num_q_classes())]


def mlp_q_to_class(q: int) -> int:
    return int(lib().hdc_mlp_q_to_class(int(q)))


def mlp_axis_features(L, M=None, dtype=HDC_C128, batch=1):
    import numpy as np
    dims = len(L)
    Mv = M if M is not None else [2 * l - 1 for l in L]
    out = (C.c_float * (dims * MLP_FEATURES))()
    _check(lib().hdc_mlp_axis_features(dims, _arr(L), _arr(Mv), dtype, int(batch), out), "mlp_axis_features")
    return np.array(out, dtype=np.float32).reshape(dims, MLP_FEATURES)


def max_outer_fft_size(dtype=HDC_C128) -> int:
    return int(lib().hdc_max_outer_fft_size(dtype))


def mlp_decode_axis(logits, L: int, M: int, dtype=HDC_C128, max_m: int = 0, rank: int = 0):
    import numpy as np
    lg = np.ascontiguousarray(logits, dtype=np.float32)
    m, p, q, D = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib().hdc_mlp_decode_axis(lg.ctypes.data_as(C.POINTER(C.c_float)), lg.size - 2, L, M, dtype, int(max_m),
                                     int(rank), C.byref(m), C.byref(p), C.byref(q), C.byref(D)), "mlp_decode_axis")
    return dict(m=m.value, p=p.value, q=q.value, D=D.value)


class MLP:
    """The parameter predictor network on the GPU (hdc_mlp_*)."""

    def __init__(self, n_in=MLP_FEATURES, hidden=MLP_HIDDEN, n_out=None):
        if n_out is None:
            n_out = lib().hdc_mlp_num_q_classes() + 2
        self.n_in, self.hidden, self.n_out = n_in, hidden, n_out
        h = C.c_void_p()
        _check(lib().hdc_mlp_create(C.byref(h), n_in, hidden, n_out), "mlp_create")
        self._h = h
        self.n_params = int(lib().hdc_mlp_num_params(h))

    def set_params(self, params):
        import numpy as np
        a = np.ascontiguousarray(params, dtype=np.float32)
        assert a.size == self.n_params
        _check(lib().hdc_mlp_set_params(self._h, a.ctypes.data_as(C.POINTER(C.c_float))), "mlp_set_params")

    def params(self):
        import numpy as np
        a = np.empty(self.n_params, dtype=np.float32)
        _check(lib().hdc_mlp_get_params(self._h, a.ctypes.data_as(C.POINTER(C.c_float))), "mlp_get_params")
        return a

    def grads(self):
        import numpy as np
        a = np.empty(self.n_params, dtype=np.float32)
        _check(lib().hdc_mlp_get_grads(self._h, a.ctypes.data_as(C.POINTER(C.c_float))), "mlp_get_grads")
        return a

    def _check_inputs(self, X, *labels):
        if X.dim() != 2 or X.shape[1] != self.n_in or X.dtype != _torch().float32 or not X.is_contiguous():
            raise ValueError(f"X must be a contiguous float32 (n, {self.n_in}) tensor")
        for y in labels:
            if y.shape != (X.shape[0],) or y.dtype != _torch().int32:
                raise ValueError("labels must be int32 (n,) tensors")

    def forward(self, X, stream=None):
        torch = _torch()
        self._check_inputs(X)
        out = torch.empty((X.shape[0], self.n_out), dtype=torch.float32, device=X.device)
        st = stream if stream is not None else torch.cuda.current_stream(X.device)
        _check(lib().hdc_mlp_forward(self._h, X.data_ptr(), X.shape[0], out.data_ptr(), st.cuda_stream), "mlp_forward")
        return out

    def loss_grad(self, X, yq, yd, loss_out, stream=None):
        """Device tensors: X float32 (n, n_in), yq / yd int32 (n,), loss_out float32 (1,)."""
        torch = _torch()
        self._check_inputs(X, yq, yd)
        st = stream if stream is not None else torch.cuda.current_stream(X.device)
        _check(lib().hdc_mlp_loss_grad(self._h, X.data_ptr(), yq.data_ptr(), yd.data_ptr(), X.shape[0],
                                       self.n_out - 2, loss_out.data_ptr(), st.cuda_stream), "mlp_loss_grad")

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        torch = _torch()
        st = stream if stream is not None else torch.cuda.current_stream()
        _check(lib().hdc_mlp_adam(self._h, lr, beta1, beta2, eps, st.cuda_stream), "mlp_adam")

    def save(self, path):
        _check(lib().hdc_mlp_save(self._h, str(path).encode()), "mlp_save")

    def load(self, path):
        _check(lib().hdc_mlp_load(self._h, str(path).encode()), "mlp_load")

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.hdc_mlp_destroy(self._h)
            self._h = None


# ------------------------------------------------------ load path, status

def set_tma(enable: bool) -> None:
    """Allow (default) or forbid the TMA-staged loads of the strided fold
    for later launches; both paths give the same result."""
    _check(lib().hdc_set_tma(int(bool(enable))), "set_tma")


def set_cluster(mode) -> None:
    """hdc_set_cluster: the thread-block-cluster route of short 1-D
    convolutions never (False / 0), where it is faster (True / 1, the
    default) or wherever it fits (2); same results either way."""
    _check(lib().hdc_set_cluster(int(mode)), "hdc_set_cluster")
    _CLUSTER_MODE[0] = int(mode)


def device_status(clear: bool = True) -> int:
    """0, or HDC_ERR_TIMEOUT if a kernel gave up waiting for a copy since the
    last clear (synchronises with the device)."""
    st = C.c_int()
    _check(lib().hdc_device_status(C.byref(st), int(bool(clear))), "device_status")
    return st.value


# ------------------------------------------------------- launch statistics

def stats_reset() -> None:
    lib().hdc_stats_reset()


def stats_timing(on: bool) -> None:
    lib().hdc_stats_timing(int(bool(on)))


def total_launches() -> int:
    return int(lib().hdc_stats_total_launches())


def stats() -> dict:
    """{kernel: {launches, ms, flops, bytes}} since the last reset (read
    after synchronising)."""
    out = {}
    for k in range(lib().hdc_stats_kernel_count()):
        n = C.c_int64()
        ms, fl, by = C.c_double(), C.c_double(), C.c_double()
        _check(lib().hdc_stats_get(k, C.byref(n), C.byref(ms), C.byref(fl), C.byref(by)), "stats_get")
        out[lib().hdc_stats_kernel_name(k).decode()] = dict(launches=n.value, ms=ms.value, flops=fl.value,
                                                             bytes=by.value)
    return out


def conv1d_noalloc(f, g, m, M=None, p=0, q=0, D=0, out=None, stream=None):
    """hdc_conv1d_noalloc: the 1-D convolution with the library's fixed
    device scratch array instead of a workspace (no device allocation in the
    call; `out` must be given by callers that cannot allocate either)."""
    torch = _torch()
    if not (f.is_cuda and g.is_cuda) or f.shape != g.shape or f.dtype != g.dtype:
        raise ValueError("f and g must be CUDA tensors of one shape and dtype")
    L = int(f.shape[-1])
    batch = f.numel() // L if L else 0
    h = out if out is not None else torch.empty_like(f)
    st = stream if stream is not None else torch.cuda.current_stream(f.device)
    with torch.cuda.device(f.device):
        rc = lib().hdc_conv1d_noalloc(f.data_ptr(), g.data_ptr(), h.data_ptr(), L,
                                      int(M) if M is not None else 2 * L - 1, int(m), int(p), int(q), int(D),
                                      dtype_code(f.dtype), batch, st.cuda_stream)
    _check(rc, "hdc_conv1d_noalloc")
    return h


def release_caches() -> None:
    _check(lib().hdc_release_caches(), "release_caches")
    _PREPARED.clear()
