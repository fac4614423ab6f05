"""CPU oracle for hybrid dealiased convolution (ctypes over plain C).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path and never imports it.

Functions (complex arrays are numpy complex128; see hdc_oracle.c for the
formula each one writes out):

* ``conv_direct(f, g)``           -- Eq. 4 per axis, double-double sums (O1)
* ``conv_direct_at(f, g, idx)``   -- the same at chosen flat output indices
* ``conv_fft(f, g)``              -- explicitly zero-padded radix-2 FFT (O2)
* ``conv_int_exact(fre, fim, gre, gim, method)`` -- exact integers (O3)
* ``closed_form_exp(A, B, P, L)`` / ``closed_form_geom(...)`` -- (O4)
* ``residue_forward / residue_backward / conv_hybrid`` -- Eq. 1, Eq. 2 (O5)
* ``conv_hermitian_direct / conv_hermitian_fft`` -- centered Hermitian (O6)
* ``dft(x, sign)``                -- the DFT by its definition
* ``mlp_loss_grad(params, sizes, X, yq, yd, n_q)`` / ``adam_step`` -- the
  parameter predictor's network in FP64 (O7)
* ``conv_unequal(f, g, m, lam, M, o, Lw)`` -- unequal lengths with residue
  matching, Section 3.5 (O8)
* ``conv_multi(xs, m, p, q, op)`` -- first L outputs of the n-fold
  convolution of n arrays, or of the sum of pairwise convolutions (O9)
* ``conv_real(f, g, m, p, q)`` -- real inputs through the packed sequence
  f + i g and conjugate residue pairs (O10)
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None
_i64 = C.c_int64
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int64)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.hdco_conv_direct.argtypes = [C.c_int, _ip, _dp, _dp, _dp]
        L.hdco_conv_direct_at.argtypes = [C.c_int, _ip, _dp, _dp, _ip, _i64, _dp]
        L.hdco_conv_fft.argtypes = [C.c_int, _ip, _dp, _dp, _dp]
        L.hdco_dft.argtypes = [_dp, _i64, C.c_int, _dp]
        L.hdco_dft.restype = None
        L.hdco_conv_int_exact_1d.argtypes = [_ip, _ip, _ip, _ip, _i64, C.c_int, _ip, _ip]
        L.hdco_closed_form_exp_1d.argtypes = [_i64, _i64, _i64, _i64, _dp]
        L.hdco_closed_form_exp_1d.restype = None
        L.hdco_closed_form_geom_1d.argtypes = [C.c_double, _i64, C.c_double, _i64, _i64, _i64, _dp]
        L.hdco_closed_form_geom_1d.restype = None
        L.hdco_residue_forward_1d.argtypes = [_dp, _i64, _i64, _i64, _i64, _dp]
        L.hdco_residue_backward_1d.argtypes = [_dp, _i64, _i64, _i64, _i64, _dp]
        L.hdco_conv_hybrid_1d.argtypes = [_dp, _dp, _i64, _i64, _i64, _i64, _dp]
        L.hdco_conv_real_1d.argtypes = [_dp, _dp, _i64, _i64, _i64, _i64, _dp]
        L.hdco_conv_multi_1d.argtypes = [_dp, C.c_int, C.c_int, _i64, _i64, _i64, _i64, _dp]
        L.hdco_conv_unequal_1d.argtypes = [_dp, _i64, _dp, _i64, _i64, _i64, _i64, _i64, _i64, _dp]
        L.hdco_conv_hermitian_2d_direct.argtypes = [_dp, _dp, _i64, _dp]
        L.hdco_conv_hermitian_2d_fft.argtypes = [_dp, _dp, _i64, _dp]
        _ip32 = C.POINTER(C.c_int)
        L.hdco_mlp_loss_grad.argtypes = [_dp, C.c_int, C.c_int, C.c_int, C.c_int, _dp, _ip32, _ip32, C.c_int,
                                         _dp, _dp, _dp]
        L.hdco_adam_step.argtypes = [_dp, _dp, _dp, _dp, C.c_long, C.c_double, C.c_double, C.c_double,
                                     C.c_double, C.c_long]
        L.hdco_adam_step.restype = None
        L.hdco_root_of_unity.argtypes = [_i64, _i64, _dp]
        L.hdco_root_of_unity.restype = None
        L.hdco_num_threads.restype = C.c_int
        L.hdco_set_num_threads.argtypes = [C.c_int]
        L.hdco_set_num_threads.restype = None
        _lib = L
    return _lib


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _dptr(a):
    return a.ctypes.data_as(_dp)


def _iptr(a):
    return a.ctypes.data_as(_ip)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def num_threads() -> int:
    return int(lib().hdco_num_threads())


def set_num_threads(n: int) -> None:
    lib().hdco_set_num_threads(int(n))


def root_of_unity(k: int, n: int) -> complex:
    out = np.zeros(2)
    lib().hdco_root_of_unity(int(k), int(n), _dptr(out))
    return complex(out[0], out[1])


def conv_direct(f, g):
    f = _c128(f)
    g = _c128(g)
    assert f.shape == g.shape and 1 <= f.ndim <= 3
    dims = np.array(f.shape, dtype=np.int64)
    h = np.empty_like(f)
    _check(lib().hdco_conv_direct(f.ndim, _iptr(dims), _dptr(f), _dptr(g), _dptr(h)), "conv_direct")
    return h


def conv_direct_at(f, g, idx):
    f = _c128(f)
    g = _c128(g)
    dims = np.array(f.shape, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty(idx.size, dtype=np.complex128)
    _check(lib().hdco_conv_direct_at(f.ndim, _iptr(dims), _dptr(f), _dptr(g), _iptr(idx),
                                     idx.size, _dptr(out)), "conv_direct_at")
    return out


def conv_fft(f, g):
    f = _c128(f)
    g = _c128(g)
    assert f.shape == g.shape and 1 <= f.ndim <= 3
    dims = np.array(f.shape, dtype=np.int64)
    h = np.empty_like(f)
    _check(lib().hdco_conv_fft(f.ndim, _iptr(dims), _dptr(f), _dptr(g), _dptr(h)), "conv_fft")
    return h


def dft(x, sign=+1):
    x = _c128(x)
    X = np.empty_like(x)
    lib().hdco_dft(_dptr(x), x.size, int(sign), _dptr(X))
    return X


def conv_int_exact(fre, fim, gre, gim, method: str = "auto"):
    """Exact first-L convolution of complex integer sequences; returns
    (re, im) int64 arrays.  method: 'direct', 'ntt' or 'auto'."""
    arrs = [np.ascontiguousarray(a, dtype=np.int64) for a in (fre, fim, gre, gim)]
    L = arrs[0].size
    if method == "auto":
        method = "direct" if L <= 4096 else "ntt"
    hre = np.empty(L, dtype=np.int64)
    him = np.empty(L, dtype=np.int64)
    _check(lib().hdco_conv_int_exact_1d(*[_iptr(a) for a in arrs], L,
                                        1 if method == "ntt" else 0, _iptr(hre), _iptr(him)),
           "conv_int_exact")
    return hre, him


def closed_form_exp(A: int, B: int, P: int, L: int):
    h = np.empty(L, dtype=np.complex128)
    lib().hdco_closed_form_exp_1d(A, B, P, L, _dptr(h))
    return h


def closed_form_geom(ra: float, A: int, rb: float, B: int, P: int, L: int):
    h = np.empty(L, dtype=np.complex128)
    lib().hdco_closed_form_geom_1d(ra, A, rb, B, P, L, _dptr(h))
    return h


def residue_forward(x, L: int, m: int, p: int, q: int):
    x = _c128(x)
    F = np.empty(q * m, dtype=np.complex128)
    _check(lib().hdco_residue_forward_1d(_dptr(x), L, m, p, q, _dptr(F)), "residue_forward")
    return F


def residue_backward(F, L: int, m: int, p: int, q: int):
    F = _c128(F)
    x = np.zeros(L, dtype=np.complex128)
    _check(lib().hdco_residue_backward_1d(_dptr(F), L, m, p, q, _dptr(x)), "residue_backward")
    return x


def conv_hybrid(f, g, m: int, p: int, q: int):
    f = _c128(f)
    g = _c128(g)
    h = np.empty_like(f)
    _check(lib().hdco_conv_hybrid_1d(_dptr(f), _dptr(g), f.size, m, p, q, _dptr(h)), "conv_hybrid")
    return h


def conv_unequal(f, g, m: int, lam: int = 1, M: int | None = None, o: int = 0, Lw: int | None = None):
    """Outputs [o, o + Lw) of the linear convolution of 1-D f and g of any
    lengths, by Section 3.5's residue matching (O8).  Defaults: M = Lf + Lg -
    1 - o, Lw = len(g)."""
    f = _c128(f)
    g = _c128(g)
    Lf, Lg = f.size, g.size
    if M is None:
        M = Lf + Lg - 1 - o
    if Lw is None:
        Lw = Lg
    h = np.empty(Lw, dtype=np.complex128)
    _check(lib().hdco_conv_unequal_1d(_dptr(f), Lf, _dptr(g), Lg, m, lam, M, o, Lw, _dptr(h)), "conv_unequal")
    return h


def conv_multi(xs, m: int, p: int = 0, q: int = 0, op: str = "product"):
    """First L outputs, for xs of shape (n, L), of x_0 * x_1 * ... * x_{n-1}
    (op 'product') or x_0 * x_1 + x_2 * x_3 + ... (op 'dot'), by the residue
    transforms (O9); p, q default to ceil(L/m) and the least alias-free q."""
    xs = np.ascontiguousarray(xs, dtype=np.complex128)
    n, L = xs.shape
    opc = {"product": 0, "dot": 1}[op]
    if p == 0:
        p = -(-L // m)
    if q == 0:
        span = n * (L - 1) + 1 if opc == 0 else 2 * L - 1
        q = -(-span // m)
    h = np.empty(L, dtype=np.complex128)
    _check(lib().hdco_conv_multi_1d(_dptr(xs), n, opc, L, m, p, q, _dptr(h)), "conv_multi")
    return h


def conv_real(f, g, m: int, p: int = 0, q: int = 0):
    """First L outputs of the convolution of real 1-D f and g by O10; p, q
    default to ceil(L/m) and ceil((2L - 1)/m)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    L = f.size
    if p == 0:
        p = -(-L // m)
    if q == 0:
        q = -(-(2 * L - 1) // m)
    h = np.empty(L, dtype=np.float64)
    _check(lib().hdco_conv_real_1d(_dptr(f), _dptr(g), L, m, p, q, _dptr(h)), "conv_real")
    return h


def conv_hermitian_direct(f, g):
    f = _c128(f)
    g = _c128(g)
    K = f.shape[1]
    assert f.shape == (2 * K - 1, K) == g.shape
    h = np.empty_like(f)
    _check(lib().hdco_conv_hermitian_2d_direct(_dptr(f), _dptr(g), K, _dptr(h)), "herm_direct")
    return h


def conv_hermitian_fft(f, g):
    f = _c128(f)
    g = _c128(g)
    K = f.shape[1]
    assert f.shape == (2 * K - 1, K) == g.shape
    h = np.empty_like(f)
    _check(lib().hdco_conv_hermitian_2d_fft(_dptr(f), _dptr(g), K, _dptr(h)), "herm_fft")
    return h


def mlp_num_params(n_in, H, n_out):
    dims = [n_in, H, H, H, n_out]
    return sum(dims[l] * dims[l + 1] + dims[l + 1] for l in range(4))


def mlp_loss_grad(params, n_in, H, n_out, X, yq, yd, n_q):
    """FP64 loss, gradient and logits of the predictor network (O7)."""
    P = np.ascontiguousarray(params, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    n = X.shape[0]
    yq = np.ascontiguousarray(yq, dtype=np.int32)
    yd = np.ascontiguousarray(yd, dtype=np.int32)
    grad = np.zeros_like(P)
    logits = np.zeros((n, n_out))
    loss = C.c_double()
    ip = C.POINTER(C.c_int)
    _check(lib().hdco_mlp_loss_grad(_dptr(P), n_in, H, n_out, n_q, _dptr(X), yq.ctypes.data_as(ip),
                                    yd.ctypes.data_as(ip), n, C.byref(loss), _dptr(grad), _dptr(logits)),
           "mlp_loss_grad")
    return loss.value, grad, logits


def adam_step(p, g, m, v, lr, b1, b2, eps, t):
    """In place on float64 arrays p, m, v."""
    lib().hdco_adam_step(_dptr(p), _dptr(np.ascontiguousarray(g, dtype=np.float64)), _dptr(m), _dptr(v), p.size,
                         lr, b1, b2, eps, t)
