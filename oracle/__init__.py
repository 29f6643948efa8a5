"""Python access to the plain FP64 CPU oracle (``vqe_oracle.c``).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library: it loads its own gcc-built ``libvqe_oracle.so``.

Each function restates one definition of the method (Sec. II-B Eqs. 2-7,
Sec. II-D and III-D); the C source documents the conventions.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_u64_p = ctypes.POINTER(ctypes.c_uint64)


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.orc_threads.restype = ctypes.c_int
        lib.orc_slim.restype = ctypes.c_size_t
        _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(_c_double_p)


def _u(a):
    return a.ctypes.data_as(_c_u64_p)


def _terms(x, z, c):
    x = np.ascontiguousarray(x, dtype=np.uint64)
    z = np.ascontiguousarray(z, dtype=np.uint64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    assert x.shape == z.shape == c.shape
    return x, z, c


def threads() -> int:
    return _load().orc_threads()


def ansatz_state(n: int, depth: int, params) -> np.ndarray:
    """psi(params) = U(params)|0...0> as complex128 (Sec. II-B, Eq. 6)."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    assert p.size == 2 * n * depth
    psi = np.empty(1 << n, dtype=np.complex128)
    _load().orc_ansatz(ctypes.c_int(n), ctypes.c_int(depth), _d(p),
                       psi.ctypes.data_as(ctypes.c_void_p))
    return psi


def apply_1q(psi: np.ndarray, q: int, u) -> np.ndarray:
    n = int(psi.size).bit_length() - 1
    out = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    m = np.ascontiguousarray(np.asarray(u, dtype=np.complex128).reshape(4))
    _load().orc_apply_1q(ctypes.c_int(n), out.ctypes.data_as(ctypes.c_void_p), ctypes.c_int(q),
                         m.ctypes.data_as(ctypes.c_void_p))
    return out


def ry_matrix(theta: float) -> np.ndarray:
    u = np.empty(4, dtype=np.complex128)
    _load().orc_ry_matrix(ctypes.c_double(theta), u.ctypes.data_as(ctypes.c_void_p))
    return u.reshape(2, 2)


def rz_matrix(phi: float) -> np.ndarray:
    u = np.empty(4, dtype=np.complex128)
    _load().orc_rz_matrix(ctypes.c_double(phi), u.ctypes.data_as(ctypes.c_void_p))
    return u.reshape(2, 2)


def pauli_apply(psi: np.ndarray, x: int, z: int) -> np.ndarray:
    n = int(psi.size).bit_length() - 1
    src = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty_like(src)
    _load().orc_pauli_apply(ctypes.c_int(n), src.ctypes.data_as(ctypes.c_void_p),
                            ctypes.c_uint64(x), ctypes.c_uint64(z),
                            out.ctypes.data_as(ctypes.c_void_p))
    return out


def expectation(psi: np.ndarray, x, z, c):
    """Unnormalised <psi|H|psi> as (real, imag) and <psi|psi> (Eq. 7 parts)."""
    n = int(psi.size).bit_length() - 1
    x, z, c = _terms(x, z, c)
    src = np.ascontiguousarray(psi, dtype=np.complex128)
    er, ei, nn = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _load().orc_expectation(ctypes.c_int(n), src.ctypes.data_as(ctypes.c_void_p),
                            ctypes.c_size_t(c.size), _u(x), _u(z), _d(c),
                            ctypes.byref(er), ctypes.byref(ei), ctypes.byref(nn))
    return er.value, ei.value, nn.value


def energy(psi: np.ndarray, x, z, c):
    """E = <psi|H|psi>/<psi|psi> and <psi|psi> (Eq. 7)."""
    er, _, nn = expectation(psi, x, z, c)
    return er / nn, nn


def apply_h(psi: np.ndarray, x, z, c) -> np.ndarray:
    n = int(psi.size).bit_length() - 1
    x, z, c = _terms(x, z, c)
    src = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty_like(src)
    _load().orc_apply_h(ctypes.c_int(n), src.ctypes.data_as(ctypes.c_void_p),
                        ctypes.c_size_t(c.size), _u(x), _u(z), _d(c),
                        out.ctypes.data_as(ctypes.c_void_p))
    return out


def slim(x, z, c, threshold: float):
    """Merge, drop exact zeros, drop |c| < threshold (Sec. II-D, III-D).

    Returns ``(x, z, c, sum_abs_dropped)`` sorted by ``(x, z)``.
    """
    x, z, c = _terms(x, z, c)
    xo, zo, co = np.empty_like(x), np.empty_like(z), np.empty_like(c)
    dropped = ctypes.c_double()
    k = _load().orc_slim(ctypes.c_size_t(c.size), _u(x), _u(z), _d(c), ctypes.c_double(threshold),
                         _u(xo), _u(zo), _d(co), ctypes.byref(dropped))
    return xo[:k].copy(), zo[:k].copy(), co[:k].copy(), dropped.value


def gradient_adjoint(n: int, depth: int, params, x, z, c):
    """Adjoint-method gradient of <psi|H|psi>; returns (grad, energy)."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    x, z, c = _terms(x, z, c)
    g = np.empty(2 * n * depth)
    e = ctypes.c_double()
    _load().orc_gradient_adjoint(ctypes.c_int(n), ctypes.c_int(depth), _d(p), ctypes.c_size_t(c.size),
                                 _u(x), _u(z), _d(c), _d(g), ctypes.byref(e))
    return g, e.value


def gradient_shift(n: int, depth: int, params, x, z, c) -> np.ndarray:
    p = np.ascontiguousarray(params, dtype=np.float64)
    x, z, c = _terms(x, z, c)
    g = np.empty(2 * n * depth)
    _load().orc_gradient_shift(ctypes.c_int(n), ctypes.c_int(depth), _d(p), ctypes.c_size_t(c.size),
                               _u(x), _u(z), _d(c), _d(g))
    return g


def gradient_fd(n: int, depth: int, params, x, z, c, h: float = 1e-5) -> np.ndarray:
    p = np.ascontiguousarray(params, dtype=np.float64)
    x, z, c = _terms(x, z, c)
    g = np.empty(2 * n * depth)
    _load().orc_gradient_fd(ctypes.c_int(n), ctypes.c_int(depth), _d(p), ctypes.c_size_t(c.size),
                            _u(x), _u(z), _d(c), ctypes.c_double(h), _d(g))
    return g


# ---------------------------------------------------------------- particle-conserving ansatz

def _exc(exc):
    e = np.ascontiguousarray(exc, dtype=np.int32).reshape(-1, 4)
    return e, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def apply_excitation(psi: np.ndarray, exc, theta: float) -> np.ndarray:
    """exp(theta (T - T^dag)) psi for one excitation (p, q, r, s) (Sec. II-B, Eq. 5)."""
    n = int(psi.size).bit_length() - 1
    out = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    e, ep = _exc(exc)
    _load().orc_apply_excitation(ctypes.c_int(n), out.ctypes.data_as(ctypes.c_void_p), ep,
                                 ctypes.c_double(theta))
    return out


def excitation_generator(psi: np.ndarray, exc) -> np.ndarray:
    n = int(psi.size).bit_length() - 1
    src = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty_like(src)
    e, ep = _exc(exc)
    _load().orc_excitation_generator(ctypes.c_int(n), src.ctypes.data_as(ctypes.c_void_p), ep,
                                     out.ctypes.data_as(ctypes.c_void_p))
    return out


def pc_ansatz_state(n: int, n_elec: int, exc, theta) -> np.ndarray:
    """psi(theta) = U(theta) psi_HF of the particle-conserving ansatz (Eqs. 5-6)."""
    e, ep = _exc(exc)
    t = np.ascontiguousarray(theta, dtype=np.float64)
    assert t.size == e.shape[0]
    psi = np.empty(1 << n, dtype=np.complex128)
    _load().orc_pc_ansatz(ctypes.c_int(n), ctypes.c_int(n_elec), ctypes.c_int(e.shape[0]), ep, _d(t),
                          psi.ctypes.data_as(ctypes.c_void_p))
    return psi


def pc_gradient_adjoint(n: int, n_elec: int, exc, theta, x, z, c):
    """Adjoint gradient of <psi|H|psi> for the particle-conserving ansatz; (grad, energy)."""
    e, ep = _exc(exc)
    t = np.ascontiguousarray(theta, dtype=np.float64)
    x, z, c = _terms(x, z, c)
    g = np.empty(max(e.shape[0], 1))
    en = ctypes.c_double()
    _load().orc_pc_gradient_adjoint(ctypes.c_int(n), ctypes.c_int(n_elec), ctypes.c_int(e.shape[0]),
                                    ep, _d(t), ctypes.c_size_t(c.size), _u(x), _u(z), _d(c), _d(g),
                                    ctypes.byref(en))
    return g[:e.shape[0]], en.value


def pc_gradient_fd(n: int, n_elec: int, exc, theta, x, z, c, h: float = 1e-5) -> np.ndarray:
    e, ep = _exc(exc)
    t = np.ascontiguousarray(theta, dtype=np.float64)
    x, z, c = _terms(x, z, c)
    g = np.empty(max(e.shape[0], 1))
    _load().orc_pc_gradient_fd(ctypes.c_int(n), ctypes.c_int(n_elec), ctypes.c_int(e.shape[0]), ep,
                               _d(t), ctypes.c_size_t(c.size), _u(x), _u(z), _d(c),
                               ctypes.c_double(h), _d(g))
    return g[:e.shape[0]]
