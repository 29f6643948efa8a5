"""Single amplitudes of the ansatz state by a sum over computational paths.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA library.

The ansatz of Sec. II-B (Eq. 6, hardware-efficient form) with D layers is
    U = prod_l  CZchain * prod_q RZ(phi_lq) RY(theta_lq),
applied to |0...0>.  Expanding the matrix product in the computational basis,
every qubit wire q carries a path b_q = (b_q0, ..., b_q,D-1) of bit values
(b_ql = the value of qubit q after the rotations of layer l), starting from 0
and ending at bit q of the output index i.  Then

    <i|U|0> = sum over all paths  prod_q w_q(b_q) * prod_{q<n-1} (-1)^{<b_q, b_q+1>}

with the single-wire weight
    w_q(b) = prod_l RY(theta_lq)[b_l, b_(l-1)] * RZ(phi_lq)[b_l, b_l]   (b_(-1) = 0)
and <b, c> = sum_l b_l c_l (mod 2), the sign of the CZ(q, q+1) gates of all
layers.  Summing the wires one at a time along the chain,

    F_0 = w_0,   F_(q+1)(c) = w_(q+1)(c) * sum_b F_q(b) (-1)^{<b, c>},
    <i|U|0> = sum_b F_(n-1)(b),

where the inner sum is a Walsh-Hadamard transform over the D path bits.  One
amplitude costs about n * D * 2^D operations, so single amplitudes of 32-qubit
states (D = 8) or 24-qubit states (D = 12) are cheap, while the full state
never exists.  Conventions as in the rest of the oracle:
RY(t) = [[c, -s], [s, c]], RZ(p) = diag(e^{-ip/2}, e^{ip/2}), qubit q = bit q,
params[(l*n + q)*2] = theta, +1 = phi.
"""
from __future__ import annotations

import numpy as np


def _wire_weights(theta, phi, out_bit: int) -> np.ndarray:
    """w(b) for every path b (bit l of the path index = value after layer l)."""
    D = len(theta)
    paths = np.arange(1 << D)
    w = np.ones(1 << D, dtype=np.complex128)
    prev = np.zeros(1 << D, dtype=np.int64)
    for l in range(D):
        cur = (paths >> l) & 1
        c, s = np.cos(theta[l] / 2.0), np.sin(theta[l] / 2.0)
        ry = np.array([[c, -s], [s, c]])
        rz = np.array([np.exp(-0.5j * phi[l]), np.exp(0.5j * phi[l])])
        w = w * ry[cur, prev] * rz[cur]
        prev = cur
    # the path must end at the requested output bit
    w[((paths >> (D - 1)) & 1) != out_bit] = 0.0
    return w


def _wht(v: np.ndarray) -> np.ndarray:
    """sum_b v(b) (-1)^{popc(b & c)} for every c (unnormalised)."""
    D = int(np.log2(v.size))
    a = v.reshape((2,) * D).copy()
    for ax in range(D):
        x0 = np.take(a, 0, axis=ax)
        x1 = np.take(a, 1, axis=ax)
        a = np.stack([x0 + x1, x0 - x1], axis=ax)
    return a.reshape(-1)


def amplitude(n: int, depth: int, params, index: int) -> complex:
    """<index| U(params) |0...0> for the n-qubit, depth-D ansatz."""
    p = np.asarray(params, dtype=np.float64).reshape(depth, n, 2)
    F = None
    for q in range(n):
        w = _wire_weights(p[:, q, 0], p[:, q, 1], (int(index) >> q) & 1)
        F = w if F is None else w * _wht(F)
    return complex(F.sum())


def amplitudes(n: int, depth: int, params, indices) -> np.ndarray:
    """amplitude() for each index."""
    return np.array([amplitude(n, depth, params, int(i)) for i in indices], dtype=np.complex128)
