"""Dense-matrix constructions used as independent pins (test side only).

Everything here is built from the textbook single-qubit matrices with
Kronecker products (qubit q = bit q, so qubit n-1 is the leftmost factor)
and library routines (scipy.linalg.expm, numpy.linalg.eigh); it shares no
code with the oracle or the CUDA library.
"""
import numpy as np
from scipy.linalg import expm

I2 = np.eye(2, dtype=complex)
X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)


def kron_list(mats):
    out = np.array([[1.0 + 0j]])
    for m in mats:
        out = np.kron(out, m)
    return out


def op_on(n, q, m):
    """Single-qubit matrix m on qubit q of n."""
    return kron_list([m if k == q else I2 for k in reversed(range(n))])


def pauli_matrix(n, x, z):
    mats = []
    for k in reversed(range(n)):
        xb, zb = (x >> k) & 1, (z >> k) & 1
        mats.append({(0, 0): I2, (1, 0): X, (0, 1): Z, (1, 1): Y}[(xb, zb)])
    return kron_list(mats)


def hamiltonian_matrix(n, x, z, c):
    H = np.zeros((1 << n, 1 << n), dtype=complex)
    for xi, zi, ci in zip(x, z, c):
        H += ci * pauli_matrix(n, int(xi), int(zi))
    return H


def ry(theta):
    return expm(-0.5j * theta * Y)


def rz(phi):
    return expm(-0.5j * phi * Z)


def cz(n, a, b):
    d = np.ones(1 << n)
    i = np.arange(1 << n)
    d[((i >> a) & 1) & ((i >> b) & 1) == 1] = -1.0
    return np.diag(d).astype(complex)


def ansatz_unitary(n, depth, params):
    """Product of the ansatz gates in time order (RY then RZ per qubit, then the CZ chain)."""
    U = np.eye(1 << n, dtype=complex)
    for l in range(depth):
        for q in range(n):
            U = op_on(n, q, ry(params[(l * n + q) * 2])) @ U
            U = op_on(n, q, rz(params[(l * n + q) * 2 + 1])) @ U
        for q in range(n - 1):
            U = cz(n, q, q + 1) @ U
    return U


def number_ops(n):
    Nup = np.zeros((1 << n, 1 << n))
    Ndn = np.zeros((1 << n, 1 << n))
    i = np.arange(1 << n)
    for m in range(n):
        occ = ((i >> m) & 1).astype(float)
        if m % 2 == 0:
            Nup += np.diag(occ)
        else:
            Ndn += np.diag(occ)
    return Nup, Ndn


def sector_ground(H, n, n_up, n_dn):
    """Lowest eigenvalue of H in the sector with n_up / n_dn occupied even/odd modes."""
    i = np.arange(1 << n)
    up = sum(((i >> m) & 1) for m in range(0, n, 2))
    dn = sum(((i >> m) & 1) for m in range(1, n, 2))
    sel = np.where((up == n_up) & (dn == n_dn))[0]
    sub = H[np.ix_(sel, sel)]
    return float(np.linalg.eigvalsh(sub)[0])
