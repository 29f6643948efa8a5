"""Seeded synthetic inputs for the VQE hot path.

This module builds inputs only: ansatz parameter vectors and qubit
Hamiltonians given as Pauli sums ``(x_mask, z_mask, coeff)``.  It holds none
of the method's own arithmetic (no circuit, no expectation value, no term
cutoff, no gradient), so both the CPU oracle side and the CUDA side can use it.

Conventions
-----------
* Qubit ``q`` is bit ``q`` of a basis-state index (little endian).
* A Pauli string is the pair of bit masks ``(x, z)``: per qubit ``(0,0)=I``,
  ``(1,0)=X``, ``(0,1)=Z``, ``(1,1)=Y``.  The coefficient ``c`` multiplies the
  tensor product of those single-qubit matrices (Sec. II-B, Eqs. 2-4).
* Fermionic mode ``m`` maps to qubit ``m`` by the Jordan-Wigner transform
  (Sec. II-B), with the occupied state of a mode being ``|1>``.
* Random numbers come from SplitMix64 (Steele, Lea, Flood 2014), a counter
  based generator: value ``k`` of stream ``seed`` is ``mix(seed + (k+1)*G)``
  with ``G = 0x9E3779B97F4A7C15``.  Uniforms use the top 53 bits; normals use
  Box-Muller.  No library generator is used, so values are identical on every
  machine.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "PauliSum", "splitmix64", "uniform01", "normal", "ansatz_params",
    "hubbard_1d", "hubbard_2d_snake", "synthetic_molecular", "batched_instances",
    "fermion_op", "merge_terms", "random_pauli_sum",
]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` 64-bit outputs of SplitMix64 stream ``seed`` starting at ``offset``."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        return _mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN)


def _substream(seed: int, stream: int) -> int:
    with np.errstate(over="ignore"):
        return int(_mix64(np.array([seed ^ (stream * 0xD1B54A32D192ED03 & 0xFFFFFFFFFFFFFFFF)],
                                   dtype=np.uint64))[0])


def uniform01(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each output."""
    u = splitmix64(_substream(seed, stream), count)
    return (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller on consecutive uniform pairs."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m, stream)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))          # 1-u1 lies in (0, 1]
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(2.0 * math.pi * u2)
    out[1::2] = r * np.sin(2.0 * math.pi * u2)
    return out[:count]


def ansatz_params(seed: int, n_qubits: int, depth: int, stream: int = 1) -> np.ndarray:
    """i.i.d. U[-pi, pi) angles for the hardware-efficient ansatz.

    Layout: ``params[(l*n + q)*2 + 0]`` is the RY angle and ``+1`` the RZ
    angle of qubit ``q`` in layer ``l``.
    """
    u = uniform01(seed, 2 * n_qubits * depth, stream)
    return -math.pi + 2.0 * math.pi * u


# --------------------------------------------------------------------------
# Pauli sums
# --------------------------------------------------------------------------

@dataclasses.dataclass
class PauliSum:
    """``H = sum_i c[i] * P(x[i], z[i])`` on ``n`` qubits (Sec. II-B, Eq. 2)."""
    n: int
    x: np.ndarray   # uint64
    z: np.ndarray   # uint64
    c: np.ndarray   # float64

    def __len__(self) -> int:
        return len(self.c)

    @property
    def n_groups(self) -> int:
        return len(np.unique(self.x))

    def sum_abs(self) -> float:
        return float(np.abs(self.c).sum())


def merge_terms(x, z, c, drop_abs: float = 0.0):
    """Sum coefficients of identical ``(x, z)`` keys; drop ``|c| <= drop_abs``.

    Returns arrays sorted by the key ``(x, z)``.
    """
    x = np.asarray(x, dtype=np.uint64)
    z = np.asarray(z, dtype=np.uint64)
    c = np.asarray(c)
    if len(c) == 0:
        return x, z, c
    keys = np.stack([x, z], axis=1)
    uniq, inv = np.unique(keys, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    if np.iscomplexobj(c):
        cs = (np.bincount(inv, weights=c.real, minlength=len(uniq))
              + 1j * np.bincount(inv, weights=c.imag, minlength=len(uniq)))
    else:
        cs = np.bincount(inv, weights=c, minlength=len(uniq))
    keep = np.abs(cs) > drop_abs
    return uniq[keep, 0].copy(), uniq[keep, 1].copy(), cs[keep]


def _popcount(a: np.ndarray) -> np.ndarray:
    return np.bitwise_count(a).astype(np.int64)


def _ladder_terms(mode: np.ndarray, dagger: bool):
    """Jordan-Wigner image of a_m (or a_m^dagger) in ``Z^z X^x`` form.

    ``a_m = Z_{<m} (X_m + i Y_m) / 2`` with ``Y = -i Z X`` gives
    ``a_m = Z_{<m} (X_m + Z_m X_m) / 2``; the adjoint has ``-`` in front of
    the ``Z_m X_m`` term.  Returns ``(coef[2], x[2, K], z[2, K])``.
    """
    mode = np.asarray(mode, dtype=np.uint64)
    e = np.left_shift(np.uint64(1), mode)
    below = e - np.uint64(1)
    xs = np.stack([e, e])
    zs = np.stack([below, below | e])
    coef = np.array([0.5, -0.5 if dagger else 0.5])
    return coef, xs, zs


def fermion_op(modes: np.ndarray, daggers, coefs: np.ndarray):
    """Products of ladder operators, one product per row of ``modes``.

    ``modes`` is a ``(K, r)`` integer array, ``daggers`` a length-``r``
    sequence of bools, ``coefs`` a length-``K`` array.  Row ``k`` stands for
    ``coefs[k] * prod_j a_{modes[k, j]}^{(dagger_j)}`` (left to right).
    Returns unmerged Pauli-string terms ``(x, z, complex c)``.

    Multiplication in ``Z^z X^x`` form uses
    ``(Z^z1 X^x1)(Z^z2 X^x2) = (-1)^{popc(x1 & z2)} Z^{z1^z2} X^{x1^x2}``;
    at the end ``Z^z X^x = i^{popc(x&z)} P(x, z)`` converts to Pauli strings.
    """
    modes = np.atleast_2d(np.asarray(modes, dtype=np.int64))
    K, r = modes.shape
    coefs = np.asarray(coefs, dtype=np.complex128).reshape(K)
    acc_c = coefs[None, :].copy()
    acc_x = np.zeros((1, K), dtype=np.uint64)
    acc_z = np.zeros((1, K), dtype=np.uint64)
    for j in range(r):
        lc, lx, lz = _ladder_terms(modes[:, j], daggers[j])
        new_c, new_x, new_z = [], [], []
        for s in range(2):
            sign = 1.0 - 2.0 * (_popcount(acc_x & lz[s][None, :]) & 1)
            new_c.append(acc_c * lc[s] * sign)
            new_x.append(acc_x ^ lx[s][None, :])
            new_z.append(acc_z ^ lz[s][None, :])
        acc_c = np.concatenate(new_c)
        acc_x = np.concatenate(new_x)
        acc_z = np.concatenate(new_z)
    kappa = _popcount(acc_x & acc_z) & 3
    acc_c = acc_c * (1j ** kappa)
    return acc_x.reshape(-1), acc_z.reshape(-1), acc_c.reshape(-1)


def _finish(n: int, parts, drop_abs: float = 1e-12, imag_tol: float = 1e-10) -> PauliSum:
    xs = np.concatenate([p[0] for p in parts])
    zs = np.concatenate([p[1] for p in parts])
    cs = np.concatenate([p[2] for p in parts])
    x, z, c = merge_terms(xs, zs, cs, drop_abs=drop_abs)
    if len(c) and np.max(np.abs(c.imag)) > imag_tol * max(1.0, np.max(np.abs(c.real))):
        raise ValueError("Hamiltonian is not Hermitian: imaginary Pauli coefficient")
    return PauliSum(n=n, x=x, z=z, c=np.ascontiguousarray(c.real))


def _hubbard(n_sites: int, bonds, t: float, U: float) -> PauliSum:
    """``H = -t sum_{<ij>,s} (a+_{is} a_{js} + h.c.) + U sum_i n_{i up} n_{i dn}``.

    Modes are interleaved: mode ``2*site + spin`` (spin 0 = up, 1 = down).
    Each bond is counted once; there is no chemical potential.
    """
    parts = []
    hop_modes, hop_c = [], []
    for (i, j) in bonds:
        for s in range(2):
            p, q = 2 * i + s, 2 * j + s
            hop_modes += [(p, q), (q, p)]
            hop_c += [-t, -t]
    if hop_modes:
        parts.append(fermion_op(np.array(hop_modes), (True, False), np.array(hop_c)))
    if U != 0.0:
        dens = [(2 * i, 2 * i, 2 * i + 1, 2 * i + 1) for i in range(n_sites)]
        # n_up n_dn = a+_up a_up a+_dn a_dn
        parts.append(fermion_op(np.array(dens), (True, False, True, False),
                                np.full(n_sites, U)))
    if not parts:
        return PauliSum(2 * n_sites, np.zeros(0, np.uint64), np.zeros(0, np.uint64), np.zeros(0))
    return _finish(2 * n_sites, parts)


def _dedupe_bonds(bonds):
    seen, out = set(), []
    for (i, j) in bonds:
        if i == j:
            continue
        key = (min(i, j), max(i, j))
        if key not in seen:
            seen.add(key)
            out.append(key)
    return out


def hubbard_1d(L: int, t: float = 1.0, U: float = 4.0, periodic: bool = False) -> PauliSum:
    """1D Fermi-Hubbard chain of ``L`` sites on ``2L`` qubits."""
    bonds = [(i, i + 1) for i in range(L - 1)]
    if periodic and L > 2:
        bonds.append((L - 1, 0))
    return _hubbard(L, _dedupe_bonds(bonds), t, U)


def snake_site(Lx: int, r: int, col: int) -> int:
    """Site index of row ``r``, column ``col`` in snake order."""
    return r * Lx + (col if r % 2 == 0 else Lx - 1 - col)


def hubbard_2d_snake(Lx: int, Ly: int, t: float = 1.0, U: float = 4.0,
                     periodic: bool = True) -> PauliSum:
    """2D Fermi-Hubbard model on an ``Lx x Ly`` lattice, sites in snake order.

    Row ``r`` is traversed left to right when ``r`` is even, right to left
    otherwise; periodic boundaries in both directions when ``periodic``.
    """
    bonds = []
    for r in range(Ly):
        for col in range(Lx):
            s = snake_site(Lx, r, col)
            if col + 1 < Lx or (periodic and Lx > 2):
                bonds.append((s, snake_site(Lx, r, (col + 1) % Lx)))
            if r + 1 < Ly or (periodic and Ly > 2):
                bonds.append((s, snake_site(Lx, (r + 1) % Ly, col)))
    return _hubbard(Lx * Ly, _dedupe_bonds(bonds), t, U)


def synthetic_integrals(n_spatial: int, seed: int):
    """Random real one- and two-body integrals with molecular-like structure.

    ``h_pq ~ N(0,1) exp(-|p-q|/2)`` symmetric; ``g_pqrs ~ N(0, 0.1^2)
    exp(-(|p-q|+|r-s|)/2)`` with the 8-fold real symmetry of chemist-notation
    integrals ``(pq|rs)``.
    """
    m = n_spatial
    idx = np.arange(m)
    dist = np.abs(idx[:, None] - idx[None, :])
    pair = np.maximum(idx[:, None], idx[None, :]) * (np.maximum(idx[:, None], idx[None, :]) + 1) // 2 \
        + np.minimum(idx[:, None], idx[None, :])
    n_pair = m * (m + 1) // 2
    h_draw = normal(seed, n_pair, stream=11)
    h = h_draw[pair] * np.exp(-dist / 2.0)
    n_quad = n_pair * (n_pair + 1) // 2
    g_draw = 0.1 * normal(seed, n_quad, stream=12)
    P = pair[:, :, None, None]
    R = pair[None, None, :, :]
    hi, lo = np.maximum(P, R), np.minimum(P, R)
    quad = hi * (hi + 1) // 2 + lo
    env = np.exp(-(dist[:, :, None, None] + dist[None, None, :, :]) / 2.0)
    g = g_draw[quad] * env
    return h, g


def synthetic_molecular(n_spatial: int = 12, seed: int = 2024) -> PauliSum:
    """Jordan-Wigner image of a random molecular-style Hamiltonian (cf. Eq. 1).

    ``H = sum_{pq,s} h_pq a+_{ps} a_{qs}
        + 1/2 sum_{pqrs,s,t} g_pqrs a+_{ps} a+_{rt} a_{st} a_{qs}``
    on ``2*n_spatial`` qubits, modes interleaved (``2p + s``), no constant.
    """
    h, g = synthetic_integrals(n_spatial, seed)
    m = n_spatial
    parts = []
    p, q, s = np.meshgrid(np.arange(m), np.arange(m), np.arange(2), indexing="ij")
    p, q, s = p.ravel(), q.ravel(), s.ravel()
    parts.append(fermion_op(np.stack([2 * p + s, 2 * q + s], axis=1), (True, False), h[p, q]))
    P, Q, R, S, sg, tg = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), np.arange(m),
                                     np.arange(2), np.arange(2), indexing="ij")
    P, Q, R, S, sg, tg = (a.ravel() for a in (P, Q, R, S, sg, tg))
    modes = np.stack([2 * P + sg, 2 * R + tg, 2 * S + tg, 2 * Q + sg], axis=1)
    coef = 0.5 * g[P, Q, R, S]
    nz = coef != 0.0
    parts.append(fermion_op(modes[nz], (True, True, False, False), coef[nz]))
    return _finish(2 * m, parts)


def batched_instances(count: int = 512, seed: int = 7, n_min: int = 12, n_max: int = 18):
    """Uneven batch: ``n`` uniform on ``{n_min..n_max}``, open Hubbard with
    ``floor(n/2)`` sites, ``t = 1``, ``U ~ U[1, 8]``, depth ``floor(n/2)``, and
    per-instance ansatz parameters.  An odd ``n`` leaves the top qubit out of
    the Hamiltonian (it still carries ansatz gates).
    """
    u = uniform01(seed, 2 * count, stream=21)
    out = []
    for k in range(count):
        n = n_min + min(int(u[2 * k] * (n_max - n_min + 1)), n_max - n_min)
        U = 1.0 + 7.0 * u[2 * k + 1]
        L = n // 2
        H = hubbard_1d(L, 1.0, U, periodic=False)
        H = PauliSum(n=n, x=H.x, z=H.z, c=H.c)
        depth = n // 2
        params = ansatz_params(seed * 1000003 + k, n, depth)
        out.append({"n": n, "depth": depth, "U": U, "H": H, "params": params})
    return out


def random_pauli_sum(n: int, n_terms: int, seed: int, with_identity: bool = True,
                     duplicates: int = 0) -> PauliSum:
    """Random real-coefficient Pauli sum: uniform masks (any mix of I/X/Y/Z),
    coefficients N(0,1); optionally an identity term and ``duplicates``
    repeated strings (to exercise merging).  Not merged."""
    u = splitmix64(_substream(seed, 31), 2 * n_terms)
    lim = np.uint64((1 << n) - 1)
    x = u[0::2] & lim
    z = u[1::2] & lim
    c = normal(seed, n_terms, stream=32)
    if with_identity:
        x = np.concatenate([x, np.zeros(1, np.uint64)])
        z = np.concatenate([z, np.zeros(1, np.uint64)])
        c = np.concatenate([c, [0.75]])
    if duplicates:
        k = min(duplicates, len(c))
        x = np.concatenate([x, x[:k]])
        z = np.concatenate([z, z[:k]])
        c = np.concatenate([c, 0.5 * c[:k]])
    return PauliSum(n=n, x=x, z=z, c=c)


def excitations(n_qubits: int, n_elec: int, n_singles: int | None = None,
                n_doubles: int | None = None, seed: int = 0) -> np.ndarray:
    """Excitation list of the particle-conserving ansatz (Sec. II-B, Eq. 5):
    rows ``(p, q, r, s)``, singles ``(p, -1, r, -1)`` = a_p^dag a_r and doubles
    ``(p, q, r, s)`` = a_p^dag a_q^dag a_r a_s, from the occupied modes of the
    Hartree-Fock state (modes ``0 .. n_elec-1``) to the virtual ones, spin
    conserving (mode ``2*site + spin``).  The paper picks its excitations from
    CISD coefficients it does not print; here ``n_singles`` / ``n_doubles``
    (``None`` = all) are drawn without replacement by a seeded shuffle.
    Rows are in the order of application: Eq. 5's product read in time order
    (as the ansatz layer of Eq. 6 is), so the D gates act first and the S
    gates last, the singles acting as an orbital rotation of the correlated
    state."""
    occ = [m for m in range(n_elec)]
    vir = [m for m in range(n_elec, n_qubits)]
    singles = [(p, -1, r, -1) for r in occ for p in vir if (p & 1) == (r & 1)]
    doubles = []
    for i, r in enumerate(occ):
        for s in occ[i + 1:]:
            for j, p in enumerate(vir):
                for q in vir[j + 1:]:
                    if (p & 1) + (q & 1) == (r & 1) + (s & 1):
                        doubles.append((p, q, r, s))

    def pick(items, k, stream):
        if k is None or k >= len(items):
            return items
        keys = uniform01(seed, len(items), stream=stream)
        order = np.sort(np.argsort(keys, kind="stable")[:k])
        return [items[i] for i in order]

    rows = pick(doubles, n_doubles, 42) + pick(singles, n_singles, 41)
    return np.array(rows, dtype=np.int32).reshape(-1, 4)


def excitation_params(seed: int, n_exc: int, scale: float = 0.5, stream: int = 43) -> np.ndarray:
    """Excitation angles, i.i.d. U[-scale*pi, scale*pi)."""
    return (2.0 * uniform01(seed, n_exc, stream=stream) - 1.0) * scale * np.pi
