"""Pins of the oracle's particle-conserving ansatz (Sec. II-B, Eqs. 5-6):
single and double excitation gates exp(theta (T - T^dag)) on the
Hartree-Fock state, checked against what mathematics fixes independently of
the oracle's code:

  * each gate equals scipy's expm of the generator built from Kronecker
    products of Jordan-Wigner ladder matrices (a dense construction that
    shares nothing with the oracle's bit loops),
  * the circuit is orthogonal and conserves particle number and S_z,
  * hand-derived 2- and 4-qubit closed forms,
  * the converged VQE on the 2-site Hubbard model reaches the exact
    ground energy (U - sqrt(U^2 + 16 t^2)) / 2 of the half-filled sector,
  * the adjoint gradient equals central differences.
"""
import numpy as np
import pytest
from scipy.linalg import expm
from scipy.optimize import minimize

import vqe_inputs as vi

SIGMA_MINUS = np.array([[0.0, 1.0], [0.0, 0.0]])   # |1> -> |0> in the basis (|0>, |1>)
ZMAT = np.diag([1.0, -1.0])


def ladder(n, m):
    """Dense a_m on n qubits (qubit q = bit q of the index): Z on every qubit
    below m, sigma^- on m, identity above.  np.kron's left factor is the most
    significant bit."""
    out = np.array([[1.0]])
    for q in range(n - 1, -1, -1):
        f = SIGMA_MINUS if q == m else (ZMAT if q < m else np.eye(2))
        out = np.kron(out, f)
    return out


def generator(n, exc):
    p, q, r, s = exc
    a = {m: ladder(n, m) for m in {p, q, r, s} if m >= 0}
    if q < 0:
        T = a[p].T @ a[r]
    else:
        T = a[p].T @ a[q].T @ a[r] @ a[s]
    return T - T.T


def gate_matrix_oracle(oracle_mod, n, exc, theta):
    dim = 1 << n
    U = np.zeros((dim, dim), dtype=complex)
    for j in range(dim):
        e = np.zeros(dim, dtype=complex)
        e[j] = 1.0
        U[:, j] = oracle_mod.apply_excitation(e, exc, theta)
    return U


EXCITATIONS_6 = [
    (1, -1, 0, -1), (5, -1, 0, -1), (4, -1, 2, -1), (0, -1, 5, -1),
    (4, 5, 0, 1), (3, 5, 0, 2), (2, 4, 5, 1), (5, 4, 1, 0),
]


@pytest.mark.parametrize("exc", EXCITATIONS_6)
def test_gate_is_expm_of_jordan_wigner_generator(oracle_mod, exc):
    n, theta = 6, 0.731
    U = gate_matrix_oracle(oracle_mod, n, exc, theta)
    ref = expm(theta * generator(n, exc))
    assert np.max(np.abs(U - ref)) <= 1e-13
    # the generator itself, on a random state
    rng = np.random.default_rng(3)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    assert np.max(np.abs(oracle_mod.excitation_generator(psi, exc) - generator(n, exc) @ psi)) <= 1e-13


def test_circuit_orthogonal_and_conserves_number_and_sz(oracle_mod):
    n, ne = 6, 3
    exc = vi.excitations(n, ne)
    theta = vi.excitation_params(5, len(exc))
    dim = 1 << n
    U = np.eye(dim, dtype=complex)
    for e, t in zip(exc, theta):
        U = gate_matrix_oracle(oracle_mod, n, e, t) @ U
    assert np.max(np.abs(U.conj().T @ U - np.eye(dim))) <= 1e-13
    assert np.max(np.abs(U.imag)) == 0.0                       # real rotations only
    idx = np.arange(dim)
    N = np.array([bin(i).count("1") for i in idx])
    SZ = np.array([bin(i & 0x55555555).count("1") - bin(i & 0xAAAAAAAA).count("1") for i in idx])
    mixes = (N[:, None] != N[None, :]) | (SZ[:, None] != SZ[None, :])
    assert np.max(np.abs(U[mixes])) == 0.0
    # the ansatz state is U applied to the Hartree-Fock basis state
    psi = oracle_mod.pc_ansatz_state(n, ne, exc, theta)
    assert np.max(np.abs(psi - U[:, (1 << ne) - 1])) <= 1e-13
    assert abs(np.vdot(psi, psi).real - 1.0) <= 1e-13


def test_closed_forms_two_and_four_qubits(oracle_mod):
    t = 0.3
    # single a_1^dag a_0 on |01> (mode 0 occupied, index 1): no mode in between
    psi = oracle_mod.pc_ansatz_state(2, 1, [[1, -1, 0, -1]], [t])
    assert np.allclose(psi, [0, np.cos(t), np.sin(t), 0], atol=1e-15)
    # double a_2^dag a_3^dag a_0 a_1 on |0011> (index 3): a_1 passes the
    # occupied mode 0 (-1), a_0, a_3^dag and a_2^dag pass none, so the pair
    # (|0011>, |1100>) turns as (cos t, -sin t)
    psi = oracle_mod.pc_ansatz_state(4, 2, [[2, 3, 0, 1]], [t])
    ref = np.zeros(16)
    ref[3], ref[12] = np.cos(t), -np.sin(t)
    assert np.allclose(psi, ref, atol=1e-15)
    # single a_3^dag a_0 on |0111>: the occupied modes 1, 2 lie between: sign +1
    psi = oracle_mod.pc_ansatz_state(4, 3, [[3, -1, 0, -1]], [t])
    assert abs(psi[7] - np.cos(t)) <= 1e-15 and abs(psi[14] - np.sin(t)) <= 1e-15
    # ... and with one occupied mode between (|0101> -> |1100>): sign -1
    e = np.zeros(16, dtype=complex)
    e[5] = 1.0
    out = oracle_mod.apply_excitation(e, [3, -1, 0, -1], t)
    assert abs(out[5] - np.cos(t)) <= 1e-15 and abs(out[12] + np.sin(t)) <= 1e-15


@pytest.mark.parametrize("U", [2.0, 4.0, 8.0])
def test_two_site_hubbard_vqe_reaches_exact_ground_energy(oracle_mod, U):
    t = 1.0
    H = vi.hubbard_1d(2, t, U, periodic=False)
    exc = vi.excitations(4, 2)            # one double, then two singles
    e0 = (U - np.sqrt(U * U + 16.0 * t * t)) / 2.0
    seen = []

    def f(th):
        g, e = oracle_mod.pc_gradient_adjoint(4, 2, exc, th, H.x, H.z, H.c)
        seen.append(e)
        return e, g

    best = min(minimize(f, vi.excitation_params(s, len(exc)), jac=True, method="BFGS",
                        options={"gtol": 1e-12}).fun for s in range(4))
    assert abs(best - e0) <= 1e-9
    assert min(seen) >= e0 - 1e-12                # variational


def test_adjoint_gradient_matches_central_differences(oracle_mod):
    n, ne = 8, 4
    H = vi.hubbard_1d(4, 1.0, 4.0, periodic=False)
    exc = vi.excitations(n, ne)
    th = vi.excitation_params(11, len(exc))
    g, e = oracle_mod.pc_gradient_adjoint(n, ne, exc, th, H.x, H.z, H.c)
    fd = oracle_mod.pc_gradient_fd(n, ne, exc, th, H.x, H.z, H.c, 1e-5)
    assert np.max(np.abs(g - fd)) <= 1e-8 * max(1.0, np.max(np.abs(g)))
    psi = oracle_mod.pc_ansatz_state(n, ne, exc, th)
    e_ref, _ = oracle_mod.energy(psi, H.x, H.z, H.c)
    assert abs(e - e_ref) <= 1e-12 * H.sum_abs()
    # all amplitude stays in the 4-electron sector
    N = np.array([bin(i).count("1") for i in range(1 << n)])
    assert np.sum(np.abs(psi[N != ne]) ** 2) == 0.0


def test_excitation_list_structure():
    exc = vi.excitations(8, 4)
    doubles = exc[exc[:, 1] >= 0]
    singles = exc[exc[:, 1] < 0]
    assert len(singles) == 8 and len(doubles) == 18
    assert np.all(exc[: len(doubles), 1] >= 0)    # doubles first
    for p, q, r, s in doubles:
        assert r < 4 and s < 4 and p >= 4 and q >= 4
        assert (p & 1) + (q & 1) == (r & 1) + (s & 1)
    for p, _, r, _ in singles:
        assert r < 4 <= p and (p & 1) == (r & 1)
    sub = vi.excitations(32, 16, 16, 102, seed=1)
    assert len(sub) == 118 and np.sum(sub[:, 1] < 0) == 16
