"""Pins of the FP64 oracle to facts outside itself (closed forms, textbook
matrices built independently, library eigensolvers, brute force).

Which plausible oracle mistake each pin catches:
  rotation sign / half-angle (RY, RZ)     -> test_gate_matrices_match_exponentials, P3
  gate order inside a layer, CZ chain     -> test_ansatz_matches_dense_unitary
  qubit <-> bit order, parameter layout    -> test_ansatz_matches_dense_unitary, P2
  Pauli phase of Y, X/Z placement         -> test_pauli_terms_match_kron, test_y_eigenstate
  dropped or doubled term in <H>          -> test_pauli_terms_match_kron, P1, P6, P7
  normalisation of Eq. 7                  -> test_energy_is_normalised
  cutoff comparison / bound               -> test_slim_*, P9
  adjoint gradient                        -> P10 (parameter shift is exact)
"""
import math
import os

import numpy as np
import pytest

import vqe_inputs as vi
import dense as dn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


def test_gate_matrices_match_exponentials(oracle_mod):
    for t in np.linspace(-7, 7, 29):
        assert np.allclose(oracle_mod.ry_matrix(t), dn.ry(t), atol=1e-15)
        assert np.allclose(oracle_mod.rz_matrix(t), dn.rz(t), atol=1e-15)


def test_brute_force_one_qubit(oracle_mod):
    """P11: RY(t)|0> = (cos t/2, sin t/2); RZ(p) on |+> gives <X> = cos p, <Y> = sin p."""
    for t in (0.3, 1.7, -2.9):
        psi = oracle_mod.ansatz_state(1, 1, [t, 0.0])
        assert np.allclose(psi, [math.cos(t / 2), math.sin(t / 2)], atol=1e-15)
        psi = oracle_mod.ansatz_state(1, 1, [math.pi / 2, t])
        ex, _, _ = oracle_mod.expectation(psi, [1], [0], [1.0])
        ey, _, _ = oracle_mod.expectation(psi, [1], [1], [1.0])
        assert abs(ex - math.cos(t)) < 1e-14 and abs(ey - math.sin(t)) < 1e-14


def test_y_eigenstate(oracle_mod):
    psi = np.array([1, 1j]) / math.sqrt(2)
    e, im, nn = oracle_mod.expectation(psi, [1], [1], [1.0])
    assert abs(e - 1.0) < 1e-15 and abs(im) < 1e-15
    e, _, _ = oracle_mod.expectation(np.array([1, -1j]) / math.sqrt(2), [1], [1], [1.0])
    assert abs(e + 1.0) < 1e-15


@pytest.mark.parametrize("n,depth", [(1, 2), (2, 2), (3, 3), (5, 2), (6, 2)])
def test_ansatz_matches_dense_unitary(oracle_mod, n, depth):
    """P5: circuit unitary from Kronecker products; U^dag U = I."""
    p = vi.ansatz_params(11 * n + depth, n, depth)
    U = dn.ansatz_unitary(n, depth, p)
    assert np.allclose(U.conj().T @ U, np.eye(1 << n), atol=1e-12)
    psi = oracle_mod.ansatz_state(n, depth, p)
    assert np.max(np.abs(psi - U[:, 0])) < 1e-13


@pytest.mark.parametrize("n", [1, 2, 4, 6])
def test_pauli_terms_match_kron(oracle_mod, n):
    """P5: every Pauli string <psi|P|psi> and P psi against kron-built matrices."""
    rng = np.random.default_rng(n)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    for x in range(1 << n):
        for z in range(1 << n):
            M = dn.pauli_matrix(n, x, z)
            assert np.allclose(oracle_mod.pauli_apply(psi, x, z), M @ psi, atol=1e-13)
            if (x * 7 + z) % 5 == 0:
                e, im, nn = oracle_mod.expectation(psi, [x], [z], [1.0])
                ref = np.vdot(psi, M @ psi)
                assert abs(e - ref.real) < 1e-12 and abs(im - ref.imag) < 1e-12


@pytest.mark.parametrize("n,T", [(4, 30), (8, 60)])
def test_energy_and_apply_h_match_dense(oracle_mod, n, T):
    H = vi.random_pauli_sum(n, T, seed=n, duplicates=5)
    Hd = dn.hamiltonian_matrix(n, H.x, H.z, H.c)
    assert np.allclose(Hd, Hd.conj().T)
    p = vi.ansatz_params(n, n, 3)
    psi = oracle_mod.ansatz_state(n, 3, p)
    e, im, nn = oracle_mod.expectation(psi, H.x, H.z, H.c)
    assert abs(e - np.vdot(psi, Hd @ psi).real) < 1e-12
    assert abs(im) < 1e-12 * H.sum_abs()
    assert np.allclose(oracle_mod.apply_h(psi, H.x, H.z, H.c), Hd @ psi, atol=1e-12)


def test_energy_is_normalised(oracle_mod):
    """Eq. 7 divides by <psi|psi>: scaling psi leaves E unchanged."""
    H = vi.hubbard_1d(3, 1.0, 4.0)
    psi = oracle_mod.ansatz_state(6, 2, vi.ansatz_params(1, 6, 2))
    e1, n1 = oracle_mod.energy(psi, H.x, H.z, H.c)
    e2, n2 = oracle_mod.energy(3.0 * psi, H.x, H.z, H.c)
    assert abs(e1 - e2) < 1e-13 and abs(n2 - 9.0 * n1) < 1e-12


@pytest.mark.parametrize("n", [8, 12, 16])
def test_unitarity(oracle_mod, n):
    """P8: |<psi|psi> - 1| <= 1e-13 after a random circuit."""
    psi = oracle_mod.ansatz_state(n, 4, vi.ansatz_params(n, n, 4))
    assert abs(np.vdot(psi, psi).real - 1.0) <= 1e-13


def test_theta_zero_gives_z_only_sum(oracle_mod):
    """P1: params = 0 leaves |0..0>; E = sum of coefficients of terms with x = 0."""
    H = vi.random_pauli_sum(7, 50, seed=4)
    psi = oracle_mod.ansatz_state(7, 2, np.zeros(28))
    e, _ = oracle_mod.energy(psi, H.x, H.z, H.c)
    assert abs(e - H.c[H.x == 0].sum()) < 1e-13
    Hh = vi.hubbard_1d(4, 1.0, 4.0)
    e, _ = oracle_mod.energy(oracle_mod.ansatz_state(8, 1, np.zeros(16)), Hh.x, Hh.z, Hh.c)
    assert abs(e) < 1e-14   # Hubbard vacuum energy is 0


def test_basis_state_preparation(oracle_mod):
    """P2: RY(pi) on a set of qubits gives a Fock state; Hubbard E = U * (#doubly occupied)."""
    L, U = 4, 3.0
    H = vi.hubbard_1d(L, 1.0, U)
    n = 2 * L
    for occ in ([0, 1], [0, 1, 4, 5], [0, 3], list(range(n)), [2, 3, 6]):
        p = np.zeros(2 * n)
        for q in occ:
            p[2 * q] = math.pi
        psi = oracle_mod.ansatz_state(n, 1, p)
        m = sum(1 << q for q in occ)
        assert abs(abs(psi[m]) - 1.0) < 1e-14
        e, _ = oracle_mod.energy(psi, H.x, H.z, H.c)
        doubly = sum(1 for s in range(L) if 2 * s in occ and 2 * s + 1 in occ)
        assert abs(e - U * doubly) < 1e-13


def test_product_state_closed_form(oracle_mod):
    """P3: depth 1, H = sum c_q Z_q + c Z_a Z_b: E = sum c_q cos t_q + c cos t_a cos t_b."""
    n = 6
    p = vi.ansatz_params(77, n, 1)
    cq = np.linspace(0.3, 1.3, n)
    x = np.zeros(n + 1, np.uint64)
    z = np.array([1 << q for q in range(n)] + [(1 << 1) | (1 << 4)], np.uint64)
    c = np.concatenate([cq, [0.8]])
    psi = oracle_mod.ansatz_state(n, 1, p)
    e, _ = oracle_mod.energy(psi, x, z, c)
    th = p[0::2]
    ref = float(np.sum(cq * np.cos(th)) + 0.8 * math.cos(th[1]) * math.cos(th[4]))
    assert abs(e - ref) < 1e-13


def test_two_site_hubbard_closed_form():
    """P6: 2-site Hubbard, N=2, S_z=0: E0 = (U - sqrt(U^2 + 16 t^2)) / 2 (golden file)."""
    g = read_golden("closed_forms.txt")
    for U in (1.0, 4.0, 8.0):
        H = vi.hubbard_1d(2, 1.0, U, periodic=False)
        M = dn.hamiltonian_matrix(4, H.x, H.z, H.c)
        e0 = dn.sector_ground(M, 4, 1, 1)
        assert abs(e0 - (U - math.sqrt(U * U + 16)) / 2) < 1e-12
    H = vi.hubbard_1d(2, 1.0, 4.0)
    e0 = dn.sector_ground(dn.hamiltonian_matrix(4, H.x, H.z, H.c), 4, 1, 1)
    assert abs(e0 - g["hubbard_2site_U4_t1_E0"]) < 1e-12


def test_free_fermions_closed_form():
    """P7: U = 0, 4-site open chain at half filling: E0 = 2 * (eps_1 + eps_2),
    eps_k = -2t cos(k pi / (L+1))."""
    g = read_golden("closed_forms.txt")
    H = vi.hubbard_1d(4, 1.0, 0.0)
    M = dn.hamiltonian_matrix(8, H.x, H.z, H.c)
    e0 = dn.sector_ground(M, 8, 2, 2)
    eps = [-2 * math.cos(k * math.pi / 5) for k in (1, 2)]
    assert abs(e0 - 2 * sum(eps)) < 1e-12
    assert abs(e0 - g["free_fermion_4site_open_halffilling_E0"]) < 1e-12


def test_slim_counts_and_bound(oracle_mod):
    """P9 and the cutoff rule: drop |c| < th (strict), merged terms, bound holds for any state."""
    H = vi.random_pauli_sum(8, 120, seed=8, duplicates=30)
    H.c = H.c * np.exp(-np.linspace(0, 9, len(H.c)))
    xs0, zs0, cs0, d0 = oracle_mod.slim(H.x, H.z, H.c, 0.0)
    x, z, c = vi.merge_terms(H.x, H.z, H.c)
    assert len(cs0) == np.count_nonzero(c) and d0 == 0.0
    psi = oracle_mod.ansatz_state(8, 3, vi.ansatz_params(8, 8, 3))
    e_full, _ = oracle_mod.energy(psi, xs0, zs0, cs0)
    for th in (1e-4, 1e-3, 1e-2, 0.1, 1.0):
        xs, zs, cs, d = oracle_mod.slim(H.x, H.z, H.c, th)
        assert np.all(np.abs(cs) >= th)
        assert len(cs) == np.count_nonzero(np.abs(c) >= th)
        assert abs(d - np.abs(c[np.abs(c) < th]).sum()) < 1e-12
        e, _ = oracle_mod.energy(psi, xs, zs, cs)
        assert abs(e_full - e) <= d + 1e-13
    # a coefficient exactly at the threshold is kept
    xs, zs, cs, d = oracle_mod.slim([1, 2], [0, 0], [0.5, 0.25], 0.5)
    assert len(cs) == 1 and cs[0] == 0.5 and d == 0.25


@pytest.mark.parametrize("n,depth", [(3, 2), (6, 2)])
def test_gradient_adjoint_vs_shift_and_fd(oracle_mod, n, depth):
    """P10: adjoint == parameter shift (exact for exp(-i t P/2) gates) and central FD."""
    H = vi.random_pauli_sum(n, 20, seed=n)
    p = vi.ansatz_params(5, n, depth)
    g, e = oracle_mod.gradient_adjoint(n, depth, p, H.x, H.z, H.c)
    gs = oracle_mod.gradient_shift(n, depth, p, H.x, H.z, H.c)
    gf = oracle_mod.gradient_fd(n, depth, p, H.x, H.z, H.c, 1e-5)
    assert np.max(np.abs(g - gs)) < 1e-10
    assert np.max(np.abs(g - gf)) < 1e-7
    psi = oracle_mod.ansatz_state(n, depth, p)
    e2, _, _ = oracle_mod.expectation(psi, H.x, H.z, H.c)
    assert abs(e - e2) < 1e-12


def test_gradient_against_dense_derivative(oracle_mod):
    """Gradient of <0|U^dag H U|0> by differentiating the dense unitary numerically (library expm)."""
    n, depth = 3, 2
    H = vi.hubbard_1d(1, 1.0, 2.0)
    H = vi.random_pauli_sum(n, 12, seed=2)
    Hd = dn.hamiltonian_matrix(n, H.x, H.z, H.c)
    p = vi.ansatz_params(9, n, depth)
    g, _ = oracle_mod.gradient_adjoint(n, depth, p, H.x, H.z, H.c)
    h = 1e-6
    for j in range(len(p)):
        pp, pm = p.copy(), p.copy()
        pp[j] += h
        pm[j] -= h
        up, um = dn.ansatz_unitary(n, depth, pp)[:, 0], dn.ansatz_unitary(n, depth, pm)[:, 0]
        fd = (np.vdot(up, Hd @ up).real - np.vdot(um, Hd @ um).real) / (2 * h)
        assert abs(fd - g[j]) < 1e-7


# ---------------------------------------------------------------- path-sum amplitudes

from oracle import pathsum as _pathsum
from dense import ansatz_unitary as _ansatz_unitary


@pytest.mark.parametrize("n,D", [(1, 1), (2, 2), (3, 1), (4, 3), (6, 2)])
def test_pathsum_matches_dense_unitary(n, D):
    """Single amplitudes by the path sum equal column 0 of the Kronecker-built
    circuit unitary (an independent construction of Eq. 6's ansatz)."""
    p = vi.ansatz_params(100 + 7 * n + D, n, D)
    col = _ansatz_unitary(n, D, p)[:, 0]
    a = _pathsum.amplitudes(n, D, p, range(1 << n))
    assert np.max(np.abs(a - col)) <= 1e-13


@pytest.mark.parametrize("n,D", [(9, 4), (10, 6), (12, 3)])
def test_pathsum_matches_full_state_oracle(oracle_mod, n, D):
    p = vi.ansatz_params(200 + n + D, n, D)
    psi = oracle_mod.ansatz_state(n, D, p)
    idx = np.random.default_rng(n).integers(0, 1 << n, 48)
    assert np.max(np.abs(_pathsum.amplitudes(n, D, p, idx) - psi[idx])) <= 1e-13


def test_pathsum_closed_forms():
    """theta = 0: |0..0>.  Depth 1 product state with the CZ chain:
    <i|U|0> = prod_q (cos or sin)(theta_q/2) e^{-+i phi_q/2} * (-1)^{popc(i & i>>1)}."""
    n, D = 7, 2
    z = np.zeros(2 * n * D)
    assert abs(_pathsum.amplitude(n, D, z, 0) - 1.0) <= 1e-15
    assert abs(_pathsum.amplitude(n, D, z, 5)) <= 1e-15
    n = 6
    p = vi.ansatz_params(17, n, 1)
    for i in (0, 1, 6, 45, 63):
        want = 1.0 + 0j
        for q in range(n):
            th, ph = p[2 * q], p[2 * q + 1]
            if (i >> q) & 1:
                want *= np.sin(th / 2) * np.exp(0.5j * ph)
            else:
                want *= np.cos(th / 2) * np.exp(-0.5j * ph)
        if bin(i & (i >> 1)).count("1") % 2:
            want = -want
        assert abs(_pathsum.amplitude(n, 1, p, i) - want) <= 1e-15
