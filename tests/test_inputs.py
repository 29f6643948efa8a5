"""Input generators: RNG, Jordan-Wigner mapping, Hubbard and molecular builders."""
import numpy as np
import pytest

import vqe_inputs as vi
from dense import hamiltonian_matrix, number_ops, I2, X, Y, Z, kron_list


def test_splitmix64_published_first_output():
    # SplitMix64 from state 0: the first output is 0xE220A8397B1DCDAF
    assert int(vi.splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF


def test_rng_deterministic_and_uniform():
    a = vi.uniform01(42, 100000)
    b = vi.uniform01(42, 100000)
    assert np.array_equal(a, b)
    assert 0.0 <= a.min() and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 0.01
    g = vi.normal(7, 200000)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1.0) < 0.01
    p = vi.ansatz_params(3, 20, 10)
    assert p.size == 400 and p.min() >= -np.pi and p.max() < np.pi


@pytest.mark.parametrize("L,periodic,terms,groups", [(4, False, 25, 7), (10, True, 71, 21)])
def test_hubbard_1d_sizes(L, periodic, terms, groups):
    H = vi.hubbard_1d(L, 1.0, 4.0, periodic)
    assert len(H) == terms and H.n_groups == groups


def test_hubbard_2d_snake_size():
    H = vi.hubbard_2d_snake(4, 4, 1.0, 4.0, periodic=True)
    assert H.n == 32 and len(H) == 177 and H.n_groups == 65


@pytest.mark.parametrize("L,U", [(2, 4.0), (3, 2.5), (4, 4.0)])
def test_hubbard_trace_identity_coefficient(L, U):
    """Tr(H)/2^n equals the identity coefficient, which is U*L/4 for this Hubbard form."""
    H = vi.hubbard_1d(L, 1.0, U, periodic=False)
    M = hamiltonian_matrix(H.n, H.x, H.z, H.c)
    assert abs(np.trace(M).real / 2 ** H.n - U * L / 4) < 1e-12
    ci = H.c[(H.x == 0) & (H.z == 0)]
    assert abs(ci[0] - U * L / 4) < 1e-14
    assert np.allclose(M, M.conj().T)


def test_jordan_wigner_anticommutation():
    """{a_p, a_q^dagger} = delta_pq and {a_p, a_q} = 0 for the generated ladder operators."""
    n = 4
    def ladder(m, dag):
        x, z, c = vi.fermion_op(np.array([[m]]), (dag,), np.array([1.0]))
        return hamiltonian_matrix(n, x, z, c)
    for p in range(n):
        for q in range(n):
            ap, aqd, aq = ladder(p, False), ladder(q, True), ladder(q, False)
            anti = ap @ aqd + aqd @ ap
            assert np.allclose(anti, np.eye(1 << n) * (p == q))
            assert np.allclose(ap @ aq + aq @ ap, 0)
    # occupied = |1>: a_0^dagger |0000> = |0001>
    v = np.zeros(1 << n); v[0] = 1
    assert np.allclose(ladder(0, True) @ v, np.eye(1 << n)[1])


def test_hubbard_conserves_particle_number_and_spin():
    H = vi.hubbard_1d(3, 1.0, 3.0, periodic=True)
    M = hamiltonian_matrix(H.n, H.x, H.z, H.c)
    Nup, Ndn = number_ops(H.n)
    assert np.allclose(M @ Nup, Nup @ M) and np.allclose(M @ Ndn, Ndn @ M)


def test_synthetic_molecular_structure():
    M = vi.synthetic_molecular(4, seed=9)
    assert M.n == 8
    Md = hamiltonian_matrix(M.n, M.x, M.z, M.c)
    assert np.allclose(Md, Md.conj().T)
    Nup, Ndn = number_ops(M.n)
    assert np.allclose(Md @ (Nup + Ndn), (Nup + Ndn) @ Md)
    # JW image: every term has an even number of X/Y factors
    assert np.all(np.bitwise_count(M.x) % 2 == 0)


def test_synthetic_molecular_24q_shape():
    M = vi.synthetic_molecular(12, seed=2024)
    assert M.n == 24
    assert 20000 < len(M) < 200000
    a = np.abs(M.c)
    assert a.max() > 0.5 and a.min() < 1e-6


def test_batched_instances():
    inst = vi.batched_instances(64, seed=3)
    ns = [d["n"] for d in inst]
    assert min(ns) >= 12 and max(ns) <= 18 and len(set(ns)) >= 5
    for d in inst:
        assert d["depth"] == d["n"] // 2 and 1.0 <= d["U"] <= 8.0
        assert d["params"].size == 2 * d["n"] * d["depth"]
        assert d["H"].n == d["n"] and (d["H"].x < (1 << d["n"])).all()
