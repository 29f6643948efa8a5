"""VQE loops on the GPU through the C ABI (adjoint gradient), pinned to the
exact ground-state energy from dense diagonalisation (tests/dense.py)."""
import numpy as np
import pytest

import vqe_inputs as vi

import dense as dn

pytestmark = pytest.mark.gpu


def _ground(H):
    return float(np.linalg.eigvalsh(dn.hamiltonian_matrix(H.n, H.x, H.z, H.c))[0])


def _engine(H, D, prec):
    import paper_2402_11878_gb300 as pkg
    eng = pkg.Engine(H.n, D, prec)
    eng.set_hamiltonian(H.x, H.z, H.c)
    return eng


def test_lbfgs_two_site_hubbard_c128(lib_built):
    from paper_2402_11878_gb300 import minimize_energy
    H = vi.hubbard_1d(2, 1.0, 4.0, periodic=False)
    e0 = _ground(H)
    eng = _engine(H, 4, "c128")
    r = minimize_energy(eng, vi.ansatz_params(103, H.n, 4))
    eng.close()
    assert abs(r["energy"] - e0) < 1e-9
    assert r["history"].min() >= e0 - 1e-10       # variational principle


def test_adam_multistart_two_site_hubbard_c64(lib_built):
    """Eight starts advanced together, one batched complex64 gradient per step."""
    from paper_2402_11878_gb300 import minimize_batch
    H = vi.hubbard_1d(2, 1.0, 4.0, periodic=False)
    e0 = _ground(H)
    eng = _engine(H, 4, "c64")
    P0 = np.stack([vi.ansatz_params(200 + s, H.n, 4) for s in range(8)])
    r = minimize_batch(eng, P0, steps=300, lr=0.05)
    eng.close()
    assert r["energies"][r["best"]] - e0 < 1e-4
    assert r["history"].min() >= e0 - 1e-5 * H.sum_abs()


def test_lbfgs_four_site_hubbard_variational_bound(lib_built):
    """8 qubits, depth 6: the loop lowers the energy and never goes below the
    exact ground state."""
    from paper_2402_11878_gb300 import minimize_energy
    H = vi.hubbard_1d(4, 1.0, 4.0, periodic=False)
    e0 = _ground(H)
    eng = _engine(H, 6, "c128")
    p0 = vi.ansatz_params(7, H.n, 6)
    r = minimize_energy(eng, p0, maxiter=300)
    eng.close()
    assert r["energy"] < r["history"][0] - 0.5
    assert r["history"].min() >= e0 - 1e-10


def test_cutoff_ratio_search_c128(lib_built):
    """Algorithm 1 through the C ABI: 2-site Hubbard plus 30 tiny terms; the
    search keeps every Hubbard term and stops at the first ratio that cuts
    one."""
    from paper_2402_11878_gb300 import cutoff_ratio_search
    Hb = vi.hubbard_1d(2, 1.0, 4.0, periodic=False)
    Hs = vi.random_pauli_sum(4, 30, seed=9)
    H = vi.PauliSum(4, np.concatenate([Hb.x, Hs.x]), np.concatenate([Hb.z, Hs.z]),
                    np.concatenate([Hb.c, 1e-5 * Hs.c / np.abs(Hs.c).max()]))
    eng = _engine(H, 4, "c128")
    out = cutoff_ratio_search(eng, H.x, H.z, H.c, vi.ansatz_params(103, 4, 4), delta_e=1e-3)
    kept, dropped = eng.slim(out["threshold"])
    eng.close()
    assert out["threshold"] <= np.abs(Hb.c[Hb.c != 0]).min()
    assert dropped <= 30 * 1e-5 + 1e-12
    e_full = out["runs"][0][2]
    assert all(abs(e - e_full) < 1e-3 for r, k, e in out["runs"] if r >= out["ratio"] - 1e-9)
