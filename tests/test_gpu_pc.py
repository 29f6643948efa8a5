"""GPU parity of the particle-conserving ansatz (Sec. II-B, Eqs. 5-6) through
the C ABI (vqe_create_pc) against the FP64 oracle: states, energies and
adjoint gradients, from one tile (every mode in shared memory) to many tiles
and passes, in both precisions.

Tolerances as for the hardware-efficient ansatz: FP64 amplitudes 1e-12,
|dE| <= 1e-11 sum|c|, gradients 1e-10 max(1, |g|_inf); complex64 amplitudes
2e-6, |dE| <= 1e-5 sum|c|, gradients |dg|_inf / |g|_inf <= 1e-4.
"""
import numpy as np
import pytest

import vqe_inputs as vi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg(lib_built):
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2402_11878_gb300 as p
    return p


def _case(n):
    """(n_elec, excitations, Hamiltonian): half filling; all singles and
    doubles up to 8 qubits, a seeded subset above."""
    ne = n // 2
    if n == 2:
        exc = np.array([[1, -1, 0, -1]], dtype=np.int32)   # spin-flipping single: the only one
    elif n <= 8:
        exc = vi.excitations(n, ne)
    else:
        exc = vi.excitations(n, ne, n_singles=10, n_doubles=30, seed=n)
    H = vi.hubbard_1d(n // 2, 1.0, 4.0, periodic=n >= 6)
    return ne, exc, H


SIZES = [2, 4, 6, 8, 10, 12, 13, 14, 16, 18]


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n", SIZES)
def test_pc_state_and_energy(pkg, oracle_mod, prec, n):
    ne, exc, H = _case(n)
    th = vi.excitation_params(100 + n, len(exc))
    eng = pkg.Engine.particle_conserving(n, ne, exc, prec)
    eng.set_hamiltonian(H.x, H.z, H.c)
    eng.apply_ansatz(th)
    psi = eng.get_state()
    ref = oracle_mod.pc_ansatz_state(n, ne, exc, th)
    tol = 1e-12 if prec == "c128" else 2e-6
    assert np.max(np.abs(psi - ref)) <= tol
    E, nn = eng.energy()
    E_ref, _ = oracle_mod.energy(ref, H.x, H.z, H.c)
    assert abs(E - E_ref) <= (1e-11 if prec == "c128" else 1e-5) * H.sum_abs()
    # the state stays in the n_elec sector
    N = np.array([bin(i).count("1") for i in range(1 << n)])
    assert np.max(np.abs(psi[N != ne])) == 0.0
    eng.close()


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n", [4, 8, 12, 14, 17])
def test_pc_adjoint_gradient(pkg, oracle_mod, prec, n):
    ne = n // 2
    exc = vi.excitations(n, ne) if n <= 8 else vi.excitations(n, ne, 8, 24, seed=3 * n)
    H = vi.hubbard_1d(n // 2, 1.0, 3.0, periodic=True)
    H = vi.PauliSum(n, H.x, H.z, H.c)       # odd n: the top qubit carries no term
    th = vi.excitation_params(200 + n, len(exc))
    eng = pkg.Engine.particle_conserving(n, ne, exc, prec)
    eng.set_hamiltonian(H.x, H.z, H.c)
    g, E = eng.gradient(th)
    g_ref, E_ref = oracle_mod.pc_gradient_adjoint(n, ne, exc, th, H.x, H.z, H.c)
    scale = max(float(np.max(np.abs(g_ref))), 1e-30)
    if prec == "c128":
        assert abs(E - E_ref) <= 1e-11 * H.sum_abs()
        assert np.max(np.abs(g - g_ref)) <= 1e-10 * max(1.0, scale)
    else:
        assert abs(E - E_ref) <= 1e-5 * H.sum_abs()
        assert np.max(np.abs(g - g_ref)) / scale <= 1e-4
    eng.close()


def test_pc_batch_and_molecular(pkg, oracle_mod):
    """Batched energies and gradients on the synthetic molecular Hamiltonian
    (5 spatial orbitals, 10 qubits, 4 electrons)."""
    import torch
    n, ne, B = 10, 4, 5
    H = vi.synthetic_molecular(5, seed=9)
    exc = vi.excitations(n, ne)
    P = np.stack([vi.excitation_params(300 + b, len(exc)) for b in range(B)])
    eng = pkg.Engine.particle_conserving(n, ne, exc, "c128")
    eng.set_hamiltonian(H.x, H.z, H.c)
    E, nn = eng.energy_batch(P)
    G, Eg = eng.gradient_batch(P)
    for b in range(B):
        g_ref, E_ref = oracle_mod.pc_gradient_adjoint(n, ne, exc, P[b], H.x, H.z, H.c)
        assert abs(E[b] - E_ref) <= 1e-11 * H.sum_abs()
        assert abs(Eg[b] - E_ref) <= 1e-11 * H.sum_abs()
        assert abs(nn[b] - 1.0) <= 1e-13
        assert np.max(np.abs(G[b] - g_ref)) <= 1e-10 * max(1.0, np.max(np.abs(g_ref)))
    # device-buffer path gives the same numbers
    Pd = torch.tensor(P, device="cuda")
    Gd = torch.empty_like(Pd)
    Ed = torch.empty(B, dtype=torch.float64, device="cuda")
    eng.gradient_batch_dev(Pd, Gd, Ed)
    assert np.array_equal(Gd.cpu().numpy(), G)
    eng.close()


def test_pc_two_site_hubbard_vqe_reaches_ground_state(pkg):
    """The converged VQE through the C ABI reaches the exact half-filled
    ground energy of the 2-site Hubbard model, (U - sqrt(U^2 + 16 t^2)) / 2."""
    U, t = 4.0, 1.0
    H = vi.hubbard_1d(2, t, U, periodic=False)
    exc = vi.excitations(4, 2)
    eng = pkg.Engine.particle_conserving(4, 2, exc, "c128")
    eng.set_hamiltonian(H.x, H.z, H.c)
    e0 = (U - np.sqrt(U * U + 16 * t * t)) / 2
    best = min(pkg.minimize_energy(eng, vi.excitation_params(s, len(exc)))["energy"] for s in range(3))
    assert abs(best - e0) <= 1e-9
    eng.close()


def test_pc_rejects_bad_excitations(pkg):
    from paper_2402_11878_gb300.binding import VQEError
    for bad in ([[4, -1, 0, -1]],            # mode beyond n
                [[1, 1, 0, 2]],               # repeated mode
                [[1, -1, 1, -1]],             # single onto itself
                [[2, -1, 0, 3]]):             # single with a fourth mode
        with pytest.raises(VQEError):
            pkg.Engine.particle_conserving(4, 2, bad, "c128")
    eng = pkg.Engine.particle_conserving(4, 2, [[2, -1, 0, -1]], "c128")
    with pytest.raises(VQEError):
        eng.set_plan_options(10, 0, 0)
    eng.close()
