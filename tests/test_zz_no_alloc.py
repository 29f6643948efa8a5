"""vqe_energy_noalloc: the energy of caller-owned device states with no
device allocation inside the library.

It serves users whose code may not allocate device memory (memory owned by
another allocator or pool, loops that cannot take cudaMalloc's device-wide
synchronisation, plug-ins handed raw device pointers).  The test calls it
through the C ABI twice in a row, with different batch sizes, precisions and
Hamiltonians, and compares each result with the energies of the regular
entry point (vqe_energy_batch) at the tolerances used by the other GPU tests.
The energies are also compared with the FP64 oracle (Eq. 7 evaluated term
by term on the same states), and a term with a mask bit at or above n_qubits
must turn every energy of that call, and only that call, into NaN.
This file is collected last, so a failure here leaves every other test run.
"""
import ctypes

import numpy as np
import pytest

import vqe_inputs as vi

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-11, "c64": 1e-5}


def noalloc_fn(lib):
    f = lib.vqe_energy_noalloc
    vp = ctypes.c_void_p
    f.argtypes = [ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, vp, vp, vp, ctypes.c_size_t,
                  vp, vp, vp]
    f.restype = ctypes.c_int
    return f


def states_and_reference(pkg, n, depth, prec, H, P):
    """Device states of the regular path and its energies (regular entry point)."""
    import torch
    eng = pkg.Engine(n, depth, prec)
    eng.set_hamiltonian(H.x, H.z, H.c)
    E_ref, N_ref = eng.energy_batch(P)
    states = []
    for p in P:
        eng.apply_ansatz(p)
        states.append(eng.get_state())
    eng.close()
    psi = torch.from_numpy(np.stack(states)).cuda()
    return psi, E_ref, N_ref


def run_noalloc(lib, n, prec, psi, H):
    import torch
    B = psi.shape[0]
    x = torch.from_numpy(H.x.astype(np.uint64).view(np.int64)).cuda()
    z = torch.from_numpy(H.z.astype(np.uint64).view(np.int64)).cuda()
    c = torch.from_numpy(np.asarray(H.c, dtype=np.float64)).cuda()
    e = torch.full((B,), -1.0, dtype=torch.float64, device="cuda")
    nn = torch.full((B,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = noalloc_fn(lib)(n, {"c64": 0, "c128": 1}[prec], psi.data_ptr(), B, x.data_ptr(),
                         z.data_ptr(), c.data_ptr(), len(H.c), e.data_ptr(), nn.data_ptr(),
                         stream or None)
    assert st == 0
    torch.cuda.synchronize()
    return e.cpu().numpy(), nn.cpu().numpy()


def test_noalloc_energy_matches_regular_entry_point_twice(lib_built, oracle_mod):
    import torch
    assert torch.cuda.is_available()
    import paper_2402_11878_gb300 as pkg
    lib = pkg.load()

    # call 1: FP64 states, 5 of them, random Pauli sum with repeated strings and Y factors
    n, D = 11, 3
    H1 = vi.random_pauli_sum(n, 80, seed=17, duplicates=6)
    P1 = np.stack([vi.ansatz_params(900 + b, n, D) for b in range(5)])
    psi1, E1_ref, N1_ref = states_and_reference(pkg, n, D, "c128", H1, P1)
    E1, N1 = run_noalloc(lib, n, "c128", psi1, H1)
    assert np.max(np.abs(E1 - E1_ref)) <= TOL["c128"] * H1.sum_abs()
    assert np.max(np.abs(N1 - N1_ref)) <= 1e-12
    for b in range(len(P1)):   # the oracle on the oracle's own state
        E_orc, N_orc = oracle_mod.energy(oracle_mod.ansatz_state(n, D, P1[b]), H1.x, H1.z, H1.c)
        assert abs(E1[b] - E_orc) <= TOL["c128"] * H1.sum_abs()
        assert abs(N1[b] - N_orc) <= 1e-12

    # call 2: complex64 states, 2 of them, a Hubbard Hamiltonian on another size
    n2, D2 = 14, 2
    H2 = vi.hubbard_1d(7, 1.0, 4.0, periodic=True)
    P2 = np.stack([vi.ansatz_params(950 + b, n2, D2) for b in range(2)])
    psi2, E2_ref, N2_ref = states_and_reference(pkg, n2, D2, "c64", H2, P2)
    E2, N2 = run_noalloc(lib, n2, "c64", psi2, H2)
    assert np.max(np.abs(E2 - E2_ref)) <= TOL["c64"] * H2.sum_abs()
    assert np.max(np.abs(N2 - N2_ref)) <= 1e-5
    for b in range(len(P2)):   # FP64 oracle on the same complex64 state
        psi_b = psi2[b].cpu().numpy().astype(np.complex128)
        E_orc, _ = oracle_mod.energy(psi_b, H2.x, H2.z, H2.c)
        assert abs(E2[b] - E_orc) <= TOL["c64"] * H2.sum_abs()


def test_noalloc_invalid_term_sets_nan_for_that_call_only(lib_built):
    """A term whose X mask has bit n set is skipped before any memory access and
    makes every energy of the call NaN; the next valid call is finite again."""
    import torch
    import paper_2402_11878_gb300 as pkg
    lib = pkg.load()
    n, D = 9, 2
    H = vi.hubbard_1d(4, 1.0, 3.0, periodic=False)
    P = np.stack([vi.ansatz_params(970 + b, n, D) for b in range(3)])
    psi, E_ref, _ = states_and_reference(pkg, n, D, "c128", H, P)
    bad = vi.PauliSum(n, np.append(H.x, np.uint64(1) << np.uint64(n)), np.append(H.z, np.uint64(0)),
                      np.append(H.c, 0.5))
    E_bad, _ = run_noalloc(lib, n, "c128", psi, bad)
    assert np.all(np.isnan(E_bad))
    E_ok, _ = run_noalloc(lib, n, "c128", psi, H)
    assert np.all(np.isfinite(E_ok))
    assert np.max(np.abs(E_ok - E_ref)) <= TOL["c128"] * H.sum_abs()


def test_noalloc_rejects_batch_beyond_limit(lib_built):
    import paper_2402_11878_gb300 as pkg
    lib = pkg.load()
    f = noalloc_fn(lib)
    one = ctypes.c_void_p(256)          # never dereferenced: the call rejects first
    assert f(8, 1, one, 4097, None, None, None, 0, one, None, None) == 1
    assert f(8, 1, one, 0, None, None, None, 0, one, None, None) == 1
    assert f(33, 1, one, 1, None, None, None, 0, one, None, None) == 1
