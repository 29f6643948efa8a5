"""Error contract of the C ABI: a failed call leaves the handle's
Hamiltonian, state and workspace as they were.  Device allocations are made
to fail on the host (vqe_testing_fail_allocations), so no GPU fault is
involved."""
import numpy as np
import pytest

import vqe_inputs as vi

pytestmark = pytest.mark.gpu

OOM = 3


@pytest.fixture()
def lib(lib_built):
    from paper_2402_11878_gb300 import binding
    L = binding.load()
    yield L
    L.vqe_testing_fail_allocations(-1)


def _engine(n, D, prec, H):
    import paper_2402_11878_gb300 as pkg
    e = pkg.Engine(n, D, prec)
    e.set_hamiltonian(H.x, H.z, H.c)
    return e


@pytest.mark.parametrize("after", [0, 1, 3, 6])
def test_failed_set_hamiltonian_keeps_previous_plan(lib, oracle_mod, after):
    n, D = 12, 2
    HA = vi.hubbard_1d(6, 1.0, 4.0, periodic=True)
    HB = vi.random_pauli_sum(n, 60, seed=5)
    p = vi.ansatz_params(31, n, D)
    eng = _engine(n, D, "c128", HA)
    eng.slim(0.6)                      # a cutoff that must survive the failure
    eng.apply_ansatz(p)
    E_A, _ = eng.energy()
    lib.vqe_testing_fail_allocations(after)
    with pytest.raises(Exception) as ei:
        eng.set_hamiltonian(HB.x, HB.z, HB.c)
    lib.vqe_testing_fail_allocations(-1)
    assert getattr(ei.value, "status", None) == OOM
    E_again, _ = eng.energy()
    assert E_again == E_A
    st = eng.stats()
    assert st["n_terms_kept"] < st["n_terms_canonical"]      # the cutoff is still in force
    # the handle still works for a new Hamiltonian afterwards
    eng.set_hamiltonian(HB.x, HB.z, HB.c)
    E_B, _ = eng.energy()
    ref = oracle_mod.ansatz_state(n, D, p)
    E_ref, _ = oracle_mod.energy(ref, HB.x, HB.z, HB.c)
    assert abs(E_B - E_ref) <= 1e-11 * HB.sum_abs()
    eng.close()


def test_failed_slim_keeps_previous_cutoff(lib):
    n, D = 10, 2
    H = vi.synthetic_molecular(5, seed=4)
    p = vi.ansatz_params(8, n, D)
    eng = _engine(n, D, "c128", H)
    eng.apply_ansatz(p)
    E0, _ = eng.energy()
    lib.vqe_testing_fail_allocations(0)
    with pytest.raises(Exception) as ei:
        eng.slim(1e-2)
    lib.vqe_testing_fail_allocations(-1)
    assert getattr(ei.value, "status", None) == OOM
    assert eng.energy()[0] == E0
    assert eng.stats()["n_terms_kept"] == eng.stats()["n_terms_canonical"]
    eng.close()


def test_workspace_growth_failure_runs_in_chunks(lib):
    """A batch that needs a larger workspace than the handle holds: when the
    larger allocation fails, the existing workspace is kept and the batch runs
    in chunks of the size it holds, with the same results."""
    import torch
    n, D, B = 10, 2, 24
    H = vi.hubbard_1d(5, 1.0, 2.0, periodic=False)
    P = torch.tensor(np.stack([vi.ansatz_params(600 + b, n, D) for b in range(B)]), device="cuda")
    E_all = torch.empty(B, dtype=torch.float64, device="cuda")
    E_chunk = torch.empty(B, dtype=torch.float64, device="cuda")
    eng = _engine(n, D, "c128", H)
    eng.energy_batch_dev(P, E_all)                 # one chunk of 24 states
    eng2 = _engine(n, D, "c128", H)
    eng2.energy_batch_dev(P[:2], E_chunk[:2])      # workspace and scratch for 2 states
    lib.vqe_testing_fail_allocations(0)
    try:
        eng2.energy_batch_dev(P, E_chunk)          # 12 chunks of 2, nothing allocated
        torch.cuda.synchronize()
    finally:
        lib.vqe_testing_fail_allocations(-1)
    # chunking changes only the reduction order of the energy sums
    assert float((E_chunk - E_all).abs().max()) <= 1e-12 * H.sum_abs()
    for e in (eng, eng2):
        e.close()
