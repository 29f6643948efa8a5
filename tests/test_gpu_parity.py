"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (fixed by the accuracy targets of the two precision modes):
  VQE_C128: |dE| <= 1e-11 * sum|c|, amplitudes max-abs <= 1e-12,
            gradients max-abs <= 1e-10 * max(1, |g_ref|_inf)
  VQE_C64:  |dE| <= 1e-5 * sum|c|, gradients |g - g_ref|_inf / |g_ref|_inf <= 1e-4
"""
import numpy as np
import pytest

import vqe_inputs as vi

pytestmark = pytest.mark.gpu

E_TOL = {"c128": 1e-11, "c64": 1e-5}


@pytest.fixture(scope="module")
def eng_mod(lib_built):
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2402_11878_gb300 as pkg
    return pkg


def make(pkg, n, depth, prec, H):
    e = pkg.Engine(n, depth, prec)
    e.set_hamiltonian(H.x, H.z, H.c)
    return e


def check_energy(E, E_ref, H, prec):
    tol = E_TOL[prec] * max(H.sum_abs(), 1e-300)
    assert abs(E - E_ref) <= tol, (E, E_ref, abs(E - E_ref), tol)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_config_small_hubbard_c128_state_and_energy(eng_mod, oracle_mod, seed):
    """8 qubits, 4-site open Hubbard t=1 U=4, depth 4, FP64: state and energy."""
    n, D = 8, 4
    H = vi.hubbard_1d(4, 1.0, 4.0, periodic=False)
    p = vi.ansatz_params(seed, n, D)
    eng = make(eng_mod, n, D, "c128", H)
    eng.apply_ansatz(p)
    psi = eng.get_state()
    ref = oracle_mod.ansatz_state(n, D, p)
    assert np.max(np.abs(psi - ref)) <= 1e-12
    E, nn = eng.energy()
    E_ref, n_ref = oracle_mod.energy(ref, H.x, H.z, H.c)
    check_energy(E, E_ref, H, "c128")
    assert abs(nn - 1.0) <= 1e-13


SIZES = [1, 2, 3, 4, 5, 7, 8, 9, 12, 13, 14, 15, 16, 17, 18]


# tile plans: the default, and two others the autotuner considers (smaller
# tiles with 4 amplitudes per thread; larger tiles)
PLANS = [(0, 0, 0), (9, 2, 2), (12, 0, 3)]


@pytest.mark.parametrize("plan", PLANS)
@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n", SIZES)
def test_random_pauli_sum_all_sizes(eng_mod, oracle_mod, prec, n, plan):
    """Every plan shape (single tile, multi-pass, ragged groups) on random Pauli sums with Y
    terms, under three tile plans."""
    D = 2 if n > 12 else 3
    H = vi.random_pauli_sum(n, 40, seed=100 + n, duplicates=3)
    p = vi.ansatz_params(7 + n, n, D)
    eng = make(eng_mod, n, D, prec, H)
    eng.set_plan_options(*plan)
    eng.apply_ansatz(p)
    psi = eng.get_state()
    ref = oracle_mod.ansatz_state(n, D, p)
    amp_tol = 1e-12 if prec == "c128" else 2e-6
    assert np.max(np.abs(psi - ref)) <= amp_tol
    E, nn = eng.energy()
    E_ref, _ = oracle_mod.energy(ref, H.x, H.z, H.c)
    check_energy(E, E_ref, H, prec)


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_batched_energies(eng_mod, oracle_mod, prec):
    n, D, B = 10, 3, 7
    H = vi.hubbard_1d(5, 1.0, 2.5, periodic=True)
    P = np.stack([vi.ansatz_params(50 + b, n, D) for b in range(B)])
    eng = make(eng_mod, n, D, prec, H)
    E, nn = eng.energy_batch(P)
    for b in range(B):
        ref = oracle_mod.ansatz_state(n, D, P[b])
        E_ref, _ = oracle_mod.energy(ref, H.x, H.z, H.c)
        check_energy(E[b], E_ref, H, prec)


@pytest.mark.parametrize("plan", PLANS)
@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n,D", [(2, 2), (3, 2), (8, 4), (13, 2), (14, 2), (16, 2), (17, 1)])
def test_adjoint_gradient(eng_mod, oracle_mod, prec, n, D, plan):
    H = vi.random_pauli_sum(n, 30, seed=200 + n) if n % 2 else vi.hubbard_1d(n // 2, 1.0, 4.0)
    H = vi.PauliSum(n, H.x, H.z, H.c)
    p = vi.ansatz_params(300 + n, n, D)
    eng = make(eng_mod, n, D, prec, H)
    eng.set_plan_options(*plan)
    g, E = eng.gradient(p)
    g_ref, E_ref = oracle_mod.gradient_adjoint(n, D, p, H.x, H.z, H.c)
    check_energy(E, E_ref, H, prec)
    scale = max(np.max(np.abs(g_ref)), 1e-30)
    err = np.max(np.abs(g - g_ref))
    if prec == "c64":
        assert err / scale <= 1e-4, (err, scale)
    else:
        assert err <= 1e-10 * max(1.0, scale), (err, scale)


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("case", ["hubbard", "molecular"])
def test_windowed_apply_h_gradient(eng_mod, oracle_mod, prec, case):
    """20 qubits, a batch large enough for the windowed apply-H (lambda = H psi
    accumulated window by window): adjoint gradients and energies vs the
    oracle's adjoint gradient, with every form of lambda = H psi (global
    sweep, windows, bit-ordered sweeps)."""
    n, D, B = 20, 2, 4
    H = vi.hubbard_1d(10, 1.0, 4.0, periodic=True) if case == "hubbard" else vi.synthetic_molecular(10, seed=3)
    P = np.stack([vi.ansatz_params(500 + b, n, D) for b in range(B)])
    eng = make(eng_mod, n, D, prec, H)
    refs = {b: oracle_mod.gradient_adjoint(n, D, P[b], H.x, H.z, H.c) for b in (0, B - 1)}
    for form in (0, 1, 2):
        assert eng.set_apply_mode(form) == form
        G, E = eng.gradient_batch(P)
        for b, (g_ref, E_ref) in refs.items():
            check_energy(E[b], E_ref, H, prec)
            scale = max(np.max(np.abs(g_ref)), 1e-30)
            err = np.max(np.abs(G[b] - g_ref))
            if prec == "c64":
                assert err / scale <= 1e-4, (form, err, scale)
            else:
                assert err <= 1e-10 * max(1.0, scale), (form, err, scale)


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n", [1, 2, 5, 9, 13, 17])
def test_sweep_apply_h_random_sums(eng_mod, oracle_mod, prec, n):
    """The sweep form of lambda = H psi on random Pauli sums with Y terms:
    groups in pattern form with several terms per pattern, groups with more
    X bits than the pattern form takes (terms unmerged), the diagonal; from
    one qubit (a single sweep smaller than a chunk) up."""
    D = 2
    H = vi.random_pauli_sum(n, 40, seed=700 + n, duplicates=3)
    p = vi.ansatz_params(710 + n, n, D)
    eng = make(eng_mod, n, D, prec, H)
    assert eng.set_apply_mode(2) == 2
    g, E = eng.gradient(p)
    g_ref, E_ref = oracle_mod.gradient_adjoint(n, D, p, H.x, H.z, H.c)
    check_energy(E, E_ref, H, prec)
    scale = max(np.max(np.abs(g_ref)), 1e-30)
    err = np.max(np.abs(g - g_ref))
    if prec == "c64":
        assert err / scale <= 1e-4, (err, scale)
    else:
        assert err <= 1e-10 * max(1.0, scale), (err, scale)


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_sweep_apply_h_several_sweeps_22q(eng_mod, oracle_mod, prec):
    """22 qubits on the 4x3 open lattice minus one site (hopping groups whose
    X bits span more than one sweep's fast bits): the sweep form runs several
    sweeps, lambda accumulated across them; the energy it yields against the
    oracle, its gradient against the windowed form's (checked against the
    oracle in test_windowed_apply_h_gradient) and, in FP64, the oracle's
    gradient."""
    from paper_2402_11878_gb300 import plans
    n, D = 22, 1
    H = vi.hubbard_2d_snake(11, 1, 1.0, 4.0, periodic=True)
    assert H.n == n
    sp = plans.sweeps(n, prec, H.x, H.z, H.c, diag_terms=False)
    assert len(sp["sweeps"]) >= 2
    p = vi.ansatz_params(2222, n, D)
    eng = make(eng_mod, n, D, prec, H)
    assert eng.set_apply_mode(2) == 2
    g2, E2 = eng.gradient(p)
    assert eng.set_apply_mode(1) == 1
    g1, E1 = eng.gradient(p)
    ref = oracle_mod.ansatz_state(n, D, p)
    E_ref, _ = oracle_mod.energy(ref, H.x, H.z, H.c)
    check_energy(E2, E_ref, H, prec)
    scale = max(np.max(np.abs(g1)), 1e-30)
    if prec == "c64":
        assert np.max(np.abs(g2 - g1)) / scale <= 1e-5
    else:
        assert np.max(np.abs(g2 - g1)) <= 1e-12 * max(1.0, scale)
        g_ref, _ = oracle_mod.gradient_adjoint(n, D, p, H.x, H.z, H.c)
        assert np.max(np.abs(g2 - g_ref)) <= 1e-10 * max(1.0, np.max(np.abs(g_ref)))


def test_gradient_batch_matches_single(eng_mod, oracle_mod):
    n, D, B = 9, 2, 3
    H = vi.random_pauli_sum(n, 25, seed=9)
    P = np.stack([vi.ansatz_params(400 + b, n, D) for b in range(B)])
    eng = make(eng_mod, n, D, "c128", H)
    G, E = eng.gradient_batch(P)
    for b in range(B):
        g_ref, E_ref = oracle_mod.gradient_adjoint(n, D, P[b], H.x, H.z, H.c)
        assert np.max(np.abs(G[b] - g_ref)) <= 1e-10 * max(1.0, np.max(np.abs(g_ref)))
        check_energy(E[b], E_ref, H, "c128")


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_slimming_against_oracle(eng_mod, oracle_mod, prec):
    """Cutoff: kept set, sum|c_dropped|, slimmed energy, and the Sec. II-D bound."""
    n, D = 12, 2
    M = vi.random_pauli_sum(n, 300, seed=5, duplicates=20)
    M.c = M.c * np.exp(-np.linspace(0, 12, len(M.c)))    # spread |c| over ~5 decades
    p = vi.ansatz_params(11, n, D)
    eng = make(eng_mod, n, D, prec, M)
    ref = oracle_mod.ansatz_state(n, D, p)
    eng.apply_ansatz(p)
    E_full, _ = eng.energy()
    for th in [0.0, 1e-4, 1e-3, 1e-2, 0.1, 10.0]:
        kept, dropped = eng.slim(th)
        xs, zs, cs, dref = oracle_mod.slim(M.x, M.z, M.c, th)
        assert kept == len(cs)
        assert abs(dropped - dref) <= 1e-12 * max(1.0, dref)
        E, _ = eng.energy()
        E_ref, _ = oracle_mod.energy(ref, xs, zs, cs) if len(cs) else (0.0, 1.0)
        check_energy(E, E_ref, M, prec)
        assert abs(E_full - E) <= dropped * (1 + 1e-9) + E_TOL[prec] * M.sum_abs()


def test_pergate_reference_kernel(eng_mod, oracle_mod):
    import torch
    n, D, B = 14, 3, 4
    H = vi.hubbard_1d(7, 1.0, 4.0, periodic=True)
    P = np.stack([vi.ansatz_params(70 + b, n, D) for b in range(B)])
    eng = make(eng_mod, n, D, "c128", H)
    pd = torch.tensor(P, device="cuda")
    e1 = torch.empty(B, dtype=torch.float64, device="cuda")
    e2 = torch.empty(B, dtype=torch.float64, device="cuda")
    eng.energy_batch_dev(pd, e1)
    eng.energy_batch_dev(pd, e2, pergate=True)
    torch.cuda.synchronize()
    for b in range(B):
        ref = oracle_mod.ansatz_state(n, D, P[b])
        E_ref, _ = oracle_mod.energy(ref, H.x, H.z, H.c)
        check_energy(float(e1[b]), E_ref, H, "c128")
        check_energy(float(e2[b]), E_ref, H, "c128")


def test_full_size_20q_fp64_hubbard(eng_mod, oracle_mod):
    """20 qubits FP64, 10-site periodic Hubbard, depth 10: whole state and energies vs oracle."""
    n, D = 20, 10
    for U in (2.0, 8.0):
        H = vi.hubbard_1d(10, 1.0, U, periodic=True)
        p = vi.ansatz_params(int(U) * 17, n, D)
        eng = make(eng_mod, n, D, "c128", H)
        eng.apply_ansatz(p)
        psi = eng.get_state()
        ref = oracle_mod.ansatz_state(n, D, p)
        assert np.max(np.abs(psi - ref)) <= 1e-12
        E, _ = eng.energy()
        E_ref, _ = oracle_mod.energy(ref, H.x, H.z, H.c)
        check_energy(E, E_ref, H, "c128")


def test_theta_zero_and_basis_states(eng_mod):
    """theta = 0 leaves |0..0>: E = sum of z-only coefficients; RY(pi) on all
    qubits prepares |1..1>, whose Hubbard energy is U * L (all sites doubly occupied)."""
    n, D = 12, 2
    H = vi.hubbard_1d(6, 1.0, 3.0)
    eng = make(eng_mod, n, D, "c128", H)
    eng.apply_ansatz(np.zeros(2 * n * D))
    E, _ = eng.energy()
    zonly = H.c[H.x == 0].sum()
    assert abs(E - zonly) <= 1e-12 * H.sum_abs()
    p = np.zeros(2 * n * D)
    p[0:2 * n:2] = np.pi
    eng.apply_ansatz(p)
    E, _ = eng.energy()
    assert abs(E - 3.0 * 6) <= 1e-11 * H.sum_abs()


def test_bitwise_determinism(eng_mod):
    n, D = 16, 3
    H = vi.random_pauli_sum(n, 60, seed=3)
    p = vi.ansatz_params(5, n, D)
    eng = make(eng_mod, n, D, "c64", H)
    g1, e1 = eng.gradient(p)
    g2, e2 = eng.gradient(p)
    assert e1 == e2 and np.array_equal(g1, g2)


def test_argument_errors(eng_mod):
    pkg = eng_mod
    eng = pkg.Engine(6, 2, "c64")
    with pytest.raises(pkg.VQEError) as ei:
        eng.energy()
    assert ei.value.status == 2
    with pytest.raises(pkg.VQEError) as ei:
        eng.set_hamiltonian([1 << 6], [0], [1.0])
    assert ei.value.status == 1
    with pytest.raises(pkg.VQEError):
        eng.set_hamiltonian([1], [0], [float("nan")])
    eng.set_hamiltonian([1], [0], [1.0])
    with pytest.raises(pkg.VQEError):
        eng.apply_ansatz(np.full(24, np.inf))
    with pytest.raises(pkg.VQEError):
        eng.slim(-1.0)


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("case", ["hubbard", "random", "molecular"])
def test_windowed_energy_batch(eng_mod, oracle_mod, prec, case):
    """Batches large enough for the windowed expectation kernel (tile windows + wide groups)."""
    if case == "hubbard":
        H = vi.hubbard_1d(9, 1.0, 2.0, periodic=True)
    elif case == "random":
        H = vi.random_pauli_sum(18, 80, seed=77, duplicates=5)
    else:
        H = vi.synthetic_molecular(9, seed=3)
    n, D, B = H.n, 2, 16
    P = np.stack([vi.ansatz_params(800 + b, n, D) for b in range(B)])
    eng = make(eng_mod, n, D, prec, H)
    E, nn = eng.energy_batch(P)
    for b in (0, 7, 15):
        ref = oracle_mod.ansatz_state(n, D, P[b])
        E_ref, _ = oracle_mod.energy(ref, H.x, H.z, H.c)
        check_energy(E[b], E_ref, H, prec)


def test_20q_fp64_windowed_energy_bench_chunks(eng_mod, oracle_mod):
    """20 qubits FP64 with a batch of 64 states (the chunk the 20-qubit bench
    workload runs): the windowed expectation kernel must be the one taken, and
    three of the states' energies must match the oracle to 1e-11 sum|c|."""
    import torch
    n, D, B = 20, 10, 64
    H = vi.hubbard_1d(10, 1.0, 4.0, periodic=True)
    P = np.stack([vi.ansatz_params(7000 + b, n, D) for b in range(B)])
    eng = make(eng_mod, n, D, "c128", H)
    Pd = torch.tensor(P, device="cuda")
    E = torch.empty(B, dtype=torch.float64, device="cuda")
    eng.profile(True)
    eng.energy_batch_dev(Pd, E)
    prof = eng.profile_read()
    eng.profile(False)
    from paper_2402_11878_gb300 import plans
    wins = plans.windows(n, "c128", H.x, H.z, H.c, diag_terms=False)
    n_win = len(wins["windows"])
    assert n_win >= 2
    assert prof["energy"]["launches"] == n_win      # one launch per window: the windowed kernel
    E = E.cpu().numpy()
    for b in (0, 31, 63):
        ref = oracle_mod.ansatz_state(n, D, P[b])
        E_ref, _ = oracle_mod.energy(ref, H.x, H.z, H.c)
        check_energy(E[b], E_ref, H, "c128")
    eng.close()


@pytest.mark.parametrize("batch", [1, 4])
def test_c64_energy_accumulation_matches_fp64_on_same_state(eng_mod, oracle_mod, batch):
    """Complex64 mode keeps its energy sums at FP64-level accuracy: a
    Hamiltonian dominated by a large identity and large Z terms, with small
    hopping terms, evaluated by the complex64 kernels (global sweep for one
    state, windows for four) against the FP64 oracle on the very same
    complex64 state.  Every coefficient and every diagonal sum is a dyadic
    number that FP32 holds exactly, so the only differences left are the
    independent roundings of FP32 amplitude products and the accumulation;
    the bound is far below what FP32 running sums over 2^20 amplitudes would
    leave."""
    import torch
    n, D = 20, 2
    base = vi.hubbard_1d(10, 1.0, 4.0, periodic=True)    # coefficients +-1/2, +-1, U/4
    zx = np.array([0] * n, dtype=np.uint64)
    zz = np.array([1 << q for q in range(n)], dtype=np.uint64)
    zc = 100.0 + 10.0 * np.arange(n)
    x = np.concatenate([base.x, zx, [0]]).astype(np.uint64)
    z = np.concatenate([base.z, zz, [0]]).astype(np.uint64)
    c = np.concatenate([base.c / 64.0, zc, [1024.0]])
    assert np.array_equal(c.astype(np.float32).astype(np.float64), c)
    H = vi.PauliSum(n, x, z, c)
    P = np.stack([vi.ansatz_params(8100 + b, n, D) for b in range(batch)])
    eng = make(eng_mod, n, D, "c64", H)
    eng.apply_ansatz(P[0])
    psi = eng.get_state().astype(np.complex128)
    E_same, _ = oracle_mod.energy(psi, H.x, H.z, H.c)
    Pd = torch.tensor(P, device="cuda")
    E = torch.empty(batch, dtype=torch.float64, device="cuda")
    eng.energy_batch_dev(Pd, E)
    got = float(E[0])
    assert abs(got - E_same) <= 2e-9 * H.sum_abs(), (got, E_same, abs(got - E_same) / H.sum_abs())
    eng.close()


def test_fp64_twelve_bit_tile_programs(eng_mod, oracle_mod):
    """The unrolled FP64 programs of 2^12-amplitude tiles (the shapes the
    32-qubit plan with tile_bits_max 12 uses, all four present at 16 qubits,
    depth 3): state, energy and gradient against the oracle."""
    n, D = 16, 3
    H = vi.hubbard_1d(8, 1.0, 4.0, periodic=True)
    p = vi.ansatz_params(1612, n, D)
    eng = make(eng_mod, n, D, "c128", H)
    eng.set_plan_options(12, 2, 3)
    eng.apply_ansatz(p)
    ref = oracle_mod.ansatz_state(n, D, p)
    assert np.max(np.abs(eng.get_state() - ref)) <= 1e-12
    g, E = eng.gradient(p)
    g_ref, E_ref = oracle_mod.gradient_adjoint(n, D, p, H.x, H.z, H.c)
    check_energy(E, E_ref, H, "c128")
    assert np.max(np.abs(g - g_ref)) <= 1e-10 * max(1.0, np.max(np.abs(g_ref)))
    eng.close()
