"""Full-size GPU checks through the C ABI: 24-qubit synthetic molecular
Hamiltonian in complex64 and the 32-qubit 4x4 Hubbard lattice (64 GiB FP64
state).  The oracle cannot hold these states, so the checks are

  * single amplitudes against the path-sum oracle (oracle/pathsum.py),
  * the exact properties of Sec. II-B/II-D that hold at any size: norm 1,
    the vacuum energy at theta = 0, the cutoff bound of Sec. II-D,
  * complex64 against complex128 energies, and the complex64 adjoint
    gradient against FP64 parameter shifts on sampled components.
"""
import numpy as np
import pytest

import vqe_inputs as vi
from oracle import pathsum

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _engine(n, D, prec, H):
    import paper_2402_11878_gb300 as pkg
    eng = pkg.Engine(n, D, prec)
    eng.set_hamiltonian(H.x, H.z, H.c)
    return eng


def _indices(n, count, seed):
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, 1 << n, count, dtype=np.uint64).astype(np.int64)
    return np.concatenate([np.array([0, (1 << n) - 1], dtype=np.int64), idx])


def _gather(ws, idx):
    return ws[torch.as_tensor(idx, device=ws.device)].cpu().numpy().astype(np.complex128)


def _c64_amplitude_tol(n, D, ref):
    # Each amplitude passes through about D * (n + 2) FP32 roundings (one
    # scaled butterfly per qubit and layer, the diagonal product), each at most
    # 2^-24 relative, with intermediate growth of at most sqrt(2) per butterfly
    # form: bound 8 * D * (n + 2) * 2^-24 of the largest sampled amplitude.
    return 8.0 * D * (n + 2) * 2.0 ** -24 * float(np.max(np.abs(ref)))


def _shift_gradient(eng, p, j):
    """Exact parameter-shift derivative of <H> for the exp(-i t P / 2) gate j."""
    vals = []
    for s in (+1.0, -1.0):
        q = p.copy()
        q[j] += s * np.pi / 2
        eng.apply_ansatz(q)
        vals.append(eng.energy()[0])
    return 0.5 * (vals[0] - vals[1])


@pytest.mark.slow
def test_24q_molecular_c64_amplitudes_energy_gradient():
    """Synthetic molecular Hamiltonian, 24 qubits, depth 12, complex64 state:
    sampled amplitudes, norm, cutoff bound at every threshold, C64 vs FP64
    energy, adjoint gradient vs FP64 parameter shift."""
    n, D = 24, 12
    H = vi.synthetic_molecular(12, 2024)
    sabs = H.sum_abs()
    p = vi.ansatz_params(2424, n, D)

    e64 = _engine(n, D, "c64", H)
    ws = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    e64.bind_workspace(ws)
    e64.apply_ansatz(p)
    E64, n64 = e64.energy()
    idx = _indices(n, 24, 1)
    ref = pathsum.amplitudes(n, D, p, idx)
    got = _gather(ws, idx)
    assert np.max(np.abs(got - ref)) <= _c64_amplitude_tol(n, D, ref)
    assert abs(n64 - 1.0) <= 1e-5
    for th in (1e-6, 1e-4, 1e-3):
        kept, dropped = e64.slim(th)
        Es, ns = e64.energy()
        assert kept < H.c.size
        assert abs(Es - E64) <= dropped * ns + 1e-5 * sabs
    e64.slim(0.0)

    e128 = _engine(n, D, "c128", H)
    e128.apply_ansatz(p)
    E128, n128 = e128.energy()
    assert abs(n128 - 1.0) <= 1e-12
    assert abs(E64 - E128) <= 1e-5 * sabs

    P = torch.tensor(p[None, :], device="cuda")
    G = torch.empty(1, 2 * n * D, dtype=torch.float64, device="cuda")
    Eg = torch.empty(1, dtype=torch.float64, device="cuda")
    e64.bind_workspace(None)
    e64.gradient_batch_dev(P, G, Eg)
    g = G[0].cpu().numpy()
    assert abs(float(Eg[0]) - E128) <= 1e-5 * sabs
    gmax = np.max(np.abs(g))
    for j in (0, 1, 2 * n * D // 2 + 7, 2 * n * D - 2, 2 * n * D - 1):
        gs = _shift_gradient(e128, p, j)
        assert abs(g[j] - gs) <= 1e-4 * gmax, (j, g[j], gs)
    e64.close()
    e128.close()


@pytest.mark.slow
def test_32q_hubbard_2d_fp64_energy_and_c64_gradient():
    """4x4 periodic Hubbard in snake order, 32 qubits, depth 8: FP64 energy on
    a 64 GiB caller-owned state (amplitudes vs path sum, norm, vacuum energy,
    cutoff bound), the FP64 adjoint gradient through the benchmark's call
    path, then the complex64 adjoint gradient on psi and lambda (2 x 32 GiB),
    both against FP64 parameter shifts."""
    if torch.cuda.get_device_properties(0).total_memory < 200e9:
        pytest.skip("needs a GPU with at least 200 GB of memory")
    n, D = 32, 8
    H = vi.hubbard_2d_snake(4, 4, 1.0, 4.0)
    sabs = H.sum_abs()
    p = vi.ansatz_params(3232, n, D)
    jobs = (0, 2 * n * D - 1, 2 * (3 * n + 17))   # first theta, last phi, a middle theta

    eng = _engine(n, D, "c128", H)
    ws = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
    eng.bind_workspace(ws)
    eng.apply_ansatz(p)
    E, nrm = eng.energy()
    assert abs(nrm - 1.0) <= 1e-12
    idx = _indices(n, 30, 2)
    ref = pathsum.amplitudes(n, D, p, idx)
    assert np.max(np.abs(_gather(ws, idx) - ref)) <= 1e-12
    kept, dropped = eng.slim(0.6)     # drops every hopping term (|c| = t/2)
    Es, ns = eng.energy()
    assert abs(Es - E) <= dropped * ns + 1e-11 * sabs
    eng.slim(0.0)
    shifts = {j: _shift_gradient(eng, p, j) for j in jobs}
    eng.apply_ansatz(np.zeros(2 * n * D))
    E0, _ = eng.energy()
    assert abs(E0) <= 1e-11 * sabs      # vacuum: no particle, no energy
    # the benchmark's own call path: FP64 energy + adjoint gradient through
    # vqe_gradient_batch_dev on library-allocated psi and lambda (2 x 64 GiB)
    eng.bind_workspace(None)
    del ws
    torch.cuda.empty_cache()
    P = torch.tensor(p[None, :], device="cuda")
    G = torch.empty(1, 2 * n * D, dtype=torch.float64, device="cuda")
    Eg = torch.empty(1, dtype=torch.float64, device="cuda")
    eng.gradient_batch_dev(P, G, Eg)
    g = G[0].cpu().numpy()
    assert abs(float(Eg[0]) - E) <= 1e-11 * sabs
    gmax = max(1.0, float(np.max(np.abs(g))))
    for j, gs in shifts.items():
        assert abs(g[j] - gs) <= 1e-10 * gmax, (j, g[j], gs)
    eng.close()
    torch.cuda.empty_cache()

    e64 = _engine(n, D, "c64", H)
    P = torch.tensor(p[None, :], device="cuda")
    G = torch.empty(1, 2 * n * D, dtype=torch.float64, device="cuda")
    Eg = torch.empty(1, dtype=torch.float64, device="cuda")
    e64.gradient_batch_dev(P, G, Eg)
    g = G[0].cpu().numpy()
    assert abs(float(Eg[0]) - E) <= 1e-5 * sabs
    gmax = np.max(np.abs(g))
    for j, gs in shifts.items():
        assert abs(g[j] - gs) <= 1e-4 * gmax, (j, g[j], gs)
    e64.close()
    torch.cuda.empty_cache()


@pytest.mark.slow
def test_32q_particle_conserving_fp64_and_c64():
    """The particle-conserving ansatz at 32 qubits (4x4 lattice at half
    filling, 102 doubles + 16 singles, the benchmark's pc32 workload): the
    FP64 state keeps every amplitude outside the 16-electron sector exactly
    zero and its norm at 1; the energy from the gradient call equals the
    energy call; the FP64 adjoint gradient matches central differences of
    FP64 energies on sampled components; complex64 agrees with FP64 within
    its tolerances."""
    if torch.cuda.get_device_properties(0).total_memory < 200e9:
        pytest.skip("needs a GPU with at least 200 GB of memory")
    import paper_2402_11878_gb300 as pkg
    n, ne = 32, 16
    H = vi.hubbard_2d_snake(4, 4, 1.0, 4.0)
    sabs = H.sum_abs()
    exc = vi.excitations(n, ne, n_singles=16, n_doubles=102, seed=32)
    th = vi.excitation_params(3232, len(exc))
    eng = pkg.Engine.particle_conserving(n, ne, exc, "c128")
    eng.set_hamiltonian(H.x, H.z, H.c)
    ws = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
    eng.bind_workspace(ws)
    eng.apply_ansatz(th)
    E, nrm = eng.energy()
    assert abs(nrm - 1.0) <= 1e-12
    idx = _indices(n, 4000, 5)
    amp = _gather(ws, idx)
    N = np.array([bin(int(i)).count("1") for i in idx])
    assert np.max(np.abs(amp[N != ne])) == 0.0
    assert abs(_gather(ws, np.array([(1 << ne) - 1]))[0]) > 0.0     # psi_HF itself stays

    def energy_at(t):
        eng.apply_ansatz(t)
        return eng.energy()[0]

    h = 1e-4
    jobs = (0, 57, len(exc) - 1)                 # a double, a double, the last single
    fd = {}
    for j in jobs:
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        fd[j] = (energy_at(tp) - energy_at(tm)) / (2 * h)
    eng.bind_workspace(None)
    del ws
    torch.cuda.empty_cache()
    P = torch.tensor(th[None, :], device="cuda")
    G = torch.empty(1, len(exc), dtype=torch.float64, device="cuda")
    Eg = torch.empty(1, dtype=torch.float64, device="cuda")
    eng.gradient_batch_dev(P, G, Eg)
    g = G[0].cpu().numpy()
    assert abs(float(Eg[0]) - E) <= 1e-11 * sabs
    gmax = max(1.0, float(np.max(np.abs(g))))
    for j, v in fd.items():
        assert abs(g[j] - v) <= 1e-6 * gmax, (j, g[j], v)   # central differences: O(h^2)
    eng.close()
    torch.cuda.empty_cache()

    e64 = pkg.Engine.particle_conserving(n, ne, exc, "c64")
    e64.set_hamiltonian(H.x, H.z, H.c)
    G64 = torch.empty_like(G)
    e64.gradient_batch_dev(P, G64, Eg)
    assert abs(float(Eg[0]) - E) <= 1e-5 * sabs
    assert float((G64[0].cpu() - torch.from_numpy(g)).abs().max()) <= 1e-4 * float(np.max(np.abs(g)))
    e64.close()
    torch.cuda.empty_cache()
