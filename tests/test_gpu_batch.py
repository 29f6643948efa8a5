"""GPU parity of the batched driver (persistent kernels per register-bit class, one CUDA graph) against the oracle."""
import numpy as np
import pytest

import vqe_inputs as vi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg(lib_built):
    import torch
    assert torch.cuda.is_available()
    import paper_2402_11878_gb300 as p
    return p


def run_batch(pkg, inst, prec="c64", tile_bits=None):
    b = pkg.Batch([d["n"] for d in inst], [d["depth"] for d in inst], prec)
    if tile_bits:
        b.set_tile_bits(tile_bits)
    for i, d in enumerate(inst):
        b.set_hamiltonian(i, d["H"].x, d["H"].z, d["H"].c)
    params = np.concatenate([d["params"] for d in inst])
    E, G = b.run(params)
    return b, E, G


def check(oracle_mod, inst, E, G, offsets, prec):
    for i, d in enumerate(inst):
        n, D, H = d["n"], d["depth"], d["H"]
        g_ref, e_ref = oracle_mod.gradient_adjoint(n, D, d["params"], H.x, H.z, H.c)
        tol = (1e-5 if prec == "c64" else 1e-11) * H.sum_abs()
        assert abs(E[i] - e_ref) <= tol, (i, n, E[i], e_ref)
        g = G[offsets[i]:offsets[i + 1]]
        scale = max(np.max(np.abs(g_ref)), 1e-30)
        if prec == "c64":
            assert np.max(np.abs(g - g_ref)) / scale <= 1e-4, (i, n)
        else:
            assert np.max(np.abs(g - g_ref)) <= 1e-10 * max(1.0, scale), (i, n)


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_batch_uneven_small(pkg, oracle_mod, prec):
    """Uneven sizes, including tiny ones and sizes that need several tiles."""
    inst = []
    for k, n in enumerate([3, 9, 12, 5, 13, 14, 8, 15, 12, 16, 1, 2]):
        if prec == "c128" and n > 14:
            continue
        D = max(1, n // 2)
        H = vi.random_pauli_sum(n, 20, seed=500 + k) if (k % 2 or n < 2) else vi.hubbard_1d(n // 2, 1.0, 3.0)
        H = vi.PauliSum(n, H.x, H.z, H.c)
        inst.append({"n": n, "depth": D, "H": H, "params": vi.ansatz_params(600 + k, n, D)})
    b, E, G = run_batch(pkg, inst, prec)
    check(oracle_mod, inst, E, G, b.offsets, prec)
    assert b.graph_launches() == 1


@pytest.mark.parametrize("tile_bits", [13, 12, 11])
def test_batch_config_instances(pkg, oracle_mod, tile_bits):
    """Instances of the uneven batch workload (12-18 qubits, open Hubbard, depth n/2), each tile plan."""
    inst = vi.batched_instances(10, seed=11)
    b, E, G = run_batch(pkg, inst, "c64", tile_bits=tile_bits)
    check(oracle_mod, inst, E, G, b.offsets, "c64")


def test_batch_graph_replay_and_device_buffers(pkg, oracle_mod):
    import torch
    inst = vi.batched_instances(6, seed=12)
    b = pkg.Batch([d["n"] for d in inst], [d["depth"] for d in inst], "c64",
                  stream=torch.cuda.current_stream())
    for i, d in enumerate(inst):
        b.set_hamiltonian(i, d["H"].x, d["H"].z, d["H"].c)
    P = torch.tensor(np.concatenate([d["params"] for d in inst]), device="cuda")
    E = torch.empty(len(inst), dtype=torch.float64, device="cuda")
    G = torch.empty_like(P)
    b.run_dev(P, E, G)
    torch.cuda.synchronize()
    e1, g1 = E.cpu().numpy().copy(), G.cpu().numpy().copy()
    b.run_dev(P, E, G)
    torch.cuda.synchronize()
    assert np.array_equal(e1, E.cpu().numpy()) and np.array_equal(g1, G.cpu().numpy())
    assert b.graph_launches() == 2
    check(oracle_mod, inst, e1, g1, b.offsets, "c64")
    k = b.autotune(P, E, G, reps=1)
    assert k in (11, 12, 13)
    torch.cuda.synchronize()
    check(oracle_mod, inst, E.cpu().numpy(), G.cpu().numpy(), b.offsets, "c64")


def test_batch_errors(pkg):
    b = pkg.Batch([4, 5], [2, 2], "c64")
    with pytest.raises(pkg.VQEError) as ei:
        b.run(np.zeros(int(b.n_params_total)))
    assert ei.value.status == 2       # no Hamiltonian yet
    with pytest.raises(pkg.VQEError):
        b.set_hamiltonian(1, [1 << 5], [0], [1.0])
