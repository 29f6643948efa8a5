"""The torch.autograd.Function around the library's adjoint gradient, checked
against the FP64 oracle's parameter-shift gradient and central finite
differences (Sec. II-C: the gradient the paper obtains from per-parameter
circuit runs).

Tolerances: FP64 mode |g - g_shift|_inf <= 1e-10 max(1, |g|_inf) (parameter
shift is exact for exp(-i t P / 2) gates); central differences with h = 1e-5
carry an O(h^2) truncation error, so they are held to 1e-7.  Complex64 mode:
relative infinity-norm error <= 1e-4.
"""
import numpy as np
import pytest

import vqe_inputs as vi

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg(lib_built):
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2402_11878_gb300 as p
    return p


@pytest.mark.parametrize("device", ["cpu", "cuda"])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_energy_function_gradient_vs_shift_and_fd(pkg, oracle_mod, prec, device):
    n, D = 8, 3
    H = vi.hubbard_1d(4, 1.0, 4.0, periodic=False)
    p0 = vi.ansatz_params(4242, n, D)
    eng = pkg.Engine(n, D, prec)
    eng.set_hamiltonian(H.x, H.z, H.c)
    theta = torch.tensor(p0, dtype=torch.float64, device=device, requires_grad=True)
    E = pkg.EnergyFunction.apply(theta, eng)
    E.backward()
    g = theta.grad.detach().cpu().numpy()
    g_shift = oracle_mod.gradient_shift(n, D, p0, H.x, H.z, H.c)
    g_fd = oracle_mod.gradient_fd(n, D, p0, H.x, H.z, H.c, 1e-5)
    psi = oracle_mod.ansatz_state(n, D, p0)
    E_ref, _ = oracle_mod.energy(psi, H.x, H.z, H.c)
    scale = max(1.0, float(np.max(np.abs(g_shift))))
    if prec == "c128":
        assert abs(float(E) - E_ref) <= 1e-11 * H.sum_abs()
        assert np.max(np.abs(g - g_shift)) <= 1e-10 * scale
        assert np.max(np.abs(g - g_fd)) <= 1e-7 * scale
    else:
        assert abs(float(E) - E_ref) <= 1e-5 * H.sum_abs()
        assert np.max(np.abs(g - g_shift)) / float(np.max(np.abs(g_shift))) <= 1e-4
    eng.close()


def test_energy_function_chain_rule_and_energy_only(pkg, oracle_mod):
    """backward scales by the upstream gradient; without requires_grad only the
    energy runs (fewer kernel launches than an adjoint evaluation)."""
    n, D = 6, 2
    H = vi.hubbard_1d(3, 1.0, 2.0, periodic=False)
    p0 = vi.ansatz_params(77, n, D)
    eng = pkg.Engine(n, D, "c128")
    eng.set_hamiltonian(H.x, H.z, H.c)
    theta = torch.tensor(p0, dtype=torch.float64, device="cuda", requires_grad=True)
    E = pkg.EnergyFunction.apply(theta, eng)
    (3.0 * E).backward()
    g_shift = oracle_mod.gradient_shift(n, D, p0, H.x, H.z, H.c)
    assert np.max(np.abs(theta.grad.cpu().numpy() - 3.0 * g_shift)) <= 3e-10 * max(1.0, np.max(np.abs(g_shift)))

    l0 = eng.stats()["kernel_launches"]
    with torch.no_grad():
        E2 = pkg.EnergyFunction.apply(theta.detach(), eng)
    l_energy = eng.stats()["kernel_launches"] - l0
    l0 = eng.stats()["kernel_launches"]
    pkg.EnergyFunction.apply(theta.detach().requires_grad_(True), eng)
    l_grad = eng.stats()["kernel_launches"] - l0
    assert abs(float(E2) - float(E)) <= 1e-12 * H.sum_abs()
    assert l_energy < l_grad
    eng.close()
