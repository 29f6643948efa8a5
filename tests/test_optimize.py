"""Host VQE drivers (paper_2402_11878_gb300/optimize.py) on the CPU.

The drivers only call an engine's ``gradient`` / ``gradient_batch``; here
the engine is either an exact quadratic or the oracle's adjoint gradient, and
the converged energy is pinned to the exact ground-state energy from dense
diagonalisation (tests/dense.py), an independent route.
"""
import numpy as np
import pytest

import vqe_inputs as vi
from paper_2402_11878_gb300.optimize import minimize_batch, minimize_energy

import dense as dn


class _Quadratic:
    """f(p) = sum a_i (p_i - b_i)^2 + c, exact gradient."""

    def __init__(self, k, seed=0):
        rng = np.random.default_rng(seed)
        self.a = rng.uniform(0.5, 3.0, k)
        self.b = rng.uniform(-1.0, 1.0, k)
        self.c = -2.5

    def gradient(self, p):
        d = np.asarray(p) - self.b
        return 2.0 * self.a * d, float(np.sum(self.a * d * d) + self.c)

    def gradient_batch(self, P):
        out = [self.gradient(p) for p in np.asarray(P)]
        return np.array([o[0] for o in out]), np.array([o[1] for o in out])


class _OracleEngine:
    """The oracle's FP64 adjoint gradient behind the Engine's methods."""

    def __init__(self, oracle_mod, n, depth, H):
        self.o, self.n, self.depth, self.H = oracle_mod, n, depth, H

    def gradient(self, p):
        return self.o.gradient_adjoint(self.n, self.depth, p, self.H.x, self.H.z, self.H.c)

    def gradient_batch(self, P):
        out = [self.gradient(p) for p in np.asarray(P)]
        return np.array([o[0] for o in out]), np.array([o[1] for o in out])


def test_minimize_energy_quadratic():
    q = _Quadratic(12)
    r = minimize_energy(q, np.zeros(12))
    assert np.allclose(r["params"], q.b, atol=1e-6)
    assert abs(r["energy"] - q.c) < 1e-10
    assert r["evaluations"] == len(r["history"]) and r["history"][-1] <= r["history"][0]


def test_minimize_batch_quadratic():
    q = _Quadratic(6, seed=1)
    P0 = np.random.default_rng(2).uniform(-2, 2, (5, 6))
    r = minimize_batch(q, P0, steps=800, lr=0.05)
    assert r["params"].shape == P0.shape and r["history"].shape == (800, 5)
    assert np.allclose(r["params"], q.b[None, :], atol=1e-4)
    assert np.all(r["energies"] - q.c < 1e-7)
    with pytest.raises(ValueError):
        minimize_batch(q, np.zeros(6))


def test_vqe_two_site_hubbard_reaches_exact_ground_state(oracle_mod):
    """2-site open Hubbard (4 qubits, t = 1, U = 4), depth 4: L-BFGS on the
    adjoint gradient reaches the exact ground-state energy (-1 here), and no
    evaluated energy lies below it (variational principle)."""
    H = vi.hubbard_1d(2, 1.0, 4.0, periodic=False)
    n, D = H.n, 4
    e0 = float(np.linalg.eigvalsh(dn.hamiltonian_matrix(n, H.x, H.z, H.c))[0])
    r = minimize_energy(_OracleEngine(oracle_mod, n, D, H), vi.ansatz_params(103, n, D))
    assert abs(r["energy"] - e0) < 1e-9
    assert r["history"].min() >= e0 - 1e-10
