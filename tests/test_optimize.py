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


def test_threshold_for_ratio_keeps_the_largest_terms(oracle_mod):
    """The threshold for a ratio keeps exactly ceil(ratio * N) merged terms
    (distinct |c|), checked with the oracle's cutoff rule."""
    from paper_2402_11878_gb300.optimize import merged_abs_coefficients, threshold_for_ratio
    H = vi.random_pauli_sum(7, 40, seed=8, duplicates=3)
    a = merged_abs_coefficients(H.x, H.z, H.c)
    assert np.all(np.diff(a) <= 0) and np.unique(a).size == a.size
    for ratio in np.round(np.arange(0.1, 1.01, 0.1), 12):
        th = threshold_for_ratio(a, ratio)
        kept = oracle_mod.slim(H.x, H.z, H.c, th)[0]
        assert len(kept) == int(np.ceil(ratio * a.size - 1e-9)), ratio


class _SlimRecorder:
    def __init__(self, n_terms):
        self.n, self.th = n_terms, None

    def slim(self, th):
        self.th = th
        return self.n, 0.0


@pytest.mark.parametrize("fail_at,expect", [(0.6, 0.7), (0.9, 1.0), (None, 0.1)])
def test_cutoff_ratio_search_return_rule(fail_at, expect):
    """Algorithm 1 as read: ratios 1, 0.9, ... ; stop at the first energy off
    by >= delta_e and return the ratio before it; 0.1 when none fails."""
    from paper_2402_11878_gb300.optimize import cutoff_ratio_search
    x = np.arange(1, 11, dtype=np.uint64)
    z = np.zeros(10, dtype=np.uint64)
    c = np.linspace(1.0, 0.1, 10)
    eng = _SlimRecorder(10)
    seen = []

    def vqe(e, p0):
        r = 1.0 if e.th == 0.0 else float(np.sum(c >= e.th)) / 10.0
        seen.append(r)
        return 1.0 if (fail_at is not None and r <= fail_at + 1e-9) else 0.0

    out = cutoff_ratio_search(eng, x, z, c, None, delta_e=0.5, vqe=vqe)
    assert abs(out["ratio"] - expect) < 1e-9
    assert seen[0] == 1.0 and np.allclose(np.diff(seen), -0.1)
    assert abs(eng.th - out["threshold"]) < 1e-15   # engine left at the answer


class _OracleSlimEngine(_OracleEngine):
    """Oracle adjoint gradient on the terms kept by the cutoff."""

    def __init__(self, oracle_mod, n, depth, H):
        super().__init__(oracle_mod, n, depth, H)
        self.full = H

    def slim(self, th):
        kx, kz, kc, dropped = self.o.slim(self.full.x, self.full.z, self.full.c, th)
        self.H = vi.PauliSum(self.n, kx, kz, kc)
        return len(kc), dropped


def test_cutoff_ratio_search_drops_only_small_terms(oracle_mod):
    """2-site Hubbard plus 30 tiny terms (|c| <= 1e-5): with delta_e = 1e-3
    the search cuts tiny terms only and stops at the first ratio that cuts a
    Hubbard term (its converged energy moves by more than delta_e)."""
    from paper_2402_11878_gb300.optimize import cutoff_ratio_search, merged_abs_coefficients
    Hb = vi.hubbard_1d(2, 1.0, 4.0, periodic=False)
    Hs = vi.random_pauli_sum(4, 30, seed=9)
    H = vi.PauliSum(4, np.concatenate([Hb.x, Hs.x]), np.concatenate([Hb.z, Hs.z]),
                    np.concatenate([Hb.c, 1e-5 * Hs.c / np.abs(Hs.c).max()]))
    eng = _OracleSlimEngine(oracle_mod, 4, 4, H)
    p0 = vi.ansatz_params(103, 4, 4)
    out = cutoff_ratio_search(eng, H.x, H.z, H.c, p0, delta_e=1e-3)
    big = np.abs(Hb.c[Hb.c != 0]).min()
    assert out["threshold"] <= big                       # every Hubbard term kept
    e_full = out["runs"][0][2]
    assert all(abs(e - e_full) < 1e-3 for r, k, e in out["runs"] if r >= out["ratio"] - 1e-9)
    assert out["ratio"] < 1.0 and len(merged_abs_coefficients(H.x, H.z, H.c)) > out["runs"][-1][1]
