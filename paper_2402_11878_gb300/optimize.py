"""Host VQE loop driven by the library's adjoint gradient.

The paper's optimiser (SLSQP, Sec. II-C) needs the energy at N_p + N_s
parameter points per iteration and spreads them over workers.  Here each
iteration costs one energy-and-gradient evaluation: the forward sweep,
lambda = H psi and the adjoint backward sweep of the library, however many
parameters there are.

Two drivers:

  * ``minimize_energy``: one start, quasi-Newton (L-BFGS-B from SciPy).
  * ``minimize_batch``: many starts advanced together with Adam, each step
    one batched gradient call (all starts' states in one launch sequence).

Both accept any object with the Engine's ``gradient`` / ``gradient_batch``
methods, so the host logic is testable without a GPU.

``cutoff_ratio_search`` is the paper's way of choosing the cutoff of
Sec. II-D (Algorithm 1): converge VQE on a smaller problem at decreasing
kept fractions of the terms and keep the smallest fraction whose energy stays
within the required accuracy; ``threshold_for_ratio`` turns that fraction
into the threshold for a larger problem.
"""
from __future__ import annotations

import numpy as np


def minimize_energy(engine, params0, maxiter: int = 500, gtol: float = 1e-9,
                    callback=None) -> dict:
    """Minimise <H>(theta) from ``params0`` with L-BFGS-B on the adjoint
    gradient.  Returns {"params", "energy", "iterations", "evaluations",
    "history"} where history holds the energy of every evaluation."""
    from scipy.optimize import minimize

    history = []

    def fun(p):
        g, e = engine.gradient(p)
        history.append(float(e))
        return float(e), np.asarray(g, dtype=np.float64)

    res = minimize(fun, np.asarray(params0, dtype=np.float64), jac=True, method="L-BFGS-B",
                   options={"maxiter": int(maxiter), "gtol": float(gtol), "ftol": 1e-15},
                   callback=callback)
    return {"params": np.asarray(res.x), "energy": float(res.fun), "iterations": int(res.nit),
            "evaluations": len(history), "history": np.asarray(history)}


def minimize_batch(engine, params0, steps: int = 300, lr: float = 0.05,
                   beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-12) -> dict:
    """Advance S starts (``params0``: S x n_params) together with Adam
    (Kingma and Ba, 2015: bias-corrected first and second moment estimates),
    one batched adjoint gradient per step.  Returns {"params" (S x n_params),
    "energies" (S,), "best" (index of the lowest), "history" (steps x S)}."""
    P = np.array(params0, dtype=np.float64, copy=True)
    if P.ndim != 2:
        raise ValueError("params0 must be starts x n_params")
    m = np.zeros_like(P)
    v = np.zeros_like(P)
    hist = np.empty((int(steps), P.shape[0]))
    for t in range(1, int(steps) + 1):
        G, E = engine.gradient_batch(P)
        G = np.asarray(G, dtype=np.float64).reshape(P.shape)
        hist[t - 1] = E
        m = beta1 * m + (1.0 - beta1) * G
        v = beta2 * v + (1.0 - beta2) * G * G
        mh = m / (1.0 - beta1 ** t)
        vh = v / (1.0 - beta2 ** t)
        P -= lr * mh / (np.sqrt(vh) + eps)
    _, E = engine.gradient_batch(P)
    E = np.asarray(E, dtype=np.float64)
    return {"params": P, "energies": E, "best": int(np.argmin(E)), "history": hist}


# ---------------------------------------------------------------- cutoff ratio

def merged_abs_coefficients(x_masks, z_masks, coeffs, n_qubits: int = 0) -> np.ndarray:
    """|c| of the Pauli strings after merging equal (x, z) pairs and dropping
    exact zeros (the terms the library's cutoff acts on), largest first.

    The canonical terms come from the library's own canonicalisation (its
    host-side plan inspection), so the threshold chosen from them matches what
    ``vqe_slim`` keeps.  ``n_qubits`` defaults to the highest mask bit + 1."""
    from . import plans
    x = np.ascontiguousarray(x_masks, dtype=np.uint64)
    z = np.ascontiguousarray(z_masks, dtype=np.uint64)
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    if not n_qubits:
        top = int(np.bitwise_or.reduce(x | z)) if x.size else 0
        n_qubits = max(1, top.bit_length())
    prep = plans.hamiltonian(n_qubits, x, z, c, 0.0)
    a = np.abs(np.asarray(prep["tc"], dtype=np.float64))
    return np.sort(a)[::-1]


def threshold_for_ratio(abs_coeffs_desc, ratio: float) -> float:
    """Cutoff threshold that keeps the ceil(ratio * N) largest-|c| terms of a
    Hamiltonian whose merged |c| are given largest first (Sec. II-D: terms
    with |c| < threshold are dropped; terms tied with the last kept one stay
    too).  ratio >= 1 keeps every term (threshold 0)."""
    a = np.asarray(abs_coeffs_desc, dtype=np.float64)
    if ratio >= 1.0 or a.size == 0:
        return 0.0
    k = max(1, int(np.ceil(ratio * a.size - 1e-9)))
    return float(a[k - 1])


def cutoff_ratio_search(engine, x_masks, z_masks, coeffs, params0, delta_e: float,
                        step: float = 0.1, min_ratio: float = 0.1, vqe=None) -> dict:
    """The cutoff-ratio search of Sec. II-D (Algorithm 1), on a problem small
    enough to converge: starting from the whole Hamiltonian (ratio 1), lower
    the kept fraction of terms (largest |c| first) by ``step`` while the
    converged VQE energy stays within ``delta_e`` of the whole Hamiltonian's;
    the answer is the smallest ratio that still met the accuracy (the ratio
    before the first failure, or ``min_ratio`` if none failed).  Apply it to a
    larger problem with ``threshold_for_ratio``.

    ``vqe(engine, params0)`` returns the converged energy (default: L-BFGS
    from ``params0``).  The engine is left slimmed to the returned ratio.
    Returns {"ratio", "threshold", "runs": [(ratio, kept, energy), ...]}."""
    if vqe is None:
        def vqe(eng, p0):
            return minimize_energy(eng, p0)["energy"]
    a = merged_abs_coefficients(x_masks, z_masks, coeffs)
    runs = []
    e_full = None
    ratio = 1.0
    best = 1.0
    n_steps = int(round((1.0 - min_ratio) / step))
    for i in range(n_steps + 1):
        ratio = round(1.0 - i * step, 12)
        th = threshold_for_ratio(a, ratio)
        kept, _ = engine.slim(th)
        e = float(vqe(engine, params0))
        runs.append((ratio, int(kept), e))
        if e_full is None:
            e_full = e
        if abs(e - e_full) >= delta_e:
            break
        best = ratio
    th = threshold_for_ratio(a, best)
    engine.slim(th)
    return {"ratio": best, "threshold": th, "runs": runs}
