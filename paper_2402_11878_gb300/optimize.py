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
    """Advance S starts (``params0``: S x n_params) together with Adam, one
    batched adjoint gradient per step.  Returns {"params" (S x n_params),
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
