"""The single-handle autotuner (vqe_autotune): every plan it may choose, and
every form of lambda = H psi, give the oracle's energies and adjoint
gradients; the tuned handle keeps producing them.

CANDIDATES mirrors the plans (tile_bits_max, run_bits, reg_bits; 0 = the
default) that the autotuner times, in its order.
"""
import numpy as np
import pytest

import vqe_inputs as vi

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

CANDIDATES = {
    "c128": [(0, 0, 0), (10, 2, 3), (12, 2, 3), (11, 2, 2), (11, 3, 3), (9, 2, 2)],
    "c64": [(0, 0, 0), (12, 3, 4), (10, 3, 4), (11, 3, 3), (12, 4, 4), (13, 3, 4)],
}


def _check(prec, E, g, E_ref, g_ref, H):
    scale = max(float(np.max(np.abs(g_ref))), 1e-30)
    if prec == "c128":
        assert abs(E - E_ref) <= 1e-11 * H.sum_abs()
        assert np.max(np.abs(g - g_ref)) <= 1e-10 * max(1.0, scale)
    else:
        assert abs(E - E_ref) <= 1e-5 * H.sum_abs()
        assert np.max(np.abs(g - g_ref)) / scale <= 1e-4


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_every_candidate_plan_and_apply_form_matches_oracle(lib_built, oracle_mod, prec):
    import paper_2402_11878_gb300 as pkg
    n, D = 15, 2
    H = vi.hubbard_1d(7, 1.0, 4.0, periodic=True)
    H = vi.PauliSum(n, H.x, H.z, H.c)          # the top qubit carries ansatz gates only
    p = vi.ansatz_params(1515, n, D)
    g_ref, E_ref = oracle_mod.gradient_adjoint(n, D, p, H.x, H.z, H.c)
    eng = pkg.Engine(n, D, prec)
    eng.set_hamiltonian(H.x, H.z, H.c)
    for plan in CANDIDATES[prec]:
        eng.set_plan_options(*plan)
        for form in (0, 1, 2):
            assert eng.set_apply_mode(form) == form
            g, E = eng.gradient(p)
            _check(prec, E, g, E_ref, g_ref, H)
    eng.close()


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_autotuned_handle_matches_oracle(lib_built, oracle_mod, prec):
    import paper_2402_11878_gb300 as pkg
    n, D, B = 16, 3, 8
    H = vi.hubbard_1d(8, 1.0, 4.0, periodic=True)
    P = np.stack([vi.ansatz_params(1600 + b, n, D) for b in range(B)])
    eng = pkg.Engine(n, D, prec)
    eng.set_hamiltonian(H.x, H.z, H.c)
    Pd = torch.tensor(P, device="cuda")
    t = eng.autotune(Pd, gradient=True, budget_ms=1e9)
    assert t["candidates"] == len(CANDIDATES[prec])
    assert t["ms_best"] <= t["ms_default"] + 1e-9
    assert t["apply_ms_global"] > 0 and t["apply_ms_windows"] > 0 and t["apply_ms_sweeps"] > 0
    assert t["apply_form"] in (0, 1, 2)
    G, E = eng.gradient_batch(P)
    for b in (0, B - 1):
        g_ref, E_ref = oracle_mod.gradient_adjoint(n, D, P[b], H.x, H.z, H.c)
        _check(prec, E[b], G[b], E_ref, g_ref, H)
    st = eng.stats()
    assert st["tile_bits_max"] == t["tile_bits_max"] or st["tile_bits_max"] <= n
    eng.close()
