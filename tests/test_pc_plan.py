"""Host checks of the excitation-pass plan (vqe_inspect_pc_plan) on the CPU:
a NumPy replay of what the pass kernel does with the plan's records -- tile
gather through the high-part offsets and the tile-number bits, pair
enumeration around the fixed bits, the split Jordan-Wigner sign, the
rotation, the adjoint's gradient rows -- must reproduce the oracle's state
and adjoint gradient.  No GPU."""
import numpy as np
import pytest

import vqe_inputs as vi


def _plan(n, prec, exc, ne=0):
    from paper_2402_11878_gb300 import plans
    return plans.pc_plan(n, prec, exc, ne)


def _tile_indices(n, P, hoff, tile):
    bm, base, tn = int(P.bmask), 0, tile
    while bm:
        bit = (bm & -bm).bit_length() - 1
        base |= (tn & 1) << bit
        tn >>= 1
        bm &= bm - 1
    e = np.arange(1 << P.k, dtype=np.int64)
    low = e & ((1 << P.m) - 1)
    high = hoff[P.hoff + (e >> P.m)].astype(np.int64)
    return base, base | low | high


def _pairs(G, k):
    npairs = 1 << (k - G.n_fixed)
    f = np.arange(npairs, dtype=np.int64)
    for i in range(G.n_fixed):
        b = int(G.fixed[i])
        f = ((f >> b) << (b + 1)) | (f & ((1 << b) - 1))
    e = f | int(G.amask)
    return e, e ^ (int(G.amask) | int(G.cmask))


def _parity(a):
    a = np.asarray(a, dtype=np.int64)
    return np.array([bin(int(v)).count("1") & 1 for v in a.ravel()]).reshape(a.shape)


def emulate(n, ne, exc, theta, H=None, oracle_mod=None, prec="c128"):
    pl = _plan(n, prec, exc, ne)
    psi = np.zeros(1 << n, dtype=complex)
    psi[(1 << ne) - 1] = 1.0
    for P in pl["passes"]:
        for tile in range(1 << (n - P.k)):
            base, g = _tile_indices(n, P, pl["hoff"], tile)
            if (base & int(P.zmask)) != int(P.zval):
                # outside the support: the kernel skips the tile (the first
                # pass writes it as zeros); it must be zero
                assert np.all(psi[g] == 0)
                continue
            t = psi[g].copy()
            for G in pl["gates"][P.g_begin:P.g_begin + P.n_gates]:
                e, e2 = _pairs(G, P.k)
                sb = (bin(base & int(G.smask_g)).count("1") + int(G.sign0)) & 1
                sg = 1 - 2 * (sb ^ _parity(e & int(G.smask_t)))
                c, s = np.cos(theta[G.param]), np.sin(theta[G.param])
                x, y = t[e].copy(), t[e2].copy()
                t[e], t[e2] = c * x - sg * s * y, c * y + sg * s * x
            psi[g] = t
    if H is None:
        return psi, None
    lam = oracle_mod.apply_h(psi, H.x, H.z, H.c)
    grad = np.zeros(len(exc))
    for P in reversed(pl["passes"]):
        for tile in range(1 << (n - P.k)):
            base, g = _tile_indices(n, P, pl["hoff"], tile)
            if (base & int(P.bzmask)) != int(P.bzval):
                # outside the support of the state after this pass: skipped,
                # zero partials; psi is zero there up to rounding
                assert np.max(np.abs(psi[g])) <= 1e-12
                continue
            t, l = psi[g].copy(), lam[g].copy()
            for G in reversed(pl["gates"][P.g_begin:P.g_begin + P.n_gates]):
                e, e2 = _pairs(G, P.k)
                sb = (bin(base & int(G.smask_g)).count("1") + int(G.sign0)) & 1
                sg = 1 - 2 * (sb ^ _parity(e & int(G.smask_t)))
                grad[G.param] += 2.0 * np.sum(sg * (np.real(np.conj(l[e2]) * t[e]) -
                                                    np.real(np.conj(l[e]) * t[e2])))
                c, s = np.cos(theta[G.param]), np.sin(theta[G.param])
                x, y, lx, ly = t[e].copy(), t[e2].copy(), l[e].copy(), l[e2].copy()
                t[e], t[e2] = c * x + sg * s * y, c * y - sg * s * x
                l[e], l[e2] = c * lx + sg * s * ly, c * ly - sg * s * lx
            psi[g], lam[g] = t, l
    return psi, grad


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n", [6, 13, 14])
def test_replayed_plan_matches_oracle(oracle_mod, lib_built, prec, n):
    ne = n // 2
    exc = vi.excitations(n, ne) if n <= 6 else vi.excitations(n, ne, 6, 14, seed=n)
    th = vi.excitation_params(n, len(exc))
    H = vi.hubbard_1d(n // 2, 1.0, 4.0, periodic=True)
    H = vi.PauliSum(n, H.x, H.z, H.c)
    psi, g = emulate(n, ne, exc, th, H, oracle_mod, prec)
    hf = np.zeros(1 << n)
    hf[(1 << ne) - 1] = 1.0
    # the backward sweep undoes the circuit on the tiles it visits (the
    # skipped ones keep the rounding residue of the passes undone before)
    assert np.max(np.abs(psi - hf)) <= 1e-12
    ref = oracle_mod.pc_ansatz_state(n, ne, exc, th)
    psi_f, _ = emulate(n, ne, exc, th, prec=prec)
    assert np.max(np.abs(psi_f - ref)) <= 1e-13
    g_ref, _ = oracle_mod.pc_gradient_adjoint(n, ne, exc, th, H.x, H.z, H.c)
    assert np.max(np.abs(g - g_ref)) <= 1e-12 * max(1.0, np.max(np.abs(g_ref)))


def test_plan_structure(lib_built):
    n = 20
    exc = vi.excitations(n, 10, 12, 40, seed=2)
    for prec, k, m in (("c128", 11, 4), ("c64", 12, 5)):
        pl = _plan(n, prec, exc, 10)
        assert sum(P.n_gates for P in pl["passes"]) == len(exc)
        for P in pl["passes"]:
            assert (P.k, P.m) == (k, m) and 1 <= P.n_gates <= 16
            tile_bits = ((1 << m) - 1) | int(np.bitwise_or.reduce(pl["hoff"][P.hoff:P.hoff + (1 << (k - m))]))
            assert bin(tile_bits).count("1") == k
            assert tile_bits & int(P.bmask) == 0 and (tile_bits | int(P.bmask)) == (1 << n) - 1
            for G in pl["gates"][P.g_begin:P.g_begin + P.n_gates]:
                p, q, r, s = exc[G.param]
                modes = [x for x in (p, q, r, s) if x >= 0]
                assert all((tile_bits >> md) & 1 for md in modes)   # every mode in the tile
        assert [G.param for G in pl["gates"]] == list(range(len(exc)))   # order kept
        # support masks: before the first pass only the Hartree-Fock tile is
        # live; the masks lie in the tile-number bits with values of psi_HF;
        # the modes touched after pass a (its backward mask) are those touched
        # before pass a + 1 (the next forward mask), seen through each pass's
        # own tile-number bits
        hf = (1 << 10) - 1
        P0 = pl["passes"][0]
        assert P0.zmask == P0.bmask and P0.zval == hf & P0.bmask
        for P in pl["passes"]:
            for msk, val in ((P.zmask, P.zval), (P.bzmask, P.bzval)):
                assert msk & ~P.bmask == 0 and val == hf & msk
            assert P.bzmask & ~P.zmask == 0            # the support only grows
        for a, b in zip(pl["passes"], pl["passes"][1:]):
            touched_a = a.bmask & ~a.bzmask
            touched_b = b.bmask & ~b.zmask
            assert touched_a & b.bmask == touched_b & a.bmask
