"""Host logic of the library, checked on the CPU (no GPU): the tile-pass
planner (index arithmetic emulated exactly as the kernels execute it),
Hamiltonian canonicalisation, cutoff and X-mask grouping."""
import numpy as np
import pytest

import vqe_inputs as vi
from kernel_emulator import Emu, energy_terms, apply_h_terms
from paper_2402_11878_gb300 import plans as P

SMEM_MAX = 227 * 1024


def pass_smem(d, backward, elem):
    threads = 1 << (d.k - d.R)
    warps = (threads + 31) // 32
    coef = 24 if elem == 16 else 12
    buf = (1 << d.k) + ((1 << d.k) >> (3 if elem == 16 else 4))   # padded tile buffer
    return (buf * elem * (2 if backward else 1) + (warps * d.k * 16 if backward else 0)
            + d.n_slots * d.k * coef + 2528)


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("n", list(range(1, 33)))
def test_plan_invariants(n, prec):
    D = 3
    pl = P.plan(n, D, prec)
    elem = 16 if prec == "c128" else 8
    covered = {}
    cz_seen = {}
    gid = 0
    for d, b in zip(pl["fwd"], pl["bwd"]):
        assert 1 <= d.R <= d.k <= 14 and d.k <= n
        assert (1 << (d.k - d.R)) <= 512
        assert pass_smem(b, True, elem) <= SMEM_MAX
        assert d.n_ops <= P.K_MAX_OPS and b.n_ops <= P.K_MAX_OPS
        assert d.n_slots == b.n_slots <= P.K_MAX_SLOTS
        for s in range(d.n_slots):
            l = d.slot_layer[s]
            for j in range(d.k):
                if (d.slot_gated[s] >> j) & 1:
                    q = j if j < d.m else d.a + (j - d.m)
                    assert (l, q) not in covered, "qubit gated twice in a layer"
                    covered[(l, q)] = gid
            for q in range(32):
                if (d.slot_czmask[s] >> q) & 1:
                    assert (l, q) not in cz_seen
                    cz_seen[(l, q)] = gid
            gid += 1
    assert len(covered) == n * D
    assert len(cz_seen) == (n - 1) * D
    # every CZ comes after both of its RY gates and before the next layer's
    for (l, q), g in cz_seen.items():
        assert g >= covered[(l, q)] and g >= covered[(l, q + 1)]
        if l + 1 < D:
            assert g < covered[(l + 1, q)] and g < covered[(l + 1, q + 1)]


CASES = [(1, 2, "c64"), (2, 3, "c128"), (3, 2, "c64"), (5, 2, "c128"), (8, 4, "c128"),
         (8, 4, "c64"), (12, 3, "c128"), (13, 2, "c64"), (14, 2, "c64"), (14, 2, "c128"),
         (16, 2, "c128"), (17, 2, "c64"), (13, 45, "c64")]


@pytest.mark.parametrize("n,D,prec", CASES)
def test_emulated_kernels_match_oracle(oracle_mod, n, D, prec):
    """The plan, executed with the kernels' index arithmetic, reproduces the oracle."""
    H = vi.random_pauli_sum(n, 25, seed=n + D, duplicates=2)
    p = vi.ansatz_params(1000 + n, n, D)
    emu = Emu(n, D, prec)
    psi = emu.forward(p)
    ref = oracle_mod.ansatz_state(n, D, p)
    assert np.max(np.abs(psi - ref)) < 1e-12
    ham = P.hamiltonian(n, H.x, H.z, H.c)
    e, nn = energy_terms(ham, n, psi)
    e_ref, _, n_ref = oracle_mod.expectation(ref, H.x, H.z, H.c)
    assert abs(e - e_ref) < 1e-12 * H.sum_abs() and abs(nn - n_ref) < 1e-12
    lam = apply_h_terms(ham, n, psi)
    assert np.max(np.abs(lam - oracle_mod.apply_h(ref, H.x, H.z, H.c))) < 1e-12 * H.sum_abs()
    if n <= 14:
        g, eg = emu.gradient(p, lambda s: apply_h_terms(ham, n, s))
        g_ref, _ = oracle_mod.gradient_adjoint(n, D, p, H.x, H.z, H.c)
        assert np.max(np.abs(g - g_ref)) < 1e-11 * max(1.0, np.max(np.abs(g_ref)))


@pytest.mark.parametrize("n,D,prec", [(20, 10, "c128"), (24, 4, "c64"), (28, 4, "c64"), (32, 8, "c128")])
def test_forward_zero_tile_masks(n, D, prec):
    """Forward passes start from |0...0>: the first pass's zmask holds every
    qubit (only the tile at base 0 is nonzero), each later pass's mask drops
    the qubits the earlier passes rotated, once every qubit has been rotated
    the mask is empty; backward pass p carries the forward mask of pass p + 1."""
    pl = P.plan(n, D, prec)
    nmask = (1 << n) - 1
    rotated = 0
    for i, d in enumerate(pl["fwd"]):
        assert d.zmask == nmask & ~rotated
        for j in range(d.k):
            if (d.slot_gated[0] >> j) & 1:
                rotated |= 1 << (j if j < d.m else d.a + j - d.m)
    assert i == 0 or pl["fwd"][0].zmask == nmask
    assert rotated == nmask and pl["fwd"][-1].zmask == 0
    fw = pl["fwd"]
    assert [d.zmask for d in pl["bwd"]] == [fw[i + 1].zmask for i in range(len(fw) - 1)] + [0]


def test_emulated_full_size_20q_plan(oracle_mod):
    """The 20-qubit FP64 plan of the benchmark workload, checked end to end."""
    n, D = 20, 10
    H = vi.hubbard_1d(10, 1.0, 4.0, periodic=True)
    p = vi.ansatz_params(4, n, D)
    psi = Emu(n, D, "c128").forward(p)
    ref = oracle_mod.ansatz_state(n, D, p)
    assert np.max(np.abs(psi - ref)) < 1e-12
    ham = P.hamiltonian(n, H.x, H.z, H.c)
    e, _ = energy_terms(ham, n, psi)
    e_ref, _, _ = oracle_mod.expectation(ref, H.x, H.z, H.c)
    assert abs(e - e_ref) < 1e-11 * H.sum_abs()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_canonicalise_and_slim_match_oracle(oracle_mod, seed):
    n = 10
    H = vi.random_pauli_sum(n, 400, seed=seed, duplicates=60)
    H.c = H.c * np.exp(-np.linspace(0, 14, len(H.c)))
    # add exact cancellations: they must disappear in the canonical form
    x = np.concatenate([H.x, H.x[:5], H.x[:5]])
    z = np.concatenate([H.z, H.z[:5], H.z[:5]])
    c = np.concatenate([H.c, np.full(5, 2.0), np.full(5, -2.0)])
    for th in [0.0, 1e-6, 1e-4, 1e-3, 0.05, 100.0]:
        ham = P.hamiltonian(n, x, z, c, threshold=th)
        xs, zs, cs, dref = oracle_mod.slim(x, z, c, th)
        assert len(ham["tz"]) == len(cs)
        assert abs(ham["sum_abs_dropped"] - dref) <= 1e-12 * max(1.0, dref)
        # same kept strings (bit exact)
        kept = set()
        for G in ham["groups"]:
            for t in range(G.t_begin, G.t_end):
                kept.add((G.x, int(ham["tz"][t])))
        assert kept == set(zip(xs.astype(int).tolist(), zs.astype(int).tolist()))


def test_grouping_signs_match_pauli_phase(oracle_mod):
    """Folding (-i)^kappa into class A/B signs reproduces every single Pauli string."""
    n = 5
    rng = np.random.default_rng(0)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    for x in range(1 << n):
        for z in range(0, 1 << n, 3):
            ham = P.hamiltonian(n, [x], [z], [1.0])
            e, _ = energy_terms(ham, n, psi)
            e_ref, _, _ = oracle_mod.expectation(psi, [x], [z], [1.0])
            assert abs(e - e_ref) < 1e-12


def test_inspect_rejects_bad_input():
    with pytest.raises(ValueError):
        P.hamiltonian(4, [1 << 4], [0], [1.0])
    with pytest.raises(ValueError):
        P.hamiltonian(4, [1], [0], [float("inf")])


OPTION_CASES = [((13, 4, 5), "c64"), ((12, 3, 5), "c128"), ((10, 1, 3), "c128"), ((11, 2, 3), "c128"), ((12, 2, 4), "c128"), ((12, 3, 4), "c128"),
                ((13, 2, 4), "c64"), ((12, 2, 4), "c64"), ((11, 4, 3), "c64"),
                ((9, 1, 2), "c64")]


@pytest.mark.parametrize("opts,prec", OPTION_CASES)
@pytest.mark.parametrize("n", [7, 16, 21])
def test_plan_options_emulated(oracle_mod, opts, prec, n):
    """Alternative tile plans (as the autotuner may pick) stay exact."""
    D = 2
    pl = P.plan(n, D, prec, opts)
    elem = 16 if prec == "c128" else 8
    for d in pl["bwd"]:
        assert (1 << (d.k - d.R)) <= 512
        assert pass_smem(d, opts[2] <= 4, elem) <= SMEM_MAX
    if n > 16:
        return
    emu = Emu(n, D, prec)
    emu.plan = pl
    p = vi.ansatz_params(77 + n, n, D)
    psi = emu.forward(p)
    assert np.max(np.abs(psi - oracle_mod.ansatz_state(n, D, p))) < 1e-12
    if opts[2] == 5:
        return      # 32 amplitudes per thread: forward (energy) plans only
    H = vi.random_pauli_sum(n, 10, seed=n)
    ham = P.hamiltonian(n, H.x, H.z, H.c)
    g, _ = emu.gradient(p, lambda s: apply_h_terms(ham, n, s))
    g_ref, _ = oracle_mod.gradient_adjoint(n, D, p, H.x, H.z, H.c)
    assert np.max(np.abs(g - g_ref)) < 1e-11 * max(1.0, np.max(np.abs(g_ref)))


def test_plan_options_rejected():
    with pytest.raises(ValueError):
        P.plan(20, 2, "c128", (14, 3, 3))   # 2^11 threads
    with pytest.raises(ValueError):
        P.plan(20, 2, "c128", (12, 12, 3))  # run bits >= tile bits


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("case", ["hubbard", "random", "molecular"])
def test_energy_windows_emulated(oracle_mod, prec, case):
    """The windowed expectation plan covers every group exactly once and reproduces the oracle."""
    from kernel_emulator import energy_windows
    if case == "hubbard":
        H = vi.hubbard_1d(8, 1.0, 3.0, periodic=True)
    elif case == "random":
        H = vi.random_pauli_sum(16, 60, seed=21, duplicates=4)
    else:
        H = vi.synthetic_molecular(8, seed=5)
    n = H.n
    p = vi.ansatz_params(31, n, 1)
    psi = oracle_mod.ansatz_state(n, 1, p)
    ham = P.hamiltonian(n, H.x, H.z, H.c)
    e_ref, _, n_ref = oracle_mod.expectation(psi, H.x, H.z, H.c)
    # the diagonal of H from the x = 0 group, as the library precomputes it
    i = np.arange(1 << n, dtype=np.int64)
    hdiag = np.zeros(1 << n)
    for G in ham["groups"]:
        if G.x == 0:
            for t in range(G.t_begin, G.t_mid):
                hdiag += ham["tc"][t] * (1 - 2 * (np.vectorize(lambda v: bin(v).count("1"))(i & int(ham["tz"][t])) & 1))
    for diag_terms in (True, False):
        win = P.windows(n, prec, H.x, H.z, H.c, diag_terms=diag_terms)
        assert win["windows"], "expected windows above the tile size"
        # pair groups are split into virtual groups (one per pattern of the
        # X bits below the top one, vanishing patterns dropped): at most
        # 2^3 per group, never more terms than the group had
        assert len(win["wgroups"]) + len(win["wide"]) <= 8 * len(ham["groups"])
        assert len(win["wterms"]) <= len(ham["tz"]) * 8
        e, nn = energy_windows(ham, win, n, psi, hdiag=None if diag_terms else hdiag)
        assert abs(e - e_ref) < 1e-11 * H.sum_abs() and abs(nn - n_ref) < 1e-12


def _tile_map_ok(n, k, m, a):
    """Tile bits [0, m) and [a, a + k - m) (global positions), the other n - k
    bits from the tile number: the map (tile, e) -> global index must be a
    bijection onto [0, 2^n) (checked structurally, as the kernels compute it)."""
    assert 0 <= m <= k <= n
    assert a >= m and a + (k - m) <= n
    if k == m:
        assert a == m   # the low tile: base bits are [k, n)
    mid = a - m
    tiles = 1 << (n - k)
    # the largest tile number maps to the largest base; with every tile bit set
    # the global index is 2^n - 1, never beyond
    t = tiles - 1
    base = ((t & ((1 << mid) - 1)) << m) | ((t >> mid) << (a + (k - m)))
    e = (1 << k) - 1
    g = base | (e & ((1 << m) - 1)) | ((e >> m) << a)
    assert g == (1 << n) - 1
    # tile and in-tile bits are disjoint
    tile_bits = ((1 << m) - 1) | (((1 << (k - m)) - 1) << a)
    assert base & tile_bits == 0


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("n,D", [(24, 12), (26, 4), (28, 4), (32, 8)])
def test_full_size_index_ranges(n, D, prec):
    """At the full sizes the GPU runs (up to 32 qubits), every pass's tile map
    stays inside [0, 2^n) and every table offset fits the 31-bit fields."""
    pl = P.plan(n, D, prec)
    for d in pl["fwd"] + pl["bwd"]:
        _tile_map_ok(n, d.k, d.m, d.a)
        for s in range(d.n_slots):
            assert 0 <= d.slot_grad_off[s] < 2 ** 31
            assert 0 <= d.slot_dtab_off[s] < 2 ** 31
            assert (d.slot_czmask[s] >> (n - 1)) == 0
    tiles_max = max(1 << (n - d.k) for d in pl["fwd"])
    assert pl["grad_stride"] < 2 ** 31
    assert tiles_max <= 2 ** 31 - 1   # grid.x
    H = vi.hubbard_2d_snake(4, 4, 1.0, 4.0) if n == 32 else vi.hubbard_1d(n // 2, 1.0, 4.0, periodic=True)
    w = P.windows(n, prec, H.x, H.z, H.c)
    for W in w["windows"]:
        assert bin(W.bmask).count("1") == n - W.k and W.bmask < (1 << n)
        hoff = w["hoff"][W.hoff:W.hoff + (1 << (W.k - W.m))]
        hbits = int(np.bitwise_or.reduce(hoff)) if hoff.size else 0
        # tile bits: the low run, the offset table's bits and the tile-number bits partition [0, n)
        assert hbits & W.bmask == 0 and hbits & ((1 << W.m) - 1) == 0
        assert (hbits | W.bmask | ((1 << W.m) - 1)) == (1 << n) - 1
        assert (1 << (n - W.k)) <= 2 ** 31 - 1
        assert W.t_count <= P.K_WIN_MAX_TERMS


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("n", [11, 20, 24, 32])
def test_padded_layout_conflict_free_for_default_plans(n, prec):
    """Every register-round access of the default plans hits distinct bank
    groups within a shared-memory wavefront: 16 lanes of 8-byte elements, or
    8 lanes of 16-byte elements, must fall on distinct slots modulo 16 / 8."""
    from kernel_emulator import elem_of, pad
    pl = P.plan(n, 2, prec)
    lanes_per_wave = 8 if prec == "c128" else 16
    for d in pl["fwd"] + pl["bwd"]:
        R = d.R
        threads = 1 << (d.k - R)
        chunks = {op.chunk for op in d.ops[:d.n_ops] if op.kind == P.OP_ROUND}
        for p in chunks:
            for w0 in range(0, threads, 32):
                lanes = np.arange(w0, min(w0 + 32, threads))
                for r in range(1 << R):
                    slots = pad(elem_of(lanes, r, p, R), prec)
                    for h in range(0, lanes.size, lanes_per_wave):
                        part = slots[h:h + lanes_per_wave] % lanes_per_wave
                        assert np.unique(part).size == part.size, (d.k, R, p, r)


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("case", ["hubbard", "molecular"])
def test_apply_h_windows_emulated(oracle_mod, prec, case):
    """The windowed apply-H over the expectation's windows (pair groups, split
    by pattern where the plan splits them) reproduces the oracle's
    lambda = H psi and Re<psi|lambda>, with and without the precomputed
    diagonal."""
    from kernel_emulator import apply_h_windows
    H = vi.hubbard_1d(8, 1.0, 3.0, periodic=True) if case == "hubbard" else vi.synthetic_molecular(8, seed=5)
    n = H.n
    psi = oracle_mod.ansatz_state(n, 1, vi.ansatz_params(33, n, 1))
    lam_ref = oracle_mod.apply_h(psi, H.x, H.z, H.c)
    ham = P.hamiltonian(n, H.x, H.z, H.c)
    i = np.arange(1 << n, dtype=np.int64)
    hdiag = np.zeros(1 << n)
    for G in ham["groups"]:
        if G.x == 0:
            for t in range(G.t_begin, G.t_mid):
                hdiag += ham["tc"][t] * (1 - 2 * (np.vectorize(lambda v: bin(v).count("1"))(i & int(ham["tz"][t])) & 1))
    for diag_terms in (True, False):
        win = P.windows(n, prec, H.x, H.z, H.c, diag_terms=diag_terms)
        assert not win["wide"]
        lam, e, nn = apply_h_windows(win, n, psi, hdiag=None if diag_terms else hdiag)
        assert np.max(np.abs(lam - lam_ref)) < 1e-12 * H.sum_abs()
        assert abs(e - float(np.real(np.vdot(psi, lam_ref)))) < 1e-11 * H.sum_abs()
        assert abs(nn - float(np.vdot(psi, psi).real)) < 1e-12


def _smem_wavefronts(elem_index, elem_bytes, pad_shift):
    """Shared-memory wavefronts of one warp reading 32 elements: the largest
    number of distinct 128-byte rows that hit one 4-byte bank."""
    slot = elem_index + (elem_index >> pad_shift) if pad_shift else elem_index
    words = (slot[:, None] * elem_bytes + 4 * np.arange(elem_bytes // 4)[None, :]).ravel()
    bank, row = (words // 4) % 32, words // 128
    return max(len(set(row[bank == b].tolist())) for b in range(32))


@pytest.mark.parametrize("case", ["hubbard20_c128", "molecular24_c64"])
def test_window_pair_reads_spread_over_banks(case):
    """The window kernels' padded tile layout (one pad element per 128-byte
    row) keeps a warp's pair reads near the minimum number of shared-memory
    wavefronts (4 for 16-byte, 2 for 8-byte elements), where the unpadded
    layout reaches 16-32 for groups that fix low tile bits."""
    from kernel_emulator import _spread
    if case == "hubbard20_c128":
        H, prec, esz, shift, worst = vi.hubbard_1d(10, 1.0, 4.0, periodic=True), "c128", 16, 3, 4
    else:
        H, prec, esz, shift, worst = vi.synthetic_molecular(12, 2024), "c64", 8, 4, 8
    win = P.windows(H.n, prec, H.x, H.z, H.c, diag_terms=False)
    padded, plain = [], []
    for W in win["windows"][:40]:
        for G in win["wgroups"][W.g_begin:W.g_end]:
            if G.xl == 0:
                continue
            fm, plog, npat = int(G.fmask), int(G.plog), int(G.npat)
            for warp in (0, 5):
                p = np.arange(32, dtype=np.int64) + 32 * warp
                u = p >> plog
                if u.max() >= npat:
                    continue
                fv = np.array([int(G.fval[x]) for x in u], dtype=np.int64)
                i0 = _spread(p & ((1 << plog) - 1), fm) | fv
                for idx in (i0, i0 ^ int(G.xl)):
                    padded.append(_smem_wavefronts(idx, esz, shift))
                    plain.append(_smem_wavefronts(idx, esz, 0))
    assert padded and max(padded) <= worst
    assert np.mean(padded) <= np.mean(plain)


def test_window_cover_of_the_molecular_hamiltonian():
    """The greedy cover in decreasing X-mask order: every group of the 24-qubit
    synthetic molecular Hamiltonian lands in a window (none swept globally),
    within the per-window caps, in at most 110 windows (C64) / 126 (C128);
    ordering by the number of high bits needed 246."""
    H = vi.synthetic_molecular(12, 2024)
    for prec, most in (("c64", 110), ("c128", 126)):
        win = P.windows(H.n, prec, H.x, H.z, H.c, diag_terms=False)
        assert not win["wide"]
        assert len(win["windows"]) <= most
        for W in win["windows"]:
            assert W.g_end - W.g_begin <= P.K_WIN_MAX_GROUPS and W.t_count <= P.K_WIN_MAX_TERMS


def _popc_parity(v):
    v = np.asarray(v, dtype=np.uint64)
    p = np.zeros(v.shape, dtype=np.int64)
    for b in range(64):
        p ^= ((v >> np.uint64(b)) & np.uint64(1)).astype(np.int64)
    return p


def emulate_sweeps(n, prec, H, psi, diag_terms=True):
    """NumPy replay of the sweep form of lambda = H psi from the library's
    plan (vqe_inspect_sweeps): per sweep and group, the pattern of each state
    at the group's X bits selects its merged terms, whose sign sums multiply
    the gathered partner; the first sweep adds the diagonal."""
    sp = P.sweeps(n, prec, H.x, H.z, H.c, diag_terms=diag_terms)
    a = np.arange(1 << n, dtype=np.uint64)
    lam = np.zeros(1 << n, dtype=complex)
    for S in sp["sweeps"]:
        # the bit order maps the counter one to one onto the states
        tab = sp["order"][1024 * S.order:1024 * (S.order + 1)].astype(np.uint64)
        s = a
        img = (tab[(s & np.uint64(255)).astype(np.int64)] |
               tab[256 + ((s >> np.uint64(8)) & np.uint64(255)).astype(np.int64)] |
               tab[512 + ((s >> np.uint64(16)) & np.uint64(255)).astype(np.int64)] |
               tab[768 + ((s >> np.uint64(24)) & np.uint64(255)).astype(np.int64)])
        assert np.array_equal(np.sort(img), a)
        if S.diag and not diag_terms:
            lam += diag_of(n, H) * psi
        for G in sp["groups"][S.g_begin:S.g_end]:
            nxb = G.flags & 255
            if (G.flags >> 10) & 1:
                # parity form: one term where popc(i & x) has parity p
                pk = (G.flags >> 11) & 1
                t = S.t_begin + G.pat
                kept = _popc_parity(a & np.uint64(G.x)) == pk
                sg = 1 - 2 * _popc_parity(a & np.uint64(sp["tz"][t]))
                f = np.where(kept, (sp["ta"][t] - 1j * sp["tb"][t]) * sg, 0)
                lam += psi[(a ^ np.uint64(G.x)).astype(np.int64)] * f
                continue
            pv = np.zeros(1 << n, dtype=np.int64)
            for k in range(nxb):
                pv |= ((a >> np.uint64((G.xbits >> (5 * k)) & 31)) & np.uint64(1)).astype(np.int64) << k
            multi = (G.flags >> 9) & 1
            fa = np.zeros(1 << n)
            fb = np.zeros(1 << n)
            for u in range(1 << nxb):
                sel = pv == u
                if multi:       # pattern entries: first term | count << 16
                    e = int(sp["pat"][S.p_begin + G.pat + u])
                    r0, cnt = e & 0xFFFF, e >> 16
                else:           # one term slot per pattern (zero when empty)
                    r0, cnt = G.pat + u, 1
                assert ((G.flags >> 8) & 1) or all(sp["tb"][S.t_begin + r] == 0 for r in range(r0, r0 + cnt))
                for r in range(r0, r0 + cnt):
                    t = S.t_begin + r
                    sg = 1 - 2 * _popc_parity(a[sel] & np.uint64(sp["tz"][t]))
                    fa[sel] += sp["ta"][t] * sg
                    fb[sel] += sp["tb"][t] * sg
            lam += psi[(a ^ np.uint64(G.x)).astype(np.int64)] * (fa - 1j * fb)
    return lam, sp


def diag_of(n, H):
    a = np.arange(1 << n, dtype=np.uint64)
    d = np.zeros(1 << n)
    for x, z, c in zip(H.x, H.z, H.c):
        if int(x) == 0:
            d += np.real(c) * (1 - 2 * _popc_parity(a & np.uint64(z)))
    return d


SWEEP_CASES = {
    "hubbard1d": lambda: vi.hubbard_1d(6, 1.0, 4.0, periodic=True),
    "lattice": lambda: vi.hubbard_2d_snake(3, 2, 1.0, 4.0),
    "molecular": lambda: vi.synthetic_molecular(6, 2024),
    "random": lambda: vi.random_pauli_sum(11, 40, seed=11),
    "tiny": lambda: vi.random_pauli_sum(2, 6, seed=2),
}


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("case", sorted(SWEEP_CASES))
@pytest.mark.parametrize("diag_terms", [True, False])
def test_apply_h_sweeps_emulated(oracle_mod, prec, case, diag_terms):
    """The sweep form of lambda = H psi (vqe_set_apply_mode 2), replayed from
    the library's plan, equals the oracle's H psi; every group sits in one
    sweep, inside that sweep's fast bits unless it has more X bits than a
    sweep holds."""
    H = SWEEP_CASES[case]()
    n = H.n
    if case in ("hubbard1d", "lattice"):
        # every hopping group takes the parity form
        sp0 = P.sweeps(n, prec, H.x, H.z, H.c, diag_terms=diag_terms)
        assert all((G.flags >> 10) & 1 for G in sp0["groups"] if G.x != 0)
    rng = np.random.default_rng(n)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    lam, sp = emulate_sweeps(n, prec, H, psi, diag_terms)
    ref = oracle_mod.apply_h(psi, H.x, H.z, H.c)
    assert np.max(np.abs(lam - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    hp = P.hamiltonian(n, H.x, H.z, H.c)
    xs = sorted(int(G.x) for G in hp["groups"] if G.x != 0)
    got = sorted(int(G.x) for G in sp["groups"] if G.x != 0)
    assert set(got) <= set(xs) and len(got) == len(set(got))   # a group at most once (vanishing ones dropped)
    mlo = min(n, 4 if prec == "c128" else 5)
    for S in sp["sweeps"]:
        assert S.fast & ((1 << mlo) - 1) == (1 << mlo) - 1
        assert bin(S.fast).count("1") <= max(20, mlo)
        for G in sp["groups"][S.g_begin:S.g_end]:
            high = int(G.x) & ~((1 << mlo) - 1)
            if bin(high).count("1") <= 20 - mlo:
                assert int(G.x) & ~S.fast == 0


def test_sweep_plan_caps(oracle_mod):
    """More groups than one sweep holds split over several sweeps (the replay
    still equals the oracle's H psi); a group with more merged terms than a
    sweep holds makes the sweep form impossible (the library then keeps
    another form)."""
    n = 12
    rng = np.random.default_rng(12)
    # 300 distinct X masks with two terms each: more than the 256 groups a sweep takes
    xs = rng.choice(np.arange(1, 1 << n), size=300, replace=False).astype(np.uint64)
    x = np.concatenate([xs, xs])
    z = rng.integers(0, 1 << n, size=x.size).astype(np.uint64)
    c = rng.standard_normal(x.size)
    H = vi.PauliSum(n, x, z, c)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    lam, sp = emulate_sweeps(n, "c128", H, psi)
    assert len(sp["sweeps"]) >= 2
    assert all(S.g_end - S.g_begin <= 256 for S in sp["sweeps"])
    ref = oracle_mod.apply_h(psi, H.x, H.z, H.c)
    assert np.max(np.abs(lam - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    # one X mask with 4100 distinct Z masks (> 4096 merged terms in one pattern)
    n2 = 14
    zz = rng.choice(np.arange(1 << n2), size=4100, replace=False).astype(np.uint64)
    x2 = np.full(zz.size, (1 << n2) - 1, dtype=np.uint64)
    H2 = vi.PauliSum(n2, x2, zz, rng.standard_normal(zz.size))
    with pytest.raises(ValueError):
        P.sweeps(n2, "c64", H2.x, H2.z, H2.c)
