"""NumPy emulation of the library's tile-pass and energy kernels on the CPU.

Test infrastructure.  It interprets the plan records the library's host
planner produces (``paper_2402_11878_gb300.plans``) with the same index
arithmetic as the CUDA kernels (register chunks, shared-memory swizzle,
tile base addresses, coefficient/table/partial offsets) and checks every
index against its buffer.  Running it against the oracle validates the
planner and the kernels' addressing before any GPU run; it is never a
fallback for the library.
"""
from __future__ import annotations

import numpy as np

from paper_2402_11878_gb300 import plans as P


def popc(a):
    return np.bitwise_count(np.asarray(a, dtype=np.uint64)).astype(np.int64)


def elem_of(t, r, p, R):
    lo = t & ((1 << p) - 1)
    return lo | (r << p) | ((t >> p) << (p + R))


def pad(e, prec):
    """Shared-memory slot of tile element e between register rounds: one pad
    element per 128-byte row (8 complex128 or 16 complex64 elements)."""
    return e + (e >> (3 if prec == "c128" else 4))


def tile_buf_elems(k, prec):
    return (1 << k) + ((1 << k) >> (3 if prec == "c128" else 4))


class Emu:
    def __init__(self, n, depth, prec):
        self.n, self.depth, self.prec = n, depth, prec
        self.plan = P.plan(n, depth, prec)

    # ------------------------------------------------------------ staging
    def stage(self, params):
        """Coefficients and diagonal tables exactly as the staging kernel builds them."""
        n = self.n
        pl = self.plan
        cv = np.zeros(pl["coef_stride"])
        cg = np.zeros(pl["coef_stride"])
        cm = np.full(pl["coef_stride"], -1, dtype=np.int64)
        dt = np.full(pl["dtab_stride"], np.nan, dtype=np.complex128)
        for S in pl["stage"]:
            size = 1 << S.k
            assert S.coef_off + S.k <= pl["coef_stride"]
            assert S.dtab_off + size <= pl["dtab_stride"]
            e = np.arange(size)
            tab = np.ones(size, dtype=np.complex128)
            sigma = 1.0
            scales = {}
            for j in range(S.n_gated):
                q, tb = S.qubit[j], S.tile_bit[j]
                assert 0 <= q < n and 0 <= tb < S.k
                th = params[(S.layer * n + q) * 2]
                ph = params[(S.layer * n + q) * 2 + 1]
                c, s = np.cos(th / 2), np.sin(th / 2)
                if abs(c) >= abs(s):
                    cv[S.coef_off + tb], cm[S.coef_off + tb], sc = s / c, 0, c
                else:
                    cv[S.coef_off + tb], cm[S.coef_off + tb], sc = c / s, 1, s
                sigma *= sc
                scales[tb] = sc
                bit = (e >> tb) & 1
                tab *= np.where(bit == 1, np.exp(0.5j * ph), np.exp(-0.5j * ph))
            dt[S.dtab_off:S.dtab_off + size] = sigma * tab
            for j in range(S.n_gated):
                tb = S.tile_bit[j]
                pb = np.prod([scales[u] for u in scales if (S.before[j] >> u) & 1])
                f = sigma / pb
                cg[S.coef_off + tb] = 1.0 / (f * f)
        self._cg = cg
        return cv, cm, dt

    # ------------------------------------------------------------ passes
    def _run_pass(self, d, psi, lam, cv, cm, dt, init_zero, backward, gpart):
        n, prec = self.n, self.prec
        k, m, a, R = d.k, d.m, d.a, d.R
        assert 1 <= R <= k <= P.K_MAX_TILE_BITS and k <= n
        assert 0 < d.n_ops <= P.K_MAX_OPS and d.n_slots <= P.K_MAX_SLOTS
        hbits = k - m
        mid = a - m
        assert mid >= 0 and a + hbits <= n
        tiles = 1 << (n - k)
        threads = 1 << (k - R)
        assert threads <= 1024
        NR = 1 << R
        tile = np.arange(tiles, dtype=np.int64)[:, None, None]
        t = np.arange(threads, dtype=np.int64)[None, :, None]
        r = np.arange(NR, dtype=np.int64)[None, None, :]
        base = ((tile & ((1 << mid) - 1)) << m) | ((tile >> mid) << (a + hbits))
        lowmask = (1 << m) - 1

        def gaddr(e):
            return base | (e & lowmask) | ((e >> m) << a)

        v = w = None
        chunk = -1
        warps = max(1, threads // 32)
        written = {}
        for oi in range(d.n_ops):
            op = d.ops[oi]
            if op.kind == P.OP_ROUND:
                p = op.chunk
                assert p + R <= k
                e = elem_of(t, r, p, R)
                if chunk < 0:
                    g = gaddr(e)
                    gf = np.broadcast_to(g, (tiles, threads, NR)).ravel()
                    assert gf.min() >= 0 and gf.max() < (1 << n)
                    assert np.unique(gf).size == gf.size == (1 << n), "tiles must partition the state"
                    if init_zero:
                        v = (g == 0).astype(np.complex128) + 0j * g
                    else:
                        v = psi[g]
                    if backward:
                        w = lam[g]
                else:
                    e_old = elem_of(t, r, chunk, R)
                    s_old = pad(np.broadcast_to(e_old, (1, threads, NR)), prec)
                    s_new = pad(np.broadcast_to(e, (1, threads, NR)), prec)
                    nbuf = tile_buf_elems(k, prec)
                    for s_ in (s_old, s_new):
                        flat = s_.ravel()
                        assert flat.min() >= 0 and flat.max() < nbuf
                        assert np.unique(flat).size == (1 << k), "smem slots must be distinct"
                    sm = np.empty((tiles, nbuf), dtype=np.complex128)
                    sm[:, s_old[0].ravel()] = v.reshape(tiles, -1)
                    v = sm[:, s_new[0].ravel()].reshape(tiles, threads, NR)
                    if backward:
                        sl = np.empty((tiles, nbuf), dtype=np.complex128)
                        sl[:, s_old[0].ravel()] = w.reshape(tiles, -1)
                        w = sl[:, s_new[0].ravel()].reshape(tiles, threads, NR)
                chunk = p
            elif op.kind == P.OP_BF:
                s = op.slot
                assert s < d.n_slots and chunk >= 0
                coff = d.slot_coef_off[s]
                for j in range(R):
                    if not (op.mask >> j) & 1:
                        continue
                    bit = chunk + j
                    assert (d.slot_gated[s] >> bit) & 1, "butterfly on a bit the slot does not gate"
                    idx = coff + bit
                    assert 0 <= idx < len(cv) and cm[idx] in (0, 1)
                    c, mode = cv[idx], cm[idx]
                    r0 = [rr for rr in range(NR) if not rr & (1 << j)]
                    r1 = [rr | (1 << j) for rr in r0]
                    if backward:
                        p0, p1, l0, l1 = v[..., r0], v[..., r1], w[..., r0], w[..., r1]
                        gs = self._cg[idx]
                        gt = gs * (np.real(np.conj(l1) * p0) - np.real(np.conj(l0) * p1)).sum(axis=(1, 2))
                        key = (s, bit)
                        assert key not in written, "theta partial written twice"
                        written[key] = gt
                    bufs = [v] + ([w] if backward else [])
                    for u in bufs:
                        x, y = u[..., r0].copy(), u[..., r1].copy()
                        if not backward:
                            if mode == 0:
                                u[..., r0], u[..., r1] = x - c * y, y + c * x
                            else:
                                u[..., r0], u[..., r1] = c * x - y, x + c * y
                        else:
                            if mode == 0:
                                u[..., r0], u[..., r1] = x + c * y, y - c * x
                            else:
                                u[..., r0], u[..., r1] = c * x + y, c * y - x
            elif op.kind == P.OP_DIAG:
                s = op.slot
                e = elem_of(t, r, chunk, R)
                g = gaddr(e)
                if backward:
                    # phi partials for every gated bit, before the diagonal is undone
                    u = np.imag(np.conj(w) * v)
                    eb = np.broadcast_to(e, u.shape)
                    for bit in range(k):
                        if (d.slot_gated[s] >> bit) & 1:
                            sg = np.where((eb >> bit) & 1, -1.0, 1.0)
                            key = ("phi", s, bit)
                            assert key not in written
                            written[key] = (sg * u).sum(axis=(1, 2))
                cz = d.slot_czmask[s]
                sgn = popc(g & (g >> 1) & cz) & 1
                off = d.slot_dtab_off[s]
                assert off + (1 << k) <= len(dt)
                tab = dt[off + np.broadcast_to(e, g.shape)]
                assert not np.isnan(tab).any(), "table entry never staged"
                fac = np.where(sgn == 1, -1.0, 1.0)
                if not backward:
                    v = v * tab * fac
                else:
                    v = v * np.conj(tab) * fac
                    w = w * np.conj(tab) * fac
            elif op.kind == P.OP_FLUSH:
                assert backward
                s = op.slot
                for bit in range(k):
                    if not (d.slot_gated[s] >> bit) & 1:
                        continue
                    gt = written.pop((s, bit))
                    gp = written.pop(("phi", s, bit))
                    base_off = d.slot_grad_off[s] + np.arange(tiles) * (2 * k) + bit * 2
                    assert base_off.max() + 1 < len(gpart)
                    skip = (base[:, 0, 0] & int(d.zmask)) != 0   # tiles the kernel skips: zero partials
                    gpart[base_off] = np.where(skip, 0.0, gt)
                    gpart[base_off + 1] = np.where(skip, 0.0, gp)
            else:
                raise AssertionError(f"unknown op kind {op.kind}")
        assert not written, "gradient partials left unflushed"
        g = gaddr(elem_of(t, r, chunk, R))
        if not backward and init_zero and d.n_slots == 1:
            # the kernels write the first pass's tile at base 0 as a product:
            # one factor per tile bit (tan form (1, v), cot form (v, 1), an
            # ungated bit (1, 0)), then the slot's table entry and CZ sign
            e = elem_of(t, r, chunk, R)
            f = np.ones(np.broadcast_shapes(e.shape, (1, threads, NR)))
            for j in range(k):
                bit = (e >> j) & 1
                if not (d.slot_gated[0] >> j) & 1:
                    f = np.where(bit == 1, 0.0, f)
                    continue
                idx = d.slot_coef_off[0] + j
                c, mode = cv[idx], cm[idx]
                f = f * np.where((bit ^ mode) == 1, c, 1.0)
            off = d.slot_dtab_off[0]
            tab = dt[off + np.broadcast_to(e, g.shape)]
            sgn = np.where(popc(g & (g >> 1) & d.slot_czmask[0]) & 1, -1.0, 1.0)
            prod = tab * f * sgn
            z0 = base[:, 0, 0] == 0
            assert np.abs(prod[z0] - v[z0]).max() <= 1e-13 * max(1.0, np.abs(v).max())
            v = np.where(z0[:, None, None], prod, v)
        # forward from |0...0>: tiles whose base has a bit of zmask are
        # written as zeros without being transformed; they must be zero
        zt = (base[:, 0, 0] & int(d.zmask)) != 0
        if backward:
            # skipped tiles: psi is zero there up to the rounding of the passes
            # already undone; the kernel leaves psi and lambda untouched and
            # writes zero partials
            if zt.any():
                assert np.abs(psi[g][zt]).max() <= 1e-12
            v = np.where(zt[:, None, None], psi[g], v)
            w = np.where(zt[:, None, None], lam[g], w)
        else:
            assert np.all(psi[g[zt]] == 0) if not init_zero else True
            assert np.allclose(v[zt], 0, atol=1e-300), "a tile marked zero is not"
            v = np.where(zt[:, None, None], 0, v)
        psi[g] = v
        if backward:
            lam[g] = w

    def forward(self, params):
        cv, cm, dt = self.stage(params)
        psi = np.zeros(1 << self.n, dtype=np.complex128)
        for i, d in enumerate(self.plan["fwd"]):
            self._run_pass(d, psi, None, cv, cm, dt, i == 0, False, None)
        return psi

    def gradient(self, params, lam_of):
        """Adjoint gradient; ``lam_of(psi)`` returns H psi (from the emulated apply-H)."""
        cv, cm, dt = self.stage(params)
        psi = self.forward(params)
        lam = lam_of(psi)
        energy = np.vdot(psi, lam).real
        gpart = np.full(self.plan["grad_stride"], np.nan)
        for d in reversed(self.plan["bwd"]):
            self._run_pass(d, psi, lam, cv, cm, dt, False, True, gpart)
        gm = self.plan["grad_map"]
        grad = np.empty(len(gm))
        for pidx, (off, cnt, step) in enumerate(gm):
            idx = off + np.arange(cnt) * step
            assert idx.max() < len(gpart)
            vals = gpart[idx]
            assert not np.isnan(vals).any(), "gradient partial never written"
            grad[pidx] = vals.sum()
        return grad, energy


def energy_terms(ham, n, psi):
    """The energy kernel's grouped formula on the CPU: (unnormalised E, norm)."""
    N = 1 << n
    groups, tz, tc = ham["groups"], ham["tz"], ham["tc"]
    i = np.arange(N, dtype=np.int64)
    acc, nrm = 0.0, 0.0
    for G in groups:
        if G.x == 0:
            a = np.abs(psi) ** 2
            f = np.zeros(N)
            for t_ in range(G.t_begin, G.t_mid):
                f += tc[t_] * (1 - 2 * (popc(i & int(tz[t_])) & 1))
            assert G.t_mid == G.t_end, "x = 0 terms are all of class A"
            acc += float((a * f).sum())
            nrm += float(a.sum())
        else:
            h = G.h
            assert (G.x >> h) == 1
            p = np.arange(N // 2, dtype=np.int64)
            i0 = ((p >> h) << (h + 1)) | (p & ((1 << h) - 1))
            i1 = i0 ^ G.x
            assert i1.max() < N and ((i0 >> h) & 1).max() == 0
            g = np.conj(psi[i0]) * psi[i1]
            fa = np.zeros(N // 2)
            fb = np.zeros(N // 2)
            for t_ in range(G.t_begin, G.t_mid):
                fa += tc[t_] * (1 - 2 * (popc(i0 & int(tz[t_])) & 1))
            for t_ in range(G.t_mid, G.t_end):
                fb += tc[t_] * (1 - 2 * (popc(i0 & int(tz[t_])) & 1))
            acc += 2.0 * float((g.real * fa + g.imag * fb).sum())
    return acc, nrm


def apply_h_terms(ham, n, psi):
    """The apply-H kernel's formula on the CPU."""
    N = 1 << n
    i = np.arange(N, dtype=np.int64)
    lam = np.zeros(N, dtype=np.complex128)
    for G in ham["groups"]:
        pj = psi[i ^ G.x]
        fa = np.zeros(N)
        fb = np.zeros(N)
        for t_ in range(G.t_begin, G.t_mid):
            fa += ham["tc"][t_] * (1 - 2 * (popc(i & int(ham["tz"][t_])) & 1))
        for t_ in range(G.t_mid, G.t_end):
            fb += ham["tc"][t_] * (1 - 2 * (popc(i & int(ham["tz"][t_])) & 1))
        lam += pj * (fa - 1j * fb)
    return lam


def _insert0(p, hl):
    return ((p >> hl) << (hl + 1)) | (p & ((1 << hl) - 1))


def _spread(p, mask):
    """p with a zero inserted at every set bit of mask, ascending."""
    p = np.asarray(p, dtype=np.int64)
    for q in range(32):
        if (mask >> q) & 1:
            p = ((p >> q) << (q + 1)) | (p & ((1 << q) - 1))
    return p


def _wht_last(F):
    """f[..., j] = sum_v F[..., v] (-1)^{popc(j & v)} (unnormalised)."""
    F = F.copy()
    N = F.shape[-1]
    h = 1
    while h < N:
        for i in range(N):
            if i & h:
                continue
            x, y = F[..., i].copy(), F[..., i | h].copy()
            F[..., i], F[..., i | h] = x + y, x - y
        h <<= 1
    return F


def energy_windows(ham, win, n, psi, hdiag=None):
    """The windowed expectation kernel on the CPU, step by step as the device
    runs it: base bits from the tile number, elements placed through the
    window's offset table, coefficients with the base sign folded in, per-run
    sign sums at each thread's first pair and a Walsh-Hadamard transform over
    the register patterns; wide groups swept; (E, norm)."""
    tz, tc = ham["tz"], ham["tc"]
    acc, nrm = 0.0, 0.0
    norms = 0
    LT, THR = 9, 512
    tid = np.arange(THR, dtype=np.int64)
    for W in win["windows"]:
        k, m = W.k, W.m
        EPT = 1 << (k - LT)
        PPT = EPT // 2
        tiles = 1 << (n - k)
        assert W.t_count <= P.K_WIN_MAX_TERMS and W.g_end - W.g_begin <= P.K_WIN_MAX_GROUPS
        bpos = [bb for bb in range(32) if (W.bmask >> bb) & 1]
        assert len(bpos) == n - k and max(bpos + [0]) < n
        tn = np.arange(tiles, dtype=np.int64)
        base = np.zeros(tiles, dtype=np.int64)
        for i, bb in enumerate(bpos):
            base |= ((tn >> i) & 1) << bb
        hoff = np.asarray(win["hoff"][W.hoff:W.hoff + (1 << (k - m))], dtype=np.int64)
        assert hoff.size == 1 << (k - m)
        e = np.arange(1 << k, dtype=np.int64)
        g = base[:, None] | (e & ((1 << m) - 1))[None, :] | hoff[e >> m][None, :]
        flat = g.ravel()
        assert flat.min() >= 0 and flat.max() < (1 << n)
        assert np.unique(flat).size == flat.size == (1 << n), "tiles must partition the state"
        sp = psi[g]
        terms = win["wterms"][W.t_begin:W.t_begin + W.t_count]
        zt = np.array([t.zt for t in terms], dtype=np.int64)
        zout = np.array([t.zout for t in terms], dtype=np.int64)
        cc = np.array([t.c for t in terms], dtype=np.float64)
        assert np.all(zout & ~W.bmask == 0) and np.all(zt < (1 << k))
        sc = cc[None, :] * (1 - 2 * (popc(base[:, None] & zout[None, :]) & 1)) if len(terms) else np.zeros((tiles, 0))
        if W.with_norm:
            nrm += float((np.abs(sp) ** 2).sum())
            norms += 1
        for G in win["wgroups"][W.g_begin:W.g_end]:
            NV = PPT if G.xl else EPT
            if G.xl and G.direct:
                NV = int(G.npat)
            assert 0 <= G.a_begin <= G.b_begin <= G.b_end <= W.t_count
            assert G.arun[0] == 0 and G.a_begin + G.arun[NV] == G.b_begin
            assert G.brun[0] == 0 and G.b_begin + G.brun[NV] == G.b_end
            assert all(G.arun[v] <= G.arun[v + 1] for v in range(NV))
            assert all(G.brun[v] <= G.brun[v + 1] for v in range(NV))

            def run_sums(run, begin, e0):
                F = np.zeros((tiles, THR, NV))
                for v in range(NV):
                    for t in range(begin + run[v], begin + run[v + 1]):
                        sgn = 1 - 2 * (popc(e0 & zt[t]) & 1)
                        F[:, :, v] += sc[:, t][:, None] * sgn[None, :]
                return _wht_last(F)

            if G.xl == 0:
                el = tid[:, None] + THR * np.arange(EPT)[None, :]          # (THR, EPT)
                w2 = np.abs(sp[:, el]) ** 2                                 # (tiles, THR, EPT)
                if hdiag is not None:
                    f = hdiag[g[:, el]]
                else:
                    f = run_sums(G.arun, G.a_begin, tid)
                acc += float((w2 * f).sum())
                continue
            xl, hl = int(G.xl), int(G.hl)
            assert xl < (1 << k) and (xl >> hl) == 1
            # pattern u fixes the tile bits fmask of the lower element to
            # fval[u]; pair P = tid + 512 s has u = P >> plog and free index
            # P mod 2^plog, spread around fmask
            fm, plog, npat = int(G.fmask), int(G.plog), int(G.npat)
            assert (fm >> hl) & 1 and fm < (1 << k) and plog == k - popc(fm)
            assert 1 <= npat <= 8 and (npat == 1 or G.direct)
            fval = [int(G.fval[u]) for u in range(npat)]
            assert all(v & ~fm == 0 and not (v >> hl) & 1 for v in fval)
            assert len(set(fval)) == npat
            t0 = tid & (511 if plog >= 9 else (1 << plog) - 1)
            e0 = sum((t0 & int(G.smask[q])) << q for q in range(5))
            dsum = np.zeros(PPT, dtype=np.int64)
            for j in range(PPT):
                for bb in range(4):
                    if (j >> bb) & 1:
                        dsum[j] |= int(G.dj[bb])
            pj = tid[:, None] + THR * np.arange(PPT)[None, :]
            u = pj >> plog
            valid = u < npat
            fv = np.array(fval + [0] * (9 - npat), dtype=np.int64)[np.minimum(u, 8)]
            il = np.where(valid, e0[:, None] | dsum[None, :] | fv, 0)
            # the kernel's composition equals the definition spread(f) | fval[u]
            ref = _spread(pj & ((1 << plog) - 1), fm) | fv
            assert np.array_equal(il[valid], ref[valid])
            assert il.max() < (1 << k) and (il ^ xl).max() < (1 << k)
            x0, x1 = sp[:, il], sp[:, il ^ xl]
            prod = np.where(valid[None, :, :], np.conj(x0) * x1, 0)
            il0 = e0

            def direct_sums(begin, run):
                f = np.zeros((tiles, THR, PPT))
                for uu in range(npat):
                    sel = (u == uu)
                    for t in range(begin + run[uu], begin + run[uu + 1]):
                        sgn = 1 - 2 * (popc(il & zt[t]) & 1)          # (THR, PPT)
                        f += sc[:, t][:, None, None] * (sgn * sel)[None, :, :]
                return f

            if G.direct:
                assert G.a_begin + G.arun[npat] == G.b_begin and G.b_begin + G.brun[npat] == G.b_end
                # the kernel holds a pattern's terms in registers: at most 3 per class
                assert all(G.arun[v + 1] - G.arun[v] <= 3 and G.brun[v + 1] - G.brun[v] <= 3
                           for v in range(npat))
                part = (prod.real * direct_sums(G.a_begin, G.arun)).sum()
                if G.b_end > G.b_begin:
                    part += (prod.imag * direct_sums(G.b_begin, G.brun)).sum()
            else:
                assert npat == 1 and plog == k - 1 and fval == [0]
                part = (prod.real * run_sums(G.arun, G.a_begin, il0)).sum()
                if G.b_end > G.b_begin:
                    part += (prod.imag * run_sums(G.brun, G.b_begin, il0)).sum()
            acc += 2.0 * float(part)
    if win["wide"]:
        sub = {"groups": win["wide"], "tz": tz, "tc": tc}
        e_w, n_w = energy_terms(sub, n, psi)
        acc += e_w
        if any(G.x == 0 for G in win["wide"]):
            nrm += n_w
            norms += 1
    assert norms == 1
    return acc, nrm


def apply_h_windows(win, n, psi, hdiag=None):
    """The windowed apply-H kernel on the CPU: the expectation's windows and
    pair groups; a shared-memory tile of lambda per window (first window from
    zero, later ones from the previous window's lambda); per pair (i0, i1) the
    sign sums FA, FB at i0 (direct per pattern, or runs plus a Walsh-Hadamard
    transform), lambda_i0 += psi_i1 (FA - i FB), lambda_i1 += psi_i0 (FA + i FB);
    the last window's Re<psi|lambda> and norm.  (lambda, E, norm)."""
    LT, THR = 9, 512
    tid = np.arange(THR, dtype=np.int64)
    lam = np.zeros(1 << n, dtype=np.complex128)
    wins = win["windows"]
    assert not win["wide"], "apply-H windows cover every group"
    acc = nrm = 0.0
    for wi, W in enumerate(wins):
        k, m = W.k, W.m
        EPT = 1 << (k - LT)
        PPT = EPT // 2
        tiles = 1 << (n - k)
        bpos = [bb for bb in range(32) if (W.bmask >> bb) & 1]
        tn = np.arange(tiles, dtype=np.int64)
        base = np.zeros(tiles, dtype=np.int64)
        for i, bb in enumerate(bpos):
            base |= ((tn >> i) & 1) << bb
        hoff = np.asarray(win["hoff"][W.hoff:W.hoff + (1 << (k - m))], dtype=np.int64)
        e = np.arange(1 << k, dtype=np.int64)
        g = base[:, None] | (e & ((1 << m) - 1))[None, :] | hoff[e >> m][None, :]
        assert np.unique(g.ravel()).size == (1 << n)
        sp = psi[g]
        terms = win["wterms"][W.t_begin:W.t_begin + W.t_count]
        zt = np.array([t.zt for t in terms], dtype=np.int64)
        zout = np.array([t.zout for t in terms], dtype=np.int64)
        cc = np.array([t.c for t in terms], dtype=np.float64)
        sc = cc[None, :] * (1 - 2 * (popc(base[:, None] & zout[None, :]) & 1)) if len(terms) else np.zeros((tiles, 0))
        sl = np.zeros((tiles, 1 << k), dtype=np.complex128) if wi == 0 else lam[g]
        el = tid[:, None] + THR * np.arange(EPT)[None, :]          # (THR, EPT) element of (thread, j)
        for G in win["wgroups"][W.g_begin:W.g_end]:
            if G.xl == 0:
                if hdiag is not None:
                    f = hdiag[g[:, el]]
                else:
                    F = np.zeros((tiles, THR, EPT))
                    for v in range(EPT):
                        for t in range(G.a_begin + G.arun[v], G.a_begin + G.arun[v + 1]):
                            F[:, :, v] += sc[:, t][:, None] * (1 - 2 * (popc(tid & zt[t]) & 1))[None, :]
                    f = _wht_last(F)
                sl[:, el] += sp[:, el] * f
                continue
            xl, hl = int(G.xl), int(G.hl)
            fm, plog, npat = int(G.fmask), int(G.plog), int(G.npat)
            assert (fm >> hl) & 1 and plog == k - popc(fm) and 1 <= npat <= 8
            fval = [int(G.fval[u]) for u in range(npat)]
            t0 = tid & (511 if plog >= 9 else (1 << plog) - 1)
            e0 = sum((t0 & int(G.smask[q])) << q for q in range(5))
            dsum = np.zeros(PPT, dtype=np.int64)
            for j in range(PPT):
                for bb in range(4):
                    if (j >> bb) & 1:
                        dsum[j] |= int(G.dj[bb])
            pj = tid[:, None] + THR * np.arange(PPT)[None, :]
            u = pj >> plog
            valid = u < npat
            fv = np.array(fval + [0] * (9 - npat), dtype=np.int64)[np.minimum(u, 8)]
            il = e0[:, None] | dsum[None, :] | fv
            assert np.array_equal(il[valid], (_spread(pj & ((1 << plog) - 1), fm) | fv)[valid])
            fa = np.zeros((tiles, THR, PPT))
            fb = np.zeros((tiles, THR, PPT))
            if G.direct:
                for uu in range(npat):
                    sel = (u == uu)
                    for t in range(G.a_begin + G.arun[uu], G.a_begin + G.arun[uu + 1]):
                        fa += sc[:, t][:, None, None] * ((1 - 2 * (popc(il & zt[t]) & 1)) * sel)[None]
                    for t in range(G.b_begin + G.brun[uu], G.b_begin + G.brun[uu + 1]):
                        fb += sc[:, t][:, None, None] * ((1 - 2 * (popc(il & zt[t]) & 1)) * sel)[None]
            else:
                assert npat == 1 and plog == k - 1 and np.all(valid)
                for F, run, begin in ((fa, G.arun, G.a_begin), (fb, G.brun, G.b_begin)):
                    R = np.zeros((tiles, THR, PPT))
                    for v in range(PPT):
                        for t in range(begin + run[v], begin + run[v + 1]):
                            R[:, :, v] += sc[:, t][:, None] * (1 - 2 * (popc(e0 & zt[t]) & 1))[None, :]
                    F += _wht_last(R)
            i0, i1 = il[valid], il[valid] ^ xl
            assert i0.max() < (1 << k) and i1.max() < (1 << k)
            # a group's pairs are disjoint: no element is written twice
            assert np.unique(np.concatenate([i0, i1])).size == 2 * i0.size
            x0, x1 = sp[:, i0], sp[:, i1]
            FA, FB = fa[:, valid], fb[:, valid]
            sl[:, i0] += x1 * (FA - 1j * FB)
            sl[:, i1] += x0 * (FA + 1j * FB)
        lam[g] = sl
        if wi == len(wins) - 1:
            acc = float((sp.real * sl.real + sp.imag * sl.imag).sum())
            nrm = float((np.abs(sp) ** 2).sum())
    return lam, acc, nrm
