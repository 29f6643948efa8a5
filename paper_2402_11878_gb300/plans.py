"""Host-only views of the plans libvqe_gb300 builds (include/vqe_inspect.h).

The library's own planners run on the host and their records are copied
out, so tests can check index arithmetic and plan semantics without a GPU.
The ctypes records below mirror the library's internal layouts; their sizes
are checked against ``vqe_inspect_sizeof`` on every call.
"""
from __future__ import annotations

import ctypes

import numpy as np

from .binding import load

K_MAX_OPS = 384
K_MAX_SLOTS = 40
K_MAX_TILE_BITS = 14
OP_ROUND, OP_BF, OP_DIAG, OP_FLUSH = 0, 1, 2, 3


class PassOp(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint8), ("chunk", ctypes.c_uint8), ("mask", ctypes.c_uint8),
                ("slot", ctypes.c_uint8)]


class PassDesc(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("m", ctypes.c_int), ("a", ctypes.c_int), ("R", ctypes.c_int),
                ("n_ops", ctypes.c_int), ("n_slots", ctypes.c_int), ("zmask", ctypes.c_uint32),
                ("slot_layer", ctypes.c_int * K_MAX_SLOTS),
                ("slot_czmask", ctypes.c_uint32 * K_MAX_SLOTS),
                ("slot_gated", ctypes.c_uint32 * K_MAX_SLOTS),
                ("slot_coef_off", ctypes.c_int * K_MAX_SLOTS),
                ("slot_dtab_off", ctypes.c_int * K_MAX_SLOTS),
                ("slot_grad_off", ctypes.c_int * K_MAX_SLOTS),
                ("ops", PassOp * K_MAX_OPS)]


class StageSlot(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("layer", ctypes.c_int), ("coef_off", ctypes.c_int),
                ("dtab_off", ctypes.c_int), ("n_gated", ctypes.c_int),
                ("tile_bit", ctypes.c_uint8 * K_MAX_TILE_BITS),
                ("qubit", ctypes.c_uint8 * K_MAX_TILE_BITS),
                ("before", ctypes.c_uint16 * K_MAX_TILE_BITS)]


class GroupDesc(ctypes.Structure):
    _fields_ = [("x", ctypes.c_uint32), ("h", ctypes.c_int), ("t_begin", ctypes.c_int),
                ("t_mid", ctypes.c_int), ("t_end", ctypes.c_int)]


K_WIN_MAX_RUNS = 16
K_WIN_MAX_TERMS = 2048
K_WIN_MAX_GROUPS = 96


class WinDesc(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("m", ctypes.c_int), ("g_begin", ctypes.c_int),
                ("g_end", ctypes.c_int), ("t_begin", ctypes.c_int), ("t_count", ctypes.c_int),
                ("hoff", ctypes.c_int), ("bmask", ctypes.c_uint32), ("block_off", ctypes.c_int),
                ("with_norm", ctypes.c_int), ("any_runs", ctypes.c_int)]


class WinGroup(ctypes.Structure):
    _fields_ = [("xl", ctypes.c_uint32), ("hl", ctypes.c_int), ("direct", ctypes.c_int),
                ("fmask", ctypes.c_uint32), ("plog", ctypes.c_int), ("npat", ctypes.c_int),
                ("fval", ctypes.c_uint32 * 8), ("smask", ctypes.c_uint32 * 5),
                ("dj", ctypes.c_uint32 * 4),
                ("a_begin", ctypes.c_int),
                ("b_begin", ctypes.c_int), ("b_end", ctypes.c_int),
                ("arun", ctypes.c_uint16 * (K_WIN_MAX_RUNS + 1)),
                ("brun", ctypes.c_uint16 * (K_WIN_MAX_RUNS + 1))]


class WinTerm(ctypes.Structure):
    _fields_ = [("zt", ctypes.c_uint32), ("zout", ctypes.c_uint32), ("c", ctypes.c_double)]


class ExcPass(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("m", ctypes.c_int), ("g_begin", ctypes.c_int),
                ("n_gates", ctypes.c_int), ("hoff", ctypes.c_int), ("bmask", ctypes.c_uint32),
                ("grad_off", ctypes.c_int), ("zmask", ctypes.c_uint32), ("zval", ctypes.c_uint32),
                ("bzmask", ctypes.c_uint32), ("bzval", ctypes.c_uint32)]


class ExcGate(ctypes.Structure):
    _fields_ = [("amask", ctypes.c_uint32), ("cmask", ctypes.c_uint32),
                ("smask_t", ctypes.c_uint32), ("smask_g", ctypes.c_uint32),
                ("sign0", ctypes.c_uint32), ("n_fixed", ctypes.c_int),
                ("fixed", ctypes.c_uint8 * 4), ("param", ctypes.c_int)]


class SweepDesc(ctypes.Structure):
    _fields_ = [("g_begin", ctypes.c_int), ("g_end", ctypes.c_int), ("p_begin", ctypes.c_int),
                ("n_pat", ctypes.c_int), ("t_begin", ctypes.c_int), ("t_count", ctypes.c_int),
                ("order", ctypes.c_int), ("diag", ctypes.c_int), ("fast", ctypes.c_uint32)]


class SGroup(ctypes.Structure):
    _fields_ = [("x", ctypes.c_uint32), ("pat", ctypes.c_int), ("xbits", ctypes.c_uint32),
                ("flags", ctypes.c_uint32)]


def _check_layouts(lib):
    for which, cls in enumerate((PassDesc, StageSlot, GroupDesc, WinDesc, WinGroup, WinTerm,
                                 ExcPass, ExcGate, SweepDesc, SGroup)):
        got = lib.vqe_inspect_sizeof(which)
        if got != ctypes.sizeof(cls):
            raise RuntimeError(f"record layout mismatch for {cls.__name__}: library {got}, "
                               f"binding {ctypes.sizeof(cls)}")


def plan(n_qubits: int, depth: int, precision: str = "c64", options=(0, 0, 0)) -> dict:
    """The tile-pass plan: forward/backward pass records, staging slots, gradient map.

    ``options`` = (tile_bits_max, run_bits, reg_bits), 0 = default."""
    lib = load()
    _check_layouts(lib)
    prec = {"c64": 0, "c128": 1}[precision]
    strides = (ctypes.c_uint64 * 3)()
    counts = (ctypes.c_int * 3)()
    opts = (ctypes.c_int * 3)(*options)
    rc = lib.vqe_inspect_plan(n_qubits, depth, prec, opts, None, None, 0, None, 0, None, 0,
                              strides, counts)
    if rc != 0 and counts[0] == 0:
        raise ValueError("vqe_inspect_plan rejected the arguments")
    npass, nstage, nparams = counts[0], counts[1], counts[2]
    fwd = (PassDesc * npass)()
    bwd = (PassDesc * npass)()
    stage = (StageSlot * nstage)()
    gmap = np.zeros(3 * nparams, dtype=np.int32)
    rc = lib.vqe_inspect_plan(n_qubits, depth, prec, opts, ctypes.addressof(fwd),
                              ctypes.addressof(bwd), npass, ctypes.addressof(stage), nstage,
                              gmap.ctypes.data, nparams, strides, counts)
    if rc != 0:
        raise ValueError("vqe_inspect_plan rejected the arguments")
    return {"fwd": list(fwd), "bwd": list(bwd), "stage": list(stage),
            "grad_map": gmap.reshape(nparams, 3), "coef_stride": strides[0],
            "dtab_stride": strides[1], "grad_stride": strides[2]}


def hamiltonian(n_qubits: int, x, z, c, threshold: float = 0.0) -> dict:
    """Canonical, cut and grouped terms as the library prepares them."""
    lib = load()
    _check_layouts(lib)
    x = np.ascontiguousarray(x, dtype=np.uint64)
    z = np.ascontiguousarray(z, dtype=np.uint64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    counts = (ctypes.c_int * 2)()
    dropped = ctypes.c_double()
    ncanon = ctypes.c_uint64()
    lib.vqe_inspect_hamiltonian(n_qubits, x.ctypes.data, z.ctypes.data, c.ctypes.data, c.size,
                                float(threshold), None, 0, None, None, 0, counts,
                                ctypes.byref(dropped), ctypes.byref(ncanon))
    ng, nt = counts[0], counts[1]
    groups = (GroupDesc * max(ng, 1))()
    tz = np.zeros(max(nt, 1), dtype=np.uint32)
    tc = np.zeros(max(nt, 1), dtype=np.float64)
    rc = lib.vqe_inspect_hamiltonian(n_qubits, x.ctypes.data, z.ctypes.data, c.ctypes.data, c.size,
                                     float(threshold), ctypes.addressof(groups), ng, tz.ctypes.data,
                                     tc.ctypes.data, nt, counts, ctypes.byref(dropped),
                                     ctypes.byref(ncanon))
    if rc != 0:
        raise ValueError("vqe_inspect_hamiltonian rejected the input")
    return {"groups": list(groups)[:ng], "tz": tz[:nt], "tc": tc[:nt],
            "sum_abs_dropped": dropped.value, "n_canonical": ncanon.value}


def windows(n_qubits: int, precision: str, x, z, c, threshold: float = 0.0,
            diag_terms: bool = True) -> dict:
    """Windows of the windowed expectation and apply-H kernels, as the library plans them:
    window records, window groups, window terms, high-part offsets, wide groups."""
    lib = load()
    _check_layouts(lib)
    prec = {"c64": 0, "c128": 1}[precision]
    x = np.ascontiguousarray(x, dtype=np.uint64)
    z = np.ascontiguousarray(z, dtype=np.uint64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    counts = (ctypes.c_int * 5)()
    lib.vqe_inspect_windows(n_qubits, prec, x.ctypes.data, z.ctypes.data, c.ctypes.data, c.size,
                            float(threshold), int(diag_terms), None, 0, None, 0,
                            None, 0, None, 0, None, 0, counts)
    nw, ng, nt, nh, nd = (counts[i] for i in range(5))
    wins = (WinDesc * max(nw, 1))()
    wg = (WinGroup * max(ng, 1))()
    wt = (WinTerm * max(nt, 1))()
    hoff = np.zeros(max(nh, 1), dtype=np.uint32)
    wide = (GroupDesc * max(nd, 1))()
    rc = lib.vqe_inspect_windows(n_qubits, prec, x.ctypes.data, z.ctypes.data, c.ctypes.data,
                                 c.size, float(threshold), int(diag_terms),
                                 ctypes.addressof(wins),
                                 nw, ctypes.addressof(wg), ng, ctypes.addressof(wt), nt,
                                 hoff.ctypes.data, nh, ctypes.addressof(wide), nd, counts)
    if rc != 0:
        raise ValueError("vqe_inspect_windows rejected the input")
    return {"windows": list(wins)[:nw], "wgroups": list(wg)[:ng], "wterms": list(wt)[:nt],
            "hoff": hoff[:nh], "wide": list(wide)[:nd]}


def sweeps(n_qubits: int, precision: str, x, z, c, threshold: float = 0.0,
           diag_terms: bool = True) -> dict:
    """Sweeps of the sweep form of lambda = H psi, as the library plans them:
    sweep records, sweep groups, pattern entries (first term | count << 16),
    merged terms (z, A and B coefficients) and the bit-order tables (1024 per
    sweep)."""
    lib = load()
    _check_layouts(lib)
    prec = {"c64": 0, "c128": 1}[precision]
    x = np.ascontiguousarray(x, dtype=np.uint64)
    z = np.ascontiguousarray(z, dtype=np.uint64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    counts = (ctypes.c_int * 4)()
    lib.vqe_inspect_sweeps(n_qubits, prec, x.ctypes.data, z.ctypes.data, c.ctypes.data, c.size,
                           float(threshold), int(diag_terms), None, 0, None, 0, None, 0, None,
                           None, None, 0, None, 0, counts)
    ns, ng, npat, nt = (counts[i] for i in range(4))
    sw = (SweepDesc * max(ns, 1))()
    sg = (SGroup * max(ng, 1))()
    pat = np.zeros(max(npat, 1), dtype=np.uint32)
    tz = np.zeros(max(nt, 1), dtype=np.uint32)
    ta = np.zeros(max(nt, 1), dtype=np.float64)
    tb = np.zeros(max(nt, 1), dtype=np.float64)
    order = np.zeros(max(1024 * ns, 1), dtype=np.uint32)
    rc = lib.vqe_inspect_sweeps(n_qubits, prec, x.ctypes.data, z.ctypes.data, c.ctypes.data,
                                c.size, float(threshold), int(diag_terms), ctypes.addressof(sw),
                                ns, ctypes.addressof(sg), ng, pat.ctypes.data, npat,
                                tz.ctypes.data, ta.ctypes.data, tb.ctypes.data, nt,
                                order.ctypes.data, 1024 * ns, counts)
    if rc != 0:
        raise ValueError("vqe_inspect_sweeps rejected the input")
    return {"sweeps": list(sw)[:ns], "groups": list(sg)[:ng], "pat": pat[:npat], "tz": tz[:nt],
            "ta": ta[:nt], "tb": tb[:nt], "order": order[:1024 * ns]}


def pc_plan(n_qubits: int, precision: str, excitations, n_elec: int = 0) -> dict:
    """Pass plan of the particle-conserving ansatz as the library builds it
    (n_elec: electrons of psi_HF, for the support masks)."""
    lib = load()
    _check_layouts(lib)
    prec = {"c64": 0, "c128": 1}[precision]
    exc = np.ascontiguousarray(excitations, dtype=np.int32).reshape(-1, 4)
    counts = (ctypes.c_int * 3)()
    rc = lib.vqe_inspect_pc_plan(n_qubits, n_elec, prec, exc.shape[0], exc.ctypes.data, None, 0,
                                 None, 0, None, 0, counts)
    if counts[0] == 0:
        raise ValueError("vqe_inspect_pc_plan rejected the arguments")
    npass, ng, nh = counts[0], counts[1], counts[2]
    passes = (ExcPass * npass)()
    gates = (ExcGate * ng)()
    hoff = np.zeros(nh, dtype=np.uint32)
    rc = lib.vqe_inspect_pc_plan(n_qubits, n_elec, prec, exc.shape[0], exc.ctypes.data,
                                 ctypes.addressof(passes), npass, ctypes.addressof(gates), ng,
                                 hoff.ctypes.data, nh, counts)
    if rc != 0:
        raise ValueError("vqe_inspect_pc_plan rejected the arguments")
    return {"passes": list(passes), "gates": list(gates), "hoff": hoff}
