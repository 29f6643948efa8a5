"""ctypes binding of libvqe_gb300 (include/vqe.h): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels; this module
converts Python/NumPy/PyTorch arguments into plain pointers and sizes, and
raises on any non-zero status.  There is no CPU fallback: if the library is
missing, importing the engine raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libvqe_gb300.so")

VQE_C64, VQE_C128 = 0, 1
STATUS = {0: "VQE_OK", 1: "VQE_ERR_ARG", 2: "VQE_ERR_STATE", 3: "VQE_ERR_OOM",
          4: "VQE_ERR_CUDA", 5: "VQE_ERR_TIMEOUT", 6: "VQE_ERR_DEVICE"}

# C ABI entry points declared in include/vqe.h and include/vqe_inspect.h
EXPORTED = [
    "vqe_create", "vqe_create_pc", "vqe_destroy", "vqe_workspace_size", "vqe_bind_workspace", "vqe_set_plan_options",
    "vqe_set_apply_mode", "vqe_autotune", "vqe_set_hamiltonian", "vqe_slim", "vqe_apply_ansatz", "vqe_energy", "vqe_get_state",
    "vqe_gradient", "vqe_energy_batch_dev", "vqe_gradient_batch_dev", "vqe_energy_batch",
    "vqe_gradient_batch", "vqe_energy_batch_pergate_dev", "vqe_get_stats", "vqe_last_error",
    "vqe_version", "vqe_profile", "vqe_profile_read", "vqe_inspect_sizeof", "vqe_inspect_plan",
    "vqe_inspect_hamiltonian", "vqe_inspect_windows", "vqe_inspect_sweeps", "vqe_inspect_pc_plan", "vqe_energy_noalloc", "vqe_batch_create", "vqe_batch_destroy",
    "vqe_batch_set_hamiltonian", "vqe_batch_param_offsets", "vqe_batch_run_dev", "vqe_batch_run",
    "vqe_batch_set_tile_bits", "vqe_batch_autotune", "vqe_batch_launch_count",
    "vqe_batch_last_error", "vqe_measure_fma_peak", "vqe_testing_fail_allocations",
]


class VQEError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_uint64), ("n_terms_input", ctypes.c_uint64),
                ("n_terms_canonical", ctypes.c_uint64), ("n_terms_kept", ctypes.c_uint64),
                ("n_groups", ctypes.c_uint64), ("sum_abs_dropped", ctypes.c_double),
                ("threshold", ctypes.c_double), ("ansatz_passes", ctypes.c_uint32),
                ("tile_bits_max", ctypes.c_uint32)]


class Tuning(ctypes.Structure):
    _fields_ = [("tile_bits_max", ctypes.c_int), ("run_bits", ctypes.c_int),
                ("reg_bits", ctypes.c_int), ("apply_form", ctypes.c_int),
                ("candidates", ctypes.c_int), ("ms_default", ctypes.c_double),
                ("ms_best", ctypes.c_double), ("apply_ms_global", ctypes.c_double),
                ("apply_ms_windows", ctypes.c_double), ("apply_ms_sweeps", ctypes.c_double)]


class KernelTimes(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64 * 4), ("ms", ctypes.c_double * 4),
                ("chunks", ctypes.c_uint64 * 4)]


KERNEL_GROUPS = ("forward_passes", "energy", "apply_h", "backward_passes")

_lib = None


def library_path() -> str:
    return LIB_PATH


def load() -> ctypes.CDLL:
    """Load libvqe_gb300.so; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libvqe_gb300.so not built ({LIB_PATH}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, sz, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p
    sig = {
        "vqe_create": [i, i, i, vp, ctypes.POINTER(vp)],
        "vqe_create_pc": [i, i, i, vp, i, vp, ctypes.POINTER(vp)],
        "vqe_destroy": [vp],
        "vqe_workspace_size": [vp, i, i, ctypes.POINTER(sz)],
        "vqe_bind_workspace": [vp, vp, sz],
        "vqe_set_hamiltonian": [vp, vp, vp, vp, sz],
        "vqe_slim": [vp, ctypes.c_double, ctypes.POINTER(sz), ctypes.POINTER(ctypes.c_double)],
        "vqe_apply_ansatz": [vp, dp],
        "vqe_energy": [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
        "vqe_get_state": [vp, vp, sz],
        "vqe_gradient": [vp, dp, dp, ctypes.POINTER(ctypes.c_double)],
        "vqe_energy_batch_dev": [vp, dp, i, dp, dp],
        "vqe_gradient_batch_dev": [vp, dp, i, dp, dp],
        "vqe_energy_batch": [vp, dp, i, dp, dp],
        "vqe_gradient_batch": [vp, dp, i, dp, dp],
        "vqe_energy_batch_pergate_dev": [vp, dp, i, dp, dp],
        "vqe_get_stats": [vp, ctypes.POINTER(Stats)],
        "vqe_last_error": [vp],
        "vqe_version": [],
        "vqe_profile": [vp, i],
        "vqe_profile_read": [vp, ctypes.POINTER(KernelTimes)],
        "vqe_inspect_sizeof": [i],
        "vqe_batch_create": [i, vp, vp, i, vp, ctypes.POINTER(vp)],
        "vqe_batch_destroy": [vp],
        "vqe_batch_set_hamiltonian": [vp, i, vp, vp, vp, sz],
        "vqe_batch_param_offsets": [vp, vp],
        "vqe_batch_run_dev": [vp, dp, dp, dp],
        "vqe_batch_run": [vp, dp, dp, dp],
        "vqe_batch_set_tile_bits": [vp, i],
        "vqe_batch_autotune": [vp, dp, dp, dp, i, ctypes.POINTER(i)],
        "vqe_batch_launch_count": [vp, ctypes.POINTER(ctypes.c_uint64)],
        "vqe_batch_last_error": [vp],
        "vqe_measure_fma_peak": [i, vp, ctypes.POINTER(ctypes.c_double)],
        "vqe_inspect_plan": [i, i, i, vp, vp, vp, i, vp, i, vp, i, vp, vp],
        "vqe_set_plan_options": [vp, i, i, i],
        "vqe_set_apply_mode": [vp, i, ctypes.POINTER(i)],
        "vqe_autotune": [vp, dp, i, i, ctypes.c_double, ctypes.POINTER(Tuning)],
        "vqe_inspect_hamiltonian": [i, vp, vp, vp, sz, ctypes.c_double, vp, i, vp, vp, i, vp,
                                    vp, vp],
        "vqe_inspect_windows": [i, i, vp, vp, vp, sz, ctypes.c_double, i, vp, i, vp, i, vp,
                                i, vp, i, vp, i, vp],
        "vqe_inspect_sweeps": [i, i, vp, vp, vp, sz, ctypes.c_double, i, vp, i, vp, i, vp, i,
                               vp, vp, vp, i, vp, i, vp],
        "vqe_inspect_pc_plan": [i, i, i, i, vp, vp, i, vp, i, vp, i, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.vqe_testing_fail_allocations.argtypes = [i]
    lib.vqe_testing_fail_allocations.restype = None
    lib.vqe_last_error.restype = ctypes.c_char_p
    lib.vqe_batch_last_error.restype = ctypes.c_char_p
    lib.vqe_version.restype = ctypes.c_char_p
    lib.vqe_inspect_sizeof.restype = ctypes.c_size_t
    _lib = lib
    return lib


def _ptr(a) -> int:
    """Raw address of a NumPy array or a torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream or None
    return int(stream) or None


class Engine:
    """One VQE problem size on the current CUDA device (a vqe_handle).

    ``Engine(n, depth, precision)`` uses the hardware-efficient ansatz;
    ``Engine.particle_conserving(n, n_elec, excitations, precision)`` the
    excitation-gate ansatz on the Hartree-Fock state (vqe_create_pc)."""

    def __init__(self, n_qubits: int, depth: int, precision: str = "c64", stream=None,
                 _excitations=None, _n_elec: int = 0):
        lib = load()
        self._lib = lib
        self.n = int(n_qubits)
        self.depth = int(depth)
        self.precision = precision
        prec = {"c64": VQE_C64, "c128": VQE_C128}[precision]
        self.state_dtype = np.complex64 if prec == VQE_C64 else np.complex128
        h = ctypes.c_void_p()
        if _excitations is None:
            self.n_params = 2 * self.n * self.depth
            st = lib.vqe_create(self.n, self.depth, prec, _stream_ptr(stream), ctypes.byref(h))
        else:
            exc = np.ascontiguousarray(_excitations, dtype=np.int32).reshape(-1, 4)
            self.n_params = exc.shape[0]
            self.excitations = exc
            st = lib.vqe_create_pc(self.n, int(_n_elec), exc.shape[0], exc.ctypes.data, prec,
                                   _stream_ptr(stream), ctypes.byref(h))
        if st != 0:
            raise VQEError(st, "vqe_create failed (is a CUDA device available?)")
        self._h = h

    @classmethod
    def particle_conserving(cls, n_qubits: int, n_elec: int, excitations, precision: str = "c64",
                            stream=None) -> "Engine":
        """Excitation rows (p, q, r, s) as vqe_create_pc takes them; one
        parameter per row."""
        return cls(n_qubits, 1, precision, stream, _excitations=excitations, _n_elec=n_elec)

    def _check(self, st: int):
        if st != 0:
            raise VQEError(st, self._lib.vqe_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.vqe_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- Hamiltonian --------------------------------------------------------
    def set_hamiltonian(self, x, z, c):
        x, z, c = _u64(x), _u64(z), _f64(c)
        if not (x.shape == z.shape == c.shape):
            raise ValueError("x, z, c must have equal length")
        self._check(self._lib.vqe_set_hamiltonian(self._h, x.ctypes.data, z.ctypes.data,
                                                  c.ctypes.data, c.size))

    def slim(self, threshold: float):
        kept = ctypes.c_size_t()
        dropped = ctypes.c_double()
        self._check(self._lib.vqe_slim(self._h, float(threshold), ctypes.byref(kept),
                                       ctypes.byref(dropped)))
        return kept.value, dropped.value

    # -- single evaluation (host buffers) -----------------------------------
    def apply_ansatz(self, params):
        p = _f64(params)
        if p.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters")
        self._check(self._lib.vqe_apply_ansatz(self._h, p.ctypes.data))

    def energy(self):
        e, nn = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.vqe_energy(self._h, ctypes.byref(e), ctypes.byref(nn)))
        return e.value, nn.value

    def get_state(self) -> np.ndarray:
        out = np.empty(1 << self.n, dtype=self.state_dtype)
        self._check(self._lib.vqe_get_state(self._h, out.ctypes.data, out.nbytes))
        return out

    def gradient(self, params):
        p = _f64(params)
        if p.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters")
        g = np.empty(self.n_params)
        e = ctypes.c_double()
        self._check(self._lib.vqe_gradient(self._h, p.ctypes.data, g.ctypes.data, ctypes.byref(e)))
        return g, e.value

    # -- batches --------------------------------------------------------------
    def energy_batch(self, params):
        """Host params (batch x n_params) -> (energies, norms) on the host."""
        p = _f64(params).reshape(-1, self.n_params)
        e = np.empty(p.shape[0])
        nn = np.empty(p.shape[0])
        self._check(self._lib.vqe_energy_batch(self._h, p.ctypes.data, p.shape[0], e.ctypes.data,
                                               nn.ctypes.data))
        return e, nn

    def energy_batch_into(self, params, energies, norms=None):
        """Host buffers (NumPy arrays or pinned CPU tensors), written in place."""
        count = params.numel() if hasattr(params, "numel") else params.size
        b = count // self.n_params
        self._check(self._lib.vqe_energy_batch(self._h, _ptr(params), b, _ptr(energies),
                                               _ptr(norms)))

    def gradient_batch(self, params):
        p = _f64(params).reshape(-1, self.n_params)
        g = np.empty_like(p)
        e = np.empty(p.shape[0])
        self._check(self._lib.vqe_gradient_batch(self._h, p.ctypes.data, p.shape[0],
                                                 g.ctypes.data, e.ctypes.data))
        return g, e

    def gradient_batch_into(self, params, grads, energies=None):
        """Host buffers (NumPy arrays or pinned CPU tensors), written in place."""
        count = params.numel() if hasattr(params, "numel") else params.size
        b = count // self.n_params
        self._check(self._lib.vqe_gradient_batch(self._h, _ptr(params), b, _ptr(grads),
                                                 _ptr(energies)))

    def energy_batch_dev(self, params_dev, energies_dev, norms_dev=None, pergate=False):
        """Device tensors: params (batch x n_params, float64), energies (batch)."""
        b = params_dev.numel() // self.n_params
        f = self._lib.vqe_energy_batch_pergate_dev if pergate else self._lib.vqe_energy_batch_dev
        self._check(f(self._h, _ptr(params_dev), b, _ptr(energies_dev), _ptr(norms_dev)))

    def gradient_batch_dev(self, params_dev, grads_dev, energies_dev=None):
        b = params_dev.numel() // self.n_params
        self._check(self._lib.vqe_gradient_batch_dev(self._h, _ptr(params_dev), b,
                                                     _ptr(grads_dev), _ptr(energies_dev)))

    def set_plan_options(self, tile_bits_max: int = 0, run_bits: int = 0, reg_bits: int = 0):
        """Choose the tile plan (0 = default); see vqe_set_plan_options."""
        self._check(self._lib.vqe_set_plan_options(self._h, tile_bits_max, run_bits, reg_bits))

    def set_apply_mode(self, mode: int) -> int:
        """lambda = H psi form: -1 automatic, 0 global sweep, 1 windows, 2
        bit-ordered sweeps; returns the form the current Hamiltonian will use."""
        out = ctypes.c_int()
        self._check(self._lib.vqe_set_apply_mode(self._h, int(mode), ctypes.byref(out)))
        return out.value

    def autotune(self, params_dev, gradient: bool = True, budget_ms: float = 60000.0) -> dict:
        """Time candidate tile plans (and apply-H forms) on device params and
        keep the fastest (vqe_autotune); returns the choice."""
        b = params_dev.numel() // self.n_params
        t = Tuning()
        self._check(self._lib.vqe_autotune(self._h, _ptr(params_dev), b, int(gradient),
                                           float(budget_ms), ctypes.byref(t)))
        return {f: getattr(t, f) for f, _ in Tuning._fields_}

    def workspace_size(self, batch: int, gradient: bool = False) -> int:
        out = ctypes.c_size_t()
        self._check(self._lib.vqe_workspace_size(self._h, batch, int(gradient), ctypes.byref(out)))
        return out.value

    def bind_workspace(self, tensor):
        """Use a caller-owned device tensor as state workspace (None to unbind)."""
        if tensor is None:
            self._check(self._lib.vqe_bind_workspace(self._h, None, 0))
        else:
            nbytes = tensor.numel() * tensor.element_size()
            self._check(self._lib.vqe_bind_workspace(self._h, _ptr(tensor), nbytes))
        self._workspace = tensor

    def profile(self, enable: bool = True):
        """Start (clearing counters) or stop event timing of kernel groups."""
        self._check(self._lib.vqe_profile(self._h, int(enable)))

    def profile_read(self) -> dict:
        t = KernelTimes()
        self._check(self._lib.vqe_profile_read(self._h, ctypes.byref(t)))
        return {g: {"launches": t.launches[i], "ms": t.ms[i], "chunks": t.chunks[i]}
                for i, g in enumerate(KERNEL_GROUPS)}

    def stats(self) -> dict:
        s = Stats()
        self._check(self._lib.vqe_get_stats(self._h, ctypes.byref(s)))
        return {name: getattr(s, name) for name, _ in Stats._fields_}


class Batch:
    """Many independent problems of uneven size in one graph launch (vqe_batch_*)."""

    def __init__(self, n_qubits, depths, precision: str = "c64", stream=None):
        lib = load()
        self._lib = lib
        self.n = np.ascontiguousarray(n_qubits, dtype=np.int32)
        self.depth = np.ascontiguousarray(depths, dtype=np.int32)
        self.count = len(self.n)
        prec = {"c64": VQE_C64, "c128": VQE_C128}[precision]
        h = ctypes.c_void_p()
        st = lib.vqe_batch_create(self.count, self.n.ctypes.data, self.depth.ctypes.data, prec,
                                  _stream_ptr(stream), ctypes.byref(h))
        if st != 0:
            raise VQEError(st, "vqe_batch_create failed")
        self._h = h
        off = np.zeros(self.count + 1, dtype=np.uint64)
        self._check(lib.vqe_batch_param_offsets(self._h, off.ctypes.data))
        self.offsets = off.astype(np.int64)
        self.n_params_total = int(self.offsets[-1])

    def _check(self, st: int):
        if st != 0:
            raise VQEError(st, self._lib.vqe_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.vqe_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_hamiltonian(self, i: int, x, z, c):
        x, z, c = _u64(x), _u64(z), _f64(c)
        self._check(self._lib.vqe_batch_set_hamiltonian(self._h, i, x.ctypes.data, z.ctypes.data,
                                                        c.ctypes.data, c.size))

    def run(self, params):
        """Host params (concatenated) -> (energies, grads) on the host."""
        p = _f64(params)
        assert p.size == self.n_params_total
        e = np.empty(self.count)
        g = np.empty_like(p)
        self._check(self._lib.vqe_batch_run(self._h, p.ctypes.data, e.ctypes.data, g.ctypes.data))
        return e, g

    def run_dev(self, params_dev, energies_dev, grads_dev):
        self._check(self._lib.vqe_batch_run_dev(self._h, _ptr(params_dev), _ptr(energies_dev),
                                                _ptr(grads_dev)))

    def set_tile_bits(self, k: int):
        self._check(self._lib.vqe_batch_set_tile_bits(self._h, k))

    def autotune(self, params_dev, energies_dev, grads_dev, reps: int = 2) -> int:
        out = ctypes.c_int()
        self._check(self._lib.vqe_batch_autotune(self._h, _ptr(params_dev), _ptr(energies_dev),
                                                 _ptr(grads_dev), reps, ctypes.byref(out)))
        return out.value

    def graph_launches(self) -> int:
        out = ctypes.c_uint64()
        self._check(self._lib.vqe_batch_launch_count(self._h, ctypes.byref(out)))
        return out.value


def version() -> str:
    return load().vqe_version().decode()


def measure_fma_peak(fp64: bool = True, stream=None) -> float:
    """Measured FMA throughput of the current GPU in TFLOP/s (FP64 or FP32)."""
    lib = load()
    out = ctypes.c_double()
    st = lib.vqe_measure_fma_peak(1 if fp64 else 0, _stream_ptr(stream), ctypes.byref(out))
    if st:
        raise VQEError(st, "vqe_measure_fma_peak failed")
    return out.value
