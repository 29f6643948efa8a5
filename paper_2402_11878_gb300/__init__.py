"""GB300-native hot path of the VQE simulation of arXiv 2402.11878.

``Engine`` wraps one handle of the C ABI in ``include/vqe.h`` (the CUDA
library ``_lib/libvqe_gb300.so``); ``energy_and_grad`` exposes the adjoint
gradient to ``torch.autograd``.  The library is loaded on first use and its
absence raises ImportError (there is no other code path).
"""
from .binding import Batch, Engine, VQEError, load, version, library_path  # noqa: F401

__all__ = ["Batch", "Engine", "VQEError", "load", "version", "library_path", "EnergyFunction",
           "energy_and_grad", "minimize_energy", "minimize_batch", "cutoff_ratio_search",
           "threshold_for_ratio", "merged_abs_coefficients"]


def __getattr__(name):
    if name in ("EnergyFunction", "energy_and_grad"):
        from . import autograd as _ag
        return getattr(_ag, name)
    if name in ("minimize_energy", "minimize_batch", "cutoff_ratio_search", "threshold_for_ratio",
                "merged_abs_coefficients"):
        from . import optimize as _opt
        return getattr(_opt, name)
    raise AttributeError(name)
