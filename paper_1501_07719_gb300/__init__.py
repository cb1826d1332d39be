"""GPU RIME predict + weighted chi^2 for GB300 (sm_103a), after Montblanc
(arXiv 1501.07719).

The computation lives in librime.so (CUDA, C ABI in include/rime.h); this
package is its thin Python binding. ``Rime`` wraps one context.
"""
from ._abi import (RIME_FP32, RIME_FP64, RimeError, lib, rime_chi2, rime_chi2_async, rime_chi2_noalloc,
                   rime_chi2_grad,
                   rime_create, rime_destroy, rime_last_error, rime_ln_norm, rime_nbl,
                   rime_predict, rime_set_data, rime_set_gains, rime_set_sources,
                   rime_set_uvw, rime_sync)
from .context import Rime
from .autograd import RimeChi2

__all__ = ["RIME_FP32", "RIME_FP64", "RimeError", "Rime", "RimeChi2", "lib", "rime_chi2", "rime_chi2_async", "rime_chi2_noalloc", "rime_chi2_grad",
           "rime_create", "rime_destroy", "rime_last_error", "rime_ln_norm", "rime_nbl",
           "rime_predict", "rime_set_data", "rime_set_gains", "rime_set_sources", "rime_set_uvw",
           "rime_sync"]
