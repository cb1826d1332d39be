"""GPU RIME predict + weighted chi^2 for GB300 (sm_103a), after Montblanc
(arXiv 1501.07719).

The computation lives in librime.so (CUDA, C ABI in include/rime.h); this
package is its thin Python binding. ``Rime`` wraps one context.
"""
from ._abi import (RIME_BEAM_COS3, RIME_BEAM_JINC, RIME_PIPE_DFMA, RIME_PIPE_EX2, RIME_PIPE_FFMA, RIME_PIPE_FFMA2, RIME_FP32, RIME_FP64, RIME_KERNEL_AUTO, RIME_KERNEL_NARROW, RIME_KERNEL_TILED, RIME_TC_OFF, RIME_TC_SPLIT_BF16, RIME_TC_SPLIT_F16, RIME_TC_SPLIT_TF32, RimeError, lib,
                   rime_batched_config, rime_chains_accept, rime_chains_init, rime_chains_propose, rime_chi2, rime_chi2_async, rime_chi2_batched, rime_chi2_grad,
                   rime_chi2_noalloc, rime_chi2_streamed, rime_create, rime_destroy, rime_last_error, rime_ln_norm, rime_nbl,
                   rime_predict, rime_set_batched_config, rime_set_data, rime_set_gains, rime_set_sources,
                   rime_set_beam, rime_set_kernel, rime_set_tensor_mode, rime_set_uvw, rime_set_wait_limit, rime_sync,
                   rime_phase_turns, rime_pipe_rate, rime_split_tiles)
from .context import Rime
from .autograd import RimeChi2

__all__ = ["RIME_BEAM_COS3", "RIME_BEAM_JINC", "RIME_PIPE_DFMA", "RIME_PIPE_EX2", "RIME_PIPE_FFMA", "RIME_PIPE_FFMA2", "RIME_FP32", "RIME_FP64", "RIME_KERNEL_AUTO", "RIME_KERNEL_NARROW", "RIME_KERNEL_TILED", "RIME_TC_OFF", "RIME_TC_SPLIT_BF16", "RIME_TC_SPLIT_F16", "RIME_TC_SPLIT_TF32", "RimeError", "Rime",
           "RimeChi2", "lib", "rime_batched_config", "rime_chains_accept", "rime_chains_init",
           "rime_chains_propose", "rime_chi2", "rime_chi2_async", "rime_chi2_batched",
           "rime_chi2_grad", "rime_chi2_noalloc", "rime_chi2_streamed", "rime_create", "rime_destroy", "rime_last_error", "rime_ln_norm",
           "rime_nbl", "rime_predict", "rime_set_batched_config", "rime_set_data", "rime_set_gains",
           "rime_set_beam", "rime_set_kernel", "rime_set_sources", "rime_set_tensor_mode", "rime_set_uvw",
           "rime_set_wait_limit", "rime_sync", "rime_phase_turns", "rime_pipe_rate",
           "rime_split_tiles"]
